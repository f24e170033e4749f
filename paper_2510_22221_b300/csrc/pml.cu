// The two passes of the convolutional PML (absorbing layers) before each
// step, one kernel per axis and pass; see pml.h for the scheme and the data
// layout.
#include "pml.h"

namespace fl {
namespace {

constexpr int kPT = 256;

// HPASS: the H memories of axis AX from E^n (forward differences) and
// H^{n+1/2} -= (dt/mu0) times the CPML terms of axis AX.  Otherwise: the E
// memories of AX from H^{n+1/2} (backward differences) and E^n += (cb/ca)
// times the CPML terms of AX.  With b = AX+1, c = AX+2 (mod 3): component b
// of a curl holds -d/dAX of component c, component c holds +d/dAX of b.
// One thread per cell of the two slabs of axis AX, the thread index being
// the cell's index in the axis's memory arrays (pml_index), so the memories
// move coalesced and neighbouring threads hold neighbouring cells along x
// (along the layer index for AX = x).  A cell in the layers of several axes
// is updated by each axis's kernel in turn (x, then y, then z).  Launched
// as the programmatic dependent of the kernel before it (all but the first
// of a step): the cell's memories, coefficients and class id, which no other
// kernel of the chain writes, are loaded before the wait for that kernel's
// fields.
template <bool HPASS, typename ClsT, int AX>
__global__ void __launch_bounds__(kPT) pml_axis_kernel(const PmlLaunch P, int src)
{
    constexpr int B = (AX + 1) % 3, CC = (AX + 2) % 3;
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const unsigned q = blockIdx.x * kPT + threadIdx.x;
    const unsigned vol = P.pvol[AX];
    if (q >= vol) return;
    const unsigned d = (unsigned)P.pd[AX];
    const unsigned nx = (unsigned)P.n[0], ny = (unsigned)P.n[1], nz = (unsigned)P.n[2];
    unsigned i, j, k, s, t;
    if (AX == 0) {
        t = q % d; const unsigned r = q / d; j = r % ny; const unsigned r2 = r / ny; k = r2 % nz; s = r2 / nz;
        i = s ? nx - d + t : t;
    } else if (AX == 1) {
        i = q % nx; const unsigned r = q / nx; t = r % d; const unsigned r2 = r / d; k = r2 % nz; s = r2 / nz;
        j = s ? ny - d + t : t;
    } else {
        i = q % nx; const unsigned r = q / nx; j = r % ny; const unsigned r2 = r / ny; t = r2 % d; s = r2 / d;
        k = s ? nz - d + t : t;
    }
    const unsigned c = AX == 0 ? i : (AX == 1 ? j : k), n = AX == 0 ? nx : (AX == 1 ? ny : nz);
    const unsigned st = AX == 0 ? 1u : (AX == 1 ? (unsigned)P.px : P.plane);
    const unsigned off = k * P.plane + j * (unsigned)P.px + i;
    const unsigned fs = P.fs;
    float *const F = P.F[src];
    const float *__restrict__ D = F + (HPASS ? 0 : 3 * fs);   // the differentiated field
    float *const T = F + (HPASS ? 3 * fs : 0);                // the corrected field
    float *const ps = P.psi[AX] + (HPASS ? 2 * vol : 0u) + q;
    // memories, coefficients and class id: written by no kernel of the chain
    const float p1 = ps[0], p2 = ps[vol];
    const float4 co = __ldg(P.pco[AX] + (s * d + t) * 2 + (HPASS ? 1 : 0));
    int cl = 0;
    if (!HPASS) cl = (int)static_cast<const ClsT *>(P.cls)[off];
    // the fields, once the kernel before this one has finished
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const float dc = D[CC * fs + off], db = D[B * fs + off];
    float dcn = 0.f, dbn = 0.f;
    const bool nb = HPASS ? c + 1 < n : c > 0;   // the wall's edges (index n; E at 0) hold 0
    if (nb) {
        dcn = D[CC * fs + (HPASS ? off + st : off - st)];
        dbn = D[B * fs + (HPASS ? off + st : off - st)];
    }
    const float tb = T[B * fs + off], tc = T[CC * fs + off];
    float g1 = 0.f, g2 = 0.f;   // d/dAX of component c (enters b) and of component b (enters c)
    if (HPASS) {
        g1 = (dcn - dc) * P.id[AX];
        g2 = (dbn - db) * P.id[AX];
    } else if (nb) {
        g1 = (dc - dcn) * P.id[AX];
        g2 = (db - dbn) * P.id[AX];
    }
    const float n1 = fmaf(co.x, p1, co.y * g1), n2 = fmaf(co.x, p2, co.y * g2);
    ps[0] = n1;
    ps[vol] = n2;
    const float corb = -fmaf(co.z, g1, n1), corc = fmaf(co.z, g2, n2);
    if (HPASS) {
        T[B * fs + off] = fmaf(-P.dtmu, corb, tb);
        T[CC * fs + off] = fmaf(-P.dtmu, corc, tc);
    } else {
        // the class table holds ca - 1
        const float4 A = __ldg(P.ctab + 3 * cl), C = __ldg(P.ctab + 3 * cl + 1);
        const float cab = 1.f + (B == 0 ? A.x : (B == 1 ? A.y : A.z)), cbb = B == 0 ? C.x : (B == 1 ? C.y : C.z);
        const float cac = 1.f + (CC == 0 ? A.x : (CC == 1 ? A.y : A.z)), cbc = CC == 0 ? C.x : (CC == 1 ? C.y : C.z);
        if (cbb != 0.f) T[B * fs + off] = fmaf(cbb * __frcp_rn(cab), corb, tb);
        if (cbc != 0.f) T[CC * fs + off] = fmaf(cbc * __frcp_rn(cac), corc, tc);
    }
}

// One axis's kernel of a pass; every launch but the first of the chain is a
// programmatic dependent of the one before it.
template <bool HPASS, typename ClsT, int AX>
static cudaError_t launch_axis(const PmlLaunch &P, int src, cudaStream_t s, bool &first)
{
    if (P.pd[AX] <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((P.pvol[AX] + kPT - 1) / kPT);
    cfg.blockDim = dim3(kPT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = first ? 0 : 1;
    first = false;
    return cudaLaunchKernelEx(&cfg, pml_axis_kernel<HPASS, ClsT, AX>, P, src);
}

template <bool HPASS, typename ClsT>
static cudaError_t launch_axes(const PmlLaunch &P, int src, cudaStream_t s, bool &first)
{
    cudaError_t e = launch_axis<HPASS, ClsT, 0>(P, src, s, first);
    if (e == cudaSuccess) e = launch_axis<HPASS, ClsT, 1>(P, src, s, first);
    if (e == cudaSuccess) e = launch_axis<HPASS, ClsT, 2>(P, src, s, first);
    return e;
}

}  // namespace

cudaError_t launch_pml(const PmlLaunch *P, int np, int src, bool cls16, cudaStream_t s)
{
    // the first kernel waits for all earlier work of the stream (a plain
    // launch: the magnet kernel of the previous step may outlast its sweep)
    bool first = true;
    for (int q = 0; q < np; ++q) {
        cudaError_t e = launch_axes<true, uint8_t>(P[q], src, s, first);
        if (e == cudaSuccess)
            e = cls16 ? launch_axes<false, uint16_t>(P[q], src, s, first) : launch_axes<false, uint8_t>(P[q], src, s, first);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace fl
