// The two passes of the convolutional PML (absorbing layers) before each
// step; see pml.h for the scheme and the data layout.
#include "pml.h"

namespace fl {
namespace {

constexpr int kPT = 256;

// Side s and layer t of cell index q on an axis of n cells with d layers at
// each end; false outside the layers.
__device__ __forceinline__ bool layer_of(int q, int n, int d, int &s, int &t)
{
    if (d <= 0) return false;
    if (q < d) { s = 0; t = q; return true; }
    if (q >= n - d) { s = 1; t = q - (n - d); return true; }
    return false;
}

// HPASS: memories of the H faces from E^n (forward differences), H^{n+1/2}
// -= (dt/mu0) times the CPML terms.  Otherwise: memories of the E edges from
// H^{n+1/2} (backward differences), E^n += (cb/ca) times the CPML terms.
// For axis a with b = a+1, c = a+2 (mod 3): component b of a curl holds
// -d/da of component c, component c holds +d/da of component b.
// One cell per thread; the block's box and every descriptor come from the
// parameters, so the first global loads are the fields', all issued before
// any store.
template <bool HPASS, typename ClsT>
__global__ void __launch_bounds__(kPT, 5) pml_kernel(const PmlLaunch P, int src)
{
    const int blk = blockIdx.x;
    PmlBox B = P.box[0];
    int b0 = 0;
#pragma unroll
    for (int q = 1; q < kPmlBoxes; ++q)
        if (q < P.nbox && blk >= P.blk[q]) { B = P.box[q]; b0 = P.blk[q]; }
    const unsigned r = (unsigned)(blk - b0) * kPT + threadIdx.x;
    if (r >= (unsigned)(B.bx * B.by * B.bz)) return;
    // r = (lk by + lj) bx + li; a multiplier is set only where r bx (q1 by)
    // stays below 2^32, which makes the multiplicative quotient exact
    const unsigned q1 = B.mbx ? __umulhi(r, B.mbx) : r / (unsigned)B.bx;
    const unsigned q2 = B.mby ? __umulhi(q1, B.mby) : q1 / (unsigned)B.by;
    const int c[3] = {B.i0 + (int)(r - q1 * B.bx), B.j0 + (int)(q1 - q2 * B.by), B.k0 + (int)q2};
    const unsigned st[3] = {1u, (unsigned)P.px, P.plane};
    const unsigned off = (unsigned)c[2] * P.plane + (unsigned)c[1] * P.px + (unsigned)c[0];
    const unsigned fs = P.fs;
    float *const F = P.F[src];
    const float *__restrict__ D = F + (HPASS ? 0 : 3 * fs);   // the differentiated field (read only here)
    float *const T = F + (HPASS ? 3 * fs : 0);                // the corrected field
    int side[3], tl[3];
    bool lay[3];
    unsigned need = 0;   // components of D (and of T) that the active axes use
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lay[a] = ((B.axes >> a) & 1) && layer_of(c[a], P.n[a], P.pd[a], side[a], tl[a]);
        if (lay[a]) need |= 7u & ~(1u << a);
    }
    // loads: own and neighbour values of D, memories, coefficients, targets
    float dself[3], tv[3], d1b[3], d1c[3], p1[3], p2[3];
    float4 co[3];
    float *ps[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        dself[q] = (need >> q) & 1 ? __ldg(D + q * fs + off) : 0.f;
        tv[q] = (need >> q) & 1 ? T[q * fs + off] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d1b[a] = d1c[a] = p1[a] = p2[a] = 0.f;
        ps[a] = nullptr;
        co[a] = make_float4(1.f, 0.f, 0.f, 0.f);
        if (!lay[a]) continue;
        const int b = a == 2 ? 0 : a + 1, cc = a == 0 ? 2 : a - 1;
        if (HPASS) {
            if (c[a] + 1 < P.n[a]) {   // the wall's edges (index n) hold 0
                d1c[a] = __ldg(D + cc * fs + off + st[a]);
                d1b[a] = __ldg(D + b * fs + off + st[a]);
            }
        } else if (c[a] > 0) {        // edges on the wall a = 0 stay 0 (their class has cb = 0)
            d1c[a] = __ldg(D + cc * fs + off - st[a]);
            d1b[a] = __ldg(D + b * fs + off - st[a]);
        }
        co[a] = __ldg(P.pco[a] + (side[a] * P.pd[a] + tl[a]) * 2 + (HPASS ? 1 : 0));
        ps[a] = P.psi[a] + (HPASS ? 2 * P.pvol[a] : 0u) +
                pml_index(a, side[a], tl[a], P.pd[a], P.n[0], P.n[1], P.n[2], c[0], c[1], c[2]);
        p1[a] = ps[a][0];
        p2[a] = ps[a][P.pvol[a]];
    }
    int cl = 0;
    if (!HPASS) cl = (int)static_cast<const ClsT *>(P.cls)[off];
    // arithmetic, then stores
    float corr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!lay[a]) continue;
        const int b = a == 2 ? 0 : a + 1, cc = a == 0 ? 2 : a - 1;
        float g1, g2;   // d/da of component cc (enters b) and of component b (enters cc)
        if (HPASS) {
            g1 = (d1c[a] - dself[cc]) * P.id[a];
            g2 = (d1b[a] - dself[b]) * P.id[a];
        } else if (c[a] > 0) {
            g1 = (dself[cc] - d1c[a]) * P.id[a];
            g2 = (dself[b] - d1b[a]) * P.id[a];
        } else {
            g1 = g2 = 0.f;
        }
        const float n1 = fmaf(co[a].x, p1[a], co[a].y * g1);
        const float n2 = fmaf(co[a].x, p2[a], co[a].y * g2);
        ps[a][0] = n1;
        ps[a][P.pvol[a]] = n2;
        corr[b] -= fmaf(co[a].z, g1, n1);
        corr[cc] += fmaf(co[a].z, g2, n2);
    }
    if (HPASS) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if ((need >> q) & 1) T[q * fs + off] = fmaf(-P.dtmu, corr[q], tv[q]);
    } else {
        const float4 A = __ldg(P.ctab + 3 * cl), C = __ldg(P.ctab + 3 * cl + 1);
        const float ca[3] = {A.x, A.y, A.z}, cb[3] = {C.x, C.y, C.z};
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (((need >> q) & 1) && cb[q] != 0.f) T[q * fs + off] = fmaf(cb[q] * __frcp_rn(ca[q]), corr[q], tv[q]);
    }
}

}  // namespace

cudaError_t launch_pml(const PmlLaunch *P, int np, int src, bool cls16, cudaStream_t s)
{
    for (int q = 0; q < np; ++q) {
        const int grid = P[q].blk[P[q].nbox];
        if (grid <= 0) continue;
        pml_kernel<true, uint8_t><<<grid, kPT, 0, s>>>(P[q], src);
        if (cls16) pml_kernel<false, uint16_t><<<grid, kPT, 0, s>>>(P[q], src);
        else pml_kernel<false, uint8_t><<<grid, kPT, 0, s>>>(P[q], src);
    }
    return cudaGetLastError();
}

}  // namespace fl
