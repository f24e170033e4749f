// Convolutional PML (absorbing layers) of the Yee-Maxwell + LLG solver: the
// device data of the layers and the launcher of their two kernels.  Not part
// of the public ABI.
//
// The stretch s = kappa + sigma / (alpha + j w eps0) of axis a turns every
// derivative d/da of the two curls into (1/kappa) d/da + psi, with the memory
// psi <- b psi + c d/da (Roden and Gedney's recursive convolution).  The
// layers occupy the first and last d_a cells of axis a.  The field sweep
// computes plain curls, so the layers act as two passes before each step:
//   H pass: psi_H from E^n; H^{n+1/2} -= (dt/mu0) [(1/kappa - 1) dE + psi_H]
//           (the whole-step CPML term of the leapfrog H^{n-1/2} -> H^{n+1/2});
//   E pass: psi_E from that H^{n+1/2}; E^n += (cb/ca) [(1/kappa - 1) dH + psi_E],
//           so that the sweep's ca E^n + cb curl H equals
//           ca E^n + cb (curl H + the CPML terms).
// Each pass is one kernel per lined axis (x, then y, then z), one thread per
// cell of that axis's two slabs: it advances the axis's two memories of the
// cell and adds the axis's terms to the cell's two components, so no value
// is written by two threads of one kernel (no atomics), and a cell in the
// layers of several axes takes their terms in a fixed order.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace fl {

// A box of layer cells (x fastest); the boxes of an instance are disjoint
// and together cover every cell with a layer on some axis.
struct PmlBox {
    int i0, j0, k0, bx, by, bz;
    unsigned mbx, mby;          // ceil(2^32 / bx), ceil(2^32 / by): division by multiplication
    int axes;                   // bit a: cells of the box may lie in the layers of axis a
};
constexpr int kPmlBoxes = 6;   // z layers (two), y layers between them, x layers in the rest

// One instance's layers, passed to the kernels by value (the constant bank:
// no global loads before the fields).  For axis a with b = a+1, c = a+2
// (mod 3), psi[a] holds four arrays of pvol[a] floats: the memories of E_b
// (d/da of H_c), E_c (d/da of H_b), H_b (d/da of E_c) and H_c (d/da of E_b),
// each indexed by pml_index.  pco[a] holds, per side and layer t,
// {b, c, 1/kappa - 1, 0} at the layer's integer coordinate (E) and then at
// its half-integer one (H).  Box q takes blocks [blk[q], blk[q + 1]).
struct PmlLaunch {
    PmlBox box[kPmlBoxes];
    int blk[kPmlBoxes + 1];
    int nbox;
    int pd[3];
    float *psi[3];
    const float4 *pco[3];
    unsigned pvol[3];
    float *F[2];                // the instance's two field buffers (Ex, Ey, Ez, Hx, Hy, Hz, fs apart)
    unsigned fs, plane;         // 32-bit offsets: 6 fs and every pvol below 2^31 (checked by the host)
    int n[3], px;
    float id[3];                // 1/dx, 1/dy, 1/dz
    float dtmu;                 // dt / mu0
    const void *cls;            // class ids, [nz][ny][px]
    const float4 *ctab;         // (ca - 1, flags) (cb) (eps/2) per class
};

// Index of cell (i, j, k) in a psi array of axis a (side s, layer t).
__host__ __device__ inline unsigned pml_index(int a, int s, int t, int d, int nx, int ny, int nz, int i, int j, int k)
{
    if (a == 0) return (((unsigned)s * nz + k) * ny + j) * d + t;
    if (a == 1) return (((unsigned)s * nz + k) * d + t) * nx + i;
    return (((unsigned)s * d + t) * ny + j) * nx + i;
}

// The H pass then the E pass of every lined instance on stream s, for field
// buffer src: one launch per lined axis and pass, the first a plain launch
// and each later one a programmatic dependent of the one before it (which
// it waits for before touching the fields); nothing when P is empty.
cudaError_t launch_pml(const PmlLaunch *P, int np, int src, bool cls16, cudaStream_t s);

}  // namespace fl
