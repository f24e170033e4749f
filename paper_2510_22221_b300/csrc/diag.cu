// Diagnostic: the discrete divergence of B / mu0 = H + M_face at every cell
// centre (B = mu0 (H + M), section "Numerical Model"; M_face the mean of the
// magnetisation of the cells beside a face, as the faces' H takes half of
// each adjacent cell's change of M).  A test aid, not part of the step: the
// leap-frog keeps div(B^n - B^0) at rounding, which the tests check on the
// GPU state.  FP64 arithmetic on the FP32 state.
#include "diag.h"

namespace fl {
namespace {

// M of every magnetic cell, global components: Ms h + R^T m (m the stored
// deviation in the bias frame); the array is zero elsewhere.
__global__ void div_m_kernel(const Inst *I, const MagComp *comps, double *M, long long nc)
{
    const MagComp C = comps[blockIdx.x];
    const int nx = I->nx, ny = I->ny;
    for (int v = threadIdx.x; v < C.V; v += blockDim.x) {
        const int mt = C.mat[v];
        if (mt == 0xFF) continue;
        const int li = v % C.bx, lj = (v / C.bx) % C.by, lk = v / (C.bx * C.by);
        const long long c = ((long long)(C.z0 + lk) * ny + (C.y0 + lj)) * nx + (C.x0 + li);
        const double m0 = C.m[v], m1 = C.m[C.V + v], m2 = C.m[2 * C.V + v];
        const double Ms = I->mm[mt].Ms;
        for (int d = 0; d < 3; ++d)
            M[d * nc + c] = Ms * I->u[d] + (double)I->R[d] * m0 + (double)I->R[3 + d] * m1 + (double)I->R[6 + d] * m2;
    }
}

// H component a of buffer F at face (i, j, k) (the far-wall arrays hold the
// normal H on the walls i = nx, j = ny, k = nz)
__device__ __forceinline__ double h_at(const Inst *I, int F, int a, int i, int j, int k)
{
    const int nx = I->nx, ny = I->ny, nz = I->nz;
    if (a == 0 && i == nx) return I->wHx[(long long)k * ny + j];
    if (a == 1 && j == ny) return I->wHy[(long long)k * nx + i];
    if (a == 2 && k == nz) return I->wHz[(long long)j * nx + i];
    return I->F[F][3 + a][(long long)k * I->plane + (long long)j * I->px + i];
}

__global__ void div_b_kernel(const Inst *I, int F, const double *M, double dx, double dy, double dz, double *out)
{
    const int nx = I->nx, ny = I->ny, nz = I->nz;
    const long long nc = (long long)nx * ny * nz;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    auto cell = [&](int d, int ii, int jj, int kk) { return M[d * nc + ((long long)kk * ny + jj) * nx + ii]; };
    double b[3][2];
    for (int t = 0; t < 2; ++t) {
        const int fi = i + t, fj = j + t, fk = k + t;
        double mx = 0.0, my = 0.0, mz = 0.0;
        if (fi - 1 >= 0 && fi - 1 < nx) mx += 0.5 * cell(0, fi - 1, j, k);
        if (fi < nx) mx += 0.5 * cell(0, fi, j, k);
        if (fj - 1 >= 0 && fj - 1 < ny) my += 0.5 * cell(1, i, fj - 1, k);
        if (fj < ny) my += 0.5 * cell(1, i, fj, k);
        if (fk - 1 >= 0 && fk - 1 < nz) mz += 0.5 * cell(2, i, j, fk - 1);
        if (fk < nz) mz += 0.5 * cell(2, i, j, fk);
        b[0][t] = h_at(I, F, 0, fi, j, k) + mx;
        b[1][t] = h_at(I, F, 1, i, fj, k) + my;
        b[2][t] = h_at(I, F, 2, i, j, fk) + mz;
    }
    out[c] = (b[0][1] - b[0][0]) / dx + (b[1][1] - b[1][0]) / dy + (b[2][1] - b[2][0]) / dz;
}

}  // namespace

cudaError_t launch_div_b(const Inst *dI, const MagComp *dcomps, int ncomp, int F, long long nc, double dx, double dy,
                         double dz, double *M, double *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(M, 0, 3 * (size_t)nc * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (ncomp > 0) div_m_kernel<<<ncomp, 256, 0, s>>>(dI, dcomps, M, nc);
    div_b_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(dI, F, M, dx, dy, dz, out);
    return cudaGetLastError();
}

}  // namespace fl
