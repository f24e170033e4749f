// Kernels of the Yee-Maxwell + LLG step for sm_103a (arxiv 2510.22221,
// section "Numerical Model").
//
// The state alternates between two field buffers: a step reads E^n and
// H^{n+1/2} from buffer src and writes E^{n+1} and H^{n+3/2} to buffer dst.
//
//   step_kernel : one sweep over the grid computing, plane by plane in z,
//                 E^{n+1} = ca E^n + cb (curl H^{n+1/2} - J(t_{n+1/2})) (Eq. Ampere
//                 with time-centred H and J) on a shared-memory tile extended by
//                 one cell, then the two half-pushes H^{n+1/2} -> H^{n+1} ->
//                 H^{n+3/2} of every non-magnetic face (M = 0 there, the plain
//                 Faraday update); FP64 energy partials and probe samples.
//   mag_kernel  : the two H/M half-pushes of every magnetic face and cell (Eq.
//                 iterate_H with the trapezoidal LLG solve of Eqs. llg_tra4-6,
//                 Jacobi-iterated until max |M^r - M^{r-1}|/Ms < tol), one CTA per
//                 face-connected magnetic region; it recomputes E^{n+1} at its
//                 own faces from buffer src, so it runs concurrently with
//                 step_kernel (the two write disjoint faces of buffer dst).
//   h_half_kernel + mag_kernel<false> : the start-up half-push that moves H and
//                 M from integer time to half a step ahead, in place.
// The last CTA to finish a step, over both kernels, sums the energy partials
// in a fixed order and advances the device step counter (no extra launch).
#include "fdtd_llg_internal.h"

namespace fl {

namespace {

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }

// Sum over the block; result valid in thread 0.  `sh` holds one double per warp.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < nw) ? sh[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ float block_max(float v, float *sh)
{
    const int tid = threadIdx.x;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    float r = sh[0];
    for (int w = 1; w < nw; ++w) r = fmaxf(r, sh[w]);
    __syncthreads();
    return r;
}

// Modulated Gaussian source (section "Modeling Setup"), FP64.
__device__ double source_value(const double *p, double t)
{
    const double u = t - p[3];
    return p[0] * exp(-u * u / (2.0 * p[2] * p[2])) * cos(2.0 * kPi * p[1] * t);
}

__device__ __forceinline__ int class_at(const LaunchSet &L, const Inst *I, long long off)
{
    return L.cls16 ? (int)static_cast<const uint16_t *>(I->cls)[off] : (int)static_cast<const uint8_t *>(I->cls)[off];
}

// Called by every CTA of a step (field and magnet kernels) after its partials
// are written: the last one sums them per instance and advances the step.
__device__ void finish_step(const LaunchSet &L, long long n, double *sred, int *s_last)
{
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nth = blockDim.x * blockDim.y;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&L.ctl->counter, 1u);
        *s_last = (prev == (unsigned)(L.nftiles + L.ncomp) - 1u);
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (L.energy) {
        for (int ii = 0; ii < L.ninst; ++ii) {
            const Inst *I = L.insts + ii;
            const int t0 = I->ftile_off, t1 = t0 + I->fntx * I->fnty * I->fntz;
            double s = 0.0;
            for (int t = t0 + tid; t < t1; t += nth) s += ld_cg(L.part_f + t);
            for (int c = I->mag_off + tid; c < I->mag_off + I->nmag; c += nth) s += ld_cg(L.part_m + c);
            s = block_sum(s, sred);
            if (tid == 0) {
                const double W = s * I->dV;
                I->energy_buf[n % I->cap] = W;
                if (!isfinite(W)) atomicOr(&L.ctl->status, ST_UNSTABLE);
            }
        }
    }
    if (tid == 0) {
        L.ctl->counter = 0u;
        L.ctl->step = n + 1;
        __threadfence();
    }
}

// ------------------------------------------------------ start-up half-push
template <typename ClsT>
__global__ void __launch_bounds__(kTX *kTY) h_half_kernel(LaunchSet L)
{
    for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
        const Inst *I = L.insts + L.tile_inst[t];
        const int lt = t - I->tile_off;
        const int tx = lt % I->ntx, ty = (lt / I->ntx) % I->nty, tz = lt / (I->ntx * I->nty);
        const int i = tx * kTX + threadIdx.x, j = ty * kTY + threadIdx.y;
        const int nx = I->nx, ny = I->ny, nz = I->nz, px = I->px;
        if (i >= nx || j >= ny) continue;
        const long long plane = I->plane;
        const int k0 = tz * kKC, k1 = min(k0 + kKC, nz);
        float *const *F = I->F[L.src];
        const float *__restrict__ Ex = F[0];
        const float *__restrict__ Ey = F[1];
        const float *__restrict__ Ez = F[2];
        const ClsT *__restrict__ cls = static_cast<const ClsT *>(I->cls);
        const bool has_mag = I->nmag > 0;
        const float idx = I->idx, idy = I->idy, idz = I->idz, ch = I->ch;
        for (int k = k0; k < k1; ++k) {
            const long long o = (long long)k * plane + (long long)j * px + i;
            const bool kp = k + 1 < nz, jp = j + 1 < ny, ip = i + 1 < nx;
            const float ex = Ex[o], ey = Ey[o], ez = Ez[o];
            const float cx = ((jp ? Ez[o + px] : 0.f) - ez) * idy - ((kp ? Ey[o + plane] : 0.f) - ey) * idz;
            const float cy = ((kp ? Ex[o + plane] : 0.f) - ex) * idz - ((ip ? Ez[o + 1] : 0.f) - ez) * idx;
            const float cz = ((ip ? Ey[o + 1] : 0.f) - ey) * idx - ((jp ? Ex[o + px] : 0.f) - ex) * idy;
            uint32_t fl = 0;
            if (has_mag) fl = __float_as_uint(__ldg(I->ctab + 3 * (int)cls[o]).w);
            if (!(fl & CF_MAG_HX)) F[3][o] -= ch * cx;
            if (!(fl & CF_MAG_HY)) F[4][o] -= ch * cy;
            if (!(fl & CF_MAG_HZ)) F[5][o] -= ch * cz;
        }
    }
}

// ------------------------------------------------------------ magnet pass
__device__ __forceinline__ float *hx_ptr(const Inst *I, float *const *F, int i, int j, int k)
{
    return (i == I->nx) ? I->wHx + (long long)k * I->ny + j : F[3] + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hy_ptr(const Inst *I, float *const *F, int i, int j, int k)
{
    return (j == I->ny) ? I->wHy + (long long)k * I->nx + i : F[4] + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hz_ptr(const Inst *I, float *const *F, int i, int j, int k)
{
    return (k == I->nz) ? I->wHz + (long long)j * I->nx + i : F[5] + (long long)k * I->plane + (long long)j * I->px + i;
}

// E of component comp at edge (i,j,k): as stored in F (ADVANCE false), or
// advanced to E^{n+1} from F's E^n and H^{n+1/2} with the same arithmetic as
// step_kernel (ADVANCE true).  Edges beyond the far walls are zero.
template <bool ADVANCE>
__device__ float e_edge(const LaunchSet &L, const Inst *I, float *const *F, int comp, int i, int j, int k, long long n)
{
    if (i >= I->nx || j >= I->ny || k >= I->nz) return 0.f;
    const long long plane = I->plane;
    const long long off = (long long)k * plane + (long long)j * I->px + i;
    if (!ADVANCE) return __ldg(F[comp] + off);
    const float *Hx = F[3], *Hy = F[4], *Hz = F[5];
    float cu;
    if (comp == 0)
        cu = (Hz[off] - (j > 0 ? Hz[off - I->px] : 0.f)) * I->idy - (Hy[off] - (k > 0 ? Hy[off - plane] : 0.f)) * I->idz;
    else if (comp == 1)
        cu = (Hx[off] - (k > 0 ? Hx[off - plane] : 0.f)) * I->idz - (Hz[off] - (i > 0 ? Hz[off - 1] : 0.f)) * I->idx;
    else
        cu = (Hy[off] - (i > 0 ? Hy[off - 1] : 0.f)) * I->idx - (Hx[off] - (j > 0 ? Hx[off - I->px] : 0.f)) * I->idy;
    for (int s = 0; s < I->nsrc; ++s)
        if (I->src[s][0] == comp && I->src[s][1] == i && I->src[s][2] == j && I->src[s][3] == k)
            cu -= (float)source_value(I->srcp[s], ((double)n + 0.5) * I->dt);
    const int c = class_at(L, I, off);
    const float4 A = __ldg(I->ctab + 3 * c), B = __ldg(I->ctab + 3 * c + 1);
    const float ca = comp == 0 ? A.x : (comp == 1 ? A.y : A.z);
    const float cb = comp == 0 ? B.x : (comp == 1 ? B.y : B.z);
    return ca * F[comp][off] + cb * cu;
}

// curl of E at the x-face (i, j+1/2, k+1/2), y-face (i+1/2, j, k+1/2), z-face (i+1/2, j+1/2, k)
template <bool ADVANCE>
__device__ float face_curl(const LaunchSet &L, const Inst *I, float *const *F, int a, int i, int j, int k, long long n)
{
    if (a == 0)
        return (e_edge<ADVANCE>(L, I, F, 2, i, j + 1, k, n) - e_edge<ADVANCE>(L, I, F, 2, i, j, k, n)) * I->idy -
               (e_edge<ADVANCE>(L, I, F, 1, i, j, k + 1, n) - e_edge<ADVANCE>(L, I, F, 1, i, j, k, n)) * I->idz;
    if (a == 1)
        return (e_edge<ADVANCE>(L, I, F, 0, i, j, k + 1, n) - e_edge<ADVANCE>(L, I, F, 0, i, j, k, n)) * I->idz -
               (e_edge<ADVANCE>(L, I, F, 2, i + 1, j, k, n) - e_edge<ADVANCE>(L, I, F, 2, i, j, k, n)) * I->idx;
    return (e_edge<ADVANCE>(L, I, F, 1, i + 1, j, k, n) - e_edge<ADVANCE>(L, I, F, 1, i, j, k, n)) * I->idx -
           (e_edge<ADVANCE>(L, I, F, 0, i, j + 1, k, n) - e_edge<ADVANCE>(L, I, F, 0, i, j, k, n)) * I->idy;
}

// The LLG solve runs in the bias frame (rows of I->R: e1, e2, e3 = h) on the
// deviation m = M - Ms e3, so the transverse components that carry the
// precession are resolved to full FP32 relative precision even when Ms h has
// three large global components, and the change of M that feeds the faces is
// computed from small terms only (never as the difference of two large
// values).  The normalisation keeps |M| at its stored value, equal to Ms up to
// FP32 storage rounding.  The face coupling and the neighbour terms of H_eff
// stay in global components (they act per axis).
__device__ __forceinline__ void to_frame(const float *R, float gx, float gy, float gz, float &lx, float &ly, float &lz)
{
    lx = R[0] * gx + R[1] * gy + R[2] * gz;
    ly = R[3] * gx + R[4] * gy + R[5] * gz;
    lz = R[6] * gx + R[7] * gy + R[8] * gz;
}
__device__ __forceinline__ void from_frame(const float *R, float lx, float ly, float lz, float &gx, float &gy, float &gz)
{
    gx = R[0] * lx + R[3] * ly + R[6] * lz;
    gy = R[1] * lx + R[4] * ly + R[7] * lz;
    gz = R[2] * lx + R[5] * ly + R[8] * lz;
}

// FUSED: a full step, H^s from buffer src, results to buffer dst, curl of
// E^{n+1}.  Otherwise: the start-up half-push, in place, curl of the stored E.
template <bool FUSED>
__global__ void __launch_bounds__(kMagThreads) mag_kernel(LaunchSet L)
{
    extern __shared__ float smem[];
    __shared__ float sredf[kMagThreads / 32];
    __shared__ double sredd[kMagThreads / 32];
    __shared__ int s_last;
    const int Vm = L.vmax;
    float *sM = smem;            // m at the start of the half-push (bias frame)
    float *sB = sM + 3 * Vm;     // b - M^n of Eq. llg_tra6 (bias frame)
    float *sA = sB + 3 * Vm;     // cell mean of H^* (H after the curl push), global
    float *sD = sA + 3 * Vm;     // M^{r} - M^{n}, current iterate, global
    uint8_t *smat = reinterpret_cast<uint8_t *>(sD + 3 * Vm);

    const MagComp C = L.comps[blockIdx.x];
    const Inst *I = L.insts + C.inst;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int V = C.V, bx = C.bx, by = C.by, bz = C.bz, bxy = bx * by;
    const long long n = *(volatile long long *)&L.ctl->step;
    const float ch = I->ch, h0n = I->h0n;
    float *const *Fs = I->F[L.src];
    float *const *Fd = I->F[FUSED ? L.dst : L.src];
    float R[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = I->R[q];
    const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nfz = bx * by * (bz + 1);

    for (int v = tid; v < V; v += nth) {
        smat[v] = C.mat[v];
        sM[v] = C.m[v];
        sM[Vm + v] = C.m[V + v];
        sM[2 * Vm + v] = C.m[2 * V + v];
    }
    __syncthreads();
    // curl E at every face of the region, once for both half-pushes
    for (int f = tid; f < nfx + nfy + nfz; f += nth) {
        int a, fi, fj, fk;
        if (f < nfx) { a = 0; fi = f % (bx + 1); fj = (f / (bx + 1)) % by; fk = f / ((bx + 1) * by); }
        else if (f < nfx + nfy) { const int g = f - nfx; a = 1; fi = g % bx; fj = (g / bx) % (by + 1); fk = g / (bx * (by + 1)); }
        else { const int g = f - nfx - nfy; a = 2; fi = g % bx; fj = (g / bx) % by; fk = g / bxy; }
        int vl = -1, vr = -1;
        if (a == 0) { if (fi > 0) vl = (fk * by + fj) * bx + fi - 1; if (fi < bx) vr = (fk * by + fj) * bx + fi; }
        else if (a == 1) { if (fj > 0) vl = (fk * by + fj - 1) * bx + fi; if (fj < by) vr = (fk * by + fj) * bx + fi; }
        else { if (fk > 0) vl = ((fk - 1) * by + fj) * bx + fi; if (fk < bz) vr = (fk * by + fj) * bx + fi; }
        const bool own = (vl >= 0 && smat[vl] != 0xFF) || (vr >= 0 && smat[vr] != 0xFF);
        C.fcurl[f] = own ? face_curl<FUSED>(L, I, Fs, a, C.x0 + fi, C.y0 + fj, C.z0 + fk, n) : 0.f;
    }
    __syncthreads();

    double eacc = 0.0;
    const int nhalf = FUSED ? 2 : 1;
    for (int hp = 0; hp < nhalf; ++hp) {
        float *const *Fin = hp == 0 ? Fs : Fd;   // H^s of this half-push
        // cell means of H^s and H^*, and b - M^n
        for (int v = tid; v < V; v += nth) {
            const int m = smat[v];
            sD[v] = sD[Vm + v] = sD[2 * Vm + v] = 0.f;
            if (m == 0xFF) {
                sB[v] = sB[Vm + v] = sB[2 * Vm + v] = 0.f;
                sA[v] = sA[Vm + v] = sA[2 * Vm + v] = 0.f;
                continue;
            }
            const int li = v % bx, lj = (v / bx) % by, lk = v / bxy;
            const int i = C.x0 + li, j = C.y0 + lj, k = C.z0 + lk;
            const float hx0 = *hx_ptr(I, Fin, i, j, k), hx1 = *hx_ptr(I, Fin, i + 1, j, k);
            const float hy0 = *hy_ptr(I, Fin, i, j, k), hy1 = *hy_ptr(I, Fin, i, j + 1, k);
            const float hz0 = *hz_ptr(I, Fin, i, j, k), hz1 = *hz_ptr(I, Fin, i, j, k + 1);
            const float cx0 = C.fcurl[(lk * by + lj) * (bx + 1) + li], cx1 = C.fcurl[(lk * by + lj) * (bx + 1) + li + 1];
            const float cy0 = C.fcurl[nfx + (lk * (by + 1) + lj) * bx + li], cy1 = C.fcurl[nfx + (lk * (by + 1) + lj + 1) * bx + li];
            const float cz0 = C.fcurl[nfx + nfy + (lk * by + lj) * bx + li], cz1 = C.fcurl[nfx + nfy + ((lk + 1) * by + lj) * bx + li];
            sA[v] = 0.5f * ((hx0 - ch * cx0) + (hx1 - ch * cx1));
            sA[Vm + v] = 0.5f * ((hy0 - ch * cy0) + (hy1 - ch * cy1));
            sA[2 * Vm + v] = 0.5f * ((hz0 - ch * cz0) + (hz1 - ch * cz1));
            float hex, hey, hez;   // H_eff^s in the bias frame
            to_frame(R, 0.5f * (hx0 + hx1), 0.5f * (hy0 + hy1), 0.5f * (hz0 + hz1), hex, hey, hez);
            hez += h0n;
            const float mx = sM[v], my = sM[Vm + v], mz = sM[2 * Vm + v];
            const float Mz = I->mm[m].Ms + mz;
            const float kap = I->mm[m].kappa;
            // b - M^n of Eq. llg_tra6: -kappa M^n x H_eff^n
            sB[v] = -kap * (my * hez - Mz * hey);
            sB[Vm + v] = -kap * (Mz * hex - mx * hez);
            sB[2 * Vm + v] = -kap * (mx * hey - my * hex);
        }
        __syncthreads();

        // Jacobi iteration of Eq. llg_tra4 with H_eff^{r-1} from the previous iterate
        float dl[kMagCPT][3];   // last iterate's change of m, bias frame
#pragma unroll
        for (int q = 0; q < kMagCPT; ++q) dl[q][0] = dl[q][1] = dl[q][2] = 0.f;
        int r = 0;
        for (;;) {
            ++r;
            float res = 0.f;
            float dn[kMagCPT][3];
#pragma unroll
            for (int q = 0; q < kMagCPT; ++q) {
                dn[q][0] = dn[q][1] = dn[q][2] = 0.f;
                const int v = tid + q * nth;
                if (v >= V) continue;
                const int m = smat[v];
                if (m == 0xFF) continue;
                const int li = v % bx, lj = (v / bx) % by, lk = v / bxy;
                const float d0 = sD[v], d1 = sD[Vm + v], d2 = sD[2 * Vm + v];
                const float dxm = li > 0 ? sD[v - 1] : 0.f, dxp = li < bx - 1 ? sD[v + 1] : 0.f;
                const float dym = lj > 0 ? sD[Vm + v - bx] : 0.f, dyp = lj < by - 1 ? sD[Vm + v + bx] : 0.f;
                const float dzm = lk > 0 ? sD[2 * Vm + v - bxy] : 0.f, dzp = lk < bz - 1 ? sD[2 * Vm + v + bxy] : 0.f;
                float hex, hey, hez;
                to_frame(R, sA[v] - 0.25f * (dxm + 2.f * d0 + dxp), sA[Vm + v] - 0.25f * (dym + 2.f * d1 + dyp),
                         sA[2 * Vm + v] - 0.25f * (dzm + 2.f * d2 + dzp), hex, hey, hez);
                hez += h0n;
                const MagMat mm = I->mm[m];
                const float mx = sM[v], my = sM[Vm + v], mz = sM[2 * Vm + v];
                const float Mz = mm.Ms + mz;
                const float dam = mm.alpha * mm.inv_Ms;
                const float ax = -(mm.kappa * hex + dam * mx);
                const float ay = -(mm.kappa * hey + dam * my);
                const float az = -(mm.kappa * hez + mm.alpha + dam * mz);
                // Eq. llg_tra4 written for the increment d = M~ - M^n, which solves
                // d + a x d = r with r = b - M^n - a x M^n = -kappa M^n x (H_eff^n + H_eff^{r-1})
                // (the damping part of a is parallel to M^n); every term is small,
                // so d keeps full FP32 relative precision however large M^n is.
                const float rx = sB[v] - mm.kappa * (my * hez - Mz * hey);
                const float ry = sB[Vm + v] - mm.kappa * (Mz * hex - mx * hez);
                const float rz = sB[2 * Vm + v] - mm.kappa * (mx * hey - my * hex);
                const float ar = ax * rx + ay * ry + az * rz;
                const float inv1 = 1.f / (1.f + ax * ax + ay * ay + az * az);
                const float ddx = (rx + ar * ax - (ay * rz - az * ry)) * inv1;
                const float ddy = (ry + ar * ay - (az * rx - ax * rz)) * inv1;
                const float ddz = (rz + ar * az - (ax * ry - ay * rx)) * inv1;
                // N(M~) = |M^n| M~ / |M~|; the change is d + s1 M~ with
                // s1 = |M^n|/|M~| - 1 = -(2 M^n.d + |d|^2) / (|M~| (|M^n| + |M~|))
                const float nM2 = mx * mx + my * my + Mz * Mz;
                const float md2 = 2.f * (mx * ddx + my * ddy + Mz * ddz) + (ddx * ddx + ddy * ddy + ddz * ddz);
                const float nM = sqrtf(nM2), nMt = sqrtf(nM2 + md2);
                const float s1 = -md2 / (nMt * (nM + nMt));
                dl[q][0] = ddx + s1 * (mx + ddx);
                dl[q][1] = ddy + s1 * (my + ddy);
                dl[q][2] = ddz + s1 * (Mz + ddz);
                from_frame(R, dl[q][0], dl[q][1], dl[q][2], dn[q][0], dn[q][1], dn[q][2]);
                const float e0 = dn[q][0] - d0, e1 = dn[q][1] - d1, e2 = dn[q][2] - d2;
                res = fmaxf(res, sqrtf(e0 * e0 + e1 * e1 + e2 * e2) * mm.inv_Ms);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kMagCPT; ++q) {
                const int v = tid + q * nth;
                if (v < V && smat[v] != 0xFF) {
                    sD[v] = dn[q][0];
                    sD[Vm + v] = dn[q][1];
                    sD[2 * Vm + v] = dn[q][2];
                }
            }
            res = block_max(res, sredf);
            if (L.llg_fixed_iter > 0) {
                if (r >= L.llg_fixed_iter) break;
            } else {
                if (res < L.llg_tol) break;
                if (r >= L.llg_max_iter) {
                    if (tid == 0) atomicOr(&L.ctl->status, ST_NOCONV);
                    break;
                }
            }
        }

        // faces: H = H^s - (dt/2mu0) curl E - (dM_left + dM_right)/2
        const bool rec = FUSED && hp == 0;
        for (int f = tid; f < nfx + nfy + nfz; f += nth) {
            int a, fi, fj, fk;
            if (f < nfx) { a = 0; fi = f % (bx + 1); fj = (f / (bx + 1)) % by; fk = f / ((bx + 1) * by); }
            else if (f < nfx + nfy) { const int g = f - nfx; a = 1; fi = g % bx; fj = (g / bx) % (by + 1); fk = g / (bx * (by + 1)); }
            else { const int g = f - nfx - nfy; a = 2; fi = g % bx; fj = (g / bx) % by; fk = g / bxy; }
            int vl = -1, vr = -1;
            if (a == 0) { if (fi > 0) vl = (fk * by + fj) * bx + fi - 1; if (fi < bx) vr = (fk * by + fj) * bx + fi; }
            else if (a == 1) { if (fj > 0) vl = (fk * by + fj - 1) * bx + fi; if (fj < by) vr = (fk * by + fj) * bx + fi; }
            else { if (fk > 0) vl = ((fk - 1) * by + fj) * bx + fi; if (fk < bz) vr = (fk * by + fj) * bx + fi; }
            const bool inl = vl >= 0 && smat[vl] != 0xFF, inr = vr >= 0 && smat[vr] != 0xFF;
            if (!inl && !inr) continue;
            const int i = C.x0 + fi, j = C.y0 + fj, k = C.z0 + fk;
            const float dlv = inl ? sD[a * Vm + vl] : 0.f, drv = inr ? sD[a * Vm + vr] : 0.f;
            const float hin = a == 0 ? *hx_ptr(I, Fin, i, j, k) : (a == 1 ? *hy_ptr(I, Fin, i, j, k) : *hz_ptr(I, Fin, i, j, k));
            float *hout = a == 0 ? hx_ptr(I, Fd, i, j, k) : (a == 1 ? hy_ptr(I, Fd, i, j, k) : hz_ptr(I, Fd, i, j, k));
            const float h = (hin - ch * C.fcurl[f]) - 0.5f * (dlv + drv);
            *hout = h;
            if (rec) eacc += (double)(h * h);
        }
#pragma unroll
        for (int q = 0; q < kMagCPT; ++q) {
            const int v = tid + q * nth;
            if (v < V && smat[v] != 0xFF) {
                sM[v] += dl[q][0];
                sM[Vm + v] += dl[q][1];
                sM[2 * Vm + v] += dl[q][2];
            }
        }
        __syncthreads();
        if (rec) {
            eacc *= 0.5 * kMu0;
            // Zeeman energy mu0 (|H0| Ms - H0.M) = mu0 |H0|/(2 Ms) |M - Ms h|^2 on |M| = Ms
            float z = 0.f;
            for (int v = tid; v < V; v += nth) {
                const int m = smat[v];
                if (m == 0xFF) continue;
                const float qx = sM[v], qy = sM[Vm + v], qz = sM[2 * Vm + v];
                z += (qx * qx + qy * qy + qz * qz) * I->mm[m].inv_Ms;
            }
            eacc += (double)z * (0.5 * kMu0 * (double)h0n);
            // probe samples of magnetic faces and of M at step n+1
            for (int p = tid; p < I->nprobe; p += nth) {
                const int pi = I->probe[p][0] - C.x0, pj = I->probe[p][1] - C.y0, pk = I->probe[p][2] - C.z0;
                if (pi < 0 || pj < 0 || pk < 0 || pi > bx || pj > by || pk > bz) continue;
                double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + p) * 9;
                const int gi = I->probe[p][0], gj = I->probe[p][1], gk = I->probe[p][2];
                if (pj < by && pk < bz) {
                    const bool l = pi > 0 && smat[(pk * by + pj) * bx + pi - 1] != 0xFF;
                    if (l || (pi < bx && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[3] = *hx_ptr(I, Fd, gi, gj, gk);
                }
                if (pi < bx && pk < bz) {
                    const bool l = pj > 0 && smat[(pk * by + pj - 1) * bx + pi] != 0xFF;
                    if (l || (pj < by && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[4] = *hy_ptr(I, Fd, gi, gj, gk);
                }
                if (pi < bx && pj < by) {
                    const bool l = pk > 0 && smat[((pk - 1) * by + pj) * bx + pi] != 0xFF;
                    if (l || (pk < bz && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[5] = *hz_ptr(I, Fd, gi, gj, gk);
                }
                if (pi < bx && pj < by && pk < bz) {
                    const int vc = (pk * by + pj) * bx + pi;
                    const int m = smat[vc];
                    if (m != 0xFF) {
                        // M = Ms h + R^T m, in FP64
                        const double mx = sM[vc], my = sM[Vm + vc], mz = sM[2 * Vm + vc];
                        const double Ms = I->mm[m].Ms;
                        for (int d = 0; d < 3; ++d)
                            row[6 + d] = Ms * I->u[d] + (double)R[d] * mx + (double)R[3 + d] * my + (double)R[6 + d] * mz;
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int v = tid; v < V; v += nth) {
        C.m[v] = sM[v];
        C.m[V + v] = sM[Vm + v];
        C.m[2 * V + v] = sM[2 * Vm + v];
    }
    if (FUSED) {
        const double s = block_sum(eacc, sredd);
        if (tid == 0) L.part_m[blockIdx.x] = s;
        finish_step(L, n, sredd, &s_last);
    }
}

// ---------------------------------------------------------- fused step
// 4-byte asynchronous global -> shared copy; src_bytes 0 writes a zero and
// reads nothing (the source pointer given is still a valid address).
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc, int src_bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct FusedSmem {
    float h[3][3][kHN];     // H^{n+1/2} planes k-1, k, k+1 (ring of three), halo tile
    float e[2][3][kEN];     // E^{n+1} planes k-1, k (ring of two), extended tile
    float en[2][3][kEN];    // E^n planes k, k+1, extended tile
    uint16_t c[3][kEN];     // class ids, planes k-1, k, k+1
};

template <typename ClsT>
__global__ void __launch_bounds__(kFT, 2) step_kernel(LaunchSet L)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    FusedSmem &S = *reinterpret_cast<FusedSmem *>(smraw);
    __shared__ double sred[kFT / 32];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const long long n = *(volatile long long *)&L.ctl->step;
    const int t = blockIdx.x;
    const Inst *I = L.insts + L.ftile_inst[t];
    const int lt = t - I->ftile_off;
    const int tx = lt % I->fntx, ty = (lt / I->fntx) % I->fnty, tz = lt / (I->fntx * I->fnty);
    const int nx = I->nx, ny = I->ny, nz = I->nz, px = I->px;
    const long long plane = I->plane;
    const int i0 = tx * kFX, j0 = ty * kFY, k0 = tz * I->fkc;
    const int k1 = min(k0 + I->fkc, nz);
    const int kend = k1 < nz ? k1 : nz;
    const float *__restrict__ Fs = I->F[L.src][0];   // component c at Fs + c * fs
    float *__restrict__ Fd = I->F[L.dst][0];
    const long long fs = I->fstride;
    const ClsT *__restrict__ cls = static_cast<const ClsT *>(I->cls);
    const float4 *__restrict__ ctab = I->ctab;
    const bool has_mag = I->nmag > 0;
    const float idx = I->idx, idy = I->idy, idz = I->idz, ch = I->ch;

    // sources and probes whose column lies in this tile's extended / interior area
    unsigned smask = 0, pmask = 0;
    for (int s = 0; s < I->nsrc; ++s) {
        const int si = I->src[s][1] - i0, sj = I->src[s][2] - j0;
        if (si >= 0 && si <= kFX && sj >= 0 && sj <= kFY) smask |= 1u << s;
    }
    for (int p = 0; p < I->nprobe; ++p) {
        const int pi = I->probe[p][0] - i0, pj = I->probe[p][1] - j0;
        if (pi >= 0 && pi < kFX && pj >= 0 && pj < kFY && I->probe[p][2] >= k0 && I->probe[p][2] < k1) pmask |= 1u << p;
    }
    const double tn = ((double)n + 0.5) * I->dt;

    int rc[kEQ];              // class ids of the next plane, on their way to shared memory

    // H of plane kk (zero outside the grid) into S.h[b], asynchronously
#define FL_LOAD_H(kk, b)                                                                                        \
    _Pragma("unroll") for (int q = 0; q < kHQ; ++q) {                                                           \
        const int p = tid + q * kFT;                                                                            \
        if (p < kHN) {                                                                                          \
            const int hi = i0 - 1 + p % kHX, hj = j0 - 1 + p / kHX;                                            \
            const bool ok = hi >= 0 && hi < nx && hj >= 0 && hj < ny && (kk) >= 0 && (kk) < nz;               \
            const long long o = ok ? (long long)(kk) * plane + (long long)hj * px + hi : 0;                    \
            cp_async4(&S.h[b][0][p], Fs + 3 * fs + o, ok ? 4 : 0);                                              \
            cp_async4(&S.h[b][1][p], Fs + 4 * fs + o, ok ? 4 : 0);                                              \
            cp_async4(&S.h[b][2][p], Fs + 5 * fs + o, ok ? 4 : 0);                                              \
        }                                                                                                       \
    }
    // E^n of plane kk into S.en[kk & 1] asynchronously, class ids into rc
#define FL_LOAD_E(kk)                                                                                           \
    _Pragma("unroll") for (int q = 0; q < kEQ; ++q) {                                                           \
        const int p = tid + q * kFT;                                                                            \
        rc[q] = 0;                                                                                              \
        if (p < kEN) {                                                                                          \
            const int ei = i0 + p % kEX, ej = j0 + p / kEX;                                                     \
            const bool ok = ei < nx && ej < ny;                                                                 \
            const long long o = ok ? (long long)(kk) * plane + (long long)ej * px + ei : 0;                    \
            cp_async4(&S.en[(kk) & 1][0][p], Fs + o, ok ? 4 : 0);                                               \
            cp_async4(&S.en[(kk) & 1][1][p], Fs + fs + o, ok ? 4 : 0);                                          \
            cp_async4(&S.en[(kk) & 1][2][p], Fs + 2 * fs + o, ok ? 4 : 0);                                      \
            if (ok) rc[q] = (int)cls[o];                                                                        \
        }                                                                                                       \
    }
#define FL_STORE_C(b)                                                                                           \
    _Pragma("unroll") for (int q = 0; q < kEQ; ++q) {                                                           \
        const int p = tid + q * kFT;                                                                            \
        if (p < kEN) S.c[b][p] = (uint16_t)rc[q];                                                               \
    }

    // prologue: H of plane k0-1 (zero below the grid) and H, E^n, classes of plane k0
    FL_LOAD_H(k0 - 1, (k0 + 2) % 3);
    FL_LOAD_H(k0, k0 % 3);
    FL_LOAD_E(k0);
    cp_async_commit();
    cp_async_wait_all();
    FL_STORE_C(k0 % 3);
    __syncthreads();

    float acc = 0.f;
    for (int k = k0; k <= kend; ++k) {
        const bool pre = k + 1 <= kend && k + 1 < nz;
        if (pre) {
            FL_LOAD_H(k + 1, (k + 1) % 3);
            FL_LOAD_E(k + 1);
            cp_async_commit();
        }
        const int b = k % 3, bm = (k + 2) % 3, eb = k & 1;
        // ---- E^{n+1} of plane k on the extended tile
#pragma unroll
        for (int q = 0; q < kEQ; ++q) {
            const int p = tid + q * kFT;
            if (p >= kEN) continue;
            const int px_ = p % kEX, py_ = p / kEX;
            const int i = i0 + px_, j = j0 + py_;
            float ex = 0.f, ey = 0.f, ez = 0.f;
            if (k < nz && i < nx && j < ny) {
                const int hp = (py_ + 1) * kHX + px_ + 1;
                const float hx = S.h[b][0][hp], hy = S.h[b][1][hp], hz = S.h[b][2][hp];
                const float hz_jm = S.h[b][2][hp - kHX], hx_jm = S.h[b][0][hp - kHX];
                const float hz_im = S.h[b][2][hp - 1], hy_im = S.h[b][1][hp - 1];
                const float hx_km = S.h[bm][0][hp], hy_km = S.h[bm][1][hp];
                float cx = (hz - hz_jm) * idy - (hy - hy_km) * idz;
                float cy = (hx - hx_km) * idz - (hz - hz_im) * idx;
                float cz = (hy - hy_im) * idx - (hx - hx_jm) * idy;
                if (smask) {
                    for (int s = 0; s < I->nsrc; ++s)
                        if (((smask >> s) & 1u) && I->src[s][1] == i && I->src[s][2] == j && I->src[s][3] == k) {
                            const float J = (float)source_value(I->srcp[s], tn);
                            if (I->src[s][0] == 0) cx -= J;
                            else if (I->src[s][0] == 1) cy -= J;
                            else cz -= J;
                        }
                }
                const int c = S.c[b][p];
                const float4 A = __ldg(ctab + 3 * c);
                const float4 B = __ldg(ctab + 3 * c + 1);
                ex = A.x * S.en[eb][0][p] + B.x * cx;
                ey = A.y * S.en[eb][1][p] + B.y * cy;
                ez = A.z * S.en[eb][2][p] + B.z * cz;
                if (px_ < kFX && py_ < kFY && k < k1) {
                    const long long o = (long long)k * plane + (long long)j * px + i;
                    Fd[o] = ex;
                    Fd[fs + o] = ey;
                    Fd[2 * fs + o] = ez;
                    if (L.energy) {
                        const float4 Q = __ldg(ctab + 3 * c + 2);
                        acc += Q.x * ex * ex + Q.y * ey * ey + Q.z * ez * ez;
                    }
                    if (pmask) {
                        for (int pp = 0; pp < I->nprobe; ++pp)
                            if (((pmask >> pp) & 1u) && I->probe[pp][0] == i && I->probe[pp][1] == j && I->probe[pp][2] == k) {
                                double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + pp) * 9;
                                row[0] = ex;
                                row[1] = ey;
                                row[2] = ez;
                            }
                    }
                }
            }
            S.e[eb][0][p] = ex;
            S.e[eb][1][p] = ey;
            S.e[eb][2][p] = ez;
        }
        __syncthreads();
        // ---- H^{n+1} and H^{n+3/2} of plane k-1 on the interior
        if (k > k0) {
            const int kh = k - 1, hb = kh % 3, e0 = kh & 1;
#pragma unroll
            for (int q = 0; q < kIQ; ++q) {
                const int p = tid + q * kFT;
                const int pi = p % kFX, pj = p / kFX;
                const int i = i0 + pi, j = j0 + pj;
                if (i >= nx || j >= ny) continue;
                const int ep = pj * kEX + pi;
                const float ex = S.e[e0][0][ep], ey = S.e[e0][1][ep], ez = S.e[e0][2][ep];
                const float ex_jp = S.e[e0][0][ep + kEX], ez_jp = S.e[e0][2][ep + kEX];
                const float ey_ip = S.e[e0][1][ep + 1], ez_ip = S.e[e0][2][ep + 1];
                const float ex_kp = S.e[eb][0][ep], ey_kp = S.e[eb][1][ep];
                const float cx = (ez_jp - ez) * idy - (ey_kp - ey) * idz;
                const float cy = (ex_kp - ex) * idz - (ez_ip - ez) * idx;
                const float cz = (ey_ip - ey) * idx - (ex_jp - ex) * idy;
                uint32_t fl = 0;
                if (has_mag) fl = __float_as_uint(__ldg(ctab + 3 * (int)S.c[hb][ep]).w);
                const int hp = (pj + 1) * kHX + pi + 1;
                const long long o = (long long)kh * plane + (long long)j * px + i;
                float hmx = 0.f, hmy = 0.f, hmz = 0.f;
                if (!(fl & CF_MAG_HX)) { hmx = S.h[hb][0][hp] - ch * cx; Fd[3 * fs + o] = hmx - ch * cx; }
                if (!(fl & CF_MAG_HY)) { hmy = S.h[hb][1][hp] - ch * cy; Fd[4 * fs + o] = hmy - ch * cy; }
                if (!(fl & CF_MAG_HZ)) { hmz = S.h[hb][2][hp] - ch * cz; Fd[5 * fs + o] = hmz - ch * cz; }
                if (L.energy) acc += (float)(0.5 * kMu0) * (hmx * hmx + hmy * hmy + hmz * hmz);
                if (pmask) {
                    for (int pp = 0; pp < I->nprobe; ++pp)
                        if (((pmask >> pp) & 1u) && I->probe[pp][0] == i && I->probe[pp][1] == j && I->probe[pp][2] == kh) {
                            double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + pp) * 9;
                            if (!(fl & CF_MAG_HX)) row[3] = hmx;
                            if (!(fl & CF_MAG_HY)) row[4] = hmy;
                            if (!(fl & CF_MAG_HZ)) row[5] = hmz;
                        }
                }
            }
        }
        if (pre) {
            cp_async_wait_all();
            FL_STORE_C((k + 1) % 3);
        }
        __syncthreads();
    }
#undef FL_LOAD_H
#undef FL_LOAD_E
#undef FL_STORE_C
    if (L.energy) {
        const double s = block_sum((double)acc, sred);
        if (tid == 0) L.part_f[t] = s;
    }
    finish_step(L, n, sred, &s_last);
}

}  // namespace

int h_half_blocks_per_sm(bool cls16)
{
    int nb = 0;
    if (cls16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_half_kernel<uint16_t>, kTX * kTY, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_half_kernel<uint8_t>, kTX * kTY, 0);
    return nb > 0 ? nb : 1;
}

static size_t mag_smem(const LaunchSet &L) { return (size_t)12 * L.vmax * sizeof(float) + (size_t)L.vmax; }

cudaError_t launch_half(const LaunchSet &L, cudaStream_t s)
{
    if (L.ncomp) {
        const size_t sm = mag_smem(L);
        cudaError_t e = cudaFuncSetAttribute(mag_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        mag_kernel<false><<<L.ncomp, kMagThreads, sm, s>>>(L);
    }
    const dim3 blk(kTX, kTY);
    if (L.cls16) h_half_kernel<uint16_t><<<L.grid_h, blk, 0, s>>>(L);
    else h_half_kernel<uint8_t><<<L.grid_h, blk, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_step(const LaunchSet &L, cudaStream_t s, cudaStream_t s_mag, cudaEvent_t ev_fork, cudaEvent_t ev_join,
                        cudaEvent_t *prof)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(step_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FusedSmem));
        cudaFuncSetAttribute(step_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FusedSmem));
        attr_set = true;
    }
    if (L.ncomp) {
        const size_t sm = mag_smem(L);
        cudaError_t e = cudaFuncSetAttribute(mag_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        cudaEventRecord(ev_fork, s);
        cudaStreamWaitEvent(s_mag, ev_fork, 0);
        if (prof) cudaEventRecord(prof[2], s_mag);
        mag_kernel<true><<<L.ncomp, kMagThreads, sm, s_mag>>>(L);
        if (prof) cudaEventRecord(prof[3], s_mag);
        cudaEventRecord(ev_join, s_mag);
    }
    if (prof) cudaEventRecord(prof[0], s);
    if (L.cls16) step_kernel<uint16_t><<<L.nftiles, kFT, sizeof(FusedSmem), s>>>(L);
    else step_kernel<uint8_t><<<L.nftiles, kFT, sizeof(FusedSmem), s>>>(L);
    if (prof) cudaEventRecord(prof[1], s);
    if (L.ncomp) cudaStreamWaitEvent(s, ev_join, 0);
    return cudaGetLastError();
}

}  // namespace fl
