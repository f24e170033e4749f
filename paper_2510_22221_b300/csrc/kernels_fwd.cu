// Forward kernels of the Yee-Maxwell + LLG step for sm_103a (arxiv 2510.22221,
// section "Numerical Model").
//
//   e_pass   : E^{n+1} = ca E^n + cb (curl H^{n+1/2} - J(t_{n+1/2}))  (Eq. Ampere
//              discretised with time-centred H and J); electric energy and
//              probe samples of E^{n+1}.
//   mag_pass : the two H/M half-pushes of every magnetic face and cell (Eq.
//              iterate_H with the trapezoidal LLG solve of Eqs. llg_tra4-6,
//              Jacobi-iterated until max |M^r - M^{r-1}|/Ms < tol), one CTA per
//              face-connected magnetic region held in shared memory.
//   h_pass   : the two half-pushes H^{n+1/2} -> H^{n+1} -> H^{n+3/2} of every
//              non-magnetic face (M = 0 there, the plain Faraday update);
//              magnetic energy, H probe samples, and the final FP64 energy sum
//              by the last CTA to finish (no extra launch).
//
// E and H are FP32 in HBM, one array per component, x fastest with a row
// pitch of a multiple of 32 floats.  Energies are summed per thread in FP32
// and across threads and tiles in FP64.
#include "fdtd_llg_internal.h"

namespace fl {

namespace {

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }

// Sum over the block (blockDim.x * blockDim.y threads, multiple of 32);
// result valid in thread 0.  `sh` holds one double per warp.
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

__device__ __forceinline__ void tile_coords(const Inst *I, int t, int &tx, int &ty, int &tz)
{
    const int lt = t - I->tile_off;
    tx = lt % I->ntx;
    const int r = lt / I->ntx;
    ty = r % I->nty;
    tz = r / I->nty;
}

// Modulated Gaussian source (section "Modeling Setup"), FP64.
__device__ double source_value(const double *p, double t)
{
    const double u = t - p[3];
    return p[0] * exp(-u * u / (2.0 * p[2] * p[2])) * cos(2.0 * kPi * p[1] * t);
}

// ------------------------------------------------------------------ E pass
template <typename ClsT>
__global__ void __launch_bounds__(kTX *kTY) e_pass_kernel(LaunchSet L)
{
    __shared__ double sred[kTX * kTY / 32];
    const long long n = *(volatile long long *)&L.ctl->step;
    for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
        const Inst *I = L.insts + L.tile_inst[t];
        int tx, ty, tz;
        tile_coords(I, t, tx, ty, tz);
        const int i = tx * kTX + threadIdx.x, j = ty * kTY + threadIdx.y;
        const int nx = I->nx, ny = I->ny, nz = I->nz, px = I->px;
        float acc = 0.f;
        if (i < nx && j < ny) {
            const long long plane = I->plane;
            const int k0 = tz * kKC, k1 = min(k0 + kKC, nz);
            float *__restrict__ Ex = I->Ex;
            float *__restrict__ Ey = I->Ey;
            float *__restrict__ Ez = I->Ez;
            const float *__restrict__ Hx = I->Hx;
            const float *__restrict__ Hy = I->Hy;
            const float *__restrict__ Hz = I->Hz;
            const ClsT *__restrict__ cls = static_cast<const ClsT *>(I->cls);
            const float4 *__restrict__ ctab = I->ctab;
            const float idx = I->idx, idy = I->idy, idz = I->idz;
            long long o = (long long)k0 * plane + (long long)j * px + i;
            float hx_km = (k0 > 0) ? __ldg(Hx + o - plane) : 0.f;
            float hy_km = (k0 > 0) ? __ldg(Hy + o - plane) : 0.f;
            // sources and probes of this column
            unsigned smask = 0, pmask = 0;
            for (int s = 0; s < I->nsrc; ++s)
                if (I->src[s][1] == i && I->src[s][2] == j && I->src[s][3] >= k0 && I->src[s][3] < k1) smask |= 1u << s;
            for (int p = 0; p < I->nprobe; ++p)
                if (I->probe[p][0] == i && I->probe[p][1] == j && I->probe[p][2] >= k0 && I->probe[p][2] < k1) pmask |= 1u << p;
            for (int k = k0; k < k1; ++k, o += plane) {
                const float hx = __ldg(Hx + o), hy = __ldg(Hy + o), hz = __ldg(Hz + o);
                const float hz_jm = (j > 0) ? __ldg(Hz + o - px) : 0.f;
                const float hx_jm = (j > 0) ? __ldg(Hx + o - px) : 0.f;
                const float hz_im = (i > 0) ? __ldg(Hz + o - 1) : 0.f;
                const float hy_im = (i > 0) ? __ldg(Hy + o - 1) : 0.f;
                float cx = (hz - hz_jm) * idy - (hy - hy_km) * idz;
                float cy = (hx - hx_km) * idz - (hz - hz_im) * idx;
                float cz = (hy - hy_im) * idx - (hx - hx_jm) * idy;
                if (smask) {
                    const double tn = ((double)n + 0.5) * I->dt;
                    for (int s = 0; s < I->nsrc; ++s)
                        if (((smask >> s) & 1u) && I->src[s][3] == k) {
                            const float J = (float)source_value(I->srcp[s], tn);
                            if (I->src[s][0] == 0) cx -= J;
                            else if (I->src[s][0] == 1) cy -= J;
                            else cz -= J;
                        }
                }
                const int c = cls[o];
                const float4 A = __ldg(ctab + 3 * c);
                const float4 B = __ldg(ctab + 3 * c + 1);
                const float ex = A.x * Ex[o] + B.x * cx;
                const float ey = A.y * Ey[o] + B.y * cy;
                const float ez = A.z * Ez[o] + B.z * cz;
                Ex[o] = ex;
                Ey[o] = ey;
                Ez[o] = ez;
                if (L.energy) {
                    const float4 Q = __ldg(ctab + 3 * c + 2);
                    acc += Q.x * ex * ex + Q.y * ey * ey + Q.z * ez * ez;
                }
                if (pmask) {
                    for (int p = 0; p < I->nprobe; ++p)
                        if (((pmask >> p) & 1u) && I->probe[p][2] == k) {
                            double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + p) * 9;
                            row[0] = ex;
                            row[1] = ey;
                            row[2] = ez;
                        }
                }
                hx_km = hx;
                hy_km = hy;
            }
        }
        if (L.energy) {
            const double s = block_sum((double)acc, sred);
            if (threadIdx.x == 0 && threadIdx.y == 0) L.part_e[t] = s;
        }
    }
}

// ------------------------------------------------------------------ H pass
template <typename ClsT, int MODE>
__global__ void __launch_bounds__(kTX *kTY) h_pass_kernel(LaunchSet L)
{
    __shared__ double sred[kTX * kTY / 32];
    __shared__ int s_last;
    const long long n = *(volatile long long *)&L.ctl->step;
    const int tid = threadIdx.x + kTX * threadIdx.y;
    for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
        const Inst *I = L.insts + L.tile_inst[t];
        int tx, ty, tz;
        tile_coords(I, t, tx, ty, tz);
        const int i = tx * kTX + threadIdx.x, j = ty * kTY + threadIdx.y;
        const int nx = I->nx, ny = I->ny, nz = I->nz, px = I->px;
        float acc = 0.f;
        if (i < nx && j < ny) {
            const long long plane = I->plane;
            const int k0 = tz * kKC, k1 = min(k0 + kKC, nz);
            const float *__restrict__ Ex = I->Ex;
            const float *__restrict__ Ey = I->Ey;
            const float *__restrict__ Ez = I->Ez;
            float *__restrict__ Hx = I->Hx;
            float *__restrict__ Hy = I->Hy;
            float *__restrict__ Hz = I->Hz;
            const ClsT *__restrict__ cls = static_cast<const ClsT *>(I->cls);
            const float4 *__restrict__ ctab = I->ctab;
            const bool has_mag = I->nmag > 0;
            const float idx = I->idx, idy = I->idy, idz = I->idz, ch = I->ch;
            const bool ip = i + 1 < nx, jp = j + 1 < ny;
            long long o = (long long)k0 * plane + (long long)j * px + i;
            float ex = __ldg(Ex + o), ey = __ldg(Ey + o);
            unsigned pmask = 0;
            if (MODE == 1)
                for (int p = 0; p < I->nprobe; ++p)
                    if (I->probe[p][0] == i && I->probe[p][1] == j && I->probe[p][2] >= k0 && I->probe[p][2] < k1) pmask |= 1u << p;
            for (int k = k0; k < k1; ++k, o += plane) {
                const bool kp = k + 1 < nz;
                const float ez = __ldg(Ez + o);
                const float ex_kp = kp ? __ldg(Ex + o + plane) : 0.f;
                const float ey_kp = kp ? __ldg(Ey + o + plane) : 0.f;
                const float ex_jp = jp ? __ldg(Ex + o + px) : 0.f;
                const float ez_jp = jp ? __ldg(Ez + o + px) : 0.f;
                const float ey_ip = ip ? __ldg(Ey + o + 1) : 0.f;
                const float ez_ip = ip ? __ldg(Ez + o + 1) : 0.f;
                const float cx = (ez_jp - ez) * idy - (ey_kp - ey) * idz;
                const float cy = (ex_kp - ex) * idz - (ez_ip - ez) * idx;
                const float cz = (ey_ip - ey) * idx - (ex_jp - ex) * idy;
                uint32_t fl = 0;
                if (has_mag) fl = __float_as_uint(__ldg(ctab + 3 * (int)cls[o]).w);
                float hmx = 0.f, hmy = 0.f, hmz = 0.f;
                if (!(fl & CF_MAG_HX)) {
                    const float h = Hx[o];
                    hmx = h - ch * cx;
                    Hx[o] = MODE ? hmx - ch * cx : hmx;
                }
                if (!(fl & CF_MAG_HY)) {
                    const float h = Hy[o];
                    hmy = h - ch * cy;
                    Hy[o] = MODE ? hmy - ch * cy : hmy;
                }
                if (!(fl & CF_MAG_HZ)) {
                    const float h = Hz[o];
                    hmz = h - ch * cz;
                    Hz[o] = MODE ? hmz - ch * cz : hmz;
                }
                if (MODE == 1) {
                    acc += hmx * hmx + hmy * hmy + hmz * hmz;
                    if (pmask) {
                        for (int p = 0; p < I->nprobe; ++p)
                            if (((pmask >> p) & 1u) && I->probe[p][2] == k) {
                                double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + p) * 9;
                                if (!(fl & CF_MAG_HX)) row[3] = hmx;
                                if (!(fl & CF_MAG_HY)) row[4] = hmy;
                                if (!(fl & CF_MAG_HZ)) row[5] = hmz;
                            }
                    }
                }
                ex = ex_kp;
                ey = ey_kp;
            }
        }
        if (MODE == 1 && L.energy) {
            const double s = block_sum((double)acc, sred) * (0.5 * kMu0);
            if (tid == 0) L.part_h[t] = s;
        }
    }
    if (MODE == 1) {
        // last CTA: per-instance energy in a fixed order, then step += 1
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&L.ctl->counter, 1u);
            s_last = (prev == gridDim.x - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (L.energy) {
                for (int ii = 0; ii < L.ninst; ++ii) {
                    const Inst *I = L.insts + ii;
                    const int t0 = I->tile_off, t1 = t0 + I->ntx * I->nty * I->ntz;
                    double s = 0.0;
                    for (int t = t0 + tid; t < t1; t += blockDim.x * blockDim.y)
                        s += ld_cg(L.part_e + t) + ld_cg(L.part_h + t);
                    for (int c = I->mag_off + tid; c < I->mag_off + I->nmag; c += blockDim.x * blockDim.y)
                        s += ld_cg(L.part_m + c);
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
    }
}

// ------------------------------------------------------------ magnet pass
__device__ __forceinline__ float e_at(const float *A, const Inst *I, int i, int j, int k)
{
    if (i >= I->nx || j >= I->ny || k >= I->nz) return 0.f;
    return __ldg(A + (long long)k * I->plane + (long long)j * I->px + i);
}

__device__ __forceinline__ float *hx_ptr(const Inst *I, int i, int j, int k)
{
    return (i == I->nx) ? I->wHx + (long long)k * I->ny + j : I->Hx + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hy_ptr(const Inst *I, int i, int j, int k)
{
    return (j == I->ny) ? I->wHy + (long long)k * I->nx + i : I->Hy + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hz_ptr(const Inst *I, int i, int j, int k)
{
    return (k == I->nz) ? I->wHz + (long long)j * I->nx + i : I->Hz + (long long)k * I->plane + (long long)j * I->px + i;
}

// curl of E at the x-face (i, j+1/2, k+1/2), y-face (i+1/2, j, k+1/2), z-face (i+1/2, j+1/2, k)
__device__ __forceinline__ float curl_x(const Inst *I, int i, int j, int k)
{
    return (e_at(I->Ez, I, i, j + 1, k) - e_at(I->Ez, I, i, j, k)) * I->idy -
           (e_at(I->Ey, I, i, j, k + 1) - e_at(I->Ey, I, i, j, k)) * I->idz;
}
__device__ __forceinline__ float curl_y(const Inst *I, int i, int j, int k)
{
    return (e_at(I->Ex, I, i, j, k + 1) - e_at(I->Ex, I, i, j, k)) * I->idz -
           (e_at(I->Ez, I, i + 1, j, k) - e_at(I->Ez, I, i, j, k)) * I->idx;
}
__device__ __forceinline__ float curl_z(const Inst *I, int i, int j, int k)
{
    return (e_at(I->Ey, I, i + 1, j, k) - e_at(I->Ey, I, i, j, k)) * I->idx -
           (e_at(I->Ex, I, i, j + 1, k) - e_at(I->Ex, I, i, j, k)) * I->idy;
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

__global__ void __launch_bounds__(kMagThreads) mag_pass_kernel(LaunchSet L, int mode)
{
    extern __shared__ float smem[];
    __shared__ float sredf[kMagThreads / 32];
    __shared__ double sredd[kMagThreads / 32];
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
    float R[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = I->R[q];

    for (int v = tid; v < V; v += nth) {
        smat[v] = C.mat[v];
        sM[v] = C.m[v];
        sM[Vm + v] = C.m[V + v];
        sM[2 * Vm + v] = C.m[2 * V + v];
    }
    __syncthreads();

    double eacc = 0.0;
    const int nhalf = mode ? 2 : 1;
    for (int hp = 0; hp < nhalf; ++hp) {
        // cell means of H^s and H^*, and b
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
            const float hx0 = *hx_ptr(I, i, j, k), hx1 = *hx_ptr(I, i + 1, j, k);
            const float hy0 = *hy_ptr(I, i, j, k), hy1 = *hy_ptr(I, i, j + 1, k);
            const float hz0 = *hz_ptr(I, i, j, k), hz1 = *hz_ptr(I, i, j, k + 1);
            const float cx0 = curl_x(I, i, j, k), cx1 = curl_x(I, i + 1, j, k);
            const float cy0 = curl_y(I, i, j, k), cy1 = curl_y(I, i, j + 1, k);
            const float cz0 = curl_z(I, i, j, k), cz1 = curl_z(I, i, j, k + 1);
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
        const bool rec = mode && hp == 0;
        const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nfz = bx * by * (bz + 1);
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
            float *hp_ = a == 0 ? hx_ptr(I, i, j, k) : (a == 1 ? hy_ptr(I, i, j, k) : hz_ptr(I, i, j, k));
            const float cu = a == 0 ? curl_x(I, i, j, k) : (a == 1 ? curl_y(I, i, j, k) : curl_z(I, i, j, k));
            const float h = (*hp_ - ch * cu) - 0.5f * (dlv + drv);
            *hp_ = h;
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
                    if (l || (pi < bx && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[3] = *hx_ptr(I, gi, gj, gk);
                }
                if (pi < bx && pk < bz) {
                    const bool l = pj > 0 && smat[(pk * by + pj - 1) * bx + pi] != 0xFF;
                    if (l || (pj < by && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[4] = *hy_ptr(I, gi, gj, gk);
                }
                if (pi < bx && pj < by) {
                    const bool l = pk > 0 && smat[((pk - 1) * by + pj) * bx + pi] != 0xFF;
                    if (l || (pk < bz && smat[(pk * by + pj) * bx + pi] != 0xFF)) row[5] = *hz_ptr(I, gi, gj, gk);
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
    if (mode) {
        const double s = block_sum(eacc, sredd);
        if (tid == 0) L.part_m[blockIdx.x] = s;
    }
}

}  // namespace

int e_pass_blocks_per_sm(bool cls16)
{
    int nb = 0;
    if (cls16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e_pass_kernel<uint16_t>, kTX * kTY, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e_pass_kernel<uint8_t>, kTX * kTY, 0);
    return nb > 0 ? nb : 1;
}

int h_pass_blocks_per_sm(bool cls16)
{
    int nb = 0;
    if (cls16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_pass_kernel<uint16_t, 1>, kTX * kTY, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_pass_kernel<uint8_t, 1>, kTX * kTY, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_e_pass(const LaunchSet &L, cudaStream_t s)
{
    const dim3 blk(kTX, kTY);
    if (L.cls16) e_pass_kernel<uint16_t><<<L.grid_e, blk, 0, s>>>(L);
    else e_pass_kernel<uint8_t><<<L.grid_e, blk, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_h_pass(const LaunchSet &L, int mode, cudaStream_t s)
{
    const dim3 blk(kTX, kTY);
    if (L.cls16) {
        if (mode) h_pass_kernel<uint16_t, 1><<<L.grid_h, blk, 0, s>>>(L);
        else h_pass_kernel<uint16_t, 0><<<L.grid_h, blk, 0, s>>>(L);
    } else {
        if (mode) h_pass_kernel<uint8_t, 1><<<L.grid_h, blk, 0, s>>>(L);
        else h_pass_kernel<uint8_t, 0><<<L.grid_h, blk, 0, s>>>(L);
    }
    return cudaGetLastError();
}

cudaError_t launch_mag_pass(const LaunchSet &L, int mode, cudaStream_t s)
{
    if (L.ncomp == 0) return cudaSuccess;
    const size_t sm = (size_t)12 * L.vmax * sizeof(float) + (size_t)L.vmax;
    cudaError_t e = cudaFuncSetAttribute(mag_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    mag_pass_kernel<<<L.ncomp, kMagThreads, sm, s>>>(L, mode);
    return cudaGetLastError();
}

}  // namespace fl
