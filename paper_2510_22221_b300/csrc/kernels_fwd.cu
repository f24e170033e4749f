// Kernels of the Yee-Maxwell + LLG step for sm_103a (arxiv 2510.22221,
// section "Numerical Model").
//
// The state alternates between two field buffers: a step reads E^n and
// H^{n+1/2} from buffer src and writes E^{n+1} and H^{n+3/2} to buffer dst.
//
//   step_kernel     : one sweep over the grid.  Each CTA marches a column of
//                     64 x 8 cells through up to 16 z-planes; every plane of H,
//                     E^n and class ids arrives by TMA in a 4-stage
//                     shared-memory ring (two planes in flight while one is
//                     computed).  Per plane it computes E^{n+1} = ca E^n +
//                     cb (curl H^{n+1/2} - J(t_{n+1/2})) (Eq. Ampere with
//                     time-centred H and J) on the tile extended by one cell,
//                     in place, then the two half-pushes H^{n+1/2} -> H^{n+1}
//                     -> H^{n+3/2} of the plane below for every non-magnetic
//                     face (M = 0 there: the plain Faraday update), with FP64
//                     energy partials and probe samples.
//   mag_kernel      : the H/M half-pushes of every magnetic face and cell (Eq.
//                     iterate_H with the trapezoidal LLG solve of Eqs.
//                     llg_tra4-6, Jacobi-iterated until max |M^r - M^{r-1}|/Ms
//                     < tol), one CTA per face-connected magnetic region, its
//                     cells, faces and face curls resident in shared memory;
//                     it first evaluates E^{n+1} (with the arithmetic of
//                     step_kernel) at the edges of its box.  It runs on a
//                     second, high-priority stream, launched ahead of and
//                     concurrently with step_kernel: it reads only buffer src
//                     and writes only magnetic faces of buffer dst, which
//                     step_kernel never writes.
//   h_half_kernel + mag_kernel with one half-push : the start-up
//                     half-push that moves H and M from integer time to half a
//                     step ahead, in place.
// The last CTA to finish a step, over both kernels, sums the energy partials
// in a fixed order and advances the device step counter (no extra launch).
#include "fdtd_llg_internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

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


// Step m's energy of an instance is the sum of its partials (written by the
// step's sweep warps and magnet CTAs) in energy_chunks() fixed chunks, the
// magnet partials in the last one; the chunk sums are added in chunk order.
// A chunk is summed by one CTA: thread q adds the chunk's slots q, q + nth,
// ... in order, B loads in flight (any B gives the same bits), and block_sum
// adds the threads in a fixed tree.  The value is then the same whether one
// CTA forms every chunk (a reduction task inside the next step's sweep) or
// one CTA each (the flush after the last step of a run).  Valid in thread 0.
template <int B>
__device__ double chunk_sum(const Inst *I, int c, int nch, const double *pf, const double *pm, int mcs, double *sred)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = I->ftile_off * kSW, s1 = (I->ftile_off + I->fntask) * kSW;
    const int len = (s1 - s0 + nch - 1) / nch, a = s0 + c * len, e = min(s1, a + len);
    double s = 0.0;
    int q = a + tid;
    for (; q + (B - 1) * nth < e; q += B * nth) {
        double v[B];
#pragma unroll
        for (int u = 0; u < B; ++u) v[u] = ld_cg(pf + q + u * nth);
#pragma unroll
        for (int u = 0; u < B; ++u) s += v[u];
    }
    for (; q < e; q += 8 * nth) {   // the rest, eight at a time; slots past the end add +0.0 (partials are >= 0)
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = q + u * nth < e ? ld_cg(pf + q + u * nth) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    if (c == nch - 1)
        for (int k = I->mag_off * mcs + tid; k < (I->mag_off + I->nmag) * mcs; k += nth) s += ld_cg(pm + k);
    return block_sum(s, sred);
}

__device__ __forceinline__ void store_energy(const LaunchSet &L, const Inst *I, double t, long long m)
{
    const double W = t * I->dV;
    I->energy_buf[m % I->cap] = W;
    if (!isfinite(W)) atomicOr(&L.ctl->status, ST_UNSTABLE);
}

__device__ __forceinline__ bool energy_pending(const LaunchSet &L, long long m)
{
    return m >= 0 && *(volatile long long *)&L.ctl->epend == m;
}

// Reduction task of the sweep: every chunk of instance ii, in order.
template <int B>
__device__ void reduce_energy(const LaunchSet &L, int ii, long long m, double *sred)
{
    if (!energy_pending(L, m)) return;
    const Inst *I = L.insts + ii;
    const double *pf = L.part_f + (m & 1) * L.part_stride, *pm = L.part_m + (m & 1) * L.part_stride;
    const int nch = energy_chunks(I->fntask);
    double t = 0.0;
    for (int c = 0; c < nch; ++c) t += chunk_sum<B>(I, c, nch, pf, pm, L.mag_cs, sred);
    if (threadIdx.x == 0) store_energy(L, I, t, m);
}

// Called by every CTA of a step (field and magnet kernels) after its partials
// are written: the last one advances the step and marks its partials pending.
__device__ void finish_step(const LaunchSet &L, long long n, int *s_last)
{
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&L.ctl->counter, 1u);
        *s_last = (prev == (unsigned)(L.nfblocks + L.ncomp * L.mag_cs) - 1u);
    }
    __syncthreads();
    if (!*s_last) return;
    if (tid == 0) {
        __threadfence();
        L.ctl->counter = 0u;
        L.ctl->work = 0u;
        L.ctl->epend = L.energy ? n : -1;
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

// ------------------------------------------------- shared E^{n+1} arithmetic
// Written with explicit round-to-nearest and fused operations so that
// step_kernel and mag_kernel produce bitwise the same E^{n+1}.
// (a1 - b1) i1 - (a2 - b2) i2: one component of a Yee curl.
__device__ __forceinline__ float curl2(float a1, float b1, float i1, float a2, float b2, float i2)
{
    return __fmaf_rn(__fsub_rn(a1, b1), i1, -__fmul_rn(__fsub_rn(a2, b2), i2));
}
// ca E^n + cb (curl H - J), as E^n + ((ca - 1) E^n + cb (curl H - J)) from
// the class table's ca - 1 (cam1), which FP32 holds to full relative
// precision where ca itself would be rounded next to 1
__device__ __forceinline__ float e_next(float cam1, float e, float cb, float c)
{
    return __fadd_rn(e, __fmaf_rn(cam1, e, __fmul_rn(cb, c)));
}

// ------------------------------------------------------------ magnet pass
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// 4-byte asynchronous copy global -> shared (completion: cp_async_wait_all)
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ float *hx_ptr(const Inst *I, float *F0, int i, int j, int k)
{
    return (i == I->nx) ? I->wHx + (long long)k * I->ny + j : F0 + 3 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hy_ptr(const Inst *I, float *F0, int i, int j, int k)
{
    return (j == I->ny) ? I->wHy + (long long)k * I->nx + i : F0 + 4 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hz_ptr(const Inst *I, float *F0, int i, int j, int k)
{
    return (k == I->nz) ? I->wHz + (long long)j * I->nx + i : F0 + 5 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}
// H component c (0: x, 1: y, 2: z) of buffer F0 at cell (i, j, k) where it is
// stored (the far-wall arrays hold Hx at i = nx, Hy at j = ny, Hz at k = nz);
// NULL where nothing is stored, which the kernels read as zero
__device__ __forceinline__ const float *h_src(const Inst *I, float *F0, int c, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0) return nullptr;
    const int nx = I->nx, ny = I->ny, nz = I->nz;
    if (c == 0) return (i <= nx && j < ny && k < nz) ? hx_ptr(I, F0, i, j, k) : nullptr;
    if (c == 1) return (i < nx && j <= ny && k < nz) ? hy_ptr(I, F0, i, j, k) : nullptr;
    return (i < nx && j < ny && k <= nz) ? hz_ptr(I, F0, i, j, k) : nullptr;
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

// Cascaded compensated accumulation of FP32 terms (Ogita, Rump and Oishi's
// Sum2): TwoSum gives the exact rounding error of every addition, which is
// summed separately, so s + c carries the running sum as if in twice the
// precision and the FP64 total does not depend on how terms are grouped.
__device__ __forceinline__ void sum2_add(float &s, float &c, float x)
{
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    c = __fadd_rn(c, err);
    s = t;
}

// FUSED: a full step (two half-pushes), H^{n+1/2} from buffer src, results to
// buffer dst, curl of E^{n+1}.  Otherwise: the start-up half-push, in place on
// buffer src, curl of the stored E.
//
// A region is split along its longest axis A (C.ax) into L.mag_cs slabs, one
// per CTA of a thread-block cluster (L.mag_cs = 1: one CTA, no cluster).  A
// CTA holds the cells of its slab and every face and edge of the slab's box,
// so the faces on a cut plane are evaluated by the CTAs on both sides, with
// the same operands in the same order, and written by the one above the cut
// (or, on the region's far face, by the last CTA).  What couples the slabs is
// the A-component of the change of M of the layer beside a cut (a face normal
// to A subtracts half the change of each adjacent cell; the cell means of H
// read it the same way): after every Jacobi iterate each CTA exports that
// component of its first and last layer into shared memory, double-buffered
// by the iterate's parity, and reads its neighbours' exports through
// distributed shared memory after one cluster barrier.  The residual test
// takes the maximum over the cluster, so every CTA stops at the same iterate.
// Each cell and face sees the same values in the same order as with one CTA:
// fields, M and the adjoint tape (written in the region's own indexing) do
// not depend on the split; only the energy partials are grouped per CTA.
//
// CL: the launch splits regions (L.mag_cs > 1); without it none of the
// cluster code is compiled in and a CTA holds a whole region.
//
// Set-up of a CTA: it copies what it reads of buffer src into shared memory
// with asynchronous copies (m, E at the slab box's edges, then per block of
// edge sites H and the class ids), so that the set-up costs one memory round
// trip per block instead of one per dependent load, and evaluates E^{n+1} at
// every edge of the slab box with the arithmetic of step_kernel.
template <bool FUSED, typename ClsT, int CPT, bool CL>
__global__ void __launch_bounds__(kMagThreads) mag_kernel(LaunchSet L)
{
    extern __shared__ float smem[];
    __shared__ float sredf[kMagThreads / 32];
    __shared__ double sredd[kMagThreads / 32];
    __shared__ MagMat smm[kMaxMagMat];
    __shared__ float sres[2];   // this CTA's residual by iterate parity, read by the cluster
    __shared__ int s_last;
    // in a full step the field sweep, launched right behind this kernel on the
    // same stream, may start now: it writes only non-magnetic faces and E of
    // buffer dst and reads nothing this kernel writes
    if (FUSED) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int cs = CL ? L.mag_cs : 1;
    const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
    const MagComp C = L.comps[blockIdx.x / cs];
    const Inst *I = L.insts + C.inst;
    const int tid = threadIdx.x, nth = blockDim.x;
    // the region's box, the split axis A and this CTA's slab [a0, a1) along it
    const int A = C.ax;
    const int ext = A == 0 ? C.bx : (A == 1 ? C.by : C.bz);
    const int a0 = rank * ext / cs, a1 = (rank + 1) * ext / cs;
    const bool lo_cut = CL && a0 > 0, hi_cut = CL && a1 < ext, last = !CL || rank == cs - 1;
    const int wo0 = A == 0 ? a0 : 0, wo1 = A == 1 ? a0 : 0, wo2 = A == 2 ? a0 : 0;   // slab origin in the region box
    const int bx = A == 0 ? a1 - a0 : C.bx, by = A == 1 ? a1 - a0 : C.by, bz = A == 2 ? a1 - a0 : C.bz;
    const int bA = a1 - a0, bxy = bx * by;
    const int V = bx * by * bz;
    const int RBx = C.bx, RBy = C.by, RV = C.V;
    const int gx0 = C.x0 + wo0, gy0 = C.y0 + wo1, gz0 = C.z0 + wo2;            // slab origin in the grid
    const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nfz = bx * by * (bz + 1);
    const int nf = nfx + nfy + nfz;
    const int ex = bx + 1, exy = (bx + 1) * (by + 1), ne = exy * (bz + 1);
    // the region's own face and edge numbering (tape layout)
    const int RnfX = (RBx + 1) * RBy * C.bz, RnfY = RBx * (RBy + 1) * C.bz;
    const int Rnf = RnfX + RnfY + RBx * RBy * (C.bz + 1);
    const int Rne = (RBx + 1) * (RBy + 1) * (C.bz + 1);
    // cross-section of the region normal to A (the slab's other two extents)
    const int XS = A == 0 ? by * bz : (A == 1 ? bx * bz : bx * by);
    const BoxDiv BD(bx, by);
    float *sX = smem;                    // exports [parity][low layer, high layer][L.mag_xs]: one offset in every CTA
    float *sM = smem + 4 * L.mag_xs;     // m (bias frame), 3 blocks of V
    float *sH = sM + 3 * V;              // face H: H^s of the half-push, then its result
    float *sE = sH + nf;                 // E at the box edges, 3 blocks of ne (until the faces are set up)
    float *sD = sE;                      // then M^{r} - M^{n} of the current iterate (global axes), 3 blocks of V
    // stage of one block of at most qx x py x ps edge sites: H of buffer src
    // on the block grown by one cell on its low sides, then the class id of
    // each site; once the edges and faces are set up the area holds sC
    const int sst = (C.qx + 1) * (C.py + 1) * (C.ps + 1);
    float *sS = sE + (3 * ne > 3 * V ? 3 * ne : 3 * V);
    float *sC = sS;                      // (dt/2mu0) curl E at the face
    uint16_t *scl = reinterpret_cast<uint16_t *>(sS + 3 * sst);
    const int narea = max(nf, 3 * sst + (C.qx * C.py * C.ps + 1) / 2);
    uint8_t *smat = reinterpret_cast<uint8_t *>(sS + narea);
    uint8_t *shalo = smat + V;           // magnet material of the layer below the slab, then of the layer above (XS each)
    const long long n = *(volatile long long *)&L.ctl->step;
    const float ch = I->ch, h0n = I->h0n;
    float *Fs = I->F[L.src][0];
    float *Fd = I->F[FUSED ? L.dst : L.src][0];
    const int nx = I->nx, ny = I->ny, nz = I->nz, px = I->px;
    const long long fs = I->fstride, plane = I->plane;
    float R[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = I->R[q];

    // slab-local cell (li, lj, lk) -> the region's cell index; the position of
    // a cell (or of a face normal to A) in the cross-section normal to A
    auto rcell = [&](int li, int lj, int lk) { return ((lk + wo2) * RBy + lj + wo1) * RBx + li + wo0; };
    // the region's index of slab cell v (the same index without a split)
    auto rcell_v = [&](int v) {
        if constexpr (!CL) return v;
        int li, lj, lk;
        cell_decode(v, BD, li, lj, lk);
        return rcell(li, lj, lk);
    };
    auto xsec = [&](int li, int lj, int lk) { return A == 0 ? lk * by + lj : (A == 1 ? lk * bx + li : lj * bx + li); };
    auto acoord = [&](int li, int lj, int lk) { return A == 0 ? li : (A == 1 ? lj : lk); };
    // whether the cells below (inl) and above (inr) face f belong to the
    // region, the cells beyond a cut read from the staged halo layers
    auto sides = [&](int a, int fi, int fj, int fk, int vl, int vr, bool &inl, bool &inr) {
        if constexpr (CL) {
            inl = vl >= 0 ? smat[vl] != 0xFF : (a == A && lo_cut && shalo[xsec(fi, fj, fk)] != 0xFF);
            inr = vr >= 0 ? smat[vr] != 0xFF : (a == A && hi_cut && shalo[XS + xsec(fi, fj, fk)] != 0xFF);
        } else {
            inl = vl >= 0 && smat[vl] != 0xFF;
            inr = vr >= 0 && smat[vr] != 0xFF;
        }
    };
    // faces written (and counted in the energy) by this CTA
    auto owned = [&](int a, int fi, int fj, int fk) { return !CL || a != A || acoord(fi, fj, fk) < bA || last; };
    auto rface = [&](int a, int fi, int fj, int fk) {
        const int i = fi + wo0, j = fj + wo1, k = fk + wo2;
        if (a == 0) return (k * RBy + j) * (RBx + 1) + i;
        if (a == 1) return RnfX + (k * (RBy + 1) + j) * RBx + i;
        return RnfX + RnfY + (k * RBy + j) * RBx + i;
    };

    // m, the material ids (with the halo layers) and E^n at every box edge:
    // one batch of asynchronous copies (edges beyond the far walls are zero)
    for (int v = tid; v < V; v += nth) {
        const int rv = rcell_v(v);
        smat[v] = C.mat[rv];
        cp_async4(sM + v, C.m + rv);
        cp_async4(sM + V + v, C.m + RV + rv);
        cp_async4(sM + 2 * V + v, C.m + 2 * RV + rv);
    }
    for (int t = tid; t < (CL ? 2 * XS : 0); t += nth) {
        const int side = t >= XS, q = t - side * XS;
        const int la = side ? bA : -1;   // slab-local A coordinate of the halo layer
        uint8_t mv = 0xFF;
        if (side ? hi_cut : lo_cut) {
            int li, lj, lk;
            if (A == 0) { li = la; lj = q % by; lk = q / by; }
            else if (A == 1) { lj = la; li = q % bx; lk = q / bx; }
            else { lk = la; li = q % bx; lj = q / bx; }
            mv = C.mat[rcell(li, lj, lk)];
        }
        shalo[t] = mv;
    }
    if (tid < kMaxMagMat) smm[tid] = I->mm[tid];
    {
        const UDiv dex(ex), dey(by + 1);
        for (int e = tid; e < 3 * ne; e += nth) {
            const int comp = e >= 2 * ne ? 2 : (e >= ne ? 1 : 0), r = e - comp * ne;
            const unsigned q1 = dex.div(r), q2 = dey.div(q1);
            const int i = gx0 + r - (int)(q1 * ex), j = gy0 + (int)(q1 - q2 * (by + 1)), k = gz0 + (int)q2;
            if (i < nx && j < ny && k < nz) cp_async4(sE + e, Fs + comp * fs + k * plane + (long long)j * px + i);
            else sE[e] = 0.f;
        }
    }
    // per block of edge sites [xa, xb) x [ya, yb) x [za, zb): stage H (and the
    // class ids), then E^{n+1} at the block's edges (with the arithmetic of
    // step_kernel) and H^s at the faces whose indices lie in the block
    bool first = true;
    for (int za = 0; za <= bz; za += C.ps)
    for (int ya = 0; ya <= by; ya += C.py)
    for (int xa = 0; xa <= bx; xa += C.qx) {
        const int xb = min(xa + C.qx, bx + 1), yb = min(ya + C.py, by + 1), zb = min(za + C.ps, bz + 1);
        const int nbx = xb - xa, nby = yb - ya, nbz = zb - za;
        const int SX = nbx + 1, SXY = SX * (nby + 1), nsc = SXY * (nbz + 1), nsite = nbx * nby * nbz;
        const UDiv dsx(SX), dsxy(SXY), dbx(nbx), dby(nby);
        if (!first) __syncthreads();   // the previous block is done with the stage
        first = false;
        for (int q = tid; q < 3 * nsc; q += nth) {
            const int c = q >= 2 * nsc ? 2 : (q >= nsc ? 1 : 0), r = q - c * nsc;
            const unsigned kk = dsxy.div(r), r2 = r - kk * SXY, jj = dsx.div(r2), ii = r2 - jj * SX;
            const float *src = h_src(I, Fs, c, gx0 + xa - 1 + (int)ii, gy0 + ya - 1 + (int)jj, gz0 + za - 1 + (int)kk);
            float *dst = sS + c * sst + r;
            if (src) cp_async4(dst, src);
            else *dst = 0.f;
        }
        if (FUSED) {
            for (int q = tid; q < nsite; q += nth) {
                const unsigned q1 = dbx.div(q), q2 = dby.div(q1);
                const int i = gx0 + xa + q - (int)(q1 * nbx), j = gy0 + ya + (int)(q1 - q2 * nby), k = gz0 + za + (int)q2;
                scl[q] = (i < nx && j < ny && k < nz) ? (uint16_t) static_cast<const ClsT *>(I->cls)[k * plane + (long long)j * px + i] : 0;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // stage value of H component c at slab-local cell (li, lj, lk), each
        // index at most one below the block
        auto hs = [&](int c, int li, int lj, int lk) {
            return sS[c * sst + (lk - za + 1) * SXY + (lj - ya + 1) * SX + li - xa + 1];
        };
        if (FUSED) {
            for (int q = tid; q < 3 * nsite; q += nth) {
                const int comp = q >= 2 * nsite ? 2 : (q >= nsite ? 1 : 0), r = q - comp * nsite;
                const unsigned q1 = dbx.div(r), q2 = dby.div(q1);
                const int li = xa + r - (int)(q1 * nbx), lj = ya + (int)(q1 - q2 * nby), lk = za + (int)q2;
                const int i = gx0 + li, j = gy0 + lj, k = gz0 + lk;
                if (i >= nx || j >= ny || k >= nz) continue;
                float cu;
                if (comp == 0)
                    cu = curl2(hs(2, li, lj, lk), hs(2, li, lj - 1, lk), I->idy, hs(1, li, lj, lk), hs(1, li, lj, lk - 1), I->idz);
                else if (comp == 1)
                    cu = curl2(hs(0, li, lj, lk), hs(0, li, lj, lk - 1), I->idz, hs(2, li, lj, lk), hs(2, li - 1, lj, lk), I->idx);
                else
                    cu = curl2(hs(1, li, lj, lk), hs(1, li - 1, lj, lk), I->idx, hs(0, li, lj, lk), hs(0, li, lj - 1, lk), I->idy);
                for (int so = 0; so < I->nsrc; ++so)
                    if (I->src[so][0] == comp && I->src[so][1] == i && I->src[so][2] == j && I->src[so][3] == k)
                        cu = __fsub_rn(cu, (float)source_value(I->srcp[so], ((double)n + 0.5) * I->dt));
                const int c = scl[r];
                const float4 Ac = __ldg(I->ctab + 3 * c), Bc = __ldg(I->ctab + 3 * c + 1);
                const float ca = comp == 0 ? Ac.x : (comp == 1 ? Ac.y : Ac.z);
                const float cb = comp == 0 ? Bc.x : (comp == 1 ? Bc.y : Bc.z);
                const int e = comp * ne + (lk * (by + 1) + lj) * ex + li;
                sE[e] = e_next(ca, sE[e], cb, cu);
            }
        }
        for (int f = tid; f < nf; f += nth) {
            int a, fi, fj, fk, vl, vr;
            face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
            if (fi < xa || fi >= xb || fj < ya || fj >= yb || fk < za || fk >= zb) continue;
            bool inl, inr;
            sides(a, fi, fj, fk, vl, vr, inl, inr);
            sH[f] = (inl || inr) ? hs(a, fi, fj, fk) : 0.f;
        }
    }
    __syncthreads();
    // (dt/2mu0) curl E at every face of the slab box
    {
        const float *Ex = sE, *Ey = Ex + ne, *Ez = Ey + ne;
        for (int f = tid; f < nf; f += nth) {
            int a, fi, fj, fk, vl, vr;
            face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
            bool inl, inr;
            sides(a, fi, fj, fk, vl, vr, inl, inr);
            float c = 0.f;
            if (inl || inr) {
                const int e0 = fk * exy + fj * ex + fi;
                float cu;
                if (a == 0) cu = curl2(Ez[e0 + ex], Ez[e0], I->idy, Ey[e0 + exy], Ey[e0], I->idz);
                else if (a == 1) cu = curl2(Ex[e0 + exy], Ex[e0], I->idz, Ez[e0 + 1], Ez[e0], I->idx);
                else cu = curl2(Ey[e0 + 1], Ey[e0], I->idx, Ex[e0 + ex], Ex[e0], I->idy);
                c = ch * cu;
            }
            sC[f] = c;
        }
    }
    __syncthreads();
    // adjoint recording (mag_tape_floats, the region's indexing): this step's
    // tape slot, else NULL; each CTA writes its own cells, faces and edges
    float *T = nullptr;
    if (FUSED && L.rec && C.tape) {
        if (n < L.rec_n0 || n - L.rec_n0 >= L.rec_slots || L.llg_fixed_iter < 1) {
            if (tid == 0) atomicOr(&L.ctl->status, ST_TAPE);   // out of the tape: record nothing
        } else {
            T = C.tape + (n - L.rec_n0) * C.tstride;
        }
    }
    const int RI = L.llg_fixed_iter;
    if (T) {   // m and face H at the start of the step, E^{n+1} at the box edges
        for (int v = tid; v < V; v += nth) {
            const int rv = rcell_v(v);
            for (int d = 0; d < 3; ++d) T[d * RV + rv] = sM[d * V + v];
        }
        for (int f = tid; f < nf; f += nth) {
            int a, fi, fj, fk, vl, vr;
            face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
            if (owned(a, fi, fj, fk)) T[3 * RV + rface(a, fi, fj, fk)] = sH[f];
        }
        const UDiv dex(ex), dey(by + 1);
        for (int e = tid; e < 3 * ne; e += nth) {
            const int comp = e >= 2 * ne ? 2 : (e >= ne ? 1 : 0), r = e - comp * ne;
            const unsigned q1 = dex.div(r), q2 = dey.div(q1);
            const int li = r - (int)(q1 * ex), lj = (int)(q1 - q2 * (by + 1)), lk = (int)q2;
            if (acoord(li, lj, lk) < bA || last)
                T[3 * RV + Rnf + comp * Rne + ((lk + wo2) * (RBy + 1) + lj + wo1) * (RBx + 1) + li + wo0] = sE[e];
        }
    }
    __syncthreads();   // sE becomes sD

    // the exports of the CTA below (its high layer) and above (its low layer)
    // in parity 0; parity p is 2 p L.mag_xs floats further
    const float *pxl = nullptr, *pxh = nullptr;
    if constexpr (CL) {
        cg::cluster_group cl = cg::this_cluster();
        if (lo_cut) pxl = cl.map_shared_rank(sX + L.mag_xs, rank - 1);
        if (hi_cut) pxh = cl.map_shared_rank(sX, rank + 1);
    }

    double eacc = 0.0;
    const int nhalf = FUSED ? 2 : 1;
    for (int hp = 0; hp < nhalf; ++hp) {
        for (int v = tid; v < V; v += nth) sD[v] = sD[V + v] = sD[2 * V + v] = 0.f;
        __syncthreads();
        // Jacobi iteration of Eq. llg_tra4 with H_eff^{r-1} from the previous iterate
        float dl[CPT][3];   // last iterate's change of m, bias frame
#pragma unroll
        for (int q = 0; q < CPT; ++q) dl[q][0] = dl[q][1] = dl[q][2] = 0.f;
        int r = 0;
        for (;;) {
            ++r;
            float res = 0.f;
            float dn[CPT][3];
            // the neighbours' exports of the previous iterate (none in the first: the change starts at zero)
            const int po = 2 * ((r - 1) & 1) * L.mag_xs;
            const float *nl = (r > 1 && pxl) ? pxl + po : nullptr, *nh = (r > 1 && pxh) ? pxh + po : nullptr;
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                dn[q][0] = dn[q][1] = dn[q][2] = 0.f;
                const int v = tid + q * nth;
                if (v >= V) continue;
                const int m = smat[v];
                if (m == 0xFF) continue;
                int li, lj, lk;
                cell_decode(v, BD, li, lj, lk);
                const int fx0 = (lk * by + lj) * (bx + 1) + li, fy0 = nfx + (lk * (by + 1) + lj) * bx + li,
                          fz0 = nfx + nfy + (lk * by + lj) * bx + li;
                const float hx0 = sH[fx0], hx1 = sH[fx0 + 1], hy0 = sH[fy0], hy1 = sH[fy0 + bx];
                const float hz0 = sH[fz0], hz1 = sH[fz0 + bxy];
                // cell means of H^* = H^s - (dt/2mu0) curl E
                const float ax_ = 0.5f * ((hx0 - sC[fx0]) + (hx1 - sC[fx0 + 1]));
                const float ay_ = 0.5f * ((hy0 - sC[fy0]) + (hy1 - sC[fy0 + bx]));
                const float az_ = 0.5f * ((hz0 - sC[fz0]) + (hz1 - sC[fz0 + bxy]));
                const float d0 = sD[v], d1 = sD[V + v], d2 = sD[2 * V + v];
                float dxm = li > 0 ? sD[v - 1] : 0.f, dxp = li < bx - 1 ? sD[v + 1] : 0.f;
                float dym = lj > 0 ? sD[V + v - bx] : 0.f, dyp = lj < by - 1 ? sD[V + v + bx] : 0.f;
                float dzm = lk > 0 ? sD[2 * V + v - bxy] : 0.f, dzp = lk < bz - 1 ? sD[2 * V + v + bxy] : 0.f;
                if (CL && (nl || nh)) {   // neighbours across a cut: the other CTA's export
                    const int la = acoord(li, lj, lk), xq = xsec(li, lj, lk);
                    const float lo = (nl && la == 0) ? nl[xq] : 0.f, hi = (nh && la == bA - 1) ? nh[xq] : 0.f;
                    if (A == 0) { if (nl && la == 0) dxm = lo; if (nh && la == bA - 1) dxp = hi; }
                    else if (A == 1) { if (nl && la == 0) dym = lo; if (nh && la == bA - 1) dyp = hi; }
                    else { if (nl && la == 0) dzm = lo; if (nh && la == bA - 1) dzp = hi; }
                }
                float hex, hey, hez;   // H_eff^{r-1} in the bias frame
                to_frame(R, ax_ - 0.25f * (dxm + 2.f * d0 + dxp), ay_ - 0.25f * (dym + 2.f * d1 + dyp),
                         az_ - 0.25f * (dzm + 2.f * d2 + dzp), hex, hey, hez);
                hez += h0n;
                float sx, sy, sz;      // H_eff^s (start of the half-push) in the bias frame
                to_frame(R, 0.5f * (hx0 + hx1), 0.5f * (hy0 + hy1), 0.5f * (hz0 + hz1), sx, sy, sz);
                sz += h0n;
                const MagMat mm = smm[m];
                const float mx = sM[v], my = sM[V + v], mz = sM[2 * V + v];
                const float Mz = mm.Ms + mz;
                const float dam = mm.alpha * mm.inv_Ms;
                const float ax = -(mm.kappa * hex + dam * mx);
                const float ay = -(mm.kappa * hey + dam * my);
                const float az = -(mm.kappa * hez + mm.alpha + dam * mz);
                // Eq. llg_tra4 written for the increment d = M~ - M^n, which solves
                // d + a x d = r with r = b - M^n - a x M^n = -kappa M^n x (H_eff^s + H_eff^{r-1})
                // (Eq. llg_tra6 gives b - M^n = -kappa M^n x H_eff^s; the damping part
                // of a is parallel to M^n); every term is small, so d keeps full FP32
                // relative precision however large M^n is.
                const float bx_ = -mm.kappa * (my * sz - Mz * sy);
                const float by_ = -mm.kappa * (Mz * sx - mx * sz);
                const float bz_ = -mm.kappa * (mx * sy - my * sx);
                const float rx = bx_ - mm.kappa * (my * hez - Mz * hey);
                const float ry = by_ - mm.kappa * (Mz * hex - mx * hez);
                const float rz = bz_ - mm.kappa * (mx * hey - my * hex);
                const float ar = ax * rx + ay * ry + az * rz;
                const float inv1 = __frcp_rn(1.f + ax * ax + ay * ay + az * az);
                const float ddx = (rx + ar * ax - (ay * rz - az * ry)) * inv1;
                const float ddy = (ry + ar * ay - (az * rx - ax * rz)) * inv1;
                const float ddz = (rz + ar * az - (ax * ry - ay * rx)) * inv1;
                // N(M~) = |M^n| M~ / |M~|; the change is d + s1 M~ with
                // s1 = |M^n|/|M~| - 1 = -(2 M^n.d + |d|^2) / (|M~| (|M^n| + |M~|))
                const float nM2 = mx * mx + my * my + Mz * Mz;
                const float md2 = 2.f * (mx * ddx + my * ddy + Mz * ddz) + (ddx * ddx + ddy * ddy + ddz * ddz);
                // (reciprocal square roots and one reciprocal: s1 is second
                // order in d, so their last-bit errors leave |M| at FP32 rounding)
                const float rnM = rsqrtf(nM2), rnMt = rsqrtf(nM2 + md2);
                const float nM = nM2 * rnM, nMt = (nM2 + md2) * rnMt;
                const float s1 = -md2 * __frcp_rn(nMt * (nM + nMt));
                dl[q][0] = ddx + s1 * (mx + ddx);
                dl[q][1] = ddy + s1 * (my + ddy);
                dl[q][2] = ddz + s1 * (Mz + ddz);
                from_frame(R, dl[q][0], dl[q][1], dl[q][2], dn[q][0], dn[q][1], dn[q][2]);
                if (L.llg_fixed_iter <= 0) {   // the residual decides only a tolerance-stopped solve
                    const float e0 = dn[q][0] - d0, e1 = dn[q][1] - d1, e2 = dn[q][2] - d2;
                    res = fmaxf(res, sqrtf(e0 * e0 + e1 * e1 + e2 * e2) * mm.inv_Ms);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int v = tid + q * nth;
                if (v < V && smat[v] != 0xFF) {
                    sD[v] = dn[q][0];
                    sD[V + v] = dn[q][1];
                    sD[2 * V + v] = dn[q][2];
                }
            }
            if (T && r <= RI) {   // iterate r of half-push hp (zero outside the region); this thread's own cells
                float *TD = T + 3 * RV + Rnf + 3 * Rne + (long long)((hp * RI + r - 1) * 3) * RV;
                for (int v = tid; v < V; v += nth) {
                    const int rv = rcell_v(v);
                    TD[rv] = sD[v];
                    TD[RV + rv] = sD[V + v];
                    TD[2 * RV + rv] = sD[2 * V + v];
                }
            }
            // (either also orders every sD write before the exports below)
            if (L.llg_fixed_iter <= 0) res = block_max(res, sredf);
            else __syncthreads();
            if constexpr (CL) {
                // the A-component of the change of M on the first and last
                // layer (zero outside the region) for the CTAs beside this one
                float *xw = sX + 2 * (r & 1) * L.mag_xs;
                const float *dA = sD + A * V;
                const int st = A == 0 ? 1 : (A == 1 ? bx : bxy), last_off = (bA - 1) * st;
                for (int t = tid; t < XS; t += nth) {
                    const int p = t % (A == 0 ? by : bx), q = t / (A == 0 ? by : bx);
                    // cell of cross-section t on layer 0: A = x: (0, p, q); y: (p, 0, q); z: (p, q, 0)
                    const int v0 = A == 0 ? (q * by + p) * bx : (A == 1 ? q * bxy + p : q * bx + p);
                    xw[t] = dA[v0];
                    xw[L.mag_xs + t] = dA[v0 + last_off];
                }
                // every CTA's iterate is complete and exported; then the
                // residual is the cluster's maximum
                if (tid == 0) sres[r & 1] = res;
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();   // every CTA's iterate is complete and exported
                if (L.llg_fixed_iter <= 0)
                    for (int q = 0; q < cs; ++q) res = fmaxf(res, *cl.map_shared_rank(&sres[r & 1], q));
            }
            if (L.llg_fixed_iter > 0) {
                if (r >= L.llg_fixed_iter) break;
            } else {
                // the test compares two iterates: from r = 2 on (the first
                // iterate against M^n measures only the change of M)
                if (r >= 2 && res < L.llg_tol) break;
                if (r >= L.llg_max_iter) {
                    if (tid == 0) atomicOr(&L.ctl->status, ST_NOCONV);
                    break;
                }
            }
        }

        // faces: H = H^s - (dt/2mu0) curl E - (dM_low + dM_high)/2, the cells
        // beyond a cut from the other CTA's last export
        const float *fl = pxl ? pxl + 2 * (r & 1) * L.mag_xs : nullptr, *fh = pxh ? pxh + 2 * (r & 1) * L.mag_xs : nullptr;
        const bool rec = FUSED && hp == 0;
        float es = 0.f, ec = 0.f;   // face energy of this thread, compensated
        for (int f = tid; f < nf; f += nth) {
            int a, fi, fj, fk, vl, vr;
            face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
            bool inl, inr;
            sides(a, fi, fj, fk, vl, vr, inl, inr);
            if (!inl && !inr) continue;
            const float dlv = inl ? (vl >= 0 ? sD[a * V + vl] : fl[xsec(fi, fj, fk)]) : 0.f;
            const float drv = inr ? (vr >= 0 ? sD[a * V + vr] : fh[xsec(fi, fj, fk)]) : 0.f;
            const float h = (sH[f] - sC[f]) - 0.5f * (dlv + drv);
            sH[f] = h;
            if (rec && owned(a, fi, fj, fk)) sum2_add(es, ec, h * h);
        }
        if (rec) eacc += (double)es + (double)ec;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int v = tid + q * nth;
            if (v < V && smat[v] != 0xFF) {
                sM[v] += dl[q][0];
                sM[V + v] += dl[q][1];
                sM[2 * V + v] += dl[q][2];
            }
        }
        __syncthreads();
        if (T && hp == 0) {   // face H and m after the first half-push
            float *TH = T + 3 * RV + Rnf + 3 * Rne + 6LL * RI * RV;
            for (int f = tid; f < nf; f += nth) {
                int a, fi, fj, fk, vl, vr;
                face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
                if (owned(a, fi, fj, fk)) TH[rface(a, fi, fj, fk)] = sH[f];
            }
            for (int v = tid; v < V; v += nth) {
                const int rv = rcell_v(v);
                for (int d = 0; d < 3; ++d) TH[Rnf + d * RV + rv] = sM[d * V + v];
            }
        }
        if (rec) {
            eacc *= 0.5 * kMu0;
            // Zeeman energy mu0 (|H0| Ms - H0.M) = mu0 |H0|/(2 Ms) |M - Ms h|^2 on |M| = Ms
            float z = 0.f;
            for (int v = tid; v < V; v += nth) {
                const int m = smat[v];
                if (m == 0xFF) continue;
                const float qx = sM[v], qy = sM[V + v], qz = sM[2 * V + v];
                z += (qx * qx + qy * qy + qz * qz) * smm[m].inv_Ms;
            }
            eacc += (double)z * (0.5 * kMu0 * (double)h0n);
            // probe samples of the magnetic faces and cells this CTA owns, at step n+1
            for (int p = tid; p < I->nprobe; p += nth) {
                const int pi = I->probe[p][0] - gx0, pj = I->probe[p][1] - gy0, pk = I->probe[p][2] - gz0;
                if (pi < 0 || pj < 0 || pk < 0 || pi > bx || pj > by || pk > bz) continue;
                double *row = I->probe_buf + ((long long)(n % I->cap) * I->nprobe + p) * 9;
                // the face of axis a at the probe cell's low side, if it is a magnetic face of this CTA
                auto face_at = [&](int a) -> int {
                    if ((a != 0 && pi >= bx) || (a != 1 && pj >= by) || (a != 2 && pk >= bz)) return -1;
                    int f, vl = -1, vr = -1;
                    if (a == 0) {
                        f = (pk * by + pj) * (bx + 1) + pi;
                        if (pi > 0) vl = (pk * by + pj) * bx + pi - 1;
                        if (pi < bx) vr = (pk * by + pj) * bx + pi;
                    } else if (a == 1) {
                        f = nfx + (pk * (by + 1) + pj) * bx + pi;
                        if (pj > 0) vl = (pk * by + pj - 1) * bx + pi;
                        if (pj < by) vr = (pk * by + pj) * bx + pi;
                    } else {
                        f = nfx + nfy + (pk * by + pj) * bx + pi;
                        if (pk > 0) vl = ((pk - 1) * by + pj) * bx + pi;
                        if (pk < bz) vr = (pk * by + pj) * bx + pi;
                    }
                    bool inl, inr;
                    sides(a, pi, pj, pk, vl, vr, inl, inr);
                    return ((inl || inr) && owned(a, pi, pj, pk)) ? f : -1;
                };
                for (int a = 0; a < 3; ++a) {
                    const int f = face_at(a);
                    if (f >= 0) row[3 + a] = sH[f];
                }
                if (pi < bx && pj < by && pk < bz) {
                    const int vc = (pk * by + pj) * bx + pi;
                    const int m = smat[vc];
                    if (m != 0xFF) {
                        // M = Ms h + R^T m, in FP64
                        const double mx = sM[vc], my = sM[V + vc], mz = sM[2 * V + vc];
                        const double Ms = smm[m].Ms;
                        for (int d = 0; d < 3; ++d)
                            row[6 + d] = Ms * I->u[d] + (double)R[d] * mx + (double)R[3 + d] * my + (double)R[6 + d] * mz;
                    }
                }
            }
        }
        // the other CTAs have read this half-push's exports before the next
        // one writes them (and before any CTA of the cluster exits)
        if constexpr (CL) cg::this_cluster().sync();
        else __syncthreads();
    }
    // results: the magnetic faces this CTA owns in the output buffer (and the
    // far-wall arrays), m of its cells
    for (int f = tid; f < nf; f += nth) {
        int a, fi, fj, fk, vl, vr;
        face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
        bool inl, inr;
        sides(a, fi, fj, fk, vl, vr, inl, inr);
        if (!(inl || inr) || !owned(a, fi, fj, fk)) continue;
        const int i = gx0 + fi, j = gy0 + fj, k = gz0 + fk;
        float *out = a == 0 ? hx_ptr(I, Fd, i, j, k) : (a == 1 ? hy_ptr(I, Fd, i, j, k) : hz_ptr(I, Fd, i, j, k));
        *out = sH[f];
    }
    for (int v = tid; v < V; v += nth) {
        const int rv = rcell_v(v);
        C.m[rv] = sM[v];
        C.m[RV + rv] = sM[V + v];
        C.m[2 * RV + rv] = sM[2 * V + v];
    }
    if (FUSED) {
        const double s = block_sum(eacc, sredd);
        if (tid == 0) L.part_m[(n & 1) * L.part_stride + blockIdx.x] = s;
        finish_step(L, n, &s_last);
    }
}

// ---------------------------------------------------------- fused step
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity: false after `polls`
// polls (2^22 by default).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, int polls = 1 << 22)
{
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *tm)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(tm) : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
// class ids of the cell pair (x, x+1), x even
__device__ __forceinline__ void cls2(const uint8_t *p, int &c0, int &c1)
{
    const unsigned v = *reinterpret_cast<const uint16_t *>(p);
    c0 = (int)(v & 0xFFu);
    c1 = (int)(v >> 8);
}
__device__ __forceinline__ void cls2(const uint16_t *p, int &c0, int &c1)
{
    const unsigned v = *reinterpret_cast<const uint32_t *>(p);
    c0 = (int)(v & 0xFFFFu);
    c1 = (int)(v >> 16);
}

// Persistent CTAs drawing tasks: column (tx, ty) of SX x SY cells (Tile<SX>),
// planes [k0, k1).  The CTA walks the items k = k0-1 (H only, for the curl of
// plane k0), k0, ..., k1 (the plane above, for E^{n+1} there; zeros beyond the
// grid).  Item q lives in stage q % kNS.  Each tile row is SX/2 lanes, each
// lane owning the cell pair (x, x+1), so shared-memory and global accesses
// move float2 pairs and x neighbours come from the pair itself.  Per item: E^{n+1} of
// plane k at the tile's own cells, one barrier, then H of plane k-1 and
// E^{n+1} of plane k at the halo edges that the next item's H update reads (Ex
// and Ez of the row above the tile, Ey and Ez of the column beyond it).  After
// the barrier of item q the stage of item q-2 has no readers left and receives
// item q + kNS - 2.  The tensor maps zero-fill everything outside the grid and
// class 0 has zero coefficients, so cells beyond the far walls get E^{n+1} = 0
// and H = 0 without a branch.
template <typename ClsT, bool STAB, int SX>
__global__ void __launch_bounds__(kST, 3) step_kernel(LaunchSet L)
{
    extern __shared__ __align__(128) unsigned char stg[];
    __shared__ uint64_t bar[kNS];
    __shared__ float4 stab[STAB ? 3 * kTabMax : 1];
    __shared__ double sred[kST / 32];
    __shared__ int s_last, s_abort, s_task;
    __shared__ uint64_t s_never;   // the diagnostic wait's barrier (L.test_wait): nothing arrives on it
    using TL = Tile<SX>;
    constexpr int SY = TL::Y, LPR = TL::LPR, HBX = TL::HBX, HC = TL::HC, EBX = TL::EBX, EBY = TL::EBY, EC = TL::EC;
    constexpr int CBX = sizeof(ClsT) == 1 ? TL::CBX8 : TL::CBX16;
    constexpr unsigned kClsBytes = CBX * EBY * sizeof(ClsT);
    static_assert((SX == 64 || SX == 32) && LPR * SY == kST && kClsBytes <= (unsigned)(kStageBytes - kStageCOff),
                  "one cell pair per lane; the class box fits its stage area");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long n = *(volatile long long *)&L.ctl->step;
    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) mbar_init(&bar[s], 1);
        mbar_init(&s_never, 1);
        fence_barrier_init();
        fence_proxy_async();
        s_abort = 0;
    }
    __syncthreads();
    // persistent CTA: tasks come from a device counter; item g (counted over
    // all of this CTA's tasks) lives in stage g % kNS with phase parity (g / kNS) & 1
    long long gbase = 0;                      // items of the earlier tasks
    long long issued = 0, consumed = 0;       // items issued (thread 0) / waited for
    const Inst *Iprev = nullptr;
    // the first nred values of the task counter are the previous step's
    // per-instance energy sums, the rest the sweep tasks
    const int nred = L.energy ? L.ninst : 0;
    double *const pf = L.part_f + (n & 1) * L.part_stride;
    for (;;) {
    if (tid == 0) s_task = (int)atomicAdd(&L.ctl->work, 1u);
    fence_proxy_async();
    __syncthreads();
    const int v = s_task;
    if (v >= nred + L.nftiles || s_abort) break;
    if (v < nred) {
        reduce_energy<8>(L, v, n - 1, sred);
        __syncthreads();   // every thread has read s_task before thread 0 draws again
        continue;
    }
    // task t of the host's schedule: instance, column (tx, ty), planes
    // [k0, k1), slot of its energy partials within the instance's range
    const int4 tk = L.ftask[v - nred];
    const Inst *I = L.insts + tk.x;
    const int tx = (int)((unsigned)tk.y & 0xFFFFu), ty = (int)((unsigned)tk.y >> 16);
    const int k0 = (int)((unsigned)tk.z & 0xFFFFu), k1 = (int)((unsigned)tk.z >> 16), slot = tk.w;
    const int nx = I->nx, ny = I->ny, px = I->px;
    const unsigned plane = (unsigned)I->plane;
    const long long fs = I->fstride;
    const int i0 = tx * SX, j0 = ty * SY;
    const int nitems = k1 - k0 + 2;
    const float4 *__restrict__ ctab = I->ctab;
    const bool has_mag = I->nmag > 0;
    const float idx = I->idx, idy = I->idy, idz = I->idz, ch = I->ch;
    const CUtensorMap *tmH = &I->tm[TM_H0 + L.src], *tmE = &I->tm[TM_E0 + L.src], *tmC = &I->tm[TM_CLS];
    auto tab = [&](int i) -> float4 {
        if constexpr (STAB) return stab[i];
        else return __ldg(ctab + i);
    };

    auto issue = [&](int q) {
        const int k = k0 - 1 + q;
        const long long g = gbase + q;
        unsigned char *base = stg + (int)(g % kNS) * kStageBytes;
        uint64_t *b = &bar[g % kNS];
        if (q == 0) {
            mbar_expect_tx(b, kStageH);
            tma_load_4d(base + kStageHOff, tmH, i0 - 4, j0 - 1, k, 3, b);
        } else {
            mbar_expect_tx(b, kStageH + kStageE + kClsBytes);
            tma_load_4d(base + kStageHOff, tmH, i0 - 4, j0 - 1, k, 3, b);
            tma_load_4d(base + kStageEOff, tmE, i0, j0, k, 0, b);
            tma_load_3d(base + kStageCOff, tmC, i0, j0, k, b);
        }
        issued = g + 1;
    };
    if (tid == 0) {
        if (I != Iprev) {
            tmap_acquire(tmH);
            tmap_acquire(tmE);
            tmap_acquire(tmC);
        }
        for (int q = 0; q < min(kNS - 1, nitems); ++q) issue(q);
    }
    if constexpr (STAB) {
        if (I != Iprev) {   // the class table of this task's instance
            for (int c = tid; c < 3 * I->nclass; c += kST) stab[c] = __ldg(ctab + c);
        }
    }
    Iprev = I;

    // sources and probes whose column lies in this tile's extended / interior area
    unsigned smask = 0, pmask = 0;
    for (int s = 0; s < I->nsrc; ++s) {
        const int si = I->src[s][1] - i0, sj = I->src[s][2] - j0;
        if (si >= 0 && si <= SX && sj >= 0 && sj <= SY) smask |= 1u << s;
    }
    for (int p = 0; p < I->nprobe; ++p) {
        const int pi = I->probe[p][0] - i0, pj = I->probe[p][1] - j0;
        if (pi >= 0 && pi < SX && pj >= 0 && pj < SY && I->probe[p][2] >= k0 && I->probe[p][2] < k1) pmask |= 1u << p;
    }
    const double tn = ((double)n + 0.5) * I->dt;
    // source current (FP64 time evaluation) subtracted from one curl component
    auto add_src = [&](int i, int j, int k, float &cx, float &cy, float &cz) {
        for (int so = 0; so < I->nsrc; ++so)
            if (((smask >> so) & 1u) && I->src[so][1] == i && I->src[so][2] == j && I->src[so][3] == k) {
                const float J = (float)source_value(I->srcp[so], tn);
                if (I->src[so][0] == 0) cx = __fsub_rn(cx, J);
                else if (I->src[so][0] == 1) cy = __fsub_rn(cy, J);
                else cz = __fsub_rn(cz, J);
            }
    };
    auto probe_row = [&](int pp) { return I->probe_buf + ((long long)(n % I->cap) * I->nprobe + pp) * 9; };

    // this thread's cells: (x, y), (x+1, y); output pointers per component
    const int x = 2 * (lane % LPR), y = w * (32 / LPR) + lane / LPR;
    const int gi = i0 + x, gj = j0 + y;
    const bool in = gi < nx && gj < ny;   // gi + 1 < px always: the pair stays in the padded row
    const unsigned ob = (unsigned)gj * (unsigned)px + (unsigned)gi;
    float *const F0 = I->F[L.dst][0];
    float *const Fx = F0, *const Fy = F0 + fs, *const Fz = F0 + 2 * fs;
    float *const Gx = F0 + 3 * fs, *const Gy = F0 + 4 * fs, *const Gz = F0 + 5 * fs;
    const int hp = (y + 1) * HBX + x + 4;   // (x, y) in the H box
    const int ep = y * EBX + x;             // (x, y) in the E box
    __syncthreads();

    float acc = 0.f, acc_c = 0.f;   // energy of this thread's cells, compensated
    // this thread's own two cells carried from plane to plane in registers: H
    // of the previous plane, E^{n+1} of the previous plane; only neighbours'
    // values come from shared memory
    float2 cHX = make_float2(0.f, 0.f), cHY = cHX, cHZ = cHX, cEX = cHX, cEY = cHX, cEZ = cHX;
    for (int q = 0; q < nitems; ++q) {
        const long long g = gbase + q;
        const int s = (int)(g % kNS), sp = (int)((g + kNS - 1) % kNS);
        bool landed = mbar_wait(&bar[s], (unsigned)(g / kNS) & 1u);
        // diagnostic of the timeout path (L.test_wait > 0): after its first
        // item has landed, CTA 0 also waits on a barrier that nothing arrives
        // on, at most L.test_wait polls, as for a copy that never lands
        if (landed && L.test_wait > 0 && blockIdx.x == 0 && g == 0) landed = mbar_wait(&s_never, 0u, L.test_wait);
        if (!landed) {
            atomicOr(&L.ctl->status, ST_TIMEOUT);
            s_abort = 1;
        }
        consumed = g + 1;
        const int k = k0 - 1 + q;
        unsigned char *cur = stg + s * kStageBytes, *prv = stg + sp * kStageBytes;
        const float *Hc = reinterpret_cast<const float *>(cur + kStageHOff);
        const float *Hp = reinterpret_cast<const float *>(prv + kStageHOff);
        float *Ec = reinterpret_cast<float *>(cur + kStageEOff);
        const ClsT *Cc = reinterpret_cast<const ClsT *>(cur + kStageCOff);
        float2 nHX, nHY, nHZ, nEX, nEY, nEZ;   // this plane's values of the own cells
        if (q == 0) {
            nHX = ld2(Hc + hp);
            nHY = ld2(Hc + HC + hp);
            nHZ = ld2(Hc + 2 * HC + hp);
            nEX = nEY = nEZ = make_float2(0.f, 0.f);
        } else {
            // ---- E^{n+1} of plane k at the tile's cells, in place over E^n
            const float2 HX = ld2(Hc + hp), HY = ld2(Hc + HC + hp), HZ = ld2(Hc + 2 * HC + hp);
            const float2 HXj = ld2(Hc + hp - HBX), HZj = ld2(Hc + 2 * HC + hp - HBX);
            const float hyi = Hc[HC + hp - 1], hzi = Hc[2 * HC + hp - 1];
            const float2 HXk = cHX, HYk = cHY;
            const float2 EX = ld2(Ec + ep), EY = ld2(Ec + EC + ep), EZ = ld2(Ec + 2 * EC + ep);
            int c0, c1;
            cls2(Cc + y * CBX + x, c0, c1);
            float cx0 = curl2(HZ.x, HZj.x, idy, HY.x, HYk.x, idz);
            float cy0 = curl2(HX.x, HXk.x, idz, HZ.x, hzi, idx);
            float cz0 = curl2(HY.x, hyi, idx, HX.x, HXj.x, idy);
            float cx1 = curl2(HZ.y, HZj.y, idy, HY.y, HYk.y, idz);
            float cy1 = curl2(HX.y, HXk.y, idz, HZ.y, HZ.x, idx);
            float cz1 = curl2(HY.y, HY.x, idx, HX.y, HXj.y, idy);
            if (smask) {
                add_src(gi, gj, k, cx0, cy0, cz0);
                add_src(gi + 1, gj, k, cx1, cy1, cz1);
            }
            const float4 A0 = tab(3 * c0), B0 = tab(3 * c0 + 1), A1 = tab(3 * c1), B1 = tab(3 * c1 + 1);
            const float ex0 = e_next(A0.x, EX.x, B0.x, cx0), ey0 = e_next(A0.y, EY.x, B0.y, cy0), ez0 = e_next(A0.z, EZ.x, B0.z, cz0);
            const float ex1 = e_next(A1.x, EX.y, B1.x, cx1), ey1 = e_next(A1.y, EY.y, B1.y, cy1), ez1 = e_next(A1.z, EZ.y, B1.z, cz1);
            st2(Ec + ep, ex0, ex1);
            st2(Ec + EC + ep, ey0, ey1);
            st2(Ec + 2 * EC + ep, ez0, ez1);
            nHX = HX;
            nHY = HY;
            nHZ = HZ;
            nEX = make_float2(ex0, ex1);
            nEY = make_float2(ey0, ey1);
            nEZ = make_float2(ez0, ez1);
            if (k < k1 && in) {
                const unsigned o = (unsigned)k * plane + ob;
                st2(Fx + o, ex0, ex1);
                st2(Fy + o, ey0, ey1);
                st2(Fz + o, ez0, ez1);
                const float4 Q0 = tab(3 * c0 + 2), Q1 = tab(3 * c1 + 2);
                sum2_add(acc, acc_c, Q0.x * ex0 * ex0 + Q0.y * ey0 * ey0 + Q0.z * ez0 * ez0 + Q1.x * ex1 * ex1 +
                                          Q1.y * ey1 * ey1 + Q1.z * ez1 * ez1);
                if (pmask) {
                    for (int pp = 0; pp < I->nprobe; ++pp)
                        if (((pmask >> pp) & 1u) && I->probe[pp][1] == gj && I->probe[pp][2] == k &&
                            (I->probe[pp][0] == gi || I->probe[pp][0] == gi + 1)) {
                            const bool second = I->probe[pp][0] != gi;
                            double *row = probe_row(pp);
                            row[0] = second ? ex1 : ex0;
                            row[1] = second ? ey1 : ey0;
                            row[2] = second ? ez1 : ez0;
                        }
                }
            }
        }
        // every generic write to the stage of item q-2 is ordered before the
        // TMA that overwrites it
        fence_proxy_async();
        __syncthreads();
        if (s_abort) break;
        if (tid == 0 && q >= 1 && q + kNS - 2 < nitems) issue(q + kNS - 2);
        // ---- H^{n+1} and H^{n+3/2} of plane k-1 at the tile's cells
        if (q > 1) {
            const float *Ep = reinterpret_cast<const float *>(prv + kStageEOff);
            const ClsT *Cp = reinterpret_cast<const ClsT *>(prv + kStageCOff);
            const float2 EX = cEX, EY = cEY, EZ = cEZ;
            const float2 EXj = ld2(Ep + ep + EBX), EZj = ld2(Ep + 2 * EC + ep + EBX);
            const float eyi = Ep[EC + ep + 2], ezi = Ep[2 * EC + ep + 2];
            const float2 EXk = nEX, EYk = nEY;
            const float2 HX = cHX, HY = cHY, HZ = cHZ;
            const float cx0 = curl2(EZj.x, EZ.x, idy, EYk.x, EY.x, idz);
            const float cy0 = curl2(EXk.x, EX.x, idz, EZ.y, EZ.x, idx);
            const float cz0 = curl2(EY.y, EY.x, idx, EXj.x, EX.x, idy);
            const float cx1 = curl2(EZj.y, EZ.y, idy, EYk.y, EY.y, idz);
            const float cy1 = curl2(EXk.y, EX.y, idz, ezi, EZ.y, idx);
            const float cz1 = curl2(eyi, EY.y, idx, EXj.y, EX.y, idy);
            uint32_t f0 = 0, f1 = 0;
            if (has_mag) {
                int c0, c1;
                cls2(Cp + y * CBX + x, c0, c1);
                f0 = __float_as_uint(tab(3 * c0).w);
                f1 = __float_as_uint(tab(3 * c1).w);
            }
            // the two half-pushes H - ch c - ch c, each one fused step; zero
            // where the face is magnetic (the magnet kernel owns it)
            const float mch = -ch;
            const float hx0 = (f0 & CF_MAG_HX) ? 0.f : __fmaf_rn(mch, cx0, HX.x);
            const float hy0 = (f0 & CF_MAG_HY) ? 0.f : __fmaf_rn(mch, cy0, HY.x);
            const float hz0 = (f0 & CF_MAG_HZ) ? 0.f : __fmaf_rn(mch, cz0, HZ.x);
            const float hx1 = (f1 & CF_MAG_HX) ? 0.f : __fmaf_rn(mch, cx1, HX.y);
            const float hy1 = (f1 & CF_MAG_HY) ? 0.f : __fmaf_rn(mch, cy1, HY.y);
            const float hz1 = (f1 & CF_MAG_HZ) ? 0.f : __fmaf_rn(mch, cz1, HZ.y);
            if (in) {
                const unsigned o = (unsigned)(k - 1) * plane + ob;
                if (!((f0 | f1) & (CF_MAG_HX | CF_MAG_HY | CF_MAG_HZ))) {
                    st2(Gx + o, __fmaf_rn(mch, cx0, hx0), __fmaf_rn(mch, cx1, hx1));
                    st2(Gy + o, __fmaf_rn(mch, cy0, hy0), __fmaf_rn(mch, cy1, hy1));
                    st2(Gz + o, __fmaf_rn(mch, cz0, hz0), __fmaf_rn(mch, cz1, hz1));
                } else {
                    if (!(f0 & CF_MAG_HX)) Gx[o] = __fmaf_rn(mch, cx0, hx0);
                    if (!(f0 & CF_MAG_HY)) Gy[o] = __fmaf_rn(mch, cy0, hy0);
                    if (!(f0 & CF_MAG_HZ)) Gz[o] = __fmaf_rn(mch, cz0, hz0);
                    if (!(f1 & CF_MAG_HX)) Gx[o + 1] = __fmaf_rn(mch, cx1, hx1);
                    if (!(f1 & CF_MAG_HY)) Gy[o + 1] = __fmaf_rn(mch, cy1, hy1);
                    if (!(f1 & CF_MAG_HZ)) Gz[o + 1] = __fmaf_rn(mch, cz1, hz1);
                }
                sum2_add(acc, acc_c, (float)(0.5 * kMu0) * (hx0 * hx0 + hy0 * hy0 + hz0 * hz0 + hx1 * hx1 + hy1 * hy1 + hz1 * hz1));
                if (pmask) {
                    for (int pp = 0; pp < I->nprobe; ++pp)
                        if (((pmask >> pp) & 1u) && I->probe[pp][1] == gj && I->probe[pp][2] == k - 1 &&
                            (I->probe[pp][0] == gi || I->probe[pp][0] == gi + 1)) {
                            const bool second = I->probe[pp][0] != gi;
                            const uint32_t f = second ? f1 : f0;
                            double *row = probe_row(pp);
                            if (!(f & CF_MAG_HX)) row[3] = second ? hx1 : hx0;
                            if (!(f & CF_MAG_HY)) row[4] = second ? hy1 : hy0;
                            if (!(f & CF_MAG_HZ)) row[5] = second ? hz1 : hz0;
                        }
                }
            }
        }
        // ---- E^{n+1} of plane k at the halo edges read by the next item:
        // threads [0, SX) Ex and Ez of row SY (cell pairs), the next 2 SY Ey
        // and Ez of column SX (64 x 8: warps 0, 1 and half of warp 2; 32 x 16:
        // warps 0 and 1)
        if (q > 0 && q + 1 < nitems && tid < SX + 2 * SY) {
            if (tid < SX) {
                const int hx = 2 * (tid % LPR);   // pair of row SY
                const int hr = (SY + 1) * HBX + hx + 4, er = SY * EBX + hx;
                const int hgi = i0 + hx;
                int c0, c1;
                cls2(Cc + SY * CBX + hx, c0, c1);
                const float4 A0 = tab(3 * c0), B0 = tab(3 * c0 + 1), A1 = tab(3 * c1), B1 = tab(3 * c1 + 1);
                if (tid < LPR) {
                    const float2 HZ = ld2(Hc + 2 * HC + hr), HZj = ld2(Hc + 2 * HC + hr - HBX);
                    const float2 HY = ld2(Hc + HC + hr), HYk = ld2(Hp + HC + hr);
                    float cx0 = curl2(HZ.x, HZj.x, idy, HY.x, HYk.x, idz), cx1 = curl2(HZ.y, HZj.y, idy, HY.y, HYk.y, idz);
                    if (smask) {
                        float d0 = 0.f, d1 = 0.f;
                        add_src(hgi, j0 + SY, k, cx0, d0, d1);
                        add_src(hgi + 1, j0 + SY, k, cx1, d0, d1);
                    }
                    const float2 EN = ld2(Ec + er);
                    st2(Ec + er, e_next(A0.x, EN.x, B0.x, cx0), e_next(A1.x, EN.y, B1.x, cx1));
                } else {
                    const float2 HY = ld2(Hc + HC + hr), HX = ld2(Hc + hr), HXj = ld2(Hc + hr - HBX);
                    const float hyi = Hc[HC + hr - 1];
                    float cz0 = curl2(HY.x, hyi, idx, HX.x, HXj.x, idy), cz1 = curl2(HY.y, HY.x, idx, HX.y, HXj.y, idy);
                    if (smask) {
                        float d0 = 0.f, d1 = 0.f;
                        add_src(hgi, j0 + SY, k, d0, d1, cz0);
                        add_src(hgi + 1, j0 + SY, k, d0, d1, cz1);
                    }
                    const float2 EN = ld2(Ec + 2 * EC + er);
                    st2(Ec + 2 * EC + er, e_next(A0.z, EN.x, B0.z, cz0), e_next(A1.z, EN.y, B1.z, cz1));
                }
            } else {
                const int cid = tid - SX, yc = cid % SY;   // cid < SY: Ey, else Ez of row yc
                const int hc = (yc + 1) * HBX + SX + 4, ec = yc * EBX + SX;
                const int c = (int)Cc[yc * CBX + SX];
                const float4 A = tab(3 * c), B = tab(3 * c + 1);
                if (cid < SY) {
                    float cy = curl2(Hc[hc], Hp[hc], idz, Hc[2 * HC + hc], Hc[2 * HC + hc - 1], idx);
                    if (smask) {
                        float d0 = 0.f, d1 = 0.f;
                        add_src(i0 + SX, j0 + yc, k, d0, cy, d1);
                    }
                    Ec[EC + ec] = e_next(A.y, Ec[EC + ec], B.y, cy);
                } else {
                    float cz = curl2(Hc[HC + hc], Hc[HC + hc - 1], idx, Hc[hc], Hc[hc - HBX], idy);
                    if (smask) {
                        float d0 = 0.f, d1 = 0.f;
                        add_src(i0 + SX, j0 + yc, k, d0, d1, cz);
                    }
                    Ec[2 * EC + ec] = e_next(A.z, Ec[2 * EC + ec], B.z, cz);
                }
            }
        }
        cHX = nHX;
        cHY = nHY;
        cHZ = nHZ;
        cEX = nEX;
        cEY = nEY;
        cEZ = nEZ;
    }
    if (L.energy) {   // one partial per warp: no block barrier per task
        double e = (double)acc + (double)acc_c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) pf[(long long)slot * kSW + w] = e;
    }
    gbase += nitems;
    }
    // after a timed-out wait: wait (bounded) for the copies still in flight
    if (tid == 0)
        for (long long g = consumed; g < issued; ++g) mbar_wait(&bar[g % kNS], (unsigned)(g / kNS) & 1u);
    finish_step(L, n, &s_last);
}

// Steps [n0, n1) of instance I's probe rows and energies from the device
// rings into the host ring R (every thread of the CTA).  Only the newest
// min(I->cap, R.cap) steps: the device rings hold the last I->cap, and an
// older step would share a host slot with a newer one.
__device__ void copy_out(const Inst *I, const HostRing &R, long long n0, long long n1)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long dcap = I->cap;
    const long long a = max(n0, n1 - min(dcap, R.cap));
    if (R.energy)
        for (long long st = a + tid; st < n1; st += nth) R.energy[st % R.cap] = I->energy_buf[st % dcap];
    const int w = I->nprobe * 9;
    if (R.rows && w)
        for (long long q = tid; q < (n1 - a) * w; q += nth) {
            const long long st = a + q / w;
            const int r = (int)(q % w);
            R.rows[(st % R.cap) * w + r] = I->probe_buf[(st % dcap) * w + r];
        }
}

// After the last step of a call.  With the energy on, one CTA per chunk of
// the pending step's partials (kST threads, as the sweep's reduction task,
// so that the sums are the same bits): the CTA that sums an instance's last
// outstanding chunk adds the chunk sums in order, and the CTA that completes
// the last instance clears the pending step (the next step's sweep then does
// not sum it again).  With the energy off, one CTA per instance.  The CTA that
// completes an instance (with nothing pending, its first one) then copies the
// call's steps [n0, n1) of the instance's results into its host ring (n1 < 0:
// the one step that the device step counter last completed).
__global__ void __launch_bounds__(kST) energy_flush_kernel(LaunchSet L, const HostRing *rings, long long n0, long long n1)
{
    __shared__ double sred[kST / 32];
    __shared__ int s_out;
    const int tid = threadIdx.x;
    if (n1 < 0) {   // a replayed one-step call: the step just completed
        n1 = *(volatile long long *)&L.ctl->step;
        n0 = n1 - 1;
    }
    int ii = blockIdx.x, c = 0;
    if (L.energy) {
        const int2 rt = L.ered[blockIdx.x];
        ii = rt.x;
        c = rt.y;
    }
    const Inst *I = L.insts + ii;
    const long long m = L.energy ? *(volatile long long *)&L.ctl->epend : -1;
    if (m >= 0) {
        const double *pf = L.part_f + (m & 1) * L.part_stride, *pm = L.part_m + (m & 1) * L.part_stride;
        const int nch = energy_chunks(I->fntask);
        const double sc = chunk_sum<32>(I, c, nch, pf, pm, L.mag_cs, sred);
        if (tid == 0) {
            int done = 0;
            L.esum[ii * kEChunks + c] = sc;
            __threadfence();
            if (atomicAdd(&L.ecnt[ii], 1u) == (unsigned)(nch - 1)) {
                __threadfence();
                double t = 0.0;
                for (int k = 0; k < nch; ++k) t += __ldcg(L.esum + ii * kEChunks + k);
                store_energy(L, I, t, m);
                L.ecnt[ii] = 0u;
                done = 1;
                if (atomicAdd(&L.ctl->eflush, 1u) == (unsigned)(L.ninst - 1)) {
                    L.ctl->eflush = 0u;
                    L.ctl->epend = -1;
                }
            }
            s_out = done;
        }
    } else if (tid == 0) {
        s_out = c == 0;
    }
    __syncthreads();
    if (s_out && rings && n1 > n0) copy_out(I, rings[ii], n0, n1);
}

__global__ void set_step_kernel(StepCtl *ctl, long long n)
{
    ctl->step = n;
    ctl->counter = 0u;
    ctl->work = 0u;
    ctl->epend = -1;
    ctl->eflush = 0u;
}

}  // namespace

cudaError_t set_device_step(StepCtl *ctl, long long n, cudaStream_t s)
{
    set_step_kernel<<<1, 1, 0, s>>>(ctl, n);
    return cudaGetLastError();
}

int h_half_blocks_per_sm(bool cls16)
{
    int nb = 0;
    if (cls16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_half_kernel<uint16_t>, kTX * kTY, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h_half_kernel<uint8_t>, kTX * kTY, 0);
    return nb > 0 ? nb : 1;
}

static constexpr int kStepSmem = kNS * kStageBytes;

using StepFn = void (*)(LaunchSet);
// The sweep instantiation for a class width, a class table in shared memory
// or not, and a tile width (64 or 32).
static StepFn step_fn(bool cls16, bool stab, int sx)
{
    if (sx == 32) {
        if (cls16) return stab ? step_kernel<uint16_t, true, 32> : step_kernel<uint16_t, false, 32>;
        return stab ? step_kernel<uint8_t, true, 32> : step_kernel<uint8_t, false, 32>;
    }
    if (cls16) return stab ? step_kernel<uint16_t, true, 64> : step_kernel<uint16_t, false, 64>;
    return stab ? step_kernel<uint8_t, true, 64> : step_kernel<uint8_t, false, 64>;
}

// The magnet kernel with c cells per thread (1, 2, 4 or kMagCPT): the fewest
// that cover the largest region of the launch, so that the per-thread
// arrays and the unrolled cell loop hold no cells that cannot exist.
template <bool FUSED, typename ClsT, bool CL>
static void (*mag_fn_cl(int c))(LaunchSet)
{
    static_assert(kMagCPT == 8, "cells per thread: 1, 2, 4 or 8");
    if (c <= 1) return mag_kernel<FUSED, ClsT, 1, CL>;
    if (c <= 2) return mag_kernel<FUSED, ClsT, 2, CL>;
    if (c <= 4) return mag_kernel<FUSED, ClsT, 4, CL>;
    return mag_kernel<FUSED, ClsT, 8, CL>;
}
// the instantiation for c cells per thread, split over a cluster or not
template <bool FUSED, typename ClsT>
static void (*mag_fn(int c, bool cl))(LaunchSet)
{
    return cl ? mag_fn_cl<FUSED, ClsT, true>(c) : mag_fn_cl<FUSED, ClsT, false>(c);
}

static int mag_cpt(int vmax) { return vmax <= kMagThreads ? 1 : vmax <= 2 * kMagThreads ? 2 : vmax <= 4 * kMagThreads ? 4 : 8; }
// Threads of a magnet CTA.  Unsplit regions: one per cell of the launch's
// largest region when it holds at most kMagThreads cells (rounded up to a
// power of two, at least 128), so that small regions leave the SM's
// registers to the field sweep running beside them; kMagThreads otherwise.
// Regions split over a cluster (cs > 1, chosen where the magnet kernel bounds
// the step): kMagThreads, since a slab has about three faces and as many edge
// components per cell, whose set-up, face and output loops then take one pass
// instead of several (measured on the 16x16x4 block of the 128x128x64 design
// case at 8 CTAs: 31.0 -> 25.4 us per magnet launch).
static int mag_threads(int vmax, int cs)
{
    if (cs > 1) return kMagThreads;
    int t = 128;
    while (t < vmax && t < kMagThreads) t *= 2;
    return t;
}

static cudaError_t step_attrs()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 8 && e == cudaSuccess; ++q)
        e = cudaFuncSetAttribute(step_fn(q & 1, (q >> 1) & 1, (q & 4) ? 32 : 64), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kStepSmem);
    for (int c = 1; c <= kMagCPT && e == cudaSuccess; c *= 2)
        for (int cl = 0; cl < 2 && e == cudaSuccess; ++cl) {
            e = cudaFuncSetAttribute(mag_fn<true, uint8_t>(c, cl), cudaFuncAttributeMaxDynamicSharedMemorySize, kMagSmemMax);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(mag_fn<true, uint16_t>(c, cl), cudaFuncAttributeMaxDynamicSharedMemorySize, kMagSmemMax);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(mag_fn<false, uint8_t>(c, cl), cudaFuncAttributeMaxDynamicSharedMemorySize, kMagSmemMax);
        }
    done = e == cudaSuccess;
    return e;
}

int step_blocks_per_sm(bool cls16, bool stab, int sx)
{
    if (step_attrs() != cudaSuccess) return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_fn(cls16, stab, sx), kST, kStepSmem);
    return nb;
}

// The magnet kernel fn over every region, L.mag_cs CTAs (one cluster) each.
static cudaError_t launch_mag(void (*fn)(LaunchSet), const LaunchSet &L, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(L.ncomp * L.mag_cs);
    cfg.blockDim = dim3(mag_threads(L.vmax, L.mag_cs));
    cfg.dynamicSmemBytes = L.mag_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = L.mag_cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = L.mag_cs > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fn, L);
}

cudaError_t launch_half(const LaunchSet &L, cudaStream_t s)
{
    cudaError_t e = step_attrs();
    if (e != cudaSuccess) return e;
    if (L.ncomp) {
        e = launch_mag(mag_fn<false, uint8_t>(mag_cpt(L.vmax), L.mag_cs > 1), L, s);
        if (e != cudaSuccess) return e;
    }
    const dim3 blk(kTX, kTY);
    if (L.cls16) h_half_kernel<uint16_t><<<L.grid_h, blk, 0, s>>>(L);
    else h_half_kernel<uint8_t><<<L.grid_h, blk, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_energy_flush(const LaunchSet &L, const HostRing *rings, long long n0, long long n1, cudaStream_t s)
{
    const int grid = L.energy ? L.nred : (rings ? L.ninst : 0);
    if (grid < 1) return cudaSuccess;
    energy_flush_kernel<<<grid, kST, 0, s>>>(L, rings, n0, n1);
    return cudaGetLastError();
}

// One full step on stream s: the magnet kernel first, then the field sweep as
// its programmatic dependent (PDL), so the sweep's CTAs are dispatched as soon
// as the magnet CTAs are resident and the two run side by side; the next
// step's magnet kernel, a plain launch, waits for both.  With prof (four
// events) the events split the two and they run one after the other.
cudaError_t launch_step(const LaunchSet &L, cudaStream_t s, cudaEvent_t *prof)
{
    cudaError_t e = step_attrs();
    if (e != cudaSuccess) return e;
    if (L.ncomp) {
        if (prof) cudaEventRecord(prof[2], s);
        e = launch_mag(L.cls16 ? mag_fn<true, uint16_t>(mag_cpt(L.vmax), L.mag_cs > 1)
                               : mag_fn<true, uint8_t>(mag_cpt(L.vmax), L.mag_cs > 1), L, s);
        if (e != cudaSuccess) return e;
        if (prof) cudaEventRecord(prof[3], s);
    }
    if (prof) cudaEventRecord(prof[0], s);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(L.nfblocks);
    cfg.blockDim = dim3(kST);
    cfg.dynamicSmemBytes = kStepSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (L.ncomp && !prof) ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, step_fn(L.cls16, L.stab, L.sx), L);
    if (e != cudaSuccess) return e;
    if (prof) cudaEventRecord(prof[1], s);
    return cudaGetLastError();
}

}  // namespace fl
