// Kernels of the physics-informed sequence surrogate (include/lem_surrogate.h):
// the LEM encoder-decoder forward pass (Eq. discrete_lem), the data and
// trapezoidal-LLG physics losses (Eqs. ml_tra1-3 with Eqs. llg_tra4-6), the
// back-propagation through both stacks, the gate-gradient sums that give the
// weight gradients, and Adam.
//
// Recurrent kernels.  One CTA advances 4 R sequences (R = 1 or 2) through
// every step of both stacks, with the two cells' weights of the stack in
// shared memory (about 200 KB at D = 64) and the states beside them; 4 D
// threads.  In a product W y (or W^T g) thread (i, r) sums, for output i,
// the summed indices of quarter r for every sequence of the CTA, so each
// weight read from shared memory serves all 4 R sequences; the 4 lanes of
// an output then reduce-scatter by warp shuffles, lane r keeping the sums of
// sequences r + 4 rr, whose element-wise updates it makes.  The time loop is
// sequential, so a step costs a chain of dependent phases (the gates and z,
// one barrier, y, one barrier, per cell; the head, one barrier) rather than
// bandwidth; the batch is spread over ceil(batch / 4 R) CTAs.  Activations
// of every step are saved (y, z, the two sigmoid gates and the two tanh
// values) for the reverse pass.
//
// Weight gradients.  The reverse kernel stores the gradients of the four gate
// pre-activations of every step; each weight gradient is then a sum over
// (step, sequence) rows of an outer product with a saved activation, summed
// by row chunks into partials and the partials in chunk order, so the result
// is the same bits for any batch split.
#include "../../include/fdtd_llg.h"
#include "../../include/lem_surrogate.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

namespace fl {
void set_last_error(const char *msg);
}

namespace {

constexpr int kG = 4;            // sequence groups per CTA
// sequences per thread R (1 or 2, chosen at launch so that the batch covers
// the SMs); a CTA holds kG R sequences
constexpr int kMMax = 4;         // largest input / output width
constexpr int kQ = 6;            // saved values per unit and step: y, z, s1, s2, tz, ty
constexpr int kKC = 2048;        // rows per chunk of the weight-gradient sums
constexpr int kLossThreads = 256;

__host__ __device__ inline long long cell_params(int d, int mc) { return 4LL * d * d + 4LL * d * mc + 4LL * d; }
__host__ __device__ inline int cell_width(int c, int m, int d) { return (c & 1) ? d : m; }
// offset of cell c (0 enc0, 1 enc1, 2 dec0, 3 dec1); c = 4: the head Wo
__host__ __device__ inline long long cell_offset(int c, int d, int m)
{
    long long o = 0;
    for (int q = 0; q < c; ++q) o += cell_params(d, cell_width(q, m, d));
    return o;
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Work-space layout (offsets in bytes, 256-aligned)
struct Layout {
    size_t act[2][2];   // [phase][layer] -> [T_ph + 1][B][kQ][D]
    size_t dg[2][2];    // [phase][layer] -> [T_ph][B][4][D]
    size_t xdec;        // [t_out][B][m] decoder inputs
    size_t recon, out, drec, dout, dot;
    size_t lpart, loss; // per-block loss partials [nblk][3] (double), losses [4] (double)
    size_t grad;        // [P] float
    size_t wpart;       // weight-gradient partials (float)
    size_t total;
    int nlblk;
    long long nwpart;
};

struct WProd {
    const float *A, *A2, *B, *B2;   // B == nullptr: the constant 1
    long long lda, ldb, K1, K;
    int aoff, boff, R, J;
    long long goff, poff;
    int chunk0, nchunk;
};
constexpr int kMaxProd = 17;
struct WProdSet {
    WProd p[kMaxProd];
    int np, nchunks;
};

bool shape_ok(const fdtd_llg_lem_shape *s)
{
    return s && (s->d == 16 || s->d == 32 || s->d == 64) && s->m >= 1 && s->m <= kMMax && s->batch >= 1 &&
           s->t_in >= 1 && s->t_out >= 1 && (long long)s->t_in + s->t_out <= 65536 && s->dt > 0.f &&
           std::isfinite(s->dt);
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(const fdtd_llg_lem_shape *s)
{
    Layout L{};
    const size_t B = s->batch, D = s->d, m = s->m;
    const size_t T[2] = {(size_t)s->t_in, (size_t)s->t_out};
    size_t o = 0;
    for (int ph = 0; ph < 2; ++ph)
        for (int l = 0; l < 2; ++l) {
            L.act[ph][l] = o;
            o += al((T[ph] + 1) * B * kQ * D * sizeof(float));
        }
    for (int ph = 0; ph < 2; ++ph)
        for (int l = 0; l < 2; ++l) {
            L.dg[ph][l] = o;
            o += al(T[ph] * B * 4 * D * sizeof(float));
        }
    L.xdec = o; o += al(T[1] * B * m * sizeof(float));
    L.recon = o; o += al(T[0] * B * m * sizeof(float));
    L.out = o; o += al(T[1] * B * m * sizeof(float));
    L.drec = o; o += al(T[0] * B * m * sizeof(float));
    L.dout = o; o += al(T[1] * B * m * sizeof(float));
    L.dot = o; o += al(T[1] * B * m * sizeof(float));
    const size_t nl = (T[0] * B * m + T[1] * B + kLossThreads - 1) / kLossThreads;
    L.nlblk = (int)nl;
    L.lpart = o; o += al(nl * 3 * sizeof(double));
    L.loss = o; o += al(4 * sizeof(double));
    L.grad = o; o += al((size_t)fdtd_llg_lem_param_count(s->d, s->m) * sizeof(float));
    // partials: per product ceil(K / kKC) chunks of R x J
    long long np = 0;
    for (int ph = 0; ph < 2; ++ph) {
        const long long K = (long long)T[ph] * B, nc = (K + kKC - 1) / kKC;
        for (int l = 0; l < 2; ++l) {
            const long long mc = l ? D : m;
            np += nc * (3 * D * D + D * D + 4 * D * mc + 4 * D);
        }
    }
    np += ((long long)(T[0] + T[1]) * B + kKC - 1) / kKC * (long long)(m * D);
    L.nwpart = np;
    L.wpart = o; o += al((size_t)np * sizeof(float));
    L.total = o;
    return L;
}

struct LemArgs {
    int B, m, t_in, t_out;
    float dt;
    const float *theta, *u;
    unsigned char *w;   // work space base
    Layout L;
};

template <typename T>
__device__ __forceinline__ T *wp(const LemArgs &A, size_t off)
{
    return reinterpret_cast<T *>(A.w + off);
}

}  // namespace

namespace {

// Row stride of the per-sequence state rows in shared memory: D + 8, so
// that the element-wise updates of 4 sequences x 8 units in a warp fall in
// distinct banks; a multiple of 4 floats, for the float4 reads.
template <int D>
__host__ __device__ constexpr int row_stride()
{
    return D + 8;
}

// Shared-memory floats of the recurrent kernels for width D
template <int D, int R>
constexpr int fwd_smem_floats()
{
    return 3 * 4 * D * D + 4 * kMMax * D + 2 * 4 * D + kMMax * D + 2 * 2 * (kG * R) * row_stride<D>() +
           (kG * R) * kMMax;
}
template <int D, int R>
constexpr int bwd_smem_floats()
{
    return 3 * 4 * D * D + 4 * kMMax * D + kMMax * D + 2 * 4 * (kG * R) * row_stride<D>() + (kG * R) * kMMax;
}

// Position of entry (o, k) of a D x D product matrix (output o, summed
// index k) in shared memory: k in blocks of 16, each block a [D][16] slab, so
// that lane (o, r) reads the float4 of k = 16 t + 4 r .. + 3 and the 32 lanes
// of a warp (8 outputs x 4 quarters) read 512 contiguous bytes.
template <int D>
__device__ __forceinline__ int qx(int o, int k)
{
    return ((k >> 4) * D + o) * 16 + (k & 15);
}

// Weights of cell c into shared memory.  W (and V of a width-D input) in
// the product layout qx: REV false for the forward products (output = row
// i, summed index = column j), true for the reverse products W^T g (output =
// column, summed index = row).  The m-wide input weights of a first cell:
// [q][c][i] forward, as stored ([q][i][c]) reverse.
template <int D, bool REV>
__device__ void load_cell(const float *theta, int c, int m, float *W, float *V, float *bb)
{
    const int mc = (c & 1) ? D : m;
    const float *src = theta + cell_offset(c, D, m);
    for (int e = threadIdx.x; e < 4 * D * D; e += blockDim.x) {
        const int q = e / (D * D), rc = e % (D * D), row = rc / D, col = rc % D;
        W[q * D * D + (REV ? qx<D>(col, row) : qx<D>(row, col))] = src[e];
    }
    src += 4 * D * D;
    for (int e = threadIdx.x; e < 4 * D * mc; e += blockDim.x) {
        const int q = e / (D * mc), rc = e % (D * mc), row = rc / mc, col = rc % mc;
        if (mc == D) V[q * D * D + (REV ? qx<D>(col, row) : qx<D>(row, col))] = src[e];
        else V[REV ? e : (q * mc + col) * D + row] = src[e];
    }
    src += 4 * D * mc;
    if (bb)
        for (int e = threadIdx.x; e < 4 * D; e += blockDim.x) bb[e] = src[e];
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float dot4(float4 w, float4 v, float a)
{
    return fmaf(w.w, v.w, fmaf(w.z, v.z, fmaf(w.y, v.y, fmaf(w.x, v.x, a))));
}

// Reduce-scatter over the 4 lanes (o, 0..3) of one output: lane r holds
// the quarter-r partials a0..a3 of sequences 0..3 of a group and gets the
// whole sum of sequence r.  Every sequence's sum is (q0 + q2) + (q1 + q3)
// of its quarter partials, whichever lane finishes it.
__device__ __forceinline__ float rs4(float a0, float a1, float a2, float a3, int r)
{
    const bool hi = r & 2, lo = r & 1;
    float k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
    k0 += __shfl_xor_sync(0xffffffffu, hi ? a0 : a2, 2);
    k1 += __shfl_xor_sync(0xffffffffu, hi ? a1 : a3, 2);
    return (lo ? k1 : k0) + __shfl_xor_sync(0xffffffffu, lo ? k0 : k1, 1);
}

// Sum over the 32 lanes of a warp (the same bits in every lane)
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Forward pass of kG R sequences (see the file comment).  Thread (i, r) =
// (tid / 4, tid % 4): in the products, output unit i over the summed
// indices of quarter r for every sequence of the CTA; in the element-wise
// updates, unit i of sequences r + 4 rr, rr < R.
template <int D, int R>
__global__ void __launch_bounds__(kG *D, 1) lem_fwd_kernel(LemArgs A)
{
    constexpr int kBT = kG * R, kT = D / 16, kNW = D / 8, kHO = (kBT * kMMax + kNW - 1) / kNW;
    constexpr int SD = row_stride<D>();
    extern __shared__ __align__(16) float sm[];
    float *W0 = sm, *W1 = W0 + 4 * D * D, *V1 = W1 + 4 * D * D, *V0 = V1 + 4 * D * D;
    float *bb0 = V0 + 4 * kMMax * D, *bb1 = bb0 + 4 * D, *Wo = bb1 + 4 * D;
    float *Y = Wo + kMMax * D, *Z = Y + 2 * kBT * SD, *X = Z + 2 * kBT * SD;
    const int tid = threadIdx.x, i = tid >> 2, r = tid & 3, lane = tid & 31, warp = tid >> 5;
    const int m = A.m, B = A.B, b0 = blockIdx.x * kBT;
    const float dt = A.dt;
    for (int e = tid; e < m * D; e += blockDim.x) Wo[e] = A.theta[cell_offset(4, D, m) + e];
    for (int e = tid; e < 2 * kBT * SD; e += blockDim.x) Y[e] = Z[e] = 0.f;
    for (int ph = 0; ph < 2; ++ph) {
        const int T = ph ? A.t_out : A.t_in;
        float *act[2] = {wp<float>(A, A.L.act[ph][0]), wp<float>(A, A.L.act[ph][1])};
        float *res = wp<float>(A, ph ? A.L.out : A.L.recon);
        float *xdec = wp<float>(A, A.L.xdec);
        __syncthreads();   // the previous phase is done with the weights
        load_cell<D, false>(A.theta, 2 * ph, m, W0, V0, bb0);
        load_cell<D, false>(A.theta, 2 * ph + 1, m, W1, V1, bb1);
        // the first input: u_0 (encoder) or 0 (decoder)
        for (int t = tid; t < kBT * m; t += blockDim.x) {
            const int s = t / m, c = t % m, b = b0 + s;
            const float v = (ph == 0 && b < B) ? A.u[(long long)b * m + c] : 0.f;
            X[s * kMMax + c] = v;
            if (ph == 1 && b < B) xdec[(long long)b * m + c] = 0.f;
        }
        // slot 0 of the saved activations: the initial states
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const int s = r + kG * rr, b = b0 + s;
                if (b < B) {
                    float *a = act[l] + (long long)b * kQ * D + i;
                    a[0] = Y[(l * kBT + s) * SD + i];
                    a[D] = Z[(l * kBT + s) * SD + i];
                }
            }
        __syncthreads();
        for (int n = 0; n < T; ++n) {
            // the encoder's next input, fetched now for the head at the end of the step
            float un[kHO];
#pragma unroll
            for (int h = 0; h < kHO; ++h) {
                const int o = warp + h * kNW, s = o / m, c = o % m, b = b0 + s;
                un[h] = (ph == 0 && n + 1 < T && lane == 0 && o < kBT * m && b < B)
                            ? A.u[((long long)(n + 1) * B + b) * m + c]
                            : 0.f;
            }
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const float *W = l ? W1 : W0, *bb = l ? bb1 : bb0;
                const float *yv = Y + l * kBT * SD, *xv = Y;   // cell 1's input is cell 0's y_n
                constexpr int kNQ = 4;
                float acc[kNQ][kBT];
#pragma unroll
                for (int q = 0; q < kNQ; ++q)
#pragma unroll
                    for (int s = 0; s < kBT; ++s) acc[q][s] = 0.f;
                // gates: W y_{n-1} (+ V x_n for cell 1), quarter r of the summed index
#pragma unroll
                for (int t = 0; t < kT; ++t) {
                    const int wo = (t * D + i) * 16 + 4 * r, vo = 16 * t + 4 * r;
                    float4 w[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) w[q] = ld4(W + q * D * D + wo);
#pragma unroll
                    for (int s = 0; s < kBT; ++s) {
                        const float4 y4 = ld4(yv + s * SD + vo);
#pragma unroll
                        for (int q = 0; q < 3; ++q) acc[q][s] = dot4(w[q], y4, acc[q][s]);
                    }
                    if (l) {
                        float4 v[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = ld4(V1 + q * D * D + wo);
#pragma unroll
                        for (int s = 0; s < kBT; ++s) {
                            const float4 x4 = ld4(xv + s * SD + vo);
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[q][s] = dot4(v[q], x4, acc[q][s]);
                        }
                    }
                }
                float s1[R], s2[R], ay[R], yp[R], zn[R], tz[R];
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    float g[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        g[q] = (q < 3 || l) ? rs4(acc[q][4 * rr], acc[q][4 * rr + 1], acc[q][4 * rr + 2],
                                                  acc[q][4 * rr + 3], r)
                                            : 0.f;
                    const int s = r + kG * rr;
                    float a1 = bb[i], a2 = bb[D + i], az = bb[2 * D + i], a4 = bb[3 * D + i];
                    if (!l) {
                        const float *x = X + s * kMMax;
                        for (int c = 0; c < m; ++c) {
                            const float xc = x[c];
                            a1 = fmaf(V0[(0 * m + c) * D + i], xc, a1);
                            a2 = fmaf(V0[(1 * m + c) * D + i], xc, a2);
                            az = fmaf(V0[(2 * m + c) * D + i], xc, az);
                            a4 = fmaf(V0[(3 * m + c) * D + i], xc, a4);
                        }
                    }
                    a1 += g[0];
                    a2 += g[1];
                    az += g[2];
                    ay[rr] = a4 + g[3];
                    yp[rr] = yv[s * SD + i];
                    const float zp = Z[(l * kBT + s) * SD + i];
                    s1[rr] = sigm(a1);
                    s2[rr] = sigm(a2);
                    tz[rr] = tanhf(az);
                    const float h1 = dt * s1[rr];
                    zn[rr] = fmaf(h1, tz[rr], (1.f - h1) * zp);
                    // z_n of unit i: read by no other thread before the barrier
                    Z[(l * kBT + s) * SD + i] = zn[rr];
                }
                __syncthreads();
                // y gate: a4 += W_4 z_n
                float a4p[kBT];
#pragma unroll
                for (int s = 0; s < kBT; ++s) a4p[s] = 0.f;
                const float *zv = Z + l * kBT * SD;
#pragma unroll
                for (int t = 0; t < kT; ++t) {
                    const float4 w = ld4(W + 3 * D * D + (t * D + i) * 16 + 4 * r);
#pragma unroll
                    for (int s = 0; s < kBT; ++s) a4p[s] = dot4(w, ld4(zv + s * SD + 16 * t + 4 * r), a4p[s]);
                }
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const float a4 = ay[rr] + rs4(a4p[4 * rr], a4p[4 * rr + 1], a4p[4 * rr + 2], a4p[4 * rr + 3], r);
                    const int s = r + kG * rr, b = b0 + s;
                    const float ty = tanhf(a4), h2 = dt * s2[rr];
                    const float yn = fmaf(h2, ty, (1.f - h2) * yp[rr]);
                    Y[(l * kBT + s) * SD + i] = yn;
                    if (b < B) {
                        float *a = act[l] + ((long long)(n + 1) * B + b) * kQ * D + i;
                        a[0] = yn;
                        a[D] = zn[rr];
                        a[2 * D] = s1[rr];
                        a[3 * D] = s2[rr];
                        a[4 * D] = tz[rr];
                        a[5 * D] = ty;
                    }
                }
                __syncthreads();
            }
            // the head: o = Wo y of the top cell, one warp per output; the next input
#pragma unroll
            for (int h = 0; h < kHO; ++h) {
                const int o = warp + h * kNW;
                if (o < kBT * m) {
                    const int s = o / m, c = o % m, b = b0 + s;
                    const float *yv = Y + (kBT + s) * SD;
                    float p = 0.f;
#pragma unroll
                    for (int k = lane; k < D; k += 32) p = fmaf(Wo[c * D + k], yv[k], p);
                    p = warp_sum(p);
                    if (lane == 0) {
                        if (b < B) res[((long long)n * B + b) * m + c] = p;
                        if (n + 1 < T) {
                            const float x = ph == 0 ? un[h] : p;
                            if (ph == 1 && b < B) xdec[((long long)(n + 1) * B + b) * m + c] = p;
                            X[s * kMMax + c] = x;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

namespace {

// ------------------------------------------------------------------ losses
// A value with its derivatives along two directions (p and q): forward-mode
// differentiation of the trapezoidal LLG map for the physics-loss gradient.
struct Dual {
    float v, a, b;
};
__device__ __forceinline__ Dual dmk(float v) { return {v, 0.f, 0.f}; }
__device__ __forceinline__ Dual operator+(Dual x, Dual y) { return {x.v + y.v, x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ Dual operator-(Dual x, Dual y) { return {x.v - y.v, x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ Dual operator-(Dual x) { return {-x.v, -x.a, -x.b}; }
__device__ __forceinline__ Dual operator*(Dual x, Dual y) { return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b}; }
__device__ __forceinline__ Dual operator*(float s, Dual x) { return {s * x.v, s * x.a, s * x.b}; }
__device__ __forceinline__ Dual operator/(Dual x, Dual y)
{
    const float r = 1.f / y.v, q = x.v * r;
    return {q, (x.a - q * y.a) * r, (x.b - q * y.b) * r};
}
__device__ __forceinline__ Dual dsqrt(Dual x)
{
    const float s = sqrtf(x.v), h = 0.5f / s;
    return {s, x.a * h, x.b * h};
}
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ float mkv(float v, float) { return v; }
__device__ __forceinline__ Dual mkv(float v, Dual) { return dmk(v); }

// One trapezoidal LLG step of m = (p, q, 1) (Eqs. llg_tra4-6): a = -(kappa
// H^{k+1} + alpha m), b = m - kappa m x H^k, M~ = (b + (a.b) a - a x b) /
// (1 + |a|^2), normalised to |m|; returns its two transverse components.
template <typename T>
__device__ void llg_map(T p, T q, const float *hk, const float *hk1, float kappa, float alpha, float h0, T &Fp, T &Fq)
{
    const T one = mkv(1.f, p);
    const float H0x = hk[0], H0y = hk[1], H0z = hk[2] + h0;
    const float H1x = hk1[0], H1y = hk1[1], H1z = hk1[2] + h0;
    // m x H^k
    const T cx = q * mkv(H0z, p) - one * mkv(H0y, p);
    const T cy = one * mkv(H0x, p) - p * mkv(H0z, p);
    const T cz = p * mkv(H0y, p) - q * mkv(H0x, p);
    const T bx = p - kappa * cx, by = q - kappa * cy, bz = one - kappa * cz;
    const T ax = -(mkv(kappa * H1x, p) + alpha * p), ay = -(mkv(kappa * H1y, p) + alpha * q),
            az = -(mkv(kappa * H1z, p) + alpha * one);
    const T ab = ax * bx + ay * by + az * bz;
    const T den = one + ax * ax + ay * ay + az * az;
    // a x b
    const T xx = ay * bz - az * by, xy = az * bx - ax * bz, xz = ax * by - ay * bx;
    const T mx = (bx + ab * ax - xx) / den, my = (by + ab * ay - xy) / den, mz = (bz + ab * az - xz) / den;
    const T s = dsqrt(p * p + q * q + one) / dsqrt(mx * mx + my * my + mz * mz);
    Fp = mx * s;
    Fq = my * s;
}

__device__ double block_sum_d(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh[q];   // the same order in every thread
    return t;
}

struct LossArgs {
    int B, m, t_in, t_out;
    float lam, kappa, alpha, h0;
    const float *u, *target, *h, *recon, *out;
    float *drec, *dout;
    double *lpart;
};

// One thread per reconstructed value, then one per (predicted step,
// sequence).  Per-block sums of the three losses go to lpart in block order.
__global__ void __launch_bounds__(kLossThreads) lem_loss_kernel(LossArgs A)
{
    __shared__ double sh[kLossThreads / 32];
    const long long NR = (long long)A.t_in * A.B * A.m, NP = (long long)A.t_out * A.B;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double lr = 0.0, lp = 0.0, lf = 0.0;
    if (t < NR) {
        const float e = A.recon[t] - A.u[t];
        lr = (double)e * e;
        A.drec[t] = 2.f * e / (float)NR;
    } else if (t < NR + NP) {
        const long long q = t - NR;
        const int k = (int)(q / A.B), m = A.m;
        const long long o = q * m;
        float dv[kMMax];
        for (int c = 0; c < m; ++c) {
            const float e = A.out[o + c] - A.target[o + c];
            lp += (double)e * e;
            dv[c] = 2.f * e / (float)(NP * m);
        }
        if (m == 2 && A.t_out > 1 && A.h) {
            const float cf = A.lam / (float)((long long)(A.t_out - 1) * A.B);
            const float *hk = A.h + q * 3;
            if (k + 1 < A.t_out) {   // pair (k, k+1): residual and its derivative in o_k
                Dual Fp, Fq;
                llg_map(Dual{A.out[o], 1.f, 0.f}, Dual{A.out[o + 1], 0.f, 1.f}, hk, hk + (long long)A.B * 3, A.kappa,
                        A.alpha, A.h0, Fp, Fq);
                const float rp = Fp.v - A.out[o + (long long)A.B * m], rq = Fq.v - A.out[o + (long long)A.B * m + 1];
                lf = ((double)rp * rp + (double)rq * rq) / (2.0 * (double)(A.t_out - 1) * A.B);
                dv[0] += cf * (Fp.a * rp + Fq.a * rq);
                dv[1] += cf * (Fp.b * rp + Fq.b * rq);
            }
            if (k >= 1) {   // pair (k-1, k): the residual's direct term in o_k
                const long long op = o - (long long)A.B * m;
                float Fp, Fq;
                llg_map(A.out[op], A.out[op + 1], hk - (long long)A.B * 3, hk, A.kappa, A.alpha, A.h0, Fp, Fq);
                dv[0] -= cf * (Fp - A.out[o]);
                dv[1] -= cf * (Fq - A.out[o + 1]);
            }
        }
        for (int c = 0; c < m; ++c) A.dout[o + c] = dv[c];
    }
    lr = block_sum_d(lr, sh);
    lp = block_sum_d(lp, sh);
    lf = block_sum_d(lf, sh);
    if (threadIdx.x == 0) {
        A.lpart[3 * blockIdx.x] = lr;
        A.lpart[3 * blockIdx.x + 1] = lp;
        A.lpart[3 * blockIdx.x + 2] = lf;
    }
}

// The four losses from the block partials, summed in block order.
__global__ void lem_loss_final_kernel(const double *lpart, int nblk, long long NR, long long NPM, double lam,
                                      double *loss)
{
    __shared__ double sh[kLossThreads / 32];
    double s[3];
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int q = threadIdx.x; q < nblk; q += blockDim.x) v += lpart[3 * q + c];
        s[c] = block_sum_d(v, sh);
    }
    if (threadIdx.x == 0) {
        const double r = s[0] / (double)NR, p = s[1] / (double)NPM;
        loss[0] = r + p + lam * s[2];
        loss[1] = r;
        loss[2] = p;
        loss[3] = s[2];
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------- reverse
// The saved values of one unit, sequence and step that the reverse step
// reads: y_{n-1}, z_{n-1} (slot n) and the gates and tanh values of step n
// (slot n + 1).
struct Saved {
    float yp, zp, s1, s2, tz, ty;
};
template <int D>
__device__ __forceinline__ Saved fetch_saved(const float *act, int B, int n, int b, int i)
{
    const float *a0 = act + ((long long)n * B + b) * kQ * D + i;
    const float *a1 = act + ((long long)(n + 1) * B + b) * kQ * D + i;
    return {a0[0], a0[D], a1[2 * D], a1[3 * D], a1[4 * D], a1[5 * D]};
}

// Back-propagation through both stacks for kG R sequences: the decoder's steps
// in reverse (with the output feedback: the gradient of step k+1's input is
// added to the gradient of output k), then the encoder's.  Thread (i, r) =
// (tid / 4, tid % 4) carries dL/dy and dL/dz of unit i of sequences r + 4 rr
// for both cells in registers and, in the products W^T g, sums quarter r of
// the summed index for every sequence of the CTA.  The gate gradients of
// each step go to shared memory for those products and to the work space
// for the weight sums; the saved activations are fetched one step ahead.
template <int D, int R>
__global__ void __launch_bounds__(kG *D, 1) lem_bwd_kernel(LemArgs A)
{
    constexpr int kBT = kG * R, kT = D / 16, kNW = D / 8, kHO = (kBT * kMMax + kNW - 1) / kNW;
    constexpr int SD = row_stride<D>();
    extern __shared__ __align__(16) float sm[];
    float *W0 = sm, *W1 = W0 + 4 * D * D, *V1 = W1 + 4 * D * D, *V0 = V1 + 4 * D * D;
    float *Wo = V0 + 4 * kMMax * D, *DG = Wo + kMMax * D;   // DG [2][4][kBT][SD]
    float *DO = DG + 2 * 4 * kBT * SD;
    const int tid = threadIdx.x, i = tid >> 2, r = tid & 3, lane = tid & 31, warp = tid >> 5;
    const int m = A.m, B = A.B, b0 = blockIdx.x * kBT;
    const float dt = A.dt;
    for (int e = tid; e < m * D; e += blockDim.x) Wo[e] = A.theta[cell_offset(4, D, m) + e];
    float dy[2][R], dz[2][R];
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) dy[l][rr] = dz[l][rr] = 0.f;
    for (int ph = 1; ph >= 0; --ph) {
        const int T = ph ? A.t_out : A.t_in;
        const float *act[2] = {wp<float>(A, A.L.act[ph][0]), wp<float>(A, A.L.act[ph][1])};
        float *dgo[2] = {wp<float>(A, A.L.dg[ph][0]), wp<float>(A, A.L.dg[ph][1])};
        const float *dsrc = wp<float>(A, ph ? A.L.dout : A.L.drec);
        float *dot = wp<float>(A, A.L.dot);
        __syncthreads();   // the previous phase is done with the weights
        load_cell<D, true>(A.theta, 2 * ph, m, W0, V0, nullptr);
        load_cell<D, true>(A.theta, 2 * ph + 1, m, W1, V1, nullptr);
        // step T-1's saved values and loss gradients
        Saved sv[2][R];
        float dl[kHO];
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int rr = 0; rr < R; ++rr) sv[l][rr] = fetch_saved<D>(act[l], B, T - 1, min(b0 + r + kG * rr, B - 1), i);
#pragma unroll
        for (int h = 0; h < kHO; ++h) {
            const int o = warp + h * kNW, b = b0 + o / m;
            dl[h] = (lane == 0 && o < kBT * m && b < B) ? dsrc[((long long)(T - 1) * B + b) * m + o % m] : 0.f;
        }
        __syncthreads();
        for (int n = T - 1; n >= 0; --n) {
            // gradient at the head's output: the loss's, plus (decoder) the
            // feedback from step n+1's input through cell 0's input weights
            // (cell 0's gate gradients of step n+1 are still in DG)
#pragma unroll
            for (int h = 0; h < kHO; ++h) {
                const int o = warp + h * kNW;
                if (o < kBT * m) {
                    const int s = o / m, c = o % m, b = b0 + s;
                    float fb = 0.f;
                    if (ph && n + 1 < T) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int k = lane; k < D; k += 32)
                                fb = fmaf(V0[(q * D + k) * m + c], DG[(q * kBT + s) * SD + k], fb);
                        fb = warp_sum(fb);
                    }
                    if (lane == 0) {
                        float v = 0.f;
                        if (b < B) {
                            v = dl[h];
                            if (ph) {
                                v += fb;
                                dot[((long long)n * B + b) * m + c] = v;
                            }
                        }
                        DO[s * kMMax + c] = v;
                    }
                    // the next step's loss gradient
                    dl[h] = (lane == 0 && n > 0 && b < B) ? dsrc[((long long)(n - 1) * B + b) * m + c] : 0.f;
                }
            }
            // the next step's saved values
            Saved nx[2][R];
#pragma unroll
            for (int l = 0; l < 2; ++l)
#pragma unroll
                for (int rr = 0; rr < R; ++rr)
                    nx[l][rr] = fetch_saved<D>(act[l], B, n > 0 ? n - 1 : 0, min(b0 + r + kG * rr, B - 1), i);
            __syncthreads();
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const int s = r + kG * rr;
                float a = dy[1][rr];
                for (int c = 0; c < m; ++c) a = fmaf(Wo[c * D + i], DO[s * kMMax + c], a);
                dy[1][rr] = a;
            }
#pragma unroll
            for (int l = 1; l >= 0; --l) {
                const float *W = l ? W1 : W0;
                float *dgl = DG + l * 4 * kBT * SD;
                float dg2[R], dgy[R], dyp[R];
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const Saved &v = sv[l][rr];
                    const float gy = dy[l][rr];
                    dg2[rr] = gy * (v.ty - v.yp) * dt * v.s2 * (1.f - v.s2);
                    dgy[rr] = gy * dt * v.s2 * (1.f - v.ty * v.ty);
                    dgl[(3 * kBT + r + kG * rr) * SD + i] = dgy[rr];
                    dyp[rr] = gy * (1.f - dt * v.s2);
                }
                __syncthreads();
                // dz: W_4^T of the y gate's gradient
                float az[kBT];
#pragma unroll
                for (int s = 0; s < kBT; ++s) az[s] = 0.f;
#pragma unroll
                for (int t = 0; t < kT; ++t) {
                    const float4 w = ld4(W + 3 * D * D + (t * D + i) * 16 + 4 * r);
#pragma unroll
                    for (int s = 0; s < kBT; ++s) az[s] = dot4(w, ld4(dgl + (3 * kBT + s) * SD + 16 * t + 4 * r), az[s]);
                }
                float dzp[R];
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const Saved &v = sv[l][rr];
                    const int s = r + kG * rr, b = b0 + s;
                    const float dzt = dz[l][rr] + rs4(az[4 * rr], az[4 * rr + 1], az[4 * rr + 2], az[4 * rr + 3], r);
                    const float dg1 = dzt * (v.tz - v.zp) * dt * v.s1 * (1.f - v.s1);
                    const float dgz = dzt * dt * v.s1 * (1.f - v.tz * v.tz);
                    dzp[rr] = dzt * (1.f - dt * v.s1);
                    dgl[(0 * kBT + s) * SD + i] = dg1;
                    dgl[(1 * kBT + s) * SD + i] = dg2[rr];
                    dgl[(2 * kBT + s) * SD + i] = dgz;
                    if (b < B) {
                        float *o = dgo[l] + ((long long)n * B + b) * 4 * D + i;
                        o[0] = dg1;
                        o[D] = dg2[rr];
                        o[2 * D] = dgz;
                        o[3 * D] = dgy[rr];
                    }
                }
                __syncthreads();
                // dy_{n-1}: W^T of the other three gates; cell 1 also gives
                // cell 0's dy_n through V^T of all four
                float ay[kBT], ax[kBT];
#pragma unroll
                for (int s = 0; s < kBT; ++s) ay[s] = ax[s] = 0.f;
#pragma unroll
                for (int t = 0; t < kT; ++t) {
                    const int wo = (t * D + i) * 16 + 4 * r, go = 16 * t + 4 * r;
                    float4 w[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) w[q] = ld4(W + q * D * D + wo);
                    float4 v[4];
                    if (l) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = ld4(V1 + q * D * D + wo);
                    }
#pragma unroll
                    for (int s = 0; s < kBT; ++s) {
                        float4 g[4];
#pragma unroll
                        for (int q = 0; q < (l ? 4 : 3); ++q) g[q] = ld4(dgl + (q * kBT + s) * SD + go);
#pragma unroll
                        for (int q = 0; q < 3; ++q) ay[s] = dot4(w[q], g[q], ay[s]);
                        if (l) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) ax[s] = dot4(v[q], g[q], ax[s]);
                        }
                    }
                }
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    dy[l][rr] = dyp[rr] + rs4(ay[4 * rr], ay[4 * rr + 1], ay[4 * rr + 2], ay[4 * rr + 3], r);
                    dz[l][rr] = dzp[rr];
                    if (l) dy[0][rr] += rs4(ax[4 * rr], ax[4 * rr + 1], ax[4 * rr + 2], ax[4 * rr + 3], r);
                }
            }
#pragma unroll
            for (int l = 0; l < 2; ++l)
#pragma unroll
                for (int rr = 0; rr < R; ++rr) sv[l][rr] = nx[l][rr];
        }
    }
}

}  // namespace

namespace {

// --------------------------------------------------------- weight sums
// Asynchronous global -> shared copies (completion by groups)
__device__ __forceinline__ void cpa4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kWRows = 32;                  // rows per staged tile
constexpr int kWA = 4 * 64 + 4, kWB = 64 + 4;   // row strides of the staged A and B tiles
constexpr int kWgradSmem = 2 * kWRows * (kWA + kWB) * (int)sizeof(float);

// Partial sums over one chunk of kKC rows of one product: C[r][j] =
// sum_k A[k][aoff + r] B[k][boff + j] (B absent: 1), rows k >= K1 from the
// second segment.  Tiles of 32 rows are staged by asynchronous copies, two
// buffers deep (the next tile lands while this one is summed).  Thread (rt,
// jt) of group q accumulates an 8 x 8 block over the staged rows kk = q (mod
// G), G = 256 / (threads per block of outputs); the groups' blocks are then
// added in group order.
__global__ void __launch_bounds__(256) lem_wgrad_kernel(WProdSet S, float *part)
{
    extern __shared__ __align__(16) float wsm[];
    int p = 0;
    while (p + 1 < S.np && (int)blockIdx.x >= S.p[p + 1].chunk0) ++p;
    const WProd &P = S.p[p];
    const int chunk = blockIdx.x - P.chunk0, tid = threadIdx.x;
    const long long k0 = (long long)chunk * kKC, k1 = min(k0 + kKC, P.K);
    const int RT = (P.R + 7) / 8, JT = (P.J + 7) / 8, NB = RT * JT, G = 256 / NB;
    const int q = tid / NB, rt = (tid % NB) % RT, jt = (tid % NB) / RT;
    const bool act = q < G;
    // 16-byte copies where rows, offsets and widths allow them
    const bool va = (P.lda % 4 == 0) && (P.aoff % 4 == 0) && (P.R % 4 == 0);
    const bool vb = P.B && (P.ldb % 4 == 0) && (P.boff % 4 == 0) && (P.J % 4 == 0);
    auto sa = [&](int buf, int kk) { return wsm + (buf * kWRows + kk) * kWA; };
    auto sb = [&](int buf, int kk) { return wsm + 2 * kWRows * kWA + (buf * kWRows + kk) * kWB; };
    auto stage = [&](int buf, long long kb) {
        const int nk = (int)min((long long)kWRows, k1 - kb);
        if (va) {
            const int w = P.R / 4;
            for (int e = tid; e < nk * w; e += blockDim.x) {
                const int kk = e / w, r = (e % w) * 4;
                const long long row = kb + kk;
                const float *src = row < P.K1 ? P.A + row * P.lda : P.A2 + (row - P.K1) * P.lda;
                cpa16(sa(buf, kk) + r, src + P.aoff + r);
            }
        } else {
            for (int e = tid; e < nk * P.R; e += blockDim.x) {
                const int kk = e / P.R, r = e % P.R;
                const long long row = kb + kk;
                const float *src = row < P.K1 ? P.A + row * P.lda : P.A2 + (row - P.K1) * P.lda;
                cpa4(sa(buf, kk) + r, src + P.aoff + r);
            }
        }
        if (!P.B) {
            for (int e = tid; e < nk * P.J; e += blockDim.x) sb(buf, e / P.J)[e % P.J] = 1.f;
        } else if (vb) {
            const int w = P.J / 4;
            for (int e = tid; e < nk * w; e += blockDim.x) {
                const int kk = e / w, j = (e % w) * 4;
                const long long row = kb + kk;
                const float *src = row < P.K1 ? P.B + row * P.ldb : P.B2 + (row - P.K1) * P.ldb;
                cpa16(sb(buf, kk) + j, src + P.boff + j);
            }
        } else {
            for (int e = tid; e < nk * P.J; e += blockDim.x) {
                const int kk = e / P.J, j = e % P.J;
                const long long row = kb + kk;
                const float *src = row < P.K1 ? P.B + row * P.ldb : P.B2 + (row - P.K1) * P.ldb;
                cpa4(sb(buf, kk) + j, src + P.boff + j);
            }
        }
        cpa_commit();
    };
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    stage(0, k0);
    int buf = 0;
    for (long long kb = k0; kb < k1; kb += kWRows, buf ^= 1) {
        const int nk = (int)min((long long)kWRows, k1 - kb);
        if (kb + kWRows < k1) {
            stage(buf ^ 1, kb + kWRows);
            cpa_wait<1>();
        } else {
            cpa_wait<0>();
        }
        __syncthreads();
        if (act)
            for (int kk = q; kk < nk; kk += G) {
                const float *ra = sa(buf, kk) + rt * 8, *rb = sb(buf, kk) + jt * 8;
                const float4 a0 = *reinterpret_cast<const float4 *>(ra), a1 = *reinterpret_cast<const float4 *>(ra + 4);
                const float4 b0 = *reinterpret_cast<const float4 *>(rb), b1 = *reinterpret_cast<const float4 *>(rb + 4);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
            }
        __syncthreads();   // this buffer is free for the tile after next
    }
    // groups 1 .. G-1 add their blocks into group 0's, one group at a time
    // (the A buffers as the exchange area: R x J <= 8192 floats whenever G > 1)
    float *xb = wsm;
    for (int g = 1; g < G; ++g) {
        if (q == g)
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int r = rt * 8 + a, j = jt * 8 + b;
                    if (r < P.R && j < P.J) xb[r * P.J + j] = acc[a][b];
                }
        __syncthreads();
        if (q == 0)
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int r = rt * 8 + a, j = jt * 8 + b;
                    if (r < P.R && j < P.J) acc[a][b] += xb[r * P.J + j];
                }
        __syncthreads();
    }
    if (q != 0) return;
    float *o = part + P.poff + (long long)chunk * P.R * P.J;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int r = rt * 8 + a, j = jt * 8 + b;
            if (r < P.R && j < P.J) o[(long long)r * P.J + j] = acc[a][b];
        }
}

// Every output of every product: the sum of its chunk partials in chunk
// order, into the gradient vector.
__global__ void lem_wreduce_kernel(WProdSet S, const float *part, float *grad)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < S.np; ++p) {
        const WProd &P = S.p[p];
        const long long n = (long long)P.R * P.J;
        if (e < n) {
            float s = 0.f;
            for (int c = 0; c < P.nchunk; ++c) s += part[P.poff + c * n + e];
            grad[P.goff + e] = s;
            return;
        }
        e -= n;
    }
}

__global__ void lem_adam_kernel(long long n, float *th, const float *g, float *mo, float *ve, float lr, float b1,
                                float b2, float eps, float c1, float c2)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = fmaf(b1, mo[q], (1.f - b1) * gq);
    const float vq = fmaf(b2, ve[q], (1.f - b2) * gq * gq);
    mo[q] = mq;
    ve[q] = vq;
    th[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

int fail(int code, const char *msg)
{
    fl::set_last_error(msg);
    return code;
}
int cuda_fail(cudaError_t e, const char *where)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    fl::set_last_error(buf);
    return FDTD_E_CUDA;
}

LemArgs args(const fdtd_llg_lem_shape *s, const float *theta, const float *u, void *work)
{
    LemArgs A{};
    A.B = s->batch;
    A.m = s->m;
    A.t_in = s->t_in;
    A.t_out = s->t_out;
    A.dt = s->dt;
    A.theta = theta;
    A.u = u;
    A.w = static_cast<unsigned char *>(work);
    A.L = layout(s);
    return A;
}

WProdSet products(const fdtd_llg_lem_shape *s, const LemArgs &A)
{
    WProdSet S{};
    const int D = s->d, m = s->m, B = s->batch;
    const long long rowq = (long long)kQ * D;
    auto f = [&](size_t off) { return reinterpret_cast<const float *>(A.w + off); };
    long long poff = 0;
    int chunk0 = 0;
    auto add = [&](WProd P) {
        P.nchunk = (int)((P.K + kKC - 1) / kKC);
        P.chunk0 = chunk0;
        P.poff = poff;
        chunk0 += P.nchunk;
        poff += (long long)P.nchunk * P.R * P.J;
        S.p[S.np++] = P;
    };
    for (int ph = 0; ph < 2; ++ph)
        for (int l = 0; l < 2; ++l) {
            const int c = 2 * ph + l, mc = cell_width(c, m, D);
            const long long base = cell_offset(c, D, m), K = (long long)(ph ? s->t_out : s->t_in) * B;
            const float *dg = f(A.L.dg[ph][l]), *act = f(A.L.act[ph][l]);
            WProd P{};
            P.A = P.A2 = dg;
            P.lda = 4LL * D;
            P.K1 = P.K = K;
            // W1, W2, Wz against y_{n-1} (slot n)
            P.aoff = 0; P.R = 3 * D; P.B = P.B2 = act; P.ldb = rowq; P.boff = 0; P.J = D; P.goff = base;
            add(P);
            // Wy against z_n (slot n+1)
            P.aoff = 3 * D; P.R = D; P.B = P.B2 = act + (long long)B * rowq; P.boff = D; P.goff = base + 3LL * D * D;
            add(P);
            // V against the cell input
            P.aoff = 0; P.R = 4 * D; P.boff = 0; P.goff = base + 4LL * D * D;
            if (l) { P.B = P.B2 = f(A.L.act[ph][0]) + (long long)B * rowq; P.ldb = rowq; P.J = D; }
            else { P.B = P.B2 = ph ? f(A.L.xdec) : A.u; P.ldb = m; P.J = m; }
            add(P);
            // biases
            P.B = P.B2 = nullptr; P.ldb = 0; P.J = 1; P.goff = base + 4LL * D * D + 4LL * D * mc;
            add(P);
        }
    WProd H{};
    H.A = f(A.L.drec); H.A2 = f(A.L.dot); H.lda = m; H.aoff = 0; H.R = m;
    H.B = f(A.L.act[0][1]) + (long long)B * rowq; H.B2 = f(A.L.act[1][1]) + (long long)B * rowq;
    H.ldb = rowq; H.boff = 0; H.J = D;
    H.K1 = (long long)s->t_in * B; H.K = (long long)(s->t_in + s->t_out) * B;
    H.goff = cell_offset(4, D, m);
    add(H);
    S.nchunks = chunk0;
    return S;
}

// Sequences per thread: 2 once the batch fills every SM with two-per-thread
// CTAs (each weight load then feeds two sequences), else 1 (more CTAs).
int seq_per_thread(int B)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 148;
    }
    return (B + 2 * kG - 1) / (2 * kG) >= nsm ? 2 : 1;
}
template <int D, int R>
cudaError_t launch_fwd_r(const LemArgs &A, cudaStream_t st)
{
    constexpr int smem = fwd_smem_floats<D, R>() * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(lem_fwd_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    lem_fwd_kernel<D, R><<<(A.B + kG * R - 1) / (kG * R), kG * D, smem, st>>>(A);
    return cudaGetLastError();
}
template <int D, int R>
cudaError_t launch_bwd_r(const LemArgs &A, cudaStream_t st)
{
    constexpr int smem = bwd_smem_floats<D, R>() * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(lem_bwd_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    lem_bwd_kernel<D, R><<<(A.B + kG * R - 1) / (kG * R), kG * D, smem, st>>>(A);
    return cudaGetLastError();
}
template <int D>
cudaError_t launch_fwd(const LemArgs &A, cudaStream_t st)
{
    return seq_per_thread(A.B) == 2 ? launch_fwd_r<D, 2>(A, st) : launch_fwd_r<D, 1>(A, st);
}
template <int D>
cudaError_t launch_bwd(const LemArgs &A, cudaStream_t st)
{
    return seq_per_thread(A.B) == 2 ? launch_bwd_r<D, 2>(A, st) : launch_bwd_r<D, 1>(A, st);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" long long fdtd_llg_lem_param_count(int d, int m)
{
    if (!(d == 16 || d == 32 || d == 64) || m < 1 || m > kMMax) return 0;
    return cell_offset(4, d, m) + (long long)m * d;
}

extern "C" int fdtd_llg_lem_workspace_bytes(const fdtd_llg_lem_shape *s, size_t *bytes)
{
    if (!shape_ok(s) || !bytes) return fail(FDTD_E_INVAL, "lem: bad shape (d in {16,32,64}, 1 <= m <= 4, sizes >= 1)");
    *bytes = layout(s).total;
    return FDTD_OK;
}

extern "C" int fdtd_llg_lem_views(const fdtd_llg_lem_shape *s, void *work, float **recon, float **out, float **grad,
                                  double **loss)
{
    if (!shape_ok(s) || !work) return fail(FDTD_E_INVAL, "lem_views: bad shape or NULL work space");
    const Layout L = layout(s);
    unsigned char *w = static_cast<unsigned char *>(work);
    if (recon) *recon = reinterpret_cast<float *>(w + L.recon);
    if (out) *out = reinterpret_cast<float *>(w + L.out);
    if (grad) *grad = reinterpret_cast<float *>(w + L.grad);
    if (loss) *loss = reinterpret_cast<double *>(w + L.loss);
    return FDTD_OK;
}

extern "C" int fdtd_llg_lem_forward(const fdtd_llg_lem_shape *s, const float *theta, const float *u, void *work,
                                    void *stream)
{
    if (!shape_ok(s) || !theta || !u || !work) return fail(FDTD_E_INVAL, "lem_forward: bad shape or NULL pointer");
    const LemArgs A = args(s, theta, u, work);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = s->d == 64 ? launch_fwd<64>(A, st) : s->d == 32 ? launch_fwd<32>(A, st) : launch_fwd<16>(A, st);
    return e == cudaSuccess ? FDTD_OK : cuda_fail(e, "lem_forward");
}

extern "C" int fdtd_llg_lem_loss(const fdtd_llg_lem_shape *s, const fdtd_llg_lem_physics *p, const float *u,
                                 const float *target, const float *h, void *work, void *stream)
{
    if (!shape_ok(s) || !p || !u || !target || !work) return fail(FDTD_E_INVAL, "lem_loss: bad shape or NULL pointer");
    if (p->lam != 0.f && !h) return fail(FDTD_E_INVAL, "lem_loss: the physics term needs h");
    if (p->lam != 0.f && s->m != 2) return fail(FDTD_E_INVAL, "lem_loss: the physics term needs m = 2");
    const Layout L = layout(s);
    unsigned char *w = static_cast<unsigned char *>(work);
    LossArgs A{};
    A.B = s->batch; A.m = s->m; A.t_in = s->t_in; A.t_out = s->t_out;
    A.lam = p->lam; A.kappa = p->kappa; A.alpha = p->alpha; A.h0 = p->h0;
    A.u = u; A.target = target; A.h = h;
    A.recon = reinterpret_cast<const float *>(w + L.recon);
    A.out = reinterpret_cast<const float *>(w + L.out);
    A.drec = reinterpret_cast<float *>(w + L.drec);
    A.dout = reinterpret_cast<float *>(w + L.dout);
    A.lpart = reinterpret_cast<double *>(w + L.lpart);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    lem_loss_kernel<<<L.nlblk, kLossThreads, 0, st>>>(A);
    const long long NR = (long long)s->t_in * s->batch * s->m, NPM = (long long)s->t_out * s->batch * s->m;
    lem_loss_final_kernel<<<1, kLossThreads, 0, st>>>(A.lpart, L.nlblk, NR, NPM, (double)p->lam,
                                                       reinterpret_cast<double *>(w + L.loss));
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FDTD_OK : cuda_fail(e, "lem_loss");
}

extern "C" int fdtd_llg_lem_backward(const fdtd_llg_lem_shape *s, const float *theta, const float *u, void *work,
                                     void *stream)
{
    if (!shape_ok(s) || !theta || !u || !work) return fail(FDTD_E_INVAL, "lem_backward: bad shape or NULL pointer");
    const LemArgs A = args(s, theta, u, work);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = s->d == 64 ? launch_bwd<64>(A, st) : s->d == 32 ? launch_bwd<32>(A, st) : launch_bwd<16>(A, st);
    if (e != cudaSuccess) return cuda_fail(e, "lem_backward");
    const WProdSet S = products(s, A);
    float *part = reinterpret_cast<float *>(A.w + A.L.wpart), *grad = reinterpret_cast<float *>(A.w + A.L.grad);
    e = cudaFuncSetAttribute(lem_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgradSmem);
    if (e != cudaSuccess) return cuda_fail(e, "lem_backward");
    lem_wgrad_kernel<<<S.nchunks, 256, kWgradSmem, st>>>(S, part);
    const long long P = fdtd_llg_lem_param_count(s->d, s->m);
    lem_wreduce_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(S, part, grad);
    e = cudaGetLastError();
    return e == cudaSuccess ? FDTD_OK : cuda_fail(e, "lem_backward");
}

extern "C" int fdtd_llg_lem_adam(long long n, float *theta, const float *grad, float *mom, float *vel, float lr,
                                 float beta1, float beta2, float eps, int t, void *stream)
{
    if (n < 1 || !theta || !grad || !mom || !vel || t < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(FDTD_E_INVAL, "lem_adam: bad argument");
    const float c1 = (float)(1.0 - std::pow((double)beta1, t)), c2 = (float)(1.0 - std::pow((double)beta2, t));
    lem_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, theta, grad, mom, vel, lr, beta1, beta2, eps, c1, c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FDTD_OK : cuda_fail(e, "lem_adam");
}

extern "C" int fdtd_llg_lem_train_step(const fdtd_llg_lem_shape *s, const fdtd_llg_lem_physics *p, float *theta,
                                       const float *u, const float *target, const float *h, float *mom, float *vel,
                                       float lr, int t, void *work, void *stream)
{
    int r = fdtd_llg_lem_forward(s, theta, u, work, stream);
    if (r == FDTD_OK) r = fdtd_llg_lem_loss(s, p, u, target, h, work, stream);
    if (r == FDTD_OK) r = fdtd_llg_lem_backward(s, theta, u, work, stream);
    if (r == FDTD_OK) {
        float *grad = nullptr;
        fdtd_llg_lem_views(s, work, nullptr, nullptr, &grad, nullptr);
        r = fdtd_llg_lem_adam(fdtd_llg_lem_param_count(s->d, s->m), theta, grad, mom, vel, lr, 0.9f, 0.999f, 1e-8f, t,
                              stream);
    }
    return r;
}
