// Reverse-time (adjoint) kernels of the Yee-Maxwell + LLG step (arxiv
// 2510.22221, section "Numerical Model"): the exact transpose of the discrete
// forward map of kernels_fwd.cu, one reverse step at a time.
//
// Forward step n:  E' = ca E + cb (C_H H - J);  then two half-pushes
//   H* = H - ch C_E E',  M' = LLG(M, H*),  H' = H* - P (M' - M)
// (P: half the change of each adjacent cell's M on a face).  Its transpose,
// with lambda the adjoint of the step's outputs:
//   magnetic regions (adj_mag_kernel): both half-pushes reversed through the
//     fixed number of Jacobi iterates of the trapezoidal LLG solve, which the
//     forward magnet kernel recorded on the tape during the segment's
//     recomputation (the transposed 3 x 9 Jacobian of one cell's increment
//     applied in one reverse-mode pass, llg_inc_vjp), giving
//     the adjoint of the faces' H and of M at the step's start, of the curl
//     terms, and d J / d |H_bias|;
//   adj_curl_h_kernel:  the probe seed dJ/dE^n is added to lambda_E, then
//     lambda_E' = lambda_E - (dt/mu0) C_H lambda_H (for a non-magnetic face
//     both half-pushes pass lambda_H through; magnetic faces carry the magnet
//     kernel's curl adjoint here); it stores w = cb lambda_E' (per step
//     parity) and lambda_E = ca lambda_E' (the class lookup once per edge),
//     and on the design-box edges adds d J / d eps_edge += (w/dt) (E^n -
//     E^{n+1}).  Its curls leave the magnetic faces out; adj_face_fix_kernel
//     then writes those faces' values from the magnet kernel and adds their
//     part to the edges beside them (lists built once per reverse sweep);
//   adj_curl_e_kernel:  lambda_H += C_E w, except at the magnetic faces, to
//     which the next reverse step's magnet kernel adds C_E w as it reads them
//     (adj_fix_kernel after the last);
//   the magnetic faces then take their own adjoint: the next reverse step's
//     magnet kernel adds the pending correction as it reads them
//     (adj_fix_kernel applies the last one after the sweep).
// So the magnet kernel of a step shares no data with the two curl sweeps
// beside which it runs (on a second stream, adj_reverse_step).
// C_E^T = C_H on the Yee grid, so the transposed curls are the forward curls.
#include "fdtd_llg_internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace fl {

namespace {

// Reverse mode of one cell's LLG increment dl = M^{r} - M^n in the bias frame
// (the arithmetic of mag_kernel; m deviation from Ms e3, hs = H_eff at the
// start of the half-push, h = H_eff of the previous iterate, both with the
// bias on e3): given ld, the adjoint of dl, returns the
// adjoints gm, ghs, gh of m, hs and h (J^T ld for the 3 x 9 Jacobian).  With
// M = m + Ms e3 and S = hs + h the increment is
//   a = -(kappa h + (alpha/Ms) M),  r = -kappa M x S,
//   d = (r + (a.r) a - a x r) / (1 + a.a),
//   dl = d + s1 (M + d),  s1 = -md2 / (|M~| (|M| + |M~|)),
//   md2 = 2 M.d + d.d,  |M~| = sqrt(|M|^2 + md2),
// and the adjoints below run those lines backwards.
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ void llg_inc_vjp(const float m[3], const float hs[3], const float h[3], const MagMat &mm, const float ld[3],
                            float gm[3], float ghs[3], float gh[3])
{
    const float k = mm.kappa, dam = mm.alpha * mm.inv_Ms;
    const float M[3] = {m[0], m[1], m[2] + mm.Ms};
    const float S[3] = {hs[0] + h[0], hs[1] + h[1], hs[2] + h[2]};
    float a[3], r[3], MxS[3], axr[3], u[3], d[3], Md[3];
    for (int c = 0; c < 3; ++c) a[c] = -(k * h[c] + dam * M[c]);
    cross3(M, S, MxS);
    for (int c = 0; c < 3; ++c) r[c] = -k * MxS[c];
    const float ar = dot3(a, r);
    const float inv1 = __frcp_rn(1.f + dot3(a, a));
    cross3(a, r, axr);
    for (int c = 0; c < 3; ++c) {
        u[c] = r[c] + ar * a[c] - axr[c];
        d[c] = u[c] * inv1;
        Md[c] = M[c] + d[c];
    }
    const float nM2 = dot3(M, M);
    const float md2 = 2.f * dot3(M, d) + dot3(d, d);
    // reciprocals from the intrinsics (the chain's latency; the adjoint
    // tolerates their last-bit differences from the forward's sqrt and divide)
    const float rnM = rsqrtf(nM2), rnMt = rsqrtf(nM2 + md2);
    const float nM = nM2 * rnM, nMt = (nM2 + md2) * rnMt;
    const float P = nMt * (nM + nMt), rP = __frcp_rn(P);
    const float s1 = -md2 * rP;
    // dl = d + s1 (M + d)
    float gd[3], gM[3];
    for (int c = 0; c < 3; ++c) {
        gd[c] = ld[c] * (1.f + s1);
        gM[c] = ld[c] * s1;
    }
    const float gs1 = dot3(ld, Md);
    // s1 = -md2 / P, P = nMt nM + nMt^2
    float gmd2 = -gs1 * rP;
    const float gP = gs1 * md2 * rP * rP;
    const float gnMt = gP * (nM + 2.f * nMt), gnM = gP * nMt;
    const float gt = 0.5f * gnMt * rnMt;       // nMt = sqrt(nM2 + md2)
    gmd2 += gt;
    const float gnM2 = gt + 0.5f * gnM * rnM;
    // md2 = 2 M.d + d.d,  nM2 = M.M
    for (int c = 0; c < 3; ++c) {
        gM[c] += 2.f * gmd2 * d[c] + 2.f * gnM2 * M[c];
        gd[c] += 2.f * gmd2 * (M[c] + d[c]);
    }
    // d = u inv1,  inv1 = 1 / (1 + a.a)
    float gu[3], ga[3], gr[3];
    const float ginv1 = dot3(gd, u);
    for (int c = 0; c < 3; ++c) {
        gu[c] = gd[c] * inv1;
        ga[c] = -2.f * ginv1 * inv1 * inv1 * a[c];
    }
    // u = r + (a.r) a - a x r
    const float gar = dot3(gu, a);
    float uxr[3], axu[3];
    cross3(gu, r, uxr);   // adjoint of a in -(a x r): gu x r
    cross3(a, gu, axu);   // adjoint of r in -(a x r): a x gu
    for (int c = 0; c < 3; ++c) {
        gr[c] = gu[c] + axu[c] + gar * a[c];
        ga[c] += ar * gu[c] + uxr[c] + gar * r[c];
    }
    // a = -(kappa h + dam M),  r = -kappa M x S
    float Sxg[3], gxM[3];
    cross3(S, gr, Sxg);
    cross3(gr, M, gxM);
    for (int c = 0; c < 3; ++c) {
        gm[c] = gM[c] - dam * ga[c] - k * Sxg[c];
        const float gS = -k * gxM[c];
        ghs[c] = gS;
        gh[c] = gS - k * ga[c];
    }
}

__device__ __forceinline__ void to_fr(const float *R, const float g[3], float l[3])
{
    l[0] = R[0] * g[0] + R[1] * g[1] + R[2] * g[2];
    l[1] = R[3] * g[0] + R[4] * g[1] + R[5] * g[2];
    l[2] = R[6] * g[0] + R[7] * g[1] + R[8] * g[2];
}
__device__ __forceinline__ void from_fr(const float *R, const float l[3], float g[3])
{
    g[0] = R[0] * l[0] + R[3] * l[1] + R[6] * l[2];
    g[1] = R[1] * l[0] + R[4] * l[1] + R[7] * l[2];
    g[2] = R[2] * l[0] + R[5] * l[1] + R[8] * l[2];
}
__device__ __forceinline__ float curl2a(float a1, float b1, float i1, float a2, float b2, float i2)
{
    return __fsub_rn(__fmul_rn(__fsub_rn(a1, b1), i1), __fmul_rn(__fsub_rn(a2, b2), i2));
}

// Component a of C_E w at the face (i, j, k) of the field arrays (w zero
// beyond the far walls): what adj_curl_e_kernel adds to lambda_H there, with
// its arithmetic, for the magnetic faces that it leaves to the magnet kernels.
__device__ __forceinline__ float face_curl_w(const Inst *I, const float *w, int a, int i, int j, int k)
{
    const long long fs = I->fstride, plane = I->plane;
    const int px = I->px;
    const long long o = (long long)k * plane + (long long)j * px + i;
    const float *wx = w, *wy = w + fs, *wz = w + 2 * fs;
    const bool xi = i + 1 < I->nx, yj = j + 1 < I->ny, zk = k + 1 < I->nz;
    if (a == 0) return curl2a(yj ? wz[o + px] : 0.f, wz[o], I->idy, zk ? wy[o + plane] : 0.f, wy[o], I->idz);
    if (a == 1) return curl2a(zk ? wx[o + plane] : 0.f, wx[o], I->idz, xi ? wz[o + 1] : 0.f, wz[o], I->idx);
    return curl2a(xi ? wy[o + 1] : 0.f, wy[o], I->idx, yj ? wx[o + px] : 0.f, wx[o], I->idy);
}

// Magnetic neighbours of face f (cells on its low and high side, -1 where
// outside the box or not magnetic), built once per kernel in shared memory.
struct FaceNb {
    int vl, vr;
};
__device__ __forceinline__ int face_axis(int f, int nfx, int nfy) { return f < nfx ? 0 : (f < nfx + nfy ? 1 : 2); }

__device__ __forceinline__ float *hx_at(const Inst *I, float *F0, int i, int j, int k, float *wall)
{
    return (i == I->nx) ? wall + (long long)k * I->ny + j : F0 + 3 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hy_at(const Inst *I, float *F0, int i, int j, int k, float *wall)
{
    return (j == I->ny) ? wall + (long long)I->ny * I->nz + (long long)k * I->nx + i
                        : F0 + 4 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}
__device__ __forceinline__ float *hz_at(const Inst *I, float *F0, int i, int j, int k, float *wall)
{
    return (k == I->nz) ? wall + (long long)I->ny * I->nz + (long long)I->nx * I->nz + (long long)j * I->nx + i
                        : F0 + 5 * I->fstride + (long long)k * I->plane + (long long)j * I->px + i;
}

// Workspace of one region (floats), nf faces, V cells:
//   C, lamHout, lamHin, lamC, fix (5 nf);  lamM, lamDl, lamA, lamHsm, lamHg[2] (6 x 3V);
//   dq (nf).
// fix carries the magnetic faces' pending correction from one reverse step to
// the next; everything the forward step computed comes from the tape.  lamHg
// is double-buffered by the parity of the iterate, so a cell's new value
// never overwrites one that a neighbour may still read.  dq: the value a
// magnetic face must show the curl sweep (q/2, for adj_face_fix_kernel).
struct RegionWS {
    float *C, *lamHout, *lamHin, *lamC, *fix;
    float *lamM, *lamDl, *lamA, *lamHsm, *lamHg[2];
    float *dq;
};
__device__ __forceinline__ RegionWS carve(float *w, int nf, int V)
{
    RegionWS r;
    r.C = w; r.lamHout = r.C + nf; r.lamHin = r.lamHout + nf; r.lamC = r.lamHin + nf; r.fix = r.lamC + nf;
    float *p = r.fix + nf;
    r.lamM = p; r.lamDl = p + 3 * V; r.lamA = p + 6 * V; r.lamHsm = p + 9 * V;
    r.lamHg[0] = p + 12 * V; r.lamHg[1] = p + 15 * V;
    r.dq = p + 18 * V;
    return r;
}

// Cell v's inputs to iteration r of a half-push: hs (bias frame, with bias),
// h (bias frame, from D^{r-1}; Dprev NULL for r = 1), m.
__device__ void cell_inputs(const MagComp &C, const BoxDiv &BD, const Inst *I, const float *R9, const uint8_t *smat, int V,
                            const float *Hs, const float *Cc, const float *Dprev, const float *m, int v, float hs[3],
                            float h[3], float mm[3], int nfx, int nfy)
{
    const int bx = C.bx, by = C.by, bxy = C.bx * C.by;
    int li, lj, lk;
    cell_decode(v, BD, li, lj, lk);
    const int fx0 = (lk * by + lj) * (bx + 1) + li, fy0 = nfx + (lk * (by + 1) + lj) * bx + li,
              fz0 = nfx + nfy + (lk * by + lj) * bx + li;
    const int f0[3] = {fx0, fy0, fz0}, f1[3] = {fx0 + 1, fy0 + bx, fz0 + bxy};
    float Hm[3], A[3];
    for (int a = 0; a < 3; ++a) {
        Hm[a] = 0.5f * (Hs[f0[a]] + Hs[f1[a]]);
        A[a] = 0.5f * ((Hs[f0[a]] - Cc[f0[a]]) + (Hs[f1[a]] - Cc[f1[a]]));
    }
    if (Dprev) {
        const int st[3] = {1, bx, bxy};
        const bool lo[3] = {li > 0, lj > 0, lk > 0}, hi[3] = {li < bx - 1, lj < by - 1, lk < C.bz - 1};
        // the neighbours' values are loaded with their material ids, not
        // after them (a non-magnetic cell's tape entry is in bounds, unused)
        for (int a = 0; a < 3; ++a) {
            const float dmv = lo[a] ? Dprev[a * V + v - st[a]] : 0.f, dpv = hi[a] ? Dprev[a * V + v + st[a]] : 0.f;
            const bool ml = lo[a] && smat[v - st[a]] != 0xFF, mh = hi[a] && smat[v + st[a]] != 0xFF;
            const float dm = ml ? dmv : 0.f, dp = mh ? dpv : 0.f;
            A[a] -= 0.25f * (dm + 2.f * Dprev[a * V + v] + dp);
        }
    }
    to_fr(R9, Hm, hs);
    to_fr(R9, A, h);
    hs[2] += I->h0n;
    h[2] += I->h0n;
    mm[0] = m[v];
    mm[1] = m[V + v];
    mm[2] = m[2 * V + v];
}

// A region's reverse pass may be split over the cs CTAs of a thread-block
// cluster: CTA rank takes every cell and face index in the blocks
// rank * nth + [0, nth) of each cs * nth (part0 = rank * nth, pstep = cs *
// nth), all of its data in the region's global workspace, and every barrier
// of the pass is the cluster's (release and acquire at cluster scope, so the
// other CTAs' workspace writes are visible after it).
__device__ __forceinline__ void region_sync(int cs)
{
    if (cs > 1) cg::this_cluster().sync();
    else __syncthreads();
}

// Reverse of one half-push.  In: lamHout (faces), lamM (adjoint of the output
// m, bias frame; overwritten with the adjoint of the input m).  Out: lamHin,
// lamC (faces); *gh0 accumulates d J / d |H_bias| of this thread's cells.
// A thread keeps the same cells and faces in every loop, so only what a loop
// reads of other threads' cells or faces needs a barrier before it: one after
// each iterate's cell pass (the neighbours' lamHg, and at the end their lamA
// and lamHsm for the faces).  The caller separates two calls by a barrier.
__device__ void rev_half(const MagComp &C, const BoxDiv &BD, const FaceNb *fnb, const Inst *I, const float *R9,
                         const uint8_t *smat, int V, int nf, int R, const float *Hs, const float *Cc, const float *m,
                         const float *D, RegionWS &W, const float *lamHout, float *lamHin, float *lamC, double *gh0, int nfx,
                         int nfy, int cs)
{
    const int tid = threadIdx.x + (cs > 1 ? (int)cg::this_cluster().block_rank() : 0) * blockDim.x;
    const int nth = blockDim.x * cs;
    const int bx = C.bx, by = C.by, bxy = bx * by;
    // direct terms of H_out = H* - P D^R, H* = Hs - C: the adjoint of dl^R
    for (int v = tid; v < V; v += nth) {
        for (int a = 0; a < 3; ++a) W.lamA[a * V + v] = W.lamHsm[a * V + v] = 0.f;
        if (smat[v] == 0xFF) {
            for (int a = 0; a < 3; ++a) W.lamDl[a * V + v] = 0.f;
            continue;
        }
        int li, lj, lk;
        cell_decode(v, BD, li, lj, lk);
        const int fx0 = (lk * by + lj) * (bx + 1) + li, fy0 = nfx + (lk * (by + 1) + lj) * bx + li,
                  fz0 = nfx + nfy + (lk * by + lj) * bx + li;
        const float lD[3] = {-0.5f * (lamHout[fx0] + lamHout[fx0 + 1]), -0.5f * (lamHout[fy0] + lamHout[fy0 + bx]),
                             -0.5f * (lamHout[fz0] + lamHout[fz0 + bxy])};
        float l[3];
        to_fr(R9, lD, l);   // D = R^T dl, so the adjoint of dl is R times that of D
        for (int a = 0; a < 3; ++a) W.lamDl[a * V + v] = W.lamM[a * V + v] + l[a];
    }
    double g = 0.0;
    for (int r = R; r >= 1; --r) {
        const float *Dp = r >= 2 ? D + 3 * V * (r - 2) : nullptr;
        float *lamHg = W.lamHg[r & 1];
        for (int v = tid; v < V; v += nth) {
            const int mt = smat[v];
            if (mt == 0xFF) {
                lamHg[v] = lamHg[V + v] = lamHg[2 * V + v] = 0.f;
                continue;
            }
            float hs[3], h[3], mm[3];
            cell_inputs(C, BD, I, R9, smat, V, Hs, Cc, Dp, m, v, hs, h, mm, nfx, nfy);
            const float ld[3] = {W.lamDl[v], W.lamDl[V + v], W.lamDl[2 * V + v]};
            // the cell's accumulators, loaded before the arithmetic
            float lM[3], lsm[3], lA[3];
            for (int a = 0; a < 3; ++a) {
                lM[a] = W.lamM[a * V + v];
                lsm[a] = W.lamHsm[a * V + v];
                lA[a] = W.lamA[a * V + v];
            }
            // J^T lambda in one reverse pass: gin = (m, hs, h) adjoints
            float gin[9];
            llg_inc_vjp(mm, hs, h, I->mm[mt], ld, gin, gin + 3, gin + 6);
            for (int a = 0; a < 3; ++a) {
                W.lamM[a * V + v] = lM[a] + gin[a];
                lsm[a] += gin[3 + a];   // bias frame
            }
            if (r == 1) {   // the last iterate: hs's adjoint to global axes
                float gq[3];
                from_fr(R9, lsm, gq);
                for (int a = 0; a < 3; ++a) lsm[a] = gq[a];
            }
            for (int a = 0; a < 3; ++a) W.lamHsm[a * V + v] = lsm[a];
            g += (double)gin[5] + (double)gin[8];     // |H_bias| enters hs and h on e3
            float lh[3] = {gin[6], gin[7], gin[8]}, lg[3];
            from_fr(R9, lh, lg);
            for (int a = 0; a < 3; ++a) {
                lamHg[a * V + v] = lg[a];
                W.lamA[a * V + v] = lA[a] + lg[a];
            }
        }
        region_sync(cs);
        if (r >= 2) {
            // h depends on D^{r-1} through -1/4 (D_{v-1} + 2 D_v + D_{v+1}) per component
            for (int v = tid; v < V; v += nth) {
                if (smat[v] == 0xFF) {
                    W.lamDl[v] = W.lamDl[V + v] = W.lamDl[2 * V + v] = 0.f;
                    continue;
                }
                int li, lj, lk;
                cell_decode(v, BD, li, lj, lk);
                const int st[3] = {1, bx, bxy};
                const bool lo[3] = {li > 0, lj > 0, lk > 0}, hi[3] = {li < bx - 1, lj < by - 1, lk < C.bz - 1};
                float lD[3];
                for (int a = 0; a < 3; ++a) {
                    const float gm = lo[a] ? lamHg[a * V + v - st[a]] : 0.f;
                    const float gp = hi[a] ? lamHg[a * V + v + st[a]] : 0.f;
                    lD[a] = -0.25f * (gm + 2.f * lamHg[a * V + v] + gp);
                }
                float l[3];
                to_fr(R9, lD, l);
                for (int a = 0; a < 3; ++a) W.lamDl[a * V + v] = l[a];
            }
        }
    }
    *gh0 += g;
    // faces: A = mean(Hs - C), hs = R mean(Hs) + bias
    for (int f = tid; f < nf; f += nth) {
        const FaceNb q = fnb[f];
        const int a = face_axis(f, nfx, nfy);
        float sA = 0.f, sH = 0.f;
        if (q.vl >= 0) { sA += 0.5f * W.lamA[a * V + q.vl]; sH += 0.5f * W.lamHsm[a * V + q.vl]; }
        if (q.vr >= 0) { sA += 0.5f * W.lamA[a * V + q.vr]; sH += 0.5f * W.lamHsm[a * V + q.vr]; }
        lamHin[f] = lamHout[f] + (sA + sH);
        lamC[f] = -lamHout[f] - sA;
    }
}

// rev_half when the region has no more cells than the cluster has threads:
// thread tid owns cell v = tid (if v < V), whose face-derived inputs (mean H^s
// and mean H^s - C), start-of-step m and own accumulators (adjoints of m, of
// dl, of hs, the sum of the h adjoints) stay in registers through the
// iterates, and whose tape values D^{r-1} for the next iterate are fetched
// while the present one computes.  Only lamHg (read by the neighbours) and,
// at the end, lamA, lamHsm and lamM go through the workspace.  The same
// float operations in the same order as rev_half: the same bits.
__device__ void rev_half_1(const MagComp &C, const BoxDiv &BD, const FaceNb *fnb, const Inst *I, const float *R9,
                           const uint8_t *smat, int V, int nf, int R, const float *Hs, const float *Cc, const float *m,
                           const float *D, RegionWS &W, const float *lamHout, float *lamHin, float *lamC, double *gh0,
                           int nfx, int nfy, int cs)
{
    const int tid = threadIdx.x + (cs > 1 ? (int)cg::this_cluster().block_rank() : 0) * blockDim.x;
    const int nth = blockDim.x * cs;
    const int bx = C.bx, by = C.by, bxy = bx * by;
    const int v = tid;
    const bool in = v < V, has = in && smat[v] != 0xFF;
    const int mt = in ? smat[v] : 0xFF;
    int li = 0, lj = 0, lk = 0;
    if (in) cell_decode(v, BD, li, lj, lk);
    const int st[3] = {1, bx, bxy};
    const bool lo[3] = {li > 0, lj > 0, lk > 0}, hi[3] = {li < bx - 1, lj < by - 1, lk < C.bz - 1};
    bool ml[3], mh[3];   // magnetic neighbours below and above
    for (int a = 0; a < 3; ++a) {
        ml[a] = in && lo[a] && smat[v - st[a]] != 0xFF;
        mh[a] = in && hi[a] && smat[v + st[a]] != 0xFF;
    }
    float Hm[3] = {0.f, 0.f, 0.f}, A0[3] = {0.f, 0.f, 0.f}, mm[3] = {0.f, 0.f, 0.f};
    float lM[3] = {0.f, 0.f, 0.f}, lDl[3] = {0.f, 0.f, 0.f};
    if (has) {
        const int fx0 = (lk * by + lj) * (bx + 1) + li, fy0 = nfx + (lk * (by + 1) + lj) * bx + li,
                  fz0 = nfx + nfy + (lk * by + lj) * bx + li;
        const int f0[3] = {fx0, fy0, fz0}, f1[3] = {fx0 + 1, fy0 + bx, fz0 + bxy};
        for (int a = 0; a < 3; ++a) {
            Hm[a] = 0.5f * (Hs[f0[a]] + Hs[f1[a]]);
            A0[a] = 0.5f * ((Hs[f0[a]] - Cc[f0[a]]) + (Hs[f1[a]] - Cc[f1[a]]));
            mm[a] = m[a * V + v];
            lM[a] = W.lamM[a * V + v];
        }
        // direct terms of H_out = H* - P D^R, H* = Hs - C: the adjoint of dl^R
        const float lD[3] = {-0.5f * (lamHout[fx0] + lamHout[fx0 + 1]), -0.5f * (lamHout[fy0] + lamHout[fy0 + bx]),
                             -0.5f * (lamHout[fz0] + lamHout[fz0 + bxy])};
        float l[3];
        to_fr(R9, lD, l);   // D = R^T dl, so the adjoint of dl is R times that of D
        for (int a = 0; a < 3; ++a) lDl[a] = lM[a] + l[a];
    }
    // D^{r-1} at the cell and its neighbours along each axis (0 where not magnetic)
    float dc[3], dm[3], dp[3];
    auto fetch = [&](int r) {
        const float *Dp = D + 3 * V * (r - 2);
        for (int a = 0; a < 3; ++a) {
            const float dmv = lo[a] && has ? Dp[a * V + v - st[a]] : 0.f, dpv = hi[a] && has ? Dp[a * V + v + st[a]] : 0.f;
            dc[a] = has ? Dp[a * V + v] : 0.f;
            dm[a] = ml[a] ? dmv : 0.f;
            dp[a] = mh[a] ? dpv : 0.f;
        }
    };
    if (R >= 2) fetch(R);
    float lsm[3] = {0.f, 0.f, 0.f}, lA[3] = {0.f, 0.f, 0.f};
    double g = 0.0;
    for (int r = R; r >= 1; --r) {
        float *lamHg = W.lamHg[r & 1];
        if (has) {
            float A[3] = {A0[0], A0[1], A0[2]};
            if (r >= 2)
                for (int a = 0; a < 3; ++a) A[a] -= 0.25f * (dm[a] + 2.f * dc[a] + dp[a]);
            if (r - 1 >= 2) fetch(r - 1);   // the next iterate's tape values, while this one computes
            float hs[3], h[3];
            to_fr(R9, Hm, hs);
            to_fr(R9, A, h);
            hs[2] += I->h0n;
            h[2] += I->h0n;
            // J^T lambda in one reverse pass: gin = (m, hs, h) adjoints
            float gin[9];
            llg_inc_vjp(mm, hs, h, I->mm[mt], lDl, gin, gin + 3, gin + 6);
            for (int a = 0; a < 3; ++a) {
                lM[a] = lM[a] + gin[a];
                lsm[a] += gin[3 + a];   // bias frame
            }
            if (r == 1) {   // the last iterate: hs's adjoint to global axes
                float gq[3];
                from_fr(R9, lsm, gq);
                for (int a = 0; a < 3; ++a) lsm[a] = gq[a];
            }
            g += (double)gin[5] + (double)gin[8];     // |H_bias| enters hs and h on e3
            float lh[3] = {gin[6], gin[7], gin[8]}, lg[3];
            from_fr(R9, lh, lg);
            for (int a = 0; a < 3; ++a) {
                lamHg[a * V + v] = lg[a];
                lA[a] = lA[a] + lg[a];
            }
        } else if (in) {
            lamHg[v] = lamHg[V + v] = lamHg[2 * V + v] = 0.f;
        }
        if (r == 1 && in)   // what the face loop reads of the neighbours, and m's adjoint
            for (int a = 0; a < 3; ++a) {
                W.lamA[a * V + v] = lA[a];
                W.lamHsm[a * V + v] = lsm[a];
                W.lamM[a * V + v] = lM[a];
            }
        region_sync(cs);
        if (r >= 2) {
            // h depends on D^{r-1} through -1/4 (D_{v-1} + 2 D_v + D_{v+1}) per component
            if (has) {
                float lD[3];
                for (int a = 0; a < 3; ++a) {
                    const float gm = lo[a] ? lamHg[a * V + v - st[a]] : 0.f;
                    const float gp = hi[a] ? lamHg[a * V + v + st[a]] : 0.f;
                    lD[a] = -0.25f * (gm + 2.f * lamHg[a * V + v] + gp);
                }
                to_fr(R9, lD, lDl);
            }
        }
    }
    *gh0 += g;
    // faces: A = mean(Hs - C), hs = R mean(Hs) + bias
    for (int f = tid; f < nf; f += nth) {
        const FaceNb q = fnb[f];
        const int a = face_axis(f, nfx, nfy);
        float sA = 0.f, sH = 0.f;
        if (q.vl >= 0) { sA += 0.5f * W.lamA[a * V + q.vl]; sH += 0.5f * W.lamHsm[a * V + q.vl]; }
        if (q.vr >= 0) { sA += 0.5f * W.lamA[a * V + q.vr]; sH += 0.5f * W.lamHsm[a * V + q.vr]; }
        lamHin[f] = lamHout[f] + (sA + sH);
        lamC[f] = -lamHout[f] - sA;
    }
}

__global__ void __launch_bounds__(kMagThreads) adj_mag_kernel(LaunchSet L, AdjSet A, int slot, int wpar)
{
    extern __shared__ FaceNb fnb[];   // nf entries (every CTA of a region holds the whole table), then V material ids
    __shared__ double sred[kMagThreads / 32];
    const int cs = A.cs, rc = blockIdx.x / cs;
    const int rank = cs > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const MagComp C = L.comps[rc];
    const Inst *I = L.insts + C.inst;
    // this CTA's part of the region's cells and faces (see region_sync)
    const int tid = threadIdx.x + rank * blockDim.x, nth = blockDim.x * cs;
    const int V = C.V, bx = C.bx, by = C.by, bz = C.bz;
    const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nf = nfx + nfy + bx * by * (bz + 1);
    const int ex = bx + 1, exy = (bx + 1) * (by + 1), ne = exy * (bz + 1);
    const int R = A.R;
    float *wsb = A.ws + A.ws_off[rc];
    RegionWS W = carve(wsb + (V + 3) / 4, nf, V);
    uint8_t *smat = reinterpret_cast<uint8_t *>(fnb + nf);   // the box's material ids, in shared memory
    float R9[9];
    for (int q = 0; q < 9; ++q) R9[q] = I->R[q];
    // the forward step's records (mag_tape_floats): m and faces at its start,
    // E^{n+1} at the box edges, the Jacobi iterates of both half-pushes, faces
    // and m after the first half-push
    const float *T = C.tape + (long long)slot * C.tstride;
    const float *m1 = T, *Hs1 = T + 3 * V;
    const float *Ex = T + 3 * V + nf, *Ey = Ex + ne, *Ez = Ey + ne;
    const float *D1 = T + 3 * V + nf + 3 * ne, *D2 = D1 + 3LL * R * V;
    const float *Hs2 = D2 + 3LL * R * V, *m2 = Hs2 + nf;
    const BoxDiv BD(bx, by);
    for (int v = threadIdx.x; v < V; v += blockDim.x) smat[v] = C.mat[v];
    __syncthreads();
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        int a, fi, fj, fk, vl, vr;
        face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
        fnb[f] = {vl >= 0 && smat[vl] != 0xFF ? vl : -1, vr >= 0 && smat[vr] != 0xFF ? vr : -1};
    }
    const float ch = I->ch;
    // this CTA's faces (each written to fnb by the same thread above)
    for (int f = tid; f < nf; f += nth) {
        int a, fi, fj, fk, vl, vr;
        face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
        const int e0 = fk * exy + fj * ex + fi;
        float cu = 0.f;
        if (a == 0) cu = curl2a(Ez[e0 + ex], Ez[e0], I->idy, Ey[e0 + exy], Ey[e0], I->idz);
        else if (a == 1) cu = curl2a(Ex[e0 + exy], Ex[e0], I->idz, Ez[e0 + 1], Ez[e0], I->idx);
        else cu = curl2a(Ey[e0 + 1], Ey[e0], I->idx, Ex[e0 + ex], Ex[e0], I->idy);
        W.C[f] = ch * cu;
        // adjoint of the step's output faces (H^{n+3/2}): field arrays or
        // walls, plus the correction the later step left pending in fix
        const int i = C.x0 + fi, j = C.y0 + fj, k = C.z0 + fk;
        const bool own = fnb[f].vl >= 0 || fnb[f].vr >= 0;
        // the adjoint of the step's output face: lambda_H, with C_E w of the
        // later step added here for a magnetic face off the far walls (the
        // H-curl sweep leaves those faces out), then the pending correction
        float lh = 0.f;
        if (own) {
            const bool wall = (a == 0 && i == I->nx) || (a == 1 && j == I->ny) || (a == 2 && k == I->nz);
            lh = *(a == 0 ? hx_at(I, A.lamH, i, j, k, A.lamW)
                          : (a == 1 ? hy_at(I, A.lamH, i, j, k, A.lamW) : hz_at(I, A.lamH, i, j, k, A.lamW)));
            if (!wall) lh = lh + face_curl_w(I, A.lamEn[wpar], a, i, j, k);
            lh = lh + W.fix[f];
        }
        W.lamHout[f] = lh;
    }
    region_sync(cs);
    // reverse: second half-push, then the first
    double g = 0.0;
    const bool one = V <= nth;   // one cell per thread: rev_half_1
    if (one) rev_half_1(C, BD, fnb, I, R9, smat, V, nf, R, Hs2, W.C, m2, D2, W, W.lamHout, W.lamHin, W.lamC, &g, nfx, nfy, cs);
    else rev_half(C, BD, fnb, I, R9, smat, V, nf, R, Hs2, W.C, m2, D2, W, W.lamHout, W.lamHin, W.lamC, &g, nfx, nfy, cs);
    for (int f = tid; f < nf; f += nth) {   // the faces rev_half gave this thread
        W.lamHout[f] = W.lamHin[f];      // adjoint of H^{n+1}
        W.fix[f] = W.lamC[f];            // curl adjoint of the second half-push
    }
    region_sync(cs);
    if (one) rev_half_1(C, BD, fnb, I, R9, smat, V, nf, R, Hs1, W.C, m1, D1, W, W.lamHout, W.lamHin, W.lamC, &g, nfx, nfy, cs);
    else rev_half(C, BD, fnb, I, R9, smat, V, nf, R, Hs1, W.C, m1, D1, W, W.lamHout, W.lamHin, W.lamC, &g, nfx, nfy, cs);
    // write back: for a magnetic face the curl sweep must see q/2 with
    // q = -(lamC1 + lamC2) (a plain face contributes 2 lambda_H); afterwards
    // the face takes lamHin, restored from fix by the next reverse step's
    // magnet kernel (or adj_fix_kernel after the last).  The curl sweep,
    // running beside this kernel, leaves magnetic faces out of its curls;
    // adj_face_fix_kernel adds their q/2 afterwards and writes it to them.
    for (int f = tid; f < nf; f += nth) {
        if (fnb[f].vl < 0 && fnb[f].vr < 0) continue;
        int a, fi, fj, fk, vl, vr;
        face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
        const int i = C.x0 + fi, j = C.y0 + fj, k = C.z0 + fk;
        const float q = -(W.lamC[f] + W.fix[f]);
        const bool wall = (a == 0 && i == I->nx) || (a == 1 && j == I->ny) || (a == 2 && k == I->nz);
        float *p = a == 0 ? hx_at(I, A.lamH, i, j, k, A.lamW) : (a == 1 ? hy_at(I, A.lamH, i, j, k, A.lamW) : hz_at(I, A.lamH, i, j, k, A.lamW));
        if (wall) {
            *p = W.lamHin[f];            // the sweeps never touch the wall arrays
            W.fix[f] = 0.f;
        } else {
            W.dq[f] = 0.5f * q;
            W.fix[f] = W.lamHin[f] - 0.5f * q;
        }
    }
    // block sum of d J / d |H_bias|, fixed order (one partial per CTA)
    for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) s += sred[w];
        A.gh0[blockIdx.x] += s;
    }
    // no CTA of the cluster exits while another may still read the workspace
    // it wrote (all reads of this step are done at the last barrier)
    if (cs > 1) cg::this_cluster().sync();
}

// magnetic faces after the last reverse step: lambda_H = (q/2 + C_E w of
// that step, which the H-curl sweep left out) + (lamHin - q/2)
__global__ void adj_fix_kernel(LaunchSet L, AdjSet A, int wpar)
{
    const MagComp C = L.comps[blockIdx.x];
    const Inst *I = L.insts + C.inst;
    const int V = C.V, bx = C.bx, by = C.by, bz = C.bz;
    const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nf = nfx + nfy + bx * by * (bz + 1);
    float *wsb = A.ws + A.ws_off[blockIdx.x];
    RegionWS W = carve(wsb + (V + 3) / 4, nf, V);
    const BoxDiv BD(bx, by);
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        int a, fi, fj, fk, vl, vr;
        face_decode(f, BD, bx, by, bz, a, fi, fj, fk, vl, vr);
        const bool own = (vl >= 0 && C.mat[vl] != 0xFF) || (vr >= 0 && C.mat[vr] != 0xFF);
        if (!own) continue;
        const int i = C.x0 + fi, j = C.y0 + fj, k = C.z0 + fk;
        const bool wall = (a == 0 && i == I->nx) || (a == 1 && j == I->ny) || (a == 2 && k == I->nz);
        if (wall) continue;
        float *p = a == 0 ? hx_at(I, A.lamH, i, j, k, A.lamW) : (a == 1 ? hy_at(I, A.lamH, i, j, k, A.lamW) : hz_at(I, A.lamH, i, j, k, A.lamW));
        *p = (*p + face_curl_w(I, A.lamEn[wpar], a, i, j, k)) + W.fix[f];
    }
}

// Step n's seed dJ/dE at the probe cells, then lambda_E' = lambda_E - (dt/mu0)
// C_H lambda_H at every edge (i, j, k); stores w = cb lambda_E' and lambda_E =
// ca lambda_E', and on the design-box edges adds d J / d eps_edge += (w/dt)
// (E^n - E^{n+1}) from design-tape slots slot and slot + 1.
template <typename ClsT>
__global__ void __launch_bounds__(256) adj_curl_h_kernel(LaunchSet L, AdjSet A, long long n, int slot)
{
    const Inst *I = L.insts;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= I->nx || j >= I->ny || k >= I->nz) return;
    const long long fs = I->fstride, plane = I->plane;
    const int px = I->px;
    const long long o = (long long)k * plane + (long long)j * px + i;
    const float *lx = A.lamH + 3 * fs, *ly = A.lamH + 4 * fs, *lz = A.lamH + 5 * fs;
    const float c2 = 2.f * I->ch;   // dt / mu0: both half-pushes
    const int c = (int)static_cast<const ClsT *>(I->cls)[o];
    const float4 Ca = __ldg(I->ctab + 3 * c), Cb = __ldg(I->ctab + 3 * c + 1);
    // faces at o, o-1, o-px, o-plane; a magnetic one (flag of the class of
    // the cell it bounds from below) counts 0 here: the magnet kernel runs
    // beside this one and adj_face_fix_kernel adds its part
    float hx0 = lx[o], hy0 = ly[o], hz0 = lz[o];
    float hzj = j > 0 ? lz[o - px] : 0.f, hxj = j > 0 ? lx[o - px] : 0.f;
    float hyk = k > 0 ? ly[o - plane] : 0.f, hxk = k > 0 ? lx[o - plane] : 0.f;
    float hzi = i > 0 ? lz[o - 1] : 0.f, hyi = i > 0 ? ly[o - 1] : 0.f;
    // (only cells in the box of the magnetic faces, or one above it, read a
    // magnetic face here)
    if (L.ncomp && i >= A.mlo[0] && j >= A.mlo[1] && k >= A.mlo[2] && i <= A.mhi[0] + 1 && j <= A.mhi[1] + 1 &&
        k <= A.mhi[2] + 1) {
        auto flags = [&](long long oc) {
            return __float_as_uint(__ldg(I->ctab + 3 * (int)static_cast<const ClsT *>(I->cls)[oc]).w);
        };
        const unsigned f0 = __float_as_uint(Ca.w);
        const unsigned fi = i > 0 ? flags(o - 1) : 0u, fj = j > 0 ? flags(o - px) : 0u, fk = k > 0 ? flags(o - plane) : 0u;
        if (f0 & CF_MAG_HX) hx0 = 0.f;
        if (f0 & CF_MAG_HY) hy0 = 0.f;
        if (f0 & CF_MAG_HZ) hz0 = 0.f;
        if (fi & CF_MAG_HY) hyi = 0.f;
        if (fi & CF_MAG_HZ) hzi = 0.f;
        if (fj & CF_MAG_HX) hxj = 0.f;
        if (fj & CF_MAG_HZ) hzj = 0.f;
        if (fk & CF_MAG_HX) hxk = 0.f;
        if (fk & CF_MAG_HY) hyk = 0.f;
    }
    const float cx = curl2a(hz0, hzj, I->idy, hy0, hyk, I->idz);
    const float cy = curl2a(hx0, hxk, I->idz, hz0, hzi, I->idx);
    const float cz = curl2a(hy0, hyi, I->idx, hx0, hxj, I->idy);
    float l0 = A.lamE[o], l1 = A.lamE[fs + o], l2 = A.lamE[2 * fs + o];
    for (int p = 0; p < A.nprobe; ++p)
        if (I->probe[p][0] == i && I->probe[p][1] == j && I->probe[p][2] == k) {
            const double *sd = A.seed + (n * A.nprobe + p) * 3;
            l0 += (float)sd[0];
            l1 += (float)sd[1];
            l2 += (float)sd[2];
        }
    const float ex = l0 - c2 * cx, ey = l1 - c2 * cy, ez = l2 - c2 * cz;
    const float w[3] = {Cb.x * ex, Cb.y * ey, Cb.z * ez};   // w = cb lambda_E'
    float *wn = A.lamEn[n & 1];
    wn[o] = w[0];
    wn[fs + o] = w[1];
    wn[2 * fs + o] = w[2];
    A.lamE[o] = __fmaf_rn(Ca.x, ex, ex);   // lambda_E = ca lambda_E' (the table holds ca - 1)
    A.lamE[fs + o] = __fmaf_rn(Ca.y, ey, ey);
    A.lamE[2 * fs + o] = __fmaf_rn(Ca.z, ez, ez);
    if (A.geps) {
        const int li = i - A.di0, lj = j - A.dj0, lk = k - A.dk0;
        if (li >= 0 && lj >= 0 && lk >= 0 && li <= A.dbx && lj <= A.dby && lk <= A.dbz) {
            const int bex = A.dbx + 1, bey = A.dby + 1, ne = bex * bey * (A.dbz + 1);
            const int r = (lk * bey + lj) * bex + li;
            for (int q = 0; q < 3; ++q) {
                if (w[q] == 0.f) continue;
                const int e = q * ne + r;
                const float En = A.dtape[(long long)slot * 3 * ne + e], En1 = A.dtape[(long long)(slot + 1) * 3 * ne + e];
                A.geps[e] += (double)w[q] / I->dt * ((double)En - (double)En1);
            }
        }
    }
}

// lambda_H += C_E w  (w = cb lambda_E' of a step of parity par, zero beyond
// the far walls) at every face except the magnetic ones: the next reverse
// step's magnet kernel adds C_E w to those as it reads them (adj_fix_kernel
// after the last), so this sweep can run beside it
__global__ void __launch_bounds__(256) adj_curl_e_kernel(LaunchSet L, AdjSet A, int par)
{
    const Inst *I = L.insts;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= I->nx || j >= I->ny || k >= I->nz) return;
    const long long fs = I->fstride, plane = I->plane;
    const int px = I->px;
    const long long o = (long long)k * plane + (long long)j * px + i;
    const float *wx_ = A.lamEn[par], *wy_ = wx_ + fs, *wz_ = wx_ + 2 * fs;
    const bool xi = i + 1 < I->nx, yj = j + 1 < I->ny, zk = k + 1 < I->nz;
    const float wx = wx_[o], wy = wy_[o], wz = wz_[o];
    const float cx = curl2a(yj ? wz_[o + px] : 0.f, wz, I->idy, zk ? wy_[o + plane] : 0.f, wy, I->idz);
    const float cy = curl2a(zk ? wx_[o + plane] : 0.f, wx, I->idz, xi ? wz_[o + 1] : 0.f, wz, I->idx);
    const float cz = curl2a(xi ? wy_[o + 1] : 0.f, wy, I->idx, yj ? wx_[o + px] : 0.f, wx, I->idy);
    unsigned fl = 0u;   // the magnetic-face flags of cell o's class (none outside the box of those faces)
    if (L.ncomp && i >= A.mlo[0] && j >= A.mlo[1] && k >= A.mlo[2] && i <= A.mhi[0] && j <= A.mhi[1] && k <= A.mhi[2]) {
        const int c = L.cls16 ? (int)static_cast<const uint16_t *>(I->cls)[o] : (int)static_cast<const uint8_t *>(I->cls)[o];
        fl = __float_as_uint(__ldg(I->ctab + 3 * c).w);
    }
    if (!(fl & CF_MAG_HX)) A.lamH[3 * fs + o] += cx;
    if (!(fl & CF_MAG_HY)) A.lamH[4 * fs + o] += cy;
    if (!(fl & CF_MAG_HZ)) A.lamH[5 * fs + o] += cz;
}

// After adj_mag_kernel and adj_curl_h_kernel (which ran side by side, the
// sweep's curls without the magnetic faces): the magnetic faces take the
// values the magnet kernel left in the workspace (lambda_H = dq), and each
// edge beside them their part of lambda_E' = lambda_E - (dt/mu0) C_H
// lambda_H, d = -(dt/mu0) times the sum of coefficient x dq over its listed
// faces, passed on as adj_curl_h_kernel passes lambda_E': w += cb d, lambda_E
// += ca d, and on a design-box edge d J / d eps_edge += (cb d / dt) (E^n -
// E^{n+1}).
__global__ void __launch_bounds__(256) adj_face_fix_kernel(LaunchSet L, AdjSet A, int slot, int par)
{
    const Inst *I = L.insts;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < A.nmf) {
        A.lamH[A.mf_lam[q]] = A.ws[A.mf_ws[q]];
        return;
    }
    const int e = q - A.nmf;
    if (e >= A.nfe) return;
    float sum = 0.f;
    for (int c = A.fe_start[e]; c < A.fe_start[e + 1]; ++c) sum = fmaf(A.fc_coef[c], A.ws[A.fc_ws[c]], sum);
    const float d = -(2.f * I->ch) * sum;
    const int comp = A.fe_comp[e];
    const long long o = A.fe_off[e], fs = I->fstride;
    const int cl = L.cls16 ? (int)static_cast<const uint16_t *>(I->cls)[o] : (int)static_cast<const uint8_t *>(I->cls)[o];
    const float4 Ca = __ldg(I->ctab + 3 * cl), Cb = __ldg(I->ctab + 3 * cl + 1);
    const float ca = comp == 0 ? Ca.x : (comp == 1 ? Ca.y : Ca.z), cb = comp == 0 ? Cb.x : (comp == 1 ? Cb.y : Cb.z);
    const float dw = cb * d;
    A.lamEn[par][comp * fs + o] += dw;
    A.lamE[comp * fs + o] += __fmaf_rn(ca, d, d);   // ca d from the table's ca - 1
    if (A.geps && dw != 0.f) {
        const long long plane = I->plane;
        const int px = I->px;
        const int k = (int)(o / plane), j = (int)((o % plane) / px), i = (int)(o % px);
        const int li = i - A.di0, lj = j - A.dj0, lk = k - A.dk0;
        if (li >= 0 && lj >= 0 && lk >= 0 && li <= A.dbx && lj <= A.dby && lk <= A.dbz) {
            const int bex = A.dbx + 1, bey = A.dby + 1, ne = bex * bey * (A.dbz + 1);
            const int ed = comp * ne + (lk * bey + lj) * bex + li;
            const float En = A.dtape[(long long)slot * 3 * ne + ed], En1 = A.dtape[(long long)(slot + 1) * 3 * ne + ed];
            A.geps[ed] += (double)dw / I->dt * ((double)En - (double)En1);
        }
    }
}

// E at the design-box edges after the current step, from buffer buf, into slot
__global__ void adj_record_design_kernel(LaunchSet L, AdjSet A, int slot, int buf)
{
    const Inst *I = L.insts;
    const int ex = A.dbx + 1, ey = A.dby + 1, ez = A.dbz + 1, ne = ex * ey * ez;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * ne) return;
    const int comp = e / ne, r = e - comp * ne;
    const int i = A.di0 + r % ex, j = A.dj0 + (r / ex) % ey, k = A.dk0 + r / (ex * ey);
    float v = 0.f;
    if (i < I->nx && j < I->ny && k < I->nz)
        v = I->F[buf][comp][(long long)k * I->plane + (long long)j * I->px + i];
    A.dtape[(long long)slot * 3 * ne + e] = v;
}

}  // namespace

long long adj_ws_floats(int bx, int by, int bz, int R)
{
    (void)R;
    const long long V = (long long)bx * by * bz;
    return (V + 3) / 4 + 6 * mag_faces(bx, by, bz) + 18 * V;
}

long long adj_dq_index(int bx, int by, int bz, int f)
{
    const long long V = (long long)bx * by * bz;
    return (V + 3) / 4 + 5 * mag_faces(bx, by, bz) + 18 * V + f;
}

cudaError_t adj_record_design(const LaunchSet &L, const AdjSet &A, int slot, int buf, cudaStream_t s)
{
    const int ne3 = 3 * (A.dbx + 1) * (A.dby + 1) * (A.dbz + 1);
    adj_record_design_kernel<<<(ne3 + 255) / 256, 256, 0, s>>>(L, A, slot, buf);
    return cudaGetLastError();
}

// Reverse of forward step n, whose records sit in tape slot `slot`
// (magnets) and design slots slot, slot+1 (E^n, E^{n+1}).  On stream st.b,
// after everything now on s (the face fix of step n+1, a segment's
// recomputation): the magnet kernel.  On s beside it: the H-curl sweep of
// step n+1 (deferred from the previous call) and the E-curl sweep of step
// n; then, after the magnet kernel, the face fix.  The H-curl sweep of step
// n waits for the next call (or adj_finish).  The two share no data: the
// sweeps leave the magnetic faces to the magnet kernels, and w is kept per
// step parity (the magnet kernel reads step n+1's, the E-curl sweep writes
// step n's).
cudaError_t adj_reverse_step(const LaunchSet &L, const AdjSet &A, long long n, int slot, cudaStream_t s,
                             AdjStreams &st)
{
    const dim3 blk(32, 8), grid((A.nx + 31) / 32, (A.ny + 7) / 8, A.nz);
    if (L.ncomp) {
        cudaError_t e = cudaFuncSetAttribute(adj_mag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, A.fnb_bytes);
        if (e == cudaSuccess) e = cudaEventRecord(st.a_ready, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st.b, st.a_ready, 0);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(L.ncomp * A.cs);
        cfg.blockDim = dim3(kMagThreads);
        cfg.dynamicSmemBytes = A.fnb_bytes;
        cfg.stream = st.b;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = A.cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = A.cs > 1 ? 1 : 0;
        e = cudaLaunchKernelEx(&cfg, adj_mag_kernel, L, A, slot, (int)((n + 1) & 1));
        if (e == cudaSuccess) e = cudaEventRecord(st.mag_done, st.b);
        if (e != cudaSuccess) return e;
    }
    if (st.pending >= 0) adj_curl_e_kernel<<<grid, blk, 0, s>>>(L, A, (int)(st.pending & 1));
    st.pending = -1;
    if (L.cls16) adj_curl_h_kernel<uint16_t><<<grid, blk, 0, s>>>(L, A, n, slot);
    else adj_curl_h_kernel<uint8_t><<<grid, blk, 0, s>>>(L, A, n, slot);
    const int nfix = A.nmf + A.nfe;
    if (L.ncomp) {
        const cudaError_t e = cudaStreamWaitEvent(s, st.mag_done, 0);
        if (e != cudaSuccess) return e;
        if (nfix > 0) adj_face_fix_kernel<<<(nfix + 255) / 256, 256, 0, s>>>(L, A, slot, (int)(n & 1));
    }
    st.pending = n;
    return cudaGetLastError();
}

// The H-curl sweep of the last reverse step, then the magnetic faces' C_E w
// and pending correction.
cudaError_t adj_finish(const LaunchSet &L, const AdjSet &A, cudaStream_t s, AdjStreams &st)
{
    const dim3 blk(32, 8), grid((A.nx + 31) / 32, (A.ny + 7) / 8, A.nz);
    int par = 0;
    if (st.pending >= 0) {
        par = (int)(st.pending & 1);
        adj_curl_e_kernel<<<grid, blk, 0, s>>>(L, A, par);
    }
    st.pending = -1;
    if (L.ncomp) adj_fix_kernel<<<L.ncomp, 256, 0, s>>>(L, A, par);
    return cudaGetLastError();
}

}  // namespace fl
