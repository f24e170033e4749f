/*
 * yee_llg_oracle.c -- plain FP64 CPU oracle of the coupled Maxwell + LLG
 * time step (arxiv 2510.22221, section "Numerical Model").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * What it computes, in the order the paper states it:
 *   Ampere's law (Eq. "Ampere") discretised on a staggered Yee grid,
 *   Faraday's law with B = mu0 (H + M) (Eq. "Faraday", Eq. "iterate_H"),
 *   the trapezoidal LLG solve (Eqs. "llg_tra4"-"llg_tra6"), normalised to
 *   |M| = Ms and iterated until the domain-wide maximum of
 *   |M^{r} - M^{r-1}| / Ms falls below the tolerance.
 *
 * Readings of points the paper leaves open:
 *   R1  Yee layout, cell (i,j,k) spans [i,i+1]x[j,j+1]x[k,k+1] cells:
 *       Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) on edges,
 *       Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k) on faces,
 *       M at cell centres of magnetic cells.
 *   R2  Each step is H/M half-push (curl E^n), full E push (curl H^{n+1/2},
 *       J at t=(n+1/2)dt), H/M half-push (curl E^{n+1}).  The factor
 *       dt/(2 mu0) of Eq. iterate_H and mu0|gamma|dt/4 of Eqs. llg_tra5-6
 *       are the half-push over h = dt/2.
 *   R3  H_eff at a cell centre = mean of the two face values of each
 *       component + H_bias; a face subtracts half the change of M of each of
 *       its (up to two) adjacent cells (the transpose of that mean).
 *   R4  Edge eps_r and sigma = mean over the four cells sharing the edge; an
 *       edge touching a PEC cell, and every edge lying in a domain wall, has
 *       E = 0.
 *   R5  Iteration starts from M^{n+1,0} = M^n; residual = Euclidean norm of
 *       M^{r}-M^{r-1} divided by Ms, maximum over every magnetic cell; the
 *       test is applied from r = 2 on (it compares two iterates).  At r = 1
 *       it would compare the first iterate with the starting guess M^n, i.e.
 *       measure the change of M itself, which is below tol*Ms whenever the
 *       precession is small; stopping there keeps only the explicit part of
 *       the M-H coupling, and the coupled scheme then gains energy without
 *       bound (an FDTD cavity with a magnet grew 10^4-fold in 3000 steps).
 *   R6  Source J(t) = J0 exp(-(t-tpk)^2/(2 Tp^2)) cos(2 pi f0 t) on one edge.
 *   R7  Energy W = sum_edges eps E^2/2 dV + sum_faces mu0 H^2/2 dV
 *                + sum_cells mu0 (|H0| Ms - H0.M) dV, the last term evaluated
 *       as mu0 |H0|/(2 Ms) |M - Ms h|^2 (equal on |M| = Ms).
 *   R15 Absorbing layers (the paper's device is bounded by PMLs whose
 *       formulation it does not give): the convolutional PML of Roden and
 *       Gedney (2000) with the complex-frequency-shifted stretch
 *       s = kappa + sigma / (alpha + j w eps0) on each axis.  Every
 *       derivative d/da of the two curls becomes (1/kappa_a) d/da plus a
 *       memory psi with psi <- b psi + c d/da, b = exp(-(sigma/kappa + alpha)
 *       dt/eps0), c = sigma (b - 1) / (kappa (sigma + kappa alpha)).  The
 *       layers fill the first and last pml_n[a] cells of axis a (inside the
 *       grid, ended by its PEC walls); at depth rho in [0, 1] (rho = 1 on the
 *       wall) sigma = sigma_max rho^m, kappa = 1 + (kappa_max - 1) rho^m,
 *       alpha = alpha_max (1 - rho), sigma_max = scale 0.8 (m+1)/(eta0 d_a).
 *       Time placement: the E memory is updated from H^{n+1/2} in the E push;
 *       the H memory from E^n, and its whole-step term -(dt/mu0)[(1/kappa-1)
 *       dE + psi] enters before the first half-push, so that H^{n-1/2} ->
 *       H^{n+1/2} is the standard CPML leapfrog update while H^{n+1} (probes,
 *       energy) stays the mean of the two half-step values' plain pushes.
 *
 * Threads: built with -fopenmp, the loops over z-planes (and over the
 * magnetic cells of an LLG iterate) are split across threads.  Every value
 * is computed by the same expression in the same order whatever the thread
 * count; the energy sums each z-plane separately and adds the plane sums in
 * plane order, so its bits do not depend on the thread count either.
 *
 * Array layout: C order with i fastest.  Full staggered sizes:
 *   Ex nx*(ny+1)*(nz+1)  Ey (nx+1)*ny*(nz+1)  Ez (nx+1)*(ny+1)*nz
 *   Hx (nx+1)*ny*nz      Hy nx*(ny+1)*nz      Hz nx*ny*(nz+1)
 *   M  3 blocks (x,y,z) of nx*ny*nz.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MU0 (4.0e-7 * ORC_PI)
#define ORC_C0 299792458.0
#define ORC_EPS0 (1.0 / (ORC_MU0 * ORC_C0 * ORC_C0))

typedef struct {
    int32_t nx, ny, nz, nmat;
    double dx, dy, dz, dt;
    const double *mat_eps_r, *mat_sigma, *mat_Ms, *mat_alpha, *mat_gamma;
    const int32_t *mat_pec;
    const uint8_t *mat_id;     /* nx*ny*nz                                  */
    const double *eps_r_cell;  /* NULL or nx*ny*nz: replaces mat_eps_r       */
    double hbias[3];           /* A/m                                        */
    int32_t nsrc, nprobe;
    const int32_t *src;        /* nsrc*4   : comp(0..2), i, j, k of the edge  */
    const double *src_par;     /* nsrc*4   : J0, f0, Tp, tpk                  */
    const int32_t *probe;      /* nprobe*3 : i, j, k                          */
    double llg_tol;
    int32_t llg_max_iter;
    int32_t llg_fixed_iter;    /* > 0: always exactly this many iterations   */
    /* convolutional PML (R15); pml_n[a] = 0 on every axis: none              */
    int32_t pml_n[3];          /* layers at both ends of axis x, y, z        */
    int32_t pml_pad_;
    double pml_order;          /* grading exponent m                         */
    double pml_scale;          /* sigma_max in units of 0.8 (m+1)/(eta0 d)   */
    double pml_kappa_max;      /* kappa at the outer wall (>= 1)             */
    double pml_alpha_max;      /* CFS alpha at the inner face (S/m)          */
} orc_problem;

typedef struct {
    double *Ex, *Ey, *Ez, *Hx, *Hy, *Hz, *M;
    int64_t step;
    double *psi;               /* PML memory, orc_psi_size doubles; NULL without PML */
} orc_state;

/* ---------------------------------------------------------------- indexing */
#define NX (p->nx)
#define NY (p->ny)
#define NZ (p->nz)
static inline int64_t iEx(const orc_problem *p, int i, int j, int k) { return i + (int64_t)NX * (j + (int64_t)(NY + 1) * k); }
static inline int64_t iEy(const orc_problem *p, int i, int j, int k) { return i + (int64_t)(NX + 1) * (j + (int64_t)NY * k); }
static inline int64_t iEz(const orc_problem *p, int i, int j, int k) { return i + (int64_t)(NX + 1) * (j + (int64_t)(NY + 1) * k); }
static inline int64_t iHx(const orc_problem *p, int i, int j, int k) { return i + (int64_t)(NX + 1) * (j + (int64_t)NY * k); }
static inline int64_t iHy(const orc_problem *p, int i, int j, int k) { return i + (int64_t)NX * (j + (int64_t)(NY + 1) * k); }
static inline int64_t iHz(const orc_problem *p, int i, int j, int k) { return i + (int64_t)NX * (j + (int64_t)NY * k); }
static inline int64_t iC(const orc_problem *p, int i, int j, int k) { return i + (int64_t)NX * (j + (int64_t)NY * k); }

static inline int64_t nEx(const orc_problem *p) { return (int64_t)NX * (NY + 1) * (NZ + 1); }
static inline int64_t nEy(const orc_problem *p) { return (int64_t)(NX + 1) * NY * (NZ + 1); }
static inline int64_t nEz(const orc_problem *p) { return (int64_t)(NX + 1) * (NY + 1) * NZ; }
static inline int64_t nHx(const orc_problem *p) { return (int64_t)(NX + 1) * NY * NZ; }
static inline int64_t nHy(const orc_problem *p) { return (int64_t)NX * (NY + 1) * NZ; }
static inline int64_t nHz(const orc_problem *p) { return (int64_t)NX * NY * (NZ + 1); }
static inline int64_t nC(const orc_problem *p) { return (int64_t)NX * NY * NZ; }

static inline int in_grid(const orc_problem *p, int i, int j, int k)
{
    return i >= 0 && i < NX && j >= 0 && j < NY && k >= 0 && k < NZ;
}

static double cell_eps_r(const orc_problem *p, int i, int j, int k)
{
    int64_t c = iC(p, i, j, k);
    if (p->eps_r_cell) return p->eps_r_cell[c];
    return p->mat_eps_r[p->mat_id[c]];
}
static double cell_Ms(const orc_problem *p, int64_t c) { return p->mat_Ms[p->mat_id[c]]; }

/* ------------------------------------------------- edge material, R4 */
typedef struct { double eps, sig; int frozen; } edge_coef;

/* cells sharing an edge: for comp 0 (Ex) the cells (i, j-a, k-b), a,b in {0,1};
 * comp 1 (Ey): (i-a, j, k-b); comp 2 (Ez): (i-a, j-b, k). */
static edge_coef edge_material(const orc_problem *p, int comp, int i, int j, int k)
{
    edge_coef e = {0.0, 0.0, 0};
    int wall;
    if (comp == 0) wall = (j == 0 || j == NY || k == 0 || k == NZ);
    else if (comp == 1) wall = (i == 0 || i == NX || k == 0 || k == NZ);
    else wall = (i == 0 || i == NX || j == 0 || j == NY);
    int n = 0;
    double se = 0.0, ss = 0.0;
    int pec = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int ci = i, cj = j, ck = k;
            if (comp == 0) { cj -= a; ck -= b; }
            else if (comp == 1) { ci -= a; ck -= b; }
            else { ci -= a; cj -= b; }
            if (!in_grid(p, ci, cj, ck)) continue;
            int m = p->mat_id[iC(p, ci, cj, ck)];
            se += cell_eps_r(p, ci, cj, ck);
            ss += p->mat_sigma[m];
            if (p->mat_pec[m]) pec = 1;
            ++n;
        }
    if (n > 0) { e.eps = ORC_EPS0 * se / n; e.sig = ss / n; }
    e.frozen = wall || pec;
    return e;
}

/* ------------------------------------------------------------- source, R6 */
double orc_source_value(const double *par, double t)
{
    double J0 = par[0], f0 = par[1], Tp = par[2], tpk = par[3];
    double u = t - tpk;
    return J0 * exp(-u * u / (2.0 * Tp * Tp)) * cos(2.0 * ORC_PI * f0 * t);
}

double orc_courant_dt(double dx, double dy, double dz, double cfl)
{
    return cfl / (ORC_C0 * sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
}

double orc_mu0(void) { return ORC_MU0; }

/* Threads of the parallel loops (<= 0: all available); returns the count in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n <= 0) n = omp_get_num_procs();
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}

/* A loop is split across threads only when it has at least this many
 * elements (small grids run faster on one thread). */
#define ORC_PAR_MIN 32768
double orc_eps0(void) { return ORC_EPS0; }
double orc_c0(void) { return ORC_C0; }

/* ----------------------------------------------------- curl of E on faces */
static double curlE_x(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* face (i, j+1/2, k+1/2) */
    return (s->Ez[iEz(p, i, j + 1, k)] - s->Ez[iEz(p, i, j, k)]) / p->dy
         - (s->Ey[iEy(p, i, j, k + 1)] - s->Ey[iEy(p, i, j, k)]) / p->dz;
}
static double curlE_y(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* face (i+1/2, j, k+1/2) */
    return (s->Ex[iEx(p, i, j, k + 1)] - s->Ex[iEx(p, i, j, k)]) / p->dz
         - (s->Ez[iEz(p, i + 1, j, k)] - s->Ez[iEz(p, i, j, k)]) / p->dx;
}
static double curlE_z(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* face (i+1/2, j+1/2, k) */
    return (s->Ey[iEy(p, i + 1, j, k)] - s->Ey[iEy(p, i, j, k)]) / p->dx
         - (s->Ex[iEx(p, i, j + 1, k)] - s->Ex[iEx(p, i, j, k)]) / p->dy;
}

/* ----------------------------------------------------- curl of H on edges */
static double curlH_x(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* edge (i+1/2, j, k), interior only */
    return (s->Hz[iHz(p, i, j, k)] - s->Hz[iHz(p, i, j - 1, k)]) / p->dy
         - (s->Hy[iHy(p, i, j, k)] - s->Hy[iHy(p, i, j, k - 1)]) / p->dz;
}
static double curlH_y(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* edge (i, j+1/2, k) */
    return (s->Hx[iHx(p, i, j, k)] - s->Hx[iHx(p, i, j, k - 1)]) / p->dz
         - (s->Hz[iHz(p, i, j, k)] - s->Hz[iHz(p, i - 1, j, k)]) / p->dx;
}
static double curlH_z(const orc_problem *p, const orc_state *s, int i, int j, int k)
{   /* edge (i, j, k+1/2) */
    return (s->Hy[iHy(p, i, j, k)] - s->Hy[iHy(p, i - 1, j, k)]) / p->dx
         - (s->Hx[iHx(p, i, j, k)] - s->Hx[iHx(p, i, j - 1, k)]) / p->dy;
}

/* ------------------------------------------------------------ vector ops */
static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* One evaluation of Eqs. llg_tra4-6 for a single cell followed by the
 * normalisation N(M) = Ms M/|M|:
 *   b = M^n - kappa (M^n x He^n)
 *   a = -[kappa He^{n+1} + (alpha/Ms) M^n]
 *   M~ = (b + (a.b) a - a x b) / (1 + |a|^2)       (solves M~ + a x M~ = b)
 * with kappa = mu0 |gamma| h / 2 for a substep of length h. */
void orc_llg_trapezoid(const double Mn[3], const double He_n[3], const double He_np1[3],
                       double kappa, double alpha, double Ms, double Mout[3])
{
    double MxH[3], b[3], a[3], axb[3];
    cross3(Mn, He_n, MxH);
    for (int q = 0; q < 3; ++q) b[q] = Mn[q] - kappa * MxH[q];
    for (int q = 0; q < 3; ++q) a[q] = -(kappa * He_np1[q] + (alpha / Ms) * Mn[q]);
    double ab = dot3(a, b), aa = dot3(a, a);
    cross3(a, b, axb);
    double Mt[3];
    for (int q = 0; q < 3; ++q) Mt[q] = (b[q] + ab * a[q] - axb[q]) / (1.0 + aa);
    double nrm = sqrt(dot3(Mt, Mt));
    for (int q = 0; q < 3; ++q) Mout[q] = Ms * Mt[q] / nrm;
}

/* ------------------------------------------------------------------ PML, R15 */
static int pml_on(const orc_problem *p)
{
    return p->pml_n[0] > 0 || p->pml_n[1] > 0 || p->pml_n[2] > 0;
}

/* b, c and kappa of the stretch on axis a at coordinate x (in cells, integer
 * or half-integer); outside the layers b = 1, c = 0, kappa = 1. */
static void pml_coef(const orc_problem *p, int a, double x, double *b, double *c, double *kap)
{
    const int n = a == 0 ? NX : a == 1 ? NY : NZ, d = p->pml_n[a];
    const double del = a == 0 ? p->dx : a == 1 ? p->dy : p->dz;
    double rho = 0.0;
    if (d > 0) {
        if (x < d) rho = (d - x) / d;
        else if (x > n - d) rho = (x - (n - d)) / d;
    }
    *b = 1.0; *c = 0.0; *kap = 1.0;
    if (rho <= 0.0) return;
    const double eta0 = ORC_MU0 * ORC_C0;
    const double smax = p->pml_scale * 0.8 * (p->pml_order + 1.0) / (eta0 * del);
    const double g = pow(rho, p->pml_order);
    const double sig = smax * g, k = 1.0 + (p->pml_kappa_max - 1.0) * g, al = p->pml_alpha_max * (1.0 - rho);
    *b = exp(-(sig / k + al) * p->dt / ORC_EPS0);
    *c = sig > 0.0 ? sig * (*b - 1.0) / (k * (sig + k * al)) : 0.0;
    *kap = k;
}

/* psi blocks, each the full staggered size of its component:
 * E: Ex|y Ex|z Ey|z Ey|x Ez|x Ez|y, then H: Hx|y Hx|z Hy|z Hy|x Hz|x Hz|y
 * (component | axis of the stretched derivative). */
int64_t orc_psi_size(const orc_problem *p)
{
    return 2 * (nEx(p) + nEy(p) + nEz(p) + nHx(p) + nHy(p) + nHz(p));
}
static double *psi_block(const orc_problem *p, const orc_state *s, int blk)
{
    const int64_t sz[12] = {nEx(p), nEx(p), nEy(p), nEy(p), nEz(p), nEz(p),
                            nHx(p), nHx(p), nHy(p), nHy(p), nHz(p), nHz(p)};
    double *q = s->psi;
    for (int i = 0; i < blk; ++i) q += sz[i];
    return q;
}

/* One stretched derivative term: the memory at q advanced with derivative
 * g, returning g / kappa + psi. */
static double pml_term(const orc_problem *p, int a, double x, double *q, double g)
{
    double b, c, k;
    pml_coef(p, a, x, &b, &c, &k);
    *q = b * *q + c * g;
    return g / k + *q;
}

/* The H side of R15 before the first half-push: H -= (dt/mu0) times the
 * stretched curl of E^n minus the plain one, memories advanced from E^n. */
static void pml_h_update(const orc_problem *p, orc_state *s)
{
    const double f = p->dt / ORC_MU0;
    double *qxy = psi_block(p, s, 6), *qxz = psi_block(p, s, 7), *qyz = psi_block(p, s, 8);
    double *qyx = psi_block(p, s, 9), *qzx = psi_block(p, s, 10), *qzy = psi_block(p, s, 11);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i <= NX; ++i) {   /* Hx at (i, j+1/2, k+1/2) */
                const int64_t h = iHx(p, i, j, k);
                const double dyEz = (s->Ez[iEz(p, i, j + 1, k)] - s->Ez[iEz(p, i, j, k)]) / p->dy;
                const double dzEy = (s->Ey[iEy(p, i, j, k + 1)] - s->Ey[iEy(p, i, j, k)]) / p->dz;
                const double st = pml_term(p, 1, j + 0.5, qxy + h, dyEz) - pml_term(p, 2, k + 0.5, qxz + h, dzEy);
                s->Hx[h] -= f * (st - (dyEz - dzEy));
            }
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i < NX; ++i) {   /* Hy at (i+1/2, j, k+1/2) */
                const int64_t h = iHy(p, i, j, k);
                const double dzEx = (s->Ex[iEx(p, i, j, k + 1)] - s->Ex[iEx(p, i, j, k)]) / p->dz;
                const double dxEz = (s->Ez[iEz(p, i + 1, j, k)] - s->Ez[iEz(p, i, j, k)]) / p->dx;
                const double st = pml_term(p, 2, k + 0.5, qyz + h, dzEx) - pml_term(p, 0, i + 0.5, qyx + h, dxEz);
                s->Hy[h] -= f * (st - (dzEx - dxEz));
            }
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {   /* Hz at (i+1/2, j+1/2, k) */
                const int64_t h = iHz(p, i, j, k);
                const double dxEy = (s->Ey[iEy(p, i + 1, j, k)] - s->Ey[iEy(p, i, j, k)]) / p->dx;
                const double dyEx = (s->Ex[iEx(p, i, j + 1, k)] - s->Ex[iEx(p, i, j, k)]) / p->dy;
                const double st = pml_term(p, 0, i + 0.5, qzx + h, dxEy) - pml_term(p, 1, j + 0.5, qzy + h, dyEx);
                s->Hz[h] -= f * (st - (dxEy - dyEx));
            }
}

/* Stretched curl of H at an interior edge of component comp (E side of R15). */
static double pml_curl_h(const orc_problem *p, orc_state *s, int comp, int i, int j, int k)
{
    if (comp == 0) {   /* Ex at (i+1/2, j, k) */
        const int64_t e = iEx(p, i, j, k);
        const double dyHz = (s->Hz[iHz(p, i, j, k)] - s->Hz[iHz(p, i, j - 1, k)]) / p->dy;
        const double dzHy = (s->Hy[iHy(p, i, j, k)] - s->Hy[iHy(p, i, j, k - 1)]) / p->dz;
        return pml_term(p, 1, j, psi_block(p, s, 0) + e, dyHz) - pml_term(p, 2, k, psi_block(p, s, 1) + e, dzHy);
    }
    if (comp == 1) {   /* Ey at (i, j+1/2, k) */
        const int64_t e = iEy(p, i, j, k);
        const double dzHx = (s->Hx[iHx(p, i, j, k)] - s->Hx[iHx(p, i, j, k - 1)]) / p->dz;
        const double dxHz = (s->Hz[iHz(p, i, j, k)] - s->Hz[iHz(p, i - 1, j, k)]) / p->dx;
        return pml_term(p, 2, k, psi_block(p, s, 2) + e, dzHx) - pml_term(p, 0, i, psi_block(p, s, 3) + e, dxHz);
    }
    {                  /* Ez at (i, j, k+1/2) */
        const int64_t e = iEz(p, i, j, k);
        const double dxHy = (s->Hy[iHy(p, i, j, k)] - s->Hy[iHy(p, i - 1, j, k)]) / p->dx;
        const double dyHx = (s->Hx[iHx(p, i, j, k)] - s->Hx[iHx(p, i, j - 1, k)]) / p->dy;
        return pml_term(p, 0, i, psi_block(p, s, 4) + e, dxHy) - pml_term(p, 1, j, psi_block(p, s, 5) + e, dyHx);
    }
}

/* ---------------------------------------------------------------- workspace */
typedef struct {
    double *Hsx, *Hsy, *Hsz;    /* H after the curl push (H^*)            */
    double *dM, *dMn;           /* change of M, current / next iterate    */
    double *Mst;                /* M at the start of the half-push        */
    double *b, *a0;             /* per magnetic cell                      */
    int64_t *mcell;             /* list of magnetic cells                 */
    int64_t nm;
    edge_coef *cx, *cy, *cz;    /* per-edge eps, sigma, frozen            */
} orc_ws;

static void ws_free(orc_ws *w)
{
    free(w->Hsx); free(w->Hsy); free(w->Hsz); free(w->dM); free(w->dMn); free(w->Mst);
    free(w->b); free(w->a0); free(w->mcell); free(w->cx); free(w->cy); free(w->cz);
    memset(w, 0, sizeof(*w));
}

static int ws_init(const orc_problem *p, orc_ws *w)
{
    memset(w, 0, sizeof(*w));
    int64_t nc = nC(p);
    w->Hsx = malloc(sizeof(double) * nHx(p));
    w->Hsy = malloc(sizeof(double) * nHy(p));
    w->Hsz = malloc(sizeof(double) * nHz(p));
    w->dM = calloc(3 * nc, sizeof(double));
    w->dMn = calloc(3 * nc, sizeof(double));
    w->Mst = calloc(3 * nc, sizeof(double));
    w->b = calloc(3 * nc, sizeof(double));
    w->a0 = calloc(3 * nc, sizeof(double));
    w->mcell = malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    w->cx = malloc(sizeof(edge_coef) * nEx(p));
    w->cy = malloc(sizeof(edge_coef) * nEy(p));
    w->cz = malloc(sizeof(edge_coef) * nEz(p));
    if (!w->Hsx || !w->Hsy || !w->Hsz || !w->dM || !w->dMn || !w->Mst || !w->b || !w->a0 ||
        !w->mcell || !w->cx || !w->cy || !w->cz) { ws_free(w); return -1; }
    w->nm = 0;
    for (int64_t c = 0; c < nc; ++c)
        if (cell_Ms(p, c) > 0.0) w->mcell[w->nm++] = c;
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i < NX; ++i) w->cx[iEx(p, i, j, k)] = edge_material(p, 0, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i <= NX; ++i) w->cy[iEy(p, i, j, k)] = edge_material(p, 1, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i <= NX; ++i) w->cz[iEz(p, i, j, k)] = edge_material(p, 2, i, j, k);
    return 0;
}

/* Face value of H during the iteration: H^* minus half the change of M of the
 * adjacent cells (cells outside the grid contribute nothing), R3. */
static double face_x(const orc_problem *p, const orc_ws *w, const double *dM, int i, int j, int k)
{
    int64_t nc = nC(p);
    double v = w->Hsx[iHx(p, i, j, k)];
    if (i - 1 >= 0) v -= 0.5 * dM[0 * nc + iC(p, i - 1, j, k)];
    if (i < NX) v -= 0.5 * dM[0 * nc + iC(p, i, j, k)];
    return v;
}
static double face_y(const orc_problem *p, const orc_ws *w, const double *dM, int i, int j, int k)
{
    int64_t nc = nC(p);
    double v = w->Hsy[iHy(p, i, j, k)];
    if (j - 1 >= 0) v -= 0.5 * dM[1 * nc + iC(p, i, j - 1, k)];
    if (j < NY) v -= 0.5 * dM[1 * nc + iC(p, i, j, k)];
    return v;
}
static double face_z(const orc_problem *p, const orc_ws *w, const double *dM, int i, int j, int k)
{
    int64_t nc = nC(p);
    double v = w->Hsz[iHz(p, i, j, k)];
    if (k - 1 >= 0) v -= 0.5 * dM[2 * nc + iC(p, i, j, k - 1)];
    if (k < NZ) v -= 0.5 * dM[2 * nc + iC(p, i, j, k)];
    return v;
}

static void cell_ijk(const orc_problem *p, int64_t c, int *i, int *j, int *k)
{
    *i = (int)(c % NX);
    *j = (int)((c / NX) % NY);
    *k = (int)(c / ((int64_t)NX * NY));
}

/* H/M half-push over h = dt/2 using the curl of the E currently in s.
 * Returns the number of LLG iterations taken; *noconv set when the
 * tolerance was not reached within llg_max_iter. */
static int half_push(const orc_problem *p, orc_state *s, orc_ws *w, int *noconv, double *res_out)
{
    const double h = 0.5 * p->dt;
    const double c = h / ORC_MU0;
    const int64_t nc = nC(p);

    /* H^* = H - (h/mu0) curl E  (Eq. iterate_H without the M terms) */
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i <= NX; ++i)
                w->Hsx[iHx(p, i, j, k)] = s->Hx[iHx(p, i, j, k)] - c * curlE_x(p, s, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i < NX; ++i)
                w->Hsy[iHy(p, i, j, k)] = s->Hy[iHy(p, i, j, k)] - c * curlE_y(p, s, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i)
                w->Hsz[iHz(p, i, j, k)] = s->Hz[iHz(p, i, j, k)] - c * curlE_z(p, s, i, j, k);

    int iters = 0;
    double res = 0.0;
    if (w->nm > 0) {
        /* fixed part of each cell's solve: b (Eq. llg_tra6) and the M^n term of a */
#pragma omp parallel for schedule(static) if (w->nm >= ORC_PAR_MIN / 8)
        for (int64_t q = 0; q < w->nm; ++q) {
            int64_t cc = w->mcell[q];
            int i, j, k;
            cell_ijk(p, cc, &i, &j, &k);
            int m = p->mat_id[cc];
            double Ms = p->mat_Ms[m], al = p->mat_alpha[m];
            double kap = ORC_MU0 * p->mat_gamma[m] * h / 2.0;
            double M[3] = {s->M[cc], s->M[nc + cc], s->M[2 * nc + cc]};
            double He[3] = {
                0.5 * (s->Hx[iHx(p, i, j, k)] + s->Hx[iHx(p, i + 1, j, k)]) + p->hbias[0],
                0.5 * (s->Hy[iHy(p, i, j, k)] + s->Hy[iHy(p, i, j + 1, k)]) + p->hbias[1],
                0.5 * (s->Hz[iHz(p, i, j, k)] + s->Hz[iHz(p, i, j, k + 1)]) + p->hbias[2]};
            double MxH[3];
            cross3(M, He, MxH);
            for (int d = 0; d < 3; ++d) {
                w->Mst[d * nc + cc] = M[d];
                w->b[d * nc + cc] = M[d] - kap * MxH[d];
                w->a0[d * nc + cc] = -(al / Ms) * M[d];
                w->dM[d * nc + cc] = 0.0;      /* M^{n+1,0} = M^n */
            }
        }
        for (;;) {
            ++iters;
            res = 0.0;
#pragma omp parallel for schedule(static) reduction(max : res) if (w->nm >= ORC_PAR_MIN / 8)
            for (int64_t q = 0; q < w->nm; ++q) {
                int64_t cc = w->mcell[q];
                int i, j, k;
                cell_ijk(p, cc, &i, &j, &k);
                int m = p->mat_id[cc];
                double Ms = p->mat_Ms[m];
                double kap = ORC_MU0 * p->mat_gamma[m] * h / 2.0;
                double He[3] = {
                    0.5 * (face_x(p, w, w->dM, i, j, k) + face_x(p, w, w->dM, i + 1, j, k)) + p->hbias[0],
                    0.5 * (face_y(p, w, w->dM, i, j, k) + face_y(p, w, w->dM, i, j + 1, k)) + p->hbias[1],
                    0.5 * (face_z(p, w, w->dM, i, j, k) + face_z(p, w, w->dM, i, j, k + 1)) + p->hbias[2]};
                double a[3], b[3], axb[3], Mt[3];
                for (int d = 0; d < 3; ++d) {
                    a[d] = -kap * He[d] + w->a0[d * nc + cc];
                    b[d] = w->b[d * nc + cc];
                }
                double ab = dot3(a, b), aa = dot3(a, a);
                cross3(a, b, axb);
                for (int d = 0; d < 3; ++d) Mt[d] = (b[d] + ab * a[d] - axb[d]) / (1.0 + aa);
                double nrm = sqrt(dot3(Mt, Mt));
                double diff2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double Mnew = Ms * Mt[d] / nrm;
                    double Mold = w->Mst[d * nc + cc] + w->dM[d * nc + cc];
                    diff2 += (Mnew - Mold) * (Mnew - Mold);
                    w->dMn[d * nc + cc] = Mnew - w->Mst[d * nc + cc];
                }
                double r = sqrt(diff2) / Ms;
                if (r > res) res = r;
            }
            /* Jacobi: every cell of this iterate used the previous iterate */
            for (int64_t q = 0; q < w->nm; ++q) {
                int64_t cc = w->mcell[q];
                for (int d = 0; d < 3; ++d) w->dM[d * nc + cc] = w->dMn[d * nc + cc];
            }
            if (p->llg_fixed_iter > 0) {
                if (iters >= p->llg_fixed_iter) break;
            } else {
                /* R5: the test compares two iterates, so it applies from r = 2 */
                if (iters >= 2 && res < p->llg_tol) break;
                if (iters >= p->llg_max_iter) { *noconv = 1; break; }
            }
        }
    }

    /* (H, M)^{n+1} = (H, M)^{n+1,r} */
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i <= NX; ++i) s->Hx[iHx(p, i, j, k)] = face_x(p, w, w->dM, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i < NX; ++i) s->Hy[iHy(p, i, j, k)] = face_y(p, w, w->dM, i, j, k);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) s->Hz[iHz(p, i, j, k)] = face_z(p, w, w->dM, i, j, k);
    for (int64_t q = 0; q < w->nm; ++q) {
        int64_t cc = w->mcell[q];
        for (int d = 0; d < 3; ++d) s->M[d * nc + cc] = w->Mst[d * nc + cc] + w->dM[d * nc + cc];
    }
    if (res_out) *res_out = res;
    return iters;
}

/* E^{n+1} = (sigma/2 + eps/dt)^{-1} [curl H - (sigma/2 - eps/dt) E^n - J]  */
static void e_push(const orc_problem *p, orc_state *s, const orc_ws *w, double t_half)
{
    const double dt = p->dt;
    const int pml = pml_on(p) && s->psi;
    /* new values into the workspace first would be needed only if the update
       read E neighbours; it reads only H, so in-place is exact. */
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i < NX; ++i) {
                int64_t e = iEx(p, i, j, k);
                edge_coef cf = w->cx[e];
                if (cf.frozen) { s->Ex[e] = 0.0; continue; }
                double curl = pml ? pml_curl_h(p, s, 0, i, j, k) : curlH_x(p, s, i, j, k);
                double J = 0.0;
                for (int q = 0; q < p->nsrc; ++q)
                    if (p->src[4 * q] == 0 && p->src[4 * q + 1] == i && p->src[4 * q + 2] == j && p->src[4 * q + 3] == k)
                        J += orc_source_value(p->src_par + 4 * q, t_half);
                s->Ex[e] = (curl - (cf.sig / 2 - cf.eps / dt) * s->Ex[e] - J) / (cf.sig / 2 + cf.eps / dt);
            }
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k <= NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i <= NX; ++i) {
                int64_t e = iEy(p, i, j, k);
                edge_coef cf = w->cy[e];
                if (cf.frozen) { s->Ey[e] = 0.0; continue; }
                double curl = pml ? pml_curl_h(p, s, 1, i, j, k) : curlH_y(p, s, i, j, k);
                double J = 0.0;
                for (int q = 0; q < p->nsrc; ++q)
                    if (p->src[4 * q] == 1 && p->src[4 * q + 1] == i && p->src[4 * q + 2] == j && p->src[4 * q + 3] == k)
                        J += orc_source_value(p->src_par + 4 * q, t_half);
                s->Ey[e] = (curl - (cf.sig / 2 - cf.eps / dt) * s->Ey[e] - J) / (cf.sig / 2 + cf.eps / dt);
            }
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j <= NY; ++j)
            for (int i = 0; i <= NX; ++i) {
                int64_t e = iEz(p, i, j, k);
                edge_coef cf = w->cz[e];
                if (cf.frozen) { s->Ez[e] = 0.0; continue; }
                double curl = pml ? pml_curl_h(p, s, 2, i, j, k) : curlH_z(p, s, i, j, k);
                double J = 0.0;
                for (int q = 0; q < p->nsrc; ++q)
                    if (p->src[4 * q] == 2 && p->src[4 * q + 1] == i && p->src[4 * q + 2] == j && p->src[4 * q + 3] == k)
                        J += orc_source_value(p->src_par + 4 * q, t_half);
                s->Ez[e] = (curl - (cf.sig / 2 - cf.eps / dt) * s->Ez[e] - J) / (cf.sig / 2 + cf.eps / dt);
            }
}

/* ------------------------------------------------------------ energy, R7 */
/* Sum of w[e] v[e]^2 over nplanes z-planes of psize entries each: every
 * plane summed on its own (entries in order), then the plane sums in order,
 * so that the result does not depend on the thread count. */
static double plane_sum_sq(const double *v, const edge_coef *cf, double wconst, int64_t nplanes, int64_t psize,
                           double *part)
{
#pragma omp parallel for schedule(static) if (nplanes * psize >= ORC_PAR_MIN)
    for (int64_t k = 0; k < nplanes; ++k) {
        double s = 0.0;
        for (int64_t e = k * psize; e < (k + 1) * psize; ++e) s += 0.5 * (cf ? cf[e].eps : wconst) * v[e] * v[e];
        part[k] = s;
    }
    double t = 0.0;
    for (int64_t k = 0; k < nplanes; ++k) t += part[k];
    return t;
}

static double energy_ws(const orc_problem *p, const orc_state *s, const orc_ws *w)
{
    double *part = malloc(sizeof(double) * (NZ + 1));
    if (!part) return NAN;
    /* staggered sizes are (planes in z) x (entries per plane) */
    double We = plane_sum_sq(s->Ex, w->cx, 0.0, NZ + 1, (int64_t)NX * (NY + 1), part)
              + plane_sum_sq(s->Ey, w->cy, 0.0, NZ + 1, (int64_t)(NX + 1) * NY, part)
              + plane_sum_sq(s->Ez, w->cz, 0.0, NZ, (int64_t)(NX + 1) * (NY + 1), part);
    double Wh = plane_sum_sq(s->Hx, NULL, ORC_MU0, NZ, (int64_t)(NX + 1) * NY, part)
              + plane_sum_sq(s->Hy, NULL, ORC_MU0, NZ, (int64_t)NX * (NY + 1), part)
              + plane_sum_sq(s->Hz, NULL, ORC_MU0, NZ + 1, (int64_t)NX * NY, part);
    free(part);
    double Wz = 0.0;
    /* mu0 (|H0| Ms - H0.M) equals mu0 |H0| / (2 Ms) |M - Ms h|^2 when |M| = Ms
     * (h = H0/|H0|); the second form is evaluated because the first cancels
     * to rounding noise (and can turn negative) for small precession angles. */
    const int64_t nc = nC(p);
    const double h0 = sqrt(dot3(p->hbias, p->hbias));
    if (h0 > 0.0)
        for (int64_t q = 0; q < w->nm; ++q) {
            int64_t cc = w->mcell[q];
            double Ms = cell_Ms(p, cc);
            double d2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                double dv = s->M[d * nc + cc] - Ms * p->hbias[d] / h0;
                d2 += dv * dv;
            }
            Wz += ORC_MU0 * h0 / (2.0 * Ms) * d2;
        }
    return (We + Wh + Wz) * p->dx * p->dy * p->dz;
}

double orc_energy(const orc_problem *p, const orc_state *s)
{
    orc_ws w;
    if (ws_init(p, &w)) return NAN;
    double W = energy_ws(p, s, &w);
    ws_free(&w);
    return W;
}

/* Divergence of B/mu0 = H + M_face at every cell centre, where M_face is the
 * mean of the magnetisation of the cells adjacent to a face (R3). */
void orc_div_b(const orc_problem *p, const orc_state *s, double *out)
{
    const int64_t nc = nC(p);
#pragma omp parallel for schedule(static) if (nC(p) >= ORC_PAR_MIN)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                double bx[2], by[2], bz[2];
                for (int t = 0; t < 2; ++t) {
                    int fi = i + t, fj = j + t, fk = k + t;
                    double mx = 0, my = 0, mz = 0;
                    if (fi - 1 >= 0 && fi - 1 < NX) mx += 0.5 * s->M[iC(p, fi - 1, j, k)];
                    if (fi < NX) mx += 0.5 * s->M[iC(p, fi, j, k)];
                    if (fj - 1 >= 0 && fj - 1 < NY) my += 0.5 * s->M[nc + iC(p, i, fj - 1, k)];
                    if (fj < NY) my += 0.5 * s->M[nc + iC(p, i, fj, k)];
                    if (fk - 1 >= 0 && fk - 1 < NZ) mz += 0.5 * s->M[2 * nc + iC(p, i, j, fk - 1)];
                    if (fk < NZ) mz += 0.5 * s->M[2 * nc + iC(p, i, j, fk)];
                    bx[t] = s->Hx[iHx(p, fi, j, k)] + mx;
                    by[t] = s->Hy[iHy(p, i, fj, k)] + my;
                    bz[t] = s->Hz[iHz(p, i, j, fk)] + mz;
                }
                out[iC(p, i, j, k)] = (bx[1] - bx[0]) / p->dx + (by[1] - by[0]) / p->dy + (bz[1] - bz[0]) / p->dz;
            }
}

/* --------------------------------------------------------------- driver */
static void record_probes(const orc_problem *p, const orc_state *s, double *row)
{
    const int64_t nc = nC(p);
    for (int q = 0; q < p->nprobe; ++q) {
        int i = p->probe[3 * q], j = p->probe[3 * q + 1], k = p->probe[3 * q + 2];
        double *r = row + 9 * q;
        int64_t cc = iC(p, i, j, k);
        r[0] = s->Ex[iEx(p, i, j, k)];
        r[1] = s->Ey[iEy(p, i, j, k)];
        r[2] = s->Ez[iEz(p, i, j, k)];
        r[3] = s->Hx[iHx(p, i, j, k)];
        r[4] = s->Hy[iHy(p, i, j, k)];
        r[5] = s->Hz[iHz(p, i, j, k)];
        r[6] = s->M[cc];
        r[7] = s->M[nc + cc];
        r[8] = s->M[2 * nc + cc];
    }
}

/* Advance nsteps full steps.  Outputs (each may be NULL):
 *   probe_out  nsteps*nprobe*9: E,H,M at every probe after each step
 *   energy_out nsteps: W after each step
 *   iters_out  nsteps*2: LLG iterations of the two half-pushes
 * Returns 0, or 1 when an LLG solve hit llg_max_iter, -1 on allocation
 * failure, -2 when PML layers are set but s->psi is NULL. */
int orc_run(const orc_problem *p, orc_state *s, int64_t nsteps,
            double *probe_out, double *energy_out, int32_t *iters_out)
{
    if (pml_on(p) && !s->psi) return -2;
    orc_ws w;
    if (ws_init(p, &w)) return -1;
    int noconv = 0;
    for (int64_t n = 0; n < nsteps; ++n) {
        double t_half = ((double)s->step + 0.5) * p->dt;
        if (pml_on(p) && s->psi) pml_h_update(p, s);
        int it1 = half_push(p, s, &w, &noconv, NULL);
        e_push(p, s, &w, t_half);
        int it2 = half_push(p, s, &w, &noconv, NULL);
        s->step += 1;
        if (probe_out) record_probes(p, s, probe_out + n * p->nprobe * 9);
        if (energy_out) energy_out[n] = energy_ws(p, s, &w);
        if (iters_out) { iters_out[2 * n] = it1; iters_out[2 * n + 1] = it2; }
    }
    ws_free(&w);
    return noconv ? 1 : 0;
}

/* One H/M half-push alone (curl of the present E), e.g. to move H, M from
 * integer time n to n+1/2 for comparison with a solver that stores H
 * half a step ahead.  Returns the iteration count, or -1. */
int orc_half_push(const orc_problem *p, orc_state *s)
{
    orc_ws w;
    if (ws_init(p, &w)) return -1;
    int noconv = 0;
    int it = half_push(p, s, &w, &noconv, NULL);
    ws_free(&w);
    return it;
}
