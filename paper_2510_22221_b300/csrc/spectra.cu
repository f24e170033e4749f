// Spectral post-processing of probe time series (arxiv 2510.22221): the
// Fourier magnitude of a probe component (the E_x spectra behind the
// anti-crossing maps, section "Results"), the ESPRIT extraction of mode
// frequencies, decay rates and Q factors from a time trace, and the cavity
// frequency and coupling g of Eq. omega_pm fitted to hybrid-mode pairs.
//
// The transform runs on the GPU straight from the device probe ring (FP64).
// The mode and coupling fits are small dense linear algebra on one series or
// a handful of numbers; they run on the host in FP64.
#include "../../include/fdtd_llg.h"
#include "fdtd_llg_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

namespace fl {
int probe_ring_view(fdtd_llg_t h, int32_t probe, const double **ring, int *cap, int *nprobe, long long *first,
                    int *count, double *dt, cudaStream_t *stream);
int fail_handle(fdtd_llg_t h, int code, const std::string &msg);
}  // namespace fl

using namespace fl;

namespace {

constexpr int kDftThreads = 256, kDftChunk = 1024, kResync = 64;

// |sum_t w_t x_t exp(-2 pi i f t dt)| for f = f0 + i df, one frequency per
// thread.  Samples t = 0..N-1 are ring rows first+t (mod cap) of probe p,
// component comp; they pass through shared memory in chunks, already
// windowed.  The phasor exp(-i w t) advances by one complex multiplication and
// is recomputed from sincos every kResync samples.
__global__ void __launch_bounds__(kDftThreads) probe_dft_kernel(const double *ring, int cap, int nprobe, int p, int comp,
                                                              long long first, int N, double dt, double f0, double df,
                                                              int nf, int hann, double *out)
{
    __shared__ double xs[kDftChunk];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double w = -2.0 * kPi * (f0 + (double)i * df) * dt;
    double sw, cw;
    sincos(w, &sw, &cw);
    double re = 0.0, im = 0.0, zr = 1.0, zi = 0.0;
    for (int c0 = 0; c0 < N; c0 += kDftChunk) {
        const int m = min(kDftChunk, N - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const long long row = (first + c0 + t) % cap;
            double x = ring[(row * nprobe + p) * 9 + comp];
            if (hann && N > 1) x *= 0.5 - 0.5 * cos(2.0 * kPi * (double)(c0 + t) / (double)(N - 1));
            xs[t] = x;
        }
        __syncthreads();
        if (i < nf) {
            for (int t = 0; t < m; ++t) {
                if (((c0 + t) % kResync) == 0) sincos(w * (double)(c0 + t), &zi, &zr);
                re = fma(xs[t], zr, re);
                im = fma(xs[t], zi, im);
                const double nr = zr * cw - zi * sw;
                zi = fma(zr, sw, zi * cw);
                zr = nr;
            }
        }
    }
    if (i < nf) out[i] = sqrt(re * re + im * im);
}

using cd = std::complex<double>;

// Symmetric eigenproblem by cyclic Jacobi rotations: A (n x n, row-major) is
// overwritten; eigenvalues in d, eigenvectors in the columns of V.
void jacobi_eigen(std::vector<double> &A, int n, std::vector<double> &d, std::vector<double> &V)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    d.resize(n);
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
}

// Solve M X = B (M n x n, B n x m, row-major, complex) by Gaussian elimination
// with partial pivoting; false if M is singular.
bool solve(std::vector<cd> M, std::vector<cd> &B, int n, int m)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(M[(size_t)i * n + k]) > std::abs(M[(size_t)piv * n + k])) piv = i;
        if (std::abs(M[(size_t)piv * n + k]) == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)piv * n + j]);
            for (int j = 0; j < m; ++j) std::swap(B[(size_t)k * m + j], B[(size_t)piv * m + j]);
        }
        for (int i = k + 1; i < n; ++i) {
            const cd f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
            if (f == cd(0.0)) continue;
            for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < m; ++j) {
            cd s = B[(size_t)k * m + j];
            for (int i = k + 1; i < n; ++i) s -= M[(size_t)k * n + i] * B[(size_t)i * m + j];
            B[(size_t)k * m + j] = s / M[(size_t)k * n + k];
        }
    return true;
}

// Eigenvalues of a general n x n matrix: Householder reduction to upper
// Hessenberg form, then QR iterations with Wilkinson shifts (explicit shifted
// QR by Givens rotations on the active window, deflating from the bottom).
bool eigenvalues(std::vector<cd> H, int n, std::vector<cd> &ev)
{
    auto at = [&](int i, int j) -> cd & { return H[(size_t)i * n + j]; };
    for (int k = 0; k + 2 < n; ++k) {
        const int len = n - k - 1;
        std::vector<cd> v(len);
        double alpha = 0.0;
        for (int i = 0; i < len; ++i) {
            v[i] = at(k + 1 + i, k);
            alpha += std::norm(v[i]);
        }
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const cd ph = std::abs(v[0]) > 0.0 ? v[0] / std::abs(v[0]) : cd(1.0);
        v[0] += ph * alpha;
        double vn = 0.0;
        for (auto &q : v) vn += std::norm(q);
        vn = std::sqrt(vn);
        for (auto &q : v) q /= vn;
        for (int j = 0; j < n; ++j) {   // (I - 2 v v^H) H
            cd s = 0.0;
            for (int i = 0; i < len; ++i) s += std::conj(v[i]) * at(k + 1 + i, j);
            for (int i = 0; i < len; ++i) at(k + 1 + i, j) -= 2.0 * v[i] * s;
        }
        for (int i = 0; i < n; ++i) {   // H (I - 2 v v^H)
            cd s = 0.0;
            for (int j = 0; j < len; ++j) s += at(i, k + 1 + j) * v[j];
            for (int j = 0; j < len; ++j) at(i, k + 1 + j) -= 2.0 * s * std::conj(v[j]);
        }
    }
    ev.assign(n, cd(0.0));
    int hi = n - 1, iter = 0, total = 0;
    std::vector<cd> gc(n), gs(n);
    while (hi > 0) {
        int l = hi;
        while (l > 0 && std::abs(at(l, l - 1)) > 1e-15 * (std::abs(at(l, l)) + std::abs(at(l - 1, l - 1)))) --l;
        if (l == hi) {
            ev[hi] = at(hi, hi);
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 200 * n) return false;
        const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
        const cd tr2 = 0.5 * (a + d), disc = std::sqrt(tr2 * tr2 - (a * d - b * c));
        cd mu = std::abs(tr2 + disc - d) < std::abs(tr2 - disc - d) ? tr2 + disc : tr2 - disc;
        if (++iter % 11 == 0) mu = d + cd(std::abs(c), 0.0);   // exceptional shift
        for (int k = l; k <= hi; ++k) at(k, k) -= mu;
        for (int k = l; k < hi; ++k) {   // rows: R = G H
            const cd x = at(k, k), y = at(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            const cd cc = r > 0.0 ? x / r : cd(1.0), ss = r > 0.0 ? y / r : cd(0.0);
            gc[k] = cc;
            gs[k] = ss;
            for (int j = k; j <= hi; ++j) {
                const cd t1 = at(k, j), t2 = at(k + 1, j);
                at(k, j) = std::conj(cc) * t1 + std::conj(ss) * t2;
                at(k + 1, j) = -ss * t1 + cc * t2;
            }
        }
        for (int k = l; k < hi; ++k) {   // columns: R G^H
            const cd cc = gc[k], ss = gs[k];
            for (int i = l; i <= std::min(k + 1, hi); ++i) {
                const cd t1 = at(i, k), t2 = at(i, k + 1);
                at(i, k) = t1 * cc + t2 * ss;
                at(i, k + 1) = -t1 * std::conj(ss) + t2 * std::conj(cc);
            }
        }
        for (int k = l; k <= hi; ++k) at(k, k) += mu;
    }
    ev[0] = at(0, 0);
    return true;
}

}  // namespace

extern "C" int fdtd_llg_probe_spectrum(fdtd_llg_t h, int32_t probe, int32_t comp, double f0, double f1, int32_t nf,
                                       int32_t window, double *out)
{
    if (comp < 0 || comp > 8 || nf < 1 || !out || (window != 0 && window != 1) || !(f1 >= f0) || (nf > 1 && f1 == f0))
        return fail_handle(h, FDTD_E_INVAL, "probe_spectrum: comp 0..8, nf >= 1, window 0 or 1, f1 > f0, out not NULL");
    const double *ring = nullptr;
    int cap = 0, nprobe = 0, count = 0;
    long long first = 0;
    double dt = 0;
    cudaStream_t s = nullptr;
    int rc = probe_ring_view(h, probe, &ring, &cap, &nprobe, &first, &count, &dt, &s);
    if (rc) return rc;
    if (count < 1) return fail_handle(h, FDTD_E_STATE, "probe_spectrum: no samples yet");
    double *d_out = nullptr;
    if (cudaMalloc(&d_out, (size_t)nf * sizeof(double)) != cudaSuccess)
        return fail_handle(h, FDTD_E_OOM, "probe_spectrum: device allocation failed");
    const double df = nf > 1 ? (f1 - f0) / (nf - 1) : 0.0;
    probe_dft_kernel<<<(nf + kDftThreads - 1) / kDftThreads, kDftThreads, 0, s>>>(ring, cap, nprobe, probe, comp, first,
                                                                                 count, dt, f0, df, nf, window, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, (size_t)nf * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail_handle(h, FDTD_E_CUDA, std::string("probe_spectrum: ") + cudaGetErrorString(e));
    return FDTD_OK;
}

extern "C" int fdtd_llg_fit_modes(const double *x, int64_t n, double dt, int32_t order, int32_t pencil, int32_t decimate,
                                  double fmin, double fmax, int32_t max_modes, double *freq, double *decay, double *amp,
                                  double *q, int32_t *nfound)
{
    if (!x || !freq || !decay || !amp || !q || !nfound || !(dt > 0) || order < 1 || max_modes < 1 || decimate < 1)
        return fail_handle(nullptr, FDTD_E_INVAL,
                           "fit_modes: null pointer, dt <= 0, order < 1, decimate < 1 or max_modes < 1");
    // block means of `decimate` samples (a moving-average filter sampled
    // every `decimate` steps: the frequencies of the exponentials are kept,
    // their amplitudes and phases change), then the fit at the coarser step
    std::vector<double> xd;
    if (decimate > 1) {
        xd.resize((size_t)(n / decimate));
        for (size_t b = 0; b < xd.size(); ++b) {
            double s = 0.0;
            for (int t = 0; t < decimate; ++t) s += x[(int64_t)b * decimate + t];
            xd[b] = s / decimate;
        }
        x = xd.data();
        n = (int64_t)xd.size();
        dt *= decimate;
    }
    const int L = pencil > 0 ? pencil : (int)std::min<int64_t>(n / 3, 200);
    if (L < order || n - L < order || L > 4096)
        return fail_handle(nullptr, FDTD_E_INVAL, "fit_modes: need order <= pencil <= n - order and pencil <= 4096");
    const int P = L + 1;
    const int64_t M = n - L;
    // Gram matrix R = Y^T Y of the Hankel matrix Y[m][j] = x[m + j]:
    // first row directly, then R[i+1][j+1] = R[i][j] + x[M+i] x[M+j] - x[i] x[j]
    std::vector<double> R((size_t)P * P);
    for (int j = 0; j < P; ++j) {
        double s = 0.0;
        for (int64_t m = 0; m < M; ++m) s += x[m] * x[m + j];
        R[j] = s;
    }
    for (int i = 0; i + 1 < P; ++i)
        for (int j = i; j + 1 < P; ++j)
            R[(size_t)(i + 1) * P + j + 1] = R[(size_t)i * P + j] + x[M + i] * x[M + j] - x[i] * x[j];
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < i; ++j) R[(size_t)i * P + j] = R[(size_t)j * P + i];
    std::vector<double> d, V;
    jacobi_eigen(R, P, d, V);
    std::vector<int> idx(P);
    for (int i = 0; i < P; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] > d[b]; });
    // signal subspace Vs (P x order); Phi solves Vs[0:L] Phi = Vs[1:P] in least squares
    const int r = order;
    std::vector<cd> G((size_t)r * r, cd(0.0)), B((size_t)r * r, cd(0.0));
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            double g = 0.0, h2 = 0.0;
            for (int t = 0; t < L; ++t) {
                const double va = V[(size_t)t * P + idx[a]];
                g += va * V[(size_t)t * P + idx[b]];
                h2 += va * V[(size_t)(t + 1) * P + idx[b]];
            }
            G[(size_t)a * r + b] = g;
            B[(size_t)a * r + b] = h2;
        }
    if (!solve(G, B, r, r)) return fail_handle(nullptr, FDTD_E_INVAL, "fit_modes: singular signal subspace");
    std::vector<cd> z;
    if (!eigenvalues(B, r, z)) return fail_handle(nullptr, FDTD_E_INVAL, "fit_modes: eigenvalue iteration did not converge");
    // amplitudes: least squares x_t ~ sum_k c_k z_k^t (normal equations)
    std::vector<cd> A((size_t)r * r, cd(0.0)), c((size_t)r, cd(0.0)), zt(r, cd(1.0));
    for (int64_t t = 0; t < n; ++t) {
        for (int a = 0; a < r; ++a) {
            const cd za = std::conj(zt[a]);
            c[a] += za * x[t];
            for (int b = 0; b < r; ++b) A[(size_t)a * r + b] += za * zt[b];
        }
        for (int a = 0; a < r; ++a) zt[a] *= z[a];
    }
    if (!solve(A, c, r, 1)) return fail_handle(nullptr, FDTD_E_INVAL, "fit_modes: coincident modes");
    struct Mode { double f, a, amp, q; };
    std::vector<Mode> modes;
    for (int k = 0; k < r; ++k) {
        const double f = std::arg(z[k]) / (2.0 * kPi * dt);
        if (!(f > 0.0) || f < fmin || f > fmax) continue;
        const double a = -std::log(std::abs(z[k])) / dt;
        modes.push_back({f, a, 2.0 * std::abs(c[k]), a != 0.0 ? kPi * f / a : INFINITY});
    }
    std::sort(modes.begin(), modes.end(), [](const Mode &u, const Mode &v) { return u.amp > v.amp; });
    if ((int)modes.size() > max_modes) modes.resize(max_modes);
    std::sort(modes.begin(), modes.end(), [](const Mode &u, const Mode &v) { return u.f < v.f; });
    for (size_t k = 0; k < modes.size(); ++k) {
        freq[k] = modes[k].f;
        decay[k] = modes[k].a;
        amp[k] = modes[k].amp;
        q[k] = modes[k].q;
    }
    *nfound = (int32_t)modes.size();
    return FDTD_OK;
}

extern "C" int fdtd_llg_fit_coupling(const double *f_plus, const double *f_minus, int32_t n, double *f_p, double *g)
{
    if (!f_plus || !f_minus || !f_p || !g || n < 2)
        return fail_handle(nullptr, FDTD_E_INVAL, "fit_coupling: null pointer or fewer than two pairs");
    // D^2 - S^2 = A + B S with S = f+ + f-, D = f+ - f-; centred least squares
    double Sm = 0.0, ym = 0.0;
    std::vector<double> S(n), y(n);
    for (int i = 0; i < n; ++i) {
        S[i] = f_plus[i] + f_minus[i];
        const double D = f_plus[i] - f_minus[i];
        y[i] = D * D - S[i] * S[i];
        Sm += S[i];
        ym += y[i];
    }
    Sm /= n;
    ym /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
        sxx += (S[i] - Sm) * (S[i] - Sm);
        sxy += (S[i] - Sm) * (y[i] - ym);
    }
    if (!(sxx > 0.0)) return fail_handle(nullptr, FDTD_E_INVAL, "fit_coupling: all pairs have the same f+ + f-");
    const double Bc = sxy / sxx, Ac = ym - Bc * Sm;
    const double fc = -Bc / 4.0;
    *f_p = fc;
    *g = std::sqrt(std::max(Ac / 4.0 - fc * fc, 0.0));
    return FDTD_OK;
}
