// fdtd_llg_e_push_noalloc: the E push of a uniform medium on caller-owned
// device arrays, for callers that must not allocate device memory.
//
// The per-block energy partials, which the handle-based E pass keeps in
// memory it allocates, live here in a file-scope __device__ array of fixed
// size that every GPU loading the library holds until the process exits.
#include "../../include/fdtd_llg.h"
#include "fdtd_llg_internal.h"

#include <cmath>
#include <cstdio>
#include <mutex>

using namespace fl;

namespace {

constexpr int kNoAllocMaxBlocks = 65536;   // 512 KB of FP64 partials
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// One block per 32 x 8 x kKC tile: E = ca E + cb curl H on every stored edge
// that is not in a wall, written E + ((ca - 1) E + cb curl H) from cam1 =
// ca - 1 (exact to FP32's relative precision where ca itself would be
// rounded next to 1), and the block's sum of E^2 of the new field.
__global__ void __launch_bounds__(kTX *kTY) noalloc_e_push_kernel(float *__restrict__ Ex, float *__restrict__ Ey,
                                                                  float *__restrict__ Ez, const float *__restrict__ Hx,
                                                                  const float *__restrict__ Hy, const float *__restrict__ Hz,
                                                                  int nx, int ny, int nz, float idx, float idy, float idz,
                                                                  float cam1, float cb, double *__restrict__ part)
{
    __shared__ double sred[kTX * kTY / 32];
    const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
    const int b = blockIdx.x;
    const int tx = b % ntx, ty = (b / ntx) % nty, tz = b / (ntx * nty);
    const int i = tx * kTX + threadIdx.x, j = ty * kTY + threadIdx.y;
    const long long plane = (long long)nx * ny;
    double acc = 0.0;   // E^2 of this thread's edges, summed in FP64
    if (i < nx && j < ny) {
        const int k0 = tz * kKC, k1 = min(k0 + kKC, nz);
        long long o = (long long)k0 * plane + (long long)j * nx + i;
        float hx_km = (k0 > 0) ? __ldg(Hx + o - plane) : 0.f;
        float hy_km = (k0 > 0) ? __ldg(Hy + o - plane) : 0.f;
        for (int k = k0; k < k1; ++k, o += plane) {
            const float hx = __ldg(Hx + o), hy = __ldg(Hy + o), hz = __ldg(Hz + o);
            const float hz_jm = (j > 0) ? __ldg(Hz + o - nx) : 0.f;
            const float hx_jm = (j > 0) ? __ldg(Hx + o - nx) : 0.f;
            const float hz_im = (i > 0) ? __ldg(Hz + o - 1) : 0.f;
            const float hy_im = (i > 0) ? __ldg(Hy + o - 1) : 0.f;
            const float cx = (hz - hz_jm) * idy - (hy - hy_km) * idz;
            const float cy = (hx - hx_km) * idz - (hz - hz_im) * idx;
            const float cz = (hy - hy_im) * idx - (hx - hx_jm) * idy;
            // edges lying in a wall stay at zero
            const float ex = (j > 0 && k > 0) ? Ex[o] + (cam1 * Ex[o] + cb * cx) : 0.f;
            const float ey = (i > 0 && k > 0) ? Ey[o] + (cam1 * Ey[o] + cb * cy) : 0.f;
            const float ez = (i > 0 && j > 0) ? Ez[o] + (cam1 * Ez[o] + cb * cz) : 0.f;
            Ex[o] = ex;
            Ey[o] = ey;
            Ez[o] = ez;
            acc += (double)ex * ex + (double)ey * ey + (double)ez * ez;
            hx_km = hx;
            hy_km = hy;
        }
    }
    double v = acc;
    const int tid = threadIdx.x + kTX * threadIdx.y;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
    if ((tid & 31) == 0) sred[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < kTX * kTY / 32; ++w) s += sred[w];
        part[b] = s;   // every slot the reduction reads is written by this launch
    }
}

// Fixed-order sum of the partials: W_e = (eps/2) dV sum E^2.
__global__ void __launch_bounds__(256) noalloc_energy_kernel(const double *__restrict__ part, int nb, double scale,
                                                             double *__restrict__ out)
{
    __shared__ double sred[8];
    double s = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) s += part[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sred[w];
        *out = t * scale;
    }
}

int noalloc_fail(int code, const char *msg)
{
    set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int fdtd_llg_e_push_noalloc(float *Ex, float *Ey, float *Ez, const float *Hx, const float *Hy, const float *Hz,
                                       int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz, double dt,
                                       double eps_r, double sigma, double *w_e, void *stream)
{
    if (!Ex || !Ey || !Ez || !Hx || !Hy || !Hz) return noalloc_fail(FDTD_E_INVAL, "null field pointer");
    if (nx < 1 || ny < 1 || nz < 1) return noalloc_fail(FDTD_E_INVAL, "nx, ny, nz must be >= 1");
    if (!(dx > 0 && dy > 0 && dz > 0 && dt > 0) || !(eps_r > 0) || sigma < 0)
        return noalloc_fail(FDTD_E_INVAL, "dx, dy, dz, dt and eps_r must be > 0 and sigma >= 0");
    if (dt * kC0 * std::sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)) > 1.0 + 1e-12)
        return noalloc_fail(FDTD_E_UNSTABLE, "dt exceeds the 3-D Courant limit");
    const long long nb = (((long long)nx + kTX - 1) / kTX) * (((long long)ny + kTY - 1) / kTY) *
                         (((long long)nz + kKC - 1) / kKC);
    if (nb <= 0 || nb > kNoAllocMaxBlocks) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "grid needs %lld blocks of 32x8x16 cells; fdtd_llg_e_push_noalloc is limited to %d "
                      "(its partial sums live in a fixed device array)", nb, kNoAllocMaxBlocks);
        return noalloc_fail(FDTD_E_INVAL, msg);
    }
    // an error left pending by earlier work on this thread is not this
    // call's: report it and leave it pending rather than clear it below
    if (cudaPeekAtLastError() != cudaSuccess)
        return noalloc_fail(FDTD_E_CUDA, "a CUDA error was already pending before fdtd_llg_e_push_noalloc");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return noalloc_fail(FDTD_E_CUDA, "no usable current CUDA device");
    double *scratch;
    {
        // once per device, with that device current: the device address of
        // the partials array (its host-side name is only a stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) return noalloc_fail(FDTD_E_CUDA, "cudaGetSymbolAddress of the partials failed");
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    const double eps = kEps0 * eps_r;
    const double den = eps / dt + sigma / 2;
    const float cb = (float)(1.0 / den);
    const float cam1 = (float)(-sigma / den);   // ca - 1
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_e_push_kernel<<<(unsigned)nb, dim3(kTX, kTY), 0, s>>>(Ex, Ey, Ez, Hx, Hy, Hz, nx, ny, nz, (float)(1.0 / dx),
                                                                 (float)(1.0 / dy), (float)(1.0 / dz), cam1, cb, scratch);
    if (cudaGetLastError() != cudaSuccess) return noalloc_fail(FDTD_E_CUDA, "E push kernel launch failed");
    if (w_e) {
        noalloc_energy_kernel<<<1, 256, 0, s>>>(scratch, (int)nb, 0.5 * eps * dx * dy * dz, w_e);
        if (cudaGetLastError() != cudaSuccess) return noalloc_fail(FDTD_E_CUDA, "energy kernel launch failed");
    }
    return FDTD_OK;
}
