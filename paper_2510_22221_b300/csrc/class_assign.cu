// Per-cell edge classes on the device (see class_assign.h): the host finds
// the distinct neighbourhoods and their classes, the device gives every cell
// its class, so the host writes nothing per cell.
#include "class_assign.h"

namespace fl {

namespace {

template <typename T>
__global__ void class_assign_kernel(const uint8_t *mid, int nx, int ny, int nz, int px, const uint64_t *keys,
                                    const uint16_t *ids, int nkeys, T *cls)
{
    const long long n = (long long)nz * ny * px;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % px);
        const long long r = q / px;
        const int j = (int)(r % ny), k = (int)(r / ny);
        T c = 0;
        if (i < nx) {
            const uint64_t key = nbhd_key(mid, nx, ny, i, j, k);
            int lo = 0, hi = nkeys;   // first index with keys[idx] >= key
            while (lo < hi) {
                const int mid_ = (lo + hi) >> 1;
                if (keys[mid_] < key) lo = mid_ + 1;
                else hi = mid_;
            }
            if (lo < nkeys && keys[lo] == key) c = (T)ids[lo];
        }
        cls[q] = c;
    }
}

template <typename T>
__global__ void class_override_kernel(const long long *off, const uint16_t *id, int n, T *cls)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) cls[off[q]] = (T)id[q];
}

}  // namespace

cudaError_t launch_class_assign(const uint8_t *mid, int nx, int ny, int nz, int px, const uint64_t *keys,
                                const uint16_t *ids, int nkeys, const long long *over_off, const uint16_t *over_id,
                                int nover, void *cls, bool c16, cudaStream_t s)
{
    const long long n = (long long)nz * ny * px;
    const int grid = (int)((n + 255) / 256 < 148 * 16 ? (n + 255) / 256 : 148 * 16);
    if (n > 0) {
        if (c16) class_assign_kernel<uint16_t><<<grid, 256, 0, s>>>(mid, nx, ny, nz, px, keys, ids, nkeys, (uint16_t *)cls);
        else class_assign_kernel<uint8_t><<<grid, 256, 0, s>>>(mid, nx, ny, nz, px, keys, ids, nkeys, (uint8_t *)cls);
    }
    if (nover > 0) {
        const int g2 = (nover + 255) / 256 < 148 * 4 ? (nover + 255) / 256 : 148 * 4;
        if (c16) class_override_kernel<uint16_t><<<g2, 256, 0, s>>>(over_off, over_id, nover, (uint16_t *)cls);
        else class_override_kernel<uint8_t><<<g2, 256, 0, s>>>(over_off, over_id, nover, (uint8_t *)cls);
    }
    return cudaGetLastError();
}

}  // namespace fl
