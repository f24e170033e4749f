// Per-cell edge classes on the device (see class_assign.h): the device lists
// the distinct neighbourhoods (with their first cells) and the magnetic
// cells, the host forms the neighbourhoods' classes, the device gives every
// cell its class, so the host reads and writes nothing per cell.
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

struct MagMask {
    uint64_t w[4];
};
struct DBox {
    int x0, y0, z0, bx, by, bz, on;
};

__device__ __forceinline__ bool in_dbox(const DBox &b, int i, int j, int k)
{
    return i >= b.x0 && i < b.x0 + b.bx && j >= b.y0 && j < b.y0 + b.by && k >= b.z0 && k < b.z0 + b.bz;
}

// Do the edges or faces of cell (i, j, k) touch a design cell?  (The cell
// itself or one of the six cells below it along one or two axes.)
__device__ __forceinline__ bool touches_design(const DBox &b, int i, int j, int k)
{
    if (!b.on || i < b.x0 || j < b.y0 || k < b.z0 || i > b.x0 + b.bx || j > b.y0 + b.by || k > b.z0 + b.bz)
        return false;
    const int nb[7][3] = {{i, j, k}, {i - 1, j, k}, {i, j - 1, k}, {i, j, k - 1},
                          {i, j - 1, k - 1}, {i - 1, j, k - 1}, {i - 1, j - 1, k}};
    for (const auto &q : nb)
        if (q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && in_dbox(b, q[0], q[1], q[2])) return true;
    return false;
}

// One thread per cell (grid-stride).  A cell enters its key into the set
// unless the cell before it along x (outside the design box's reach too)
// has the same key, so the first cell of every key enters it; the slot's
// first cell is the minimum over the entries.  Probing is linear and
// bounded by the table size.
__global__ void key_scan_kernel(const uint8_t *mid, int nx, int ny, int nz, MagMask mag, DBox db, KeyScan K)
{
    const long long n = (long long)nx * ny * nz;
    const unsigned mask = K.cap - 1;
    const int lane = threadIdx.x & 31;
    unsigned top = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const long long r = c / nx;
        const int j = (int)(r % ny), k = (int)(r / ny);
        const unsigned m0 = mid[c];
        top = max(top, m0);
        // the magnetic cells, one counter update per warp
        const bool ismag = (mag.w[m0 >> 6] >> (m0 & 63)) & 1ull;
        const unsigned act = __activemask();
        const unsigned bal = __ballot_sync(act, ismag);
        if (bal) {
            const int lead = __ffs(bal) - 1;
            unsigned long long base = 0;
            if (lane == lead) base = atomicAdd(K.mcount, (unsigned long long)__popc(bal));
            base = __shfl_sync(act, base, lead);
            if (ismag) {
                const unsigned long long idx = base + (unsigned long long)__popc(bal & ((1u << lane) - 1u));
                if (idx < K.mcap) K.mlist[idx] = (unsigned long long)c;
            }
        }
        if (touches_design(db, i, j, k)) continue;
        const uint64_t key = nbhd_key(mid, nx, ny, i, j, k);
        if (i > 0 && !touches_design(db, i - 1, j, k) && nbhd_key(mid, nx, ny, i - 1, j, k) == key) continue;
        unsigned slot = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & mask;
        bool done = false;
        for (unsigned p = 0; p < K.cap && !done; ++p) {
            const unsigned long long prev = atomicCAS(&K.tk[slot], kKeyEmpty, (unsigned long long)key);
            if (prev == kKeyEmpty || prev == key) {
                atomicMin(&K.first[slot], (unsigned long long)c);
                done = true;
            } else {
                slot = (slot + 1) & mask;
            }
        }
        if (!done) atomicOr(K.overflow, 1u);
    }
    top = __reduce_max_sync(0xffffffffu, top);
    if (lane == 0) atomicMax(K.top, top);
}

__global__ void key_compact_kernel(KeyScan K)
{
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < K.cap; q += gridDim.x * blockDim.x) {
        const unsigned long long key = K.tk[q];
        if (key == kKeyEmpty) continue;
        const unsigned idx = atomicAdd(K.kcount, 1u);
        K.kout[idx] = key;
        K.fout[idx] = K.first[q];
    }
}

}  // namespace

cudaError_t launch_key_scan(const uint8_t *mid, int nx, int ny, int nz, const uint64_t mag[4], bool has_design,
                            const int db[6], const KeyScan &K, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(K.tk, 0xFF, (size_t)K.cap * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(K.first, 0xFF, (size_t)K.cap * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(K.mcount, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(K.top, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(K.overflow, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(K.kcount, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    MagMask mm;
    for (int q = 0; q < 4; ++q) mm.w[q] = mag[q];
    DBox b{db[0], db[1], db[2], db[3], db[4], db[5], has_design ? 1 : 0};
    const long long n = (long long)nx * ny * nz;
    const int grid = (int)((n + 255) / 256 < 148 * 16 ? (n + 255) / 256 : 148 * 16);
    if (n > 0) key_scan_kernel<<<grid, 256, 0, s>>>(mid, nx, ny, nz, mm, b, K);
    return cudaGetLastError();
}

cudaError_t launch_key_compact(const KeyScan &K, cudaStream_t s)
{
    const int grid = (int)((K.cap + 255) / 256 < 148 * 4 ? (K.cap + 255) / 256 : 148 * 4);
    key_compact_kernel<<<grid, 256, 0, s>>>(K);
    return cudaGetLastError();
}

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
