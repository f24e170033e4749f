// Device-side assignment of the per-cell edge classes (class_assign.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fl {

// The 59-bit neighbourhood key of cell (i, j, k) that fixes its class outside
// a design box: the material ids of the cell and of the six cells that share
// its three edges and three faces (below in x, y, z and the three diagonal
// pairs), 0xFF for a cell beyond the low walls, then three bits for the cell
// lying on the x, y, z = 0 walls.  mid: nx x ny x nz, x fastest.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint64_t nbhd_key(const uint8_t *mid, int nx, int ny, int i, int j, int k)
{
    const long long sj = nx, sk = (long long)nx * ny, c = k * sk + j * sj + i;
    const uint64_t m0 = mid[c];
    const uint64_t mi = i > 0 ? mid[c - 1] : 0xFFu;
    const uint64_t mj = j > 0 ? mid[c - sj] : 0xFFu;
    const uint64_t mk = k > 0 ? mid[c - sk] : 0xFFu;
    const uint64_t mjk = j > 0 && k > 0 ? mid[c - sj - sk] : 0xFFu;
    const uint64_t mik = i > 0 && k > 0 ? mid[c - 1 - sk] : 0xFFu;
    const uint64_t mij = i > 0 && j > 0 ? mid[c - 1 - sj] : 0xFFu;
    const uint64_t key = (m0 << 48) | (mi << 40) | (mj << 32) | (mk << 24) | (mjk << 16) | (mik << 8) | mij;
    return (key << 3) | (uint64_t)((i == 0) | ((j == 0) << 1) | ((k == 0) << 2));
}

// Class ids of every cell of an nx x ny x nz grid into cls (padded rows of
// px, 1 or 2 bytes per id; cells beyond nx get class 0): the cell's
// neighbourhood key looked up in keys[0..nkeys) (ascending) with class ids
// ids[]; a key that is not listed (a cell whose class the caller sets itself)
// gets class 0.  Then cls[over_off[q]] = over_id[q] for q < nover.  All
// pointers are device memory; asynchronous on stream s.
cudaError_t launch_class_assign(const uint8_t *mid, int nx, int ny, int nz, int px, const uint64_t *keys,
                                const uint16_t *ids, int nkeys, const long long *over_off, const uint16_t *over_id,
                                int nover, void *cls, bool c16, cudaStream_t s);

}  // namespace fl
