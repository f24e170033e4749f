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

// What the host needs of a grid's material ids before it forms the classes
// (device memory, filled by launch_key_scan):
//  * the distinct neighbourhood keys of the cells outside the design box's
//    reach, each with its first cell (the lowest linear index that has it),
//    in an open-addressing hash set of cap slots (cap a power of two, at
//    most 2^24; empty slots hold kKeyEmpty, first cells start at ~0);
//  * the magnetic cells (material ids flagged in mag), in no fixed order:
//    their number in *mcount, the first mcap of them in mlist;
//  * the largest material id in *top;
//  * *overflow != 0 if a key found no free slot.
struct KeyScan {
    unsigned long long *tk, *first;   // [cap] keys and first cells
    unsigned cap;
    unsigned long long *mlist;        // [mcap] magnetic cells
    unsigned long long mcap;
    unsigned long long *mcount;
    unsigned *top, *overflow;
    unsigned long long *kout, *fout;  // [cap] the occupied slots, compacted by launch_key_compact
    unsigned *kcount;
};
constexpr unsigned long long kKeyEmpty = ~0ull;   // keys are below 2^59

// mag: bit m set when material m is magnetic.  has_design with box db =
// (x0, y0, z0, bx, by, bz): a cell whose edges or faces touch a design cell
// is left out of the key set (its class depends on eps_r_design).  Resets
// the set and the counters first; asynchronous on stream s.
cudaError_t launch_key_scan(const uint8_t *mid, int nx, int ny, int nz, const uint64_t mag[4], bool has_design,
                            const int db[6], const KeyScan &K, cudaStream_t s);
// The occupied slots of the key set into kout / fout (in slot order, which
// depends on the insertion order: the host sorts them), their number in
// *kcount; asynchronous on stream s.
cudaError_t launch_key_compact(const KeyScan &K, cudaStream_t s);

}  // namespace fl
