// Internal structures shared by the host runtime and the sm_103a kernels of
// the Yee-Maxwell + LLG solver.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fl {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;       // vacuum permeability (H/m)
constexpr double kC0 = 299792458.0;         // speed of light (m/s)
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);

constexpr int kMaxSrc = 4;
constexpr int kMaxProbe = 32;
constexpr int kMaxMagMat = 16;

// Tile of the start-up H half-push kernel: 32 (x, one warp) x 8 (y) columns,
// each thread marching kKC planes in z.
constexpr int kTX = 32, kTY = 8, kKC = 16;

// Fused step kernel: persistent CTAs of kST threads take column tasks of
// SX x SY cells x a range of z-planes (from the host's schedule) and march
// them in z.  Each z-plane arrives by TMA in one stage of a kNS-deep
// shared-memory ring: H on the tile extended by one cell on the low x/y sides
// (box HBX x HBY, x starting 4 cells low so that the copy stays 16-byte
// aligned), E^n and the class ids on the tile extended by one cell on the high
// x/y sides.  E^{n+1} overwrites E^n in place.  A stage stays live for two
// planes (as plane k and then as plane k-1), so kNS - 2 planes are in flight
// while one is computed.  Two tile shapes, 64 x 8 and 32 x 16 (each lane owns
// a cell pair), chosen per handle: the narrow one wastes fewer lanes on grids
// whose x extent is just above a multiple of 64.  Their boxes hold the same
// number of values, so both share one stage layout.
constexpr int kSX = 64, kSY = 8, kSZ = 16, kST = 256, kNS = 4;
constexpr int kSW = kST / 32;   // warps of a sweep CTA (one energy partial each per task)
constexpr int kEChunks = 8;         // most chunks of one instance's energy sum
constexpr int kEChunkSlots = 1024;  // most sweep partials in a chunk, unless an instance needs more than kEChunks

// Chunks of the energy sum of an instance with fntask sweep tasks.
__host__ __device__ inline int energy_chunks(int fntask)
{
    const int c = (fntask * kSW + kEChunkSlots - 1) / kEChunkSlots;
    return c < 1 ? 1 : (c > kEChunks ? kEChunks : c);
}
template <int SX>
struct Tile {
    static constexpr int LPR = SX / 2;                 // lanes per tile row (one cell pair each)
    static constexpr int Y = kST / LPR;                // rows: 8 (SX 64) or 16 (SX 32)
    static constexpr int HBX = SX + 8, HBY = Y + 2, HC = HBX * HBY;   // H box, one component
    static constexpr int EBX = SX + 4, EBY = Y + 1, EC = EBX * EBY;   // E box, one component
    static constexpr int CBX8 = SX + 16, CBX16 = SX + 8;              // class box width (u8 / u16)
};
static_assert(Tile<32>::HC == Tile<64>::HC && Tile<32>::EC == Tile<64>::EC, "one stage layout for both shapes");
constexpr int kHBX = Tile<kSX>::HBX, kHBY = Tile<kSX>::HBY, kHC = Tile<kSX>::HC;
constexpr int kEBX = Tile<kSX>::EBX, kEBY = Tile<kSX>::EBY, kEC = Tile<kSX>::EC;
constexpr int kStageH = 3 * kHC * 4;                               // 8640 B
constexpr int kStageE = 3 * kEC * 4;                               // 7344 B
constexpr int kStageHOff = 0;
constexpr int kStageEOff = (kStageH + 127) / 128 * 128;
constexpr int kStageCOff = kStageEOff + (kStageE + 127) / 128 * 128;
constexpr int kClsMaxBytes = Tile<32>::CBX16 * Tile<32>::EBY * 2 > Tile<64>::CBX16 * Tile<64>::EBY * 2
                                 ? Tile<32>::CBX16 * Tile<32>::EBY * 2
                                 : Tile<64>::CBX16 * Tile<64>::EBY * 2;
constexpr int kStageBytes = kStageCOff + (kClsMaxBytes + 127) / 128 * 128;
// Class tables of at most kTabMax entries are staged in shared memory.
constexpr int kTabMax = 64;

// Magnet kernel: each face-connected magnetic region is split along its
// longest axis into cs slabs (1 <= cs <= kMagClusterMax, one per CTA of a
// thread-block cluster, the same cs for every region of a launch); a slab's
// box holds at most kMagMaxV cells, kMagCPT cells per thread, and its cells,
// faces and edges fit one CTA's shared memory (mag_cta_smem).
constexpr int kMagThreads = 512;
constexpr int kMagMaxV = 4096;
constexpr int kMagCPT = kMagMaxV / kMagThreads;
constexpr int kMagSmemMax = 226 * 1024;   // 227 KB per CTA less the static shared memory
constexpr int kMagClusterMax = 8;         // portable cluster size
constexpr int kMagCtaCells = 128;         // cells per CTA the automatic split aims at
inline long long mag_faces(int bx, int by, int bz)
{
    return (long long)(bx + 1) * by * bz + (long long)bx * (by + 1) * bz + (long long)bx * by * (bz + 1);
}
inline long long mag_edges(int bx, int by, int bz) { return 3LL * (bx + 1) * (by + 1) * (bz + 1); }
// One step of a region's adjoint tape (floats): m and face H at the step's
// start (3V, faces), E^{n+1} at the box edges, the R Jacobi iterates of both
// half-pushes (M^r - M^n, global axes, 2 R x 3V, half-push major), then face
// H and m after the first half-push (faces, 3V).
inline long long mag_tape_floats(int bx, int by, int bz, int R)
{
    const long long V = (long long)bx * by * bz;
    return 3 * V + mag_faces(bx, by, bz) + mag_edges(bx, by, bz) + 6LL * R * V + mag_faces(bx, by, bz) + 3 * V;
}
// m (3 V floats), face H (one float per face), the box-edge E (3 per edge;
// the change of M, 3 V floats, reuses it later), then one area that first
// holds the stage of a block of qx x py x ps edge sites (H on the block grown
// by one cell on its low x, y and z sides, 3 components, and the class id of
// each site as u16) and then (dt/2mu0) curl E (one float per face), the
// material byte of each cell
inline long long mag_stage_floats(int bx, int by, int bz, int qx, int py, int ps)
{
    const long long stage = 3LL * (qx + 1) * (py + 1) * (ps + 1) + ((long long)qx * py * ps + 1) / 2;
    const long long nf = mag_faces(bx, by, bz);
    return stage > nf ? stage : nf;
}
inline long long mag_smem_bytes(int bx, int by, int bz, int qx, int py, int ps)
{
    const long long V = (long long)bx * by * bz;
    const long long e = mag_edges(bx, by, bz);
    return 4 * (3 * V + mag_faces(bx, by, bz) + (e > 3 * V ? e : 3 * V) + mag_stage_floats(bx, by, bz, qx, py, ps)) + V;
}
// Dynamic shared memory of a magnet CTA whose slab box is bx x by x bz, in a
// launch whose exchange area holds xs floats per layer (0 without a cluster):
// the exports [2 parities][2 layers][xs], the slab's arrays, and the halo
// material bytes of the layers below and above the slab (hxs each, when split).
inline long long mag_cta_smem(int bx, int by, int bz, int qx, int py, int ps, int xs, int hxs)
{
    return 16LL * xs + mag_smem_bytes(bx, by, bz, qx, py, ps) + 2LL * hxs;
}
// Block of the staged box (the box has (bx+1)(by+1)(bz+1) edge sites): whole
// x rows and y columns with as many z planes as fit, else one plane and as
// many rows as fit, else one row and as many sites as fit; false when not
// even one site fits (the slab is too large for one CTA).  xs, hxs: as in
// mag_cta_smem.
inline bool mag_stage_block(int bx, int by, int bz, int &qx, int &py, int &ps, int xs = 0, int hxs = 0)
{
    qx = bx + 1;
    py = by + 1;
    for (ps = bz + 1; ps >= 1; --ps)
        if (mag_cta_smem(bx, by, bz, qx, py, ps, xs, hxs) <= kMagSmemMax) return true;
    ps = 1;
    for (py = by; py >= 1; --py)
        if (mag_cta_smem(bx, by, bz, qx, py, ps, xs, hxs) <= kMagSmemMax) return true;
    py = 1;
    for (qx = bx; qx >= 1; --qx)
        if (mag_cta_smem(bx, by, bz, qx, py, ps, xs, hxs) <= kMagSmemMax) return true;
    return false;
}
// The split axis of a region's box (its longest; z, then y, on ties), and the
// box of the largest of its cs slabs.
inline int mag_split_axis(int bx, int by, int bz) { return (bz >= by && bz >= bx) ? 2 : (by >= bx ? 1 : 0); }
inline void mag_slab_box(int bx, int by, int bz, int cs, int &sx, int &sy, int &sz)
{
    const int a = mag_split_axis(bx, by, bz);
    sx = bx; sy = by; sz = bz;
    int &e = a == 0 ? sx : (a == 1 ? sy : sz);
    e = (e + cs - 1) / cs;
}
inline int mag_cross_section(int bx, int by, int bz)
{
    const int a = mag_split_axis(bx, by, bz);
    return a == 0 ? by * bz : (a == 1 ? bx * bz : bx * by);
}

#ifdef __CUDACC__
// Division by a box dimension d by multiplication: with m = ceil(2^32 / d),
// umulhi(n, m) = floor(n / d) exactly whenever n d < 2^32 (the error term
// n (m d - 2^32) / 2^32 stays below 1).  Box indices here are below 2^16 and
// dimensions at most 4097.
struct UDiv {
    unsigned d, m;
    __device__ explicit UDiv(unsigned dd) : d(dd), m(dd > 1 ? (unsigned)(0xFFFFFFFFull / dd + 1ull) : 0u) {}
    __device__ __forceinline__ unsigned div(unsigned n) const { return d > 1 ? __umulhi(n, m) : n; }
};
struct BoxDiv {
    UDiv bx, by, bx1, by1;
    __device__ BoxDiv(int x, int y) : bx(x), by(y), bx1(x + 1), by1(y + 1) {}
};
// (li, lj, lk) of cell v of a bx x by x bz box
__device__ __forceinline__ void cell_decode(int v, const BoxDiv &D, int &li, int &lj, int &lk)
{
    const unsigned q1 = D.bx.div(v), q2 = D.by.div(q1);
    li = v - (int)(q1 * D.bx.d);
    lj = (int)(q1 - q2 * D.by.d);
    lk = (int)q2;
}

// Face f of a region's box: axis a and box-local indices; the cells on its low
// (vl) and high (vr) side, -1 outside the box.  Faces are numbered x faces
// ((bx+1) by bz), then y faces (bx (by+1) bz), then z faces (bx by (bz+1)).
__device__ __forceinline__ void face_decode(int f, const BoxDiv &D, int bx, int by, int bz, int &a, int &fi, int &fj,
                                            int &fk, int &vl, int &vr)
{
    const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz;
    vl = vr = -1;
    if (f < nfx) {
        const unsigned q1 = D.bx1.div(f), q2 = D.by.div(q1);
        a = 0; fi = f - (int)(q1 * (bx + 1)); fj = (int)(q1 - q2 * by); fk = (int)q2;
        if (fi > 0) vl = (fk * by + fj) * bx + fi - 1;
        if (fi < bx) vr = (fk * by + fj) * bx + fi;
    } else if (f < nfx + nfy) {
        const int g = f - nfx;
        const unsigned q1 = D.bx.div(g), q2 = D.by1.div(q1);
        a = 1; fi = g - (int)(q1 * bx); fj = (int)(q1 - q2 * (by + 1)); fk = (int)q2;
        if (fj > 0) vl = (fk * by + fj - 1) * bx + fi;
        if (fj < by) vr = (fk * by + fj) * bx + fi;
    } else {
        const int g = f - nfx - nfy;
        const unsigned q1 = D.bx.div(g), q2 = D.by.div(q1);
        a = 2; fi = g - (int)(q1 * bx); fj = (int)(q1 - q2 * by); fk = (int)q2;
        if (fk > 0) vl = ((fk - 1) * by + fj) * bx + fi;
        if (fk < bz) vr = (fk * by + fj) * bx + fi;
    }
}

#endif

// Class-table entry flags (bit field stored in the .w of the first float4).
enum : uint32_t { CF_MAG_HX = 1u, CF_MAG_HY = 2u, CF_MAG_HZ = 4u };

struct MagMat {
    float Ms, inv_Ms, alpha, kappa;   // kappa = mu0 |gamma| (dt/2) / 2
};

// Tensor maps of one instance (TMA descriptors, 128-byte aligned in device memory).
enum { TM_H0 = 0, TM_H1 = 1, TM_E0 = 2, TM_E1 = 3, TM_CLS = 4, TM_COUNT = 5 };

// Everything a kernel needs about one grid instance.
struct alignas(128) Inst {
    CUtensorMap tm[TM_COUNT];             // H box and E box of buffers 0/1, class box
    float *F[2][6];                       // two buffers of Ex, Ey, Ez, Hx, Hy, Hz: [nz][ny][px]
    long long fstride;                    // F[b][c] = F[b][0] + c * fstride
    float *wHx, *wHy, *wHz;               // far-wall normal H: [nz][ny], [nz][nx], [ny][nx]
    const void *cls;                      // class id per cell: uint8 or uint16
    const float4 *ctab;                   // 3 float4 per class: (ca - 1, flags) (cb) (eps/2)
    int nclass;                           // entries of ctab
    double *probe_buf;                    // [cap][nprobe][9]
    double *energy_buf;                   // [cap]
    int nx, ny, nz, px;
    long long plane;                      // ny * px
    float idx, idy, idz;                  // 1/dx, 1/dy, 1/dz
    float ch;                             // dt / (2 mu0), one half-push
    float R[9];                           // rows: bias frame axes e1, e2, e3 = h (global coords)
    float h0n;                            // |H_bias|
    double u[3];                          // h = H_bias / |H_bias| (z when zero), FP64
    double dt, dV;
    int cap;                              // probe / energy ring length (steps)
    int nsrc, nprobe;
    int src[kMaxSrc][4];                  // comp, i, j, k
    double srcp[kMaxSrc][4];              // J0, f0, Tp, tpk
    int probe[kMaxProbe][3];
    int tile_off, ntx, nty, ntz;          // half-push tiles of this instance in the tile list
    int ftile_off, fntask;              // sweep tasks: this instance's energy-partial slots [ftile_off, + fntask)
    int mag_off, nmag;                    // magnet regions of this instance
    MagMat mm[kMaxMagMat];
};

struct MagComp {
    int inst;
    int x0, y0, z0, bx, by, bz, V;
    int ax;                 // split axis of the box (mag_split_axis)
    int qx, py, ps;         // edge sites per staged block in x, y, z (mag_stage_block)
    float *m;               // deviation M - Ms h in the bias frame: 3 blocks of V
    const uint8_t *mat;     // V: magnet material index, 0xFF outside this region
    float *tape;            // adjoint recording, per step mag_tape_floats; NULL when off
    long long tstride;      // floats per step of the tape
};

// Device-resident control block of a batch.
struct StepCtl {
    long long step;         // completed steps
    unsigned int counter;   // CTAs (field and magnet kernels) that have finished this step
    int status;             // latched error bits (ST_*)
    unsigned int work;      // next field-sweep task to hand out
    long long epend;        // step whose energy partials await their sums (-1: none)
    unsigned int eflush;    // instances whose pending energy the flush has summed
};

// A caller's host ring that step results stream into by device stores
// (pinned host memory, addressed through its device mapping): per instance,
// probe rows (cap x nprobe x 9) and energies (cap); NULL: not streamed so.
struct HostRing {
    double *rows;
    double *energy;
    long long cap;
};
enum : int { ST_NOCONV = 1, ST_UNSTABLE = 2, ST_TIMEOUT = 4, ST_TAPE = 8 };

struct LaunchSet {
    const Inst *insts;
    int ninst;
    const int *tile_inst;
    int ntiles;
    const MagComp *comps;
    int ncomp;
    int vmax;               // largest slab box of the launch (cells)
    int mag_cs;             // magnet CTAs per region (cluster size)
    int mag_xs;             // floats per exported layer (largest cross-section; 0 when mag_cs = 1)
    StepCtl *ctl;
    // energy partials of one step, two sets used by step parity: part_f[t *
    // kSW + w] per sweep task t and warp w, then part_m[c * mag_cs + r] per
    // magnet CTA r of region c (part_m = part_f + nslot_f); set p starts at
    // part_f + p * part_stride
    double *part_f, *part_m;
    int nslot_f, part_stride;
    // the flush's energy chunks: nred records {instance, chunk}, chunk sums
    // esum[instance * kEChunks + chunk], chunks summed per instance ecnt
    const int2 *ered;
    int nred;
    double *esum;
    unsigned *ecnt;
    // field-sweep tasks in the order CTAs draw them: {instance, tx | ty << 16,
    // k0 | k1 << 16, energy-partial slot}
    const int4 *ftask;
    int nftiles;
    int nfblocks;                       // persistent CTAs of the field sweep
    int mag_smem;                       // dynamic shared memory of the magnet kernel (bytes)
    int src, dst;                       // field buffers read / written by a step
    int grid_h;
    bool cls16;
    float llg_tol;
    int llg_max_iter, llg_fixed_iter;
    int energy;
    bool stab;                          // every instance's class table fits kTabMax
    int sx;                             // sweep tile width: 64 (64 x 8 tiles) or 32 (32 x 16)
    int rec;                            // magnet kernel writes its tape (adjoint recomputation)
    int test_wait;                      // > 0: sweep CTA 0 also waits, this many polls, on a barrier nothing arrives on
    long long rec_n0;                   // step of tape slot 0
    int rec_slots;                      // slots of the tape
};

// Launchers (kernels_fwd.cu).  launch_half: the start-up H/M half-push that
// moves H, M from integer time to half a step ahead, in place on buffer src.
// launch_step: one full step reading buffer src and writing buffer dst on
// stream s, the magnetic regions and the field sweep side by side (the sweep
// is a programmatic dependent launch of the magnet kernel); prof, when not
// NULL, holds four events recorded around the two kernels.
cudaError_t launch_half(const LaunchSet &L, cudaStream_t s);
cudaError_t launch_step(const LaunchSet &L, cudaStream_t s, cudaEvent_t *prof);
// The energy of step n is summed during step n + 1 (by the sweep CTAs that
// draw its reduction tasks); launch_energy_flush sums the last step's after a
// run of steps, with the same arithmetic, so the values do not depend on where
// a run of steps ends.
// It also copies the call's steps [n0, n1) of probe rows and energies into
// the host rings `rings` (device array of ninst, or NULL).
cudaError_t launch_energy_flush(const LaunchSet &L, const HostRing *rings, long long n0, long long n1, cudaStream_t s);
int h_half_blocks_per_sm(bool cls16);
int step_blocks_per_sm(bool cls16, bool stab, int sx);

// ------------------------------------------------------------- adjoint
// Device pointers of one reverse sweep (adjoint.cu), single instance.
struct AdjSet {
    float *lamE;            // adjoint of E^{n+1} (3 field arrays, fstride apart), then of E^n
    float *lamEn[2];        // w = cb lambda_E' (3 arrays) of the reverse steps of each parity
    float *lamH;            // adjoint of H (3 field arrays)
    float *lamW;            // adjoint of the far-wall normal H (walls layout)
    float *ws;              // per-region workspace (ws_off[region] floats in)
    const long long *ws_off;
    double *gh0;            // per magnet CTA (region c, rank r at c * cs + r): d J / d |H_bias|
    int cs;                 // CTAs per region of adj_mag_kernel (a thread-block cluster when > 1)
    const double *seed;     // [nsteps][nprobe][3]: dJ/dE at the probe edges
    int nprobe;
    int nx, ny, nz;         // the instance's grid
    int R;                  // Jacobi iterates of every LLG solve (fixed)
    int fnb_bytes;          // dynamic shared memory of adj_mag_kernel: 8 bytes per face and 1 per cell of the largest region
    // design box (superset of the edges whose eps depends on a design cell)
    int di0, dj0, dk0, dbx, dby, dbz;   // cells; edges span (dbx+1)(dby+1)(dbz+1) per component
    float *dtape;           // [slot][3][dbz+1][dby+1][dbx+1]: E at the design-box edges after step rec_n0+slot-1
    double *geps;           // per design-box edge: d J / d eps_edge (FP64)
    // The curl sweep adj_curl_h runs beside adj_mag_kernel with the magnetic
    // faces left out of its curls; the magnet kernel puts those faces' values
    // in its workspace, which adj_face_fix_kernel then writes to the faces
    // (nmf of them: lambda_H offset, workspace index) and, times the curl's
    // coefficients, adds to the edges beside them (nfe edges: component, cell
    // offset, and the contributions fe_start[e] .. fe_start[e+1] - 1:
    // workspace index and coefficient).  Lists in a fixed order, so the sums
    // are the same bits every run.
    int nmf, nfe;
    int mlo[3], mhi[3];     // box of every magnetic face (cell indices, inclusive; empty when mlo > mhi)
    const long long *mf_lam, *mf_ws;
    const int *fe_comp, *fe_start;
    const long long *fe_off, *fc_ws;
    const float *fc_coef;
};
long long adj_ws_floats(int bx, int by, int bz, int R);
// workspace index (within the region's workspace) of the change of face f
long long adj_dq_index(int bx, int by, int bz, int f);
// stream-ordered write of the device step counter (and clear of the CTA count)
cudaError_t set_device_step(StepCtl *ctl, long long n, cudaStream_t s);
cudaError_t adj_record_design(const LaunchSet &L, const AdjSet &A, int slot, int buf, cudaStream_t s);
// The second stream of a reverse sweep: the magnet kernel of step n runs on
// b, beside the H-curl sweep of step n+1 (deferred: pending) and the E-curl
// sweep of step n on the handle's stream.
struct AdjStreams {
    cudaStream_t b;
    cudaEvent_t a_ready, mag_done;
    long long pending;      // the step whose H-curl sweep is still to launch, or -1
};
cudaError_t adj_reverse_step(const LaunchSet &L, const AdjSet &A, long long n, int slot, cudaStream_t s,
                             AdjStreams &st);
cudaError_t adj_finish(const LaunchSet &L, const AdjSet &A, cudaStream_t s, AdjStreams &st);

// fdtd_llg_last_error(NULL) message for entry points without a handle.
void set_last_error(const char *msg);

}  // namespace fl
