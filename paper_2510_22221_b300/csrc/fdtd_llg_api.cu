// Host runtime of the C ABI declared in include/fdtd_llg.h: handles, device
// memory, material preprocessing, magnetic-region discovery, launches.
#include "../../include/fdtd_llg.h"
#include "fdtd_llg_internal.h"
#include "class_assign.h"
#include "pml.h"
#include "diag.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

using namespace fl;

namespace {

thread_local std::string g_last_error;

struct Instance {
    int nx = 0, ny = 0, nz = 0, px = 0;
    double dx = 0, dy = 0, dz = 0;
    bool materials_set = false;
    // device buffers (owned through Sim's allocator)
    float *fields[2] = {nullptr, nullptr};   // two buffers of 6 arrays of nz*ny*px
    float *walls = nullptr;           // wHx, wHy, wHz
    void *cls = nullptr;
    int cls_bytes = 1;
    float4 *ctab = nullptr;
    int nclass = 0;
    double *probe_buf = nullptr;
    int probe_alloc = -1;             // probes the probe ring was sized for
    double *energy_buf = nullptr;
    // caller's host rings for streamed results (fdtd_llg_stream_results)
    // the caller's host rings: pageable ones are filled by copies queued after
    // each step call (host_*), pinned ones by the flush kernel (ring_mapped)
    double *host_rows = nullptr, *host_energy = nullptr;
    long long host_cap = 0;
    bool ring_mapped = false;
    float *mbuf = nullptr;            // all regions' deviation m (bias frame)
    uint8_t *magmat = nullptr;        // all regions' material maps
    // host descriptions
    std::vector<std::array<int, 4>> src;
    std::vector<std::array<double, 4>> srcp;
    std::vector<std::array<int, 3>> probes;
    std::vector<MagComp> comps;       // device pointers inside
    std::vector<MagMat> mm;
    std::vector<double> mm_Ms;        // Ms of each magnet material (FP64)
    double hbias[3] = {0, 0, 0};
    bool has_design = false;
    int dbox[6] = {0, 0, 0, 0, 0, 0}; // design box: i0, j0, k0, bx, by, bz
    double u[3] = {0, 0, 1};          // bias direction
    float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};   // bias frame rows (e1, e2, e3 = u)
    // absorbing layers (fdtd_llg_set_pml): layers per axis, grading
    // (order, scale, kappa_max, alpha_max), device memories and coefficients
    int pml_n[3] = {0, 0, 0};
    double pml_par[4] = {3, 1, 1, 0};
    float *psi[3] = {nullptr, nullptr, nullptr};
    float4 *pco[3] = {nullptr, nullptr, nullptr};
    long long pvol[3] = {0, 0, 0};
    bool ca_nonpos = false;           // some edge class has cb != 0 and ca = 0 (sigma = 2 eps / dt)
    bool has_pml() const { return pml_n[0] > 0 || pml_n[1] > 0 || pml_n[2] > 0; }
    size_t pml_floats() const { return 4 * (size_t)(pvol[0] + pvol[1] + pvol[2]); }
    size_t n_field() const { return (size_t)nz * ny * px; }
    size_t n_wall() const { return (size_t)ny * nz + (size_t)nx * nz + (size_t)nx * ny; }
};

struct Sim {
    std::vector<Instance> inst;
    std::vector<struct fdtd_llg_s *> members;
    double dt = 0;
    fdtd_llg_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int cur = 0;                      // field buffer holding the present state
    // device control and descriptors
    Inst *d_insts = nullptr;
    int *d_tile_inst = nullptr;
    int4 *d_ftile_inst = nullptr;      // sweep task records in claim order
    MagComp *d_comps = nullptr;
    StepCtl *d_ctl = nullptr;
    double *d_part = nullptr;         // part_e | part_h | part_m
    HostRing *d_rings = nullptr;      // per instance: the mapped host rings the flush fills
    bool rings_mapped = false;        // some instance has one
    int2 *d_ered = nullptr;           // the flush's energy chunks {instance, chunk}
    double *d_esum = nullptr;         // chunk sums, kEChunks per instance
    unsigned *d_ecnt = nullptr;       // chunks summed, per instance
    int nred = 0;
    // absorbing layers: the launch descriptor of each lined instance
    std::vector<PmlLaunch> pml;
    int ntiles = 0, nftiles = 0, ncomp = 0, vmax = 0, mag_smem = 0;
    int mag_cs = 1, mag_xs = 0;       // magnet CTAs per region (cluster size) and exported floats per layer
    int mag_cluster = 0;              // requested magnet CTAs per region (0: automatic)
    int test_wait = 0;                // fdtd_llg_test_wait_timeout: polls of the diagnostic wait (0: off)
    int mag_cs_need = 1, mag_cs_fast = 1;   // fewest magnet CTAs per region that fit; the fast split
    bool stab = false;                // every class table small enough for shared memory
    int tiling = 0;                   // requested z-planes per sweep task (0: model)
    int planes = 0;                   // z-planes per sweep task in effect
    int tile_width = 0;               // requested sweep tile width (0: fewest padded cells, 32, 64)
    int sx = 64;                      // sweep tile width in effect (Tile<sx>)
    bool cls16 = false;
    bool dirty = true;
    int nsm = 148;
    long long host_step = 0;
    bool half_ahead = false;
    // checkpointed run for the adjoint
    long long adj_N = 0;              // steps of the recorded run (0: none)
    long long adj_K = 0;              // steps between checkpoints
    float *ckpt = nullptr;            // ceil(N/K) states: fields of the present buffer, walls, m
    size_t ckpt_floats = 0;
    // adjoint tapes (run_checkpointed): slots [0, tail) hold the last `tail`
    // steps of the run (step tail0 + s), recorded as it ran; when tail < N,
    // slots [tail + 1, tail + 1 + K) take one recomputed segment
    float *tape = nullptr;            // magnet regions, region-major: slots x mag_tape_floats
    float *dtape = nullptr;           // design-box edge E: slots + 1 records
    long long tail = 0, tail0 = 0;
    long long tape_budget = -1;       // bytes recorded during the run (-1: half the free device memory)
    // CUDA graph of kGraphSteps steps (even: the buffer parity returns), replayed by long step calls
    cudaGraphExec_t graph = nullptr;
    int graph_parity = -1;            // buffer holding the state when the graph starts; -1: none
    cudaGraphExec_t graph1[2] = {nullptr, nullptr};   // one-step calls (step and flush), by starting buffer
    // graphs of r steps (0 < r < kGraphSteps) by starting buffer, built on
    // first use: the part of a call that the kGraphSteps graph does not cover
    cudaGraphExec_t graph_r[32][2] = {};
    bool graph_off = false;           // capture failed once on this stream: launch step by step
    int graph_mode = -1;              // 1 always, 0 never, -1 default (as 1)
    std::vector<void *> allocs;
    std::string err;
    // profiling: event pairs recorded around launches
    bool profiling = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
    fdtd_llg_profile prof{};

    cudaEvent_t take_event()
    {
        if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void *dalloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *p = nullptr;
        if (cfg.alloc) p = cfg.alloc(bytes, stream, cfg.alloc_user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (p) allocs.push_back(p);
        return p;
    }
    void dfree(void *p)
    {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) allocs.erase(it);
        if (cfg.free) cfg.free(p, cfg.alloc_user);
        else cudaFree(p);
    }
    ~Sim()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : ev_pool) cudaEventDestroy(e);
        for (void *p : allocs) {
            if (cfg.free) cfg.free(p, cfg.alloc_user);
            else cudaFree(p);
        }
        allocs.clear();
        if (graph) cudaGraphExecDestroy(graph);
        for (auto g1 : graph1)
            if (g1) cudaGraphExecDestroy(g1);
        for (auto &gr : graph_r)
            for (auto g : gr)
                if (g) cudaGraphExecDestroy(g);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

}  // namespace

struct fdtd_llg_s {
    Sim *sim;
    int index;          // -1: batch root
    bool owns;          // destroy frees the Sim
};

namespace {

int fail(fdtd_llg_t h, int code, const std::string &msg)
{
    g_last_error = msg;
    if (h && h->sim) h->sim->err = msg;
    return code;
}

#define CKR(h, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(h, FDTD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

double courant_limit(double dx, double dy, double dz)
{
    return 1.0 / (kC0 * std::sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
}

bool valid_cfg(const fdtd_llg_config &c, std::string &why)
{
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) { why = "nx, ny, nz must be >= 1"; return false; }
    if ((long long)c.nz * c.ny * ((c.nx + 31) / 32 * 32) >= (1LL << 32)) {
        why = "grid too large: nz * ny * (nx rounded up to 32) must be below 2^32";
        return false;
    }
    if (!(c.dx > 0 && c.dy > 0 && c.dz > 0)) { why = "dx, dy, dz must be > 0"; return false; }
    if (c.dt < 0 || (c.dt == 0 && !(c.courant_factor > 0 && c.courant_factor <= 1))) {
        why = "dt must be > 0, or dt = 0 with 0 < courant_factor <= 1";
        return false;
    }
    if (c.llg_tol < 0 || c.llg_max_iter < 0 || c.llg_fixed_iter < 0 || c.probe_capacity < 0) {
        why = "negative LLG or probe settings";
        return false;
    }
    return true;
}

Instance *inst_of(fdtd_llg_t h)
{
    if (!h || !h->sim) return nullptr;
    int i = h->index < 0 ? 0 : h->index;
    if (i >= (int)h->sim->inst.size()) return nullptr;
    return &h->sim->inst[i];
}

bool is_member(fdtd_llg_t h) { return h && h->sim && h->index >= 0; }

// Device temporaries of one call, released (after the handle's stream has
// drained) when the call returns, on every path.
struct DevTemps {
    Sim *S;
    std::vector<void *> p;
    void *get(size_t bytes)
    {
        void *q = S->dalloc(bytes);
        if (q) p.push_back(q);
        return q;
    }
    ~DevTemps()
    {
        if (p.empty()) return;
        cudaStreamSynchronize(S->stream);
        for (void *q : p) S->dfree(q);
    }
};

// ------------------------------------------------------- edge coefficients
struct ClassKey {
    uint32_t w[10];
    bool operator==(const ClassKey &o) const { return std::memcmp(w, o.w, sizeof w) == 0; }
};
struct ClassKeyHash {
    size_t operator()(const ClassKey &k) const
    {
        uint64_t h = 1469598103934665603ull;
        for (uint32_t v : k.w) { h ^= v; h *= 1099511628211ull; }
        return (size_t)h;
    }
};

uint32_t fbits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

// Orthonormal frame with third axis u (rows e1, e2, e3).
void bias_frame(const double u[3], double E[9])
{
    const double a[3] = {std::fabs(u[0]) < 0.9 ? 1.0 : 0.0, std::fabs(u[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    double e1[3] = {a[1] * u[2] - a[2] * u[1], a[2] * u[0] - a[0] * u[2], a[0] * u[1] - a[1] * u[0]};
    const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double &v : e1) v /= n1;
    const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    for (int q = 0; q < 3; ++q) { E[q] = e1[q]; E[3 + q] = e2[q]; E[6 + q] = u[q]; }
}

}  // namespace

namespace fl {
// Records a message for fdtd_llg_last_error(NULL) (used by entry points that
// have no handle).
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace fl

// ------------------------------------------------------------------ ABI
extern "C" int fdtd_llg_abi_version(void) { return FDTD_LLG_ABI_VERSION; }

extern "C" const char *fdtd_llg_last_error(fdtd_llg_t h)
{
    if (h && h->sim) return h->sim->err.c_str();
    return g_last_error.c_str();
}

static int create_impl(const fdtd_llg_config *cfgs, int32_t n, fdtd_llg_t *out)
{
    if (!cfgs || !out || n < 1) return fail(nullptr, FDTD_E_INVAL, "null argument or n < 1");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        std::string why;
        if (!valid_cfg(cfgs[i], why)) return fail(nullptr, FDTD_E_INVAL, "instance " + std::to_string(i) + ": " + why);
    }
    // common time step: explicit, or the smallest Courant step of the set
    double dt;
    if (cfgs[0].dt > 0) dt = cfgs[0].dt;
    else {
        dt = 1e300;
        for (int i = 0; i < n; ++i)
            dt = std::min(dt, cfgs[0].courant_factor * courant_limit(cfgs[i].dx, cfgs[i].dy, cfgs[i].dz));
    }
    for (int i = 0; i < n; ++i) {
        const double lim = courant_limit(cfgs[i].dx, cfgs[i].dy, cfgs[i].dz);
        if (dt > lim * (1 + 1e-12))
            return fail(nullptr, FDTD_E_UNSTABLE, "dt exceeds the 3-D Courant limit of instance " + std::to_string(i));
    }
    if (cudaSetDevice(cfgs[0].device) != cudaSuccess) return fail(nullptr, FDTD_E_CUDA, "cudaSetDevice failed");
    Sim *S = new Sim();
    S->cfg = cfgs[0];
    if (S->cfg.llg_tol == 0) S->cfg.llg_tol = 1e-6;
    if (S->cfg.llg_max_iter == 0) S->cfg.llg_max_iter = 20;
    if (S->cfg.probe_capacity == 0) S->cfg.probe_capacity = 4096;
    S->dt = dt;
    cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, cfgs[0].device);
    if (S->cfg.stream) S->stream = (cudaStream_t)S->cfg.stream;
    else {
        if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete S;
            return fail(nullptr, FDTD_E_CUDA, "cudaStreamCreate failed");
        }
        S->own_stream = true;
    }
    S->inst.resize(n);
    fdtd_llg_t root = new fdtd_llg_s{S, n == 1 ? 0 : -1, true};
    for (int i = 0; i < n; ++i) {
        Instance &I = S->inst[i];
        I.nx = cfgs[i].nx; I.ny = cfgs[i].ny; I.nz = cfgs[i].nz;
        I.px = (I.nx + 31) / 32 * 32;
        I.dx = cfgs[i].dx; I.dy = cfgs[i].dy; I.dz = cfgs[i].dz;
        I.fields[0] = (float *)S->dalloc(6 * I.n_field() * sizeof(float));
        I.fields[1] = (float *)S->dalloc(6 * I.n_field() * sizeof(float));
        I.walls = (float *)S->dalloc(I.n_wall() * sizeof(float));
        I.energy_buf = (double *)S->dalloc((size_t)S->cfg.probe_capacity * sizeof(double));
        if (!I.fields[0] || !I.fields[1] || !I.walls || !I.energy_buf) {
            fdtd_llg_destroy(root);
            return fail(nullptr, FDTD_E_OOM, "device allocation failed");
        }
        cudaMemsetAsync(I.fields[0], 0, 6 * I.n_field() * sizeof(float), S->stream);
        cudaMemsetAsync(I.fields[1], 0, 6 * I.n_field() * sizeof(float), S->stream);
        cudaMemsetAsync(I.walls, 0, I.n_wall() * sizeof(float), S->stream);
        cudaMemsetAsync(I.energy_buf, 0, (size_t)S->cfg.probe_capacity * sizeof(double), S->stream);
        S->members.push_back(n == 1 ? root : new fdtd_llg_s{S, i, false});
    }
    S->d_ctl = (StepCtl *)S->dalloc(sizeof(StepCtl));
    if (!S->d_ctl) { fdtd_llg_destroy(root); return fail(nullptr, FDTD_E_OOM, "device allocation failed"); }
    cudaMemsetAsync(S->d_ctl, 0, sizeof(StepCtl), S->stream);
    set_device_step(S->d_ctl, 0, S->stream);   // also: no energy partials pending
    if (cudaStreamSynchronize(S->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        fdtd_llg_destroy(root);
        return fail(nullptr, FDTD_E_CUDA, "initialisation failed");
    }
    *out = root;
    return FDTD_OK;
}

extern "C" int fdtd_llg_create(const fdtd_llg_config *cfg, fdtd_llg_t *out) { return create_impl(cfg, 1, out); }

extern "C" int fdtd_llg_create_batch(const fdtd_llg_config *cfgs, int32_t n, fdtd_llg_t *out)
{
    return create_impl(cfgs, n, out);
}

extern "C" int fdtd_llg_batch_member(fdtd_llg_t b, int32_t i, fdtd_llg_t *m)
{
    if (!b || !b->sim || !m) return fail(b, FDTD_E_INVAL, "null argument");
    if (i < 0 || i >= (int)b->sim->members.size()) return fail(b, FDTD_E_RANGE, "member index out of range");
    *m = b->sim->members[i];
    return FDTD_OK;
}

extern "C" void fdtd_llg_destroy(fdtd_llg_t h)
{
    if (!h) return;
    if (!h->owns) return;   // members go with their batch
    Sim *S = h->sim;
    if (S) {
        for (auto *m : S->members)
            if (m != h) delete m;
        delete S;
    }
    delete h;
}

// --------------------------------------------------------- set_materials
// The absorbing layers need every magnetic cell outside them (the magnet
// kernel owns those faces) and ca != 0 on every edge that they correct (the
// E pass folds the CPML term into E^n through cb/ca; ca < 0, a good
// conductor, is fine: the sweep multiplies the folded value by ca again).
// Whether a region's bounding box bx x by x bz can run: split along its
// longest axis into up to kMagClusterMax slabs, one per CTA of a cluster,
// its largest slab must hold at most kMagMaxV cells and fit one CTA's shared
// memory beside the exchange area of its cross-section.
static bool mag_region_fits(int bx, int by, int bz, std::string &why)
{
    const int a = mag_split_axis(bx, by, bz);
    const int ext = a == 0 ? bx : (a == 1 ? by : bz);
    const int cs = std::min(kMagClusterMax, ext);
    int sx, sy, sz, qx, py, ps;
    mag_slab_box(bx, by, bz, cs, sx, sy, sz);
    const int xs = cs > 1 ? mag_cross_section(bx, by, bz) : 0;
    const long long V = (long long)bx * by * bz, sv = (long long)sx * sy * sz;
    if (sv > kMagMaxV || !mag_stage_block(sx, sy, sz, qx, py, ps, xs, xs)) {
        why = "a magnetic region's bounding box (" + std::to_string(bx) + " x " + std::to_string(by) + " x " +
              std::to_string(bz) + " = " + std::to_string(V) + " cells) does not fit " + std::to_string(cs) +
              " magnet CTAs: each holds at most " + std::to_string(kMagMaxV) + " cells of a slab along the box's longest axis";
        return false;
    }
    return true;
}

static int pml_check(fdtd_llg_t h, const Instance &I)
{
    const int n[3] = {I.nx, I.ny, I.nz};
    for (const MagComp &C : I.comps) {
        const int lo[3] = {C.x0, C.y0, C.z0}, ext[3] = {C.bx, C.by, C.bz};
        for (int a = 0; a < 3; ++a)
            if (I.pml_n[a] > 0 && (lo[a] < I.pml_n[a] || lo[a] + ext[a] > n[a] - I.pml_n[a]))
                return fail(h, FDTD_E_INVAL, "magnetic cells inside the absorbing layers");
    }
    if (I.ca_nonpos) return fail(h, FDTD_E_INVAL, "absorbing layers need sigma != 2 eps / dt in every material (ca = 0)");
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_materials(fdtd_llg_t h, const uint8_t *mat_id, const fdtd_material *table, int32_t ntable,
                                      const double hbias[3], const double *eps_r_design, const int32_t design_box[6])
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "set_materials needs an instance handle (use fdtd_llg_batch_member)");
    if (!mat_id || !table || !hbias || ntable < 1 || ntable > 255)
        return fail(h, FDTD_E_INVAL, "null argument or ntable outside 1..255");
    Sim *S = h->sim;
    Instance &I = *inst_of(h);
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const size_t nc = (size_t)nx * ny * nz;
    // material ids on the host: the caller's array itself when it is host
    // memory, a copy when it is device memory
    std::vector<uint8_t> mid_copy;
    const uint8_t *mid = mat_id;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, mat_id) == cudaSuccess && pa.type == cudaMemoryTypeDevice) {
        mid_copy.resize(nc);
        CKR(h, cudaMemcpy(mid_copy.data(), mat_id, nc, cudaMemcpyDeviceToHost));
        mid = mid_copy.data();
    } else {
        cudaGetLastError();
    }
    for (int m = 0; m < ntable; ++m) {
        const fdtd_material &t = table[m];
        if (!(t.eps_r > 0) || t.sigma < 0 || t.Ms < 0 || t.alpha < 0 || (t.Ms > 0 && !(t.gamma > 0)))
            return fail(h, FDTD_E_INVAL, "material " + std::to_string(m) + " has an invalid parameter");
    }
    for (int q = 0; q < 3; ++q)
        if (!std::isfinite(hbias[q])) return fail(h, FDTD_E_INVAL, "hbias is not finite");
    const bool has_design = eps_r_design != nullptr;
    int db[6] = {0, 0, 0, 0, 0, 0};
    if (has_design) {
        if (!design_box) return fail(h, FDTD_E_INVAL, "eps_r_design given without design_box");
        std::memcpy(db, design_box, sizeof db);
        if (db[0] < 0 || db[1] < 0 || db[2] < 0 || db[3] < 1 || db[4] < 1 || db[5] < 1 || db[0] + db[3] > nx ||
            db[1] + db[4] > ny || db[2] + db[5] > nz)
            return fail(h, FDTD_E_INVAL, "design_box outside the grid");
        const size_t nd = (size_t)db[3] * db[4] * db[5];
        for (size_t q = 0; q < nd; ++q)
            if (!(eps_r_design[q] > 0)) return fail(h, FDTD_E_INVAL, "eps_r_design must be > 0");
    }
    auto cid = [&](int i, int j, int k) { return ((size_t)k * ny + j) * nx + i; };
    auto in_box = [&](int i, int j, int k) {
        return has_design && i >= db[0] && i < db[0] + db[3] && j >= db[1] && j < db[1] + db[4] && k >= db[2] &&
               k < db[2] + db[5];
    };
    auto eps_of = [&](int i, int j, int k) -> double {
        if (in_box(i, j, k)) return eps_r_design[((size_t)(k - db[2]) * db[4] + (j - db[1])) * db[3] + (i - db[0])];
        return table[mid[cid(i, j, k)]].eps_r;
    };
    const double dt = S->dt;
    // per-cell class: (ca - 1, cb, eps/2) of the three edges with index (i,j,k)
    // + magnetic-face flags.  ca - 1 = -sigma / den is kept instead of ca: in
    // FP32, ca = 1 - sigma dt / eps (~1 - 1e-7 for a weak conductor) would
    // be rounded to a few units of the last place below 1, changing the
    // conductive loss by up to ~10 %; ca - 1 holds it to full relative
    // precision.  Edges held at zero (walls, PEC) have ca - 1 = -1, cb = 0.
    auto edge = [&](int comp, int i, int j, int k, float &ca, float &cb, float &he) {
        bool wall;
        if (comp == 0) wall = (j == 0 || k == 0);
        else if (comp == 1) wall = (i == 0 || k == 0);
        else wall = (i == 0 || j == 0);
        ca = -1.f;
        cb = he = 0.f;
        if (wall) return;
        double se = 0, ss = 0;
        bool pec = false;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                int ci = i, cj = j, ck = k;
                if (comp == 0) { cj -= a; ck -= b; }
                else if (comp == 1) { ci -= a; ck -= b; }
                else { ci -= a; cj -= b; }
                const fdtd_material &t = table[mid[cid(ci, cj, ck)]];
                se += eps_of(ci, cj, ck);
                ss += t.sigma;
                pec = pec || t.is_pec;
            }
        if (pec) return;
        const double eps = kEps0 * se / 4, sig = ss / 4;
        const double den = eps / dt + sig / 2;
        ca = (float)(-sig / den);
        cb = (float)(1.0 / den);
        he = (float)(eps / 2);
    };
    bool magm[256] = {};
    for (int m = 0; m < ntable; ++m) magm[m] = table[m].Ms > 0;
    auto magc = [&](int i, int j, int k) { return magm[mid[cid(i, j, k)]]; };
    // the class of cell (i, j, k) from its edges' coefficients and magnetic faces
    auto class_key = [&](int i, int j, int k) {
        ClassKey key;
        float v[9];
        edge(0, i, j, k, v[0], v[3], v[6]);
        edge(1, i, j, k, v[1], v[4], v[7]);
        edge(2, i, j, k, v[2], v[5], v[8]);
        for (int q = 0; q < 9; ++q) key.w[q] = fbits(v[q]);
        uint32_t f = 0;
        if (magc(i, j, k) || (i > 0 && magc(i - 1, j, k))) f |= CF_MAG_HX;
        if (magc(i, j, k) || (j > 0 && magc(i, j - 1, k))) f |= CF_MAG_HY;
        if (magc(i, j, k) || (k > 0 && magc(i, j, k - 1))) f |= CF_MAG_HZ;
        key.w[9] = f;
        return key;
    };
    // a cell whose edges or faces touch a design cell (its class then
    // depends on eps_r_design, not only on the materials around it)
    auto touches_design = [&](int i, int j, int k) {
        if (!has_design || i < db[0] || j < db[1] || k < db[2] || i > db[0] + db[3] || j > db[1] + db[4] ||
            k > db[2] + db[5])
            return false;
        const int nb[7][3] = {{i, j, k}, {i - 1, j, k}, {i, j - 1, k}, {i, j, k - 1},
                              {i, j - 1, k - 1}, {i - 1, j, k - 1}, {i - 1, j - 1, k}};
        for (auto &q : nb)
            if (q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && in_box(q[0], q[1], q[2])) return true;
        return false;
    };
    // Classes.  Elsewhere a cell's class depends only on its neighbourhood
    // key (nbhd_key: the materials of the seven cells its edges and faces
    // touch, and the walls it lies against).  The device lists the distinct
    // keys, each with its first cell, and the magnetic cells; the keys'
    // classes, formed here in the order of their first cells, and those of
    // the cells touching the design box are the host's work, and the device
    // gives every cell its class (the host reads and writes nothing per
    // cell).  The material ids go to the device first (the caller's device
    // array itself when it is one).
    const bool on_dev = !mid_copy.empty();
    DevTemps tmpd{S};
    const uint8_t *dmid = mat_id;
    if (!on_dev) {
        uint8_t *d = (uint8_t *)tmpd.get(nc);
        if (!d) return fail(h, FDTD_E_OOM, "device allocation failed");
        CKR(h, cudaMemcpyAsync(d, mid, nc, cudaMemcpyHostToDevice, S->stream));
        dmid = d;
    }
    uint64_t magw[4] = {0, 0, 0, 0};
    for (int m = 0; m < ntable; ++m)
        if (magm[m]) magw[m >> 6] |= 1ull << (m & 63);
    // the key set starts small (a grid has few distinct neighbourhoods) and
    // grows sixteenfold whenever a scan overflows it, up to 2^20 slots; its
    // arrays and the counters share one allocation
    KeyScan K{};
    K.cap = 64;
    while (K.cap < 4096 && K.cap < 2 * nc) K.cap *= 2;
    K.mcap = std::max<unsigned long long>(1, std::min<unsigned long long>(nc, 1ull << 16));
    auto alloc_set = [&]() -> bool {
        unsigned char *p = (unsigned char *)tmpd.get((size_t)K.cap * 32 + 32);
        if (!p) return false;
        K.tk = (unsigned long long *)p;
        K.first = K.tk + K.cap;
        K.kout = K.first + K.cap;
        K.fout = K.kout + K.cap;
        unsigned char *cnt = p + (size_t)K.cap * 32;
        K.mcount = (unsigned long long *)cnt;
        K.top = (unsigned *)(cnt + 8);
        K.overflow = (unsigned *)(cnt + 12);
        K.kcount = (unsigned *)(cnt + 16);
        return true;
    };
    K.mlist = (unsigned long long *)tmpd.get((size_t)K.mcap * 8);
    if (!K.mlist || !alloc_set()) return fail(h, FDTD_E_OOM, "device allocation failed");
    struct {
        unsigned long long mcount;
        unsigned top, overflow, kcount, pad;
    } hc{};
    for (int pass = 0; pass < 8; ++pass) {
        CKR(h, launch_key_scan(dmid, nx, ny, nz, magw, has_design, db, K, S->stream));
        CKR(h, launch_key_compact(K, S->stream));
        CKR(h, cudaMemcpyAsync(&hc, K.mcount, sizeof hc, cudaMemcpyDeviceToHost, S->stream));
        CKR(h, cudaStreamSynchronize(S->stream));
        if (hc.overflow && K.cap < (1u << 20)) {   // again with a larger set
            K.cap = std::min(K.cap * 16, 1u << 20);
            if (!alloc_set()) return fail(h, FDTD_E_OOM, "device allocation failed");
            continue;
        }
        if (hc.mcount > K.mcap) {   // more magnetic cells than the list holds: again with room for all
            K.mlist = (unsigned long long *)tmpd.get((size_t)hc.mcount * 8);
            if (!K.mlist) return fail(h, FDTD_E_OOM, "device allocation failed");
            K.mcap = hc.mcount;
            continue;
        }
        break;
    }
    if (nc && hc.top >= (unsigned)ntable) return fail(h, FDTD_E_INVAL, "mat_id references a material beyond ntable");
    if (hc.mcount > K.mcap) return fail(h, FDTD_E_CUDA, "the device's list of magnetic cells overflowed");
    if (hc.overflow)
        return fail(h, FDTD_E_INVAL, "more than " + std::to_string(K.cap) + " distinct material neighbourhoods");
    std::vector<std::pair<uint64_t, uint64_t>> first_key(hc.kcount);   // (first cell, key)
    std::vector<size_t> magcells(hc.mcount);
    {
        std::vector<unsigned long long> kk(hc.kcount), ff(hc.kcount), mm(hc.mcount);
        if (hc.kcount) {
            CKR(h, cudaMemcpy(kk.data(), K.kout, hc.kcount * 8ull, cudaMemcpyDeviceToHost));
            CKR(h, cudaMemcpy(ff.data(), K.fout, hc.kcount * 8ull, cudaMemcpyDeviceToHost));
        }
        if (hc.mcount) CKR(h, cudaMemcpy(mm.data(), K.mlist, hc.mcount * 8ull, cudaMemcpyDeviceToHost));
        for (size_t q = 0; q < kk.size(); ++q) first_key[q] = {ff[q], kk[q]};
        std::sort(first_key.begin(), first_key.end());
        for (size_t q = 0; q < mm.size(); ++q) magcells[q] = (size_t)mm[q];
        std::sort(magcells.begin(), magcells.end());
    }
    std::unordered_map<ClassKey, int, ClassKeyHash> classes;
    std::vector<ClassKey> keys;
    {
        // class 0: every coefficient zero and no flags; the field kernel reads
        // it for the cells beyond the far walls, whose E^{n+1} is then zero
        ClassKey zero;
        std::memset(&zero, 0, sizeof zero);
        classes.emplace(zero, 0);
        keys.push_back(zero);
    }
    auto class_of = [&](int i, int j, int k) -> int {
        const ClassKey key = class_key(i, j, k);
        auto it = classes.find(key);
        if (it != classes.end()) return it->second;
        const int c = (int)keys.size();
        if (c >= 65536) return -1;
        classes.emplace(key, c);
        keys.push_back(key);
        return c;
    };
    const int px = I.px;
    std::unordered_map<uint64_t, int> key_class;
    for (const auto &fk : first_key) {
        const size_t c = (size_t)fk.first;
        const int cl = class_of((int)(c % nx), (int)((c / nx) % ny), (int)(c / ((size_t)nx * ny)));
        if (cl < 0) return fail(h, FDTD_E_INVAL, "more than 65536 distinct edge classes");
        key_class.emplace(fk.second, cl);
    }
    std::vector<long long> over_off;
    std::vector<uint16_t> over_id;
    if (has_design)
        for (int k = db[2]; k <= std::min(nz - 1, db[2] + db[5]); ++k)
            for (int j = db[1]; j <= std::min(ny - 1, db[1] + db[4]); ++j)
                for (int i = db[0]; i <= std::min(nx - 1, db[0] + db[3]); ++i)
                    if (touches_design(i, j, k)) {
                        const int cl = class_of(i, j, k);
                        if (cl < 0) return fail(h, FDTD_E_INVAL, "more than 65536 distinct edge classes");
                        over_off.push_back(((long long)k * ny + j) * px + i);
                        over_id.push_back((uint16_t)cl);
                    }
    std::vector<std::pair<uint64_t, uint16_t>> kc(key_class.begin(), key_class.end());
    std::sort(kc.begin(), kc.end());
    const int nclass = (int)keys.size();
    const bool c16 = nclass > 256;
    // magnetic regions: face-connected components of cells with Ms > 0,
    // numbered in the order of their first cell
    // region label per magnetic cell, by its index in the sorted list of
    // magnetic cells (every magnetic cell is in it)
    std::vector<int> label(magcells.size(), -1);
    auto mag_index = [&](size_t c) {
        return (size_t)(std::lower_bound(magcells.begin(), magcells.end(), c) - magcells.begin());
    };
    struct Box { int x0, y0, z0, x1, y1, z1; };
    std::vector<Box> boxes;
    std::vector<size_t> stack;
    for (size_t q0 = 0; q0 < magcells.size(); ++q0) {
        if (label[q0] >= 0) continue;
        const size_t c0 = magcells[q0];
        const int L = (int)boxes.size();
        Box b{nx, ny, nz, -1, -1, -1};
        stack.clear();
        stack.push_back(c0);
        label[q0] = L;
        while (!stack.empty()) {
            const size_t c = stack.back();
            stack.pop_back();
            const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((size_t)nx * ny));
            b.x0 = std::min(b.x0, i); b.y0 = std::min(b.y0, j); b.z0 = std::min(b.z0, k);
            b.x1 = std::max(b.x1, i); b.y1 = std::max(b.y1, j); b.z1 = std::max(b.z1, k);
            const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
            for (auto &q : nb) {
                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= nx || q[1] >= ny || q[2] >= nz) continue;
                const size_t cc = cid(q[0], q[1], q[2]);
                if (!magm[mid[cc]]) continue;
                const size_t qi = mag_index(cc);
                if (qi >= magcells.size() || magcells[qi] != cc)
                    return fail(h, FDTD_E_CUDA, "the device's list of magnetic cells is incomplete");
                int &lc = label[qi];
                if (lc < 0) {
                    lc = L;
                    stack.push_back(cc);
                }
            }
        }
        std::string why;
        if (!mag_region_fits(b.x1 - b.x0 + 1, b.y1 - b.y0 + 1, b.z1 - b.z0 + 1, why)) return fail(h, FDTD_E_INVAL, why);
        boxes.push_back(b);
    }
    // magnet material table (compact index per magnetic material)
    std::vector<int> mm_index(ntable, 0xFF);
    std::vector<MagMat> mm;
    std::vector<double> mm_Ms;
    const double hdt = 0.5 * dt;
    for (int m = 0; m < ntable; ++m)
        if (table[m].Ms > 0) {
            if ((int)mm.size() >= kMaxMagMat) return fail(h, FDTD_E_INVAL, "more than 16 magnetic materials");
            mm_index[m] = (int)mm.size();
            MagMat q;
            q.Ms = (float)table[m].Ms;
            q.inv_Ms = (float)(1.0 / table[m].Ms);
            q.alpha = (float)table[m].alpha;
            q.kappa = (float)(kMu0 * table[m].gamma * hdt / 2);
            mm.push_back(q);
            mm_Ms.push_back(table[m].Ms);
        }
    size_t totV = 0;
    for (auto &b : boxes) totV += (size_t)(b.x1 - b.x0 + 1) * (b.y1 - b.y0 + 1) * (b.z1 - b.z0 + 1);
    std::vector<uint8_t> hmat(totV);
    // release the previous materials of this instance
    CKR(h, cudaStreamSynchronize(S->stream));
    S->dfree(I.cls); S->dfree(I.ctab); S->dfree(I.mbuf); S->dfree(I.magmat);
    I.cls = nullptr; I.ctab = nullptr; I.mbuf = nullptr; I.magmat = nullptr;
    I.mbuf = (float *)S->dalloc(3 * totV * sizeof(float));
    I.magmat = (uint8_t *)S->dalloc(totV);
    I.cls = S->dalloc((size_t)I.nz * I.ny * I.px * (c16 ? 2 : 1));
    I.ctab = (float4 *)S->dalloc((size_t)3 * nclass * sizeof(float4));
    if (!I.mbuf || !I.magmat || !I.cls || !I.ctab) return fail(h, FDTD_E_OOM, "device allocation failed");
    I.comps.clear();
    size_t off = 0;
    for (size_t L = 0; L < boxes.size(); ++L) {
        const Box &b = boxes[L];
        MagComp C{};
        C.x0 = b.x0; C.y0 = b.y0; C.z0 = b.z0;
        C.bx = b.x1 - b.x0 + 1; C.by = b.y1 - b.y0 + 1; C.bz = b.z1 - b.z0 + 1;
        C.V = C.bx * C.by * C.bz;
        for (int lk = 0; lk < C.bz; ++lk)
            for (int lj = 0; lj < C.by; ++lj)
                for (int li = 0; li < C.bx; ++li) {
                    const int v = (lk * C.by + lj) * C.bx + li;
                    const size_t c = cid(C.x0 + li, C.y0 + lj, C.z0 + lk);
                    hmat[off + v] = magm[mid[c]] && label[mag_index(c)] == (int)L ? (uint8_t)mm_index[mid[c]] : 0xFF;
                }
        C.m = I.mbuf + 3 * off;
        C.mat = I.magmat + off;
        I.comps.push_back(C);
        off += C.V;
    }
    // bias frame: M starts at Ms h, i.e. m = 0
    const double h0n = std::sqrt(hbias[0] * hbias[0] + hbias[1] * hbias[1] + hbias[2] * hbias[2]);
    double u[3] = {0, 0, 1};
    if (h0n > 0) for (int q = 0; q < 3; ++q) u[q] = hbias[q] / h0n;
    double E[9];
    bias_frame(u, E);
    // upload: class ids in the padded layout, table, regions; zero the fields
    {
        // class ids on the device: from the material ids there, the sorted
        // keys and the overrides
        const size_t nk = kc.size(), no = over_off.size();
        const size_t o_keys = 0, o_ids = o_keys + nk * 8, o_off = (o_ids + nk * 2 + 15) / 16 * 16,
                     o_oid = o_off + no * 8, tbytes = o_oid + no * 2 + 16;
        unsigned char *tmp = (unsigned char *)S->dalloc(tbytes);
        if (!tmp) return fail(h, FDTD_E_OOM, "device allocation failed");
        std::vector<uint64_t> hk(nk);
        std::vector<uint16_t> hid(nk);
        for (size_t q = 0; q < nk; ++q) { hk[q] = kc[q].first; hid[q] = kc[q].second; }
        cudaError_t e = cudaSuccess;
        if (nk) e = cudaMemcpyAsync(tmp + o_keys, hk.data(), nk * 8, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess && nk) e = cudaMemcpyAsync(tmp + o_ids, hid.data(), nk * 2, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess && no) e = cudaMemcpyAsync(tmp + o_off, over_off.data(), no * 8, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess && no) e = cudaMemcpyAsync(tmp + o_oid, over_id.data(), no * 2, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess)
            e = launch_class_assign(dmid, nx, ny, nz, px, (const uint64_t *)(tmp + o_keys),
                                    (const uint16_t *)(tmp + o_ids), (int)nk, (const long long *)(tmp + o_off),
                                    (const uint16_t *)(tmp + o_oid), (int)no, I.cls, c16, S->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);   // the host arrays above are released next
        S->dfree(tmp);
        CKR(h, e);
        std::vector<float4> tab(3 * (size_t)nclass);
        bool ca_nonpos = false;
        for (int c = 0; c < nclass; ++c) {
            const uint32_t *w = keys[c].w;
            float v[9];
            std::memcpy(v, w, sizeof v);
            float flag;
            std::memcpy(&flag, &w[9], 4);
            tab[3 * c] = make_float4(v[0], v[1], v[2], flag);
            for (int q = 0; q < 3; ++q) ca_nonpos = ca_nonpos || (v[3 + q] != 0.f && v[q] == -1.f);   // ca = 0
            tab[3 * c + 1] = make_float4(v[3], v[4], v[5], 0.f);
            tab[3 * c + 2] = make_float4(v[6], v[7], v[8], 0.f);
        }
        CKR(h, cudaMemcpy(I.ctab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice));
        I.ca_nonpos = ca_nonpos;
        if (totV) {
            CKR(h, cudaMemset(I.mbuf, 0, 3 * totV * sizeof(float)));
            CKR(h, cudaMemcpy(I.magmat, hmat.data(), hmat.size(), cudaMemcpyHostToDevice));
        }
        CKR(h, cudaMemset(I.fields[0], 0, 6 * I.n_field() * sizeof(float)));
        CKR(h, cudaMemset(I.fields[1], 0, 6 * I.n_field() * sizeof(float)));
        CKR(h, cudaMemset(I.walls, 0, I.n_wall() * sizeof(float)));
    }
    I.cls_bytes = c16 ? 2 : 1;
    I.nclass = nclass;
    I.mm = mm;
    I.mm_Ms = mm_Ms;
    std::memcpy(I.hbias, hbias, sizeof I.hbias);
    std::memcpy(I.u, u, sizeof I.u);
    for (int q = 0; q < 9; ++q) I.R[q] = (float)E[q];
    I.materials_set = true;
    I.has_design = has_design;
    if (I.has_pml()) {
        const int rc = pml_check(h, I);
        if (rc) {
            I.materials_set = false;   // stepping refuses until materials and layers agree
            return rc;
        }
        for (int a = 0; a < 3; ++a)
            if (I.psi[a]) CKR(h, cudaMemset(I.psi[a], 0, 4 * (size_t)I.pvol[a] * sizeof(float)));
    }
    std::memcpy(I.dbox, db, sizeof db);
    // a batch's step count restarts with any instance's materials
    S->host_step = 0;
    S->half_ahead = false;
    S->cur = 0;
    S->adj_N = 0;   // a recorded run belongs to the previous materials
    S->dfree(S->tape);
    S->dfree(S->dtape);
    S->tape = S->dtape = nullptr;
    S->tail = S->tail0 = 0;
    // ordered on the handle's stream (its kernels may still run)
    CKR(h, cudaMemsetAsync(S->d_ctl, 0, sizeof(StepCtl), S->stream));
    CKR(h, set_device_step(S->d_ctl, 0, S->stream));
    CKR(h, cudaStreamSynchronize(S->stream));
    S->dirty = true;
    return FDTD_OK;
}

// {b, c, 1/kappa - 1, 0} of the CPML recursion at depth rho (0 inner face,
// 1 the wall): sigma = smax rho^m, kappa = 1 + (kmax - 1) rho^m,
// alpha = amax (1 - rho); b = exp(-(sigma/kappa + alpha) dt/eps0),
// c = sigma (b - 1) / (kappa (sigma + kappa alpha)).
static float4 pml_coefficients(double rho, double smax, const double *par, double dt)
{
    double sig = 0, kap = 1, al = par[3];
    if (rho > 0) {
        const double g = std::pow(rho, par[0]);
        sig = smax * g;
        kap = 1 + (par[2] - 1) * g;
        al = par[3] * (1 - rho);
    }
    const double b = std::exp(-(sig / kap + al) * dt / kEps0);
    const double c = sig > 0 ? sig * (b - 1) / (kap * (sig + kap * al)) : 0.0;
    return make_float4((float)b, (float)c, (float)(1 / kap - 1), 0.f);
}

extern "C" int fdtd_llg_set_pml(fdtd_llg_t h, const int32_t layers[3], double order, double scale, double kappa_max,
                                double alpha_max)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "set_pml needs an instance handle (use fdtd_llg_batch_member)");
    if (!layers) return fail(h, FDTD_E_INVAL, "null layers");
    Sim *S = h->sim;
    Instance &I = *inst_of(h);
    const int n[3] = {I.nx, I.ny, I.nz};
    for (int a = 0; a < 3; ++a)
        if (layers[a] < 0 || 2 * layers[a] > n[a]) return fail(h, FDTD_E_INVAL, "layers must be >= 0 and at most half the axis");
    if (6 * I.n_field() >= (1ull << 31))
        return fail(h, FDTD_E_INVAL, "grid too large for the layers' 32-bit offsets (6 nx' ny nz >= 2^31)");
    if (!(order >= 0) || !(scale >= 0) || !(kappa_max >= 1) || !(alpha_max >= 0))
        return fail(h, FDTD_E_INVAL, "need order >= 0, scale >= 0, kappa_max >= 1, alpha_max >= 0");
    if (S->adj_N) return fail(h, FDTD_E_STATE, "a checkpointed run is recorded; set the materials again first");
    CKR(h, cudaStreamSynchronize(S->stream));
    const int old[3] = {I.pml_n[0], I.pml_n[1], I.pml_n[2]};
    for (int a = 0; a < 3; ++a) I.pml_n[a] = layers[a];
    if (I.materials_set && I.has_pml()) {
        const int rc = pml_check(h, I);
        if (rc) {
            for (int a = 0; a < 3; ++a) I.pml_n[a] = old[a];
            return rc;
        }
    }
    const double par[4] = {order, scale, kappa_max, alpha_max};
    std::memcpy(I.pml_par, par, sizeof par);
    const double del[3] = {I.dx, I.dy, I.dz};
    for (int a = 0; a < 3; ++a) {
        S->dfree(I.psi[a]);
        S->dfree(I.pco[a]);
        I.psi[a] = nullptr;
        I.pco[a] = nullptr;
        I.pvol[a] = 0;
        const int d = layers[a];
        if (d == 0) continue;
        const long long other = (long long)n[(a + 1) % 3] * n[(a + 2) % 3];
        I.pvol[a] = 2LL * d * other;
        I.psi[a] = (float *)S->dalloc(4 * (size_t)I.pvol[a] * sizeof(float));
        I.pco[a] = (float4 *)S->dalloc((size_t)4 * d * sizeof(float4));
        if (!I.psi[a] || !I.pco[a]) return fail(h, FDTD_E_OOM, "device allocation failed");
        CKR(h, cudaMemset(I.psi[a], 0, 4 * (size_t)I.pvol[a] * sizeof(float)));
        const double smax = scale * 0.8 * (order + 1) / (kMu0 * kC0 * del[a]);
        std::vector<float4> co((size_t)4 * d);
        for (int t = 0; t < d; ++t) {
            co[2 * t] = pml_coefficients((double)(d - t) / d, smax, par, S->dt);                      // low side, E
            co[2 * t + 1] = pml_coefficients((d - t - 0.5) / d, smax, par, S->dt);                     // low side, H
            co[2 * (d + t)] = pml_coefficients((double)t / d, smax, par, S->dt);                       // high side, E
            co[2 * (d + t) + 1] = pml_coefficients((t + 0.5) / d, smax, par, S->dt);                   // high side, H
        }
        CKR(h, cudaMemcpy(I.pco[a], co.data(), co.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    S->dirty = true;
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_source(fdtd_llg_t h, int32_t comp, int32_t i, int32_t j, int32_t k, double J0, double f0,
                                   double Tp, double t_peak)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "set_source needs an instance handle");
    Instance *I = inst_of(h);
    if (comp < 0 || comp > 2) return fail(h, FDTD_E_INVAL, "comp must be 0, 1 or 2");
    if (i < 0 || j < 0 || k < 0 || i >= I->nx || j >= I->ny || k >= I->nz) return fail(h, FDTD_E_RANGE, "source edge outside the grid");
    if (!(f0 > 0) || Tp < 0 || !std::isfinite(J0)) return fail(h, FDTD_E_INVAL, "f0 must be > 0, Tp >= 0, J0 finite");
    if ((int)I->src.size() >= kMaxSrc) return fail(h, FDTD_E_INVAL, "at most 4 sources per instance");
    if (Tp == 0) Tp = 1.0 / f0;
    if (t_peak == 0) t_peak = 3.0 * Tp;
    I->src.push_back({comp, i, j, k});
    I->srcp.push_back({J0, f0, Tp, t_peak});
    h->sim->dirty = true;
    return FDTD_OK;
}

extern "C" int fdtd_llg_add_probe(fdtd_llg_t h, int32_t i, int32_t j, int32_t k, int32_t *id)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "add_probe needs an instance handle");
    Instance *I = inst_of(h);
    if (i < 0 || j < 0 || k < 0 || i >= I->nx || j >= I->ny || k >= I->nz) return fail(h, FDTD_E_RANGE, "probe cell outside the grid");
    if ((int)I->probes.size() >= kMaxProbe) return fail(h, FDTD_E_INVAL, "at most 32 probes per instance");
    if (h->sim->host_step > 0) return fail(h, FDTD_E_STATE, "add probes before the first step");
    I->probes.push_back({i, j, k});
    if (id) *id = (int32_t)I->probes.size() - 1;
    h->sim->dirty = true;
    return FDTD_OK;
}

// ----------------------------------------------------------- descriptors
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The field kernel's TMA boxes for tile width sx: per buffer, H (components
// 3-5) on HBX x HBY and E (components 0-2) on EBX x EBY of one z-plane, over a
// 4-D view (x, y, z, component) of the six arrays; the class ids on CBX x EBY.
// Reads outside (nx, ny, nz) return zeros.
static int encode_tensor_maps(fdtd_llg_t h, const Instance &I, Inst &d, int sx)
{
    const cuuint32_t hbx = sx == 32 ? Tile<32>::HBX : Tile<64>::HBX, hby = sx == 32 ? Tile<32>::HBY : Tile<64>::HBY;
    const cuuint32_t ebx = sx == 32 ? Tile<32>::EBX : Tile<64>::EBX, eby = sx == 32 ? Tile<32>::EBY : Tile<64>::EBY;
    const cuuint32_t cb8 = sx == 32 ? Tile<32>::CBX8 : Tile<64>::CBX8, cb16 = sx == 32 ? Tile<32>::CBX16 : Tile<64>::CBX16;
    auto enc = tensor_map_encoder();
    if (!enc) return fail(h, FDTD_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const cuuint64_t nf = I.n_field();
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t dims[4] = {(cuuint64_t)I.nx, (cuuint64_t)I.ny, (cuuint64_t)I.nz, 6};
        const cuuint64_t strides[3] = {(cuuint64_t)I.px * 4, (cuuint64_t)I.px * I.ny * 4, nf * 4};
        const cuuint32_t boxH[4] = {hbx, hby, 1, 3}, boxE[4] = {ebx, eby, 1, 3};
        CUresult r = enc(&d.tm[TM_H0 + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, I.fields[b], dims, strides, boxH, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = enc(&d.tm[TM_E0 + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, I.fields[b], dims, strides, boxE, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, FDTD_E_CUDA, "cuTensorMapEncodeTiled failed for a field buffer");
    }
    const bool c16 = I.cls_bytes == 2;
    const cuuint64_t cdims[3] = {(cuuint64_t)I.nx, (cuuint64_t)I.ny, (cuuint64_t)I.nz};
    const cuuint64_t cstr[2] = {(cuuint64_t)I.px * I.cls_bytes, (cuuint64_t)I.px * I.ny * I.cls_bytes};
    const cuuint32_t cbox[3] = {c16 ? cb16 : cb8, eby, 1};
    const CUresult r = enc(&d.tm[TM_CLS], c16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, I.cls,
                           cdims, cstr, cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, FDTD_E_CUDA, "cuTensorMapEncodeTiled failed for the class ids");
    return FDTD_OK;
}

// Sweep tile width: the shape (64 x 8 or 32 x 16) that pads the instances'
// x-y extents to fewer cells (64 on ties); lanes beyond the grid do no useful
// work, so the padded count is the sweep's cost in lanes.
static int choose_width(const Sim *S)
{
    long long p64 = 0, p32 = 0;
    for (const Instance &I : S->inst) {
        p64 += (long long)((I.nx + 63) / 64) * 64 * ((I.ny + Tile<64>::Y - 1) / Tile<64>::Y) * Tile<64>::Y * I.nz;
        p32 += (long long)((I.nx + 31) / 32) * 32 * ((I.ny + Tile<32>::Y - 1) / Tile<32>::Y) * Tile<32>::Y * I.nz;
    }
    return p32 < p64 ? 32 : 64;
}

// Columns (x-y tiles) of an instance at tile width sx.
static int columns_of(const Instance &I, int sx)
{
    const int sy = kST / (sx / 2);
    return ((I.nx + sx - 1) / sx) * ((I.ny + sy - 1) / sy);
}

// Plane count of the sweep tasks from a cost model.  A task of P planes
// costs about P + 1.4 plane-times (the plane below, which only loads H, ~0.4,
// and the extra E^{n+1} plane above, 1); `slots` CTAs drawing the tasks
// finish after the total over the slots plus, on average, half the longest
// task.  Fewer, longer tasks cut the per-task planes, shorter ones the tail;
// the P with the smallest modelled time wins (the smallest on ties).
// (Measured against it: a schedule of long tasks drawn first and short ones
// last was 2 % slower on a 256 x 256 x 128 grid and within 3 % elsewhere.)
// Cost model of the field sweep for P planes per task (in plane-times of one
// CTA slot): the items each slot reads (a task of p planes costs p + 1.4: the
// H plane below and the extra E^{n+1} plane above) and half the longest task
// for the tail.
static double model_cost(const Sim *S, int P, int slots)
{
    double items = 0;
    int maxt = 0;
    for (const Instance &I : S->inst) {
        const int pk = std::min(P, I.nz), nch = (I.nz + pk - 1) / pk;
        items += (double)columns_of(I, S->sx) * (I.nz + 1.4 * nch);
        maxt = std::max(maxt, pk);
    }
    return items / std::max(1, slots) + 0.5 * (maxt + 1.4);
}

static int max_planes(const Sim *S)
{
    int maxnz = 1;
    for (const Instance &I : S->inst) maxnz = std::max(maxnz, I.nz);
    return std::max(2, std::min(maxnz, 128));
}

static int model_planes(const Sim *S, int slots)
{
    int best = kSZ;
    double best_t = 1e300;
    for (int P = 2; P <= max_planes(S); ++P) {
        const double t = model_cost(S, P, slots);
        if (t < best_t * (1.0 - 1e-9)) { best_t = t; best = P; }
    }
    return best;
}

// The plane counts the model rates within frac of its best, best first, at
// most n of them: the model ignores how the tasks fill the last wave of
// CTAs, which decides between such near ties.
static std::vector<int> model_near(const Sim *S, int slots, double frac, size_t n)
{
    std::vector<std::pair<double, int>> c;
    for (int P = 2; P <= max_planes(S); ++P) c.emplace_back(model_cost(S, P, slots), P);
    std::sort(c.begin(), c.end());
    std::vector<int> out;
    for (const auto &q : c)
        if (q.first <= c[0].first * (1.0 + frac) && out.size() < n) out.push_back(q.second);
    return out;
}

static void drop_graph1(Sim *S);
static void drop_graph_r(Sim *S);

// Tilings that fdtd_llg_autotune found in this process, by the shape of the
// batch (every instance's extents, magnet regions and absorbing layers): a
// handle of the same shape whose tiling and tile width are both left to the
// library starts from the tuned pair instead of the cost model, so the
// choice does not depend on which handle, or how long a run, was tuned.
static std::mutex g_tune_mu;
struct Tuned { int planes, width, mag_cs; };
static std::map<std::vector<long long>, Tuned> g_tuned;   // shape -> tuned choices (mag_cs 0: the automatic one)

static std::vector<long long> tune_key(const Sim *S)
{
    std::vector<long long> k;
    for (const Instance &I : S->inst) {
        k.push_back(I.nx);
        k.push_back(I.ny);
        k.push_back(I.nz);
        k.push_back((long long)I.comps.size());
        k.push_back(((long long)I.pml_n[0] << 40) | ((long long)I.pml_n[1] << 20) | I.pml_n[2]);
    }
    return k;
}

static int upload_descriptors(fdtd_llg_t h)
{
    Sim *S = h->sim;
    if (!S->dirty) return FDTD_OK;
    CKR(h, cudaStreamSynchronize(S->stream));
    int want_w = S->tile_width, want_p = S->tiling, want_cs = S->mag_cluster;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const auto it = g_tuned.find(tune_key(S));
        if (it != g_tuned.end()) {
            if (!want_w && want_p <= 0) {
                want_p = it->second.planes;
                want_w = it->second.width;
            }
            if (!want_cs) want_cs = it->second.mag_cs;
        }
    }
    S->sx = want_w ? want_w : choose_width(S);
    S->planes = want_p > 0 ? want_p : model_planes(S, S->nsm * std::max(1, step_blocks_per_sm(false, true, S->sx)));
    std::vector<Inst> hi(S->inst.size());
    std::vector<int> tile_inst;
    // sweep tasks of `planes` planes: energy slots per instance by column,
    // then z; claim order plane band by plane band over all instances
    struct TaskRec { int4 t; int band; };
    std::vector<TaskRec> recs;
    std::vector<MagComp> comps;
    bool c16 = false;
    int vmax = 0, msmem = 0;
    bool stab = true;
    for (size_t ii = 0; ii < S->inst.size(); ++ii) {
        Instance &I = S->inst[ii];
        if (!I.materials_set) return fail(h, FDTD_E_STATE, "instance " + std::to_string(ii) + " has no materials");
        if ((int)I.probes.size() != I.probe_alloc) {
            S->dfree(I.probe_buf);
            const size_t pb = (size_t)S->cfg.probe_capacity * std::max<size_t>(1, I.probes.size()) * 9 * sizeof(double);
            I.probe_buf = (double *)S->dalloc(pb);
            if (!I.probe_buf) return fail(h, FDTD_E_OOM, "device allocation failed");
            CKR(h, cudaMemset(I.probe_buf, 0, pb));
            I.probe_alloc = (int)I.probes.size();
        }
        Inst &d = hi[ii];
        std::memset(&d, 0, sizeof d);
        const size_t nf = I.n_field();
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 6; ++c) d.F[b][c] = I.fields[b] + c * nf;
        d.fstride = (long long)nf;
        d.wHx = I.walls; d.wHy = I.walls + (size_t)I.ny * I.nz; d.wHz = d.wHy + (size_t)I.nx * I.nz;
        d.cls = I.cls; d.ctab = I.ctab; d.nclass = I.nclass;
        stab = stab && I.nclass <= kTabMax;
        d.probe_buf = I.probe_buf; d.energy_buf = I.energy_buf;
        d.nx = I.nx; d.ny = I.ny; d.nz = I.nz; d.px = I.px;
        d.plane = (long long)I.ny * I.px;
        d.idx = (float)(1.0 / I.dx); d.idy = (float)(1.0 / I.dy); d.idz = (float)(1.0 / I.dz);
        d.ch = (float)(S->dt / (2.0 * kMu0));
        for (int q = 0; q < 9; ++q) d.R[q] = I.R[q];
        d.h0n = (float)std::sqrt(I.hbias[0] * I.hbias[0] + I.hbias[1] * I.hbias[1] + I.hbias[2] * I.hbias[2]);
        for (int q = 0; q < 3; ++q) d.u[q] = I.u[q];
        d.dt = S->dt;
        d.dV = I.dx * I.dy * I.dz;
        d.cap = S->cfg.probe_capacity;
        d.nsrc = (int)I.src.size();
        for (int s = 0; s < d.nsrc; ++s)
            for (int q = 0; q < 4; ++q) { d.src[s][q] = I.src[s][q]; d.srcp[s][q] = I.srcp[s][q]; }
        d.nprobe = (int)I.probes.size();
        for (int p = 0; p < d.nprobe; ++p)
            for (int q = 0; q < 3; ++q) d.probe[p][q] = I.probes[p][q];
        d.ntx = (I.nx + kTX - 1) / kTX; d.nty = (I.ny + kTY - 1) / kTY; d.ntz = (I.nz + kKC - 1) / kKC;
        d.tile_off = (int)tile_inst.size();
        const int nt = d.ntx * d.nty * d.ntz;
        for (int t = 0; t < nt; ++t) tile_inst.push_back((int)ii);
        {
            const int sy = kST / (S->sx / 2);
            const int fntx = (I.nx + S->sx - 1) / S->sx, fnty = (I.ny + sy - 1) / sy;
            if (I.nz > 0xFFFF || fntx > 0xFFFF || fnty > 0x7FFF) return fail(h, FDTD_E_INVAL, "grid too large for the sweep's task records");
            const int pl = std::min(S->planes, I.nz);
            d.ftile_off = (int)recs.size();
            for (int ty = 0; ty < fnty; ++ty)
                for (int tx = 0; tx < fntx; ++tx)
                    for (int k = 0, band = 0; k < I.nz; k += pl, ++band) {
                        TaskRec r;
                        r.t = make_int4((int)ii, tx | (ty << 16), k | (std::min(I.nz, k + pl) << 16), (int)recs.size());
                        r.band = band;
                        recs.push_back(r);
                    }
            d.fntask = (int)recs.size() - d.ftile_off;
        }
        d.mag_off = (int)comps.size();
        d.nmag = (int)I.comps.size();
        for (auto C : I.comps) {
            C.inst = (int)ii;
            C.ax = mag_split_axis(C.bx, C.by, C.bz);
            comps.push_back(C);
        }
        for (size_t m = 0; m < I.mm.size(); ++m) d.mm[m] = I.mm[m];
        c16 = c16 || I.cls_bytes == 2;
    }
    // magnet CTAs per region: the requested count, else as set out below
    // (the autotuner may also time the other choice); never more than the
    // shortest split extent of any region (no empty slab) nor kMagClusterMax
    int mcs = 1, mxs = 0;
    if (!comps.empty()) {
        int maxV = 0, minext = kMagClusterMax;
        for (const MagComp &C : comps) {
            maxV = std::max(maxV, C.V);
            minext = std::min(minext, C.ax == 0 ? C.bx : (C.ax == 1 ? C.by : C.bz));
        }
        // fewest CTAs per region whose slabs fit one CTA
        int need = 1;
        for (const MagComp &C : comps) {
            int c = 1;
            for (; c < kMagClusterMax; ++c) {
                int sx, sy, sz, qx, py, ps;
                mag_slab_box(C.bx, C.by, C.bz, c, sx, sy, sz);
                const int x = c > 1 ? mag_cross_section(C.bx, C.by, C.bz) : 0;
                if ((long long)sx * sy * sz <= kMagMaxV && mag_stage_block(sx, sy, sz, qx, py, ps, x, x)) break;
            }
            need = std::max(need, c);
        }
        // split further, to about kMagCtaCells cells per CTA, only where the
        // magnet kernel would outlast the field sweep running beside it (a
        // small grid with a large region): split CTAs displace sweep CTAs
        // from more SMs.  Model: the sweep at ~5 TB/s over every cell; the
        // magnet kernel in one CTA ~15 us + 40 us per 1024 cells of the
        // largest region.  Measured per step: 128x128x64 with a 1024-cell
        // block 43 -> 33 us on 8 CTAs; 256x256x128 with a 1280-cell film 84 us
        // on 1 CTA, 84-87 us on 2-8; the 64-cube sweep 338 us on 1, 349-370
        // on 2-4.
        long long cells = 0;
        for (const Instance &I : S->inst) cells += (long long)I.nx * I.ny * I.nz;
        const double t_sweep = (double)cells * 49.0 / 5.0e6, t_mag = 15.0 + 40.0 * maxV / 1024.0;
        const int fast = std::min({kMagClusterMax, minext, (maxV + kMagCtaCells - 1) / kMagCtaCells});
        S->mag_cs_fast = std::max(need, fast);
        S->mag_cs_need = need;
        mcs = want_cs > 0 ? want_cs : (t_mag > t_sweep ? std::max(need, fast) : need);
        if (mcs > minext)
            return fail(h, FDTD_E_INVAL, "magnet cluster of " + std::to_string(mcs) + " CTAs splits a region only " +
                                             std::to_string(minext) + " cells long");
        if (mcs > 1)
            for (const MagComp &C : comps) mxs = std::max(mxs, mag_cross_section(C.bx, C.by, C.bz));
        for (MagComp &C : comps) {
            int sx, sy, sz;
            mag_slab_box(C.bx, C.by, C.bz, mcs, sx, sy, sz);
            const int hxs = mcs > 1 ? mag_cross_section(C.bx, C.by, C.bz) : 0;
            if ((long long)sx * sy * sz > kMagMaxV || !mag_stage_block(sx, sy, sz, C.qx, C.py, C.ps, mxs, hxs))
                return fail(h, FDTD_E_INVAL, "a magnetic region (" + std::to_string(C.bx) + " x " + std::to_string(C.by) +
                                                 " x " + std::to_string(C.bz) + ") does not fit " + std::to_string(mcs) +
                                                 " magnet CTAs; the batch's smallest region limits the split");
            vmax = std::max(vmax, sx * sy * sz);
            msmem = std::max(msmem, (int)mag_cta_smem(sx, sy, sz, C.qx, C.py, C.ps, mxs, hxs));
        }
    }
    if (c16)
        for (size_t ii = 0; ii < S->inst.size(); ++ii) {
            Instance &I = S->inst[ii];
            if (I.cls_bytes == 2) continue;
            // widen this instance's class ids so that a batch shares one width
            std::vector<uint8_t> narrow(I.n_field());
            CKR(h, cudaMemcpy(narrow.data(), I.cls, narrow.size(), cudaMemcpyDeviceToHost));
            std::vector<uint16_t> wide(narrow.begin(), narrow.end());
            void *w = S->dalloc(wide.size() * 2);
            if (!w) return fail(h, FDTD_E_OOM, "device allocation failed");
            CKR(h, cudaMemcpy(w, wide.data(), wide.size() * 2, cudaMemcpyHostToDevice));
            S->dfree(I.cls);
            I.cls = w;
            I.cls_bytes = 2;
            hi[ii].cls = w;
        }
    // TMA descriptors of every instance, after the class width is settled
    for (size_t ii = 0; ii < S->inst.size(); ++ii) {
        const int rc = encode_tensor_maps(h, S->inst[ii], hi[ii], S->sx);
        if (rc) return rc;
    }
    // claim order: by z band, then instance and column
    std::stable_sort(recs.begin(), recs.end(), [](const TaskRec &a, const TaskRec &b) {
        if (a.band != b.band) return a.band < b.band;
        return a.t.x < b.t.x;
    });
    std::vector<int4> ftask(recs.size());
    for (size_t q = 0; q < recs.size(); ++q) ftask[q] = recs[q].t;
    // the flush's energy chunks, one CTA each
    std::vector<int2> ered;
    for (size_t ii = 0; ii < hi.size(); ++ii)
        for (int c = 0; c < energy_chunks(hi[ii].fntask); ++c) ered.push_back(make_int2((int)ii, c));
    S->dfree(S->d_insts); S->dfree(S->d_tile_inst); S->dfree(S->d_ftile_inst); S->dfree(S->d_comps); S->dfree(S->d_part);
    S->dfree(S->d_ered); S->dfree(S->d_esum); S->dfree(S->d_ecnt);
    S->d_ered = (int2 *)S->dalloc(ered.size() * sizeof(int2));
    S->d_esum = (double *)S->dalloc(hi.size() * kEChunks * sizeof(double));
    S->d_ecnt = (unsigned *)S->dalloc(hi.size() * sizeof(unsigned));
    if (!S->d_ered || !S->d_esum || !S->d_ecnt) return fail(h, FDTD_E_OOM, "device allocation failed");
    CKR(h, cudaMemcpy(S->d_ered, ered.data(), ered.size() * sizeof(int2), cudaMemcpyHostToDevice));
    CKR(h, cudaMemset(S->d_ecnt, 0, hi.size() * sizeof(unsigned)));
    S->nred = (int)ered.size();
    S->d_insts = (Inst *)S->dalloc(hi.size() * sizeof(Inst));
    S->d_tile_inst = (int *)S->dalloc(tile_inst.size() * sizeof(int));
    S->d_ftile_inst = (int4 *)S->dalloc(std::max<size_t>(1, ftask.size()) * sizeof(int4));
    S->d_comps = (MagComp *)S->dalloc(std::max<size_t>(1, comps.size()) * sizeof(MagComp));
    const size_t part_stride = ftask.size() * kSW + comps.size() * mcs;
    S->d_part = (double *)S->dalloc((2 * part_stride + 1) * sizeof(double));
    if (!S->d_insts || !S->d_tile_inst || !S->d_ftile_inst || !S->d_comps || !S->d_part)
        return fail(h, FDTD_E_OOM, "device allocation failed");
    CKR(h, cudaMemcpy(S->d_insts, hi.data(), hi.size() * sizeof(Inst), cudaMemcpyHostToDevice));
    CKR(h, cudaMemcpy(S->d_tile_inst, tile_inst.data(), tile_inst.size() * sizeof(int), cudaMemcpyHostToDevice));
    CKR(h, cudaMemcpy(S->d_ftile_inst, ftask.data(), ftask.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!comps.empty()) CKR(h, cudaMemcpy(S->d_comps, comps.data(), comps.size() * sizeof(MagComp), cudaMemcpyHostToDevice));
    CKR(h, cudaMemset(S->d_part, 0, (2 * part_stride + 1) * sizeof(double)));
    // the pending step's partials are gone with the old buffer (its energy was
    // already summed by the flush that ended its run): epend = -1
    CKR(h, cudaMemsetAsync(&S->d_ctl->epend, 0xFF, sizeof(long long), S->stream));
    CKR(h, cudaStreamSynchronize(S->stream));
    S->ntiles = (int)tile_inst.size();
    S->nftiles = (int)ftask.size();
    S->ncomp = (int)comps.size();
    S->mag_cs = mcs;
    S->mag_xs = mxs;
    S->vmax = vmax;
    S->stab = stab;
    S->mag_smem = msmem;
    S->cls16 = c16;
    {
        // absorbing layers: per lined instance, its descriptor and the disjoint
        // boxes of its layer cells, each box a range of whole blocks
        S->pml.clear();
        for (size_t ii = 0; ii < S->inst.size(); ++ii) {
            const Instance &I = S->inst[ii];
            if (!I.has_pml()) continue;
            PmlLaunch q;
            std::memset(&q, 0, sizeof q);
            const int dx = I.pml_n[0], dy = I.pml_n[1], dz = I.pml_n[2];
            auto add = [&](int i0, int j0, int k0, int bx, int by, int bz, int axes) {
                if (bx <= 0 || by <= 0 || bz <= 0) return;
                // multipliers ceil(2^32 / d) where every dividend times d stays below
                // 2^32 (exact quotients); 0: the kernel divides
                const unsigned long long vol = (unsigned long long)bx * by * bz;
                const unsigned mbx = bx > 1 && vol * bx < (1ull << 32) ? (unsigned)(0xFFFFFFFFull / (unsigned)bx + 1) : 0u;
                const unsigned mby = by > 1 && (unsigned long long)by * by * bz < (1ull << 32)
                                         ? (unsigned)(0xFFFFFFFFull / (unsigned)by + 1) : 0u;
                q.box[q.nbox] = PmlBox{i0, j0, k0, bx, by, bz, mbx, mby, axes};
                q.blk[q.nbox + 1] = q.blk[q.nbox] + (int)(((long long)bx * by * bz + 255) / 256);
                ++q.nbox;
            };
            add(0, 0, 0, I.nx, I.ny, dz, 7);                                // z layers: whole planes
            if (dz) add(0, 0, I.nz - dz, I.nx, I.ny, dz, 7);
            add(0, 0, dz, I.nx, dy, I.nz - 2 * dz, 3);                       // y layers between them
            if (dy) add(0, I.ny - dy, dz, I.nx, dy, I.nz - 2 * dz, 3);
            add(0, dy, dz, dx, I.ny - 2 * dy, I.nz - 2 * dz, 1);             // x layers in the rest
            if (dx) add(I.nx - dx, dy, dz, dx, I.ny - 2 * dy, I.nz - 2 * dz, 1);
            for (int a = 0; a < 3; ++a) {
                q.pd[a] = I.pml_n[a];
                q.psi[a] = I.psi[a];
                q.pco[a] = I.pco[a];
                q.pvol[a] = (unsigned)I.pvol[a];
            }
            q.F[0] = I.fields[0];
            q.F[1] = I.fields[1];
            q.fs = (unsigned)I.n_field();
            q.plane = (unsigned)((size_t)I.ny * I.px);
            q.n[0] = I.nx; q.n[1] = I.ny; q.n[2] = I.nz;
            q.px = I.px;
            q.id[0] = (float)(1.0 / I.dx); q.id[1] = (float)(1.0 / I.dy); q.id[2] = (float)(1.0 / I.dz);
            q.dtmu = 2.f * (float)(S->dt / (2.0 * kMu0));
            q.cls = I.cls;
            q.ctab = I.ctab;
            S->pml.push_back(q);
        }
    }
    S->dirty = false;
    if (S->graph) { cudaGraphExecDestroy(S->graph); S->graph = nullptr; }   // its launch set is stale
    S->graph_parity = -1;
    drop_graph1(S);
    drop_graph_r(S);
    return FDTD_OK;
}

static LaunchSet launch_set(Sim *S)
{
    LaunchSet L{};
    L.insts = S->d_insts;
    L.ninst = (int)S->inst.size();
    L.tile_inst = S->d_tile_inst;
    L.ntiles = S->ntiles;
    L.comps = S->d_comps;
    L.ncomp = S->ncomp;
    L.vmax = S->vmax;
    L.mag_smem = S->mag_smem;
    L.stab = S->stab;
    L.ctl = S->d_ctl;
    L.nslot_f = S->nftiles * kSW;
    L.part_stride = L.nslot_f + S->ncomp * S->mag_cs;
    L.mag_cs = S->mag_cs;
    L.mag_xs = S->mag_xs;
    L.test_wait = S->test_wait;
    L.part_f = S->d_part;
    L.part_m = S->d_part + L.nslot_f;
    L.ftask = S->d_ftile_inst;
    L.nftiles = S->nftiles;
    L.ered = S->d_ered;
    L.nred = S->nred;
    L.esum = S->d_esum;
    L.ecnt = S->d_ecnt;
    // persistent field-sweep CTAs: as many as fit at once (late ones, queued
    // behind the magnet CTAs, take what is left of the task counter)
    L.sx = S->sx;
    L.nfblocks = std::max(1, std::min(S->nftiles, S->nsm * std::max(1, step_blocks_per_sm(S->cls16, S->stab, S->sx))));
    L.src = S->cur;
    L.dst = 1 - S->cur;
    L.cls16 = S->cls16;
    L.grid_h = std::min(S->ntiles, S->nsm * h_half_blocks_per_sm(S->cls16));
    L.llg_tol = (float)S->cfg.llg_tol;
    L.llg_max_iter = S->cfg.llg_max_iter;
    L.llg_fixed_iter = S->cfg.llg_fixed_iter;
    L.energy = S->cfg.energy_every != 0;
    return L;
}

// Steps per CUDA graph: long step calls on a stream that can be captured
// replay one graph of kGraphSteps steps instead of launching kernel by kernel.
constexpr int64_t kGraphSteps = 32;

static bool capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

static_assert(kGraphSteps <= 32, "graph_r holds graphs of fewer than 32 steps");

static void drop_graph1(Sim *S)
{
    for (auto &g1 : S->graph1)
        if (g1) { cudaGraphExecDestroy(g1); g1 = nullptr; }
}

static void drop_graph_r(Sim *S)
{
    for (auto &gr : S->graph_r)
        for (auto &g : gr)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

// Capture n steps starting from buffer S->cur (the absorbing-layer passes and
// the step's kernels, no flush) and instantiate them into *out.
static cudaError_t capture_steps(Sim *S, LaunchSet L, int64_t n, cudaGraphExec_t *out)
{
    *out = nullptr;
    cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int cur = S->cur;
    for (int64_t q = 0; q < n && e == cudaSuccess; ++q) {
        L.src = cur;
        L.dst = 1 - cur;
        e = launch_pml(S->pml.data(), (int)S->pml.size(), L.src, L.cls16, S->stream);
        if (e == cudaSuccess) e = launch_step(L, S->stream, nullptr);
        cur ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(S->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (e != cudaSuccess) *out = nullptr;
    if (g) cudaGraphDestroy(g);
    return e;
}

// The graph of a one-step call starting from buffer S->cur: the step's two
// kernels and the flush, which takes the step from the device counter.
static cudaError_t build_graph1(Sim *S, LaunchSet L)
{
    cudaGraphExec_t &g1 = S->graph1[S->cur];
    if (g1) { cudaGraphExecDestroy(g1); g1 = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    L.src = S->cur;
    L.dst = 1 - S->cur;
    e = launch_pml(S->pml.data(), (int)S->pml.size(), L.src, L.cls16, S->stream);
    if (e == cudaSuccess) e = launch_step(L, S->stream, nullptr);
    if (e == cudaSuccess) e = launch_energy_flush(L, S->rings_mapped ? S->d_rings : nullptr, -1, -1, S->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(S->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g1, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// (Re)build the graph of kGraphSteps steps starting from buffer S->cur.
static cudaError_t build_graph(Sim *S, LaunchSet L)
{
    if (S->graph) { cudaGraphExecDestroy(S->graph); S->graph = nullptr; }
    const cudaError_t e = capture_steps(S, L, kGraphSteps, &S->graph);
    S->graph_parity = e == cudaSuccess ? S->cur : -1;
    return e;
}

// Queue on the stream the copies of steps [n0, n1)'s probe rows and energies
// from the device rings into the instances' pageable host rings (those that
// stream), after everything queued so far; steps older than the device ring
// are gone.
static cudaError_t stream_out(Sim *S, long long n0, long long n1)
{
    const long long dcap = S->cfg.probe_capacity;
    for (Instance &I : S->inst) {
        if (I.host_cap < 1) continue;
        const long long np = (long long)I.probes.size();
        for (long long st = std::max(n0, n1 - dcap); st < n1;) {
            const long long ds = st % dcap, hs = st % I.host_cap;
            const long long run = std::min({n1 - st, dcap - ds, I.host_cap - hs});
            cudaError_t e = cudaSuccess;
            if (I.host_rows && np)
                e = cudaMemcpyAsync(I.host_rows + hs * np * 9, I.probe_buf + ds * np * 9, run * np * 9 * sizeof(double),
                                    cudaMemcpyDeviceToHost, S->stream);
            if (e == cudaSuccess && I.host_energy)
                e = cudaMemcpyAsync(I.host_energy + hs, I.energy_buf + ds, run * sizeof(double), cudaMemcpyDeviceToHost,
                                    S->stream);
            if (e != cudaSuccess) return e;
            st += run;
        }
    }
    return cudaSuccess;
}

extern "C" int fdtd_llg_stream_results(fdtd_llg_t h, double *rows, double *energy, int64_t capacity)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "stream_results needs an instance handle");
    if ((rows || energy) && capacity < 1) return fail(h, FDTD_E_INVAL, "capacity must be >= 1");
    Sim *S = h->sim;
    Instance *I = inst_of(h);
    CKR(h, cudaStreamSynchronize(S->stream));   // copies queued into the previous rings are done
    // pinned host memory is written by the flush kernel through its device
    // address; other host memory by copies queued after each step call
    auto mapped = [](double *p) -> double * {
        if (!p) return nullptr;
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return pa.type == cudaMemoryTypeHost ? (double *)pa.devicePointer : nullptr;
    };
    HostRing R{mapped(rows), mapped(energy), capacity};
    I->host_rows = R.rows ? nullptr : rows;
    I->host_energy = R.energy ? nullptr : energy;
    I->host_cap = (I->host_rows || I->host_energy) ? capacity : 0;
    I->ring_mapped = R.rows || R.energy;
    if (!S->d_rings) {
        S->d_rings = (HostRing *)S->dalloc(S->inst.size() * sizeof(HostRing));
        if (!S->d_rings) return fail(h, FDTD_E_OOM, "device allocation failed");
        CKR(h, cudaMemset(S->d_rings, 0, S->inst.size() * sizeof(HostRing)));
    }
    CKR(h, cudaMemcpy(S->d_rings + (I - S->inst.data()), &R, sizeof(HostRing), cudaMemcpyHostToDevice));
    S->rings_mapped = false;
    for (const Instance &J : S->inst) S->rings_mapped = S->rings_mapped || J.ring_mapped;
    drop_graph1(S);   // they pass the rings to the flush
    return FDTD_OK;
}

extern "C" int fdtd_llg_step(fdtd_llg_t h, int64_t nsteps)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    if (!h->owns) return fail(h, FDTD_E_INVAL, "step the batch handle, not a member");
    if (nsteps < 0) return fail(h, FDTD_E_INVAL, "nsteps < 0");
    Sim *S = h->sim;
    int rc = upload_descriptors(h);
    if (rc) return rc;
    LaunchSet L = launch_set(S);
    if (!S->half_ahead && nsteps > 0) {
        L.src = L.dst = S->cur;
        CKR(h, launch_half(L, S->stream));
        S->half_ahead = true;
    }
    int64_t s = 0;
    const bool want = S->graph_mode != 0;   // -1 (default): replay shortens the gaps between steps at every size
    if (want && !S->profiling && !S->graph_off && nsteps >= 2 && capturable(S->stream)) {
        // whole graphs of kGraphSteps steps, then one cached graph of the
        // remaining r < kGraphSteps steps, so that calls of any length (a
        // short call repeated, as a serving loop makes them) replay graphs
        if (nsteps >= kGraphSteps) {
            if ((!S->graph || S->graph_parity != S->cur) && build_graph(S, L) != cudaSuccess) {
                cudaGetLastError();   // not fatal: this stream is stepped launch by launch
                S->graph_off = true;
            }
            if (S->graph)
                for (; s + kGraphSteps <= nsteps; s += kGraphSteps) CKR(h, cudaGraphLaunch(S->graph, S->stream));
        }
        const int64_t r = nsteps - s;
        if (r > 0 && !S->graph_off) {
            cudaGraphExec_t &gr = S->graph_r[r][S->cur];
            if (!gr && capture_steps(S, L, r, &gr) != cudaSuccess) {
                cudaGetLastError();
                S->graph_off = true;
            }
            if (gr) {
                CKR(h, cudaGraphLaunch(gr, S->stream));
                s += r;
                if (r & 1) S->cur ^= 1;
            }
        }
    }
    if (want && nsteps == 1 && !S->profiling && !S->graph_off && capturable(S->stream)) {
        // a one-step call: one replayed graph of the step and its flush
        if (!S->graph1[S->cur] && build_graph1(S, L) != cudaSuccess) {
            cudaGetLastError();
            S->graph_off = true;
        }
        if (S->graph1[S->cur]) {
            CKR(h, cudaGraphLaunch(S->graph1[S->cur], S->stream));
            S->cur ^= 1;
            CKR(h, stream_out(S, S->host_step, S->host_step + 1));
            S->host_step += 1;
            return FDTD_OK;
        }
    }
    for (; s < nsteps; ++s) {
        L.src = S->cur;
        L.dst = 1 - S->cur;
        cudaEvent_t ev[4];
        cudaEvent_t *prof = nullptr;
        if (S->profiling) {
            for (auto &e : ev) e = S->take_event();
            prof = ev;
        }
        CKR(h, launch_pml(S->pml.data(), (int)S->pml.size(), L.src, L.cls16, S->stream));
        CKR(h, launch_step(L, S->stream, prof));
        if (prof) {
            S->recs.push_back({0, ev[0], ev[1]});
            if (L.ncomp) S->recs.push_back({1, ev[2], ev[3]});
            else { S->ev_pool.push_back(ev[2]); S->ev_pool.push_back(ev[3]); }
        }
        S->cur ^= 1;
    }
    const HostRing *rings = S->rings_mapped ? S->d_rings : nullptr;
    if (nsteps > 0) CKR(h, launch_energy_flush(L, rings, S->host_step, S->host_step + nsteps, S->stream));
    if (nsteps > 0) CKR(h, stream_out(S, S->host_step, S->host_step + nsteps));
    S->host_step += nsteps;
    return FDTD_OK;
}

static int check_status(fdtd_llg_t h, const StepCtl &c)
{
    if (c.status & ST_UNSTABLE) return fail(h, FDTD_E_UNSTABLE, "energy is not finite (unstable run)");
    if (c.status & ST_NOCONV) return fail(h, FDTD_E_LLG_NOCONV, "an LLG solve did not reach llg_tol within llg_max_iter");
    if (c.status & ST_TIMEOUT) return fail(h, FDTD_E_CUDA, "a field-kernel wait for its tile copies timed out");
    return FDTD_OK;
}

static int sync_status(fdtd_llg_t h)
{
    Sim *S = h->sim;
    CKR(h, cudaStreamSynchronize(S->stream));
    StepCtl c{};
    CKR(h, cudaMemcpy(&c, S->d_ctl, sizeof c, cudaMemcpyDeviceToHost));
    return check_status(h, c);
}

extern "C" int fdtd_llg_sync(fdtd_llg_t h)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    return sync_status(h);
}

extern "C" int fdtd_llg_time_state(fdtd_llg_t h, int64_t *step, int32_t *half)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    if (step) *step = h->sim->host_step;
    if (half) *half = h->sim->half_ahead ? 1 : 0;
    return FDTD_OK;
}

// rows of a ring holding host_step records of `stride` doubles (oldest first)
static int read_ring(fdtd_llg_t h, const double *dbuf, int stride, int col_off, int ncols, double *out, int64_t cap_rows,
                     int64_t *rows)
{
    Sim *S = h->sim;
    const long long cap = S->cfg.probe_capacity;
    const long long have = std::min<long long>(S->host_step, cap);
    const long long want = std::max<long long>(0, std::min<long long>(have, cap_rows));
    for (long long r = 0; r < want;) {
        const long long stepi = S->host_step - want + r;   // record of state stepi+1
        const long long slot = stepi % cap;
        const long long run = std::min<long long>(want - r, cap - slot);   // contiguous slots
        if (ncols == stride) {
            CKR(h, cudaMemcpyAsync(out + r * ncols, dbuf + slot * stride, run * ncols * sizeof(double),
                                   cudaMemcpyDeviceToHost, S->stream));
        } else {
            CKR(h, cudaMemcpy2DAsync(out + r * ncols, ncols * sizeof(double), dbuf + slot * stride + col_off,
                                     stride * sizeof(double), ncols * sizeof(double), run, cudaMemcpyDeviceToHost, S->stream));
        }
        r += run;
    }
    CKR(h, cudaStreamSynchronize(S->stream));
    if (rows) *rows = want;
    return FDTD_OK;
}

extern "C" int fdtd_llg_probe(fdtd_llg_t h, int32_t id, double *out, int64_t cap_rows, int64_t *rows)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "probe needs an instance handle");
    Instance *I = inst_of(h);
    if (id < 0 || id >= (int)I->probes.size()) return fail(h, FDTD_E_RANGE, "no such probe");
    if (!out && cap_rows > 0) return fail(h, FDTD_E_INVAL, "null output");
    int rc = sync_status(h);
    if (rc) return rc;
    if (!I->probe_buf || I->probe_alloc != (int)I->probes.size()) {
        if (rows) *rows = 0;
        return FDTD_OK;
    }
    return read_ring(h, I->probe_buf, (int)I->probes.size() * 9, id * 9, 9, out, cap_rows, rows);
}

extern "C" int fdtd_llg_energy(fdtd_llg_t h, double *out, int64_t cap, int64_t *written)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "energy needs an instance handle");
    Instance *I = inst_of(h);
    if (!out && cap > 0) return fail(h, FDTD_E_INVAL, "null output");
    int rc = sync_status(h);
    if (rc) return rc;
    return read_ring(h, I->energy_buf, 1, 0, 1, out, cap, written);
}

extern "C" int fdtd_llg_read_last(fdtd_llg_t h, double *probe_rows, double *energy)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "read_last needs an instance handle");
    Sim *S = h->sim;
    Instance *I = inst_of(h);
    if (S->host_step < 1) return fail(h, FDTD_E_STATE, "no step has run");
    const long long slot = (S->host_step - 1) % S->cfg.probe_capacity;
    const size_t np = I->probes.size();
    StepCtl c{};
    if (probe_rows && np)
        CKR(h, cudaMemcpyAsync(probe_rows, I->probe_buf + slot * np * 9, np * 9 * sizeof(double), cudaMemcpyDeviceToHost,
                               S->stream));
    if (energy) CKR(h, cudaMemcpyAsync(energy, I->energy_buf + slot, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
    CKR(h, cudaMemcpyAsync(&c, S->d_ctl, sizeof c, cudaMemcpyDeviceToHost, S->stream));
    CKR(h, cudaStreamSynchronize(S->stream));
    return check_status(h, c);
}

// ------------------------------------------------------------- fields
static int field_count(const Instance &I, int which, size_t &count)
{
    if ((which >= FDTD_F_EX && which <= FDTD_F_MZ) || (which >= FDTD_F_DMX && which <= FDTD_F_DMZ)) {
        count = (size_t)I.nx * I.ny * I.nz;
        return 0;
    }
    if (which == FDTD_F_HX_WALL) { count = (size_t)I.ny * I.nz; return 0; }
    if (which == FDTD_F_HY_WALL) { count = (size_t)I.nx * I.nz; return 0; }
    if (which == FDTD_F_HZ_WALL) { count = (size_t)I.nx * I.ny; return 0; }
    return -1;
}

// M of every region in global axes (FP64), as deviation (dev = true) or full value.
static int magnet_read(fdtd_llg_t h, Instance &I, std::vector<std::vector<double>> &out, std::vector<std::vector<uint8_t>> &mats,
                       bool dev)
{
    out.clear();
    mats.clear();
    for (auto &C : I.comps) {
        std::vector<float> m(3 * (size_t)C.V);
        std::vector<uint8_t> mt(C.V);
        CKR(h, cudaMemcpy(m.data(), C.m, m.size() * sizeof(float), cudaMemcpyDeviceToHost));
        CKR(h, cudaMemcpy(mt.data(), C.mat, C.V, cudaMemcpyDeviceToHost));
        std::vector<double> g(3 * (size_t)C.V, 0.0);
        for (int v = 0; v < C.V; ++v) {
            if (mt[v] == 0xFF) continue;
            const double l[3] = {m[v], m[C.V + v], m[2 * (size_t)C.V + v]};
            for (int d = 0; d < 3; ++d) {
                double val = (double)I.R[d] * l[0] + (double)I.R[3 + d] * l[1] + (double)I.R[6 + d] * l[2];
                if (!dev) val += I.mm_Ms[mt[v]] * I.u[d];
                g[(size_t)d * C.V + v] = val;
            }
        }
        out.push_back(std::move(g));
        mats.push_back(std::move(mt));
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_div_b(fdtd_llg_t h, double *out, size_t count)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "div_b needs an instance handle");
    Instance *I = inst_of(h);
    const size_t nc = (size_t)I->nx * I->ny * I->nz;
    if (!out || count < nc) return fail(h, FDTD_E_INVAL, "output too small");
    int rc = sync_status(h);
    if (rc) return rc;
    rc = upload_descriptors(h);
    if (rc) return rc;
    Sim *S = h->sim;
    const int idx = h->index < 0 ? 0 : h->index;
    double *dM = nullptr, *dout = nullptr;
    MagComp *dc = nullptr;
    const size_t ncomp = I->comps.size();
    cudaError_t e = cudaMalloc(&dM, 3 * nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, nc * sizeof(double));
    if (e == cudaSuccess && ncomp) e = cudaMalloc(&dc, ncomp * sizeof(MagComp));
    if (e == cudaSuccess && ncomp)
        e = cudaMemcpyAsync(dc, I->comps.data(), ncomp * sizeof(MagComp), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess)
        e = launch_div_b(S->d_insts + idx, dc, (int)ncomp, S->cur, (long long)nc, I->dx, I->dy, I->dz, dM, dout,
                         S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, nc * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    cudaFree(dM);
    cudaFree(dout);
    cudaFree(dc);
    if (e != cudaSuccess) return fail(h, FDTD_E_CUDA, std::string("div_b: ") + cudaGetErrorString(e));
    return FDTD_OK;
}

extern "C" int fdtd_llg_get_field(fdtd_llg_t h, int32_t which, float *out, size_t count)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "get_field needs an instance handle");
    Instance *I = inst_of(h);
    size_t need;
    if (field_count(*I, which, need)) return fail(h, FDTD_E_INVAL, "unknown field selector");
    if (!out || count < need) return fail(h, FDTD_E_INVAL, "output too small");
    int rc = sync_status(h);
    if (rc) return rc;
    const size_t nf = I->n_field();
    if (which <= FDTD_F_HZ) {
        CKR(h, cudaMemcpy2D(out, I->nx * sizeof(float), I->fields[h->sim->cur] + which * nf, I->px * sizeof(float), I->nx * sizeof(float),
                            (size_t)I->ny * I->nz, cudaMemcpyDeviceToHost));
    } else if (which <= FDTD_F_MZ || which >= FDTD_F_DMX) {
        const bool dev = which >= FDTD_F_DMX;
        const int d = dev ? which - FDTD_F_DMX : which - FDTD_F_MX;
        std::vector<std::vector<double>> g;
        std::vector<std::vector<uint8_t>> mt;
        rc = magnet_read(h, *I, g, mt, dev);
        if (rc) return rc;
        std::fill(out, out + need, 0.f);
        for (size_t c = 0; c < I->comps.size(); ++c) {
            const MagComp &C = I->comps[c];
            for (int v = 0; v < C.V; ++v) {
                if (mt[c][v] == 0xFF) continue;
                const int li = v % C.bx, lj = (v / C.bx) % C.by, lk = v / (C.bx * C.by);
                out[((size_t)(C.z0 + lk) * I->ny + (C.y0 + lj)) * I->nx + (C.x0 + li)] = (float)g[c][(size_t)d * C.V + v];
            }
        }
    } else {
        size_t off = 0;
        if (which >= FDTD_F_HY_WALL) off += (size_t)I->ny * I->nz;
        if (which >= FDTD_F_HZ_WALL) off += (size_t)I->nx * I->nz;
        CKR(h, cudaMemcpy(out, I->walls + off, need * sizeof(float), cudaMemcpyDeviceToHost));
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_field(fdtd_llg_t h, int32_t which, const float *in, size_t count)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "set_field needs an instance handle");
    Instance *I = inst_of(h);
    if (!I->materials_set) return fail(h, FDTD_E_STATE, "set materials first");
    size_t need;
    if (field_count(*I, which, need)) return fail(h, FDTD_E_INVAL, "unknown field selector");
    if (!in || count < need) return fail(h, FDTD_E_INVAL, "input too small");
    CKR(h, cudaStreamSynchronize(h->sim->stream));
    const size_t nf = I->n_field();
    if (which <= FDTD_F_HZ) {
        CKR(h, cudaMemcpy2D(I->fields[h->sim->cur] + which * nf, I->px * sizeof(float), in, I->nx * sizeof(float), I->nx * sizeof(float),
                            (size_t)I->ny * I->nz, cudaMemcpyHostToDevice));
    } else if (which <= FDTD_F_MZ || which >= FDTD_F_DMX) {
        const bool dev = which >= FDTD_F_DMX;
        const int d = dev ? which - FDTD_F_DMX : which - FDTD_F_MX;
        std::vector<std::vector<double>> g;
        std::vector<std::vector<uint8_t>> mt;
        int rc = magnet_read(h, *I, g, mt, true);
        if (rc) return rc;
        for (size_t c = 0; c < I->comps.size(); ++c) {
            const MagComp &C = I->comps[c];
            std::vector<float> m(3 * (size_t)C.V, 0.f);
            for (int v = 0; v < C.V; ++v) {
                if (mt[c][v] == 0xFF) continue;
                const int li = v % C.bx, lj = (v / C.bx) % C.by, lk = v / (C.bx * C.by);
                const double x = in[((size_t)(C.z0 + lk) * I->ny + (C.y0 + lj)) * I->nx + (C.x0 + li)];
                g[c][(size_t)d * C.V + v] = dev ? x : x - I->mm_Ms[mt[c][v]] * I->u[d];
                const double dg[3] = {g[c][v], g[c][C.V + v], g[c][2 * (size_t)C.V + v]};
                for (int q = 0; q < 3; ++q)
                    m[(size_t)q * C.V + v] = (float)((double)I->R[3 * q] * dg[0] + (double)I->R[3 * q + 1] * dg[1] +
                                                     (double)I->R[3 * q + 2] * dg[2]);
            }
            CKR(h, cudaMemcpy(C.m, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    } else {
        size_t off = 0;
        if (which >= FDTD_F_HY_WALL) off += (size_t)I->ny * I->nz;
        if (which >= FDTD_F_HZ_WALL) off += (size_t)I->nx * I->nz;
        CKR(h, cudaMemcpy(I->walls + off, in, need * sizeof(float), cudaMemcpyHostToDevice));
    }
    h->sim->half_ahead = false;
    return FDTD_OK;
}

extern "C" int fdtd_llg_planes(fdtd_llg_t h, int32_t k0, int32_t k1, float *buf, size_t count, int32_t to_handle)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "planes needs an instance handle");
    Instance *I = inst_of(h);
    if (!I->materials_set) return fail(h, FDTD_E_STATE, "set materials first");
    const int nx = I->nx, ny = I->ny, nz = I->nz;
    if (k0 < 0 || k1 > nz || k0 >= k1) return fail(h, FDTD_E_RANGE, "plane range outside the grid");
    if (to_handle && I->has_pml())
        return fail(h, FDTD_E_NOSYS, "planes cannot be written into a handle with absorbing layers (their memories are not exchanged)");
    const size_t P = (size_t)(k1 - k0), pl = (size_t)nx * ny;
    const size_t need = P * (9 * pl + nx + ny);
    if (!buf || count < need) return fail(h, FDTD_E_INVAL, "buffer too small");
    int rc = to_handle ? 0 : sync_status(h);
    if (rc) return rc;
    CKR(h, cudaStreamSynchronize(h->sim->stream));
    const size_t nf = I->n_field();
    const cudaMemcpyKind kind = to_handle ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    // E and H: six arrays of P planes, rows of nx from the padded rows of px
    for (int q = 0; q < 6; ++q) {
        float *dev = I->fields[h->sim->cur] + q * nf + (size_t)k0 * ny * I->px;
        float *host = buf + q * P * pl;
        if (to_handle)
            CKR(h, cudaMemcpy2D(dev, I->px * sizeof(float), host, nx * sizeof(float), nx * sizeof(float), P * ny, kind));
        else
            CKR(h, cudaMemcpy2D(host, nx * sizeof(float), dev, I->px * sizeof(float), nx * sizeof(float), P * ny, kind));
    }
    // far-wall normal H that has z planes: Hx at x = nx (ny per plane), Hy at y = ny (nx per plane)
    {
        float *hx = I->walls + (size_t)k0 * ny, *hy = I->walls + (size_t)ny * nz + (size_t)k0 * nx;
        float *bx = buf + 6 * P * pl, *by = bx + P * ny;
        if (to_handle) {
            CKR(h, cudaMemcpy(hx, bx, P * ny * sizeof(float), kind));
            CKR(h, cudaMemcpy(hy, by, P * nx * sizeof(float), kind));
        } else {
            CKR(h, cudaMemcpy(bx, hx, P * ny * sizeof(float), kind));
            CKR(h, cudaMemcpy(by, hy, P * nx * sizeof(float), kind));
        }
    }
    // the magnetisation deviation of magnetic cells, as stored (bias frame)
    float *bm = buf + 6 * P * pl + P * (nx + ny);
    if (!to_handle) std::fill(bm, bm + 3 * P * pl, 0.f);
    for (const MagComp &C : I->comps) {
        const int z0 = std::max(k0, C.z0), z1 = std::min(k1, C.z0 + C.bz);
        if (z0 >= z1) continue;
        std::vector<float> m(3 * (size_t)C.V);
        std::vector<uint8_t> mt(C.V);
        CKR(h, cudaMemcpy(m.data(), C.m, m.size() * sizeof(float), cudaMemcpyDeviceToHost));
        CKR(h, cudaMemcpy(mt.data(), C.mat, C.V, cudaMemcpyDeviceToHost));
        for (int k = z0; k < z1; ++k)
            for (int lj = 0; lj < C.by; ++lj)
                for (int li = 0; li < C.bx; ++li) {
                    const int v = ((k - C.z0) * C.by + lj) * C.bx + li;
                    if (mt[v] == 0xFF) continue;
                    const size_t o = ((size_t)(k - k0) * ny + (C.y0 + lj)) * nx + (C.x0 + li);
                    for (int d = 0; d < 3; ++d) {
                        if (to_handle) m[(size_t)d * C.V + v] = bm[d * P * pl + o];
                        else bm[d * P * pl + o] = m[(size_t)d * C.V + v];
                    }
                }
        if (to_handle) CKR(h, cudaMemcpy(C.m, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return FDTD_OK;
}

// ---------------------------------------------------------- checkpoints
namespace {
struct StateHeader {
    uint32_t magic, version;
    int32_t nx, ny, nz, ncomp;
    int64_t step;
    int32_t half_ahead, pad;
    uint64_t bytes;
};
constexpr uint32_t kMagic = 0x4c4c4446u;   // "FDLL"
}  // namespace

// The magnetisation deviation of region C's cells in planes [k0, k1) between
// the region's array and a plane buffer bm (3 x P x ny x nx, zero outside
// magnetic cells on read; ignored there on write).
__global__ void planes_m_kernel(MagComp C, int k0, int k1, int nx, int ny, float *bm, int to_handle)
{
    const int z0 = max(k0, C.z0), z1 = min(k1, C.z0 + C.bz);
    const long long n = (long long)(z1 - z0) * C.by * C.bx;
    const size_t P = (size_t)(k1 - k0), pl = (size_t)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int li = (int)(q % C.bx), lj = (int)((q / C.bx) % C.by), k = z0 + (int)(q / ((long long)C.bx * C.by));
        const int v = ((k - C.z0) * C.by + lj) * C.bx + li;
        if (C.mat[v] == 0xFF) continue;
        const size_t o = ((size_t)(k - k0) * ny + (C.y0 + lj)) * nx + (C.x0 + li);
        for (int d = 0; d < 3; ++d) {
            if (to_handle) C.m[(size_t)d * C.V + v] = bm[d * P * pl + o];
            else bm[d * P * pl + o] = C.m[(size_t)d * C.V + v];
        }
    }
}

extern "C" int fdtd_llg_planes_device(fdtd_llg_t h, int32_t k0, int32_t k1, float *buf, size_t count, int32_t to_handle)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "planes needs an instance handle");
    Instance *I = inst_of(h);
    Sim *S = h->sim;
    if (!I->materials_set) return fail(h, FDTD_E_STATE, "set materials first");
    const int nx = I->nx, ny = I->ny, nz = I->nz;
    if (k0 < 0 || k1 > nz || k0 >= k1) return fail(h, FDTD_E_RANGE, "plane range outside the grid");
    if (to_handle && I->has_pml())
        return fail(h, FDTD_E_NOSYS, "planes cannot be written into a handle with absorbing layers (their memories are not exchanged)");
    const size_t P = (size_t)(k1 - k0), pl = (size_t)nx * ny;
    const size_t need = P * (9 * pl + nx + ny);
    if (!buf || count < need) return fail(h, FDTD_E_INVAL, "buffer too small");
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, buf) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(h, FDTD_E_INVAL, "planes_device needs a device buffer");
    }
    const size_t nf = I->n_field();
    cudaStream_t st = S->stream;
    const cudaMemcpyKind kind = cudaMemcpyDeviceToDevice;
    for (int q = 0; q < 6; ++q) {
        float *dev = I->fields[S->cur] + q * nf + (size_t)k0 * ny * I->px;
        float *b = buf + q * P * pl;
        if (to_handle)
            CKR(h, cudaMemcpy2DAsync(dev, I->px * sizeof(float), b, nx * sizeof(float), nx * sizeof(float), P * ny, kind, st));
        else
            CKR(h, cudaMemcpy2DAsync(b, nx * sizeof(float), dev, I->px * sizeof(float), nx * sizeof(float), P * ny, kind, st));
    }
    float *hx = I->walls + (size_t)k0 * ny, *hy = I->walls + (size_t)ny * nz + (size_t)k0 * nx;
    float *bx = buf + 6 * P * pl, *by = bx + P * ny;
    if (to_handle) {
        CKR(h, cudaMemcpyAsync(hx, bx, P * ny * sizeof(float), kind, st));
        CKR(h, cudaMemcpyAsync(hy, by, P * nx * sizeof(float), kind, st));
    } else {
        CKR(h, cudaMemcpyAsync(bx, hx, P * ny * sizeof(float), kind, st));
        CKR(h, cudaMemcpyAsync(by, hy, P * nx * sizeof(float), kind, st));
    }
    float *bm = buf + 6 * P * pl + P * (nx + ny);
    if (!to_handle) CKR(h, cudaMemsetAsync(bm, 0, 3 * P * pl * sizeof(float), st));
    for (const MagComp &C : I->comps) {
        if (std::max(k0, C.z0) >= std::min(k1, C.z0 + C.bz)) continue;
        planes_m_kernel<<<64, 256, 0, st>>>(C, k0, k1, nx, ny, bm, to_handle);
        CKR(h, cudaGetLastError());
    }
    return FDTD_OK;
}

static size_t state_bytes(const Instance &I)
{
    size_t b = sizeof(StateHeader) + 6 * (size_t)I.nx * I.ny * I.nz * sizeof(float);
    b += I.n_wall() * sizeof(float);
    for (auto &C : I.comps) b += 3 * (size_t)C.V * sizeof(float);
    b += I.pml_floats() * sizeof(float);   // the absorbing layers' memories
    return b;
}

extern "C" int fdtd_llg_save_state(fdtd_llg_t h, void *buf, size_t *size)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "save_state needs an instance handle");
    Instance *I = inst_of(h);
    if (!size) return fail(h, FDTD_E_INVAL, "null size");
    const size_t need = state_bytes(*I);
    if (!buf) { *size = need; return FDTD_OK; }
    if (*size < need) { *size = need; return fail(h, FDTD_E_INVAL, "buffer too small"); }
    int rc = sync_status(h);
    if (rc) return rc;
    StateHeader hd{kMagic, 1, I->nx, I->ny, I->nz, (int32_t)I->comps.size(), h->sim->host_step, h->sim->half_ahead ? 1 : 0, 0, need};
    char *p = (char *)buf;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t nf = I->n_field();
    const size_t ncell = (size_t)I->nx * I->ny * I->nz;
    for (int f = 0; f < 6; ++f) {
        CKR(h, cudaMemcpy2D(p, I->nx * sizeof(float), I->fields[h->sim->cur] + f * nf, I->px * sizeof(float), I->nx * sizeof(float),
                            (size_t)I->ny * I->nz, cudaMemcpyDeviceToHost));
        p += ncell * sizeof(float);
    }
    CKR(h, cudaMemcpy(p, I->walls, I->n_wall() * sizeof(float), cudaMemcpyDeviceToHost));
    p += I->n_wall() * sizeof(float);
    for (auto &C : I->comps) {
        CKR(h, cudaMemcpy(p, C.m, 3 * (size_t)C.V * sizeof(float), cudaMemcpyDeviceToHost));
        p += 3 * (size_t)C.V * sizeof(float);
    }
    for (int a = 0; a < 3; ++a)
        if (I->pvol[a]) {
            CKR(h, cudaMemcpy(p, I->psi[a], 4 * (size_t)I->pvol[a] * sizeof(float), cudaMemcpyDeviceToHost));
            p += 4 * (size_t)I->pvol[a] * sizeof(float);
        }
    *size = need;
    return FDTD_OK;
}

extern "C" int fdtd_llg_load_state(fdtd_llg_t h, const void *buf, size_t size)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "load_state needs an instance handle");
    Instance *I = inst_of(h);
    if (h->sim->inst.size() > 1) return fail(h, FDTD_E_NOSYS, "load_state applies to single-instance handles");
    if (!buf || size < sizeof(StateHeader)) return fail(h, FDTD_E_INVAL, "buffer too small");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kMagic || hd.version != 1 || hd.nx != I->nx || hd.ny != I->ny || hd.nz != I->nz ||
        hd.ncomp != (int)I->comps.size() || hd.bytes != state_bytes(*I) || size < hd.bytes)
        return fail(h, FDTD_E_INVAL, "state does not match this handle");
    CKR(h, cudaStreamSynchronize(h->sim->stream));
    const char *p = (const char *)buf + sizeof hd;
    const size_t nf = I->n_field();
    const size_t ncell = (size_t)I->nx * I->ny * I->nz;
    for (int f = 0; f < 6; ++f) {
        CKR(h, cudaMemcpy2D(I->fields[h->sim->cur] + f * nf, I->px * sizeof(float), p, I->nx * sizeof(float), I->nx * sizeof(float),
                            (size_t)I->ny * I->nz, cudaMemcpyHostToDevice));
        p += ncell * sizeof(float);
    }
    CKR(h, cudaMemcpy(I->walls, p, I->n_wall() * sizeof(float), cudaMemcpyHostToDevice));
    p += I->n_wall() * sizeof(float);
    for (auto &C : I->comps) {
        CKR(h, cudaMemcpy(C.m, p, 3 * (size_t)C.V * sizeof(float), cudaMemcpyHostToDevice));
        p += 3 * (size_t)C.V * sizeof(float);
    }
    for (int a = 0; a < 3; ++a)
        if (I->pvol[a]) {
            CKR(h, cudaMemcpy(I->psi[a], p, 4 * (size_t)I->pvol[a] * sizeof(float), cudaMemcpyHostToDevice));
            p += 4 * (size_t)I->pvol[a] * sizeof(float);
        }
    Sim *S = h->sim;
    S->host_step = hd.step;
    S->half_ahead = hd.half_ahead != 0;
    CKR(h, cudaStreamSynchronize(S->stream));
    CKR(h, cudaMemsetAsync(S->d_ctl, 0, sizeof(StepCtl), S->stream));
    CKR(h, set_device_step(S->d_ctl, hd.step, S->stream));
    CKR(h, cudaStreamSynchronize(S->stream));
    return FDTD_OK;
}

// ------------------------------------------------------------- profiling
extern "C" int fdtd_llg_test_wait_timeout(fdtd_llg_t h, int32_t polls)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "set the diagnostic wait on the handle, not a member");
    if (polls < 0 || polls > (1 << 20)) return fail(h, FDTD_E_INVAL, "polls must be 0 to 2^20");
    if (polls != h->sim->test_wait) {
        h->sim->test_wait = polls;
        h->sim->dirty = true;   // graphs captured with the old launch parameters are dropped
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_magnet_cluster(fdtd_llg_t h, int32_t ctas)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "set the magnet cluster on the handle, not a member");
    if (ctas < 0 || ctas > kMagClusterMax)
        return fail(h, FDTD_E_INVAL, "magnet CTAs per region must be 0 (automatic) to " + std::to_string(kMagClusterMax));
    if (ctas != h->sim->mag_cluster) {
        h->sim->mag_cluster = ctas;
        h->sim->dirty = true;
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_get_magnet_cluster(fdtd_llg_t h, int32_t *ctas)
{
    if (!h || !h->sim || !ctas) return fail(h, FDTD_E_INVAL, "null handle or output");
    *ctas = h->sim->dirty ? 0 : (h->sim->ncomp ? h->sim->mag_cs : 0);
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_graphs(fdtd_llg_t h, int32_t mode)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "set graphs on the handle, not a member");
    if (mode < -1 || mode > 1) return fail(h, FDTD_E_INVAL, "mode must be -1, 0 or 1");
    h->sim->graph_mode = mode;
    return FDTD_OK;
}

extern "C" int fdtd_llg_get_dt(fdtd_llg_t h, double *dt)
{
    if (!h || !h->sim || !dt) return fail(h, FDTD_E_INVAL, "null handle or output");
    *dt = h->sim->dt;
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_tiling(fdtd_llg_t h, int32_t planes)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    if (!h->owns) return fail(h, FDTD_E_INVAL, "set the tiling on the batch handle, not a member");
    if (planes < 0) return fail(h, FDTD_E_INVAL, "planes must be >= 0");
    if (planes != h->sim->tiling) {
        h->sim->tiling = planes;
        h->sim->dirty = true;
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_set_tile_width(fdtd_llg_t h, int32_t width)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    if (!h->owns) return fail(h, FDTD_E_INVAL, "set the tile width on the batch handle, not a member");
    if (width != 0 && width != 32 && width != 64) return fail(h, FDTD_E_INVAL, "tile width must be 0, 32 or 64");
    if (width != h->sim->tile_width) {
        h->sim->tile_width = width;
        h->sim->dirty = true;
    }
    return FDTD_OK;
}

extern "C" int fdtd_llg_get_tile_width(fdtd_llg_t h, int32_t *width)
{
    if (!h || !h->sim || !width) return fail(h, FDTD_E_INVAL, "null handle or output");
    *width = h->sim->dirty ? 0 : h->sim->sx;
    return FDTD_OK;
}

extern "C" int fdtd_llg_get_tiling(fdtd_llg_t h, int32_t *planes)
{
    if (!h || !h->sim || !planes) return fail(h, FDTD_E_INVAL, "null handle or output");
    *planes = h->sim->dirty ? 0 : h->sim->planes;
    return FDTD_OK;
}

extern "C" int fdtd_llg_autotune(fdtd_llg_t h, int32_t trial_steps, int32_t *planes)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    if (!h->owns) return fail(h, FDTD_E_INVAL, "autotune the batch handle, not a member");
    if (trial_steps < 1) return fail(h, FDTD_E_INVAL, "trial_steps must be >= 1");
    Sim *S = h->sim;
    const int keep = S->tiling, keep_w = S->tile_width;
    int rc = fdtd_llg_set_tiling(h, 0);
    if (!rc) rc = fdtd_llg_set_tile_width(h, 0);
    if (!rc) rc = fdtd_llg_step(h, 1);   // start-up half-push and descriptors
    if (rc) return rc;
    const int w0 = S->sx;
    std::vector<int> cand = {S->planes, 8, 12, 16, 24, 32, 48, 64};
    for (int P : model_near(S, S->nsm * std::max(1, step_blocks_per_sm(false, true, S->sx)), 0.05, 12)) cand.push_back(P);
    int maxnz = 1;
    for (const Instance &I : S->inst) maxnz = std::max(maxnz, I.nz);
    for (int &c : cand) c = std::min(c, maxnz);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t e0, e1;
    CKR(h, cudaEventCreate(&e0));
    CKR(h, cudaEventCreate(&e1));
    // one setting's time: a first call of trial_steps builds its graphs (host
    // work the events would otherwise count), then the faster of two timed calls
    auto trial = [&](float &ms) -> int {
        int r = fdtd_llg_step(h, trial_steps);
        ms = -1.f;
        for (int rep = 0; rep < 2 && !r; ++rep) {
            cudaEventRecord(e0, S->stream);
            r = fdtd_llg_step(h, trial_steps);
            if (r) break;
            cudaEventRecord(e1, S->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(h, FDTD_E_CUDA, "autotune timing failed");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (ms < 0.f || t < ms) ms = t;
        }
        return r;
    };
    int best = cand[0], best_w = w0, best_cs = 0;
    float best_ms = -1.f;
    // every plane count with the width of fewest padded cells, then the other
    // width with the same counts
    for (int wi = 0; wi < 2 && !rc; ++wi) {
        const int width = wi == 0 ? w0 : (w0 == 64 ? 32 : 64);
        for (int c : cand) {
            rc = fdtd_llg_set_tiling(h, c);
            if (!rc) rc = fdtd_llg_set_tile_width(h, width);
            if (!rc) rc = fdtd_llg_step(h, 1);   // upload the new descriptors outside the timing
            float ms = 0.f;
            if (!rc) rc = trial(ms);
            if (rc) break;
            if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = c; best_w = width; }
        }
    }
    if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        fdtd_llg_set_tiling(h, keep);
        fdtd_llg_set_tile_width(h, keep_w);
        return rc;
    }
    rc = fdtd_llg_set_tiling(h, best);
    if (!rc) rc = fdtd_llg_set_tile_width(h, best_w);
    // with magnets and no split requested: the fewest magnet CTAs per region
    // against the fast split, at the chosen tiling
    if (!rc && S->ncomp && S->mag_cluster == 0 && S->mag_cs_need != S->mag_cs_fast) {
        float t[2] = {0.f, 0.f};
        const int opt[2] = {S->mag_cs_need, S->mag_cs_fast};
        for (int q = 0; q < 2 && !rc; ++q) {
            rc = fdtd_llg_set_magnet_cluster(h, opt[q]);
            if (!rc) rc = fdtd_llg_step(h, 1);
            if (!rc) rc = trial(t[q]);
        }
        if (!rc) best_cs = t[1] < t[0] ? opt[1] : opt[0];
        const int r2 = fdtd_llg_set_magnet_cluster(h, 0);
        if (!rc) rc = r2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(S)] = {best, best_w, best_cs};
        S->dirty = true;   // the tuned magnet split takes effect at the next step
    }
    if (planes) *planes = best;
    return rc;
}

extern "C" int fdtd_llg_set_profiling(fdtd_llg_t h, int32_t on)
{
    if (!h || !h->sim) return fail(h, FDTD_E_INVAL, "null handle");
    h->sim->profiling = on != 0;
    return FDTD_OK;
}

extern "C" int fdtd_llg_read_profile(fdtd_llg_t h, fdtd_llg_profile *out, int32_t reset)
{
    if (!h || !h->sim || !out) return fail(h, FDTD_E_INVAL, "null argument");
    Sim *S = h->sim;
    CKR(h, cudaStreamSynchronize(S->stream));
    for (auto &r : S->recs) {
        float ms = 0.f;
        CKR(h, cudaEventElapsedTime(&ms, r.a, r.b));
        S->prof.launches[r.kind] += 1;
        S->prof.ms[r.kind] += ms;
        S->ev_pool.push_back(r.a);
        S->ev_pool.push_back(r.b);
    }
    S->recs.clear();
    long long cells = 0;
    for (auto &I : S->inst) cells += (long long)I.nx * I.ny * I.nz;
    S->prof.cells = cells;
    *out = S->prof;
    if (reset) S->prof = fdtd_llg_profile{};
    return FDTD_OK;
}

// ------------------------------------------------ checkpointed run, adjoint
static size_t state_floats(const Instance &I)
{
    size_t totV = 0;
    for (const auto &C : I.comps) totV += C.V;
    return 6 * I.n_field() + I.n_wall() + 3 * totV;
}

// copy the present state (fields of the current buffer, walls, m) to/from dst
static cudaError_t copy_state(Sim *S, float *buf, bool save)
{
    Instance &I = S->inst[0];
    const size_t f6 = 6 * I.n_field(), nw = I.n_wall();
    size_t totV = 0;
    for (const auto &C : I.comps) totV += C.V;
    float *F = I.fields[S->cur];
    cudaError_t e = save ? cudaMemcpyAsync(buf, F, f6 * 4, cudaMemcpyDeviceToDevice, S->stream)
                         : cudaMemcpyAsync(F, buf, f6 * 4, cudaMemcpyDeviceToDevice, S->stream);
    if (e == cudaSuccess)
        e = save ? cudaMemcpyAsync(buf + f6, I.walls, nw * 4, cudaMemcpyDeviceToDevice, S->stream)
                 : cudaMemcpyAsync(I.walls, buf + f6, nw * 4, cudaMemcpyDeviceToDevice, S->stream);
    if (e == cudaSuccess && totV)
        e = save ? cudaMemcpyAsync(buf + f6 + nw, I.mbuf, 3 * totV * 4, cudaMemcpyDeviceToDevice, S->stream)
                 : cudaMemcpyAsync(I.mbuf, buf + f6 + nw, 3 * totV * 4, cudaMemcpyDeviceToDevice, S->stream);
    return e;
}

// Design-box geometry of the adjoint sets of instance I (nbe edge sites).
static long long design_set(const Instance &I, AdjSet &A)
{
    if (!I.has_design) return 0;
    A.di0 = I.dbox[0]; A.dj0 = I.dbox[1]; A.dk0 = I.dbox[2];
    A.dbx = I.dbox[3]; A.dby = I.dbox[4]; A.dbz = I.dbox[5];
    return (long long)(A.dbx + 1) * (A.dby + 1) * (A.dbz + 1);
}

extern "C" int fdtd_llg_set_tape_budget(fdtd_llg_t h, int64_t bytes)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "set_tape_budget needs the handle, not a member");
    h->sim->tape_budget = bytes < 0 ? -1 : bytes;
    return FDTD_OK;
}

extern "C" int fdtd_llg_run_checkpointed(fdtd_llg_t h, int64_t nsteps, int32_t interval)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "run_checkpointed needs the handle, not a member");
    Sim *S = h->sim;
    if (S->inst.size() != 1) return fail(h, FDTD_E_NOSYS, "the adjoint supports single-instance handles");
    if (S->inst[0].has_pml()) return fail(h, FDTD_E_NOSYS, "the adjoint does not cover absorbing layers");
    if (nsteps < 1 || interval < 0) return fail(h, FDTD_E_INVAL, "nsteps must be >= 1 and interval >= 0");
    if (S->host_step != 0) return fail(h, FDTD_E_STATE, "run_checkpointed starts at step 0 (set the materials again)");
    int rc = upload_descriptors(h);
    if (rc) return rc;
    if (S->ncomp && S->cfg.llg_fixed_iter < 2)
        return fail(h, FDTD_E_INVAL, "with magnets the adjoint needs llg_fixed_iter >= 2 (a fixed LLG map)");
    for (const MagComp &C : S->inst[0].comps) {   // the reverse magnet kernel holds a region in one CTA
        int qx, py, ps;
        if (C.V > kMagMaxV || !mag_stage_block(C.bx, C.by, C.bz, qx, py, ps))
            return fail(h, FDTD_E_NOSYS, "the adjoint covers magnetic regions of at most " + std::to_string(kMagMaxV) +
                                             " cells that fit one CTA");
    }
    const long long K = interval > 0 ? interval : (long long)std::ceil(std::sqrt((double)nsteps));
    const long long nck = (nsteps + K - 1) / K;
    const size_t sf = state_floats(S->inst[0]);
    Instance &I = S->inst[0];
    S->adj_N = 0;
    S->dfree(S->ckpt);
    S->dfree(S->tape);
    S->dfree(S->dtape);
    S->tape = S->dtape = nullptr;
    S->ckpt = (float *)S->dalloc((size_t)nck * sf * sizeof(float));
    if (!S->ckpt) return fail(h, FDTD_E_OOM, "checkpoint allocation failed");
    S->ckpt_floats = sf;
    // tapes: the trailing segments that fit the budget are recorded during
    // this run (their reverse steps need no recomputation); one more segment's
    // worth of slots serves the recomputation of the earlier ones
    const int R = std::max(2, S->cfg.llg_fixed_iter);
    const int nc = (int)I.comps.size();
    std::vector<long long> tstr(std::max(1, nc), 0);
    long long per_m = 0;
    for (int c = 0; c < nc; ++c) per_m += (tstr[c] = mag_tape_floats(I.comps[c].bx, I.comps[c].by, I.comps[c].bz, R));
    AdjSet Ad{};
    const long long per_d = 3 * design_set(I, Ad);
    auto slots = [&](long long T, long long &tail, long long &sm, long long &sd) {
        tail = T == 0 ? 0 : nsteps - (nck - T) * K;
        const long long rk = T < nck ? K : 0;
        sm = tail + (rk ? 1 + rk : 0);
        sd = tail + 1 + (rk ? rk + 1 : 0);
        return 4 * (sm * per_m + sd * per_d);
    };
    long long budget = S->tape_budget;
    if (budget < 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = (long long)(fr / 2);
    }
    long long T = 0, tail = 0, sm = 0, sd = 0;
    while (T < nck && slots(T + 1, tail, sm, sd) <= budget) ++T;
    slots(T, tail, sm, sd);
    if (per_m) S->tape = (float *)S->dalloc((size_t)(sm * per_m) * sizeof(float));
    if (per_d) S->dtape = (float *)S->dalloc((size_t)(sd * per_d) * sizeof(float));
    if ((per_m && !S->tape) || (per_d && !S->dtape)) return fail(h, FDTD_E_OOM, "adjoint tape allocation failed");
    long long off = 0;
    for (int c = 0; c < nc; ++c) {
        I.comps[c].tape = S->tape + off;
        I.comps[c].tstride = tstr[c];
        off += sm * tstr[c];
    }
    Ad.dtape = S->dtape;
    S->tail = tail;
    S->tail0 = nsteps - tail;
    S->dirty = true;
    rc = upload_descriptors(h);
    if (rc) return rc;
    if (!S->half_ahead) {
        LaunchSet L = launch_set(S);
        L.src = L.dst = S->cur;
        CKR(h, launch_half(L, S->stream));
        S->half_ahead = true;
    }
    for (long long c = 0; c < nck; ++c) {
        const long long na = c * K, ns = std::min<long long>(K, nsteps - na);
        CKR(h, copy_state(S, S->ckpt + c * sf, true));
        if (na < S->tail0) {
            rc = fdtd_llg_step(h, ns);
            if (rc) return rc;
            continue;
        }
        LaunchSet L = launch_set(S);   // recorded steps: magnet tape slot n - tail0, design slots after each step
        L.rec = 1;
        L.rec_n0 = S->tail0;
        L.rec_slots = (int)tail;
        if (na == S->tail0 && per_d) CKR(h, adj_record_design(L, Ad, 0, S->cur, S->stream));
        for (long long n = na; n < na + ns; ++n) {
            L.src = S->cur;
            L.dst = 1 - S->cur;
            CKR(h, launch_step(L, S->stream, nullptr));
            S->cur ^= 1;
            if (per_d) CKR(h, adj_record_design(L, Ad, (int)(n - S->tail0 + 1), S->cur, S->stream));
        }
        CKR(h, launch_energy_flush(L, S->rings_mapped ? S->d_rings : nullptr, S->host_step, S->host_step + ns, S->stream));
        CKR(h, stream_out(S, S->host_step, S->host_step + ns));
        S->host_step += ns;
    }
    S->adj_N = nsteps;
    S->adj_K = K;
    return FDTD_OK;
}

extern "C" int fdtd_llg_adjoint_step(fdtd_llg_t h, const double *dJ_dE, double *grad_eps, double *grad_h0)
{
    if (!h || !h->sim || !h->owns) return fail(h, FDTD_E_INVAL, "adjoint needs the handle, not a member");
    Sim *S = h->sim;
    if (S->adj_N <= 0 || !S->ckpt) return fail(h, FDTD_E_STATE, "no checkpointed run: call fdtd_llg_run_checkpointed first");
    if (!dJ_dE) return fail(h, FDTD_E_INVAL, "dJ_dE is NULL");
    Instance &I = S->inst[0];
    const long long N = S->adj_N, K = S->adj_K, nck = (N + K - 1) / K;
    const int np = (int)I.probes.size();
    const size_t nf = I.n_field(), sf = S->ckpt_floats;
    const int R = std::max(2, S->cfg.llg_fixed_iter);
    std::vector<void *> owned;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = S->dalloc(bytes);
        if (p) owned.push_back(p);
        return p;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(S->stream);
        for (void *p : owned) S->dfree(p);
    };
    AdjSet A{};
    A.lamE = (float *)alloc(3 * nf * 4);
    A.lamEn[0] = (float *)alloc(3 * nf * 4);
    A.lamEn[1] = (float *)alloc(3 * nf * 4);
    A.lamH = (float *)alloc(6 * nf * 4);
    A.lamW = (float *)alloc(I.n_wall() * 4);
    const int nc = (int)I.comps.size();
    std::vector<long long> ws_off(std::max(1, nc), 0);
    long long ws_tot = 0;
    for (int c = 0; c < nc; ++c) {
        const MagComp &C = I.comps[c];
        ws_off[c] = ws_tot;
        ws_tot += (adj_ws_floats(C.bx, C.by, C.bz, R) + 63) / 64 * 64;
    }
    A.ws = (float *)alloc(std::max<long long>(ws_tot, 1) * 4);
    long long *d_wsoff = (long long *)alloc(ws_off.size() * sizeof(long long));
    A.ws_off = d_wsoff;
    const int ngh = std::max(1, nc) * kMagClusterMax;   // one partial per magnet CTA
    A.gh0 = (double *)alloc(ngh * sizeof(double));
    const long long nseed = N * std::max(1, np) * 3;
    double *d_seed = (double *)alloc(nseed * sizeof(double));
    A.seed = d_seed;
    A.nprobe = np;
    A.nx = I.nx; A.ny = I.ny; A.nz = I.nz;
    A.R = R;
    for (int c = 0; c < nc; ++c)
        A.fnb_bytes = std::max(A.fnb_bytes, (int)(8 * mag_faces(I.comps[c].bx, I.comps[c].by, I.comps[c].bz) +
                                                  (I.comps[c].V + 15) / 16 * 16));
    // the magnet regions' faces and the edges whose curl of H reads them:
    // adj_curl_h runs beside the magnet kernel with those faces left out;
    // adj_face_fix_kernel writes their values and adds their part afterwards
    std::vector<long long> mf_lam, mf_ws, fe_off, fc_ws;
    std::vector<int> fe_comp, fe_start(1, 0);
    std::vector<float> fc_coef;
    {
        const float id[3] = {(float)(1.0 / I.dx), (float)(1.0 / I.dy), (float)(1.0 / I.dz)};
        const long long fsz = (long long)I.n_field(), plane = (long long)I.ny * I.px;
        std::map<std::pair<int, long long>, std::vector<std::pair<long long, float>>> edges;
        for (int c = 0; c < nc; ++c) {
            const MagComp &C = I.comps[c];
            std::vector<uint8_t> mat(C.V);
            if (cudaMemcpy(mat.data(), C.mat, C.V, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cleanup();
                return fail(h, FDTD_E_CUDA, "adjoint setup: reading the magnet regions failed");
            }
            const int bx = C.bx, by = C.by, bz = C.bz;
            const int nfx = (bx + 1) * by * bz, nfy = bx * (by + 1) * bz, nfz = bx * by * (bz + 1);
            auto magc = [&](int li, int lj, int lk) {
                return li >= 0 && lj >= 0 && lk >= 0 && li < bx && lj < by && lk < bz && mat[(lk * by + lj) * bx + li] != 0xFF;
            };
            for (int f = 0; f < nfx + nfy + nfz; ++f) {
                int a, fi, fj, fk;   // the magnet kernel's face numbering
                if (f < nfx) {
                    a = 0; fi = f % (bx + 1); fj = (f / (bx + 1)) % by; fk = f / ((bx + 1) * by);
                } else if (f < nfx + nfy) {
                    const int g = f - nfx;
                    a = 1; fi = g % bx; fj = (g / bx) % (by + 1); fk = g / (bx * (by + 1));
                } else {
                    const int g = f - nfx - nfy;
                    a = 2; fi = g % bx; fj = (g / bx) % by; fk = g / (bx * by);
                }
                if (!magc(fi - (a == 0), fj - (a == 1), fk - (a == 2)) && !magc(fi, fj, fk)) continue;
                const int i = C.x0 + fi, j = C.y0 + fj, k = C.z0 + fk;
                if ((a == 0 && i == I.nx) || (a == 1 && j == I.ny) || (a == 2 && k == I.nz)) continue;   // wall: the kernel writes it
                const long long wsi = ws_off[c] + adj_dq_index(bx, by, bz, f);
                mf_lam.push_back((3 + a) * fsz + k * plane + (long long)j * I.px + i);
                mf_ws.push_back(wsi);
                // the edges (component, offset) whose C_H lambda_H holds this
                // face, and its coefficient there (the curls of adj_curl_h_kernel)
                struct Term { int comp, di, dj, dk; float coef; };
                Term t[4];
                if (a == 0) { t[0] = {1, 0, 0, 0, id[2]}; t[1] = {1, 0, 0, 1, -id[2]}; t[2] = {2, 0, 0, 0, -id[1]}; t[3] = {2, 0, 1, 0, id[1]}; }
                else if (a == 1) { t[0] = {0, 0, 0, 0, -id[2]}; t[1] = {0, 0, 0, 1, id[2]}; t[2] = {2, 0, 0, 0, id[0]}; t[3] = {2, 1, 0, 0, -id[0]}; }
                else { t[0] = {0, 0, 0, 0, id[1]}; t[1] = {0, 0, 1, 0, -id[1]}; t[2] = {1, 0, 0, 0, -id[0]}; t[3] = {1, 1, 0, 0, id[0]}; }
                for (const Term &q : t) {
                    const int ei = i + q.di, ej = j + q.dj, ek = k + q.dk;
                    if (ei >= I.nx || ej >= I.ny || ek >= I.nz) continue;   // not an edge the sweep updates
                    edges[{q.comp, ek * plane + (long long)ej * I.px + ei}].push_back({wsi, q.coef});
                }
            }
        }
        for (auto &kv : edges) {
            fe_comp.push_back(kv.first.first);
            fe_off.push_back(kv.first.second);
            for (auto &cq : kv.second) {
                fc_ws.push_back(cq.first);
                fc_coef.push_back(cq.second);
            }
            fe_start.push_back((int)fc_ws.size());
        }
    }
    A.nmf = (int)mf_lam.size();
    A.nfe = (int)fe_off.size();
    // the box of every magnetic face: a face of a region box lies at cell
    // indices x0 .. x0 + bx (and so on)
    A.mlo[0] = A.mlo[1] = A.mlo[2] = 1 << 30;
    A.mhi[0] = A.mhi[1] = A.mhi[2] = -1;
    for (const MagComp &C : I.comps) {
        const int lo[3] = {C.x0, C.y0, C.z0}, hi[3] = {C.x0 + C.bx, C.y0 + C.by, C.z0 + C.bz};
        for (int a = 0; a < 3; ++a) {
            A.mlo[a] = std::min(A.mlo[a], lo[a]);
            A.mhi[a] = std::max(A.mhi[a], hi[a]);
        }
    }
    long long *d_mf = (long long *)alloc(std::max<size_t>(1, 2 * mf_lam.size()) * sizeof(long long));
    long long *d_feo = (long long *)alloc(std::max<size_t>(1, fe_off.size() + fc_ws.size()) * sizeof(long long));
    int *d_fei = (int *)alloc((fe_comp.size() + fe_start.size()) * sizeof(int));
    float *d_fcc = (float *)alloc(std::max<size_t>(1, fc_coef.size()) * sizeof(float));
    if (!d_mf || !d_feo || !d_fei || !d_fcc) { cleanup(); return fail(h, FDTD_E_OOM, "adjoint buffers: device allocation failed"); }
    A.mf_lam = d_mf; A.mf_ws = d_mf + mf_lam.size();
    A.fe_off = d_feo; A.fc_ws = d_feo + fe_off.size();
    A.fe_comp = d_fei; A.fe_start = d_fei + fe_comp.size();
    A.fc_coef = d_fcc;
    {
        cudaError_t e = cudaSuccess;
        auto up = [&](void *dst, const void *src, size_t bytes) {
            if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S->stream);
        };
        up(d_mf, mf_lam.data(), mf_lam.size() * 8);
        up(d_mf + mf_lam.size(), mf_ws.data(), mf_ws.size() * 8);
        up(d_feo, fe_off.data(), fe_off.size() * 8);
        up(d_feo + fe_off.size(), fc_ws.data(), fc_ws.size() * 8);
        up(d_fei, fe_comp.data(), fe_comp.size() * 4);
        up(d_fei + fe_comp.size(), fe_start.data(), fe_start.size() * 4);
        up(d_fcc, fc_coef.data(), fc_coef.size() * 4);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);   // before the host lists are released
        if (e != cudaSuccess) { cleanup(); return fail(h, FDTD_E_CUDA, std::string("adjoint setup: ") + cudaGetErrorString(e)); }
    }
    const long long nbe = design_set(I, A);
    if (nbe) {
        A.dtape = S->dtape;
        A.geps = (double *)alloc(3 * nbe * sizeof(double));
    }
    bool ok = A.lamE && A.lamEn[0] && A.lamEn[1] && A.lamH && A.lamW && A.ws && d_wsoff && A.gh0 && d_seed &&
              (!nbe || (A.dtape && A.geps)) && (!nc || S->tape);
    if (!ok) { cleanup(); return fail(h, FDTD_E_OOM, "adjoint buffers: device allocation failed"); }
    cudaError_t e = cudaMemsetAsync(A.lamE, 0, 3 * nf * 4, S->stream);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaMemsetAsync(A.lamEn[q], 0, 3 * nf * 4, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.lamH, 0, 6 * nf * 4, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.lamW, 0, I.n_wall() * 4, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.ws, 0, std::max<long long>(ws_tot, 1) * 4, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.gh0, 0, ngh * sizeof(double), S->stream);
    if (e == cudaSuccess && A.geps) e = cudaMemsetAsync(A.geps, 0, 3 * nbe * sizeof(double), S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_wsoff, ws_off.data(), ws_off.size() * sizeof(long long), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess && np) e = cudaMemcpyAsync(d_seed, dJ_dE, nseed * sizeof(double), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) { cleanup(); return fail(h, FDTD_E_CUDA, std::string("adjoint setup: ") + cudaGetErrorString(e)); }
    int rc = upload_descriptors(h);
    if (rc) { cleanup(); return rc; }
    LaunchSet L = launch_set(S);
    L.rec = 1;
    A.cs = std::max(1, L.mag_cs);   // the reverse magnet kernel splits regions as the forward one does
    // the second stream of the reverse steps and its two events (released,
    // after both streams drain, when this call returns)
    AdjStreams ast{};
    ast.pending = -1;
    struct StreamsGuard {
        AdjStreams &st;
        ~StreamsGuard()
        {
            if (st.b) cudaStreamSynchronize(st.b);
            if (st.a_ready) cudaEventDestroy(st.a_ready);
            if (st.mag_done) cudaEventDestroy(st.mag_done);
            if (st.b) cudaStreamDestroy(st.b);
        }
    } ast_guard{ast};
    {
        // the highest priority: the magnet kernel's cluster takes SMs before
        // the blocks of the sweeps launched beside it
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ast.b, cudaStreamNonBlocking, hi);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ast.a_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ast.mag_done, cudaEventDisableTiming);
    if (e != cudaSuccess) { cleanup(); return fail(h, FDTD_E_CUDA, std::string("adjoint setup: ") + cudaGetErrorString(e)); }
    const long long tail = S->tail, tail0 = S->tail0, base = tail + 1;
    for (long long seg = nck - 1; seg >= 0 && e == cudaSuccess; --seg) {
        const long long na = seg * K, nb = std::min(N, na + K);
        if (na >= tail0) {   // recorded during the run: tape slot n - tail0
            for (long long n = nb - 1; n >= na && e == cudaSuccess; --n)
                e = adj_reverse_step(L, A, n, (int)(n - tail0), S->stream, ast);
            continue;
        }
        // recompute the segment from its checkpoint into slots base + (n - na)
        e = copy_state(S, S->ckpt + seg * sf, false);
        // ordered on the handle's stream: earlier segments' kernels may still run
        if (e == cudaSuccess) e = set_device_step(S->d_ctl, na, S->stream);
        L.rec_n0 = na - base;
        L.rec_slots = (int)(base + K);
        if (e == cudaSuccess && nbe) e = adj_record_design(L, A, (int)base, S->cur, S->stream);
        for (long long n = na; n < nb && e == cudaSuccess; ++n) {
            L.src = S->cur;
            L.dst = 1 - S->cur;
            e = launch_step(L, S->stream, nullptr);
            S->cur ^= 1;
            if (e == cudaSuccess && nbe) e = adj_record_design(L, A, (int)(base + n - na + 1), S->cur, S->stream);
        }
        if (e == cudaSuccess) e = launch_energy_flush(L, nullptr, 0, 0, S->stream);
        for (long long n = nb - 1; n >= na && e == cudaSuccess; --n)
            e = adj_reverse_step(L, A, n, (int)(base + n - na), S->stream, ast);
        S->host_step = nb;
    }
    if (e == cudaSuccess) e = adj_finish(L, A, S->stream, ast);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ast.b);
    std::vector<double> gh(ngh, 0.0), ge(3 * nbe, 0.0);
    if (e == cudaSuccess) e = cudaMemcpy(gh.data(), A.gh0, gh.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nbe) e = cudaMemcpy(ge.data(), A.geps, ge.size() * sizeof(double), cudaMemcpyDeviceToHost);
    StepCtl st{};
    if (e == cudaSuccess) e = cudaMemcpy(&st, S->d_ctl, sizeof st, cudaMemcpyDeviceToHost);
    cudaStreamSynchronize(ast.b);   // on every path: no magnet kernel still reads the buffers freed next
    cleanup();
    if (e != cudaSuccess) return fail(h, FDTD_E_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    if (st.status & ST_UNSTABLE) return fail(h, FDTD_E_UNSTABLE, "adjoint recomputation: energy not finite");
    if (st.status & ST_TAPE) return fail(h, FDTD_E_CUDA, "adjoint recomputation: a step fell outside its tape");
    if (grad_h0) {
        double s = 0.0;
        for (int c = 0; c < nc * A.cs; ++c) s += gh[c];
        *grad_h0 = s;
    }
    if (grad_eps && I.has_design) {
        // eps of an edge = eps0 times the mean eps_r of its four cells
        const int bx = A.dbx, by = A.dby, bz = A.dbz, ex = bx + 1, ey = by + 1;
        auto g = [&](int comp, int li, int lj, int lk) { return ge[(size_t)comp * nbe + ((size_t)lk * ey + lj) * ex + li]; };
        for (int k = 0; k < bz; ++k)
            for (int j = 0; j < by; ++j)
                for (int i = 0; i < bx; ++i) {
                    double s = 0.0;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            s += g(0, i, j + a, k + b) + g(1, i + a, j, k + b) + g(2, i + a, j + b, k);
                    grad_eps[((size_t)k * by + j) * bx + i] = 0.25 * kEps0 * s;
                }
    } else if (grad_eps) {
        return fail(h, FDTD_E_STATE, "grad_eps requested but the materials have no design box");
    }
    return FDTD_OK;
}

// ---------------------------------------------- hooks for spectra.cu
namespace fl {
int fail_handle(fdtd_llg_t h, int code, const std::string &msg) { return fail(h, code, msg); }

// The device probe ring of an instance and the window of samples it holds:
// rows first .. first+count-1 (mod cap) are the states after those steps.
int probe_ring_view(fdtd_llg_t h, int32_t probe, const double **ring, int *cap, int *nprobe, long long *first,
                    int *count, double *dt, cudaStream_t *stream)
{
    if (!is_member(h)) return fail(h, FDTD_E_INVAL, "probe_spectrum needs an instance handle");
    Instance *I = inst_of(h);
    Sim *S = h->sim;
    if (probe < 0 || probe >= (int)I->probes.size()) return fail(h, FDTD_E_RANGE, "probe id out of range");
    const long long c = S->cfg.probe_capacity;
    const long long have = (I->probe_buf && I->probe_alloc == (int)I->probes.size()) ? std::min<long long>(S->host_step, c) : 0;
    *ring = I->probe_buf;
    *cap = (int)c;
    *nprobe = I->probe_alloc;
    *first = S->host_step - have;
    *count = (int)have;
    *dt = S->dt;
    *stream = S->stream;
    return FDTD_OK;
}
}  // namespace fl
