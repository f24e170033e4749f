/*
 * fdtd_llg.h -- C ABI of the B300 (sm_103a) Yee-Maxwell + LLG solver.
 *
 * Method: arxiv 2510.22221, section "Numerical Model":
 *   Ampere's law      eps0 eps_r dE/dt + sigma E = curl H - J_src   (Eq. Ampere)
 *   Faraday's law     dB/dt = -curl E,  B = mu0 (H + M)              (Eq. Faraday)
 *   LLG               dM/dt = -mu0|gamma| M x H_eff + (alpha/Ms) M x dM/dt  (Eq. LLG)
 *                     H_eff = H + H_bias, |M| = Ms
 * discretised on a staggered Yee grid with a leap-frog step: an H/M half-push
 * with curl E^n (Eq. iterate_H with the trapezoidal LLG solve of
 * Eqs. llg_tra4-6, iterated until max |M^r - M^{r-1}|/Ms < tol), the E push of
 * the Ampere update with curl H^{n+1/2} and J at t = (n+1/2) dt, and a second
 * H/M half-push with curl E^{n+1}.  Every field update runs in hand-written
 * CUDA kernels; fields are FP32, probe series, energies and gradients FP64.
 *
 * Grid and layout.  nx*ny*nz cells of size dx*dy*dz, PEC walls on all six
 * faces.  Cell (i,j,k) spans [i,i+1]x[j,j+1]x[k,k+1] in units of the cell.
 *   Ex(i,j,k) sits at (i+1/2, j, k)      Hx(i,j,k) at (i, j+1/2, k+1/2)
 *   Ey(i,j,k) at (i, j+1/2, k)           Hy(i,j,k) at (i+1/2, j, k+1/2)
 *   Ez(i,j,k) at (i, j, k+1/2)           Hz(i,j,k) at (i+1/2, j+1/2, k)
 *   M(i,j,k) at the cell centre (magnetic cells only).
 * Host arrays passed to or from the library are "compact": nx*ny*nz values,
 * i fastest, then j, then k.  Edge values in a wall are zero and are not
 * stored beyond index n-1; the normal H on the three far walls (i = nx,
 * j = ny, k = nz) is stored in separate wall arrays (FDTD_F_HX_WALL ...).
 *
 * Edge material: eps_r and sigma of an edge are the mean over its four
 * cells; an edge touching a PEC cell, or lying in a wall, holds E = 0.  The
 * E update ca E^n + cb (curl H - J) is applied in FP32 as E^n + ((ca - 1)
 * E^n + cb (curl H - J)) with ca - 1 = -sigma / (eps/dt + sigma/2), which
 * FP32 holds to full relative precision where ca next to 1 would lose a
 * weak conductor's loss to rounding.  A
 * face adjacent to a magnetic cell subtracts half of that cell's change of
 * M; H_eff at a cell centre is the mean of the two faces of each component
 * plus H_bias.  Magnetisation is held as its deviation m = M - Ms h from the
 * bias direction h = H_bias/|H_bias| (z when the bias is zero), expressed in
 * a frame whose third axis is h, so that FP32 resolves small precession
 * angles to full relative precision.
 *
 * Threading: a handle is not thread-safe; calls on one handle must be
 * serialised by the caller.  Errors: every int-returning call returns
 * FDTD_OK (0) or a negative FDTD_E_* code; fdtd_llg_last_error() returns a
 * message for the last failing call on that handle.  Kernel-side conditions
 * (LLG not converged, non-finite energy) are latched on the device and
 * reported by the next call that synchronises (fdtd_llg_sync, probe, energy,
 * get_field, save_state).
 *
 * Memory: the handle owns its device memory.  By default it is obtained with
 * cudaMalloc; a caller may supply an allocator (fdtd_llg_config.alloc/free),
 * e.g. a framework's caching allocator.  Host pointers passed in are only read
 * during the call; output buffers are caller-owned.
 */
#ifndef FDTD_LLG_H
#define FDTD_LLG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_LLG_ABI_VERSION 2

enum {
    FDTD_OK = 0,
    FDTD_E_INVAL = -1,        /* bad argument, size or geometry                */
    FDTD_E_CUDA = -2,         /* a CUDA call failed                            */
    FDTD_E_OOM = -3,          /* device or host allocation failed              */
    FDTD_E_UNSTABLE = -4,     /* dt above the Courant limit, or energy not finite */
    FDTD_E_LLG_NOCONV = -5,   /* an LLG solve did not reach llg_tol            */
    FDTD_E_STATE = -6,        /* call not valid in the handle's present state  */
    FDTD_E_RANGE = -7,        /* index out of range                            */
    FDTD_E_NOSYS = -8         /* not supported for this handle                 */
};

typedef struct fdtd_llg_s *fdtd_llg_t;

typedef void *(*fdtd_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*fdtd_free_fn)(void *ptr, void *user);

typedef struct {
    int32_t nx, ny, nz;        /* cells                                        */
    double dx, dy, dz;         /* cell size (m)                                */
    double dt;                 /* time step (s); 0: courant_factor x 3-D limit  */
    double courant_factor;     /* used when dt == 0 (e.g. 0.5; paper: 0.9)     */
    double llg_tol;            /* LLG residual tolerance; 0: 1e-6              */
    int32_t llg_max_iter;      /* 0: 20                                        */
    int32_t llg_fixed_iter;    /* > 0: exactly this many iterations, no test   */
    int32_t probe_capacity;    /* steps kept in the probe/energy rings; 0: 4096 */
    int32_t energy_every;      /* 1: energy each step; 0: never                */
    int32_t device;            /* CUDA device ordinal                          */
    void *stream;              /* cudaStream_t; NULL: a stream the handle owns  */
    fdtd_alloc_fn alloc;       /* NULL: cudaMalloc                             */
    fdtd_free_fn free;         /* NULL: cudaFree                               */
    void *alloc_user;
} fdtd_llg_config;

typedef struct {
    double eps_r;              /* relative permittivity                        */
    double sigma;              /* conductivity (S/m)                           */
    double Ms;                 /* saturation magnetisation (A/m); 0: non-magnetic */
    double alpha;              /* Gilbert damping                              */
    double gamma;              /* |gamma| (rad/(s T)), e.g. 1.76e11            */
    int32_t is_pec;            /* 1: perfect electric conductor                */
    int32_t pad_;
} fdtd_material;

/* field selectors for get_field / set_field */
enum {
    FDTD_F_EX = 0, FDTD_F_EY, FDTD_F_EZ, FDTD_F_HX, FDTD_F_HY, FDTD_F_HZ,
    FDTD_F_MX, FDTD_F_MY, FDTD_F_MZ,                  /* M (A/m), global axes      */
    FDTD_F_HX_WALL, FDTD_F_HY_WALL, FDTD_F_HZ_WALL,   /* ny*nz, nx*nz, nx*ny       */
    FDTD_F_DMX, FDTD_F_DMY, FDTD_F_DMZ                /* M - Ms h, global axes     */
};

/* Create a solver for one grid (a batch of one).  dt > Courant limit ->
 * FDTD_E_UNSTABLE.  Fields start at zero; materials must be set before the
 * first step. */
int fdtd_llg_create(const fdtd_llg_config *cfg, fdtd_llg_t *out);

/* Create n independent instances advanced together by fdtd_llg_step on the
 * returned handle (the bias-sweep pattern).  Each cfgs[i] gives an instance's
 * grid; all share dt (dt = 0 takes the smallest Courant step of the set),
 * and the device, stream, allocator and LLG settings of cfgs[0].  Instance
 * handles come from fdtd_llg_batch_member. */
int fdtd_llg_create_batch(const fdtd_llg_config *cfgs, int32_t n, fdtd_llg_t *out);

/* Handle of instance i of a batch (owned by the batch; do not destroy).
 * A single-instance handle is its own member 0. */
int fdtd_llg_batch_member(fdtd_llg_t batch, int32_t i, fdtd_llg_t *member);

/* Materials (section "Numerical Model": eps_r, sigma per cell; Ms, alpha in
 * magnets).  mat_id: nx*ny*nz bytes, compact layout, host or device pointer.
 * table: ntable <= 255 entries, host.  hbias: H_bias (A/m), host.
 * eps_r_design (nullable): per-cell eps_r over the box design_box =
 * {i0, j0, k0, ni, nj, nk} (compact in that box, host), overriding the table's
 * eps_r there.  Resets E, H to 0 and M to Ms h in magnetic cells, and the
 * batch's step count to 0.  Each face-connected magnetic region is cut
 * along its bounding box's longest axis into at most 8 slabs (one CTA of a
 * thread-block cluster each), and each slab's box must hold at most 4096
 * cells; at most 16 magnetic materials.  The distinct neighbourhoods (the
 * material ids of a cell and of the six cells below it along one or two
 * axes) are listed on the device: at most 2^20 of them.  The host reads
 * nothing per cell except, when mat_id is device memory, one copy of it.
 * Errors: FDTD_E_INVAL (an id >= ntable, bad table, box or magnet region,
 * too many distinct neighbourhoods or more than 65536 edge classes),
 * FDTD_E_OOM. */
int fdtd_llg_set_materials(fdtd_llg_t h, const uint8_t *mat_id, const fdtd_material *table,
                           int32_t ntable, const double hbias[3], const double *eps_r_design,
                           const int32_t design_box[6]);

/* Absorbing layers (the paper's device is bounded by PMLs, section
 * "Modeling Setup", which it does not formulate): the convolutional PML of
 * Roden and Gedney with the complex-frequency-shifted stretch
 * s = kappa + sigma / (alpha + j w eps0) in the first and last layers[a] cells
 * of axis a (x, y, z), inside the grid and ended by its PEC walls.  At depth
 * rho in [0, 1] (1 on the wall): sigma = scale 0.8 (order+1) / (eta0 d_a)
 * rho^order, kappa = 1 + (kappa_max - 1) rho^order, alpha = alpha_max
 * (1 - rho) (S/m).  The memories start at 0 (again at every
 * fdtd_llg_set_materials and set_pml) and are part of save_state.
 * H read back from the handle is H^{n+1/2} before the whole-step CPML term
 * of step n+1 (applied at that step's start); probes and the energy use the
 * plain midpoint H^{n}, as without layers.  layers = {0, 0, 0} removes them.
 * Errors: FDTD_E_INVAL (layers < 0 or more than half an axis, order < 0,
 * scale < 0, kappa_max < 1, alpha_max < 0, magnetic cells inside the
 * layers, a material with sigma = 2 eps / dt, where ca = 0; good conductors,
 * ca < 0, are allowed; a grid with 6 nz ny nx' >= 2^31, nx' = nx rounded up
 * to 32, beyond the layer passes' 32-bit offsets); FDTD_E_STATE after
 * fdtd_llg_run_checkpointed.  Not covered by the adjoint
 * (fdtd_llg_run_checkpointed: FDTD_E_NOSYS) nor by writes of
 * fdtd_llg_planes (FDTD_E_NOSYS). */
int fdtd_llg_set_pml(fdtd_llg_t h, const int32_t layers[3], double order, double scale, double kappa_max,
                     double alpha_max);

/* Point current density on one edge (section "Modeling Setup": modulated
 * Gaussian J = J0 exp(-(t - t_peak)^2 / (2 Tp^2)) cos(2 pi f0 t)); comp 0/1/2
 * selects an Ex/Ey/Ez edge with the indices of the layout above.  Tp = 0 ->
 * 1/f0 (one period); t_peak = 0 -> 3 Tp.  At most 4 sources per instance.
 * Adds to the sources already set. */
int fdtd_llg_set_source(fdtd_llg_t h, int32_t comp, int32_t i, int32_t j, int32_t k,
                        double J0, double f0, double Tp, double t_peak);

/* Probe at cell (i,j,k): records, after every step n, the nine values
 * Ex, Ey, Ez, Hx, Hy, Hz (the native components with index (i,j,k)) and
 * Mx, My, Mz of the cell at time n dt, in FP64 (section "Datasets Curation":
 * point samples of the fields).  At most 32 probes per instance; add probes
 * before the first step. */
int fdtd_llg_add_probe(fdtd_llg_t h, int32_t i, int32_t j, int32_t k, int32_t *id);

/* Advance nsteps full steps on the handle's stream (asynchronous; a batch
 * advances all its instances).  Kernel-side errors surface at the next
 * synchronising call. */
int fdtd_llg_step(fdtd_llg_t h, int64_t nsteps);

/* Wait for the handle's stream and report latched device errors. */
int fdtd_llg_sync(fdtd_llg_t h);

/* Copy the last min(cap_rows, steps recorded, probe_capacity) rows of probe
 * `id` to out (rows x 9 doubles, oldest first); *rows = rows written. */
int fdtd_llg_probe(fdtd_llg_t h, int32_t id, double *out, int64_t cap_rows, int64_t *rows);

/* Copy the last min(cap, steps, probe_capacity) energies
 * W = sum_edges eps E^2/2 dV + sum_faces mu0 H^2/2 dV + sum_cells mu0 (|H0| Ms - H0.M) dV
 * (oldest first, one per step) to out. */
int fdtd_llg_energy(fdtd_llg_t h, double *out, int64_t cap, int64_t *written);

/* The newest step's outputs in one call and one stream synchronisation: the
 * rows of every probe (probe_rows: nprobes x 9 doubles, in add order; may be
 * NULL) and the energy (*energy; may be NULL; 0 when the handle was created
 * without energy).  Host memory, caller-owned.  Errors: FDTD_E_INVAL (batch
 * handle), FDTD_E_STATE (no step yet), and the latched run errors of
 * fdtd_llg_sync. */
int fdtd_llg_read_last(fdtd_llg_t h, double *probe_rows, double *energy);

/* Streamed results: from the next step call on, every fdtd_llg_step (and
 * fdtd_llg_run_checkpointed) of the handle's batch queues, on the handle's
 * stream after its kernels, copies of its steps' probe rows and energies
 * into these host rings: step n's rows at rows[(n % capacity) * nprobes * 9
 * ...] (nprobes x 9 doubles, add order) and its energy at energy[n %
 * capacity].  Nothing waits for them: they are complete once a synchronising
 * call returns (fdtd_llg_sync, a read, an event recorded after the step
 * call).  Steps older than probe_capacity at the end of a call are not
 * copied.  The rings are caller-owned and must stay valid while streaming.
 * Page-locked memory (cudaHostAlloc, or registered and mapped) is written
 * directly by the kernel that ends each step call, through its device
 * address; other host memory by copies queued after it.  Either pointer may
 * be NULL; both NULL stops streaming.  The call synchronises the stream (copies
 * into earlier rings complete first).  Errors: FDTD_E_INVAL (batch handle,
 * capacity < 1). */
int fdtd_llg_stream_results(fdtd_llg_t h, double *rows, double *energy, int64_t capacity);

/* Steps completed, and whether H and M are stored half a step ahead of E
 * (1 after the first step; get_field then returns H, M at (n + 1/2) dt). */
int fdtd_llg_time_state(fdtd_llg_t h, int64_t *step, int32_t *h_half_ahead);

/* Diagnostic (section "Numerical Model", B = mu0 (H + M)): the discrete
 * divergence of B / mu0 = H + M_face at every cell centre of the present
 * state, M_face the mean of the magnetisation of the cells beside a face
 * (zero outside magnets), in FP64 from the FP32 state, into out (host,
 * caller-owned, nx*ny*nz values, compact layout).  The state holds H and M
 * half a step ahead after the first step.  The leap-frog keeps
 * div(B^n - B^0) at rounding.  Synchronises the stream.  Errors:
 * FDTD_E_INVAL (batch handle, small buffer), FDTD_E_STATE (no materials),
 * FDTD_E_CUDA. */
int fdtd_llg_div_b(fdtd_llg_t h, double *out, size_t count);

/* Read / write one field in the compact host layout (float32).  set_field
 * declares the state to be at integer time (H, M not half a step ahead).
 * FDTD_F_M* / FDTD_F_DM* entries outside magnets are zero and ignored on
 * write. */
int fdtd_llg_get_field(fdtd_llg_t h, int32_t which, float *out, size_t count);
int fdtd_llg_set_field(fdtd_llg_t h, int32_t which, const float *in, size_t count);

/* The stored state of z-planes [k0, k1) (the cells k0 .. k1-1 and their low
 * faces and edges), copied exactly between the handle and buf (host memory,
 * float32) without changing the time state: the halo exchange of one grid
 * split into z-slabs over several handles or processes (the box
 * decomposition of section "Parallelization").  to_handle = 0 reads the
 * handle into buf (after a synchronisation; latched run errors are
 * returned), 1 writes buf into the handle.  buf holds, with P = k1 - k0:
 * Ex, Ey, Ez, Hx, Hy, Hz (each P x ny x nx, compact layout), the far-wall
 * normal H of those planes (Hx at x = nx: P x ny; Hy at y = ny: P x nx), then
 * the magnetisation deviation M - Ms h of the magnetic cells in the frame of
 * the bias, as stored (3 x P x ny x nx, zero elsewhere; ignored on write
 * outside magnetic cells): P (9 nx ny + nx + ny) floats.  Errors:
 * FDTD_E_RANGE (planes outside the grid), FDTD_E_INVAL (batch handle, small
 * buffer), FDTD_E_STATE (no materials). */
int fdtd_llg_planes(fdtd_llg_t h, int32_t k0, int32_t k1, float *buf, size_t count, int32_t to_handle);

/* fdtd_llg_planes with buf in device memory (of the handle's GPU): the same
 * layout, queued on the handle's stream with no synchronisation and no host
 * round trip, so that a halo exchange between slabs stays on the GPUs (the
 * buffer then travels by NCCL send/recv or a peer copy; ghost-cell exchange
 * of section "Parallelization").  Reads see every step queued before the
 * call; writes are seen by every step queued after it.  The caller orders
 * its own use of buf with the handle's stream.  Errors as fdtd_llg_planes,
 * and FDTD_E_INVAL when buf is not device memory. */
int fdtd_llg_planes_device(fdtd_llg_t h, int32_t k0, int32_t k1, float *buf, size_t count, int32_t to_handle);

/* Checkpoint / resume of E, H, M, wall faces, step and time state.
 * buf = NULL: *size receives the byte count needed. */
int fdtd_llg_save_state(fdtd_llg_t h, void *buf, size_t *size);
int fdtd_llg_load_state(fdtd_llg_t h, const void *buf, size_t size);

/* Per-kernel device time, measured with CUDA events that the library records
 * around every launch while profiling is on (the kernels themselves are
 * unchanged).  Kinds: [0] the field sweep of a step (E push and H
 * half-push pair of every non-magnetic face), [1] the magnetic-region kernel,
 * [2] unused.  Outside profiling the two kernels of a step run side by side
 * (the sweep is a programmatic dependent launch of the magnet kernel); the
 * events between them make them run one after the other, so each is timed
 * alone. */
typedef struct {
    int64_t launches[3];
    double ms[3];              /* summed device time of those launches (ms)     */
    int64_t cells;             /* cells advanced per launch of the field sweep  */
} fdtd_llg_profile;

int fdtd_llg_set_profiling(fdtd_llg_t h, int32_t on);

/* Synchronise, add up the recorded events into *out; reset != 0 clears the
 * record afterwards. */
int fdtd_llg_read_profile(fdtd_llg_t h, fdtd_llg_profile *out, int32_t reset);

/* CUDA graphs for step calls: mode 1 replays captured graphs, 0 launches
 * kernel by kernel, -1 (default) behaves as 1 (replay shortens the gap
 * between one step's kernels and the next step's at every grid size
 * measured: 86.6 -> 84.5 us per step on 256x256x128, 537 -> 535 us on
 * 512x512x256).  A call of n >= 2 steps replays floor(n / 32) times a graph
 * of 32 steps, then a graph of the remaining n mod 32 steps; each graph is
 * captured on first use (per starting buffer) and kept until the handle's
 * launch set changes (tiling, materials, layers, sources, probes), so a
 * short call repeated costs its capture once.  A one-step call replays a
 * graph of its step and the flush that ends it.  Graphs are used only on a
 * stream that can be captured (not the legacy default stream) and never
 * while profiling.  Results are the same to the bit either way.
 * Errors: FDTD_E_INVAL. */
int fdtd_llg_set_graphs(fdtd_llg_t h, int32_t mode);

/* Magnet CTAs per magnetic region (section "Numerical Model": the LLG solve
 * of Eqs. llg_tra4-6 with Eq. iterate_H, Jacobi-iterated over a region).  A
 * region's box is split along its longest axis into `ctas` slabs, one per CTA
 * of a thread-block cluster; after each Jacobi iterate the CTAs exchange the
 * change of M of the layers beside each cut through distributed shared memory
 * and take the cluster's largest residual, so fields and M are the same to
 * the bit for every split (the energy's partial sums are grouped per CTA).
 * 0 (default): about 128 cells per CTA in the largest region while the
 * magnet CTAs of all regions number at most one per SM, and never fewer than
 * the slabs need to fit; at most 8 and at most the shortest split extent of
 * any region of the batch.  Each CTA has one thread per slab cell (128 to
 * 512).  A
 * region fits when its largest slab holds at most 4096 cells and fits one
 * CTA's shared memory, so a region's box may hold up to ~32768 cells.
 * get_magnet_cluster returns the count in effect (0 before the first step or
 * without magnets).  Errors: FDTD_E_INVAL (ctas outside 0..8; at the next
 * step, a split longer than a region or a slab too large). */
int fdtd_llg_set_magnet_cluster(fdtd_llg_t h, int32_t ctas);

/* Check of the failure path of the field sweep's bounded waits (the paper has
 * no counterpart).  Every wait of a sweep CTA for its tile copies gives up
 * after 2^22 polls: the CTA then latches a timeout in the device status,
 * stops drawing tasks, waits (bounded) for its own copies in flight and
 * exits, and the next synchronising call returns FDTD_E_CUDA ("... timed
 * out").  With polls > 0, in every following step the first sweep CTA, once
 * its first tile has landed, also waits at most `polls` polls on a
 * shared-memory barrier that nothing arrives on, and so takes that path;
 * nothing faults or hangs, the context stays usable, and the step's results
 * are incomplete.  0 (default) turns it off.  Errors: FDTD_E_INVAL. */
int fdtd_llg_test_wait_timeout(fdtd_llg_t h, int32_t polls);
int fdtd_llg_get_magnet_cluster(fdtd_llg_t h, int32_t *ctas);

/* The time step (s) shared by every instance of the handle's batch. */
int fdtd_llg_get_dt(fdtd_llg_t h, double *dt);

/* Tiling of the field sweep.  Each task of the sweep marches one column of
 * the tile shape (fdtd_llg_set_tile_width) through `planes` z-planes (the
 * last task of a column the rest); the tasks are drawn by persistent CTAs.
 * planes = 0 (the default) lets the library choose from a cost model (each
 * task also reads about 1.4 planes beyond its own, against the tail of the
 * task loop).  The tiling changes only the order in which the energy partial
 * sums are added: fields and probe samples are the same to the bit.  Takes
 * effect at the next step.  Errors: FDTD_E_INVAL (planes < 0, or a member
 * handle). */
int fdtd_llg_set_tiling(fdtd_llg_t h, int32_t planes);

/* Tile shape of the field sweep: width 64 (64 x 8 cells per task column) or
 * 32 (32 x 16), the same 512 cells and the same per-plane copies; 0 (the
 * default) takes the shape that pads the instances' x-y extents to fewer
 * cells (64 on ties).  Fields and probe samples do not depend on it.  Takes
 * effect at the next step.  Errors: FDTD_E_INVAL (not 0, 32 or 64; a member
 * handle). */
int fdtd_llg_set_tile_width(fdtd_llg_t h, int32_t width);

/* The tile width in effect; 0 before the first step or sync after materials
 * were set. */
int fdtd_llg_get_tile_width(fdtd_llg_t h, int32_t *width);

/* The z-planes per sweep task in effect (resolving planes = 0); *planes is
 * 0 before the first step or sync after materials were set. */
int fdtd_llg_get_tiling(fdtd_llg_t h, int32_t *planes);

/* Autotuner of the tiling.  Runs 3 trial_steps real steps per candidate (they
 * advance the simulation, fill the probe and energy rings and count in the
 * step number: one untimed call that builds the candidate's CUDA graphs, then
 * the faster of two timed calls) with each of a fixed list of candidate plane
 * counts (8, 12, 16, 24, 32, 48,
 * 64), the model's choice and the counts the model rates within 5 % of it
 * (at most 12: the model does not see how the tasks fill the last wave of
 * CTAs), first at the tile width of fewest padded cells and then at the
 * other width, timed with CUDA events on the handle's stream, and keeps the
 * fastest (plane count, width); the plane count is returned in *planes (may
 * be NULL), the width by fdtd_llg_get_tile_width.  The handle then holds
 * that tiling as if set with fdtd_llg_set_tiling and fdtd_llg_set_tile_width.
 * Synchronises the stream.
 * Errors: FDTD_E_INVAL (trial_steps < 1, a member handle), those of
 * fdtd_llg_step. */
int fdtd_llg_autotune(fdtd_llg_t h, int32_t trial_steps, int32_t *planes);

/* Adjoint (reverse-time) gradients of a probe objective.  Single-instance
 * handles only.
 *
 * fdtd_llg_run_checkpointed: from step 0 (right after fdtd_llg_set_materials
 * and the sources and probes), run nsteps steps like fdtd_llg_step while
 * keeping a copy of the state (E, H, walls, M: 6 field arrays + walls + 3
 * floats per magnet cell) every `interval` steps (0: ceil(sqrt(nsteps))), on
 * the device through the handle's allocator.  It also records what the
 * reverse steps read (per step: each magnet region's start state, box-edge
 * E and Jacobi iterates; E on the design-box edges) for the trailing
 * segments whose records fit the tape budget (fdtd_llg_set_tape_budget), and
 * keeps room for one more segment, into which fdtd_llg_adjoint_step
 * recomputes each earlier segment from its checkpoint.  With magnets the LLG
 * solve must be a fixed map: llg_fixed_iter >= 2 at creation.  Errors:
 * FDTD_E_INVAL, FDTD_E_STATE (not at step 0), FDTD_E_NOSYS (batch),
 * FDTD_E_OOM.
 *
 * fdtd_llg_set_tape_budget: bytes that fdtd_llg_run_checkpointed may use for
 * records taken during the run (on top of the checkpoints and of one
 * segment's records): < 0 (the default) half the free device memory at that
 * call, 0 none (every segment is recomputed once, the sqrt(N) checkpointing
 * alone).  The gradients do not depend on it.  Errors: FDTD_E_INVAL (member
 * handle).
 *
 * fdtd_llg_adjoint_step: the reverse-time counterpart of fdtd_llg_step over
 * the whole recorded run, i.e. the exact gradient of the discrete forward map
 * of that run for an objective J whose derivative with respect to the recorded probe
 * E samples is dJ_dE[n][p][c] (host, FP64, nsteps x nprobes x 3: step n's
 * row, probe p, Ex/Ey/Ez of its cell).  Reverse sweep segment by segment
 * from the last checkpoint: each segment's forward steps are recomputed
 * (recording what the reverse step needs), then reversed step by step on the
 * GPU (FP32 adjoint fields, FP64 gradient accumulation; each magnet region
 * reversed over as many CTAs of a thread-block cluster as the forward magnet
 * kernel uses, fdtd_llg_set_magnet_cluster).  Outputs, host,
 * FP64, either may be NULL: grad_eps[k][j][i], dJ/d eps_r of every cell of the
 * design box given to fdtd_llg_set_materials; *grad_h0, dJ/d |H_bias| (per
 * A/m) along the bias direction (M starts along it whatever its size).  The
 * call may be repeated with other dJ_dE; afterwards the handle's fields hold
 * the state of the run's last step or, when segments were recomputed, that
 * after the first checkpoint interval (read probes and energy before
 * calling).  Errors: FDTD_E_STATE (no checkpointed run; grad_eps without a
 * design box), FDTD_E_INVAL, FDTD_E_OOM, FDTD_E_UNSTABLE, FDTD_E_CUDA. */
int fdtd_llg_run_checkpointed(fdtd_llg_t h, int64_t nsteps, int32_t interval);
int fdtd_llg_set_tape_budget(fdtd_llg_t h, int64_t bytes);
int fdtd_llg_adjoint_step(fdtd_llg_t h, const double *dJ_dE, double *grad_eps, double *grad_h0);

/* Spectra and mode fits of probe time series (the E_x spectra behind the
 * anti-crossing maps of section "Results", the ESPRIT extraction of the
 * polariton frequencies and Q factors, and Eq. omega_pm). */

/* |sum_t w_t x_t exp(-2 pi i f t dt)| of probe `probe`, component comp (the
 * column of fdtd_llg_probe: 0-2 E, 3-5 H, 6-8 M), over the samples the ring
 * holds (the last min(steps, probe_capacity) steps, t = 0 the oldest), at
 * f = f0 + i (f1 - f0)/(nf - 1), i < nf; w = 1 (window 0) or the symmetric
 * Hann window 0.5 - 0.5 cos(2 pi t/(N-1)) (window 1).  Computed on the GPU in
 * FP64 from the device ring; out: host array of nf doubles.  Synchronises the
 * handle's stream.  Errors: FDTD_E_INVAL, FDTD_E_RANGE (probe id),
 * FDTD_E_STATE (no samples yet), FDTD_E_OOM, FDTD_E_CUDA. */
int fdtd_llg_probe_spectrum(fdtd_llg_t h, int32_t probe, int32_t comp, double f0, double f1, int32_t nf,
                            int32_t window, double *out);

/* ESPRIT on a real series x[0..n) sampled every dt (the mode extraction of
 * section "Results"): with decimate > 1 the series is first replaced by its
 * block means of `decimate` samples at step decimate dt (a moving average:
 * frequencies and decay rates of the exponentials are kept; a probe series
 * sampled far above the band of interest then spans many periods within one
 * pencil, which makes the fit well conditioned).  Then the `order` complex
 * exponentials z_k^t of the Hankel data matrix's signal subspace (pencil
 * length L = pencil, or min(n/3, 200) when pencil <= 0; needs
 * order <= L <= n - order, L <= 4096, n counted after decimation), their
 * amplitudes by least squares, and of those with positive frequency in
 * [fmin, fmax] the max_modes of largest amplitude, sorted by frequency: freq
 * (Hz), decay (1/s, amplitude ~ exp(-decay t)), amp (of the real cosine of
 * the decimated series), q = pi freq / decay.  Output arrays hold max_modes
 * doubles; *nfound receives the count.  Runs on the host in FP64; needs no
 * GPU.  Errors: FDTD_E_INVAL (message in fdtd_llg_last_error(NULL)). */
int fdtd_llg_fit_modes(const double *x, int64_t n, double dt, int32_t order, int32_t pencil, int32_t decimate,
                       double fmin, double fmax, int32_t max_modes, double *freq, double *decay, double *amp, double *q,
                       int32_t *nfound);

/* Cavity frequency f_p and coupling g of Eq. omega_pm from n >= 2 hybrid
 * pairs (f_plus[i] > f_minus[i], Hz) measured at different detunings: with
 * S = f+ + f- and D = f+ - f-, Eq. omega_pm gives D^2 - S^2 = 4 (f_p^2 + g^2)
 * - 4 f_p S, fitted by least squares.  The splitting at resonance is 2 g.
 * Host, FP64.  Errors: FDTD_E_INVAL. */
int fdtd_llg_fit_coupling(const double *f_plus, const double *f_minus, int32_t n, double *f_p, double *g);

/* E push that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (code running
 * inside another framework's memory pool, a real-time loop that forbids
 * allocation, a host that hands the library a fixed set of buffers).  It does
 * one Ampere update E = ca E + cb curl H of a uniform medium (eps_r, sigma),
 * in FP32 as E + ((ca - 1) E + cb curl H) like the solver's own update (ca - 1
 * = -sigma / (eps/dt + sigma/2) keeps its full relative precision where ca
 * next to 1 would not), with PEC walls on caller-owned device arrays in the compact layout
 * (nx*ny*nz floats each, pitch nx; wall edges stay zero) and, when w_e is not
 * NULL, writes the FP64 electric energy (eps0 eps_r / 2) sum E^2 dx dy dz of
 * the result to the device double *w_e.  Work is queued on `stream`
 * (cudaStream_t, NULL = default stream) of the current device.
 * Its per-block partial sums live in a fixed device array of 65536 doubles
 * (512 KB) that every GPU which loads the library holds until the process
 * exits; grids needing more than 65536 blocks of 32x8x16 cells are rejected
 * with FDTD_E_INVAL.  The first call on a device looks up that array's device
 * address (with that device current); make that first call before any stream
 * capture.  Every call shares the array and overwrites the slots it reads, so
 * calls that overlap on the GPU (other streams, other threads) race.  The
 * looked-up address is kept for the life of the process: after a
 * cudaDeviceReset the library must be unloaded and loaded again before this
 * entry point is used on that device.  A CUDA error already pending on the
 * calling thread is reported (FDTD_E_CUDA) and left pending.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  Errors:
 * FDTD_E_INVAL, FDTD_E_UNSTABLE (dt above the Courant limit), FDTD_E_CUDA;
 * message in fdtd_llg_last_error(NULL). */
int fdtd_llg_e_push_noalloc(float *Ex, float *Ey, float *Ez, const float *Hx, const float *Hy, const float *Hz,
                            int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz, double dt,
                            double eps_r, double sigma, double *w_e, void *stream);

/* Release everything.  NULL is accepted.  Members of a batch are released
 * with the batch. */
void fdtd_llg_destroy(fdtd_llg_t h);

/* Message of the last failing call on h (thread-local when h is NULL). */
const char *fdtd_llg_last_error(fdtd_llg_t h);

/* Version of this ABI (FDTD_LLG_ABI_VERSION). */
int fdtd_llg_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_LLG_H */
