// Internal structures shared by the host runtime and the sm_103a kernels of
// the Yee-Maxwell + LLG solver.  Not part of the public ABI.
#pragma once
#include <cstdint>
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

// Tile of the fused step kernel: kFX x kFY columns marching kFC(runtime)
// planes in z, kFT threads; shared-memory planes of H with a one-cell halo on
// the low x and y sides plus the high extension, and of E^{n+1} on the tile
// extended by one cell on the high x and y sides.
constexpr int kFX = 64, kFY = 16, kFT = 256;
constexpr int kHX = kFX + 2, kHY = kFY + 2, kHN = kHX * kHY;
constexpr int kEX = kFX + 1, kEY = kFY + 1, kEN = kEX * kEY;
constexpr int kHQ = (kHN + kFT - 1) / kFT;
constexpr int kEQ = (kEN + kFT - 1) / kFT;
constexpr int kIQ = kFX * kFY / kFT;
constexpr int kFusedPlanes = 16;   // z planes per fused-step tile

// Magnet kernel: one CTA per face-connected magnetic region, whose bounding
// box holds at most kMagMaxV cells, kMagCPT cells per thread.
constexpr int kMagThreads = 512;
constexpr int kMagMaxV = 4096;
constexpr int kMagCPT = kMagMaxV / kMagThreads;

// Class-table entry flags (bit field stored in the .w of the first float4).
enum : uint32_t { CF_MAG_HX = 1u, CF_MAG_HY = 2u, CF_MAG_HZ = 4u };

struct MagMat {
    float Ms, inv_Ms, alpha, kappa;   // kappa = mu0 |gamma| (dt/2) / 2
};

// Everything a kernel needs about one grid instance.
struct Inst {
    float *F[2][6];                       // two buffers of Ex, Ey, Ez, Hx, Hy, Hz: [nz][ny][px]
    long long fstride;                    // F[b][c] = F[b][0] + c * fstride
    float *wHx, *wHy, *wHz;               // far-wall normal H: [nz][ny], [nz][nx], [ny][nx]
    const void *cls;                      // class id per cell: uint8 or uint16
    const float4 *ctab;                   // 3 float4 per class: (ca, flags) (cb) (eps/2)
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
    int ftile_off, fntx, fnty, fntz, fkc; // fused-step tiles (kFX x kFY x fkc)
    int mag_off, nmag;                    // magnet regions of this instance
    MagMat mm[kMaxMagMat];
};

struct MagComp {
    int inst;
    int x0, y0, z0, bx, by, bz, V;
    float *m;               // deviation M - Ms h in the bias frame: 3 blocks of V
    const uint8_t *mat;     // V: magnet material index, 0xFF outside this region
    float *fcurl;           // scratch: curl E at the region's faces (x, y, z face blocks)
};

// Device-resident control block of a batch.
struct StepCtl {
    long long step;         // completed steps
    unsigned int counter;   // CTAs of the H pass that have finished this step
    int status;             // latched error bits (ST_*)
};
enum : int { ST_NOCONV = 1, ST_UNSTABLE = 2 };

struct LaunchSet {
    const Inst *insts;
    int ninst;
    const int *tile_inst;
    int ntiles;
    const MagComp *comps;
    int ncomp;
    int vmax;
    StepCtl *ctl;
    double *part_f, *part_m;            // energy partials per fused tile / per region
    const int *ftile_inst;
    int nftiles;
    int src, dst;                       // field buffers read / written by a step
    int grid_h;
    bool cls16;
    float llg_tol;
    int llg_max_iter, llg_fixed_iter;
    int energy;
};

// Launchers (kernels_fwd.cu).  launch_half: the start-up H/M half-push that
// moves H, M from integer time to half a step ahead, in place on buffer src.
// launch_step: one full step reading buffer src and writing buffer dst, the
// field kernel on s and the magnetic regions concurrently on s_mag (events
// ev_fork / ev_join order them with the surrounding work on s).
cudaError_t launch_half(const LaunchSet &L, cudaStream_t s);
cudaError_t launch_step(const LaunchSet &L, cudaStream_t s, cudaStream_t s_mag, cudaEvent_t ev_fork,
                        cudaEvent_t ev_join, cudaEvent_t *prof);
int h_half_blocks_per_sm(bool cls16);

// fdtd_llg_last_error(NULL) message for entry points without a handle.
void set_last_error(const char *msg);

}  // namespace fl
