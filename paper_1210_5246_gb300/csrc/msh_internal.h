// msh_internal.h -- shared host/device declarations of libmsh (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/msh.h"

namespace msh {

// NVTX range over a call of the ABI (visible in nsys / ncu timelines; a no-op without a
// tool attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// A-posteriori fallback passes per step (see the step kernels).
constexpr int kFallbackPasses = 4;

// Device-resident time control of a grid.  The step kernels read dt and the buffer
// parity from here; the finalize kernel writes the next dt, so a run needs no host
// round trip per step.
struct Ctrl {
  double t, t_next, t_end, dt, dt_max, dt_cfl, cfl, dt_last;
  int64_t step, max_step, first_bad, hist_cap, hist_base;
  int32_t done, status, realizable;
  int32_t force;  // bit p: fallback pass p runs even if no cell of this grid was newly tagged
                  // by pass p - 1 (slabs that share the fallback of one grid); reset per step
  int32_t nbad[kFallbackPasses + 1];  // cells newly tagged by pass p of this step (p = 0: the step)
  double totals[10];
  double *hist;
  // adjoint tape: per step s in [tape_base, tape_base + tape_len) its dt and whether its
  // a-posteriori fallback tagged cells
  double *tape_dt;
  int32_t *tape_had;
  int64_t tape_base, tape_len;
  int32_t last_tagged;  // cells the a-posteriori fallback tagged in the last step
  int32_t sg_hist;      // self-gravity: the previous step's acceleration is stored
  int32_t stage_timeout;  // a 3D step kernel's bounded wait for a bulk tensor copy ran out
                          // (the step's result is void; finalize reports MSH_E_TIMEOUT)
};

// Per-thread-block partial reductions written by the step and scan kernels.
struct Partial {
  double diag[10];
  double smax;
  long long bad;
};

template <typename T> struct StepArgs {
  T *U[2];              // ping-pong state buffers, source = U[step & 1]
  const T *acc;         // gravitational acceleration -grad Phi, [3][N], or nullptr
  Ctrl *ctrl;
  Partial *part;
  int32_t *flags;       // per cell: 8 * step tag + pass of a failed update (fallback)
  int level;            // 0: the step; p >= 1: fallback pass p
  int nx, ny, nz;
  int bc[6];
  double dx[3];
  int zchunk;
  // adjoint tape: the step kernel stores U^s in ck[(s - ck_base) / ck_K] when s - ck_base
  // is a multiple of ck_K in [0, ck_len); ck = nullptr: no tape
  T *ck;
  int64_t ck_base, ck_len;
  int ck_K;
  T *U1;                // the central scheme's first-stage state (nullptr for MUSCL-Hancock)
  int units = 0;        // 3D: work units of the launch (set by the launcher)
  int test_skip = 0;    // test hook: thread block 0 does not issue its bulk copy of plane -2
};

constexpr int kTile1D = 128;   // threads per block of the 1D step kernel
constexpr int kTileX = 30;     // interior cells per warp row of the 3D kernel
constexpr int kStripX = 28;    // updated cells per warp strip of the 2D kernel

// Default length of the chunk a thread block streams: rows (2D); 3D: 0, the balanced
// tiling (work units of equal plane counts, one per resident block).
inline int default_chunk(int ndim, const int64_t n[3]) {
  if (ndim == 3) return 0;
  if (ndim == 2) return (int)(n[1] < 16 ? n[1] : 16);
  return 1;
}
constexpr int kFinalizeThreads = 256;

// launchers (msh_step.cu)
// retry = false: the step; retry = true: the fallback pass, a no-op unless the step
// tagged cells whose second-order update was not realizable
template <typename T> cudaError_t launch_step(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s,
                                              int *nblocks_out);
// the characteristic step with the Roe-type flux (same contract as launch_step)
template <typename T> cudaError_t launch_step_roe(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s,
                                                  int *nblocks_out);
template <typename T> cudaError_t launch_step_hllc(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s,
                                                  int *nblocks_out);
// the corner-transport-upwind form of the characteristic step, SCH = 0 (HLL), 3 (Roe-type)
// or 4 (HLLC); same contract as launch_step
template <typename T, int SCH> cudaError_t launch_step_ctu(const StepArgs<T> &a, int ndim, int rows, bool retry,
                                                           cudaStream_t s, int *nblocks_out);
// stage 1 or 2 of the Kurganov-Tadmor scheme (a.U1 must be set)
template <typename T> cudaError_t launch_step_kt(const StepArgs<T> &a, int ndim, int rows, int stage, cudaStream_t s);
template <typename T> int step_blocks(int ndim, int rows, int nx, int ny, int nz, int zchunk);
template <typename T> size_t step_smem(int ndim, int rows, bool ctu, bool retry);
// partials of cells [c0, c1) (c1 = 0: all N); maxf: the corner-transport-upwind CFL speed
template <typename T> cudaError_t launch_scan(const T *U, size_t N, int nx, int ny, int ndim,
                                              const double *dx, Partial *part, int nparts,
                                              cudaStream_t s, size_t c0 = 0, size_t c1 = 0,
                                              bool maxf = false);
cudaError_t launch_set_dt(Ctrl *ctrl, double dt, cudaStream_t s);
// phased steps of slabs that share the a-posteriori fallback (msh_step_begin / _retry / _end)
cudaError_t launch_force_pass(Ctrl *ctrl, int level, cudaStream_t s);
cudaError_t launch_tags(Ctrl *ctrl, int32_t *flags, size_t c0, size_t c1, int32_t *levels, bool to_grid,
                        cudaStream_t s);
cudaError_t launch_count_tags(const Ctrl *ctrl, const int32_t *flags, size_t c0, size_t c1, int level,
                              unsigned long long *count, cudaStream_t s);
cudaError_t launch_finalize(Ctrl *ctrl, const Partial *part, int nparts, int mode, cudaStream_t s);
cudaError_t launch_run_start(Ctrl *ctrl, double t_end, int64_t max_steps, double dt_max, cudaStream_t s);
cudaError_t launch_ensemble_start(Ctrl *ctrl, int64_t step_base, int64_t nsteps, int32_t *status, cudaStream_t s);
cudaError_t launch_ensemble_end(const Ctrl *ctrl, int32_t *status, cudaStream_t s);
template <typename T> cudaError_t launch_convert(T *U, size_t N, int to_primitive, cudaStream_t s);
template <typename T> cudaError_t launch_gravity_field(const double *phi, T *acc, int ndim, int nx, int ny, int nz,
                                                       const double *dx, cudaStream_t s);

constexpr int kScanBlocks = 608;  // 4 x 152 SMs
// States in flight in an ensemble run: one uploading, one computing, one downloading and
// one spare, so that no stage waits for a slot while the other two are busy.
constexpr int kEnsembleSlots = 4;

// Thread-local error text behind msh_last_error(), shared by every translation unit.
// clear_error() also resets a stale non-sticky CUDA error so that the cudaGetLastError()
// after a launch reports only that launch.
void clear_error();
void set_error_text(const char *msg);

}  // namespace msh

// Host-side state of a grid handle (the opaque msh_grid of the C ABI).

struct msh_grid {
  int ndim = 0;
  int64_t n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, dx[3] = {1, 1, 1};
  int32_t bc[6] = {0, 0, 0, 0, 0, 0};
  int prec = MSH_FP64;
  double cfl = 0.5;
  size_t N = 0;           // cells
  size_t esize = 8;       // bytes per element
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *U[2] = {nullptr, nullptr};
  double *phi = nullptr;  // potential as given (with ghost layer)
  void *acc = nullptr;    // -grad Phi, [3][N] in the state precision
  msh::Ctrl *ctrl = nullptr;   // device
  msh::Ctrl *hctrl = nullptr;  // pinned host mirror
  int32_t *hdone = nullptr;                       // pinned completion flags of two batches
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  msh::Partial *part = nullptr;
  int part_cap = 0;
  int32_t *flags = nullptr;  // per-cell fallback tags
  double *hist = nullptr;
  int64_t hist_cap = 0;
  // adjoint tape (msh_set_tape): checkpoints every tape_K steps from step tape_base
  void *tape = nullptr;
  double *tape_dt = nullptr;
  int32_t *tape_had = nullptr;
  int32_t tape_K = 0;
  int64_t tape_base = 0, tape_len = 0;
  bool tape_valid = false;
  // slab decomposition: a halo copy made the planned CFL step stale; a second control
  // block for reductions over a range of layers
  bool dt_stale = false;
  int scheme = MSH_SCHEME_MUSCL_HANCOCK;
  bool ctu = false;    // corner-transport-upwind form of the characteristic schemes
  void *U1 = nullptr;  // first Runge-Kutta stage of the central scheme
  // periodic self-gravity (msh_set_self_gravity): G > 0 when on, cuFFT plans, the FFT
  // input / spectrum / potential, the previous and the used acceleration [3][N], and a
  // device copy of the two state-buffer pointers
  double sg_G = 0.0;
  int sg_plan_fwd = 0, sg_plan_inv = 0;
  void *sg_rho = nullptr, *sg_hat = nullptr, *sg_phi = nullptr, *sg_prev = nullptr, *sg_use = nullptr;
  void *sg_eig = nullptr;  // per-axis Laplacian eigenvalues in the state precision
  void **sg_bufs = nullptr;
  msh::Ctrl *ctrl_aux = nullptr;
  bool has_state = false;
  // phased step (msh_step_begin .. msh_step_end): the pass that ran last (-1: no step open)
  // and the number of partials the step kernel wrote
  int phase_level = -1;
  int phase_nb = 0;
  int32_t test_fault = 0;  // msh_set_test_fault: applied to the next eager step launch
  unsigned long long *tag_count = nullptr;  // device counter of msh_count_tags
  int rows = 8, zchunk = 32;
  cudaGraphExec_t graph = nullptr;
  // profiling: eager launches with events around every step-kernel launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  double prof_ms = 0.0;      // summed step-kernel time
  double prof_fin_ms = 0.0;  // summed time from the step kernel's end to the finalize kernel's end
  int64_t prof_launches = 0;
  // ensemble runs: kEnsembleSlots device slots of one state each, copy-in and copy-out
  // streams, per-slot events (uploaded, result ready, downloaded) and per-state statuses
  void *ens_slot[msh::kEnsembleSlots] = {};
  cudaStream_t ens_in = nullptr, ens_out = nullptr;
  cudaEvent_t ens_ev[3 * msh::kEnsembleSlots] = {};
  int32_t *ens_status = nullptr;
  int64_t ens_status_cap = 0;
};

namespace msh {
// self-gravity (msh_selfgrav.cu): the per-step potential and acceleration, the history
// flag, plans and buffers
cudaError_t launch_self_gravity(msh_grid *g, cudaStream_t s);
cudaError_t launch_self_gravity_mark(msh_grid *g, cudaStream_t s);
msh_status setup_self_gravity(msh_grid *g, double G);
void free_self_gravity(msh_grid *g);
}  // namespace msh
