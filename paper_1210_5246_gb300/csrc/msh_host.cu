// msh_host.cu -- C ABI of libmsh: grid lifecycle, state transfer, step/run control.
//
// A grid owns two state buffers (ping-pong by step parity), a device control block
// (time, dt, step counter, stop flags), per-block reduction partials and a cached CUDA
// graph holding kGraphSteps consecutive (step, finalize) launch pairs.  msh_run launches
// that graph until the device control block reports completion; kernels of a finished
// run return immediately, so over-launching past t_end is harmless.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/msh.h"
#include "msh_internal.h"

using namespace msh;

namespace {
thread_local std::string g_err;
}  // namespace

void msh::clear_error() {
  g_err.clear();
  (void)cudaGetLastError();
}

void msh::set_error_text(const char *msg) { g_err = msg; }

namespace {

void begin() { clear_error(); }

msh_status fail(msh_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (e_ == cudaErrorMemoryAllocation) return fail(MSH_E_NOMEM, "%s: %s", #expr, cudaGetErrorString(e_)); \
      return fail(MSH_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));                    \
    }                                                                                      \
  } while (0)

constexpr int kGraphSteps = 16;

}  // namespace


// ---------------------------------------------------------------- helpers
namespace {

template <typename T> StepArgs<T> make_args(msh_grid *g) {
  StepArgs<T> a;
  a.U[0] = (T *)g->U[0];
  a.U[1] = (T *)g->U[1];
  a.acc = (const T *)(g->sg_G > 0.0 ? g->sg_use : g->acc);
  a.ctrl = g->ctrl;
  a.part = g->part;
  a.flags = g->flags;
  a.nx = (int)g->n[0];
  a.ny = (int)g->n[1];
  a.nz = (int)g->n[2];
  for (int i = 0; i < 6; i++) a.bc[i] = g->bc[i];
  for (int i = 0; i < 3; i++) a.dx[i] = g->dx[i];
  a.zchunk = g->zchunk;
  a.level = 0;
  a.ck = g->tape_valid ? (T *)g->tape : nullptr;
  a.ck_base = g->tape_base;
  a.ck_len = g->tape_len;
  a.ck_K = g->tape_K > 0 ? g->tape_K : 1;
  a.U1 = (T *)g->U1;
  return a;
}

int blocks_for(msh_grid *g, int rows, int zchunk) {
  if (g->prec == MSH_FP32) return step_blocks<float>(g->ndim, rows, (int)g->n[0], (int)g->n[1], (int)g->n[2], zchunk);
  return step_blocks<double>(g->ndim, rows, (int)g->n[0], (int)g->n[1], (int)g->n[2], zchunk);
}

msh_status ensure_partials(msh_grid *g, int need) {
  if (need <= g->part_cap) return MSH_OK;
  if (g->part) cudaFree(g->part);
  g->part = nullptr;
  g->part_cap = 0;
  CUDA_TRY(cudaMalloc(&g->part, sizeof(Partial) * (size_t)need));
  g->part_cap = need;
  return MSH_OK;
}

void drop_graph(msh_grid *g) {
  if (g->graph) cudaGraphExecDestroy(g->graph);
  g->graph = nullptr;
}

// Copy the tape fields of the host mirror (the tail of Ctrl) to the device control block.
cudaError_t push_tape_fields(msh_grid *g) {
  const size_t off = offsetof(Ctrl, tape_dt);
  return cudaMemcpyAsync(reinterpret_cast<char *>(g->ctrl) + off, reinterpret_cast<char *>(g->hctrl) + off,
                         sizeof(Ctrl) - off, cudaMemcpyHostToDevice, g->stream);
}

// A new state or time ends the recorded trajectory: stop recording, keep the memory.
msh_status stop_tape(msh_grid *g) {
  if (!g->tape_valid) return MSH_OK;
  g->tape_valid = false;
  g->hctrl->tape_dt = nullptr;
  g->hctrl->tape_had = nullptr;
  g->hctrl->tape_len = 0;
  drop_graph(g);  // the graph's step arguments point at the tape
  CUDA_TRY(push_tape_fields(g));
  return MSH_OK;
}

void free_tape(msh_grid *g) {
  if (g->tape) cudaFree(g->tape);
  if (g->tape_dt) cudaFree(g->tape_dt);
  if (g->tape_had) cudaFree(g->tape_had);
  g->tape = nullptr;
  g->tape_dt = nullptr;
  g->tape_had = nullptr;
  g->tape_K = 0;
  g->tape_len = 0;
  g->tape_valid = false;
}

// One pass of the characteristic step with the grid's flux (HLL, Roe-type or HLLC).
template <typename T>
static cudaError_t launch_characteristic(msh_grid *g, const StepArgs<T> &a, bool retry, int *nblocks_out) {
  if (g->ctu) {  // the corner-transport-upwind form
    if (g->scheme == MSH_SCHEME_MUSCL_HANCOCK_ROE)
      return launch_step_ctu<T, 3>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
    if (g->scheme == MSH_SCHEME_MUSCL_HANCOCK_HLLC)
      return launch_step_ctu<T, 4>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
    return launch_step_ctu<T, 0>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
  }
  if (g->scheme == MSH_SCHEME_MUSCL_HANCOCK_ROE)
    return launch_step_roe<T>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
  if (g->scheme == MSH_SCHEME_MUSCL_HANCOCK_HLLC)
    return launch_step_hllc<T>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
  return launch_step<T>(a, g->ndim, g->rows, retry, g->stream, nblocks_out);
}

msh_status launch_one_step(msh_grid *g, int ev_slot) {
  g->phase_level = -1;  // a whole step closes a phased one that was left open
  int nb = 0;
  cudaError_t e;
  if (g->sg_G > 0.0) {  // the potential of U^n and the step's acceleration
    e = launch_self_gravity(g, g->stream);
    if (e == cudaSuccess) e = launch_self_gravity_mark(g, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "self-gravity: %s", cudaGetErrorString(e));
  }
  if (g->profiling && ev_slot >= 0) CUDA_TRY(cudaEventRecord(g->ev[3 * ev_slot], g->stream));
  if (g->scheme == MSH_SCHEME_KT) {
    // the two Runge-Kutta stages of the central scheme, then the finalize (no fallback)
    nb = blocks_for(g, g->rows, g->zchunk);
    for (int stage = 1; stage <= 2; stage++) {
      e = g->prec == MSH_FP32 ? launch_step_kt<float>(make_args<float>(g), g->ndim, g->rows, stage, g->stream)
                              : launch_step_kt<double>(make_args<double>(g), g->ndim, g->rows, stage, g->stream);
      if (e != cudaSuccess) return fail(MSH_E_CUDA, "central scheme stage %d launch: %s", stage, cudaGetErrorString(e));
    }
    if (g->profiling && ev_slot >= 0) CUDA_TRY(cudaEventRecord(g->ev[3 * ev_slot + 1], g->stream));
    e = launch_finalize(g->ctrl, g->part, nb, 0, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "finalize launch: %s", cudaGetErrorString(e));
    if (g->profiling && ev_slot >= 0) CUDA_TRY(cudaEventRecord(g->ev[3 * ev_slot + 2], g->stream));
    return MSH_OK;
  }
  // the characteristic step (HLL, Roe-type or HLLC flux), then its fallback passes: each
  // returns at once unless the previous pass tagged new cells
  const int32_t test_fault = g->test_fault;
  g->test_fault = 0;  // a test hook applies to one step
  for (int level = 0; level <= kFallbackPasses; level++) {
    const bool retry = level > 0;
    if (g->prec == MSH_FP32) {
      StepArgs<float> a = make_args<float>(g);
      a.level = level;
      a.test_skip = level == 0 && test_fault == 1;
      e = launch_characteristic(g, a, retry, retry ? nullptr : &nb);
    } else {
      StepArgs<double> a = make_args<double>(g);
      a.level = level;
      a.test_skip = level == 0 && test_fault == 1;
      e = launch_characteristic(g, a, retry, retry ? nullptr : &nb);
    }
    if (e != cudaSuccess)
      return fail(MSH_E_CUDA, "%s kernel launch: %s", retry ? "fallback" : "step", cudaGetErrorString(e));
    if (level == 0 && g->profiling && ev_slot >= 0) CUDA_TRY(cudaEventRecord(g->ev[3 * ev_slot + 1], g->stream));
  }
  e = launch_finalize(g->ctrl, g->part, nb, 0, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "finalize launch: %s", cudaGetErrorString(e));
  if (g->profiling && ev_slot >= 0) CUDA_TRY(cudaEventRecord(g->ev[3 * ev_slot + 2], g->stream));
  return MSH_OK;
}

msh_status build_graph(msh_grid *g) {
  if (g->graph) return MSH_OK;
  const int32_t test_fault = g->test_fault;  // test hooks never enter a graph
  g->test_fault = 0;
  struct Restore {
    msh_grid *g;
    int32_t v;
    ~Restore() { g->test_fault = v; }
  } restore{g, test_fault};
  msh_status st = ensure_partials(g, blocks_for(g, g->rows, g->zchunk));
  if (st) return st;
  cudaGraph_t graph;
  CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kGraphSteps; i++) {
    st = launch_one_step(g, i);
    if (st) {
      cudaStreamEndCapture(g->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
  }
  CUDA_TRY(cudaStreamEndCapture(g->stream, &graph));
  cudaError_t e = cudaGraphInstantiate(&g->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return MSH_OK;
}

msh_status read_ctrl(msh_grid *g) {
  CUDA_TRY(cudaMemcpyAsync(g->hctrl, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

void collect_profile(msh_grid *g, int slots) {
  if (!g->profiling) return;
  for (int i = 0; i < slots; i++) {
    float ms = 0.f;
    float ms2 = 0.f;
    if (cudaEventElapsedTime(&ms, g->ev[3 * i], g->ev[3 * i + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms2, g->ev[3 * i + 1], g->ev[3 * i + 2]) == cudaSuccess) {
      g->prof_ms += ms;
      g->prof_fin_ms += ms2;
      g->prof_launches += 1;
    } else {
      (void)cudaGetLastError();
    }
  }
}

// Scan the buffer `which` and run the finalize kernel in mode 1 (no time advance).
msh_status prime(msh_grid *g, int which) {
  msh_status st = ensure_partials(g, kScanBlocks);
  if (st) return st;
  cudaError_t e;
  if (g->prec == MSH_FP32)
    e = launch_scan<float>((const float *)g->U[which], g->N, (int)g->n[0], (int)g->n[1], g->ndim, g->dx, g->part,
                           kScanBlocks, g->stream, 0, 0, g->ctu);
  else
    e = launch_scan<double>((const double *)g->U[which], g->N, (int)g->n[0], (int)g->n[1], g->ndim, g->dx,
                            g->part, kScanBlocks, g->stream, 0, 0, g->ctu);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "scan launch: %s", cudaGetErrorString(e));
  e = launch_finalize(g->ctrl, g->part, kScanBlocks, 1, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "finalize launch: %s", cudaGetErrorString(e));
  return read_ctrl(g);
}

int cur_buf(msh_grid *g) { return (int)(g->hctrl->step & 1); }

void free_ensemble(msh_grid *g) {
  if (g->ens_in) cudaStreamSynchronize(g->ens_in);
  if (g->ens_out) cudaStreamSynchronize(g->ens_out);
  for (auto &b : g->ens_slot) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  for (auto &e : g->ens_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (g->ens_in) cudaStreamDestroy(g->ens_in);
  if (g->ens_out) cudaStreamDestroy(g->ens_out);
  if (g->ens_status) cudaFree(g->ens_status);
  g->ens_in = g->ens_out = nullptr;
  g->ens_status = nullptr;
  g->ens_status_cap = 0;
}

// Slots, streams, events and a status array for `count` states.
msh_status ensure_ensemble(msh_grid *g, int64_t count) {
  const size_t bytes = g->N * 10 * g->esize;
  for (auto &b : g->ens_slot)
    if (!b && cudaMalloc(&b, bytes) != cudaSuccess) {
      cudaGetLastError();
      free_ensemble(g);
      return fail(MSH_E_NOMEM, "ensemble slots (%d x %zu bytes)", kEnsembleSlots, bytes);
    }
  if (!g->ens_in) CUDA_TRY(cudaStreamCreateWithFlags(&g->ens_in, cudaStreamNonBlocking));
  if (!g->ens_out) CUDA_TRY(cudaStreamCreateWithFlags(&g->ens_out, cudaStreamNonBlocking));
  for (auto &e : g->ens_ev)
    if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (g->ens_status_cap < count) {
    if (g->ens_status) cudaFree(g->ens_status);
    g->ens_status = nullptr;
    g->ens_status_cap = 0;
    if (cudaMalloc(&g->ens_status, sizeof(int32_t) * (size_t)count) != cudaSuccess) {
      cudaGetLastError();
      return fail(MSH_E_NOMEM, "ensemble statuses");
    }
    g->ens_status_cap = count;
  }
  return MSH_OK;
}

// After msh_set_slab the planned CFL step belongs to the state before the copy.
msh_status refresh_dt(msh_grid *g) {
  if (!g->dt_stale) return MSH_OK;
  msh_status st = prime(g, cur_buf(g));
  if (st == MSH_OK) g->dt_stale = false;
  return st;
}

// Cells per layer of the last active axis, and the number of layers.
void layer_geometry(const msh_grid *g, size_t *per_layer, int64_t *layers) {
  const int ax = g->ndim - 1;
  size_t p = 1;
  for (int d = 0; d < ax; d++) p *= (size_t)g->n[d];
  *per_layer = p;
  *layers = g->n[ax];
}

}  // namespace

// ------------------------------------------------------------------- ABI
extern "C" {

const char *msh_last_error(void) { return g_err.c_str(); }

int32_t msh_version(void) { return 10000; }

msh_status msh_init_grid(msh_grid **out, int32_t ndim, const int64_t n[3], const double lo[3],
                         const double hi[3], const int32_t bc[6], int32_t precision, double cfl, void *stream) {
  begin();
  if (!out || !n || !lo || !hi || !bc) return fail(MSH_E_INVALID_ARG, "null argument");
  if (ndim < 1 || ndim > 3) return fail(MSH_E_INVALID_ARG, "ndim must be 1, 2 or 3 (got %d)", ndim);
  if (precision != MSH_FP32 && precision != MSH_FP64) return fail(MSH_E_INVALID_ARG, "bad precision %d", precision);
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(MSH_E_INVALID_ARG, "cfl must be in (0, 1] (got %g)", cfl);
  for (int d = 0; d < 3; d++) {
    if (d < ndim) {
      if (n[d] < 2) return fail(MSH_E_INVALID_ARG, "n[%d] must be >= 2", d);
      if (!(hi[d] > lo[d])) return fail(MSH_E_INVALID_ARG, "hi[%d] must exceed lo[%d]", d, d);
      for (int s = 0; s < 2; s++)
        if (bc[2 * d + s] < 0 || bc[2 * d + s] > 2) return fail(MSH_E_INVALID_ARG, "bad bc[%d]", 2 * d + s);
      if ((bc[2 * d] == MSH_BC_PERIODIC) != (bc[2 * d + 1] == MSH_BC_PERIODIC))
        return fail(MSH_E_INVALID_ARG, "periodic boundary of dim %d must be paired", d);
    } else if (n[d] != 1) {
      return fail(MSH_E_INVALID_ARG, "n[%d] must be 1 for an unused dimension", d);
    }
  }
  const double cells = (double)n[0] * (double)n[1] * (double)n[2];
  if (cells * 10.0 > 2147483647.0 * 8.0) return fail(MSH_E_INVALID_ARG, "grid too large");
  if (n[0] > (1 << 30) || n[1] > (1 << 30) || n[2] > (1 << 30)) return fail(MSH_E_INVALID_ARG, "grid too large");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return fail(MSH_E_CUDA, "no CUDA device available (libmsh has no CPU path)");
  msh_grid *g = new (std::nothrow) msh_grid();
  if (!g) return fail(MSH_E_NOMEM, "host allocation");
  g->ndim = ndim;
  for (int d = 0; d < 3; d++) {
    g->n[d] = n[d];
    g->lo[d] = d < ndim ? lo[d] : 0.0;
    g->hi[d] = d < ndim ? hi[d] : 1.0;
    g->dx[d] = (g->hi[d] - g->lo[d]) / (double)n[d];
  }
  for (int i = 0; i < 6; i++) g->bc[i] = (i < 2 * ndim) ? bc[i] : MSH_BC_PERIODIC;
  g->prec = precision;
  g->esize = precision == MSH_FP32 ? 4 : 8;
  g->cfl = cfl;
  g->N = (size_t)n[0] * n[1] * n[2];
  g->zchunk = default_chunk(ndim, n);
  g->rows = 8;
  auto cleanup = [&](msh_status s) {
    msh_destroy(g);
    return s;
  };
  cudaError_t e;
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(MSH_E_CUDA, "stream create: %s", cudaGetErrorString(e)));
    g->own_stream = true;
  }
  const size_t bytes = g->N * 10 * g->esize;
  for (int b = 0; b < 2; b++) {
    e = cudaMalloc(&g->U[b], bytes);
    if (e != cudaSuccess) return cleanup(fail(MSH_E_NOMEM, "state buffer (%zu bytes): %s", bytes, cudaGetErrorString(e)));
  }
  e = cudaMalloc(&g->flags, g->N * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->flags, 0, g->N * sizeof(int32_t), g->stream);
  if (e != cudaSuccess) return cleanup(fail(MSH_E_NOMEM, "fallback tags: %s", cudaGetErrorString(e)));
  e = cudaMalloc(&g->ctrl, sizeof(Ctrl));
  if (e != cudaSuccess) return cleanup(fail(MSH_E_NOMEM, "control block: %s", cudaGetErrorString(e)));
  e = cudaMallocHost(&g->hctrl, sizeof(Ctrl));
  if (e != cudaSuccess) return cleanup(fail(MSH_E_NOMEM, "pinned control block: %s", cudaGetErrorString(e)));
  e = cudaMallocHost(&g->hdone, 2 * sizeof(int32_t));
  if (e != cudaSuccess) return cleanup(fail(MSH_E_NOMEM, "pinned flags: %s", cudaGetErrorString(e)));
  for (auto &ev : g->ev_done) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(fail(MSH_E_CUDA, "event create: %s", cudaGetErrorString(e)));
  }
  memset(g->hctrl, 0, sizeof(Ctrl));
  g->hctrl->cfl = cfl;
  g->hctrl->t_end = INFINITY;
  g->hctrl->dt_max = INFINITY;
  g->hctrl->done = 1;
  g->hctrl->first_bad = -1;
  e = cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cleanup(fail(MSH_E_CUDA, "control init: %s", cudaGetErrorString(e)));
  msh_status st = ensure_partials(g, std::max(kScanBlocks, blocks_for(g, g->rows, g->zchunk)));
  if (st) return cleanup(st);
  *out = g;
  return MSH_OK;
}

msh_status msh_destroy(msh_grid *g) {
  if (!g) return MSH_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  drop_graph(g);
  for (auto &e : g->ev) cudaEventDestroy(e);
  for (int b = 0; b < 2; b++)
    if (g->U[b]) cudaFree(g->U[b]);
  if (g->phi) cudaFree(g->phi);
  if (g->acc) cudaFree(g->acc);
  if (g->ctrl) cudaFree(g->ctrl);
  if (g->hctrl) cudaFreeHost(g->hctrl);
  if (g->hdone) cudaFreeHost(g->hdone);
  for (auto &e : g->ev_done)
    if (e) cudaEventDestroy(e);
  if (g->part) cudaFree(g->part);
  if (g->flags) cudaFree(g->flags);
  if (g->hist) cudaFree(g->hist);
  if (g->ctrl_aux) cudaFree(g->ctrl_aux);
  if (g->tag_count) cudaFree(g->tag_count);
  if (g->U1) cudaFree(g->U1);
  free_self_gravity(g);
  free_tape(g);
  free_ensemble(g);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return MSH_OK;
}

msh_status msh_set_state(msh_grid *g, const void *U, int32_t where, int32_t kind) {
  msh::NvtxRange nvtx_range("msh_set_state");
  begin();
  if (!g || !U) return fail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return fail(MSH_E_INVALID_ARG, "bad where");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return fail(MSH_E_INVALID_ARG, "bad kind");
  msh_status st0 = stop_tape(g);
  if (st0) return st0;
  const int cur = cur_buf(g), nxt = cur ^ 1;
  const size_t bytes = g->N * 10 * g->esize;
  CUDA_TRY(cudaMemcpyAsync(g->U[nxt], U, bytes, where == MSH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           g->stream));
  if (kind == MSH_PRIMITIVE) {
    cudaError_t e = g->prec == MSH_FP32 ? launch_convert<float>((float *)g->U[nxt], g->N, 0, g->stream)
                                        : launch_convert<double>((double *)g->U[nxt], g->N, 0, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
  }
  // fallback tags are step numbers; a new state must not see tags of an earlier trajectory
  CUDA_TRY(cudaMemsetAsync(g->flags, 0, g->N * sizeof(int32_t), g->stream));
  msh_status st = prime(g, nxt);
  if (st) return st;
  if (!g->hctrl->realizable) {
    const int64_t bad = g->hctrl->first_bad;
    // restore the control block's view of the old state
    if (g->has_state) prime(g, cur);
    return fail(MSH_E_REALIZABILITY, "state not realizable at cell %lld (rho <= 0 or P not SPD)", (long long)bad);
  }
  CUDA_TRY(cudaMemcpyAsync(g->U[cur], g->U[nxt], bytes, cudaMemcpyDeviceToDevice, g->stream));
  // a new state has no previous self-gravity acceleration
  g->hctrl->sg_hist = 0;
  CUDA_TRY(cudaMemsetAsync(&g->ctrl->sg_hist, 0, sizeof(int32_t), g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  g->has_state = true;
  return MSH_OK;
}

msh_status msh_get_state(msh_grid *g, void *U, int32_t where, int32_t kind) {
  msh::NvtxRange nvtx_range("msh_get_state");
  begin();
  if (!g || !U) return fail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return fail(MSH_E_INVALID_ARG, "bad where");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return fail(MSH_E_INVALID_ARG, "bad kind");
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  const int cur = cur_buf(g), nxt = cur ^ 1;
  const size_t bytes = g->N * 10 * g->esize;
  const void *src = g->U[cur];
  if (kind == MSH_PRIMITIVE) {
    CUDA_TRY(cudaMemcpyAsync(g->U[nxt], g->U[cur], bytes, cudaMemcpyDeviceToDevice, g->stream));
    cudaError_t e = g->prec == MSH_FP32 ? launch_convert<float>((float *)g->U[nxt], g->N, 1, g->stream)
                                        : launch_convert<double>((double *)g->U[nxt], g->N, 1, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
    src = g->U[nxt];
  }
  CUDA_TRY(cudaMemcpyAsync(U, src, bytes, where == MSH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_run_ensemble(msh_grid *g, int64_t count, const void *const *in, void *const *out, int32_t kind,
                            int64_t nsteps, int32_t *status) {
  msh::NvtxRange nvtx_range("msh_run_ensemble");
  begin();
  if (!g || (count > 0 && (!in || !out))) return fail(MSH_E_INVALID_ARG, "null argument");
  if (count < 0 || nsteps < 1) return fail(MSH_E_INVALID_ARG, "count must be >= 0 and nsteps >= 1");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return fail(MSH_E_INVALID_ARG, "bad kind");
  for (int64_t k = 0; k < count; k++)
    if (!in[k] || !out[k]) return fail(MSH_E_INVALID_ARG, "null state pointer %lld", (long long)k);
  if (count == 0) return MSH_OK;
  msh_status st = stop_tape(g);
  if (st) return st;
  st = ensure_ensemble(g, count);
  if (st) return st;
  st = ensure_partials(g, std::max(kScanBlocks, blocks_for(g, g->rows, g->zchunk)));
  if (st) return st;
  const size_t bytes = g->N * 10 * g->esize;
  const bool fp32 = g->prec == MSH_FP32;
  // the device step counter continues from the grid's; state k starts at base + k * nsteps,
  // so its input goes to buffer (step & 1) and its result comes from ((step + nsteps) & 1)
  int64_t base = g->hctrl->step;
  cudaEvent_t *ev_in = g->ens_ev, *ev_done = g->ens_ev + kEnsembleSlots, *ev_free = g->ens_ev + 2 * kEnsembleSlots;
  for (int64_t k = 0; k < count; k++) {
    const int j = (int)(k % kEnsembleSlots);
    void *slot = g->ens_slot[j];
    // upload: slot j is free once the download of state k - kEnsembleSlots has finished
    if (k >= kEnsembleSlots) CUDA_TRY(cudaStreamWaitEvent(g->ens_in, ev_free[j], 0));
    CUDA_TRY(cudaMemcpyAsync(slot, in[k], bytes, cudaMemcpyHostToDevice, g->ens_in));
    CUDA_TRY(cudaEventRecord(ev_in[j], g->ens_in));
    // the steps, on the grid's stream
    CUDA_TRY(cudaStreamWaitEvent(g->stream, ev_in[j], 0));
    cudaError_t e = cudaSuccess;
    if (kind == MSH_PRIMITIVE)
      e = fp32 ? launch_convert<float>((float *)slot, g->N, 0, g->stream)
               : launch_convert<double>((double *)slot, g->N, 0, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
    const int64_t s0 = base + k * nsteps;
    void *src = g->U[s0 & 1];
    CUDA_TRY(cudaMemcpyAsync(src, slot, bytes, cudaMemcpyDeviceToDevice, g->stream));
    e = fp32 ? launch_scan<float>((const float *)src, g->N, (int)g->n[0], (int)g->n[1], g->ndim, g->dx, g->part,
                                  kScanBlocks, g->stream, 0, 0, g->ctu)
             : launch_scan<double>((const double *)src, g->N, (int)g->n[0], (int)g->n[1], g->ndim, g->dx, g->part,
                                   kScanBlocks, g->stream, 0, 0, g->ctu);
    if (e == cudaSuccess) e = launch_finalize(g->ctrl, g->part, kScanBlocks, 1, g->stream);
    if (e == cudaSuccess) e = launch_ensemble_start(g->ctrl, s0, nsteps, g->ens_status + k, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "ensemble start: %s", cudaGetErrorString(e));
    for (int64_t i = 0; i < nsteps; i++) {
      st = launch_one_step(g, -1);
      if (st) return st;
    }
    e = launch_ensemble_end(g->ctrl, g->ens_status + k, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "ensemble end: %s", cudaGetErrorString(e));
    CUDA_TRY(cudaMemcpyAsync(slot, g->U[(s0 + nsteps) & 1], bytes, cudaMemcpyDeviceToDevice, g->stream));
    if (kind == MSH_PRIMITIVE)
      e = fp32 ? launch_convert<float>((float *)slot, g->N, 1, g->stream)
               : launch_convert<double>((double *)slot, g->N, 1, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
    CUDA_TRY(cudaEventRecord(ev_done[j], g->stream));
    // download
    CUDA_TRY(cudaStreamWaitEvent(g->ens_out, ev_done[j], 0));
    CUDA_TRY(cudaMemcpyAsync(out[k], slot, bytes, cudaMemcpyDeviceToHost, g->ens_out));
    CUDA_TRY(cudaEventRecord(ev_free[j], g->ens_out));
  }
  CUDA_TRY(cudaStreamSynchronize(g->ens_out));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  std::vector<int32_t> hs((size_t)count);
  CUDA_TRY(cudaMemcpy(hs.data(), g->ens_status, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost));
  st = read_ctrl(g);
  if (st) return st;
  // the grid now holds the last state's result
  g->has_state = true;
  g->hctrl->sg_hist = 0;
  int64_t first_bad = -1;
  for (int64_t k = 0; k < count; k++) {
    if (status) status[k] = hs[(size_t)k];
    if (hs[(size_t)k] != 0 && first_bad < 0) first_bad = k;
  }
  for (int64_t k = 0; k < count; k++)
    if (hs[(size_t)k] == MSH_E_TIMEOUT)
      return fail(MSH_E_TIMEOUT, "ensemble state %lld: a step kernel gave up waiting for a bulk copy", (long long)k);
  if (first_bad >= 0)
    return fail(MSH_E_REALIZABILITY, "ensemble state %lld is not realizable (input or result)", (long long)first_bad);
  return MSH_OK;
}

msh_status msh_set_time(msh_grid *g, double t, int64_t step) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (step < 0 || !std::isfinite(t)) return fail(MSH_E_INVALID_ARG, "bad time or step");
  msh_status st0 = stop_tape(g);
  if (st0) return st0;
  if (((step ^ g->hctrl->step) & 1) && g->has_state) {
    // keep the current state in the buffer the new parity selects
    const size_t bytes = g->N * 10 * g->esize;
    const int cur = cur_buf(g);
    CUDA_TRY(cudaMemcpyAsync(g->U[cur ^ 1], g->U[cur], bytes, cudaMemcpyDeviceToDevice, g->stream));
  }
  CUDA_TRY(cudaMemsetAsync(g->flags, 0, g->N * sizeof(int32_t), g->stream));
  g->hctrl->t = t;
  g->hctrl->step = step;
  g->hctrl->sg_hist = 0;
  CUDA_TRY(cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_get_time(msh_grid *g, double *t, int64_t *step) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (t) *t = g->hctrl->t;
  if (step) *step = g->hctrl->step;
  return MSH_OK;
}

msh_status msh_set_potential(msh_grid *g, const double *phi, int32_t where) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  drop_graph(g);
  if (!phi) {
    if (g->phi) cudaFree(g->phi);
    if (g->acc) cudaFree(g->acc);
    g->phi = nullptr;
    g->acc = nullptr;
    return MSH_OK;
  }
  if (where != MSH_HOST && where != MSH_DEVICE) return fail(MSH_E_INVALID_ARG, "bad where");
  size_t cnt = 1;
  for (int d = 0; d < 3; d++) cnt *= (size_t)(g->n[d] + (d < g->ndim ? 2 : 0));
  if (!g->phi) CUDA_TRY(cudaMalloc(&g->phi, cnt * sizeof(double)));
  if (!g->acc) CUDA_TRY(cudaMalloc(&g->acc, 3 * g->N * g->esize));
  CUDA_TRY(cudaMemcpyAsync(g->phi, phi, cnt * sizeof(double),
                           where == MSH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream));
  cudaError_t e = g->prec == MSH_FP32
                      ? launch_gravity_field<float>(g->phi, (float *)g->acc, g->ndim, (int)g->n[0], (int)g->n[1],
                                                    (int)g->n[2], g->dx, g->stream)
                      : launch_gravity_field<double>(g->phi, (double *)g->acc, g->ndim, (int)g->n[0], (int)g->n[1],
                                                     (int)g->n[2], g->dx, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "gravity field: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_set_scheme(msh_grid *g, int32_t scheme) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (scheme != MSH_SCHEME_MUSCL_HANCOCK && scheme != MSH_SCHEME_KT && scheme != MSH_SCHEME_MUSCL_HANCOCK_ROE &&
      scheme != MSH_SCHEME_MUSCL_HANCOCK_HLLC)
    return fail(MSH_E_INVALID_ARG, "unknown scheme");
  if (scheme != MSH_SCHEME_MUSCL_HANCOCK && g->tape_valid)
    return fail(MSH_E_STATE, "the adjoint tape covers the MUSCL-Hancock scheme with HLL only");
  if (scheme == MSH_SCHEME_KT && g->ctu)
    return fail(MSH_E_STATE, "the transverse (CTU) terms belong to the characteristic schemes: switch CTU off first");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (scheme == MSH_SCHEME_KT && !g->U1) CUDA_TRY(cudaMalloc(&g->U1, g->N * 10 * g->esize));
  if (scheme != g->scheme) drop_graph(g);
  g->scheme = scheme;
  return MSH_OK;
}

msh_status msh_set_ctu(msh_grid *g, int32_t on) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (on != 0 && on != 1) return fail(MSH_E_INVALID_ARG, "on must be 0 or 1");
  if (on && g->scheme == MSH_SCHEME_KT)
    return fail(MSH_E_STATE, "the transverse (CTU) terms belong to the characteristic schemes, not the central one");
  if (on && g->tape_valid && g->ndim > 1)
    return fail(MSH_E_STATE, "the adjoint tape covers the step without transverse (CTU) terms only");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if ((bool)on == g->ctu) return MSH_OK;
  drop_graph(g);
  g->ctu = on != 0;
  // the CFL rule changed: plan the next step of the current state again
  if (g->has_state) return prime(g, cur_buf(g));
  return MSH_OK;
}

msh_status msh_get_ctu(const msh_grid *g, int32_t *on) {
  begin();
  if (!g || !on) return fail(MSH_E_INVALID_ARG, "null argument");
  *on = g->ctu ? 1 : 0;
  return MSH_OK;
}

msh_status msh_set_self_gravity(msh_grid *g, double G) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!(G >= 0.0) || !std::isfinite(G)) return fail(MSH_E_INVALID_ARG, "G must be finite and >= 0");
  for (int i = 0; i < 2 * g->ndim; i++)
    if (G > 0.0 && g->bc[i] != MSH_BC_PERIODIC)
      return fail(MSH_E_INVALID_ARG, "self-gravity needs periodic boundaries on every active dimension");
  if (G > 0.0 && g->tape_valid) return fail(MSH_E_STATE, "the adjoint tape covers external potentials only");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  drop_graph(g);
  if (G == 0.0) {
    free_self_gravity(g);
    return MSH_OK;
  }
  msh_status st = setup_self_gravity(g, G);
  if (st) return st;
  g->hctrl->sg_hist = 0;
  CUDA_TRY(cudaMemsetAsync(&g->ctrl->sg_hist, 0, sizeof(int32_t), g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_set_cell_width(msh_grid *g, const double dx[3]) {
  begin();
  if (!g || !dx) return fail(MSH_E_INVALID_ARG, "null argument");
  for (int d = 0; d < g->ndim; d++)
    if (!(dx[d] > 0.0) || !std::isfinite(dx[d])) return fail(MSH_E_INVALID_ARG, "dx[%d] must be finite and > 0", d);
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  drop_graph(g);  // the cell widths are baked into the graph's step arguments
  for (int d = 0; d < g->ndim; d++) {
    g->dx[d] = dx[d];
    g->hi[d] = g->lo[d] + (double)g->n[d] * dx[d];
  }
  if (g->phi) {  // the acceleration is a difference quotient of the potential
    cudaError_t e = g->prec == MSH_FP32
                        ? launch_gravity_field<float>(g->phi, (float *)g->acc, g->ndim, (int)g->n[0], (int)g->n[1],
                                                      (int)g->n[2], g->dx, g->stream)
                        : launch_gravity_field<double>(g->phi, (double *)g->acc, g->ndim, (int)g->n[0], (int)g->n[1],
                                                       (int)g->n[2], g->dx, g->stream);
    if (e != cudaSuccess) return fail(MSH_E_CUDA, "gravity field: %s", cudaGetErrorString(e));
  }
  if (g->has_state) g->dt_stale = true;  // the CFL step depends on dx
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_step(msh_grid *g, double dt_max, double *dt_taken) {
  msh::NvtxRange nvtx_range("msh_step");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "msh_step before msh_set_state");
  if (!(dt_max > 0.0)) return fail(MSH_E_INVALID_ARG, "dt_max must be > 0");
  msh_status st = refresh_dt(g);
  if (st) return st;
  st = ensure_partials(g, blocks_for(g, g->rows, g->zchunk));
  if (st) return st;
  cudaError_t e = launch_run_start(g->ctrl, INFINITY, 1, dt_max, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "run start: %s", cudaGetErrorString(e));
  st = launch_one_step(g, -1);
  if (st) return st;
  st = read_ctrl(g);
  if (st) return st;
  if (dt_taken) *dt_taken = g->hctrl->dt_last;
  if (g->hctrl->status == MSH_E_TIMEOUT)
    return fail(MSH_E_TIMEOUT, "a step kernel gave up waiting for a bulk copy of its staged planes");
  if (g->hctrl->status == MSH_E_REALIZABILITY)
    return fail(MSH_E_REALIZABILITY, "step produced a non-realizable cell %lld", (long long)g->hctrl->first_bad);
  return MSH_OK;
}

msh_status msh_run(msh_grid *g, double t_end, int64_t max_steps, int64_t *steps, double *t_out) {
  msh::NvtxRange nvtx_range("msh_run");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "msh_run before msh_set_state");
  if (max_steps < 0 || std::isnan(t_end)) return fail(MSH_E_INVALID_ARG, "bad t_end or max_steps");
  msh_status st = refresh_dt(g);
  if (st) return st;
  st = g->profiling ? ensure_partials(g, blocks_for(g, g->rows, g->zchunk)) : build_graph(g);
  if (st) return st;
  const int64_t s0 = g->hctrl->step;
  cudaError_t e = launch_run_start(g->ctrl, t_end, max_steps, INFINITY, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "run start: %s", cudaGetErrorString(e));
  // at most this many batches of kGraphSteps steps can be needed
  const int64_t need = (max_steps + kGraphSteps - 1) / kGraphSteps;
  if (g->profiling) {
    // profiled runs launch the same kernels eagerly, bracketed by events
    for (int64_t it = 0;; it++) {
      if (it > need) return fail(MSH_E_STATE, "run did not terminate (device control inconsistent)");
      const int64_t before = g->hctrl->step;
      for (int i = 0; i < kGraphSteps; i++) {
        st = launch_one_step(g, i);
        if (st) return st;
      }
      st = read_ctrl(g);
      if (st) return st;
      // only the launches that took a step count (the tail after completion returns at once)
      collect_profile(g, (int)(g->hctrl->step - before));
      if (g->hctrl->done) break;
    }
  } else if (max_steps < kGraphSteps) {
    // short runs: exactly max_steps launch pairs, no speculative batch
    for (int64_t i = 0; i < max_steps; i++) {
      st = launch_one_step(g, -1);
      if (st) return st;
    }
    st = read_ctrl(g);
    if (st) return st;
  } else {
    // Two graph batches in flight: launch batch it, then wait for the completion flag of
    // batch it-1, so the GPU never idles while the host polls.  Batches launched after
    // the run finished return immediately on the device.
    for (int64_t it = 0;; it++) {
      if (it > need + 1) return fail(MSH_E_STATE, "run did not terminate (device control inconsistent)");
      if (it < need) {
        CUDA_TRY(cudaGraphLaunch(g->graph, g->stream));
        CUDA_TRY(cudaMemcpyAsync(&g->hdone[it & 1], &g->ctrl->done, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 g->stream));
        CUDA_TRY(cudaEventRecord(g->ev_done[it & 1], g->stream));
      }
      if (it >= 1) {
        CUDA_TRY(cudaEventSynchronize(g->ev_done[(it - 1) & 1]));
        if (g->hdone[(it - 1) & 1] || it >= need) break;
      }
    }
    st = read_ctrl(g);
    if (st) return st;
  }
  if (steps) *steps = g->hctrl->step - s0;
  if (t_out) *t_out = g->hctrl->t;
  if (g->hctrl->status == MSH_E_TIMEOUT)
    return fail(MSH_E_TIMEOUT, "a step kernel gave up waiting for a bulk copy of its staged planes");
  if (g->hctrl->status == MSH_E_REALIZABILITY)
    return fail(MSH_E_REALIZABILITY, "non-realizable cell %lld at step %lld", (long long)g->hctrl->first_bad,
                (long long)g->hctrl->step);
  return MSH_OK;
}

msh_status msh_diagnostics(msh_grid *g, double totals[10], int32_t *realizable, int64_t *first_bad) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  if (totals) memcpy(totals, g->hctrl->totals, sizeof(double) * 10);
  if (realizable) *realizable = g->hctrl->realizable;
  if (first_bad) *first_bad = g->hctrl->first_bad;
  return MSH_OK;
}

msh_status msh_set_recording(msh_grid *g, int64_t capacity) {
  begin();
  if (!g || capacity < 0) return fail(MSH_E_INVALID_ARG, "bad argument");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (g->hist) cudaFree(g->hist);
  g->hist = nullptr;
  g->hist_cap = 0;
  if (capacity > 0) {
    CUDA_TRY(cudaMalloc(&g->hist, sizeof(double) * (size_t)capacity));
    g->hist_cap = capacity;
  }
  g->hctrl->hist = g->hist;
  g->hctrl->hist_cap = g->hist_cap;
  g->hctrl->hist_base = g->hctrl->step;
  CUDA_TRY(cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

msh_status msh_set_tape(msh_grid *g, int32_t K, int64_t max_steps) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (K < 0 || (K > 0 && max_steps < 1)) return fail(MSH_E_INVALID_ARG, "need K >= 1 and max_steps >= 1 (K = 0 frees)");
  if (K > 0 && g->scheme != MSH_SCHEME_MUSCL_HANCOCK)
    return fail(MSH_E_STATE, "the adjoint covers the MUSCL-Hancock scheme only");
  if (K > 0 && g->ctu && g->ndim > 1)
    return fail(MSH_E_STATE, "the adjoint covers the step without transverse (CTU) terms only");
  if (K > 0 && g->sg_G > 0.0) return fail(MSH_E_STATE, "the adjoint covers external potentials only");
  if (!g->has_state && K > 0) return fail(MSH_E_STATE, "msh_set_tape before msh_set_state");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  msh_status st = stop_tape(g);
  if (st) return st;
  if (K == 0) {
    free_tape(g);
    return MSH_OK;
  }
  const int64_t nck = (max_steps + K - 1) / K;
  const int64_t have_ck = g->tape_K > 0 ? (g->tape_len + g->tape_K - 1) / g->tape_K : 0;
  if (nck > have_ck || max_steps > g->tape_len) {
    free_tape(g);
    CUDA_TRY(cudaMalloc(&g->tape, (size_t)nck * g->N * 10 * g->esize));
    CUDA_TRY(cudaMalloc(&g->tape_dt, sizeof(double) * (size_t)max_steps));
    CUDA_TRY(cudaMalloc(&g->tape_had, sizeof(int32_t) * (size_t)max_steps));
  }
  g->tape_K = K;
  g->tape_len = max_steps;
  g->tape_base = g->hctrl->step;
  g->tape_valid = true;
  g->hctrl->tape_dt = g->tape_dt;
  g->hctrl->tape_had = g->tape_had;
  g->hctrl->tape_base = g->tape_base;
  g->hctrl->tape_len = g->tape_len;
  CUDA_TRY(push_tape_fields(g));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MSH_OK;
}

// ------------------------------------------------------- slab decomposition
static msh_status copy_slab(msh_grid *g, int64_t start, int64_t count, void *buf, int32_t where, bool to_grid) {
  if (!g || (!buf && count > 0)) return fail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return fail(MSH_E_INVALID_ARG, "bad where");
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  size_t per = 0;
  int64_t layers = 0;
  layer_geometry(g, &per, &layers);
  if (start < 0 || count < 0 || start + count > layers)
    return fail(MSH_E_INVALID_ARG, "layers [%lld, %lld) outside [0, %lld)", (long long)start,
                (long long)(start + count), (long long)layers);
  if (count == 0) return MSH_OK;
  char *U = static_cast<char *>(g->U[cur_buf(g)]);
  const size_t bytes = (size_t)count * per * g->esize;
  const cudaMemcpyKind kind = to_grid ? (where == MSH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice)
                                      : (where == MSH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  for (int k = 0; k < 10; k++) {
    char *dev = U + ((size_t)k * g->N + (size_t)start * per) * g->esize;
    char *other = static_cast<char *>(buf) + (size_t)k * bytes;
    CUDA_TRY(cudaMemcpyAsync(to_grid ? dev : other, to_grid ? other : dev, bytes, kind, g->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (to_grid) g->dt_stale = true;
  return MSH_OK;
}

msh_status msh_get_slab(msh_grid *g, int64_t start, int64_t count, void *buf, int32_t where) {
  begin();
  return copy_slab(g, start, count, buf, where, false);
}

msh_status msh_set_slab(msh_grid *g, int64_t start, int64_t count, const void *buf, int32_t where) {
  begin();
  return copy_slab(g, start, count, const_cast<void *>(buf), where, true);
}

msh_status msh_reduce_layers(msh_grid *g, int64_t start, int64_t count, double totals[10], double *dt_cfl,
                             int32_t *realizable) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  size_t per = 0;
  int64_t layers = 0;
  layer_geometry(g, &per, &layers);
  if (start < 0 || count < 1 || start + count > layers)
    return fail(MSH_E_INVALID_ARG, "layers [%lld, %lld) outside [0, %lld) or empty", (long long)start,
                (long long)(start + count), (long long)layers);
  if (!g->ctrl_aux) CUDA_TRY(cudaMalloc(&g->ctrl_aux, sizeof(Ctrl)));
  msh_status st = ensure_partials(g, kScanBlocks);
  if (st) return st;
  Ctrl c;
  memset(&c, 0, sizeof c);
  c.cfl = g->cfl;
  CUDA_TRY(cudaMemcpyAsync(g->ctrl_aux, &c, sizeof c, cudaMemcpyHostToDevice, g->stream));
  const size_t c0 = (size_t)start * per, c1 = (size_t)(start + count) * per;
  const int which = cur_buf(g);
  cudaError_t e = g->prec == MSH_FP32
                      ? launch_scan<float>((const float *)g->U[which], g->N, (int)g->n[0], (int)g->n[1], g->ndim,
                                           g->dx, g->part, kScanBlocks, g->stream, c0, c1, g->ctu)
                      : launch_scan<double>((const double *)g->U[which], g->N, (int)g->n[0], (int)g->n[1], g->ndim,
                                            g->dx, g->part, kScanBlocks, g->stream, c0, c1, g->ctu);
  if (e == cudaSuccess) e = launch_finalize(g->ctrl_aux, g->part, kScanBlocks, 1, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "layer reduction: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(&c, g->ctrl_aux, sizeof c, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (totals) memcpy(totals, c.totals, sizeof(double) * 10);
  if (dt_cfl) *dt_cfl = c.dt_cfl;
  if (realizable) *realizable = c.realizable;
  return MSH_OK;
}

msh_status msh_step_dt(msh_grid *g, double dt, int32_t *tagged_cells) {
  msh::NvtxRange nvtx_range("msh_step_dt");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "msh_step_dt before msh_set_state");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MSH_E_INVALID_ARG, "dt must be finite and > 0");
  msh_status st = ensure_partials(g, blocks_for(g, g->rows, g->zchunk));
  if (st) return st;
  cudaError_t e = launch_set_dt(g->ctrl, dt, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "set dt: %s", cudaGetErrorString(e));
  st = launch_one_step(g, -1);
  if (st) return st;
  st = read_ctrl(g);
  if (st) return st;
  g->dt_stale = false;  // the finalize planned from the new state
  if (tagged_cells) *tagged_cells = g->hctrl->last_tagged;
  if (g->hctrl->status == MSH_E_TIMEOUT)
    return fail(MSH_E_TIMEOUT, "a step kernel gave up waiting for a bulk copy of its staged planes");
  if (g->hctrl->status == MSH_E_REALIZABILITY)
    return fail(MSH_E_REALIZABILITY, "step produced a non-realizable cell %lld", (long long)g->hctrl->first_bad);
  return MSH_OK;
}

// ----------------------------------------- phased step: slabs sharing the fallback
static msh_status phase_layers(msh_grid *g, int64_t start, int64_t count, size_t *c0, size_t *c1) {
  size_t per = 0;
  int64_t layers = 0;
  layer_geometry(g, &per, &layers);
  if (start < 0 || count < 0 || start + count > layers)
    return fail(MSH_E_INVALID_ARG, "layers [%lld, %lld) outside [0, %lld)", (long long)start,
                (long long)(start + count), (long long)layers);
  *c0 = (size_t)start * per;
  *c1 = (size_t)(start + count) * per;
  return MSH_OK;
}

msh_status msh_step_begin(msh_grid *g, double dt) {
  msh::NvtxRange nvtx_range("msh_step_begin");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "msh_step_begin before msh_set_state");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MSH_E_INVALID_ARG, "dt must be finite and > 0");
  if (g->scheme == MSH_SCHEME_KT)
    return fail(MSH_E_STATE, "the central scheme has no fallback passes: step it with msh_step_dt");
  if (g->sg_G > 0.0) return fail(MSH_E_STATE, "a phased step does not take self-gravity");
  msh_status st = ensure_partials(g, blocks_for(g, g->rows, g->zchunk));
  if (st) return st;
  cudaError_t e = launch_set_dt(g->ctrl, dt, g->stream);
  int nb = 0;
  if (e == cudaSuccess) {
    const int32_t test_fault = g->test_fault;
    g->test_fault = 0;  // a test hook applies to one step
    if (g->prec == MSH_FP32) {
      StepArgs<float> a = make_args<float>(g);
      a.test_skip = test_fault == 1;
      e = launch_characteristic(g, a, false, &nb);
    } else {
      StepArgs<double> a = make_args<double>(g);
      a.test_skip = test_fault == 1;
      e = launch_characteristic(g, a, false, &nb);
    }
  }
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "step begin: %s", cudaGetErrorString(e));
  g->phase_level = 0;
  g->phase_nb = nb;
  return MSH_OK;
}

msh_status msh_step_retry(msh_grid *g, int32_t level) {
  msh::NvtxRange nvtx_range("msh_step_retry");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (g->phase_level < 0) return fail(MSH_E_STATE, "msh_step_retry outside msh_step_begin .. msh_step_end");
  if (level != g->phase_level + 1 || level > kFallbackPasses)
    return fail(MSH_E_INVALID_ARG, "fallback pass %d after pass %d (passes run in order 1 .. %d)", level,
                g->phase_level, kFallbackPasses);
  cudaError_t e = launch_force_pass(g->ctrl, level, g->stream);
  if (e == cudaSuccess) {
    if (g->prec == MSH_FP32) {
      StepArgs<float> a = make_args<float>(g);
      a.level = level;
      e = launch_characteristic(g, a, true, nullptr);
    } else {
      StepArgs<double> a = make_args<double>(g);
      a.level = level;
      e = launch_characteristic(g, a, true, nullptr);
    }
  }
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "fallback pass: %s", cudaGetErrorString(e));
  g->phase_level = level;
  return MSH_OK;
}

msh_status msh_step_end(msh_grid *g, int32_t *tagged_cells) {
  msh::NvtxRange nvtx_range("msh_step_end");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (g->phase_level < 0) return fail(MSH_E_STATE, "msh_step_end without msh_step_begin");
  g->phase_level = -1;
  cudaError_t e = launch_finalize(g->ctrl, g->part, g->phase_nb, 0, g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "finalize launch: %s", cudaGetErrorString(e));
  msh_status st = read_ctrl(g);
  if (st) return st;
  g->dt_stale = false;
  if (tagged_cells) *tagged_cells = g->hctrl->last_tagged;
  if (g->hctrl->status == MSH_E_TIMEOUT)
    return fail(MSH_E_TIMEOUT, "a step kernel gave up waiting for a bulk copy of its staged planes");
  if (g->hctrl->status == MSH_E_REALIZABILITY)
    return fail(MSH_E_REALIZABILITY, "step produced a non-realizable cell %lld", (long long)g->hctrl->first_bad);
  return MSH_OK;
}

static msh_status copy_tags(msh_grid *g, int64_t start, int64_t count, int32_t *levels, int32_t where,
                            bool to_grid) {
  if (!g || (!levels && count > 0)) return fail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return fail(MSH_E_INVALID_ARG, "bad where");
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  size_t c0 = 0, c1 = 0;
  msh_status st = phase_layers(g, start, count, &c0, &c1);
  if (st || c1 == c0) return st;
  const size_t bytes = (c1 - c0) * sizeof(int32_t);
  int32_t *buf = levels;
  if (where == MSH_HOST) CUDA_TRY(cudaMallocAsync(&buf, bytes, g->stream));
  cudaError_t e = cudaSuccess;
  if (to_grid && where == MSH_HOST) e = cudaMemcpyAsync(buf, levels, bytes, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = launch_tags(g->ctrl, g->flags, c0, c1, buf, to_grid, g->stream);
  if (e == cudaSuccess && !to_grid && where == MSH_HOST)
    e = cudaMemcpyAsync(levels, buf, bytes, cudaMemcpyDeviceToHost, g->stream);
  if (where == MSH_HOST) cudaFreeAsync(buf, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "fallback tags: %s", cudaGetErrorString(e));
  return MSH_OK;
}

msh_status msh_get_tags(msh_grid *g, int64_t start, int64_t count, int32_t *levels, int32_t where) {
  begin();
  return copy_tags(g, start, count, levels, where, false);
}

msh_status msh_set_tags(msh_grid *g, int64_t start, int64_t count, const int32_t *levels, int32_t where) {
  begin();
  return copy_tags(g, start, count, const_cast<int32_t *>(levels), where, true);
}

msh_status msh_count_tags(msh_grid *g, int64_t start, int64_t count, int32_t level, int64_t *n) {
  begin();
  if (!g || !n) return fail(MSH_E_INVALID_ARG, "null argument");
  if (level < 0 || level > kFallbackPasses) return fail(MSH_E_INVALID_ARG, "level must be in [0, %d]", kFallbackPasses);
  if (!g->has_state) return fail(MSH_E_STATE, "no state set");
  size_t c0 = 0, c1 = 0;
  msh_status st = phase_layers(g, start, count, &c0, &c1);
  if (st) return st;
  *n = 0;
  if (c1 == c0) return MSH_OK;
  if (!g->tag_count) CUDA_TRY(cudaMalloc(&g->tag_count, sizeof(unsigned long long)));
  unsigned long long h = 0;
  cudaError_t e = launch_count_tags(g->ctrl, g->flags, c0, c1, level, g->tag_count, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, g->tag_count, sizeof h, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail(MSH_E_CUDA, "count tags: %s", cudaGetErrorString(e));
  *n = (int64_t)h;
  return MSH_OK;
}

msh_status msh_get_dt_history(msh_grid *g, double *dts, int64_t capacity, int64_t *count) {
  begin();
  if (!g || capacity < 0 || (capacity > 0 && !dts)) return fail(MSH_E_INVALID_ARG, "bad argument");
  int64_t n = g->hist ? g->hctrl->step - g->hctrl->hist_base : 0;
  if (n > g->hist_cap) n = g->hist_cap;
  if (n < 0) n = 0;
  const int64_t m = n < capacity ? n : capacity;
  if (m > 0) {
    CUDA_TRY(cudaMemcpyAsync(dts, g->hist, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
  }
  if (count) *count = n;
  return MSH_OK;
}

msh_status msh_set_tiling(msh_grid *g, int32_t rows, int32_t zchunk) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (rows != 4 && rows != 8 && rows != 16) return fail(MSH_E_INVALID_ARG, "rows must be 4, 8 or 16");
  if (rows == 16 && g->ndim == 3 && g->prec == MSH_FP64)
    return fail(MSH_E_INVALID_ARG, "rows 16 in 3D needs FP32 (its FP64 staging exceeds shared memory)");
  if (zchunk < 0 || (zchunk == 0 && g->ndim != 3))
    return fail(MSH_E_INVALID_ARG, "zchunk must be >= 1 (or 0 in 3D: the balanced tiling)");
  const int64_t stream_len = g->ndim == 3 ? g->n[2] : g->ndim == 2 ? g->n[1] : 1;
  if (zchunk > stream_len) zchunk = (int)stream_len;
  msh_status st = ensure_partials(g, blocks_for(g, rows, zchunk));
  if (st) return st;
  if (rows != g->rows || zchunk != g->zchunk) drop_graph(g);
  g->rows = rows;
  g->zchunk = zchunk;
  return MSH_OK;
}

msh_status msh_get_tiling(msh_grid *g, int32_t *rows, int32_t *zchunk) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (rows) *rows = g->rows;
  if (zchunk) *zchunk = g->zchunk;
  return MSH_OK;
}

// Time each tile shape on copies of the current state (the state, time and step
// counter are restored afterwards) and keep the fastest.
msh_status msh_autotune(msh_grid *g, int32_t *rows_out, int32_t *zchunk_out) {
  msh::NvtxRange nvtx_range("msh_autotune");
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (!g->has_state) return fail(MSH_E_STATE, "msh_autotune before msh_set_state");
  if (g->ndim == 1) {
    if (rows_out) *rows_out = g->rows;
    if (zchunk_out) *zchunk_out = g->zchunk;
    return MSH_OK;
  }
  const size_t bytes = g->N * 10 * g->esize;
  const int cur = cur_buf(g);
  void *save = nullptr;
  CUDA_TRY(cudaMalloc(&save, bytes));
  Ctrl saved_ctrl = *g->hctrl;
  // the trial steps must not write the adjoint tape
  Ctrl trial_ctrl = saved_ctrl;
  trial_ctrl.tape_dt = nullptr;
  trial_ctrl.tape_had = nullptr;
  trial_ctrl.tape_len = 0;
  const bool tape_was_valid = g->tape_valid;
  g->tape_valid = false;
  *g->hctrl = trial_ctrl;
  msh_status st = MSH_OK;
  // the trial steps overwrite the stored self-gravity acceleration: keep a copy
  void *sg_save = nullptr;
  if (g->sg_G > 0.0 && cudaMalloc(&sg_save, 3 * g->N * g->esize) == cudaSuccess)
    cudaMemcpyAsync(sg_save, g->sg_prev, 3 * g->N * g->esize, cudaMemcpyDeviceToDevice, g->stream);
  else if (g->sg_G > 0.0)
    st = fail(MSH_E_NOMEM, "autotune: no room to keep the self-gravity history");
  if (cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
    st = fail(MSH_E_CUDA, "autotune setup: %s", cudaGetErrorString(cudaGetLastError()));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<std::pair<int, int>> cands;
  const int rows_c[3] = {4, 8, 16};
  const int zc_c[4] = {8, 16, 32, 64};
  const int64_t stream_len = g->ndim == 3 ? g->n[2] : g->n[1];
  // 2D: rows of 8..64; 3D: the balanced tiling (0) and chunks that cut z into m = 1..8
  // near-equal windows
  std::vector<int> zcs;
  if (g->ndim == 3) {
    zcs.push_back(0);
    for (int m = 1; m <= 8; m++) {
      const int z = (int)((stream_len + m - 1) / m);
      if (std::find(zcs.begin(), zcs.end(), z) == zcs.end()) zcs.push_back(z);
    }
  } else {
    for (int z : zc_c)
      if (z <= stream_len || z == zc_c[0]) zcs.push_back(z);
  }
  for (int r : rows_c)
    for (int z : zcs)
      if (!(r == 16 && g->ndim == 3 && g->prec == MSH_FP64)) cands.push_back({r, z});
  float best = 1e30f;
  std::pair<int, int> best_c = {g->rows, g->zchunk};
  const int reps = 3;
  if (st == MSH_OK && (cudaMemcpyAsync(save, g->U[cur], bytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
                       cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    st = fail(MSH_E_CUDA, "autotune setup: %s", cudaGetErrorString(cudaGetLastError()));
  }
  const bool prof = g->profiling;
  g->profiling = false;
  for (size_t i = 0; st == MSH_OK && i < cands.size(); i++) {
    st = msh_set_tiling(g, cands[i].first, cands[i].second);
    if (st) break;
    cudaError_t e = launch_run_start(g->ctrl, INFINITY, 1 << 30, INFINITY, g->stream);
    for (int w = 0; st == MSH_OK && w < 1; w++) st = launch_one_step(g, -1);
    if (st == MSH_OK) e = cudaEventRecord(e0, g->stream);
    for (int w = 0; st == MSH_OK && w < reps; w++) st = launch_one_step(g, -1);
    if (st == MSH_OK) e = cudaEventRecord(e1, g->stream);
    if (st == MSH_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == MSH_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (st == MSH_OK && e != cudaSuccess) st = fail(MSH_E_CUDA, "autotune timing: %s", cudaGetErrorString(e));
    if (st == MSH_OK && ms < best) {
      best = ms;
      best_c = cands[i];
    }
    // restore state and control block for the next candidate
    if (st == MSH_OK) {
      *g->hctrl = trial_ctrl;
      e = cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(g->U[cur], save, bytes, cudaMemcpyDeviceToDevice, g->stream);
      if (e != cudaSuccess) st = fail(MSH_E_CUDA, "autotune restore: %s", cudaGetErrorString(e));
    }
  }
  g->profiling = prof;
  *g->hctrl = saved_ctrl;
  g->tape_valid = tape_was_valid;
  if (sg_save) {
    cudaMemcpyAsync(g->sg_prev, sg_save, 3 * g->N * g->esize, cudaMemcpyDeviceToDevice, g->stream);
    cudaStreamSynchronize(g->stream);
    cudaFree(sg_save);
  }
  if (cudaMemcpyAsync(g->ctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream) != cudaSuccess && st == MSH_OK)
    st = fail(MSH_E_CUDA, "autotune restore: %s", cudaGetErrorString(cudaGetLastError()));
  drop_graph(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(g->stream);
  cudaFree(save);
  if (st) return st;
  st = msh_set_tiling(g, best_c.first, best_c.second);
  if (st) return st;
  if (rows_out) *rows_out = g->rows;
  if (zchunk_out) *zchunk_out = g->zchunk;
  return MSH_OK;
}

msh_status msh_set_test_fault(msh_grid *g, int32_t kind) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (kind != 0 && kind != 1) return fail(MSH_E_INVALID_ARG, "test fault kind must be 0 or 1");
  g->test_fault = kind;
  return MSH_OK;
}

msh_status msh_set_profiling(msh_grid *g, int32_t on) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (on && g->ev.empty()) {
    g->ev.resize(3 * kGraphSteps);
    for (auto &e : g->ev) CUDA_TRY(cudaEventCreate(&e));
  }
  if ((bool)on != g->profiling) drop_graph(g);
  g->profiling = on != 0;
  g->prof_ms = 0.0;
  g->prof_fin_ms = 0.0;
  g->prof_launches = 0;
  return MSH_OK;
}

msh_status msh_get_profile(msh_grid *g, double *step_kernel_ms, double *finalize_ms, int64_t *launches) {
  begin();
  if (!g) return fail(MSH_E_INVALID_ARG, "null grid");
  if (step_kernel_ms) *step_kernel_ms = g->prof_ms;
  if (finalize_ms) *finalize_ms = g->prof_fin_ms;
  if (launches) *launches = g->prof_launches;
  return MSH_OK;
}

}  // extern "C"
