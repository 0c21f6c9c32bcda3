// msh_noalloc.cu -- one step of the grid solver that allocates no memory.
//
// Some callers cannot allocate device memory: code that runs while the allocator is
// forbidden or already exhausted (inside a pre-sized memory pool of another framework,
// an embedded or real-time host loop that must not call into the allocator, a handler
// running under a strict memory budget), or code that only owns the two state buffers it
// was handed.  msh_step_noalloc serves them: the caller passes the input and output
// states, and all the working memory of the step (control block, per-block reduction
// partials, fallback tags) lives in one file-scope device array of fixed size that every
// GPU holds from the moment it loads the library until the process exits.
//
// That array is shared by every call: each call clears what must start at zero (the
// control block and the tags of its cells) before using it, and two calls whose work
// overlaps on the GPU (other streams, other host threads) race on it.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "../../include/msh.h"
#include "msh_internal.h"

namespace msh {

constexpr size_t kNoallocMaxCells = size_t(1) << 20;  // 1,048,576 cells
constexpr size_t kNoallocMaxBlocks = 16384;           // per-block reduction partials
constexpr size_t kNoallocCtrlBytes = 512;
constexpr size_t kNoallocBytes =
    kNoallocCtrlBytes + kNoallocMaxBlocks * sizeof(Partial) + kNoallocMaxCells * sizeof(int32_t);
static_assert(sizeof(Ctrl) <= kNoallocCtrlBytes, "control block does not fit its slot");
static_assert(sizeof(Partial) % 8 == 0, "partials must keep 8-byte alignment");

// The scratch memory.  In host code this name is only a host-side stand-in: the device
// address comes from cudaGetSymbolAddress, taken once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_noalloc_scratch per device; two host threads making the first call on
// a device at once both store the same address
std::atomic<void *> g_scratch_addr[kMaxDevices] = {};

// Start the step after the scan of U_in: a non-realizable input (rho <= 0 or P not positive
// definite in some cell; the scan's finalize has set ctrl->realizable and first_bad) is not
// stepped: the step kernels see done = 1 and return, U_out is not written, and the status is
// MSH_E_REALIZABILITY.  Otherwise the step is planned as a one-step run with dt <= dt_max.
__global__ void noalloc_start_kernel(Ctrl *c, double dt_max) {
  if (!c->realizable) {
    c->done = 1;
    c->status = MSH_E_REALIZABILITY;
    return;
  }
  c->t_end = INFINITY;
  c->max_step = c->step + 1;
  c->dt_max = dt_max;
  c->done = 0;
  c->status = 0;
  double dt = c->dt_cfl;
  if (dt > dt_max) dt = dt_max;
  c->dt = dt;
  c->t_next = c->t + dt;
}

template <typename T>
msh_status noalloc_step(int ndim, const int64_t n[3], const double dx[3], const int32_t bc[6], double cfl,
                        double dt_max, const T *Uin, T *Uout, cudaStream_t s, double *dt_taken,
                        unsigned char *base) {
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
  Partial *part = reinterpret_cast<Partial *>(base + kNoallocCtrlBytes);
  int32_t *flags = reinterpret_cast<int32_t *>(base + kNoallocCtrlBytes + kNoallocMaxBlocks * sizeof(Partial));
  const size_t N = (size_t)n[0] * n[1] * n[2];
  StepArgs<T> a;
  a.U[0] = const_cast<T *>(Uin);  // step 0 reads U[0] and writes U[1]
  a.U[1] = Uout;
  a.acc = nullptr;
  a.ctrl = ctrl;
  a.part = part;
  a.flags = flags;
  a.nx = (int)n[0];
  a.ny = (int)n[1];
  a.nz = (int)n[2];
  for (int i = 0; i < 6; i++) a.bc[i] = i < 2 * ndim ? bc[i] : MSH_BC_PERIODIC;
  for (int i = 0; i < 3; i++) a.dx[i] = dx[i];
  a.zchunk = default_chunk(ndim, n);
  a.level = 0;
  a.ck = nullptr;  // no adjoint tape
  a.ck_base = 0;
  a.ck_len = 0;
  a.ck_K = 1;
  a.U1 = nullptr;
  const int rows = 8;
  const int nb = step_blocks<T>(ndim, rows, a.nx, a.ny, a.nz, a.zchunk);
  if ((size_t)nb > kNoallocMaxBlocks)
    return set_error_text("msh_step_noalloc: grid needs more thread blocks than the fixed scratch holds"),
           MSH_E_INVALID_ARG;
  // clear the control block and the tags of these cells (the array keeps the last call's data)
  Ctrl init;
  memset(&init, 0, sizeof init);
  init.cfl = cfl;
  init.t_end = INFINITY;
  init.dt_max = INFINITY;
  init.done = 1;
  init.first_bad = -1;
  cudaError_t e = cudaMemcpyAsync(ctrl, &init, sizeof init, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, N * sizeof(int32_t), s);
  // CFL dt of the input state, then one step with dt = min(CFL dt, dt_max)
  if (e == cudaSuccess) e = launch_scan<T>(Uin, N, a.nx, a.ny, ndim, dx, part, kScanBlocks, s);
  if (e == cudaSuccess) e = launch_finalize(ctrl, part, kScanBlocks, 1, s);
  if (e == cudaSuccess) {
    noalloc_start_kernel<<<1, 1, 0, s>>>(ctrl, dt_max);
    e = cudaGetLastError();
  }
  for (int level = 0; e == cudaSuccess && level <= kFallbackPasses; level++) {
    a.level = level;
    e = launch_step<T>(a, ndim, rows, level > 0, s, nullptr);
  }
  if (e == cudaSuccess) e = launch_finalize(ctrl, part, nb, 0, s);
  Ctrl out;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&out, ctrl, sizeof out, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error_text(cudaGetErrorString(e));
    return MSH_E_CUDA;
  }
  if (out.status == MSH_E_TIMEOUT) {
    set_error_text("msh_step_noalloc: the step kernel gave up waiting for a bulk copy of its staged planes");
    return MSH_E_TIMEOUT;
  }
  if (out.status == MSH_E_REALIZABILITY) {
    char msg[160];
    snprintf(msg, sizeof msg, "msh_step_noalloc: %s (first cell %lld)",
             out.step == 0 ? "U_in is not realizable; nothing was stepped" : "the step produced a non-realizable cell",
             (long long)out.first_bad);
    set_error_text(msg);
    return MSH_E_REALIZABILITY;
  }
  if (dt_taken) *dt_taken = out.dt_last;
  return MSH_OK;
}
}  // namespace

}  // namespace msh

using namespace msh;

extern "C" msh_status msh_step_noalloc(int32_t ndim, const int64_t n[3], const double lo[3], const double hi[3],
                                       const int32_t bc[6], int32_t precision, double cfl, double dt_max,
                                       const void *U_in, void *U_out, void *stream, double *dt_taken) {
  clear_error();
  if (!n || !lo || !hi || !bc || !U_in || !U_out) return set_error_text("msh_step_noalloc: null argument"), MSH_E_INVALID_ARG;
  if (ndim < 1 || ndim > 3) return set_error_text("msh_step_noalloc: ndim must be 1, 2 or 3"), MSH_E_INVALID_ARG;
  if (precision != MSH_FP32 && precision != MSH_FP64)
    return set_error_text("msh_step_noalloc: bad precision"), MSH_E_INVALID_ARG;
  if (!(cfl > 0.0 && cfl <= 1.0)) return set_error_text("msh_step_noalloc: cfl must be in (0, 1]"), MSH_E_INVALID_ARG;
  if (!(dt_max > 0.0)) return set_error_text("msh_step_noalloc: dt_max must be > 0"), MSH_E_INVALID_ARG;
  if (U_in == U_out) return set_error_text("msh_step_noalloc: U_in and U_out must differ"), MSH_E_INVALID_ARG;
  double dx[3];
  for (int d = 0; d < 3; d++) {
    if (d < ndim) {
      if (n[d] < 2 || !(hi[d] > lo[d])) return set_error_text("msh_step_noalloc: bad extent"), MSH_E_INVALID_ARG;
      if ((bc[2 * d] == MSH_BC_PERIODIC) != (bc[2 * d + 1] == MSH_BC_PERIODIC) || bc[2 * d] < 0 || bc[2 * d] > 2 ||
          bc[2 * d + 1] < 0 || bc[2 * d + 1] > 2)
        return set_error_text("msh_step_noalloc: bad boundary"), MSH_E_INVALID_ARG;
      dx[d] = (hi[d] - lo[d]) / (double)n[d];
    } else {
      if (n[d] != 1) return set_error_text("msh_step_noalloc: unused dimension must have n = 1"), MSH_E_INVALID_ARG;
      dx[d] = 1.0;
    }
  }
  const double cells = (double)n[0] * (double)n[1] * (double)n[2];
  if (cells > (double)kNoallocMaxCells)
    return set_error_text("msh_step_noalloc: more than 1048576 cells (the fixed scratch limit); use msh_step"),
           MSH_E_INVALID_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error_text("msh_step_noalloc: no usable CUDA device"), MSH_E_CUDA;
  void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {  // first call on this device: look up the array's device address
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
      set_error_text(cudaGetErrorString(e));
      return MSH_E_CUDA;
    }
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char *base = static_cast<unsigned char *>(addr);
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == MSH_FP32)
    return noalloc_step<float>(ndim, n, dx, bc, cfl, dt_max, (const float *)U_in, (float *)U_out, s, dt_taken, base);
  return noalloc_step<double>(ndim, n, dx, bc, cfl, dt_max, (const double *)U_in, (double *)U_out, s, dt_taken, base);
}
