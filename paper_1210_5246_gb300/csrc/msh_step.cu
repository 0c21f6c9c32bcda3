// msh_step.cu -- step launchers of the MUSCL-Hancock scheme and the small kernels of a
// run: scan, gravity field, finalize (fixed-order reduction of the partials, plans the
// next step on the device), run start, conversions.  The step kernels themselves are in
// msh_step_kernels.cuh; the central scheme's stages are instantiated in msh_step_kt.cu.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "msh_step_kernels.cuh"

namespace msh {

// ----------------------------------------------------------------- scan kernel
// Partials (totals, max signal speed sum, first non-realizable cell) of the cells
// [c0, c1) of a state whose fields are N apart.  MAXF: the corner-transport-upwind speed
// (the maximum over the dims instead of the sum).
template <typename T, int NDIM, bool MAXF>
__global__ void __launch_bounds__(256) scan_kernel(const T *__restrict__ U, size_t N, size_t c0, size_t c1, T idx,
                                                   T idy, T idz, Partial *part) {
  double diag[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) diag[k] = 0.0;
  T smax = T(0);
  long long bad = LLONG_MAX;
  for (size_t c = c0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += (size_t)gridDim.x * blockDim.x) {
    T Uc[NV], W[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) Uc[k] = U[k * N + c];
    cons_to_prim(Uc, W);
    if (!realizable(W)) bad = min(bad, (long long)c);
    smax = fmax(smax, speed_sum<T, NDIM, MAXF>(W, idx, idy, idz));
#pragma unroll
    for (int k = 0; k < NV; k++) diag[k] += (double)Uc[k];
  }
  block_partial<256>(diag, (double)smax, bad, part + blockIdx.x);
}

// Acceleration a = -grad Phi by central differences from the potential with one ghost
// layer, stored [3][N] in the state's precision.
template <typename T>
__global__ void gravity_field_kernel(const double *__restrict__ phi, T *__restrict__ acc, int ndim, int nx,
                                     int ny, int nz, double dx0, double dx1, double dx2) {
  const size_t N = (size_t)nx * ny * nz;
  const int gy = ndim > 1 ? 1 : 0, gz = ndim > 2 ? 1 : 0;
  const long px = nx + 2, py = ny + 2 * gy;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const long x = (long)(c % nx), y = (long)((c / nx) % ny), z = (long)(c / ((size_t)nx * ny));
    const long ctr = ((z + gz) * py + (y + gy)) * px + (x + 1);
    acc[c] = (T)(-(phi[ctr + 1] - phi[ctr - 1]) / (2.0 * dx0));
    acc[N + c] = ndim > 1 ? (T)(-(phi[ctr + px] - phi[ctr - px]) / (2.0 * dx1)) : T(0);
    acc[2 * N + c] = ndim > 2 ? (T)(-(phi[ctr + px * py] - phi[ctr - px * py]) / (2.0 * dx2)) : T(0);
  }
}

// -------------------------------------------------------- finalize and plan
__device__ void plan(Ctrl *c) {
  if (c->t >= c->t_end || c->step >= c->max_step) {
    c->done = 1;
    return;
  }
  double dt = c->dt_cfl;
  if (dt > c->dt_max) dt = c->dt_max;
  double tn = c->t + dt;
  if (tn >= c->t_end) {
    dt = c->t_end - c->t;
    tn = c->t_end;
  }
  c->dt = dt;
  c->t_next = tn;
}

// mode 0: after a step (advance time, record dt, stop on a non-realizable cell, plan the
// next step); mode 1: after set_state (CFL dt and totals of the state only).
__global__ void __launch_bounds__(kFinalizeThreads) finalize_kernel(Ctrl *ctrl, const Partial *part,
                                                                    int nparts, int mode) {
  if (mode == 0 && ctrl->done) return;
  __shared__ double sd[kFinalizeThreads][NV + 1];
  __shared__ long long sb[kFinalizeThreads];
  const int t = threadIdx.x;
  double d[NV];
  for (int k = 0; k < NV; k++) d[k] = 0.0;
  double smax = 0.0;
  long long bad = LLONG_MAX;
  for (int i = t; i < nparts; i += kFinalizeThreads) {
    for (int k = 0; k < NV; k++) d[k] += part[i].diag[k];
    smax = fmax(smax, part[i].smax);
    bad = min(bad, part[i].bad);
  }
  for (int k = 0; k < NV; k++) sd[t][k] = d[k];
  sd[t][NV] = smax;
  sb[t] = bad;
  __syncthreads();
  for (int s = kFinalizeThreads / 2; s > 0; s >>= 1) {  // pairwise, fixed order
    if (t < s) {
      for (int k = 0; k < NV; k++) sd[t][k] += sd[t + s][k];
      sd[t][NV] = fmax(sd[t][NV], sd[t + s][NV]);
      sb[t] = min(sb[t], sb[t + s]);
    }
    __syncthreads();
  }
  if (t != 0) return;
  Ctrl *c = ctrl;
  if (mode == 0 && c->stage_timeout) {  // the step kernel gave up waiting for staged data
    c->status = 5;                     // MSH_E_TIMEOUT
    c->done = 1;
    return;
  }
  for (int k = 0; k < NV; k++) c->totals[k] = sd[0][k];
  const long long b = sb[0];
  c->realizable = (b == LLONG_MAX);
  c->first_bad = (b == LLONG_MAX) ? -1 : b;
  c->dt_cfl = c->cfl / sd[0][NV];
  if (mode == 1) {
    c->done = 1;
    return;
  }
  c->last_tagged = c->nbad[0];
  const int64_t ti = c->step - c->tape_base;
  if (c->tape_dt != nullptr && ti >= 0 && ti < c->tape_len) {
    c->tape_dt[ti] = c->dt;
    c->tape_had[ti] = c->nbad[0] > 0;
  }
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
  c->force = 0;
  const int64_t hi_ = c->step - c->hist_base;
  if (c->hist != nullptr && hi_ >= 0 && hi_ < c->hist_cap) c->hist[hi_] = c->dt;
  c->dt_last = c->dt;
  c->t = c->t_next;
  c->step += 1;
  if (!c->realizable) {
    c->status = 4;  // MSH_E_REALIZABILITY
    c->done = 1;
    return;
  }
  plan(c);
}

// One step with a given dt: no CFL limit, no end time.
__global__ void set_dt_kernel(Ctrl *c, double dt) {
  c->t_end = INFINITY;
  c->max_step = INT64_MAX;
  c->dt_max = INFINITY;
  c->done = 0;
  c->status = 0;
  c->stage_timeout = 0;
  c->force = 0;
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
  c->dt = dt;
  c->t_next = c->t + dt;
}

// A fallback pass that must run even where this grid tagged nothing in the pass before.
__global__ void force_pass_kernel(Ctrl *c, int level) { c->force |= 1 << level; }

// Per cell of [c0, c1): the fallback pass of the current step that tagged it, or -1
// (tags are 8 * (step tag) + pass; a tag of another step is no tag).
__global__ void get_tags_kernel(const Ctrl *ctrl, const int32_t *flags, size_t c0, size_t c1, int32_t *levels) {
  const int32_t tag = (int32_t)(ctrl->step & 0x0fffffff) + 1;
  for (size_t c = c0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += (size_t)gridDim.x * blockDim.x) {
    const int32_t f = flags[c];
    levels[c - c0] = (f >> 3) == tag ? (f & 7) : -1;
  }
}

__global__ void set_tags_kernel(const Ctrl *ctrl, int32_t *flags, size_t c0, size_t c1, const int32_t *levels) {
  const int32_t tag = (int32_t)(ctrl->step & 0x0fffffff) + 1;
  for (size_t c = c0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += (size_t)gridDim.x * blockDim.x) {
    const int32_t l = levels[c - c0];
    flags[c] = l >= 0 ? tag * 8 + l : 0;
  }
}

// Cells of [c0, c1) tagged by pass `level` of the current step.
__global__ void count_tags_kernel(const Ctrl *ctrl, const int32_t *flags, size_t c0, size_t c1, int level,
                                  unsigned long long *count) {
  const int32_t want = ((int32_t)(ctrl->step & 0x0fffffff) + 1) * 8 + level;
  unsigned long long n = 0;
  for (size_t c = c0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += (size_t)gridDim.x * blockDim.x)
    n += flags[c] == want;
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, n);
}

cudaError_t launch_force_pass(Ctrl *ctrl, int level, cudaStream_t s) {
  force_pass_kernel<<<1, 1, 0, s>>>(ctrl, level);
  return cudaGetLastError();
}

cudaError_t launch_tags(Ctrl *ctrl, int32_t *flags, size_t c0, size_t c1, int32_t *levels, bool to_grid,
                        cudaStream_t s) {
  const int blocks = (int)std::min<size_t>((c1 - c0 + 255) / 256 + 1, (size_t)kScanBlocks);
  if (to_grid) set_tags_kernel<<<blocks, 256, 0, s>>>(ctrl, flags, c0, c1, levels);
  else get_tags_kernel<<<blocks, 256, 0, s>>>(ctrl, flags, c0, c1, levels);
  return cudaGetLastError();
}

cudaError_t launch_count_tags(const Ctrl *ctrl, const int32_t *flags, size_t c0, size_t c1, int level,
                              unsigned long long *count, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<size_t>((c1 - c0 + 255) / 256 + 1, (size_t)kScanBlocks);
  count_tags_kernel<<<blocks, 256, 0, s>>>(ctrl, flags, c0, c1, level, count);
  return cudaGetLastError();
}

__global__ void run_start_kernel(Ctrl *c, double t_end, int64_t max_steps, double dt_max) {
  c->t_end = t_end;
  c->max_step = (max_steps > INT64_MAX - c->step) ? INT64_MAX : c->step + max_steps;
  c->dt_max = dt_max;
  c->done = 0;
  c->status = 0;
  c->stage_timeout = 0;
  c->force = 0;
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
  plan(c);
}

// Ensemble runs: after the scan of a new state (finalize mode 1), start it at t = 0 with the
// step counter at step_base (the host knows every state's base, hence its buffer parity and
// fallback tags, without reading the device); a non-realizable input is not stepped and its
// status is MSH_E_REALIZABILITY.  ensemble_end records the status of the state's steps.
__global__ void ensemble_start_kernel(Ctrl *c, int64_t step_base, int64_t nsteps, int32_t *status) {
  c->t = 0.0;
  c->step = step_base;
  c->sg_hist = 0;  // a new state has no previous self-gravity acceleration
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
  if (!c->realizable) {
    c->done = 1;
    c->status = 4;  // MSH_E_REALIZABILITY
    *status = 4;
    return;
  }
  *status = 0;
  c->t_end = INFINITY;
  c->max_step = step_base + nsteps;
  c->dt_max = INFINITY;
  c->done = 0;
  c->status = 0;
  c->stage_timeout = 0;
  plan(c);
}

__global__ void ensemble_end_kernel(const Ctrl *c, int32_t *status) {
  if (*status == 0) *status = c->status;
}

cudaError_t launch_ensemble_start(Ctrl *ctrl, int64_t step_base, int64_t nsteps, int32_t *status, cudaStream_t s) {
  ensemble_start_kernel<<<1, 1, 0, s>>>(ctrl, step_base, nsteps, status);
  return cudaGetLastError();
}

cudaError_t launch_ensemble_end(const Ctrl *ctrl, int32_t *status, cudaStream_t s) {
  ensemble_end_kernel<<<1, 1, 0, s>>>(ctrl, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------- conversions
template <typename T>
__global__ void convert_kernel(T *U, size_t N, int to_primitive) {
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    T a[NV], b[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) a[k] = U[k * N + c];
    if (to_primitive) cons_to_prim(a, b);
    else prim_to_cons(a, b);
#pragma unroll
    for (int k = 0; k < NV; k++) U[k * N + c] = b[k];
  }
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s, int *nblocks_out) {
  if (nblocks_out) *nblocks_out = step_blocks<T>(ndim, rows, a.nx, a.ny, a.nz, a.zchunk);
  return retry ? launch_step_mode<T, 0, true>(a, ndim, rows, s) : launch_step_mode<T, 0, false>(a, ndim, rows, s);
}

template <typename T>
cudaError_t launch_scan(const T *U, size_t N, int nx, int ny, int ndim, const double *dx, Partial *part,
                        int nparts, cudaStream_t s, size_t c0, size_t c1, bool maxf) {
  const T ix = (T)(1.0 / dx[0]), iy = (T)(1.0 / dx[1]), iz = (T)(1.0 / dx[2]);
  if (c1 == 0) c1 = N;
  if (ndim == 1) scan_kernel<T, 1, false><<<nparts, 256, 0, s>>>(U, N, c0, c1, ix, iy, iz, part);
  else if (ndim == 2 && maxf) scan_kernel<T, 2, true><<<nparts, 256, 0, s>>>(U, N, c0, c1, ix, iy, iz, part);
  else if (ndim == 2) scan_kernel<T, 2, false><<<nparts, 256, 0, s>>>(U, N, c0, c1, ix, iy, iz, part);
  else if (maxf) scan_kernel<T, 3, true><<<nparts, 256, 0, s>>>(U, N, c0, c1, ix, iy, iz, part);
  else scan_kernel<T, 3, false><<<nparts, 256, 0, s>>>(U, N, c0, c1, ix, iy, iz, part);
  return cudaGetLastError();
}

cudaError_t launch_set_dt(Ctrl *ctrl, double dt, cudaStream_t s) {
  set_dt_kernel<<<1, 1, 0, s>>>(ctrl, dt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gravity_field(const double *phi, T *acc, int ndim, int nx, int ny, int nz, const double *dx,
                                 cudaStream_t s) {
  gravity_field_kernel<T><<<kScanBlocks, 256, 0, s>>>(phi, acc, ndim, nx, ny, nz, dx[0], dx[1], dx[2]);
  return cudaGetLastError();
}

cudaError_t launch_finalize(Ctrl *ctrl, const Partial *part, int nparts, int mode, cudaStream_t s) {
  finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(ctrl, part, nparts, mode);
  return cudaGetLastError();
}

cudaError_t launch_run_start(Ctrl *ctrl, double t_end, int64_t max_steps, double dt_max, cudaStream_t s) {
  run_start_kernel<<<1, 1, 0, s>>>(ctrl, t_end, max_steps, dt_max);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_convert(T *U, size_t N, int to_primitive, cudaStream_t s) {
  const int blocks = (int)((N + 255) / 256 < (size_t)kScanBlocks ? (N + 255) / 256 : kScanBlocks);
  convert_kernel<T><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(U, N, to_primitive);
  return cudaGetLastError();
}

#define MSH_INST(T)                                                                                   \
  template cudaError_t launch_step<T>(const StepArgs<T> &, int, int, bool, cudaStream_t, int *);     \
  template int step_blocks<T>(int, int, int, int, int, int);                                         \
  template size_t step_smem<T>(int, int, bool, bool);                                                    \
  template cudaError_t launch_scan<T>(const T *, size_t, int, int, int, const double *, Partial *, int, \
                                      cudaStream_t, size_t, size_t, bool);                           \
  template cudaError_t launch_convert<T>(T *, size_t, int, cudaStream_t);                            \
  template cudaError_t launch_gravity_field<T>(const double *, T *, int, int, int, int, const double *, cudaStream_t);
MSH_INST(float)
MSH_INST(double)

}  // namespace msh
