// msh_batch.cu -- thousands of independent 1D Riemann problems ("tubes") in one
// persistent launch.
//
// Each thread block repeatedly takes the next tube from a device work queue (tubes are
// ordered longest first on the host, since the work of a tube grows as len^2), loads it
// into shared memory and advances it to its own t_end with a block-local CFL reduction;
// the tube never leaves shared memory until it is finished.  In shared memory a tube is held
// in primitive variables W, so the reconstruction reads its three cells without
// conversions; per step the block sweeps the tube in chunks of NT cells: reconstruction of
// the chunk's cells, HLL fluxes through their lower faces, and the conservative update
// U^{n+1} = U(W^n) - dt/dx (F_{i+1/2} - F_{i-1/2}) of the cell one behind the chunk front (a
// cell is updated once both of its faces are known; its W^n is the thread's left neighbour,
// already in registers), stored as W^{n+1} into the second tube buffer; the buffers swap
// roles after each step, so W^n stays intact for the fallback passes without a copy.
// The step is the same as the grid kernels': MUSCL-Hancock on the characteristic
// variables (Sec. 3.3), HLL flux, outflow boundaries by index clamping, CFL time step
// dt = C dx / max(|u| + sqrt(3 P_xx/rho)) with the last step clipped to t_end.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <numeric>

#include "../../include/msh.h"
#include "msh_device.cuh"
#include "msh_internal.h"

namespace msh {

template <typename T> struct TubeArgs {
  T *U;                    // [NV][total] conserved, tubes back to back
  const int64_t *off;      // [ntubes] first cell of each tube
  const int32_t *len;      // [ntubes]
  const double *t_end;     // [ntubes]
  const int32_t *order;    // [ntubes] processing order (longest first)
  int32_t *queue;          // work-queue head
  int64_t *steps;          // [ntubes] out
  double *t_out;           // [ntubes] out
  int32_t *status;         // [ntubes] out: 0 ok, 4 non-realizable, 5 step cap reached
  int64_t *fallback;       // [ntubes] out: steps whose second-order update tagged cells
  int64_t total;
  int32_t ntubes;
  int32_t cap;             // shared-memory capacity in cells (>= max len)
  double cfl;
  int64_t max_steps;
};

template <typename T> __device__ __forceinline__ void load_w(const T *sW, int cap, int c, int n, T (&W)[NV]) {
  const int cc = min(max(c, 0), n - 1);  // outflow: zero-gradient copy of the edge cell
#pragma unroll
  for (int k = 0; k < NV; k++) W[k] = sW[k * cap + cc];
}

template <typename T, int NT> __device__ __forceinline__ T block_max(T v, T *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  T m = red[0];
#pragma unroll
  for (int i = 1; i < NT / 32; i++) m = fmax(m, red[i]);
  __syncthreads();
  return m;
}

// One sweep of a tube over all its faces: reconstruction, HLL fluxes and the conservative
// update, chunk by chunk.  src holds W^n; dst receives W^{n+1} (a different buffer).  With FALLBACK, every face that
// touches a cell tagged by an earlier pass (sFl == 2) takes first-order states.  Cells whose
// update is not realizable and that carry no active tag are tagged (sFl = 1) and *s_nbad
// is set.  Returns the thread's maximum signal-speed sum of the new state.
template <typename T, int NT, bool FALLBACK>
__device__ T tube_pass(const T *src, T *dst, unsigned char *sFl, int n, int cap, T nu, T dtdx, T idx, T *sF,
                       T *sH, T *sHc, int *s_nbad, int *s_any) {
  const int t = threadIdx.x;
  T smax = T(0);
  for (int b = -1; b <= n; b += NT) {
    const int c = b + t;
    T lo[NV], hi[NV], wm[NV];  // wm: W^n of the cell this thread updates (c - 1)
    if (c <= n) {
      T w0[NV], wp[NV];
      load_w(src, cap, c - 1, n, wm);
      load_w(src, cap, c, n, w0);
      load_w(src, cap, c + 1, n, wp);
      reconstruct(wm, w0, wp, nu, lo, hi);
      if (FALLBACK) {  // tags of earlier passes (value 2) are active in this pass
        auto f = [&](int i) { return sFl[min(max(i, 0), n - 1)] == 2; };
        first_order_faces(f(c - 1), f(c), f(c + 1), w0, lo, hi);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) sH[v * NT + t] = hi[v];
    }
    __syncthreads();
    if (c >= 0 && c <= n) {
      T hl[NV], F[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) hl[v] = (t > 0) ? sH[v * NT + t - 1] : sHc[v];
      hll(hl, lo, F);
#pragma unroll
      for (int v = 0; v < NV; v++) sF[v * (NT + 1) + t + 1] = F[v];
    }
    __syncthreads();
    // the last thread hands its hi face state to the next chunk (read after the next
    // barrier; every read of the current carry happened before the barrier above)
    if (t == NT - 1 && c <= n) {
#pragma unroll
      for (int v = 0; v < NV; v++) sHc[v] = hi[v];
    }
    const int cu = b - 1 + t;  // cell whose two faces are now known (= c - 1: its W^n is wm)
    if (cu >= 0 && cu < n) {
      T U[NV], W[NV];
      prim_to_cons(wm, U);
#pragma unroll
      for (int v = 0; v < NV; v++) U[v] -= dtdx * (sF[v * (NT + 1) + t + 1] - sF[v * (NT + 1) + t]);
      cons_to_prim(U, W);
#pragma unroll
      for (int v = 0; v < NV; v++) dst[v * cap + cu] = W[v];
      if (!realizable(W)) {
        *s_any = 1;
        if (sFl[cu] != 2) {  // newly failing cell: tag it for the next pass
          sFl[cu] = 1;
          *s_nbad = 1;
        }
      }
      smax = fmax(smax, (fabs(W[1]) + T(1.7320508075688772) * sqrt_ratio(W[4], W[0])) * idx);
    }
    __syncthreads();
    if (t == 0) {  // the last face of this chunk is the lower face of the next chunk's first update
#pragma unroll
      for (int v = 0; v < NV; v++) sF[v * (NT + 1)] = sF[v * (NT + 1) + NT];
    }
  }
  return smax;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) tubes_kernel(TubeArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cap = a.cap;
  // two tube buffers (primitive): a step reads W^n from one and writes W^{n+1} to the other
  // (the fallback passes re-read the untouched W^n), then the two swap roles
  T *sU = reinterpret_cast<T *>(smem_raw);  // [NV][cap]
  T *sUo = sU + (size_t)NV * cap;           // [NV][cap]
  T *sF = sUo + (size_t)NV * cap;           // [NV][NT+1]: sF[0] = carried face, sF[t+1] = lower face of cell b+t
  T *sH = sF + NV * (NT + 1);               // [NV][NT]: hi face states of the chunk
  T *sHc = sH + NV * NT;                    // [NV]: hi face state of the cell before the chunk
  unsigned char *sFl = reinterpret_cast<unsigned char *>(sHc + NV);  // [cap] fallback tags
  __shared__ T red[NT / 32];
  __shared__ int s_q;
  __shared__ int s_nbad, s_any;
  const int t = threadIdx.x;
  for (;;) {
    if (t == 0) s_q = atomicAdd(a.queue, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= a.ntubes) break;
    const int k = a.order[q];
    const int n = a.len[k];
    const int64_t off = a.off[k];
    T *cur = sU, *nxt = sUo;  // W^n and W^{n+1} of the current step
    for (int c = t; c < n; c += NT) {
      T U[NV], W[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) U[v] = a.U[v * a.total + off + c];
      cons_to_prim(U, W);
#pragma unroll
      for (int v = 0; v < NV; v++) cur[v * cap + c] = W[v];
      sFl[c] = 0;
    }
    __syncthreads();
    const T idx = (T)n, half_idx = T(0.5) * idx;
    // signal-speed sum of the initial state
    T sm = T(0);
    for (int c = t; c < n; c += NT) {
      T W[NV];
      load_w(cur, cap, c, n, W);
      sm = fmax(sm, (fabs(W[1]) + T(1.7320508075688772) * sqrt_ratio(W[4], W[0])) * idx);
    }
    sm = block_max<T, NT>(sm, red);
    double tt = 0.0;
    const double te = a.t_end[k];
    int64_t steps = 0, fb_steps = 0;
    int status = 0;
    while (tt < te) {
      if (steps >= a.max_steps) { status = 5; break; }
      double dt = a.cfl / (double)sm;
      double tn = tt + dt;
      if (tn >= te) { dt = te - tt; tn = te; }
      const T nu = (T)dt * half_idx, dtdx = (T)dt * idx;
      if (t == 0) { s_nbad = 0; s_any = 0; }
      __syncthreads();
      T smax = tube_pass<T, NT, false>(cur, nxt, sFl, n, cap, nu, dtdx, idx, sF, sH, sHc, &s_nbad, &s_any);
      sm = block_max<T, NT>(smax, red);  // its barriers also order the carries and s_nbad
      fb_steps += s_nbad != 0;
      // a-posteriori fallback: redo the step from U^n with first-order faces at every tagged
      // cell; cells still failing are tagged too (at most kFallbackPasses passes)
      for (int pass = 1; pass <= kFallbackPasses && s_nbad; pass++) {
        __syncthreads();
        if (t == 0) { s_nbad = 0; s_any = 0; }
        __syncthreads();
        for (int c = t; c < n; c += NT)
          if (sFl[c] == 1) sFl[c] = 2;  // tags of earlier passes become active
        __syncthreads();
        smax = tube_pass<T, NT, true>(cur, nxt, sFl, n, cap, nu, dtdx, idx, sF, sH, sHc, &s_nbad, &s_any);
        sm = block_max<T, NT>(smax, red);
      }
      const bool still_bad = s_any != 0;  // some cell of the last pass is not realizable
      for (int c = t; c < n; c += NT) sFl[c] = 0;
      __syncthreads();
      T *sw = cur;  // U^{n+1} becomes the next step's U^n
      cur = nxt;
      nxt = sw;
      if (still_bad) { status = 4; tt = tn; steps++; break; }
      tt = tn;
      steps++;
    }
    __syncthreads();
    for (int c = t; c < n; c += NT) {
      T W[NV], U[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) W[v] = cur[v * cap + c];
      prim_to_cons(W, U);
#pragma unroll
      for (int v = 0; v < NV; v++) a.U[v * a.total + off + c] = U[v];
    }
    if (t == 0) {
      a.steps[k] = steps;
      a.t_out[k] = tt;
      a.status[k] = status;
      a.fallback[k] = fb_steps;
    }
    __syncthreads();
  }
}

template <typename T> size_t tube_smem(int cap, int nt) {
  return sizeof(T) * (2 * (size_t)NV * cap + (size_t)NV * (nt + 1) + (size_t)NV * nt + NV) + (size_t)cap;
}

template <typename T, int NT> static cudaError_t launch_tubes_nt(const TubeArgs<T> &a, int blocks, cudaStream_t s) {
  const size_t smem = tube_smem<T>(a.cap, NT);
  cudaError_t e = cudaFuncSetAttribute(tubes_kernel<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tubes_kernel<T, NT><<<blocks, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T> int tube_blocks(int cap, int nt) {
  int dev = 0, sms = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t per = tube_smem<T>(cap, nt) + 1024;
  int per_sm = (int)(maxsm / per);
  per_sm = std::max(1, std::min(per_sm, 2048 / nt));
  return sms * per_sm;
}

template <typename T> cudaError_t launch_tubes(const TubeArgs<T> &a, int nt, cudaStream_t s) {
  const int blocks = std::min(tube_blocks<T>(a.cap, nt), (int)a.ntubes);
  if (nt == 128) return launch_tubes_nt<T, 128>(a, blocks, s);
  if (nt == 512) return launch_tubes_nt<T, 512>(a, blocks, s);
  return launch_tubes_nt<T, 256>(a, blocks, s);
}

}  // namespace msh

// ======================================================================= host
using namespace msh;

namespace {
msh_status bfail(msh_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_text(buf);
  return s;
}
#define B_TRY(expr)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return bfail(e_ == cudaErrorMemoryAllocation ? MSH_E_NOMEM : MSH_E_CUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                     \
  } while (0)
}  // namespace

struct msh_batch {
  int ntubes = 0;
  int prec = MSH_FP32;
  size_t esize = 4;
  double cfl = 0.8;
  int64_t total = 0;
  int cap = 0;
  int threads = 0;  // chosen block size (0 = not tuned yet)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<int32_t> len;
  std::vector<int64_t> off;
  std::vector<double> t_end;
  std::vector<unsigned char> init;  // initial conserved state, host copy for reset
  void *U = nullptr;
  int64_t *d_off = nullptr;
  int32_t *d_len = nullptr, *d_order = nullptr, *d_queue = nullptr, *d_status = nullptr;
  double *d_tend = nullptr, *d_t = nullptr;
  int64_t *d_steps = nullptr;
  int64_t *d_fallback = nullptr;
  std::vector<msh_grid *> grids;  // per-tube grids of the per-launch baseline (lazily built)
};

namespace {

template <typename T> void fill_initial(msh_batch *b, const double *WL, const double *WR) {
  T *h = reinterpret_cast<T *>(b->init.data());
  for (int k = 0; k < b->ntubes; k++) {
    const int n = b->len[k];
    for (int i = 0; i < n; i++) {
      const double x = (i + 0.5) / n;
      const double *w = (x < 0.5) ? WL + 10 * k : WR + 10 * k;
      for (int v = 0; v < NV; v++) h[v * b->total + b->off[k] + i] = (T)w[v];
    }
  }
}

msh_status upload_initial(msh_batch *b) {
  const size_t bytes = (size_t)b->total * NV * b->esize;
  B_TRY(cudaMemcpyAsync(b->U, b->init.data(), bytes, cudaMemcpyHostToDevice, b->stream));
  cudaError_t e = b->prec == MSH_FP32 ? launch_convert<float>((float *)b->U, (size_t)b->total, 0, b->stream)
                                      : launch_convert<double>((double *)b->U, (size_t)b->total, 0, b->stream);
  if (e != cudaSuccess) return bfail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
  B_TRY(cudaMemsetAsync(b->d_steps, 0, sizeof(int64_t) * b->ntubes, b->stream));
  B_TRY(cudaMemsetAsync(b->d_fallback, 0, sizeof(int64_t) * b->ntubes, b->stream));
  B_TRY(cudaMemsetAsync(b->d_t, 0, sizeof(double) * b->ntubes, b->stream));
  B_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int32_t) * b->ntubes, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  return MSH_OK;
}

msh_status run_once(msh_batch *b, int nt, int64_t max_steps) {
  B_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(int32_t), b->stream));
  cudaError_t e;
  if (b->prec == MSH_FP32) {
    TubeArgs<float> a{(float *)b->U, b->d_off, b->d_len, b->d_tend, b->d_order, b->d_queue, b->d_steps, b->d_t,
                      b->d_status, b->d_fallback, b->total, b->ntubes, b->cap, b->cfl, max_steps};
    e = launch_tubes<float>(a, nt, b->stream);
  } else {
    TubeArgs<double> a{(double *)b->U, b->d_off, b->d_len, b->d_tend, b->d_order, b->d_queue, b->d_steps, b->d_t,
                       b->d_status, b->d_fallback, b->total, b->ntubes, b->cap, b->cfl, max_steps};
    e = launch_tubes<double>(a, nt, b->stream);
  }
  if (e != cudaSuccess) return bfail(MSH_E_CUDA, "tube kernel launch: %s", cudaGetErrorString(e));
  return MSH_OK;
}

msh_status check_status(msh_batch *b) {
  std::vector<int32_t> st(b->ntubes);
  B_TRY(cudaMemcpyAsync(st.data(), b->d_status, sizeof(int32_t) * b->ntubes, cudaMemcpyDeviceToHost, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < b->ntubes; k++) {
    if (st[k] == 4) return bfail(MSH_E_REALIZABILITY, "tube %d became non-realizable", k);
    if (st[k] == 5) return bfail(MSH_E_TIMEOUT, "tube %d reached max_steps before t_end", k);
  }
  return MSH_OK;
}

}  // namespace

extern "C" {

msh_status msh_batch_init(msh_batch **out, int32_t ntubes, const int32_t *len, const double *WL, const double *WR,
                          const double *t_end, int32_t precision, double cfl, void *stream) {
  clear_error();
  if (!out || !len || !WL || !WR || !t_end) return bfail(MSH_E_INVALID_ARG, "null argument");
  if (ntubes < 1) return bfail(MSH_E_INVALID_ARG, "ntubes must be >= 1");
  if (precision != MSH_FP32 && precision != MSH_FP64) return bfail(MSH_E_INVALID_ARG, "bad precision");
  if (!(cfl > 0.0 && cfl <= 1.0)) return bfail(MSH_E_INVALID_ARG, "cfl must be in (0, 1]");
  const int maxlen = precision == MSH_FP32 ? 2048 : 1024;
  int cap = 0;
  for (int k = 0; k < ntubes; k++) {
    if (len[k] < 4 || len[k] > maxlen) return bfail(MSH_E_INVALID_ARG, "len[%d] = %d outside [4, %d]", k, len[k], maxlen);
    if (!(t_end[k] > 0.0) || !std::isfinite(t_end[k])) return bfail(MSH_E_INVALID_ARG, "t_end[%d] must be > 0", k);
    for (int v = 0; v < NV; v++)
      if (!std::isfinite(WL[10 * k + v]) || !std::isfinite(WR[10 * k + v]))
        return bfail(MSH_E_INVALID_ARG, "non-finite state of tube %d", k);
    // realizability of the two input states (rho > 0, P SPD)
    for (const double *w : {WL + 10 * k, WR + 10 * k}) {
      const double m2 = w[4] * w[7] - w[5] * w[5];
      const double m3 = w[4] * (w[7] * w[9] - w[8] * w[8]) - w[5] * (w[5] * w[9] - w[8] * w[6]) +
                        w[6] * (w[5] * w[8] - w[7] * w[6]);
      if (!(w[0] > 0 && w[4] > 0 && m2 > 0 && m3 > 0))
        return bfail(MSH_E_REALIZABILITY, "input state of tube %d not realizable", k);
    }
    cap = std::max(cap, (int)len[k]);
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return bfail(MSH_E_CUDA, "no CUDA device available (libmsh has no CPU path)");
  msh_batch *b = new (std::nothrow) msh_batch();
  if (!b) return bfail(MSH_E_NOMEM, "host allocation");
  b->ntubes = ntubes;
  b->prec = precision;
  b->esize = precision == MSH_FP32 ? 4 : 8;
  b->cfl = cfl;
  b->cap = cap;
  b->len.assign(len, len + ntubes);
  b->t_end.assign(t_end, t_end + ntubes);
  b->off.resize(ntubes);
  int64_t acc = 0;
  for (int k = 0; k < ntubes; k++) {
    b->off[k] = acc;
    acc += len[k];
  }
  b->total = acc;
  std::vector<int32_t> order(ntubes);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return len[x] > len[y]; });
  b->init.resize((size_t)b->total * NV * b->esize);
  if (precision == MSH_FP32) fill_initial<float>(b, WL, WR);
  else fill_initial<double>(b, WL, WR);
  auto cleanup = [&](msh_status s) {
    msh_batch_destroy(b);
    return s;
  };
  cudaError_t e = cudaSuccess;
  if (stream) b->stream = (cudaStream_t)stream;
  else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->U, (size_t)b->total * NV * b->esize);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_off, sizeof(int64_t) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_len, sizeof(int32_t) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int32_t) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int32_t) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tend, sizeof(double) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_t, sizeof(double) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_steps, sizeof(int64_t) * ntubes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fallback, sizeof(int64_t) * ntubes);
  if (e != cudaSuccess) return cleanup(bfail(MSH_E_NOMEM, "batch allocation: %s", cudaGetErrorString(e)));
  e = cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(int64_t) * ntubes, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_len, len, sizeof(int32_t) * ntubes, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * ntubes, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tend, t_end, sizeof(double) * ntubes, cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cleanup(bfail(MSH_E_CUDA, "batch upload: %s", cudaGetErrorString(e)));
  msh_status st = upload_initial(b);
  if (st) return cleanup(st);
  *out = b;
  return MSH_OK;
}

msh_status msh_batch_reset(msh_batch *b) {
  clear_error();
  if (!b) return bfail(MSH_E_INVALID_ARG, "null batch");
  return upload_initial(b);
}

msh_status msh_batch_run(msh_batch *b, int32_t threads, int64_t max_steps) {
  msh::NvtxRange nvtx_range("msh_batch_run");
  clear_error();
  if (!b) return bfail(MSH_E_INVALID_ARG, "null batch");
  if (threads != 0 && threads != 128 && threads != 256 && threads != 512)
    return bfail(MSH_E_INVALID_ARG, "threads must be 0, 128, 256 or 512");
  if (max_steps < 1) return bfail(MSH_E_INVALID_ARG, "max_steps must be >= 1");
  int nt = threads;
  if (nt == 0 && b->threads == 0) {
    // autotune: time each block size on a full run from the initial state
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_nt = 256;
    for (int cand : {128, 256, 512}) {
      const size_t need = b->prec == MSH_FP32 ? tube_smem<float>(b->cap, cand) : tube_smem<double>(b->cap, cand);
      if (need > 227 * 1024) continue;
      msh_status st = upload_initial(b);
      if (st) return st;
      B_TRY(cudaEventRecord(e0, b->stream));
      st = run_once(b, cand, max_steps);
      if (st) return st;
      B_TRY(cudaEventRecord(e1, b->stream));
      B_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      B_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_nt = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->threads = best_nt;
    msh_status st = upload_initial(b);
    if (st) return st;
  }
  if (nt == 0) nt = b->threads;
  const size_t smem = b->prec == MSH_FP32 ? tube_smem<float>(b->cap, nt) : tube_smem<double>(b->cap, nt);
  if (smem > 227 * 1024) return bfail(MSH_E_INVALID_ARG, "tubes too long for %d threads (%zu B shared)", nt, smem);
  // one persistent launch, captured in a CUDA graph (queue reset + kernel)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  B_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  msh_status st = run_once(b, nt, max_steps);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return bfail(MSH_E_CUDA, "capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(MSH_E_CUDA, "instantiate: %s", cudaGetErrorString(e));
  e = cudaGraphLaunch(exec, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return bfail(MSH_E_CUDA, "tube run: %s", cudaGetErrorString(e));
  return check_status(b);
}

msh_status msh_batch_run_per_tube(msh_batch *b, const int32_t *tubes, int32_t count, int64_t max_steps) {
  msh::NvtxRange nvtx_range("msh_batch_run_per_tube");
  clear_error();
  if (!b) return bfail(MSH_E_INVALID_ARG, "null batch");
  if (tubes && count < 0) return bfail(MSH_E_INVALID_ARG, "bad count");
  const int m = tubes ? count : b->ntubes;
  if ((int)b->grids.size() < b->ntubes) b->grids.resize(b->ntubes, nullptr);
  for (int i = 0; i < m; i++) {
    const int k = tubes ? tubes[i] : i;
    if (k < 0 || k >= b->ntubes) return bfail(MSH_E_INVALID_ARG, "tube index %d out of range", k);
    if (!b->grids[k]) {
      const int64_t n3[3] = {b->len[k], 1, 1};
      const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
      const int32_t bc[6] = {MSH_BC_OUTFLOW, MSH_BC_OUTFLOW, 0, 0, 0, 0};
      msh_status st = msh_init_grid(&b->grids[k], 1, n3, lo, hi, bc, b->prec, b->cfl, b->stream);
      if (st) return bfail(st, "per-tube grid: %s", msh_last_error());
    }
    msh_grid *g = b->grids[k];
    const size_t n = (size_t)b->len[k];
    // gather tube k ([10][n]) from the batch state, run it alone, scatter it back
    void *tmp = nullptr;
    B_TRY(cudaMallocAsync(&tmp, n * NV * b->esize, b->stream));
    B_TRY(cudaMemcpy2DAsync(tmp, n * b->esize, (char *)b->U + b->off[k] * b->esize, b->total * b->esize,
                            n * b->esize, NV, cudaMemcpyDeviceToDevice, b->stream));
    msh_status st = msh_set_time(g, 0.0, 0);
    if (!st) st = msh_set_state(g, tmp, MSH_DEVICE, MSH_CONSERVED);
    int64_t steps = 0;
    double tt = 0.0;
    if (!st) st = msh_run(g, b->t_end[k], max_steps, &steps, &tt);
    if (!st) st = msh_get_state(g, tmp, MSH_DEVICE, MSH_CONSERVED);
    if (st) {
      cudaFreeAsync(tmp, b->stream);
      return bfail(st, "tube %d: %s", k, msh_last_error());
    }
    B_TRY(cudaMemcpy2DAsync((char *)b->U + b->off[k] * b->esize, b->total * b->esize, tmp, n * b->esize,
                            n * b->esize, NV, cudaMemcpyDeviceToDevice, b->stream));
    B_TRY(cudaFreeAsync(tmp, b->stream));
    B_TRY(cudaMemcpyAsync(b->d_steps + k, &steps, sizeof(int64_t), cudaMemcpyHostToDevice, b->stream));
    B_TRY(cudaMemcpyAsync(b->d_t + k, &tt, sizeof(double), cudaMemcpyHostToDevice, b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
  }
  return MSH_OK;
}

msh_status msh_batch_get_state(msh_batch *b, void *U, int32_t where, int32_t kind) {
  clear_error();
  if (!b || !U) return bfail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return bfail(MSH_E_INVALID_ARG, "bad where");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return bfail(MSH_E_INVALID_ARG, "bad kind");
  const size_t bytes = (size_t)b->total * NV * b->esize;
  const void *src = b->U;
  void *tmp = nullptr;
  if (kind == MSH_PRIMITIVE) {
    B_TRY(cudaMallocAsync(&tmp, bytes, b->stream));
    B_TRY(cudaMemcpyAsync(tmp, b->U, bytes, cudaMemcpyDeviceToDevice, b->stream));
    cudaError_t e = b->prec == MSH_FP32 ? launch_convert<float>((float *)tmp, (size_t)b->total, 1, b->stream)
                                        : launch_convert<double>((double *)tmp, (size_t)b->total, 1, b->stream);
    if (e != cudaSuccess) return bfail(MSH_E_CUDA, "convert: %s", cudaGetErrorString(e));
    src = tmp;
  }
  B_TRY(cudaMemcpyAsync(U, src, bytes, where == MSH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        b->stream));
  if (tmp) B_TRY(cudaFreeAsync(tmp, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  return MSH_OK;
}

msh_status msh_batch_info(msh_batch *b, int64_t *steps, double *t, int64_t *cell_updates) {
  clear_error();
  if (!b) return bfail(MSH_E_INVALID_ARG, "null batch");
  std::vector<int64_t> s(b->ntubes);
  std::vector<double> tt(b->ntubes);
  B_TRY(cudaMemcpyAsync(s.data(), b->d_steps, sizeof(int64_t) * b->ntubes, cudaMemcpyDeviceToHost, b->stream));
  B_TRY(cudaMemcpyAsync(tt.data(), b->d_t, sizeof(double) * b->ntubes, cudaMemcpyDeviceToHost, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  if (steps) memcpy(steps, s.data(), sizeof(int64_t) * b->ntubes);
  if (t) memcpy(t, tt.data(), sizeof(double) * b->ntubes);
  if (cell_updates) {
    int64_t cu = 0;
    for (int k = 0; k < b->ntubes; k++) cu += s[k] * b->len[k];
    *cell_updates = cu;
  }
  return MSH_OK;
}

msh_status msh_batch_fallback_steps(msh_batch *b, int64_t *counts) {
  clear_error();
  if (!b || !counts) return bfail(MSH_E_INVALID_ARG, "null argument");
  B_TRY(cudaMemcpyAsync(counts, b->d_fallback, sizeof(int64_t) * b->ntubes, cudaMemcpyDeviceToHost, b->stream));
  B_TRY(cudaStreamSynchronize(b->stream));
  return MSH_OK;
}

msh_status msh_batch_destroy(msh_batch *b) {
  if (!b) return MSH_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto *g : b->grids)
    if (g) msh_destroy(g);
  cudaFree(b->U);
  cudaFree(b->d_off);
  cudaFree(b->d_len);
  cudaFree(b->d_order);
  cudaFree(b->d_queue);
  cudaFree(b->d_status);
  cudaFree(b->d_tend);
  cudaFree(b->d_t);
  cudaFree(b->d_steps);
  cudaFree(b->d_fallback);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return MSH_OK;
}

}  // extern "C"
