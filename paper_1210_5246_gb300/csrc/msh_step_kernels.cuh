// msh_step_kernels.cuh -- the step kernels of libmsh and their launch templates.
//
// One launch = one full step (or one Runge-Kutta stage of the central scheme): boundary
// handling by index mapping (guardcells, Sec. 3.1), conserved -> primitive,
// per-direction reconstruction and face fluxes (characteristic MUSCL-Hancock with HLL,
// Sec. 3.3; or the Kurganov-Tadmor central scheme, Sec. 3.2), unsplit conservative update,
// gravity source after the hydro update (Sec. 3.3, last paragraph), and per-block partials
// of the next CFL time step, the FP64 conserved totals and the realizability check.
//
// 3D kernel layout: a thread block is a 32 x ROWS grid of threads covering cells
// (x0-1 .. x0+30, y0-1 .. y0+ROWS-2); the 30 x (ROWS-2) interior cells are updated, the
// ring of halo threads reconstructs the neighbours whose face states the interior needs.
// z planes stream through a three-plane shared-memory ring (2.5D): x and y fluxes come
// from the current plane, the z flux is carried in registers from plane to plane, so
// every cell is reconstructed once per direction.  Each plane of a tile's staged box
// arrives one plane ahead by one bulk tensor copy (TMA) completed on an mbarrier, the
// cells of the box outside the grid fixed up afterwards from their mapped cells; a block
// streams whole columns of tiles or equal runs of planes (balanced tiling), or chunks of
// zchunk planes.  2D: one warp per 32-column strip streamed in y (step_strip2d_kernel).
//
// Template parameter SCH: 0 MUSCL-Hancock (the step); 1, 2 the two stages of the central
// scheme (stage 1 writes U1 = U^n + dt L(U^n), stage 2 sweeps U1 and writes
// (U^n + U1 + dt L(U1)) / 2 with the source and the partials).
#pragma once
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <cstring>
#include <utility>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "msh_device.cuh"
#include "msh_internal.h"

namespace msh {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ block partials
template <int NT>
__device__ __forceinline__ void block_partial(double (&diag)[NV], double smax, long long bad,
                                              Partial *out, const double *base = nullptr) {
  __shared__ double red[NT / 32][NV + 1];
  __shared__ long long redb[NT / 32];
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; k++) diag[k] += __shfl_down_sync(FULL, diag[k], o);
    smax = fmax(smax, __shfl_down_sync(FULL, smax, o));
    bad = min(bad, __shfl_down_sync(FULL, bad, o));
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) red[warp][k] = diag[k];
    red[warp][NV] = smax;
    redb[warp] = bad;
  }
  __syncthreads();
  if (tid == 0) {
    Partial p;
    for (int k = 0; k < NV; k++) p.diag[k] = base != nullptr ? base[k] : 0.0;
    p.smax = 0.0;
    p.bad = LLONG_MAX;
    for (int w = 0; w < NT / 32; w++) {
      for (int k = 0; k < NV; k++) p.diag[k] += red[w][k];
      p.smax = fmax(p.smax, red[w][NV]);
      p.bad = min(p.bad, redb[w]);
    }
    *out = p;
  }
}

// Sum over active dims of (|u_d| + sqrt(3 P_dd / rho)) / dx_d: the CFL signal-speed sum.
// MAXF (the corner-transport-upwind step): the maximum over the dims instead of the sum.
template <typename T, int NDIM, bool MAXF = false>
__device__ __forceinline__ T speed_sum(const T (&W)[NV], T idx, T idy, T idz) {
  T s = (fabs(W[1]) + sqrt_ratio(W[4], W[0]) * T(1.7320508075688772)) * idx;
  if (NDIM > 1) {
    const T sy = (fabs(W[2]) + sqrt_ratio(W[7], W[0]) * T(1.7320508075688772)) * idy;
    s = MAXF ? fmax(s, sy) : s + sy;
  }
  if (NDIM > 2) {
    const T sz = (fabs(W[3]) + sqrt_ratio(W[9], W[0]) * T(1.7320508075688772)) * idz;
    s = MAXF ? fmax(s, sz) : s + sz;
  }
  return s;
}

// Checkpoint slot of the adjoint tape that step `step` stores U^step into, or nullptr.
template <typename T> __device__ __forceinline__ T *tape_slot(const StepArgs<T> &a, int64_t step, size_t N) {
  if (a.ck == nullptr) return nullptr;
  const int64_t ts = step - a.ck_base;
  if (ts < 0 || ts >= a.ck_len || ts % a.ck_K != 0) return nullptr;
  return a.ck + (size_t)(ts / a.ck_K) * NV * N;
}

// Per-cell tail of the step: gravity source, store, next-dt speed, realizability, totals;
// U^n also goes to the tape's checkpoint `ck` when the step has one.
// U^n of the cell is read from src[k * stride] (the state in global memory, or a staged
// copy in shared memory).
// SCH 0: U^{n+1} = U^n + dt L (MUSCL-Hancock); SCH 1: U1 = U^n + dt L(U^n) (the first
// Runge-Kutta stage, stored without sources or partials); SCH 2: U^{n+1} =
// (U^n + U1 + dt L(U1)) / 2 with src = U1 and un0 = U^n of the cell (fields N apart).
template <typename T, int NDIM, int SCH, bool RETRY, bool CTU = false>
__device__ __forceinline__ void finish_cell(const StepArgs<T> &a, const T *src, size_t stride, const T *un0,
                                            T *__restrict__ Ud, size_t N, size_t c,
                                            const T (&acc)[NV], T dt, T idx, T idy, T idz, Acc<T> &diag,
                                            T &smax, long long &bad, int32_t tag, T *__restrict__ ck) {
  T Un[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T u = src[k * stride];
    if (SCH == 0 && !RETRY && ck != nullptr) ck[k * N + c] = u;
    if (SCH == 2) Un[k] = T(0.5) * (un0[k * N] + (u + dt * acc[k]));
    else Un[k] = fma(dt, acc[k], u);
  }
  if (SCH == 1) {
#pragma unroll
    for (int k = 0; k < NV; k++) Ud[k * N + c] = Un[k];
    return;
  }
  if (a.acc != nullptr) {
    // a = -grad Phi: m += dt rho a, E += dt (mbar a^T + a mbar^T), mbar = (m* + m^{n+1})/2
    T g[3] = {T(0), T(0), T(0)};
    g[0] = a.acc[c];
    if (NDIM > 1) g[1] = a.acc[N + c];
    if (NDIM > 2) g[2] = a.acc[2 * N + c];
    T mb[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const T mn = Un[1 + i] + dt * Un[0] * g[i];
      mb[i] = T(0.5) * (Un[1 + i] + mn);
      Un[1 + i] = mn;
    }
    Un[4] += dt * T(2) * mb[0] * g[0];
    Un[5] += dt * (mb[0] * g[1] + g[0] * mb[1]);
    Un[6] += dt * (mb[0] * g[2] + g[0] * mb[2]);
    Un[7] += dt * T(2) * mb[1] * g[1];
    Un[8] += dt * (mb[1] * g[2] + g[1] * mb[2]);
    Un[9] += dt * T(2) * mb[2] * g[2];
  }
  {  // a running pointer: one 64-bit add per field instead of an index product
    T *d = Ud + c;
#pragma unroll
    for (int k = 0; k < NV; k++) {
      *d = Un[k];
      d += N;
    }
  }
  T W[NV];
  cons_to_prim(Un, W);
  if (!realizable(W)) {
    bad = min(bad, (long long)c);
    if (!kCharacteristic<SCH>) goto done;  // the central scheme has no a-posteriori fallback
    {
    // tag the cell for the next fallback pass (a cell tagged by an earlier pass keeps its tag)
    const int32_t f = a.flags[c];
    if (!((f >> 3) == tag && (f & 7) < a.level)) {
      a.flags[c] = tag * 8 + a.level;
      atomicAdd(&a.ctrl->nbad[a.level], 1);
    }
    }
  }
done:
  smax = fmax(smax, speed_sum<T, NDIM, CTU>(W, idx, idy, idz));
  diag.add(Un);
}

template <typename T, int NT>
__device__ __forceinline__ void write_partial(const Acc<T> &diag, T smax, long long bad, Partial *out) {
  double d[NV];
  diag.get(d);
  block_partial<NT>(d, (double)smax, bad, out);
}
// The same with FP64 totals `base` (block_totals) added to the threads' sums.
template <typename T, int NT>
__device__ __forceinline__ void write_partial(const Acc<T> &diag, T smax, long long bad, Partial *out,
                                              const double *base) {
  double d[NV];
  diag.get(d);
  block_partial<NT>(d, (double)smax, bad, out, base);
}

// FP64 running totals of a thread block, in shared memory (thread 0 writes them).
__device__ __forceinline__ double *block_totals() {
  __shared__ double tot[NV];
  return tot;
}

// Move the threads' running sums into the block's FP64 totals (fixed order: warps by
// shuffles, then thread 0 over the warps) and restart them from zero.  Every thread of the
// block calls it.
template <typename T, int NT> __device__ __forceinline__ void flush_totals(Acc<T> &diag, double *tot) {
  __shared__ double red[NT / 32][NV];
  double d[NV];
  diag.get(d);
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; k++) d[k] += __shfl_down_sync(FULL, d[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) red[tid >> 5][k] = d[k];
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 0; w < NT / 32; w++)
      for (int k = 0; k < NV; k++) tot[k] += red[w][k];
  }
  diag.zero();
}

// A cell takes first-order faces in fallback pass `level` if an earlier pass of this step
// tagged it.  Tags written during the current pass are ignored, so every thread block of
// a pass sees the same tagged set.
__device__ __forceinline__ bool tagged(int32_t f, int32_t tag, int level) {
  return (f >> 3) == tag && (f & 7) < level;
}

// ------------------------------------------------------------------ 1D kernel
template <typename T, int SCH, bool RETRY>
__global__ void __launch_bounds__(kTile1D) step1d_kernel(StepArgs<T> a) {
  constexpr int B = kTile1D, SXX = B + 2;
  const Ctrl *ctrl = a.ctrl;
  if (ctrl->done) return;
  if (RETRY && ctrl->nbad[a.level - 1] == 0 && !((ctrl->force >> a.level) & 1)) return;
  const int64_t step = ctrl->step;
  const int32_t tag = (int32_t)(step & 0x0fffffff) + 1;
  __shared__ unsigned char sFl[RETRY ? SXX : 1];
  // sweep source, destination and U^n (the second Runge-Kutta stage sweeps U1)
  const T *__restrict__ U0 = a.U[step & 1];
  const T *__restrict__ Us = SCH == 2 ? a.U1 : U0;
  T *__restrict__ Ud = SCH == 1 ? a.U1 : a.U[(step + 1) & 1];
  const double dtd = ctrl->dt;
  const T dt = (T)dtd, nu = (T)(0.5 * dtd / a.dx[0]), idx = (T)(1.0 / a.dx[0]);
  __shared__ T sW[NV][SXX];
  __shared__ T sH[NV][B];
  const int t = threadIdx.x;
  const int nx = a.nx;
  const size_t N = (size_t)nx;
  const int ntiles = (nx + B - 3) / (B - 2);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const int x0 = tile * (B - 2);
  for (int i = t; i < SXX; i += B) {
    bool mir;
    const int xx = map_index(x0 - 2 + i, nx, a.bc[0], a.bc[1], mir);
    T U[NV], W[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) U[k] = Us[k * N + xx];
    if (mir) {
      U[1] = -U[1]; U[5] = -U[5]; U[6] = -U[6];
    }
    cons_to_prim(U, W);
#pragma unroll
    for (int k = 0; k < NV; k++) sW[k][i] = W[k];
    if (RETRY) sFl[i] = tagged(a.flags[xx], tag, a.level);
  }
  __syncthreads();
  T wm[NV], w0[NV], wp[NV], lo[NV], hi[NV], F[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) { wm[k] = sW[k][t]; w0[k] = sW[k][t + 1]; wp[k] = sW[k][t + 2]; }
  recon<SCH>(wm, w0, wp, nu, lo, hi);
  if (RETRY) first_order_faces(sFl[t] != 0, sFl[t + 1] != 0, sFl[t + 2] != 0, w0, lo, hi);
#pragma unroll
  for (int k = 0; k < NV; k++) sH[k][t] = hi[k];
  __syncthreads();
  if (t >= 1) {
    T hl[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) hl[k] = sH[k][t - 1];
    face_flux<SCH, RETRY>(hl, lo, RETRY && (sFl[t] | sFl[t + 1]), F);
  }
  __syncthreads();
  if (t >= 1) {
#pragma unroll
    for (int k = 0; k < NV; k++) sH[k][t] = F[k];
  }
  __syncthreads();
  Acc<T> diag;
  diag.zero();
  T smax = T(0);
  long long bad = LLONG_MAX;
  const int gx = x0 - 1 + t;
  if (t >= 1 && t <= B - 2 && gx < nx) {
    T acc[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) acc[k] = (F[k] - sH[k][t + 1]) * idx;
    finish_cell<T, 1, SCH, RETRY>(a, Us + gx, N, U0 + gx, Ud, N, (size_t)gx, acc, dt, idx, T(0), T(0), diag, smax,
                                  bad, tag, (RETRY || SCH != 0) ? nullptr : tape_slot(a, step, N));
  }
  write_partial<T, B>(diag, smax, bad, a.part + tile);
  __syncthreads();  // the next tile reuses the shared arrays
  }
}

// ----------------------------------------------------------------- 3D kernel
// Raw staging slots of the 3D kernel: four keep U^n of the plane being updated in shared
// memory (FP32, 16 rows: 224 KB with everything else); two otherwise (the update re-reads
// U^n from global memory), which keeps two FP32 blocks of 8 rows per SM and FP64 within
// the shared memory of a block.
// The corner-transport-upwind form keeps two (its shared memory holds per-thread transverse
// terms instead).
template <typename T, int BY, bool CTU = false>
constexpr int kRawPlanes = (sizeof(T) == 4 && BY == 16 && !CTU) ? 4 : 2;
// Asynchronous global -> shared copies (cp.async, completion tracked per thread by commit
// groups).
// The NV fields of one staged cell: field k lands at byte k * FSTRIDE past the shared address
// s (immediate offsets) and comes from g + k N (a running pointer: one 64-bit add per field
// instead of an index product).
template <typename T, int OFF> __device__ __forceinline__ void cp_async_at(unsigned s, const T *g) {
  asm volatile("cp.async.ca.shared.global [%0+%2], [%1], %3;\n" ::"r"(s), "l"(g), "n"(OFF), "n"((int)sizeof(T))
               : "memory");
}
template <typename T, int FSTRIDE, int... K>
__device__ __forceinline__ void cp_async_fields(unsigned s, const T *g, size_t N, std::integer_sequence<int, K...>) {
  ((cp_async_at<T, K * FSTRIDE>(s, g), g += N), ...);
}
template <typename T, int FSTRIDE> __device__ __forceinline__ void cp_async_cell(T *smem, const T *g, size_t N) {
  cp_async_fields<T, FSTRIDE>((unsigned)__cvta_generic_to_shared(smem), g, N, std::make_integer_sequence<int, NV>{});
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent groups are pending
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk tensor staging of the 3D kernel.  The state is a 4D tensor [NV][nz][ny][nx]; one
// copy moves a box of kTmaBoxX x (rows + 2) x 1 plane x NV fields into a raw staging slot
// ([NV][rows+2][kTmaBoxX], dense) and completes the transaction count of the slot's
// mbarrier.  The box starts at a multiple of 4 cells in x (16-byte rule of the copy), so
// it is two columns wider than the 34 the tile needs.  Its cells outside the grid arrive
// as zeros (tiles at the grid's edges) and are fixed up cell by cell afterwards.  Tensor
// maps: one per state buffer (U[0], U[1], U1), passed as a grid-constant kernel parameter.
constexpr int kTmaBoxX = 36;
struct TileMaps {
  CUtensorMap map[3];
  int ok;  // 1: the maps are valid and the step stages by bulk tensor copies
};
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the other threads and to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with parity `parity`; false if it has not completed within
// 2^31 clocks (about a second), so a copy that never lands cannot hang the kernel.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int f,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
      : "memory");
}

template <typename T, int D, int SY, int SX>
__device__ __forceinline__ void gather(const T *__restrict__ pl, int sy, int sx, T (&w)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) w[k] = pl[(Frame<D>::g(k) * SY + sy) * SX + sx];
}

// CTU: the corner-transport-upwind form (transverse terms in the face states, max-form CFL
// speed; 8-row tiles take one block per SM and the registers that allows, 16-row tiles keep
// 16 warps per SM and spill some).  Every thread's own cell is then staged too (the four cells diagonal to the
// tile's corners join the staged box), every thread but the four corner ones forms the
// transverse terms of its cell plane by plane, and the sums each sweep needs, X_x = T_y +
// T_z and X_y = T_x + T_z, wait in thread-private shared memory from the plane before.
template <typename T, int NDIM, int BY, int SCH, bool RETRY, bool CTU = false>
__global__ void __launch_bounds__(32 * BY, (BY <= 8 && !CTU && sizeof(T) == 4 ? 2 : 1))
    step_tile_kernel(StepArgs<T> a, const __grid_constant__ TileMaps tm) {
  static_assert(NDIM == 3, "the 2D step runs in step_strip2d_kernel");
  static_assert(kTileX % 2 == 0, "bulk-copy boxes start at most two cells before the staged box");
  constexpr int SX = 34, SY = BY + 2, NQ = SY * SX;
  constexpr int PL = NV * NQ;  // one primitive plane, all fields: [NV][SY][SX]
  constexpr int RAW = kRawPlanes<T, BY, CTU>;  // raw staging slots (4: U^n of the update from shared memory)
  // Raw slots: [NV][SY][RSX].  The step stages by bulk tensor copies (rows
  // RSX = kTmaBoxX wide, slots 128-byte aligned); the fallback passes and the
  // corner-transport-upwind form stage cell by cell (rows of SX).
  constexpr bool kTma = !RETRY && !CTU;
  constexpr int RSX = kTma ? kTmaBoxX : SX, RNQ = SY * RSX;
  constexpr int RSTR = kTma ? (NV * RNQ * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T) : NV * RNQ;
  constexpr unsigned kTmaBytes = (unsigned)(kTmaBoxX * SY * NV * sizeof(T));
  const Ctrl *ctrl = a.ctrl;
  if (ctrl->done) return;
  if (RETRY && ctrl->nbad[a.level - 1] == 0 && !((ctrl->force >> a.level) & 1)) return;
  const int64_t step = ctrl->step;
  const int32_t tag = (int32_t)(step & 0x0fffffff) + 1;
  // fallback tags of the staged cells (fallback pass only)
  __shared__ unsigned char sFl[RETRY ? 3 : 1][RETRY ? NQ : 1];
  // sweep source, destination and U^n (the second Runge-Kutta stage sweeps U1)
  const T *__restrict__ U0 = a.U[step & 1];
  const T *__restrict__ Us = SCH == 2 ? a.U1 : U0;
  T *__restrict__ Ud = SCH == 1 ? a.U1 : a.U[(step + 1) & 1];
  const double dtd = ctrl->dt;
  const T dt = (T)dtd;
  const T nux = (T)(0.5 * dtd / a.dx[0]), idx = (T)(1.0 / a.dx[0]);
  const T nuy = (T)(0.5 * dtd / a.dx[1]), idy = (T)(1.0 / a.dx[1]);
  const T nuz = (T)(0.5 * dtd / a.dx[2]), idz = (T)(1.0 / a.dx[2]);
  T *const ck = (RETRY || SCH != 0) ? nullptr : tape_slot(a, step, (size_t)a.nx * a.ny * a.nz);
  // shared memory: RAW raw conserved planes filled one plane ahead (bulk tensor copies or
  // cp.async), three primitive planes (ring), the y-sweep face states and fluxes, per staged
  // position of the tile its x/y reflect flips (the same for every plane) and, for the
  // cell-by-cell staging of the fallback passes and the corner-transport-upwind form, per
  // staged cell its sign flips (bits 0..9) and fallback tag (bit 10)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T *sR = reinterpret_cast<T *>(smem_raw);
  T *sW = sR + RAW * RSTR;
  T *sXh = sW + 3 * PL;          // [NV][BY][32]
  T *sXf = sXh + NV * BY * 32;   // [NV][BY][32]
  T *sCx = sXf + NV * BY * 32;   // CTU: X_x of the thread's cell, [NV][BY * 32]
  T *sCy = sCx + (CTU ? NV * BY * 32 : 0);  // CTU: X_y, [NV][BY * 32]
  // [RAW][NQ] but for the step, which forms the flips from sFxy and the plane
  uint16_t *sMeta = reinterpret_cast<uint16_t *>(sCy + (CTU ? NV * BY * 32 : 0));
  uint16_t *sFxy = sMeta + (kTma ? 0 : RAW * NQ);  // [NQ]
  // one mbarrier per raw slot (bulk tensor staging)
  __shared__ __align__(8) uint64_t sBar[kTma ? RAW : 1];
  auto slot = [](int p) { return ((p % RAW) + RAW) % RAW; };
  // raw-slot index of staged position i (row pitch RSX instead of SX)
  auto rawi = [](int i) { return RSX == SX ? i : i + (i / SX) * (RSX - SX); };
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  // Bulk tensor staging: on when the maps are valid (block-uniform); the mbarriers keep their
  // phases across the tiles of a block, tracked by parity bits per slot (every thread waits
  // for every copy; thread 0 issues them).
  const bool tma_on = kTma && tm.ok != 0 && (smem_u32(smem_raw) & 127u) == 0;
  unsigned tma_ph = 0, tma_iss = 0;
  bool tma_dead = false;  // a wait ran out: no more copies are issued or waited for
  if (kTma && tma_on) {
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < (kTma ? RAW : 1); q++) mbar_init(&sBar[q], 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t N = (size_t)nx * ny * nz;
  // Work units (one partial each).  Chunked tiling (zchunk > 0): a unit is one chunk of
  // zchunk planes of one column of tiles (x-y tile, all of z).  Balanced tiling (zchunk =
  // 0): the columns are dealt out whole, column c to unit c mod units, as long as every unit
  // gets one; the planes of the columns left over are ordered window by window (windows of
  // wz planes, the share of one unit; within a window column by column, so that units
  // running at the same time stream neighbouring columns at the same heights and share
  // their halos in L2) and cut into `units` equal runs.  Every unit so streams the same
  // number of planes (to one), in one to three stretches, each with its own prologue.  The
  // step launches one thread block per unit; the fallback passes run on a small grid that
  // loops over the units, so a pass with nothing to do costs only its launch.
  const int tilesx = (nx + kTileX - 1) / kTileX, tilesy = (ny + BY - 3) / (BY - 2);
  const int ncols = tilesx * tilesy, units = a.units, zc = a.zchunk;
  const int nfull = zc > 0 ? 0 : ncols / units;
  const int nrcol = ncols - nfull * units;  // columns left over (balanced tiling)
  const long long nrest = zc > 0 ? 0 : (long long)nrcol * nz;
  const int wz = zc > 0 ? 1 : (int)std::max<long long>(1, (nrest + units - 1) / units);
  const int nwf = nz / wz, wlast = nz - nwf * wz;  // whole windows, planes of the last one
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
  Acc<T> diag;
  diag.zero();
  T smax = T(0);
  long long bad = LLONG_MAX;
  double *const tot = block_totals();  // FP64 running totals of the unit (FP32 states)
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) tot[k] = 0.0;
  }
  long long rp = nrest * u / units;
  const long long rend = nrest * (u + 1) / units;
  for (int item = 0;; item++) {
  int col, z0, z1;
  if (zc > 0) {  // chunked tiling: one chunk
    if (item > 0) break;
    col = u % ncols;
    z0 = (u / ncols) * zc;
    z1 = min(nz, z0 + zc);
  } else if (item < nfull) {  // a whole column
    col = u + item * units;
    z0 = 0;
    z1 = nz;
  } else {  // a run of the left-over columns' planes, up to the end of its window
    if (rp >= rend) break;
    const long long inwhole = (long long)nrcol * wz * nwf;
    int j, zend;
    if (rp < inwhole) {
      const int k = (int)(rp / ((long long)nrcol * wz));
      const int r = (int)(rp - (long long)k * nrcol * wz);
      j = r / wz;
      z0 = k * wz + (r - j * wz);
      zend = (k + 1) * wz;
    } else {
      const int r = (int)(rp - inwhole);
      j = r / wlast;
      z0 = nwf * wz + (r - j * wlast);
      zend = nz;
    }
    z1 = (int)std::min<long long>(zend, z0 + (rend - rp));
    col = nfull * units + j;
    rp += z1 - z0;
  }
  const int bxi = col % tilesx, byi = col / tilesx;
  const int x0 = bxi * kTileX, y0 = byi * (BY - 2);
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const int sx = tx + 1, sy = ty + 1;
  const bool interior = tx >= 1 && tx <= kTileX && ty >= 1 && ty <= BY - 2;
  const bool valid = interior && gx < nx && gy < ny;
  // Bulk staging: one bulk tensor copy per plane of the box from (xs, y0-2), the staged
  // box at column xo of it; cells of the box outside the grid arrive as zeros and are then
  // fixed up one by one from their mapped cells (periodic wrap, mirror images, outflow).
  const bool use_tma = tma_on;
  const int xs = (x0 - 2) & ~3, xo = use_tma ? x0 - 2 - xs : 0;
  // Rows of a tile that overhangs the grid in y: a row beyond it (gy > ny) feeds no updated
  // cell and skips its sweeps (warp-uniform; the barriers and the staging stay); the row
  // just above the last one (gy = ny) still reconstructs along y for that row's upper face.
  // The corner-transport-upwind form keeps every row (its transverse terms reach along x).
  const bool rowvalid = CTU || gy < ny, rowneed = CTU || gy <= ny;
  // CTU: the threads whose cell's face states are used (all but the four corner threads)
  const bool tneed = CTU && ((ty >= 1 && ty <= BY - 2) || (tx >= 1 && tx <= kTileX));
  // staged cells: the box without its corners (CTU: without its outer corners)
  auto staged = [](int qy, int qx) {
    return (qy >= 2 && qy <= BY - 1) || (qx >= 2 && qx <= 31) || (CTU && qy >= 1 && qy <= BY && qx >= 1 && qx <= 32);
  };

  // Staged cells: the 34 x (BY+2) box (x0-2 .. x0+31, y0-2 .. y0+BY-1) without its corners
  // (staged()).  A thread stages positions i = tid and tid + 32 BY (two cover the box);
  // their in-plane source offsets (yy nx + xx; -1 where nothing is staged) stay in its
  // registers and their x/y flips in shared memory, mapped once per tile by the thread that
  // uses them (no barrier needed).
  static_assert(NQ <= 2 * 32 * BY, "two staged positions per thread");
  int soff[2];
  unsigned fixm = 0u;  // bit j: staged position j lies outside the grid (a fix-up of the bulk copy)
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const int i = tid + j * 32 * BY;
    soff[j] = -1;
    if (i < NQ) {
      const int qy = i / SX, qx = i - qy * SX;
      const int rx = x0 - 2 + qx, ry = y0 - 2 + qy;
      bool mx, my;
      const int xx = map_index(rx, nx, a.bc[0], a.bc[1], mx);
      const int yy = map_index(ry, ny, a.bc[2], a.bc[3], my);
      if (staged(qy, qx)) {
        soff[j] = yy * nx + xx;
        if (rx < 0 || rx >= nx || ry < 0 || ry >= ny) fixm |= 1u << j;
      }
      sFxy[i] = (mx ? flip_mask(0) : 0u) ^ (my ? flip_mask(1) : 0u);
    }
  }
  // Cell by cell, a thread stages and later converts the same cells, so the copies it waits
  // for are its own and no barrier separates staging from conversion; a bulk copy is
  // issued by thread 0 and every thread waits for it on the slot's mbarrier.
  auto stage = [&](int z) {
    bool mz = false;
    const int zz = map_index(z, nz, a.bc[4], a.bc[5], mz);
    if constexpr (kTma) {
      if (use_tma) {  // thread 0 issues the plane's copy; every thread waits for it in convert
        // (test hook: block 0 leaves out the copy of plane -2, which starts a stretch from
        // z = 0, and the threads waiting for it give up)
        if (tid == 0 && !tma_dead && !(a.test_skip && blockIdx.x == 0 && z == -2)) {
          const int q = slot(z);
          fence_proxy_async();  // the slot's last reads (before the barrier) precede the copy
          mbar_expect_tx(&sBar[q], kTmaBytes);
          tma_load_4d(sR + q * RSTR, &tm.map[SCH == 2 ? 2 : (int)(step & 1)], xs, y0 - 2, zz, 0, &sBar[q]);
          tma_iss ^= 1u << q;
        }
        return;
      }
    }
    T *dst = sR + slot(z) * RSTR;
    uint16_t *meta = sMeta + slot(z) * NQ;
    const size_t zoff = (size_t)zz * ny * nx;
    const unsigned fz = mz ? flip_mask(2) : 0u;
#pragma unroll
    for (int j = 0; j < 2; j++) {
      if (soff[j] < 0) continue;
      const int i = tid + j * 32 * BY;
      const size_t c = zoff + (size_t)soff[j];
      cp_async_cell<T, RNQ * (int)sizeof(T)>(dst + rawi(i), Us + c, N);
      if constexpr (!kTma) {
        unsigned m = sFxy[i] ^ fz;
        if (RETRY && tagged(a.flags[c], tag, a.level)) m |= 1u << 10;
        meta[i] = (uint16_t)m;
      }
    }
    cp_async_commit();
  };
  // Fix-ups of a bulk-copied plane: once its copy has landed, the threads whose staged cells
  // lie outside the grid overwrite them with their mapped cells (cp.async, waited for in
  // convert).  A thread without such cells does nothing.
  auto fixups = [&](int z) {
    if constexpr (kTma) {
      if (use_tma && fixm != 0u) {
        const int q = slot(z);
        if (!tma_dead && !mbar_wait_bounded(&sBar[q], (tma_ph >> q) & 1u)) {
          tma_dead = true;
          atomicExch(&a.ctrl->stage_timeout, 1);
        }
        bool mz = false;
        const size_t zoff = (size_t)map_index(z, nz, a.bc[4], a.bc[5], mz) * ny * nx;
        T *dst = sR + q * RSTR + xo;
#pragma unroll
        for (int j = 0; j < 2; j++)
          if ((fixm >> j) & 1u)
            cp_async_cell<T, RNQ * (int)sizeof(T)>(dst + rawi(tid + j * 32 * BY), Us + zoff + (size_t)soff[j], N);
        cp_async_commit();
      }
    }
  };
  auto convert = [&](int z) {  // raw plane z -> primitive plane in ring slot z mod 3
    const int q = slot(z);
    const T *src = sR + q * RSTR;
    const uint16_t *meta = sMeta + q * NQ;
    const int b = ((z % 3) + 3) % 3;
    T *dst = sW + b * PL;
    unsigned fz = 0u;  // the step: flips of the cell = its x/y flips ^ those of a mirror plane
    if constexpr (kTma) {
      if (use_tma) {  // the plane's copy, then this thread's fix-ups
        if (!tma_dead && !mbar_wait_bounded(&sBar[q], (tma_ph >> q) & 1u)) {
          tma_dead = true;
          atomicExch(&a.ctrl->stage_timeout, 1);
        }
        tma_ph ^= 1u << q;
        if (fixm != 0u) cp_async_wait<0>();
      }
      bool mz = false;
      (void)map_index(z, nz, a.bc[4], a.bc[5], mz);
      fz = mz ? flip_mask(2) : 0u;
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      if (soff[j] < 0) continue;
      const int i = tid + j * 32 * BY;
      const unsigned m = kTma ? (unsigned)sFxy[i] ^ fz : (unsigned)meta[i];
      const int ri = rawi(i) + xo;
      T U[NV], W[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) U[k] = src[k * RNQ + ri];
      if (m & 0x3ffu) {  // a reflect image (never inside a periodic or outflow grid)
#pragma unroll
        for (int k = 0; k < NV; k++) U[k] = ((m >> k) & 1u) ? -U[k] : U[k];
      }
      cons_to_prim(U, W);
#pragma unroll
      for (int k = 0; k < NV; k++) dst[k * NQ + i] = W[k];
      if (RETRY) sFl[RETRY ? b : 0][i] = (m >> 10) & 1u;
    }
  };
  auto buf = [](int p) { return ((p % 3) + 3) % 3; };
  auto fl = [&](int b, int qy, int qx) -> bool { return RETRY ? sFl[RETRY ? b : 0][qy * SX + qx] != 0 : false; };
  // z reconstruction of cell p (planes p-1, p, p+1) in the interior threads
  auto recon_z = [&](int p, T (&lo)[NV], T (&hi)[NV]) {
    T wm[NV], w0[NV], wp[NV];
    gather<T, 2, SY, SX>(sW + buf(p - 1) * PL, sy, sx, wm);
    gather<T, 2, SY, SX>(sW + buf(p) * PL, sy, sx, w0);
    gather<T, 2, SY, SX>(sW + buf(p + 1) * PL, sy, sx, wp);
    recon<SCH>(wm, w0, wp, nuz, lo, hi);
    if (RETRY) first_order_faces(fl(buf(p - 1), sy, sx), fl(buf(p), sy, sx), fl(buf(p + 1), sy, sx), w0, lo, hi);
  };
  // CTU: z reconstruction of cell p with the transverse terms X_z = T_x + T_y (global order,
  // xg in the thread's slot of free shared memory); the cell's own T_z is added to X_x and
  // X_y in its private slots when `keep`
  auto recon_z_ctu = [&](int p, const T *xg, bool keep, T (&lo)[NV], T (&hi)[NV]) {
    T wm[NV], w0[NV], wp[NV];
    gather<T, 2, SY, SX>(sW + buf(p - 1) * PL, sy, sx, wm);
    gather<T, 2, SY, SX>(sW + buf(p) * PL, sy, sx, w0);
    gather<T, 2, SY, SX>(sW + buf(p + 1) * PL, sy, sx, wp);
    if constexpr (CTU)
      recon_ctu<SCH>(
          wm, w0, wp, nuz, [&](int k) { return xg[Frame<2>::g(k) * BY * 32 + tid]; },
          [&](int k, T v) {
            if (keep) {
              sCx[Frame<2>::g(k) * BY * 32 + tid] += v;
              sCy[Frame<2>::g(k) * BY * 32 + tid] += v;
            }
          },
          lo, hi);
    if (RETRY) first_order_faces(fl(buf(p - 1), sy, sx), fl(buf(p), sy, sx), fl(buf(p + 1), sy, sx), w0, lo, hi);
  };
  // CTU: T_x and T_y of the thread's cell in plane p (global order): X_z = T_x + T_y to xz,
  // and T_y to its X_x slot, T_x to its X_y slot (all thread-private)
  auto trans_x_y = [&](int p, T *xz) {
    const T *pl = sW + buf(p) * PL;
    T wm[NV], w0[NV], wp[NV], o[NV];
    gather<T, 0, SY, SX>(pl, sy, sx - 1, wm);
    gather<T, 0, SY, SX>(pl, sy, sx, w0);
    gather<T, 0, SY, SX>(pl, sy, sx + 1, wp);
    transverse(wm, w0, wp, nux, o);  // the x frame is the global order
#pragma unroll
    for (int k = 0; k < NV; k++) {
      xz[k * BY * 32 + tid] = o[k];
      sCy[k * BY * 32 + tid] = o[k];
    }
    gather<T, 1, SY, SX>(pl, sy - 1, sx, wm);
    gather<T, 1, SY, SX>(pl, sy, sx, w0);
    gather<T, 1, SY, SX>(pl, sy + 1, sx, wp);
    transverse(wm, w0, wp, nuy, o);
#pragma unroll
    for (int k = 0; k < NV; k++) {
      const int gk = Frame<1>::g(k);
      xz[gk * BY * 32 + tid] += o[k];
      sCx[gk * BY * 32 + tid] = o[k];
    }
  };
  // CTU: the z face states of cell p (interior threads: lo, hi) and, for every thread whose
  // cell is used (keep), X_x = T_y + T_z and X_y = T_x + T_z of cell p in its private slots.
  // X_z = T_x + T_y waits in the raw staging slot of plane p + 1, which holds no pending
  // data here (its plane is converted and the next copy into it comes after the next
  // barrier), in the thread's own cells.
  auto ctu_plane = [&](int p, bool keep, T (&lo)[NV], T (&hi)[NV]) {
    T *xz = sR + slot(p + 1) * RSTR;
    trans_x_y(p, xz);
    recon_z_ctu(p, xz, keep, lo, hi);
  };

  // prologue: planes z0-2 .. z0+2 converted; the z face state of cell z0 and the flux
  // through its lower face in registers
  if constexpr (RAW == 4) {  // the first four planes in flight at once
    stage(z0 - 2);
    stage(z0 - 1);
    stage(z0);
    stage(z0 + 1);
    fixups(z0 - 2);
    fixups(z0 - 1);
    fixups(z0);
    fixups(z0 + 1);
    cp_async_wait<2>();  // cell by cell: this thread's copies of planes z0-2 and z0-1 have landed
    convert(z0 - 2);
    convert(z0 - 1);
    cp_async_wait<1>();
    convert(z0);
  } else {
    stage(z0 - 2);
    stage(z0 - 1);
    fixups(z0 - 2);
    fixups(z0 - 1);
    cp_async_wait<0>();
    convert(z0 - 2);
    convert(z0 - 1);
    // two raw slots: plane z0 takes the slot of plane z0-2, which a bulk copy may overwrite
    // only after every thread has converted it (cell-by-cell staging rewrites only the
    // thread's own cells)
    if (use_tma) __syncthreads();
    stage(z0);
    fixups(z0);
    cp_async_wait<0>();
    convert(z0);
  }
  __syncthreads();
  T hprev[NV], Fprev[NV];
  if (interior && rowvalid) {
    T lo[NV];
    if constexpr (CTU) {
      // X_z of cell z0-1 in the raw slot of plane z0+1, which is staged only below; the X_x,
      // X_y slots written here are rewritten for plane z0 before their first use
      ctu_plane(z0 - 1, false, lo, hprev);
    } else {
      recon_z(z0 - 1, lo, hprev);
    }
  }
  if constexpr (RAW != 4) {
    stage(z0 + 1);
    fixups(z0 + 1);
  }
  cp_async_wait<0>();
  __syncthreads();  // plane z0-2 is no longer read
  convert(z0 + 1);
  stage(z0 + 2);
  __syncthreads();
  {
    T lo[NV], hi[NV];
    if constexpr (CTU) {
      if (tneed) ctu_plane(z0, true, lo, hi);
    } else if (interior && rowvalid) {
      recon_z(z0, lo, hi);
    }
    if (interior && rowvalid) {
      face_flux<SCH, RETRY>(hprev, lo, fl(buf(z0 - 1), sy, sx) || fl(buf(z0), sy, sx), Fprev);
#pragma unroll
      for (int k = 0; k < NV; k++) hprev[k] = hi[k];
    }
  }
  fixups(z0 + 2);
  cp_async_wait<0>();
  __syncthreads();  // plane z0-1 is no longer read
  convert(z0 + 2);
  __syncthreads();

  for (int z = z0; z < z1; z++) {
    // planes z, z+1, z+2 are converted
    const T *pl = sW + buf(z) * PL;
    // flux divergence of the cell, accumulated as each face flux becomes known (the lower z
    // face first; the flux registers die at once, which keeps the register count down)
    T acc[NV];
    {
      T Fg[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) Fg[Frame<2>::g(k)] = Fprev[k];
      v_mul(acc, Fg, idz);
    }
    if (ty >= 1 && ty <= BY - 2 && rowvalid) {  // x sweep, warp-uniform: one warp per row
      T wm[NV], w0[NV], wp[NV], lo[NV], hi[NV], hl[NV], F[NV];
      gather<T, 0, SY, SX>(pl, sy, sx - 1, wm);
      gather<T, 0, SY, SX>(pl, sy, sx, w0);
      gather<T, 0, SY, SX>(pl, sy, sx + 1, wp);
      if constexpr (CTU) {
        recon_ctu<SCH>(
            wm, w0, wp, nux, [&](int k) { return sCx[k * BY * 32 + tid]; }, [](int, T) {}, lo, hi);
      } else {
        recon<SCH>(wm, w0, wp, nux, lo, hi);
      }
      if (RETRY) first_order_faces(fl(buf(z), sy, sx - 1), fl(buf(z), sy, sx), fl(buf(z), sy, sx + 1), w0, lo, hi);
#pragma unroll
      for (int k = 0; k < NV; k++) hl[k] = __shfl_up_sync(FULL, hi[k], 1);
      face_flux<SCH, RETRY>(hl, lo, fl(buf(z), sy, sx - 1) || fl(buf(z), sy, sx), F);  // lower x face
      T Fu[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) Fu[k] = __shfl_down_sync(FULL, F[k], 1);
      v_sub(F, F, Fu);
      v_fma(acc, F, idx, acc);
    }
    const bool ycol = tx >= 1 && tx <= kTileX && rowneed;
    T ylo[NV];
    if (ycol) {  // y reconstruction of this cell; its upper face state goes to shared memory
      T wm[NV], w0[NV], wp[NV], hi[NV];
      gather<T, 1, SY, SX>(pl, sy - 1, sx, wm);
      gather<T, 1, SY, SX>(pl, sy, sx, w0);
      gather<T, 1, SY, SX>(pl, sy + 1, sx, wp);
      if constexpr (CTU) {
        recon_ctu<SCH>(
            wm, w0, wp, nuy, [&](int k) { return sCy[Frame<1>::g(k) * BY * 32 + tid]; }, [](int, T) {}, ylo, hi);
      } else {
        recon<SCH>(wm, w0, wp, nuy, ylo, hi);
      }
      if (RETRY) first_order_faces(fl(buf(z), sy - 1, sx), fl(buf(z), sy, sx), fl(buf(z), sy + 1, sx), w0, ylo, hi);
#pragma unroll
      for (int k = 0; k < NV; k++) sXh[(k * BY + ty) * 32 + tx] = hi[k];
    }
    __syncthreads();
    // Every thread has finished the previous plane: its raw slot (plane z-1 with four
    // slots, z+1 with two) is free for plane z+3.
    if (z + 3 <= z1 + 1) stage(z + 3);
    if (ycol && ty >= 1) {  // flux through the lower y face
      T hl[NV], Fy[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) hl[k] = sXh[(k * BY + ty - 1) * 32 + tx];
      face_flux<SCH, RETRY>(hl, ylo, fl(buf(z), sy - 1, sx) || fl(buf(z), sy, sx), Fy);
      T Fg[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) {
        sXf[(k * BY + ty) * 32 + tx] = Fy[k];
        Fg[Frame<1>::g(k)] = Fy[k];
      }
      v_fma(acc, Fg, idy, acc);
    }
    {  // z: reconstruct cell z+1, flux through the upper z face of cell z
      T lo[NV], hi[NV], F[NV];
      if constexpr (CTU) {
        if (tneed) ctu_plane(z + 1, true, lo, hi);
      } else if (interior && rowvalid) {
        recon_z(z + 1, lo, hi);
      }
      if (interior && rowvalid) {
      face_flux<SCH, RETRY>(hprev, lo, fl(buf(z), sy, sx) || fl(buf(z + 1), sy, sx), F);
      T Fg[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) {
        Fg[Frame<2>::g(k)] = F[k];
        hprev[k] = hi[k];
        Fprev[k] = F[k];
      }
      v_fma(acc, Fg, -idz, acc);
      }
    }
    // the copy of plane z+3 has had the z sweep to land: the fix-ups of its cells outside
    // the grid go out now, to land during the update
    if (z + 1 < z1) fixups(z + 3);
    __syncthreads();
    if (interior && rowvalid) {
#pragma unroll
      for (int k = 0; k < NV; k++) acc[Frame<1>::g(k)] -= sXf[(k * BY + ty + 1) * 32 + tx] * idy;  // upper y face
    }
    if (valid) {
      const size_t c = ((size_t)z * ny + gy) * nx + gx;
      if (RAW == 4)  // the swept state as staged (an interior cell is never a reflect image)
        finish_cell<T, NDIM, SCH, RETRY, CTU>(a, sR + slot(z) * RSTR + sy * RSX + sx + xo, RNQ, U0 + c, Ud, N, c, acc, dt,
                                              idx, idy, idz, diag, smax, bad, tag, ck);
      else
        finish_cell<T, NDIM, SCH, RETRY, CTU>(a, Us + c, N, U0 + c, Ud, N, c, acc, dt, idx, idy, idz, diag, smax,
                                              bad, tag, ck);
    }
    // Plane z is no longer read (every read of the primitive planes precedes the second
    // barrier); plane z+3 replaces it.  The next iteration reads it only after its first
    // barrier, and rewrites sXh / sXf only after every thread has passed this one.
    if (z + 1 < z1) {
      cp_async_wait<0>();
      convert(z + 3);
    }
    // FP32 states: every 64 planes of a stretch, and at its end, the threads' FP32 sums
    // move into the job's FP64 totals (a sum spans at most 64 planes)
    // (the barrier inside comes after every thread has finished the plane)
    if constexpr (sizeof(T) == 4) {
      if (((z + 1 - z0) & 63) == 0 && z + 1 < z1) flush_totals<T, 32 * BY>(diag, tot);
    }
  }
  cp_async_wait<0>();
  if constexpr (sizeof(T) == 4) flush_totals<T, 32 * BY>(diag, tot);  // its barrier also ends the stretch
  __syncthreads();  // the next stretch restages every buffer
  }
  write_partial<T, 32 * BY>(diag, smax, bad, a.part + u, tot);
  }
  if (kTma && tma_on && tid == 0 && tma_dead) {
    // a wait ran out: let copies still in flight land (bounded) before the block exits
#pragma unroll
    for (int q = 0; q < (kTma ? RAW : 1); q++) (void)mbar_wait_bounded(&sBar[q], ((tma_iss >> q) & 1u) ^ 1u);
  }
}

// ---------------------------------------------------------------- 2D kernel
// One warp owns a strip of 32 columns, lane l holding cell x0 - 2 + l, and streams it in
// y over `ychunk` rows; lanes 2..29 are updated (kStripX = 28 cells per strip).  x faces:
// warp shuffles of the row held in registers; y faces: a three-row register ring with the
// face state and flux of the previous row carried, so every cell is reconstructed once
// per direction.  Warps never wait on one another inside a tile; a thread block of WARPS
// strips writes one partial.
// CTU: the corner-transport-upwind form.  The y reconstruction of cell y+1 takes X_y = T_x
// of its row (formed from the row's shuffled neighbours) and yields the cell's own T_y,
// which waits in lane-private shared memory as X_x of the next row's x sweep.
template <typename T, int WARPS, int SCH, bool RETRY, bool CTU = false>
__global__ void __launch_bounds__(32 * WARPS) step_strip2d_kernel(StepArgs<T> a) {
  __shared__ T sTy[CTU ? WARPS : 1][NV][32];  // CTU: T_y of the lane's cell in the row of the x sweep
  const Ctrl *ctrl = a.ctrl;
  if (ctrl->done) return;
  if (RETRY && ctrl->nbad[a.level - 1] == 0 && !((ctrl->force >> a.level) & 1)) return;
  const int64_t step = ctrl->step;
  const int32_t tag = (int32_t)(step & 0x0fffffff) + 1;
  // sweep source, destination and U^n (the second Runge-Kutta stage sweeps U1)
  const T *__restrict__ U0 = a.U[step & 1];
  const T *__restrict__ Us = SCH == 2 ? a.U1 : U0;
  T *__restrict__ Ud = SCH == 1 ? a.U1 : a.U[(step + 1) & 1];
  const double dtd = ctrl->dt;
  const T dt = (T)dtd;
  const T nux = (T)(0.5 * dtd / a.dx[0]), idx = (T)(1.0 / a.dx[0]);
  const T nuy = (T)(0.5 * dtd / a.dx[1]), idy = (T)(1.0 / a.dx[1]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = a.nx, ny = a.ny, ych = a.zchunk;
  const size_t N = (size_t)nx * ny;
  T *const ck = (RETRY || SCH != 0) ? nullptr : tape_slot(a, step, N);
  const int stripsx = (nx + kStripX - 1) / kStripX, chunksy = (ny + ych - 1) / ych;
  const int ntiles = stripsx * chunksy;
  const int ngroups = (ntiles + WARPS - 1) / WARPS;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    Acc<T> diag;
    diag.zero();
    T smax = T(0);
    long long bad = LLONG_MAX;
    const int tile = grp * WARPS + warp;
    if (tile < ntiles) {  // warp-uniform
      const int x0 = (tile % stripsx) * kStripX, y0 = (tile / stripsx) * ych;
      const int y1 = min(y0 + ych, ny);
      const int gx = x0 - 2 + lane;
      bool mx;
      const int xx = map_index(gx, nx, a.bc[0], a.bc[1], mx);
      const bool upd = lane >= 2 && lane <= kStripX + 1 && gx < nx;
      // raw conserved row (with the reflect images' sign flips) and its fallback tag
      auto fetch = [&](int y, T (&U)[NV], bool &fl) {
        bool my;
        const int yy = map_index(y, ny, a.bc[2], a.bc[3], my);
        const unsigned flip = (mx ? flip_mask(0) : 0u) ^ (my ? flip_mask(1) : 0u);
        const size_t c = (size_t)yy * nx + xx;
        const T *__restrict__ src = Us + c;  // a running pointer: one 64-bit add per field
#pragma unroll
        for (int k = 0; k < NV; k++) {
          U[k] = *src;
          src += N;
        }
        if (flip) {  // a mirror image (never inside a periodic or outflow grid)
#pragma unroll
          for (int k = 0; k < NV; k++) U[k] = ((flip >> k) & 1u) ? -U[k] : U[k];
        }
        fl = RETRY ? tagged(a.flags[c], tag, a.level) : false;
      };
      auto ylocal = [](const T (&w)[NV], T (&o)[NV]) {
#pragma unroll
        for (int k = 0; k < NV; k++) o[k] = w[Frame<1>::g(k)];
      };
      // CTU: T_x of a row held in the y frame, returned in the y frame (all lanes take part)
      auto trans_x = [&](const T (&ry)[NV], T (&Xy)[NV]) {
        T w0[NV], wm[NV], wp[NV], o[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) w0[k] = ry[Frame<1>::g(k)];  // Frame<1> is an involution
#pragma unroll
        for (int k = 0; k < NV; k++) {
          wm[k] = __shfl_up_sync(FULL, w0[k], 1);
          wp[k] = __shfl_down_sync(FULL, w0[k], 1);
        }
        transverse(wm, w0, wp, nux, o);
#pragma unroll
        for (int k = 0; k < NV; k++) Xy[k] = o[Frame<1>::g(k)];
      };
      // y reconstruction (y frame), with CTU the transverse term X_y = T_x of the cell's row
      // and the cell's own T_y stored (global order) for the x sweep of that row
      auto recon_y = [&](const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T (&lo)[NV], T (&hi)[NV]) {
        if constexpr (CTU) {
          T Xy[NV];
          trans_x(w0, Xy);
          recon_ctu<SCH>(
              wm, w0, wp, nuy, [&](int k) { return Xy[k]; },
              [&](int k, T v) { sTy[CTU ? warp : 0][Frame<1>::g(k)][lane] = v; }, lo, hi);
        } else {
          recon<SCH>(wm, w0, wp, nuy, lo, hi);
        }
      };
      // ring: rows y, y+1, y+2 (primitive, y local frame) and their tags
      T r0[NV], r1[NV], r2[NV], hprev[NV], Fprev[NV];
      bool f0 = false, f1 = false, f2 = false;
      {
        T U[NV], w[NV], wa[NV];
        bool fa;
        fetch(y0 - 2, U, fa); cons_to_prim(U, w); ylocal(w, wa);
        fetch(y0 - 1, U, f0); cons_to_prim(U, w); ylocal(w, r0);
        fetch(y0, U, f1); cons_to_prim(U, w); ylocal(w, r1);
        fetch(y0 + 1, U, f2); cons_to_prim(U, w); ylocal(w, r2);
        T lo[NV], hi[NV];
        recon_y(wa, r0, r1, lo, hprev);  // cell y0-1
        if (RETRY) first_order_faces(fa, f0, f1, r0, lo, hprev);
        recon_y(r0, r1, r2, lo, hi);     // cell y0 (CTU: its T_y for the first x sweep)
        if (RETRY) first_order_faces(f0, f1, f2, r1, lo, hi);
        face_flux<SCH, RETRY>(hprev, lo, f0 || f1, Fprev);  // flux through y0 - 1/2
#pragma unroll
        for (int k = 0; k < NV; k++) {
          hprev[k] = hi[k];
          r0[k] = r1[k];
          r1[k] = r2[k];
        }
        f0 = f1;
        f1 = f2;
      }
      for (int y = y0; y < y1; y++) {
        T Un2[NV];
        fetch(y + 2, Un2, f2);  // issued before the x sweep hides its latency
        // flux divergence of the cell, the lower y face first (Fprev dies at once)
        T acc[NV];
        {
          T Fg[NV];
#pragma unroll
          for (int k = 0; k < NV; k++) Fg[Frame<1>::g(k)] = Fprev[k];
          v_mul(acc, Fg, idy);
        }
        {
          // x sweep of row y: local x frame = natural order
          T w0[NV], wm[NV], wp[NV], lo[NV], hi[NV], hl[NV], F[NV];
#pragma unroll
          for (int k = 0; k < NV; k++) w0[k] = r0[Frame<1>::g(k)];  // Frame<1> is an involution
#pragma unroll
          for (int k = 0; k < NV; k++) {
            wm[k] = __shfl_up_sync(FULL, w0[k], 1);
            wp[k] = __shfl_down_sync(FULL, w0[k], 1);
          }
          if constexpr (CTU) {
            recon_ctu<SCH>(
                wm, w0, wp, nux, [&](int k) { return sTy[CTU ? warp : 0][k][lane]; }, [](int, T) {}, lo, hi);
          } else {
            recon<SCH>(wm, w0, wp, nux, lo, hi);
          }
          bool fxlo = false;  // the lower x face has first-order states
          if (RETRY) {
            const bool fm = __shfl_up_sync(FULL, f0, 1), fp = __shfl_down_sync(FULL, f0, 1);
            first_order_faces(fm, f0, fp, w0, lo, hi);
            fxlo = fm || f0;
          }
#pragma unroll
          for (int k = 0; k < NV; k++) hl[k] = __shfl_up_sync(FULL, hi[k], 1);
          face_flux<SCH, RETRY>(hl, lo, fxlo, F);  // flux through the lower x face of this cell
#pragma unroll
          for (int k = 0; k < NV; k++) hl[k] = __shfl_down_sync(FULL, F[k], 1);  // upper x face
          v_sub(F, F, hl);
          v_fma(acc, F, idx, acc);
        }
        {
          // y: reconstruct cell y+1, flux through y + 1/2
          T w[NV];
          cons_to_prim(Un2, w);
          ylocal(w, r2);
          T lo[NV], hi[NV], F[NV];
          recon_y(r0, r1, r2, lo, hi);
          if (RETRY) first_order_faces(f0, f1, f2, r1, lo, hi);
          face_flux<SCH, RETRY>(hprev, lo, f0 || f1, F);
          T Fg[NV];
#pragma unroll
          for (int k = 0; k < NV; k++) {
            Fg[Frame<1>::g(k)] = F[k];
            hprev[k] = hi[k];
            Fprev[k] = F[k];
          }
          v_fma(acc, Fg, -idy, acc);
        }
        if (upd)
          finish_cell<T, 2, SCH, RETRY, CTU>(a, Us + ((size_t)y * nx + gx), N, U0 + ((size_t)y * nx + gx), Ud, N,
                                             (size_t)y * nx + gx, acc, dt, idx, idy, T(0), diag, smax, bad, tag, ck);
#pragma unroll
        for (int k = 0; k < NV; k++) {
          r0[k] = r1[k];
          r1[k] = r2[k];
        }
        f0 = f1;
        f1 = f2;
      }
    }
    write_partial<T, 32 * WARPS>(diag, smax, bad, a.part + grp);
    __syncthreads();  // the next group reuses the reduction buffers
  }
}

// ---------------------------------------------------------------- launchers
// grid of the fallback passes: two blocks per SM, looping over the tiles (any grid size
// covers every tile; the SM count of the first device asked sizes it)
inline int fallback_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 2 * (sms > 0 ? sms : 152);
  }();
  return blocks;
}

// cudaFuncSetAttribute acts on the current device only: a kernel's launches on every device
// need their own call.  One bit per device records it (devices 64 and up set it on every
// launch; a repeated call is harmless, so two host threads racing on a bit are too).
inline cudaError_t set_smem_once(std::atomic<uint64_t> &done, const void *kernel, size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
  if (bit != 0 && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// 3D: RAW raw slots of NV x (rows+2) x 34 (the step: x kTmaBoxX, each rounded up to 128
// bytes), three primitive planes of NV x (rows+2) x 34, the y-sweep face states and fluxes
// (2 x NV x rows x 32), with CTU the per-thread X_x and X_y (2 x NV x rows x 32), RAW planes
// of per-cell flags and the tile's x/y flips ((rows+2) x 34 half-words).
template <typename T> size_t step_smem(int ndim, int rows, bool ctu, bool retry) {
  if (ndim < 3) return 0;
  const size_t nq = (size_t)(rows + 2) * 34;
  const size_t raw = ctu ? 2 : rows == 16 ? kRawPlanes<T, 16> : rows == 8 ? kRawPlanes<T, 8> : kRawPlanes<T, 4>;
  const bool tma = !ctu && !retry;
  const size_t slot = tma ? ((size_t)NV * (rows + 2) * kTmaBoxX * sizeof(T) + 127) / 128 * 128 : NV * nq * sizeof(T);
  const size_t per_thread = ctu ? 4 : 2;
  return raw * slot + sizeof(T) * (3 * NV * nq + per_thread * NV * rows * 32) +
         ((tma ? 0 : raw) + 1) * nq * sizeof(uint16_t);
}

// The driver's tensor-map encoder, looked up once per process (nullptr if unavailable:
// the step then stages every tile cell by cell).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Tensor maps of the state buffers for the bulk tensor staging of rows-row tiles: each
// buffer as a [NV][nz][ny][nx] tensor of T, box kTmaBoxX x (rows+2) x 1 x NV.  ok = 0 (cell-
// by-cell staging) when the copy's rules are not met: a buffer not 16-byte aligned, a row
// of nx cells not a multiple of 16 bytes, or no encoder.  The last maps are kept per host
// thread and instantiation, so repeated launches on the same buffers encode nothing.
template <typename T, int BY> TileMaps make_tile_maps(const StepArgs<T> &a) {
  struct Key {
    const void *p[3];
    int n[3];
  };
  static thread_local Key key{};
  static thread_local TileMaps cached{};
  static thread_local bool have = false;
  const Key k = {{a.U[0], a.U[1], a.U1}, {a.nx, a.ny, a.nz}};
  if (have && std::memcmp(&k, &key, sizeof k) == 0) return cached;
  TileMaps tm;
  std::memset(&tm, 0, sizeof tm);
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  const size_t es = sizeof(T);
  bool ok = enc != nullptr && ((size_t)a.nx * es) % 16 == 0;
  const T *bufs[3] = {a.U[0], a.U[1], a.U1};
  for (int i = 0; i < 3 && ok; i++) {
    if (bufs[i] == nullptr) continue;
    if (reinterpret_cast<uintptr_t>(bufs[i]) % 16 != 0) {
      ok = false;
      break;
    }
    const cuuint64_t dim[4] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz, (cuuint64_t)NV};
    const cuuint64_t str[3] = {(cuuint64_t)a.nx * es, (cuuint64_t)a.nx * a.ny * es,
                               (cuuint64_t)a.nx * a.ny * a.nz * es};
    const cuuint32_t box[4] = {(cuuint32_t)kTmaBoxX, (cuuint32_t)(BY + 2), 1u, (cuuint32_t)NV};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r =
        enc(&tm.map[i], es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
            const_cast<T *>(bufs[i]), dim, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) ok = false;
  }
  tm.ok = ok ? 1 : 0;
  key = k;
  cached = tm;
  have = true;
  return tm;
}

// SM count of the current device, looked up once per device.
inline int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    dev = -1;
  }
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) != cudaSuccess || n < 1) {
    (void)cudaGetLastError();
    n = 1;
  }
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Thread blocks of the rows-row 3D step kernel (MUSCL-Hancock, the step pass) resident on
// one SM of the current device, from the occupancy calculator; looked up once per device.
template <typename T, int BY> int resident_tiles() {
  if constexpr (sizeof(T) == 8 && BY == 16) {
    return 1;  // not offered
  } else {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      (void)cudaGetLastError();
      dev = -1;
    }
    if (dev >= 0 && dev < 64) {
      const int c = cache[dev].load(std::memory_order_relaxed);
      if (c > 0) return c;
    }
    const void *k = (const void *)step_tile_kernel<T, 3, BY, 0, false, false>;
    const size_t smem = step_smem<T>(3, BY, false, false);
    int nb = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * BY, smem) != cudaSuccess || nb < 1) {
      (void)cudaGetLastError();
      nb = 1;
    }
    if (dev >= 0 && dev < 64) cache[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
}

// Work units of a 3D launch.  Chunked tiling (zchunk > 0): one per chunk of zchunk planes
// of a column of tiles.  Balanced tiling (zchunk = 0): as many as the SMs hold step
// blocks, but at least kMinUnitPlanes planes each and at least one.
constexpr int kMinUnitPlanes = 8;
template <typename T> int tile_units(int rows, int nx, int ny, int nz, int zchunk) {
  const long long ncols = (long long)((nx + kTileX - 1) / kTileX) * ((ny + rows - 3) / (rows - 2));
  if (zchunk > 0) return (int)(ncols * ((nz + zchunk - 1) / zchunk));
  const int per_sm = rows == 16 ? resident_tiles<T, 16>() : rows == 8 ? resident_tiles<T, 8>() : resident_tiles<T, 4>();
  const long long full = (long long)device_sms() * per_sm;
  return (int)std::max<long long>(1, std::min(full, ncols * nz / kMinUnitPlanes));
}

template <typename T> int step_blocks(int ndim, int rows, int nx, int ny, int nz, int zchunk) {
  if (ndim == 1) return (nx + kTile1D - 3) / (kTile1D - 2);
  if (ndim == 2) {
    const long tiles = (long)((nx + kStripX - 1) / kStripX) * ((ny + zchunk - 1) / zchunk);
    return (int)((tiles + rows - 1) / rows);
  }
  return tile_units<T>(rows, nx, ny, nz, zchunk);
}

template <typename T, int NDIM, int BY, int SCH, bool RETRY, bool CTU>
static cudaError_t launch_tile(const StepArgs<T> &a, cudaStream_t s) {
  if constexpr (sizeof(T) == 8 && BY == 16) {
    return cudaErrorInvalidConfiguration;  // 326 KB of shared memory: not offered for FP64
  } else {
  const size_t smem = step_smem<T>(NDIM, BY, CTU, RETRY);
  static std::atomic<uint64_t> attr_done{0};  // devices whose attribute is set, per instantiation
  cudaError_t e = set_smem_once(attr_done, (const void *)step_tile_kernel<T, NDIM, BY, SCH, RETRY, CTU>, smem);
  if (e != cudaSuccess) return e;
  StepArgs<T> b = a;
  b.units = step_blocks<T>(NDIM, BY, a.nx, a.ny, a.nz, a.zchunk);
  const int blocks = RETRY ? std::min(b.units, fallback_blocks()) : b.units;
  TileMaps tm;
  if constexpr (!RETRY && !CTU) {
    tm = make_tile_maps<T, BY>(a);
    if (SCH == 2 && a.U1 == nullptr) tm.ok = 0;  // the second central-scheme stage sweeps U1
  } else {
    std::memset(&tm, 0, sizeof tm);
  }
  step_tile_kernel<T, NDIM, BY, SCH, RETRY, CTU><<<blocks, dim3(32, BY), smem, s>>>(b, tm);
  return cudaGetLastError();
  }
}

template <typename T, int WARPS, int SCH, bool RETRY, bool CTU>
static cudaError_t launch_strip2d(const StepArgs<T> &a, cudaStream_t s) {
  const int groups = step_blocks<T>(2, WARPS, a.nx, a.ny, 1, a.zchunk);
  const int blocks = RETRY ? std::min(groups, fallback_blocks()) : groups;
  step_strip2d_kernel<T, WARPS, SCH, RETRY, CTU><<<blocks, 32 * WARPS, 0, s>>>(a);
  return cudaGetLastError();
}

// CTU: the corner-transport-upwind form of the 2D and 3D kernels (in 1D there is no
// transverse direction and the max-form CFL rule is the sum; the plain kernel runs).
template <typename T, int SCH, bool RETRY, bool CTU = false>
static cudaError_t launch_step_mode(const StepArgs<T> &a, int ndim, int rows, cudaStream_t s) {
  if (ndim == 1) {
    const int ntiles = (a.nx + kTile1D - 3) / (kTile1D - 2);
    step1d_kernel<T, SCH, RETRY><<<RETRY ? std::min(ntiles, fallback_blocks()) : ntiles, kTile1D, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (ndim == 2) {
    if (rows == 4) return launch_strip2d<T, 4, SCH, RETRY, CTU>(a, s);
    if (rows == 16) return launch_strip2d<T, 16, SCH, RETRY, CTU>(a, s);
    return launch_strip2d<T, 8, SCH, RETRY, CTU>(a, s);
  }
  if (rows == 4) return launch_tile<T, 3, 4, SCH, RETRY, CTU>(a, s);
  if (rows == 16) return launch_tile<T, 3, 16, SCH, RETRY, CTU>(a, s);
  return launch_tile<T, 3, 8, SCH, RETRY, CTU>(a, s);
}

// The corner-transport-upwind form of the characteristic step with the flux of scheme SCH
// (0 HLL, 3 Roe-type, 4 HLLC); same contract as launch_step.  Instantiated once per
// scheme in its own translation unit (msh_step_ctu_*.cu).
template <typename T, int SCH>
cudaError_t launch_step_ctu(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s, int *nblocks_out) {
  if (nblocks_out) *nblocks_out = step_blocks<T>(ndim, rows, a.nx, a.ny, a.nz, a.zchunk);
  return retry ? launch_step_mode<T, SCH, true, true>(a, ndim, rows, s)
               : launch_step_mode<T, SCH, false, true>(a, ndim, rows, s);
}

}  // namespace msh
