// msh_step.cu -- fused Godunov step kernels for the ten-moment BME on uniform grids.
//
// One launch = one full step: boundary handling by index mapping (guardcells, Sec. 3.1),
// conserved -> primitive, per-direction characteristic MUSCL-Hancock reconstruction and
// HLL fluxes (Sec. 3.3), unsplit conservative update, gravity source after the hydro
// update (Sec. 3.3, last paragraph), and per-block partials of the next CFL time step,
// the FP64 conserved totals and the realizability check.  A one-block finalize kernel
// reduces the partials in a fixed order and plans the next step on the device.
//
// 2D/3D kernel layout: a thread block is a 32 x ROWS grid of threads covering cells
// (x0-1 .. x0+30, y0-1 .. y0+ROWS-2); the 30 x (ROWS-2) interior cells are updated, the
// ring of halo threads reconstructs the neighbours whose face states the interior needs.
// 3D streams z planes through a three-plane shared-memory ring (2.5D): x and y fluxes
// come from the current plane, the z flux is carried in registers from plane to plane,
// so every cell is reconstructed once per direction.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "msh_device.cuh"
#include "msh_internal.h"

namespace msh {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ block partials
template <int NT>
__device__ __forceinline__ void block_partial(double (&diag)[NV], double smax, long long bad,
                                              Partial *out) {
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
    for (int k = 0; k < NV; k++) p.diag[k] = 0.0;
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
template <typename T, int NDIM>
__device__ __forceinline__ T speed_sum(const T (&W)[NV], T idx, T idy, T idz) {
  const T r3 = T(3) * frcp(W[0]);
  T s = (fabs(W[1]) + sqrt_ratio(W[4], W[0]) * T(1.7320508075688772)) * idx;
  if (NDIM > 1) s += (fabs(W[2]) + sqrt_ratio(W[7], W[0]) * T(1.7320508075688772)) * idy;
  if (NDIM > 2) s += (fabs(W[3]) + sqrt_ratio(W[9], W[0]) * T(1.7320508075688772)) * idz;
  (void)r3;
  return s;
}

// Per-cell tail of the step: gravity source, store, next-dt speed, realizability, totals.
template <typename T, int NDIM, bool RETRY>
__device__ __forceinline__ void finish_cell(const StepArgs<T> &a, const T *__restrict__ Us,
                                            T *__restrict__ Ud, size_t N, size_t c,
                                            const T (&acc)[NV], T dt, T idx, T idy, T idz, Acc<T> &diag,
                                            T &smax, long long &bad, int32_t tag) {
  T Un[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) Un[k] = Us[k * N + c] + dt * acc[k];
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
#pragma unroll
  for (int k = 0; k < NV; k++) Ud[k * N + c] = Un[k];
  T W[NV];
  cons_to_prim(Un, W);
  if (!realizable(W)) {
    bad = min(bad, (long long)c);
    // tag the cell for the next fallback pass (a cell tagged by an earlier pass keeps its tag)
    const int32_t f = a.flags[c];
    if (!((f >> 3) == tag && (f & 7) < a.level)) {
      a.flags[c] = tag * 8 + a.level;
      atomicAdd(&a.ctrl->nbad[a.level], 1);
    }
  }
  smax = fmax(smax, speed_sum<T, NDIM>(W, idx, idy, idz));
  diag.add(Un);
}

template <typename T, int NT>
__device__ __forceinline__ void write_partial(const Acc<T> &diag, T smax, long long bad, Partial *out) {
  double d[NV];
  diag.get(d);
  block_partial<NT>(d, (double)smax, bad, out);
}

// A cell takes first-order faces in fallback pass `level` if an earlier pass of this step
// tagged it.  Tags written during the current pass are ignored, so every thread block of
// a pass sees the same tagged set.
__device__ __forceinline__ bool tagged(int32_t f, int32_t tag, int level) {
  return (f >> 3) == tag && (f & 7) < level;
}

// ------------------------------------------------------------------ 1D kernel
template <typename T, bool RETRY>
__global__ void __launch_bounds__(kTile1D) step1d_kernel(StepArgs<T> a) {
  constexpr int B = kTile1D, SXX = B + 2;
  const Ctrl *ctrl = a.ctrl;
  if (ctrl->done) return;
  if (RETRY && ctrl->nbad[a.level - 1] == 0) return;
  const int64_t step = ctrl->step;
  const int32_t tag = (int32_t)(step & 0x0fffffff) + 1;
  __shared__ unsigned char sFl[RETRY ? SXX : 1];
  const T *__restrict__ Us = a.U[step & 1];
  T *__restrict__ Ud = a.U[(step + 1) & 1];
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
  reconstruct(wm, w0, wp, nu, lo, hi);
  if (RETRY) first_order_faces(sFl[t] != 0, sFl[t + 1] != 0, sFl[t + 2] != 0, w0, lo, hi);
#pragma unroll
  for (int k = 0; k < NV; k++) sH[k][t] = hi[k];
  __syncthreads();
  if (t >= 1) {
    T hl[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) hl[k] = sH[k][t - 1];
    hll(hl, lo, F);
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
    finish_cell<T, 1, RETRY>(a, Us, Ud, N, (size_t)gx, acc, dt, idx, T(0), T(0), diag, smax, bad, tag);
  }
  write_partial<T, B>(diag, smax, bad, a.part + tile);
  __syncthreads();  // the next tile reuses the shared arrays
  }
}

// -------------------------------------------------------------- 2D/3D kernel
template <typename T, int D, int SY, int SX>
__device__ __forceinline__ void gather(const T *__restrict__ pl, int sy, int sx, T (&w)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) w[k] = pl[(Frame<D>::g(k) * SY + sy) * SX + sx];
}

template <typename T, int NDIM, int BY, bool RETRY>
__global__ void __launch_bounds__(32 * BY, (BY <= 8 ? 2 : 1)) step_tile_kernel(StepArgs<T> a) {
  constexpr int SX = 34, SY = BY + 2;
  constexpr int NPL = (NDIM == 3) ? 3 : 1;
  constexpr int PL = NV * SY * SX;
  const Ctrl *ctrl = a.ctrl;
  if (ctrl->done) return;
  if (RETRY && ctrl->nbad[a.level - 1] == 0) return;
  const int64_t step = ctrl->step;
  const int32_t tag = (int32_t)(step & 0x0fffffff) + 1;
  // fallback tags of the staged cells (fallback pass only)
  __shared__ unsigned char sFl[RETRY ? NPL : 1][RETRY ? SY : 1][RETRY ? SX : 1];
  const T *__restrict__ Us = a.U[step & 1];
  T *__restrict__ Ud = a.U[(step + 1) & 1];
  const double dtd = ctrl->dt;
  const T dt = (T)dtd;
  const T nux = (T)(0.5 * dtd / a.dx[0]), idx = (T)(1.0 / a.dx[0]);
  const T nuy = (T)(0.5 * dtd / a.dx[1]), idy = (T)(1.0 / a.dx[1]);
  const T nuz = (T)(0.5 * dtd / a.dx[2]), idz = (T)(1.0 / a.dx[2]);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sW = reinterpret_cast<T *>(smem_raw);
  T *sX = sW + NPL * PL;  // [NV][BY][32] exchange buffer for the y sweep
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t N = (size_t)nx * ny * nz;
  // One thread block per tile for the step; the fallback passes run on a small grid that
  // loops over the tiles, so a pass with nothing to do costs only its launch.
  const int tilesx = (nx + kTileX - 1) / kTileX, tilesy = (ny + BY - 3) / (BY - 2);
  const int tilesz = NDIM == 3 ? (nz + a.zchunk - 1) / a.zchunk : 1;
  const int ntiles = tilesx * tilesy * tilesz;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const int bxi = tile % tilesx, byi = (tile / tilesx) % tilesy, bzi = tile / (tilesx * tilesy);
  const int x0 = bxi * kTileX, y0 = byi * (BY - 2);
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const int sx = tx + 1, sy = ty + 1;
  const bool interior = tx >= 1 && tx <= kTileX && ty >= 1 && ty <= BY - 2;
  const bool valid = interior && gx < nx && gy < ny;

  auto load_plane = [&](int buf, int z) {
    bool mz = false;
    const int zz = (NDIM == 3) ? map_index(z, nz, a.bc[4], a.bc[5], mz) : 0;
    T *dst = sW + buf * PL;
    for (int i = tid; i < SY * SX; i += 32 * BY) {
      const int qy = i / SX, qx = i - qy * SX;
      const bool need = (qy >= 2 && qy <= BY - 1) || (qx >= 2 && qx <= 31);
      if (!need) continue;
      bool mx, my;
      const int xx = map_index(x0 - 2 + qx, nx, a.bc[0], a.bc[1], mx);
      const int yy = map_index(y0 - 2 + qy, ny, a.bc[2], a.bc[3], my);
      const unsigned flip = (mx ? flip_mask(0) : 0u) ^ (my ? flip_mask(1) : 0u) ^ (mz ? flip_mask(2) : 0u);
      const size_t c = ((size_t)zz * ny + yy) * nx + xx;
      T U[NV], W[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) {
        const T v = Us[k * N + c];
        U[k] = ((flip >> k) & 1u) ? -v : v;
      }
      cons_to_prim(U, W);
#pragma unroll
      for (int k = 0; k < NV; k++) dst[(k * SY + qy) * SX + qx] = W[k];
      if (RETRY) sFl[buf][qy][qx] = tagged(a.flags[c], tag, a.level);
    }
  };
  auto fl = [&](int buf, int qy, int qx) -> bool { return RETRY ? sFl[RETRY ? buf : 0][RETRY ? qy : 0][RETRY ? qx : 0] != 0 : false; };

  // x and y sweeps of the plane in buffer `buf`, accumulating -dF/dx - dG/dy into acc
  auto sweep_xy = [&](int b, T (&acc)[NV]) {
    const T *pl = sW + b * PL;
    if (ty >= 1 && ty <= BY - 2) {  // warp-uniform: one warp per row
      T wm[NV], w0[NV], wp[NV], lo[NV], hi[NV], hl[NV], F[NV];
      gather<T, 0, SY, SX>(pl, sy, sx - 1, wm);
      gather<T, 0, SY, SX>(pl, sy, sx, w0);
      gather<T, 0, SY, SX>(pl, sy, sx + 1, wp);
      reconstruct(wm, w0, wp, nux, lo, hi);
      if (RETRY) first_order_faces(fl(b, sy, sx - 1), fl(b, sy, sx), fl(b, sy, sx + 1), w0, lo, hi);
#pragma unroll
      for (int k = 0; k < NV; k++) hl[k] = __shfl_up_sync(FULL, hi[k], 1);
      hll(hl, lo, F);  // flux at the lower x face of this cell
#pragma unroll
      for (int k = 0; k < NV; k++) {
        const T Fr = __shfl_down_sync(FULL, F[k], 1);
        acc[k] += (F[k] - Fr) * idx;
      }
    }
    const bool ycol = tx >= 1 && tx <= kTileX;
    T lo[NV], F[NV];
    if (ycol) {
      T wm[NV], w0[NV], wp[NV], hi[NV];
      gather<T, 1, SY, SX>(pl, sy - 1, sx, wm);
      gather<T, 1, SY, SX>(pl, sy, sx, w0);
      gather<T, 1, SY, SX>(pl, sy + 1, sx, wp);
      reconstruct(wm, w0, wp, nuy, lo, hi);
      if (RETRY) first_order_faces(fl(b, sy - 1, sx), fl(b, sy, sx), fl(b, sy + 1, sx), w0, lo, hi);
#pragma unroll
      for (int k = 0; k < NV; k++) sX[(k * BY + ty) * 32 + tx] = hi[k];
    }
    __syncthreads();
    if (ycol && ty >= 1) {
      T hl[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) hl[k] = sX[(k * BY + ty - 1) * 32 + tx];
      hll(hl, lo, F);
    }
    __syncthreads();
    if (ycol && ty >= 1) {
#pragma unroll
      for (int k = 0; k < NV; k++) sX[(k * BY + ty) * 32 + tx] = F[k];
    }
    __syncthreads();
    if (interior) {
#pragma unroll
      for (int k = 0; k < NV; k++) {
        const T Fu = sX[(k * BY + ty + 1) * 32 + tx];
        acc[Frame<1>::g(k)] += (F[k] - Fu) * idy;
      }
    }
  };

  Acc<T> diag;
  diag.zero();
  T smax = T(0);
  long long bad = LLONG_MAX;

  if (NDIM == 2) {
    load_plane(0, 0);
    __syncthreads();
    T acc[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) acc[k] = T(0);
    sweep_xy(0, acc);
    if (valid)
      finish_cell<T, NDIM, RETRY>(a, Us, Ud, N, (size_t)gy * nx + gx, acc, dt, idx, idy, idz, diag, smax, bad, tag);
  } else {
    const int z0 = bzi * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    auto buf = [](int p) { return ((p % 3) + 3) % 3; };
    // prologue: z face state of cell z0-1 and the flux through its upper face
    load_plane(buf(z0 - 2), z0 - 2);
    load_plane(buf(z0 - 1), z0 - 1);
    load_plane(buf(z0), z0);
    __syncthreads();
    T hprev[NV], Fprev[NV];
    if (interior) {
      T wm[NV], w0[NV], wp[NV], lo[NV];
      gather<T, 2, SY, SX>(sW + buf(z0 - 2) * PL, sy, sx, wm);
      gather<T, 2, SY, SX>(sW + buf(z0 - 1) * PL, sy, sx, w0);
      gather<T, 2, SY, SX>(sW + buf(z0) * PL, sy, sx, wp);
      reconstruct(wm, w0, wp, nuz, lo, hprev);
      if (RETRY)
        first_order_faces(fl(buf(z0 - 2), sy, sx), fl(buf(z0 - 1), sy, sx), fl(buf(z0), sy, sx), w0, lo, hprev);
    }
    __syncthreads();
    load_plane(buf(z0 + 1), z0 + 1);
    __syncthreads();
    if (interior) {
      T wm[NV], w0[NV], wp[NV], lo[NV], hi[NV];
      gather<T, 2, SY, SX>(sW + buf(z0 - 1) * PL, sy, sx, wm);
      gather<T, 2, SY, SX>(sW + buf(z0) * PL, sy, sx, w0);
      gather<T, 2, SY, SX>(sW + buf(z0 + 1) * PL, sy, sx, wp);
      reconstruct(wm, w0, wp, nuz, lo, hi);
      if (RETRY) first_order_faces(fl(buf(z0 - 1), sy, sx), fl(buf(z0), sy, sx), fl(buf(z0 + 1), sy, sx), w0, lo, hi);
      hll(hprev, lo, Fprev);
#pragma unroll
      for (int k = 0; k < NV; k++) hprev[k] = hi[k];
    }
    __syncthreads();
    load_plane(buf(z0 + 2), z0 + 2);
    __syncthreads();
    for (int z = z0; z < z1; z++) {
      T acc[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) acc[k] = T(0);
      sweep_xy(buf(z), acc);
      if (interior) {
        T wm[NV], w0[NV], wp[NV], lo[NV], hi[NV], F[NV];
        gather<T, 2, SY, SX>(sW + buf(z) * PL, sy, sx, wm);
        gather<T, 2, SY, SX>(sW + buf(z + 1) * PL, sy, sx, w0);
        gather<T, 2, SY, SX>(sW + buf(z + 2) * PL, sy, sx, wp);
        reconstruct(wm, w0, wp, nuz, lo, hi);  // cell z+1
        if (RETRY) first_order_faces(fl(buf(z), sy, sx), fl(buf(z + 1), sy, sx), fl(buf(z + 2), sy, sx), w0, lo, hi);
        hll(hprev, lo, F);                     // flux through the upper z face of cell z
#pragma unroll
        for (int k = 0; k < NV; k++) {
          acc[Frame<2>::g(k)] += (Fprev[k] - F[k]) * idz;
          hprev[k] = hi[k];
          Fprev[k] = F[k];
        }
      }
      if (valid)
        finish_cell<T, NDIM, RETRY>(a, Us, Ud, N, ((size_t)z * ny + gy) * nx + gx, acc, dt, idx, idy, idz, diag,
                                    smax, bad, tag);
      __syncthreads();
      if (z + 1 < z1) {
        load_plane(buf(z), z + 3);
        __syncthreads();
      }
    }
  }
  write_partial<T, 32 * BY>(diag, smax, bad, a.part + tile);
  }
}

// ----------------------------------------------------------------- scan kernel
// Partials (totals, max signal speed sum, first non-realizable cell) of a state.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) scan_kernel(const T *__restrict__ U, size_t N, T idx, T idy, T idz,
                                                   Partial *part) {
  double diag[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) diag[k] = 0.0;
  T smax = T(0);
  long long bad = LLONG_MAX;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    T Uc[NV], W[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) Uc[k] = U[k * N + c];
    cons_to_prim(Uc, W);
    if (!realizable(W)) bad = min(bad, (long long)c);
    smax = fmax(smax, speed_sum<T, NDIM>(W, idx, idy, idz));
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
  for (int k = 0; k < NV; k++) c->totals[k] = sd[0][k];
  const long long b = sb[0];
  c->realizable = (b == LLONG_MAX);
  c->first_bad = (b == LLONG_MAX) ? -1 : b;
  c->dt_cfl = c->cfl / sd[0][NV];
  if (mode == 1) {
    c->done = 1;
    return;
  }
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
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

__global__ void run_start_kernel(Ctrl *c, double t_end, int64_t max_steps, double dt_max) {
  c->t_end = t_end;
  c->max_step = (max_steps > INT64_MAX - c->step) ? INT64_MAX : c->step + max_steps;
  c->dt_max = dt_max;
  c->done = 0;
  c->status = 0;
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
  plan(c);
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

// ---------------------------------------------------------------- launchers
// grid of the fallback passes: two blocks per SM, looping over the tiles
static int fallback_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = 2 * (sms > 0 ? sms : 152);
  }
  return blocks;
}

template <typename T> size_t step_smem(int ndim, int rows) {
  if (ndim == 1) return 0;
  const int npl = ndim == 3 ? 3 : 1;
  return sizeof(T) * ((size_t)npl * NV * (rows + 2) * 34 + (size_t)NV * rows * 32);
}

template <typename T> int step_blocks(int ndim, int rows, int nx, int ny, int nz, int zchunk) {
  if (ndim == 1) return (nx + kTile1D - 3) / (kTile1D - 2);
  const int bx = (nx + kTileX - 1) / kTileX;
  const int by = (ny + rows - 3) / (rows - 2);
  const int bz = ndim == 3 ? (nz + zchunk - 1) / zchunk : 1;
  return bx * by * bz;
}

template <typename T, int NDIM, int BY, bool RETRY>
static cudaError_t launch_tile(const StepArgs<T> &a, cudaStream_t s) {
  const size_t smem = step_smem<T>(NDIM, BY);
  static bool attr_set = false;  // one attribute call per instantiation and process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(step_tile_kernel<T, NDIM, BY, RETRY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int ntiles = step_blocks<T>(NDIM, BY, a.nx, a.ny, a.nz, a.zchunk);
  const int blocks = RETRY ? std::min(ntiles, fallback_blocks()) : ntiles;
  step_tile_kernel<T, NDIM, BY, RETRY><<<blocks, dim3(32, BY), smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, bool RETRY>
static cudaError_t launch_step_mode(const StepArgs<T> &a, int ndim, int rows, cudaStream_t s) {
  if (ndim == 1) {
    const int ntiles = (a.nx + kTile1D - 3) / (kTile1D - 2);
    step1d_kernel<T, RETRY><<<RETRY ? std::min(ntiles, fallback_blocks()) : ntiles, kTile1D, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (ndim == 2) {
    if (rows == 4) return launch_tile<T, 2, 4, RETRY>(a, s);
    if (rows == 16) return launch_tile<T, 2, 16, RETRY>(a, s);
    return launch_tile<T, 2, 8, RETRY>(a, s);
  }
  if (rows == 4) return launch_tile<T, 3, 4, RETRY>(a, s);
  if (rows == 16) return launch_tile<T, 3, 16, RETRY>(a, s);
  return launch_tile<T, 3, 8, RETRY>(a, s);
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s, int *nblocks_out) {
  if (nblocks_out) *nblocks_out = step_blocks<T>(ndim, rows, a.nx, a.ny, a.nz, a.zchunk);
  return retry ? launch_step_mode<T, true>(a, ndim, rows, s) : launch_step_mode<T, false>(a, ndim, rows, s);
}

template <typename T>
cudaError_t launch_scan(const T *U, size_t N, int nx, int ny, int ndim, const double *dx, Partial *part,
                        int nparts, cudaStream_t s) {
  const T ix = (T)(1.0 / dx[0]), iy = (T)(1.0 / dx[1]), iz = (T)(1.0 / dx[2]);
  if (ndim == 1) scan_kernel<T, 1><<<nparts, 256, 0, s>>>(U, N, ix, iy, iz, part);
  else if (ndim == 2) scan_kernel<T, 2><<<nparts, 256, 0, s>>>(U, N, ix, iy, iz, part);
  else scan_kernel<T, 3><<<nparts, 256, 0, s>>>(U, N, ix, iy, iz, part);
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
  template size_t step_smem<T>(int, int);                                                            \
  template cudaError_t launch_scan<T>(const T *, size_t, int, int, int, const double *, Partial *, int, \
                                      cudaStream_t);                                                 \
  template cudaError_t launch_convert<T>(T *, size_t, int, cudaStream_t);                            \
  template cudaError_t launch_gravity_field<T>(const double *, T *, int, int, int, int, const double *, cudaStream_t);
MSH_INST(float)
MSH_INST(double)

}  // namespace msh
