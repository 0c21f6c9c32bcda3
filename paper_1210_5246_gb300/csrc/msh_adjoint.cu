// msh_adjoint.cu -- discrete adjoint of the step (msh_adjoint_run).
//
// Reverse step n maps lam^{n+1} = dL/dU^{n+1} to lam^n = dL/dU^n for the frozen time step
// dt_n, with every branch of the forward step frozen (MC limiter selection, face-state
// fallback, HLL branch and min/max of the signal speeds, a-posteriori fallback tags):
//   1. lam* = G^T lam^{n+1}           gravity source (linear in U* for a fixed -grad Phi),
//                                     evaluated where the passes below need it
//   2. per direction d, one fused pass over pencils along d (adj_pencil_kernel):
//      F^bar = (dt/dx)(lam*_j - lam*_{j-1}) through the HLL flux at face j-1/2 -> adjoints of
//      the face states hi_{j-1}, lo_j; the reconstruction of cell j reversed -> adjoints of
//      W_{j-1}, W_j, W_{j+1}; summed per cell by warp shuffles onto the padded primitive
//      adjoint (deterministic, no atomics; the first direction writes, later ones add)
//   3. fold        lam^n_i = lam*_i + (dW/dU)^T W^bar_i: in the last direction's pass for a
//                  cell no ghost cell maps to; else (within two cells of an edge) plus the
//                  ghost images of cell i (periodic wrap, outflow copy, reflect mirror with
//                  its sign flips) in adj_fold_kernel
// Forward states are checkpointed every K steps (by a forward sweep here, or by the step
// kernels of the recorded run: msh_adjoint_tape) and recomputed segment by segment during
// the reverse sweep.  Which steps tagged cells for the a-posteriori fallback is known on
// the host: only those steps launch their fallback passes when recomputed, and only those
// are re-run before their reverse, to restore their tags.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/msh.h"
#include "msh_adjoint.cuh"
#include "msh_device.cuh"
#include "msh_internal.h"
#include "msh_step_kernels.cuh"

namespace msh {

template <typename T> struct AdjArgs {
  const T *U;          // U^n [NV][N]
  const T *lam;        // lam^{n+1}
  T *out;              // lam^n
  const T *acc;        // -grad Phi [3][N] or nullptr
  const int32_t *flags;
  const Ctrl *ctrl;    // fallback pass counters of the re-run forward step
  int32_t tag;
  T *Wb;               // primitive adjoint on the padded grid [NV][Npad]
  int n[3], ndim, bc[6];
  double dx[3], dt;
  int d;               // sweep direction
};

__device__ __forceinline__ int last_pass(const Ctrl *c) {
  int p = 0;
  for (int q = 1; q <= kFallbackPasses; q++) {
    if (c->nbad[q - 1] > 0) p = q;
    else break;
  }
  return p;
}

// padded index: 2 ghost layers on every active dim
__device__ __forceinline__ size_t pad_index(const int (&n)[3], int ndim, const int (&c)[3]) {
  const int g0 = 2, g1 = ndim > 1 ? 2 : 0, g2 = ndim > 2 ? 2 : 0;
  const int p0 = n[0] + 2 * g0, p1 = n[1] + 2 * g1;
  return ((size_t)(c[2] + g2) * p1 + (c[1] + g1)) * p0 + (c[0] + g0);
}

// conserved state, mirror mask and tag of a (possibly ghost) cell
template <typename T>
__device__ __forceinline__ size_t load_cell(const AdjArgs<T> &a, const int (&c)[3], T (&U)[NV], unsigned &flip) {
  int m[3];
  flip = 0u;
  for (int e = 0; e < 3; e++) {
    if (e < a.ndim) {
      bool mir;
      m[e] = map_index(c[e], a.n[e], a.bc[2 * e], a.bc[2 * e + 1], mir);
      if (mir) flip ^= flip_mask(e);
    } else {
      m[e] = 0;
    }
  }
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  const size_t idx = ((size_t)m[2] * a.n[1] + m[1]) * a.n[0] + m[0];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T v = a.U[k * N + idx];
    U[k] = ((flip >> k) & 1u) ? -v : v;
  }
  return idx;
}

template <typename T, int D>
__device__ __forceinline__ void local_w(const AdjArgs<T> &a, int (&c)[3], int j, T (&w)[NV], bool &tagged_cell,
                                        int pass) {
  c[D] = j;
  T U[NV], W[NV];
  unsigned flip;
  const size_t idx = load_cell(a, c, U, flip);
  cons_to_prim(U, W);
#pragma unroll
  for (int k = 0; k < NV; k++) w[k] = W[Frame<D>::g(k)];
  const int32_t f = a.flags[idx];
  tagged_cell = (f >> 3) == a.tag && (f & 7) < pass;
}

// lam* = G^T lam^{n+1} of cell c (the gravity source's adjoint; identity without gravity)
template <typename T>
__device__ __forceinline__ void lam_star(const AdjArgs<T> &a, size_t N, size_t c, T (&ls)[NV]) {
  T lam[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) lam[k] = a.lam[k * N + c];
  if (a.acc) {
    const T g[3] = {a.acc[c], a.acc[N + c], a.acc[2 * N + c]};
    gravity_vjp(g, (T)a.dt, lam, ls);
  } else {
#pragma unroll
    for (int k = 0; k < NV; k++) ls[k] = lam[k];
  }
}

// Reverse of one sweep direction D, fused: one warp per segment of a pencil along D, lane l
// holding the extended position j = -2 + 26 seg - 3 + l.  Each lane converts its own cell
// once and takes its neighbours' primitive states, tags and lam* by shuffles; it recomputes
// its reconstruction (the face states lo_j, hi_j, forward branches), reverses the HLL flux
// through its lower face j-1/2 with F^bar = (dt/dx)(lam*_j - lam*_{j-1}) (faces j in
// [0, n_D]; ghost cells are not updated, so their lam* is zero), reverses its
// reconstruction with the adjoints of its two face states (the upper one from lane l+1;
// extended cells j in [-1, n_D]), and sums the three reconstruction adjoints that reach its
// cell (its own and its neighbours').  That sum is complete in lanes 3..28 (each needs
// the faces of lanes l-1 .. l+2 and the states of lanes l-3 .. l+3), which own the padded
// positions [-2, n_D + 1] segment by segment: direction 0 writes them, a later direction
// adds where the cell is inside the grid along D and writes its own ghost layers.
constexpr int kAdjSeg = 26;  // complete positions per warp segment

// A cell that some ghost cell maps to (within two cells of the grid's edge along an active
// axis, for every kind of boundary): its adjoint also collects its ghost images, which the
// fold kernel adds.
__device__ __forceinline__ bool ghost_source(const int (&n)[3], int ndim, const int (&c)[3]) {
  for (int d = 0; d < ndim; d++)
    if (c[d] <= 1 || c[d] >= n[d] - 2) return true;
  return false;
}

// The last direction's pass finishes a cell that is no ghost source at once:
// lam^n = lam* + (dW/dU)^T (W^bar of the earlier directions + s).
template <typename T>
__device__ __forceinline__ void fold_cell(const AdjArgs<T> &a, size_t N, size_t Npad, size_t ci, size_t pi,
                                          bool first, const T (&s)[NV], const T (&ls)[NV]) {
  T U[NV], Ub[NV], Wb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    U[k] = a.U[k * N + ci];
    Wb[k] = first ? s[k] : a.Wb[k * Npad + pi] + s[k];
    Ub[k] = T(0);
  }
  cons_to_prim_vjp(U, Wb, Ub);
#pragma unroll
  for (int k = 0; k < NV; k++) a.out[k * N + ci] = ls[k] + Ub[k];
}

// The warp-wide part of the fused pass: lane l holds extended position j of one pencil along
// D with its primitive state w0 (local frame), tag f0 and lam* ls (global order); returns
// in s (global order) the primitive adjoint of its cell from this direction, complete in
// lanes 3..28.
template <typename T, int D>
__device__ __forceinline__ void adj_pencil_lane(int j, int nd, T nu, T dtdx, const T (&w0)[NV], bool f0,
                                                const T (&ls)[NV], T (&s)[NV]) {
  T wm[NV], wp[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    wm[k] = __shfl_up_sync(0xffffffffu, w0[k], 1);
    wp[k] = __shfl_down_sync(0xffffffffu, w0[k], 1);
  }
  const bool fm = __shfl_up_sync(0xffffffffu, (int)f0, 1) != 0;
  const bool fp = __shfl_down_sync(0xffffffffu, (int)f0, 1) != 0;
  // forward face states of this cell
  T lo[NV], hi[NV];
  reconstruct(wm, w0, wp, nu, lo, hi);
  first_order_faces(fm, f0, fp, w0, lo, hi);
  // the flux adjoint at the lower face j-1/2: hb to hi_{j-1} (lane l-1), lb to lo_j
  T hm[NV], Fb[NV], hb[NV], lb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    hm[k] = __shfl_up_sync(0xffffffffu, hi[k], 1);
    const int gk = Frame<D>::g(k);
    Fb[k] = dtdx * (ls[gk] - __shfl_up_sync(0xffffffffu, ls[gk], 1));
    hb[k] = T(0);
    lb[k] = T(0);
  }
  if (j >= 0 && j <= nd) hll_vjp(hm, lo, Fb, hb, lb);
  T hib[NV], gm[NV], g0[NV], gp[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    hib[k] = __shfl_down_sync(0xffffffffu, hb[k], 1);
    gm[k] = g0[k] = gp[k] = T(0);
  }
  if (j >= -1 && j <= nd) reconstruct_vjp(wm, w0, wp, nu, fm, f0, fp, lb, hib, gm, g0, gp);
  // g0 + gm of lane l+1 + gp of lane l-1
#pragma unroll
  for (int k = 0; k < NV; k++)
    s[Frame<D>::g(k)] = g0[k] + __shfl_down_sync(0xffffffffu, gm[k], 1) + __shfl_up_sync(0xffffffffu, gp[k], 1);
}

// Direction 0: one warp per segment of a pencil along x (lanes along x, coalesced).  LAST: x
// is the grid's only direction (1D), and the pass finishes the cells that are no ghost source.
template <typename T, int D, bool LAST>
__global__ void __launch_bounds__(256) adj_pencil_kernel(AdjArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int nd = a.n[D];
  const int nseg = (nd + 4 + kAdjSeg - 1) / kAdjSeg;
  constexpr int O1 = D == 0 ? 1 : 0, O2 = D == 2 ? 1 : 2;  // the other two axes
  const long nwarps = (long)a.n[O1] * a.n[O2] * nseg;
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  const int g1 = a.ndim > 1 ? 2 : 0, g2 = a.ndim > 2 ? 2 : 0;
  const size_t Npad = (size_t)(a.n[0] + 4) * (a.n[1] + 2 * g1) * (a.n[2] + 2 * g2);
  const int pass = last_pass(a.ctrl);
  const T nu = (T)(0.5 * a.dt / a.dx[D]);
  const T dtdx = (T)(a.dt / a.dx[D]);
  const long wstride = (long)gridDim.x * (blockDim.x >> 5);
  const long npen = (long)a.n[O1] * a.n[O2];
  for (long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nwarps; w += wstride) {
    const long pen = w % npen;
    const int seg = (int)(w / npen);
    int c[3];
    c[O1] = (int)(pen % a.n[O1]);
    c[O2] = (int)(pen / a.n[O1]);
    const int j = -2 + seg * kAdjSeg - 3 + lane;
    T w0[NV], ls[NV], s[NV];
    bool f0;
    local_w<T, D>(a, c, j, w0, f0, pass);  // also sets c[D] = j
    if (j >= 0 && j < nd) {
      lam_star(a, N, ((size_t)c[2] * a.n[1] + c[1]) * a.n[0] + c[0], ls);
    } else {
#pragma unroll
      for (int k = 0; k < NV; k++) ls[k] = T(0);
    }
    adj_pencil_lane<T, D>(j, nd, nu, dtdx, w0, f0, ls, s);
    if (lane >= 3 && lane <= 28 && j <= nd + 1) {
      const size_t pi = pad_index(a.n, a.ndim, c);
      if (LAST && j >= 0 && j < nd && !ghost_source(a.n, a.ndim, c)) {
        fold_cell(a, N, Npad, ((size_t)c[2] * a.n[1] + c[1]) * a.n[0] + c[0], pi, D == 0, s, ls);
      } else if (D == 0 || j < 0 || j >= nd) {
#pragma unroll
        for (int k = 0; k < NV; k++) a.Wb[k * Npad + pi] = s[k];
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) a.Wb[k * Npad + pi] += s[k];
      }
    }
  }
}

// Directions 1 and 2: the same pass with the pencils' data staged through shared memory so
// that every global access runs along x.  A block of eight warps takes 8 cells along x and
// the 32 extended positions of one segment along D (26 complete, a 3-cell halo at each end),
// for one index of the remaining axis: each thread loads one cell of the tile (the conserved
// state converted to the local frame of D, lam*, tag; a row of 8 cells is one 32-byte sector
// in FP32), each warp then runs one column as a pencil (lanes along D, neighbours by
// shuffles), leaving the column's result in place of its state, and the block adds the 26
// complete rows to the padded adjoint row by row (the last direction finishes the cells
// that are no ghost source instead).  One column per warp gives several waves of tiles, so
// the last, partly filled wave is short.
constexpr int kAdjTileX = 8, kAdjTileP = 9;  // tile columns; padded row pitch (no bank conflicts)
constexpr int kAdjTileThreads = 256;

template <typename T> size_t adj_tile_smem() {
  return (2 * (size_t)NV * 32 * kAdjTileP) * sizeof(T) + 32 * kAdjTileP * sizeof(int);
}

template <typename T, int D, bool LAST>
__global__ void __launch_bounds__(kAdjTileThreads, sizeof(T) == 4 ? 2 : 1) adj_tile_kernel(AdjArgs<T> a) {
  static_assert(D == 1 || D == 2, "the staged pass runs along y or z");
  extern __shared__ __align__(16) unsigned char adj_smem[];
  T *sW = reinterpret_cast<T *>(adj_smem);            // [NV][32 along D][kAdjTileP along x]
  T *sL = sW + (size_t)NV * 32 * kAdjTileP;           // lam*, same layout (global order)
  int *sF = reinterpret_cast<int *>(sL + (size_t)NV * 32 * kAdjTileP);  // tags
  const int nd = a.n[D];
  const int nseg = (nd + 4 + kAdjSeg - 1) / kAdjSeg;
  constexpr int O = D == 1 ? 2 : 1;  // the remaining axis
  const int tilesx = (a.n[0] + kAdjTileX - 1) / kAdjTileX;
  const long ntiles = (long)tilesx * nseg * a.n[O];
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  const int g1 = a.ndim > 1 ? 2 : 0, g2 = a.ndim > 2 ? 2 : 0;
  const size_t Npad = (size_t)(a.n[0] + 4) * (a.n[1] + 2 * g1) * (a.n[2] + 2 * g2);
  const int pass = last_pass(a.ctrl);
  const T nu = (T)(0.5 * a.dt / a.dx[D]);
  const T dtdx = (T)(a.dt / a.dx[D]);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int bx = (int)(tile % tilesx);
    const int seg = (int)((tile / tilesx) % nseg);
    const int o = (int)(tile / ((long)tilesx * nseg));
    const int x0 = bx * kAdjTileX, jb = -2 + seg * kAdjSeg - 3;
    for (int i = tid; i < 32 * kAdjTileX; i += blockDim.x) {
      const int r = i / kAdjTileX, x = i - r * kAdjTileX;
      int c[3];
      c[0] = min(x0 + x, a.n[0] - 1);
      c[O] = o;
      const int j = jb + r;
      T w[NV], ls[NV];
      bool f;
      local_w<T, D>(a, c, j, w, f, pass);  // sets c[D] = j
      if (j >= 0 && j < nd) {
        lam_star(a, N, ((size_t)c[2] * a.n[1] + c[1]) * a.n[0] + c[0], ls);
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) ls[k] = T(0);
      }
#pragma unroll
      for (int k = 0; k < NV; k++) {
        sW[(k * 32 + r) * kAdjTileP + x] = w[k];
        sL[(k * 32 + r) * kAdjTileP + x] = ls[k];
      }
      sF[r * kAdjTileP + x] = f;
    }
    __syncthreads();
    for (int x = warp; x < kAdjTileX; x += blockDim.x >> 5) {
      T w0[NV], ls[NV], s[NV];
#pragma unroll
      for (int k = 0; k < NV; k++) {
        w0[k] = sW[(k * 32 + lane) * kAdjTileP + x];
        ls[k] = sL[(k * 32 + lane) * kAdjTileP + x];
      }
      const bool f0 = sF[lane * kAdjTileP + x] != 0;
      adj_pencil_lane<T, D>(jb + lane, nd, nu, dtdx, w0, f0, ls, s);
#pragma unroll
      for (int k = 0; k < NV; k++) sW[(k * 32 + lane) * kAdjTileP + x] = s[k];  // only this lane read it
    }
    __syncthreads();
    for (int i = tid; i < kAdjSeg * kAdjTileX; i += blockDim.x) {
      const int r = 3 + i / kAdjTileX, x = i % kAdjTileX;
      const int j = jb + r;
      if (x0 + x >= a.n[0] || j > nd + 1) continue;
      int c[3];
      c[0] = x0 + x;
      c[O] = o;
      c[D] = j;
      const size_t pi = pad_index(a.n, a.ndim, c);
      if (LAST && j >= 0 && j < nd && !ghost_source(a.n, a.ndim, c)) {
        T sv[NV], ls[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
          sv[k] = sW[(k * 32 + r) * kAdjTileP + x];
          ls[k] = sL[(k * 32 + r) * kAdjTileP + x];
        }
        fold_cell(a, N, Npad, ((size_t)c[2] * a.n[1] + c[1]) * a.n[0] + c[0], pi, false, sv, ls);
      } else if (j < 0 || j >= nd) {
#pragma unroll
        for (int k = 0; k < NV; k++) a.Wb[k * Npad + pi] = sW[(k * 32 + r) * kAdjTileP + x];
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) a.Wb[k * Npad + pi] += sW[(k * 32 + r) * kAdjTileP + x];
      }
    }
    __syncthreads();  // the next tile restages the shared arrays
  }
}

template <typename T, int D, bool LAST> cudaError_t launch_adj_tile(const AdjArgs<T> &a, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = set_smem_once(attr_done, (const void *)adj_tile_kernel<T, D, LAST>, adj_tile_smem<T>());
  if (e != cudaSuccess) return e;
  const int nseg = (a.n[D] + 4 + kAdjSeg - 1) / kAdjSeg;
  const long tiles = (long)((a.n[0] + kAdjTileX - 1) / kAdjTileX) * nseg * a.n[D == 1 ? 2 : 1];
  adj_tile_kernel<T, D, LAST><<<(int)std::min<long>(tiles, 1L << 20), kAdjTileThreads, adj_tile_smem<T>(), st>>>(a);
  return cudaGetLastError();
}

// fold of the ghost sources: lam^n_i = lam*_i + (dW/dU)^T Wb_i + images of ghost cells whose
// source is i (the other cells are finished by the last direction's pass)
template <typename T>
__global__ void adj_fold_kernel(AdjArgs<T> a) {
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  int g[3] = {2, a.ndim > 1 ? 2 : 0, a.ndim > 2 ? 2 : 0};
  const size_t Npad = (size_t)(a.n[0] + 2 * g[0]) * (a.n[1] + 2 * g[1]) * (a.n[2] + 2 * g[2]);
  const unsigned n0 = (unsigned)a.n[0], n1 = (unsigned)a.n[1];
  for (size_t ci = (size_t)blockIdx.x * blockDim.x + threadIdx.x; ci < N; ci += (size_t)gridDim.x * blockDim.x) {
    // (N < 2^32 cells: the grid's own limit)
    const unsigned q = (unsigned)ci / n0;
    int c[3] = {(int)((unsigned)ci - q * n0), (int)(q % n1), (int)(q / n1)};
    if (!ghost_source(a.n, a.ndim, c)) continue;  // finished by the last direction's pass
    T U[NV], Ub[NV], Wb[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
      U[k] = a.U[k * N + ci];
      Ub[k] = T(0);
    }
    size_t pi = pad_index(a.n, a.ndim, c);
#pragma unroll
    for (int k = 0; k < NV; k++) Wb[k] = a.Wb[k * Npad + pi];
    cons_to_prim_vjp(U, Wb, Ub);
    for (int d = 0; d < a.ndim; d++) {
      const int nd = a.n[d];
      const int ghosts[4] = {-2, -1, nd, nd + 1};
      for (int gi = 0; gi < 4; gi++) {
        bool mir;
        const int src = map_index(ghosts[gi], nd, a.bc[2 * d], a.bc[2 * d + 1], mir);
        if (src != c[d]) continue;
        int q[3] = {c[0], c[1], c[2]};
        q[d] = ghosts[gi];
        const size_t qi = pad_index(a.n, a.ndim, q);
        const unsigned flip = mir ? flip_mask(d) : 0u;
        T Ug[NV], Ugb[NV], Wgb[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
          Ug[k] = ((flip >> k) & 1u) ? -U[k] : U[k];
          Ugb[k] = T(0);
          Wgb[k] = a.Wb[k * Npad + qi];
        }
        cons_to_prim_vjp(Ug, Wgb, Ugb);
#pragma unroll
        for (int k = 0; k < NV; k++) Ub[k] += ((flip >> k) & 1u) ? -Ugb[k] : Ugb[k];
      }
    }
    T ls[NV];
    lam_star(a, N, ci, ls);
#pragma unroll
    for (int k = 0; k < NV; k++) a.out[k * N + ci] = ls[k] + Ub[k];
  }
}

// dL/dW0 = (dU/dW)^T dL/dU0 at the primitive initial state W
template <typename T>
__global__ void adj_prim_kernel(const T *W, const T *Ub, T *Wb, size_t N) {
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    T w[NV], ub[NV], wb[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
      w[k] = W[k * N + c];
      ub[k] = Ub[k * N + c];
      wb[k] = T(0);
    }
    prim_to_cons_vjp(w, ub, wb);
#pragma unroll
    for (int k = 0; k < NV; k++) Wb[k * N + c] = wb[k];
  }
}

// control of the adjoint's forward steps: fixed dt and step tag
__global__ void adj_setup_kernel(Ctrl *c, int64_t step, double dt) {
  c->step = step;
  c->dt = dt;
  c->done = 0;
  for (int p = 0; p <= kFallbackPasses; p++) c->nbad[p] = 0;
}

__global__ void adj_record_kernel(const Ctrl *c, int32_t *had_tags, int64_t step) {
  had_tags[step] = c->nbad[0] > 0;
}

}  // namespace msh

// ======================================================================= host
using namespace msh;

namespace {

msh_status afail(msh_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_text(buf);
  return s;
}

#define A_TRY(expr)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      st = afail(e_ == cudaErrorMemoryAllocation ? MSH_E_NOMEM : MSH_E_CUDA, "%s: %s", #expr,   \
                 cudaGetErrorString(e_));                                                       \
      goto done;                                                                                \
    }                                                                                           \
  } while (0)

int grid_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// One forward step src -> dst with the fixed dt (no finalize: the schedule is given).  The
// fallback passes are launched only when `passes` is set, i.e. when the step is known (or
// not yet known) to tag cells; a step that tagged none recomputes identically without them.
template <typename T>
cudaError_t forward_step(msh_grid *g, Ctrl *ctl, Partial *part, T *src, T *dst, int64_t step, double dt,
                         bool passes) {
  adj_setup_kernel<<<1, 1, 0, g->stream>>>(ctl, step, dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  StepArgs<T> a;
  a.U[step & 1] = src;
  a.U[(step + 1) & 1] = dst;
  a.acc = (const T *)g->acc;
  a.ctrl = ctl;
  a.part = part;
  a.flags = g->flags;
  a.nx = (int)g->n[0];
  a.ny = (int)g->n[1];
  a.nz = (int)g->n[2];
  for (int i = 0; i < 6; i++) a.bc[i] = g->bc[i];
  for (int i = 0; i < 3; i++) a.dx[i] = g->dx[i];
  a.zchunk = g->zchunk;
  a.ck = nullptr;
  a.ck_base = 0;
  a.ck_len = 0;
  a.ck_K = 1;
  a.U1 = nullptr;
  for (int level = 0; level <= (passes ? kFallbackPasses : 0); level++) {
    a.level = level;
    e = launch_step<T>(a, g->ndim, g->rows, level > 0, g->stream, nullptr);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Reverse sweep over nsteps steps from the checkpoints ck (U^{mK}, device), the dt
// schedule and the per-step fallback flags (host).  lamN / lam0 are located per `where`;
// W0 (device, may be null) is the primitive initial state for kind == MSH_PRIMITIVE.
template <typename T>
msh_status reverse_sweep(msh_grid *g, const T *ck, int64_t nsteps, const double *dts, const int32_t *had, int K,
                         const void *lamN, void *lam0, int where, const T *W0) {
  msh_status st = MSH_OK;
  const size_t N = g->N;
  const size_t S = N * NV * sizeof(T);
  const cudaMemcpyKind in_kind = where == MSH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind out_kind = where == MSH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const int64_t nck = nsteps > 0 ? (nsteps + K - 1) / K : 0;
  const int64_t seg_len = std::min<int64_t>(K, std::max<int64_t>(nsteps, 1));
  size_t Npad = 1;
  for (int d = 0; d < 3; d++) Npad *= (size_t)(g->n[d] + (d < g->ndim ? 4 : 0));
  const int nb = std::max(step_blocks<T>(g->ndim, g->rows, (int)g->n[0], (int)g->n[1], (int)g->n[2], g->zchunk),
                          1);
  T *seg = nullptr, *la = nullptr, *lb = nullptr, *scratch = nullptr;
  T *Wb = nullptr;
  Ctrl *ctl = nullptr;
  Partial *part = nullptr;
  A_TRY(cudaMalloc(&seg, S * (size_t)seg_len));
  A_TRY(cudaMalloc(&la, S));
  A_TRY(cudaMalloc(&lb, S));
  A_TRY(cudaMalloc(&scratch, S));
  A_TRY(cudaMalloc(&Wb, Npad * NV * sizeof(T)));
  A_TRY(cudaMalloc(&ctl, sizeof(Ctrl)));
  A_TRY(cudaMalloc(&part, sizeof(Partial) * (size_t)nb));
  A_TRY(cudaMemcpyAsync(ctl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream));
  A_TRY(cudaMemcpyAsync(la, lamN, S, in_kind, g->stream));
  for (int64_t sg = nck - 1; sg >= 0; sg--) {
    const int64_t n0 = sg * K, n1 = std::min<int64_t>(n0 + K, nsteps);
    // recompute the segment's states U^{n0} .. U^{n1-1}
    A_TRY(cudaMemcpyAsync(seg, ck + (size_t)sg * N * NV, S, cudaMemcpyDeviceToDevice, g->stream));
    for (int64_t n = n0; n + 1 < n1; n++)
      A_TRY(forward_step<T>(g, ctl, part, seg + (size_t)(n - n0) * N * NV, seg + (size_t)(n - n0 + 1) * N * NV, n,
                            dts[n], had[n] != 0));
    for (int64_t n = n1 - 1; n >= n0; n--) {
      T *Un = seg + (size_t)(n - n0) * N * NV;
      // restore the fallback tags of step n (only a step that tagged cells has any)
      if (had[n]) A_TRY(forward_step<T>(g, ctl, part, Un, scratch, n, dts[n], true));
      AdjArgs<T> a;
      a.U = Un;
      a.lam = la;
      a.out = lb;
      a.acc = (const T *)g->acc;
      a.flags = g->flags;
      a.ctrl = ctl;
      a.tag = (int32_t)(n & 0x0fffffff) + 1;
      a.Wb = Wb;
      for (int i = 0; i < 3; i++) {
        a.n[i] = (int)g->n[i];
        a.dx[i] = g->dx[i];
      }
      a.ndim = g->ndim;
      for (int i = 0; i < 6; i++) a.bc[i] = g->bc[i];
      a.dt = dts[n];
      for (int d = 0; d < g->ndim; d++) {
        a.d = d;
        const long warps = (long)(N / g->n[d]) * ((g->n[d] + 4 + kAdjSeg - 1) / kAdjSeg);
        const int blocks = (int)std::min<long>((warps + 7) / 8, 1L << 20);
        if (d == 0) {
          if (g->ndim == 1) adj_pencil_kernel<T, 0, true><<<blocks, 256, 0, g->stream>>>(a);
          else adj_pencil_kernel<T, 0, false><<<blocks, 256, 0, g->stream>>>(a);
          A_TRY(cudaGetLastError());
        } else if (d == 1) {
          if (g->ndim == 2) A_TRY((launch_adj_tile<T, 1, true>(a, g->stream)));
          else A_TRY((launch_adj_tile<T, 1, false>(a, g->stream)));
        } else {
          A_TRY((launch_adj_tile<T, 2, true>(a, g->stream)));
        }
      }
      adj_fold_kernel<T><<<grid_blocks(N), 256, 0, g->stream>>>(a);
      A_TRY(cudaGetLastError());
      std::swap(la, lb);
    }
  }
  if (W0 != nullptr) {
    adj_prim_kernel<T><<<grid_blocks(N), 256, 0, g->stream>>>(W0, la, lb, N);
    A_TRY(cudaGetLastError());
    std::swap(la, lb);
  }
  A_TRY(cudaMemcpyAsync(lam0, la, S, out_kind, g->stream));
  A_TRY(cudaStreamSynchronize(g->stream));
done:
  cudaStreamSynchronize(g->stream);
  for (void *p : {(void *)seg, (void *)la, (void *)lb, (void *)scratch, (void *)Wb, (void *)ctl, (void *)part})
    if (p) cudaFree(p);
  return st;
}

// msh_adjoint_run: forward sweep from U0 storing checkpoints and fallback flags, then the
// reverse sweep.
template <typename T>
msh_status adjoint_impl(msh_grid *g, const void *U0, int64_t nsteps, const double *dts, int K, const void *lamN,
                        void *lam0, int where, int kind) {
  msh_status st = MSH_OK;
  const size_t N = g->N;
  const size_t S = N * NV * sizeof(T);
  const cudaMemcpyKind in_kind = where == MSH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const int64_t nck = nsteps > 0 ? (nsteps + K - 1) / K : 1;
  const int nb = std::max(step_blocks<T>(g->ndim, g->rows, (int)g->n[0], (int)g->n[1], (int)g->n[2], g->zchunk),
                          1);
  T *ck = nullptr, *bufA = nullptr, *bufB = nullptr, *W0 = nullptr;
  Ctrl *ctl = nullptr;
  Partial *part = nullptr;
  int32_t *had = nullptr;
  std::vector<int32_t> had_h((size_t)std::max<int64_t>(nsteps, 1), 0);
  A_TRY(cudaMalloc(&ck, S * nck));
  A_TRY(cudaMalloc(&bufA, S));
  A_TRY(cudaMalloc(&bufB, S));
  A_TRY(cudaMalloc(&ctl, sizeof(Ctrl)));
  A_TRY(cudaMalloc(&part, sizeof(Partial) * (size_t)nb));
  A_TRY(cudaMalloc(&had, sizeof(int32_t) * had_h.size()));
  A_TRY(cudaMemcpyAsync(ctl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream));
  // fallback tags are step numbers: start from a clean slate (and leave one behind)
  A_TRY(cudaMemsetAsync(g->flags, 0, N * sizeof(int32_t), g->stream));
  A_TRY(cudaMemcpyAsync(ck, U0, S, in_kind, g->stream));
  if (kind == MSH_PRIMITIVE) {
    A_TRY(cudaMalloc(&W0, S));
    A_TRY(cudaMemcpyAsync(W0, ck, S, cudaMemcpyDeviceToDevice, g->stream));
    A_TRY(launch_convert<T>(ck, N, 0, g->stream));
  }
  {
    const T *cur = ck;
    for (int64_t s = 0; s < nsteps; s++) {
      T *dst = (s & 1) ? bufB : bufA;
      A_TRY(forward_step<T>(g, ctl, part, const_cast<T *>(cur), dst, s, dts[s], true));
      adj_record_kernel<<<1, 1, 0, g->stream>>>(ctl, had, s);
      A_TRY(cudaGetLastError());
      cur = dst;
      if ((s + 1) % K == 0 && s + 1 < nsteps)
        A_TRY(cudaMemcpyAsync(ck + (size_t)((s + 1) / K) * N * NV, cur, S, cudaMemcpyDeviceToDevice, g->stream));
    }
  }
  if (nsteps > 0)
    A_TRY(cudaMemcpyAsync(had_h.data(), had, sizeof(int32_t) * (size_t)nsteps, cudaMemcpyDeviceToHost, g->stream));
  A_TRY(cudaStreamSynchronize(g->stream));
  cudaFree(bufA);
  cudaFree(bufB);
  bufA = bufB = nullptr;
  st = reverse_sweep<T>(g, ck, nsteps, dts, had_h.data(), K, lamN, lam0, where, W0);
done:
  cudaMemsetAsync(g->flags, 0, N * sizeof(int32_t), g->stream);
  cudaStreamSynchronize(g->stream);
  for (void *p : {(void *)ck, (void *)bufA, (void *)bufB, (void *)W0, (void *)ctl, (void *)part, (void *)had})
    if (p) cudaFree(p);
  return st;
}

// msh_adjoint_tape: the checkpoints, dt schedule and fallback flags of the recorded run.
template <typename T>
msh_status adjoint_tape_impl(msh_grid *g, const void *lamN, void *lam0, int where, int kind) {
  msh_status st = MSH_OK;
  const size_t N = g->N;
  const size_t S = N * NV * sizeof(T);
  const int64_t nsteps = g->hctrl->step - g->tape_base;
  std::vector<double> dts((size_t)std::max<int64_t>(nsteps, 1));
  std::vector<int32_t> had((size_t)std::max<int64_t>(nsteps, 1), 0);
  T *W0 = nullptr;
  if (nsteps > 0) {
    A_TRY(cudaMemcpyAsync(dts.data(), g->tape_dt, sizeof(double) * (size_t)nsteps, cudaMemcpyDeviceToHost, g->stream));
    A_TRY(cudaMemcpyAsync(had.data(), g->tape_had, sizeof(int32_t) * (size_t)nsteps, cudaMemcpyDeviceToHost,
                          g->stream));
  }
  if (kind == MSH_PRIMITIVE) {
    A_TRY(cudaMalloc(&W0, S));
    A_TRY(cudaMemcpyAsync(W0, g->tape, S, cudaMemcpyDeviceToDevice, g->stream));
    A_TRY(launch_convert<T>(W0, N, 1, g->stream));
  }
  A_TRY(cudaStreamSynchronize(g->stream));
  st = reverse_sweep<T>(g, (const T *)g->tape, nsteps, dts.data(), had.data(), g->tape_K, lamN, lam0, where, W0);
done:
  cudaStreamSynchronize(g->stream);
  if (W0) cudaFree(W0);
  return st;
}

}  // namespace

extern "C" msh_status msh_adjoint_run(msh_grid *g, const void *U0, int64_t nsteps, const double *dt_sched, int32_t K,
                                      const void *dL_dUN, void *dL_dU0, int32_t where, int32_t kind) {
  msh::NvtxRange nvtx_range("msh_adjoint_run");
  clear_error();
  if (!g || !U0 || !dL_dUN || !dL_dU0) return afail(MSH_E_INVALID_ARG, "null argument");
  if (nsteps < 0 || (nsteps > 0 && !dt_sched)) return afail(MSH_E_INVALID_ARG, "bad nsteps or dt schedule");
  if (K < 1) return afail(MSH_E_INVALID_ARG, "checkpoint interval K must be >= 1");
  if (where != MSH_HOST && where != MSH_DEVICE) return afail(MSH_E_INVALID_ARG, "bad where");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return afail(MSH_E_INVALID_ARG, "bad kind");
  for (int64_t s = 0; s < nsteps; s++)
    if (!(dt_sched[s] > 0.0) || !std::isfinite(dt_sched[s]))
      return afail(MSH_E_INVALID_ARG, "dt_sched[%lld] must be finite and > 0", (long long)s);
  if (g->scheme != MSH_SCHEME_MUSCL_HANCOCK) return afail(MSH_E_STATE, "the adjoint covers the MUSCL-Hancock scheme only");
  if (g->ctu && g->ndim > 1)
    return afail(MSH_E_STATE, "the adjoint covers the step without transverse (CTU) terms only");
  if (g->sg_G > 0.0) return afail(MSH_E_STATE, "the adjoint covers external potentials only");
  if (g->prec == MSH_FP32)
    return adjoint_impl<float>(g, U0, nsteps, dt_sched, K, dL_dUN, dL_dU0, where, kind);
  return adjoint_impl<double>(g, U0, nsteps, dt_sched, K, dL_dUN, dL_dU0, where, kind);
}

extern "C" msh_status msh_adjoint_tape(msh_grid *g, const void *dL_dUN, void *dL_dU0, int32_t where, int32_t kind) {
  msh::NvtxRange nvtx_range("msh_adjoint_tape");
  clear_error();
  if (!g || !dL_dUN || !dL_dU0) return afail(MSH_E_INVALID_ARG, "null argument");
  if (where != MSH_HOST && where != MSH_DEVICE) return afail(MSH_E_INVALID_ARG, "bad where");
  if (kind != MSH_CONSERVED && kind != MSH_PRIMITIVE) return afail(MSH_E_INVALID_ARG, "bad kind");
  if (!g->tape_valid) return afail(MSH_E_STATE, "no adjoint tape is being recorded (msh_set_tape)");
  const int64_t nsteps = g->hctrl->step - g->tape_base;
  if (nsteps < 0 || nsteps > g->tape_len)
    return afail(MSH_E_STATE, "the run took %lld steps since msh_set_tape, the tape holds %lld", (long long)nsteps,
                 (long long)g->tape_len);
  if (g->prec == MSH_FP32) return adjoint_tape_impl<float>(g, dL_dUN, dL_dU0, where, kind);
  return adjoint_tape_impl<double>(g, dL_dUN, dL_dU0, where, kind);
}
