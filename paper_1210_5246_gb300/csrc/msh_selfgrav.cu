// msh_selfgrav.cu -- periodic self-gravity (msh_set_self_gravity).
//
// Before every step: the density of U^n goes through a real-to-complex FFT (cuFFT), each
// mode is scaled by -4 pi G / k_eff^2 with k_eff^2 = sum_d (2 sin(pi k_d / n_d) / dx_d)^2,
// the eigenvalues of the 3-point discrete Laplacian (the mean, k = 0, is dropped), and the
// inverse FFT gives the potential.  a^n = -grad Phi^n by central differences; the
// acceleration the step's gravity source uses is interpolated forward from the previous
// step's (Sec. 3.3, last paragraph):
//   a^{n+1/2} = a^n + (dt_n / (2 dt_{n-1})) (a^n - a^{n-1})   (a^n on the first step),
// plus -grad of the external potential when there is one.  Every kernel reads the step's
// buffer parity and dt from the device control block, so the sequence is captured in the
// run's CUDA graphs like the step itself.
#include <cufft.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/msh.h"
#include "msh_internal.h"

namespace msh {
namespace {

template <typename T> struct Fft;
template <> struct Fft<float> {
  using C = cufftComplex;
  static cufftResult fwd(cufftHandle p, float *in, C *out) { return cufftExecR2C(p, in, out); }
  static cufftResult inv(cufftHandle p, C *in, float *out) { return cufftExecC2R(p, in, out); }
};
template <> struct Fft<double> {
  using C = cufftDoubleComplex;
  static cufftResult fwd(cufftHandle p, double *in, C *out) { return cufftExecD2Z(p, in, out); }
  static cufftResult inv(cufftHandle p, C *in, double *out) { return cufftExecZ2D(p, in, out); }
};

// density of U^n (field 0 of the buffer the step reads) into the FFT input
template <typename T>
__global__ void sg_density_kernel(const Ctrl *ctrl, T *const *U, T *rho, size_t N) {
  if (ctrl->done) return;
  const T *src = U[ctrl->step & 1];
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x)
    rho[c] = src[c];
}

// Phi_k = -4 pi G rho_k / k_eff^2 / N on the half spectrum [nz][ny][nx/2+1]; eig holds the
// per-axis Laplacian eigenvalues (2 sin(pi k / n) / dx)^2, x then y then z (built on the
// host once), c = -4 pi G / N.
template <typename T, typename C>
__global__ void sg_scale_kernel(const Ctrl *ctrl, C *hat, const T *__restrict__ eig, int nx, int ny, int nz, T c) {
  if (ctrl->done) return;
  const int hx = nx / 2 + 1;
  const size_t M = (size_t)hx * ny * nz;
  const T *ex = eig, *ey = eig + hx, *ez = eig + hx + ny;
  for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(m % hx), ky = (int)((m / hx) % ny), kz = (int)(m / ((size_t)hx * ny));
    const T k2 = ex[kx] + ey[ky] + ez[kz];
    const T f = k2 > T(0) ? c / k2 : T(0);
    hat[m].x *= f;
    hat[m].y *= f;
  }
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// a^n = -grad Phi (central, periodic); the step's acceleration is a^n interpolated forward
// with the previous step's a^{n-1} (kept in prev), plus the external field if any.
template <typename T>
__global__ void sg_accel_kernel(const Ctrl *ctrl, const T *phi, T *prev, T *use, const T *ext, int ndim, int nx,
                                int ny, int nz, double dx0, double dx1, double dx2) {
  if (ctrl->done) return;
  const size_t N = (size_t)nx * ny * nz;
  const double hist = ctrl->sg_hist ? ctrl->dt / (2.0 * ctrl->dt_last) : 0.0;
  const T w = (T)hist;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
    T a[3] = {T(0), T(0), T(0)};
    a[0] = -(phi[((size_t)z * ny + y) * nx + wrap(x + 1, nx)] - phi[((size_t)z * ny + y) * nx + wrap(x - 1, nx)]) /
           (T)(2.0 * dx0);
    if (ndim > 1)
      a[1] = -(phi[((size_t)z * ny + wrap(y + 1, ny)) * nx + x] - phi[((size_t)z * ny + wrap(y - 1, ny)) * nx + x]) /
             (T)(2.0 * dx1);
    if (ndim > 2)
      a[2] = -(phi[((size_t)wrap(z + 1, nz) * ny + y) * nx + x] - phi[((size_t)wrap(z - 1, nz) * ny + y) * nx + x]) /
             (T)(2.0 * dx2);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const T an = a[d];
      T v = an + w * (an - prev[d * N + c]);
      if (ext) v += ext[d * N + c];
      use[d * N + c] = v;
      prev[d * N + c] = an;
    }
  }
}

__global__ void sg_mark_kernel(Ctrl *ctrl) {
  if (!ctrl->done) ctrl->sg_hist = 1;
}

int sg_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 2048 ? (b > 0 ? b : 1) : 2048);
}

template <typename T> cudaError_t sg_launch_impl(msh_grid *g, cudaStream_t s) {
  const size_t N = g->N;
  const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
  using C = typename Fft<T>::C;
  sg_density_kernel<T><<<sg_blocks(N), 256, 0, s>>>(g->ctrl, (T *const *)g->sg_bufs, (T *)g->sg_rho, N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (Fft<T>::fwd((cufftHandle)g->sg_plan_fwd, (T *)g->sg_rho, (C *)g->sg_hat) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  const size_t M = (size_t)(nx / 2 + 1) * ny * nz;
  const T c = (T)(-4.0 * M_PI * g->sg_G / ((double)nx * ny * nz));
  sg_scale_kernel<T, C><<<sg_blocks(M), 256, 0, s>>>(g->ctrl, (C *)g->sg_hat, (const T *)g->sg_eig, nx, ny, nz, c);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (Fft<T>::inv((cufftHandle)g->sg_plan_inv, (C *)g->sg_hat, (T *)g->sg_phi) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  sg_accel_kernel<T><<<sg_blocks(N), 256, 0, s>>>(g->ctrl, (const T *)g->sg_phi, (T *)g->sg_prev, (T *)g->sg_use,
                                                  (const T *)g->acc, g->ndim, nx, ny, nz, g->dx[0], g->dx[1], g->dx[2]);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_self_gravity(msh_grid *g, cudaStream_t s) {
  return g->prec == MSH_FP32 ? sg_launch_impl<float>(g, s) : sg_launch_impl<double>(g, s);
}

cudaError_t launch_self_gravity_mark(msh_grid *g, cudaStream_t s) {
  sg_mark_kernel<<<1, 1, 0, s>>>(g->ctrl);
  return cudaGetLastError();
}

void free_self_gravity(msh_grid *g) {
  if (g->sg_plan_fwd) cufftDestroy((cufftHandle)g->sg_plan_fwd);
  if (g->sg_plan_inv) cufftDestroy((cufftHandle)g->sg_plan_inv);
  for (void *p : {g->sg_rho, g->sg_hat, g->sg_phi, g->sg_prev, g->sg_use, g->sg_eig, (void *)g->sg_bufs})
    if (p) cudaFree(p);
  g->sg_plan_fwd = g->sg_plan_inv = 0;
  g->sg_rho = g->sg_hat = g->sg_phi = g->sg_prev = g->sg_use = g->sg_eig = nullptr;
  g->sg_bufs = nullptr;
  g->sg_G = 0.0;
}

// Plans and buffers for the grid's shape and precision.
msh_status setup_self_gravity(msh_grid *g, double G) {
  free_self_gravity(g);
  const size_t N = g->N, es = g->esize;
  const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
  const size_t M = (size_t)(nx / 2 + 1) * ny * nz;
  const bool f32 = g->prec == MSH_FP32;
  cufftHandle pf = 0, pi = 0;
  cufftResult r;
  const cufftType tf = f32 ? CUFFT_R2C : CUFFT_D2Z, ti = f32 ? CUFFT_C2R : CUFFT_Z2D;
  if (g->ndim == 1) {
    r = cufftPlan1d(&pf, nx, tf, 1);
    if (r == CUFFT_SUCCESS) r = cufftPlan1d(&pi, nx, ti, 1);
  } else if (g->ndim == 2) {
    r = cufftPlan2d(&pf, ny, nx, tf);
    if (r == CUFFT_SUCCESS) r = cufftPlan2d(&pi, ny, nx, ti);
  } else {
    r = cufftPlan3d(&pf, nz, ny, nx, tf);
    if (r == CUFFT_SUCCESS) r = cufftPlan3d(&pi, nz, ny, nx, ti);
  }
  g->sg_plan_fwd = pf;
  g->sg_plan_inv = pi;
  if (r == CUFFT_SUCCESS) r = cufftSetStream(pf, g->stream);
  if (r == CUFFT_SUCCESS) r = cufftSetStream(pi, g->stream);
  if (r != CUFFT_SUCCESS) {
    free_self_gravity(g);
    set_error_text("cuFFT plan creation failed");
    return MSH_E_CUDA;
  }
  cudaError_t e = cudaMalloc(&g->sg_rho, N * es);
  if (e == cudaSuccess) e = cudaMalloc(&g->sg_hat, M * 2 * es);
  if (e == cudaSuccess) e = cudaMalloc(&g->sg_phi, N * es);
  if (e == cudaSuccess) e = cudaMalloc(&g->sg_prev, 3 * N * es);
  if (e == cudaSuccess) e = cudaMalloc(&g->sg_use, 3 * N * es);
  if (e == cudaSuccess) e = cudaMalloc(&g->sg_bufs, 2 * sizeof(void *));
  if (e == cudaSuccess) e = cudaMemcpy(g->sg_bufs, g->U, 2 * sizeof(void *), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->sg_prev, 0, 3 * N * es);
  // per-axis eigenvalues of the 3-point Laplacian, (2 sin(pi k / n) / dx)^2 (0 on inactive
  // axes), x for k = 0 .. nx/2 (the half spectrum), then y, then z
  if (e == cudaSuccess) {
    const int hx = nx / 2 + 1;
    std::vector<double> eig((size_t)hx + ny + nz, 0.0);
    auto fill = [&](double *out, int count, int n, int d) {
      for (int k = 0; k < count; k++) {
        const double sv = d < g->ndim ? 2.0 * std::sin(M_PI * k / n) / g->dx[d] : 0.0;
        out[k] = sv * sv;
      }
    };
    fill(eig.data(), hx, nx, 0);
    fill(eig.data() + hx, ny, ny, 1);
    fill(eig.data() + hx + ny, nz, nz, 2);
    e = cudaMalloc(&g->sg_eig, eig.size() * es);
    if (e == cudaSuccess) {
      if (f32) {
        std::vector<float> ef(eig.begin(), eig.end());
        e = cudaMemcpy(g->sg_eig, ef.data(), ef.size() * sizeof(float), cudaMemcpyHostToDevice);
      } else {
        e = cudaMemcpy(g->sg_eig, eig.data(), eig.size() * sizeof(double), cudaMemcpyHostToDevice);
      }
    }
  }
  if (e != cudaSuccess) {
    free_self_gravity(g);
    set_error_text(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MSH_E_NOMEM : MSH_E_CUDA;
  }
  g->sg_G = G;
  return MSH_OK;
}

}  // namespace msh
