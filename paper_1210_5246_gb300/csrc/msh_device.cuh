// msh_device.cuh -- per-cell and per-face device arithmetic of the BME Godunov step.
//
// Everything here works on one 10-vector in registers.  The reconstruction and the flux
// are written in the "local frame" of a sweep direction: the normal axis is moved to
// the x slot, the two transverse axes keep their natural order.  In that frame the
// eigen-system is the ten-variable extension of the paper's x-direction system
// (Sec. 3.3, eqs jacobian, eigenvalues, righteigvec, lefteigvec):
//   eigenvalues  u -+ cf, u -+ cs (twice each), u (four contact waves),
//   cf = sqrt(3 P_xx / rho), cs = sqrt(P_xx / rho),
// and the projections below are its closed-form sparse left/right eigenvectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msh {

constexpr int NV = 10;

// Primitive/conserved component that sits at local slot k for sweep direction D.
// D = 0: (rho, u, v, w, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz)
// D = 1: normal y, transverse (x, z);  D = 2: normal z, transverse (x, y).
template <int D> struct Frame;
template <> struct Frame<0> {
  static __device__ __forceinline__ constexpr int g(int k) { return k; }
};
template <> struct Frame<1> {
  static __device__ __forceinline__ constexpr int g(int k) {
    return k == 1 ? 2 : k == 2 ? 1 : k == 4 ? 7 : k == 6 ? 8 : k == 7 ? 4 : k == 8 ? 6 : k;
  }
};
template <> struct Frame<2> {
  static __device__ __forceinline__ constexpr int g(int k) {
    return k == 1 ? 3 : k == 2 ? 1 : k == 3 ? 2 : k == 4 ? 9 : k == 5 ? 6 : k == 6 ? 8
         : k == 7 ? 4 : k == 8 ? 5 : k == 9 ? 7 : k;
  }
};

// ---------------------------------------------------------- fast arithmetic
// FP32: hardware approximate reciprocal and reciprocal square root (a few ulp, far
// inside the FP32 tolerances); FP64: IEEE division and square root.
template <typename T> __device__ __forceinline__ T frcp(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float frcp<float>(float x) { return __fdividef(1.0f, x); }
template <typename T> __device__ __forceinline__ T frsqrt(T x) { return T(1) / sqrt(x); }
template <> __device__ __forceinline__ float frsqrt<float>(float x) { return rsqrtf(x); }
// sqrt(p / r) for p, r > 0
template <typename T> __device__ __forceinline__ T sqrt_ratio(T p, T r) { return sqrt(p / r); }
template <> __device__ __forceinline__ float sqrt_ratio<float>(float p, float r) { return p * rsqrtf(p * r); }

// ------------------------------------------------------- paired FP32 arithmetic
// Componentwise operations on 10-vectors, d_k = a_k s + c_k (v_fma), d_k = a_k s (v_mul),
// d_k = a_k + b_k (v_add) and d_k = a_k - b_k (v_sub).  In FP32 components (k, k+1) go through the packed f32x2 instructions of sm_100
// (__ffma2_rn, __fadd2_rn: two single-precision operations per issued instruction, each
// rounded as its scalar form); FP64 stays scalar.
template <typename T>
__device__ __forceinline__ void v_fma(T (&d)[NV], const T (&a)[NV], T s, const T (&c)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = fma(a[k], s, c[k]);
}
template <>
__device__ __forceinline__ void v_fma<float>(float (&d)[NV], const float (&a)[NV], float s, const float (&c)[NV]) {
  const float2 ss = make_float2(s, s);
#pragma unroll
  for (int k = 0; k < NV; k += 2) {
    const float2 r = __ffma2_rn(make_float2(a[k], a[k + 1]), ss, make_float2(c[k], c[k + 1]));
    d[k] = r.x;
    d[k + 1] = r.y;
  }
}
template <typename T> __device__ __forceinline__ void v_mul(T (&d)[NV], const T (&a)[NV], T s) {
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = a[k] * s;
}
template <> __device__ __forceinline__ void v_mul<float>(float (&d)[NV], const float (&a)[NV], float s) {
  const float2 ss = make_float2(s, s);
#pragma unroll
  for (int k = 0; k < NV; k += 2) {
    const float2 r = __fmul2_rn(make_float2(a[k], a[k + 1]), ss);
    d[k] = r.x;
    d[k + 1] = r.y;
  }
}
template <typename T> __device__ __forceinline__ void v_add(T (&d)[NV], const T (&a)[NV], const T (&b)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = a[k] + b[k];
}
template <>
__device__ __forceinline__ void v_add<float>(float (&d)[NV], const float (&a)[NV], const float (&b)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k += 2) {
    const float2 r = __fadd2_rn(make_float2(a[k], a[k + 1]), make_float2(b[k], b[k + 1]));
    d[k] = r.x;
    d[k + 1] = r.y;
  }
}
template <typename T> __device__ __forceinline__ void v_sub(T (&d)[NV], const T (&a)[NV], const T (&b)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = a[k] - b[k];
}
template <>
__device__ __forceinline__ void v_sub<float>(float (&d)[NV], const float (&a)[NV], const float (&b)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k += 2) {
    const float2 r = __fadd2_rn(make_float2(a[k], a[k + 1]), make_float2(-b[k], -b[k + 1]));
    d[k] = r.x;
    d[k + 1] = r.y;
  }
}

// ---------------------------------------------------------------- conversions
// E_ij = P_ij + rho u_i u_j (Sec. 2).  The FP32 path recomputes a diagonal dispersion
// in FP64 when the kinetic part cancels more than 99.9 % of E_ii, i.e. where P_ii/rho
// approaches realizability loss.
template <typename T> __device__ __forceinline__ T diag_fix(T P, T E, T m, T rho) { return P; }
template <> __device__ __forceinline__ float diag_fix<float>(float P, float E, float m, float rho) {
  if (P < 1.0e-3f * E) {
    double r = (double)E - (double)m * (double)m / (double)rho;
    return (float)r;
  }
  return P;
}

template <typename T>
__device__ __forceinline__ void cons_to_prim(const T (&U)[NV], T (&W)[NV]) {
  const T rho = U[0];
  const T ir = frcp(rho);
  const T u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
  W[4] = diag_fix<T>(U[4] - U[1] * u, U[4], U[1], rho);
  W[5] = U[5] - U[1] * v;
  W[6] = U[6] - U[1] * w;
  W[7] = diag_fix<T>(U[7] - U[2] * v, U[7], U[2], rho);
  W[8] = U[8] - U[2] * w;
  W[9] = diag_fix<T>(U[9] - U[3] * w, U[9], U[3], rho);
}

template <typename T>
__device__ __forceinline__ void prim_to_cons(const T (&W)[NV], T (&U)[NV]) {
  const T rho = W[0];
  const T mx = rho * W[1], my = rho * W[2], mz = rho * W[3];
  U[0] = rho; U[1] = mx; U[2] = my; U[3] = mz;
  U[4] = W[4] + mx * W[1];
  U[5] = W[5] + mx * W[2];
  U[6] = W[6] + mx * W[3];
  U[7] = W[7] + my * W[2];
  U[8] = W[8] + my * W[3];
  U[9] = W[9] + mz * W[3];
}

// rho > 0 and P positive definite by its leading principal minors.
template <typename T> __device__ __forceinline__ bool realizable(const T (&W)[NV]) {
  const T m1 = W[4];
  const T m2 = W[4] * W[7] - W[5] * W[5];
  const T m3 = W[4] * (W[7] * W[9] - W[8] * W[8]) - W[5] * (W[5] * W[9] - W[8] * W[6]) +
               W[6] * (W[5] * W[8] - W[7] * W[6]);
  return W[0] > T(0) && m1 > T(0) && m2 > T(0) && m3 > T(0);
}

// ----------------------------------------------------------- reconstruction
// MC limiter on one characteristic amplitude, dC = (dL + dR)/2 by linearity of L.
template <typename T> __device__ __forceinline__ T mc_limit(T dl, T dr) {
  const T dc = T(0.5) * (dl + dr);
  const T m = fmin(fmin(T(2) * fabs(dl), fabs(dc)), T(2) * fabs(dr));
  return (dl * dr > T(0)) ? copysign(m, dc) : T(0);
}

// The same limiter doubled: 2 mc(dL, dR) = sign(dL) min(4|dL|, 4|dR|, |dL + dR|) for
// same-sign differences, else 0.  Scaling by powers of two is exact, so this is exactly
// twice mc_limit (two instructions cheaper).
template <typename T> __device__ __forceinline__ T mc_limit2(T dl, T dr) {
  const T m = fmin(T(4) * fmin(fabs(dl), fabs(dr)), fabs(dl + dr));
  return (dl * dr > T(0)) ? copysign(m, dl) : T(0);
}

// The doubled limiter on every amplitude of a 10-vector (FP32: the sum, the product and the
// factor 4 in packed f32x2 instructions; the same values as mc_limit2).
template <typename T> __device__ __forceinline__ void mc_limit2_v(const T (&dl)[NV], const T (&dr)[NV], T (&m)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) m[k] = mc_limit2(dl[k], dr[k]);
}
template <>
__device__ __forceinline__ void mc_limit2_v<float>(const float (&dl)[NV], const float (&dr)[NV], float (&m)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k += 2) {
    const float2 a = make_float2(dl[k], dl[k + 1]), b = make_float2(dr[k], dr[k + 1]);
    const float2 sum = __fadd2_rn(a, b), prod = __fmul2_rn(a, b);
    const float2 q = __fmul2_rn(make_float2(4.0f, 4.0f), make_float2(fminf(fabsf(a.x), fabsf(b.x)),
                                                                        fminf(fabsf(a.y), fabsf(b.y))));
    const float m0 = fminf(q.x, fabsf(sum.x)), m1 = fminf(q.y, fabsf(sum.y));
    m[k] = prod.x > 0.0f ? copysignf(m0, a.x) : 0.0f;
    m[k + 1] = prod.y > 0.0f ? copysignf(m1, a.y) : 0.0f;
  }
}

// Eigen-quantities of the local-frame state w0 shared by projection and back-projection.
template <typename T> struct Eig {
  T rho, u, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz;
  T cf, cs, a, b, ip, icf2, ics2;
  __device__ __forceinline__ void init(const T (&w)[NV]) {
    rho = w[0]; u = w[1];
    Pxx = w[4]; Pxy = w[5]; Pxz = w[6]; Pyy = w[7]; Pyz = w[8]; Pzz = w[9];
    ip = frcp(Pxx);
    const T s = frsqrt(Pxx * rho);       // 1 / sqrt(P_xx rho)
    cs = Pxx * s;                        // sqrt(P_xx / rho)
    const T rs = rho * s;                // 1 / cs
    cf = T(1.7320508075688772) * cs;
    a = Pxy * ip;
    b = Pxz * ip;
    icf2 = T(0.28867513459481287) * rs;  // 1 / (2 cf)
    ics2 = T(0.5) * rs;                  // 1 / (2 cs)
  }
  // characteristic amplitudes c = L d in wave order
  // (f-, sv-, sw-, c_rho, c_yy, c_yz, c_zz, sv+, sw+, f+)
  __device__ __forceinline__ void project(const T (&d)[NV], T (&c)[NV]) const {
    const T e = d[4] * ip * T(1.0 / 3.0);
    const T t1 = d[1] * icf2, t2 = T(0.5) * e;
    c[0] = t2 - t1;
    c[9] = t2 + t1;
    const T qv = (d[2] - a * d[1]) * ics2, rv = T(0.5) * (d[5] - a * d[4]) * ip;
    c[1] = rv - qv;
    c[7] = rv + qv;
    const T qw = (d[3] - b * d[1]) * ics2, rw = T(0.5) * (d[6] - b * d[4]) * ip;
    c[2] = rw - qw;
    c[8] = rw + qw;
    c[3] = d[0] - rho * e;
    c[4] = d[7] - T(2) * a * d[5] + (T(4) * a * Pxy - Pyy) * e;
    c[5] = d[8] - b * d[5] - a * d[6] + (T(4) * a * Pxz - Pyz) * e;
    c[6] = d[9] - T(2) * b * d[6] + (T(4) * b * Pxz - Pzz) * e;
  }
  // primitive vector R c
  __device__ __forceinline__ void back(const T (&c)[NV], T (&o)[NV]) const {
    const T A = c[9] + c[0], B = (c[9] - c[0]) * cf;
    const T C = c[7] + c[1], Dv = (c[7] - c[1]) * cs;
    const T E = c[8] + c[2], Fw = (c[8] - c[2]) * cs;
    o[0] = rho * A + c[3];
    o[1] = B;
    o[2] = a * B + Dv;
    o[3] = b * B + Fw;
    o[4] = T(3) * Pxx * A;
    o[5] = T(3) * Pxy * A + Pxx * C;
    o[6] = T(3) * Pxz * A + Pxx * E;
    o[7] = (Pyy + T(2) * a * Pxy) * A + T(2) * Pxy * C + c[4];
    o[8] = (Pyz + T(2) * a * Pxz) * A + Pxz * C + Pxy * E + c[5];
    o[9] = (Pzz + T(2) * b * Pxz) * A + T(2) * Pxz * E + c[6];
  }
  // R c and R (s c), s the wave speeds relative to u (-cf, -cs, -cs, 0 x 4, cs, cs, cf),
  // sharing the wave-pair sums: with A = c_f+ + c_f-, B = (c_f+ - c_f-) cf and so on, the
  // speed-weighted amplitudes give A' = B, B' = cf^2 A (cf^2 = 3 cs^2), C' = Dv, Dv' = cs^2 C,
  // E' = Fw, Fw' = cs^2 E, and no contact amplitudes.
  __device__ __forceinline__ void back2(const T (&c)[NV], T (&o)[NV], T (&os)[NV]) const {
    back(c, o);
    const T A = c[9] + c[0], C = c[7] + c[1], E = c[8] + c[2];
    const T A2 = (c[9] - c[0]) * cf, C2 = (c[7] - c[1]) * cs, E2 = (c[8] - c[2]) * cs;
    const T cs2 = cs * cs;
    const T B2 = T(3) * cs2 * A, D2 = cs2 * C, F2 = cs2 * E;
    os[0] = rho * A2;
    os[1] = B2;
    os[2] = a * B2 + D2;
    os[3] = b * B2 + F2;
    os[4] = T(3) * Pxx * A2;
    os[5] = T(3) * Pxy * A2 + Pxx * C2;
    os[6] = T(3) * Pxz * A2 + Pxx * E2;
    os[7] = (Pyy + T(2) * a * Pxy) * A2 + T(2) * Pxy * C2;
    os[8] = (Pyz + T(2) * a * Pxz) * A2 + Pxz * C2 + Pxy * E2;
    os[9] = (Pzz + T(2) * b * Pxz) * A2 + T(2) * Pxz * E2;
  }
};

// ------------------------------------------------- corner transport upwind
// Transverse term of a cell along direction t for the corner-transport-upwind form of the
// unsplit step (the data reconstruction of Lee & Deane 2009, on which FLASH's unsplit
// MUSCL-Hancock solver of Sec. 3.3 is built; the paper prints none of it): the
// quasi-linear transverse derivative -(dt/2) A_t dW/dx_t taken wave by wave from the
// upwind side,
//   T_t = -nu sum_a lam^a (L^a . dW^a) R^a,   dW^a = w0 - wm if lam^a > 0, else wp - w0,
// nu = dt / (2 dx_t), with the eigen-system of the cell along t (local frame of t).  The
// face states along d take sum_{t != d} T_t before the face-state check.
// cl, cr: the amplitudes L (w0 - wm) and L (wp - w0).
template <typename T>
__device__ __forceinline__ void upwind_terms(const Eig<T> &E, const T (&cl)[NV], const T (&cr)[NV], T nu,
                                             T (&o)[NV]) {
  const T s[NV] = {-E.cf, -E.cs, -E.cs, T(0), T(0), T(0), T(0), E.cs, E.cs, E.cf};
  T c[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T lam = E.u + s[k];
    c[k] = -nu * lam * (lam > T(0) ? cl[k] : cr[k]);
  }
  E.back(c, o);
}

template <typename T>
__device__ __forceinline__ void transverse(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu,
                                           T (&o)[NV]) {
  Eig<T> E;
  E.init(w0);
  T d[NV], cl[NV], cr[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = w0[k] - wm[k];
  E.project(d, cl);
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = wp[k] - w0[k];
  E.project(d, cr);
  upwind_terms(E, cl, cr, nu, o);
}

// Face-state check: if a face state has rho <= 0 or P_nn <= 0 both revert to w0 (first
// order).
template <typename T>
__device__ __forceinline__ void face_state_check(const T (&w0)[NV], T (&lo)[NV], T (&hi)[NV]) {
  const bool ok = hi[0] > T(0) && lo[0] > T(0) && hi[4] > T(0) && lo[4] > T(0);
  if (!ok) {
#pragma unroll
    for (int k = 0; k < NV; k++) { hi[k] = w0[k]; lo[k] = w0[k]; }
  }
}

// Reconstruction of one cell along the sweep direction, in the local frame.
//   wm, w0, wp   primitive states of cells i-1, i, i+1
//   nu           dt / (2 dx)
// Output: face states lo (at i-1/2) and hi (at i+1/2):
//   dw^m = R mc(L dw_L, L dw_R);   w0 -+ dw^m/2 - nu A dw^m,   A dw^m = R Lambda mc(...)
// CTU: both face states also take X (the other directions' transverse terms, local frame;
// xget(k) returns X_k) and the cell's own transverse term along this direction is handed to
// tput(k, T_k) (upwind_terms).  Then the face-state check.  The accessors let a kernel keep
// X and T in shared memory, read and written where they are used.
template <typename T, bool CTU, typename XG, typename TP>
__device__ __forceinline__ void reconstruct(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu,
                                            T (&lo)[NV], T (&hi)[NV], XG &&xget, TP &&tput) {
  Eig<T> E;
  E.init(w0);
  T d[NV], cl[NV], cr[NV];
  v_sub(d, w0, wm);
  E.project(d, cl);
  v_sub(d, wp, w0);
  E.project(d, cr);
  // limited amplitudes, doubled (every quantity below up to the predictor is exactly twice
  // its unscaled value, so the face states are bit for bit those of the unscaled form)
  T m[NV];
  mc_limit2_v(cl, cr, m);
  if constexpr (CTU) {
    T o[NV];
    upwind_terms(E, cl, cr, nu, o);
#pragma unroll
    for (int k = 0; k < NV; k++) tput(k, o[k]);
  }
  T dw[NV], g[NV];
  E.back2(m, dw, g);  // 2 dw^m (dw^m the limited primitive slope) and 2 (A dw^m - u dw^m)
  // hi, lo = w0 -+ dw^m/2 - nu A dw^m = (w0 - nu g / 2) + (+-1/4 - nu u / 2) 2 dw^m
  const T nu2 = T(0.5) * nu;
  T base[NV];
  v_fma(base, g, -nu2, w0);
  if constexpr (CTU) {
#pragma unroll
    for (int k = 0; k < NV; k++) base[k] += xget(k);
  }
  v_fma(hi, dw, T(0.25) - nu2 * E.u, base);
  v_fma(lo, dw, T(-0.25) - nu2 * E.u, base);
  face_state_check(w0, lo, hi);
}

template <typename T>
__device__ __forceinline__ void reconstruct(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu,
                                            T (&lo)[NV], T (&hi)[NV]) {
  reconstruct<T, false>(wm, w0, wp, nu, lo, hi, [](int) { return T(0); }, [](int, T) {});
}

// Upwind characteristic tracing for the Roe-type flux (Sec. 3.3, eqs 40-43: reference
// states traced with the fastest wave towards each face, then each wave that reaches the
// face corrected to its own speed; no eq 44-45 terms).  Summed per wave a with amplitude
// c_a = (L dw^m)_a and speed lam_a = u + s_a:
//   hi = w0 + sum_a (1/2 - nu x_a) c_a R^a,   x_a = lam_a if lam_a > 0, else max(u + cf, 0)
//   lo = w0 + sum_a (-1/2 - nu y_a) c_a R^a,  y_a = lam_a if lam_a < 0, else min(u - cf, 0)
// (eq 41 read in the mirror form of eq 40).  Same limiter, transverse terms (CTU) and
// face-state check as reconstruct.
template <typename T, bool CTU, typename XG, typename TP>
__device__ __forceinline__ void reconstruct_upwind(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV],
                                                   T nu, T (&lo)[NV], T (&hi)[NV], XG &&xget, TP &&tput) {
  Eig<T> E;
  E.init(w0);
  T d[NV], cl[NV], cr[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = w0[k] - wm[k];
  E.project(d, cl);
#pragma unroll
  for (int k = 0; k < NV; k++) d[k] = wp[k] - w0[k];
  E.project(d, cr);
  // doubled limited amplitudes: the coefficients below carry the factor 1/2
  T m[NV];
  mc_limit2_v(cl, cr, m);
  if constexpr (CTU) {
    T o[NV];
    upwind_terms(E, cl, cr, nu, o);
#pragma unroll
    for (int k = 0; k < NV; k++) tput(k, o[k]);
  }
  const T u = E.u;
  const T s[NV] = {-E.cf, -E.cs, -E.cs, T(0), T(0), T(0), T(0), E.cs, E.cs, E.cf};
  const T xM = fmax(u + E.cf, T(0)), y0 = fmin(u - E.cf, T(0)), nu2 = T(0.5) * nu;
  T ch[NV], cl2[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T lam = u + s[k];
    ch[k] = (T(0.25) - nu2 * (lam > T(0) ? lam : xM)) * m[k];
    cl2[k] = (T(-0.25) - nu2 * (lam < T(0) ? lam : y0)) * m[k];
  }
  T dh[NV], dl[NV];
  E.back(ch, dh);
  E.back(cl2, dl);
#pragma unroll
  for (int k = 0; k < NV; k++) {
    T base = w0[k];
    if constexpr (CTU) base += xget(k);
    hi[k] = base + dh[k];
    lo[k] = base + dl[k];
  }
  face_state_check(w0, lo, hi);
}

template <typename T>
__device__ __forceinline__ void reconstruct_upwind(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV],
                                                   T nu, T (&lo)[NV], T (&hi)[NV]) {
  reconstruct_upwind<T, false>(wm, w0, wp, nu, lo, hi, [](int) { return T(0); }, [](int, T) {});
}

// A-posteriori fallback: every face that touches a cell whose second-order update was
// not realizable takes first-order states (the cell-centred primitive state).  fm, f0,
// fp: tags of cells i-1, i, i+1 along the sweep.
template <typename T>
__device__ __forceinline__ void first_order_faces(bool fm, bool f0, bool fp, const T (&w0)[NV], T (&lo)[NV],
                                                  T (&hi)[NV]) {
  if (f0 || fm) {
#pragma unroll
    for (int k = 0; k < NV; k++) lo[k] = w0[k];
  }
  if (f0 || fp) {
#pragma unroll
    for (int k = 0; k < NV; k++) hi[k] = w0[k];
  }
}

// Conserved vector and normal flux of a local-frame primitive state (eqs contin,
// moment, dispers: rho u_n; rho u_i u_n + P_in; E_ij u_n + P_in u_j + P_jn u_i).
template <typename T>
__device__ __forceinline__ void phys(const T (&w)[NV], T (&U)[NV], T (&F)[NV]) {
  const T r = w[0], u = w[1], v = w[2], ww = w[3];
  const T Pxx = w[4], Pxy = w[5], Pxz = w[6], Pyy = w[7], Pyz = w[8], Pzz = w[9];
  const T mx = r * u, my = r * v, mz = r * ww;
  U[0] = r; U[1] = mx; U[2] = my; U[3] = mz;
  U[4] = Pxx + mx * u; U[5] = Pxy + mx * v; U[6] = Pxz + mx * ww;
  U[7] = Pyy + my * v; U[8] = Pyz + my * ww; U[9] = Pzz + mz * ww;
  F[0] = mx;
  F[1] = mx * u + Pxx;
  F[2] = my * u + Pxy;
  F[3] = mz * u + Pxz;
  F[4] = (U[4] + T(2) * Pxx) * u;
  F[5] = (U[5] + Pxy) * u + Pxx * v;
  F[6] = (U[6] + Pxz) * u + Pxx * ww;
  F[7] = U[7] * u + T(2) * Pxy * v;
  F[8] = U[8] * u + Pxy * ww + Pxz * v;
  F[9] = U[9] * u + T(2) * Pxz * ww;
}

// HLL flux between local-frame face states wl | wr with signal speeds
// S_L = min(u_L - cf_L, u_R - cf_R), S_R = max(u_L + cf_L, u_R + cf_R).
template <typename T>
__device__ __forceinline__ void hll(const T (&wl)[NV], const T (&wr)[NV], T (&F)[NV]) {
  T Ul[NV], Fl[NV], Ur[NV], Fr[NV];
  phys(wl, Ul, Fl);
  phys(wr, Ur, Fr);
  const T cl = T(1.7320508075688772) * sqrt_ratio(wl[4], wl[0]);
  const T cr = T(1.7320508075688772) * sqrt_ratio(wr[4], wr[0]);
  const T SL = fmin(wl[1] - cl, wr[1] - cr);
  const T SR = fmax(wl[1] + cl, wr[1] + cr);
  // F = a Fl + b Fr + c (Ur - Ul): (1, 0, 0) for SL >= 0, (0, 1, 0) for SR <= 0, else
  // (SR, -SL, SL SR) / (SR - SL); the branch selects three scalars, not ten fluxes
  T a, b, c;
  if (SL >= T(0)) {
    a = T(1); b = T(0); c = T(0);
  } else if (SR <= T(0)) {
    a = T(0); b = T(1); c = T(0);
  } else {
    const T inv = frcp(SR - SL);
    a = SR * inv;
    b = -SL * inv;
    c = SL * SR * inv;
  }
  T t[NV];
  v_sub(t, Ur, Ul);
  v_mul(t, t, c);
  v_fma(t, Fr, b, t);
  v_fma(F, Fl, a, t);
}

// ------------------------------------------------------- Kurganov-Tadmor
// Face values of one cell for the central scheme of Sec. 3.2 (local frame): primitive
// variables reconstructed component by component with the MC limiter (computed doubled:
// w0 -+ 2mc/4 is exactly w0 -+ mc/2); a face value with rho <= 0 or P_nn <= 0 reverts both
// faces to w0.
template <typename T>
__device__ __forceinline__ void kt_reconstruct(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV],
                                               T (&lo)[NV], T (&hi)[NV]) {
  T dl[NV], dr[NV], s2[NV];
  v_sub(dl, w0, wm);
  v_sub(dr, wp, w0);
  mc_limit2_v(dl, dr, s2);
  v_fma(hi, s2, T(0.25), w0);
  v_fma(lo, s2, T(-0.25), w0);
  face_state_check(w0, lo, hi);
}

// Central flux H = (f(wl) + f(wr))/2 - a (U(wr) - U(wl))/2 through a face with the value wl
// on its left side and wr on its right side; a = the larger spectral radius of df/du,
// |u_n| + sqrt(3 P_nn / rho), of the two (eqs spectralfreq, soundspeed with gamma = 3).
template <typename T>
__device__ __forceinline__ void kt_flux(const T (&wl)[NV], const T (&wr)[NV], T (&F)[NV]) {
  T Ul[NV], Fl[NV], Ur[NV], Fr[NV];
  phys(wl, Ul, Fl);
  phys(wr, Ur, Fr);
  const T al = fabs(wl[1]) + T(1.7320508075688772) * sqrt_ratio(wl[4], wl[0]);
  const T ar = fabs(wr[1]) + T(1.7320508075688772) * sqrt_ratio(wr[4], wr[0]);
  const T h = T(0.5) * fmax(al, ar);
  T dU[NV], Fs[NV];
  v_sub(dU, Ur, Ul);
  v_add(Fs, Fl, Fr);
  v_mul(Fs, Fs, T(0.5));
  v_fma(F, dU, -h, Fs);
}

// ------------------------------------------------------------ Roe-type flux
// Linearised characteristic upwind flux (local frame):
//   F = (f(wl) + f(wr)) / 2 - (dU/dW)(wm) R |Lambda| L (wr - wl) / 2,
// with wm = (wl + wr) / 2 (no Roe average is known for the ten-moment system), the
// closed-form eigen-system of wm, and Harten's entropy fix on the two fast waves only:
// |lambda| -> (lambda^2 + delta^2) / (2 delta) below delta = cf / 10.  The shear and contact
// waves are linearly degenerate and keep |lambda|, so a stationary contact is not diffused.
template <typename T>
__device__ __forceinline__ void roe_flux(const T (&wl)[NV], const T (&wr)[NV], T (&F)[NV]) {
  T wm[NV], dw[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    wm[k] = T(0.5) * (wl[k] + wr[k]);
    dw[k] = wr[k] - wl[k];
  }
  Eig<T> E;
  E.init(wm);
  T c[NV];
  E.project(dw, c);
  const T u = E.u, delta = T(0.1) * E.cf;
  auto fast = [&](T l) {
    const T al = fabs(l);
    return al < delta ? (l * l + delta * delta) * (T(0.5) * frcp(delta)) : al;
  };
  const T am = fabs(u - E.cs), ap = fabs(u + E.cs), a0 = fabs(u);
  c[0] *= fast(u - E.cf);
  c[9] *= fast(u + E.cf);
  c[1] *= am; c[2] *= am;
  c[7] *= ap; c[8] *= ap;
  c[3] *= a0; c[4] *= a0; c[5] *= a0; c[6] *= a0;
  T d[NV];
  E.back(c, d);  // primitive dissipation R |Lambda| L dw
  const T r = wm[0], ux = wm[1], uy = wm[2], uz = wm[3];
  T dU[NV];      // through the Jacobian of the conserved map at wm
  dU[0] = d[0];
  dU[1] = r * d[1] + ux * d[0];
  dU[2] = r * d[2] + uy * d[0];
  dU[3] = r * d[3] + uz * d[0];
  dU[4] = d[4] + d[0] * ux * ux + r * (T(2) * d[1] * ux);
  dU[5] = d[5] + d[0] * ux * uy + r * (d[1] * uy + ux * d[2]);
  dU[6] = d[6] + d[0] * ux * uz + r * (d[1] * uz + ux * d[3]);
  dU[7] = d[7] + d[0] * uy * uy + r * (T(2) * d[2] * uy);
  dU[8] = d[8] + d[0] * uy * uz + r * (d[2] * uz + uy * d[3]);
  dU[9] = d[9] + d[0] * uz * uz + r * (T(2) * d[3] * uz);
  T Ul[NV], Fl[NV], Ur[NV], Fr[NV];
  phys(wl, Ul, Fl);
  phys(wr, Ur, Fr);
  T Fs[NV];
  v_add(Fs, Fl, Fr);
  v_sub(Fs, Fs, dU);
  v_mul(F, Fs, T(0.5));
}

// ------------------------------------------------------------------- HLLC
// The part Pi of the normal flux F = u U + Pi (local frame) that depends only on the
// quantities continuous across a contact, u_i and P_ix:
//   Pi = (0; P_ix; P_ix u_j + P_jx u_i).
template <typename T>
__device__ __forceinline__ void pi_terms(T u, T v, T w, T pxx, T pxy, T pxz, T (&P)[NV]) {
  P[0] = T(0);
  P[1] = pxx;
  P[2] = pxy;
  P[3] = pxz;
  P[4] = T(2) * pxx * u;
  P[5] = pxy * u + pxx * v;
  P[6] = pxz * u + pxx * w;
  P[7] = T(2) * pxy * v;
  P[8] = pxy * w + pxz * v;
  P[9] = T(2) * pxz * w;
}

// Three-wave HLLC flux for the ten-moment system (local frame).  Outer waves S_L, S_R as in
// HLL (they carry the fast and shear waves), the contact S_M in between (it carries rho and
// the transverse stresses).  Every pair (u_i, P_ix) takes one star value on both sides of
// the contact, from the momentum jump conditions across S_L and S_R with C_K = rho_K
// (S_K - u_K):  u*_i = (C_R u_i,R - C_L u_i,L - (P_ix,R - P_ix,L)) / (C_R - C_L),
// P*_ix = P_ix,L + C_L (u*_i - u_i,L);  S_M = u*_x.  The star state of side K follows from
// the jump conditions across S_K, U*_K = (U_K (S_K - u_K) + Pi* - Pi_K) / (S_K - S_M), so
// the flux F_K + S_K (U*_K - U_K) of the side of the face that holds x/t = 0 is
//   F = a U_K + b Pi_K + c Pi*,  (a, b, c) = (S_M (S_K - u_K), -S_M, S_K) / (S_K - S_M),
// or (u_K, 1, 0) (the physical flux) when both waves move away from the face.  Where S_M is
// not strictly inside (S_L, S_R) the flux is HLL's.
template <typename T>
__device__ __forceinline__ void hllc_flux(const T (&wl)[NV], const T (&wr)[NV], T (&F)[NV]) {
  const T cl = T(1.7320508075688772) * sqrt_ratio(wl[4], wl[0]);
  const T cr = T(1.7320508075688772) * sqrt_ratio(wr[4], wr[0]);
  const T SL = fmin(wl[1] - cl, wr[1] - cr);
  const T SR = fmax(wl[1] + cl, wr[1] + cr);
  const T CL = wl[0] * (SL - wl[1]), CR = wr[0] * (SR - wr[1]);
  const T inv = frcp(CR - CL);
  T us[3], ps[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    us[i] = (CR * wr[1 + i] - CL * wl[1 + i] - (wr[4 + i] - wl[4 + i])) * inv;
    ps[i] = wl[4 + i] + CL * (us[i] - wl[1 + i]);
  }
  const T SM = us[0];
  if (!(SL < SM && SM < SR)) {
    hll(wl, wr, F);
    return;
  }
  const bool left = SM >= T(0);
  T wk[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) wk[k] = left ? wl[k] : wr[k];
  const T SK = left ? SL : SR, uk = wk[1];
  T a, b, c;
  if (SL >= T(0) || SR <= T(0)) {
    a = uk; b = T(1); c = T(0);
  } else {
    const T i2 = frcp(SK - SM);
    a = SM * (SK - uk) * i2;
    b = -SM * i2;
    c = SK * i2;
  }
  T Uk[NV], Fk[NV], Pk[NV], Ps[NV];
  phys(wk, Uk, Fk);
  pi_terms(wk[1], wk[2], wk[3], wk[4], wk[5], wk[6], Pk);
  pi_terms(us[0], us[1], us[2], ps[0], ps[1], ps[2], Ps);
  T t[NV];
  v_mul(t, Ps, c);
  v_fma(t, Pk, b, t);
  v_fma(F, Uk, a, t);
}

// Scheme of a step kernel: 0 the characteristic MUSCL-Hancock step with HLL (Sec. 3.3);
// 1 and 2 the two Runge-Kutta stages of the Kurganov-Tadmor scheme (Sec. 3.2); 3 the
// characteristic step with upwind tracing and the Roe-type flux; 4 the characteristic step
// with the HLLC flux.  0, 3 and 4 have the a-posteriori fallback.
template <int SCH> constexpr bool kCharacteristic = SCH == 0 || SCH == 3 || SCH == 4;

template <int SCH, typename T>
__device__ __forceinline__ void recon(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu, T (&lo)[NV],
                                      T (&hi)[NV]) {
  if constexpr (SCH == 0 || SCH == 4) reconstruct(wm, w0, wp, nu, lo, hi);
  else if constexpr (SCH == 3) reconstruct_upwind(wm, w0, wp, nu, lo, hi);
  else kt_reconstruct(wm, w0, wp, lo, hi);
}

// The characteristic schemes' reconstruction with the transverse terms X (local frame,
// xget(k) = X_k) in the face states; the cell's own transverse term along the sweep goes to
// tput(k, T_k).
template <int SCH, typename T, typename XG, typename TP>
__device__ __forceinline__ void recon_ctu(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu,
                                          XG &&xget, TP &&tput, T (&lo)[NV], T (&hi)[NV]) {
  static_assert(kCharacteristic<SCH>, "transverse terms belong to the characteristic schemes");
  if constexpr (SCH == 3) reconstruct_upwind<T, true>(wm, w0, wp, nu, lo, hi, xget, tput);
  else reconstruct<T, true>(wm, w0, wp, nu, lo, hi, xget, tput);
}

template <int SCH, typename T>
__device__ __forceinline__ void face_flux(const T (&wl)[NV], const T (&wr)[NV], T (&F)[NV]) {
  if constexpr (SCH == 0) hll(wl, wr, F);
  else if constexpr (SCH == 3) roe_flux(wl, wr, F);
  else if constexpr (SCH == 4) hllc_flux(wl, wr, F);
  else kt_flux(wl, wr, F);
}

// Flux through a face in a step pass: in a fallback pass (RETRY) a face with first-order
// states (it touches a tagged cell) takes HLL under the Roe-type and HLLC schemes too.  The
// fallback has to make the update realizable; HLL with bounding wave speeds is positively
// conservative, a linearised Roe flux is not (Einfeldt, Munz, Roe & Sjogreen 1991), and
// HLLC's star states, formed from jump conditions, need not be realizable.
template <int SCH, bool RETRY, typename T>
__device__ __forceinline__ void face_flux(const T (&wl)[NV], const T (&wr)[NV], bool first, T (&F)[NV]) {
  if constexpr ((SCH == 3 || SCH == 4) && RETRY) {
    if (first) hll(wl, wr, F);
    else face_flux<SCH>(wl, wr, F);
  } else {
    face_flux<SCH>(wl, wr, F);
  }
}

// ---------------------------------------------------------- accumulators
// Per-thread running sums of the conserved totals over the cells one thread updates.  FP64
// states add in FP64.  FP32 states add in FP32 per thread (relative rounding error of a
// k-term sum below k 2^-24, random in sign across threads) and in FP64 from the block
// reduction on, so the totals need no FP64 arithmetic per cell (FP64 throughput is a small
// fraction of FP32 on this GPU).  The 3D step moves a thread's FP32 sum into FP64 block
// totals every 64 planes of a stretch and at its end, so one FP32 sum spans at most 64
// cells; 2D strips and 1D tiles stream one chunk.
template <typename T> struct Acc {
  double v[NV];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = 0.0;
  }
  __device__ __forceinline__ void add(const T (&x)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] += x[k];
  }
  __device__ __forceinline__ void get(double (&o)[NV]) const {
#pragma unroll
    for (int k = 0; k < NV; k++) o[k] = v[k];
  }
};
template <> struct Acc<float> {
  float v[NV];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = 0.f;
  }
  __device__ __forceinline__ void add(const float (&x)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; k += 2) {
      const float2 r = __fadd2_rn(make_float2(v[k], v[k + 1]), make_float2(x[k], x[k + 1]));
      v[k] = r.x;
      v[k + 1] = r.y;
    }
  }
  __device__ __forceinline__ void get(double (&o)[NV]) const {
#pragma unroll
    for (int k = 0; k < NV; k++) o[k] = (double)v[k];
  }
};

// ------------------------------------------------------------- boundaries
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2 };

// Map a (possibly ghost) index onto the grid.  mirror = reflect image.  The result is
// clamped into [0, n) so that tile overhang beyond the ghost layers stays in bounds.
__device__ __forceinline__ int map_index(int i, int n, int bclo, int bchi, bool &mirror) {
  mirror = false;
  if (i < 0) {
    if (bclo == BC_PERIODIC) i += n;
    else if (bclo == BC_OUTFLOW) i = 0;
    else { i = -1 - i; mirror = true; }
  } else if (i >= n) {
    if (bchi == BC_PERIODIC) i -= n;
    else if (bchi == BC_OUTFLOW) i = n - 1;
    else { i = 2 * n - 1 - i; mirror = true; }
  }
  return min(max(i, 0), n - 1);
}

// Sign flips of a mirrored image across a face normal to d: m_d and E_dt (t != d).
__device__ __forceinline__ unsigned flip_mask(int d) {
  return d == 0 ? ((1u << 1) | (1u << 5) | (1u << 6))
       : d == 1 ? ((1u << 2) | (1u << 5) | (1u << 8))
                : ((1u << 3) | (1u << 6) | (1u << 8));
}

}  // namespace msh
