// msh_adjoint.cuh -- hand-written reverse mode (vector-Jacobian products) of the
// per-cell and per-face operations of the step, branches frozen at their forward values.
//
// Each *_vjp recomputes the forward quantities it needs from its inputs and accumulates
// the adjoints of its inputs (the "bar" arrays are added to, never overwritten).
#pragma once
#include "msh_device.cuh"

namespace msh {

// W = W(U): rho, u = m/rho, P = E - m m^T / rho.  Accumulates Ub += (dW/dU)^T Wb.
template <typename T>
__device__ __forceinline__ void cons_to_prim_vjp(const T (&U)[NV], const T (&Wb)[NV], T (&Ub)[NV]) {
  const T ir = T(1) / U[0];
  const T u0 = U[1] * ir, u1 = U[2] * ir, u2 = U[3] * ir;
  Ub[0] += Wb[0] - (Wb[1] * u0 + Wb[2] * u1 + Wb[3] * u2) * ir + Wb[4] * u0 * u0 + Wb[5] * u0 * u1 +
           Wb[6] * u0 * u2 + Wb[7] * u1 * u1 + Wb[8] * u1 * u2 + Wb[9] * u2 * u2;
  Ub[1] += Wb[1] * ir - T(2) * u0 * Wb[4] - u1 * Wb[5] - u2 * Wb[6];
  Ub[2] += Wb[2] * ir - u0 * Wb[5] - T(2) * u1 * Wb[7] - u2 * Wb[8];
  Ub[3] += Wb[3] * ir - u0 * Wb[6] - u1 * Wb[8] - T(2) * u2 * Wb[9];
#pragma unroll
  for (int k = 4; k < NV; k++) Ub[k] += Wb[k];
}

// U = U(W).  Accumulates Wb += (dU/dW)^T Ub.
template <typename T>
__device__ __forceinline__ void prim_to_cons_vjp(const T (&W)[NV], const T (&Ub)[NV], T (&Wb)[NV]) {
  const T r = W[0], u0 = W[1], u1 = W[2], u2 = W[3];
  Wb[0] += Ub[0] + Ub[1] * u0 + Ub[2] * u1 + Ub[3] * u2 + Ub[4] * u0 * u0 + Ub[5] * u0 * u1 + Ub[6] * u0 * u2 +
           Ub[7] * u1 * u1 + Ub[8] * u1 * u2 + Ub[9] * u2 * u2;
  Wb[1] += r * (Ub[1] + T(2) * u0 * Ub[4] + u1 * Ub[5] + u2 * Ub[6]);
  Wb[2] += r * (Ub[2] + u0 * Ub[5] + T(2) * u1 * Ub[7] + u2 * Ub[8]);
  Wb[3] += r * (Ub[3] + u0 * Ub[6] + u1 * Ub[8] + T(2) * u2 * Ub[9]);
#pragma unroll
  for (int k = 4; k < NV; k++) Wb[k] += Ub[k];
}

// Gravity source after the hydro update (linear in U* for a fixed acceleration g):
//   rho' = rho*, m' = m* + dt rho* g, E' = E* + dt (m* g^T + g m*^T) + dt^2 rho* g g^T.
// Returns lam* = (dU'/dU*)^T lam.
template <typename T>
__device__ __forceinline__ void gravity_vjp(const T (&g)[3], T dt, const T (&lam)[NV], T (&ls)[NV]) {
  const T d2 = dt * dt;
  ls[0] = lam[0] + dt * (g[0] * lam[1] + g[1] * lam[2] + g[2] * lam[3]) +
          d2 * (g[0] * g[0] * lam[4] + g[0] * g[1] * lam[5] + g[0] * g[2] * lam[6] + g[1] * g[1] * lam[7] +
                g[1] * g[2] * lam[8] + g[2] * g[2] * lam[9]);
  ls[1] = lam[1] + dt * (T(2) * g[0] * lam[4] + g[1] * lam[5] + g[2] * lam[6]);
  ls[2] = lam[2] + dt * (g[0] * lam[5] + T(2) * g[1] * lam[7] + g[2] * lam[8]);
  ls[3] = lam[3] + dt * (g[0] * lam[6] + g[1] * lam[8] + T(2) * g[2] * lam[9]);
#pragma unroll
  for (int k = 4; k < NV; k++) ls[k] = lam[k];
}

// Reverse of phys(): accumulates wb += (dU/dw)^T Ub + (dF/dw)^T Fb (local frame).
template <typename T>
__device__ __forceinline__ void phys_vjp(const T (&w)[NV], const T (&Ub)[NV], const T (&Fb)[NV], T (&wb)[NV]) {
  const T r = w[0], u = w[1], v = w[2], ww = w[3];
  const T Pxx = w[4], Pxy = w[5], Pxz = w[6];
  const T mx = r * u, my = r * v, mz = r * ww;
  const T U4 = Pxx + mx * u, U5 = Pxy + mx * v, U6 = Pxz + mx * ww;
  const T U7 = w[7] + my * v, U8 = w[8] + my * ww, U9 = w[9] + mz * ww;
  const T b4 = Ub[4] + Fb[4] * u, b5 = Ub[5] + Fb[5] * u, b6 = Ub[6] + Fb[6] * u;
  const T b7 = Ub[7] + Fb[7] * u, b8 = Ub[8] + Fb[8] * u, b9 = Ub[9] + Fb[9] * u;
  T ub = Fb[1] * mx + Fb[2] * my + Fb[3] * mz + Fb[4] * (U4 + T(2) * Pxx) + Fb[5] * (U5 + Pxy) +
         Fb[6] * (U6 + Pxz) + Fb[7] * U7 + Fb[8] * U8 + Fb[9] * U9;
  T vb = Fb[5] * Pxx + T(2) * Fb[7] * Pxy + Fb[8] * Pxz;
  T wwb = Fb[6] * Pxx + Fb[8] * Pxy + T(2) * Fb[9] * Pxz;
  wb[4] += Fb[1] + T(2) * Fb[4] * u + Fb[5] * v + Fb[6] * ww + b4;
  wb[5] += Fb[2] + Fb[5] * u + T(2) * Fb[7] * v + Fb[8] * ww + b5;
  wb[6] += Fb[3] + Fb[6] * u + Fb[8] * v + T(2) * Fb[9] * ww + b6;
  wb[7] += b7;
  wb[8] += b8;
  wb[9] += b9;
  const T mxb = Fb[0] + Fb[1] * u + Ub[1] + b4 * u + b5 * v + b6 * ww;
  const T myb = Fb[2] * u + Ub[2] + b7 * v + b8 * ww;
  const T mzb = Fb[3] * u + Ub[3] + b9 * ww;
  ub += b4 * mx;
  vb += b5 * mx + b7 * my;
  wwb += b6 * mx + b8 * my + b9 * mz;
  wb[0] += Ub[0] + mxb * u + myb * v + mzb * ww;
  wb[1] += ub + mxb * r;
  wb[2] += vb + myb * r;
  wb[3] += wwb + mzb * r;
}

// Reverse of hll() with the forward branch (and min/max selections) frozen.
template <typename T>
__device__ __forceinline__ void hll_vjp(const T (&wl)[NV], const T (&wr)[NV], const T (&Fb)[NV], T (&wlb)[NV],
                                        T (&wrb)[NV]) {
  T Ul[NV], Fl[NV], Ur[NV], Fr[NV];
  phys(wl, Ul, Fl);
  phys(wr, Ur, Fr);
  const T cl = T(1.7320508075688772) * sqrt_ratio(wl[4], wl[0]);
  const T cr = T(1.7320508075688772) * sqrt_ratio(wr[4], wr[0]);
  const T aL = wl[1] - cl, aR = wr[1] - cr, bL = wl[1] + cl, bR = wr[1] + cr;
  const T SL = fmin(aL, aR), SR = fmax(bL, bR);
  T zero[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) zero[k] = T(0);
  if (SL >= T(0)) {
    phys_vjp(wl, zero, Fb, wlb);
    return;
  }
  if (SR <= T(0)) {
    phys_vjp(wr, zero, Fb, wrb);
    return;
  }
  const T inv = T(1) / (SR - SL);
  T Flb[NV], Frb[NV], Urb[NV], Ulb[NV];
  T SLb = T(0), SRb = T(0);
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T dU = Ur[k] - Ul[k];
    const T F = (SR * Fl[k] - SL * Fr[k] + SL * SR * dU) * inv;
    Flb[k] = SR * inv * Fb[k];
    Frb[k] = -SL * inv * Fb[k];
    Urb[k] = SL * SR * inv * Fb[k];
    Ulb[k] = -Urb[k];
    SRb += Fb[k] * ((Fl[k] + SL * dU) * inv - F * inv);
    SLb += Fb[k] * ((-Fr[k] + SR * dU) * inv + F * inv);
  }
  T clb = T(0), crb = T(0);
  if (aL <= aR) { wlb[1] += SLb; clb -= SLb; } else { wrb[1] += SLb; crb -= SLb; }
  if (bL >= bR) { wlb[1] += SRb; clb += SRb; } else { wrb[1] += SRb; crb += SRb; }
  // c = sqrt(3 P / rho): dc/dP = c / (2P), dc/drho = -c / (2 rho)
  wlb[4] += clb * cl / (T(2) * wl[4]);
  wlb[0] -= clb * cl / (T(2) * wl[0]);
  wrb[4] += crb * cr / (T(2) * wr[4]);
  wrb[0] -= crb * cr / (T(2) * wr[0]);
  phys_vjp(wl, Ulb, Flb, wlb);
  phys_vjp(wr, Urb, Frb, wrb);
}

// Adjoints of the eigen-quantities of Eig<T> (and of the state entries they read).
template <typename T> struct EigBar {
  T rho, u, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz, cf, cs, a, b, ip, icf2, ics2;
  __device__ __forceinline__ void zero() {
    rho = u = Pxx = Pxy = Pxz = Pyy = Pyz = Pzz = cf = cs = a = b = ip = icf2 = ics2 = T(0);
  }
};

// Reverse of Eig::project (c = L d): accumulates db and the coefficient adjoints.
template <typename T>
__device__ __forceinline__ void project_vjp(const Eig<T> &E, const T (&d)[NV], const T (&cb)[NV], T (&db)[NV],
                                            EigBar<T> &Eb) {
  const T e = d[4] * E.ip * T(1.0 / 3.0);
  const T t2b = cb[0] + cb[9], t1b = cb[9] - cb[0];
  const T rvb = cb[1] + cb[7], qvb = cb[7] - cb[1];
  const T rwb = cb[2] + cb[8], qwb = cb[8] - cb[2];
  const T k4 = T(4) * E.a * E.Pxy - E.Pyy, k5 = T(4) * E.a * E.Pxz - E.Pyz, k6 = T(4) * E.b * E.Pxz - E.Pzz;
  const T eb = T(0.5) * t2b - E.rho * cb[3] + k4 * cb[4] + k5 * cb[5] + k6 * cb[6];
  db[0] += cb[3];
  db[7] += cb[4];
  db[8] += cb[5];
  db[9] += cb[6];
  db[1] += E.icf2 * t1b - E.a * E.ics2 * qvb - E.b * E.ics2 * qwb;
  db[2] += E.ics2 * qvb;
  db[3] += E.ics2 * qwb;
  db[4] += E.ip * T(1.0 / 3.0) * eb - T(0.5) * E.a * E.ip * rvb - T(0.5) * E.b * E.ip * rwb;
  db[5] += T(0.5) * E.ip * rvb - T(2) * E.a * cb[4] - E.b * cb[5];
  db[6] += T(0.5) * E.ip * rwb - E.a * cb[5] - T(2) * E.b * cb[6];
  Eb.ip += d[4] * T(1.0 / 3.0) * eb + T(0.5) * (d[5] - E.a * d[4]) * rvb + T(0.5) * (d[6] - E.b * d[4]) * rwb;
  Eb.icf2 += d[1] * t1b;
  Eb.ics2 += (d[2] - E.a * d[1]) * qvb + (d[3] - E.b * d[1]) * qwb;
  Eb.a += -d[1] * E.ics2 * qvb - T(0.5) * d[4] * E.ip * rvb - T(2) * d[5] * cb[4] + T(4) * E.Pxy * e * cb[4] -
          d[6] * cb[5] + T(4) * E.Pxz * e * cb[5];
  Eb.b += -d[1] * E.ics2 * qwb - T(0.5) * d[4] * E.ip * rwb - d[5] * cb[5] - T(2) * d[6] * cb[6] +
          T(4) * E.Pxz * e * cb[6];
  Eb.rho += -e * cb[3];
  Eb.Pxy += T(4) * E.a * e * cb[4];
  Eb.Pyy += -e * cb[4];
  Eb.Pxz += T(4) * E.a * e * cb[5] + T(4) * E.b * e * cb[6];
  Eb.Pyz += -e * cb[5];
  Eb.Pzz += -e * cb[6];
}

// Reverse of Eig::back (o = R c): accumulates cb and the coefficient adjoints.
template <typename T>
__device__ __forceinline__ void back_vjp(const Eig<T> &E, const T (&c)[NV], const T (&ob)[NV], T (&cb)[NV],
                                         EigBar<T> &Eb) {
  const T A = c[9] + c[0], B = (c[9] - c[0]) * E.cf;
  const T C = c[7] + c[1], Ec = c[8] + c[2];
  const T Ab = E.rho * ob[0] + T(3) * E.Pxx * ob[4] + T(3) * E.Pxy * ob[5] + T(3) * E.Pxz * ob[6] +
               (E.Pyy + T(2) * E.a * E.Pxy) * ob[7] + (E.Pyz + T(2) * E.a * E.Pxz) * ob[8] +
               (E.Pzz + T(2) * E.b * E.Pxz) * ob[9];
  const T Bb = ob[1] + E.a * ob[2] + E.b * ob[3];
  const T Cb = E.Pxx * ob[5] + T(2) * E.Pxy * ob[7] + E.Pxz * ob[8];
  const T Db = ob[2];
  const T Eb_ = E.Pxx * ob[6] + E.Pxy * ob[8] + T(2) * E.Pxz * ob[9];
  const T Fb = ob[3];
  cb[3] += ob[0];
  cb[4] += ob[7];
  cb[5] += ob[8];
  cb[6] += ob[9];
  cb[9] += Ab + E.cf * Bb;
  cb[0] += Ab - E.cf * Bb;
  cb[7] += Cb + E.cs * Db;
  cb[1] += Cb - E.cs * Db;
  cb[8] += Eb_ + E.cs * Fb;
  cb[2] += Eb_ - E.cs * Fb;
  Eb.rho += A * ob[0];
  Eb.cf += (c[9] - c[0]) * Bb;
  Eb.cs += (c[7] - c[1]) * Db + (c[8] - c[2]) * Fb;
  Eb.a += B * ob[2] + T(2) * E.Pxy * A * ob[7] + T(2) * E.Pxz * A * ob[8];
  Eb.b += B * ob[3] + T(2) * E.Pxz * A * ob[9];
  Eb.Pxx += T(3) * A * ob[4] + C * ob[5] + Ec * ob[6];
  Eb.Pxy += T(3) * A * ob[5] + (T(2) * E.a * A + T(2) * C) * ob[7] + Ec * ob[8];
  Eb.Pxz += T(3) * A * ob[6] + (T(2) * E.a * A + C) * ob[8] + (T(2) * E.b * A + T(2) * Ec) * ob[9];
  Eb.Pyy += A * ob[7];
  Eb.Pyz += A * ob[8];
  Eb.Pzz += A * ob[9];
}

// Reverse of Eig::init: adds the adjoints of the eigen-quantities into w0b (local frame).
template <typename T>
__device__ __forceinline__ void eig_init_vjp(const Eig<T> &E, const EigBar<T> &Eb, T (&w0b)[NV]) {
  const T q = E.Pxx / E.rho;
  const T rs = frsqrt(q);
  const T csb = Eb.cs + T(1.7320508075688772) * Eb.cf;
  T rsb = T(0.28867513459481287) * Eb.icf2 + T(0.5) * Eb.ics2 + csb * q;
  T qb = csb * rs - T(0.5) * rsb * rs / q;
  T Pxxb = Eb.Pxx + qb / E.rho;
  const T rhob = Eb.rho - qb * q / E.rho;
  const T ipb = Eb.ip + Eb.a * E.Pxy + Eb.b * E.Pxz;
  Pxxb -= ipb * E.ip * E.ip;
  w0b[0] += rhob;
  w0b[1] += Eb.u;
  w0b[4] += Pxxb;
  w0b[5] += Eb.Pxy + Eb.a * E.ip;
  w0b[6] += Eb.Pxz + Eb.b * E.ip;
  w0b[7] += Eb.Pyy;
  w0b[8] += Eb.Pyz;
  w0b[9] += Eb.Pzz;
}

// Reverse of reconstruct() (local frame) plus the a-posteriori first-order overrides
// (fm, f0, fp: tags of cells i-1, i, i+1 in the forward pass whose result is kept).
// Accumulates wmb, w0b, wpb from the face-state adjoints lob (at i-1/2) and hib (at i+1/2).
template <typename T>
__device__ __forceinline__ void reconstruct_vjp(const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T nu,
                                                bool fm, bool f0, bool fp, const T (&lob_in)[NV],
                                                const T (&hib_in)[NV], T (&wmb)[NV], T (&w0b)[NV], T (&wpb)[NV]) {
  T lob[NV], hib[NV];
  const bool lo_first = f0 || fm, hi_first = f0 || fp;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    lob[k] = lo_first ? T(0) : lob_in[k];
    hib[k] = hi_first ? T(0) : hib_in[k];
    if (lo_first) w0b[k] += lob_in[k];
    if (hi_first) w0b[k] += hib_in[k];
  }
  if (lo_first && hi_first) return;
  // forward recomputation
  Eig<T> E;
  E.init(w0);
  T dL[NV], dR[NV], cl[NV], cr[NV], m[NV], lm[NV], dw[NV], g[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    dL[k] = w0[k] - wm[k];
    dR[k] = wp[k] - w0[k];
  }
  E.project(dL, cl);
  E.project(dR, cr);
#pragma unroll
  for (int k = 0; k < NV; k++) m[k] = mc_limit(cl[k], cr[k]);
  lm[0] = -E.cf * m[0]; lm[1] = -E.cs * m[1]; lm[2] = -E.cs * m[2];
  lm[3] = T(0); lm[4] = T(0); lm[5] = T(0); lm[6] = T(0);
  lm[7] = E.cs * m[7]; lm[8] = E.cs * m[8]; lm[9] = E.cf * m[9];
  E.back(m, dw);
  E.back(lm, g);
  {
    T hi0 = T(0), lo0 = T(0), hi4 = T(0), lo4 = T(0);
    const T adw0 = E.u * dw[0] + g[0], adw4 = E.u * dw[4] + g[4];
    hi0 = w0[0] - nu * adw0 + T(0.5) * dw[0];
    lo0 = w0[0] - nu * adw0 - T(0.5) * dw[0];
    hi4 = w0[4] - nu * adw4 + T(0.5) * dw[4];
    lo4 = w0[4] - nu * adw4 - T(0.5) * dw[4];
    if (!(hi0 > T(0) && lo0 > T(0) && hi4 > T(0) && lo4 > T(0))) {  // face-state fallback: lo = hi = w0
#pragma unroll
      for (int k = 0; k < NV; k++) w0b[k] += lob[k] + hib[k];
      return;
    }
  }
  // reverse
  EigBar<T> Eb;
  Eb.zero();
  T dwb[NV], gb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const T predb = hib[k] + lob[k];
    const T adwb = -nu * predb;
    w0b[k] += predb;
    dwb[k] = T(0.5) * (hib[k] - lob[k]) + E.u * adwb;
    Eb.u += adwb * dw[k];
    gb[k] = adwb;
  }
  T mb[NV], lmb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) { mb[k] = T(0); lmb[k] = T(0); }
  back_vjp(E, lm, gb, lmb, Eb);
  back_vjp(E, m, dwb, mb, Eb);
  mb[0] += -E.cf * lmb[0]; mb[1] += -E.cs * lmb[1]; mb[2] += -E.cs * lmb[2];
  mb[7] += E.cs * lmb[7]; mb[8] += E.cs * lmb[8]; mb[9] += E.cf * lmb[9];
  Eb.cf += -m[0] * lmb[0] + m[9] * lmb[9];
  Eb.cs += -m[1] * lmb[1] - m[2] * lmb[2] + m[7] * lmb[7] + m[8] * lmb[8];
  // MC limiter with the forward selection frozen
  T clb[NV], crb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    clb[k] = T(0);
    crb[k] = T(0);
    const T l = cl[k], r = cr[k];
    if (l * r > T(0)) {
      const T al = T(2) * fabs(l), ac = fabs(T(0.5) * (l + r)), ar = T(2) * fabs(r);
      if (al <= ac && al <= ar) clb[k] = T(2) * mb[k];
      else if (ac <= ar) { clb[k] = T(0.5) * mb[k]; crb[k] = T(0.5) * mb[k]; }
      else crb[k] = T(2) * mb[k];
    }
  }
  T dLb[NV], dRb[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) { dLb[k] = T(0); dRb[k] = T(0); }
  project_vjp(E, dL, clb, dLb, Eb);
  project_vjp(E, dR, crb, dRb, Eb);
#pragma unroll
  for (int k = 0; k < NV; k++) {
    w0b[k] += dLb[k] - dRb[k];
    wmb[k] -= dLb[k];
    wpb[k] += dRb[k];
  }
  // the eigen-quantities (and the entries Eig reads directly) depend on w0
  eig_init_vjp(E, Eb, w0b);
}

}  // namespace msh
