"""Differentiable FP64 restatement of the step in plain PyTorch CPU ops (test infrastructure).

It computes the same step as ``msh_oracle.c`` (Sec. 3.3 of the paper: characteristic
MUSCL-Hancock reconstruction with the MC limiter, HLL flux, unsplit update, gravity source
after the hydro update), vectorised over cells with explicit batched 10x10 matrices L, R and
A of the ten-moment system, and with the same readings (face-state fallback, a-posteriori
first-order fallback).  Its purpose is the discrete adjoint: torch.autograd differentiates
the step exactly, with every branch (limiter selection, HLL branch, min/max of the signal
speeds, fallbacks) frozen at its forward value.  The C oracle pins its forward pass; central
finite differences of the C oracle pin its gradients.

Layout: U is a float64 tensor [10, nz, ny, nx]; component order as in the C oracle.
"""
from __future__ import annotations

import math

import torch

NV = 10
TI = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}


def tidx(i, j):
    return TI[(min(i, j), max(i, j))]


# local frame of a sweep direction: normal axis first, transverse axes in natural order
PERM = {0: [0, 1, 2, 3, 4, 5, 6, 7, 8, 9],
        1: [0, 2, 1, 3, 7, 5, 8, 4, 6, 9],
        2: [0, 3, 1, 2, 9, 6, 8, 4, 5, 7]}


def cons_to_prim(U):
    rho = U[0]
    u = [U[1 + i] / rho for i in range(3)]
    W = [rho] + u + [None] * 6
    for i in range(3):
        for j in range(i, 3):
            W[tidx(i, j)] = U[tidx(i, j)] - rho * u[i] * u[j]
    return torch.stack(W)


def prim_to_cons(W):
    rho = W[0]
    U = [rho] + [rho * W[1 + i] for i in range(3)] + [None] * 6
    for i in range(3):
        for j in range(i, 3):
            U[tidx(i, j)] = W[tidx(i, j)] + rho * W[1 + i] * W[1 + j]
    return torch.stack(U)


def flux(W, d):
    """Physical flux along d: rho u_d; rho u_i u_d + P_id; E_ij u_d + P_id u_j + P_jd u_i."""
    U = prim_to_cons(W)
    rho, u = W[0], W[1:4]
    F = [rho * u[d]] + [rho * u[i] * u[d] + W[tidx(i, d)] for i in range(3)] + [None] * 6
    for i in range(3):
        for j in range(i, 3):
            F[tidx(i, j)] = U[tidx(i, j)] * u[d] + W[tidx(i, d)] * u[j] + W[tidx(j, d)] * u[i]
    return torch.stack(F)


def _mat(entries, shape, like):
    M = torch.zeros(shape + (NV, NV), dtype=like.dtype)
    for (r, c), v in entries.items():
        M[..., r, c] = v
    return M


def eigen_x(w):
    """Quasi-linear Jacobian A, left eigenvectors L (rows) and right eigenvectors R (columns)
    of the x-normal ten-moment system at local-frame primitive states w [10, ...]."""
    rho, u = w[0], w[1]
    Pxx, Pxy, Pxz, Pyy, Pyz, Pzz = w[4], w[5], w[6], w[7], w[8], w[9]
    shape = tuple(rho.shape)
    cf = torch.sqrt(3.0 * Pxx / rho)
    cs = torch.sqrt(Pxx / rho)
    A = {(k, k): u for k in range(NV)}
    A.update({(0, 1): rho, (1, 4): 1 / rho, (2, 5): 1 / rho, (3, 6): 1 / rho, (4, 1): 3 * Pxx,
              (5, 1): 2 * Pxy, (5, 2): Pxx, (6, 1): 2 * Pxz, (6, 3): Pxx, (7, 1): Pyy, (7, 2): 2 * Pxy,
              (8, 1): Pyz, (8, 2): Pxz, (8, 3): Pxy, (9, 1): Pzz, (9, 3): 2 * Pxz})
    R, L = {}, {}
    for sgn, kf, kv, kw in ((-1.0, 0, 1, 2), (1.0, 9, 7, 8)):
        s = sgn * cf
        c = sgn * cs
        R.update({(0, kf): rho, (1, kf): s, (2, kf): s * Pxy / Pxx, (3, kf): s * Pxz / Pxx, (4, kf): 3 * Pxx,
                  (5, kf): 3 * Pxy, (6, kf): 3 * Pxz, (7, kf): Pyy + 2 * Pxy * Pxy / Pxx,
                  (8, kf): Pyz + 2 * Pxy * Pxz / Pxx, (9, kf): Pzz + 2 * Pxz * Pxz / Pxx})
        R.update({(2, kv): c, (5, kv): Pxx, (7, kv): 2 * Pxy, (8, kv): Pxz})
        R.update({(3, kw): c, (6, kw): Pxx, (8, kw): Pxy, (9, kw): 2 * Pxz})
        L.update({(kf, 1): 1 / (2 * s), (kf, 4): 1 / (6 * Pxx)})
        L.update({(kv, 1): -Pxy / (2 * c * Pxx), (kv, 2): 1 / (2 * c), (kv, 4): -Pxy / (2 * Pxx * Pxx),
                  (kv, 5): 1 / (2 * Pxx)})
        L.update({(kw, 1): -Pxz / (2 * c * Pxx), (kw, 3): 1 / (2 * c), (kw, 4): -Pxz / (2 * Pxx * Pxx),
                  (kw, 6): 1 / (2 * Pxx)})
    one = torch.ones_like(rho)
    R.update({(0, 3): one, (7, 4): one, (8, 5): one, (9, 6): one})
    L.update({(3, 0): one, (3, 4): -rho / (3 * Pxx),
              (4, 4): (4 * Pxy * Pxy / Pxx - Pyy) / (3 * Pxx), (4, 5): -2 * Pxy / Pxx, (4, 7): one,
              (5, 4): (4 * Pxy * Pxz / Pxx - Pyz) / (3 * Pxx), (5, 5): -Pxz / Pxx, (5, 6): -Pxy / Pxx,
              (5, 8): one,
              (6, 4): (4 * Pxz * Pxz / Pxx - Pzz) / (3 * Pxx), (6, 6): -2 * Pxz / Pxx, (6, 9): one})
    return _mat(A, shape, w), _mat(L, shape, w), _mat(R, shape, w)


def mc_limit(dL, dC, dR):
    m = torch.minimum(torch.minimum(2 * dL.abs(), dC.abs()), 2 * dR.abs())
    return torch.where(dL * dR > 0, torch.where(dC > 0, m, -m), torch.zeros_like(m))


def _ghost_index(n, bclo, bchi, g):
    """Source index and mirror flag of padded positions -g .. n+g-1."""
    src, mir = [], []
    for i in range(-g, n + g):
        m = False
        if i < 0:
            s = i + n if bclo == 0 else (0 if bclo == 1 else -1 - i)
            m = bclo == 2
        elif i >= n:
            s = i - n if bchi == 0 else (n - 1 if bchi == 1 else 2 * n - 1 - i)
            m = bchi == 2
        else:
            s = i
        src.append(s)
        mir.append(m)
    return torch.tensor(src), torch.tensor(mir)


def ghost_fill(U, ndim, bc):
    """Pad active dims with 2 ghost layers; reflect negates m_d and E_dt (t != d)."""
    V = U
    for d in range(ndim):
        axis = 3 - d  # tensor axis of dimension d ([c, z, y, x])
        n = V.shape[axis]
        src, mir = _ghost_index(n, bc[d][0], bc[d][1], 2)
        V = torch.index_select(V, axis, src)
        sign = torch.ones((NV, len(src)), dtype=U.dtype)
        flips = [1 + d] + [tidx(d, t) for t in range(3) if t != d]
        for k in flips:
            sign[k, mir] = -1.0
        shape = [NV, 1, 1, 1]
        shape[axis] = len(src)
        V = V * sign.reshape(shape)
    return V


def _flag_pad(flag, ndim, bc):
    F = flag
    for d in range(ndim):
        axis = 2 - d
        src, _ = _ghost_index(F.shape[axis], bc[d][0], bc[d][1], 2)
        F = torch.index_select(F, axis, src)
    return F


def hll(WL, WR, d):
    """HLL flux with S_L = min(u_L - cf_L, u_R - cf_R), S_R = max(u_L + cf_L, u_R + cf_R)."""
    nn = tidx(d, d)
    cL = torch.sqrt(3 * WL[nn] / WL[0])
    cR = torch.sqrt(3 * WR[nn] / WR[0])
    SL = torch.minimum(WL[1 + d] - cL, WR[1 + d] - cR)
    SR = torch.maximum(WL[1 + d] + cL, WR[1 + d] + cR)
    FL, FR = flux(WL, d), flux(WR, d)
    UL, UR = prim_to_cons(WL), prim_to_cons(WR)
    Fm = (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)
    return torch.where(SL >= 0, FL, torch.where(SR <= 0, FR, Fm))


def step_pass(U, ndim, dx, bc, dt, phi=None, flag=None):
    """One pass of the step (see msh_oracle.c step_pass).  flag: bool [nz, ny, nx] or None."""
    G = ghost_fill(U, ndim, bc)
    Wp = cons_to_prim(G)
    Fp = None if flag is None else _flag_pad(flag, ndim, bc)
    dU = torch.zeros_like(U)
    for d in range(ndim):
        axis = 3 - d
        # move the sweep axis last and the other padded dims to their interior range
        W = Wp
        Fl = Fp
        for e in range(ndim):
            if e != d:
                a = 3 - e
                W = W.narrow(a, 2, W.shape[a] - 4)
                if Fl is not None:
                    Fl = Fl.narrow(a - 1, 2, Fl.shape[a - 1] - 4)
        W = W.movedim(axis, -1)
        if Fl is not None:
            Fl = Fl.movedim(axis - 1, -1)
        wl = W[PERM[d]]                          # local frame, [10, ..., n+4]
        w0, wm, wpp = wl[..., 1:-1], wl[..., :-2], wl[..., 2:]   # cells -1 .. n
        dwL, dwC, dwR = w0 - wm, 0.5 * (wpp - wm), wpp - w0
        A, L, R = eigen_x(w0)
        mv = lambda M, v: torch.einsum("...ij,j...->i...", M, v)
        daL, daC, daR = mv(L, dwL), mv(L, dwC), mv(L, dwR)
        dam = mc_limit(daL, daC, daR)
        dwm = mv(R, dam)
        Adw = mv(A, dwm)
        nu = 0.5 * dt / dx[d]
        hi = w0 + 0.5 * dwm - nu * Adw
        lo = w0 - 0.5 * dwm - nu * Adw
        ok = (hi[0] > 0) & (lo[0] > 0) & (hi[4] > 0) & (lo[4] > 0)
        hi = torch.where(ok, hi, w0)
        lo = torch.where(ok, lo, w0)
        if Fl is not None:
            f0 = Fl[..., 1:-1]
            fm, fpp = Fl[..., :-2], Fl[..., 2:]
            lo = torch.where(f0 | fm, w0, lo)
            hi = torch.where(f0 | fpp, w0, hi)
        inv = [PERM[d].index(k) for k in range(NV)]
        lo, hi = lo[inv], hi[inv]                # back to global order
        F = hll(hi[..., :-1], lo[..., 1:], d)    # faces -1/2 .. n-1/2
        div = (F[..., 1:] - F[..., :-1]) / dx[d]
        dU = dU - div.movedim(-1, axis)
    Us = U + dt * dU
    if phi is not None:
        g = [1 if e < ndim else 0 for e in range(3)]
        nz, ny, nx = U.shape[1:]
        a = []
        for e in range(3):
            if e >= ndim:
                a.append(torch.zeros((nz, ny, nx), dtype=U.dtype))
                continue
            sl_p = [slice(g[2], g[2] + nz), slice(g[1], g[1] + ny), slice(g[0], g[0] + nx)]
            sl_m = list(sl_p)
            ax = 2 - e
            sl_p[ax] = slice(sl_p[ax].start + 1, sl_p[ax].stop + 1)
            sl_m[ax] = slice(sl_m[ax].start - 1, sl_m[ax].stop - 1)
            a.append(-(phi[tuple(sl_p)] - phi[tuple(sl_m)]) / (2 * dx[e]))
        rho = Us[0]
        m_star = [Us[1 + i] for i in range(3)]
        m_new = [m_star[i] + dt * rho * a[i] for i in range(3)]
        mbar = [0.5 * (m_star[i] + m_new[i]) for i in range(3)]
        comps = [Us[0]] + m_new + [None] * 6
        for i in range(3):
            for j in range(i, 3):
                comps[tidx(i, j)] = Us[tidx(i, j)] + dt * (mbar[i] * a[j] + a[i] * mbar[j])
        Us = torch.stack(comps)
    return Us


def realizable(U):
    W = cons_to_prim(U)
    m2 = W[4] * W[7] - W[5] * W[5]
    m3 = W[4] * (W[7] * W[9] - W[8] * W[8]) - W[5] * (W[5] * W[9] - W[8] * W[6]) + W[6] * (W[5] * W[8] - W[7] * W[6])
    return (U[0] > 0) & (W[4] > 0) & (m2 > 0) & (m3 > 0)


FALLBACK_PASSES = 4


def step(U, ndim, dx, bc, dt, phi=None):
    """The step with the a-posteriori first-order fallback: cells whose update is not
    realizable are tagged and the step recomputed with first-order faces around them, the
    tagged set growing for at most FALLBACK_PASSES passes.  The tags are found without
    gradients and are frozen in the differentiated pass."""
    with torch.no_grad():
        out = step_pass(U.detach(), ndim, dx, bc, dt, phi)
        bad = torch.zeros(U.shape[1:], dtype=torch.bool)
        for _ in range(FALLBACK_PASSES):
            new = ~realizable(out) & ~bad
            if not bool(new.any()):
                break
            bad = bad | new
            out = step_pass(U.detach(), ndim, dx, bc, dt, phi, bad)
    if bool(bad.any()):
        return step_pass(U, ndim, dx, bc, dt, phi, bad)
    return step_pass(U, ndim, dx, bc, dt, phi)


def adjoint_run(U0, ndim, dx, bc, dts, lamN, phi=None):
    """dL/dU0 = (dU_N/dU_0)^T lamN for the frozen schedule dts (reverse sweep over stored states)."""
    states = [torch.as_tensor(U0, dtype=torch.float64)]
    ph = None if phi is None else torch.as_tensor(phi, dtype=torch.float64)
    with torch.no_grad():
        for dt in dts:
            states.append(step(states[-1], ndim, dx, bc, float(dt), ph))
    lam = torch.as_tensor(lamN, dtype=torch.float64)
    for n in range(len(dts) - 1, -1, -1):
        Un = states[n].clone().requires_grad_(True)
        out = step(Un, ndim, dx, bc, float(dts[n]), ph)
        (g,) = torch.autograd.grad(out, Un, grad_outputs=lam)
        lam = g
    return lam, states[-1]
