"""Independent brute-force step for tiny grids (test helper, pins the oracle).

Nothing here uses the oracle's closed forms.  The physical flux is the velocity moment
of a Gaussian distribution (zero heat flux closure, Sec. 2), by Gauss-Hermite quadrature
(``flux_gh``) or Isserlis' theorem (``flux_moments``, pinned to the quadrature); the
primitive Jacobian A = (dU/dW)^-1 dF/dW comes from complex-step
differentiation of that flux; wave speeds are numerical eigenvalues of A; eigenvectors
are numerical null spaces of (A - lambda I).  Inside a degenerate eigenspace the basis
is fixed by the axis-aligned convention of the paper's printed eigenvectors (eq
righteigvec): the basis vectors restrict to unit vectors on the transverse velocity
components (shear waves) and on (rho, P_t1t1, P_t1t2, P_t2t2) (contact waves).  The MC
limiter is odd and positively homogeneous, so any per-vector scaling gives the same step.
"""
from __future__ import annotations

import numpy as np

_gh_x, _gh_w = np.polynomial.hermite_e.hermegauss(3)
_gh_w = _gh_w / _gh_w.sum()
TI = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}


def tidx(i, j):
    return TI[(min(i, j), max(i, j))]


def _chol3(S):
    """Cholesky of a (possibly complex-symmetric) 3x3 matrix, without conjugation."""
    L = np.zeros((3, 3), dtype=S.dtype)
    for i in range(3):
        for j in range(i + 1):
            s = S[i, j] - sum(L[i, k] * L[j, k] for k in range(j))
            L[i, j] = np.sqrt(s) if i == j else s / L[j, j]
    return L


def cons(W):
    W = np.asarray(W)
    U = np.zeros(10, dtype=W.dtype)
    rho, u = W[0], W[1:4]
    U[0] = rho
    U[1:4] = rho * u
    for i in range(3):
        for j in range(i, 3):
            U[tidx(i, j)] = W[tidx(i, j)] + rho * u[i] * u[j]
    return U


def flux_gh(W, d):
    """Flux along d as moments of f = rho N(u, P/rho): rho<v_d>, rho<v_i v_d>, rho<v_i v_j v_d>."""
    W = np.asarray(W)
    rho, u = W[0], W[1:4]
    S = np.empty((3, 3), dtype=W.dtype)
    for i in range(3):
        for j in range(3):
            S[i, j] = W[tidx(i, j)] / rho
    L = _chol3(S)
    F = np.zeros(10, dtype=W.dtype)
    for a, wa in zip(_gh_x, _gh_w):
        for b, wb in zip(_gh_x, _gh_w):
            for c, wc in zip(_gh_x, _gh_w):
                v = u + L @ np.array([a, b, c])
                w = wa * wb * wc * rho
                F[0] += w * v[d]
                for i in range(3):
                    F[1 + i] += w * v[i] * v[d]
                    for j in range(i, 3):
                        F[tidx(i, j)] += w * v[i] * v[j] * v[d]
    return F


def flux_moments(W, d):
    """Same moments from Isserlis' theorem for a Gaussian with mean u, covariance S = P/rho:
    <v_i v_j v_k> = u_i u_j u_k + u_i S_jk + u_j S_ik + u_k S_ij.  Polynomial in W, so it
    also holds for the non-positive-definite face states a Hancock predictor can produce
    (the quadrature needs a Cholesky factor)."""
    W = np.asarray(W)
    rho, u = W[0], W[1:4]
    S = [[W[tidx(i, j)] / rho for j in range(3)] for i in range(3)]
    F = np.zeros(10, dtype=W.dtype)
    F[0] = rho * u[d]
    for i in range(3):
        F[1 + i] = rho * (u[i] * u[d] + S[i][d])
        for j in range(i, 3):
            F[tidx(i, j)] = rho * (u[i] * u[j] * u[d] + u[i] * S[j][d] + u[j] * S[i][d] + u[d] * S[i][j])
    return F


def jac_cs(fun, W, h=1e-30):
    """Complex-step Jacobian d fun / d W (exact to rounding)."""
    W = np.asarray(W, dtype=np.float64)
    J = np.zeros((10, 10))
    for k in range(10):
        Wc = W.astype(np.complex128)
        Wc[k] += 1j * h
        J[:, k] = np.imag(fun(Wc)) / h
    return J


def prim_jacobian(W, d):
    dU = jac_cs(cons, W)
    dF = jac_cs(lambda w: flux_moments(w, d), W)
    return np.linalg.solve(dU, dF)


def _free_sets(d):
    t = [a for a in range(3) if a != d]
    shear = [1 + t[0], 1 + t[1]]
    contact = [0, tidx(t[0], t[0]), tidx(t[0], t[1]), tidx(t[1], t[1])]
    return shear, contact


def eigen(W, d):
    """(A, lam, R) with numerically computed eigen-decomposition (columns of R)."""
    A = prim_jacobian(W, d)
    lam = np.sort(np.linalg.eigvals(A).real)
    groups = []
    for v in lam:
        if groups and abs(v - groups[-1][0]) < 1e-7 * (1 + abs(v)):
            groups[-1][1] += 1
        else:
            groups.append([v, 1])
    shear, contact = _free_sets(d)
    cols, lams = [], []
    for v, m in groups:
        M = A - v * np.eye(10)
        _, s, Vt = np.linalg.svd(M)
        N = Vt[-m:].T  # null space basis
        if m == 1:
            B = N
        else:
            S = contact if m == 4 else shear
            B = N @ np.linalg.inv(N[S, :])
        for k in range(m):
            cols.append(B[:, k])
            lams.append(v)
    return A, np.array(lams), np.array(cols).T


def mc(dL, dC, dR):
    out = np.zeros_like(dC)
    ok = dL * dR > 0
    m = np.minimum(np.minimum(2 * np.abs(dL), np.abs(dC)), 2 * np.abs(dR))
    out[ok] = np.sign(dC[ok]) * m[ok]
    return out


def prim(U):
    W = np.zeros(10)
    rho = U[0]
    W[0] = rho
    W[1:4] = U[1:4] / rho
    for i in range(3):
        for j in range(i, 3):
            W[tidx(i, j)] = U[tidx(i, j)] - rho * W[1 + i] * W[1 + j]
    return W


def realizable(U):
    if not U[0] > 0:
        return False
    W = prim(U)
    P = np.array([[W[4], W[5], W[6]], [W[5], W[7], W[8]], [W[6], W[8], W[9]]])
    return bool(P[0, 0] > 0 and np.linalg.det(P[:2, :2]) > 0 and np.linalg.det(P) > 0)


def recon(Wm, W0, Wp, d, dtdx, check=True):
    A, lam, R = eigen(W0, d)
    Linv = np.linalg.inv(R)
    dL, dR, dC = W0 - Wm, Wp - W0, 0.5 * (Wp - Wm)
    dm = R @ mc(Linv @ dL, Linv @ dC, Linv @ dR)
    hi = W0 + 0.5 * dm - 0.5 * dtdx * (A @ dm)
    lo = W0 - 0.5 * dm - 0.5 * dtdx * (A @ dm)
    return check_states(W0, d, lo, hi) if check else (lo, hi)


def check_states(W0, d, lo, hi):
    """First-order states where a face state has rho <= 0 or P_dd <= 0."""
    nn = tidx(d, d)
    if not (hi[0] > 0 and lo[0] > 0 and hi[nn] > 0 and lo[nn] > 0):
        return W0.copy(), W0.copy()
    return lo, hi


def transverse(Wm, W0, Wp, t, dtdx):
    """Corner-transport-upwind transverse term along t, wave by wave on the numerical
    eigen-system: -(dt / 2dx_t) sum_a lam_a a_a R^a with a_a the amplitude of the upwind
    one-sided difference (backward for lam_a > 0, forward otherwise)."""
    _, lam, R = eigen(W0, t)
    Linv = np.linalg.inv(R)
    aL, aR = Linv @ (W0 - Wm), Linv @ (Wp - W0)
    a = np.where(lam > 0, aL, aR)
    return -0.5 * dtdx * (R @ (lam * a))


def recon_upwind(Wm, W0, Wp, d, dtdx, check=True):
    """Upwind characteristic tracing (eqs 40-43 with eq 41 in the mirror form of eq 40),
    summed per wave: with a = R^-1 dw^m, nu = dt / 2dx,
      hi = W0 + sum_a (1/2 - nu s_a) a_a R^a,  s_a = lam_a if lam_a > 0 else max(lam_max, 0)
      lo = W0 + sum_a (-1/2 - nu t_a) a_a R^a, t_a = lam_a if lam_a < 0 else min(lam_min, 0)."""
    _, lam, R = eigen(W0, d)
    Linv = np.linalg.inv(R)
    dL, dR, dC = W0 - Wm, Wp - W0, 0.5 * (Wp - Wm)
    a = mc(Linv @ dL, Linv @ dC, Linv @ dR)
    nu = 0.5 * dtdx
    s = np.where(lam > 0, lam, max(lam.max(), 0.0))
    t = np.where(lam < 0, lam, min(lam.min(), 0.0))
    hi = W0 + R @ ((0.5 - nu * s) * a)
    lo = W0 + R @ ((-0.5 - nu * t) * a)
    return check_states(W0, d, lo, hi) if check else (lo, hi)


def speeds(W, d):
    lam = np.linalg.eigvals(prim_jacobian(W, d)).real
    return lam.min(), lam.max()


def hll(WL, WR, d):
    aL, bL = speeds(WL, d)
    aR, bR = speeds(WR, d)
    SL, SR = min(aL, aR), max(bL, bR)
    FL, FR = flux_moments(WL, d).real, flux_moments(WR, d).real
    if SL >= 0:
        return FL
    if SR <= 0:
        return FR
    UL, UR = cons(WL), cons(WR)
    return (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)


def roe(WL, WR, d):
    """Roe-type flux from the numerically computed eigen-system of the primitive Jacobian at
    the arithmetic mean state: F = (f_L + f_R)/2 - (1/2) (dU/dW) R |Lambda| R^-1 (W_R - W_L),
    Harten's fix |l| -> (l^2 + delta^2) / (2 delta) below delta = 0.1 sqrt(3 P_dd / rho) on the
    slowest and fastest waves only."""
    Wm = 0.5 * (WL + WR)
    _, lam, R = eigen(Wm, d)
    a = np.linalg.solve(R, WR - WL)
    delta = 0.1 * np.sqrt(3 * Wm[tidx(d, d)] / Wm[0])
    al = np.abs(lam)
    for k in (0, len(lam) - 1):
        if al[k] < delta:
            al[k] = (lam[k] ** 2 + delta ** 2) / (2 * delta)
    dW = R @ (al * a)
    dUdW = jac_cs(cons, Wm).real
    FL, FR = flux_moments(WL, d).real, flux_moments(WR, d).real
    return 0.5 * (FL + FR) - 0.5 * dUdW @ dW


def _pad_line(Uline, bclo, bchi, d):
    """Two ghost cells each side along a line of conserved states (n, 10)."""
    n = Uline.shape[0]
    out = np.zeros((n + 4, 10))
    out[2:-2] = Uline
    flip = np.ones(10)
    flip[1 + d] = -1
    for t in range(3):
        if t != d:
            flip[tidx(d, t)] = -1
    for g in (1, 2):
        # lower side: ghost index -g
        if bclo == 0:
            out[2 - g] = Uline[n - g]
        elif bclo == 1:
            out[2 - g] = Uline[0]
        else:
            out[2 - g] = Uline[g - 1] * flip
        if bchi == 0:
            out[n + 1 + g] = Uline[g - 1]
        elif bchi == 1:
            out[n + 1 + g] = Uline[n - 1]
        else:
            out[n + 1 + g] = Uline[n - g] * flip
    return out


def _pad_grid(U, ndim, bc):
    """Conserved array with two ghost layers on every active axis, filled axis by axis with
    the rules of _pad_line (corner ghosts combine the rules of both axes)."""
    out = np.asarray(U, dtype=np.float64)
    for d in range(ndim):
        ax = 3 - d  # array axis of dimension d in [10][z][y][x]
        moved = np.moveaxis(out, ax, -1)  # [10, ..., n_d]
        rows = int(np.prod(moved.shape[1:-1]))
        lines = moved.reshape(10, rows, moved.shape[-1])
        padded = np.zeros((10, rows, moved.shape[-1] + 4))
        for r in range(rows):
            padded[:, r, :] = _pad_line(lines[:, r, :].T, bc[d][0], bc[d][1], d).T
        shape = list(moved.shape)
        shape[-1] += 4
        out = np.moveaxis(padded.reshape(shape), -1, ax)
    return out


def step(U, ndim, dx, bc, dt, phi=None, flux="hll", ctu=False):
    """One unsplit step on a tiny grid, with the a-posteriori fallback: if the second-order
    update leaves cells non-realizable, recompute with first-order face states on every
    face of those cells.  flux="roe": upwind tracing (recon_upwind) and the Roe-type flux
    on every face except the first-order faces of a fallback pass, which take HLL.
    ctu=True: every face state along d takes the transverse terms along the other axes
    (``transverse``) before the face-state check."""
    Un = _step_pass(U, ndim, dx, bc, dt, phi, None, flux, ctu)
    nz, ny, nx = Un.shape[1:]
    bad = np.zeros((nz, ny, nx), dtype=bool)
    for _ in range(5):  # the first check plus at most four fallback passes
        new = np.zeros_like(bad)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    new[z, y, x] = (not realizable(Un[:, z, y, x])) and not bad[z, y, x]
        if not new.any() or _ == 4:
            break
        bad |= new
        Un = _step_pass(U, ndim, dx, bc, dt, phi, bad, flux, ctu)
    return Un


def _step_pass(U, ndim, dx, bc, dt, phi, bad, flux="hll", ctu=False):
    U = np.asarray(U, dtype=np.float64)
    dU = np.zeros_like(U)
    nz, ny, nx = U.shape[1:]
    shape = (nx, ny, nz)
    g = [2 if d < ndim else 0 for d in range(3)]
    Wpad = None
    if ctu and ndim > 1:
        Up = _pad_grid(U, ndim, bc)
        Wpad = np.zeros_like(Up)
        for z in range(Up.shape[1]):
            for y in range(Up.shape[2]):
                for x in range(Up.shape[3]):
                    Wpad[:, z, y, x] = prim(Up[:, z, y, x])

    def T(t, q):  # transverse term along t of the padded cell q = (x, y, z)
        qm, qp = list(q), list(q)
        qm[t] -= 1
        qp[t] += 1
        return transverse(Wpad[:, qm[2], qm[1], qm[0]], Wpad[:, q[2], q[1], q[0]], Wpad[:, qp[2], qp[1], qp[0]],
                          t, dt / dx[t])
    for d in range(ndim):
        other = [a for a in range(3) if a != d]
        for j1 in range(shape[other[0]]):
            for j2 in range(shape[other[1]]):
                idx = [None, None, None]
                idx[other[0]], idx[other[1]] = j1, j2
                line = []
                for i in range(shape[d]):
                    idx[d] = i
                    line.append(U[:, idx[2], idx[1], idx[0]])
                P = _pad_line(np.array(line), bc[d][0], bc[d][1], d)
                Wl = [prim(u) for u in P]
                n = shape[d]
                rc = recon_upwind if flux == "roe" else recon
                if Wpad is None:
                    faces = [list(rc(Wl[k - 1], Wl[k], Wl[k + 1], d, dt / dx[d])) for k in range(1, n + 3)]
                else:
                    faces = []
                    for k in range(1, n + 3):
                        lo, hi = rc(Wl[k - 1], Wl[k], Wl[k + 1], d, dt / dx[d], check=False)
                        q = [0, 0, 0]
                        q[d] = k
                        q[other[0]], q[other[1]] = j1 + g[other[0]], j2 + g[other[1]]
                        tr = sum(T(t, q) for t in range(ndim) if t != d)
                        faces.append(list(check_states(Wl[k], d, lo + tr, hi + tr)))
                if bad is not None:
                    # flag of padded cell k (k = i + 2 for cell i), ghosts take their source cell's
                    def flag(k):
                        i = k - 2
                        if i < 0:
                            i = i + n if bc[d][0] == 0 else (0 if bc[d][0] == 1 else -1 - i)
                        elif i >= n:
                            i = i - n if bc[d][1] == 0 else (n - 1 if bc[d][1] == 1 else 2 * n - 1 - i)
                        idx2 = list(idx)
                        idx2[d] = i
                        return bad[idx2[2], idx2[1], idx2[0]]
                first = set()
                if bad is not None:
                    for k in range(1, n + 2):  # face between padded cells k and k+1
                        if flag(k) or flag(k + 1):
                            faces[k - 1][1] = Wl[k].copy()
                            faces[k][0] = Wl[k + 1].copy()
                            first.add(k)

                def F(k):  # flux through the face between padded cells k and k+1
                    f = roe if flux == "roe" and k not in first else hll
                    return f(faces[k - 1][1], faces[k][0], d)
                # faces[k-1] = (lo, hi) of padded cell k, cell i <-> padded i+2
                for i in range(n):
                    Fm, Fp = F(i + 1), F(i + 2)
                    idx[d] = i
                    dU[:, idx[2], idx[1], idx[0]] -= (Fp - Fm) / dx[d]
    Un = U + dt * dU
    if phi is not None:
        g = [1 if d < ndim else 0 for d in range(3)]
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    c = (z + g[2], y + g[1], x + g[0])
                    a = np.zeros(3)
                    for d in range(ndim):
                        e = [0, 0, 0]
                        e[2 - d] = 1
                        cp = tuple(c[k] + e[k] for k in range(3))
                        cm = tuple(c[k] - e[k] for k in range(3))
                        a[d] = -(phi[cp] - phi[cm]) / (2 * dx[d])
                    u = Un[:, z, y, x]
                    m_old = u[1:4].copy()
                    m_new = m_old + dt * u[0] * a
                    mbar = 0.5 * (m_old + m_new)
                    for i in range(3):
                        for j in range(i, 3):
                            u[tidx(i, j)] += dt * (mbar[i] * a[j] + a[i] * mbar[j])
                    u[1:4] = m_new
    return Un


def cfl_dt(U, ndim, dx, cfl, ctu=False):
    nz, ny, nx = U.shape[1:]
    smax = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                W = prim(U[:, z, y, x])
                s = 0.0
                for d in range(ndim):
                    a, b = speeds(W, d)
                    sd = max(abs(a), abs(b)) / dx[d]
                    s = max(s, sd) if ctu else s + sd
                smax = max(smax, s)
    return cfl / smax
