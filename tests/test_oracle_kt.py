"""Pins of the oracle's Kurganov-Tadmor scheme (Sec. 3.2) against what the paper and the
mathematics fix: flux consistency H(u, u) = f(u); a uniform state is a fixed point;
conservation of all ten totals on a periodic grid; convergence to the exact gamma = 3 Sod
solution; a contact no sharper than the MUSCL-Hancock scheme's (Sec. 4.1); reduction of a density bump in uniform flow to the scalar
KT scheme, restated here; mirror symmetry."""
import numpy as np
import pytest

from oracle import exact_riemann

KT = 1


def _rand_states(rng, m):
    W = np.zeros((m, 10))
    W[:, 0] = np.exp(rng.uniform(-1, 1, m))
    W[:, 1:4] = rng.uniform(-1, 1, (m, 3))
    for i in range(m):
        A = np.tril(rng.normal(0, 0.3, (3, 3)))
        A[np.diag_indices(3)] = rng.uniform(0.3, 1.0, 3)
        P = A @ A.T
        W[i, 4:] = [P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]]
    return W


def test_flux_consistency(oracle):
    rng = np.random.default_rng(1)
    for W in _rand_states(rng, 20):
        for d in range(3):
            np.testing.assert_array_equal(oracle.kt_flux(W, W, d), oracle.flux(W, d))


def test_kt_flux_formula(oracle):
    """H = (f(WL) + f(WR))/2 - a (U(WR) - U(WL))/2 with a = max |u_d| + sqrt(3 P_dd / rho)."""
    rng = np.random.default_rng(2)
    S = _rand_states(rng, 12)
    nn = {0: 4, 1: 7, 2: 9}
    for WL, WR in zip(S[:6], S[6:]):
        for d in range(3):
            a = max(abs(W[1 + d]) + np.sqrt(3 * W[nn[d]] / W[0]) for W in (WL, WR))
            UL = oracle.prim_to_cons(WL.reshape(10, 1)).ravel()
            UR = oracle.prim_to_cons(WR.reshape(10, 1)).ravel()
            H = 0.5 * (oracle.flux(WL, d) + oracle.flux(WR, d)) - 0.5 * a * (UR - UL)
            np.testing.assert_allclose(oracle.kt_flux(WL, WR, d), H, rtol=1e-13, atol=1e-13)


def test_uniform_state_is_fixed(oracle):
    W = _rand_states(np.random.default_rng(3), 1)[0]
    for n, bc in [((16,), ((0, 0),)), ((8, 6), ((1, 1), (0, 0))), ((5, 4, 6), ((0, 0), (2, 2), (1, 1)))]:
        shape = (10,) + (1,) * (3 - len(n)) + tuple(reversed(n))
        Wf = np.broadcast_to(W.reshape((10,) + (1,) * 3), shape).copy()
        if any(b[0] == 2 for b in bc):
            Wf[1:4] = 0.0
            Wf[5], Wf[6], Wf[8] = 0.0, 0.0, 0.0  # reflect images of a uniform state: no shear
        g = oracle.Grid(n, (0,) * len(n), (1,) * len(n), bc, 0.4, scheme=KT)
        U = oracle.prim_to_cons(Wf)
        U1 = oracle.step(g, U, 1e-3)
        np.testing.assert_allclose(U1, U, rtol=1e-15, atol=1e-15)


def test_conservation_periodic(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.turb(n=12)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, 0.4, scheme=KT)
    U0 = oracle.prim_to_cons(p.W)
    U, ns, _, rc, _ = oracle.run(g, U0, np.inf, max_steps=6)
    assert rc == 0 and ns == 6
    t0, t1 = oracle.diagnostics(g, U0)[0], oracle.diagnostics(g, U)[0]
    scale = np.array([t0[0]] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)


def _sod(oracle, n, scheme, cfl=0.4):
    from paper_1210_5246_gb300 import inputs
    p = inputs.sod(n)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, cfl, scheme=scheme)
    U, ns, t, rc, _ = oracle.run(g, oracle.prim_to_cons(p.W), p.t_end)
    assert rc == 0 and t == p.t_end
    return oracle.cons_to_prim(U).reshape(10, -1), (np.arange(n) + 0.5) / n


def test_sod_converges_to_exact_gamma3(oracle):
    errs = []
    for n in (128, 256, 512):
        W, x = _sod(oracle, n, KT)
        rho, _, _, _ = exact_riemann.sample((x - 0.5) / 0.2, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gamma=3.0)
        errs.append(np.abs(W[0] - rho).mean())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 6e-3


def _contact_width(W, x):
    """Cells with density between 10 % and 90 % of the jump across the contact (x near 0.62)."""
    rl, rr = 0.6486437, 0.1707036  # exact gamma = 3 star densities left and right of the contact
    m = (x > 0.45) & (x < 0.85)
    r = W[0][m]
    lo, hi = rr + 0.1 * (rl - rr), rr + 0.9 * (rl - rr)
    return int(np.sum((r > lo) & (r < hi)))


def test_contact_not_sharper_than_muscl_hancock(oracle):
    """Sec. 4.1 finds the KT contact about twice as wide as that of the characteristic
    scheme with HLLC, which resolves contacts.  HLL (the flux of the hot path) does not, so
    here KT's contact is no sharper than MUSCL-Hancock's and both spread over a few cells."""
    Wk, x = _sod(oracle, 256, KT)
    Wm, _ = _sod(oracle, 256, 0)
    wk, wm = _contact_width(Wk, x), _contact_width(Wm, x)
    assert wk >= wm and 3 <= wm <= 12 and wk <= 12, (wk, wm)


def _scalar_kt(rho, u, P, dx, dt, steps):
    """The scalar scheme a density bump in uniform velocity u and dispersion P follows:
    rho_t + (rho u)_x = 0 with MC-limited face values, H = (rho- + rho+) u / 2
    - a (rho+ - rho-) / 2, a = |u| + sqrt(3 P / min(rho-, rho+)), Heun's RK2 (periodic)."""
    def mc(dl, dc, dr):
        m = np.minimum(2 * np.abs(dl), np.minimum(np.abs(dc), 2 * np.abs(dr)))
        return np.where(dl * dr > 0, np.sign(dc) * m, 0.0)

    def L(r):
        rm, rp = np.roll(r, 1), np.roll(r, -1)
        s = mc(r - rm, 0.5 * (rp - rm), rp - r)
        left = r + 0.5 * s              # value on the left side of face i+1/2
        right = np.roll(r - 0.5 * s, -1)  # value on its right side (from cell i+1)
        a = np.abs(u) + np.sqrt(3 * P / np.minimum(left, right))
        H = 0.5 * (left + right) * u - 0.5 * a * (right - left)
        return -(H - np.roll(H, 1)) / dx

    for _ in range(steps):
        r1 = rho + dt * L(rho)
        rho = 0.5 * (rho + (r1 + dt * L(r1)))
    return rho


def test_density_bump_reduces_to_scalar_kt(oracle):
    n, u, P = 64, 0.7, 0.3
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.exp(-((x - 0.4) / 0.08) ** 2) + 0.2 * (np.abs(x - 0.75) < 0.06)
    W = np.zeros((10, 1, 1, n))
    W[0, 0, 0] = rho
    W[1] = u
    W[4] = W[7] = W[9] = P
    g = oracle.Grid((n,), (0.0,), (1.0,), ((0, 0),), 0.4, scheme=KT)
    dt = 0.3 / n
    U = oracle.prim_to_cons(W)
    for _ in range(20):
        U = oracle.step(g, U, dt)
    ref = _scalar_kt(rho, u, P, 1.0 / n, dt, 20)
    np.testing.assert_allclose(U[0].ravel(), ref, rtol=1e-12, atol=1e-12)
    Wn = oracle.cons_to_prim(U)
    np.testing.assert_allclose(Wn[1].ravel(), u, rtol=1e-12)
    np.testing.assert_allclose(Wn[4].ravel(), P, rtol=1e-11)


def test_mirror_symmetry(oracle):
    rng = np.random.default_rng(7)
    n = 40
    W = np.zeros((10, 1, 1, n))
    S = _rand_states(rng, n)
    W[:, 0, 0, :] = S.T
    g = oracle.Grid((n,), (0.0,), (1.0,), ((1, 2),), 0.4, scheme=KT)
    gm = oracle.Grid((n,), (0.0,), (1.0,), ((2, 1),), 0.4, scheme=KT)
    flip = np.ones(10)
    flip[[1, 5, 6]] = -1  # u_x, P_xy, P_xz change sign under x -> -x
    Wm = W[:, :, :, ::-1] * flip[:, None, None, None]
    U, _, _, rc, _ = oracle.run(g, oracle.prim_to_cons(W), np.inf, max_steps=5)
    Um, _, _, rcm, _ = oracle.run(gm, oracle.prim_to_cons(Wm), np.inf, max_steps=5)
    assert rc == rcm == 0
    flipU = np.ones(10)
    flipU[[1, 5, 6]] = -1
    np.testing.assert_allclose(Um[:, :, :, ::-1] * flipU[:, None, None, None], U, rtol=1e-13, atol=1e-13)
