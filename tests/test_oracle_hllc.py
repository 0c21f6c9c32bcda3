"""Pins of the oracle's HLLC flux for the ten-moment system and the scheme built on it:
consistency F(W, W) = f(W); the supersonic branches; an isolated contact (jumps in rho and
the transverse stresses only) resolved exactly, where HLL smears it; reduction to the
textbook gamma = 3 HLLC of gas dynamics (Toro's star states with E = E_nn / 2 and a passive
P_tt / rho) for diagonal stresses without transverse velocity; for random states the star
velocities agree on both sides of the contact and the star states average to the HLL state
(integral consistency); the scheme converges to the exact gamma = 3 Sod solution, keeps a
stationary contact exactly, resolves the moving contact more sharply than HLL and conserves
every total; the fallback passes restore realizability."""
import numpy as np
import pytest

from oracle import exact_riemann

HLLC, HLL = 3, 0
TI = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}


def ti(i, j):
    return TI[(min(i, j), max(i, j))]


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


def test_consistency(oracle):
    for W in _rand_states(np.random.default_rng(1), 20):
        for d in range(3):
            np.testing.assert_allclose(oracle.hllc_flux(W, W, d), oracle.flux(W, d), rtol=0, atol=1e-14)


def test_supersonic(oracle):
    rng = np.random.default_rng(2)
    Ws = _rand_states(rng, 10)
    for i in range(0, 10, 2):
        WL, WR = Ws[i].copy(), Ws[i + 1].copy()
        for d in range(3):
            L, R = WL.copy(), WR.copy()
            shift = 5.0 * max(np.sqrt(3 * L[ti(d, d)] / L[0]), np.sqrt(3 * R[ti(d, d)] / R[0])) + 2.0
            L[1 + d] += shift
            R[1 + d] += shift
            np.testing.assert_array_equal(oracle.hllc_flux(L, R, d), oracle.flux(L, d))
            L[1 + d] -= 2 * shift
            R[1 + d] -= 2 * shift
            np.testing.assert_array_equal(oracle.hllc_flux(L, R, d), oracle.flux(R, d))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_isolated_contact_is_exact(oracle, d):
    """W_R differs from W_L in rho and the stresses P_tt' transverse to d only (the fields
    the contact wave carries): the flux is the physical flux of the upwind side."""
    rng = np.random.default_rng(3 + d)
    t = [a for a in range(3) if a != d]
    for W in _rand_states(rng, 6):
        for sgn in (1.0, -1.0):
            L = W.copy()
            L[1 + d] = sgn * 0.3 * np.sqrt(3 * L[ti(d, d)] / L[0])  # subsonic: HLL is not upwind here
            R = L.copy()
            R[0] *= 2.5
            for (i, j) in ((t[0], t[0]), (t[0], t[1]), (t[1], t[1])):
                R[ti(i, j)] += 0.3 * L[ti(i, j)] if i == j else 0.05
            # keep the transverse block positive definite
            assert np.all(np.linalg.eigvalsh(np.array([[R[ti(a, b)] for b in range(3)] for a in range(3)])) > 0)
            want = oracle.flux(L if sgn > 0 else R, d)
            got = oracle.hllc_flux(L, R, d)
            assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
            assert np.abs(oracle.hll(L, R, d) - want).max() > 1e-3 * np.abs(want).max()


def _toro_hllc(WL, WR, d):
    """Gas-dynamics HLLC (Toro, Riemann Solvers, Sec. 10.4), gamma = 3, pressure P_dd,
    Davis speeds from c = sqrt(3 P_dd / rho); returns the fluxes of (rho, rho u, E) and of
    the passive density rho P_tt / rho for the transverse diagonal stresses."""
    g = 3.0
    nn = ti(d, d)
    rL, uL, pL = WL[0], WL[1 + d], WL[nn]
    rR, uR, pR = WR[0], WR[1 + d], WR[nn]
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    SL, SR = min(uL - cL, uR - cR), max(uL + cL, uR + cR)
    EL = 0.5 * rL * uL ** 2 + pL / (g - 1)
    ER = 0.5 * rR * uR ** 2 + pR / (g - 1)
    t = [a for a in range(3) if a != d]
    phis = [(ti(a, a)) for a in t]

    def U(r, u, E, W):
        return np.array([r, r * u, E] + [W[k] for k in phis])

    def F(r, u, p, E, W):
        return np.array([r * u, r * u * u + p, (E + p) * u] + [W[k] * u for k in phis])

    UL_, UR_ = U(rL, uL, EL, WL), U(rR, uR, ER, WR)
    FL_, FR_ = F(rL, uL, pL, EL, WL), F(rR, uR, pR, ER, WR)
    if SL >= 0:
        return FL_
    if SR <= 0:
        return FR_
    SM = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(r, u, p, E, W, S):
        f = r * (S - u) / (S - SM)
        return f * np.array([1.0, SM, E / r + (SM - u) * (SM + p / (r * (S - u)))] + [W[k] / r for k in phis])

    if SM >= 0:
        return FL_ + SL * (star(rL, uL, pL, EL, WL, SL) - UL_)
    return FR_ + SR * (star(rR, uR, pR, ER, WR, SR) - UR_)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_reduces_to_gas_dynamics_hllc(oracle, d):
    rng = np.random.default_rng(10 + d)
    for _ in range(20):
        WL, WR = np.zeros(10), np.zeros(10)
        for W in (WL, WR):
            W[0] = np.exp(rng.uniform(-1.5, 1.5))
            W[1 + d] = rng.uniform(-1.5, 1.5)
            for a in range(3):
                W[ti(a, a)] = np.exp(rng.uniform(-1.5, 1.0))
        F = oracle.hllc_flux(WL, WR, d)
        T = _toro_hllc(WL, WR, d)
        t = [a for a in range(3) if a != d]
        mine = np.array([F[0], F[1 + d], 0.5 * F[ti(d, d)]] + [F[ti(a, a)] for a in t])
        assert np.abs(mine - T).max() <= 1e-12 * np.abs(T).max()
        for a in t:  # no transverse momentum or shear stress appears
            assert F[1 + a] == 0.0 and F[ti(d, a)] == 0.0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_star_states(oracle, d):
    """Random states: the star velocities u*_i of both sides agree (the shear and normal
    stress pairs are solved consistently) and equal S_M along d, and the star states average
    to the HLL state: (S_M - S_L) U*_L + (S_R - S_M) U*_R = S_R U_R - S_L U_L - (F_R - F_L)."""
    rng = np.random.default_rng(30 + d)
    Ws = _rand_states(rng, 40)
    n_ok = 0
    for i in range(0, 40, 2):
        WL, WR = Ws[i], Ws[i + 1]
        ok, UsL, UsR, (SL, SM, SR) = oracle.hllc_star(WL, WR, d)
        if not ok:
            continue
        n_ok += 1
        vL, vR = UsL[1:4] / UsL[0], UsR[1:4] / UsR[0]
        np.testing.assert_allclose(vL, vR, rtol=1e-12, atol=1e-12)
        assert abs(vL[d] - SM) <= 1e-12 * (1 + abs(SM))
        UL, UR = oracle.prim_to_cons(WL.reshape(10, 1, 1, 1)).ravel(), oracle.prim_to_cons(WR.reshape(10, 1, 1, 1)).ravel()
        lhs = (SM - SL) * UsL + (SR - SM) * UsR
        rhs = SR * UR - SL * UL - (oracle.flux(WR, d) - oracle.flux(WL, d))
        assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()
    assert n_ok >= 15


def _sod(oracle, n, scheme):
    from paper_1210_5246_gb300 import inputs
    p = inputs.sod(n)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl, scheme=scheme)
    U, _, t, rc, _ = oracle.run(g, oracle.prim_to_cons(p.W), p.t_end)
    assert rc == 0 and t == p.t_end
    return oracle.cons_to_prim(U).reshape(10, -1), (np.arange(n) + 0.5) / n


def _contact_width(W, x):
    rl, rr = 0.6486437, 0.1707036
    m = (x > 0.45) & (x < 0.85)
    r = W[0][m]
    lo, hi = rr + 0.1 * (rl - rr), rr + 0.9 * (rl - rr)
    return int(np.sum((r > lo) & (r < hi)))


def test_sod_converges_and_contact_sharper_than_hll(oracle):
    errs = []
    for n in (128, 256, 512):
        W, x = _sod(oracle, n, HLLC)
        rho, _, _, _ = exact_riemann.sample((x - 0.5) / 0.2, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gamma=3.0)
        errs.append(np.abs(W[0] - rho).mean())
        if n >= 256:
            Wh, _ = _sod(oracle, n, HLL)
            assert _contact_width(W, x) < _contact_width(Wh, x)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3, errs


def test_stationary_contact_is_exact(oracle):
    n = 64
    W = np.zeros((10, 1, 1, n))
    x = (np.arange(n) + 0.5) / n
    W[0, 0, 0] = np.where(np.abs(x - 0.5) < 0.25, 2.0, 0.5)
    W[4] = 1.0
    W[7, 0, 0] = np.where(np.abs(x - 0.5) < 0.25, 0.7, 1.3)
    W[9] = 1.0
    W[5] = 0.1
    W[2] = 0.2
    g = oracle.Grid((n,), (0.0,), (1.0,), ((0, 0),), 0.5, scheme=HLLC)
    U, ns, _, rc, _ = oracle.run(g, oracle.prim_to_cons(W), np.inf, max_steps=40)
    assert rc == 0 and ns == 40
    np.testing.assert_allclose(oracle.cons_to_prim(U), W, rtol=1e-13, atol=1e-15)


def test_conservation_periodic(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.turb(n=12)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl, scheme=HLLC)
    U0 = oracle.prim_to_cons(p.W)
    U, ns, _, rc, _ = oracle.run(g, U0, np.inf, max_steps=5)
    assert rc == 0 and ns == 5
    t0, t1 = oracle.diagnostics(g, U0)[0], oracle.diagnostics(g, U)[0]
    scale = np.array([t0[0]] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)


@pytest.mark.parametrize("seed", [1, 13])
def test_fallback_restores_realizability(oracle, seed):
    from tests.test_oracle_pins import _extreme_tiny
    W = _extreme_tiny(seed)
    g = oracle.Grid((8,), (0,), (1,), ((0, 0),), 0.8, scheme=HLLC)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    A = oracle.step(g, U, dt)
    tot0 = oracle.diagnostics(g, U)[0]
    tot1, ok, _ = oracle.diagnostics(g, A)
    assert ok
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(tot0).max())
