"""Pins of the oracle's Roe-type flux (the characteristic scheme with a linearised upwind
flux): consistency F(W, W) = f(W); upwinding (a supersonic state gets the upwind flux
exactly); a stationary contact is kept exactly (the contact waves have speed 0 and are not
entropy-fixed) while HLL smears it; the moving contact of the gamma = 3 Sod problem is
sharper than HLL's; convergence to the exact Sod solution; conservation of every total."""
import numpy as np
import pytest

from oracle import exact_riemann

ROE, HLL = 2, 0


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
            np.testing.assert_allclose(oracle.roe_flux(W, W, d), oracle.flux(W, d), rtol=0, atol=1e-15)


def test_supersonic_upwinding(oracle):
    """With every wave speed of the mean state positive (negative), the flux is the left
    (right) physical flux exactly in linear problems; for close states to O(jump^2)."""
    rng = np.random.default_rng(2)
    for W in _rand_states(rng, 8):
        W = W.copy()
        W[1] = 3.0 + 3 * np.sqrt(3 * W[4] / W[0])  # u > cf: all waves to the right
        V = W * (1 + 1e-4 * rng.normal(size=10))
        F = oracle.roe_flux(W, V, 0)
        assert np.abs(F - oracle.flux(W, 0)).max() <= 1e-6 * np.abs(oracle.flux(W, 0)).max()
        W2, V2 = W.copy(), V.copy()
        W2[1], V2[1] = -W[1], -V[1]
        F2 = oracle.roe_flux(W2, V2, 0)
        assert np.abs(F2 - oracle.flux(V2, 0)).max() <= 1e-6 * np.abs(oracle.flux(V2, 0)).max()


def _contact(oracle, scheme, n=64, steps=40, u=0.0):
    W = np.zeros((10, 1, 1, n))
    x = (np.arange(n) + 0.5) / n
    W[0, 0, 0] = np.where(np.abs(x - 0.5) < 0.25, 2.0, 0.5)
    W[1] = u
    W[4] = W[7] = W[9] = 1.0
    W[5] = 0.1
    g = oracle.Grid((n,), (0.0,), (1.0,), ((0, 0),), 0.5, scheme=scheme)
    U, ns, _, rc, _ = oracle.run(g, oracle.prim_to_cons(W), np.inf, max_steps=steps)
    assert rc == 0 and ns == steps
    return oracle.cons_to_prim(U)[0, 0, 0], W[0, 0, 0]


def test_stationary_contact_is_exact(oracle):
    rho, rho0 = _contact(oracle, ROE)
    np.testing.assert_allclose(rho, rho0, rtol=1e-13)
    rho_h, _ = _contact(oracle, HLL)
    assert np.abs(rho_h - rho0).max() > 0.1  # HLL diffuses the same contact


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


def test_sod_contact_sharper_than_hll(oracle):
    Wr, x = _sod(oracle, 256, ROE)
    Wh, _ = _sod(oracle, 256, HLL)
    assert _contact_width(Wr, x) < _contact_width(Wh, x), (_contact_width(Wr, x), _contact_width(Wh, x))


def test_sod_converges_to_exact_gamma3(oracle):
    errs = []
    for n in (128, 256, 512):
        W, x = _sod(oracle, n, ROE)
        rho, _, _, _ = exact_riemann.sample((x - 0.5) / 0.2, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gamma=3.0)
        errs.append(np.abs(W[0] - rho).mean())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3, errs


def test_conservation_periodic(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.turb(n=12)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl, scheme=ROE)
    U0 = oracle.prim_to_cons(p.W)
    U, ns, _, rc, _ = oracle.run(g, U0, np.inf, max_steps=5)
    assert rc == 0 and ns == 5
    t0, t1 = oracle.diagnostics(g, U0)[0], oracle.diagnostics(g, U)[0]
    scale = np.array([t0[0]] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)


def test_roe_flux_matches_bruteforce(oracle):
    """Against the flux built from a numerically computed eigen-system (SVD null spaces of
    the complex-step Jacobian), for near and far state pairs in every direction."""
    from tests import bruteforce as BF
    rng = np.random.default_rng(5)
    Ws = _rand_states(rng, 12)
    for i in range(0, 12, 2):
        WL = Ws[i]
        for WR in (WL * (1 + 0.05 * rng.normal(size=10)), Ws[i + 1]):
            for d in range(3):
                F, B = oracle.roe_flux(WL, WR, d), BF.roe(WL, WR, d)
                assert np.abs(F - B).max() <= 1e-9 * (np.abs(B).max() + 1), (d, np.abs(F - B).max())


@pytest.mark.parametrize("seed", [1, 13])
def test_fallback_takes_hll_on_first_order_faces(oracle, seed):
    """Extreme states: the Roe-type second-order update leaves cells non-realizable; the
    fallback passes (first-order states and the HLL flux on every face of a tagged cell, the
    Roe-type flux elsewhere) make it realizable and conservative, and match the brute-force
    step with the same rule."""
    from tests import bruteforce as BF
    from tests.test_oracle_pins import _extreme_tiny
    W = _extreme_tiny(seed)
    g = oracle.Grid((8,), (0,), (1,), ((0, 0),), 0.8, scheme=ROE)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    assert not oracle.diagnostics(g, oracle.step_second_order_only(g, U, dt))[1]
    A = oracle.step(g, U, dt)
    tot0 = oracle.diagnostics(g, U)[0]
    tot1, ok, _ = oracle.diagnostics(g, A)
    assert ok
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(tot0).max())
    B = BF.step(U, 1, [1 / 8] * 3, ((0, 0),), dt, flux="roe")
    scale = np.abs(B).reshape(10, -1).max(axis=1)[:, None, None, None] + 1e-300
    assert np.max(np.abs(A - B) / scale) < 1e-10


def test_kt_contact_wider_than_roe(oracle):
    """Sec. 4.1 finds the central scheme's contact about twice as wide as that of a
    contact-resolving upwind flux: the Kurganov-Tadmor contact of the gamma = 3 Sod problem
    is wider than the Roe-type one at every resolution."""
    KT = 1
    for n in (256, 512):
        Wr, x = _sod(oracle, n, ROE)
        Wk, _ = _sod(oracle, n, KT)
        assert _contact_width(Wk, x) > _contact_width(Wr, x)


def _triples(rng, m):
    """m (Wm, W0, Wp) triples of nearby realizable states."""
    return [[W * (1 + 0.05 * rng.normal(size=10)) for _ in range(3)] for W in _rand_states(rng, m)]


@pytest.mark.parametrize("d", [0, 1, 2])
def test_upwind_tracing_matches_bruteforce(oracle, d):
    """The oracle's tracing, written as eqs 40-43, equals the per-wave form on a numerically
    computed eigen-system, subsonic and supersonic."""
    from tests import bruteforce as BF
    rng = np.random.default_rng(20 + d)
    for Wm, W0, Wp in _triples(rng, 6):
        for shift in (0.0, 4.0, -4.0):
            s = np.zeros(10)
            s[1 + d] = shift * np.sqrt(3 * W0[4 + [0, 3, 5][d]] / W0[0])
            lo, hi = oracle.reconstruct_upwind(Wm + s, W0 + s, Wp + s, d, 0.3)
            blo, bhi = BF.recon_upwind(Wm + s, W0 + s, Wp + s, d, 0.3)
            scale = np.abs(W0 + s).max()
            assert np.abs(lo - blo).max() <= 1e-10 * scale and np.abs(hi - bhi).max() <= 1e-10 * scale


def test_upwind_tracing_supersonic_closed_forms(oracle):
    """All waves moving right (u > cf): the i+1/2 state is the full Hancock predictor and the
    i-1/2 state is untraced, w - dw^m / 2.  All waves moving left: the mirror.  (The second
    case fixes the reading of eq 41: its printed form would leave the traced i-1/2 state off
    the Hancock one.)"""
    rng = np.random.default_rng(8)
    for Wm, W0, Wp in _triples(rng, 6):
        for sgn in (1.0, -1.0):
            s = np.zeros(10)
            s[1] = sgn * 3.0 * np.sqrt(3 * W0[4] / W0[0])
            A = [w + s for w in (Wm, W0, Wp)]
            hlo, hhi = oracle.reconstruct(*A, 0, 0.3)
            dwm = hhi - hlo  # the Hancock states differ by exactly dw^m
            lo, hi = oracle.reconstruct_upwind(*A, 0, 0.3)
            tol = 1e-12 * np.abs(A[1]).max()
            if sgn > 0:
                assert np.abs(hi - hhi).max() <= tol
                assert np.abs(lo - (A[1] - 0.5 * dwm)).max() <= tol
            else:
                assert np.abs(lo - hlo).max() <= tol
                assert np.abs(hi - (A[1] + 0.5 * dwm)).max() <= tol
