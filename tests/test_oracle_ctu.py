"""Pins of the oracle's corner-transport-upwind option (transverse terms in the face states,
max-form CFL): agreement with the brute-force step (transverse terms wave by wave on a
numerically computed eigen-system, padded grid filled axis by axis) on tiny 2D and 3D
grids with every boundary kind; no effect in 1D; a flow that varies along x only on a 2D
grid reproduces the 1D run bit for bit; diagonal advection at max-form CFL 0.8 in 2D and 3D
stays accurate where the plain unsplit step on the same time steps diverges, and converges
at second order; conservation; x <-> y symmetry."""
import numpy as np
import pytest

from tests import bruteforce as BF


def _rand_W(rng, shape, amp=0.15):
    W = np.zeros((10,) + shape)
    W[0] = 1 + amp * rng.uniform(-1, 1, shape)
    W[1:4] = 0.3 * rng.uniform(-1, 1, (3,) + shape)
    W[4] = 0.8 + 0.2 * rng.uniform(-1, 1, shape)
    W[7] = 0.7 + 0.2 * rng.uniform(-1, 1, shape)
    W[9] = 0.6 + 0.2 * rng.uniform(-1, 1, shape)
    for k in (5, 6, 8):
        W[k] = 0.05 * rng.uniform(-1, 1, shape)
    return W


@pytest.mark.parametrize("n,bc,scheme,flux", [
    ((6, 5), ((0, 0), (1, 2)), 0, "hll"),
    ((5, 6), ((2, 1), (0, 0)), 2, "roe"),
    ((4, 4, 3), ((0, 0), (2, 2), (1, 0)), 0, "hll"),
])
def test_matches_bruteforce(oracle, n, bc, scheme, flux):
    nd = len(n)
    rng = np.random.default_rng(sum(n))
    shape = (1,) * (3 - nd) + tuple(reversed(n))
    W = _rand_W(rng, shape)
    g = oracle.Grid(n, (0,) * nd, (1,) * nd, bc, 0.8, scheme=scheme, ctu=True)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    assert abs(dt - BF.cfl_dt(U, nd, list(g.dx), 0.8, ctu=True)) <= 1e-13 * dt
    A = oracle.step(g, U, dt)
    B = BF.step(U, nd, list(g.dx), bc, dt, flux=flux, ctu=True)
    scale = np.abs(B).reshape(10, -1).max(axis=1)[:, None, None, None] + 1e-300
    assert np.max(np.abs(A - B) / scale) < 1e-11
    # the transverse terms matter here: the plain step differs
    P = oracle.step(oracle.Grid(n, (0,) * nd, (1,) * nd, bc, 0.8, scheme=scheme), U, dt)
    assert np.max(np.abs(A - P) / scale) > 1e-6


def test_no_effect_in_1d(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.sod(64)
    outs = []
    for ctu in (False, True):
        g = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl, ctu=ctu)
        outs.append(oracle.run(g, oracle.prim_to_cons(p.W), 0.1)[0])
    np.testing.assert_array_equal(outs[0], outs[1])


def test_x_only_flow_equals_1d(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.sod(48)
    W2 = np.repeat(p.W, 5, axis=2)  # [10][1][5][48]
    g2 = oracle.Grid((48, 5), (0.0, 0.0), (1.0, 0.3), ((1, 1), (0, 0)), 0.6, ctu=True)
    U2, _, _, rc, dts = oracle.run(g2, oracle.prim_to_cons(W2), 0.1, record=True)
    assert rc == 0
    g1 = oracle.Grid((48,), (0.0,), (1.0,), ((1, 1),), 0.6)
    U1 = oracle.run_schedule(g1, oracle.prim_to_cons(p.W), dts)
    for j in range(5):
        np.testing.assert_array_equal(U2[:, :, j:j + 1, :], U1)


def _advection(nd, n):
    xs = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([xs] * nd), indexing="ij")
    shape = (1,) * (3 - nd) + (n,) * nd
    W = np.zeros((10,) + shape)
    W[0] = (1 + 0.2 * sum(np.sin(2 * np.pi * g) for g in grids)).reshape(shape)
    vel = [1.0, 0.8, 0.6][:nd]
    for d in range(nd):
        W[1 + d] = vel[d]
    W[4] = W[7] = W[9] = 0.1
    return W, vel


def _exact(nd, n, vel, t):
    xs = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([xs] * nd), indexing="ij")
    # grids[a] is the coordinate of array axis a = reversed dimension order (z, y, x)
    r = sum(np.sin(2 * np.pi * (grids[a] - vel[nd - 1 - a] * t)) for a in range(nd))
    return (1 + 0.2 * r).reshape((1,) * (3 - nd) + (n,) * nd)


@pytest.mark.parametrize("nd,n", [(2, 48), (3, 20)])
def test_stable_at_max_cfl_08(oracle, nd, n):
    W, vel = _advection(nd, n)
    U0 = oracle.prim_to_cons(W)
    g = oracle.Grid((n,) * nd, (0,) * nd, (1,) * nd, ((0, 0),) * nd, 0.8, ctu=True)
    U, ns, t, rc, dts = oracle.run(g, U0, 1.0, record=True)
    assert rc == 0
    err = np.abs(U[0] - _exact(nd, n, vel, t)).max()
    assert err < 0.05, err
    plain = oracle.Grid((n,) * nd, (0,) * nd, (1,) * nd, ((0, 0),) * nd, 0.8)
    with np.errstate(all="ignore"):
        Up = oracle.run_schedule(plain, U0, dts)
        bad = not np.all(np.isfinite(Up[0])) or np.abs(Up[0] - 1).max() > 1.0
    assert bad


def test_second_order_at_max_cfl_08(oracle):
    errs = []
    for n in (32, 64, 128):
        W, vel = _advection(2, n)
        g = oracle.Grid((n, n), (0, 0), (1, 1), ((0, 0), (0, 0)), 0.8, ctu=True)
        U, ns, t, rc, _ = oracle.run(g, oracle.prim_to_cons(W), 0.5)
        assert rc == 0
        errs.append(np.abs(U[0] - _exact(2, n, vel, t)).mean())
    assert np.log2(errs[1] / errs[2]) >= 1.8, errs


def test_conservation_periodic(oracle):
    from paper_1210_5246_gb300 import inputs
    p = inputs.turb(n=12)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, 0.7, ctu=True)
    U0 = oracle.prim_to_cons(p.W)
    U, ns, _, rc, _ = oracle.run(g, U0, np.inf, max_steps=5)
    assert rc == 0 and ns == 5
    t0, t1 = oracle.diagnostics(g, U0)[0], oracle.diagnostics(g, U)[0]
    scale = np.array([t0[0]] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)


def test_xy_swap_symmetry(oracle):
    rng = np.random.default_rng(4)
    n = 16
    W = _rand_W(rng, (1, n, n))
    # swap x and y: transpose the grid and exchange the x/y components
    perm = [0, 2, 1, 3, 7, 5, 8, 4, 6, 9]
    Ws = W[perm].transpose(0, 1, 3, 2).copy()
    outs = []
    for w in (W, Ws):
        g = oracle.Grid((n, n), (0, 0), (1, 1), ((0, 0), (0, 0)), 0.8, ctu=True)
        outs.append(oracle.run(g, oracle.prim_to_cons(w), np.inf, max_steps=6)[0])
    back = outs[1][perm].transpose(0, 1, 3, 2)
    assert np.abs(back - outs[0]).max() <= 1e-13 * np.abs(outs[0]).max()
