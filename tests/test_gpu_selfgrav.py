"""Periodic self-gravity on the GPU (cuFFT Poisson solve, forward-interpolated acceleration)
against the oracle's self-gravity: FP64 <= 1e-10 relative L_inf per field, FP32 within the
FP32 tolerances; 1D/2D/3D, both schemes, with an external potential, through the CUDA
graphs; the linear Jeans growth rate; errors."""
import numpy as np
import pytest

from tests.parity import assert_fp32, assert_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs


def _periodic_field(shape, seed, sigma2=0.3):
    rng = np.random.default_rng(seed)
    W = np.zeros((10,) + shape)
    W[0] = np.exp(0.3 * rng.normal(size=shape))
    W[1:4] = 0.2 * rng.normal(size=(3,) + shape)
    W[4], W[7], W[9] = sigma2, 0.8 * sigma2, 0.9 * sigma2
    W[5] = 0.05 * sigma2 * rng.normal(size=shape)
    return W


def _compare(msh, oracle, n, W, steps, G, precision=None, scheme=0, phi_ext=None, cfl=0.4, profiled=False,
             ctu=False):
    from oracle import selfgrav
    precision = msh.FP64 if precision is None else precision
    nd = len(n)
    lo, hi = (0.0,) * nd, (1.0,) * nd
    bc = ((0, 0),) * nd
    g = msh.Grid(n, lo, hi, bc, cfl, precision)
    if scheme:
        g.set_scheme(scheme)
    if ctu:
        g.set_ctu(True)
    if phi_ext is not None:
        g.set_potential(phi_ext)
    g.set_self_gravity(G)
    g.set_profiling(profiled)
    Wg = W.astype(np.float32) if precision == msh.FP32 else W
    g.set_state(Wg, msh.PRIMITIVE)
    ns, _ = g.run(max_steps=steps)
    assert ns == steps
    U, Wout = g.get_state().astype(np.float64), g.get_state(msh.PRIMITIVE).astype(np.float64)
    g.close()
    og = oracle.Grid(n, lo, hi, bc, cfl, scheme=scheme, ctu=ctu)
    Uo, _ = selfgrav.run(og, oracle.prim_to_cons(Wg.astype(np.float64)), steps, G, phi_ext=phi_ext)
    return U, Wout, Uo, oracle.cons_to_prim(Uo)


@pytest.mark.parametrize("shape,n,steps", [((1, 1, 64), (64,), 12), ((1, 24, 40), (40, 24), 10),
                                           ((12, 10, 16), (16, 10, 12), 6)])
def test_fp64_matches_oracle(env, oracle, shape, n, steps):
    msh, _ = env
    W = _periodic_field(shape, len(n))
    U, _, Uo, _ = _compare(msh, oracle, n, W, steps, G=2.0)
    assert_fp64(U, Uo, what=f"self-gravity {n}")


def test_fp32_matches_oracle(env, oracle):
    msh, _ = env
    W = _periodic_field((1, 24, 40), 5)
    _, Wg, _, Wo = _compare(msh, oracle, (40, 24), W, 10, G=2.0, precision=msh.FP32)
    assert_fp32(Wg, Wo, what="self-gravity fp32")


def test_central_scheme_and_external_potential(env, oracle):
    msh, _ = env
    n = (32, 20)
    W = _periodic_field((1, 20, 32), 7)
    x = (np.arange(-1, n[0] + 1) + 0.5) / n[0]
    y = (np.arange(-1, n[1] + 1) + 0.5) / n[1]
    X, Y = np.meshgrid(x, y, indexing="xy")
    phi = (0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).reshape(1, n[1] + 2, n[0] + 2)
    U, _, Uo, _ = _compare(msh, oracle, n, W, 8, G=1.5, scheme=msh.KT, phi_ext=phi)
    assert_fp64(U, Uo, what="self-gravity kt + external")


def test_graph_runs_equal_eager_and_oracle(env, oracle):
    msh, _ = env
    W = _periodic_field((1, 1, 48), 9)
    U, _, Uo, _ = _compare(msh, oracle, (48,), W, 40, G=3.0)
    Ue, _, _, _ = _compare(msh, oracle, (48,), W, 40, G=3.0, profiled=True)
    assert_fp64(U, Uo, what="self-gravity graph")
    np.testing.assert_array_equal(U, Ue)


def test_new_state_resets_the_history(env):
    msh, _ = env
    W = _periodic_field((1, 16, 16), 11)
    g = msh.Grid((16, 16), (0, 0), (1, 1), ((0, 0), (0, 0)), 0.4, msh.FP64)
    g.set_self_gravity(2.0)
    g.set_state(W, msh.PRIMITIVE)
    g.run(max_steps=5)
    g.set_state(W, msh.PRIMITIVE)
    g.set_time(0.0, 0)
    g.run(max_steps=5)
    a = g.get_state()
    h = msh.Grid((16, 16), (0, 0), (1, 1), ((0, 0), (0, 0)), 0.4, msh.FP64)
    h.set_self_gravity(2.0)
    h.set_state(W, msh.PRIMITIVE)
    h.run(max_steps=5)
    np.testing.assert_array_equal(a, h.get_state())
    g.close()
    h.close()


def test_jeans_growth_rate(env):
    """Linear Jeans growth of the ten-moment system on the GPU: rate sqrt(4 pi G rho0 - 3 sigma^2 k^2)."""
    msh, _ = env
    n, L, sigma2, eps = 64, 4.0, 0.01, 1e-4
    G = 1.0 / (4 * np.pi)
    x = (np.arange(n) + 0.5) * L / n
    k = 2 * np.pi / L
    gamma = np.sqrt(1.0 - 3 * sigma2 * k * k)
    W = np.zeros((10, 1, 1, n))
    W[0, 0, 0] = 1 + eps * np.cos(k * x)
    W[1, 0, 0] = -gamma / k * eps * np.sin(k * x)
    W[4, 0, 0] = sigma2 * (1 + 3 * eps * np.cos(k * x))
    W[7] = W[9] = sigma2
    g = msh.Grid((n,), (0.0,), (L,), ((0, 0),), 0.2, msh.FP64)
    g.set_self_gravity(G)
    g.set_state(W, msh.PRIMITIVE)
    ts, amps = [], []
    for _ in range(12):
        g.run(max_steps=10)
        rho = g.get_state()[0, 0, 0]
        ts.append(g.time()[0])
        amps.append(2 * np.sum((rho - 1) * np.cos(k * x)) / n)
    g.close()
    fit = np.polyfit(ts[1:], np.log(np.abs(amps[1:])), 1)[0]
    assert abs(fit - gamma) <= 0.03 * gamma, (fit, gamma)


def test_errors(env):
    msh, I = env
    g = msh.Grid((16,), (0.0,), (1.0,), ((1, 1),), 0.4, msh.FP64)
    with pytest.raises(msh.MshError) as ei:
        g.set_self_gravity(1.0)
    assert ei.value.status == msh.MSH_E_INVALID_ARG
    g.close()
    g = msh.Grid((16,), (0.0,), (1.0,), ((0, 0),), 0.4, msh.FP64)
    g.set_self_gravity(1.0)
    W = _periodic_field((1, 1, 16), 3)
    g.set_state(W, msh.PRIMITIVE)
    U0 = g.get_state()
    with pytest.raises(msh.MshError) as ei:
        g.adjoint_run(U0, [1e-3], U0, K=1)
    assert ei.value.status == msh.MSH_E_STATE
    with pytest.raises(msh.MshError):
        g.set_self_gravity(-1.0)
    g.set_self_gravity(0.0)
    g.adjoint_run(U0, [1e-3], U0, K=1)  # allowed again without self-gravity
    g.close()


@pytest.mark.parametrize("shape,n,steps", [((1, 24, 40), (40, 24), 10), ((12, 10, 16), (16, 10, 12), 6)])
def test_ctu_matches_oracle(env, oracle, shape, n, steps):
    """Self-gravity with the corner-transport-upwind step (max-form CFL, CFL 0.7)."""
    msh, _ = env
    W = _periodic_field(shape, len(n) + 7)
    U, _, Uo, _ = _compare(msh, oracle, n, W, steps, G=2.0, cfl=0.7, ctu=True)
    assert_fp64(U, Uo, what=f"self-gravity ctu {n}")
