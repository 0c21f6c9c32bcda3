"""GPU discrete adjoint (msh_adjoint_run) against the oracle's adjoint (autograd of the FP64
PyTorch restatement of the step, pinned to central finite differences in
test_adjoint_oracle.py), on the same frozen dt schedule."""
import numpy as np
import pytest
import torch

from oracle import torch_step as ts
from tests.parity import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import msh as m
    m.load()
    return m


def _smooth(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    axes = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                       indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, (10, 3))
    amp = np.array([0.2, 0.1, 0.1, 0.1, 0.1, 0.04, 0.04, 0.1, 0.03, 0.1])
    base = np.array([1.0, 0.3, -0.2, 0.1, 0.6, 0.0, 0.0, 0.5, 0.0, 0.4])
    W = np.zeros((10,) + shape)
    for k in range(10):
        W[k] = base[k] + amp[k] * np.sin(2 * np.pi * axes[2] + ph[k, 0]) * np.cos(2 * np.pi * axes[1] + ph[k, 1]) \
            * np.cos(2 * np.pi * axes[0] + ph[k, 2])
    return W


def _case(name, oracle):
    from paper_1210_5246_gb300 import inputs as I
    if name == "sod":
        p = I.sod(48)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, None, 5
    if name == "smooth2d_gravity_reflect":
        n = 14
        W = _smooth((1, n, n), 1)
        xs = (np.arange(-1, n + 1) + 0.5) / n
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        phi = (0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).reshape(1, n + 2, n + 2)
        W[3] = 0.0  # reflect in y keeps u_z = 0 and P_xz = P_yz = 0 physical
        return W, (n, n), (0, 0), (1, 1), ((0, 0), (2, 2)), 0.4, phi, 4
    if name == "turb3d":
        p = I.turb(n=8, nsteps=3)
        return p.W, p.n, p.lo, p.hi, ((0, 0), (1, 1), (2, 1)), p.cfl, None, 3
    if name == "disc":
        p = I.disc(n=20, nsteps=3)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, p.phi, 3
    if name == "fallback1d":
        from tests.test_oracle_pins import _extreme_tiny
        return _extreme_tiny(1), (8,), (0,), (1,), ((0, 0),), 0.8, None, 2
    if name == "tiles2d":
        # several x tiles of the staged pass (8 columns, the last one ragged) and three
        # 26-position segments along y; periodic x, reflect y
        W = _smooth((1, 61, 70), 2)
        W[3] = 0.0
        return W, (70, 61), (0, 0), (1, 1), ((0, 0), (2, 2)), 0.4, None, 2
    if name == "tiles3d":
        # segments along y and z, ragged x tiles; outflow x, periodic y, reflect/outflow z
        W = _smooth((33, 30, 19), 3)
        return W, (19, 30, 33), (0, 0, 0), (1, 1, 1), ((1, 1), (0, 0), (2, 1)), 0.4, None, 2
    raise KeyError(name)


def _oracle_adjoint(W, n, bc, dx, dts, lam, phi, kind):
    U0 = ts.prim_to_cons(torch.tensor(W))
    if kind == "primitive":
        Wt = torch.tensor(W).requires_grad_(True)
        Ut = ts.prim_to_cons(Wt)
        out = Ut
        for dt in dts:
            out = ts.step(out, len(n), dx, bc, float(dt), None if phi is None else torch.tensor(phi))
        (g,) = torch.autograd.grad(out, Wt, grad_outputs=torch.tensor(lam))
        return g.numpy()
    g, _ = ts.adjoint_run(U0, len(n), dx, bc, dts, torch.tensor(lam), None if phi is None else torch.tensor(phi))
    return g.numpy()


@pytest.mark.parametrize("name", ["sod", "smooth2d_gravity_reflect", "turb3d", "disc", "fallback1d", "tiles2d",
                                  "tiles3d"])
def test_adjoint_fp64_matches_oracle(msh, oracle, name):
    W, n, lo, hi, bc, cfl, phi, steps = _case(name, oracle)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    U0 = oracle.prim_to_cons(W)
    dts = oracle.run(og, U0, np.inf, max_steps=steps, phi=phi, record=True)[4]
    lam = np.random.default_rng(7).normal(size=U0.shape)
    ref = _oracle_adjoint(W, n, bc, og.dx, dts, lam, phi, "conserved")
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    if phi is not None:
        g.set_potential(phi)
    got = g.adjoint_run(U0, dts, lam, K=2)
    e = field_errors(got, ref, "linf")
    assert e.max() <= 1e-10, e
    g.close()


def test_adjoint_primitive_kind_and_device_buffers(msh, oracle):
    W, n, lo, hi, bc, cfl, phi, steps = _case("disc", oracle)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    dts = oracle.run(og, oracle.prim_to_cons(W), np.inf, max_steps=steps, phi=phi, record=True)[4]
    lam = np.random.default_rng(8).normal(size=W.shape)
    ref = _oracle_adjoint(W, n, bc, og.dx, dts, lam, phi, "primitive")
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    g.set_potential(phi)
    got = g.adjoint_run(torch.tensor(W, device="cuda"), dts, torch.tensor(lam, device="cuda"), K=1,
                        kind=msh.PRIMITIVE)
    e = field_errors(got.cpu().numpy(), ref, "linf")
    assert e.max() <= 1e-10, e
    g.close()


def test_adjoint_fp32(msh, oracle):
    """FP32 adjoint against the FP64 oracle adjoint: relative L2 error <= 1e-3."""
    W, n, lo, hi, bc, cfl, phi, steps = _case("smooth2d_gravity_reflect", oracle)
    W32 = W.astype(np.float32).astype(np.float64)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    U0 = oracle.prim_to_cons(W32)
    dts = oracle.run(og, U0, np.inf, max_steps=steps, phi=phi, record=True)[4]
    lam = np.random.default_rng(9).normal(size=U0.shape)
    ref = _oracle_adjoint(W32, n, bc, og.dx, dts, lam, phi, "conserved")
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP32)
    g.set_potential(phi)
    got = g.adjoint_run(U0.astype(np.float32), dts, lam.astype(np.float32), K=3).astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel
    g.close()


def test_adjoint_does_not_touch_grid_state(msh, oracle):
    from paper_1210_5246_gb300 import inputs as I
    p = I.sod(32, t_end=0.02)
    g = msh.Grid.from_problem(p, msh.FP64)
    g.set_state(p.W, msh.PRIMITIVE)
    g.run(max_steps=3)
    before = g.get_state(), g.time()
    U0 = oracle.prim_to_cons(p.W)
    g.adjoint_run(U0, [1e-3, 1e-3], np.ones_like(U0), K=1)
    np.testing.assert_array_equal(g.get_state(), before[0])
    assert g.time() == before[1]
    g.close()


# ------------------------------------------------------------------ adjoint tape
def _taped_run(msh, case, K, autotune=False):
    W, n, lo, hi, bc, cfl, phi, steps = case
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    if phi is not None:
        g.set_potential(phi)
    g.set_state(W, msh.PRIMITIVE)
    U0 = g.get_state()
    g.set_recording(steps)
    g.set_tape(K, steps)
    if autotune and len(n) > 1:
        g.autotune()
    ns, _ = g.run(max_steps=steps)
    assert ns == steps
    return g, U0, g.dt_history()


@pytest.mark.parametrize("name,K", [("sod", 2), ("smooth2d_gravity_reflect", 3), ("turb3d", 1), ("disc", 2),
                                    ("fallback1d", 1)])
def test_tape_equals_forward_sweep_adjoint_and_oracle(msh, oracle, name, K):
    """The adjoint from the recorded tape equals msh_adjoint_run on the same state and
    schedule bit for bit (same checkpoints, same kernels), and the oracle's adjoint."""
    case = _case(name, oracle)
    W, n, lo, hi, bc, cfl, phi, steps = case
    g, U0, dts = _taped_run(msh, case, K, autotune=(name == "disc"))
    lam = np.random.default_rng(11).normal(size=U0.shape)
    got = g.adjoint_tape(lam)
    ref_run = g.adjoint_run(U0, dts, lam, K=K)
    np.testing.assert_array_equal(got, ref_run)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    ref = _oracle_adjoint(W, n, bc, og.dx, dts, lam, phi, "conserved")
    assert field_errors(got, ref, "linf").max() <= 1e-10
    if name == "disc":
        gp = g.adjoint_tape(torch.tensor(lam, device="cuda"), kind=msh.PRIMITIVE).cpu().numpy()
        refp = _oracle_adjoint(W, n, bc, og.dx, dts, lam, phi, "primitive")
        assert field_errors(gp, refp, "linf").max() <= 1e-10
    g.close()


def test_tape_does_not_change_the_run(msh, oracle):
    case = _case("turb3d", oracle)
    W, n, lo, hi, bc, cfl, phi, steps = case
    g, _, _ = _taped_run(msh, case, 1)
    taped = g.get_state()
    g.close()
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    g.set_state(W, msh.PRIMITIVE)
    g.run(max_steps=steps)
    np.testing.assert_array_equal(g.get_state(), taped)
    g.close()


def test_tape_errors(msh, oracle):
    W, n, lo, hi, bc, cfl, phi, steps = _case("sod", oracle)
    g = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    lam = np.ones((10, 1, 1, n[0]))
    with pytest.raises(msh.MshError) as ei:
        g.set_tape(2, 4)  # no state yet
    assert ei.value.status == msh.MSH_E_STATE
    g.set_state(W, msh.PRIMITIVE)
    with pytest.raises(msh.MshError) as ei:
        g.adjoint_tape(lam)  # nothing recorded
    assert ei.value.status == msh.MSH_E_STATE
    with pytest.raises(msh.MshError) as ei:
        g.set_tape(-1, 4)
    assert ei.value.status == msh.MSH_E_INVALID_ARG
    g.set_tape(2, 3)
    g.run(max_steps=4)  # one step past the tape
    with pytest.raises(msh.MshError) as ei:
        g.adjoint_tape(lam)
    assert ei.value.status == msh.MSH_E_STATE
    g.set_tape(2, 3)
    g.run(max_steps=2)
    g.adjoint_tape(lam)
    g.set_state(W, msh.PRIMITIVE)  # a new state ends the recording
    with pytest.raises(msh.MshError) as ei:
        g.adjoint_tape(lam)
    assert ei.value.status == msh.MSH_E_STATE
    g.set_tape(0, 0)  # frees
    g.close()
