"""Pins of the oracle's discrete adjoint (PyTorch restatement of the step, autograd).

Forward: identical to the C oracle (to rounding) on every workload.  Gradients: the
vector-Jacobian product over several steps with a frozen dt schedule agrees with central
finite differences of the C oracle along random directions, and forward-mode JVPs agree
with reverse-mode VJPs (dot-product test)."""
import numpy as np
import pytest
import torch

from oracle import torch_step as ts
from paper_1210_5246_gb300 import inputs as I


def _problem(name):
    if name == "sod":
        return I.sod(48), 4
    if name == "blast":
        return I.blast(n=16, nsteps=3), 3
    if name == "turb":
        return I.turb(n=8, nsteps=2), 2
    if name == "disc":
        return I.disc(n=20, nsteps=3), 3
    raise KeyError(name)


@pytest.mark.parametrize("name", ["sod", "blast", "turb", "disc"])
def test_torch_step_matches_c_oracle(oracle, name):
    p, steps = _problem(name)
    g = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)
    U = oracle.prim_to_cons(p.W)
    dts = oracle.run(g, U, np.inf, max_steps=steps, phi=p.phi, record=True)[4]
    Uc = oracle.run_schedule(g, U, dts, phi=p.phi)
    Ut = torch.tensor(U)
    ph = None if p.phi is None else torch.tensor(p.phi)
    with torch.no_grad():
        for dt in dts:
            Ut = ts.step(Ut, p.ndim, g.dx, p.bc, float(dt), ph)
    assert np.abs(Ut.numpy() - Uc).max() <= 1e-13 * np.abs(Uc).max()


def _smooth_2d(n=12, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    # every field varies (an exactly constant field puts its characteristic slopes on the
    # MC limiter's kink, where one-sided finite differences and the frozen branch differ)
    ph = rng.uniform(0, 2 * np.pi, (10, 2))
    amp = np.array([0.2, 0.1, 0.1, 0.1, 0.1, 0.04, 0.04, 0.1, 0.03, 0.1])
    base = np.array([1.0, 0.3, -0.2, 0.1, 0.6, 0.0, 0.0, 0.5, 0.0, 0.4])
    W = np.zeros((10, 1, n, n))
    for k in range(10):
        W[k, 0] = base[k] + amp[k] * np.sin(2 * np.pi * X + ph[k, 0]) * np.cos(2 * np.pi * Y + ph[k, 1])
    return W


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_matches_central_fd(oracle, seed):
    """<dL/dU0, v> from the reverse sweep equals (L(U0 + h v) - L(U0 - h v)) / 2h with
    L(U0) = <lam, U_N(U0)> computed by the C oracle over a frozen dt schedule."""
    n = 12
    W = _smooth_2d(n, seed)
    g = oracle.Grid((n, n), (0, 0), (1, 1), ((0, 0), (1, 1)), 0.4)
    xs = (np.arange(-1, n + 1) + 0.5) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    phi = (0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).reshape(1, n + 2, n + 2)
    U0 = oracle.prim_to_cons(W)
    dts = oracle.run(g, U0, np.inf, max_steps=4, phi=phi, record=True)[4]
    rng = np.random.default_rng(100 + seed)
    lam = rng.normal(size=U0.shape)
    grad, UN = ts.adjoint_run(torch.tensor(U0), 2, g.dx, ((0, 0), (1, 1)), dts, torch.tensor(lam),
                              torch.tensor(phi))
    np.testing.assert_allclose(UN.numpy(), oracle.run_schedule(g, U0, dts, phi=phi), rtol=0, atol=1e-13)
    for k in range(3):
        v = rng.normal(size=U0.shape) * np.abs(U0).max(axis=(1, 2, 3), keepdims=True) * 1e-3
        h = 1e-5  # small enough not to cross a limiter switch
        Lp = (lam * oracle.run_schedule(g, U0 + h * v, dts, phi=phi)).sum()
        Lm = (lam * oracle.run_schedule(g, U0 - h * v, dts, phi=phi)).sum()
        fd = (Lp - Lm) / (2 * h)
        ad = float((grad.numpy() * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 2e-9, (fd, ad)  # 2e-9: FD rounding of L ~ O(10)


def test_jvp_vjp_dot_product():
    """<J v, w> = <v, J^T w> between forward-mode (torch.func.jvp) and reverse mode."""
    n = 10
    W = _smooth_2d(n, 3)
    U0 = torch.tensor(ts.prim_to_cons(torch.tensor(W)).numpy())
    dx = (1 / n, 1 / n, 1.0)
    bc = ((0, 0), (2, 2))
    f = lambda U: ts.step(ts.step(U, 2, dx, bc, 0.01), 2, dx, bc, 0.008)
    rng = np.random.default_rng(5)
    v = torch.tensor(rng.normal(size=W.shape))
    w = torch.tensor(rng.normal(size=W.shape))
    _, Jv = torch.func.jvp(f, (U0,), (v,))
    U = U0.clone().requires_grad_(True)
    (JTw,) = torch.autograd.grad(f(U), U, grad_outputs=w)
    a, b = float((Jv * w).sum()), float((v * JTw).sum())
    assert abs(a - b) <= 1e-10 * abs(a)
