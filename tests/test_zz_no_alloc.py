"""msh_step_noalloc: one grid step for callers that cannot allocate device memory (code
inside another framework's pre-sized memory pool, real-time loops that must stay out of
the allocator, code that only owns the two state buffers it was handed).  Its working
memory is a fixed file-scope device array; this test checks, through the C ABI, that two
calls in a row give the same states as two msh_step calls on an ordinary grid.  It lives
in a file of its own that pytest collects last."""
import numpy as np
import pytest

from tests.parity import assert_fp32, assert_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import msh as m
    m.load()
    return m


def _state(shape, seed):
    rng = np.random.default_rng(seed)
    W = np.zeros((10,) + shape)
    W[0] = np.exp(rng.uniform(-0.5, 0.5, shape))
    W[1:4] = rng.uniform(-0.3, 0.3, (3,) + shape)
    W[4], W[7], W[9] = 0.8, 0.7, 0.6
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, shape)
    return W


@pytest.mark.parametrize("n,bc,prec", [((61, 45), ((2, 2), (1, 1)), "fp64"),
                                       ((33, 17, 9), ((1, 2), (0, 0), (2, 1)), "fp32"),
                                       ((300,), ((2, 1),), "fp64")])
def test_noalloc_step_matches_msh_step_twice(msh, n, bc, prec):
    import torch
    precision = msh.FP64 if prec == "fp64" else msh.FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    nd = len(n)
    lo, hi = (0.0,) * nd, (1.0, 1.5, 0.5)[:nd]
    shape = (n[2] if nd > 2 else 1, n[1] if nd > 1 else 1, n[0])
    W = _state(shape, seed=sum(n))
    g = msh.Grid(n, lo, hi, bc, 0.5, precision)
    g.set_state(W.astype(g.dtype), msh.PRIMITIVE)
    U0 = g.get_state()
    dt1 = g.step()
    A1 = g.get_state()
    dt2 = g.step()
    A2 = g.get_state()
    g.close()
    u0 = torch.tensor(U0, device="cuda", dtype=dtype)
    u1 = torch.empty_like(u0)
    u2 = torch.empty_like(u0)
    e1 = msh.msh_step_noalloc(n, lo, hi, bc, precision, 0.5, u0, u1)
    e2 = msh.msh_step_noalloc(n, lo, hi, bc, precision, 0.5, u1, u2)
    assert abs(e1 - dt1) <= 1e-12 * dt1 and abs(e2 - dt2) <= 1e-12 * dt2
    B1, B2 = u1.cpu().numpy(), u2.cpu().numpy()
    if prec == "fp64":
        assert_fp64(B1, A1, what="first call")
        assert_fp64(B2, A2, what="second call")
    else:
        assert_fp32(_prim(B1), _prim(A1), what="first call")
        assert_fp32(_prim(B2), _prim(A2), what="second call")


def _prim(U):
    U = U.astype(np.float64)
    W = U.copy()
    r = U[0]
    u = U[1:4] / r
    W[1:4] = u
    pairs = {4: (0, 0), 5: (0, 1), 6: (0, 2), 7: (1, 1), 8: (1, 2), 9: (2, 2)}
    for k, (i, j) in pairs.items():
        W[k] = U[k] - r * u[i] * u[j]
    return W


def test_noalloc_rejects_oversized_grid(msh):
    import torch
    u = torch.zeros(10, device="cuda", dtype=torch.float64)
    with pytest.raises(msh.MshError) as ei:
        msh.msh_step_noalloc((1100, 1000), (0, 0), (1, 1), ((0, 0), (0, 0)), msh.FP64, 0.5, u,
                             torch.zeros_like(u))
    assert ei.value.status == msh.MSH_E_INVALID_ARG and "1048576" in str(ei.value)


def test_noalloc_rejects_non_realizable_input(msh):
    """A state with one cell whose P_xx P_yy < P_xy^2 is refused before any step, the
    output buffer untouched; the next call on a realizable state steps normally."""
    import torch
    n, lo, hi, bc = (40, 24), (0.0, 0.0), (1.0, 1.0), ((0, 0), (1, 1))
    W = _state((1, n[1], n[0]), seed=11)
    W[5, 0, 7, 13] = 2.0  # P_xy^2 = 4 > P_xx P_yy = 0.56
    U = W.copy()
    r = W[0]
    U[1:4] = r * W[1:4]
    pairs = {4: (1, 1), 5: (1, 2), 6: (1, 3), 7: (2, 2), 8: (2, 3), 9: (3, 3)}
    for k, (i, j) in pairs.items():
        U[k] = W[k] + r * W[i] * W[j]
    u0 = torch.tensor(U, device="cuda", dtype=torch.float64)
    u1 = torch.full_like(u0, 7.0)
    with pytest.raises(msh.MshError) as ei:
        msh.msh_step_noalloc(n, lo, hi, bc, msh.FP64, 0.5, u0, u1)
    assert ei.value.status == msh.MSH_E_REALIZABILITY
    assert f"first cell {7 * n[0] + 13}" in str(ei.value)
    assert bool((u1 == 7.0).all())
    W[5, 0, 7, 13] = 0.0
    U[5] = W[5] + r * W[1] * W[2]
    u0 = torch.tensor(U, device="cuda", dtype=torch.float64)
    assert msh.msh_step_noalloc(n, lo, hi, bc, msh.FP64, 0.5, u0, u1) > 0
    assert bool(torch.isfinite(u1).all()) and not bool((u1 == 7.0).any())

