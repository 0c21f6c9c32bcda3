"""msh_run_ensemble: independent states streamed through host memory with uploads, steps
and downloads overlapped.  Every state's result equals, bit for bit, the same state run
alone on a fresh grid (set_state, run, get_state) — FP32 and FP64, conserved and primitive
input, several steps, gravity, every scheme — and matches the oracle (FP64 1e-10); a
non-realizable input is reported for its state alone; the grid keeps the last result."""
import numpy as np
import pytest

from tests.parity import assert_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs, torch


def _pinned(torch, shape, dtype):
    t = torch.empty(shape, dtype=torch.float32 if dtype == np.float32 else torch.float64).pin_memory()
    return t.numpy()


def _alone(msh, p, W, prec, kind, nsteps, scheme=None, ctu=False):
    g = msh.Grid.from_problem(p, prec)
    if scheme is not None:
        g.set_scheme(scheme)
    if ctu:
        g.set_ctu(True)
    if kind == msh.CONSERVED:
        g.set_state(W, msh.PRIMITIVE)
        U = g.get_state()
        g.close()
        g = msh.Grid.from_problem(p, prec)
        if scheme is not None:
            g.set_scheme(scheme)
        if ctu:
            g.set_ctu(True)
        g.set_state(U, msh.CONSERVED)
    else:
        g.set_state(W, msh.PRIMITIVE)
    g.run(max_steps=nsteps)
    out = g.get_state(kind)
    g.close()
    return out


def _states(inputs, n, count):
    return [inputs.turb(n=n, nsteps=4, seed=10 + k) for k in range(count)]


@pytest.mark.parametrize("prec_name,kind_name,nsteps", [("FP32", "PRIMITIVE", 1), ("FP64", "PRIMITIVE", 3),
                                                         ("FP32", "CONSERVED", 2), ("FP64", "CONSERVED", 1)])
def test_equals_states_run_alone(env, prec_name, kind_name, nsteps):
    msh, inputs, torch = env
    prec, kind = getattr(msh, prec_name), getattr(msh, kind_name)
    ps = _states(inputs, 20, 5)
    dt = np.float32 if prec == msh.FP32 else np.float64
    g = msh.Grid.from_problem(ps[0], prec)
    ins, want = [], []
    for p in ps:
        a = _pinned(torch, p.W.shape, dt)
        if kind == msh.PRIMITIVE:
            a[...] = p.W.astype(dt)
        else:
            h = msh.Grid.from_problem(p, prec)
            h.set_state(p.W.astype(dt), msh.PRIMITIVE)
            a[...] = h.get_state()
            h.close()
        ins.append(a)
        want.append(_alone(msh, p, p.W.astype(dt), prec, kind, nsteps))
    outs = [_pinned(torch, p.W.shape, dt) for _ in ps]
    st = g.run_ensemble(ins, outs, kind=kind, nsteps=nsteps)
    assert list(st) == [0] * len(ps)
    for k in range(len(ps)):
        np.testing.assert_array_equal(outs[k], want[k])
    # the grid holds the last state's result
    np.testing.assert_array_equal(g.get_state(kind), want[-1])
    g.close()


def test_matches_oracle_fp64(env, oracle):
    msh, inputs, torch = env
    ps = _states(inputs, 16, 3)
    g = msh.Grid.from_problem(ps[0], msh.FP64)
    ins = [np.ascontiguousarray(p.W) for p in ps]
    outs = [np.empty_like(p.W) for p in ps]
    g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=2)
    g.close()
    for p, o in zip(ps, outs):
        og = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)
        Uo = oracle.run(og, oracle.prim_to_cons(p.W), np.inf, max_steps=2)[0]
        assert_fp64(oracle.prim_to_cons(o), Uo, what="ensemble vs oracle")


@pytest.mark.parametrize("scheme_name", ["KT", "MUSCL_HANCOCK_ROE", "MUSCL_HANCOCK_HLLC"])
def test_schemes_and_gravity(env, scheme_name):
    msh, inputs, torch = env
    scheme = getattr(msh, scheme_name)
    ps = [inputs.disc(n=48, nsteps=3, seed=20 + k) for k in range(4)]
    g = msh.Grid.from_problem(ps[0], msh.FP64)
    g.set_scheme(scheme)
    ins = [np.ascontiguousarray(p.W) for p in ps]
    outs = [np.empty_like(p.W) for p in ps]
    g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=3)
    g.close()
    for p, o in zip(ps, outs):
        np.testing.assert_array_equal(o, _alone(msh, p, p.W, msh.FP64, msh.PRIMITIVE, 3, scheme))


def test_non_realizable_input_is_isolated(env):
    msh, inputs, torch = env
    ps = _states(inputs, 12, 4)
    bad = ps[1].W.copy()
    bad[0, 3, 4, 5] = -1.0  # negative density in one cell
    ins = [np.ascontiguousarray(ps[0].W), bad, np.ascontiguousarray(ps[2].W), np.ascontiguousarray(ps[3].W)]
    outs = [np.empty_like(ps[0].W) for _ in ins]
    g = msh.Grid.from_problem(ps[0], msh.FP64)
    st = g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=2, check=False)
    assert list(st) == [0, msh.MSH_E_REALIZABILITY, 0, 0]
    for k in (0, 2, 3):
        np.testing.assert_array_equal(outs[k], _alone(msh, ps[k], ps[k].W, msh.FP64, msh.PRIMITIVE, 2))
    with pytest.raises(msh.MshError) as ei:
        g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=2)
    assert ei.value.status == msh.MSH_E_REALIZABILITY
    # the grid still works as a plain grid afterwards
    g.set_state(ps[0].W, msh.PRIMITIVE)
    g.run(max_steps=2)
    np.testing.assert_array_equal(g.get_state(msh.PRIMITIVE), outs[0])
    g.close()


def test_arguments(env):
    msh, inputs, torch = env
    p = inputs.turb(n=8, nsteps=1)
    g = msh.Grid.from_problem(p, msh.FP64)
    assert len(g.run_ensemble([], [])) == 0
    W = np.ascontiguousarray(p.W)
    with pytest.raises(msh.MshError) as ei:
        g.run_ensemble([W], [np.empty_like(W)], nsteps=0)
    assert ei.value.status == msh.MSH_E_INVALID_ARG
    with pytest.raises(ValueError):
        g.run_ensemble([W.astype(np.float32)], [np.empty_like(W)])
    with pytest.raises(ValueError):
        g.run_ensemble([W], [])
    g.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP32"])
def test_ctu_equals_states_run_alone(env, prec_name):
    """The corner-transport-upwind step in an ensemble: each state's start re-plans with the
    max-form CFL rule; every result equals the state run alone, bit for bit."""
    msh, inputs, torch = env
    prec = getattr(msh, prec_name)
    dtype = np.float32 if prec == msh.FP32 else np.float64
    ps = _states(inputs, 20, 5)
    g = msh.Grid.from_problem(ps[0], prec)
    g.set_ctu(True)
    ins = [np.ascontiguousarray(p.W.astype(dtype)) for p in ps]
    outs = [np.empty_like(w) for w in ins]
    st = g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=4)
    g.close()
    assert list(st) == [0] * len(ps)
    for p, w, o in zip(ps, ins, outs):
        np.testing.assert_array_equal(o, _alone(msh, p, w, prec, msh.PRIMITIVE, 4, ctu=True))
