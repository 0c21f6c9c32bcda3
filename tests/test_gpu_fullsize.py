"""Parity at the workloads' full sizes, in the launch configuration the benchmark times
(autotuned tiling, graph-launched msh_run on a dedicated stream).

* 2D blast, 1024^2 periodic, all 200 steps: FP64 against the oracle (rel L_inf <= 1e-10),
  FP32 against the oracle run from the FP32-rounded input (rel L1 <= 2e-4 / 5e-4).
* 3D box, 256^3 periodic, all 50 steps: FP64 element by element against the oracle
  (rel L_inf <= 1e-10, the dt sequence to 1e-12) and FP32 against the same FP64 oracle run
  (rel L1 <= 2e-4 / 5e-4; the FP32 input is the rounded FP64 one, a 6e-8 perturbation far
  below the tolerance; the oracle needs ~3 s per step on 16 cores, so one oracle run
  serves both); the full runs also by properties that hold at any size: all ten totals
  conserved to round-off (periodic), every cell realizable, device totals against an FP64
  sum of the state, FP32 against FP64.
* Disc, 512^2 outflow with gravity, all 2000 steps: FP32 and FP64 against the oracle.
* Corner transport upwind: the blast's first 50 steps at CFL 0.8 (FP64 and FP32) and the
  box's first 2 steps at CFL 0.6 (FP32) against the oracle's CTU step.
"""
import numpy as np
import pytest

from tests.parity import assert_fp32, assert_fp64, field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs, torch.cuda.Stream()


def _gpu_run(msh, p, precision, stream, steps, record=0):
    g = msh.Grid.from_problem(p, precision, stream=stream.cuda_stream)
    W = p.W.astype(np.float32) if precision == msh.FP32 else p.W
    g.set_state(W, msh.PRIMITIVE)
    g.autotune()
    g.set_state(W, msh.PRIMITIVE)
    g.set_time(0.0, 0)
    if record:
        g.set_recording(record)
    ns, t = g.run(max_steps=steps)
    assert ns == steps
    out = {"U": g.get_state().astype(np.float64), "W": g.get_state(msh.PRIMITIVE).astype(np.float64),
           "diag": g.diagnostics(), "t": t, "tiling": g.tiling()}
    if record:
        out["dts"] = g.dt_history()
    g.close()
    return out


def _oracle_run(oracle, p, W, steps, record=False):
    og = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)
    U, ns, t, rc, h = oracle.run(og, oracle.prim_to_cons(W.astype(np.float64)), np.inf, max_steps=steps,
                                 phi=p.phi, record=record)
    assert rc == 0 and ns == steps
    return U, t, h


# ------------------------------------------------------------------ 2D blast
def test_blast_1024_fp64_all_steps(env, oracle):
    msh, I, s = env
    p = I.blast()
    G = _gpu_run(msh, p, msh.FP64, s, p.nsteps)
    Uo, to, _ = _oracle_run(oracle, p, p.W, p.nsteps)
    assert abs(G["t"] - to) <= 1e-13 * to
    assert_fp64(G["U"], Uo, what=f"blast 1024^2 fp64 tiling={G['tiling']}")


def test_blast_1024_fp32_all_steps(env, oracle):
    msh, I, s = env
    p = I.blast()
    G = _gpu_run(msh, p, msh.FP32, s, p.nsteps)
    Uo, _, _ = _oracle_run(oracle, p, p.W.astype(np.float32), p.nsteps)
    assert_fp32(G["W"], oracle.cons_to_prim(Uo), what=f"blast 1024^2 fp32 tiling={G['tiling']}")


# ------------------------------------------------------------------- 3D box
@pytest.fixture(scope="module")
def box(env):
    msh, I, s = env
    return I.turb()


def test_box_256_all_50_steps_elementwise(env, oracle, box):
    msh, I, s = env
    p = box
    Uo, to, ho = _oracle_run(oracle, p, p.W, p.nsteps, record=True)
    G64 = _gpu_run(msh, p, msh.FP64, s, p.nsteps, record=p.nsteps)
    np.testing.assert_allclose(G64["dts"], ho, rtol=1e-12)
    assert abs(G64["t"] - to) <= 1e-12 * to
    assert_fp64(G64["U"], Uo, what=f"box 256^3 fp64, {p.nsteps} steps, tiling={G64['tiling']}")
    del G64
    Wo = oracle.cons_to_prim(Uo)
    del Uo
    G32 = _gpu_run(msh, p, msh.FP32, s, p.nsteps)
    assert_fp32(G32["W"], Wo, what=f"box 256^3 fp32, {p.nsteps} steps, tiling={G32['tiling']}")


def test_box_256_full_run_properties(env, box):
    msh, I, s = env
    p = box
    res = {}
    for prec in (msh.FP64, msh.FP32):
        g = msh.Grid.from_problem(p, prec, stream=s.cuda_stream)
        W = p.W.astype(np.float32) if prec == msh.FP32 else p.W
        g.set_state(W, msh.PRIMITIVE)
        g.autotune()
        g.set_state(W, msh.PRIMITIVE)
        g.set_time(0.0, 0)
        t0, ok0, _ = g.diagnostics()
        ns, t = g.run(max_steps=p.nsteps)
        t1, ok1, bad = g.diagnostics()
        assert ns == p.nsteps and ok0 and ok1 and bad == -1
        scale = np.array([abs(t0[0])] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
        # FP64: round-off of 16.7M cells x 50 steps; FP32: the state itself is rounded to
        # 2^-24 per cell and per step
        tol = 1e-12 if prec == msh.FP64 else 2e-6
        drift = np.abs(t1 - t0) / scale
        assert np.all(drift < tol), (prec, drift)
        # the device totals against an FP64 sum of the returned state (FP32 grids sum each
        # thread's cells in FP32, then in FP64)
        Ug = g.get_state().astype(np.float64).reshape(10, -1)
        ref_tot = Ug.sum(axis=1)
        tol_tot = 1e-13 if prec == msh.FP64 else 1e-7
        assert np.all(np.abs(t1 - ref_tot) / scale < tol_tot), (prec, (t1 - ref_tot) / scale)
        res[prec] = g.get_state(msh.PRIMITIVE).astype(np.float64)
        g.close()
    e = field_errors(res[msh.FP32], res[msh.FP64], "l1")
    assert e[0] <= 2e-4 and max(e[k] for k in (4, 5, 6, 7, 8, 9)) <= 5e-4, e


# --------------------------------------------------------------------- disc
def test_disc_512_fp32_all_steps(env, oracle):
    msh, I, s = env
    p = I.disc()
    G = _gpu_run(msh, p, msh.FP32, s, p.nsteps)
    Uo, _, _ = _oracle_run(oracle, p, p.W.astype(np.float32), p.nsteps)
    assert_fp32(G["W"], oracle.cons_to_prim(Uo), what=f"disc 512^2 fp32, {p.nsteps} steps")


def test_disc_512_fp64_all_steps(env, oracle):
    msh, I, s = env
    p = I.disc()
    G = _gpu_run(msh, p, msh.FP64, s, p.nsteps)
    Uo, to, _ = _oracle_run(oracle, p, p.W, p.nsteps)
    assert abs(G["t"] - to) <= 1e-12 * to
    assert_fp64(G["U"], Uo, what=f"disc 512^2 fp64, {p.nsteps} steps")


# ------------------------------------------------- corner transport upwind
def _gpu_run_ctu(msh, p, precision, stream, steps, cfl):
    g = msh.Grid(p.n, p.lo, p.hi, p.bc, cfl, precision, stream=stream.cuda_stream)
    g.set_ctu(True)
    W = p.W.astype(np.float32) if precision == msh.FP32 else p.W
    g.set_state(W, msh.PRIMITIVE)
    g.autotune()
    g.set_state(W, msh.PRIMITIVE)
    g.set_time(0.0, 0)
    ns, t = g.run(max_steps=steps)
    assert ns == steps
    out = {"U": g.get_state().astype(np.float64), "W": g.get_state(msh.PRIMITIVE).astype(np.float64), "t": t,
           "tiling": g.tiling()}
    g.close()
    return out


def _oracle_run_ctu(oracle, p, W, steps, cfl):
    og = oracle.Grid(p.n, p.lo, p.hi, p.bc, cfl, ctu=True)
    U, ns, t, rc, _ = oracle.run(og, oracle.prim_to_cons(W.astype(np.float64)), np.inf, max_steps=steps)
    assert rc == 0 and ns == steps
    return U, t


def test_ctu_blast_1024_first_50_steps(env, oracle):
    """The corner-transport-upwind step at CFL 0.8 (the CTU line of the benchmark suite) on
    the full 1024^2 blast: FP64 element by element, FP32 against the FP32-rounded input."""
    msh, I, s = env
    p = I.blast()
    G = _gpu_run_ctu(msh, p, msh.FP64, s, 50, 0.8)
    Uo, to = _oracle_run_ctu(oracle, p, p.W, 50, 0.8)
    assert abs(G["t"] - to) <= 1e-13 * to
    assert_fp64(G["U"], Uo, what=f"ctu blast 1024^2 fp64 tiling={G['tiling']}")
    G = _gpu_run_ctu(msh, p, msh.FP32, s, 50, 0.8)
    Uo, _ = _oracle_run_ctu(oracle, p, p.W.astype(np.float32), 50, 0.8)
    assert_fp32(G["W"], oracle.cons_to_prim(Uo), what=f"ctu blast 1024^2 fp32 tiling={G['tiling']}")


def test_ctu_box_256_first_steps_fp32(env, oracle):
    """The corner-transport-upwind step at CFL 0.6 (the largest realizable one of the
    benchmark suite's ladder) on the full 256^3 box, FP32, its first two steps element by
    element against the oracle run from the FP32-rounded input."""
    msh, I, s = env
    p = I.turb()
    G = _gpu_run_ctu(msh, p, msh.FP32, s, 2, 0.6)
    Uo, to = _oracle_run_ctu(oracle, p, p.W.astype(np.float32), 2, 0.6)
    assert abs(G["t"] - to) <= 1e-5 * to
    assert_fp32(G["W"], oracle.cons_to_prim(Uo), what=f"ctu box 256^3 fp32 tiling={G['tiling']}")
