"""Slab decomposition with libmsh grids on one GPU: the slabs of one process (the
in-process form of the multi-GPU path; no kernel waits on another) advance in lockstep
through msh_get_slab / msh_set_slab / msh_reduce_layers / msh_step_dt and must reproduce
the single-grid run bit for bit, in FP64 and FP32."""
import numpy as np
import pytest

from paper_1210_5246_gb300 import decomp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs


def _problem(I, name):
    if name == "box3d":
        p = I.turb(n=20, nsteps=5)
        return p, 5
    if name == "blast2d":
        p = I.blast(n=64, nsteps=6)
        return p, 6
    if name == "disc2d":
        p = I.disc(n=48, nsteps=6)
        return p, 6
    if name == "sod1d":
        p = I.sod(96)
        return p, 8
    raise KeyError(name)


@pytest.mark.parametrize("name,world", [("box3d", 3), ("box3d", 2), ("blast2d", 4), ("disc2d", 3), ("sod1d", 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_slabs_equal_single_grid(env, name, world, prec):
    msh, I = env
    p, steps = _problem(I, name)
    precision = msh.FP64 if prec == "fp64" else msh.FP32
    W = p.W.astype(np.float32) if precision == msh.FP32 else p.W
    g = msh.Grid.from_problem(p, precision)
    g.set_state(W, msh.PRIMITIVE)
    U0 = g.get_state()
    g.run(max_steps=steps)
    ref, (t_ref, _) = g.get_state(), g.time()
    tot_ref, _, _ = g.diagnostics()
    g.close()
    S = decomp.Slabs(p.n[-1], world, p.bc[-1][0] == 0)
    st = decomp.make_grid_steppers(msh, p.n, p.lo, p.hi, p.bc, p.cfl, precision, U0, S, range(world), phi=p.phi)
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].g.get_state() for r in range(world)], p.n, S)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref)
    tot, _, ok = drv.reduce()
    assert ok
    # FP32 grids sum each thread's cells in FP32 before the FP64 reduction
    scale = np.abs(tot_ref).max()
    tol = 1e-12 if precision == msh.FP64 else 1e-7
    np.testing.assert_allclose(tot, tot_ref, rtol=tol, atol=tol * scale)
    for s in st.values():
        s.g.close()


def test_slab_calls(env):
    msh, I = env
    p, _ = _problem(I, "box3d")
    g = msh.Grid.from_problem(p, msh.FP64)
    g.set_state(p.W, msh.PRIMITIVE)
    U = g.get_state()
    layers, per = g.layer_shape()
    assert (layers, per) == (p.n[2], p.n[0] * p.n[1])
    # get_slab returns the layers of every field
    s = g.get_slab(3, 4)
    np.testing.assert_array_equal(s.reshape(10, 4, p.n[1], p.n[0]), U[:, 3:7])
    # set_slab writes them back elsewhere
    g.set_slab(10, 4, s)
    V = g.get_state()
    np.testing.assert_array_equal(V[:, 10:14], U[:, 3:7])
    # reductions over a range of layers equal the totals of those layers
    tot, dt, ok = g.reduce_layers(10, 4)
    np.testing.assert_allclose(tot, V[:, 10:14].reshape(10, -1).sum(axis=1), rtol=1e-13, atol=1e-13)
    tot_all, dt_all, _ = g.reduce_layers(0, layers)
    assert ok and dt >= dt_all > 0
    # a step with a fixed dt advances the time by exactly dt
    t0 = g.time()[0]
    assert g.step_dt(0.5 * dt_all) == 0
    assert g.time() == (t0 + 0.5 * dt_all, 1)
    for bad in [(-1, 2), (layers - 1, 2)]:
        with pytest.raises(msh.MshError) as ei:
            g.get_slab(*bad)
        assert ei.value.status == msh.MSH_E_INVALID_ARG
    with pytest.raises(msh.MshError):
        g.step_dt(0.0)
    with pytest.raises(msh.MshError):
        g.set_cell_width((0.1, -1.0, 0.1))
    g.close()


def test_cell_width_override(env):
    """A grid whose widths are set explicitly steps like one built with those widths."""
    msh, I = env
    p, steps = _problem(I, "disc2d")
    a = msh.Grid.from_problem(p, msh.FP64)
    b = msh.Grid(p.n, (0.0, 0.0), (1.0, 1.0), p.bc, p.cfl, msh.FP64)
    b.set_cell_width(tuple((p.hi[d] - p.lo[d]) / p.n[d] for d in range(2)))
    b.set_potential(p.phi)
    for g in (a, b):
        g.set_state(p.W, msh.PRIMITIVE)
        g.run(max_steps=steps)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("name,world,cfl", [("box3d", 3, 0.5), ("blast2d", 4, 0.8)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ctu_slabs_equal_single_grid(env, name, world, cfl, prec):
    """The corner-transport-upwind form across slabs: bit-identical to the single grid (at
    CFL numbers whose steps tag no fallback cell, which would couple the slabs within a
    step; the box tags one in its third step at 0.8)."""
    msh, I = env
    p, steps = _problem(I, name)
    precision = msh.FP64 if prec == "fp64" else msh.FP32
    W = p.W.astype(np.float32) if precision == msh.FP32 else p.W
    g = msh.Grid(p.n, p.lo, p.hi, p.bc, cfl, precision)
    g.set_ctu(True)
    g.set_state(W, msh.PRIMITIVE)
    U0 = g.get_state()
    g.run(max_steps=steps)
    ref, (t_ref, _) = g.get_state(), g.time()
    g.close()
    S = decomp.Slabs(p.n[-1], world, p.bc[-1][0] == 0)
    st = decomp.make_grid_steppers(msh, p.n, p.lo, p.hi, p.bc, cfl, precision, U0, S, range(world), ctu=True)
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].g.get_state() for r in range(world)], p.n, S)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref)
    for s in st.values():
        s.g.close()


def _extreme_2d():
    """The extreme 2D periodic case of the CPU decomposition tests (density contrasts up to
    2000, velocity jumps up to 6, CFL 0.9): the fallback tags cells next to every slab
    boundary."""
    from tests.test_decomp import _extreme_2d as mk
    return mk()


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fallback_across_slabs_equals_single_grid(env, world, prec):
    """libmsh slabs sharing the a-posteriori fallback (msh_step_begin / msh_get_tags /
    msh_set_tags / msh_count_tags / msh_step_retry / msh_step_end): bit for bit the single
    grid's msh_step_dt run, with tags on both sides of every slab boundary; FP64 also
    against the oracle."""
    msh, I = env
    precision = msh.FP64 if prec == "fp64" else msh.FP32
    W = _extreme_2d()
    W = W.astype(np.float32) if precision == msh.FP32 else W
    n, lo, hi, bc, cfl, steps = (14, 24), (0.0, 0.0), (1.0, 1.0), ((0, 0), (0, 0)), 0.9, 3
    g = msh.Grid(n, lo, hi, bc, cfl, precision)
    g.set_state(W, msh.PRIMITIVE)
    U0 = g.get_state()
    g.run(max_steps=steps)
    ref, (t_ref, _) = g.get_state(), g.time()
    g.close()
    S = decomp.Slabs(n[-1], world, True)
    st = decomp.make_grid_steppers(msh, n, lo, hi, bc, cfl, precision, U0, S, range(world))
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].g.get_state() for r in range(world)], n, S)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref)
    if precision == msh.FP64:
        from oracle import oracle
        from tests.parity import assert_fp64
        og = oracle.Grid(n, lo, hi, bc, cfl)
        Uo, so, to, rc, _ = oracle.run(og, oracle.prim_to_cons(W), np.inf, max_steps=steps)
        assert rc == 0
        assert_fp64(got, Uo, what=f"fallback across {world} slabs")
    for r in range(world):
        st[r].g.close()


def test_phased_step_equals_step_dt_and_tags_round_trip(env):
    """On one grid, msh_step_begin + the passes msh_step_dt would run + msh_step_end give the
    msh_step_dt result bit for bit; msh_get_tags / msh_set_tags / msh_count_tags agree with
    one another; retry out of order and end without begin are refused."""
    msh, I = env
    W = _extreme_2d()
    n, lo, hi, bc, cfl = (14, 24), (0.0, 0.0), (1.0, 1.0), ((0, 0), (0, 0)), 0.9
    a = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    a.set_state(W, msh.PRIMITIVE)
    dt = a.step()  # the CFL step: the reference
    b = msh.Grid(n, lo, hi, bc, cfl, msh.FP64)
    b.set_state(W, msh.PRIMITIVE)
    b.step_begin(dt)
    levels = b.get_tags(0, n[1])
    assert (levels == 0).sum() == b.count_tags(0, n[1], 0) > 0 and set(np.unique(levels)) <= {-1, 0}
    lvl = 1
    while lvl <= 4 and b.count_tags(0, n[1], lvl - 1) > 0:
        b.step_retry(lvl)
        lvl += 1
    with pytest.raises(msh.MshError):
        b.step_retry(lvl + 1)
    b.step_end()
    np.testing.assert_array_equal(b.get_state(), a.get_state())
    assert b.time() == a.time()
    with pytest.raises(msh.MshError) as ei:
        b.step_end()
    assert ei.value.status == msh.MSH_E_STATE
    # tags written by msh_set_tags are read back (the current step's tag of each cell)
    b.step_begin(dt)
    rng = np.random.default_rng(1)
    lv = rng.integers(-1, 3, n[0] * 5).astype(np.int32)
    b.set_tags(3, 5, lv)
    np.testing.assert_array_equal(b.get_tags(3, 5), lv)
    assert b.count_tags(3, 5, 2) == int((lv == 2).sum())
    with pytest.raises(msh.MshError) as ei:  # no fallback pass ran: the update is not realizable
        b.step_end()
    assert ei.value.status == msh.MSH_E_REALIZABILITY
    a.close()
    b.close()

