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
