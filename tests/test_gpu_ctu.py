"""The corner-transport-upwind form of the characteristic schemes on the GPU (transverse
terms of every other direction in the face states, max-form CFL rule) against the oracle's:
FP64 <= 1e-10 relative L_inf per field, FP32 within the FP32 tolerances; HLL, Roe-type and
HLLC fluxes; 2D strips and 3D tiles of every shape, every boundary kind, gravity, the
a-posteriori fallback; no effect in 1D; switching re-plans the step; refusals."""
import numpy as np
import pytest

from tests.parity import assert_fp32, assert_fp64
from tests.test_gpu_parity import _extreme

pytestmark = pytest.mark.gpu
# (name of the scheme in the binding, oracle scheme number)
SCHEMES = [("MUSCL_HANCOCK", 0), ("MUSCL_HANCOCK_ROE", 2), ("MUSCL_HANCOCK_HLLC", 3)]


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs


@pytest.fixture(params=SCHEMES, ids=[s[0] for s in SCHEMES])
def scheme(request):
    return request.param


def _run(msh, oracle, scheme, n, lo, hi, bc, cfl, W, precision, steps=None, t_end=np.inf, phi=None, tiling=None):
    g = msh.Grid(n, lo, hi, bc, cfl, precision)
    g.set_scheme(getattr(msh, scheme[0]))
    g.set_ctu(True)
    assert g.get_ctu()
    if phi is not None:
        g.set_potential(phi)
    if tiling:
        g.set_tiling(*tiling)
    Wg = W.astype(np.float32) if precision == msh.FP32 else W
    g.set_state(Wg, msh.PRIMITIVE)
    ns, t = g.run(t_end, steps if steps is not None else (1 << 62))
    U, Wout = g.get_state().astype(np.float64), g.get_state(msh.PRIMITIVE).astype(np.float64)
    g.close()
    og = oracle.Grid(n, lo, hi, bc, cfl, scheme=scheme[1], ctu=True)
    Uo, no, to, rc, _ = oracle.run(og, oracle.prim_to_cons(Wg.astype(np.float64)), t_end,
                                   max_steps=steps if steps is not None else (1 << 62), phi=phi)
    assert rc == 0 and ns == no and abs(t - to) <= (1e-13 if precision == msh.FP64 else 1e-5) * to
    return U, Wout, Uo, oracle.cons_to_prim(Uo)


def _blast_W(p, scheme):
    """The blast's initial state; for the Roe-type scheme with a uniform drift.  Its upwind
    tracing (eqs 40-43) is discontinuous where an eigenvalue crosses zero (a wave of speed
    0+ enters the face state with weight 1/2, one of speed 0- with 1/2 - nu max(u + cf, 0)),
    and the blast's contact waves sit at exactly u = 0 in a noisy density: which side of
    zero their speeds fall on after the first step is decided by rounding, so the GPU and the
    oracle could take different branches.  A drift moves the eigenvalues off zero."""
    W = p.W.copy()
    if scheme[0] == "MUSCL_HANCOCK_ROE":
        W[1] += 0.25
        W[2] -= 0.15
    return W


def _random(shape, seed):
    rng = np.random.default_rng(seed)
    W = np.zeros((10,) + shape)
    W[0] = np.exp(rng.uniform(-0.5, 0.5, shape))
    W[1:4] = rng.uniform(-0.3, 0.3, (3,) + shape)
    W[4], W[7], W[9] = 0.8, 0.7, 0.6
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, shape)
    return W


@pytest.mark.parametrize("tiling", [(4, 8), (8, 16), (16, 64)])
def test_blast(env, oracle, scheme, tiling):
    msh, I = env
    p = I.blast(n=97, nsteps=12)
    U, _, Uo, _ = _run(msh, oracle, scheme, p.n, p.lo, p.hi, p.bc, 0.8, _blast_W(p, scheme), msh.FP64, steps=12,
                       tiling=tiling)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} blast {tiling}")


def test_blast_fp32(env, oracle, scheme):
    msh, I = env
    p = I.blast(n=97, nsteps=12)
    _, W, _, Wo = _run(msh, oracle, scheme, p.n, p.lo, p.hi, p.bc, 0.8, _blast_W(p, scheme), msh.FP32, steps=12)
    assert_fp32(W, Wo, what=f"ctu {scheme[0]} blast fp32")


@pytest.mark.parametrize("shape,bc", [((31, 7), ((1, 1), (2, 2))), ((61, 45), ((2, 2), (1, 2))),
                                      ((40, 33), ((0, 0), (0, 0)))])
def test_2d_shapes(env, oracle, scheme, shape, bc):
    msh, _ = env
    W = _random((1, shape[1], shape[0]), shape[0] * 100 + shape[1])
    U, _, Uo, _ = _run(msh, oracle, scheme, shape, (0.0, 0.0), (1.0, 2.0), bc, 0.8, W, msh.FP64, steps=5)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} 2d {shape}")


@pytest.mark.parametrize("tiling", [(8, 32), (4, 5)])
def test_turb(env, oracle, scheme, tiling):
    msh, I = env
    p = I.turb(n=24, nsteps=5)
    U, _, Uo, _ = _run(msh, oracle, scheme, p.n, p.lo, p.hi, p.bc, 0.8, p.W, msh.FP64, steps=5, tiling=tiling)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} turb {tiling}")


@pytest.mark.parametrize("tiling", [(16, 7), (8, 32), (4, 9)])
def test_turb_fp32(env, oracle, scheme, tiling):
    msh, I = env
    p = I.turb(n=32, nsteps=8)
    _, W, _, Wo = _run(msh, oracle, scheme, p.n, p.lo, p.hi, p.bc, 0.8, p.W, msh.FP32, steps=8, tiling=tiling)
    assert_fp32(W, Wo, what=f"ctu {scheme[0]} turb fp32 {tiling}")


@pytest.mark.parametrize("shape,bc", [((33, 17, 9), ((1, 2), (2, 1), (0, 0))),
                                      ((31, 15, 6), ((2, 2), (0, 0), (1, 2)))])
def test_3d_shapes(env, oracle, scheme, shape, bc):
    msh, _ = env
    W = _random(tuple(reversed(shape)), sum(shape))
    U, _, Uo, _ = _run(msh, oracle, scheme, shape, (0, 0, 0), (1, 1.5, 0.5), bc, 0.8, W, msh.FP64, steps=4,
                       tiling=(8, 4))
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} 3d {shape}")


def test_disc_gravity(env, oracle, scheme):
    msh, I = env
    p = I.disc(n=64, nsteps=12)
    U, _, Uo, _ = _run(msh, oracle, scheme, p.n, p.lo, p.hi, p.bc, 0.8, p.W, msh.FP64, steps=12, phi=p.phi)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} disc")


@pytest.mark.parametrize("shape,n,bc,cfl", [((1, 12, 12), (12, 12), ((0, 0), (1, 2)), 0.5),
                                            ((6, 7, 9), (9, 7, 6), ((2, 1), (0, 0), (1, 1)), 0.5)])
def test_fallback(env, oracle, scheme, shape, n, bc, cfl):
    msh, _ = env
    nd = len(n)
    U, _, Uo, _ = _run(msh, oracle, scheme, n, (0,) * nd, (1,) * nd, bc, cfl, _extreme(shape, 0), msh.FP64, steps=20)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} fallback {n}")


@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_supersonic_drift(env, oracle, scheme, sgn):
    """Every wave moving one way along x and y: the one-sided branches of the transverse terms."""
    msh, _ = env
    shape = (1, 19, 37)
    W = _random(shape, 5)
    W[1] += sgn * 3.0 * np.sqrt(3 * W[4] / W[0])
    W[2] -= sgn * 3.0 * np.sqrt(3 * W[7] / W[0])
    U, _, Uo, _ = _run(msh, oracle, scheme, (37, 19), (0.0, 0.0), (1.0, 1.0), ((0, 0), (1, 1)), 0.8, W, msh.FP64,
                       steps=6)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} supersonic {sgn}")


def test_no_effect_in_1d(env):
    msh, I = env
    p = I.sod(128)
    outs = []
    for ctu in (False, True):
        g = msh.Grid.from_problem(p, msh.FP64)
        g.set_ctu(ctu)
        g.set_state(p.W, msh.PRIMITIVE)
        g.run(p.t_end)
        outs.append(g.get_state())
        g.close()
    np.testing.assert_array_equal(outs[0], outs[1])


def test_switch_replans_step(env, oracle):
    """The planned step follows the CFL rule in force: the max form after switching on, the
    sum form after switching off again (both against the oracle's rule)."""
    msh, I = env
    p = I.turb(n=16, nsteps=1)
    g = msh.Grid.from_problem(p, msh.FP64)
    g.set_state(p.W, msh.PRIMITIVE)
    U = oracle.prim_to_cons(p.W)
    for ctu in (True, False, True):
        g.set_ctu(ctu)
        dt = g.step()
        og = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl, ctu=ctu)
        assert abs(dt - oracle.cfl_dt(og, U)) <= 1e-13 * dt
        g.set_state(p.W, msh.PRIMITIVE)
    g.close()


def test_refusals(env):
    msh, I = env
    p = I.blast(n=16, nsteps=1)
    g = msh.Grid.from_problem(p, msh.FP64)
    g.set_state(p.W, msh.PRIMITIVE)
    g.set_scheme(msh.KT)
    with pytest.raises(msh.MshError) as ei:
        g.set_ctu(True)
    assert ei.value.status == msh.MSH_E_STATE
    g.set_scheme(msh.MUSCL_HANCOCK)
    g.set_ctu(True)
    with pytest.raises(msh.MshError) as ei:
        g.set_scheme(msh.KT)
    assert ei.value.status == msh.MSH_E_STATE
    U0 = g.get_state()
    with pytest.raises(msh.MshError) as ei:
        g.adjoint_run(U0, [1e-4], U0, K=1)
    assert ei.value.status == msh.MSH_E_STATE
    with pytest.raises(msh.MshError) as ei:
        g.set_tape(1, 4)
    assert ei.value.status == msh.MSH_E_STATE
    g.close()


@pytest.mark.parametrize("n,bc", [((2, 3), ((2, 2), (2, 1))), ((3, 2), ((1, 2), (0, 0))),
                                  ((2, 2, 2), ((2, 2), (2, 2), (2, 2))), ((3, 2, 4), ((2, 1), (0, 0), (2, 2)))])
def test_tiny_grids(env, oracle, scheme, n, bc):
    """Grids of two or three cells per axis: nearly every neighbour a transverse term reads is
    a boundary image, the corner images with reflections along two axes at once."""
    msh, _ = env
    nd = len(n)
    shape = tuple(reversed(n)) if nd == 3 else (1,) + tuple(reversed(n))
    W = _random(shape, sum(n) + 11)
    U, _, Uo, _ = _run(msh, oracle, scheme, n, (0,) * nd, (1,) * nd, bc, 0.7, W, msh.FP64, steps=6)
    assert_fp64(U, Uo, what=f"ctu {scheme[0]} tiny {n}")
