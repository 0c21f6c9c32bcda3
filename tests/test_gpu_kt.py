"""The Kurganov-Tadmor central scheme (Sec. 3.2) on the GPU against the oracle's KT scheme:
FP64 <= 1e-10 relative L_inf per field after the run, FP32 within 2e-4 (rho) / 5e-4 (P_ij)
relative L1 of the FP64 oracle run from the FP32-rounded input; 1D/2D/3D, every boundary
kind, ragged tiles and strips, several tile shapes, gravity; slabs of a KT grid equal the
single grid; the adjoint refuses the central scheme."""
import numpy as np
import pytest

from paper_1210_5246_gb300 import decomp
from tests.parity import assert_fp32, assert_fp64

pytestmark = pytest.mark.gpu
KT_CFL = 0.4


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import inputs, msh
    msh.load()
    return msh, inputs


def _run(msh, oracle, n, lo, hi, bc, cfl, W, precision, steps=None, t_end=np.inf, phi=None, tiling=None):
    g = msh.Grid(n, lo, hi, bc, cfl, precision)
    g.set_scheme(msh.KT)
    if phi is not None:
        g.set_potential(phi)
    if tiling:
        g.set_tiling(*tiling)
    Wg = W.astype(np.float32) if precision == msh.FP32 else W
    g.set_state(Wg, msh.PRIMITIVE)
    ns, t = g.run(t_end, steps if steps is not None else (1 << 62))
    U = g.get_state().astype(np.float64)
    Wout = g.get_state(msh.PRIMITIVE).astype(np.float64)
    g.close()
    og = oracle.Grid(n, lo, hi, bc, cfl, scheme=oracle.SCHEME_KT)
    Uo, no, to, rc, _ = oracle.run(og, oracle.prim_to_cons(Wg.astype(np.float64)), t_end,
                                   max_steps=steps if steps is not None else (1 << 62), phi=phi)
    # FP32 grids take their dt from FP32 signal speeds
    assert rc == 0 and ns == no and abs(t - to) <= (1e-13 if precision == msh.FP64 else 1e-5) * to
    return U, Wout, Uo, oracle.cons_to_prim(Uo)


def test_sod_fp64(env, oracle):
    msh, I = env
    p = I.sod(256)
    U, _, Uo, _ = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP64, t_end=p.t_end)
    assert_fp64(U, Uo, what="kt sod fp64")


def test_sod_fp32(env, oracle):
    msh, I = env
    p = I.sod(256)
    _, W, _, Wo = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP32, t_end=p.t_end)
    assert_fp32(W, Wo, what="kt sod fp32")


@pytest.mark.parametrize("n,bc", [(5, (0, 0)), (127, (1, 2)), (300, (2, 1))])
def test_1d_ragged_and_boundaries(env, oracle, n, bc):
    msh, _ = env
    rng = np.random.default_rng(n)
    W = np.zeros((10, 1, 1, n))
    W[0] = np.exp(rng.uniform(-0.5, 0.5, (1, 1, n)))
    W[1:4] = rng.uniform(-0.3, 0.3, (3, 1, 1, n))
    W[4], W[7], W[9] = 0.8, 0.7, 0.5
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, (1, 1, n))
    U, _, Uo, _ = _run(msh, oracle, (n,), (0.0,), (1.0,), (bc,), KT_CFL, W, msh.FP64, steps=7)
    assert_fp64(U, Uo, what=f"kt 1d {n}")


@pytest.mark.parametrize("tiling", [(4, 8), (8, 16), (16, 64)])
def test_blast_fp64(env, oracle, tiling):
    msh, I = env
    p = I.blast(n=97, nsteps=15)
    U, _, Uo, _ = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP64, steps=15, tiling=tiling)
    assert_fp64(U, Uo, what=f"kt blast fp64 {tiling}")


def test_blast_fp32(env, oracle):
    msh, I = env
    p = I.blast(n=97, nsteps=15)
    _, W, _, Wo = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP32, steps=15)
    assert_fp32(W, Wo, what="kt blast fp32")


@pytest.mark.parametrize("shape,bc", [((31, 7), ((1, 1), (2, 2))), ((61, 45), ((2, 2), (1, 2)))])
def test_2d_shapes_and_boundaries(env, oracle, shape, bc):
    msh, _ = env
    nx, ny = shape
    rng = np.random.default_rng(nx * 100 + ny)
    W = np.zeros((10, 1, ny, nx))
    W[0] = np.exp(rng.uniform(-0.5, 0.5, (1, ny, nx)))
    W[1:4] = rng.uniform(-0.3, 0.3, (3, 1, ny, nx))
    W[4], W[7], W[9] = 0.8, 0.7, 0.5
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, (1, ny, nx))
    U, _, Uo, _ = _run(msh, oracle, shape, (0.0, 0.0), (1.0, 2.0), bc, KT_CFL, W, msh.FP64, steps=5)
    assert_fp64(U, Uo, what=f"kt 2d {shape}")


@pytest.mark.parametrize("tiling", [(8, 32), (4, 5), (16, 7)])
def test_turb_fp64(env, oracle, tiling):
    msh, I = env
    p = I.turb(n=24, nsteps=5)
    U, _, Uo, _ = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP64, steps=5,
                       tiling=tiling if tiling[0] != 16 else None)
    assert_fp64(U, Uo, what=f"kt turb fp64 {tiling}")


def test_turb_fp32_rows16(env, oracle):
    msh, I = env
    p = I.turb(n=32, nsteps=8)
    _, W, _, Wo = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP32, steps=8, tiling=(16, 7))
    assert_fp32(W, Wo, what="kt turb fp32")


@pytest.mark.parametrize("shape,bc", [((33, 17, 9), ((1, 2), (2, 1), (0, 0))), ((5, 40, 3), ((2, 2), (0, 0), (1, 1)))])
def test_3d_shapes_and_boundaries(env, oracle, shape, bc):
    msh, _ = env
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + 7 * ny + 31 * nz)
    W = np.zeros((10, nz, ny, nx))
    W[0] = np.exp(rng.uniform(-0.5, 0.5, (nz, ny, nx)))
    W[1:4] = rng.uniform(-0.3, 0.3, (3, nz, ny, nx))
    W[4], W[7], W[9] = 0.8, 0.7, 0.6
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, (nz, ny, nx))
    U, _, Uo, _ = _run(msh, oracle, shape, (0, 0, 0), (1, 1.5, 0.5), bc, KT_CFL, W, msh.FP64, steps=4, tiling=(8, 4))
    assert_fp64(U, Uo, what=f"kt 3d {shape}")


def test_disc_gravity(env, oracle):
    msh, I = env
    p = I.disc(n=64, nsteps=15)
    U, _, Uo, _ = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP64, steps=15, phi=p.phi)
    assert_fp64(U, Uo, what="kt disc fp64")
    _, W, _, Wo = _run(msh, oracle, p.n, p.lo, p.hi, p.bc, KT_CFL, p.W, msh.FP32, steps=15, phi=p.phi)
    assert_fp32(W, Wo, what="kt disc fp32")


def test_switching_schemes(env, oracle):
    """A grid switched to KT and back steps like a grid that never left MUSCL-Hancock."""
    msh, I = env
    p = I.blast(n=40, nsteps=4)
    a = msh.Grid.from_problem(p, msh.FP64)
    b = msh.Grid.from_problem(p, msh.FP64)
    b.set_scheme(msh.KT)
    b.set_scheme(msh.MUSCL_HANCOCK)
    for g in (a, b):
        g.set_state(p.W, msh.PRIMITIVE)
        g.run(max_steps=4)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_kt_slabs_equal_single_grid(env):
    msh, I = env
    p = I.turb(n=20, nsteps=4)
    g = msh.Grid(p.n, p.lo, p.hi, p.bc, KT_CFL, msh.FP64)
    g.set_scheme(msh.KT)
    g.set_state(p.W, msh.PRIMITIVE)
    U0 = g.get_state()
    g.run(max_steps=4)
    ref, (t_ref, _) = g.get_state(), g.time()
    g.close()
    S = decomp.Slabs(p.n[-1], 3, True, halo=decomp.halo_width(msh.KT))
    st = decomp.make_grid_steppers(msh, p.n, p.lo, p.hi, p.bc, KT_CFL, msh.FP64, U0, S, range(3), scheme=msh.KT)
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(4)
    assert ns == 4 and t == t_ref
    np.testing.assert_array_equal(decomp.join_owned([st[r].g.get_state() for r in range(3)], p.n, S), ref)
    for s in st.values():
        s.g.close()


def test_adjoint_refuses_kt(env):
    msh, I = env
    p = I.sod(32)
    g = msh.Grid.from_problem(p, msh.FP64)
    g.set_state(p.W, msh.PRIMITIVE)
    g.set_scheme(msh.KT)
    U0 = g.get_state()
    for call in (lambda: g.adjoint_run(U0, [1e-3], U0, K=1), lambda: g.set_tape(2, 4)):
        with pytest.raises(msh.MshError) as ei:
            call()
        assert ei.value.status == msh.MSH_E_STATE
    with pytest.raises(msh.MshError) as ei:
        g.set_scheme(7)
    assert ei.value.status == msh.MSH_E_INVALID_ARG
    g.close()
