"""3D steps that stage their planes by bulk tensor copies, against the oracle.

The 3D step stages every plane of a tile with one bulk tensor copy of the box from the
4-cell-aligned column xs = (x0 - 2) & ~3 and row y0 - 2 when a row of nx cells is a
multiple of 16 bytes; cells of the box outside the grid arrive as zeros and are fixed up
from their mapped cells (periodic wrap, mirror images, outflow) once the copy has landed.
The grids here hold tiles of every kind (x tiles at x0 = 0, 30 and 60: boxes from -4, 28
and 56, the staged box 2, 0 and 2 columns into them; edge tiles in x and y; tiles inside),
with every boundary kind in x, y and z (mirror planes take the z sign flips of the copied
plane), every tiling of the step (16, 8 and 4 rows; two raw slots for 8 and 4 rows), every
scheme that stages this way (MUSCL-Hancock with HLL, Roe-type and HLLC fluxes, both stages
of the central scheme) and a run whose a-posteriori fallback tags cells.  FP64 <= 1e-10
relative L_inf per field, FP32 within 2e-4 (rho) / 5e-4 (P_ij) relative L1 of the FP64
oracle from the FP32-rounded input.  A grid whose rows are not a multiple of 16 bytes
(nx = 94 in FP32, 97 in both precisions) stages every tile cell by cell and must give the
same answer.  zchunk 0 is the balanced tiling (equal plane counts per block: whole
columns, then runs of the rest window by window); a grid with more columns of tiles than
the device has block slots takes both parts."""
import numpy as np
import pytest

from tests.parity import assert_fp32, assert_fp64
from tests.test_gpu_parity import _extreme

pytestmark = pytest.mark.gpu

# (name in the binding, oracle scheme number, CFL)
SCHEMES = {"MH": ("MUSCL_HANCOCK", 0, 0.5), "ROE": ("MUSCL_HANCOCK_ROE", 2, 0.5),
           "HLLC": ("MUSCL_HANCOCK_HLLC", 3, 0.5), "KT": ("KT", 1, 0.4)}


@pytest.fixture(scope="module")
def msh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import msh as m
    m.load()
    return m


def _state(shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    W = np.zeros((10, nz, ny, nx))
    W[0] = np.exp(rng.uniform(-0.5, 0.5, (nz, ny, nx)))
    W[1:4] = rng.uniform(-0.3, 0.3, (3, nz, ny, nx))
    W[4], W[7], W[9] = 0.8, 0.7, 0.6
    for k in (5, 6, 8):
        W[k] = rng.uniform(-0.1, 0.1, (nz, ny, nx))
    return W


def _run(msh, oracle, n, bc, W, precision, scheme, rows, zchunk, steps):
    name, osch, cfl = SCHEMES[scheme]
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.5, 0.125)
    g = msh.Grid(n, lo, hi, bc, cfl, precision)
    if scheme != "MH":
        g.set_scheme(getattr(msh, name))
    g.set_tiling(rows, zchunk)
    Wg = W.astype(np.float32) if precision == msh.FP32 else W
    g.set_state(Wg, msh.PRIMITIVE)
    ns, t = g.run(np.inf, steps)
    U = g.get_state().astype(np.float64)
    Wout = g.get_state(msh.PRIMITIVE).astype(np.float64)
    g.close()
    og = oracle.Grid(n, lo, hi, bc, cfl, scheme=osch)
    Uo, no, to, rc, _ = oracle.run(og, oracle.prim_to_cons(Wg.astype(np.float64)), np.inf, max_steps=steps)
    assert rc == 0 and ns == no == steps
    assert abs(t - to) <= (1e-13 if precision == msh.FP64 else 1e-5) * to
    return U, Wout, Uo, oracle.cons_to_prim(Uo)


# z boundaries: periodic, mirror on both sides, outflow below and mirror above
BCS = {"zper": ((0, 0), (0, 0), (0, 0)), "zrefl": ((1, 1), (0, 0), (2, 2)), "zmix": ((2, 1), (1, 2), (1, 2))}


@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("rows,zchunk", [(8, 5), (4, 12), (8, 0)])
def test_mh_fp64_mixed_tiles(msh, oracle, bcname, rows, zchunk):
    n = (96, 46, 12)
    W = _state(n[::-1], 11)
    U, _, Uo, _ = _run(msh, oracle, n, BCS[bcname], W, msh.FP64, "MH", rows, zchunk, 4)
    assert_fp64(U, Uo, what=f"bulk-staged mh fp64 {bcname} rows={rows}")


@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("rows,zchunk", [(16, 5), (8, 12), (4, 3), (16, 0), (4, 0)])
def test_mh_fp32_mixed_tiles(msh, oracle, bcname, rows, zchunk):
    n = (96, 46, 12)
    W = _state(n[::-1], 12)
    _, Wg, _, Wo = _run(msh, oracle, n, BCS[bcname], W, msh.FP32, "MH", rows, zchunk, 4)
    assert_fp32(Wg, Wo, what=f"bulk-staged mh fp32 {bcname} rows={rows}")


@pytest.mark.parametrize("scheme", ["ROE", "HLLC", "KT"])
@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_other_schemes_mixed_tiles(msh, oracle, scheme, precision):
    n = (96, 46, 10)
    W = _state(n[::-1], 13)
    if scheme == "ROE":  # eigenvalues off zero (the upwind tracing switches at zero speed)
        W[1] += 0.25
        W[2] -= 0.15
    p = getattr(msh, precision)
    rows = 16 if precision == "FP32" else 8
    U, Wg, Uo, Wo = _run(msh, oracle, n, BCS["zmix"], W, p, scheme, rows, 4, 3)
    if precision == "FP64":
        assert_fp64(U, Uo, what=f"bulk-staged {scheme} fp64")
    else:
        assert_fp32(Wg, Wo, what=f"bulk-staged {scheme} fp32")


@pytest.mark.parametrize("nx", [94, 97])
@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_rows_off_the_copy_alignment(msh, oracle, nx, precision):
    n = (nx, 40, 8)
    W = _state(n[::-1], nx)
    p = getattr(msh, precision)
    U, Wg, Uo, Wo = _run(msh, oracle, n, BCS["zrefl"], W, p, "MH", 16 if precision == "FP32" else 8, 8, 3)
    if precision == "FP64":
        assert_fp64(U, Uo, what=f"nx={nx} fp64")
    else:
        assert_fp32(Wg, Wo, what=f"nx={nx} fp32")


def test_fallback_with_bulk_staged_tiles_fp64(msh, oracle):
    """Extreme states over 3 steps of the oracle's dt schedule: the step stages by bulk
    copies, the fallback passes (which tag cells here) stage cell by cell."""
    n = (92, 44, 8)
    W = _extreme(n[::-1], 5)
    bc = ((0, 0), (1, 2), (2, 2))
    og = oracle.Grid(n, (0, 0, 0), (1, 1, 1), bc, 0.5)
    Uo, no, to, rc, dts = oracle.run(og, oracle.prim_to_cons(W), np.inf, max_steps=3, record=True)
    assert rc == 0 and no == 3
    g = msh.Grid(n, (0, 0, 0), (1, 1, 1), bc, 0.5, msh.FP64)
    g.set_tiling(8, 8)
    g.set_state(W, msh.PRIMITIVE)
    tagged = [g.step_dt(float(dt)) for dt in dts]
    assert sum(tagged) > 0, "the extreme state should make the fallback tag cells"
    assert_fp64(g.get_state(), Uo, what="bulk-staged fallback fp64")
    g.close()


@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_balanced_tiling_whole_columns_and_runs(msh, oracle, precision):
    """600 x 120 x 12 cells: 20 x 9 = 180 columns of 16-row tiles (8-row in FP64: 20 x 20),
    more than one per block slot, so blocks stream whole columns and then runs of the
    columns left over."""
    n = (600, 120, 12)
    W = _state(n[::-1], 21)
    p = getattr(msh, precision)
    rows = 16 if precision == "FP32" else 8
    U, Wg, Uo, Wo = _run(msh, oracle, n, BCS["zmix"], W, p, "MH", rows, 0, 3)
    if precision == "FP64":
        assert_fp64(U, Uo, what="balanced fp64")
    else:
        assert_fp32(Wg, Wo, what="balanced fp32")


def test_bulk_copy_wait_runs_out(msh):
    """The bound on the waits for bulk copies: with the test hook, thread block 0 of the next
    step leaves its first copy out, the threads waiting for that plane give up after about
    2^31 SM clocks, and the step returns MSH_E_TIMEOUT instead of hanging.  The context stays
    usable: after msh_set_state the grid steps exactly as a fresh grid does, and a second
    step without the hook succeeds."""
    n = (96, 46, 12)
    W = _state(n[::-1], 31).astype(np.float32)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.5, 0.125)

    def grid():
        g = msh.Grid(n, lo, hi, BCS["zper"], 0.5, msh.FP32)
        g.set_tiling(16, 0)
        g.set_state(W, msh.PRIMITIVE)
        return g

    g = grid()
    g.set_test_fault(1)
    with pytest.raises(msh.MshError) as ei:
        g.step()
    assert ei.value.status == msh.MSH_E_TIMEOUT
    g.set_state(W, msh.PRIMITIVE)
    g.step()
    g.step()
    ref = grid()
    ref.step()
    ref.step()
    assert np.array_equal(g.get_state(), ref.get_state())
    g.close()
    ref.close()
