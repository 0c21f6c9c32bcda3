"""Slab decomposition on the CPU: the driver's host logic (partition, halo exchange, global
dt and totals) with the FP64 oracle stepping each slab, in one process and as two gloo
ranks.  Every case must reproduce the single-grid oracle run bit for bit: a slab's owned
cells see exactly the neighbour values and the dt of the whole grid."""
import math
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1210_5246_gb300 import decomp, inputs


class OracleStepper:
    """A slab stepped by the oracle (test helper)."""

    def __init__(self, oracle, n, lo, hi, bc, cfl, U, dx, phi=None, scheme=0, ctu=False):
        self.o = oracle
        self.n, self.bc, self.cfl, self.dx = tuple(n), tuple(bc), cfl, tuple(dx)
        self.scheme, self.ctu = scheme, ctu
        self.g = self._grid(self.n)
        self.U = np.array(U, dtype=np.float64).reshape((10,) + (1,) * (3 - len(n)) + tuple(reversed(n)))
        self.phi = phi
        self.ax = 4 - len(n)

    def _grid(self, n):
        """Oracle grid of n cells with this slab's cell widths set exactly."""
        g = self.o.Grid(n, (0.0,) * len(n), tuple(m * d for m, d in zip(n, self.dx)), self.bc, self.cfl,
                        scheme=self.scheme, ctu=self.ctu)
        for d, w in enumerate(self.dx):
            g._g.dx[d] = w
        return g

    def layers(self):
        return self.n[-1]

    def _sl(self, start, count):
        s = [slice(None)] * 4
        s[self.ax] = slice(start, start + count)
        return tuple(s)

    def get(self, start, count):
        return self.U[self._sl(start, count)].reshape(10, -1).copy()

    def set(self, start, count, buf):
        shape = list(self.U.shape)
        shape[self.ax] = count
        self.U[self._sl(start, count)] = np.asarray(buf).reshape(shape)

    def reduce(self, start, count):
        g = self._grid(self.n[:-1] + (count,))
        Us = np.ascontiguousarray(self.U[self._sl(start, count)])
        tot, ok, _ = self.o.diagnostics(g, Us)
        return np.asarray(tot), self.o.cfl_dt(g, Us), bool(ok)

    def step(self, dt):
        self.U = self.o.step(self.g, self.U, dt, phi=self.phi).reshape(self.U.shape)
        return 0

    # the shared a-posteriori fallback, pass by pass (the oracle's og_step repeats og_step_pass
    # with the growing tagged set on one grid; here the driver decides when a pass runs)
    @property
    def phased(self):
        return self.scheme != 1

    def begin(self, dt):
        self.dt = dt
        self.Unew = self.o.step_pass(self.g, self.U, dt, None, phi=self.phi)
        self.tags = np.where(self.o.realizable_cells(self.g, self.Unew), -1, 0).astype(np.int32)

    def retry(self, level):
        self.Unew = self.o.step_pass(self.g, self.U, self.dt, self.tags >= 0, phi=self.phi)
        new = ~self.o.realizable_cells(self.g, self.Unew) & (self.tags < 0)
        self.tags[new] = level

    def end(self):
        self.U = self.Unew.reshape(self.U.shape)
        return int((self.tags == 0).sum())

    def _tsl(self, start, count):
        s = [slice(None)] * 3
        s[self.ax - 1] = slice(start, start + count)
        return tuple(s)

    def count_tags(self, start, count, level):
        return int((self.tags[self._tsl(start, count)] == level).sum())

    def get_tags(self, start, count):
        return self.tags[self._tsl(start, count)].reshape(-1).copy()

    def set_tags(self, start, count, levels):
        t = self.tags[self._tsl(start, count)]
        self.tags[self._tsl(start, count)] = np.asarray(levels, dtype=np.int32).reshape(t.shape)


def _extreme_2d(n=(14, 24), seed=4):
    """2D periodic states with density contrasts of up to 2000 and velocity jumps of up to 6:
    at CFL 0.9 the second-order update of 44 cells of the first step is not realizable, in
    every row of the grid, so the a-posteriori fallback tags cells on both sides of every
    slab boundary (and in the next steps a few more)."""
    rng = np.random.default_rng(seed)
    nx, ny = n
    W = np.zeros((10, 1, ny, nx))
    W[0] = np.exp(rng.uniform(np.log(0.05), np.log(100), (1, ny, nx)))
    W[1:3] = rng.uniform(-3.0, 3.0, (2, 1, ny, nx))
    for y in range(ny):
        for x in range(nx):
            L = np.tril(rng.normal(0, 0.3, (3, 3)))
            L[np.diag_indices(3)] = rng.uniform(0.1, 1, 3)
            P = L @ L.T
            W[4:, 0, y, x] = [P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]]
    return W


def _problem(name):
    if name == "extreme2d":
        W = _extreme_2d()
        return W, (14, 24), (0.0, 0.0), (1.0, 1.0), ((0, 0), (0, 0)), 0.9, None, 3
    if name == "box3d":
        p = inputs.turb(n=12, nsteps=4)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, None, 4
    if name == "blast2d":
        p = inputs.blast(n=20, nsteps=5)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, None, 5
    if name == "disc2d":
        p = inputs.disc(n=24, nsteps=4)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, p.phi, 4
    if name == "sod1d":
        p = inputs.sod(40)
        return p.W, p.n, p.lo, p.hi, p.bc, p.cfl, None, 6
    raise KeyError(name)


def _steppers(oracle, name, slabs, ranks):
    W, n, lo, hi, bc, cfl, phi, _ = _problem(name)
    U = oracle.prim_to_cons(W)
    parts = decomp.split_state(U, n, slabs)
    periodic = bc[-1][0] == 0
    out = {}
    for r in ranks:
        sl = slabs[r]
        n_l, lo_l, hi_l, bc_l, dx = decomp.local_geometry(n, lo, hi, bc, sl)
        ph = None if phi is None else decomp.local_potential(phi, n, sl, periodic)
        out[r] = OracleStepper(oracle, n_l, lo_l, hi_l, bc_l, cfl, parts[r], dx, ph)
    return out


def _single(oracle, name):
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    U, ns, t, rc, _ = oracle.run(og, oracle.prim_to_cons(W), np.inf, max_steps=steps, phi=phi)
    assert rc == 0 and ns == steps
    return U.reshape((10,) + (1,) * (3 - len(n)) + tuple(reversed(n))), t


# ------------------------------------------------------------------ host logic
@pytest.mark.parametrize("n,world,periodic", [(10, 1, True), (10, 2, True), (11, 3, False), (9, 4, True),
                                              (8, 4, False)])
def test_partition(n, world, periodic):
    S = decomp.Slabs(n, world, periodic)
    owned = np.concatenate([np.arange(s.start, s.start + s.count) for s in S.slabs])
    assert np.array_equal(owned, np.arange(n))
    assert max(s.count for s in S.slabs) - min(s.count for s in S.slabs) <= 1
    for s in S.slabs:
        assert s.count >= (decomp.HALO if world > 1 else 1)
        if world == 1:
            assert s.lo_halo == s.hi_halo == 0
        else:
            assert (s.lower is None) == (not periodic and s.rank == 0)
            assert (s.upper is None) == (not periodic and s.rank == world - 1)
            if s.upper is not None:
                assert S[s.upper].lower == s.rank
    with pytest.raises(ValueError):
        decomp.Slabs(5, 3, True)


def test_local_geometry():
    rng = np.random.default_rng(4)
    for _ in range(200):
        nd = int(rng.integers(1, 4))
        n = tuple(int(v) for v in rng.integers(4, 60, nd))
        lo = tuple(float(v) for v in rng.uniform(-3, 3, nd))
        hi = tuple(l + float(w) for l, w in zip(lo, rng.uniform(0.1, 7, nd)))
        periodic = bool(rng.integers(0, 2))
        bc = ((0, 0),) * (nd - 1) + (((0, 0),) if periodic else ((2, 1),))
        S = decomp.Slabs(n[-1], min(3, n[-1] // 2), periodic)
        for sl in S.slabs:
            n_l, lo_l, hi_l, bc_l, dx = decomp.local_geometry(n, lo, hi, bc, sl)
            assert dx == tuple((hi[d] - lo[d]) / n[d] for d in range(nd))
            assert n_l[:-1] == n[:-1] and n_l[-1] == sl.local_layers
            assert bc_l[-1][0] == (1 if sl.lo_halo else bc[-1][0]) and bc_l[-1][1] == (1 if sl.hi_halo else bc[-1][1])


def test_split_and_join_round_trip():
    rng = np.random.default_rng(5)
    for n in [(17,), (6, 9), (5, 4, 11)]:
        U = rng.normal(size=(10,) + (1,) * (3 - len(n)) + tuple(reversed(n)))
        for world, per in [(1, False), (2, True), (3, False), (4, True)]:
            if n[-1] // world < 2:
                continue
            S = decomp.Slabs(n[-1], world, per)
            assert np.array_equal(decomp.join_owned(decomp.split_state(U, n, S), n, S), U)


# ------------------------------------------------------------ in one process
@pytest.mark.parametrize("name,world", [("box3d", 3), ("blast2d", 2), ("blast2d", 4), ("disc2d", 3),
                                        ("sod1d", 3)])
def test_inprocess_slabs_equal_single_grid(oracle, name, world):
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    S = decomp.Slabs(n[-1], world, bc[-1][0] == 0)
    st = _steppers(oracle, name, S, range(world))
    drv = decomp.SlabDriver(S, st)
    tot0, _, ok0 = drv.reduce()
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].U for r in range(world)], n, S)
    ref, t_ref = _single(oracle, name)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref)
    tot1, _, ok1 = drv.reduce()
    assert ok0 and ok1
    og = oracle.Grid(n, lo, hi, bc, cfl)
    np.testing.assert_allclose(tot1, oracle.diagnostics(og, ref)[0], rtol=1e-13, atol=1e-13 * np.abs(tot1).max())


# ------------------------------------------------------------- two gloo ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir, name):
    import torch.distributed as dist
    from oracle import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo")
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    S = decomp.Slabs(n[-1], world, bc[-1][0] == 0)
    st = _steppers(oracle, name, S, [rank])
    drv = decomp.SlabDriver(S, st, decomp.TorchDist("cpu"))
    ns, t = drv.run(steps)
    parts = [None] * world
    dist.all_gather_object(parts, st[rank].U)
    if rank == 0:
        np.save(os.path.join(outdir, "state.npy"), decomp.join_owned(parts, n, S))
        np.save(os.path.join(outdir, "time.npy"), np.array([ns, t]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["box3d", "disc2d"])
def test_two_gloo_ranks_equal_single_grid(oracle, name):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d, name), nprocs=2, join=True, start_method="spawn")
        got = np.load(os.path.join(d, "state.npy"))
        ns, t = np.load(os.path.join(d, "time.npy"))
    ref, t_ref = _single(oracle, name)
    assert ns == _problem(name)[-1] and t == t_ref
    np.testing.assert_array_equal(got, ref)


def test_kt_slabs_need_four_halo_layers(oracle):
    """The central scheme's two stages reach four cells: four halo layers reproduce the
    single grid, two do not."""
    from paper_1210_5246_gb300 import inputs
    p = inputs.turb(n=16)
    n, steps = p.n, 3
    og = oracle.Grid(n, p.lo, p.hi, p.bc, 0.4, scheme=1)
    ref, _, t_ref, rc, _ = oracle.run(og, oracle.prim_to_cons(p.W), np.inf, max_steps=steps)
    for halo, equal in ((decomp.halo_width(1), True), (decomp.HALO, False)):
        S = decomp.Slabs(n[-1], 3, True, halo=halo)
        parts = decomp.split_state(oracle.prim_to_cons(p.W), n, S)
        st = {}
        for r in range(3):
            n_l, lo_l, hi_l, bc_l, dx = decomp.local_geometry(n, p.lo, p.hi, p.bc, S[r])
            st[r] = OracleStepper(oracle, n_l, lo_l, hi_l, bc_l, 0.4, parts[r], dx, scheme=1)
        drv = decomp.SlabDriver(S, st)
        ns, t = drv.run(steps)
        got = decomp.join_owned([st[r].U for r in range(3)], n, S)
        assert np.array_equal(got, ref.reshape(got.shape)) == equal


@pytest.mark.parametrize("name,scheme", [("box3d", 0), ("blast2d", 2), ("box3d", 3)])
def test_ctu_slabs_equal_single_grid(oracle, name, scheme):
    """The corner-transport-upwind form (transverse terms reach one cell along each axis,
    max-form CFL reduced over the slabs) stays inside the two halo layers: three slabs
    reproduce the single grid bit for bit."""
    p = inputs.turb(n=16) if name == "box3d" else inputs.blast(n=32)
    n, steps = p.n, 3
    og = oracle.Grid(n, p.lo, p.hi, p.bc, 0.8, scheme=scheme, ctu=True)
    ref, _, t_ref, rc, _ = oracle.run(og, oracle.prim_to_cons(p.W), np.inf, max_steps=steps)
    assert rc == 0
    S = decomp.Slabs(n[-1], 3, True)
    parts = decomp.split_state(oracle.prim_to_cons(p.W), n, S)
    st = {}
    for r in range(3):
        n_l, lo_l, hi_l, bc_l, dx = decomp.local_geometry(n, p.lo, p.hi, p.bc, S[r])
        st[r] = OracleStepper(oracle, n_l, lo_l, hi_l, bc_l, 0.8, parts[r], dx, scheme=scheme, ctu=True)
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].U for r in range(3)], n, S)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref.reshape(got.shape))


# ------------------------------------------------ fallback across slab boundaries
def _single_tags(oracle, name):
    """Per step of the single-grid oracle run: the cells its fallback tagged (pass 0)."""
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    og = oracle.Grid(n, lo, hi, bc, cfl)
    U = oracle.prim_to_cons(W)
    out = []
    for _ in range(steps):
        dt = oracle.cfl_dt(og, U)
        out.append(~oracle.realizable_cells(og, oracle.step_pass(og, U, dt, None)))
        U = oracle.step(og, U, dt)
    return out


@pytest.mark.parametrize("world", [2, 3, 4])
def test_fallback_across_slab_boundaries_equals_single_grid(oracle, world):
    """The fallback tags cells on both sides of every slab boundary in every step; the slabs
    share its passes (tags exchanged into the halos before each pass) and reproduce the
    single-grid oracle run bit for bit."""
    name = "extreme2d"
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    S = decomp.Slabs(n[-1], world, True)
    tags = _single_tags(oracle, name)
    for sl in S.slabs:  # the single grid tags cells in the layers next to each boundary
        assert any(t[0, sl.start].any() or t[0, sl.start - 1].any() for t in tags), sl
    st = _steppers(oracle, name, S, range(world))
    drv = decomp.SlabDriver(S, st)
    ns, t = drv.run(steps)
    got = decomp.join_owned([st[r].U for r in range(world)], n, S)
    ref, t_ref = _single(oracle, name)
    assert ns == steps and t == t_ref
    np.testing.assert_array_equal(got, ref)


def test_fallback_without_tag_exchange_differs(oracle):
    """The same slabs with the tag exchange switched off (each slab sees only its own tags)
    no longer reproduce the single grid: the test above depends on the exchange."""
    name = "extreme2d"
    W, n, lo, hi, bc, cfl, phi, steps = _problem(name)
    S = decomp.Slabs(n[-1], 3, True)
    st = _steppers(oracle, name, S, range(3))
    drv = decomp.SlabDriver(S, st)
    real = drv.exchange
    drv.exchange = lambda tags=False: None if tags else real()
    drv.run(steps)
    got = decomp.join_owned([st[r].U for r in range(3)], n, S)
    ref, _ = _single(oracle, name)
    assert not np.array_equal(got, ref)


def _worker_fb(rank, world, port, outdir):
    import torch.distributed as dist
    from oracle import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo")
    W, n, lo, hi, bc, cfl, phi, steps = _problem("extreme2d")
    S = decomp.Slabs(n[-1], world, True)
    st = _steppers(oracle, "extreme2d", S, [rank])
    drv = decomp.SlabDriver(S, st, decomp.TorchDist("cpu"))
    ns, t = drv.run(steps)
    parts = [None] * world
    dist.all_gather_object(parts, st[rank].U)
    if rank == 0:
        np.save(os.path.join(outdir, "state.npy"), decomp.join_owned(parts, n, S))
        np.save(os.path.join(outdir, "time.npy"), np.array([ns, t]))
    dist.barrier()
    dist.destroy_process_group()


def test_fallback_across_two_gloo_ranks_equals_single_grid(oracle):
    """Two gloo ranks, each stepping one slab with the oracle, the fallback tags crossing
    both slab boundaries (periodic axis): bit for bit the single-grid run."""
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker_fb, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        got = np.load(os.path.join(d, "state.npy"))
        ns, t = np.load(os.path.join(d, "time.npy"))
    ref, t_ref = _single(oracle, "extreme2d")
    assert ns == 3 and t == t_ref
    np.testing.assert_array_equal(got, ref)

