"""Slab decomposition of one grid over several ranks (one GPU each).

The unsplit step (Sec. 3.3) reaches two cells to each side, so a grid cut into slabs
along its last active axis (z in 3D, y in 2D, x in 1D) advances exactly like the whole grid
if, before every step, each slab receives two halo layers from each neighbour (four for
the central scheme of Sec. 3.2, whose two Runge-Kutta stages each reach two cells) and all
slabs take the same dt: the minimum over slabs of the CFL dt of the layers each owns.  The
conserved totals are the sum over slabs of the owned layers' totals.  This is the only
place where the path has an exchange step; everything else (independent grids, the
batched tubes) shards with no collective (see ``replicas``).

A rank's local grid holds its owned layers plus the halo layers on every side that has a
neighbour (both sides when the axis is periodic; none at a non-periodic end of the global
grid, which keeps the global boundary condition).  A halo side's own boundary condition is
a placeholder: the cells it affects are halo cells, overwritten by the next exchange.

The a-posteriori fallback couples cells within a step: a cell whose second-order update is
not realizable is tagged, and the step is recomputed with first-order states on every face
of every tagged cell, up to four passes.  A face's states depend on the tags of the two
cells it joins, so before each pass every slab receives its neighbours' tags in its halo
layers (the guardcell exchange of Sec. 3.1, applied to the tags), and a pass runs on every
slab when any slab's owned cells were newly tagged by the pass before (a sum over the
slabs).  With that the slabs reproduce the single grid bit for bit in every step.

A stepper is any object with
    layers()                 -> number of local layers
    get(start, count)        -> array [10, count * cells per layer] (conserved)
    set(start, count, buf)
    reduce(start, count)     -> (totals[10], cfl dt, realizable) of those layers
    step(dt)                 -> cells the fallback tagged (a whole step, fallback inside)
and, for the shared fallback (``phased`` true):
    begin(dt)                the second-order pass (its failing cells are tagged by pass 0)
    retry(level)             fallback pass `level` with the tags of the passes before
    end()                    finishes the step
    count_tags(start, count, level), get_tags(start, count), set_tags(start, count, levels)
                             the tags of layers, one int per cell: the pass that tagged it, or -1.
A stepper without ``phased`` (the central scheme, which has no fallback) takes whole steps,
and a step in which it tags cells raises ``FallbackAcrossSlabs``.
``GridStepper`` wraps a libmsh grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

HALO = 2  # stencil radius of the MUSCL-Hancock step
FALLBACK_PASSES = 4  # a-posteriori fallback passes per step (the library's rule)


def halo_width(scheme=0):
    """Halo layers a slab needs per step: two for the MUSCL-Hancock step; four for the
    central scheme, whose two Runge-Kutta stages each reach two cells."""
    return 2 * HALO if scheme == 1 else HALO


class FallbackAcrossSlabs(RuntimeError):
    pass


class NotRealizable(RuntimeError):
    """A step left an owned cell of some slab non-realizable (rho <= 0 or P not positive
    definite) after every fallback pass."""


@dataclass
class Slab:
    rank: int
    start: int       # first owned global layer
    count: int       # owned layers
    lo_halo: int     # halo layers below (0 or HALO)
    hi_halo: int     # halo layers above (0 or HALO)
    lower: int | None  # rank owning the layers below the halo, if any
    upper: int | None

    @property
    def local_layers(self):
        return self.lo_halo + self.count + self.hi_halo

    @property
    def first_local_layer(self):
        """Global layer index of local layer 0 (may be negative or >= n on a periodic axis)."""
        return self.start - self.lo_halo


class Slabs:
    """Even partition of ``n`` layers into ``world`` slabs (the first n % world slabs one
    layer longer), each owning at least ``halo`` layers, the halo width of the scheme."""

    def __init__(self, n: int, world: int, periodic: bool, halo: int = HALO):
        if world < 1:
            raise ValueError("world must be >= 1")
        if world > 1 and n // world < halo:
            raise ValueError(f"{n} layers cannot give {world} slabs of at least {halo} layers")
        self.n, self.world, self.periodic, self.halo = n, world, periodic, halo
        base, extra = divmod(n, world)
        self.slabs = []
        s = 0
        for r in range(world):
            c = base + (1 if r < extra else 0)
            if world == 1:
                lower = upper = None
            else:
                lower = (r - 1) % world if (r > 0 or periodic) else None
                upper = (r + 1) % world if (r < world - 1 or periodic) else None
            self.slabs.append(Slab(r, s, c, halo if lower is not None else 0, halo if upper is not None else 0,
                                   lower, upper))
            s += c

    def __getitem__(self, r) -> Slab:
        return self.slabs[r]


def local_geometry(n, lo, hi, bc, slab: Slab, placeholder_bc=1):
    """(cells, lo, hi, boundary conditions, cell widths) of the local grid of ``slab`` for
    the global grid (n, lo, hi, bc).  (hi - lo) / m cannot reproduce the global width in
    floating point for every layer count m, so the widths are returned separately and the
    local grid takes them explicitly (``msh_set_cell_width``); its bounds along the cut axis
    are nominal."""
    nd = len(n)
    a = nd - 1
    dx = tuple((hi[d] - lo[d]) / n[d] for d in range(nd))
    m = slab.local_layers
    n_l = list(n)
    n_l[a] = m
    lo_l = list(lo)
    hi_l = list(hi)
    lo_l[a] = lo[a] + slab.first_local_layer * dx[a]
    hi_l[a] = lo_l[a] + m * dx[a]
    bc_l = [tuple(b) for b in bc]
    bc_l[a] = (placeholder_bc if slab.lo_halo else bc[a][0], placeholder_bc if slab.hi_halo else bc[a][1])
    return tuple(n_l), tuple(lo_l), tuple(hi_l), tuple(bc_l), dx


def _cut_axis(nd):
    """Array axis of the cut layers in a state [10][nz][ny][nx] (the potential has no field
    axis: subtract one)."""
    return 4 - nd


def local_potential(phi, n, slab: Slab, periodic: bool):
    """Slice of a potential with one ghost layer per active axis ([nz+2gz][ny+2gy][nx+2gx])
    for the local grid of ``slab``: global layers first_local_layer - 1 .. + local_layers."""
    nd = len(n)
    a = nd - 1
    phi = np.asarray(phi, dtype=np.float64)
    phi = phi.reshape((1,) * (3 - phi.ndim) + phi.shape)
    idx = []
    for j in range(slab.local_layers + 2):
        gl = slab.first_local_layer - 1 + j
        if periodic and not (-1 <= gl <= n[a]):
            gl %= n[a]
        idx.append(gl + 1)
    return np.ascontiguousarray(np.take(phi, idx, axis=_cut_axis(nd) - 1))


def split_state(U, n, slabs: Slabs):
    """Local initial states (owned layers and halos) of every slab from a global state."""
    nd = len(n)
    U = np.asarray(U).reshape((10,) + (1,) * (3 - nd) + tuple(reversed(n)))
    out = []
    for sl in slabs.slabs:
        idx = [(sl.first_local_layer + j) % slabs.n for j in range(sl.local_layers)]
        out.append(np.ascontiguousarray(np.take(U, idx, axis=_cut_axis(nd))))
    return out


def join_owned(parts, n, slabs: Slabs):
    """Global state [10][nz][ny][nx] from every slab's local state (owned layers only)."""
    nd = len(n)
    ax = _cut_axis(nd)
    owned = []
    for sl, P in zip(slabs.slabs, parts):
        shape = [10] + [1] * (3 - nd) + list(reversed(n))
        shape[ax] = sl.local_layers
        P = np.asarray(P).reshape(shape)
        owned.append(np.take(P, range(sl.lo_halo, sl.lo_halo + sl.count), axis=ax))
    return np.concatenate(owned, axis=ax)


class InProcess:
    """Communicator for slabs that all live in this process (no collectives)."""

    def min(self, x):
        return x

    def sum(self, x):
        return x


class TorchDist:
    """Communicator over torch.distributed (gloo on the CPU, NCCL on GPUs): halo layers
    move by isend/irecv between neighbours, dt by all_reduce(MIN), totals by all_reduce(SUM)."""

    def __init__(self, device="cpu"):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.device = torch, dist, device

    def min(self, x):
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
        return float(t.item())

    def sum(self, x):
        t = self.torch.tensor(np.asarray(x, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.cpu().numpy()

    def exchange(self, sends, recvs):
        """sends: [(peer, tag, array)], recvs: [(peer, tag, shape, dtype)] -> {tag: array}."""
        torch, dist = self.torch, self.dist
        reqs, bufs = [], {}
        for peer, tag, shape, dtype in recvs:
            b = torch.empty(shape, dtype=torch.from_numpy(np.empty(0, dtype=dtype)).dtype, device=self.device)
            bufs[tag] = b
            reqs.append(dist.irecv(b, src=peer, tag=tag))
        keep = []
        for peer, tag, arr in sends:
            t = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device)
            keep.append(t)
            reqs.append(dist.isend(t, dst=peer, tag=tag))
        for q in reqs:
            q.wait()
        return {tag: b.cpu().numpy() for tag, b in bufs.items()}


class SlabDriver:
    """Advances the slabs this process holds (``steppers``: rank -> stepper) in lockstep
    with the slabs of the other processes (``comm``)."""

    def __init__(self, slabs: Slabs, steppers: dict, comm=None):
        self.slabs, self.steppers = slabs, steppers
        self.comm = comm if comm is not None else InProcess()
        self.t = 0.0
        self.steps = 0

    # tags: (receiver rank, side) so that every message is unique within one exchange
    @staticmethod
    def _tag(dst, side):
        return 2 * dst + side

    def exchange(self, tags=False):
        """Copy the halo's width of owned layers to each neighbour's halo: the conserved state,
        or with ``tags`` the fallback tags of the current step.  Messages to other processes
        go out in a fixed order (to the lower neighbour, then to the upper one) and are
        received in the matching order (from the upper neighbour, then the lower one)."""
        S = self.slabs
        h = S.halo
        sends, recvs, local = [], [], []
        for r, st in self.steppers.items():
            sl = S[r]
            get = st.get_tags if tags else st.get
            if sl.lower is not None:  # my lowest owned layers -> the lower neighbour's upper halo
                arr = get(sl.lo_halo, h)
                if sl.lower in self.steppers:
                    local.append((sl.lower, 1, arr))
                else:
                    sends.append((sl.lower, self._tag(sl.lower, 1), arr))
            if sl.upper is not None:  # my highest owned layers -> the upper neighbour's lower halo
                arr = get(sl.lo_halo + sl.count - h, h)
                if sl.upper in self.steppers:
                    local.append((sl.upper, 0, arr))
                else:
                    sends.append((sl.upper, self._tag(sl.upper, 0), arr))
            if sl.upper is not None and sl.upper not in self.steppers:
                recvs.append((sl.upper, r, 1))
            if sl.lower is not None and sl.lower not in self.steppers:
                recvs.append((sl.lower, r, 0))
        got = {}
        if recvs:
            shape, dtype = sends[0][2].shape, sends[0][2].dtype  # every layer block has one size
            got = self.comm.exchange(sends, [(peer, self._tag(r, side), shape, dtype) for peer, r, side in recvs])
        def put(r, start, arr):
            st = self.steppers[r]
            (st.set_tags if tags else st.set)(start, h, arr)
        for dst, side, arr in local:
            sl = S[dst]
            put(dst, 0 if side == 0 else sl.lo_halo + sl.count, arr)
        for peer, r, side in recvs:
            sl = S[r]
            put(r, 0 if side == 0 else sl.lo_halo + sl.count, got[self._tag(r, side)])

    def reduce(self):
        """(totals, cfl dt, realizable) over the whole grid."""
        tot = np.zeros(10)
        dt = math.inf
        ok = True
        for r, st in self.steppers.items():
            sl = self.slabs[r]
            t_r, dt_r, ok_r = st.reduce(sl.lo_halo, sl.count)
            tot += t_r
            dt = min(dt, dt_r)
            ok = ok and ok_r
        return self.comm.sum(tot), self.comm.min(dt), self.comm.min(1.0 if ok else 0.0) > 0.0

    def step(self, t_end=math.inf, dt_max=math.inf):
        """One step of the whole grid; returns dt (0 if t_end was reached)."""
        if self.t >= t_end:
            return 0.0
        self.exchange()
        _, dt, _ = self.reduce()
        dt = min(dt, dt_max)
        if self.t + dt >= t_end:
            dt = t_end - self.t
        if all(getattr(st, "phased", False) for st in self.steppers.values()):
            self._phased_step(dt)
        else:
            tagged = 0
            for st in self.steppers.values():
                tagged += st.step(dt)
            tagged = int(self.comm.sum(np.array([float(tagged)]))[0])
            if tagged:
                raise FallbackAcrossSlabs(f"step {self.steps}: the a-posteriori fallback tagged {tagged} cells")
        # A stepper checks every local cell, its halo cells too, whose update is discarded;
        # where one reported a non-realizable cell, the owned layers decide (all ranks).
        flagged = sum(1.0 for st in self.steppers.values() if getattr(st, "local_bad", False))
        for st in self.steppers.values():
            st.local_bad = False
        if self.comm.sum(np.array([flagged]))[0] > 0:
            _, _, ok = self.reduce()
            if not ok:
                raise NotRealizable(f"step {self.steps}: an owned cell is not realizable after the fallback")
        self.t += dt
        self.steps += 1
        return dt

    def owned_tags(self, level):
        """Cells of every slab's owned layers tagged by pass `level` of this step (all ranks)."""
        n = 0
        for r, st in self.steppers.items():
            sl = self.slabs[r]
            n += st.count_tags(sl.lo_halo, sl.count, level)
        return int(self.comm.sum(np.array([float(n)]))[0])

    def _phased_step(self, dt):
        """One step with the a-posteriori fallback shared by the slabs: pass p runs on every
        slab, after the tags of the passes before it have reached the neighbours' halos,
        whenever some slab's owned cells were newly tagged by pass p - 1."""
        for st in self.steppers.values():
            st.begin(dt)
        for level in range(1, FALLBACK_PASSES + 1):
            if self.owned_tags(level - 1) == 0:
                break
            self.exchange(tags=True)
            for st in self.steppers.values():
                st.retry(level)
        for st in self.steppers.values():
            st.end()

    def run(self, max_steps, t_end=math.inf):
        for _ in range(max_steps):
            if self.step(t_end) == 0.0:
                break
        return self.steps, self.t


class GridStepper:
    """A libmsh grid as a slab stepper (host buffers for the halo copies).  The
    characteristic schemes share the fallback (``phased``); the central scheme has none."""

    def __init__(self, grid, scheme=0):
        self.g = grid
        self.phased = scheme != 1
        self.local_bad = False

    def _checked(self, call, *args):
        """A step call whose MSH_E_REALIZABILITY (some local cell, halo cells included) is
        left to the driver's check of the owned layers; the step itself has been taken."""
        from . import msh
        try:
            return call(*args)
        except msh.MshError as e:
            if e.status != msh.MSH_E_REALIZABILITY:
                raise
            self.local_bad = True
            return 0

    def layers(self):
        return self.g.layer_shape()[0]

    def get(self, start, count):
        return self.g.get_slab(start, count)

    def set(self, start, count, buf):
        self.g.set_slab(start, count, buf)

    def reduce(self, start, count):
        return self.g.reduce_layers(start, count)

    def step(self, dt):
        return self._checked(self.g.step_dt, dt)

    def begin(self, dt):
        self.g.step_begin(dt)

    def retry(self, level):
        self.g.step_retry(level)

    def end(self):
        return self._checked(self.g.step_end)

    def count_tags(self, start, count, level):
        return self.g.count_tags(start, count, level)

    def get_tags(self, start, count):
        return self.g.get_tags(start, count)

    def set_tags(self, start, count, levels):
        self.g.set_tags(start, count, levels)


def make_grid_steppers(msh, n, lo, hi, bc, cfl, precision, U, slabs: Slabs, ranks, phi=None, stream=None,
                       scheme=0, ctu=False):
    """Local libmsh grids (state set, potential sliced, scheme and its corner-transport-upwind
    form selected) for the given ranks.  The transverse terms of a cell reach one cell along
    each axis, inside the two halo layers of the characteristic step."""
    parts = split_state(U, n, slabs)
    a = len(n) - 1
    periodic = bc[a][0] == 0
    out = {}
    for r in ranks:
        sl = slabs[r]
        n_l, lo_l, hi_l, bc_l, dx = local_geometry(n, lo, hi, bc, sl)
        g = msh.Grid(n_l, lo_l, hi_l, bc_l, cfl, precision, stream=stream)
        g.set_cell_width(dx)
        if scheme:
            g.set_scheme(scheme)
        if ctu:
            g.set_ctu(True)
        if phi is not None:
            g.set_potential(local_potential(phi, n, sl, periodic))
        g.set_state(parts[r].astype(g.dtype), msh.CONSERVED)
        out[r] = GridStepper(g, scheme)
    return out
