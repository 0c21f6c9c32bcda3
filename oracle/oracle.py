"""ctypes wrapper around ``msh_oracle.c`` (plain FP64 loops, OpenMP over pencils).

Test infrastructure only (see the package docstring).  Arrays are numpy float64 in
structure-of-arrays layout ``[10][nz][ny][nx]``; conserved component order is
(rho, m_x, m_y, m_z, E_xx, E_xy, E_xz, E_yy, E_yz, E_zz) and primitive order is
(rho, u_x, u_y, u_z, P_xx, P_xy, P_xz, P_yy, P_yz, P_zz), with E_ij = P_ij + rho u_i u_j
(Sec. 2, below eq. dispers).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "msh_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

PERIODIC, OUTFLOW, REFLECT = 0, 1, 2
SCHEME_MH, SCHEME_KT, SCHEME_MH_ROE, SCHEME_MH_HLLC = 0, 1, 2, 3
NV = 10

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", "-ffp-contract=off", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class OgGrid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("pad0", C.c_int32), ("n", C.c_int64 * 3),
                ("dx", C.c_double * 3), ("bc", C.c_int32 * 6), ("cfl", C.c_double),
                ("scheme", C.c_int32), ("ctu", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(OgGrid)
            lib.og_step.argtypes = [gp, dp, dp, C.c_double, dp]
            lib.og_step.restype = C.c_int
            lib.og_cfl_dt.argtypes = [gp, dp]
            lib.og_cfl_dt.restype = C.c_double
            lib.og_step_second_order_only.argtypes = [gp, dp, dp, C.c_double, dp]
            lib.og_step_second_order_only.restype = C.c_int
            lib.og_run.argtypes = [gp, dp, dp, C.c_double, C.c_double, C.c_int64, C.c_double,
                                   dp, C.POINTER(C.c_int64), dp]
            lib.og_run.restype = C.c_int
            lib.og_run_schedule.argtypes = [gp, dp, dp, dp, C.c_int64]
            lib.og_run_schedule.restype = C.c_int
            lib.og_diagnostics.argtypes = [gp, dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
            lib.og_ghost_fill.argtypes = [gp, dp, dp]
            lib.og_flux.argtypes = [dp, C.c_int, dp]
            lib.og_hll.argtypes = [dp, dp, C.c_int, dp]
            lib.og_kt_flux.argtypes = [dp, dp, C.c_int, dp]
            lib.og_roe.argtypes = [dp, dp, C.c_int, dp]
            lib.og_hllc.argtypes = [dp, dp, C.c_int, dp]
            lib.og_hllc_star.argtypes = [dp, dp, C.c_int, dp, dp, dp]
            lib.og_hllc_star.restype = C.c_int
            lib.og_kt_reconstruct.argtypes = [dp, dp, dp, C.c_int, dp, dp]
            lib.og_reconstruct.argtypes = [dp, dp, dp, C.c_int, C.c_double, dp, dp]
            lib.og_reconstruct_upwind.argtypes = [dp, dp, dp, C.c_int, C.c_double, dp, dp]
            for f in ("og_jacobian_x", "og_right_x", "og_left_x"):
                getattr(lib, f).argtypes = [dp, dp]
            lib.og_eigenvalues_x.argtypes = [dp, dp]
            lib.og_prim_to_cons_arr.argtypes = [dp, dp, C.c_int64]
            lib.og_cons_to_prim_arr.argtypes = [dp, dp, C.c_int64]
            lib.og_step_pass.argtypes = [gp, dp, dp, C.c_double, C.c_void_p, dp]
            lib.og_step_pass.restype = C.c_int
            lib.og_realizable_cells.argtypes = [gp, dp, C.c_void_p]
            lib.og_num_threads.restype = C.c_int
            lib.og_set_num_threads.argtypes = [C.c_int]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Uniform grid description: ``n`` cells per dim on [lo, hi], boundaries
    ``bc[d] = (lower, upper)`` (PERIODIC / OUTFLOW / REFLECT), CFL number ``cfl``."""

    def __init__(self, n, lo, hi, bc, cfl, scheme=0, ctu=False):
        """scheme: SCHEME_MH (MUSCL-Hancock + HLL, Sec. 3.3), SCHEME_KT (Kurganov-Tadmor
        + RK2, Sec. 3.2), SCHEME_MH_ROE (MUSCL-Hancock with upwind tracing and the Roe-type
        flux) or SCHEME_MH_HLLC (MUSCL-Hancock with the HLLC flux).  ctu: the characteristic
        schemes add the transverse terms of ``og_transverse`` to the face states and take
        the max-form CFL rule."""
        n = list(n)
        self.ndim = len(n)
        self.n = tuple(n) + (1,) * (3 - len(n))
        lo = list(lo) + [0.0] * (3 - len(lo))
        hi = list(hi) + [1.0] * (3 - len(hi))
        self.dx = tuple((hi[d] - lo[d]) / self.n[d] for d in range(3))
        self.lo, self.hi = tuple(lo), tuple(hi)
        self.bc = tuple(tuple(b) for b in bc) + ((PERIODIC, PERIODIC),) * (3 - len(bc))
        self.cfl = float(cfl)
        g = OgGrid()
        g.ndim = self.ndim
        for d in range(3):
            g.n[d] = self.n[d]
            g.dx[d] = self.dx[d]
            g.bc[2 * d] = self.bc[d][0]
            g.bc[2 * d + 1] = self.bc[d][1]
        g.cfl = self.cfl
        g.scheme = int(scheme)
        g.ctu = int(bool(ctu))
        self.scheme = int(scheme)
        self.ctu = bool(ctu)
        self._g = g

    @property
    def shape(self):
        return (NV, self.n[2], self.n[1], self.n[0])

    @property
    def ncells(self):
        return self.n[0] * self.n[1] * self.n[2]

    def phi_shape(self):
        g = [1 if d < self.ndim else 0 for d in range(3)]
        return (self.n[2] + 2 * g[2], self.n[1] + 2 * g[1], self.n[0] + 2 * g[0])


def prim_to_cons(W):
    W = _f64(W)
    U = np.empty_like(W)
    _load().og_prim_to_cons_arr(_p(W), _p(U), W.size // NV)
    return U


def cons_to_prim(U):
    U = _f64(U)
    W = np.empty_like(U)
    _load().og_cons_to_prim_arr(_p(U), _p(W), U.size // NV)
    return W


def cfl_dt(grid: Grid, U) -> float:
    U = _f64(U)
    return _load().og_cfl_dt(C.byref(grid._g), _p(U))


def step(grid: Grid, U, dt, phi=None):
    """One step of size ``dt`` (a1-a8); returns the new conserved state."""
    U = _f64(U).reshape(grid.shape)
    out = np.empty_like(U)
    ph = None if phi is None else _f64(phi).reshape(grid.phi_shape())
    rc = _load().og_step(C.byref(grid._g), _p(U), None if ph is None else _p(ph), float(dt),
                         _p(out))
    if rc:
        raise MemoryError("oracle step failed to allocate")
    return out


def step_second_order_only(grid: Grid, U, dt, phi=None):
    """The step without the a-posteriori first-order fallback."""
    U = _f64(U).reshape(grid.shape)
    out = np.empty_like(U)
    ph = None if phi is None else _f64(phi).reshape(grid.phi_shape())
    if _load().og_step_second_order_only(C.byref(grid._g), _p(U), None if ph is None else _p(ph),
                                         float(dt), _p(out)):
        raise MemoryError("oracle step failed to allocate")
    return out


def run(grid: Grid, U, t_end, max_steps=1 << 62, dt_max=float("inf"), phi=None, t0=0.0,
        record=False):
    """Advance to ``t_end`` (last step clipped) or ``max_steps``.
    Returns (U, steps, t, status, dt_history or None)."""
    U = _f64(U).reshape(grid.shape).copy()
    ph = None if phi is None else _f64(phi).reshape(grid.phi_shape())
    cap = int(min(max_steps, 10_000_000)) if record else 0
    hist = np.zeros(max(cap, 1))
    ns = C.c_int64(0)
    tt = C.c_double(0.0)
    rc = _load().og_run(C.byref(grid._g), _p(U), None if ph is None else _p(ph), float(t0),
                        float(t_end), int(max_steps), float(dt_max),
                        _p(hist) if record else None, C.byref(ns), C.byref(tt))
    return U, ns.value, tt.value, rc, (hist[: ns.value].copy() if record else None)


def step_pass(grid: Grid, U, dt, tagged=None, phi=None):
    """One pass of the characteristic step (``og_step_pass``): second order without
    ``tagged``; with ``tagged`` (bool per cell) first-order faces at every tagged cell."""
    U = _f64(U).reshape(grid.shape)
    out = np.empty_like(U)
    ph = None if phi is None else _f64(phi).reshape(grid.phi_shape())
    tg = None
    if tagged is not None:
        tg = np.ascontiguousarray(np.asarray(tagged, dtype=np.uint8).reshape(-1))
        if tg.size != grid.ncells:
            raise ValueError("tagged must have one entry per cell")
    rc = _load().og_step_pass(C.byref(grid._g), _p(U), None if ph is None else _p(ph), float(dt),
                              None if tg is None else tg.ctypes.data, _p(out))
    if rc:
        raise MemoryError("oracle step failed to allocate")
    return out


def realizable_cells(grid: Grid, U):
    """Per cell: realizable (rho > 0, P positive definite)."""
    U = _f64(U).reshape(grid.shape)
    out = np.empty(grid.ncells, dtype=np.uint8)
    _load().og_realizable_cells(C.byref(grid._g), _p(U), out.ctypes.data)
    return out.astype(bool).reshape(grid.shape[1:])


def run_schedule(grid: Grid, U, dts, phi=None):
    """Replay a fixed dt schedule."""
    U = _f64(U).reshape(grid.shape).copy()
    d = _f64(dts)
    ph = None if phi is None else _f64(phi).reshape(grid.phi_shape())
    rc = _load().og_run_schedule(C.byref(grid._g), _p(U), None if ph is None else _p(ph), _p(d),
                                 len(d))
    if rc:
        raise MemoryError("oracle step failed to allocate")
    return U


def diagnostics(grid: Grid, U):
    """(totals[10], realizable, first_bad_cell)."""
    U = _f64(U).reshape(grid.shape)
    tot = np.zeros(NV)
    ok = C.c_int32(0)
    bad = C.c_int64(0)
    _load().og_diagnostics(C.byref(grid._g), _p(U), _p(tot), C.byref(ok), C.byref(bad))
    return tot, bool(ok.value), bad.value


def ghost_fill(grid: Grid, U):
    g = [2 if d < grid.ndim else 0 for d in range(3)]
    shp = (NV, grid.n[2] + 2 * g[2], grid.n[1] + 2 * g[1], grid.n[0] + 2 * g[0])
    out = np.empty(shp)
    _load().og_ghost_fill(C.byref(grid._g), _p(_f64(U).reshape(grid.shape)), _p(out))
    return out


# --- single-state building blocks (used by the pins) -----------------------------
def flux(W, d):
    W = _f64(W)
    F = np.empty(NV)
    _load().og_flux(_p(W), int(d), _p(F))
    return F


def hll(WL, WR, d):
    F = np.empty(NV)
    _load().og_hll(_p(_f64(WL)), _p(_f64(WR)), int(d), _p(F))
    return F


def roe_flux(WL, WR, d):
    """Roe-type flux between the face states WL and WR (primitive, global order)."""
    F = np.zeros(NV)
    _load().og_roe(_p(_f64(WL)), _p(_f64(WR)), int(d), _p(F))
    return F


def hllc_flux(WL, WR, d):
    """HLLC flux between the face states WL and WR (primitive, global order)."""
    F = np.zeros(NV)
    _load().og_hllc(_p(_f64(WL)), _p(_f64(WR)), int(d), _p(F))
    return F


def hllc_star(WL, WR, d):
    """(ok, U*_L, U*_R, (S_L, S_M, S_R)) of the HLLC flux; ok False where HLLC reverts to HLL."""
    UsL, UsR, S = np.zeros(NV), np.zeros(NV), np.zeros(3)
    ok = _load().og_hllc_star(_p(_f64(WL)), _p(_f64(WR)), int(d), _p(UsL), _p(UsR), _p(S))
    return bool(ok), UsL, UsR, tuple(S)


def kt_flux(WL, WR, d):
    """Kurganov-Tadmor flux between the face values WL (left side) and WR (right side)."""
    F = np.zeros(NV)
    _load().og_kt_flux(_p(_f64(WL)), _p(_f64(WR)), int(d), _p(F))
    return F


def kt_reconstruct(Wm, W0, Wp, d):
    """(lo, hi) face values of a cell in the KT scheme (componentwise MC on primitives)."""
    lo, hi = np.zeros(NV), np.zeros(NV)
    _load().og_kt_reconstruct(_p(_f64(Wm)), _p(_f64(W0)), _p(_f64(Wp)), int(d), _p(lo), _p(hi))
    return lo, hi


def reconstruct(Wm, W0, Wp, d, dtdx):
    lo, hi = np.empty(NV), np.empty(NV)
    _load().og_reconstruct(_p(_f64(Wm)), _p(_f64(W0)), _p(_f64(Wp)), int(d), float(dtdx),
                           _p(lo), _p(hi))
    return lo, hi


def reconstruct_upwind(Wm, W0, Wp, d, dtdx):
    """(lo, hi) face states with the upwind characteristic tracing of the Roe-type scheme."""
    lo, hi = np.empty(NV), np.empty(NV)
    _load().og_reconstruct_upwind(_p(_f64(Wm)), _p(_f64(W0)), _p(_f64(Wp)), int(d), float(dtdx),
                                  _p(lo), _p(hi))
    return lo, hi


def eigensystem_x(W):
    """(A, lam, R, L) of the x-normal quasi-linear primitive system."""
    W = _f64(W)
    A, R, L = (np.empty((NV, NV)) for _ in range(3))
    lam = np.empty(NV)
    lib = _load()
    lib.og_jacobian_x(_p(W), _p(A))
    lib.og_eigenvalues_x(_p(W), _p(lam))
    lib.og_right_x(_p(W), _p(R))
    lib.og_left_x(_p(W), _p(L))
    return A, lam, R, L


def num_threads() -> int:
    return _load().og_num_threads()


def set_num_threads(n: int) -> None:
    _load().og_set_num_threads(int(n))
