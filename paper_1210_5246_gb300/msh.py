"""Thin ctypes binding of libmsh (``include/msh.h``).

Argument marshalling only: every step of the solver runs in the CUDA library.  The
module-level functions keep the C names (``msh_init_grid``, ``msh_step``, ...); the
``Grid`` and ``Batch`` classes are conveniences over them.  Host arrays are numpy,
device arrays are torch CUDA tensors (torch provides device memory and streams only).

There is no fallback: if ``libmsh.so`` is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MSH_OK, MSH_E_INVALID_ARG, MSH_E_CUDA, MSH_E_NOMEM, MSH_E_REALIZABILITY, MSH_E_TIMEOUT, MSH_E_STATE = range(7)
PERIODIC, OUTFLOW, REFLECT = 0, 1, 2
FP32, FP64 = 0, 1
MUSCL_HANCOCK, KT, MUSCL_HANCOCK_ROE, MUSCL_HANCOCK_HLLC = 0, 1, 2, 3
HOST, DEVICE = 0, 1
CONSERVED, PRIMITIVE = 0, 1

_STATUS_NAMES = {1: "MSH_E_INVALID_ARG", 2: "MSH_E_CUDA", 3: "MSH_E_NOMEM", 4: "MSH_E_REALIZABILITY",
                 5: "MSH_E_TIMEOUT", 6: "MSH_E_STATE"}


class MshError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

# (name, argtypes) of every exported entry point; restype is int32 unless noted
_vp, _i32, _i64, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_P = C.POINTER
SIGNATURES = {
    "msh_last_error": [],
    "msh_version": [],
    "msh_init_grid": [_P(_vp), _i32, _P(_i64), _P(_dbl), _P(_dbl), _P(_i32), _i32, _dbl, _vp],
    "msh_destroy": [_vp],
    "msh_set_state": [_vp, _vp, _i32, _i32],
    "msh_get_state": [_vp, _vp, _i32, _i32],
    "msh_set_time": [_vp, _dbl, _i64],
    "msh_get_time": [_vp, _P(_dbl), _P(_i64)],
    "msh_set_potential": [_vp, _vp, _i32],
    "msh_step": [_vp, _dbl, _P(_dbl)],
    "msh_run": [_vp, _dbl, _i64, _P(_i64), _P(_dbl)],
    "msh_run_ensemble": [_vp, _i64, _P(_vp), _P(_vp), _i32, _i64, _P(_i32)],
    "msh_diagnostics": [_vp, _P(_dbl), _P(_i32), _P(_i64)],
    "msh_set_recording": [_vp, _i64],
    "msh_get_dt_history": [_vp, _P(_dbl), _i64, _P(_i64)],
    "msh_set_tiling": [_vp, _i32, _i32],
    "msh_get_tiling": [_vp, _P(_i32), _P(_i32)],
    "msh_autotune": [_vp, _P(_i32), _P(_i32)],
    "msh_set_profiling": [_vp, _i32],
    "msh_set_test_fault": [_vp, _i32],
    "msh_get_profile": [_vp, _P(_dbl), _P(_dbl), _P(_i64)],
    "msh_adjoint_run": [_vp, _vp, _i64, _P(_dbl), _i32, _vp, _vp, _i32, _i32],
    "msh_set_tape": [_vp, _i32, _i64],
    "msh_set_scheme": [_vp, _i32],
    "msh_set_ctu": [_vp, _i32],
    "msh_get_ctu": [_vp, _P(_i32)],
    "msh_set_self_gravity": [_vp, _dbl],
    "msh_set_cell_width": [_vp, _P(_dbl)],
    "msh_get_slab": [_vp, _i64, _i64, _vp, _i32],
    "msh_set_slab": [_vp, _i64, _i64, _vp, _i32],
    "msh_reduce_layers": [_vp, _i64, _i64, _P(_dbl), _P(_dbl), _P(_i32)],
    "msh_step_dt": [_vp, _dbl, _P(_i32)],
    "msh_adjoint_tape": [_vp, _vp, _vp, _i32, _i32],
    "msh_batch_init": [_P(_vp), _i32, _P(_i32), _P(_dbl), _P(_dbl), _P(_dbl), _i32, _dbl, _vp],
    "msh_batch_reset": [_vp],
    "msh_batch_run": [_vp, _i32, _i64],
    "msh_batch_run_per_tube": [_vp, _P(_i32), _i32, _i64],
    "msh_batch_get_state": [_vp, _vp, _i32, _i32],
    "msh_batch_info": [_vp, _P(_i64), _P(_dbl), _P(_i64)],
    "msh_batch_fallback_steps": [_vp, _P(_i64)],
    "msh_batch_destroy": [_vp],
    "msh_step_begin": [_vp, _dbl],
    "msh_step_retry": [_vp, _i32],
    "msh_step_end": [_vp, _P(_i32)],
    "msh_get_tags": [_vp, _i64, _i64, _vp, _i32],
    "msh_set_tags": [_vp, _i64, _i64, _vp, _i32],
    "msh_count_tags": [_vp, _i64, _i64, _i32, _P(_i64)],
    "msh_step_noalloc": [_i32, _P(_i64), _P(_dbl), _P(_dbl), _P(_i32), _i32, _dbl, _dbl, _vp, _vp, _vp, _P(_dbl)],
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmsh.so.  Raises if it is missing (unless ``build_if_missing``)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise ImportError(f"libmsh.so not built ({path}); run __graft_entry__.build() "
                                      "or python -m paper_1210_5246_gb300.build")
                _build.build()
            lib = C.CDLL(path)
            for name, args in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = C.c_char_p if name == "msh_last_error" else C.c_int32
            _lib = lib
    return _lib


def _check(status):
    if status != MSH_OK:
        raise MshError(status, load().msh_last_error().decode())


def _ptr_dbl(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------- C-named calls
def msh_last_error() -> str:
    return load().msh_last_error().decode()


def msh_version() -> int:
    return load().msh_version()


def msh_init_grid(ndim, n, lo, hi, bc, precision, cfl, stream=None):
    h = C.c_void_p()
    n3 = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    lo3 = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    hi3 = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    flat = [b for pair in bc for b in pair] + [0] * (6 - 2 * len(bc))
    bc6 = (C.c_int32 * 6)(*flat)
    _check(load().msh_init_grid(C.byref(h), int(ndim), n3, lo3, hi3, bc6, int(precision), float(cfl),
                                C.c_void_p(stream) if stream else None))
    return h


def msh_destroy(h):
    _check(load().msh_destroy(h))


def msh_step(h, dt_max=float("inf")):
    dt = C.c_double(0.0)
    _check(load().msh_step(h, float(dt_max), C.byref(dt)))
    return dt.value


def msh_run(h, t_end=float("inf"), max_steps=(1 << 62)):
    s = C.c_int64(0)
    t = C.c_double(0.0)
    _check(load().msh_run(h, float(t_end), int(max_steps), C.byref(s), C.byref(t)))
    return s.value, t.value


def msh_step_noalloc(n, lo, hi, bc, precision, cfl, U_in, U_out, dt_max=float("inf"), stream=None):
    """One grid step that allocates no memory (see include/msh.h).  U_in and U_out are
    device tensors (torch, contiguous [10][nz][ny][nx]) of the given precision.
    Returns the step size."""
    ndim = len(n)
    n3 = (C.c_int64 * 3)(*(list(n) + [1] * (3 - ndim)))
    lo3 = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - ndim)))
    hi3 = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - ndim)))
    bc6 = (C.c_int32 * 6)(*([b for pair in bc for b in pair] + [0] * (6 - 2 * ndim)))
    dt = C.c_double(0.0)
    _check(load().msh_step_noalloc(ndim, n3, lo3, hi3, bc6, int(precision), float(cfl), float(dt_max),
                                   C.c_void_p(U_in.data_ptr()), C.c_void_p(U_out.data_ptr()),
                                   C.c_void_p(stream) if stream else None, C.byref(dt)))
    return dt.value


# ------------------------------------------------------------------ classes
def _torch():
    import torch
    return torch


class Grid:
    """A uniform 1D/2D/3D grid on the GPU (see ``msh_init_grid``)."""

    def __init__(self, n, lo, hi, bc, cfl, precision=FP64, stream=None):
        self.ndim = len(n)
        self.n = tuple(n) + (1,) * (3 - len(n))
        self.precision = precision
        self.dtype = np.float32 if precision == FP32 else np.float64
        self.h = msh_init_grid(self.ndim, n, lo, hi, bc, precision, cfl, stream)
        self.shape = (10, self.n[2], self.n[1], self.n[0])

    @classmethod
    def from_problem(cls, p, precision=FP64, stream=None):
        g = cls(p.n, p.lo, p.hi, p.bc, p.cfl, precision, stream)
        if p.phi is not None:
            g.set_potential(p.phi)
        return g

    def close(self):
        if self.h:
            msh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ----------------------------------------------------------------
    def _buf(self, a):
        """(pointer, where, keepalive) for a numpy host array or a torch CUDA tensor."""
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=self.dtype)
            if a.size != int(np.prod(self.shape)):
                raise ValueError(f"state must have {np.prod(self.shape)} elements")
            return a.ctypes.data_as(C.c_void_p), HOST, a
        t = a
        if not t.is_contiguous() or t.numel() != int(np.prod(self.shape)):
            raise ValueError("device state must be contiguous with 10*N elements")
        want = _torch().float32 if self.precision == FP32 else _torch().float64
        if t.dtype != want:
            raise ValueError(f"device state must be {want}")
        return C.c_void_p(t.data_ptr()), DEVICE, t

    def set_state(self, U, kind=CONSERVED):
        p, where, keep = self._buf(U)
        _check(load().msh_set_state(self.h, p, where, kind))

    def get_state(self, kind=CONSERVED, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, where, keep = self._buf(out)
        _check(load().msh_get_state(self.h, p, where, kind))
        return out

    def set_potential(self, phi):
        if phi is None:
            _check(load().msh_set_potential(self.h, None, HOST))
            return
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        _check(load().msh_set_potential(self.h, phi.ctypes.data_as(C.c_void_p), HOST))

    def set_time(self, t, step=0):
        _check(load().msh_set_time(self.h, float(t), int(step)))

    def time(self):
        t = C.c_double(0.0)
        s = C.c_int64(0)
        _check(load().msh_get_time(self.h, C.byref(t), C.byref(s)))
        return t.value, s.value

    # -- stepping -------------------------------------------------------------
    def step(self, dt_max=float("inf")):
        return msh_step(self.h, dt_max)

    def run(self, t_end=float("inf"), max_steps=(1 << 62)):
        return msh_run(self.h, t_end, max_steps)

    def run_ensemble(self, inputs, outputs, kind=CONSERVED, nsteps=1, check=True):
        """Advance every host state inputs[k] by nsteps CFL steps from t = 0 into outputs[k],
        uploads, steps and downloads overlapped (see ``msh_run_ensemble``); page-locked
        arrays (e.g. ``torch.empty(...).pin_memory().numpy()``) let the copies overlap.
        Returns the per-state statuses; check=True raises MshError if a state failed."""
        n = len(inputs)
        if len(outputs) != n:
            raise ValueError("inputs and outputs differ in length")
        size = int(np.prod(self.shape))

        def ptr(a, writable):
            ok = (isinstance(a, np.ndarray) and a.dtype == self.dtype and a.flags.c_contiguous and a.size == size
                  and (a.flags.writeable or not writable))
            if not ok:
                raise ValueError("ensemble states must be C-contiguous host arrays of the grid's dtype and size")
            return a.ctypes.data

        ins = (C.c_void_p * max(n, 1))(*[ptr(a, False) for a in inputs])
        outs = (C.c_void_p * max(n, 1))(*[ptr(a, True) for a in outputs])
        status = np.zeros(max(n, 1), dtype=np.int32)
        st = load().msh_run_ensemble(self.h, n, ins, outs, int(kind), int(nsteps),
                                     status.ctypes.data_as(C.POINTER(C.c_int32)))
        if check or st != MSH_E_REALIZABILITY:
            _check(st)
        return status[:n]

    def diagnostics(self):
        tot = np.zeros(10)
        ok = C.c_int32(0)
        bad = C.c_int64(0)
        _check(load().msh_diagnostics(self.h, _ptr_dbl(tot), C.byref(ok), C.byref(bad)))
        return tot, bool(ok.value), bad.value

    def set_recording(self, capacity):
        _check(load().msh_set_recording(self.h, int(capacity)))

    def dt_history(self, capacity=None):
        cnt = C.c_int64(0)
        _check(load().msh_get_dt_history(self.h, None, 0, C.byref(cnt)))
        n = cnt.value if capacity is None else min(cnt.value, capacity)
        out = np.zeros(max(n, 1))
        _check(load().msh_get_dt_history(self.h, _ptr_dbl(out), n, C.byref(cnt)))
        return out[:n]

    def set_tiling(self, rows, zchunk=1):
        _check(load().msh_set_tiling(self.h, int(rows), int(zchunk)))

    def tiling(self):
        r, z = C.c_int32(0), C.c_int32(0)
        _check(load().msh_get_tiling(self.h, C.byref(r), C.byref(z)))
        return r.value, z.value

    def autotune(self):
        r, z = C.c_int32(0), C.c_int32(0)
        _check(load().msh_autotune(self.h, C.byref(r), C.byref(z)))
        return r.value, z.value

    def set_profiling(self, on=True):
        _check(load().msh_set_profiling(self.h, int(bool(on))))

    def set_test_fault(self, kind):
        """Test hook of the bounded bulk-copy waits of the 3D step (see msh_set_test_fault)."""
        _check(load().msh_set_test_fault(self.h, int(kind)))

    def profile(self):
        """(summed step-kernel ms, summed finalize ms, timed launches) since profiling began."""
        ms = C.c_double(0.0)
        fin = C.c_double(0.0)
        n = C.c_int64(0)
        _check(load().msh_get_profile(self.h, C.byref(ms), C.byref(fin), C.byref(n)))
        return ms.value, fin.value, n.value

    # -- adjoint --------------------------------------------------------------
    def adjoint_run(self, U0, dt_sched, dL_dUN, K=50, kind=CONSERVED, out=None):
        """dL/dU0 = (dU_N/dU_0)^T dL/dU_N for the frozen schedule ``dt_sched``."""
        dts = np.ascontiguousarray(dt_sched, dtype=np.float64)
        p0, w0, k0 = self._buf(U0)
        pg, wg, kg = self._buf(dL_dUN)
        if w0 != wg:
            raise ValueError("U0 and dL_dUN must both be host or both be device arrays")
        if out is None:
            if w0 == HOST:
                out = np.empty(self.shape, dtype=self.dtype)
            else:
                out = _torch().empty_like(dL_dUN)
        po, wo, ko = self._buf(out)
        _check(load().msh_adjoint_run(self.h, p0, len(dts), _ptr_dbl(dts), int(K), pg, po, w0, kind))
        return out

    def set_self_gravity(self, G):
        """Periodic self-gravity with constant G (0: off); see ``msh_set_self_gravity``."""
        _check(load().msh_set_self_gravity(self.h, float(G)))

    def set_scheme(self, scheme):
        """MUSCL_HANCOCK (default, HLL), MUSCL_HANCOCK_ROE, MUSCL_HANCOCK_HLLC or KT (see
        ``msh_set_scheme``)."""
        _check(load().msh_set_scheme(self.h, int(scheme)))

    def set_ctu(self, on=True):
        """Corner-transport-upwind form of the characteristic schemes (transverse terms in
        the face states, max-form CFL rule; see ``msh_set_ctu``)."""
        _check(load().msh_set_ctu(self.h, 1 if on else 0))

    def get_ctu(self):
        r = C.c_int32()
        _check(load().msh_get_ctu(self.h, C.byref(r)))
        return bool(r.value)

    # -- slab decomposition -------------------------------------------------------
    def set_cell_width(self, dx):
        """Cell widths of the active dims (see ``msh_set_cell_width``)."""
        w = np.zeros(3)
        w[: len(dx)] = dx
        _check(load().msh_set_cell_width(self.h, _ptr_dbl(w)))

    def layer_shape(self):
        """(layers, cells per layer) of the last active axis."""
        layers = self.n[self.ndim - 1]
        return layers, int(np.prod(self.n[: self.ndim - 1]))

    def get_slab(self, start, count, out=None):
        """Layers [start, start+count) of the conserved state as [10, count * cells per layer]
        (numpy, or a torch CUDA tensor when ``out`` is one)."""
        _, per = self.layer_shape()
        if out is None:
            out = np.empty((10, count * per), dtype=self.dtype)
        p, w, keep = self._slab_buf(out, count * per)
        _check(load().msh_get_slab(self.h, int(start), int(count), p, w))
        return out

    def set_slab(self, start, count, buf):
        _, per = self.layer_shape()
        p, w, keep = self._slab_buf(buf, count * per)
        _check(load().msh_set_slab(self.h, int(start), int(count), p, w))

    def _slab_buf(self, a, cells):
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=self.dtype)
            if a.size != 10 * cells:
                raise ValueError(f"slab buffer must have {10 * cells} elements")
            return a.ctypes.data_as(C.c_void_p), HOST, a
        want = _torch().float32 if self.precision == FP32 else _torch().float64
        if not a.is_contiguous() or a.numel() != 10 * cells or a.dtype != want:
            raise ValueError("device slab buffer must be contiguous, of the grid's dtype and size")
        return C.c_void_p(a.data_ptr()), DEVICE, a

    def reduce_layers(self, start, count):
        """(totals[10], CFL dt, realizable) over layers [start, start+count)."""
        tot = np.zeros(10)
        dt = C.c_double(0.0)
        ok = C.c_int32(0)
        _check(load().msh_reduce_layers(self.h, int(start), int(count), _ptr_dbl(tot), C.byref(dt), C.byref(ok)))
        return tot, dt.value, bool(ok.value)

    def step_dt(self, dt):
        """One step with exactly dt; returns the number of cells the fallback tagged."""
        tagged = C.c_int32(0)
        _check(load().msh_step_dt(self.h, float(dt), C.byref(tagged)))
        return tagged.value

    # -- phased step (slabs sharing the a-posteriori fallback; see msh_step_begin) ----
    def step_begin(self, dt):
        _check(load().msh_step_begin(self.h, float(dt)))

    def step_retry(self, level):
        _check(load().msh_step_retry(self.h, int(level)))

    def step_end(self):
        """Finishes the phased step; returns the cells this grid's pass 0 tagged."""
        tagged = C.c_int32(0)
        _check(load().msh_step_end(self.h, C.byref(tagged)))
        return tagged.value

    def get_tags(self, start, count):
        """Per cell of layers [start, start + count): the pass of this step that tagged it, or -1."""
        per = int(np.prod(self.layer_shape()[1:]))
        out = np.empty(count * per, dtype=np.int32)
        _check(load().msh_get_tags(self.h, int(start), int(count), out.ctypes.data_as(C.c_void_p), HOST))
        return out

    def set_tags(self, start, count, levels):
        lv = np.ascontiguousarray(levels, dtype=np.int32).reshape(-1)
        per = int(np.prod(self.layer_shape()[1:]))
        if lv.size != count * per:
            raise ValueError("levels must have one entry per cell of the layers")
        _check(load().msh_set_tags(self.h, int(start), int(count), lv.ctypes.data_as(C.c_void_p), HOST))

    def count_tags(self, start, count, level):
        n = C.c_int64(0)
        _check(load().msh_count_tags(self.h, int(start), int(count), int(level), C.byref(n)))
        return n.value

    def set_tape(self, K, max_steps):
        """Record checkpoints every K steps, dts and fallback flags of the next max_steps
        steps (K = 0 frees the tape); see ``msh_set_tape``."""
        _check(load().msh_set_tape(self.h, int(K), int(max_steps)))

    def adjoint_tape(self, dL_dUN, kind=CONSERVED, out=None):
        """dL/dU0 over the steps recorded since ``set_tape`` (see ``msh_adjoint_tape``)."""
        pg, wg, kg = self._buf(dL_dUN)
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype) if wg == HOST else _torch().empty_like(dL_dUN)
        po, wo, ko = self._buf(out)
        if wo != wg:
            raise ValueError("dL_dUN and out must both be host or both be device arrays")
        _check(load().msh_adjoint_tape(self.h, pg, po, wg, kind))
        return out


class Batch:
    """Batched independent 1D Riemann tubes (see ``msh_batch_init``)."""

    def __init__(self, length, WL, WR, t_end, cfl=0.8, precision=FP32, stream=None):
        self.length = np.ascontiguousarray(length, dtype=np.int32)
        self.ntubes = len(self.length)
        WL = np.ascontiguousarray(WL, dtype=np.float64)
        WR = np.ascontiguousarray(WR, dtype=np.float64)
        te = np.ascontiguousarray(np.broadcast_to(np.asarray(t_end, dtype=np.float64), (self.ntubes,)))
        self.precision = precision
        self.dtype = np.float32 if precision == FP32 else np.float64
        self.total = int(self.length.sum())
        self.offsets = np.concatenate([[0], np.cumsum(self.length)])
        h = C.c_void_p()
        _check(load().msh_batch_init(C.byref(h), self.ntubes,
                                     self.length.ctypes.data_as(C.POINTER(C.c_int32)), _ptr_dbl(WL),
                                     _ptr_dbl(WR), _ptr_dbl(te), int(precision), float(cfl),
                                     C.c_void_p(stream) if stream else None))
        self.h = h

    def close(self):
        if self.h:
            _check(load().msh_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(load().msh_batch_reset(self.h))

    def run(self, threads=0, max_steps=1 << 40):
        _check(load().msh_batch_run(self.h, int(threads), int(max_steps)))

    def run_per_tube(self, tubes=None, max_steps=1 << 40):
        if tubes is None:
            _check(load().msh_batch_run_per_tube(self.h, None, 0, int(max_steps)))
        else:
            t = np.ascontiguousarray(tubes, dtype=np.int32)
            _check(load().msh_batch_run_per_tube(self.h, t.ctypes.data_as(C.POINTER(C.c_int32)), len(t),
                                                 int(max_steps)))

    def get_state(self, kind=CONSERVED):
        out = np.empty((10, self.total), dtype=self.dtype)
        _check(load().msh_batch_get_state(self.h, out.ctypes.data_as(C.c_void_p), HOST, kind))
        return out

    def tube(self, U, k):
        return U[:, self.offsets[k]:self.offsets[k + 1]]

    def info(self):
        steps = np.zeros(self.ntubes, dtype=np.int64)
        t = np.zeros(self.ntubes)
        cu = C.c_int64(0)
        _check(load().msh_batch_info(self.h, steps.ctypes.data_as(C.POINTER(C.c_int64)), _ptr_dbl(t),
                                     C.byref(cu)))
        return steps, t, cu.value

    def fallback_steps(self):
        """Per tube, the steps of the last run that took the a-posteriori fallback passes."""
        counts = np.zeros(self.ntubes, dtype=np.int64)
        _check(load().msh_batch_fallback_steps(self.h, counts.ctypes.data_as(C.POINTER(C.c_int64))))
        return counts
