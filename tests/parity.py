"""Norms and comparison helpers for GPU-vs-oracle parity (test helper).

Norms (the paper defines none): per field, relative L_inf = max|d| / max|x_oracle| and
relative L1 = sum|d| / sum|x_oracle|.  A field that is identically zero in the oracle is
compared in absolute terms against the scale of its family (rho for momenta, the largest
|P| component for the stress tensor).
"""
import numpy as np

P_FIELDS = (4, 5, 6, 7, 8, 9)


def field_errors(gpu, ref, kind="linf"):
    g = np.asarray(gpu, dtype=np.float64).reshape(10, -1)
    r = np.asarray(ref, dtype=np.float64).reshape(10, -1)
    d = np.abs(g - r)
    rho_scale = np.abs(r[0]).max()
    p_scale = np.abs(r[4:]).max()
    out = np.zeros(10)
    for k in range(10):
        scale = np.abs(r[k]).max() if kind == "linf" else np.abs(r[k]).sum()
        if scale == 0.0:
            fam = rho_scale if k < 4 else p_scale
            out[k] = d[k].max() / fam
        else:
            out[k] = (d[k].max() if kind == "linf" else d[k].sum()) / scale
    return out


def assert_fp64(gpu_U, ref_U, tol=1e-10, what=""):
    e = field_errors(gpu_U, ref_U, "linf")
    assert e.max() <= tol, f"{what}: FP64 rel Linf per field {e}"
    return e


def assert_fp32(gpu_W, ref_W, tol_rho=2e-4, tol_P=5e-4, what=""):
    """FP32 GPU vs FP64 oracle: relative L1 on density and on each P_ij (primitive)."""
    e = field_errors(gpu_W, ref_W, "l1")
    assert e[0] <= tol_rho, f"{what}: FP32 rel L1 rho {e[0]:.3e}"
    for k in P_FIELDS:
        assert e[k] <= tol_P, f"{what}: FP32 rel L1 of field {k} = {e[k]:.3e}"
    return e
