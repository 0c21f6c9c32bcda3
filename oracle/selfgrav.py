"""Self-gravity for the oracle (TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the
CPU legs of bench.py may use it; the CUDA path shares nothing with it).

Periodic grids: the potential solves the discrete Poisson equation
    sum_d (Phi_{i+e_d} - 2 Phi_i + Phi_{i-e_d}) / dx_d^2 = 4 pi G (rho_i - mean rho)
(the mean is removed, as on any periodic domain), by the FFT: the 3-point Laplacian has the
eigenvalues -sum_d (2 sin(k_d dx_d / 2) / dx_d)^2 on the modes exp(i k . x).  The gravity
source is the step's (a8: a = -grad Phi by central differences after the hydro update).
Sec. 3.3 (last paragraph) keeps it second order in time by storing the previous step's
acceleration and interpolating forward; read here as
    a^{n+1/2} = a^n + (dt_n / (2 dt_{n-1})) (a^n - a^{n-1})   (a^{1/2} = a^0),
applied through the potential, on which a depends linearly.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def poisson_periodic(rho, dx, G=1.0):
    """Potential [nz][ny][nx] of the density rho [nz][ny][nx] (active dims: the last len(dx))."""
    rho = np.asarray(rho, dtype=np.float64)
    nd = len(dx)
    axes = tuple(range(3 - nd, 3))
    rk = np.fft.fftn(rho - rho.mean(), axes=axes)
    lap = np.zeros(rho.shape)
    for j, d in enumerate(range(nd)):
        ax = 2 - d  # array axis of dimension d in [nz][ny][nx]
        n = rho.shape[ax]
        k = 2.0 * np.pi * np.fft.fftfreq(n)  # k dx
        eig = (2.0 * np.sin(k / 2.0) / dx[d]) ** 2
        shape = [1, 1, 1]
        shape[ax] = n
        lap = lap + eig.reshape(shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = np.where(lap > 0.0, -4.0 * np.pi * G * rk / lap, 0.0)
    return np.real(np.fft.ifftn(pk, axes=axes))


def with_ghosts(phi, nd):
    """Periodic ghost layer on the active dims: [nz+2gz][ny+2gy][nx+2gx]."""
    pads = [(0, 0)] * (3 - nd) + [(1, 1)] * nd
    return np.pad(phi, pads, mode="wrap")


def run(grid: O.Grid, U, steps, G=1.0, history=None, phi_ext=None):
    """``steps`` CFL steps with self-gravity; returns (U, dt list).  ``history`` (a dict,
    updated in place) carries the previous step's potential and dt across calls;
    ``phi_ext`` (with its ghost layer) is an external potential added to the self-potential."""
    nd = grid.ndim
    dx = grid.dx[:nd]
    U = np.array(U, dtype=np.float64).reshape(grid.shape)
    h = history if history is not None else {}
    dts = []
    for _ in range(steps):
        dt = O.cfl_dt(grid, U)
        phi = poisson_periodic(U[0], dx, G)
        prev = h.get("phi")
        phi_half = phi if prev is None else phi + (dt / (2.0 * h["dt"])) * (phi - prev)
        ph = with_ghosts(phi_half, nd)
        if phi_ext is not None:
            ph = ph + np.asarray(phi_ext, dtype=np.float64).reshape(ph.shape)
        U = O.step(grid, U, dt, phi=ph)
        h["phi"], h["dt"] = phi, dt
        dts.append(dt)
    return U, dts
