"""Pins of the oracle's periodic self-gravity: the FFT potential satisfies the 3-point
discrete Poisson equation, checked by applying the stencil in real space; the linear Jeans
problem of the ten-moment system (dispersion relation omega^2 = 3 sigma^2 k^2 - 4 pi G rho0
from the continuity, momentum and P_xx equations with Poisson's equation) grows at its
rate below the Jeans wavenumber and oscillates at its frequency above it."""
import numpy as np
import pytest

from oracle import selfgrav


def _laplacian(phi, dx):
    nd = len(dx)
    out = np.zeros_like(phi)
    for d in range(nd):
        ax = 2 - d
        out += (np.roll(phi, 1, ax) - 2 * phi + np.roll(phi, -1, ax)) / dx[d] ** 2
    return out


@pytest.mark.parametrize("shape,dx", [((1, 1, 32), (0.1,)), ((1, 12, 20), (0.05, 0.2)), ((6, 10, 8), (0.3, 0.1, 0.2))])
def test_potential_solves_discrete_poisson(shape, dx):
    rng = np.random.default_rng(len(dx))
    rho = np.exp(rng.normal(0, 0.5, shape))
    G = 0.7
    phi = selfgrav.poisson_periodic(rho, dx, G)
    res = _laplacian(phi, dx) - 4 * np.pi * G * (rho - rho.mean())
    assert np.abs(res).max() <= 1e-10 * np.abs(4 * np.pi * G * rho).max()
    assert abs(phi.mean()) <= 1e-12 * np.abs(phi).max()


def _jeans(oracle, k_mult, steps_to, sigma2=0.01, n=64, L=4.0, eps=1e-4, cfl=0.2, every=10):
    """1D periodic medium rho0 = 1, P = sigma2 I, G = 1/(4 pi) (4 pi G rho0 = 1), density mode
    k = 2 pi k_mult / L; returns (times, signed amplitudes of the cos(kx) mode, omega^2)."""
    G = 1.0 / (4 * np.pi)
    x = (np.arange(n) + 0.5) * L / n
    k = 2 * np.pi * k_mult / L
    om2 = 3 * sigma2 * k * k - 1.0
    W = np.zeros((10, 1, 1, n))
    W[0, 0, 0] = 1 + eps * np.cos(k * x)
    W[4, 0, 0] = sigma2 * (1 + 3 * eps * np.cos(k * x))  # dP_xx / P = 3 drho / rho
    W[7] = W[9] = sigma2
    if om2 < 0:  # growing mode: du = -(gamma / k) eps sin(kx)
        W[1, 0, 0] = -np.sqrt(-om2) / k * eps * np.sin(k * x)
    g = oracle.Grid((n,), (0.0,), (L,), ((0, 0),), cfl)
    U = oracle.prim_to_cons(W)
    ts, amps = [0.0], [eps]
    t = 0.0
    hist = {}
    while t < steps_to:
        U, dts = selfgrav.run(g, U, every, G, hist)
        t += sum(dts)
        rho = U[0, 0, 0]
        ts.append(t)
        amps.append(2 * np.sum((rho - 1) * np.cos(k * x)) / n)
    return np.array(ts), np.array(amps), om2


def test_jeans_growth_rate(oracle):
    ts, amps, om2 = _jeans(oracle, 1, 3.0)
    gamma = np.sqrt(-om2)
    fit = np.polyfit(ts[2:], np.log(np.abs(amps[2:])), 1)[0]
    assert abs(fit - gamma) <= 0.03 * gamma, (fit, gamma)


def test_jeans_oscillation_frequency(oracle):
    """Above the Jeans wavenumber a standing density wave released from rest oscillates as
    cos(omega t): its first zero comes at pi / (2 omega)."""
    ts, amps, om2 = _jeans(oracle, 6, 2.0, every=1)
    omega = np.sqrt(om2)
    t0 = np.pi / (2 * omega)
    i = int(np.argmax(amps < 0))  # first sample past the zero
    tz = ts[i - 1] + (ts[i] - ts[i - 1]) * amps[i - 1] / (amps[i - 1] - amps[i])
    assert abs(tz - t0) <= 0.05 * t0, (tz, t0)
