"""Seeded synthetic inputs (initial conditions and external potentials).

This module is shared by the tests, the benchmark and the oracle harness.  It holds
no arithmetic of the solver itself: it only draws random numbers and evaluates the
initial-condition formulas, and it returns PRIMITIVE states
W = (rho, u_x, u_y, u_z, P_xx, P_xy, P_xz, P_yy, P_yz, P_zz) as float64 arrays of
shape [10][nz][ny][nx].  The conversion to conserved variables belongs to each side
(the CUDA library and the oracle) separately.

Each generator uses numpy's PCG64 seeded with the workload number, so both sides see
identical inputs.  The workloads mirror the paper's test problems (Sec. 4):

* ``sod``   -- 1D shock tube of Sec. 4.1 (gamma = 3 reduction of Sec. 4);
* ``blast`` -- 2D anisotropic-stress blast, periodic unit square;
* ``turb``  -- 3D periodic box with lognormal density, k^-2 Gaussian random fields
              and a random SPD stress tensor per cell;
* ``tubes`` -- thousands of independent 1D Riemann problems of uneven length;
* ``disc``  -- 2D stellar disc in a fixed logarithmic potential with Toomre Q = 1.2
              (Sec. 4.4's Q_T definition; the paper's own disc model is not available,
              so this is a synthetic stand-in).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, OUTFLOW, REFLECT = 0, 1, 2


@dataclass
class Problem:
    """A grid problem: primitive state ``W`` [10][nz][ny][nx], geometry and run control."""
    name: str
    W: np.ndarray
    lo: tuple
    hi: tuple
    bc: tuple                       # ((lo, hi),) per active dim
    cfl: float
    t_end: float = math.inf
    nsteps: int | None = None
    phi: np.ndarray | None = None   # potential with one ghost layer on active dims
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.bc)

    @property
    def n(self):
        nz, ny, nx = self.W.shape[1:]
        return (nx, ny, nz)[: self.ndim]


def _spd_field(rng, shape, diag_lo, diag_hi, off_sigma):
    """P = L L^T per cell, L lower triangular with U[diag_lo, diag_hi] diagonal and
    N(0, off_sigma) off-diagonal entries.  Returns the six components in primitive
    order (xx, xy, xz, yy, yz, zz)."""
    l11, l22, l33 = (rng.uniform(diag_lo, diag_hi, shape) for _ in range(3))
    l21, l31, l32 = (rng.normal(0.0, off_sigma, shape) for _ in range(3))
    Pxx = l11 * l11
    Pxy = l21 * l11
    Pxz = l31 * l11
    Pyy = l21 * l21 + l22 * l22
    Pyz = l31 * l21 + l32 * l22
    Pzz = l31 * l31 + l32 * l32 + l33 * l33
    return Pxx, Pxy, Pxz, Pyy, Pyz, Pzz


# ----------------------------------------------------------------------------- sod
def sod(n=256, t_end=0.2, cfl=0.8, x0=0.5):
    """1D shock tube: left rho = 1, P = 1 I; right rho = 0.125, P = 0.1 I; u = 0;
    outflow boundaries on [0, 1]."""
    x = (np.arange(n) + 0.5) / n
    left = x < x0
    W = np.zeros((10, 1, 1, n))
    W[0, 0, 0] = np.where(left, 1.0, 0.125)
    for c in (4, 7, 9):
        W[c, 0, 0] = np.where(left, 1.0, 0.1)
    return Problem("sod", W, (0.0,), (1.0,), ((OUTFLOW, OUTFLOW),), cfl, t_end=t_end,
                   extra={"x0": x0,
                          "left": dict(rho=1.0, u=0.0, Pxx=1.0, Pyy=1.0, Pzz=1.0),
                          "right": dict(rho=0.125, u=0.0, Pxx=0.1, Pyy=0.1, Pzz=0.1)})


# --------------------------------------------------------------------------- blast
def blast(n=1024, nsteps=200, cfl=0.5, seed=2, radius=0.1):
    """2D anisotropic-stress blast on the periodic unit square.  Background rho = 1,
    u = 0, P = diag(0.1, 0.1, 0.1); disc of radius ``radius`` about the centre with
    P_xx = 10, P_yy = 1, P_xy = 2 (P_zz = 0.1, P_xz = P_yz = 0); 1 % uniform density
    noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    disc = (X - 0.5) ** 2 + (Y - 0.5) ** 2 < radius ** 2
    W = np.zeros((10, 1, n, n))
    W[0, 0] = 1.0 + 0.01 * rng.uniform(-1.0, 1.0, (n, n))
    W[4, 0] = np.where(disc, 10.0, 0.1)
    W[5, 0] = np.where(disc, 2.0, 0.0)
    W[7, 0] = np.where(disc, 1.0, 0.1)
    W[9, 0] = 0.1
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
    return Problem("blast", W, (0.0, 0.0), (1.0, 1.0), bc, cfl, nsteps=nsteps)


# ---------------------------------------------------------------------------- turb
def gaussian_random_field(rng, n, slope=-2.0, kmax=None):
    """Unit-variance periodic Gaussian random field on n^3 with energy spectrum
    E(k) ~ k^slope for 1 <= |k| <= kmax (3D power ~ k^(slope-2)); k = 0 removed."""
    kmax = n // 2 if kmax is None else kmax
    k = np.fft.fftfreq(n, d=1.0 / n)
    kz = k[:, None, None]
    ky = k[None, :, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    band = (kk >= 1.0) & (kk <= kmax)
    amp[band] = kk[band] ** ((slope - 2.0) / 2.0)
    noise = rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape)
    f = np.fft.irfftn(noise * amp, s=(n, n, n), axes=(0, 1, 2))
    f -= f.mean()
    f /= f.std()
    return f


def turb(n=256, nsteps=50, cfl=0.5, seed=3):
    """3D periodic turbulent box: lognormal density (sigma = 0.5, mean 1) from a k^-2
    Gaussian random field, velocity from three independent k^-2 fields with rms |u| = 1,
    and P = L L^T per cell (diagonal U[0.3, 1], off-diagonal N(0, 0.1))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = np.zeros((10, n, n, n))
    g = gaussian_random_field(rng, n)
    W[0] = np.exp(0.5 * g - 0.125)
    vel = [gaussian_random_field(rng, n) for _ in range(3)]
    rms = math.sqrt(float(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)))
    for i in range(3):
        W[1 + i] = vel[i] / rms
    P = _spd_field(rng, (n, n, n), 0.3, 1.0, 0.1)
    for c, v in zip((4, 5, 6, 7, 8, 9), P):
        W[c] = v
    bc = ((PERIODIC, PERIODIC),) * 3
    return Problem("turb", W, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), bc, cfl, nsteps=nsteps)


# --------------------------------------------------------------------------- tubes
@dataclass
class Tubes:
    """Independent 1D Riemann problems on [0, 1] (interface 0.5, outflow, CFL ``cfl``).
    ``length[k]`` cells; ``WL[k]``, ``WR[k]`` primitive left/right states (10 each)."""
    length: np.ndarray
    WL: np.ndarray
    WR: np.ndarray
    t_end: float
    cfl: float

    def initial_tube(self, k):
        n = int(self.length[k])
        x = (np.arange(n) + 0.5) / n
        W = np.where((x < 0.5)[None, :], self.WL[k][:, None], self.WR[k][:, None])
        return W.reshape(10, 1, 1, n)


def tubes(ntubes=4096, nmin=128, nmax=2048, t_end=0.1, cfl=0.8, seed=4):
    """Batched Riemann problems: lengths log-uniform in [nmin, nmax]; per side rho
    log-uniform [0.1, 10], u_x uniform [-1, 1], u_y = u_z = 0, P = L L^T (diagonal
    U[0.1, 1], off-diagonal N(0, 0.2)); draws whose exact solution contains vacuum are
    redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    length = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), ntubes))).astype(np.int32)

    def draw(m):
        W = np.zeros((m, 10))
        W[:, 0] = np.exp(rng.uniform(math.log(0.1), math.log(10.0), m))
        W[:, 1] = rng.uniform(-1.0, 1.0, m)
        P = _spd_field(rng, (m,), 0.1, 1.0, 0.2)
        for c, v in zip((4, 5, 6, 7, 8, 9), P):
            W[:, c] = v
        return W

    WL, WR = draw(ntubes), draw(ntubes)
    # Riemann problems whose exact solution contains vacuum (the two states separate faster
    # than the sum of their fast speeds, u_R - u_L >= cf_L + cf_R with cf = sqrt(3 P_xx/rho))
    # are redrawn: zero density is outside the moment closure's validity.
    while True:
        cf = lambda W: np.sqrt(3.0 * W[:, 4] / W[:, 0])
        vac = np.where(WR[:, 1] - WL[:, 1] >= cf(WL) + cf(WR))[0]
        if len(vac) == 0:
            break
        WL[vac], WR[vac] = draw(len(vac)), draw(len(vac))
    return Tubes(length, WL, WR, t_end, cfl)


# ---------------------------------------------------------------------------- disc
DISC_DEFAULTS = dict(L=20.0, v0=1.0, Rc=1.0, Rd=3.0, Sigma0=0.1, G=1.0, Q=1.2,
                     sigma_floor=0.05, R_loss=10.0)


def disc_potential(n=512, L=20.0, v0=1.0, Rc=1.0):
    """Phi = v0^2/2 ln(Rc^2 + R^2) at cell centres with one ghost layer: [1][n+2][n+2]."""
    dx = 2.0 * L / n
    c = -L + (np.arange(-1, n + 1) + 0.5) * dx
    X, Y = np.meshgrid(c, c, indexing="xy")
    return (0.5 * v0 * v0 * np.log(Rc * Rc + X * X + Y * Y)).reshape(1, n + 2, n + 2)


def disc_profiles(R, v0=1.0, Rc=1.0, Rd=3.0, Sigma0=0.1, G=1.0, Q=1.2, sigma_floor=0.05):
    """Axisymmetric surface density, radial dispersion (Toomre Q_T = sigma kappa /
    (3.36 G Sigma), Sec. 4.4) and circular speed of the unperturbed disc."""
    Sigma = Sigma0 * np.exp(-R / Rd)
    kappa = np.sqrt(v0 * v0 * (2.0 * R * R + 4.0 * Rc * Rc)) / (R * R + Rc * Rc)
    sigR = np.maximum(3.36 * Q * G * Sigma / kappa, sigma_floor * v0)
    vc2 = v0 * v0 * R * R / (R * R + Rc * Rc)
    return Sigma, sigR, vc2


def disc_noise(n=512, seed=5):
    """The seeded perturbation field xi ~ U[-1, 1] (delta = 0.01 xi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, (n, n))


def disc_base(n=512, **kw):
    """Unperturbed fields of the disc on the n x n grid: dict with Sigma (unperturbed
    surface density), sig2 (sigma_R^2), vc2, jeans = (R/Sigma) d(Sigma sigma_R^2)/dR,
    cphi, sphi, R, and the parameters."""
    p = dict(DISC_DEFAULTS)
    p.update(kw)
    L = p["L"]
    dx = 2.0 * L / n
    c = -L + (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(c, c, indexing="xy")
    R = np.sqrt(X * X + Y * Y)
    prof = dict(v0=p["v0"], Rc=p["Rc"], Rd=p["Rd"], Sigma0=p["Sigma0"], G=p["G"], Q=p["Q"],
                sigma_floor=p["sigma_floor"])
    Sigma, sigR, vc2 = disc_profiles(R, **prof)
    h = 1e-5
    f = lambda r: (lambda s, sr, _: s * sr * sr)(*disc_profiles(r, **prof))
    dfdR = (f(R + h) - f(np.maximum(R - h, 0.0))) / (R + h - np.maximum(R - h, 0.0))
    Rs = np.maximum(R, 1e-30)
    return dict(Sigma=Sigma, sig2=sigR * sigR, vc2=vc2, jeans=R / Sigma * dfdR, cphi=X / Rs, sphi=Y / Rs,
                R=R, X=X, Y=Y, dx=dx, params=p)


def disc_compose(base, delta, beta, xp=np):
    """Primitive disc state [10, 1, n, n] from the base fields, the perturbation field delta
    and the anisotropy beta.  Written with the array module ``xp`` (numpy or torch), so the
    same composition serves the seeded input and a differentiable map of (delta, beta)."""
    S = base["Sigma"] * (1.0 + delta)
    sig2 = base["sig2"]
    vphi = xp.sqrt(xp.clamp(base["vc2"] - beta * sig2 + base["jeans"], min=0.0) if xp is not np
                   else np.maximum(base["vc2"] - beta * sig2 + base["jeans"], 0.0))
    c, s = base["cphi"], base["sphi"]
    Pr = S * sig2
    Pp = S * sig2 * (1.0 + beta)
    zero = 0.0 * S
    comps = [S, -vphi * s, vphi * c, zero, Pr * c * c + Pp * s * s, (Pr - Pp) * c * s, zero,
             Pr * s * s + Pp * c * c, zero, S * sig2]
    W = xp.stack(comps)
    return W.reshape((10, 1) + tuple(S.shape))


def disc(n=512, nsteps=2000, cfl=0.5, seed=5, beta=0.0, delta=None, **kw):
    """2D stellar disc over [-L, L]^2 (outflow) in the fixed logarithmic potential.
    Sigma = Sigma0 exp(-R/Rd) (1 + delta) with delta = 0.01 xi; in-plane dispersion
    P = Sigma sigma_R^2 [e_R e_R^T + (1 + beta) e_phi e_phi^T], P_zz = Sigma sigma_R^2;
    rotation from the Jeans (asymmetric drift) relation
    v_phi^2 = v_c^2 + sigma_R^2 - sigma_phi^2 + (R/Sigma) d(Sigma sigma_R^2)/dR."""
    base = disc_base(n, **kw)
    p = base["params"]
    L = p["L"]
    if delta is None:
        delta = 0.01 * disc_noise(n, seed)
    W = disc_compose(base, delta, beta)
    phi = disc_potential(n, L, p["v0"], p["Rc"])
    bc = ((OUTFLOW, OUTFLOW), (OUTFLOW, OUTFLOW))
    return Problem("disc", W, (-L, -L), (L, L), bc, cfl, nsteps=nsteps, phi=phi,
                   extra={"R_loss": p["R_loss"], "beta": beta, "params": p})


def small(name):
    """Small variants of each workload for parity tests (seconds on the oracle)."""
    if name == "sod":
        return sod(256)
    if name == "blast":
        return blast(n=96, nsteps=20)
    if name == "turb":
        return turb(n=24, nsteps=6)
    if name == "disc":
        return disc(n=64, nsteps=20)
    raise KeyError(name)
