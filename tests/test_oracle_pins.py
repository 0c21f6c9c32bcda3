"""Pins for the FP64 oracle: each test checks the oracle against something other than
itself -- moment integrals of a Gaussian velocity distribution, complex-step Jacobians,
exact Riemann solutions, conservation, symmetries, textbook special cases and an
independent brute-force step on tiny grids."""
import math

import numpy as np
import pytest

from oracle.exact_riemann import bme_sod_solution, sample, star_state, wave_speeds
from paper_1210_5246_gb300 import inputs as I
from tests import bruteforce as BF

RNG = np.random.default_rng(1234)


def random_state(rng, u_scale=1.0, off=0.3):
    W = np.zeros(10)
    W[0] = math.exp(rng.uniform(-1, 1))
    W[1:4] = rng.uniform(-u_scale, u_scale, 3)
    L = np.tril(rng.normal(0, off, (3, 3)))
    L[np.diag_indices(3)] = rng.uniform(0.4, 1.2, 3)
    P = L @ L.T
    for (i, j), k in BF.TI.items():
        W[k] = P[i, j]
    return W


def grid_of(o, p):
    return o.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)


# ------------------------------------------------------------------ flux, eigen
@pytest.mark.parametrize("seed", range(5))
def test_flux_equals_gaussian_moments(oracle, seed):
    """Eqs contin/moment/dispers with Q_ijk = 0: the fluxes are the velocity moments of a
    Gaussian distribution (zero heat flux); Gauss-Hermite quadrature is exact here."""
    rng = np.random.default_rng(seed)
    W = random_state(rng)
    for d in range(3):
        np.testing.assert_allclose(oracle.flux(W, d), BF.flux_gh(W, d).real, rtol=1e-13,
                                   atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_isserlis_moments_equal_quadrature(seed):
    """The brute-force step's polynomial moment flux equals the quadrature moments."""
    W = random_state(np.random.default_rng(50 + seed))
    for d in range(3):
        np.testing.assert_allclose(BF.flux_moments(W, d), BF.flux_gh(W, d).real, rtol=1e-13, atol=1e-13)


def test_flux_diagonal_case_matches_printed_vector(oracle):
    """Sec. 3.3 eq conservedfluxes (diagonal stress): F = (rho v_x, rho v_x^2 + P_xx,
    rho v_y v_x, rho v_z v_x, (E_xx + 2 P_xx) v_x, E_yy v_x, E_zz v_x)."""
    W = np.array([1.3, 0.4, -0.2, 0.7, 0.9, 0.0, 0.0, 0.5, 0.0, 0.3])
    rho, vx, vy, vz, Pxx, Pyy, Pzz = W[0], W[1], W[2], W[3], W[4], W[7], W[9]
    Exx, Eyy, Ezz = Pxx + rho * vx * vx, Pyy + rho * vy * vy, Pzz + rho * vz * vz
    F = oracle.flux(W, 0)
    np.testing.assert_allclose(F[[0, 1, 2, 3, 4, 7, 9]],
                               [rho * vx, rho * vx * vx + Pxx, rho * vy * vx, rho * vz * vx,
                                (Exx + 2 * Pxx) * vx, Eyy * vx, Ezz * vx], rtol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_eigensystem(oracle, seed):
    """A from the oracle equals the complex-step primitive Jacobian of the Gaussian-moment
    flux; L R = I; A R = R Lambda; eigenvalues u -+ sqrt(3 Pxx/rho), u -+ sqrt(Pxx/rho), u."""
    rng = np.random.default_rng(100 + seed)
    W = random_state(rng)
    A, lam, R, L = oracle.eigensystem_x(W)
    np.testing.assert_allclose(A, BF.prim_jacobian(W, 0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(L @ R, np.eye(10), atol=1e-13)
    np.testing.assert_allclose(A @ R, R * lam[None, :], atol=1e-12)
    num = np.sort(np.linalg.eigvals(BF.prim_jacobian(W, 0)).real)
    np.testing.assert_allclose(np.sort(lam), num, atol=1e-7)
    cf, cs = math.sqrt(3 * W[4] / W[0]), math.sqrt(W[4] / W[0])
    assert abs(lam.max() - (W[1] + cf)) < 1e-14 and abs(lam.min() - (W[1] - cf)) < 1e-14
    assert abs(sorted(lam)[1] - (W[1] - cs)) < 1e-14


def test_eigensystem_reduces_to_paper_diagonal_case(oracle):
    """With P_xy = P_xz = 0 the fast-wave columns are (rho, +-a, 0, 0, rho a^2, ...) as in
    eq righteigvec, and the fast-wave rows are (0, +-1/(2a), 0, 0, 1/(2 rho a^2), ...)
    as in eq lefteigvec, with a = sqrt(3 P_xx / rho)."""
    W = np.array([0.7, 0.1, 0.0, 0.0, 0.4, 0.0, 0.0, 0.3, 0.0, 0.2])
    A, lam, R, L = oracle.eigensystem_x(W)
    a = math.sqrt(3 * W[4] / W[0])
    rho = W[0]
    np.testing.assert_allclose(R[[0, 1, 4], 9], [rho, a, rho * a * a], rtol=1e-14)
    np.testing.assert_allclose(R[[0, 1, 4], 0], [rho, -a, rho * a * a], rtol=1e-14)
    # the paper's rows are the ones for columns scaled by rho; compare L*rho
    np.testing.assert_allclose(L[9, [1, 4]] * rho, [1 / (2 * a) * rho, 1 / (2 * rho * a * a) * rho],
                               rtol=1e-14)
    np.testing.assert_allclose(L[0, [1, 4]] * rho, [-1 / (2 * a) * rho, 1 / (2 * rho * a * a) * rho],
                               rtol=1e-14)


# ------------------------------------------------------------------- exact Sod
def test_exact_riemann_rankine_hugoniot_and_invariants():
    """Star state of the gamma = 3 Sod problem satisfies the Rankine-Hugoniot jump
    conditions across the shock and the Riemann invariant across the rarefaction."""
    g = 3.0
    rL, uL, pL, rR, uR, pR = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    ps, us, rsL, rsR = star_state(rL, uL, pL, rR, uR, pR, g)
    S = wave_speeds(rL, uL, pL, rR, uR, pR, g)["right_shock"]
    E = lambda r, u, p: p / (g - 1) + 0.5 * r * u * u
    jump = lambda a, b: a - b
    assert abs(jump(rsR * (us - S), rR * (uR - S))) < 1e-12
    assert abs(jump(rsR * us * (us - S) + ps, rR * uR * (uR - S) + pR)) < 1e-12
    assert abs(jump((E(rsR, us, ps)) * (us - S) + ps * us, E(rR, uR, pR) * (uR - S) + pR * uR)) < 1e-12
    cL, csL = math.sqrt(g * pL / rL), math.sqrt(g * ps / rsL)
    assert abs((uL + 2 * cL / (g - 1)) - (us + 2 * csL / (g - 1))) < 1e-12
    assert abs(ps / rsL ** g - pL / rL ** g) < 1e-12
    # the textbook gamma = 1.4 Sod star state
    ps14, us14, _, _ = star_state(rL, uL, pL, rR, uR, pR, 1.4)
    assert abs(ps14 - 0.30313) < 1e-5 and abs(us14 - 0.92745) < 1e-5


def test_exact_sampling_continuity():
    """The sampled solution is continuous through the rarefaction fan edges."""
    S = wave_speeds(1, 0, 1, 0.125, 0, 0.1, 3.0)
    for edge in (S["left_head"], S["left_tail"]):
        r, u, p, _ = sample(np.array([edge - 1e-9, edge + 1e-9]), 1, 0, 1, 0.125, 0, 0.1, 3.0)
        assert abs(r[0] - r[1]) < 1e-7 and abs(p[0] - p[1]) < 1e-7 and abs(u[0] - u[1]) < 1e-7


def _sod_errors(oracle, n):
    p = I.sod(n)
    g = grid_of(oracle, p)
    U, ns, t, rc, _ = oracle.run(g, oracle.prim_to_cons(p.W), p.t_end)
    assert rc == 0 and t == p.t_end
    W = oracle.cons_to_prim(U).reshape(10, -1)
    x = (np.arange(n) + 0.5) / n
    Wex = bme_sod_solution(x, p.t_end, 0.5, p.extra["left"], p.extra["right"])
    return W, Wex, x


def test_sod_converges_to_gamma3_solution(oracle):
    """Sec. 4: the 1D moment equations are classic hydrodynamics with gamma = 3; the
    numerical Sod solution converges to that analytic solution under refinement."""
    errs = []
    for n in (128, 256, 512):
        W, Wex, _ = _sod_errors(oracle, n)
        errs.append([np.abs(W[k] - Wex[k]).mean() for k in (0, 1, 4, 7, 9)])
    errs = np.array(errs)
    assert np.all(errs[1] < 0.75 * errs[0]) and np.all(errs[2] < 0.75 * errs[1])
    assert errs[2, 0] < 3e-3
    # transverse components stay exactly zero
    W, _, _ = _sod_errors(oracle, 128)
    assert np.all(W[[2, 3, 5, 6, 8]] == 0.0)


def test_sod_shock_and_contact_width(oracle):
    """Sec. 4.1: the shock is captured within about two zones and the contact within
    about six (HLLC in the paper; HLL is more diffusive at the contact, so the contact
    allowance here is eight zones)."""
    n = 256
    W, Wex, x = _sod_errors(oracle, n)
    S = wave_speeds(1, 0, 1, 0.125, 0, 0.1, 3.0)
    rho, r_ex = W[0], Wex[0]
    xs = 0.5 + S["right_shock"] * 0.2
    xc = 0.5 + S["contact"] * 0.2
    rsR = S["rho_star_R"]
    mid = 0.5 * (rsR + 0.125)
    ish = np.where((rho > 0.125 + 0.1 * (rsR - 0.125)) & (rho < rsR - 0.1 * (rsR - 0.125)) & (x > xc + 0.05))[0]
    assert len(ish) <= 3 and np.all(np.abs(x[ish] - xs) < 3.0 / n)
    rsL = S["rho_star_L"]
    ict = np.where((rho > rsR + 0.1 * (rsL - rsR)) & (rho < rsL - 0.1 * (rsL - rsR)) & (np.abs(x - xc) < 0.1))[0]
    assert len(ict) <= 8
    assert abs(x[np.argmin(np.abs(rho - mid))] - xs) < 2.0 / n


# --------------------------------------------------------------- conservation
def test_periodic_conservation_all_fields(oracle):
    """Periodic, no gravity: telescoping fluxes conserve all ten totals to round-off."""
    p = I.blast(n=48, nsteps=15)
    g = grid_of(oracle, p)
    U0 = oracle.prim_to_cons(p.W)
    U1, ns, _, rc, _ = oracle.run(g, U0, np.inf, max_steps=15)
    t0, _, _ = oracle.diagnostics(g, U0)
    t1, ok, _ = oracle.diagnostics(g, U1)
    assert rc == 0 and ok and ns == 15
    scale = np.array([t0[0]] * 4 + [abs(t0[4]) + abs(t0[7]) + abs(t0[9])] * 6)
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)


def test_gravity_momentum_budget(oracle):
    """With gravity, sum(m) changes by exactly dt sum(rho a) (sources, Sec. 3.3), mass is
    conserved and P is untouched by the source (u += dt a)."""
    n = 32
    rng = np.random.default_rng(7)
    W = np.zeros((10, 1, n, n))
    W[0, 0] = 1 + 0.2 * rng.uniform(-1, 1, (n, n))
    W[1, 0], W[2, 0] = 0.1, -0.2
    W[4, 0], W[7, 0], W[9, 0], W[5, 0] = 0.5, 0.4, 0.3, 0.05
    g = oracle.Grid((n, n), (0, 0), (1, 1), ((0, 0), (0, 0)), 0.5)
    xs = (np.arange(-1, n + 1) + 0.5) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    phi = (np.sin(2 * np.pi * X) + 0.5 * np.cos(2 * np.pi * Y)).reshape(1, n + 2, n + 2)
    U0 = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U0)
    Uh = oracle.step(g, U0, dt)
    Ug = oracle.step(g, U0, dt, phi=phi)
    ax = -(phi[0, 1:-1, 2:] - phi[0, 1:-1, :-2]) / (2 / n)
    ay = -(phi[0, 2:, 1:-1] - phi[0, :-2, 1:-1]) / (2 / n)
    np.testing.assert_allclose(Ug[1, 0], Uh[1, 0] + dt * Uh[0, 0] * ax, rtol=0, atol=1e-15)
    np.testing.assert_allclose(Ug[2, 0], Uh[2, 0] + dt * Uh[0, 0] * ay, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(Ug[0], Uh[0])
    Wh, Wg = oracle.cons_to_prim(Uh), oracle.cons_to_prim(Ug)
    np.testing.assert_allclose(Wg[4:], Wh[4:], atol=1e-14)
    np.testing.assert_allclose(Wg[1, 0], Wh[1, 0] + dt * ax, atol=1e-14)


# ------------------------------------------------------------------- symmetry
def _mirror_x(U):
    V = U[..., ::-1].copy()
    for k in (1, 5, 6):  # m_x, E_xy, E_xz change sign
        V[k] *= -1
    return V


def test_mirror_symmetry(oracle):
    """x -> -x (reverse cells, negate m_x, E_xy, E_xz) commutes with the step."""
    p = I.blast(n=40, nsteps=5)
    W = p.W.copy()
    W[1, 0] = 0.3 * np.sin(2 * np.pi * (np.arange(40) + 0.5) / 40)[None, :]
    W[5, 0] += 0.01
    g = grid_of(oracle, p)
    U = oracle.prim_to_cons(W)
    A = oracle.run(g, U, np.inf, max_steps=5)[0]
    B = oracle.run(g, _mirror_x(U), np.inf, max_steps=5)[0]
    np.testing.assert_allclose(_mirror_x(B), A, atol=1e-13, rtol=0)


def _swap_xy(U):
    V = np.swapaxes(U, -1, -2).copy()
    perm = [0, 2, 1, 3, 7, 5, 8, 4, 6, 9]
    return V[perm]


def test_xy_swap_symmetry(oracle):
    """Swapping x and y (on a square grid) commutes with the step."""
    rng = np.random.default_rng(3)
    n = 24
    W = np.zeros((10, 1, n, n))
    W[0] = 1 + 0.3 * rng.uniform(-1, 1, (1, n, n))
    W[1:3] = 0.3 * rng.uniform(-1, 1, (2, 1, n, n))
    W[4], W[7], W[9] = 0.6, 0.4, 0.3
    W[5] = 0.1 * rng.uniform(-1, 1, (1, n, n))
    g = oracle.Grid((n, n), (0, 0), (1, 1), ((1, 2), (1, 2)), 0.5)
    U = oracle.prim_to_cons(W)
    A = oracle.run(g, U, np.inf, max_steps=4)[0]
    B = oracle.run(g, _swap_xy(U), np.inf, max_steps=4)[0]
    np.testing.assert_allclose(_swap_xy(B), A, atol=1e-13, rtol=0)


def test_3d_cyclic_symmetry(oracle):
    """Cyclic relabelling x -> y -> z -> x of a periodic cube commutes with the step."""
    p = I.turb(n=12, nsteps=2)
    g = grid_of(oracle, p)
    U = oracle.prim_to_cons(p.W)

    def cyc(V):
        # new axes: (z,y,x) array; x->y, y->z, z->x
        out = np.transpose(V, (0, 2, 3, 1)).copy()  # [c][y][x][z] -> as (z',y',x') with z'=y...
        perm = [0, 3, 1, 2, 9, 6, 8, 4, 5, 7]
        return out[perm]

    A = oracle.run(g, U, np.inf, max_steps=2)[0]
    B = oracle.run(g, cyc(U), np.inf, max_steps=2)[0]
    np.testing.assert_allclose(cyc(A), B, atol=1e-13, rtol=0)


def test_reflect_equals_mirrored_periodic(oracle):
    """A reflecting wall at both ends equals the periodic problem on the mirror-doubled
    domain (ghost cells of a reflect boundary are the mirror images)."""
    rng = np.random.default_rng(11)
    n = 20
    W = np.zeros((10, 1, 1, n))
    W[0] = 1 + 0.4 * rng.uniform(-1, 1, n)
    W[1:4] = 0.3 * rng.uniform(-1, 1, (3, 1, 1, n))
    W[4], W[7], W[9] = 0.6, 0.5, 0.4
    W[5], W[6], W[8] = 0.05, -0.04, 0.03
    U = oracle.prim_to_cons(W)
    gr = oracle.Grid((n,), (0,), (1,), ((2, 2),), 0.8)
    gp = oracle.Grid((2 * n,), (-1,), (1,), ((0, 0),), 0.8)
    Ud = np.concatenate([_mirror_x(U), U], axis=-1)
    A = oracle.run(gr, U, np.inf, max_steps=6)[0]
    B = oracle.run(gp, Ud, np.inf, max_steps=6)[0]
    np.testing.assert_allclose(B[..., n:], A, atol=1e-13, rtol=0)


# ------------------------------------------------------------- special cases
def test_uniform_state_stays_uniform(oracle):
    W = np.zeros((10, 4, 5, 6))
    W[:, ...] = random_state(np.random.default_rng(5))[:, None, None, None]
    g = oracle.Grid((6, 5, 4), (0, 0, 0), (1, 1, 1), ((0, 0), (1, 1), (2, 2)), 0.5)
    U = oracle.prim_to_cons(W)
    # reflect would flip a uniform velocity, so use a state with u_z = 0 and P_xz = P_yz = 0
    W2 = W.copy()
    W2[3], W2[6], W2[8] = 0.0, 0.0, 0.0
    U = oracle.prim_to_cons(W2)
    U1 = oracle.run(g, U, np.inf, max_steps=3)[0]
    np.testing.assert_allclose(U1, U, rtol=1e-14, atol=1e-15)


def _scalar_muscl_hll(rho, u, P, dx, dt):
    """Textbook scalar MUSCL-Hancock + MC limiter + HLL for rho_t + u rho_x = 0 with
    signal speeds u -+ sqrt(3 P / rho) on periodic cells."""
    dL = rho - np.roll(rho, 1)
    dR = np.roll(rho, -1) - rho
    dC = 0.5 * (dL + dR)
    s = np.where(dL * dR > 0, np.sign(dC) * np.minimum(np.minimum(2 * abs(dL), abs(dC)), 2 * abs(dR)), 0.0)
    hi = rho + 0.5 * s - 0.5 * dt / dx * u * s
    lo = rho - 0.5 * s - 0.5 * dt / dx * u * s
    rL, rR = hi, np.roll(lo, -1)  # face i+1/2
    cL, cR = np.sqrt(3 * P / rL), np.sqrt(3 * P / rR)
    SL = np.minimum(u - cL, u - cR)
    SR = np.maximum(u + cL, u + cR)
    F = np.where(SL >= 0, rL * u, np.where(SR <= 0, rR * u,
                 (SR * rL * u - SL * rR * u + SL * SR * (rR - rL)) / (SR - SL)))
    return rho - dt / dx * (F - np.roll(F, 1))


def test_density_bump_reduces_to_scalar_scheme(oracle):
    """Uniform u and P with a density bump: only the density contact wave is active and
    the step reduces to the scalar MUSCL-Hancock/MC/HLL advection of rho, while u and P
    stay exactly uniform."""
    n = 64
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.5 * np.exp(-((x - 0.4) / 0.08) ** 2) + 0.3 * (x > 0.7)
    W = np.zeros((10, 1, 1, n))
    W[0, 0, 0] = rho
    W[1], W[4], W[7], W[9] = 0.7, 0.3, 0.2, 0.1
    g = oracle.Grid((n,), (0,), (1,), ((0, 0),), 0.8)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    U1 = oracle.step(g, U, dt)
    ref = _scalar_muscl_hll(rho, 0.7, 0.3, 1.0 / n, dt)
    np.testing.assert_allclose(U1[0, 0, 0], ref, rtol=1e-13)
    W1 = oracle.cons_to_prim(U1)
    np.testing.assert_allclose(W1[1], 0.7, rtol=1e-13)
    np.testing.assert_allclose(W1[4], 0.3, rtol=1e-12)


def test_cfl_dt_closed_form(oracle):
    """dt = C / max_cells sum_d (|u_d| + sqrt(3 P_dd/rho)) / dx_d."""
    W = np.zeros((10, 1, 2, 3))
    W[0], W[4], W[7], W[9] = 1.0, 0.12, 0.27, 1.0
    W[1, 0, 1, 2], W[2, 0, 1, 2] = -0.5, 0.25
    g = oracle.Grid((3, 2), (0, 0), (3, 1), ((1, 1), (1, 1)), 0.4)
    s = (0.5 + math.sqrt(0.36)) / 1.0 + (0.25 + math.sqrt(0.81)) / 0.5
    assert abs(oracle.cfl_dt(g, oracle.prim_to_cons(W)) - 0.4 / s) < 1e-15


def test_ghost_fill_rules(oracle):
    n = 5
    U = np.arange(10 * n, dtype=float).reshape(10, 1, 1, n) + 1
    for bc, expect in (((0, 0), lambda c: [c[3], c[4], *c, c[0], c[1]]),
                       ((1, 1), lambda c: [c[0], c[0], *c, c[4], c[4]]),
                       ((2, 2), lambda c: [c[1], c[0], *c, c[4], c[3]])):
        G = oracle.ghost_fill(oracle.Grid((n,), (0,), (1,), (bc,), 0.5), U)
        for k in range(10):
            e = np.array(expect(list(U[k, 0, 0])))
            if bc == (2, 2) and k in (1, 5, 6):
                e[[0, 1, -2, -1]] *= -1
            np.testing.assert_array_equal(G[k, 0, 0], e)


def test_realizability_flag(oracle):
    W = np.zeros((10, 1, 1, 4))
    W[0], W[4], W[7], W[9] = 1.0, 1.0, 1.0, 1.0
    W[5, 0, 0, 2] = 1.5  # P_xx P_yy - P_xy^2 < 0
    g = oracle.Grid((4,), (0,), (1,), ((1, 1),), 0.5)
    tot, ok, bad = oracle.diagnostics(g, oracle.prim_to_cons(W))
    assert not ok and bad == 2
    W[5, 0, 0, 2] = 0.5
    assert oracle.diagnostics(g, oracle.prim_to_cons(W))[1]


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("case", ["periodic1d", "outflow1d", "reflect1d", "periodic2d", "gravity2d"])
def test_bruteforce_tiny_grids(oracle, case, seed):
    """8-cell grids: the oracle's step equals the independent brute-force step (numerical
    eigen-decomposition of the complex-step Jacobian of the Gaussian-moment flux)."""
    rng = np.random.default_rng(sum(map(ord, case)) * 7919 + seed)
    ndim = 2 if "2d" in case else 1
    n = 8
    shape = (10, 1, n if ndim == 2 else 1, n)
    W = np.zeros(shape)
    for idx in np.ndindex(shape[1:]):
        W[(slice(None),) + idx] = random_state(rng, u_scale=0.5, off=0.15)
    bcv = {"periodic": 0, "outflow": 1, "reflect": 2, "gravity": 1}[case[:-2].rstrip("0123456789")]
    bc = ((bcv, bcv),) * ndim
    g = oracle.Grid((n,) * ndim, (0,) * ndim, (1,) * ndim, bc, 0.6)
    U = oracle.prim_to_cons(W)
    phi = None
    if case == "gravity2d":
        xs = (np.arange(-1, n + 1) + 0.5) / n
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        phi = (0.5 * X * X - 0.3 * np.sin(3 * Y)).reshape(1, n + 2, n + 2)
    dx = [1.0 / n] * 3
    dt_bf = BF.cfl_dt(U, ndim, dx, 0.6)
    dt = oracle.cfl_dt(g, U)
    assert abs(dt - dt_bf) < 1e-13 * dt
    for _ in range(2):
        A = oracle.step(g, U, dt, phi=phi)
        B = BF.step(U, ndim, dx, bc, dt, phi=phi)
        scale = np.abs(B).reshape(10, -1).max(axis=1)[:, None, None, None] + 1e-300
        assert np.max(np.abs(A - B) / scale) < 1e-11
        U = A
        dt = oracle.cfl_dt(g, U)


# ------------------------------------------------------- a-posteriori fallback
def _extreme_tiny(seed, n=8):
    rng = np.random.default_rng(seed)
    W = np.zeros((10, 1, 1, n))
    W[0] = np.exp(rng.uniform(np.log(0.05), np.log(20), n))
    W[1] = rng.uniform(-1.5, 1.5, n)
    for c in range(n):
        L = np.tril(rng.normal(0, 0.3, (3, 3)))
        L[np.diag_indices(3)] = rng.uniform(0.1, 1, 3)
        P = L @ L.T
        W[4:, 0, 0, c] = [P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]]
    return W


@pytest.mark.parametrize("seed", [1, 13, 31])
def test_fallback_restores_realizability_and_matches_bruteforce(oracle, seed):
    """Extreme 8-cell states where the second-order update leaves a cell non-realizable:
    the step with the first-order fallback is realizable, conserves every total on the
    periodic grid, and equals the independent brute-force step with the same fallback."""
    W = _extreme_tiny(seed)
    g = oracle.Grid((8,), (0,), (1,), ((0, 0),), 0.8)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    assert not oracle.diagnostics(g, oracle.step_second_order_only(g, U, dt))[1]
    A = oracle.step(g, U, dt)
    tot0 = oracle.diagnostics(g, U)[0]
    tot1, ok, _ = oracle.diagnostics(g, A)
    assert ok
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(tot0).max())
    B = BF.step(U, 1, [1 / 8] * 3, ((0, 0),), dt)
    scale = np.abs(B).reshape(10, -1).max(axis=1)[:, None, None, None] + 1e-300
    assert np.max(np.abs(A - B) / scale) < 1e-11


@pytest.mark.parametrize("seed", [1, 13, 31])
def test_step_equals_its_passes_repeated(oracle, seed):
    """og_step is og_step_pass repeated: the second-order pass, then passes with first-order
    faces at every cell tagged so far, a cell being tagged when its update is not realizable,
    at most four fallback passes.  Restated here pass by pass from the exported single pass
    and realizability test (the form a driver uses to share the fallback between slabs):
    bit for bit og_step, on states that take one or more fallback passes."""
    W = _extreme_tiny(seed)
    g = oracle.Grid((8,), (0,), (1,), ((0, 0),), 0.8)
    U = oracle.prim_to_cons(W)
    dt = oracle.cfl_dt(g, U)
    Un = oracle.step_pass(g, U, dt)
    tagged = ~oracle.realizable_cells(g, Un)
    assert tagged.any()
    new, passes = tagged.copy(), 0
    while new.any() and passes < 4:
        Un = oracle.step_pass(g, U, dt, tagged)
        new = ~oracle.realizable_cells(g, Un) & ~tagged
        tagged |= new
        passes += 1
    np.testing.assert_array_equal(Un, oracle.step(g, U, dt))
    np.testing.assert_array_equal(oracle.step_pass(g, U, dt), oracle.step_second_order_only(g, U, dt))


def test_fallback_inactive_on_smooth_data(oracle):
    """Where the second-order update is realizable the fallback changes nothing."""
    p = I.blast(n=24, nsteps=1)
    g = grid_of(oracle, p)
    U = oracle.prim_to_cons(p.W)
    dt = oracle.cfl_dt(g, U)
    np.testing.assert_array_equal(oracle.step(g, U, dt), oracle.step_second_order_only(g, U, dt))
