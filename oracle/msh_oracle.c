/*
 * msh_oracle.c -- plain, slow, FP64 reference ("oracle") for one Godunov step of
 * the ten-moment collisionless Boltzmann moment equations (BME) of Mitchell,
 * Vorobyov & Hensler, "Collisionless stellar hydrodynamics as an efficient
 * alternative to N-body methods" (arXiv:1210.5246).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path shares no code, header or constant with it.
 *
 * The step follows the paper's order:
 *   a1  ghost fill                           (guardcells, Sec. 3.1)
 *   a2  conserved -> primitive               (primitive form W, Sec. 3.3)
 *   a3  slopes dw_L, dw_C, dw_R and characteristic projection du = L dw
 *                                             (Sec. 3.3, slope and projection eqs)
 *   a4  MC limiter, back-projection dw^m = R du^m (Sec. 3.3, TVD constraint)
 *   a5  Hancock face states: Stone (2008) eqs 40-45 summed over all waves,
 *       which for the HLL family is w +- dw^m/2 - (dt/2dx) A dw^m (Sec. 3.3)
 *   a6  HLL Riemann flux with the fast eigenvalue as signal speed (Sec. 3.3)
 *   a7  unsplit conservative update (MUSCL-Hancock unsplit, Sec. 3.3)
 *   a8  gravity source after the hydro step (operator splitting, Sec. 3.3
 *       last paragraph; sources of eqs contin/moment/dispers, Sec. 2)
 *   a9  CFL time step from the wave speeds a = sqrt(3 P_dd / rho) (Sec. 3.2/3.3)
 *   a10 FP64 conserved totals and realizability (rho > 0, P SPD)
 *
 * Other schemes of the paper, selected by og_grid.scheme: the Kurganov-Tadmor central
 * scheme with second-order Runge-Kutta (Sec. 3.2, og_step_kt); the characteristic step with
 * upwind tracing (eqs 40-43, og_reconstruct_upwind) and a Roe-type flux (og_roe); the
 * characteristic step with the Hancock predictor and an HLLC flux (og_hllc).
 *
 * Readings where the paper is silent or garbled:
 *   - full ten-moment system (the paper prints only the diagonal 7-variable case);
 *   - the ten-moment Jacobian / eigenvectors derived from eqs contin/moment/dispers
 *     with zero heat flux (the printed 7x7 Jacobian misses rho in row 1 and the
 *     P_yy u', P_zz u' couplings);
 *   - limiter returns 0 when dw_L * dw_R <= 0;
 *   - face state fallback: if a Hancock face state of a cell has rho <= 0 or
 *     P_nn <= 0, both face states of that cell in that direction revert to W_i;
 *   - a-posteriori fallback: cells whose second-order update is not realizable get
 *     first-order face states on all their faces and the step is recomputed; cells
 *     still failing join the tagged set and the step is recomputed again (at most
 *     OG_FALLBACK_PASSES passes);
 *   - CFL: dt = C / max_cells sum_d (|u_d| + sqrt(3 P_dd/rho)) / dx_d;
 *   - gravity: a = -grad(Phi) by central differences, m += dt rho a,
 *     E += dt (mbar a^T + a mbar^T) with mbar the mean of m before/after;
 *   - Roe-type and HLLC fluxes: faces with first-order states in a fallback pass take HLL.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 10
/* maximum number of a-posteriori fallback passes per step */
#define OG_FALLBACK_PASSES 4
/* conserved order: rho, m_x, m_y, m_z, E_xx, E_xy, E_xz, E_yy, E_yz, E_zz
 * primitive order: rho, u_x, u_y, u_z, P_xx, P_xy, P_xz, P_yy, P_yz, P_zz   */

typedef struct {
    int32_t ndim;        /* 1, 2 or 3 */
    int32_t pad0;
    int64_t n[3];        /* cells per dimension, n[d] = 1 for unused d */
    double dx[3];        /* cell widths */
    int32_t bc[6];       /* bc[2d+0] lower face, bc[2d+1] upper face: 0 periodic, 1 outflow, 2 reflect */
    double cfl;
    int32_t scheme;      /* OG_SCHEME_MH (Sec. 3.3, HLL), OG_SCHEME_KT (Sec. 3.2),
                            OG_SCHEME_MH_ROE (Sec. 3.3, Roe-type flux, eqs 40-43 tracing) or
                            OG_SCHEME_MH_HLLC (Sec. 3.3, HLLC flux, eqs 40-45 tracing) */
    int32_t ctu;         /* characteristic schemes: 1 adds the transverse terms to the face
                            states and takes the max-form CFL rule (og_transverse) */
} og_grid;

enum { OG_PERIODIC = 0, OG_OUTFLOW = 1, OG_REFLECT = 2 };
enum { OG_SCHEME_MH = 0, OG_SCHEME_KT = 1, OG_SCHEME_MH_ROE = 2, OG_SCHEME_MH_HLLC = 3 };

/* index of the symmetric tensor component (i,j) inside the 10-vector */
static int tens_idx(int i, int j)
{
    static const int t[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
    return t[i][j];
}

/* ---------------------------------------------------------------- a2 ----- */
/* E_ij = P_ij + rho u_i u_j  (Sec. 2, definition below eq dispers) */
static void cons_to_prim(const double *U, double *W)
{
    double rho = U[0];
    W[0] = rho;
    for (int i = 0; i < 3; i++) W[1 + i] = U[1 + i] / rho;
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++)
            W[tens_idx(i, j)] = U[tens_idx(i, j)] - rho * W[1 + i] * W[1 + j];
}

static void prim_to_cons(const double *W, double *U)
{
    double rho = W[0];
    U[0] = rho;
    for (int i = 0; i < 3; i++) U[1 + i] = rho * W[1 + i];
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++)
            U[tens_idx(i, j)] = W[tens_idx(i, j)] + rho * W[1 + i] * W[1 + j];
}

/* Physical flux along direction d (eqs contin, moment, dispers with Q_ijk = 0):
 *   rho u_d ;  rho u_i u_d + P_id ;  E_ij u_d + P_id u_j + P_jd u_i            */
void og_flux(const double *W, int d, double *F)
{
    double U[NV];
    prim_to_cons(W, U);
    double rho = W[0];
    const double *u = W + 1;
    F[0] = rho * u[d];
    for (int i = 0; i < 3; i++) F[1 + i] = rho * u[i] * u[d] + W[tens_idx(i, d)];
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++)
            F[tens_idx(i, j)] = U[tens_idx(i, j)] * u[d] + W[tens_idx(i, d)] * u[j] +
                                W[tens_idx(j, d)] * u[i];
}

/* ------------------------------------------------ eigen-system, x-normal ---- */
/* Local frame for direction d: the normal axis becomes "x".  perm[d][k] gives
 * the global primitive component that sits at local position k.  Transverse
 * axes keep their natural order: d=y -> (y, x, z), d=z -> (z, x, y).          */
static const int perm[3][NV] = {
    {0, 1, 2, 3, 4, 5, 6, 7, 8, 9},
    {0, 2, 1, 3, 7, 5, 8, 4, 6, 9},
    {0, 3, 1, 2, 9, 6, 8, 4, 5, 7},
};

/* Quasi-linear primitive Jacobian A_x(W):  W_t + A_x W_x = 0, derived from the
 * ten moment equations with zero heat flux (the 10-variable extension of the
 * paper's eq jacobian).  Row order = primitive order.                          */
void og_jacobian_x(const double *W, double A[NV][NV])
{
    double rho = W[0], u = W[1];
    double Pxx = W[4], Pxy = W[5], Pxz = W[6], Pyy = W[7], Pyz = W[8], Pzz = W[9];
    memset(A, 0, sizeof(double) * NV * NV);
    for (int k = 0; k < NV; k++) A[k][k] = u;
    A[0][1] = rho;                      /* rho_t + u rho_x + rho u_x */
    A[1][4] = 1.0 / rho;                /* u_t + u u_x + Pxx_x / rho */
    A[2][5] = 1.0 / rho;                /* v_t + u v_x + Pxy_x / rho */
    A[3][6] = 1.0 / rho;                /* w_t + u w_x + Pxz_x / rho */
    A[4][1] = 3.0 * Pxx;                /* Pxx_t + u Pxx_x + 3 Pxx u_x */
    A[5][1] = 2.0 * Pxy; A[5][2] = Pxx; /* Pxy: 2 Pxy u_x + Pxx v_x */
    A[6][1] = 2.0 * Pxz; A[6][3] = Pxx; /* Pxz: 2 Pxz u_x + Pxx w_x */
    A[7][1] = Pyy; A[7][2] = 2.0 * Pxy; /* Pyy: Pyy u_x + 2 Pxy v_x */
    A[8][1] = Pyz; A[8][2] = Pxz; A[8][3] = Pxy; /* Pyz */
    A[9][1] = Pzz; A[9][3] = 2.0 * Pxz; /* Pzz: Pzz u_x + 2 Pxz w_x */
}

/* Eigenvalues in wave order: fast-, shear_y-, shear_z-, contact rho, contact yy,
 * contact yz, contact zz, shear_y+, shear_z+, fast+   (eq eigenvalues extended). */
void og_eigenvalues_x(const double *W, double lam[NV])
{
    double u = W[1];
    double cf = sqrt(3.0 * W[4] / W[0]);
    double cs = sqrt(W[4] / W[0]);
    lam[0] = u - cf;
    lam[1] = u - cs; lam[2] = u - cs;
    lam[3] = u; lam[4] = u; lam[5] = u; lam[6] = u;
    lam[7] = u + cs; lam[8] = u + cs;
    lam[9] = u + cf;
}

/* Right eigenvectors as columns R[:,k] (10-variable extension of eq righteigvec). */
void og_right_x(const double *W, double R[NV][NV])
{
    double rho = W[0];
    double Pxx = W[4], Pxy = W[5], Pxz = W[6], Pyy = W[7], Pyz = W[8], Pzz = W[9];
    double cf = sqrt(3.0 * Pxx / rho), cs = sqrt(Pxx / rho);
    memset(R, 0, sizeof(double) * NV * NV);
    for (int sgn = -1; sgn <= 1; sgn += 2) {
        int kf = (sgn < 0) ? 0 : 9;      /* fast wave, s = +-cf */
        double s = sgn * cf;
        R[0][kf] = rho;
        R[1][kf] = s;
        R[2][kf] = s * Pxy / Pxx;
        R[3][kf] = s * Pxz / Pxx;
        R[4][kf] = 3.0 * Pxx;
        R[5][kf] = 3.0 * Pxy;
        R[6][kf] = 3.0 * Pxz;
        R[7][kf] = Pyy + 2.0 * Pxy * Pxy / Pxx;
        R[8][kf] = Pyz + 2.0 * Pxy * Pxz / Pxx;
        R[9][kf] = Pzz + 2.0 * Pxz * Pxz / Pxx;
        int kv = (sgn < 0) ? 1 : 7;      /* shear wave in v, s = +-cs */
        int kw = (sgn < 0) ? 2 : 8;      /* shear wave in w */
        double c = sgn * cs;
        R[2][kv] = c; R[5][kv] = Pxx; R[7][kv] = 2.0 * Pxy; R[8][kv] = Pxz;
        R[3][kw] = c; R[6][kw] = Pxx; R[8][kw] = Pxy; R[9][kw] = 2.0 * Pxz;
    }
    R[0][3] = 1.0;  /* contact: density      */
    R[7][4] = 1.0;  /* contact: P_yy          */
    R[8][5] = 1.0;  /* contact: P_yz          */
    R[9][6] = 1.0;  /* contact: P_zz          */
}

/* Left eigenvectors as rows L[k,:], L R = I (10-variable extension of eq lefteigvec). */
void og_left_x(const double *W, double L[NV][NV])
{
    double rho = W[0];
    double Pxx = W[4], Pxy = W[5], Pxz = W[6], Pyy = W[7], Pyz = W[8], Pzz = W[9];
    double cf = sqrt(3.0 * Pxx / rho), cs = sqrt(Pxx / rho);
    memset(L, 0, sizeof(double) * NV * NV);
    for (int sgn = -1; sgn <= 1; sgn += 2) {
        int kf = (sgn < 0) ? 0 : 9;
        double s = sgn * cf;
        L[kf][1] = 1.0 / (2.0 * s);
        L[kf][4] = 1.0 / (6.0 * Pxx);
        int kv = (sgn < 0) ? 1 : 7;
        int kw = (sgn < 0) ? 2 : 8;
        double c = sgn * cs;
        L[kv][1] = -Pxy / (2.0 * c * Pxx);
        L[kv][2] = 1.0 / (2.0 * c);
        L[kv][4] = -Pxy / (2.0 * Pxx * Pxx);
        L[kv][5] = 1.0 / (2.0 * Pxx);
        L[kw][1] = -Pxz / (2.0 * c * Pxx);
        L[kw][3] = 1.0 / (2.0 * c);
        L[kw][4] = -Pxz / (2.0 * Pxx * Pxx);
        L[kw][6] = 1.0 / (2.0 * Pxx);
    }
    L[3][0] = 1.0;
    L[3][4] = -rho / (3.0 * Pxx);
    L[4][4] = (4.0 * Pxy * Pxy / Pxx - Pyy) / (3.0 * Pxx);
    L[4][5] = -2.0 * Pxy / Pxx;
    L[4][7] = 1.0;
    L[5][4] = (4.0 * Pxy * Pxz / Pxx - Pyz) / (3.0 * Pxx);
    L[5][5] = -Pxz / Pxx;
    L[5][6] = -Pxy / Pxx;
    L[5][8] = 1.0;
    L[6][4] = (4.0 * Pxz * Pxz / Pxx - Pzz) / (3.0 * Pxx);
    L[6][6] = -2.0 * Pxz / Pxx;
    L[6][9] = 1.0;
}

static void matvec(double M[NV][NV], const double *x, double *y)
{
    for (int i = 0; i < NV; i++) {
        double s = 0.0;
        for (int j = 0; j < NV; j++) s += M[i][j] * x[j];
        y[i] = s;
    }
}

/* ---------------------------------------------------------------- a4 ----- */
/* Monotonised-central limiter on one characteristic component. */
static double mc_limit(double dL, double dC, double dR)
{
    if (dL * dR <= 0.0) return 0.0;
    double m = fmin(2.0 * fabs(dL), fmin(fabs(dC), 2.0 * fabs(dR)));
    return (dC > 0.0) ? m : -m;
}

/* ------------------------------------------------------------- a3 - a5 ---- */
/* Reconstruction of cell i along direction d from its neighbours Wm, W0, Wp
 * (global primitive order).  dtdx = dt/dx_d.  Writes the face states at i-1/2
 * (lo) and i+1/2 (hi) in global primitive order.                             */
static void hancock_states(const double *Wm, const double *W0, const double *Wp, int d,
                           double dtdx, double *lo, double *hi)
{
    const int *p = perm[d];
    double w0[NV], dwL[NV], dwC[NV], dwR[NV];
    for (int k = 0; k < NV; k++) {
        w0[k] = W0[p[k]];
        dwL[k] = W0[p[k]] - Wm[p[k]];              /* dw_L = w_i - w_{i-1}       */
        dwC[k] = 0.5 * (Wp[p[k]] - Wm[p[k]]);      /* dw_C = (w_{i+1}-w_{i-1})/2 */
        dwR[k] = Wp[p[k]] - W0[p[k]];              /* dw_R = w_{i+1} - w_i       */
    }
    double L[NV][NV], R[NV][NV], A[NV][NV];
    og_left_x(w0, L);
    og_right_x(w0, R);
    og_jacobian_x(w0, A);
    double daL[NV], daC[NV], daR[NV], dam[NV], dwm[NV], Adw[NV];
    matvec(L, dwL, daL);
    matvec(L, dwC, daC);
    matvec(L, dwR, daR);
    for (int k = 0; k < NV; k++) dam[k] = mc_limit(daL[k], daC[k], daR[k]);
    matvec(R, dam, dwm);
    matvec(A, dwm, Adw);
    for (int k = 0; k < NV; k++) {
        hi[p[k]] = w0[k] + 0.5 * dwm[k] - 0.5 * dtdx * Adw[k];
        lo[p[k]] = w0[k] - 0.5 * dwm[k] - 0.5 * dtdx * Adw[k];
    }
}

/* face-state fallback (reading): revert to first order if a face state along d has
 * non-positive density or non-positive normal dispersion */
static void face_state_check(const double *W0, int d, double *lo, double *hi)
{
    int nn = tens_idx(d, d);
    if (!(hi[0] > 0.0 && lo[0] > 0.0 && hi[nn] > 0.0 && lo[nn] > 0.0)) {
        for (int k = 0; k < NV; k++) hi[k] = lo[k] = W0[k];
    }
}

void og_reconstruct(const double *Wm, const double *W0, const double *Wp, int d,
                    double dtdx, double *lo, double *hi)
{
    hancock_states(Wm, W0, Wp, d, dtdx, lo, hi);
    face_state_check(W0, d, lo, hi);
}

/* Transverse term of a cell along direction t for the corner-transport-upwind form of the
 * unsplit step (the data reconstruction of Lee & Deane 2009, which FLASH's unsplit
 * MUSCL-Hancock solver used by Sec. 3.3 follows; the paper prints none of it): the
 * quasi-linear transverse derivative -(dt/2) A_t dW/dx_t taken wave by wave from the
 * upwind side,
 *   T_t = -(dt / (2 dx_t)) sum_a lam^a (L^a . dW^a) R^a,
 *   dW^a = W_i - W_{i-e_t} if lam^a > 0, W_{i+e_t} - W_i otherwise,
 * with the eigen-system of cell i along t.  The face states along d then take
 * sum_{t != d} T_t before the face-state check.  dtdx = dt / dx_t. */
void og_transverse(const double *Wm, const double *W0, const double *Wp, int t, double dtdx, double *T)
{
    const int *p = perm[t];
    double w0[NV], dL[NV], dR[NV];
    for (int k = 0; k < NV; k++) {
        w0[k] = W0[p[k]];
        dL[k] = W0[p[k]] - Wm[p[k]];
        dR[k] = Wp[p[k]] - W0[p[k]];
    }
    double L[NV][NV], R[NV][NV], lam[NV], aL[NV], aR[NV], c[NV], o[NV];
    og_left_x(w0, L);
    og_right_x(w0, R);
    og_eigenvalues_x(w0, lam);
    matvec(L, dL, aL);
    matvec(L, dR, aR);
    for (int a = 0; a < NV; a++) c[a] = lam[a] * (lam[a] > 0.0 ? aL[a] : aR[a]);
    matvec(R, c, o);
    for (int k = 0; k < NV; k++) T[p[k]] = -0.5 * dtdx * o[k];
}

/* Characteristic tracing for a Riemann solver that resolves every wave (Sec. 3.3, eqs 40-43;
 * Colella 1990, Stone et al. 2008): the limited slope dw^m as in og_reconstruct; reference
 * states traced with the fastest wave towards each face,
 *   wt_L(i+1/2) = w + [1/2 - max(lam^M, 0) dt/(2dx)] dw^m                          (eq 40)
 *   wt_R(i-1/2) = w - [1/2 + min(lam^0, 0) dt/(2dx)] dw^m                          (eq 41)
 * (eq 41 read in the mirror form of eq 40: the printed -max(lam^0, 0) leaves the reference
 * state untraced whenever lam^0 < 0), then every wave that reaches the face within dt/2
 * corrected from the reference speed to its own,
 *   w_L = wt_L + dt/(2dx) sum_{lam^a > 0} (lam^M - lam^a) (L^a . dw^m) R^a           (eq 42)
 *   w_R = wt_R + dt/(2dx) sum_{lam^a < 0} (lam^0 - lam^a) (L^a . dw^m) R^a           (eq 43)
 * lam^M, lam^0 the largest and smallest eigenvalues of cell i; L^a the rows of L, R^a the
 * columns of R.  No eq 44-45 terms (those belong to HLL).  Face-state fallback as in
 * og_reconstruct (og_reconstruct_upwind). */
static void upwind_states(const double *Wm, const double *W0, const double *Wp, int d,
                          double dtdx, double *lo, double *hi)
{
    const int *p = perm[d];
    double w0[NV], dwL[NV], dwC[NV], dwR[NV];
    for (int k = 0; k < NV; k++) {
        w0[k] = W0[p[k]];
        dwL[k] = W0[p[k]] - Wm[p[k]];
        dwC[k] = 0.5 * (Wp[p[k]] - Wm[p[k]]);
        dwR[k] = Wp[p[k]] - W0[p[k]];
    }
    double L[NV][NV], R[NV][NV], lam[NV];
    og_left_x(w0, L);
    og_right_x(w0, R);
    og_eigenvalues_x(w0, lam);
    double daL[NV], daC[NV], daR[NV], dam[NV], dwm[NV];
    matvec(L, dwL, daL);
    matvec(L, dwC, daC);
    matvec(L, dwR, daR);
    for (int k = 0; k < NV; k++) dam[k] = mc_limit(daL[k], daC[k], daR[k]);
    matvec(R, dam, dwm);
    double lmax = lam[0], lmin = lam[0];
    for (int k = 1; k < NV; k++) {
        lmax = fmax(lmax, lam[k]);
        lmin = fmin(lmin, lam[k]);
    }
    double hi_l[NV], lo_l[NV];
    const double h = 0.5 * dtdx;
    for (int k = 0; k < NV; k++) {
        hi_l[k] = w0[k] + (0.5 - fmax(lmax, 0.0) * h) * dwm[k];                   /* eq 40 */
        lo_l[k] = w0[k] - (0.5 + fmin(lmin, 0.0) * h) * dwm[k];                   /* eq 41 */
    }
    for (int a = 0; a < NV; a++) {
        double la = 0.0; /* L^a . dw^m */
        for (int k = 0; k < NV; k++) la += L[a][k] * dwm[k];
        if (lam[a] > 0.0)
            for (int k = 0; k < NV; k++) hi_l[k] += h * (lmax - lam[a]) * la * R[k][a];   /* eq 42 */
        if (lam[a] < 0.0)
            for (int k = 0; k < NV; k++) lo_l[k] += h * (lmin - lam[a]) * la * R[k][a];   /* eq 43 */
    }
    for (int k = 0; k < NV; k++) {
        lo[p[k]] = lo_l[k];
        hi[p[k]] = hi_l[k];
    }
}

void og_reconstruct_upwind(const double *Wm, const double *W0, const double *Wp, int d,
                           double dtdx, double *lo, double *hi)
{
    upwind_states(Wm, W0, Wp, d, dtdx, lo, hi);
    face_state_check(W0, d, lo, hi);
}

/* ---------------------------------------------------------------- a6 ----- */
/* HLL flux along direction d between face states WL (left) and WR (right). */
void og_hll(const double *WL, const double *WR, int d, double *F)
{
    double FL[NV], FR[NV], UL[NV], UR[NV];
    og_flux(WL, d, FL);
    og_flux(WR, d, FR);
    prim_to_cons(WL, UL);
    prim_to_cons(WR, UR);
    int nn = tens_idx(d, d);
    double cL = sqrt(3.0 * WL[nn] / WL[0]);
    double cR = sqrt(3.0 * WR[nn] / WR[0]);
    double SL = fmin(WL[1 + d] - cL, WR[1 + d] - cR);
    double SR = fmax(WL[1 + d] + cL, WR[1 + d] + cR);
    if (SL >= 0.0) {
        for (int k = 0; k < NV; k++) F[k] = FL[k];
    } else if (SR <= 0.0) {
        for (int k = 0; k < NV; k++) F[k] = FR[k];
    } else {
        for (int k = 0; k < NV; k++)
            F[k] = (SR * FL[k] - SL * FR[k] + SL * SR * (UR[k] - UL[k])) / (SR - SL);
    }
}

/* ------------------------------------------------------ Roe-type flux ---- */
/* Linearised characteristic upwind flux (Roe 1981) through a face normal to d:
 *   F = (f(WL) + f(WR)) / 2 - (1/2) (dU/dW)(Wm) R(Wm) |Lambda(Wm)| L(Wm) (WR - WL),
 * with the eigen-system of the local frame (og_left_x, og_right_x, og_eigenvalues_x).
 * Readings (no Roe average is known for the ten-moment system): Wm = (WL + WR) / 2, the
 * primitive jump in place of (dW/dU)(UR - UL), and Harten's entropy fix on the two fast
 * (genuinely nonlinear) waves: |lambda| -> (lambda^2 + delta^2) / (2 delta) where
 * |lambda| < delta = 0.1 cf(Wm).  The shear and contact waves are linearly degenerate and
 * keep |lambda|, so a stationary contact gets no dissipation.                           */
void og_roe(const double *WL, const double *WR, int d, double *F)
{
    const int *p = perm[d];
    double wm[NV], dw[NV];
    for (int k = 0; k < NV; k++) {
        wm[k] = 0.5 * (WL[p[k]] + WR[p[k]]);
        dw[k] = WR[p[k]] - WL[p[k]];
    }
    double L[NV][NV], R[NV][NV], lam[NV], a[NV], dd[NV];
    og_left_x(wm, L);
    og_right_x(wm, R);
    og_eigenvalues_x(wm, lam);
    matvec(L, dw, a);
    double delta = 0.1 * sqrt(3.0 * wm[4] / wm[0]);
    for (int k = 0; k < NV; k++) {
        double al = fabs(lam[k]);
        if ((k == 0 || k == NV - 1) && al < delta) al = (lam[k] * lam[k] + delta * delta) / (2.0 * delta);
        a[k] *= al;
    }
    matvec(R, a, dd);
    /* back to the global order, then through the Jacobian of prim_to_cons at Wm */
    double Wg[NV], Dg[NV];
    for (int k = 0; k < NV; k++) {
        Wg[p[k]] = wm[k];
        Dg[p[k]] = dd[k];
    }
    double dU[NV];
    dU[0] = Dg[0];
    for (int i = 0; i < 3; i++) dU[1 + i] = Wg[0] * Dg[1 + i] + Wg[1 + i] * Dg[0];
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++)
            dU[tens_idx(i, j)] = Dg[tens_idx(i, j)] + Dg[0] * Wg[1 + i] * Wg[1 + j] +
                                 Wg[0] * (Dg[1 + i] * Wg[1 + j] + Wg[1 + i] * Dg[1 + j]);
    double FL[NV], FR[NV];
    og_flux(WL, d, FL);
    og_flux(WR, d, FR);
    for (int k = 0; k < NV; k++) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * dU[k];
}

/* ------------------------------------------------------------- HLLC ---- */
/* Three-wave HLLC flux (Toro, Spruce & Speares 1994; Batten et al. 1997) for the ten-moment
 * system through a face normal to d.  The flux is F = u_d U + Pi with
 *   Pi = (0; P_id; P_id u_j + P_jd u_i),
 * and Pi depends only on u and on the stresses P_id on the face, the quantities that are
 * continuous across the contact wave (rho, P_tt' jump there).  Readings: the outer waves
 * S_L, S_R are HLL's (Davis speeds from the fast eigenvalue) and carry the fast and shear
 * waves together; the middle wave is the contact S_M.  The star values of every pair
 * (u_i, P_id) are common to both star states and follow from the momentum jump
 * conditions across S_L and S_R, u*_i = u_i,K + (P*_id - P_id,K) / C_K with
 * C_K = rho_K (S_K - u_d,K):
 *   P*_id = (C_L C_R (u_i,R - u_i,L) + C_R P_id,L - C_L P_id,R) / (C_R - C_L),
 * for i = d the usual contact speed S_M = u*_d and normal stress.  Each star state then
 * follows from the jump conditions across its outer wave,
 *   U*_K = (U_K (S_K - u_d,K) + Pi* - Pi_K) / (S_K - S_M),
 * so that (S_M - S_L) U*_L + (S_R - S_M) U*_R equals (S_R - S_L) times the HLL state and
 * the two star fluxes satisfy the contact's jump condition.  With diagonal stresses and no
 * transverse velocity jump this is the gamma = 3 HLLC of gas dynamics (E_dd / 2 as the
 * energy); an isolated contact is resolved exactly.  Where S_M is not strictly inside
 * (S_L, S_R) the flux is HLL's.  Returns 1 if the star states were formed, 0 otherwise. */
int og_hllc_star(const double *WL, const double *WR, int d, double *UsL, double *UsR, double *S)
{
    int nn = tens_idx(d, d);
    double cL = sqrt(3.0 * WL[nn] / WL[0]);
    double cR = sqrt(3.0 * WR[nn] / WR[0]);
    double SL = fmin(WL[1 + d] - cL, WR[1 + d] - cR);
    double SR = fmax(WL[1 + d] + cL, WR[1 + d] + cR);
    double CL = WL[0] * (SL - WL[1 + d]), CR = WR[0] * (SR - WR[1 + d]);
    double us[3], Ps[3]; /* star u_i and P_id */
    for (int i = 0; i < 3; i++) {
        int id = tens_idx(i, d);
        Ps[i] = (CL * CR * (WR[1 + i] - WL[1 + i]) + CR * WL[id] - CL * WR[id]) / (CR - CL);
        us[i] = WL[1 + i] + (Ps[i] - WL[id]) / CL;
    }
    double SM = us[d];
    S[0] = SL; S[1] = SM; S[2] = SR;
    if (!(SL < SM && SM < SR)) return 0;
    /* Pi at the star values and at each side */
    double Pis[NV], PiL[NV], PiR[NV];
    const double *W2[2] = {WL, WR};
    double *Pi2[2] = {PiL, PiR};
    for (int side = 0; side < 3; side++) {
        double *Pi = side < 2 ? Pi2[side] : Pis;
        double u[3], Pd[3];
        for (int i = 0; i < 3; i++) {
            u[i] = side < 2 ? W2[side][1 + i] : us[i];
            Pd[i] = side < 2 ? W2[side][tens_idx(i, d)] : Ps[i];
        }
        Pi[0] = 0.0;
        for (int i = 0; i < 3; i++) Pi[1 + i] = Pd[i];
        for (int i = 0; i < 3; i++)
            for (int j = i; j < 3; j++) Pi[tens_idx(i, j)] = Pd[i] * u[j] + Pd[j] * u[i];
    }
    double UL[NV], UR[NV];
    prim_to_cons(WL, UL);
    prim_to_cons(WR, UR);
    for (int k = 0; k < NV; k++) {
        UsL[k] = (UL[k] * (SL - WL[1 + d]) + Pis[k] - PiL[k]) / (SL - SM);
        UsR[k] = (UR[k] * (SR - WR[1 + d]) + Pis[k] - PiR[k]) / (SR - SM);
    }
    return 1;
}

void og_hllc(const double *WL, const double *WR, int d, double *F)
{
    double UsL[NV], UsR[NV], S[3], UL[NV], UR[NV], FL[NV], FR[NV];
    if (!og_hllc_star(WL, WR, d, UsL, UsR, S)) {
        og_hll(WL, WR, d, F);
        return;
    }
    og_flux(WL, d, FL);
    og_flux(WR, d, FR);
    prim_to_cons(WL, UL);
    prim_to_cons(WR, UR);
    if (S[0] >= 0.0) {
        for (int k = 0; k < NV; k++) F[k] = FL[k];
    } else if (S[2] <= 0.0) {
        for (int k = 0; k < NV; k++) F[k] = FR[k];
    } else if (S[1] >= 0.0) {
        for (int k = 0; k < NV; k++) F[k] = FL[k] + S[0] * (UsL[k] - UL[k]);
    } else {
        for (int k = 0; k < NV; k++) F[k] = FR[k] + S[2] * (UsR[k] - UR[k]);
    }
}

/* Face flux of the characteristic scheme: HLL (the hot path), the Roe-type or the HLLC flux.  A
 * face with first-order states in a fallback pass (first != 0) takes HLL in all three: the
 * fallback has to make the update realizable, and a linearised Roe flux is not positively
 * conservative (Einfeldt, Munz, Roe & Sjogreen 1991) where HLL with bounding wave speeds
 * is; HLLC's star states, formed from the jump conditions, need not be realizable either. */
static void face_flux(const og_grid *Gr, const double *WL, const double *WR, int d, int first, double *F)
{
    if (Gr->scheme == OG_SCHEME_MH_ROE && !first) og_roe(WL, WR, d, F);
    else if (Gr->scheme == OG_SCHEME_MH_HLLC && !first) og_hllc(WL, WR, d, F);
    else og_hll(WL, WR, d, F);
}

/* ---------------------------------------------------------------- a1 ----- */
/* Padded array layout: [NV][pz][py][px] with 2 ghost layers on active dims. */
typedef struct {
    int64_t n[3], g[3], p[3];
} og_pad;

static og_pad make_pad(const og_grid *G)
{
    og_pad P;
    for (int d = 0; d < 3; d++) {
        P.n[d] = G->n[d];
        P.g[d] = (d < G->ndim) ? 2 : 0;
        P.p[d] = P.n[d] + 2 * P.g[d];
    }
    return P;
}

static inline int64_t pidx(const og_pad *P, int64_t x, int64_t y, int64_t z)
{
    return ((z + P->g[2]) * P->p[1] + (y + P->g[1])) * P->p[0] + (x + P->g[0]);
}

/* source cell of ghost index i along a dimension of n cells, and whether the
 * copy is mirrored (reflect boundary) */
static int64_t ghost_src(int64_t i, int64_t n, int bclo, int bchi, int *mirror)
{
    *mirror = 0;
    if (i < 0) {
        if (bclo == OG_PERIODIC) return i + n;
        if (bclo == OG_OUTFLOW) return 0;
        *mirror = 1;
        return -1 - i;
    }
    if (i >= n) {
        if (bchi == OG_PERIODIC) return i - n;
        if (bchi == OG_OUTFLOW) return n - 1;
        *mirror = 1;
        return 2 * n - 1 - i;
    }
    return i;
}

/* Fill the padded conserved array G (NV * p0*p1*p2) from U ([NV][nz][ny][nx]).
 * Reflect negates m_d and E_dt (t != d) of the mirrored copy.               */
void og_ghost_fill(const og_grid *Gr, const double *U, double *G)
{
    og_pad P = make_pad(Gr);
    int64_t N = P.n[0] * P.n[1] * P.n[2];
    int64_t NP = P.p[0] * P.p[1] * P.p[2];
    for (int64_t z = -P.g[2]; z < P.n[2] + P.g[2]; z++)
        for (int64_t y = -P.g[1]; y < P.n[1] + P.g[1]; y++)
            for (int64_t x = -P.g[0]; x < P.n[0] + P.g[0]; x++) {
                int64_t c[3] = {x, y, z}, s[3];
                int mir[3];
                for (int d = 0; d < 3; d++)
                    s[d] = ghost_src(c[d], P.n[d], Gr->bc[2 * d], Gr->bc[2 * d + 1], &mir[d]);
                int64_t src = (s[2] * P.n[1] + s[1]) * P.n[0] + s[0];
                int64_t dst = pidx(&P, x, y, z);
                for (int k = 0; k < NV; k++) {
                    double v = U[k * N + src];
                    for (int d = 0; d < 3; d++) {
                        if (!mir[d]) continue;
                        if (k == 1 + d) v = -v;                          /* m_d   */
                        for (int t = 0; t < 3; t++)
                            if (t != d && k == tens_idx(d, t)) v = -v;   /* E_dt  */
                    }
                    G[k * NP + dst] = v;
                }
            }
}

/* ---------------------------------------------------------------- a9 ----- */
double og_cfl_dt(const og_grid *G, const double *U)
{
    int64_t N = G->n[0] * G->n[1] * G->n[2];
    double smax = 0.0;
#pragma omp parallel for reduction(max : smax)
    for (int64_t c = 0; c < N; c++) {
        double Uc[NV], W[NV];
        for (int k = 0; k < NV; k++) Uc[k] = U[k * N + c];
        cons_to_prim(Uc, W);
        double s = 0.0;
        for (int d = 0; d < G->ndim; d++) {
            double sd = (fabs(W[1 + d]) + sqrt(3.0 * W[tens_idx(d, d)] / W[0])) / G->dx[d];
            s = G->ctu ? fmax(s, sd) : s + sd; /* CTU: max over directions, else the sum */
        }
        if (s > smax) smax = s;
    }
    return G->cfl / smax;
}

/* Realizability of one conserved state: rho > 0 and P positive definite. */
static int cell_realizable(const double *Uc)
{
    if (!(Uc[0] > 0.0)) return 0;
    double W[NV];
    cons_to_prim(Uc, W);
    double m1 = W[4];
    double m2 = W[4] * W[7] - W[5] * W[5];
    double m3 = W[4] * (W[7] * W[9] - W[8] * W[8]) - W[5] * (W[5] * W[9] - W[8] * W[6]) +
                W[6] * (W[5] * W[8] - W[7] * W[6]);
    return m1 > 0.0 && m2 > 0.0 && m3 > 0.0;
}

/* ---------------------------------------------------------------- a8 ----- */
/* Gravity source on the updated state Us of cell c: a = -grad Phi by central
 * differences of the potential (one ghost layer on active dims), m += dt rho a,
 * E += dt (mbar a^T + a mbar^T) with mbar the mean of m before and after. */
static void gravity_source(const og_grid *Gr, const double *phi, double dt, int64_t c, double *Us)
{
    int64_t n0 = Gr->n[0], n1 = Gr->n[1];
    int64_t gx = (Gr->ndim > 0), gy = (Gr->ndim > 1), gz = (Gr->ndim > 2);
    int64_t px = n0 + 2 * gx, py = n1 + 2 * gy;
    int64_t x = c % n0, y = (c / n0) % n1, z = c / (n0 * n1);
    double a[3] = {0.0, 0.0, 0.0};
    int64_t ctr = ((z + gz) * py + (y + gy)) * px + (x + gx);
    int64_t stride[3] = {1, px, px * py};
    for (int d = 0; d < Gr->ndim; d++)
        a[d] = -(phi[ctr + stride[d]] - phi[ctr - stride[d]]) / (2.0 * Gr->dx[d]);
    double m_star[3], m_new[3], mbar[3];
    for (int i = 0; i < 3; i++) {
        m_star[i] = Us[1 + i];
        m_new[i] = m_star[i] + dt * Us[0] * a[i];
        mbar[i] = 0.5 * (m_star[i] + m_new[i]);
    }
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++)
            Us[tens_idx(i, j)] += dt * (mbar[i] * a[j] + a[i] * mbar[j]);
    for (int i = 0; i < 3; i++) Us[1 + i] = m_new[i];
}

/* -------------------------------------------------------------- a1 - a8 --- */
/* One pass of the step.  flag: NULL, or per padded cell 1 where the faces of that
 * cell take first-order face states (the cell-centred W on both sides). */
static int step_pass(const og_grid *Gr, const double *U, const double *phi, double dt,
                     const unsigned char *flag, double *Unew)
{
    og_pad P = make_pad(Gr);
    int64_t N = P.n[0] * P.n[1] * P.n[2];
    int64_t NP = P.p[0] * P.p[1] * P.p[2];
    double *G = (double *)malloc(sizeof(double) * NV * NP);
    double *Wp = (double *)malloc(sizeof(double) * NV * NP);
    double *dU = (double *)calloc((size_t)NV * N, sizeof(double));
    if (!G || !Wp || !dU) { free(G); free(Wp); free(dU); return 1; }
    og_ghost_fill(Gr, U, G);                                           /* a1 */
#pragma omp parallel for
    for (int64_t c = 0; c < NP; c++) {                                 /* a2 */
        double Uc[NV], W[NV];
        for (int k = 0; k < NV; k++) Uc[k] = G[k * NP + c];
        cons_to_prim(Uc, W);
        for (int k = 0; k < NV; k++) Wp[k * NP + c] = W[k];
    }
    /* transverse terms of every padded cell whose neighbours along t exist (CTU form) */
    double *Ttr = NULL;
    if (Gr->ctu && Gr->ndim > 1 && Gr->scheme != OG_SCHEME_KT) {
        Ttr = (double *)calloc((size_t)Gr->ndim * NV * NP, sizeof(double));
        if (!Ttr) { free(G); free(Wp); free(dU); return 1; }
        for (int t = 0; t < Gr->ndim; t++) {
            int64_t st = (t == 0) ? 1 : (t == 1 ? P.p[0] : P.p[0] * P.p[1]);
#pragma omp parallel for
            for (int64_t c = 0; c < NP; c++) {
                int64_t q[3] = {c % P.p[0], (c / P.p[0]) % P.p[1], c / (P.p[0] * P.p[1])};
                if (q[t] < 1 || q[t] > P.p[t] - 2) continue;
                double Wc[3][NV], T[NV];
                for (int o = -1; o <= 1; o++)
                    for (int k = 0; k < NV; k++) Wc[o + 1][k] = Wp[k * NP + c + o * st];
                og_transverse(Wc[0], Wc[1], Wc[2], t, dt / Gr->dx[t], T);
                for (int k = 0; k < NV; k++) Ttr[((size_t)t * NV + k) * NP + c] = T[k];
            }
        }
    }
    for (int d = 0; d < Gr->ndim; d++) {                               /* a3-a7 */
        int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;              /* the other axes */
        int64_t n1 = P.n[a1], n2 = P.n[a2], nd = P.n[d];
        double dtdx = dt / Gr->dx[d];
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
        for (int64_t j2 = 0; j2 < n2; j2++)
            for (int64_t j1 = 0; j1 < n1; j1++) {
                /* pencil along d; face states of cells -1 .. nd */
                double *lo = (double *)malloc(sizeof(double) * NV * (nd + 2));
                double *hi = (double *)malloc(sizeof(double) * NV * (nd + 2));
                unsigned char *first = (unsigned char *)calloc((size_t)(nd + 1), 1); /* face i-1/2 at i */
                for (int64_t i = -1; i <= nd; i++) {
                    double Wc[3][NV];
                    for (int o = -1; o <= 1; o++) {
                        int64_t c3[3];
                        c3[d] = i + o; c3[a1] = j1; c3[a2] = j2;
                        int64_t pi = pidx(&P, c3[0], c3[1], c3[2]);
                        for (int k = 0; k < NV; k++) Wc[o + 1][k] = Wp[k * NP + pi];
                    }
                    double *li = lo + NV * (i + 1), *hi_ = hi + NV * (i + 1);
                    if (Gr->scheme == OG_SCHEME_MH_ROE)
                        upwind_states(Wc[0], Wc[1], Wc[2], d, dtdx, li, hi_);
                    else
                        hancock_states(Wc[0], Wc[1], Wc[2], d, dtdx, li, hi_);
                    if (Ttr) {
                        int64_t c3[3];
                        c3[d] = i; c3[a1] = j1; c3[a2] = j2;
                        int64_t pc = pidx(&P, c3[0], c3[1], c3[2]);
                        for (int t = 0; t < Gr->ndim; t++) {
                            if (t == d) continue;
                            for (int k = 0; k < NV; k++) {
                                double v = Ttr[((size_t)t * NV + k) * NP + pc];
                                li[k] += v;
                                hi_[k] += v;
                            }
                        }
                    }
                    face_state_check(Wc[1], d, li, hi_);
                }
                if (flag) {
                    /* first-order states on every face that touches a flagged cell */
                    for (int64_t i = -1; i < nd; i++) {
                        int64_t ca[3], cb[3];
                        ca[d] = i; ca[a1] = j1; ca[a2] = j2;
                        cb[d] = i + 1; cb[a1] = j1; cb[a2] = j2;
                        int64_t pa = pidx(&P, ca[0], ca[1], ca[2]), pb = pidx(&P, cb[0], cb[1], cb[2]);
                        if (!(flag[pa] || flag[pb])) continue;
                        first[i + 1] = 1;
                        for (int k = 0; k < NV; k++) {
                            hi[NV * (i + 1) + k] = Wp[k * NP + pa];
                            lo[NV * (i + 2) + k] = Wp[k * NP + pb];
                        }
                    }
                }
                /* faces i-1/2 for i = 0 .. nd, flux difference into dU */
                double Fm[NV], Fp[NV];
                face_flux(Gr, hi + NV * 0, lo + NV * 1, d, first[0], Fm);        /* face -1/2 */
                for (int64_t i = 0; i < nd; i++) {
                    face_flux(Gr, hi + NV * (i + 1), lo + NV * (i + 2), d, first[i + 1], Fp); /* face i+1/2 */
                    int64_t c3[3];
                    c3[d] = i; c3[a1] = j1; c3[a2] = j2;
                    int64_t c = (c3[2] * P.n[1] + c3[1]) * P.n[0] + c3[0];
                    for (int k = 0; k < NV; k++) dU[k * N + c] -= (Fp[k] - Fm[k]) / Gr->dx[d];
                    memcpy(Fm, Fp, sizeof Fm);
                }
                free(lo);
                free(hi);
                free(first);
            }
    }
#pragma omp parallel for
    for (int64_t c = 0; c < N; c++) {                                  /* a7, a8 */
        double Us[NV];
        for (int k = 0; k < NV; k++) Us[k] = U[k * N + c] + dt * dU[k * N + c];
        if (phi) gravity_source(Gr, phi, dt, c, Us);
        for (int k = 0; k < NV; k++) Unew[k * N + c] = Us[k];
    }
    free(G);
    free(Wp);
    free(dU);
    free(Ttr);
    return 0;
}

/* Tags of the grid's cells (bad[N]) on the padded grid: a ghost cell carries the tag of
 * its source cell (a1's mapping). */
static void padded_flags(const og_grid *Gr, const unsigned char *bad, unsigned char *flag)
{
    og_pad P = make_pad(Gr);
    for (int64_t z = -P.g[2]; z < P.n[2] + P.g[2]; z++)
        for (int64_t y = -P.g[1]; y < P.n[1] + P.g[1]; y++)
            for (int64_t x = -P.g[0]; x < P.n[0] + P.g[0]; x++) {
                int64_t c[3] = {x, y, z}, s[3];
                int mir;
                for (int d = 0; d < 3; d++)
                    s[d] = ghost_src(c[d], P.n[d], Gr->bc[2 * d], Gr->bc[2 * d + 1], &mir);
                flag[pidx(&P, x, y, z)] = bad[(s[2] * P.n[1] + s[1]) * P.n[0] + s[0]];
            }
}

/* One pass of the characteristic step from U to Unew: the second-order pass with
 * tagged == NULL, else the pass of og_step's a-posteriori fallback with first-order face
 * states on every face that touches a cell whose tagged[c] is non-zero (tagged[N] over the
 * grid's cells).  og_step is this pass repeated with the growing tagged set; a driver that
 * shares the fallback across several grids (slabs of one grid) repeats it itself.
 * Returns 0, or 1 on allocation failure. */
int og_step_pass(const og_grid *Gr, const double *U, const double *phi, double dt, const unsigned char *tagged,
                 double *Unew)
{
    if (!tagged) return step_pass(Gr, U, phi, dt, NULL, Unew);
    og_pad P = make_pad(Gr);
    unsigned char *flag = (unsigned char *)calloc((size_t)(P.p[0] * P.p[1] * P.p[2]), 1);
    if (!flag) return 1;
    padded_flags(Gr, tagged, flag);
    int rc = step_pass(Gr, U, phi, dt, flag, Unew);
    free(flag);
    return rc;
}

/* Per cell of U: 1 if realizable (rho > 0, P positive definite), else 0. */
void og_realizable_cells(const og_grid *Gr, const double *U, unsigned char *out)
{
    int64_t N = Gr->n[0] * Gr->n[1] * Gr->n[2];
    for (int64_t c = 0; c < N; c++) {
        double Uc[NV];
        for (int k = 0; k < NV; k++) Uc[k] = U[k * N + c];
        out[c] = (unsigned char)cell_realizable(Uc);
    }
}

/* One step of size dt from U to Unew ([NV][nz][ny][nx]).  phi: NULL or the
 * potential with one ghost layer on active dims ([nz+2gz][ny+2gy][nx+2gx]).
 * A-posteriori fallback (reading; the paper is silent on positivity): if the
 * second-order update leaves a cell non-realizable, the step is recomputed from U
 * with first-order face states on every face of every such cell (MOOD-style
 * detection, Clain, Diot & Loubere 2011); face fluxes stay shared, so the update
 * stays conservative.  Cells still non-realizable after that are left for the
 * caller's realizability check.  Returns 0, or 1 on allocation failure. */
int og_step_kt(const og_grid *Gr, const double *U, const double *phi, double dt, double *Unew);

int og_step(const og_grid *Gr, const double *U, const double *phi, double dt, double *Unew)
{
    if (Gr->scheme == OG_SCHEME_KT) return og_step_kt(Gr, U, phi, dt, Unew);
    if (step_pass(Gr, U, phi, dt, NULL, Unew)) return 1;
    og_pad P = make_pad(Gr);
    int64_t N = P.n[0] * P.n[1] * P.n[2];
    int64_t NP = P.p[0] * P.p[1] * P.p[2];
    unsigned char *bad = (unsigned char *)calloc((size_t)N, 1);
    if (!bad) return 1;
    int64_t nbad = 0;
    for (int64_t c = 0; c < N; c++) {
        double Uc[NV];
        for (int k = 0; k < NV; k++) Uc[k] = Unew[k * N + c];
        if (!cell_realizable(Uc)) { bad[c] = 1; nbad++; }
    }
    /* Each fallback pass adds the cells that are still non-realizable to the tagged set,
     * so the first-order region grows until the update is realizable (at most
     * OG_FALLBACK_PASSES passes). */
    unsigned char *flag = NULL;
    for (int pass = 0; nbad > 0 && pass < OG_FALLBACK_PASSES; pass++) {
        if (!flag) flag = (unsigned char *)calloc((size_t)NP, 1);
        if (!flag) { free(bad); return 1; }
        padded_flags(Gr, bad, flag);
        if (step_pass(Gr, U, phi, dt, flag, Unew)) { free(flag); free(bad); return 1; }
        nbad = 0;
        for (int64_t c = 0; c < N; c++) {
            double Uc[NV];
            for (int k = 0; k < NV; k++) Uc[k] = Unew[k * N + c];
            if (!cell_realizable(Uc) && !bad[c]) { bad[c] = 1; nbad++; }
        }
    }
    free(flag);
    free(bad);
    return 0;
}

/* ------------------------------------------------------------ KT scheme -- */
/* The Kurganov-Tadmor central scheme with second-order Runge-Kutta time integration
 * (Sec. 3.2; Kurganov & Tadmor 2000, eq 4.2):
 *   du_i/dt = L(u)_i = - sum_d (H_{d,i+1/2} - H_{d,i-1/2}) / dx_d,
 *   H_{i+1/2} = (f(u+) + f(u-)) / 2 - a_{i+1/2} (u+ - u-) / 2,
 * u- the value on the left side of face i+1/2 (from cell i), u+ on its right side (from
 * cell i+1), and a_{i+1/2} the larger spectral radius of df/du at u- and u+ (eq
 * spectralfreq), which for the BME is |u_n| + sqrt(3 P_nn / rho) (eq soundspeed, gamma = 3).
 * Readings (the paper defers the rest to KT2000):
 *   - u-/u+ come from a piecewise-linear reconstruction of the primitive variables,
 *     component by component, with the MC limiter (the generalised minmod with theta = 2);
 *     a cell with a face value of rho <= 0 or P_nn <= 0 takes first-order face values;
 *   - the time integration is Heun's two-stage Runge-Kutta method:
 *     u1 = u + dt L(u), u_new = (u + u1 + dt L(u1)) / 2;
 *   - gravity as a8, after the two stages;
 *   - the CFL rule a9 with the grid's CFL number.                                   */
void og_kt_reconstruct(const double *Wm, const double *W0, const double *Wp, int d, double *lo, double *hi)
{
    for (int k = 0; k < NV; k++) {
        double s = mc_limit(W0[k] - Wm[k], 0.5 * (Wp[k] - Wm[k]), Wp[k] - W0[k]);
        hi[k] = W0[k] + 0.5 * s;
        lo[k] = W0[k] - 0.5 * s;
    }
    int nn = tens_idx(d, d);
    if (!(hi[0] > 0.0 && lo[0] > 0.0 && hi[nn] > 0.0 && lo[nn] > 0.0))
        for (int k = 0; k < NV; k++) hi[k] = lo[k] = W0[k];
}

/* KT flux through a face normal to d: WL = u- (left side), WR = u+ (right side). */
void og_kt_flux(const double *WL, const double *WR, int d, double *H)
{
    double FL[NV], FR[NV], UL[NV], UR[NV];
    og_flux(WL, d, FL);
    og_flux(WR, d, FR);
    prim_to_cons(WL, UL);
    prim_to_cons(WR, UR);
    int nn = tens_idx(d, d);
    double aL = fabs(WL[1 + d]) + sqrt(3.0 * WL[nn] / WL[0]);
    double aR = fabs(WR[1 + d]) + sqrt(3.0 * WR[nn] / WR[0]);
    double a = fmax(aL, aR);
    for (int k = 0; k < NV; k++) H[k] = 0.5 * (FR[k] + FL[k]) - 0.5 * a * (UR[k] - UL[k]);
}

/* dU = L(U), the semi-discrete right-hand side, with the ghost cells of a1. */
static int kt_rhs(const og_grid *Gr, const double *U, double *dU)
{
    og_pad P = make_pad(Gr);
    int64_t N = P.n[0] * P.n[1] * P.n[2];
    int64_t NP = P.p[0] * P.p[1] * P.p[2];
    double *G = (double *)malloc(sizeof(double) * NV * NP);
    double *Wp = (double *)malloc(sizeof(double) * NV * NP);
    if (!G || !Wp) { free(G); free(Wp); return 1; }
    memset(dU, 0, sizeof(double) * NV * N);
    og_ghost_fill(Gr, U, G);
#pragma omp parallel for
    for (int64_t c = 0; c < NP; c++) {
        double Uc[NV], W[NV];
        for (int k = 0; k < NV; k++) Uc[k] = G[k * NP + c];
        cons_to_prim(Uc, W);
        for (int k = 0; k < NV; k++) Wp[k * NP + c] = W[k];
    }
    for (int d = 0; d < Gr->ndim; d++) {
        int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
        int64_t n1 = P.n[a1], n2 = P.n[a2], nd = P.n[d];
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
        for (int64_t j2 = 0; j2 < n2; j2++)
            for (int64_t j1 = 0; j1 < n1; j1++) {
                double *lo = (double *)malloc(sizeof(double) * NV * (nd + 2));
                double *hi = (double *)malloc(sizeof(double) * NV * (nd + 2));
                unsigned char *first = (unsigned char *)calloc((size_t)(nd + 1), 1); /* face i-1/2 at i */
                for (int64_t i = -1; i <= nd; i++) {
                    double Wc[3][NV];
                    for (int o = -1; o <= 1; o++) {
                        int64_t c3[3];
                        c3[d] = i + o; c3[a1] = j1; c3[a2] = j2;
                        int64_t pi = pidx(&P, c3[0], c3[1], c3[2]);
                        for (int k = 0; k < NV; k++) Wc[o + 1][k] = Wp[k * NP + pi];
                    }
                    og_kt_reconstruct(Wc[0], Wc[1], Wc[2], d, lo + NV * (i + 1), hi + NV * (i + 1));
                }
                double Hm[NV], Hp[NV];
                og_kt_flux(hi + NV * 0, lo + NV * 1, d, Hm);           /* face -1/2 */
                for (int64_t i = 0; i < nd; i++) {
                    og_kt_flux(hi + NV * (i + 1), lo + NV * (i + 2), d, Hp);
                    int64_t c3[3];
                    c3[d] = i; c3[a1] = j1; c3[a2] = j2;
                    int64_t c = (c3[2] * P.n[1] + c3[1]) * P.n[0] + c3[0];
                    for (int k = 0; k < NV; k++) dU[k * N + c] -= (Hp[k] - Hm[k]) / Gr->dx[d];
                    memcpy(Hm, Hp, sizeof Hm);
                }
                free(lo);
                free(hi);
            }
    }
    free(G);
    free(Wp);
    return 0;
}

int og_step_kt(const og_grid *Gr, const double *U, const double *phi, double dt, double *Unew)
{
    int64_t N = Gr->n[0] * Gr->n[1] * Gr->n[2];
    double *L0 = (double *)malloc(sizeof(double) * NV * N);
    double *U1 = (double *)malloc(sizeof(double) * NV * N);
    int rc = (!L0 || !U1);
    if (!rc) rc = kt_rhs(Gr, U, L0);
    if (!rc) {
        for (int64_t i = 0; i < NV * N; i++) U1[i] = U[i] + dt * L0[i];
        rc = kt_rhs(Gr, U1, L0);                 /* L0 <- L(U1) */
    }
    if (!rc) {
#pragma omp parallel for
        for (int64_t c = 0; c < N; c++) {
            double Us[NV];
            for (int k = 0; k < NV; k++)
                Us[k] = 0.5 * (U[k * N + c] + (U1[k * N + c] + dt * L0[k * N + c]));
            if (phi) gravity_source(Gr, phi, dt, c, Us);
            for (int k = 0; k < NV; k++) Unew[k * N + c] = Us[k];
        }
    }
    free(L0);
    free(U1);
    return rc ? 1 : 0;
}

/* --------------------------------------------------------------- a10 ----- */
/* Totals of the ten conserved fields, realizability (rho > 0 and P SPD by its
 * leading minors) and the first offending cell (-1 if none).                */
void og_diagnostics(const og_grid *G, const double *U, double *tot, int32_t *realizable,
                    int64_t *first_bad)
{
    int64_t N = G->n[0] * G->n[1] * G->n[2];
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int64_t c = 0; c < N; c++) s += U[k * N + c];
        tot[k] = s;
    }
    *first_bad = -1;
    for (int64_t c = 0; c < N; c++) {
        double Uc[NV], W[NV];
        for (int k = 0; k < NV; k++) Uc[k] = U[k * N + c];
        int ok = Uc[0] > 0.0;
        if (ok) {
            cons_to_prim(Uc, W);
            double m1 = W[4];
            double m2 = W[4] * W[7] - W[5] * W[5];
            double m3 = W[4] * (W[7] * W[9] - W[8] * W[8]) - W[5] * (W[5] * W[9] - W[8] * W[6]) +
                        W[6] * (W[5] * W[8] - W[7] * W[6]);
            ok = (m1 > 0.0) && (m2 > 0.0) && (m3 > 0.0);
        }
        if (!ok) { *first_bad = c; break; }
    }
    *realizable = (*first_bad < 0);
}

/* Run from t0 to t_end (last step clipped to land on t_end) or max_steps.
 * dt_max caps each step.  dt_hist (may be NULL) receives each dt taken.
 * Returns 0, or 4 if a step produced a non-realizable state (stops there).   */
int og_run(const og_grid *G, double *U, const double *phi, double t0, double t_end,
           int64_t max_steps, double dt_max, double *dt_hist, int64_t *nsteps, double *t_out)
{
    int64_t N = G->n[0] * G->n[1] * G->n[2];
    double *Un = (double *)malloc(sizeof(double) * NV * N);
    double t = t0;
    int64_t s = 0;
    int rc = 0;
    while (t < t_end && s < max_steps) {
        double dt = og_cfl_dt(G, U);
        if (dt > dt_max) dt = dt_max;
        double t_new = t + dt;
        if (t_new >= t_end) { dt = t_end - t; t_new = t_end; }
        if (og_step(G, U, phi, dt, Un)) { rc = 3; break; }
        memcpy(U, Un, sizeof(double) * NV * N);
        if (dt_hist) dt_hist[s] = dt;
        t = t_new;
        s++;
        double tot[NV];
        int32_t ok;
        int64_t bad;
        og_diagnostics(G, U, tot, &ok, &bad);
        if (!ok) { rc = 4; break; }
    }
    free(Un);
    *nsteps = s;
    *t_out = t;
    return rc;
}

/* Replay a given dt schedule (no CFL evaluation): U <- step^n(U). */
int og_run_schedule(const og_grid *G, double *U, const double *phi, const double *dts,
                    int64_t nsteps)
{
    int64_t N = G->n[0] * G->n[1] * G->n[2];
    double *Un = (double *)malloc(sizeof(double) * NV * N);
    for (int64_t s = 0; s < nsteps; s++) {
        if (og_step(G, U, phi, dts[s], Un)) { free(Un); return 3; }
        memcpy(U, Un, sizeof(double) * NV * N);
    }
    free(Un);
    return 0;
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void og_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Array helpers for the test harness: [NV][N] primitive <-> conserved. */
void og_prim_to_cons_arr(const double *W, double *U, int64_t N)
{
    for (int64_t c = 0; c < N; c++) {
        double w[NV], u[NV];
        for (int k = 0; k < NV; k++) w[k] = W[k * N + c];
        prim_to_cons(w, u);
        for (int k = 0; k < NV; k++) U[k * N + c] = u[k];
    }
}

void og_cons_to_prim_arr(const double *U, double *W, int64_t N)
{
    for (int64_t c = 0; c < N; c++) {
        double w[NV], u[NV];
        for (int k = 0; k < NV; k++) u[k] = U[k * N + c];
        cons_to_prim(u, w);
        for (int k = 0; k < NV; k++) W[k * N + c] = w[k];
    }
}

/* The step without the a-posteriori fallback (for tests of the fallback itself). */
int og_step_second_order_only(const og_grid *Gr, const double *U, const double *phi, double dt,
                              double *Unew)
{
    return step_pass(Gr, U, phi, dt, NULL, Unew);
}
