/*
 * msh.h -- C ABI of libmsh, a GB300 (sm_103a) solver for the collisionless Boltzmann
 * moment equations (BME) of Mitchell, Vorobyov & Hensler, arXiv:1210.5246.
 *
 * The operation behind every call is one Godunov finite-volume step of the ten moment
 * equations (Sec. 2, eqs contin, moment, dispers, closed with zero heat flux):
 * characteristic-traced MUSCL-Hancock reconstruction on the eigenvectors of the
 * primitive Jacobian (Sec. 3.3, eqs jacobian, eigenvalues, righteigvec, lefteigvec,
 * extended to ten variables), an HLL Riemann flux with the fast speed
 * sqrt(3 P_nn / rho) (Sec. 3.2 eq soundspeed, Sec. 3.3), an unsplit conservative
 * update, the gravity source applied after the hydro step (operator splitting, last
 * paragraph of Sec. 3.3) and a CFL time-step reduction.
 *
 * Conventions shared by all calls
 * -------------------------------
 * State layout: structure of arrays [10][nz][ny][nx], x fastest, no ghost cells, in
 * the grid's precision (float for MSH_FP32, double for MSH_FP64).  Component order:
 *   conserved U = (rho, m_x, m_y, m_z, E_xx, E_xy, E_xz, E_yy, E_yz, E_zz)
 *   primitive W = (rho, u_x, u_y, u_z, P_xx, P_xy, P_xz, P_yy, P_yz, P_zz)
 * with m = rho u and E_ij = P_ij + rho u_i u_j (Sec. 2, below eq dispers).
 * Unused dimensions have n = 1 (1D: n = {nx,1,1}; 2D: n = {nx,ny,1}).
 *
 * Memory: `where` = MSH_HOST means a host pointer (pageable or pinned), MSH_DEVICE a
 * device pointer on the current CUDA device.  The caller keeps ownership of every
 * pointer it passes; the library copies what it needs before returning (or, for
 * device pointers, in stream order on the grid's stream).  The library owns the
 * buffers behind a handle until msh_destroy / msh_batch_destroy.
 *
 * Errors: every call returns an msh_status.  On error nothing is written to the
 * caller's output arguments and msh_last_error() (thread-local) describes the cause.
 * No C++ exception crosses the ABI.  There is no CPU fallback: without a usable CUDA
 * device the calls that need one return MSH_E_CUDA.
 */
#ifndef MSH_H
#define MSH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t msh_status;
#define MSH_OK 0
#define MSH_E_INVALID_ARG 1   /* bad size, pointer, enum or order of arguments          */
#define MSH_E_CUDA 2          /* a CUDA runtime call failed (message has the CUDA error) */
#define MSH_E_NOMEM 3         /* device or pinned allocation failed                     */
#define MSH_E_REALIZABILITY 4 /* rho <= 0 or P not positive definite in some cell       */
#define MSH_E_TIMEOUT 5       /* a bounded device-side wait ran out                     */
#define MSH_E_STATE 6         /* call made in the wrong order (e.g. step before state)  */

#define MSH_BC_PERIODIC 0     /* wrap-around                                            */
#define MSH_BC_OUTFLOW 1      /* zero-gradient copy of the edge cell                    */
#define MSH_BC_REFLECT 2      /* mirror; negates m_n and E_nt (t != n) of the image     */

#define MSH_FP32 0
#define MSH_FP64 1

#define MSH_SCHEME_MUSCL_HANCOCK 0     /* characteristic MUSCL-Hancock + HLL (Sec. 3.3)     */
#define MSH_SCHEME_KT 1                /* Kurganov-Tadmor central scheme + RK2 (Sec. 3.2)   */
#define MSH_SCHEME_MUSCL_HANCOCK_ROE 2 /* characteristic MUSCL-Hancock + Roe-type flux     */
#define MSH_SCHEME_MUSCL_HANCOCK_HLLC 3 /* characteristic MUSCL-Hancock + HLLC flux        */

#define MSH_HOST 0
#define MSH_DEVICE 1

#define MSH_CONSERVED 0
#define MSH_PRIMITIVE 1

typedef struct msh_grid msh_grid;
typedef struct msh_batch msh_batch;

/* Description of the last error on the calling thread ("" if none).  The pointer stays
 * valid until the next msh_* call on this thread. */
const char *msh_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t msh_version(void);

/*
 * Create a uniform grid (the paper's Sec. 3.1 block of cells without AMR).
 *   ndim      1, 2 or 3
 *   n[3]      cells per dimension, n[d] >= 2 for d < ndim, n[d] == 1 otherwise
 *   lo, hi    domain corners; hi[d] > lo[d] for d < ndim (cell width (hi-lo)/n)
 *   bc[6]     bc[2d] lower, bc[2d+1] upper boundary of dimension d (MSH_BC_*); a
 *             periodic side must be paired with a periodic side
 *   precision MSH_FP32 or MSH_FP64 (arithmetic and storage of the state)
 *   cfl       Courant number C in (0, 1]: dt = C / max sum_d (|u_d| + sqrt(3 P_dd/rho))/dx_d
 *   stream    cudaStream_t to run on, or NULL for a stream the grid creates and owns
 * Allocates two state buffers, reduction scratch and control block on the current
 * device.  *out receives the handle.
 */
msh_status msh_init_grid(msh_grid **out, int32_t ndim, const int64_t n[3], const double lo[3],
                         const double hi[3], const int32_t bc[6], int32_t precision, double cfl,
                         void *stream);

/* Release everything the grid owns.  NULL is accepted. */
msh_status msh_destroy(msh_grid *g);

/*
 * Copy a state into the grid (and reset nothing else: time and step count are kept).
 *   U     [10][nz][ny][nx] in the grid precision, conserved or primitive (kind)
 * Rejects a state with rho <= 0 or non positive-definite P (Sylvester minors) with
 * MSH_E_REALIZABILITY, leaving the previous state in place.  Computes the CFL time
 * step of the new state.
 */
msh_status msh_set_state(msh_grid *g, const void *U, int32_t where, int32_t kind);

/* Copy the current state out ([10][nz][ny][nx], grid precision, conserved or primitive). */
msh_status msh_get_state(msh_grid *g, void *U, int32_t where, int32_t kind);

/* Set the simulation time and step counter (e.g. when resuming from a saved state). */
msh_status msh_set_time(msh_grid *g, double t, int64_t step);

/* Current simulation time (accumulated in FP64) and number of steps taken. */
msh_status msh_get_time(msh_grid *g, double *t, int64_t *step);

/*
 * External gravitational potential Phi at cell centres, including one ghost layer on
 * each active dimension: [nz+2gz][ny+2gy][nx+2gx] doubles, g = 1 for active dims, 0
 * otherwise.  The acceleration a = -grad Phi is taken by central differences and applied
 * after the hydro update (Sec. 3.3, operator splitting; sources of eqs moment/dispers):
 * m += dt rho a, E += dt (mbar a^T + a mbar^T), mbar = (m_before + m_after)/2.
 * phi == NULL removes gravity.  The library copies the array.
 */
msh_status msh_set_potential(msh_grid *g, const double *phi, int32_t where);

/*
 * One step with dt = min(CFL dt of the current state, dt_max).  *dt_taken (may be NULL)
 * receives the step size.  Returns MSH_E_REALIZABILITY (and keeps the new state, so it
 * can be inspected) if the step produced a non-realizable cell.
 */
msh_status msh_step(msh_grid *g, double dt_max, double *dt_taken);

/*
 * Advance until t_end (the last step is clipped to land on t_end exactly) or until
 * max_steps more steps were taken.  Steps are launched from CUDA graphs with the time
 * control on the device; the host synchronises only to test for completion.
 * *steps (may be NULL) receives the number of steps taken by this call, *t_out (may be
 * NULL) the final time.  Stops early with MSH_E_REALIZABILITY on a non-realizable cell.
 */
msh_status msh_run(msh_grid *g, double t_end, int64_t max_steps, int64_t *steps, double *t_out);

/*
 * Ensemble of independent states through host memory: each of the `count` states is
 * uploaded, advanced from t = 0 by exactly `nsteps` CFL steps of the grid's scheme (same
 * geometry, boundaries, potential, self-gravity and CFL number as msh_run; Sec. 3.3 per
 * step) and downloaded.  Uploads, steps and downloads of different states overlap: four
 * device slots of one state each, a copy-in and a copy-out stream besides the grid's
 * stream.
 *   in[k]    host pointer to state k, [10][nz][ny][nx] in the grid's precision, `kind`
 *            (MSH_CONSERVED or MSH_PRIMITIVE); page-locked memory lets the copies overlap
 *   out[k]   host pointer receiving the result of state k (same layout and kind); no out[j]
 *            may overlap any in[k] (a download can run during a later upload); out[j] may
 *            repeat (downloads run in order)
 *   status   NULL or count int32: MSH_OK, or MSH_E_REALIZABILITY if state k's input was not
 *            realizable (it is not stepped) or one of its steps produced a non-realizable
 *            cell; the content of out[k] is then unspecified
 * Returns MSH_E_INVALID_ARG (null pointers, count < 0, nsteps < 1), MSH_E_NOMEM (four
 * more state buffers), MSH_E_REALIZABILITY if any state failed (the others are complete),
 * MSH_E_CUDA.  Afterwards the grid holds the last state's result, its time and a step
 * counter advanced by count * nsteps; a recording tape ends (as with msh_set_state).
 */
msh_status msh_run_ensemble(msh_grid *g, int64_t count, const void *const *in, void *const *out, int32_t kind,
                            int64_t nsteps, int32_t *status);

/*
 * FP64 totals of the ten conserved fields over the grid (pairwise reduced, fixed order)
 * as of the last step or set_state, realizability flag (1 = every cell has rho > 0 and
 * P positive definite) and the first offending cell's linear index (-1 if none).
 * Any output pointer may be NULL.
 */
msh_status msh_diagnostics(msh_grid *g, double totals[10], int32_t *realizable, int64_t *first_bad);

/*
 * Record the dt of every following step into a device-side history of `capacity`
 * entries (0 disables and frees it).  Needed by msh_adjoint_run's callers that replay a
 * forward run.  msh_get_dt_history copies at most `capacity` entries (host pointer) and
 * returns the number recorded in *count.
 */
msh_status msh_set_recording(msh_grid *g, int64_t capacity);
msh_status msh_get_dt_history(msh_grid *g, double *dts, int64_t capacity, int64_t *count);

/*
 * Tile shape of the 2D/3D step kernels.  3D: `rows` = thread rows per block (4, 8 or 16,
 * each a warp of 32 cells in x) and `zchunk` = z planes each block streams, or 0 for the
 * balanced tiling: one block per block slot of the device's SMs, each streaming the same
 * number of planes (whole columns of tiles first, then equal runs of the rest, at least 8
 * planes each).  2D: `rows` = warps per block (4, 8 or 16, each a strip of 28 updated
 * columns) and `zchunk` = grid rows each warp streams in y.  1D ignores both.  `zchunk` >=
 * 1 (3D: >= 0), clipped to the streamed axis.  3D FP64 grids take rows 4 or 8 (rows 16
 * would need more shared memory than a thread block has).  Defaults: rows 8; zchunk 0
 * (3D) or 16 (2D).  msh_autotune times the candidates (3D: rows 4/8/16 with the balanced
 * tiling and with chunks cutting z into 1..8 near-equal windows; 2D: rows 4/8/16 with
 * zchunk 8..64) on this grid's current state (without changing it or the tape) and keeps
 * the fastest; the chosen values are returned in *rows / *zchunk (may be NULL).
 */
msh_status msh_set_tiling(msh_grid *g, int32_t rows, int32_t zchunk);
msh_status msh_get_tiling(msh_grid *g, int32_t *rows, int32_t *zchunk);
msh_status msh_autotune(msh_grid *g, int32_t *rows, int32_t *zchunk);

/*
 * Kernel timing: with profiling on, msh_run launches the same kernels without the CUDA
 * graph and brackets every step-kernel launch with CUDA events on the grid's stream,
 * accumulating their elapsed times.  msh_get_profile returns the summed step-kernel time,
 * the summed time from each step kernel's end to its finalize kernel's end (both in
 * ms) and the number of timed launches since profiling was switched on.
 */
msh_status msh_set_profiling(msh_grid *g, int32_t on);
msh_status msh_get_profile(msh_grid *g, double *step_kernel_ms, double *finalize_ms, int64_t *launches);

/*
 * Test hook for the bounded waits of the 3D step (no counterpart in the paper).  kind 1:
 * in the next characteristic step (HLL, Roe-type or HLLC flux) taken eagerly (msh_step,
 * msh_step_dt, msh_step_begin; never inside the CUDA graph of msh_run), thread block 0 of
 * the step kernel does not issue its bulk tensor copy of plane -2 (the first copy of a
 * stretch from z = 0, which every tiling gives block 0 first), so the threads waiting for
 * that plane give up after about 2^31 SM clocks (about a second), the step's result is
 * void and the call returns MSH_E_TIMEOUT; the grid stays usable after msh_set_state.
 * Grids whose 3D step stages cell by cell (rows not a multiple of 16 bytes), 1D and 2D
 * grids ignore it.  kind 0 clears it.  The hook applies to one step.  Errors:
 * MSH_E_INVALID_ARG for a null grid or another kind.
 */
msh_status msh_set_test_fault(msh_grid *g, int32_t kind);

/*
 * Discrete adjoint (vector-Jacobian product) of `nsteps` forward steps taken from U0
 * with the frozen time-step schedule dt_sched[nsteps] (host doubles), limiter branches,
 * HLL branches and face-state fallbacks frozen at their forward values:
 *     dL_dU0 = (d U_N / d U_0)^T dL_dUN.
 *   U0, dL_dUN, dL_dU0   [10][nz][ny][nx] in the grid precision, located per `where`;
 *                        if kind == MSH_PRIMITIVE, U0 is primitive and dL_dU0 is the
 *                        gradient with respect to the primitive initial state
 *   K                    checkpoint interval (>= 1): the forward states are stored every
 *                        K steps and recomputed in between during the reverse sweep
 * Uses the grid's potential and boundaries; does not change the grid's state or time.
 */
msh_status msh_adjoint_run(msh_grid *g, const void *U0, int64_t nsteps, const double *dt_sched,
                           int32_t K, const void *dL_dUN, void *dL_dU0, int32_t where,
                           int32_t kind);

/*
 * Adjoint tape of a forward run.  msh_set_tape(g, K, max_steps) starts recording at the
 * grid's current step s0: the step kernel of every step s0 + mK stores its input state
 * U^{s0+mK} in device memory owned by the grid (ceil(max_steps / K) states), and the
 * finalize kernel records each step's dt and whether its a-posteriori fallback tagged
 * cells, for the first max_steps steps.  Recording costs one extra write of the state
 * every K steps and no launches.  msh_set_state and msh_set_time end the recording (the
 * memory is kept for the next msh_set_tape); K = 0 frees it.  Needs a state.
 *
 * msh_adjoint_tape(g, dL_dUN, dL_dU0, where, kind) is msh_adjoint_run over the recorded
 * steps s0 .. current step, with U0 = U^{s0} and the recorded dt schedule, without the
 * forward sweep msh_adjoint_run needs to build its checkpoints.  kind == MSH_PRIMITIVE
 * returns the gradient with respect to W0 = primitive(U^{s0}).  Errors: MSH_E_STATE if no
 * tape is being recorded or the run went past max_steps.
 */
msh_status msh_set_tape(msh_grid *g, int32_t K, int64_t max_steps);
msh_status msh_adjoint_tape(msh_grid *g, const void *dL_dUN, void *dL_dU0, int32_t where, int32_t kind);

/*
 * Scheme of the grid's steps (default MSH_SCHEME_MUSCL_HANCOCK).  MSH_SCHEME_KT is the
 * semi-discrete central scheme of Kurganov & Tadmor (Sec. 3.2, eq 4.2 of their paper):
 *   du_i/dt = -sum_d (H_{i+1/2} - H_{i-1/2}) / dx_d,
 *   H_{i+1/2} = (f(u+) + f(u-)) / 2 - a_{i+1/2} (u+ - u-) / 2,
 * with a_{i+1/2} the larger spectral radius |u_n| + sqrt(3 P_nn / rho) of the two face
 * values (eqs spectralfreq, soundspeed with gamma = 3), face values from the primitive
 * variables reconstructed component by component with the MC limiter (first order where a
 * face value has rho <= 0 or P_nn <= 0), Heun's second-order Runge-Kutta stages
 * (u1 = u + dt L(u), u_new = (u + u1 + dt L(u1)) / 2), the gravity source after them and
 * the same CFL rule; it has no a-posteriori fallback.  Selecting it allocates one more
 * state buffer.  MSH_SCHEME_MUSCL_HANCOCK_ROE is the characteristic step of Sec. 3.3 with
 * the tracing a Riemann solver that resolves every wave takes (eqs 40-43: the reference
 * states traced with the fastest wave towards each face, each wave that reaches the face
 * corrected to its own speed; eq 41 in the mirror form of eq 40) and a Roe-type flux
 * (Roe 1981) in place of HLL:
 *   F = (f(wl) + f(wr)) / 2 - (dU/dW)(wm) R |Lambda| L (wr - wl) / 2,  wm = (wl + wr) / 2,
 * the closed-form eigen-system of wm and Harten's entropy fix on the two fast waves
 * (delta = cf / 10).  MSH_SCHEME_MUSCL_HANCOCK_HLLC is the characteristic step with the
 * Hancock predictor and a three-wave HLLC flux: outer waves as in HLL, the contact between
 * them; the pairs (u_i, P_in) take common star values from the momentum jump conditions
 * across the outer waves, the star states follow from the jump conditions (HLL where the
 * contact speed is not strictly between the outer ones).  Both have the a-posteriori
 * fallback of HLL, whose faces with first-order states take the HLL flux.  The adjoint
 * (msh_adjoint_run, msh_set_tape) covers MUSCL-Hancock with HLL only: MSH_E_STATE otherwise.
 */
msh_status msh_set_scheme(msh_grid *g, int32_t scheme);

/*
 * Corner-transport-upwind (CTU) form of the characteristic schemes (on = 1; 0 switches it
 * off, the default).  Sec. 3.3 uses FLASH's unsplit MUSCL-Hancock solver (Lee & Deane 2009)
 * but prints no transverse coupling; with CTU every face state along d also takes
 *   sum_{t != d} T_t,  T_t = -(dt / (2 dx_t)) sum_a lam^a (L^a . dW^a) R^a,
 *   dW^a = W_i - W_{i-e_t} if lam^a > 0, else W_{i+e_t} - W_i,
 * the quasi-linear transverse derivative -(dt/2) A_t dW/dx_t of cell i taken wave by wave
 * from the upwind side (eigen-system of cell i along t), before the face-state check; the
 * first-order faces of the a-posteriori fallback take none.  The CFL rule becomes
 *   dt = C / max_cells max_d (|u_d| + sqrt(3 P_dd / rho)) / dx_d
 * (the maximum over the directions instead of the sum), so a step can be up to ndim times
 * longer.  No effect in 1D.  Switching it re-plans the next step of the current state.
 * Errors: MSH_E_STATE with the central scheme (MSH_SCHEME_KT) or a recording adjoint tape;
 * the adjoint (msh_adjoint_run, msh_set_tape) refuses a 2D/3D grid with CTU on.
 * msh_get_ctu reads the setting.
 */
msh_status msh_set_ctu(msh_grid *g, int32_t on);
msh_status msh_get_ctu(const msh_grid *g, int32_t *on);

/*
 * Periodic self-gravity with the gravitational constant G (> 0; 0 switches it off).  Needs
 * periodic boundaries on every active dimension (MSH_E_INVALID_ARG otherwise).  Before every
 * step the potential of the density of U^n solves the 3-point discrete Poisson equation
 *   sum_d (Phi_{i+e_d} - 2 Phi_i + Phi_{i-e_d}) / dx_d^2 = 4 pi G (rho_i - mean rho)
 * by FFT (cuFFT); a^n = -grad Phi^n by central differences, and the step's gravity source
 * (applied after the hydro update, Sec. 3.3) uses the acceleration interpolated forward in
 * time from the stored previous one (Sec. 3.3, last paragraph):
 *   a^{n+1/2} = a^n + (dt_n / (2 dt_{n-1})) (a^n - a^{n-1}),  a^n on a state's first step,
 * plus -grad of the external potential if one is set.  Works with both schemes; not with
 * the adjoint (MSH_E_STATE) and not within a slab decomposition (the solve is global).
 */
msh_status msh_set_self_gravity(msh_grid *g, double G);

/*
 * Slab decomposition: several grids, each owning a slab of one global grid along its last
 * active axis (z in 3D, y in 2D, x in 1D) plus two halo layers copied from the
 * neighbouring slabs before every step (the stencil radius of the step is two cells,
 * Sec. 3.3).  A layer is one index of that axis, with all cells of the other axes.
 *   msh_get_slab / msh_set_slab   copy `count` layers from layer `start` of the conserved
 *                                 state to / from buf [10][count][...] in the grid's
 *                                 precision (host or device per `where`; the caller owns
 *                                 buf).  After msh_set_slab the next msh_step / msh_run
 *                                 first recomputes the CFL time step.
 *   msh_reduce_layers             FP64 totals, CFL dt (cfl / max over the layers of
 *                                 sum_d (|u_d| + sqrt(3 P_dd/rho))/dx_d) and realizability of
 *                                 layers [start, start + count) only (a slab without its halo);
 *                                 any output may be NULL.
 *   msh_step_dt                   one step with exactly dt (> 0; no CFL limit, no end time);
 *                                 *tagged_cells (may be NULL) receives the number of cells the
 *                                 a-posteriori fallback tagged in it.  The fallback couples
 *                                 cells within a step, so a slab run equals the single-grid run
 *                                 only for steps in which no rank tagged cells; the phased step
 *                                 below shares the fallback between slabs.
 *   msh_set_cell_width            replaces the cell widths dx[d] (> 0, active dims) that
 *                                 msh_init_grid derived from (hi - lo) / n: a slab of m
 *                                 layers takes the global grid's widths exactly, which
 *                                 (hi - lo) / m cannot always reproduce in floating point.
 * Errors: MSH_E_INVALID_ARG for layers outside the grid, MSH_E_STATE without a state.
 */
msh_status msh_set_cell_width(msh_grid *g, const double dx[3]);
msh_status msh_get_slab(msh_grid *g, int64_t start, int64_t count, void *buf, int32_t where);
msh_status msh_set_slab(msh_grid *g, int64_t start, int64_t count, const void *buf, int32_t where);
msh_status msh_reduce_layers(msh_grid *g, int64_t start, int64_t count, double totals[10], double *dt_cfl,
                             int32_t *realizable);
msh_status msh_step_dt(msh_grid *g, double dt, int32_t *tagged_cells);

/*
 * Phased step: msh_step_dt split at the passes of its a-posteriori fallback, so that slabs
 * of one grid take their fallback passes together (the guardcell exchange of Sec. 3.1
 * applied to the fallback tags; the fallback itself is this library's positivity rule: a
 * cell whose second-order update is not realizable is tagged, and the step is recomputed
 * with first-order face states on every face of every tagged cell, at most 4 passes, cells
 * still failing joining the tagged set).  A face's states depend on the tags of the two
 * cells it joins, so a slab needs its neighbours' tags in its first halo layer before each
 * pass.  The protocol, per step, on every slab:
 *   msh_step_begin(g, dt)          the second-order pass with exactly dt; its failing cells
 *                                  are tagged by pass 0;
 *   then for p = 1, 2, ... 4, while some slab's owned layers hold cells tagged by pass p-1
 *   (msh_count_tags, summed over the slabs):
 *     msh_set_tags on the halo layers from the neighbours' msh_get_tags of their owned
 *     boundary layers, then msh_step_retry(g, p): fallback pass p from the same U^n with
 *     first-order faces at every cell tagged by passes 0 .. p-1 of this step, run even where
 *     this grid tagged nothing itself; its newly failing cells are tagged by pass p;
 *   msh_step_end(g, &tagged)       the step's totals, CFL dt of the new state, time and step
 *                                  counter advance (MSH_E_REALIZABILITY as msh_step_dt).
 * On one grid, the passes msh_step_dt would run give its result bit for bit.
 *   msh_get_tags / msh_set_tags    per cell of layers [start, start + count) (int32
 *                                  levels[count][cells per layer], host or device per
 *                                  `where`, owned by the caller): the pass of the current step
 *                                  that tagged it, or -1.  msh_set_tags overwrites the tags of
 *                                  those layers (-1 clears).
 *   msh_count_tags                 *n = cells of layers [start, start + count) tagged by pass
 *                                  `level` (0 .. 4) of the current step.
 * The central scheme has no fallback (msh_step_begin: MSH_E_STATE; step it with
 * msh_step_dt), nor does a grid with self-gravity take a phased step.  msh_step_retry out
 * of order or outside begin .. end, and msh_step_end without begin: MSH_E_STATE or
 * MSH_E_INVALID_ARG; any other stepping call closes an open phased step.
 */
msh_status msh_step_begin(msh_grid *g, double dt);
msh_status msh_step_retry(msh_grid *g, int32_t level);
msh_status msh_step_end(msh_grid *g, int32_t *tagged_cells);
msh_status msh_get_tags(msh_grid *g, int64_t start, int64_t count, int32_t *levels, int32_t where);
msh_status msh_set_tags(msh_grid *g, int64_t start, int64_t count, const int32_t *levels, int32_t where);
msh_status msh_count_tags(msh_grid *g, int64_t start, int64_t count, int32_t level, int64_t *n);

/*
 * Batched independent 1D Riemann problems ("tubes") on [0, 1] with the interface at 0.5
 * and outflow boundaries, each advanced to its own t_end with its own CFL time step.
 *   ntubes           number of tubes (>= 1)
 *   len[ntubes]      cells per tube, 4 <= len <= 2048 (FP32) or 1024 (FP64) (host)
 *   WL, WR           [ntubes][10] primitive left / right states (host doubles)
 *   t_end[ntubes]    final times (host doubles, > 0)
 *   precision        MSH_FP32 or MSH_FP64
 * The tubes are stored back to back, [10][sum len] (tube k starts at the prefix sum of
 * len).  msh_batch_run advances all tubes in one persistent launch captured in a CUDA
 * graph; thread blocks take tubes longest first from a device work queue.  Cells whose
 * second-order update is not realizable trigger the same a-posteriori first-order
 * fallback as msh_step (the step is recomputed from U^n with first-order faces there);
 * a tube still non-realizable after it stops with MSH_E_REALIZABILITY.  threads is
 * the block size (0 = autotuned: the fastest of the candidates on a warm-up run).
 * max_steps caps the steps of each tube (MSH_E_TIMEOUT if a tube hits it before t_end).
 */
msh_status msh_batch_init(msh_batch **out, int32_t ntubes, const int32_t *len, const double *WL,
                          const double *WR, const double *t_end, int32_t precision, double cfl,
                          void *stream);
msh_status msh_batch_reset(msh_batch *b);
msh_status msh_batch_run(msh_batch *b, int32_t threads, int64_t max_steps);
/* One tube per launch sequence: the same tubes advanced with one step-kernel launch per
 * step (the baseline the persistent form is compared with).  tubes == NULL runs all. */
msh_status msh_batch_run_per_tube(msh_batch *b, const int32_t *tubes, int32_t count,
                                  int64_t max_steps);
msh_status msh_batch_get_state(msh_batch *b, void *U, int32_t where, int32_t kind);
/* steps[ntubes] and t[ntubes] (host, either may be NULL); *cell_updates = sum steps*len. */
msh_status msh_batch_info(msh_batch *b, int64_t *steps, double *t, int64_t *cell_updates);
/* Per tube, the number of steps of the last msh_batch_run whose second-order update left
 * cells non-realizable, i.e. that took the a-posteriori fallback passes (counts[ntubes],
 * host).  Zero after msh_batch_init / msh_batch_reset, and for tubes stepped by
 * msh_batch_run_per_tube. */
msh_status msh_batch_fallback_steps(msh_batch *b, int64_t *counts);
msh_status msh_batch_destroy(msh_batch *b);

/*
 * One step of a 1D/2D/3D grid (no gravity) that allocates no memory, for callers that
 * cannot allocate device memory: code running inside another framework's pre-sized memory
 * pool, a real-time or embedded host loop that must not enter the allocator, or any code
 * that owns nothing but the two state buffers it was given.  The paper has no counterpart;
 * this is a convenience of the library.
 *   ndim, n, lo, hi, bc, precision, cfl   as for msh_init_grid
 *   dt_max     the step is dt = min(CFL dt of U_in, dt_max)
 *   U_in       device pointer, conserved state [10][nz][ny][nx] in the given precision
 *   U_out      device pointer receiving U after one step (must not alias U_in)
 *   stream     cudaStream_t to run on (NULL: the default stream); the call synchronises it
 *   dt_taken   host pointer receiving the step size (may be NULL)
 * The step is always the default one of a new grid: characteristic MUSCL-Hancock with the
 * HLL flux, no corner-transport-upwind terms, the a-posteriori fallback, the default tiling
 * (8 rows); a grid set to another scheme, to CTU or to another tiling steps differently.
 * A non-realizable U_in (rho <= 0 or P not positive definite in some cell) is rejected with
 * MSH_E_REALIZABILITY before any step, U_out untouched; a step whose result stays
 * non-realizable after the fallback passes also returns MSH_E_REALIZABILITY (U_out then
 * holds that result).  msh_last_error() names the first offending cell.
 * The working memory (control block, reduction partials, fallback tags) is one file-scope
 * device array of about 5.6 MB that every GPU holds from the moment it loads the library
 * until the process exits; grids of more than 1,048,576 cells (or needing more than 16384
 * thread blocks) are rejected with MSH_E_INVALID_ARG.  The first call on a device looks up
 * that array's device address, so make the first call before any stream capture.  Every
 * call shares the array: each call clears what must start at zero, and calls that overlap
 * on the GPU (from other streams or host threads) race on it.  No cudaMalloc, cudaFree or
 * other allocating routine is called.
 */
msh_status msh_step_noalloc(int32_t ndim, const int64_t n[3], const double lo[3], const double hi[3],
                            const int32_t bc[6], int32_t precision, double cfl, double dt_max,
                            const void *U_in, void *U_out, void *stream, double *dt_taken);

#ifdef __cplusplus
}
#endif

#endif /* MSH_H */
