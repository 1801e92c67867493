/*
 * hydro.h -- C ABI of the GB300 (sm_103a) WENO5 / Lax-Friedrichs / SSP-RK3 solver of the 2D Euler
 * equations with a level-set flame scalar.
 *
 * The method is the hydrodynamics update of Leung, Chu & Lin (2015), "A new hydrodynamics code for
 * Type Ia supernovae": the conservative Euler equations in (r,z) with geometric and gravity source
 * terms (Sec. 2.1, Eq. euler2D), finite-difference WENO reconstruction of fluxes split by a global
 * Lax-Friedrichs splitting (Sec. 2.1), the three-stage third-order SSP Runge-Kutta scheme named there
 * as the original prescription (Sec. 2.1), the CFL time step dt = c_cfl Delta / (c_s + |v_r| + |v_z|)
 * (Sec. 5.4), and the level-set scalar S advected by v + v_flame (Sec. 2.2).
 *
 * Conventions shared by every entry point
 *   - State arrays are structure-of-arrays U[f][j][i] with i (x, or r) contiguous: nfields planes
 *     of ny rows of nx values, dtype float (HYDRO_F32) or double (HYDRO_F64). Fields:
 *     0 rho, 1 rho*u (rho v_r), 2 rho*v (rho v_z), 3 total energy density tau, 4 level set phi.
 *     Values are point values at cell centres x_i = x0 + (i + 1/2) dx, y_j = y0 + (j + 1/2) dy.
 *   - Pointers named U / lambda are DEVICE pointers owned by the caller unless the name says host.
 *     The library owns only its context and the scratch it allocates in hydro_init (three padded
 *     working states, reduction slots, logs) and frees in hydro_destroy.
 *   - All device work runs on the context's stream, asynchronously, except calls that return host
 *     values (time, dt, totals, status), which synchronise that stream.
 *   - Return codes: HYDRO_OK (0) or a negative HYDRO_E* code; nothing aborts. hydro_last_error gives
 *     the context's message for the last failure.
 */
#ifndef HYDRO_H
#define HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_ctx hydro_ctx;

typedef enum { HYDRO_F32 = 0, HYDRO_F64 = 1 } hydro_dtype;

/* Boundary kinds (Sec. 2.1 and the code tests of Sec. 5): periodic; transmissive (outflow, zero
 * gradient); reflecting wall (mirror, normal momentum reversed); symmetry axis r = 0 of an (r,z)
 * grid (same mirror rule, x-lo face only). Ghost images of phi are even mirrors. */
typedef enum {
  HYDRO_BC_PERIODIC = 0,
  HYDRO_BC_TRANSMISSIVE = 1,
  HYDRO_BC_REFLECT = 2,
  HYDRO_BC_AXIS = 3
} hydro_bc;

enum {
  HYDRO_OK = 0,
  HYDRO_EINVAL = -1,        /* bad argument: null pointer, size, bc pair, dtype, nfields        */
  HYDRO_ECUDA = -2,         /* a CUDA call failed (message in hydro_last_error)                 */
  HYDRO_ENONPHYSICAL = -3,  /* the device saw a non-finite value, rho <= 0 or p <= 0             */
  HYDRO_ETIMEOUT = -4,      /* a device wait or a host wait on the stream exceeded its limit     */
  HYDRO_ESTATE = -5,        /* call out of order (e.g. adjoint sweep without a recorded run)     */
  HYDRO_ESIZE = -6          /* a size beyond a fixed limit of an allocation-free entry point     */
};

/* Flux reconstruction (Sec. 2.1). COMPONENT: WENO5 of each conserved component's Lax-Friedrichs split
 * flux. CHARACTERISTIC: the "WENO-Roe" construction the paper names (Jiang & Shu 1996): at every face
 * the split fluxes of the six stencil cells are projected on the left eigenvectors of the flux Jacobian
 * at the Roe average of the face's two cells, reconstructed per characteristic field with WENO5, and
 * projected back; the same global alpha serves every field. The adjoint entry points and batched steps
 * take COMPONENT contexts only (HYDRO_EINVAL otherwise). */
typedef enum { HYDRO_SCHEME_COMPONENT = 0, HYDRO_SCHEME_CHARACTERISTIC = 1 } hydro_scheme;

typedef struct {
  int nx, ny;               /* interior cells, >= 3 each                                         */
  double x0, x1, y0, y1;    /* domain; with geometry 1, x is r and x0 >= 0                        */
  double gamma;             /* ideal gas p = (gamma - 1) rho eps, gamma > 1                       */
  double cfl;               /* Courant number c_cfl > 0                                          */
  int geometry;             /* 0 Cartesian (x, y); 1 axisymmetric (r, z): adds -(1/r) sources     */
  double gravity_y;         /* constant acceleration along y (z); sources (0,0,rho g, m_y g)      */
  int bc[4];                /* hydro_bc of faces x-lo, x-hi, y-lo, y-hi                           */
  int nfields;              /* 4 (hydro) or 5 (hydro + level set phi)                             */
  double flame_speed;       /* burning speed s_f of the level-set front (phi > 0 ash)             */
  int dtype;                /* hydro_dtype                                                       */
  int scheme;               /* hydro_scheme: how the hydro fluxes are reconstructed               */
  int rk_stages;            /* time discretisation: 3 (or 0) the three-stage SSP-RK3; 5 the paper's  *
                             * five-stage third-order scheme (Sec. 2.1), read as Spiteri & Ruuth's  *
                             * SSP(5,3). Recording, frozen steps and the adjoint are of the 3-stage *
                             * scheme (HYDRO_EINVAL on a 5-stage context).                          */
} hydro_config;

/* Create a context for one grid: validates cfg (HYDRO_EINVAL on a bad field, an unpaired periodic
 * face or an axis face that is not x-lo of an (r,z) grid with x0 = 0), allocates the padded working
 * states and scratch on the current device, and binds the CUDA stream (cudaStream_t, NULL = legacy
 * default stream). *out receives the context; on failure *out is NULL. */
int hydro_init(const hydro_config* cfg, void* stream, hydro_ctx** out);

/* Release the context and all of its device memory (synchronises its stream). NULL is ignored. */
void hydro_destroy(hydro_ctx* ctx);

/* Message of the last failure on this context ("" if none). Valid until the next call on ctx. */
const char* hydro_last_error(hydro_ctx* ctx);

/* Rebind the context to another stream (interface plumbing; no counterpart in the paper). */
int hydro_set_stream(hydro_ctx* ctx, void* stream);

/* Advance U (device, [nfields][ny][nx], caller-owned) by nsteps SSP-RK3 steps in place (Sec. 2.1).
 * Each step takes dt from the CFL condition on U^n (Sec. 5.4) and the global Lax-Friedrichs speeds
 * alpha_x = max(|u| + c), alpha_y = max(|v| + c) from each stage's input. *t_inout (may be NULL) is
 * advanced by the sum of the steps' dt, accumulated in FP64 on the device; *dt_last (may be NULL)
 * receives the last dt. Returns HYDRO_ENONPHYSICAL if any stage produced a non-finite value,
 * rho <= 0 or p <= 0 (U then holds the state of the failing step). Synchronises the stream. */
int hydro_step(hydro_ctx* ctx, void* U, int nsteps, double* t_inout, double* dt_last);

/* Same as hydro_step (the update of Sec. 2.1) for a state in HOST memory, on the context's stream. Pinned (page-locked) memory is
 * used in place: the kernel that builds the padded working state reads it over the host link, and the
 * last stage of the last step runs in row bands while a second stream of the context copies each finished
 * band back into it (copy engine, overlapped with the next band). Pageable memory is copied to a device
 * buffer, stepped and copied back. */
int hydro_step_host(hydro_ctx* ctx, void* U_host, int nsteps, double* t_inout, double* dt_last);

/* Spatial operator L(U) = -(dF/dx + dG/dy) + S(U) of Eq. euler2D (Sec. 2.1) and the level-set right-hand
 * side -H_hat (Sec. 2.2), with the Lax-Friedrichs speeds given (not computed): L is a caller-owned device
 * array shaped like U. Asynchronous. */
int hydro_rhs(hydro_ctx* ctx, const void* U, double alpha_x, double alpha_y, void* L);

/* Conserved totals sum_cells U_f dV (f = 0..4; dV = dx dy, or 2 pi r_i dr dz in (r,z)) of a device
 * state -- the mass and energy whose relative changes the Gresho test reports (Sec. 5.2) -- accumulated
 * in FP64 in a fixed order (bitwise repeatable); out is a host array of 5. out[4] is 0 when nfields = 4.
 * Synchronises the stream. */
int conserved_totals(hydro_ctx* ctx, const void* U, double out[5]);

/* Totals of the state written by the last completed hydro_step / hydro_batch_step, accumulated by the
 * last stage kernel of each step. FP64 contexts: FP64 sums of U_f dV. FP32 contexts: each warp's cells of
 * a tile are summed in FP32 (U_f, times r_i in (r,z)), each warp's tile partials in a compensated FP32
 * sum (value plus error term), and those across the grid in FP64, dV applied once, so the result agrees
 * with conserved_totals to about 1e-7 of sum |U_f dV|. Atomics: the last bits may vary between runs. */
int hydro_last_totals(hydro_ctx* ctx, double out[5]);

/* Conserved totals of a device state WITHOUT allocating anything and without a context, for callers
 * that cannot call cudaMalloc (code in host callbacks or allocator hooks, processes with a fixed
 * memory pool, frameworks that forbid device allocation on their threads). The paper has no
 * counterpart: this is an interface addition. Same result definition as conserved_totals (FP64
 * sums of U_f dV in a fixed order, out[4] = 0 for nfields = 4); U is a device [nfields][ny][nx]
 * array of dtype; the domain (x0, x1, y0, y1) and geometry give dV; out is a host array of 5.
 * Scratch: a file-scope device array of 16384 x 5 + 5 doubles (655 KB) that every GPU loading the
 * library keeps until the process exits; hence ny <= 16384, else HYDRO_ESIZE (nothing launched).
 * Every call looks up that array's address in the current context (cheap once the module is loaded).
 * With lazy module loading (the CUDA default) the FIRST call in a context loads the library's device
 * code, and the driver places the array then: a caller that must not allocate at all makes one
 * warm-up call beforehand, outside its hook (or sets CUDA_MODULE_LOADING=EAGER). The call cannot be
 * used during stream capture: it reads the result back and synchronises the stream. All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. An error already pending in the calling thread's CUDA state is left in
 * place and reported as HYDRO_ECUDA without launching. Runs on `stream` and synchronises it. */
int conserved_totals_noalloc(const void* U, int nx, int ny, int nfields, int dtype, int geometry, double x0,
                             double x1, double y0, double y1, void* stream, double out[5]);

/* Level-set reinitialisation of phi (field 4 of a device state with nfields = 5), in place (Sec. 2.2):
 * the front points are the linear-interpolation zeros of phi along every pair of neighbouring cells (in
 * x and in y, inside the grid) whose values lie on opposite sides of zero (> 0 ash, <= 0 fuel); every
 * cell's distance d to the front is its smallest distance to those points (Euclidean, no periodic
 * images); phi_new = H(d) phi_old + (1 - H(d)) sign(phi_old) d with H(d) = [1 - tanh((d - d0)/(Delta/3))]
 * / [1 - tanh(-d0/(Delta/3))], d0 = 3 Delta, Delta = min(dx, dy). phi is unchanged when there is no
 * front. Cost O(cells x front points). *npoints (may be NULL) receives the number of front points.
 * Allocates its point buffer (2 points per cell) on first use. Synchronises the stream. */
int hydro_reinit(hydro_ctx* ctx, void* U, int* npoints);

/* Measured fused multiply-add throughput of the context's GPU in dtype (HYDRO_F32 or HYDRO_F64): every
 * thread of 8 x 256 threads per SM runs 8 independent FMA chains of 16 x iters FMAs; *fma_per_s receives
 * FMAs per second (a flop rate is twice that). The cross-check of the arithmetic roofline. Allocates and
 * frees 8 bytes; synchronises the stream. */
int hydro_fma_probe(hydro_ctx* ctx, int dtype, int iters, double* fma_per_s);

/* Self-test of the device failure path: one thread runs the stage kernel's bounded wait on an mbarrier
 * that nothing completes, for `polls` polls (1 .. 2^24; ~2^20 take a few milliseconds), and the call
 * returns what a lost tile copy returns: HYDRO_ETIMEOUT ("a device wait gave up"). No GPU state is left
 * behind and the context stays usable. HYDRO_EINVAL for polls outside the range. Synchronises the
 * stream. */
int hydro_wait_selftest(hydro_ctx* ctx, unsigned polls);

/* Self-gravity potential Phi of the density rho = U[0] on an (r,z) grid (geometry 1), Sec. 2.1:
 * (1/r) d/dr (r dPhi/dr) + d2Phi/dz2 = 4 pi G rho, solved by successive over-relaxation of red-black
 * Gauss-Seidel sweeps (red: i + j even, then black) with
 *   Phi_GS = (aE Phi_E + aW Phi_W + aN Phi_N + aS Phi_S - 4 pi G rho) / (aE + aW + aN + aS),
 *   aE = r_{i+1/2} / (r_i dr^2), aW = r_{i-1/2} / (r_i dr^2), aN = aS = 1 / dz^2,
 *   Phi <- (1 - omega) Phi + omega Phi_GS,
 * every operation rounded once in that order (FP64 whatever the state's dtype). Inner boundaries
 * reflect: the x-lo face (the axis, where aW = 0 at r = 0, or a wall) and the y-lo face when its bc is
 * HYDRO_BC_REFLECT (the missing neighbour is the cell's own value). The other faces hold the Roche value
 * -G M / sqrt(r^2 + z^2) at the ghost cell centre, M the mass, doubled when y-lo reflects (a z = 0
 * symmetry plane). The mass of the grid, sum of rho 2 pi r dr dz with each term rounded in that order,
 * is summed exactly and rounded once (correctly rounded, independent of summation order).
 * The sweeps stop after the first sweep in which every cell's relative change |new - old| / |new| is
 * below tol (cells with 0/0 are ignored), or after max_iters sweeps; tol <= 0 runs exactly max_iters.
 *   U        device state [nfields][ny][nx] (only the rho plane is read)
 *   phi      device double [ny][nx]: the initial guess on entry, the potential on exit (caller-owned)
 *   omega    relaxation factor, 0 < omega < 2
 *   iters    (may be NULL) receives the sweeps done; mass (may be NULL) the grid mass (not doubled)
 * Errors: HYDRO_EINVAL for a Cartesian grid, null pointers, omega outside (0, 2), max_iters < 0, ny >
 * 131070; HYDRO_ESIZE beyond 2^31 - 1 cells; HYDRO_ENONPHYSICAL when rho holds inf or NaN (phi is then
 * NaN). Allocates its work arrays (5 nx + ny doubles and a few KB) on first use. Synchronises the stream. */
int hydro_poisson(hydro_ctx* ctx, const void* U, double G, double omega, double tol, int max_iters, double* phi,
                  int* iters, double* mass);

/* Correctly rounded sum of n device doubles x (round to nearest, ties to even, once): the terms are added
 * exactly into a fixed-point long accumulator, so the result does not depend on the order of summation.
 * It is the summation the Poisson solve uses for its mass. *out is a host double. Errors: HYDRO_ESIZE
 * for n > 2^31 - 1; HYDRO_ENONPHYSICAL (and *out = NaN) when a term is inf or NaN. Allocates on first
 * use like hydro_poisson. Synchronises the stream. */
int hydro_exact_sum(hydro_ctx* ctx, const double* x, long long n, double* out);

/* ---- recording and the discrete adjoint (frozen alpha and dt) ---------------------------------
 * The paper has no adjoint: these entry points are the exact discrete adjoint (reverse mode) of the
 * component-wise update of Sec. 2.1 / 2.2 as this library computes it. alpha_x, alpha_y and dt are
 * maxima/minima over the grid and have no derivative; the adjoint and the finite-difference checks
 * freeze them at the values the forward run used. The characteristic scheme has no adjoint here:
 * HYDRO_EINVAL on such a context. lambda arrays are caller-owned device arrays shaped like U. */

/* Start recording: the next steps log dt (one double per step) and the stage alphas (six doubles per
 * step) for up to max_steps steps. max_steps = 0 stops recording and frees the log. */
int hydro_record(hydro_ctx* ctx, int max_steps);
/* Copy the first n logged entries to host arrays dt_log[n], alpha_log[6n]. Returns the number of
 * steps recorded so far through *n_recorded (may be NULL). HYDRO_EINVAL for n beyond the recorded
 * count or null arrays with n > 0. Synchronises the stream. */
int hydro_get_log(hydro_ctx* ctx, int n, double* dt_log, double* alpha_log, int* n_recorded);

/* Forward map (Sec. 2.1) with dt and stage alphas frozen at host-given values (nsteps entries /
 * 6*nsteps host doubles). HYDRO_EINVAL for null arrays with nsteps > 0. */
int hydro_step_frozen(hydro_ctx* ctx, void* U, int nsteps, const double* dt_log, const double* alpha_log);

/* Discrete adjoint of one frozen SSP-RK3 step: lambda (device, shaped like U) holds dJ/dU^{n+1} on
 * entry and dJ/dU^n on exit; U_n is the step's input state; alpha holds (alpha_x, alpha_y) of the
 * three stages. The stage states are recomputed from U_n. */
int hydro_adjoint_step(hydro_ctx* ctx, const void* U_n, void* lambda, double dt, const double alpha[6]);

/* Forward run of nsteps steps from U (device, advanced in place to U^N) keeping checkpoints for a
 * later reverse sweep: every checkpoint_every-th state is stored in library memory (checkpoint_every
 * <= 0 picks sqrt(nsteps)), and dt / alphas are recorded. */
int hydro_forward_checkpointed(hydro_ctx* ctx, void* U, int nsteps, int checkpoint_every);
/* Reverse sweep over the last checkpointed forward run: lambda holds dJ/dU^N on entry and dJ/dU^0 on
 * exit. Segments are recomputed from their checkpoints (two-level checkpointing); the stored run is
 * kept, so the sweep may be repeated for another lambda. HYDRO_ESTATE when no checkpointed run exists. */
int hydro_adjoint_sweep(hydro_ctx* ctx, void* lambda);

/* Forward run of nsteps steps from U (advanced in place to U^N) for a reverse sweep on a binomial
 * checkpoint schedule (revolve: Griewank & Walther, ACM TOMS 26, 2000) under a memory budget: only U^0
 * and the recorded dt / alphas are kept; the next hydro_adjoint_sweep reverses the run with `snapshots`
 * (0 .. 4096) further state slots, recomputing forward segments from the nearest stored state, and takes
 * the least recomputation that budget allows (with s slots and t sweeps over the run, C(s + t, s) steps can
 * be reversed). Device memory: snapshots + 2 states. *sweep_forward_steps (may be NULL) receives the
 * forward steps the sweep will recompute. The adjoint steps see the same states as under
 * hydro_forward_checkpointed, so the gradient is the same, bit for bit. HYDRO_EINVAL for bad arguments or a
 * characteristic-scheme context. */
int hydro_forward_revolve(hydro_ctx* ctx, void* U, int nsteps, int snapshots, long long* sweep_forward_steps);

/* ---- batched ensembles ------------------------------------------------------------------------ */

/* Advance nmembers independent grids (each with its own context, all of one dtype and nfields) by
 * nsteps steps of the update of Sec. 2.1 (each member its own alphas and dt): each RK stage of all members is ONE persistent kernel launch that walks a table of
 * (member, tile) work items; the three launches of a step are replayed from a CUDA graph. U[m] is
 * member m's device state, t[m] (host, may be NULL) its time. Runs on members[0]'s stream. The work table
 * and graph are kept on members[0] and reused while the same contexts (by identity, not address) with
 * unchanged parameters come back in the same order; any other call, or a member whose parameters changed
 * (hydro_record, hydro_set_tile_variant, hydro_autotune), rebuilds them. HYDRO_EINVAL when members differ
 * in dtype, nfields or device, or use the characteristic scheme; a member's non-physical state or device
 * timeout is reported with its index in hydro_last_error(members[0]). Synchronises the stream. */
int hydro_batch_step(hydro_ctx* const* members, void* const* U, int nmembers, int nsteps, double* t);

/* ---- tuning and timing ------------------------------------------------------------------------
 * Performance plumbing with no counterpart in the paper; results of the update do not depend on the
 * tile variant (bitwise). */

/* Number of tile variants and the current one; select a variant (0 .. n-1) for this context
 * (HYDRO_EINVAL for no such variant or one that does not fit on the device). A new context starts with
 * variant 2 (60 x 30 cells, 640 threads) for component-wise FP32 grids of at least one such tile per SM,
 * else 1. */
int hydro_tile_variants(hydro_ctx* ctx, int* n, int* current);
/* Tile rows of the discrete adjoint's line kernel for this context: 16 (two CTAs of 16 x 32 output points
 * per SM), 32 (FP32 only: one CTA of 32 x 32 per SM), or 0 (the default: 32 in FP32 where the padded grid
 * holds at least one 32 x 32 tile per SM, else 16). Every choice gives the same bits. HYDRO_EINVAL for
 * another value. */
int hydro_set_adjoint_tile_rows(hydro_ctx* ctx, int rows);
int hydro_set_tile_variant(hydro_ctx* ctx, int variant);
/* Describe a variant: tile width and height in cells, threads per CTA, shared memory bytes. */
int hydro_tile_info(hydro_ctx* ctx, int variant, int* tile_x, int* tile_y, int* threads, int* smem_bytes);
/* Time every variant on a copy of U (device; U is not modified) for `steps` steps each and keep the
 * fastest; per-variant milliseconds per step go to ms_out[n] (may be NULL). */
int hydro_autotune(hydro_ctx* ctx, const void* U, int steps, double* ms_out);

/* Autotuner of a batched ensemble's plan (the members and states of hydro_batch_step). Times, on the
 * batch's own mixed-size work list, every combination of tile variant v (0 .. 2), persistent grid size w
 * (0: one wave of resident CTAs, 1: two waves) and work-list layout l (0: each CTA a contiguous run of
 * the member-ordered tiles, row by row; 1: the same run with each member's tiles column by column; 2: the
 * tiles dealt out one by one), `steps` graph-replayed steps each after one untimed step, on the members'
 * working copies: U is read, never written. Keeps the fastest as the plan of later hydro_batch_step calls
 * with these members (members[0] holds it). ms_out[18] (may be NULL) receives ms per step of trial
 * (v * 2 + w) * 3 + l, -1 where the variant does not fit; *best (may be NULL) the trial kept. Errors as
 * hydro_batch_step; a non-physical state does not stop the timing. Synchronises the stream. */
int hydro_batch_autotune(hydro_ctx* const* members, void* const* U, int nmembers, int steps, double* ms_out,
                         int* best);

/* Per-launch timing of the stage kernels: with enable = 1, every stage launch is bracketed by CUDA
 * events on the context's stream; hydro_stage_timing returns the launches and the summed device time
 * since the last enable (synchronises the stream). */
int hydro_profile(hydro_ctx* ctx, int enable);
int hydro_stage_timing(hydro_ctx* ctx, int* launches, double* total_ms);

/* Number of kernel launches the library issued on this context since it was created. */
long long hydro_launch_count(hydro_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_H */
