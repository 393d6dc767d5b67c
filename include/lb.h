/*
 * lb.h - C ABI of the GB300 (sm_103a) library for the tunable-surface-tension
 * pseudopotential lattice Boltzmann method of Li & Luo (arXiv 1306.6445).
 *
 * One context = one D2Q9 lattice of nx * ny sites on one GPU. Each call of
 * lb_step advances it by whole time steps of the MRT pseudopotential update:
 *   rho = sum f, psi(rho)                          (Sec. II, Eq. 6 and text after Eq. 7)
 *   F = -G psi(x) sum_a w_a psi(x + e_a) e_a      (Eq. 7, w(1) = 1/3, w(2) = 1/12)
 *   Q = kappa G/2 psi(x) sum_a w_a [psi(x + e_a) - psi(x)] e_a e_a     (Eq. 19)
 *   rho v = sum e f + F/2                          (Eq. 6)
 *   m* = m - Lambda (m - m_eq) + (I - Lambda/2) S + C                  (Eq. 17)
 *     with m_eq of Eq. 3, S of Eq. 5 whose S_1 is Eq. 8, C of Eq. 18
 *   f* = M^-1 m*, then streaming f_a(x + e_a, t + 1) = f*_a(x, t)      (Eq. 4)
 * Lattice units c = delta_x = delta_t = 1, c_s^2 = 1/3.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Velocities e_0..e_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
 * - Host field arrays are row-major [y][x] (x fastest), nx * ny doubles, owned by
 *   the caller. Host population arrays are [alpha][y][x], 9 * ny * nx elements of
 *   the context's storage type (double for LB_FP64, float for LB_FP32, and for LB_BF16 the
 *   16-bit stored patterns of f_a - w_a rho_s, see lb_prec).
 * - Populations are stored on the device as 9 planes of ny rows of `pitch`
 *   elements (pitch = lb_pitch(nx, prec) >= nx + 2 H, a multiple of 32 elements, with
 *   H = 8 for LB_FP32 and 4 for LB_FP64 and LB_BF16). Column x of a row sits at element
 *   x + H; elements H-2, H-1 and nx+H, nx+H+1 hold periodic images of columns nx-2, nx-1
 *   and 0, 1 (copies of the edge columns for LB_BC_OPEN). The stored array is the state
 *   g from which the populations of the current time are PULLED,
 *   f_a(x, t) = g_a(x - e_a) (bounce-back at walls), i.e. the post-collision values
 *   of the previous step before streaming. lb_get/set_populations convert.
 * - Every function returns an lb_status; nothing throws across the ABI. After
 *   LB_ENONFINITE, LB_EDOMAIN or LB_ETIMEOUT the context is poisoned: every later
 *   call except lb_free / lb_last_error / lb_status_of returns that code again.
 * - Calls on one context are not thread-safe. Work is queued on the context's
 *   stream; calls that return data to the host synchronise that stream.
 */
#ifndef PAPER_1306_6445_GB300_LB_H
#define PAPER_1306_6445_GB300_LB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,      /* bad argument (sizes, rates, kappa, buffer size, ...) */
    LB_ENOMEM = 2,      /* device or host allocation failed */
    LB_ECUDA = 3,       /* a CUDA runtime call failed (message in lb_last_error) */
    LB_ENONFINITE = 4,  /* a reduction found a non-finite mass or momentum */
    LB_EDOMAIN = 5,     /* psi^2 < 0 or rho <= 0 at some site: EOS left its real branch */
    LB_ETIMEOUT = 6     /* a bounded device-side wait gave up */
} lb_status;

typedef enum { LB_EOS_CS = 0, LB_EOS_EXP = 1, LB_EOS_PIECEWISE = 2 } lb_eos_kind;
/* Storage / arithmetic precision of a context's populations:
 *  LB_FP64, LB_FP32: stored and computed in that type;
 *  LB_BF16: stored as BF16 (round to nearest even, or stochastically) of the shifted
 *           population f_a - w_a rho_s, w = 4/9, 1/9 (a = 1..4), 1/36 (a = 5..8), rho_s set
 *           by lb_set_storage_shift (default 0); a step computes in FP32 on the shifted
 *           values (the shift enters the moments rho, e and zeta), and f_a = float(stored)
 *           + w_a rho_s everywhere else. Single contexts only (not batches). */
typedef enum { LB_FP64 = 0, LB_FP32 = 1, LB_BF16 = 2 } lb_prec;
/* Boundaries: LB_BC_PERIODIC in x and y; LB_BC_WALLS_Y periodic in x with half-way
 * bounce-back (no-slip) walls below row 0 and above row ny-1 (Sec. V.B); LB_BC_OPEN a
 * bounce-back wall below row 0 and open boundaries above row ny-1 and beyond columns 0 and
 * nx-1, where a population entering the lattice is taken from the nearest lattice site
 * (zero gradient), and psi outside the lattice is that of the nearest site: the
 * droplet-splash geometry of Sec. V.C, whose open condition the paper does not name.
 * LB_BC_OPEN is compiled for LB_FP32 and LB_FP64 and supports lb_set_viscosity_switch. */
typedef enum { LB_BC_PERIODIC = 0, LB_BC_WALLS_Y = 1, LB_BC_OPEN = 2 } lb_bc;

/* Equation of state / pseudopotential (Sec. II; Eq. 23).
 *  LB_EOS_CS:        p = rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2, eta = b rho/4;
 *                    psi = sqrt(2 (p - rho/3) / G)
 *  LB_EOS_EXP:       psi = psi0 exp(-rho0 / rho)
 *  LB_EOS_PIECEWISE: p of Eq. 23 with theta_v, theta_m, theta_l, rho1, rho2;
 *                    psi = sqrt(2 (p - rho/3) / G)                                   */
typedef struct {
    int kind;                              /* lb_eos_kind */
    double a, b, R, T;                     /* Carnahan-Starling */
    double psi0, rho0;                     /* exponential potential */
    double theta_v, theta_m, theta_l, rho1, rho2;  /* Eq. 23 */
} lb_eos;

/* Relaxation rates s = 1/tau of Lambda = diag(s_rho, s_e, s_zeta, s_j, s_q, s_j, s_q, s_v, s_v)
 * (Sec. II, text after Eq. 1). Each must lie in (0, 2). */
typedef struct {
    double s_rho, s_e, s_zeta, s_j, s_q, s_v;
} lb_rates;

typedef struct lb_ctx lb_ctx;

/* Row pitch (elements) of the device population planes for a lattice of width nx. */
size_t lb_pitch(int nx, int prec);

/* Bytes of ONE device population buffer: 9 * ny * lb_pitch(nx, prec) * element size. */
size_t lb_buffer_bytes(int nx, int ny, int prec);

/* Create a context and allocate its two device population buffers (ping-pong).
 *  nx, ny       lattice size, each >= 3.
 *  eos, G       pseudopotential and interaction strength of Eq. 7 (G != 0 for the
 *               EOS-based potentials, which divide by G).
 *  kappa        surface-tension parameter of Eq. 19, in [0, 1).
 *  sigma_force  the constant sigma of Eq. 8 (>= 0; 0 gives the forcing of Eq. 5).
 *               When it is non-zero the paper requires s_zeta == s_e (text after Eq. 8).
 *  rates        relaxation rates, each in (0, 2).
 *  prec         LB_FP64 or LB_FP32 (storage and arithmetic type of the update).
 *  bc           LB_BC_PERIODIC, or LB_BC_WALLS_Y: periodic in x, no-slip walls below
 *               row 0 and above row ny-1 (half-way bounce-back; psi of the adjacent
 *               fluid row is used at the wall, Sec. V.B names no scheme).
 *  stream       a cudaStream_t to queue work on, or NULL for the legacy default stream.
 * The populations are left uninitialised: call lb_set_rho_u or lb_set_populations.
 * Errors: LB_EINVAL for any argument outside the ranges above, LB_ENOMEM, LB_ECUDA. */
lb_status lb_init(lb_ctx **out, int nx, int ny, const lb_eos *eos, double G, double kappa,
                  double sigma_force, const lb_rates *rates, int prec, int bc, void *stream);

/* As lb_init, but the two device population buffers belong to the caller (for example
 * memory from a tensor library). Each must hold lb_buffer_bytes(nx, ny, prec) bytes,
 * be 256-byte aligned and stay valid until lb_free. The library never frees them.
 * Errors: as lb_init, plus LB_EINVAL for NULL or misaligned buffers. */
lb_status lb_init_ex(lb_ctx **out, int nx, int ny, const lb_eos *eos, double G, double kappa,
                     double sigma_force, const lb_rates *rates, int prec, int bc, void *stream,
                     void *f_a, void *f_b);

/* Number of compiled variants of the step kernel: strip width x shared-memory ring depth
 * x ring kind. Variants 0-3 stage whole stored rows of the strip (all nine populations,
 * three rows in use at a time); variants 4-6 stage, per psi row, exactly the three plane
 * groups that row is pulled from (one stage in use at a time, so more CTAs fit on an SM).
 * Every variant gives identical results. Contexts and batches start with variant 4. */
int lb_launch_variants(void);

/* Density-dependent viscosity of Sec. V.C (LB_BC_OPEN contexts): sites with rho < rho_1
 * relax the viscous moments p_xx, p_xy at s_v_vapour (the vapour viscosity
 * (1/s_v_vapour - 1/2)/3), the others at the context's s_v; rho is the site density of
 * the step (Eq. 6). Off until called. Synchronises. Errors: LB_EINVAL for another boundary
 * kind, a non-finite rho_1 or s_v_vapour outside (0, 2). */
lb_status lb_set_viscosity_switch(lb_ctx *ctx, double rho_1, double s_v_vapour);

/* rho_s of the LB_BF16 storage shift (stored value = BF16(f_a - w_a rho_s)). Call it before
 * lb_set_rho_u / lb_set_populations: populations already stored keep their bits and are
 * read with the new shift. A rho_s near the density of most sites keeps the stored
 * differences small (BF16 keeps 8 significant bits). Synchronises. Errors: LB_EINVAL for a
 * context that is not LB_BF16 or a non-finite rho_s. */
lb_status lb_set_storage_shift(lb_ctx *ctx, double rho_s);

/* Rounding of the values an LB_BF16 step stores (f_a - w_a rho_s, FP32, to BF16).
 * LB_ROUND_NEAREST (the default): round to nearest even. LB_ROUND_STOCHASTIC: the magnitude
 * rounds up with probability (dropped bits) / 2^16, so each stored value is unbiased; the
 * random bits come from a counter-based generator (MurmurHash3's 32-bit finaliser) keyed by
 * the site, the step count and the population, so runs are reproducible and do not depend
 * on the launch variant. The initial state of lb_set_rho_u is rounded to nearest. Library
 * plumbing for the precision study (the paper has no counterpart). Synchronises.
 * Errors: LB_EINVAL for a context that is not LB_BF16 or an unknown mode. */
enum { LB_ROUND_NEAREST = 0, LB_ROUND_STOCHASTIC = 1 };
lb_status lb_set_storage_rounding(lb_ctx *ctx, int mode);

/* Choose the step kernel's variant (0 .. lb_launch_variants()-1) and the number of rows
 * each CTA marches over (rows = 0: about three waves of resident CTAs, at least 8 rows).
 * Synchronises the stream. Errors: LB_EINVAL for an unknown variant or rows < 0. */
lb_status lb_set_launch(lb_ctx *ctx, int variant, int rows);

/* Autotuner: time every compiled variant with rows per CTA from {default, 6, 8, 9, 10,
 * 11, 12, 13, 14, 15, 16, 20, 24} (at most ny) on this lattice and keep the fastest. Each
 * candidate runs one untimed launch and then three timed runs of `trial_steps` >= 1
 * launches (its time is the fastest run). The trial launches take real steps on a scratch
 * copy of the state (a temporary device buffer of lb_buffer_bytes, freed before return),
 * ping-ponging with the spare buffer in the alternating visiting order of lb_step, so every
 * candidate meets the cache reuse of real stepping; without memory for the copy they read
 * the state and write the spare buffer. The state is only read, so the state and the step
 * count are unchanged. Per-site results do not depend on the choice. Writes the choice
 * if the pointers are not NULL. Synchronises. Errors: LB_EINVAL, LB_ECUDA, and the
 * sticky errors of lb_sync. */
lb_status lb_autotune(lb_ctx *ctx, int trial_steps, int *variant, int *rows);

/* Current launch: variant, lattice columns per CTA, rows per CTA, resident CTAs per SM. */
lb_status lb_get_launch(const lb_ctx *ctx, int *variant, int *tx, int *rows, int *ctas_per_sm);

/* Test hook for the failure path of the bounded device-side waits: from the next lb_step
 * on, the step kernel never requests lattice row `row` (as staged in its shared-memory
 * ring), so the CTAs that need it give up after about one second and the next
 * synchronising call returns LB_ETIMEOUT. Nothing faults and no copy is left in flight.
 * INT_MIN (the default) switches it off. Not part of the method; for tests only. */
lb_status lb_debug_stall_row(lb_ctx *ctx, int row);

/* f = f_eq(rho, u) = M^-1 m_eq(rho, u) of Eq. 3 at every site (the initial state).
 * rho, ux, uy: host arrays of nx*ny doubles, [y][x]. The step counter is reset to 0.
 * Synchronises the stream. Errors: LB_EINVAL (NULL), LB_EDOMAIN if psi(rho) is not real
 * and positive at some site (rho <= 0, or (p_EOS - rho/3)/G <= 0), LB_ECUDA. */
lb_status lb_set_rho_u(lb_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* Advance n >= 0 time steps (Eqs. 4-8, 17-19), one kernel launch per step. Queued on the
 * stream; returns without waiting. A psi-domain violation found on the device is reported
 * by the next call that synchronises (lb_sync, lb_get_*, lb_reduce) as LB_EDOMAIN; a
 * device-side wait that gave up (about one second) as LB_ETIMEOUT. */
lb_status lb_step(lb_ctx *ctx, int n);

/* Wait for queued work and report device-side errors (LB_EDOMAIN, LB_ECUDA). */
lb_status lb_sync(lb_ctx *ctx);

/* Density rho = sum_a f_a (Eq. 6) into a host array of nx*ny doubles. Synchronises. */
lb_status lb_get_rho(lb_ctx *ctx, double *rho);

/* Velocity v = (sum_a e_a f_a + F/2) / rho (Eq. 6, with F of Eq. 7) into two host arrays
 * of nx*ny doubles. Synchronises. */
lb_status lb_get_u(lb_ctx *ctx, double *ux, double *uy);

/* Copy the current populations to / from a packed host array [alpha][y][x] of
 * 9*ny*nx elements of the storage type; `bytes` must equal that size exactly.
 * The array travels as one contiguous copy through the context's spare device buffer,
 * where a kernel converts between the host layout and the stored state.
 * lb_set_populations resets nothing else (the step counter is kept). Both synchronise.
 * Errors: LB_EINVAL on a size mismatch or NULL, LB_ECUDA. */
lb_status lb_get_populations(lb_ctx *ctx, void *dst, size_t bytes);
lb_status lb_set_populations(lb_ctx *ctx, const void *src, size_t bytes);

/* Global diagnostics in FP64 with a fixed reduction order (bit-reproducible):
 * out[0] = sum rho, out[1] = sum rho v_x, out[2] = sum rho v_y (v of Eq. 6),
 * out[3] = max |v|. Synchronises. LB_ENONFINITE (and poisoning) if any is not finite. */
lb_status lb_reduce(lb_ctx *ctx, double out[4]);

/* lb_reduce without any device allocation, for callers that cannot allocate: for
 * example a plugin confined to a device-memory budget given to it by its host
 * application, or a loop that must not call cudaMalloc/cudaFree because they can
 * synchronise the whole device. The paper has no counterpart; this is library plumbing.
 * Same outputs as lb_reduce (out[0] = sum rho, out[1..2] = sum rho v, out[3] = max |v|,
 * FP64, fixed reduction order), written to the caller's host array; synchronises the
 * context's stream. Its scratch is one static device array of 4104 doubles (32.8 KB) that
 * every GPU loading this library holds until the process exits; lattices of at most
 * 2^24 sites are accepted (LB_EINVAL with a message otherwise). The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress), so make that first
 * call before any stream capture. All calls share the array: calls that overlap on the
 * GPU (for example on two streams) race and must be serialised by the caller.
 * Errors: as lb_reduce (LB_EDOMAIN, LB_ENONFINITE poison the context), LB_ECUDA, and
 * LB_EINVAL for an LB_BF16 or LB_BC_OPEN context (use lb_reduce). Errors that kernels queued
 * before this call recorded in the context (LB_ETIMEOUT, LB_EDOMAIN) are returned and poison
 * the context exactly as in lb_reduce. */
lb_status lb_reduce_noalloc(lb_ctx *ctx, double out[4]);

/* Laplace-law measurement of a droplet centred at ((nx-1)/2, (ny-1)/2) (Sec. V.A), on the
 * GPU from the current state: FP64 sums over all sites in a fixed order (the same bits on
 * every call), with the definitions of lb_batch_measure. radius: nominal droplet radius,
 * used only for the masks (inside r < radius/2, outside r > radius + 0.3 min(nx, ny)/2).
 * out[0] = theta = (p_in - p_out) R, 1 = rho_in, 2 = rho_out (mask means), 3 = R from the
 * mass, sqrt((M - rho_out N) / (pi (rho_in - rho_out))), 4 = p_in, 5 = p_out (means of
 * p = rho/3 + G psi^2/2, the bulk part of Eq. 20), 6 = M = total mass, 7 = 1 if a site has
 * a non-finite density or pressure or psi off its real branch (else 0). The context is
 * not poisoned by a failed measurement. Synchronises.
 * Errors: LB_EINVAL for a NULL out or a radius that is not positive and finite, LB_ENOMEM,
 * LB_ECUDA, and the sticky errors of lb_sync. */
lb_status lb_measure_droplet(lb_ctx *ctx, double radius, double out[8]);

/* Height of the liquid-vapour interface in every column (Sec. V.B capillary wave), on
 * the GPU from the current state: heights[x] = (y - 1) + (rho(x, y-1) - rho_mid) /
 * (rho(x, y-1) - rho(x, y)) with y the lowest row whose density is below rho_mid (liquid
 * below the interface), the densities those of lb_get_rho; NaN where row 0 is already
 * below rho_mid or no row is. heights: caller-owned host buffer of nx doubles.
 * Synchronises. Errors: LB_EINVAL for a NULL buffer or a non-finite rho_mid, LB_ENOMEM,
 * LB_ECUDA, and the sticky errors of lb_sync. */
lb_status lb_interface_height(lb_ctx *ctx, double rho_mid, double *heights);

/* Number of time steps taken since lb_set_rho_u. */
long long lb_steps_done(const lb_ctx *ctx);

/* Number of kernel launches one lb_step(ctx, 1) queues (for launch accounting). */
int lb_kernels_per_step(const lb_ctx *ctx);

/* Last error message of the context (static string "no context" for NULL). */
const char *lb_last_error(const lb_ctx *ctx);

/* Sticky status of the context (LB_OK unless poisoned). */
lb_status lb_status_of(const lb_ctx *ctx);

/* Release the context and the device memory the library allocated. NULL is a no-op. */
void lb_free(lb_ctx *ctx);

/* ---------------------------------------------------------------------------------
 * Batched lattices: many independent periodic lattices of uneven size and parameters
 * (for example a sweep of droplets over temperature, kappa and viscosity) advanced
 * together. Each time step is ONE launch of a persistent kernel whose CTAs walk a fixed
 * list of work items (lattice, strip, row block); runs of 64 steps are captured once in a
 * CUDA graph and replayed. The update of each lattice is the one of lb_step (Eqs. 4-8,
 * 17-19), bit for bit. All lattices share the precision and the EOS kind.
 * --------------------------------------------------------------------------------- */
typedef struct {
    int nx, ny;                        /* lattice size, each >= 3 (periodic in x and y) */
    lb_eos eos;                        /* same kind for every lattice of a batch */
    double G, kappa, sigma_force;      /* as in lb_init */
    lb_rates rates;
} lb_lattice_desc;

typedef struct lb_batch lb_batch;

/* How a lattice of width nx is cut into strips of at most tx columns (tx a multiple of 4)
 * for the batched step: ceil(nx/tx) strips whose widths differ by at most 7 and all start
 * on a multiple of 4 columns (only the last width may be any size). Writes the widths and
 * returns the strip count, or -1 for bad arguments or too small a `widths` array. Host only. */
int lb_strip_widths(int nx, int tx, int *widths, int max_strips);

/* Create a batch of n lattices (device memory for all populations in one allocation).
 * Errors: LB_EINVAL (mixed EOS kinds or any argument lb_init would reject), LB_ENOMEM,
 * LB_ECUDA. The populations start at zero: set every lattice with lb_batch_set_rho_u. */
lb_status lb_batch_create(lb_batch **out, int n, const lb_lattice_desc *descs, int prec,
                          void *stream);

/* f = f_eq(rho, u) (Eq. 3) for lattice i from host arrays of nx*ny doubles, [y][x].
 * Synchronises. Errors: LB_EINVAL, LB_EDOMAIN (psi not real at some site), LB_ECUDA. */
lb_status lb_batch_set_rho_u(lb_batch *b, int i, const double *rho, const double *ux,
                             const double *uy);

/* Advance every lattice n >= 0 time steps (queued; returns without waiting). */
lb_status lb_batch_step(lb_batch *b, int n);

/* Wait for queued work. LB_ETIMEOUT (and poisoning) if a bounded device wait gave up;
 * per-lattice psi-domain errors do not stop the batch (see lb_batch_errors). */
lb_status lb_batch_sync(lb_batch *b);

/* Per-lattice error bits (1 = psi domain left, 2 = wait timed out) into flags[n]. */
lb_status lb_batch_errors(lb_batch *b, int *flags);

/* Density of lattice i (Eq. 6) into a host array of nx*ny doubles. Synchronises. */
lb_status lb_batch_get_rho(lb_batch *b, int i, double *rho);

/* Populations of lattice i ([alpha][y][x], 9*ny*nx elements of the storage type; `bytes`
 * must match). Synchronises. */
lb_status lb_batch_get_populations(lb_batch *b, int i, void *dst, size_t bytes);

/* Laplace-law measurement of every lattice on the GPU (FP64 sums in a fixed order).
 * radius[i]: nominal droplet radius of lattice i (droplet centred at ((nx-1)/2, (ny-1)/2)).
 * Writes 8 doubles per lattice: out[8i + 0] = theta = (p_in - p_out) R (Laplace law,
 * Sec. V.A), 1 = rho_in (mean over r < R/2), 2 = rho_out (mean over r > R + 0.3 min(nx,ny)/2),
 * 3 = R from the mass, 4 = p_in, 5 = p_out (p = rho/3 + G psi^2/2, the bulk part of
 * Eq. 20), 6 = total mass, 7 = 1 if the lattice failed (non-finite, psi domain), else 0.
 * Synchronises. */
lb_status lb_batch_measure(lb_batch *b, const double *radius, double *out);

/* Time a few steps of every compiled variant and rows-per-item choice in {8, 12, 16, 24,
 * 32} on this batch and keep the fastest. The trial launches take real steps of the
 * current states (set them first: the cost of a step depends on the state), after the
 * populations, per-lattice error flags, phase and step count have been saved to a
 * temporary device buffer the size of the batch's pool; they are restored afterwards, so
 * the batch is unchanged. Writes the choice if the pointers are not NULL. Synchronises.
 * Errors: LB_EINVAL, LB_ENOMEM (no room for the copy; nothing changed), LB_ECUDA. */
lb_status lb_batch_autotune(lb_batch *b, int trial_steps, int *variant, int *rows);

/* Choose the variant and rows per work item directly; report the current launch. */
lb_status lb_batch_set_launch(lb_batch *b, int variant, int rows);
lb_status lb_batch_get_launch(const lb_batch *b, int *variant, int *rows, int *grid,
                              int *items);

/* Choose which lattices lb_batch_step advances (active[i] != 0), for example to stop the
 * lattices that have converged while the others run on; an inactive lattice keeps its
 * state, can still be read and measured, and can be made active again. All lattices start
 * active. Must be called when the batch's step count is even (every multiple of 64 steps
 * is); rebuilds the work list and drops the captured graphs. Synchronises.
 * Errors: LB_EINVAL (NULL or an odd step count), LB_ENOMEM, LB_ECUDA. Library plumbing
 * (the paper has no counterpart). */
lb_status lb_batch_set_active(lb_batch *b, const unsigned char *active);

/* Steps lattice i has been advanced (it is not advanced while inactive); -1 for a bad i. */
long long lb_batch_lattice_steps(const lb_batch *b, int i);

/* Steps of the batch as a whole (every lb_batch_step call counts, active lattices or not). */
long long lb_batch_steps_done(const lb_batch *b);
int lb_batch_size(const lb_batch *b);
const char *lb_batch_last_error(const lb_batch *b);
void lb_batch_free(lb_batch *b);

/* ---------------------------------------------------------------------------------
 * Measurement (no counterpart in the paper).
 * --------------------------------------------------------------------------------- */

/* FP64 fused multiply-add throughput of the current device, the ALU roof of the LB_FP64
 * update: 8 blocks of 256 threads per SM, each thread running 8 independent chains of
 * `iters` FP64 FMAs, timed with CUDA events on `cuda_stream` (a cudaStream_t, or NULL for
 * the legacy default stream) after one untimed launch. *fma_per_s receives FP64 FMA
 * thread instructions per second (one FMA = 2 flops). iters = 4096 runs about 15 ms on a
 * GPU with GB300's FP64 rate. Synchronises the stream.
 * Errors: LB_EINVAL for iters < 1 or a NULL output, LB_ENOMEM, LB_ECUDA. */
lb_status lb_probe_fp64_fma_rate(void *cuda_stream, int iters, double *fma_per_s);

/* ---------------------------------------------------------------------------------
 * Host-side thermodynamic set-up helpers (no GPU work). They give the Carnahan-
 * Starling critical point and the Maxwell coexistence densities used to build
 * initial droplets (Sec. II; the Maxwell rule is equal area in 1/rho).
 * --------------------------------------------------------------------------------- */

/* Critical temperature and density of the Carnahan-Starling EOS with a, b, R.
 * Errors: LB_EINVAL for non-positive a, b or R. */
lb_status lb_cs_critical(double a, double b, double R, double *Tc, double *rhoc);

/* Maxwell coexistence densities and pressure of `eos` (with interaction strength G for
 * the exponential potential, whose pressure is rho/3 + G psi^2/2).
 * Errors: LB_EINVAL when the EOS has no van der Waals loop or the solve fails. */
lb_status lb_maxwell(const lb_eos *eos, double G, double *rho_v, double *rho_l, double *p_b);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1306_6445_GB300_LB_H */
