/*
 * swpic.h -- C ABI of the GB300 decorated-particle (Scovel-Weinstein, k = 2)
 * step for the 1D1V periodic Vlasov-Poisson system.
 *
 * Model (paper: "A Structure-Preserving Decorated Particle Method for the
 * Vlasov-Poisson System", Quashie, Burby, Christlieb, Tang):
 *   decorated particle a carries (Q_a, P_a, q*_a, p*_a, psi*_a)      Sec. 3.2, Sec. 5
 *   charge  rho = sum_a psi*_a delta(q - Q_a) + p*_a delta'(q - Q_a)   Eq. (rho)
 *   potential: periodic P1 Galerkin, int phi_h' v' = sum_a psi* v(Q) - p* v'(Q),
 *              zero-mean gauge                                          Eq. (galerkin), (lin-sys)
 *   motion : dQ/dt = P, dP/dt = -phi_h'(Q), d(q*)/dt = p* phi_h''(Q),
 *            d(p*)/dt = -q*, psi* constant                              Eq. (sw-evolution)
 *   time   : leapfrog (kick (P, q*) / drift (Q, p*) / kick)            Sec. 5
 * Units e = m = eps0 = 1.  The mesh of a run has nx uniform P1 elements on
 * [0, L); h = L/nx; node j sits at q_j = j h; element i = [q_i, q_{i+1}).
 *
 * Conventions
 *  - Every call returns swpic_status; SWPIC_OK == 0.  On failure the context
 *    keeps a message readable with swpic_last_error().  Nothing aborts, exits
 *    or traps; a device-side anomaly (fixed-point overflow of the charge
 *    accumulator, a non-finite field) is recorded in a device flag and
 *    reported as SWPIC_ENUMERIC by the next synchronous call.
 *  - Device work is enqueued on the stream given to swpic_bind_state() and
 *    is asynchronous unless a call says "synchronous".
 *  - Particle state is caller-owned device memory (structure of arrays, one
 *    array per variable, element type float or double per the precision of
 *    the context).  The context borrows the pointers; it never frees them.
 *  - All runs of a batch share one precision, decoration flag, deposit mode
 *    and phi'' reading; each run has its own L, nx, dt and particle count.
 *    Particles of run r occupy [offsets[r], offsets[r+1]) of every array.
 */
#ifndef SWPIC_H
#define SWPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWPIC_ABI_VERSION 1
#define SWPIC_NX_MAX 4096          /* mesh elements per run (shared-memory tile) */
#define SWPIC_STATIC_NX_MAX 4096   /* mesh elements of swpic_deposit_static */

typedef enum swpic_status {
    SWPIC_OK = 0,
    SWPIC_EINVAL = 1,        /* bad argument or configuration                    */
    SWPIC_ENOMEM = 2,        /* device or host allocation failed                 */
    SWPIC_ECUDA = 3,         /* a CUDA runtime call failed                       */
    SWPIC_ETIMEOUT = 4,      /* a bounded device wait ran out                    */
    SWPIC_ENUMERIC = 5,      /* accumulator overflow or non-finite field          */
    SWPIC_EUNSUPPORTED = 6,  /* feature not available for this context           */
    SWPIC_ESTATE = 7,        /* call out of order (e.g. no state bound)          */
    SWPIC_EIO = 8            /* file could not be read or written                */
} swpic_status;

typedef enum swpic_precision { SWPIC_F32 = 32, SWPIC_F64 = 64 } swpic_precision;

/* Deposit accumulation.
 * ATOMIC:        per-CTA shared-memory float/double atomics, then 64-bit
 *                fixed-point global atomics; run-to-run bits may differ in the
 *                last place of b.
 * DETERMINISTIC: per-thread sums in a fixed particle order, then 64-bit
 *                fixed-point integer atomics in shared and global memory;
 *                integer addition is associative, so b is bitwise identical
 *                from run to run for a fixed launch configuration.        */
typedef enum swpic_deposit_mode {
    SWPIC_DEPOSIT_ATOMIC = 0,
    SWPIC_DEPOSIT_DETERMINISTIC = 1
} swpic_deposit_mode;

/* Reading of "phi_h'' reconstructed through an auxiliary projection" (Sec. 5):
 * LUMPED: g = lumped-mass L2 projection of phi_h' onto P1, g_j =
 *         (Phi_{j+1} - Phi_{j-1})/(2h); phi'' = g' (constant per element).
 * NODAL:  s_j = -btilde_j/h, the lumped L2 projection of phi'' = n0 - rho
 *         (Eq. poisson), interpolated linearly inside each element.
 * P2:     the field itself in V_h^(2) (quadratic Lagrange elements, the
 *         degree-k space of Sec. 5 with k = 2): phi_h' is linear and phi_h''
 *         constant inside each element, both from the element's quadratic,
 *         no projection.  The deposit adds one accumulator per element
 *         (the midpoint degree of freedom).                              */
typedef enum swpic_d2_mode { SWPIC_D2_LUMPED = 0, SWPIC_D2_NODAL = 2, SWPIC_D2_P2 = 3 } swpic_d2_mode;

typedef struct swpic_config {
    double  L;                 /* domain length (> 0)                            */
    double  dt;                /* time step (> 0)                                */
    int32_t nx;                /* mesh elements, 2 <= nx <= SWPIC_NX_MAX          */
    int32_t precision;         /* SWPIC_F32 or SWPIC_F64 (state + push + deposit) */
    int32_t decorated;         /* 1: monopole + dipole; 0: point-particle PIC     */
    int32_t deposit_mode;      /* swpic_deposit_mode                             */
    int32_t d2_mode;           /* swpic_d2_mode                                  */
    int32_t resort_every;      /* stable sort by cell every K steps; 0 = never   */
    int32_t threads_per_block; /* 0 = default (256); a multiple of 32 in 64..768
                                  (FP32 state) or 64..512 (FP64 state)           */
    int32_t blocks_per_sm;     /* 0 = default (3 FP32, 2 FP64)                   */
    int32_t use_graphs;        /* 1 = capture swpic_step() in CUDA graphs        */
    int32_t diag_capacity;     /* diagnostic records kept per run (0 = 4096)     */
} swpic_config;

/* One diagnostic record (all FP64), Eq. (Hh) and Eq. (Eamp):
 * mass = sum psi*, momentum = sum(psi* P + q*), kinetic = sum(psi* P^2/2 + q* P),
 * field_energy = (1/2) Phi^T A Phi = (h/2) sum_i E_i^2, H = kinetic + field,
 * E_amp = ((1/L) int E^2)^{1/2}; (P, q*) taken at the integer time t.        */
typedef struct swpic_diag {
    double t, mass, momentum, kinetic, field_energy, hamiltonian, e_amp;
    int64_t step;
} swpic_diag;

/* Lattice initialisation of one run (reading of Sec. 4.2 / Alg. 1 with each
 * phase-space lattice cell taken as the cluster S_a of the continuum f0):
 *   centre (x_i, v_j) = ((i + 1/2) dx, vmin + (j + 1/2) dv), particle index i*nv + j
 *   Q = wrap(x_i + jx dx), P = v_j + jv dv              (jitter in cells)
 *   psi* = f0(x_i, v_j) dx dv
 *   p*   = int_cell f0(q,p) (L/2pi) sin(2pi (Q - q)/L) dq dp    (periodic c, Sec. 4.2)
 *   q*   = -int_cell f0(q,p) (P - p) dq dp                       (Eq. moment-def)
 * cell integrals by an n x n Gauss-Legendre rule (1 <= n <= 5).
 * f0(x, v) = (1 + alpha cos(kx x)) sum_m amp_m (c0_m + c2_m v^2) exp(-beta_m (v - u_m)^2) */
typedef struct swpic_lattice {
    int32_t nq, nv;            /* lattice points in x and in v; nq*nv = particles of the run */
    double  vmin, vmax;
    double  alpha, kx;
    int32_t n_terms;           /* 1..4 */
    int32_t quad_order;        /* Gauss-Legendre points per axis, 1..5 (4 typical) */
    double  amp[4], c0[4], c2[4], beta[4], u[4];
    int32_t decorate;          /* 1: compute p*, q*; 0: set them to zero */
    int32_t reserved;
} swpic_lattice;

typedef struct swpic_ctx swpic_ctx;
typedef struct CUstream_st *swpic_stream;   /* same type as cudaStream_t */

/* ---- lifetime ------------------------------------------------------------ */

/* Single run of n_particles (>= 0).  Validates cfg; allocates the context's
 * own device buffers (mesh accumulators, field tables, sort histograms,
 * diagnostics ring).  *out receives the context or NULL on failure. */
swpic_status swpic_create(const swpic_config *cfg, int64_t n_particles, swpic_ctx **out);

/* Ensemble of n_runs independent runs advanced by the same launches.
 * cfgs[n_runs]: per-run L, dt, nx (the shared fields are taken from cfgs[0]
 * and must agree); particle_offsets[n_runs + 1]: host array, offsets[0] == 0,
 * non-decreasing.  Runs with no particles are allowed. */
swpic_status swpic_create_batch(const swpic_config *cfgs, int32_t n_runs,
                                const int64_t *particle_offsets, swpic_ctx **out);

/* Frees only what the context owns.  NULL is accepted. */
void swpic_destroy(swpic_ctx *ctx);

/* Message of the last failure on ctx (owned by ctx; valid until the next call). */
const char *swpic_last_error(const swpic_ctx *ctx);
const char *swpic_status_string(swpic_status s);
int32_t swpic_abi_version(void);

/* Bytes of caller-provided scratch needed by the stable sort (ping-pong copy
 * of the particle arrays): 5 (or 3 without decoration) * N * element size,
 * rounded up to 256-byte segments.  Synchronous, host only. */
swpic_status swpic_scratch_bytes(const swpic_ctx *ctx, int64_t *bytes);

/* Bind caller-owned device arrays (each 16-byte aligned, N elements of the
 * context's precision).  qs/ps may be NULL when decorated == 0.  scratch may be
 * NULL (sorting then unavailable) or point to >= swpic_scratch_bytes bytes.
 * stream: the CUDA stream all later work is enqueued on (NULL = legacy default). */
swpic_status swpic_bind_state(swpic_ctx *ctx, void *Q, void *P, void *qs, void *ps,
                              void *psi, void *scratch, int64_t scratch_bytes,
                              swpic_stream stream);

/* ---- initialisation -------------------------------------------------------- */

/* Copy a host FP64 state (all runs, concatenated; n == total particles) into
 * the bound arrays, converting to the context's precision.  qs/ps may be NULL
 * (zero decoration).  Then prepares the run: mass, fixed-point scale, field of
 * the initial positions (deposit + solve) and a diagnostic record at t = 0. */
swpic_status swpic_init_particles(swpic_ctx *ctx, const double *Q, const double *P,
                                  const double *qs, const double *ps, const double *psi,
                                  int64_t n);

/* Fill run `run` on the device from a lattice description (see swpic_lattice);
 * jitter_x / jitter_v: host FP64 arrays of nq*nv jitter values in lattice cells,
 * or NULL.  The field and t = 0 record are prepared lazily by the next call
 * that needs them (or by swpic_refresh). */
swpic_status swpic_init_lattice(swpic_ctx *ctx, int32_t run, const swpic_lattice *spec,
                                const double *jitter_x, const double *jitter_v);

/* Re-derive everything that depends on the bound arrays (mass, fixed-point
 * scale, field, t = 0 record, step counters reset to 0) after the caller wrote
 * them directly. */
swpic_status swpic_refresh(swpic_ctx *ctx);

/* ---- the step, in pieces (Sec. 5) ------------------------------------------- */

/* a1 + a3 + a4: deposit the charge of the current (Q, p*, psi*) (Eq.
 * rhs-assembly) and remove its mean (the uniform background, Eq. neutrality).
 * The result btilde is kept on the device (read it with swpic_get_mesh). */
swpic_status swpic_deposit(swpic_ctx *ctx);

/* a5: solve A Phi = btilde with 1^T Phi = 0 (Eq. lin-sys) and build the field
 * tables used by the push (phi_h' per element, phi_h'' per the d2 reading). */
swpic_status swpic_solve_field(swpic_ctx *ctx);

/* a6: kick then drift with the current tables:
 *   P  <- P  - kick_fraction dt phi_h'(Q),   q* <- q* + kick_fraction dt p* phi_h''(Q)
 *   Q  <- wrap(Q + drift_fraction dt P),      p* <- p* - drift_fraction dt q*
 * KDK = gather_push(0.5, 1) ; deposit ; solve_field ; gather_push(0.5, 0). */
swpic_status swpic_gather_push(swpic_ctx *ctx, double kick_fraction, double drift_fraction);

/* a2: stable counting sort of every run's particles by element index
 * (key = clamp(floor(Q * (nx/L)), 0, nx-1) in the state's precision).
 * Needs scratch. */
swpic_status swpic_sort(swpic_ctx *ctx);

/* n_steps full KDK steps of every run (fused kernels; one launch per step for
 * all runs; CUDA-graph captured when use_graphs).  A diagnostic record is
 * appended at every step s with s % diag_every == 0 (diag_every <= 0: none).
 * The state is at integer time on return.  Re-sorts every resort_every steps. */
swpic_status swpic_step(swpic_ctx *ctx, int32_t n_steps, int32_t diag_every);

/* ---- results --------------------------------------------------------------- */

/* Synchronous.  Copies up to max_records of run `run`'s records (oldest first)
 * into out[]; *n_records receives the number copied. */
swpic_status swpic_diagnostics(swpic_ctx *ctx, int32_t run, swpic_diag *out,
                               int32_t max_records, int32_t *n_records);

/* Synchronous copy-out of run `run`'s mesh data (host arrays of nx doubles,
 * any may be NULL): b (deposit), btilde (b - mean b), Phi (zero-mean nodal
 * potential), E (field on each element = -phi_h'), d2 (phi'' table). */
swpic_status swpic_get_mesh(swpic_ctx *ctx, int32_t run, double *b, double *btilde,
                            double *Phi, double *E, double *d2);

/* Synchronous copy-out of the element index of every particle (a1):
 * keys[a] = clamp(floor(Q_a * (nx/L)), 0, nx-1) computed in the state's
 * precision, with the run-local nx and L.  keys: host int32 array of n. */
swpic_status swpic_get_keys(swpic_ctx *ctx, int32_t *keys, int64_t n);

/* Waits for the bound stream and reports a device anomaly recorded since the
 * last report (SWPIC_ENUMERIC; the message names the number of runs and the
 * first one).  Anomalies are per run: a run whose charge accumulator
 * overflowed or whose field became non-finite keeps its flag (see
 * swpic_run_status) while the other runs of a batch are unaffected; its own
 * overflowing contributions are dropped.  Flags are cleared by swpic_refresh,
 * swpic_init_particles and swpic_load. */
swpic_status swpic_synchronize(swpic_ctx *ctx);

/* Synchronous.  flags[r] = anomaly bits of run r (1: fixed-point charge
 * accumulator overflow, 2: non-finite field, 4: a bounded wait for a bulk
 * copy ran out, reported by swpic_synchronize as SWPIC_ETIMEOUT); n_runs
 * must equal the runs. */
swpic_status swpic_run_status(swpic_ctx *ctx, int32_t *flags, int32_t n_runs);

/* ---- decorated particles from marker particles ---------------------------------- */

/* Sec. 4.1-4.2 "Initialization" and Alg. lumping_procedure: k-means in phase
 * space, then one decorated particle per non-empty cluster with
 *   psi* = sum psi (Eq. psi-star),  (Q, P) = the member nearest to the cluster's
 *   psi-weighted mean,  p* = sum psi (L/2pi) sin(2pi (Q - Qm)/L),
 *   q* = -sum psi (P - Pm)  (Eq. moment-def with the periodic c).
 * k-means: n_iter Lloyd iterations in (q, p), q differences by the minimum
 * image; the nearest-center decision is taken in FP32 (ties to the smaller
 * cluster index); centers move to the psi-weighted member means (q unwrapped
 * about the current center, wrapped into [0, L)); an empty cluster keeps its
 * center.  Member sums are exact (64-bit fixed point), so results do not
 * depend on thread order except the FP64 atomic sums of p*, q*.
 * All arrays are DEVICE memory, FP64 unless noted:
 *   Qm, Pm, wm [M]   markers: positions in [0, L), momenta, weights (> 0);
 *                    M < 2^32
 *   cq, cp [K]       initial centers in, final centers out (K >= 1)
 *   assign [M]       int32, final cluster of every marker; may be NULL
 *   Q, P, qs, ps, psi [K]  the decorated particles of the non-empty clusters,
 *                    in cluster order (Q, P, q*, p*, psi*)
 *   n_out            HOST int64: number of decorated particles written
 * Allocates its work buffers (stream-ordered) and frees them; synchronous.
 * Errors: SWPIC_EINVAL for bad sizes/pointers, SWPIC_ENOMEM, SWPIC_ENUMERIC
 * for non-finite weights or momenta, SWPIC_ECUDA. */
swpic_status swpic_kmeans_lump(const double *Qm, const double *Pm, const double *wm, int64_t M,
                               double *cq, double *cp, int32_t K, double L, int32_t n_iter,
                               int32_t *assign, double *Q, double *P, double *qs, double *ps,
                               double *psi, int64_t *n_out, swpic_stream stream);

/* ---- deposit without device allocation ---------------------------------------- */

/* Mesh charge b_j = sum_a psi*_a phi_j(Q_a) - p*_a phi_j'(Q_a) of one run, for
 * callers that cannot let this library allocate device memory (for example an
 * application that owns the whole device-memory budget through its own pool
 * and forbids other code from calling cudaMalloc/cudaFree).  No counterpart in
 * the paper: it is a memory-management variant of swpic_deposit + the b of
 * swpic_get_mesh.  It allocates nothing: its scratch (a fixed-point charge
 * accumulator of SWPIC_STATIC_NX_MAX int64 words and two doubles, 32 KB per
 * device) lives in file-scope device arrays that every GPU which loads the
 * library holds until the process exits.
 *   Q, ps, psi: caller's device arrays of n elements, float (precision 32) or
 *               double (64); ps may be NULL (no decoration).  Q is read as a
 *               position on the torus: values outside [0, L) are wrapped into
 *               it as the particle pass wraps them (the arrays are not written).
 *   b:          caller's device array of nx doubles (output).
 *   L, nx:      the periodic mesh; 2 <= nx <= SWPIC_STATIC_NX_MAX, else
 *               SWPIC_EINVAL (the scratch holds at most that many nodes).
 *   stream:     work is enqueued here, asynchronously.
 * The first call on a device looks up the device addresses of the scratch
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  The addresses are kept for the life of the process and do
 * not survive a cudaDeviceReset of that device: do not call this entry point on
 * a device after resetting it.  Every call clears and reuses the same scratch,
 * so calls whose work overlaps on the GPU (different streams, or different host
 * threads on one device) race and must be serialised by the caller.
 * Errors: SWPIC_EINVAL for bad sizes or pointers; SWPIC_ECUDA when a launch
 * fails, or when a CUDA error left pending by earlier work is found on entry
 * (it is reported and left pending, not cleared). */
swpic_status swpic_deposit_static(const void *Q, const void *ps, const void *psi, int64_t n,
                                  int32_t precision, double L, int32_t nx, double *b,
                                  swpic_stream stream);

/* ---- end to end from host memory --------------------------------------------- */

/* Host-memory form of swpic_step for callers that keep the state on the host:
 * copies the host arrays (context precision, n == total particles; qs/ps may
 * be NULL when decorated == 0) into the bound device arrays, prepares the field
 * of that state, runs n_steps steps, and copies the final (Q, P, q*, p*) back
 * to the host outputs (NULL outputs are skipped).  Synchronous.  Pinned host
 * memory gives the full copy bandwidth. */
swpic_status swpic_step_host(swpic_ctx *ctx, const void *Q, const void *P, const void *qs,
                             const void *ps, const void *psi, void *Q_out, void *P_out,
                             void *qs_out, void *ps_out, int64_t n, int32_t n_steps,
                             int32_t diag_every);

/* ---- checkpoint ------------------------------------------------------------- */

/* Synchronous.  Writes/reads the particle arrays, per-run step counters,
 * field tables and configuration as raw little-endian binary.  load requires a
 * context created with the same configuration and bound arrays; the loading
 * context's diagnostic records are discarded (its records start at the
 * checkpoint). */
swpic_status swpic_save(swpic_ctx *ctx, const char *path);
swpic_status swpic_load(swpic_ctx *ctx, const char *path);

/* ---- launch shape, tuning and measurement --------------------------------- */

/* Threads per block and resident blocks per SM of the particle kernels
 * (0 keeps the current value).  Invalidates captured graphs. */
swpic_status swpic_set_launch(swpic_ctx *ctx, int32_t threads_per_block,
                              int32_t blocks_per_sm, int32_t resort_every);
swpic_status swpic_get_launch(const swpic_ctx *ctx, int32_t *threads_per_block,
                              int32_t *blocks_per_sm, int32_t *resort_every);

/* How the particle pass moves particle data (no counterpart in the paper; a
 * property of this implementation).  A warp works in turns of 512 bytes per
 * array (64 FP32 or 32 FP64 two-particle vectors); lane l takes vectors l and
 * 32 + l of a turn.  stages = 0: each thread loads its 16-byte vectors into
 * registers, one vector ahead of the one it pushes.  stages = 2..8: every warp
 * runs its own pipeline: lane 0 copies the warp's next turns global -> shared
 * memory with bulk asynchronous copies (one 1-D copy per array and turn,
 * completion counted in bytes on the stage's mbarrier), up to `stages` turns
 * ahead; the lanes read a stage into registers, lane 0 refills it, and the
 * updated particles are written back with plain stores.  The stage count
 * actually used is the largest <= stages that fits in shared memory at
 * blocks_per_sm CTAs per SM (register loads when fewer than two fit).  Both
 * streams give every thread the same particles in the same order, so results
 * do not depend on the choice beyond the deposit-order freedom of
 * SWPIC_DEPOSIT_ATOMIC.  Default 4.  Invalidates captured graphs.
 * *effective receives the stage count that the current launch shape gets
 * (0 = register loads). */
swpic_status swpic_set_pipeline(swpic_ctx *ctx, int32_t stages);
swpic_status swpic_get_pipeline(const swpic_ctx *ctx, int32_t *requested, int32_t *effective);

/* Where swpic_step solves the field of each deposit (Eq. swpic_poisson; no
 * counterpart in the paper, a property of this implementation):
 * LAST_CTA: the CTA that finishes a run's last particles of the depositing
 *           pass solves it at the end of that pass and writes the run's table.
 * AT_START: the depositing pass only deposits; every CTA of the next pass
 *           solves the field of the finished deposit into its own shared-memory
 *           table at its start, while its first particle copies are in flight,
 *           and the CTA holding the run's first particle also writes the run's
 *           table, snapshot, W, E_amp and gauge to global memory.  No pass ends
 *           in a one-CTA solve.  Each CTA solves once per run it touches.
 * AUTO (default): AT_START for batches of at most 4 runs, LAST_CTA otherwise.
 * Both give bitwise the same fields, states and records (the solve is exact
 * integer arithmetic followed by the same roundings).  The charge
 * accumulators rotate over three buffers per run.  Invalidates captured
 * graphs.  EINVAL for any other mode. */
typedef enum swpic_field_solve {
    SWPIC_FIELD_SOLVE_AUTO = 0,
    SWPIC_FIELD_SOLVE_LAST_CTA = 1,
    SWPIC_FIELD_SOLVE_AT_START = 2
} swpic_field_solve;
swpic_status swpic_set_field_solve(swpic_ctx *ctx, int32_t mode);
swpic_status swpic_get_field_solve(const swpic_ctx *ctx, int32_t *mode, int32_t *effective);

/* Times a small grid of launch shapes (threads per block 128, 192, 256, 384,
 * 512, 768 up to the precision's limit, x CTAs per SM 1..8 within 2048
 * threads), particle-load pipelines and re-sort intervals on the bound state,
 * then, for the best shape with the bulk-copy stream, 2, 3 and 4 stages with
 * and without issuing each CTA's first copies before it stages its field
 * table (which is saved before and restored after, bit
 * for bit; trial steps record diagnostics every step) and keeps the fastest.
 * Tune on a state like the one to be run: the fastest shape for a freshly
 * initialised (ordered) lattice differs from the one for a mixed plasma.
 * steps_per_trial > 0.  cache_path: JSON file read before and updated after tuning, keyed by (GPU, precision, decoration, deposit mode,
 * runs, particles, total mesh size); NULL = no cache.  Synchronous. */
swpic_status swpic_autotune(swpic_ctx *ctx, int32_t steps_per_trial, const char *cache_path);

/* When enabled, swpic_step records a CUDA event pair around every particle
 * pass it launches (inside the captured graph too); swpic_pass_times returns
 * the device durations (ms) of the passes of the most recent swpic_step call
 * (synchronous). */
swpic_status swpic_set_timing(swpic_ctx *ctx, int32_t enable);
swpic_status swpic_pass_times(swpic_ctx *ctx, float *ms, int32_t max_passes, int32_t *n_passes);

/* Failure-path hook for tests (no counterpart in the paper): every wait of
 * the bulk-copy stream for its copies is bounded, and one that runs out flags
 * the run (reported by swpic_synchronize as SWPIC_ETIMEOUT, bit 4 of
 * swpic_run_status); the warp then waits, again bounded, for the copies it has
 * in flight, and its CTA leaves the pass.  stall_warp >= 0 makes that warp
 * (grid-wide index blockIdx * warps per block + warp) leave the stage of its
 * first turn unarmed in every later pass: no copy is issued into it, so its
 * wait can only run out, while every copy that is issued still lands.
 * wait_limit_ns bounds each wait (0 = the default of 1 s).  A pass that timed
 * out leaves the run's field stale; swpic_refresh recovers it.  stall_warp =
 * -1 with wait_limit_ns = 0 restores normal operation.  Invalidates captured
 * graphs.  Only the bulk-copy stream waits (swpic_set_pipeline with >= 2
 * stages that fit). */
swpic_status swpic_set_wait_test(swpic_ctx *ctx, int32_t stall_warp, int64_t wait_limit_ns);

/* Number of kernel launches this context has issued so far (a graph replay
 * counts each kernel node it contains). */
swpic_status swpic_launch_count(const swpic_ctx *ctx, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
