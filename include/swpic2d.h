/*
 * swpic2d.h -- C ABI of the GB300 decorated-particle (Scovel-Weinstein, k = 2)
 * step for the 2D2V periodic Vlasov-Poisson system.
 *
 * Model (general-d form of the paper, Sec. 3.3, on the torus T^2, with S_h =
 * delta and units e = m = eps0 = 1):
 *   decorated particle a carries Q_a, P_a, q*_a, p*_a in R^2 and psi*_a
 *   potential: int grad phi_h . grad v = sum_a psi*_a v(Q_a) - p*_a . grad v(Q_a)
 *              - n0 int v for all v in E, zero mean              Eq. (swpic_poisson)
 *   motion : dQ/dt = P, dP/dt = -grad phi_h(Q), d(q*)/dt = H(Q) p*,
 *            d(p*)/dt = -q*, psi* constant                       Eq. (swpic_dynamics)
 *   time   : leapfrog, kick (P, q*) / drift (Q, p*) / kick        Sec. 5
 * Discretisation (the paper gives none for d > 1):
 *   E = periodic bilinear (Q1) elements on an nx x ny uniform mesh of
 *       [0, Lx) x [0, Ly); node (i, j) at (i hx, j hy), index j nx + i;
 *       cell (i, j) = [i hx, (i+1) hx) x [j hy, (j+1) hy); a particle on a
 *       mesh line belongs to the cell on its right / above.
 *   H_ik = d_k g_i, g = lumped-mass L2 projection of grad phi_h onto E
 *       (the 2D form of the 1D "auxiliary projection", reading LUMPED):
 *       g_x(i,j) = (2/3) C_x(i,j) + (1/6) (C_x(i,j-1) + C_x(i,j+1)),
 *       C_x(i,j) = (Phi_{i+1,j} - Phi_{i-1,j}) / (2 hx); g_y likewise.
 *   The Q1 system is solved exactly by the discrete Fourier transform: its
 *   stiffness is diagonal in Fourier modes with symbol
 *       (2 - 2 cos tx)(4 + 2 cos ty) hy/(6 hx) + (2 - 2 cos ty)(4 + 2 cos tx) hx/(6 hy);
 *   the zero mode carries the neutralising background and the gauge.
 *
 * Conventions are those of swpic.h: swpic_status results, caller-owned
 * device state (structure of arrays in the context's precision), work
 * enqueued on the bound stream, device anomalies reported as SWPIC_ENUMERIC
 * by the next synchronous call, nothing aborts or traps.
 */
#ifndef SWPIC2D_H
#define SWPIC2D_H

#include <stdint.h>
#include "swpic.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SWPIC2D_N_MAX 1024            /* cells per axis (a power of two, >= 4) */
#define SWPIC2D_NODES_MAX_F32 8192    /* nx * ny of an FP32 context (shared-memory table) */
#define SWPIC2D_NODES_MAX_F64 4096    /* nx * ny of an FP64 context */

typedef struct swpic2d_config {
    double  Lx, Ly;            /* domain lengths (> 0)                                  */
    double  dt;                /* time step (> 0)                                       */
    int32_t nx, ny;            /* cells per axis: powers of two in [4, SWPIC2D_N_MAX]    */
    int32_t precision;         /* SWPIC_F32 or SWPIC_F64 (state, push and deposit)      */
    int32_t decorated;         /* 1: monopole + dipole; 0: point-particle PIC            */
    int32_t threads_per_block; /* 0 = default (256); 64..256, multiple of 32             */
    int32_t blocks_per_sm;     /* 0 = default (as many as the shared memory allows, <= 8) */
    int32_t diag_capacity;     /* diagnostic records kept (0 = 4096); later ones dropped  */
    int32_t reserved;
} swpic2d_config;

/* One diagnostic record (FP64) at integer time t = step dt:
 * mass = sum psi*, momentum = sum(psi* P + q*), kinetic = sum(psi* |P|^2/2 + q* . P),
 * field_energy W = (1/2) int |grad phi_h|^2 = (1/2) Phi^T btilde, H = kinetic + W,
 * e_amp = (2 W / (Lx Ly))^(1/2).                                                       */
typedef struct swpic2d_diag {
    double t, mass, momentum_x, momentum_y, kinetic, field_energy, hamiltonian, e_amp;
    int64_t step;
} swpic2d_diag;

/* Lattice initialisation (the cluster reading of Sec. 4.2 / Alg. 1 used in
 * 1D, one dimension up): each cell of an nqx x nqy x nvx x nvy phase-space
 * lattice on [0, Lx) x [0, Ly) x [vmin, vmax]^2 is the cluster S_a of
 *   f0 = (1 + alpha cos(kx x + ky y)) exp(-|v|^2 / (2 vth^2)) / (2 pi vth^2);
 * particle index ((k nvy + l) nqy + j) nqx + i (positions fastest, so the
 * lanes of a warp sit in neighbouring cells);  Q, P = the cell centre;
 *   psi* = f0(centre) dx dy dvx dvy
 *   p*_x = int_cell f0 (Lx/2pi) sin(2pi (Qx - x)/Lx), p*_y likewise  (periodic c)
 *   q*   = - int_cell f0 (P - p)                                   (Eq. moment-def)
 * cell integrals by a quad_order^4 Gauss-Legendre rule (1 <= quad_order <= 4),
 * evaluated in FP64 and stored in the context's precision.                 */
typedef struct swpic2d_lattice {
    int32_t nqx, nqy, nvx, nvy;
    double  vmin, vmax, alpha, kx, ky, vth;
    int32_t quad_order;
    int32_t decorate;          /* 0: p*, q* = 0 */
} swpic2d_lattice;

typedef struct swpic2d_ctx swpic2d_ctx;

/* Validate cfg, allocate the context's own device buffers (charge
 * accumulator, spectral work array, potential, node table, diagnostics).
 * n_particles >= 0.  *out receives the context or NULL on failure. */
swpic_status swpic2d_create(const swpic2d_config *cfg, int64_t n_particles, swpic2d_ctx **out);
void swpic2d_destroy(swpic2d_ctx *ctx);
const char *swpic2d_last_error(const swpic2d_ctx *ctx);

/* Borrow the caller's device state: state[9] = Qx, Qy, Px, Py, qx, qy, px, py,
 * psi (q*, p* entries may be NULL when not decorated), each n_particles
 * elements of the context's precision.  stream: where all work is enqueued
 * (NULL = the legacy default stream).  The context never frees them. */
swpic_status swpic2d_bind_state(swpic2d_ctx *ctx, void *const state[9], swpic_stream stream);

/* Synchronous.  Take the fixed-point unit of the charge accumulator from
 * the bound state (sum psi* + 2 sum |p*_x|/hx + 2 sum |p*_y|/hy maps to
 * 2^58 in FP64 contexts, 2^54 in FP32 ones; the limit is 2^62, and the
 * decorations p* grow in time) and compute the field of the state (deposit,
 * solve, node table).  Call after writing the state and before
 * swpic2d_step; a run whose decorations outgrow the headroom reports
 * SWPIC_ENUMERIC, and a refresh takes a new unit. */
swpic_status swpic2d_refresh(swpic2d_ctx *ctx);

/* Synchronous.  Write the lattice state into the bound arrays (the product
 * nqx nqy nvx nvy must equal the context's particle count) and take its
 * field (as swpic2d_refresh). */
swpic_status swpic2d_init_lattice(swpic2d_ctx *ctx, const swpic2d_lattice *spec);

/* Advance n_steps >= 0 leapfrog steps (asynchronous).  The closing half-kick
 * of a step and the opening half-kick of the next share one fused pass over
 * the particles, which also deposits the drifted charge.  diag_every > 0:
 * a record at every integer time t = s dt with s % diag_every == 0 (once per
 * s, including the starting time). */
swpic_status swpic2d_step(swpic2d_ctx *ctx, int32_t n_steps, int32_t diag_every);

/* Synchronous.  The whole path from host memory: copy the nine host arrays
 * in[9] (Qx, Qy, Px, Py, qx, qy, px, py, psi in the context's precision;
 * a NULL decoration array is taken as zero) into the bound device state,
 * take its field (as swpic2d_refresh), advance n_steps, and copy the eight
 * evolving arrays back into out[8] (NULL entries are skipped).  Pinned host
 * memory makes the copies asynchronous. */
swpic_status swpic2d_step_host(swpic2d_ctx *ctx, const void *const in[9], void *const out[8],
                               int32_t n_steps, int32_t diag_every);

/* Synchronous: copy up to max_records records into out (host). */
swpic_status swpic2d_diagnostics(swpic2d_ctx *ctx, swpic2d_diag *out, int32_t max_records,
                                 int32_t *n_records);

/* Synchronous: the current field on the nodes, host arrays of ny*nx doubles
 * (node index j nx + i); any pointer may be NULL.  b is the deposited load
 * of the last field update, Phi the zero-mean potential (FP32 contexts: the
 * FP32 values of the node table), gx, gy the projected gradient held
 * (rounded to the state precision) in the node table. */
swpic_status swpic2d_get_field(swpic2d_ctx *ctx, double *b, double *Phi, double *gx, double *gy);

/* Synchronous: wait for the stream; report a device anomaly flag. */
swpic_status swpic2d_synchronize(swpic2d_ctx *ctx);

/* Checkpoint (synchronous).  swpic2d_save writes the bound state (the nine
 * arrays, or five without decorations, in the context's precision), the step
 * count and the geometry to a binary file; SWPIC_EIO when it cannot be
 * written.  swpic2d_load reads such a file into the bound arrays of a
 * context with the same precision, decoration flag, particle count, mesh,
 * domain and dt (SWPIC_EINVAL otherwise, SWPIC_EIO when unreadable),
 * restores the step count and takes the field of the state (as
 * swpic2d_refresh).  The loading context's diagnostic records are discarded:
 * its records start at the checkpoint (the records before it stay with the
 * context that made them). */
swpic_status swpic2d_save(swpic2d_ctx *ctx, const char *path);
swpic_status swpic2d_load(swpic2d_ctx *ctx, const char *path);

/* Per-pass device durations (CUDA events around every particle pass of
 * swpic2d_step while enabled; read and cleared by swpic2d_pass_times). */
swpic_status swpic2d_set_timing(swpic2d_ctx *ctx, int32_t enable);
swpic_status swpic2d_pass_times(swpic2d_ctx *ctx, float *ms, int32_t max_passes, int32_t *n_passes);

/* Kernels this context has launched so far. */
swpic_status swpic2d_launch_count(const swpic2d_ctx *ctx, int64_t *count);

#ifdef __cplusplus
}
#endif

#endif
