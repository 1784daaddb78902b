/*
 * swpic_oracle.c -- plain, slow, FP64 CPU oracle for the 1D1V periodic
 * monopole-dipole (k = 2) Scovel-Weinstein decorated-particle step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and never calls it.
 *
 * Every routine follows the paper (Quashie, Burby, Christlieb, Tang,
 * "A Structure-Preserving Decorated Particle Method for the Vlasov-Poisson
 * System") in its own notation:
 *   state of decorated particle a:  (Q_a, P_a, q*_a, p*_a, psi*_a)     (Sec. 3.2, Sec. 5)
 *   units e = m = eps0 = 1, periodic domain [0, L)                       (Sec. 5, Eq. poisson)
 *   mesh: nx uniform P1 elements, h = L/nx, node j at q_j = j h,
 *         element i = [q_i, q_{i+1})                                     (Sec. 5, V_h^(1))
 *
 * Nothing is blocked, fused or reordered beyond what the paper states: each
 * routine is one loop over particles or one dense linear-algebra step.
 * All floating point is IEEE double; build with -ffp-contract=off so that the
 * x86 and aarch64 builds round identically.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Small helpers                                                             */
/* ------------------------------------------------------------------------ */

/* Neumaier compensated summation: returns sum + compensation. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *acc, double x) {
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
    else                          acc->c += (x - t) + acc->s;
    acc->s = t;
}
static double nsum_val(const nsum *acc) { return acc->s + acc->c; }

/* Host threads for the particle loops of or_run (default 1: the plain serial
 * loops that every test uses).  With T > 1 (an OpenMP build) the particles
 * are split into T contiguous blocks: gather, kick and drift act particle by
 * particle (same results), while the deposit and the particle sums of the
 * diagnostics give one partial per block, added in block order, so the
 * results depend on T only through that summation order.  This exists to
 * time the oracle on all host cores; it changes none of its arithmetic. */
static int g_threads = 1;
int or_set_threads(int t) {
#ifdef _OPENMP
    g_threads = t < 1 ? 1 : t;
#else
    (void)t;
    g_threads = 1;
#endif
    return g_threads;
}
static void block_of(int64_t n, int T, int t, int64_t *a0, int64_t *a1) {
    *a0 = n * t / T;
    *a1 = n * (t + 1) / T;
}

/* Periodic wrap of a position into [0, L) (torus T = R mod L, Sec. 2).
 * A value that rounds up to exactly L is mapped to L - L = 0 (reading A5). */
double or_wrap(double Q, double L) {
    double w = Q - L * floor(Q / L);
    if (w >= L) w -= L;
    if (w < 0.0) w += L;
    return w;
}

/* Element containing Q: i = floor(Q/h), clamped to [0, nx-1].  A particle
 * exactly on node q_i belongs to the element on its right (reading A5). */
int32_t or_element(double Q, double L, int32_t nx) {
    double h = L / (double)nx;
    double s = floor(Q / h);
    int32_t i = (int32_t)s;
    if (i < 0) i = 0;
    if (i > nx - 1) i = nx - 1;
    return i;
}

/* Element decided in FP32 from an FP32-stored position:
 * floor(fl32(Q) * fl32(nx/L)), clamped.  Used when the state is kept in FP32
 * storage, so the integer decision is taken in the storage precision. */
int32_t or_element_f32(double Q, double L, int32_t nx) {
    float q = (float)Q;
    float inv_h = (float)((double)nx / L);
    float prod = q * inv_h;
    float s = floorf(prod);
    int32_t i = (s != s) ? 0 : (int32_t)s;
    if (i < 0) i = 0;
    if (i > nx - 1) i = nx - 1;
    return i;
}

/* Round a value to FP32 storage (and back to double). */
static double to_f32(double x) { return (double)(float)x; }

/* ------------------------------------------------------------------------ */
/* Deposit: right-hand side assembly, Eq. (rhs-assembly) of Sec. 5           */
/*   b_j = sum_a [ psi*_a phi_j(Q_a) - p*_a phi_j'(Q_a) ]                    */
/* For P1 hats on element i with local coordinate xi = (Q - q_i)/h:          */
/*   phi_i = 1 - xi, phi_{i+1} = xi, phi_i' = -1/h, phi_{i+1}' = +1/h.       */
/* If elem != NULL the element of particle a is elem[a] (a decision taken by */
/* the caller, e.g. in FP32); otherwise it is or_element(Q_a).               */
/* p_star may be NULL (decoration off: point-particle PIC, Eq. pic_poisson). */
/* ------------------------------------------------------------------------ */
void or_deposit(int64_t n, const double *Q, const double *p_star,
                const double *psi_star, const int32_t *elem,
                double L, int32_t nx, double *b) {
    double h = L / (double)nx;
    for (int32_t j = 0; j < nx; ++j) b[j] = 0.0;
    for (int64_t a = 0; a < n; ++a) {
        int32_t i = elem ? elem[a] : or_element(Q[a], L, nx);
        int32_t ip1 = (i + 1 == nx) ? 0 : i + 1;
        double xi = (Q[a] - (double)i * h) / h;
        double ps = p_star ? p_star[a] : 0.0;
        /* monopole psi* phi_j(Q), dipole - p* phi_j'(Q) */
        b[i]   += psi_star[a] * (1.0 - xi) - ps * (-1.0 / h);
        b[ip1] += psi_star[a] * xi         - ps * (+1.0 / h);
    }
}

/* Independent brute-force form of the same assembly: every hat function phi_j
 * is evaluated at every particle from the periodic distance d = Q - q_j
 * (wrapped into [-L/2, L/2)).  phi_j(Q) = 1 - |d|/h for |d| < h; its
 * derivative is -1/h to the right of the node (0 <= d < h) and +1/h to the
 * left (-h <= d < 0).  O(N nx); for tiny inputs only. */
void or_deposit_bruteforce(int64_t n, const double *Q, const double *p_star,
                           const double *psi_star, double L, int32_t nx,
                           double *b) {
    double h = L / (double)nx;
    for (int32_t j = 0; j < nx; ++j) {
        double acc = 0.0;
        double qj = (double)j * h;
        for (int64_t a = 0; a < n; ++a) {
            double d = Q[a] - qj;
            d -= L * floor(d / L + 0.5);          /* into [-L/2, L/2) */
            double phi = 0.0, dphi = 0.0;
            if (d >= 0.0 && d < h)       { phi = 1.0 - d / h; dphi = -1.0 / h; }
            else if (d < 0.0 && d >= -h) { phi = 1.0 + d / h; dphi = +1.0 / h; }
            double ps = p_star ? p_star[a] : 0.0;
            acc += psi_star[a] * phi - ps * dphi;
        }
        b[j] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Stiffness matrix, Eq. (lin-sys): A_ij = int_0^L phi_i' phi_j' dq,         */
/* assembled element by element (each element e = [q_i, q_{i+1}] adds        */
/* (1/h) [[1, -1], [-1, 1]] to rows/cols {i, i+1 mod nx}).  Dense nx x nx.   */
/* ------------------------------------------------------------------------ */
void or_stiffness(int32_t nx, double L, double *A) {
    double h = L / (double)nx;
    memset(A, 0, sizeof(double) * (size_t)nx * (size_t)nx);
    for (int32_t e = 0; e < nx; ++e) {
        int32_t i = e, j = (e + 1) % nx;
        A[(size_t)i * nx + i] += 1.0 / h;
        A[(size_t)j * nx + j] += 1.0 / h;
        A[(size_t)i * nx + j] -= 1.0 / h;
        A[(size_t)j * nx + i] -= 1.0 / h;
    }
}

/* Dense LU with partial pivoting of an m x m matrix (row-major, in place). */
static int lu_factor(int32_t m, double *M, int32_t *piv) {
    for (int32_t k = 0; k < m; ++k) {
        int32_t p = k;
        double best = fabs(M[(size_t)k * m + k]);
        for (int32_t r = k + 1; r < m; ++r) {
            double v = fabs(M[(size_t)r * m + k]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int32_t c = 0; c < m; ++c) {
                double t = M[(size_t)k * m + c];
                M[(size_t)k * m + c] = M[(size_t)p * m + c];
                M[(size_t)p * m + c] = t;
            }
        for (int32_t r = k + 1; r < m; ++r) {
            double f = M[(size_t)r * m + k] / M[(size_t)k * m + k];
            M[(size_t)r * m + k] = f;
            for (int32_t c = k + 1; c < m; ++c)
                M[(size_t)r * m + c] -= f * M[(size_t)k * m + c];
        }
    }
    return 0;
}
static void lu_solve(int32_t m, const double *M, const int32_t *piv, double *x) {
    for (int32_t k = 0; k < m; ++k) {
        int32_t p = piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
    for (int32_t r = 0; r < m; ++r) {
        double s = x[r];
        for (int32_t c = 0; c < r; ++c) s -= M[(size_t)r * m + c] * x[c];
        x[r] = s;
    }
    for (int32_t r = m - 1; r >= 0; --r) {
        double s = x[r];
        for (int32_t c = r + 1; c < m; ++c) s -= M[(size_t)r * m + c] * x[c];
        x[r] = s / M[(size_t)r * m + r];
    }
}

/* Factorised Galerkin Poisson operator (Eq. galerkin / lin-sys).  The test
 * space carries the zero-mean constraint, so A Phi - b must be orthogonal to
 * every zero-mean coefficient vector: A Phi + lambda 1 = b, 1^T Phi = 0.
 * That bordered (nx+1) x (nx+1) system is what is factorised.  Its
 * multiplier is lambda = mean(b): the uniform background n0 (Eq. neutrality)
 * is removed by the constraint, as Sec. 5 states. */
typedef struct {
    int32_t nx;
    double L;
    double *M;     /* (nx+1)^2 LU factors */
    int32_t *piv;
} or_poisson;

or_poisson *or_poisson_new(int32_t nx, double L) {
    or_poisson *s = (or_poisson *)calloc(1, sizeof(or_poisson));
    int32_t m = nx + 1;
    s->nx = nx; s->L = L;
    s->M = (double *)calloc((size_t)m * m, sizeof(double));
    s->piv = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    double *A = (double *)calloc((size_t)nx * nx, sizeof(double));
    or_stiffness(nx, L, A);
    for (int32_t r = 0; r < nx; ++r) {
        for (int32_t c = 0; c < nx; ++c) s->M[(size_t)r * m + c] = A[(size_t)r * nx + c];
        s->M[(size_t)r * m + nx] = 1.0;
        s->M[(size_t)nx * m + r] = 1.0;
    }
    s->M[(size_t)nx * m + nx] = 0.0;
    free(A);
    if (lu_factor(m, s->M, s->piv) != 0) { free(s->M); free(s->piv); free(s); return NULL; }
    return s;
}
void or_poisson_free(or_poisson *s) {
    if (!s) return;
    free(s->M); free(s->piv); free(s);
}
/* Solve for the nodal potential Phi (zero mean) and the multiplier lambda. */
void or_poisson_solve(const or_poisson *s, const double *b, double *Phi, double *lambda) {
    int32_t nx = s->nx, m = nx + 1;
    double *x = (double *)malloc(sizeof(double) * (size_t)m);
    for (int32_t j = 0; j < nx; ++j) x[j] = b[j];
    x[nx] = 0.0;
    lu_solve(m, s->M, s->piv, x);
    for (int32_t j = 0; j < nx; ++j) Phi[j] = x[j];
    if (lambda) *lambda = x[nx];
    free(x);
}
/* One-shot convenience form. Returns 0 on success. */
int or_solve(int32_t nx, double L, const double *b, double *Phi, double *lambda) {
    or_poisson *s = or_poisson_new(nx, L);
    if (!s) return -1;
    or_poisson_solve(s, b, Phi, lambda);
    or_poisson_free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Field tables (Sec. 5: phi_h' from the Lagrange basis, phi_h'' through an  */
/* auxiliary projection).                                                    */
/*   dphi[i] = phi_h' on element i = (Phi_{i+1} - Phi_i)/h.                  */
/* The projection the paper leaves unspecified is taken in one of three      */
/* readings (d2_mode):                                                       */
/*   0 LUMPED:     g = M_L^{-1} r, r_j = int phi_h' phi_j dq, M_L = h I;     */
/*                 phi'' on element i = (g_{i+1} - g_i)/h   (per element)    */
/*   1 CONSISTENT: g = M^{-1} r with the consistent P1 mass matrix           */
/*                 M_jk = int phi_j phi_k dq; phi'' = (g_{i+1} - g_i)/h      */
/*   2 NODAL:      s = M_L^{-1} m, m_j = int (n0 - rho) phi_j dq = -btilde_j,*/
/*                 i.e. s_j = -btilde_j / h, the lumped projection of        */
/*                 phi'' = n0 - rho (Eq. poisson); per NODE, interpolated    */
/*                 linearly inside each element by the push.                 */
/* d2 has nx entries in every mode (per element for 0/1, per node for 2).    */
/* btilde (b - mean b) is needed only for mode 2 and may be NULL otherwise.  */
/* ------------------------------------------------------------------------ */
int or_field_tables(int32_t nx, double L, const double *Phi, const double *btilde,
                    int32_t d2_mode, double *dphi, double *d2) {
    if (nx < 1) return -1;
    double h = L / (double)nx;
    for (int32_t i = 0; i < nx; ++i) {
        int32_t ip1 = (i + 1) % nx;
        dphi[i] = (Phi[ip1] - Phi[i]) / h;
    }
    if (d2_mode == 2) {
        if (!btilde) return -1;
        for (int32_t j = 0; j < nx; ++j) d2[j] = -btilde[j] / h;
        return 0;
    }
    /* r_j = int phi_h' phi_j: elements j-1 and j each give (h/2) * slope */
    double *r = (double *)malloc(sizeof(double) * (size_t)nx);
    double *g = (double *)malloc(sizeof(double) * (size_t)nx);
    for (int32_t j = 0; j < nx; ++j) {
        int32_t jm1 = (j - 1 + nx) % nx;
        r[j] = 0.5 * h * dphi[jm1] + 0.5 * h * dphi[j];
    }
    if (d2_mode == 0) {
        for (int32_t j = 0; j < nx; ++j) g[j] = r[j] / h;
    } else if (d2_mode == 1) {
        /* consistent mass: element [q_i, q_{i+1}] adds (h/6)[[2,1],[1,2]] */
        double *M = (double *)calloc((size_t)nx * nx, sizeof(double));
        int32_t *piv = (int32_t *)calloc((size_t)nx, sizeof(int32_t));
        for (int32_t e = 0; e < nx; ++e) {
            int32_t i = e, j = (e + 1) % nx;
            M[(size_t)i * nx + i] += 2.0 * h / 6.0;
            M[(size_t)j * nx + j] += 2.0 * h / 6.0;
            M[(size_t)i * nx + j] += 1.0 * h / 6.0;
            M[(size_t)j * nx + i] += 1.0 * h / 6.0;
        }
        for (int32_t j = 0; j < nx; ++j) g[j] = r[j];
        int rc = lu_factor(nx, M, piv);
        if (rc == 0) lu_solve(nx, M, piv, g);
        free(M); free(piv);
        if (rc != 0) { free(r); free(g); return -1; }
    } else {
        free(r); free(g);
        return -1;
    }
    for (int32_t i = 0; i < nx; ++i) {
        int32_t ip1 = (i + 1) % nx;
        d2[i] = (g[ip1] - g[i]) / h;
    }
    free(r); free(g);
    return 0;
}

/* Gather phi_h'(Q_a) and the projected phi_h''(Q_a) for every particle. */
void or_gather(int64_t n, const double *Q, const int32_t *elem, double L, int32_t nx,
               const double *dphi, const double *d2, int32_t d2_mode,
               double *dV, double *d2V) {
    double h = L / (double)nx;
    for (int64_t a = 0; a < n; ++a) {
        int32_t i = elem ? elem[a] : or_element(Q[a], L, nx);
        dV[a] = dphi[i];
        if (d2_mode == 2) {
            int32_t ip1 = (i + 1) % nx;
            double xi = (Q[a] - (double)i * h) / h;
            d2V[a] = d2[i] * (1.0 - xi) + d2[ip1] * xi;
        } else {
            d2V[a] = d2[i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The two halves of the leapfrog (Sec. 5, Eq. sw-evolution).                */
/* Hamilton's equations (App. B, Eq. HamApp) with H_h of Eq. (Hh) give       */
/*   dQ/dt = P, dP/dt = -phi_h'(Q), d(q*)/dt = p* phi_h''(Q), d(p*)/dt = -q* */
/* The fields depend only on (Q, p*), and the velocities of (Q, p*) only on  */
/* (P, q*), so the leapfrog alternates:                                      */
/*   kick : P  <- P  - c phi_h'(Q),   q* <- q* + c p* phi_h''(Q)             */
/*   drift: Q  <- wrap(Q + c P),      p* <- p* - c q*                        */
/* The kick takes the per-particle field values so that a prescribed         */
/* potential (Sec. 3.3 / 7.1) can be fed in directly.                        */
/* ------------------------------------------------------------------------ */
void or_kick_values(int64_t n, const double *p_star, double *P, double *q_star,
                    const double *dV, const double *d2V, double c) {
    for (int64_t a = 0; a < n; ++a) {
        P[a] = P[a] - c * dV[a];
        if (q_star && p_star) q_star[a] = q_star[a] + c * p_star[a] * d2V[a];
    }
}
void or_drift(int64_t n, double *Q, const double *P, const double *q_star,
              double *p_star, double L, double c) {
    for (int64_t a = 0; a < n; ++a) {
        Q[a] = or_wrap(Q[a] + c * P[a], L);
        if (q_star && p_star) p_star[a] = p_star[a] - c * q_star[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics.                                                              */
/*  mass      = sum psi*                        (a Casimir, Sec. 3.1)        */
/*  momentum  = sum (psi* P + q*) = <Gamma_2, p>  (pairing Eq. pairing with  */
/*              the ansatz Eq. sw_f_ansatz)                                  */
/*  kinetic   = sum (psi* P^2/2 + q* P)         (Eq. Hh, m = 1)              */
/*  field     = (1/2) Phi^T A Phi                (Eq. Hh), A assembled       */
/*  H_h       = kinetic + field                                              */
/*  E_amp     = ( (1/L) int_0^L E^2 dq )^{1/2}   (Eq. Eamp), E = -phi_h'     */
/* out = {mass, momentum, kinetic, field, H, E_amp}                          */
/* ------------------------------------------------------------------------ */
static void particle_sums(int64_t a0, int64_t a1, const double *P, const double *q_star,
                          const double *psi_star, nsum out[3]) {
    nsum mass = {0, 0}, mom = {0, 0}, kin = {0, 0};
    for (int64_t a = a0; a < a1; ++a) {
        double qs = q_star ? q_star[a] : 0.0;
        nsum_add(&mass, psi_star[a]);
        nsum_add(&mom, psi_star[a] * P[a] + qs);
        nsum_add(&kin, 0.5 * psi_star[a] * P[a] * P[a] + qs * P[a]);
    }
    out[0] = mass; out[1] = mom; out[2] = kin;
}

void or_diagnostics(int64_t n, const double *P, const double *q_star,
                    const double *psi_star, int32_t nx, double L,
                    const double *Phi, double *out) {
    nsum mass = {0, 0}, mom = {0, 0}, kin = {0, 0};
    if (g_threads <= 1) {
        nsum r[3];
        particle_sums(0, n, P, q_star, psi_star, r);
        mass = r[0]; mom = r[1]; kin = r[2];
    } else {
        const int T = g_threads;
        nsum *part = (nsum *)calloc((size_t)T * 3, sizeof(nsum));
#pragma omp parallel for num_threads(T) schedule(static, 1)
        for (int t = 0; t < T; ++t) {
            int64_t a0, a1;
            block_of(n, T, t, &a0, &a1);
            particle_sums(a0, a1, P, q_star, psi_star, part + 3 * t);
        }
        for (int t = 0; t < T; ++t) {       /* block order */
            nsum_add(&mass, nsum_val(&part[3 * t]));
            nsum_add(&mom, nsum_val(&part[3 * t + 1]));
            nsum_add(&kin, nsum_val(&part[3 * t + 2]));
        }
        free(part);
    }
    double *A = (double *)malloc(sizeof(double) * (size_t)nx * nx);
    or_stiffness(nx, L, A);
    nsum w = {0, 0};
    for (int32_t i = 0; i < nx; ++i)
        for (int32_t j = 0; j < nx; ++j)
            if (A[(size_t)i * nx + j] != 0.0) nsum_add(&w, Phi[i] * A[(size_t)i * nx + j] * Phi[j]);
    free(A);
    double h = L / (double)nx;
    nsum e2 = {0, 0};
    for (int32_t i = 0; i < nx; ++i) {
        double E = -(Phi[(i + 1) % nx] - Phi[i]) / h;   /* constant on element i */
        nsum_add(&e2, E * E * h);                        /* int over element i */
    }
    out[0] = nsum_val(&mass);
    out[1] = nsum_val(&mom);
    out[2] = nsum_val(&kin);
    out[3] = 0.5 * nsum_val(&w);
    out[4] = out[2] + out[3];
    out[5] = sqrt(nsum_val(&e2) / L);
}

/* ------------------------------------------------------------------------ */
/* Whole run: KDK leapfrog (Sec. 5, "leapfrog ... as in standard PIC")       */
/*   field(Q^n, p*^n) -> kick(dt/2) -> drift(dt) -> field(Q^{n+1}, p*^{n+1}) */
/*   -> kick(dt/2)                                                           */
/* with the field step = deposit (Eq. rhs-assembly) -> Galerkin solve        */
/* (Eq. lin-sys with the zero-mean gauge) -> tables.                         */
/* State arrays are updated in place (integer-time values on return).       */
/* If diag != NULL, a record of 7 doubles {t, mass, momentum, kinetic,       */
/* field, H, E_amp} is written at every step s with s % diag_every == 0      */
/* (s = 0 .. n_steps); *n_diag receives the number of records written.       */
/* decorated = 0 runs the point-particle PIC step (q*, p* ignored, may be    */
/* NULL).  store_f32 = 1 keeps the state in FP32 storage: every updated      */
/* value is rounded to FP32, element decisions are taken in FP32 from the    */
/* stored positions, the field tables and the step coefficients dt/2, dt   */
/* are rounded to FP32; arithmetic stays FP64.  Returns 0 on success.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nx, d2_mode, decorated, store_f32;
    double L;
    or_poisson *solver;
    double *b, *btilde, *Phi, *dphi, *d2, *dV, *d2V;
    int32_t *elem;     /* FP32-storage element decisions (store_f32 only) */
} or_field;

/* P2 elements (d2_mode 3): defined below */
int or_p2_field(int64_t n, const double *Q, const double *p_star, const double *psi_star,
                const int32_t *elem, double L, int32_t nx, double *Phi2, double *a_el, double *beta_el);
void or_p2_gather(int64_t n, const double *Q, const int32_t *elem, double L, int32_t nx,
                  const double *a_el, const double *beta_el, double *dV, double *d2V);
void or_p2_energy(int32_t nx, double L, const double *a_el, const double *beta_el, double *W, double *E_amp);

static void decide_elements(or_field *f, int64_t n, const double *Q) {
    for (int64_t a = 0; a < n; ++a) f->elem[a] = or_element_f32(Q[a], f->L, f->nx);
}

static int field_update(or_field *f, int64_t n, const double *Q, const double *p_star,
                        const double *psi_star) {
    if (f->store_f32) decide_elements(f, n, Q);
    if (f->d2_mode == 3) {
        /* P2: dphi <- a (element midpoint phi'), d2 <- beta; Phi <- vertex values */
        double *Phi2 = (double *)malloc(sizeof(double) * 2 * (size_t)f->nx);
        int rc = or_p2_field(n, Q, f->decorated ? p_star : NULL, psi_star, f->store_f32 ? f->elem : NULL,
                             f->L, f->nx, Phi2, f->dphi, f->d2);
        for (int32_t j = 0; j < f->nx; ++j) f->Phi[j] = Phi2[2 * j];
        free(Phi2);
        if (f->store_f32)
            for (int32_t j = 0; j < f->nx; ++j) { f->dphi[j] = to_f32(f->dphi[j]); f->d2[j] = to_f32(f->d2[j]); }
        return rc;
    }
    if (g_threads <= 1 || f->store_f32) {
        or_deposit(n, Q, f->decorated ? p_star : NULL, psi_star, f->store_f32 ? f->elem : NULL,
                   f->L, f->nx, f->b);
    } else {
        /* one mesh per particle block, added in block order */
        const int T = g_threads;
        const int32_t nx = f->nx;
        double *part = (double *)malloc(sizeof(double) * (size_t)T * nx);
#pragma omp parallel for num_threads(T) schedule(static, 1)
        for (int t = 0; t < T; ++t) {
            int64_t a0, a1;
            block_of(n, T, t, &a0, &a1);
            or_deposit(a1 - a0, Q + a0, (f->decorated && p_star) ? p_star + a0 : NULL, psi_star + a0, NULL,
                       f->L, nx, part + (size_t)t * nx);
        }
        for (int32_t j = 0; j < nx; ++j) {
            double v = 0.0;
            for (int t = 0; t < T; ++t) v += part[(size_t)t * nx + j];
            f->b[j] = v;
        }
        free(part);
    }
    double lambda = 0.0;
    or_poisson_solve(f->solver, f->b, f->Phi, &lambda);
    for (int32_t j = 0; j < f->nx; ++j) f->btilde[j] = f->b[j] - lambda;
    int rc = or_field_tables(f->nx, f->L, f->Phi, f->btilde, f->d2_mode, f->dphi, f->d2);
    if (f->store_f32)
        for (int32_t j = 0; j < f->nx; ++j) { f->dphi[j] = to_f32(f->dphi[j]); f->d2[j] = to_f32(f->d2[j]); }
    return rc;
}

/* FP32 storage of the particle state after an update (store_f32 only).  The
 * domain stays [0, L) with the exact L: a position whose FP32 rounding lands
 * on or beyond L is wrapped by L (in FP64) and rounded again. */
static void store_state(const or_field *f, int64_t n, double *Q, double *P, double *qs, double *ps) {
    if (!f->store_f32) return;
    for (int64_t a = 0; a < n; ++a) {
        if (Q) {
            float q = (float)Q[a];
            if ((double)q >= f->L) q = (float)((double)q - f->L);
            if (q < 0.0f) q = (float)((double)q + f->L);
            Q[a] = (double)q;
        }
        P[a] = to_f32(P[a]);
        if (qs) qs[a] = to_f32(qs[a]);
        if (ps) ps[a] = to_f32(ps[a]);
    }
}

static void write_diag(double *rec, double t, int64_t n, const double *P, const double *q_star,
                       const double *psi_star, const or_field *f) {
    double out[6];
    or_diagnostics(n, P, f->decorated ? q_star : NULL, psi_star, f->nx, f->L, f->Phi, out);
    if (f->d2_mode == 3) {        /* P2: field energy and E_amp of the quadratic phi_h */
        or_p2_energy(f->nx, f->L, f->dphi, f->d2, &out[3], &out[5]);
        out[4] = out[2] + out[3];
    }
    rec[0] = t;
    for (int k = 0; k < 6; ++k) rec[1 + k] = out[k];
}

int or_run(int64_t n, double *Q, double *P, double *q_star, double *p_star,
           const double *psi_star, int32_t nx, double L, double dt,
           int32_t d2_mode, int32_t decorated, int32_t n_steps, int32_t diag_every,
           double *diag, int32_t *n_diag, double *Phi_out, int32_t store_f32) {
    or_field f;
    memset(&f, 0, sizeof(f));
    f.nx = nx; f.L = L; f.d2_mode = d2_mode; f.decorated = decorated; f.store_f32 = store_f32;
    f.elem = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    f.solver = or_poisson_new(nx, L);
    if (!f.solver) return -1;
    f.b = (double *)calloc((size_t)nx, sizeof(double));
    f.btilde = (double *)calloc((size_t)nx, sizeof(double));
    f.Phi = (double *)calloc((size_t)nx, sizeof(double));
    f.dphi = (double *)calloc((size_t)nx, sizeof(double));
    f.d2 = (double *)calloc((size_t)nx, sizeof(double));
    f.dV = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    f.d2V = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *qs = decorated ? q_star : NULL;
    double *ps = decorated ? p_star : NULL;
    int rc = field_update(&f, n, Q, ps, psi_star);
    int32_t nd = 0;
    if (rc == 0 && diag && diag_every > 0) write_diag(diag + 7 * (nd++), 0.0, n, P, qs, psi_star, &f);
    /* FP32 storage keeps the step coefficients in FP32 as well */
    const double half = store_f32 ? to_f32(0.5 * dt) : 0.5 * dt;
    const double full = store_f32 ? to_f32(dt) : dt;
    /* threaded particle loops (see or_set_threads): P1 field, FP64 storage */
    const int T = (g_threads > 1 && d2_mode != 3 && !store_f32) ? g_threads : 1;
    for (int32_t s = 1; rc == 0 && s <= n_steps; ++s) {
        if (T > 1) {
#pragma omp parallel for num_threads(T) schedule(static, 1)
            for (int t = 0; t < T; ++t) {
                int64_t a0, a1;
                block_of(n, T, t, &a0, &a1);
                or_gather(a1 - a0, Q + a0, NULL, L, nx, f.dphi, f.d2, d2_mode, f.dV + a0, f.d2V + a0);
                or_kick_values(a1 - a0, ps ? ps + a0 : NULL, P + a0, qs ? qs + a0 : NULL, f.dV + a0,
                               f.d2V + a0, half);
                or_drift(a1 - a0, Q + a0, P + a0, qs ? qs + a0 : NULL, ps ? ps + a0 : NULL, L, full);
            }
            rc = field_update(&f, n, Q, ps, psi_star);
            if (rc != 0) break;
#pragma omp parallel for num_threads(T) schedule(static, 1)
            for (int t = 0; t < T; ++t) {
                int64_t a0, a1;
                block_of(n, T, t, &a0, &a1);
                or_gather(a1 - a0, Q + a0, NULL, L, nx, f.dphi, f.d2, d2_mode, f.dV + a0, f.d2V + a0);
                or_kick_values(a1 - a0, ps ? ps + a0 : NULL, P + a0, qs ? qs + a0 : NULL, f.dV + a0,
                               f.d2V + a0, half);
            }
            if (diag && diag_every > 0 && s % diag_every == 0)
                write_diag(diag + 7 * (nd++), (double)s * dt, n, P, qs, psi_star, &f);
            continue;
        }
        if (d2_mode == 3) or_p2_gather(n, Q, store_f32 ? f.elem : NULL, L, nx, f.dphi, f.d2, f.dV, f.d2V);
        else or_gather(n, Q, store_f32 ? f.elem : NULL, L, nx, f.dphi, f.d2, d2_mode, f.dV, f.d2V);
        or_kick_values(n, ps, P, qs, f.dV, f.d2V, half);
        store_state(&f, n, NULL, P, qs, NULL);
        or_drift(n, Q, P, qs, ps, L, full);
        store_state(&f, n, Q, P, qs, ps);
        rc = field_update(&f, n, Q, ps, psi_star);
        if (rc != 0) break;
        if (d2_mode == 3) or_p2_gather(n, Q, store_f32 ? f.elem : NULL, L, nx, f.dphi, f.d2, f.dV, f.d2V);
        else or_gather(n, Q, store_f32 ? f.elem : NULL, L, nx, f.dphi, f.d2, d2_mode, f.dV, f.d2V);
        or_kick_values(n, ps, P, qs, f.dV, f.d2V, half);
        store_state(&f, n, NULL, P, qs, NULL);
        if (diag && diag_every > 0 && s % diag_every == 0)
            write_diag(diag + 7 * (nd++), (double)s * dt, n, P, qs, psi_star, &f);
    }
    if (n_diag) *n_diag = nd;
    if (Phi_out) for (int32_t j = 0; j < nx; ++j) Phi_out[j] = f.Phi[j];
    or_poisson_free(f.solver);
    free(f.b); free(f.btilde); free(f.Phi); free(f.dphi); free(f.d2); free(f.dV); free(f.d2V);
    free(f.elem);
    return rc;
}

/* Field of a given state: deposit -> solve -> tables, all outputs length nx. */
int or_field_of_state(int64_t n, const double *Q, const double *p_star, const double *psi_star,
                      int32_t nx, double L, int32_t d2_mode, int32_t decorated,
                      double *b, double *btilde, double *Phi, double *dphi, double *d2) {
    or_field f;
    memset(&f, 0, sizeof(f));
    f.nx = nx; f.L = L; f.d2_mode = d2_mode; f.decorated = decorated;
    f.solver = or_poisson_new(nx, L);
    if (!f.solver) return -1;
    f.b = b; f.btilde = btilde; f.Phi = Phi; f.dphi = dphi; f.d2 = d2;
    int rc = field_update(&f, n, Q, decorated ? p_star : NULL, psi_star);
    or_poisson_free(f.solver);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Initialisation on a phase-space lattice (reading of Sec. 4.2 / Alg. 1     */
/* with each lattice cell taken as the cluster S_a of the continuum f0).     */
/*   centre      (x_i, v_j) = ((i + 1/2) dx, vmin + (j + 1/2) dv)            */
/*   particle    Q = wrap(x_i + jx dx), P = v_j + jv dv  (jitter in cells)   */
/*   psi*        = f0(x_i, v_j) dx dv                     (midpoint weight)  */
/*   p*          = int_cell f0(q,p) c(Q, q) dq dp,   c = (L/2pi) sin(2pi(Q-q)/L)  (Sec. 4.2) */
/*   q*          = - int_cell f0(q,p) (P - p) dq dp                (Eq. moment-def)      */
/* with the cell integrals taken by an n x n Gauss-Legendre rule.  Particle  */
/* index = i * nv + j (x-major).                                            */
/* f0(x, v) = (1 + alpha cos(kx x)) * sum_m amp_m (c0_m + c2_m v^2)          */
/*            exp(-beta_m (v - u_m)^2)                                       */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on the        */
/* Legendre polynomial P_n (three-term recurrence).                          */
int or_gauss_legendre(int32_t npts, double *x, double *w) {
    if (npts < 1 || npts > 64) return -1;
    const double pi = 3.14159265358979323846;
    for (int32_t k = 0; k < npts; ++k) {
        /* initial guess near the k-th largest root, then Newton on P_n */
        double z = cos(pi * ((double)k + 0.75) / ((double)npts + 0.5));
        double pn = 0.0, pnm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            pn = z; pnm1 = 1.0;
            if (npts == 1) { pn = z; pnm1 = 1.0; }
            for (int32_t m = 2; m <= npts; ++m) {
                double pm = ((2.0 * m - 1.0) * z * pn - (m - 1.0) * pnm1) / (double)m;
                pnm1 = pn; pn = pm;
            }
            /* P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1) */
            dp = (double)npts * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        pn = z; pnm1 = 1.0;
        for (int32_t m = 2; m <= npts; ++m) {
            double pm = ((2.0 * m - 1.0) * z * pn - (m - 1.0) * pnm1) / (double)m;
            pnm1 = pn; pn = pm;
        }
        dp = (double)npts * (z * pn - pnm1) / (z * z - 1.0);
        x[k] = -z;                         /* ascending order */
        w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

typedef struct {
    double alpha, kx;
    int32_t n_terms;
    double amp[4], c0[4], c2[4], beta[4], u[4];
} or_f0;

static double f0_eval(const or_f0 *f, double x, double v) {
    double s = 0.0;
    for (int32_t m = 0; m < f->n_terms; ++m)
        s += f->amp[m] * (f->c0[m] + f->c2[m] * v * v) * exp(-f->beta[m] * (v - f->u[m]) * (v - f->u[m]));
    return (1.0 + f->alpha * cos(f->kx * x)) * s;
}

int or_init_lattice(int32_t nq, int32_t nv, double L, double vmin, double vmax,
                    double alpha, double kx, int32_t n_terms, const double *amp,
                    const double *c0, const double *c2, const double *beta,
                    const double *u, int32_t quad_order, int32_t decorate,
                    const double *jitter_x, const double *jitter_v,
                    double *Q, double *P, double *q_star, double *p_star, double *psi_star) {
    if (n_terms < 1 || n_terms > 4 || nq < 1 || nv < 1) return -1;
    or_f0 f;
    memset(&f, 0, sizeof(f));
    f.alpha = alpha; f.kx = kx; f.n_terms = n_terms;
    for (int32_t m = 0; m < n_terms; ++m) {
        f.amp[m] = amp[m]; f.c0[m] = c0[m]; f.c2[m] = c2[m]; f.beta[m] = beta[m]; f.u[m] = u[m];
    }
    double gx[64], gw[64];
    if (decorate && or_gauss_legendre(quad_order, gx, gw) != 0) return -1;
    const double pi = 3.14159265358979323846;
    double dx = L / (double)nq, dv = (vmax - vmin) / (double)nv;
    for (int32_t i = 0; i < nq; ++i) {
        double xc = ((double)i + 0.5) * dx;
        for (int32_t j = 0; j < nv; ++j) {
            int64_t a = (int64_t)i * nv + j;
            double vc = vmin + ((double)j + 0.5) * dv;
            double jx = jitter_x ? jitter_x[a] : 0.0;
            double jv = jitter_v ? jitter_v[a] : 0.0;
            double Qa = or_wrap(xc + jx * dx, L);
            double Pa = vc + jv * dv;
            Q[a] = Qa;
            P[a] = Pa;
            psi_star[a] = f0_eval(&f, xc, vc) * dx * dv;
            if (!decorate) {
                if (q_star) q_star[a] = 0.0;
                if (p_star) p_star[a] = 0.0;
                continue;
            }
            double ps = 0.0, qs = 0.0;
            for (int32_t r = 0; r < quad_order; ++r) {
                double q = xc + 0.5 * dx * gx[r];
                for (int32_t s = 0; s < quad_order; ++s) {
                    double p = vc + 0.5 * dv * gx[s];
                    double wgt = gw[r] * gw[s] * 0.25 * dx * dv;
                    double fv = f0_eval(&f, q, p);
                    ps += wgt * fv * (L / (2.0 * pi)) * sin(2.0 * pi * (Qa - q) / L);
                    qs += -wgt * fv * (Pa - p);
                }
            }
            p_star[a] = ps;
            q_star[a] = qs;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Decorated-particle initialization from marker particles                   */
/* (Sec. 4.1-4.2 "Initialization", Alg. lumping_procedure, Eqs. psi-star and */
/* moment-def, with the periodic c of the T^d subsection).                   */
/*                                                                           */
/* Reading of "k-means on the phase-space coordinates" on the torus: Lloyd    */
/* iterations in (q, p) with the minimum-image difference in q.  The         */
/* assignment is a decision, taken in FP32 (the precision of the GPU path):  */
/* dq = Qm - cq (floats, folded once into [-L/2, L/2)), dp = Pm - cp,         */
/* d2 = dq*dq + dp*dp, ties to the smaller cluster index.  Centers are the   */
/* psi-weighted member means in FP64, q unwrapped about the current center   */
/* and wrapped into [0, L); an empty cluster keeps its center.               */
/* ------------------------------------------------------------------------ */
static float km_fold(float d, float L, float half) {
    if (d >= half) return d - L;
    if (d < -half) return d + L;
    return d;
}
static double km_fold_d(double d, double L) {
    if (d >= 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

/* nearest center of every marker (FP32 decision) */
void or_kmeans_assign(int64_t M, const double *Qm, const double *Pm, int32_t K,
                      const double *cq, const double *cp, double L, int32_t *assign) {
    const float Lf = (float)L, half = (float)(0.5 * L);
    for (int64_t A = 0; A < M; ++A) {
        const float qf = (float)Qm[A], pf = (float)Pm[A];
        float best = INFINITY;
        int32_t bi = 0;
        for (int32_t k = 0; k < K; ++k) {
            const float dq = km_fold(qf - (float)cq[k], Lf, half);
            const float dp = pf - (float)cp[k];
            const float d2 = dq * dq + dp * dp;
            if (d2 < best) { best = d2; bi = k; }
        }
        assign[A] = bi;
    }
}

/* psi-weighted member means about the given centers (FP64, marker order);
   w_sum[k] = 0 leaves the center unchanged */
void or_kmeans_means(int64_t M, const double *Qm, const double *Pm, const double *wm,
                     const int32_t *assign, int32_t K, double L, const double *cq, const double *cp,
                     double *mq, double *mp, double *w_sum) {
    double *sq = (double *)calloc((size_t)K, sizeof(double));
    double *sp = (double *)calloc((size_t)K, sizeof(double));
    for (int32_t k = 0; k < K; ++k) w_sum[k] = 0.0;
    for (int64_t A = 0; A < M; ++A) {
        const int32_t k = assign[A];
        w_sum[k] += wm[A];
        sq[k] += wm[A] * km_fold_d(Qm[A] - cq[k], L);
        sp[k] += wm[A] * Pm[A];
    }
    for (int32_t k = 0; k < K; ++k) {
        if (w_sum[k] != 0.0) {
            mq[k] = or_wrap(cq[k] + sq[k] / w_sum[k], L);
            mp[k] = sp[k] / w_sum[k];
        } else {
            mq[k] = cq[k];
            mp[k] = cp[k];
        }
    }
    free(sq);
    free(sp);
}

/* n_iter Lloyd iterations from the given centers (updated in place), then the
   final assignment */
void or_kmeans(int64_t M, const double *Qm, const double *Pm, const double *wm, int32_t K,
               double L, int32_t n_iter, double *cq, double *cp, int32_t *assign) {
    double *mq = (double *)malloc(sizeof(double) * (size_t)K);
    double *mp = (double *)malloc(sizeof(double) * (size_t)K);
    double *ws = (double *)malloc(sizeof(double) * (size_t)K);
    for (int32_t it = 0; it < n_iter; ++it) {
        or_kmeans_assign(M, Qm, Pm, K, cq, cp, L, assign);
        or_kmeans_means(M, Qm, Pm, wm, assign, K, L, cq, cp, mq, mp, ws);
        memcpy(cq, mq, sizeof(double) * (size_t)K);
        memcpy(cp, mp, sizeof(double) * (size_t)K);
    }
    or_kmeans_assign(M, Qm, Pm, K, cq, cp, L, assign);
    free(mq);
    free(mp);
    free(ws);
}

/* Alg. lumping_procedure for the clusters of `assign` (centers cq, cp: the q
   unwrap reference of each cluster).  For every non-empty cluster, in cluster
   order: psi* = sum psi (Eq. psi-star); (Q, P) = the member nearest (FP32
   decision, ties to the smaller marker index) to the psi-weighted mean;
   p* = sum psi (L/2pi) sin(2pi (Q - Qm)/L), q* = -sum psi (P - Pm)
   (Eq. moment-def with the periodic c).  Returns the number of particles. */
int64_t or_lump(int64_t M, const double *Qm, const double *Pm, const double *wm,
                const int32_t *assign, int32_t K, double L, const double *cq, const double *cp,
                double *Q, double *P, double *q_star, double *p_star, double *psi_star) {
    const double pi = 3.14159265358979323846;
    const float Lf = (float)L, half = (float)(0.5 * L);
    double *mq = (double *)malloc(sizeof(double) * (size_t)K);
    double *mp = (double *)malloc(sizeof(double) * (size_t)K);
    double *ws = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t *a0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    float *best = (float *)malloc(sizeof(float) * (size_t)K);
    or_kmeans_means(M, Qm, Pm, wm, assign, K, L, cq, cp, mq, mp, ws);
    for (int32_t k = 0; k < K; ++k) { a0[k] = -1; best[k] = INFINITY; }
    for (int64_t A = 0; A < M; ++A) {
        const int32_t k = assign[A];
        const float dq = km_fold((float)Qm[A] - (float)mq[k], Lf, half);
        const float dp = (float)Pm[A] - (float)mp[k];
        const float d2 = dq * dq + dp * dp;
        if (a0[k] < 0 || d2 < best[k]) { best[k] = d2; a0[k] = A; }
    }
    /* compact index of each non-empty cluster */
    int64_t n = 0;
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    for (int32_t k = 0; k < K; ++k) {
        slot[k] = (a0[k] >= 0) ? n++ : -1;
        if (slot[k] < 0) continue;
        Q[slot[k]] = Qm[a0[k]];
        P[slot[k]] = Pm[a0[k]];
        psi_star[slot[k]] = 0.0;
        p_star[slot[k]] = 0.0;
        q_star[slot[k]] = 0.0;
    }
    for (int64_t A = 0; A < M; ++A) {
        const int64_t s = slot[assign[A]];
        psi_star[s] += wm[A];
        p_star[s] += wm[A] * (L / (2.0 * pi)) * sin(2.0 * pi * (Q[s] - Qm[A]) / L);
        q_star[s] += -wm[A] * (P[s] - Pm[A]);
    }
    free(mq); free(mp); free(ws); free(a0); free(best); free(slot);
    return n;
}

/* ------------------------------------------------------------------------ */
/* P2 (quadratic Lagrange) elements, V_h^(2) of Sec. 5 (degree k = 2):       */
/* phi_h' and phi_h'' both come from the element's quadratic, no projection. */
/* Degrees of freedom: vertex j -> 2j, midpoint of element i -> 2i + 1      */
/* (2 nx in all, periodic).  On element i with xi = (Q - q_i)/h:             */
/*   N_v0 = (1-xi)(1-2xi), N_m = 4 xi (1-xi), N_v1 = xi (2xi - 1),           */
/*   h N' = (4xi - 3, 4 - 8xi, 4xi - 1).                                     */
/* Eq. lin-sys with the P2 stiffness (element (1/3h)[[7,-8,1],[-8,16,-8],    */
/* [1,-8,7]]), Eq. rhs-assembly b_k = sum psi N_k(Q) - p* N_k'(Q), and the   */
/* zero-mean test space as a bordered system with c_k = int N_k (h/3 per    */
/* vertex, 2h/3 per midpoint): A Phi + lambda c = b, c^T Phi = 0.  Dense.    */
/* Outputs per element i: a_i = phi_h' at the element midpoint and           */
/* beta_i with phi_h'(xi) = a_i + beta_i (1 - 2 xi), phi_h'' = -2 beta_i/h.  */
/* ------------------------------------------------------------------------ */
static void p2_basis(double xi, double h, double N[3], double dN[3]) {
    N[0] = (1.0 - xi) * (1.0 - 2.0 * xi);
    N[1] = 4.0 * xi * (1.0 - xi);
    N[2] = xi * (2.0 * xi - 1.0);
    dN[0] = (4.0 * xi - 3.0) / h;
    dN[1] = (4.0 - 8.0 * xi) / h;
    dN[2] = (4.0 * xi - 1.0) / h;
}

int or_p2_field(int64_t n, const double *Q, const double *p_star, const double *psi_star,
                const int32_t *elem, double L, int32_t nx, double *Phi2, double *a_el, double *beta_el) {
    const int32_t nd = 2 * nx, m = nd + 1;
    const double h = L / (double)nx;
    double *M = (double *)calloc((size_t)m * m, sizeof(double));
    int32_t *piv = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    double *x = (double *)calloc((size_t)m, sizeof(double));
    if (!M || !piv || !x) { free(M); free(piv); free(x); return -1; }
    static const double K[3][3] = {{7, -8, 1}, {-8, 16, -8}, {1, -8, 7}};
    for (int32_t e = 0; e < nx; ++e) {
        const int32_t d[3] = {2 * e, 2 * e + 1, (2 * e + 2) % nd};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[(size_t)d[r] * m + d[c]] += K[r][c] / (3.0 * h);
        M[(size_t)d[0] * m + nd] += h / 6.0;
        M[(size_t)d[2] * m + nd] += h / 6.0;
        M[(size_t)d[1] * m + nd] += 2.0 * h / 3.0;
        M[(size_t)nd * m + d[0]] += h / 6.0;
        M[(size_t)nd * m + d[2]] += h / 6.0;
        M[(size_t)nd * m + d[1]] += 2.0 * h / 3.0;
    }
    for (int64_t a = 0; a < n; ++a) {
        const int32_t e = elem ? elem[a] : or_element(Q[a], L, nx);
        const double xi = (Q[a] - (double)e * h) / h;
        double N[3], dN[3];
        p2_basis(xi, h, N, dN);
        const int32_t d[3] = {2 * e, 2 * e + 1, (2 * e + 2) % nd};
        for (int k = 0; k < 3; ++k)
            x[d[k]] += psi_star[a] * N[k] - (p_star ? p_star[a] : 0.0) * dN[k];
    }
    x[nd] = 0.0;
    int rc = lu_factor(m, M, piv);
    if (rc == 0) {
        lu_solve(m, M, piv, x);
        for (int32_t k = 0; k < nd; ++k) Phi2[k] = x[k];
        for (int32_t e = 0; e < nx; ++e) {
            const double v0 = x[2 * e], vm = x[2 * e + 1], v1 = x[(2 * e + 2) % nd];
            a_el[e] = (v1 - v0) / h;                           /* phi' at xi = 1/2 */
            beta_el[e] = (4.0 * vm - 2.0 * v0 - 2.0 * v1) / h;  /* phi'(xi) = a + beta (1 - 2 xi) */
        }
    }
    free(M); free(piv); free(x);
    return rc;
}

/* phi_h'(Q) and phi_h''(Q) from the P2 element tables */
void or_p2_gather(int64_t n, const double *Q, const int32_t *elem, double L, int32_t nx,
                  const double *a_el, const double *beta_el, double *dV, double *d2V) {
    const double h = L / (double)nx;
    for (int64_t a = 0; a < n; ++a) {
        const int32_t e = elem ? elem[a] : or_element(Q[a], L, nx);
        const double xi = (Q[a] - (double)e * h) / h;
        dV[a] = a_el[e] + beta_el[e] * (1.0 - 2.0 * xi);
        d2V[a] = -2.0 * beta_el[e] / h;
    }
}

/* W = (1/2) int phi_h'^2 = (h/2) sum (a^2 + beta^2/3); E_amp = ((1/L) int phi_h'^2)^(1/2) */
void or_p2_energy(int32_t nx, double L, const double *a_el, const double *beta_el, double *W, double *E_amp) {
    const double h = L / (double)nx;
    double s = 0.0;
    for (int32_t e = 0; e < nx; ++e) s += h * (a_el[e] * a_el[e] + beta_el[e] * beta_el[e] / 3.0);
    *W = 0.5 * s;
    *E_amp = sqrt(s / L);
}
