/*
 * swpic2d_oracle.c -- plain, slow, FP64 CPU oracle for the 2D2V periodic
 * monopole-dipole (k = 2) Scovel-Weinstein decorated-particle step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and never calls it.
 *
 * The model is the general-d form of the paper (Sec. 3.3, Eq. swpic_poisson and
 * Eq. swpic_dynamics) on the torus T^2 (end of Sec. 3.3), with S_h = delta
 * and units e = m = eps0 = 1:
 *   state of decorated particle a: Q, P, q*, p* in R^2 (Q on the torus), psi* > 0
 *   potential: phi_h in a finite-element subspace E of H^1(T^2) with
 *       int grad phi_h . grad v = sum_a [psi*_a v(Q_a) - p*_a . grad v(Q_a)] - n0 int v
 *       for every v in E, zero mean                                    (Eq. swpic_poisson)
 *   motion: dQ/dt = P, dP/dt = -grad phi_h(Q), d(p*)/dt = -q*,
 *           d(q*)/dt = (grad grad phi_h)(Q) p*, psi* constant             (Eq. swpic_dynamics)
 * Readings (the paper gives no 2D discretisation):
 *   E = periodic bilinear (Q1) elements on an nx x ny uniform mesh of
 *       [0, Lx) x [0, Ly); node (i, j) at (i hx, j hy), index j nx + i;
 *       cell (i, j) = [i hx, (i+1) hx) x [j hy, (j+1) hy)
 *   grad grad phi_h is taken, as in 1D (reading LUMPED), from the lumped-mass
 *       L2 projection g of grad phi_h onto E (each component): g_j =
 *       int grad phi_h N_j / int N_j, and (grad grad phi_h)_{ik} := d_k g_i.
 *   time: KDK leapfrog on the split (P, q*) kick / (Q, p*) drift (Sec. 5).
 *
 * Integrals are taken by the 2 x 2 Gauss rule per cell, which is exact for
 * every integrand here (at most quadratic in each coordinate).  Nothing is
 * blocked or fused; linear algebra is one dense LU of the bordered system.
 * Build with -ffp-contract=off (x86 and aarch64 round alike).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Mesh geometry                                                             */
/* ------------------------------------------------------------------------ */

/* Wrap a coordinate into [0, L); a value that rounds up to L maps to 0. */
static double wrap2(double Q, double L) {
    double w = Q - L * floor(Q / L);
    if (w >= L) w -= L;
    if (w < 0.0) w += L;
    return w;
}

/* Cell index along one axis: floor(Q/h) clamped to [0, n-1] (a particle on
 * a mesh line belongs to the cell on its right / above). */
int32_t or2d_cell(double Q, double L, int32_t n) {
    double s = floor(Q / (L / (double)n));
    int32_t i = (s != s) ? 0 : (int32_t)s;
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    return i;
}

/* The same decision taken in FP32 from an FP32-stored coordinate:
 * floor(fl32(fl32(Q) * fl32(n/L))), clamped. */
int32_t or2d_cell_f32(double Q, double L, int32_t n) {
    float q = (float)Q;
    float inv_h = (float)((double)n / L);
    float s = floorf(q * inv_h);
    int32_t i = (s != s) ? 0 : (int32_t)s;
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    return i;
}

/* Bilinear basis of the four corners of a cell at local (xi, eta) in [0,1]^2,
 * corner order c = 0:(0,0) 1:(1,0) 2:(0,1) 3:(1,1); N and its gradient. */
static void q1_basis(double xi, double eta, double hx, double hy, double N[4], double Nx[4], double Ny[4]) {
    N[0] = (1.0 - xi) * (1.0 - eta);
    N[1] = xi * (1.0 - eta);
    N[2] = (1.0 - xi) * eta;
    N[3] = xi * eta;
    Nx[0] = -(1.0 - eta) / hx; Nx[1] = (1.0 - eta) / hx; Nx[2] = -eta / hx; Nx[3] = eta / hx;
    Ny[0] = -(1.0 - xi) / hy;  Ny[1] = -xi / hy;         Ny[2] = (1.0 - xi) / hy; Ny[3] = xi / hy;
}

/* Global node indices of the corners of cell (i, j). */
static void cell_nodes(int32_t i, int32_t j, int32_t nx, int32_t ny, int32_t d[4]) {
    const int32_t i1 = (i + 1) % nx, j1 = (j + 1) % ny;
    d[0] = j * nx + i; d[1] = j * nx + i1; d[2] = j1 * nx + i; d[3] = j1 * nx + i1;
}

static const double GP[2] = {0.21132486540518711775, 0.78867513459481288225};  /* (1 -+ 1/sqrt 3)/2 */

/* ------------------------------------------------------------------------ */
/* Deposit (right-hand side of Eq. swpic_poisson with S_h = delta):          */
/*   b_j = sum_a [ psi*_a N_j(Q_a) - p*_a . grad N_j(Q_a) ]                  */
/* cx, cy: optional cell decisions (e.g. taken in FP32); ps may be NULL.     */
/* ------------------------------------------------------------------------ */
void or2d_deposit(int64_t n, const double *Qx, const double *Qy, const double *psx, const double *psy,
                  const double *psi, const int32_t *cx, const int32_t *cy, double Lx, double Ly,
                  int32_t nx, int32_t ny, double *b) {
    const double hx = Lx / nx, hy = Ly / ny;
    memset(b, 0, sizeof(double) * (size_t)nx * ny);
    for (int64_t a = 0; a < n; ++a) {
        const int32_t i = cx ? cx[a] : or2d_cell(Qx[a], Lx, nx);
        const int32_t j = cy ? cy[a] : or2d_cell(Qy[a], Ly, ny);
        const double xi = (Qx[a] - i * hx) / hx, eta = (Qy[a] - j * hy) / hy;
        double N[4], Nx[4], Ny[4];
        int32_t d[4];
        q1_basis(xi, eta, hx, hy, N, Nx, Ny);
        cell_nodes(i, j, nx, ny, d);
        for (int c = 0; c < 4; ++c) {
            double v = psi[a] * N[c];
            if (psx) v -= psx[a] * Nx[c] + psy[a] * Ny[c];
            b[d[c]] += v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra (partial pivoting)                                   */
/* ------------------------------------------------------------------------ */
static int lu2_factor(int32_t m, double *M, int32_t *piv) {
    for (int32_t k = 0; k < m; ++k) {
        int32_t p = k;
        double best = fabs(M[(size_t)k * m + k]);
        for (int32_t r = k + 1; r < m; ++r)
            if (fabs(M[(size_t)r * m + k]) > best) { best = fabs(M[(size_t)r * m + k]); p = r; }
        if (best == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int32_t c = 0; c < m; ++c) {
                double t = M[(size_t)k * m + c]; M[(size_t)k * m + c] = M[(size_t)p * m + c]; M[(size_t)p * m + c] = t;
            }
        const double inv = 1.0 / M[(size_t)k * m + k];
        for (int32_t r = k + 1; r < m; ++r) {
            const double f = M[(size_t)r * m + k] * inv;
            M[(size_t)r * m + k] = f;
            if (f != 0.0)
                for (int32_t c = k + 1; c < m; ++c) M[(size_t)r * m + c] -= f * M[(size_t)k * m + c];
        }
    }
    return 0;
}

/* Rows were swapped whole in the factorisation, so all swaps go first. */
static void lu2_solve(int32_t m, const double *M, const int32_t *piv, double *x) {
    for (int32_t k = 0; k < m; ++k) {
        const int32_t p = piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
    for (int32_t k = 0; k < m; ++k)
        for (int32_t r = k + 1; r < m; ++r) x[r] -= M[(size_t)r * m + k] * x[k];
    for (int32_t k = m - 1; k >= 0; --k) {
        double s = x[k];
        for (int32_t c = k + 1; c < m; ++c) s -= M[(size_t)k * m + c] * x[c];
        x[k] = s / M[(size_t)k * m + k];
    }
}

/* ------------------------------------------------------------------------ */
/* Poisson solve: the Galerkin system of Eq. swpic_poisson on E = Q1,        */
/*   K Phi + lambda m = b,  m^T Phi = 0,                                      */
/* K_jk = int grad N_j . grad N_k, m_j = int N_j (zero-mean gauge; lambda is  */
/* the neutralising background n0 = sum b / |Omega|).  Assembled by the 2 x 2 */
/* Gauss rule per cell; factored once per mesh.                               */
/* ------------------------------------------------------------------------ */
typedef struct or2d_solver {
    int32_t nx, ny, m;
    double Lx, Ly;
    double *K;       /* the assembled stiffness (nx ny)^2, kept for the energy */
    double *M;       /* LU of the bordered matrix */
    int32_t *piv;
} or2d_solver;

void or2d_stiffness(int32_t nx, int32_t ny, double Lx, double Ly, double *K) {
    const int32_t N = nx * ny;
    const double hx = Lx / nx, hy = Ly / ny;
    memset(K, 0, sizeof(double) * (size_t)N * N);
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int32_t d[4];
            cell_nodes(i, j, nx, ny, d);
            for (int gx = 0; gx < 2; ++gx)
                for (int gy = 0; gy < 2; ++gy) {
                    double N4[4], Nx[4], Ny[4];
                    q1_basis(GP[gx], GP[gy], hx, hy, N4, Nx, Ny);
                    const double w = 0.25 * hx * hy;
                    for (int r = 0; r < 4; ++r)
                        for (int c = 0; c < 4; ++c)
                            K[(size_t)d[r] * N + d[c]] += w * (Nx[r] * Nx[c] + Ny[r] * Ny[c]);
                }
        }
}

or2d_solver *or2d_solver_new(int32_t nx, int32_t ny, double Lx, double Ly) {
    const int32_t N = nx * ny, m = N + 1;
    or2d_solver *s = (or2d_solver *)calloc(1, sizeof(or2d_solver));
    if (!s) return NULL;
    s->nx = nx; s->ny = ny; s->m = m; s->Lx = Lx; s->Ly = Ly;
    s->K = (double *)malloc(sizeof(double) * (size_t)N * N);
    s->M = (double *)calloc((size_t)m * m, sizeof(double));
    s->piv = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    if (!s->K || !s->M || !s->piv) { free(s->K); free(s->M); free(s->piv); free(s); return NULL; }
    or2d_stiffness(nx, ny, Lx, Ly, s->K);
    const double mass = (Lx / nx) * (Ly / ny);      /* int N_j (four quarter-cells) */
    for (int32_t r = 0; r < N; ++r) {
        memcpy(s->M + (size_t)r * m, s->K + (size_t)r * N, sizeof(double) * N);
        s->M[(size_t)r * m + N] = mass;
        s->M[(size_t)N * m + r] = mass;
    }
    if (lu2_factor(m, s->M, s->piv) != 0) { free(s->K); free(s->M); free(s->piv); free(s); return NULL; }
    return s;
}

void or2d_solver_free(or2d_solver *s) {
    if (!s) return;
    free(s->K); free(s->M); free(s->piv); free(s);
}

void or2d_solver_apply(const or2d_solver *s, const double *b, double *Phi, double *lambda) {
    const int32_t N = s->nx * s->ny;
    double *x = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    memcpy(x, b, sizeof(double) * N);
    x[N] = 0.0;
    lu2_solve(s->m, s->M, s->piv, x);
    memcpy(Phi, x, sizeof(double) * N);
    if (lambda) *lambda = x[N];
    free(x);
}

/* One-shot solve (factors the mesh's matrix each call). */
int or2d_solve(int32_t nx, int32_t ny, double Lx, double Ly, const double *b, double *Phi, double *lambda) {
    or2d_solver *s = or2d_solver_new(nx, ny, Lx, Ly);
    if (!s) return -1;
    or2d_solver_apply(s, b, Phi, lambda);
    or2d_solver_free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lumped-mass projection of grad phi_h onto E (reading of the paper's       */
/* auxiliary projection, as in 1D):  g_j = int grad phi_h N_j / int N_j.     */
/* ------------------------------------------------------------------------ */
void or2d_project(int32_t nx, int32_t ny, double Lx, double Ly, const double *Phi, double *gx, double *gy) {
    const int32_t N = nx * ny;
    const double hx = Lx / nx, hy = Ly / ny;
    memset(gx, 0, sizeof(double) * N);
    memset(gy, 0, sizeof(double) * N);
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int32_t d[4];
            cell_nodes(i, j, nx, ny, d);
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    double N4[4], Nx[4], Ny[4];
                    q1_basis(GP[a], GP[c], hx, hy, N4, Nx, Ny);
                    double ex = 0.0, ey = 0.0;
                    for (int k = 0; k < 4; ++k) { ex += Phi[d[k]] * Nx[k]; ey += Phi[d[k]] * Ny[k]; }
                    const double w = 0.25 * hx * hy;
                    for (int k = 0; k < 4; ++k) { gx[d[k]] += w * ex * N4[k]; gy[d[k]] += w * ey * N4[k]; }
                }
        }
    const double inv_m = 1.0 / (hx * hy);
    for (int32_t k = 0; k < N; ++k) { gx[k] *= inv_m; gy[k] *= inv_m; }
}

/* ------------------------------------------------------------------------ */
/* Gather at the particles: grad phi_h(Q) = sum_j Phi_j grad N_j(Q) and      */
/* H_ik(Q) = d_k g_i(Q) = sum_j g_i,j d_k N_j(Q).  Out: Ex = d_x phi,         */
/* Ey = d_y phi, Hxx = d_x g_x, Hxy = d_y g_x, Hyx = d_x g_y, Hyy = d_y g_y.  */
/* ------------------------------------------------------------------------ */
void or2d_gather(int64_t n, const double *Qx, const double *Qy, const int32_t *cx, const int32_t *cy,
                 double Lx, double Ly, int32_t nx, int32_t ny, const double *Phi, const double *gx,
                 const double *gy, double *Ex, double *Ey, double *Hxx, double *Hxy, double *Hyx, double *Hyy) {
    const double hx = Lx / nx, hy = Ly / ny;
    for (int64_t a = 0; a < n; ++a) {
        const int32_t i = cx ? cx[a] : or2d_cell(Qx[a], Lx, nx);
        const int32_t j = cy ? cy[a] : or2d_cell(Qy[a], Ly, ny);
        const double xi = (Qx[a] - i * hx) / hx, eta = (Qy[a] - j * hy) / hy;
        double N[4], Nx[4], Ny[4];
        int32_t d[4];
        q1_basis(xi, eta, hx, hy, N, Nx, Ny);
        cell_nodes(i, j, nx, ny, d);
        double ex = 0, ey = 0, hxx = 0, hxy = 0, hyx = 0, hyy = 0;
        for (int c = 0; c < 4; ++c) {
            ex += Phi[d[c]] * Nx[c];
            ey += Phi[d[c]] * Ny[c];
            hxx += gx[d[c]] * Nx[c];
            hxy += gx[d[c]] * Ny[c];
            hyx += gy[d[c]] * Nx[c];
            hyy += gy[d[c]] * Ny[c];
        }
        Ex[a] = ex; Ey[a] = ey; Hxx[a] = hxx; Hxy[a] = hxy; Hyx[a] = hyx; Hyy[a] = hyy;
    }
}

/* W = (1/2) int |grad phi_h|^2 (2 x 2 Gauss per cell, exact). */
double or2d_field_energy(int32_t nx, int32_t ny, double Lx, double Ly, const double *Phi) {
    const double hx = Lx / nx, hy = Ly / ny;
    double W = 0.0;
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int32_t d[4];
            cell_nodes(i, j, nx, ny, d);
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    double N4[4], Nx[4], Ny[4];
                    q1_basis(GP[a], GP[c], hx, hy, N4, Nx, Ny);
                    double ex = 0.0, ey = 0.0;
                    for (int k = 0; k < 4; ++k) { ex += Phi[d[k]] * Nx[k]; ey += Phi[d[k]] * Ny[k]; }
                    W += 0.5 * 0.25 * hx * hy * (ex * ex + ey * ey);
                }
        }
    return W;
}

/* ------------------------------------------------------------------------ */
/* Run: KDK leapfrog (Sec. 5 split, Eq. swpic_dynamics)                       */
/*   kick  c: P -= c grad phi_h(Q);  q*_i += c sum_k H_ik(Q) p*_k              */
/*   drift c: Q += c P (wrapped);    p* -= c q*                                */
/* diag record (8 doubles): t, mass, mom_x, mom_y, kinetic, W, H, E_amp with  */
/*   mom = sum(psi* P + q*), kinetic = sum(psi* |P|^2/2 + q* . P),             */
/*   W = (1/2) int |grad phi_h|^2, E_amp = (2 W / (Lx Ly))^(1/2).              */
/* store_f32: the state is kept in FP32 storage (rounded after every update;  */
/* cells decided in FP32; the nodal table and step coefficients in FP32).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, decorated, store_f32;
    double Lx, Ly;
    or2d_solver *solver;
    int32_t *cx, *cy;
    double *b, *Phi, *gx, *gy, *Ex, *Ey, *Hxx, *Hxy, *Hyx, *Hyy;
    double W;
} or2d_field;

static double f32r(double x) { return (double)(float)x; }

static void field2_update(or2d_field *f, int64_t n, const double *Qx, const double *Qy,
                          const double *psx, const double *psy, const double *psi) {
    const int32_t N = f->nx * f->ny;
    if (f->store_f32)
        for (int64_t a = 0; a < n; ++a) {
            f->cx[a] = or2d_cell_f32(Qx[a], f->Lx, f->nx);
            f->cy[a] = or2d_cell_f32(Qy[a], f->Ly, f->ny);
        }
    or2d_deposit(n, Qx, Qy, f->decorated ? psx : NULL, psy, psi, f->store_f32 ? f->cx : NULL,
                 f->store_f32 ? f->cy : NULL, f->Lx, f->Ly, f->nx, f->ny, f->b);
    or2d_solver_apply(f->solver, f->b, f->Phi, NULL);
    f->W = or2d_field_energy(f->nx, f->ny, f->Lx, f->Ly, f->Phi);
    or2d_project(f->nx, f->ny, f->Lx, f->Ly, f->Phi, f->gx, f->gy);
    if (f->store_f32)
        for (int32_t k = 0; k < N; ++k) { f->Phi[k] = f32r(f->Phi[k]); f->gx[k] = f32r(f->gx[k]); f->gy[k] = f32r(f->gy[k]); }
}

static void kick2(or2d_field *f, int64_t n, const double *Qx, const double *Qy, double *Px, double *Py,
                  double *qx, double *qy, const double *px, const double *py, double c) {
    or2d_gather(n, Qx, Qy, f->store_f32 ? f->cx : NULL, f->store_f32 ? f->cy : NULL, f->Lx, f->Ly, f->nx,
                f->ny, f->Phi, f->gx, f->gy, f->Ex, f->Ey, f->Hxx, f->Hxy, f->Hyx, f->Hyy);
    for (int64_t a = 0; a < n; ++a) {
        Px[a] -= c * f->Ex[a];
        Py[a] -= c * f->Ey[a];
        if (f->decorated) {
            const double dqx = c * (f->Hxx[a] * px[a] + f->Hxy[a] * py[a]);
            const double dqy = c * (f->Hyx[a] * px[a] + f->Hyy[a] * py[a]);
            qx[a] += dqx;
            qy[a] += dqy;
        }
        if (f->store_f32) {
            Px[a] = f32r(Px[a]); Py[a] = f32r(Py[a]);
            if (f->decorated) { qx[a] = f32r(qx[a]); qy[a] = f32r(qy[a]); }
        }
    }
}

static void drift2(const or2d_field *f, int64_t n, double *Qx, double *Qy, const double *Px, const double *Py,
                   const double *qx, const double *qy, double *px, double *py, double c) {
    for (int64_t a = 0; a < n; ++a) {
        double x = wrap2(Qx[a] + c * Px[a], f->Lx);
        double y = wrap2(Qy[a] + c * Py[a], f->Ly);
        if (f->store_f32) {
            x = f32r(x); if (x >= f->Lx) x = f32r(x - f->Lx);
            y = f32r(y); if (y >= f->Ly) y = f32r(y - f->Ly);
        }
        Qx[a] = x; Qy[a] = y;
        if (f->decorated) {
            px[a] -= c * qx[a];
            py[a] -= c * qy[a];
            if (f->store_f32) { px[a] = f32r(px[a]); py[a] = f32r(py[a]); }
        }
    }
}

static void diag2(const or2d_field *f, double *rec, double t, int64_t n, const double *Px, const double *Py,
                  const double *qx, const double *qy, const double *psi) {
    double mass = 0, mx = 0, my = 0, kin = 0;
    for (int64_t a = 0; a < n; ++a) {
        mass += psi[a];
        mx += psi[a] * Px[a] + (f->decorated ? qx[a] : 0.0);
        my += psi[a] * Py[a] + (f->decorated ? qy[a] : 0.0);
        kin += 0.5 * psi[a] * (Px[a] * Px[a] + Py[a] * Py[a]);
        if (f->decorated) kin += qx[a] * Px[a] + qy[a] * Py[a];
    }
    rec[0] = t; rec[1] = mass; rec[2] = mx; rec[3] = my; rec[4] = kin;
    rec[5] = f->W; rec[6] = kin + f->W; rec[7] = sqrt(2.0 * f->W / (f->Lx * f->Ly));
}

int or2d_run(int64_t n, double *Qx, double *Qy, double *Px, double *Py, double *qx, double *qy,
             double *px, double *py, const double *psi, int32_t nx, int32_t ny, double Lx, double Ly,
             double dt, int32_t decorated, int32_t n_steps, int32_t diag_every, double *diag,
             int32_t *n_diag, double *Phi_out, int32_t store_f32) {
    or2d_field f;
    memset(&f, 0, sizeof(f));
    f.nx = nx; f.ny = ny; f.Lx = Lx; f.Ly = Ly; f.decorated = decorated; f.store_f32 = store_f32;
    const int32_t N = nx * ny;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    f.solver = or2d_solver_new(nx, ny, Lx, Ly);
    if (!f.solver) return -1;
    f.cx = (int32_t *)calloc(nn, sizeof(int32_t)); f.cy = (int32_t *)calloc(nn, sizeof(int32_t));
    f.b = (double *)calloc(N, sizeof(double)); f.Phi = (double *)calloc(N, sizeof(double));
    f.gx = (double *)calloc(N, sizeof(double)); f.gy = (double *)calloc(N, sizeof(double));
    double **pa[6] = {&f.Ex, &f.Ey, &f.Hxx, &f.Hxy, &f.Hyx, &f.Hyy};
    for (int k = 0; k < 6; ++k) *pa[k] = (double *)calloc(nn, sizeof(double));
    const double half = store_f32 ? f32r(0.5 * dt) : 0.5 * dt;
    const double full = store_f32 ? f32r(dt) : dt;
    field2_update(&f, n, Qx, Qy, px, py, psi);
    int32_t nd = 0;
    if (diag && diag_every > 0) diag2(&f, diag + 8 * (nd++), 0.0, n, Px, Py, qx, qy, psi);
    for (int32_t s = 1; s <= n_steps; ++s) {
        kick2(&f, n, Qx, Qy, Px, Py, qx, qy, px, py, half);
        drift2(&f, n, Qx, Qy, Px, Py, qx, qy, px, py, full);
        field2_update(&f, n, Qx, Qy, px, py, psi);
        kick2(&f, n, Qx, Qy, Px, Py, qx, qy, px, py, half);
        if (diag && diag_every > 0 && s % diag_every == 0)
            diag2(&f, diag + 8 * (nd++), (double)s * dt, n, Px, Py, qx, qy, psi);
    }
    if (n_diag) *n_diag = nd;
    if (Phi_out) memcpy(Phi_out, f.Phi, sizeof(double) * N);
    or2d_solver_free(f.solver);
    free(f.cx); free(f.cy); free(f.b); free(f.Phi); free(f.gx); free(f.gy);
    for (int k = 0; k < 6; ++k) free(*pa[k]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice initialisation in 2D2V: the reading of Sec. 4.2 / Alg. 1 used in   */
/* 1D, one dimension up.  Each cell of a 4D phase-space lattice is the        */
/* cluster S_a of the continuum f0; particle index ((k nvy + l) nqy + j) nqx  */
/* + i (positions fastest);  Q = cell centre in (x, y), P = cell centre in     */
/* (vx, vy);                                                                  */
/*   psi*  = f0(centre) dx dy dvx dvy                        (midpoint)        */
/*   p*_x  = int_cell f0 (Lx/2pi) sin(2pi (Qx - x)/Lx)   (periodic c, Sec. 4.2) */
/*   p*_y  = int_cell f0 (Ly/2pi) sin(2pi (Qy - y)/Ly)                         */
/*   q*    = - int_cell f0 (P - p)                          (Eq. moment-def)  */
/* by an n^4 Gauss-Legendre rule.                                             */
/* f0 = (1 + alpha cos(kx x + ky y)) exp(-(vx^2 + vy^2)/(2 vth^2)) / (2 pi vth^2) */
/* ------------------------------------------------------------------------ */
int or_gauss_legendre(int32_t npts, double *x, double *w);

static double f0_2d(double alpha, double kx, double ky, double vth, double x, double y, double vx, double vy) {
    const double pi = 3.14159265358979323846;
    return (1.0 + alpha * cos(kx * x + ky * y)) * exp(-(vx * vx + vy * vy) / (2.0 * vth * vth)) /
           (2.0 * pi * vth * vth);
}

int or2d_init_lattice(int32_t nqx, int32_t nqy, int32_t nvx, int32_t nvy, double Lx, double Ly,
                      double vmin, double vmax, double alpha, double kx, double ky, double vth,
                      int32_t quad_order, int32_t decorate, double *Qx, double *Qy, double *Px, double *Py,
                      double *qx, double *qy, double *px, double *py, double *psi) {
    if (nqx < 1 || nqy < 1 || nvx < 1 || nvy < 1 || quad_order < 1 || quad_order > 8) return -1;
    double g[64], gw[64];
    if (or_gauss_legendre(quad_order, g, gw) != 0) return -1;
    const double pi = 3.14159265358979323846;
    const double dx = Lx / nqx, dy = Ly / nqy, dvx = (vmax - vmin) / nvx, dvy = (vmax - vmin) / nvy;
    const int32_t n = quad_order;
    for (int32_t i = 0; i < nqx; ++i)
        for (int32_t j = 0; j < nqy; ++j)
            for (int32_t k = 0; k < nvx; ++k)
                for (int32_t l = 0; l < nvy; ++l) {
                    const int64_t a = (((int64_t)k * nvy + l) * nqy + j) * nqx + i;
                    const double xc = (i + 0.5) * dx, yc = (j + 0.5) * dy;
                    const double uc = vmin + (k + 0.5) * dvx, wc = vmin + (l + 0.5) * dvy;
                    Qx[a] = xc; Qy[a] = yc; Px[a] = uc; Py[a] = wc;
                    psi[a] = f0_2d(alpha, kx, ky, vth, xc, yc, uc, wc) * dx * dy * dvx * dvy;
                    double sx = 0.0, sy = 0.0, tx = 0.0, ty = 0.0;
                    if (decorate) {
                        for (int32_t r = 0; r < n; ++r)
                            for (int32_t s = 0; s < n; ++s)
                                for (int32_t t = 0; t < n; ++t)
                                    for (int32_t u = 0; u < n; ++u) {
                                        const double x = xc + 0.5 * dx * g[r], y = yc + 0.5 * dy * g[s];
                                        const double vx = uc + 0.5 * dvx * g[t], vy = wc + 0.5 * dvy * g[u];
                                        const double wgt = gw[r] * gw[s] * gw[t] * gw[u] * 0.0625 * dx * dy * dvx * dvy;
                                        const double fv = wgt * f0_2d(alpha, kx, ky, vth, x, y, vx, vy);
                                        sx += fv * (Lx / (2.0 * pi)) * sin(2.0 * pi * (xc - x) / Lx);
                                        sy += fv * (Ly / (2.0 * pi)) * sin(2.0 * pi * (yc - y) / Ly);
                                        tx += -fv * (uc - vx);
                                        ty += -fv * (wc - vy);
                                    }
                    }
                    px[a] = sx; py[a] = sy; qx[a] = tx; qy[a] = ty;
                }
    return 0;
}
