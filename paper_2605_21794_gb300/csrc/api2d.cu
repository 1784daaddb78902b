// C ABI of the 2D2V decorated-particle step (include/swpic2d.h): context,
// validation, the fixed-point unit, the fused-pass / spectral-solve sequence
// of a step, diagnostics and read-outs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "swpic2d_internal.cuh"

using namespace swpic2d;

namespace {
// The deposit bound of the state at refresh maps to 2^58 units (FP64) or
// 2^54 units (FP32); the accumulator's limit is 2^62.  The dipole weights p*
// grow in time (dp*/dt = -q*, the shear of nearby characteristics), so the
// bound grows too: FP32 runs keep 2^8 of headroom for it, at a quantum far
// below FP32 resolution; FP64 runs keep 2^4 and a quantum of 2^-58 of the bound.
constexpr int kFixedBits2dF64 = 58;
constexpr int kFixedBits2dF32 = 54;
}

struct swpic2d_ctx {
    swpic2d_config cfg{};
    int64_t n = 0;
    int prec = SWPIC_F32, nn = 0, tpb = 256, grid = 1, cap = 4096;
    bool dec = true, bound = false, ready = false, timing = false;
    size_t smem_dep = 0, smem_nodep = 0;
    void *st[9] = {};
    cudaStream_t stream = nullptr;
    // device buffers
    unsigned long long *acc = nullptr;
    double *b = nullptr, *phi = nullptr, *inv_lam = nullptr, *diag_acc = nullptr, *W = nullptr;
    double *rec = nullptr, *bsum = nullptr;
    double2 *spec = nullptr, *tw = nullptr;
    float2 *twf = nullptr;
    float *inv_lamf = nullptr;
    unsigned int *done = nullptr;
    long long *braw = nullptr;
    void *table = nullptr;
    int *err = nullptr;
    double fx_scale = 1.0, fx_inv = 1.0;
    int fx_k = 0;
    int64_t step = 0, last_rec = -1, n_rec = 0, launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    std::string msg;
};

namespace {

swpic_status fail(swpic2d_ctx *c, swpic_status s, const std::string &m) {
    if (c) c->msg = m;
    return s;
}

#define CK2(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(ctx, SWPIC_ECUDA, std::string(#call) + ": " +   \
                                           cudaGetErrorString(e_));                        \
    } while (0)

bool pow2(int v) { return v >= 4 && v <= SWPIC2D_N_MAX && (v & (v - 1)) == 0; }
int ilog2(int v) { int k = 0; while ((1 << k) < v) ++k; return k; }

void free_all(swpic2d_ctx *c) {
    void *ptrs[] = {c->acc, c->b, c->phi, c->inv_lam, c->diag_acc, c->W, c->rec, c->bsum, c->spec, c->tw,
                    c->table, c->err, c->twf, c->inv_lamf, c->done, c->braw};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &e : c->events) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    c->events.clear();
}

PassArgs2d pass_args(const swpic2d_ctx *c) {
    PassArgs2d a{};
    a.Qx = c->st[0]; a.Qy = c->st[1]; a.Px = c->st[2]; a.Py = c->st[3];
    a.qx = c->st[4]; a.qy = c->st[5]; a.px = c->st[6]; a.py = c->st[7]; a.psi = c->st[8];
    a.n = c->n;
    a.table = c->table;
    a.acc = c->acc;
    a.diag_acc = c->diag_acc;
    a.err = c->err;
    a.Lx = c->cfg.Lx; a.Ly = c->cfg.Ly;
    a.inv_hx = (double)c->cfg.nx / c->cfg.Lx;
    a.inv_hy = (double)c->cfg.ny / c->cfg.Ly;
    a.inv_Lx = 1.0 / c->cfg.Lx;
    a.inv_Ly = 1.0 / c->cfg.Ly;
    a.fx_scale = c->fx_scale;
    a.nx = c->cfg.nx; a.ny = c->cfg.ny;
    return a;
}

SolveArgs2d solve_args(const swpic2d_ctx *c) {
    SolveArgs2d s{};
    s.acc = c->acc; s.b = c->b; s.spec = c->spec; s.phi = c->phi; s.inv_lam = c->inv_lam; s.tw = c->tw;
    s.W = c->W; s.table = c->table; s.err = c->err;
    s.fx_inv = c->fx_inv;
    s.inv_hx = (double)c->cfg.nx / c->cfg.Lx;
    s.inv_hy = (double)c->cfg.ny / c->cfg.Ly;
    s.inv_nn = 1.0 / (double)c->nn;
    s.nx = c->cfg.nx; s.ny = c->cfg.ny;
    s.lognx = ilog2(c->cfg.nx); s.logny = ilog2(c->cfg.ny);
    s.ntw = std::max(c->cfg.nx, c->cfg.ny);
    s.twf = c->twf;
    s.inv_lamf = c->inv_lamf;
    s.fx_k = c->fx_k;
    s.braw = c->braw;
    return s;
}

RecordArgs2d record_args(swpic2d_ctx *c, int64_t s) {
    RecordArgs2d r{};
    r.diag_acc = c->diag_acc;
    r.W = c->W;
    r.rec = (c->n_rec < c->cap) ? c->rec + 9 * c->n_rec : nullptr;   // full: later records dropped
    r.err = c->err;
    r.t = (double)s * c->cfg.dt;
    r.area = c->cfg.Lx * c->cfg.Ly;
    r.step = s;
    if (c->n_rec < c->cap) ++c->n_rec;
    return r;
}

swpic_status check_flag(swpic2d_ctx *ctx) {
    int f = 0;
    CK2(cudaMemcpy(&f, ctx->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        CK2(cudaMemset(ctx->err, 0, sizeof(int)));
        return fail(ctx, SWPIC_ENUMERIC, (f & kErrOverflow) ? "charge accumulator overflow (refresh the unit)"
                                                            : "non-finite charge or field");
    }
    return SWPIC_OK;
}

// one fused pass: kick c1, diagnostics, kick c2, drift cd, deposit.  FP32:
// the pass's last CTA also writes the record at integer step rec_step (diag)
// and solves the new field (dep); FP64: separate record and solve kernels.
swpic_status pass(swpic2d_ctx *ctx, double c1, double c2, double cd, bool dep, bool diag, int64_t rec_step) {
    PassArgs2d a = pass_args(ctx);
    a.k1 = c1 * ctx->cfg.dt;
    a.k2 = c2 * ctx->cfg.dt;
    a.kd = cd * ctx->cfg.dt;
    const bool tail = ctx->prec == SWPIC_F32;
    if (tail) {
        a.tail = (diag ? 1 : 0) | (dep ? 2 : 0);
        a.done = ctx->done;
        if (diag) a.rec = record_args(ctx, rec_step);
        a.solve = solve_args(ctx);
    }
    const size_t smem = dep ? ctx->smem_dep : ctx->smem_nodep;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->timing) {
        CK2(cudaEventCreate(&e0));
        CK2(cudaEventCreate(&e1));
        CK2(cudaEventRecord(e0, ctx->stream));
    }
    CK2(launch_pass(ctx->prec, ctx->dec, dep, diag, a, ctx->grid, ctx->tpb, smem, ctx->stream));
    ++ctx->launches;
    if (ctx->timing) {
        CK2(cudaEventRecord(e1, ctx->stream));
        ctx->events.emplace_back(e0, e1);
    }
    if (!tail) {
        if (diag) {
            CK2(launch_record(record_args(ctx, rec_step), ctx->stream));
            ++ctx->launches;
        }
        if (dep) CK2(launch_solve(ctx->prec, solve_args(ctx), ctx->stream, &ctx->launches));
    }
    return SWPIC_OK;
}

}  // namespace

extern "C" {

swpic_status swpic2d_create(const swpic2d_config *cfg, int64_t n_particles, swpic2d_ctx **out) {
    if (!out) return SWPIC_EINVAL;
    *out = nullptr;
    if (!cfg || n_particles < 0) return SWPIC_EINVAL;
    const swpic2d_config &c = *cfg;
    if (!(c.Lx > 0.0) || !(c.Ly > 0.0) || !(c.dt > 0.0) || !std::isfinite(c.Lx) || !std::isfinite(c.Ly) ||
        !std::isfinite(c.dt))
        return SWPIC_EINVAL;
    if (!pow2(c.nx) || !pow2(c.ny)) return SWPIC_EINVAL;
    if (c.precision != SWPIC_F32 && c.precision != SWPIC_F64) return SWPIC_EINVAL;
    const int nn = c.nx * c.ny;
    if (nn > (c.precision == SWPIC_F64 ? SWPIC2D_NODES_MAX_F64 : SWPIC2D_NODES_MAX_F32)) return SWPIC_EINVAL;
    if (c.threads_per_block != 0 && (c.threads_per_block < 64 || c.threads_per_block > 256 ||
                                     c.threads_per_block % 32))
        return SWPIC_EINVAL;
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 32 || c.diag_capacity < 0) return SWPIC_EINVAL;

    swpic2d_ctx *ctx = new swpic2d_ctx();
    ctx->cfg = c;
    ctx->n = n_particles;
    ctx->prec = c.precision;
    ctx->dec = c.decorated != 0;
    ctx->nn = nn;
    ctx->tpb = c.threads_per_block ? c.threads_per_block : 256;
    ctx->cap = c.diag_capacity ? c.diag_capacity : 4096;
    ctx->smem_dep = pass_smem_bytes(ctx->prec, c.nx, c.ny, true);
    ctx->smem_nodep = pass_smem_bytes(ctx->prec, c.nx, c.ny, false);
    const size_t es = (ctx->prec == SWPIC_F64) ? 8 : 4;
    const int ntw = std::max(c.nx, c.ny);
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) { ok = ok && cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
    alloc((void **)&ctx->acc, sizeof(unsigned long long) * nn);
    alloc((void **)&ctx->b, sizeof(double) * nn);
    alloc((void **)&ctx->phi, sizeof(double) * nn);
    alloc((void **)&ctx->inv_lam, sizeof(double) * nn);
    alloc((void **)&ctx->spec, sizeof(double2) * nn);
    alloc((void **)&ctx->tw, sizeof(double2) * (ntw / 2));
    alloc((void **)&ctx->table, 4 * es * nn);
    alloc((void **)&ctx->diag_acc, sizeof(double) * 4);
    alloc((void **)&ctx->W, sizeof(double));
    alloc((void **)&ctx->bsum, sizeof(double));
    alloc((void **)&ctx->rec, sizeof(double) * 9 * ctx->cap);
    alloc((void **)&ctx->err, sizeof(int));
    alloc((void **)&ctx->twf, sizeof(float2) * (ntw / 2));
    alloc((void **)&ctx->inv_lamf, sizeof(float) * nn);
    alloc((void **)&ctx->done, sizeof(unsigned int));
    alloc((void **)&ctx->braw, sizeof(long long) * nn);
    if (!ok) {
        free_all(ctx);
        delete ctx;
        return SWPIC_ENOMEM;
    }
    // twiddles exp(-2 pi i k / ntw) and the inverse symbol of the Q1 stiffness
    std::vector<double2> tw(ntw / 2);
    for (int k = 0; k < ntw / 2; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)ntw;
        tw[k] = make_double2(std::cos(a), std::sin(a));
    }
    const double hx = c.Lx / c.nx, hy = c.Ly / c.ny;
    std::vector<double> il(nn);
    for (int ky = 0; ky < c.ny; ++ky)
        for (int kx = 0; kx < c.nx; ++kx) {
            const double cx = std::cos(2.0 * M_PI * kx / c.nx), cy = std::cos(2.0 * M_PI * ky / c.ny);
            const double lam = (2.0 - 2.0 * cx) * (4.0 + 2.0 * cy) * hy / (6.0 * hx) +
                               (2.0 - 2.0 * cy) * (4.0 + 2.0 * cx) * hx / (6.0 * hy);
            il[ky * c.nx + kx] = (kx == 0 && ky == 0) ? 0.0 : 1.0 / lam;
        }
    std::vector<float2> twf(tw.size());
    for (size_t k = 0; k < tw.size(); ++k) twf[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    std::vector<float> ilf(nn);
    for (int k = 0; k < nn; ++k) ilf[k] = (float)il[k];
    bool okc = cudaMemcpy(ctx->tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(ctx->twf, twf.data(), sizeof(float2) * twf.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(ctx->inv_lamf, ilf.data(), sizeof(float) * nn, cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(ctx->done, 0, sizeof(unsigned int)) == cudaSuccess &&
               cudaMemset(ctx->braw, 0, sizeof(long long) * nn) == cudaSuccess &&
               cudaMemcpy(ctx->inv_lam, il.data(), sizeof(double) * nn, cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(ctx->acc, 0, sizeof(unsigned long long) * nn) == cudaSuccess &&
               cudaMemset(ctx->table, 0, 4 * es * nn) == cudaSuccess &&
               cudaMemset(ctx->b, 0, sizeof(double) * nn) == cudaSuccess &&
               cudaMemset(ctx->phi, 0, sizeof(double) * nn) == cudaSuccess &&
               cudaMemset(ctx->diag_acc, 0, sizeof(double) * 4) == cudaSuccess &&
               cudaMemset(ctx->W, 0, sizeof(double)) == cudaSuccess &&
               cudaMemset(ctx->err, 0, sizeof(int)) == cudaSuccess;
    // launch shape: CTAs per SM from the occupancy of the depositing pass
    int dev = 0, sms = 1, occ = 1;
    okc = okc && cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    const void *fn = pass_kernel(ctx->prec, ctx->dec, true, true);
    okc = okc && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_dep) ==
                     cudaSuccess &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, ctx->tpb, ctx->smem_dep) == cudaSuccess;
    if (!okc || occ < 1) {
        free_all(ctx);
        delete ctx;
        return okc ? SWPIC_EINVAL : SWPIC_ECUDA;
    }
    const int bpsm = c.blocks_per_sm ? std::min(c.blocks_per_sm, occ) : std::min(occ, 8);
    const int64_t need = (n_particles + ctx->tpb - 1) / ctx->tpb;
    ctx->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * bpsm, need));
    *out = ctx;
    return SWPIC_OK;
}

void swpic2d_destroy(swpic2d_ctx *ctx) {
    if (!ctx) return;
    if (ctx->bound) cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

const char *swpic2d_last_error(const swpic2d_ctx *ctx) { return ctx ? ctx->msg.c_str() : "no context"; }

swpic_status swpic2d_bind_state(swpic2d_ctx *ctx, void *const state[9], swpic_stream stream) {
    if (!ctx || !state) return SWPIC_EINVAL;
    for (int k = 0; k < 9; ++k) {
        const bool optional = (k >= 4 && k <= 7) && !ctx->dec;
        if (!state[k] && !optional && ctx->n > 0) return fail(ctx, SWPIC_EINVAL, "missing state array");
        const size_t al = (ctx->prec == SWPIC_F64) ? 8 : 4;
        if (state[k] && (reinterpret_cast<uintptr_t>(state[k]) % al))
            return fail(ctx, SWPIC_EINVAL, "misaligned state array");
    }
    for (int k = 0; k < 9; ++k) ctx->st[k] = state[k];
    if (!ctx->dec)
        for (int k = 4; k < 8; ++k) ctx->st[k] = nullptr;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    ctx->bound = true;
    ctx->ready = false;
    return SWPIC_OK;
}

swpic_status swpic2d_refresh(swpic2d_ctx *ctx) {
    if (!ctx) return SWPIC_EINVAL;
    if (!ctx->bound) return fail(ctx, SWPIC_ESTATE, "no state bound");
    double m = 0.0;
    if (ctx->n > 0) {
        CK2(cudaMemsetAsync(ctx->bsum, 0, sizeof(double), ctx->stream));
        CK2(launch_bound(ctx->prec, pass_args(ctx), ctx->bsum, std::min(ctx->grid, 1024), ctx->stream));
        ++ctx->launches;
        CK2(cudaMemcpyAsync(&m, ctx->bsum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK2(cudaStreamSynchronize(ctx->stream));
    }
    if (!std::isfinite(m)) return fail(ctx, SWPIC_ENUMERIC, "non-finite particle weights");
    const int bits = (ctx->prec == SWPIC_F64) ? kFixedBits2dF64 : kFixedBits2dF32;
    int k = bits;
    if (m > 0.0) k = bits - (int)std::ceil(std::log2(m));
    k = std::max(-1000, std::min(1000, k));
    ctx->fx_scale = std::ldexp(1.0, k);
    ctx->fx_inv = std::ldexp(1.0, -k);
    ctx->fx_k = k;
    CK2(cudaMemsetAsync(ctx->acc, 0, sizeof(unsigned long long) * ctx->nn, ctx->stream));
    CK2(cudaMemsetAsync(ctx->diag_acc, 0, sizeof(double) * 4, ctx->stream));
    swpic_status s = pass(ctx, 0.0, 0.0, 0.0, true, false, 0);      // deposit, then the field
    if (s != SWPIC_OK) return s;
    CK2(cudaStreamSynchronize(ctx->stream));
    s = check_flag(ctx);
    if (s != SWPIC_OK) return s;
    ctx->ready = true;
    return SWPIC_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term
// recurrence of P_n), n <= 8: out[0..n) nodes, out[8..8+n) weights.
static void gauss_legendre(int n, double *out) {
    for (int k = 0; k < n; ++k) {
        double z = std::cos(M_PI * (k + 0.75) / (n + 0.5)), pn = 0.0, pm = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            pn = z; pm = 1.0;
            for (int m = 2; m <= n; ++m) { const double q = ((2.0 * m - 1.0) * z * pn - (m - 1.0) * pm) / m; pm = pn; pn = q; }
            if (n == 1) { pn = z; pm = 1.0; }
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        pn = z; pm = 1.0;
        for (int m = 2; m <= n; ++m) { const double q = ((2.0 * m - 1.0) * z * pn - (m - 1.0) * pm) / m; pm = pn; pn = q; }
        dp = n * (z * pn - pm) / (z * z - 1.0);
        out[k] = -z;
        out[8 + k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

swpic_status swpic2d_init_lattice(swpic2d_ctx *ctx, const swpic2d_lattice *spec) {
    if (!ctx || !spec) return SWPIC_EINVAL;
    if (!ctx->bound) return fail(ctx, SWPIC_ESTATE, "no state bound");
    const swpic2d_lattice &f = *spec;
    if (f.nqx < 1 || f.nqy < 1 || f.nvx < 1 || f.nvy < 1 || f.quad_order < 1 || f.quad_order > 4 ||
        !(f.vmax > f.vmin) || !(f.vth > 0.0) || !std::isfinite(f.alpha) || !std::isfinite(f.kx) ||
        !std::isfinite(f.ky))
        return fail(ctx, SWPIC_EINVAL, "bad lattice");
    if ((int64_t)f.nqx * f.nqy * f.nvx * f.nvy != ctx->n)
        return fail(ctx, SWPIC_EINVAL, "nqx nqy nvx nvy must equal the particle count");
    double gl[16] = {};
    gauss_legendre(f.quad_order, gl);
    double *dgl = nullptr;
    CK2(cudaMalloc(&dgl, sizeof(gl)));
    cudaError_t e = cudaMemcpyAsync(dgl, gl, sizeof(gl), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        swpic2d_lattice g = f;
        if (!ctx->dec) g.decorate = 0;
        e = launch_init_lattice(ctx->prec, g, ctx->cfg.Lx, ctx->cfg.Ly, dgl, ctx->st, ctx->stream);
        ++ctx->launches;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dgl);
    CK2(e);
    return swpic2d_refresh(ctx);
}

swpic_status swpic2d_step(swpic2d_ctx *ctx, int32_t n_steps, int32_t diag_every) {
    if (!ctx || n_steps < 0 || diag_every < 0) return SWPIC_EINVAL;
    if (!ctx->ready) return fail(ctx, SWPIC_ESTATE, "call swpic2d_refresh after binding or writing the state");
    if (n_steps == 0) return SWPIC_OK;
    for (int32_t p = 0; p <= n_steps; ++p) {
        const bool first = (p == 0), last = (p == n_steps);
        const int64_t s = ctx->step + p;           // integer time seen after the closing kick
        const bool diag = diag_every > 0 && s % diag_every == 0 && s != ctx->last_rec;
        swpic_status st = pass(ctx, first ? 0.0 : 0.5, last ? 0.0 : 0.5, last ? 0.0 : 1.0, !last, diag, s);
        if (st != SWPIC_OK) return st;
        if (diag) ctx->last_rec = s;
    }
    ctx->step += n_steps;
    return SWPIC_OK;
}

swpic_status swpic2d_diagnostics(swpic2d_ctx *ctx, swpic2d_diag *out, int32_t max_records, int32_t *n_records) {
    if (!ctx || max_records < 0 || (!out && max_records > 0)) return SWPIC_EINVAL;
    CK2(cudaStreamSynchronize(ctx->stream));
    swpic_status s = check_flag(ctx);
    if (s != SWPIC_OK) return s;
    const int n = (int)std::min<int64_t>(ctx->n_rec, max_records);
    std::vector<double> h((size_t)9 * std::max(n, 1));
    if (n > 0) CK2(cudaMemcpy(h.data(), ctx->rec, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost));
    for (int r = 0; r < n; ++r) {
        const double *v = &h[9 * r];
        out[r] = swpic2d_diag{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], (int64_t)v[8]};
    }
    if (n_records) *n_records = n;
    return SWPIC_OK;
}

swpic_status swpic2d_get_field(swpic2d_ctx *ctx, double *b, double *Phi, double *gx, double *gy) {
    if (!ctx) return SWPIC_EINVAL;
    CK2(cudaStreamSynchronize(ctx->stream));
    const int nn = ctx->nn;
    const bool f32 = ctx->prec == SWPIC_F32;       // FP32: integer loads and the FP32 Phi of the table
    if (b && f32) {
        std::vector<long long> raw(nn);
        CK2(cudaMemcpy(raw.data(), ctx->braw, sizeof(long long) * nn, cudaMemcpyDeviceToHost));
        for (int k = 0; k < nn; ++k) b[k] = (double)raw[k] * ctx->fx_inv;
    } else if (b) {
        CK2(cudaMemcpy(b, ctx->b, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    }
    if (Phi && !f32) CK2(cudaMemcpy(Phi, ctx->phi, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    if (gx || gy || (Phi && f32)) {
        const size_t es = (ctx->prec == SWPIC_F64) ? 8 : 4;
        std::vector<unsigned char> t(4 * es * nn);
        CK2(cudaMemcpy(t.data(), ctx->table, t.size(), cudaMemcpyDeviceToHost));
        for (int k = 0; k < nn; ++k) {
            double vp, vx, vy;
            if (es == 8) {
                vp = reinterpret_cast<const double *>(t.data())[4 * k];
                vx = reinterpret_cast<const double *>(t.data())[4 * k + 1];
                vy = reinterpret_cast<const double *>(t.data())[4 * k + 2];
            } else {
                vp = reinterpret_cast<const float *>(t.data())[4 * k];
                vx = reinterpret_cast<const float *>(t.data())[4 * k + 1];
                vy = reinterpret_cast<const float *>(t.data())[4 * k + 2];
            }
            if (Phi && f32) Phi[k] = vp;
            if (gx) gx[k] = vx;
            if (gy) gy[k] = vy;
        }
    }
    return check_flag(ctx);
}

swpic_status swpic2d_step_host(swpic2d_ctx *ctx, const void *const in[9], void *const out[8],
                               int32_t n_steps, int32_t diag_every) {
    if (!ctx || !in || n_steps < 0 || diag_every < 0) return SWPIC_EINVAL;
    if (!ctx->bound) return fail(ctx, SWPIC_ESTATE, "no state bound");
    const size_t bytes = (size_t)ctx->n * (ctx->prec == SWPIC_F64 ? 8 : 4);
    for (int k = 0; k < 9; ++k) {
        if (!ctx->st[k] || bytes == 0) continue;
        if (in[k]) CK2(cudaMemcpyAsync(ctx->st[k], in[k], bytes, cudaMemcpyHostToDevice, ctx->stream));
        else if (k >= 4 && k <= 7) CK2(cudaMemsetAsync(ctx->st[k], 0, bytes, ctx->stream));
        else return fail(ctx, SWPIC_EINVAL, "missing host array");
    }
    swpic_status s = swpic2d_refresh(ctx);
    if (s != SWPIC_OK) return s;
    s = swpic2d_step(ctx, n_steps, diag_every);
    if (s != SWPIC_OK) return s;
    if (out)
        for (int k = 0; k < 8; ++k)
            if (out[k] && ctx->st[k] && bytes)
                CK2(cudaMemcpyAsync(out[k], ctx->st[k], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return swpic2d_synchronize(ctx);
}

// ---- checkpoint ----------------------------------------------------------
static const char kMagic2d[8] = {'S', 'W', 'P', '2', 'D', 'v', '1', 0};

struct Header2d {
    int32_t prec, dec, nx, ny;
    int64_t n, step, last_rec;
    double Lx, Ly, dt;
};

swpic_status swpic2d_save(swpic2d_ctx *ctx, const char *path) {
    if (!ctx || !path) return SWPIC_EINVAL;
    if (!ctx->bound) return fail(ctx, SWPIC_ESTATE, "no state bound");
    CK2(cudaStreamSynchronize(ctx->stream));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, SWPIC_EIO, std::string("cannot open ") + path);
    const Header2d h{ctx->prec, ctx->dec ? 1 : 0, ctx->cfg.nx, ctx->cfg.ny, ctx->n, ctx->step, ctx->last_rec,
                     ctx->cfg.Lx, ctx->cfg.Ly, ctx->cfg.dt};
    bool ok = std::fwrite(kMagic2d, 1, 8, f) == 8 && std::fwrite(&h, sizeof(h), 1, f) == 1;
    const size_t bytes = (size_t)ctx->n * (ctx->prec == SWPIC_F64 ? 8 : 4);
    std::vector<unsigned char> buf(bytes);
    for (int k = 0; k < 9 && ok; ++k) {
        if (!ctx->st[k] || bytes == 0) continue;
        const cudaError_t e = cudaMemcpy(buf.data(), ctx->st[k], bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, SWPIC_ECUDA, std::string("save: ") + cudaGetErrorString(e));
        }
        ok = std::fwrite(buf.data(), 1, bytes, f) == bytes;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SWPIC_OK : fail(ctx, SWPIC_EIO, std::string("cannot write ") + path);
}

swpic_status swpic2d_load(swpic2d_ctx *ctx, const char *path) {
    if (!ctx || !path) return SWPIC_EINVAL;
    if (!ctx->bound) return fail(ctx, SWPIC_ESTATE, "no state bound");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, SWPIC_EIO, std::string("cannot open ") + path);
    char magic[8];
    Header2d h{};
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic2d, 8) != 0 ||
        std::fread(&h, sizeof(h), 1, f) != 1) {
        std::fclose(f);
        return fail(ctx, SWPIC_EIO, std::string("not a 2D checkpoint: ") + path);
    }
    if (h.prec != ctx->prec || h.dec != (ctx->dec ? 1 : 0) || h.nx != ctx->cfg.nx || h.ny != ctx->cfg.ny ||
        h.n != ctx->n || h.Lx != ctx->cfg.Lx || h.Ly != ctx->cfg.Ly || h.dt != ctx->cfg.dt) {
        std::fclose(f);
        return fail(ctx, SWPIC_EINVAL, "checkpoint does not match this context");
    }
    CK2(cudaStreamSynchronize(ctx->stream));
    const size_t bytes = (size_t)ctx->n * (ctx->prec == SWPIC_F64 ? 8 : 4);
    std::vector<unsigned char> buf(bytes);
    for (int k = 0; k < 9; ++k) {
        if (!ctx->st[k] || bytes == 0) continue;
        if (std::fread(buf.data(), 1, bytes, f) != bytes) {
            std::fclose(f);
            return fail(ctx, SWPIC_EIO, std::string("truncated checkpoint: ") + path);
        }
        const cudaError_t e = cudaMemcpy(ctx->st[k], buf.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, SWPIC_ECUDA, std::string("load: ") + cudaGetErrorString(e));
        }
    }
    std::fclose(f);
    ctx->step = h.step;
    ctx->last_rec = h.last_rec;
    ctx->n_rec = 0;               // the records start at the checkpoint, as in the 1D load
    return swpic2d_refresh(ctx);
}

swpic_status swpic2d_synchronize(swpic2d_ctx *ctx) {
    if (!ctx) return SWPIC_EINVAL;
    CK2(cudaStreamSynchronize(ctx->stream));
    return check_flag(ctx);
}

swpic_status swpic2d_set_timing(swpic2d_ctx *ctx, int32_t enable) {
    if (!ctx) return SWPIC_EINVAL;
    ctx->timing = enable != 0;
    return SWPIC_OK;
}

swpic_status swpic2d_pass_times(swpic2d_ctx *ctx, float *ms, int32_t max_passes, int32_t *n_passes) {
    if (!ctx || max_passes < 0 || (!ms && max_passes > 0)) return SWPIC_EINVAL;
    CK2(cudaStreamSynchronize(ctx->stream));
    int n = 0;
    for (auto &e : ctx->events) {
        float t = 0.f;
        CK2(cudaEventElapsedTime(&t, e.first, e.second));
        if (n < max_passes) ms[n++] = t;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    ctx->events.clear();
    if (n_passes) *n_passes = n;
    return SWPIC_OK;
}

swpic_status swpic2d_launch_count(const swpic2d_ctx *ctx, int64_t *count) {
    if (!ctx || !count) return SWPIC_EINVAL;
    *count = ctx->launches;
    return SWPIC_OK;
}

}  // extern "C"
