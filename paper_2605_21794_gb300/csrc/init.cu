// Initialisation kernels (sm_103a): lattice decorated particles, FP64 -> state
// conversion, and the per-run mass sums that fix the fixed-point scale.
//
// Lattice reading of Sec. 4.2 / Alg. 1 (each lattice cell is the cluster):
//   psi* = f0(x_i, v_j) dx dv
//   p*   = int_cell f0(q, p) c(Q, q) dq dp,  c(Q, q) = (L/2pi) sin(2pi (Q - q)/L)
//   q*   = -int_cell f0(q, p) (P - p) dq dp
// f0(x, v) = X(x) V(v) with X = 1 + alpha cos(kx x) and V a sum of Gaussians
// times (c0 + c2 v^2), so the n x n Gauss-Legendre rule factorises:
//   p* = [sum_r w_r X(q_ir) c(Q, q_ir) dx/2] [sum_s w_s V(p_js) dv/2]
//   q* = -[sum_r w_r X(q_ir) dx/2] [sum_s w_s V(p_js) (P - p_js) dv/2]
// X(q_ir) depends only on the column i and V(p_js) only on the row j: they are
// tabulated once (k_lattice_tables).  The small angles 2pi(Q - q_ir)/L are
// formed from the offsets (jitter and node) so nothing cancels:
//   sin(a - b_r) = sin a cos b_r - cos a sin b_r,  a = 2pi jx dx/L,
//   b_r = pi g_r dx/L  (g_r the Gauss-Legendre node on [-1, 1]).
#include <math.h>

#include "swpic_internal.cuh"

namespace swpic {

__device__ double f0_X(const LatticeDev &t, double x) { return 1.0 + t.alpha * cos(t.kx * x); }
__device__ double f0_V(const LatticeDev &t, double v) {
    double s = 0.0;
    for (int m = 0; m < t.n_terms; ++m) {
        const double d = v - t.u[m];
        s += t.amp[m] * (t.c0[m] + t.c2[m] * v * v) * exp(-t.beta[m] * d * d);
    }
    return s;
}

// columns: Xc[i] = X(x_i), Xq[i*n + r] = X(q_ir); rows: Vc[j] = V(v_j), Vq[j*n + s] = V(p_js)
__global__ void k_lattice_tables(LatticeDev t, double L, double *Xc, double *Xq, double *Vc,
                                 double *Vq) {
    const int n = t.quad_order;
    const double dx = L / t.nq, dv = (t.vmax - t.vmin) / t.nv;
    const int total = t.nq + t.nv;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        if (k < t.nq) {
            const double xc = (k + 0.5) * dx;
            Xc[k] = f0_X(t, xc);
            for (int r = 0; r < n; ++r) Xq[(size_t)k * n + r] = f0_X(t, xc + 0.5 * dx * t.gx[r]);
        } else {
            const int j = k - t.nq;
            const double vc = t.vmin + (j + 0.5) * dv;
            Vc[j] = f0_V(t, vc);
            for (int s = 0; s < n; ++s) Vq[(size_t)j * n + s] = f0_V(t, vc + 0.5 * dv * t.gx[s]);
        }
    }
}

template <typename T>
__global__ void k_init_lattice(T *Q, T *P, T *qs, T *ps, T *psi, int64_t p0, double L, LatticeDev t,
                               const double *jx, const double *jv, const double *Xc,
                               const double *Xq, const double *Vc, const double *Vq, double sb[5],
                               double cb[5]) {
    const int n = t.quad_order;
    const int64_t total = (int64_t)t.nq * t.nv;
    const double dx = L / t.nq, dv = (t.vmax - t.vmin) / t.nv;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(a / t.nv), j = (int)(a % t.nv);
        const double xc = (i + 0.5) * dx, vc = t.vmin + (j + 0.5) * dv;
        const double ox = jx ? jx[a] : 0.0, ov = jv ? jv[a] : 0.0;
        double Qa = xc + ox * dx;
        Qa = Qa - L * floor(Qa / L);
        if (Qa >= L) Qa -= L;
        if (Qa < 0.0) Qa += L;
        const double Pa = vc + ov * dv;
        const double w = Xc[i] * Vc[j] * dx * dv;
        T Qt = (T)Qa;
        if ((double)Qt >= L) Qt = (T)((double)Qt - L);   // rounded onto/over L: wrap exactly
        const int64_t o = p0 + a;
        Q[o] = Qt;
        P[o] = (T)Pa;
        psi[o] = (T)w;
        if (qs == nullptr) continue;
        if (!t.decorate) { qs[o] = T(0); ps[o] = T(0); continue; }
        double sa = 0.0, ca = 1.0;
        if (ox != 0.0) sincos(two_pi * ox * dx / L, &sa, &ca);
        double px = 0.0, xint = 0.0, vint = 0.0, vmom = 0.0;
        for (int r = 0; r < n; ++r) {
            const double xr = t.gw[r] * Xq[(size_t)i * n + r];
            xint += xr;
            px += xr * (sa * cb[r] - ca * sb[r]);        // sin(2pi (Q - q_ir)/L)
        }
        for (int s = 0; s < n; ++s) {
            const double vs = t.gw[s] * Vq[(size_t)j * n + s];
            vint += vs;
            vmom += vs * (ov - 0.5 * t.gx[s]);            // (P - p_js)/dv
        }
        const double hx = 0.5 * dx, hv = 0.5 * dv;
        ps[o] = (T)((L / two_pi) * px * hx * vint * hv);
        qs[o] = (T)(-(xint * hx) * (vmom * dv * hv));
    }
}

template <typename T>
__global__ void k_convert(const double *src, T *dst, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = (T)src[k];
}

// per chunk: psi* summed as an unevaluated FP32 pair (hi + lo, Knuth's two-sum,
// error-free per addition) in FP32 state, in FP64 in FP64 state; |psi*| and |p*|
// (only a bound for the fixed-point scale) as plain sums.  Partial sums are
// combined in a fixed order, so the result depends only on the run's own data.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

template <typename T>
struct MassAcc {
    double s = 0.0, sa = 0.0, sp = 0.0;
    __device__ __forceinline__ void add(T x, T p) {
        s += x;
        sa += fabs(x);
        sp += fabs(p);
    }
    __device__ __forceinline__ void get(double &a, double &b, double &c) const { a = s; b = sa; c = sp; }
};

template <>
struct MassAcc<float> {
    float hi = 0.f, lo = 0.f, sa = 0.f, sp = 0.f;
    __device__ __forceinline__ void add(float x, float p) {
        two_sum_acc(hi, lo, x);
        sa += fabsf(x);
        sp += fabsf(p);
    }
    __device__ __forceinline__ void get(double &a, double &b, double &c) const {
        a = (double)hi + (double)lo;
        b = (double)sa;
        c = (double)sp;
    }
};

__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double (*sh)[32]) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = 0.0;
        for (int k = 0; k < nw; ++k) { a += sh[0][k]; b += sh[1][k]; c += sh[2][k]; }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mass_partial(const T *psi, const T *ps,
                                                      const SortChunk *chunks, double *partials) {
    __shared__ double sh[3][32];
    const SortChunk c = chunks[blockIdx.x];
    MassAcc<T> acc;
    for (int64_t k = c.start + threadIdx.x; k < c.end; k += blockDim.x)
        acc.add(psi[k], ps ? ps[k] : T(0));
    double a, b, d;
    acc.get(a, b, d);
    block_sum3(a, b, d, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = d;
    }
}

// one block per run: mass[r] = sum psi*; bound[r] = (sum |psi*|, sum |p*|)
__global__ void __launch_bounds__(256) k_mass_final(const double *partials, const SortChunk *chunks,
                                                    int n_chunks, double *mass, double *bound) {
    __shared__ double sh[3][32];
    __shared__ int s_lo;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) {
        // chunks are ordered by run: binary search the first chunk of run r
        int lo = 0, hi = n_chunks;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (chunks[mid].run < r) lo = mid + 1; else hi = mid;
        }
        s_lo = lo;
    }
    __syncthreads();
    const int lo = s_lo;
    double a = 0.0, b = 0.0, d = 0.0;
    for (int c = lo + threadIdx.x; c < n_chunks && chunks[c].run == r; c += blockDim.x) {
        a += partials[3 * c];
        b += partials[3 * c + 1];
        d += partials[3 * c + 2];
    }
    block_sum3(a, b, d, sh);
    if (threadIdx.x == 0) {
        mass[r] = a;
        bound[2 * r] = b;
        bound[2 * r + 1] = d;
    }
}

cudaError_t launch_init_lattice(int prec, bool decorated, void *Q, void *P, void *qs, void *ps,
                                void *psi, int64_t p0, double L, const LatticeDev &lat,
                                const double *jx, const double *jv, cudaStream_t s) {
    const int n = lat.quad_order;
    double *tabs = nullptr;
    const size_t nd = (size_t)lat.nq * (n + 1) + (size_t)lat.nv * (n + 1) + 10;
    cudaError_t e = cudaMallocAsync((void **)&tabs, nd * sizeof(double), s);
    if (e != cudaSuccess) return e;
    double *Xc = tabs, *Xq = Xc + lat.nq, *Vc = Xq + (size_t)lat.nq * n, *Vq = Vc + lat.nv;
    double *sbcb = Vq + (size_t)lat.nv * n;
    double h_sbcb[10];
    const double pi = 3.14159265358979323846;
    const double dx = L / lat.nq;
    for (int r = 0; r < 5; ++r) {
        const double b = (r < n) ? pi * lat.gx[r] * dx / L : 0.0;
        h_sbcb[r] = sin(b);
        h_sbcb[5 + r] = cos(b);
    }
    e = cudaMemcpyAsync(sbcb, h_sbcb, sizeof(h_sbcb), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFreeAsync(tabs, s); return e; }
    const int tg = (lat.nq + lat.nv + 255) / 256;
    k_lattice_tables<<<tg, 256, 0, s>>>(lat, L, Xc, Xq, Vc, Vq);
    const int64_t total = (int64_t)lat.nq * lat.nv;
    const int grid = (int)((total + 255) / 256 < 65536 ? (total + 255) / 256 : 65536);
    if (total > 0) {
        if (prec == SWPIC_F64)
            k_init_lattice<double><<<grid, 256, 0, s>>>(
                (double *)Q, (double *)P, decorated ? (double *)qs : nullptr,
                decorated ? (double *)ps : nullptr, (double *)psi, p0, L, lat, jx, jv, Xc, Xq, Vc,
                Vq, sbcb, sbcb + 5);
        else
            k_init_lattice<float><<<grid, 256, 0, s>>>(
                (float *)Q, (float *)P, decorated ? (float *)qs : nullptr,
                decorated ? (float *)ps : nullptr, (float *)psi, p0, L, lat, jx, jv, Xc, Xq, Vc, Vq,
                sbcb, sbcb + 5);
    }
    e = cudaGetLastError();
    cudaFreeAsync(tabs, s);
    return e;
}

cudaError_t launch_convert(int prec, const double *src, void *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    if (prec == SWPIC_F64) k_convert<double><<<grid, 256, 0, s>>>(src, (double *)dst, n);
    else k_convert<float><<<grid, 256, 0, s>>>(src, (float *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_mass(int prec, const void *psi, const void *ps, const SortChunk *chunks,
                        int n_chunks, double *partials, int n_runs, double *mass, double *bound,
                        cudaStream_t s) {
    if (n_chunks > 0) {
        if (prec == SWPIC_F64)
            k_mass_partial<double><<<n_chunks, 256, 0, s>>>((const double *)psi, (const double *)ps,
                                                            chunks, partials);
        else
            k_mass_partial<float><<<n_chunks, 256, 0, s>>>((const float *)psi, (const float *)ps,
                                                           chunks, partials);
    }
    if (n_runs > 0) k_mass_final<<<n_runs, 256, 0, s>>>(partials, chunks, n_chunks, mass, bound);
    return cudaGetLastError();
}

}  // namespace swpic
