// Kernels of the 2D2V decorated-particle step (general-d model of Sec. 3.3 on
// the torus T^2, bilinear elements, leapfrog of Sec. 5).
//
//   k_pass2d      one fused pass over the particles: gather grad phi_h and the
//                 projected Hessian from the node table in shared memory,
//                 closing half-kick, diagnostics at the integer time, opening
//                 half-kick, drift, wrap, deposit of the drifted monopole +
//                 dipole charge into a per-CTA shared mesh, flush to a global
//                 64-bit fixed-point accumulator (Eq. swpic_poisson, S_h = delta);
//                 in FP32 contexts its last CTA writes the diagnostic record and
//                 solves the new field in FP32 (solve_tail_f32); consecutive
//                 passes use programmatic dependent launch (each waits for its
//                 predecessor before it reads memory)
//   FP64 contexts solve in four kernels:
//   k_rows_fwd    node loads -> FP64, forward DFT of every mesh row
//   k_cols        per column: forward DFT, divide by the Q1 stiffness symbol
//                 (zero mode dropped: neutralising background + zero-mean gauge),
//                 inverse DFT
//   k_rows_inv    inverse DFT of every row -> Phi, field energy (1/2) Phi^T b
//   k_table       lumped projection g of grad phi_h, node table (Phi, g) in the
//                 state precision
//   k_record      one diagnostic record (FP64 contexts)
//   k_init_lattice2d  the lattice start
//
// The DFTs are radix-2 in shared memory: one CTA per row or column in FP64,
// the whole mesh in one CTA in FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "swpic2d_internal.cuh"

namespace swpic2d {

// node table entry (Phi, g_x, g_y, pad): one 16-byte load (FP32) or two (FP64)
struct alignas(16) Node64 { double x, y, z, w; };
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = Node64; };

__device__ __forceinline__ float flr(float x) { return floorf(x); }
__device__ __forceinline__ double flr(double x) { return floor(x); }

// floor(c) and its integer for c = s clamped to [0, cmax], cmax = n - 1/2,
// without a float <-> int conversion instruction (they run on this GPU's
// narrow FP64/conversion pipe): adding 2^23 (2^52) rounding down leaves
// floor(c) in the low mantissa bits.  NaN clamps to 0.
__device__ __forceinline__ int cell_index(float s, float cmax, float &fi) {
    const float c = fminf(fmaxf(s, 0.0f), cmax);
    const float y = __fadd_rd(c, 8388608.0f);
    fi = y - 8388608.0f;
    return __float_as_int(y) - 0x4B000000;
}
__device__ __forceinline__ int cell_index(double s, double cmax, double &fi) {
    const double c = fmin(fmax(s, 0.0), cmax);
    const double y = __dadd_rd(c, 4503599627370496.0);
    fi = y - 4503599627370496.0;
    return (int)(__double_as_longlong(y) - 0x4330000000000000ll);
}

// Cell along one axis: floor(Q / h) as one multiply by 1/h in the state
// precision, clamped to [0, n-1]; frac = Q/h - i (the local coordinate).
template <typename T>
__device__ __forceinline__ int cell_of(T Q, T inv_h, T cmax, T &frac) {
    const T s = Q * inv_h;
    T fi;
    const int i = cell_index(s, cmax, fi);
    frac = s - fi;
    return i;
}

// Periodic wrap into [0, L); a value that rounds up to L maps to 0.
template <typename T>
__device__ __forceinline__ T wrap(T Q, T L, T inv_L) {
    if (Q >= T(0) && Q < L) return Q;
    T w = Q - L * flr(Q * inv_L);
    if (w >= L) w -= L;
    if (w < T(0)) w += L;
    if (w >= L) w = T(0);
    return w;
}

template <typename T>
struct Kahan {
    T s, c;
    __device__ __forceinline__ void add(T x) {
        const T y = x - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 block sum; every thread of the block must call it.  Result valid in thread 0.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < nw; ++k) s += sh[k];
    return s;
}

// v 2^k rounded to an integer; |v 2^k| < 2^62 or the flag is set.  FP32
// values scale in FP32 (exact: a power of two) when 2^k is an FP32 normal.
__device__ __forceinline__ unsigned long long to_fixed(double v, double scale, int *err) {
    const double x = v * scale;
    if (!(fabs(x) < 4.611686018427388e18)) {       // 2^62; also catches NaN
        atomicOr(err, isfinite(v) ? kErrOverflow : kErrNonFinite);
        return 0ull;
    }
    return (unsigned long long)__double2ll_rn(x);
}
__device__ __forceinline__ unsigned long long to_fixed(float v, double scale, int *err) {
    if (scale < 0x1p-125 || scale > 0x1p125) return to_fixed((double)v, scale, err);
    const float x = v * (float)scale;
    if (!(fabsf(x) < 4.611686e18f)) {
        atomicOr(err, isfinite(v) ? kErrOverflow : kErrNonFinite);
        return 0ull;
    }
    return (unsigned long long)__float2ll_rn(x);
}

// ---------------------------------------------------------------------------
// Diagnostic record and the one-CTA FP32 solve (the tail of an FP32 pass)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bit_reverse(int i, int logn) {
    return (logn == 0) ? 0 : (int)(__brev((unsigned)i) >> (32 - logn));
}

// One record from the pass's partial sums at the integer time and the field
// energy of the field the pass used; clears the partial sums.  One thread.
__device__ void write_record(const RecordArgs2d &r) {
    if (r.rec) {
        const double W = *r.W;
        double *o = r.rec;
        o[0] = r.t;
        o[1] = r.diag_acc[0];
        o[2] = r.diag_acc[1];
        o[3] = r.diag_acc[2];
        o[4] = r.diag_acc[3];
        o[5] = W;
        o[6] = r.diag_acc[3] + W;
        o[7] = sqrt(fmax(2.0 * W / r.area, 0.0));
        o[8] = (double)r.step;
        if (!isfinite(o[6])) atomicOr(r.err, kErrNonFinite);
    }
    for (int q = 0; q < 4; ++q) r.diag_acc[q] = 0.0;
}

// Radix-2 DIT stages over the rows (stride 1, ROWS) or the columns (stride
// nx) of an ny x nx complex FP32 array whose lines are in bit-reversed order.
// nx = 2^lx, ny = 2^ly, ntw = 2^lt; tw in shared memory.
template <bool ROWS>
__device__ void fft_lines_f32(float2 *z, int lx, int ly, const float2 *tw, int lt, bool inverse) {
    const int nx = 1 << lx;
    const int ln = ROWS ? lx : ly, lh = ln - 1, total = 1 << (lx + ly - 1);
    for (int s = 0; s < ln; ++s) {                  // half = 2^s, len = 2^(s+1)
        const int half = 1 << s, tshift = lt - s - 1;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            int line, r;
            if (ROWS) { line = b >> lh; r = b & ((1 << lh) - 1); }
            else { line = b & (nx - 1); r = b >> lx; }
            const int g = r >> s, pos = r & (half - 1), k0 = (g << (s + 1)) + pos;
            const int i0 = ROWS ? (line << lx) + k0 : (k0 << lx) + line;
            const int i1 = i0 + (ROWS ? half : half << lx);
            float2 w = tw[pos << tshift];
            if (inverse) w.y = -w.y;
            const float2 u = z[i0], v = z[i1];
            const float2 t = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            z[i0] = make_float2(u.x + t.x, u.y + t.y);
            z[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

// In-place bit-reversal permutation of every row (ROWS) or column.
template <bool ROWS>
__device__ void brev_lines_f32(float2 *z, int lx, int ly) {
    const int nx = 1 << lx;
    for (int b = threadIdx.x; b < (1 << (lx + ly)); b += blockDim.x) {
        const int i = b & (nx - 1), j = b >> lx;
        const int k = ROWS ? i : j, r = bit_reverse(k, ROWS ? lx : ly);
        if (k < r) {
            const int o = ROWS ? (j << lx) + r : (r << lx) + i;
            const float2 t = z[b];
            z[b] = z[o];
            z[o] = t;
        }
    }
    __syncthreads();
}

__device__ long long block_sum_ll(long long v, long long *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    long long s = 0;
    for (int k = 0; k < nw; ++k) s += sh[k];
    return s;                                   // every thread
}

// The new field from the accumulated node loads, by one CTA in FP32 (FP32
// contexts): btilde = b - S/nn from the exact integers, forward DFT of the
// rows and columns, division by the Q1 symbol (zero mode dropped), inverse
// DFTs, W = (1/2) Phi^T btilde, the node table.  smem: 20 bytes per node.
__device__ void solve_tail_f32(const SolveArgs2d &s, unsigned char *smem) {
    __shared__ long long sh_ll[32];
    __shared__ double sh_d[32];
    const int nx = s.nx, ny = s.ny, nn = nx * ny, lognn = s.lognx + s.logny;
    long long *bi = reinterpret_cast<long long *>(smem);
    float2 *z = reinterpret_cast<float2 *>(smem + 8 * (size_t)nn);
    float *bt = reinterpret_cast<float *>(smem + 16 * (size_t)nn);
    long long part = 0;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const long long v = (long long)__ldcg(s.acc + k);
        s.acc[k] = 0ull;
        bi[k] = v;
        part += v;
        s.braw[k] = v;                  // the read-out scales it on the host
    }
    const long long S = block_sum_ll(part, sh_ll);
    const long long q = S >> lognn, rem = S & (long long)(nn - 1);
    const float frac = (float)rem * (float)s.inv_nn;
    const bool fsc = s.fx_k >= -125 && s.fx_k <= 125;       // 2^-k an FP32 normal: one exact multiply
    const float sc = fsc ? (float)s.fx_inv : 1.0f;
    const int lx = s.lognx, ly = s.logny;
    int lt = 0;
    while ((1 << lt) < s.ntw) ++lt;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const float u = (float)(bi[k] - q) - frac;
        const float v = fsc ? u * sc : scalbnf(u, -s.fx_k);
        bt[k] = v;
        const int i = k & (nx - 1), j = k >> lx;
        z[(j << lx) + bit_reverse(i, lx)] = make_float2(v, 0.0f);
    }
    __syncthreads();
    float2 *tw = reinterpret_cast<float2 *>(bi);             // the integers are no longer needed
    for (int k = threadIdx.x; k < (s.ntw >> 1); k += blockDim.x) tw[k] = s.twf[k];
    __syncthreads();
    fft_lines_f32<true>(z, lx, ly, tw, lt, false);
    brev_lines_f32<false>(z, lx, ly);
    fft_lines_f32<false>(z, lx, ly, tw, lt, false);
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const float il = s.inv_lamf[k];
        z[k] = make_float2(z[k].x * il, z[k].y * il);
    }
    __syncthreads();
    brev_lines_f32<false>(z, lx, ly);
    fft_lines_f32<false>(z, lx, ly, tw, lt, true);
    brev_lines_f32<true>(z, lx, ly);
    fft_lines_f32<true>(z, lx, ly, tw, lt, true);
    float *ph = reinterpret_cast<float *>(bi);            // the twiddles are no longer needed
    const float inv_nn = (float)s.inv_nn;
    float e = 0.0f;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const float phi = z[k].x * inv_nn;
        ph[k] = phi;                    // Phi is read out from the node table
        e += phi * bt[k];
    }
    __syncthreads();
    const float ihx = (float)s.inv_hx, ihy = (float)s.inv_hy;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const int i = k & (nx - 1), j = k >> lx;
        const int im = (i - 1) & (nx - 1), ip = (i + 1) & (nx - 1);
        const int jm = (j - 1) & (ny - 1), jp = (j + 1) & (ny - 1);
        auto cx = [&](int r) { return (ph[(r << lx) + ip] - ph[(r << lx) + im]) * (0.5f * ihx); };
        auto cy = [&](int c) { return (ph[(jp << lx) + c] - ph[(jm << lx) + c]) * (0.5f * ihy); };
        const float gx = (2.0f / 3.0f) * cx(j) + (1.0f / 6.0f) * (cx(jm) + cx(jp));
        const float gy = (2.0f / 3.0f) * cy(i) + (1.0f / 6.0f) * (cy(im) + cy(ip));
        reinterpret_cast<float4 *>(s.table)[k] = make_float4(ph[k], gx, gy, 0.0f);
    }
    const double Wt = block_sum((double)e, sh_d);
    if (threadIdx.x == 0) {
        *s.W = 0.5 * Wt;
        if (!isfinite(Wt)) atomicOr(s.err, kErrNonFinite);
    }
}

// ---------------------------------------------------------------------------
// The fused particle pass
// ---------------------------------------------------------------------------
template <typename T> struct Part { T x, y, vx, vy, w, sx, sy, rx, ry; };

template <typename T, bool DEC, bool DEP, bool DIAG>
__global__ void __launch_bounds__(256, 3) k_pass2d(PassArgs2d a) {
    using T4 = typename V4<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[32];
    // table and mesh rows are padded to nx + 1 entries, so that particles
    // stacked in y (an ordered or cold plasma) do not all hit one bank
    const int nx = a.nx, ny = a.ny, nn = nx * ny, rs = nx + 1, lgx = __ffs(nx) - 1;
    T4 *tab = reinterpret_cast<T4 *>(smem);
    T *mesh = reinterpret_cast<T *>(smem + (size_t)rs * ny * sizeof(T4));
    const T4 *gtab = reinterpret_cast<const T4 *>(a.table);
    // Programmatic dependent launch: this grid may be scheduled while the
    // previous pass is still finishing; wait for it before touching memory.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const int pk = (k >> lgx) * rs + (k & (nx - 1));
        tab[pk] = gtab[k];
        if (DEP) {
            mesh[pk] = T(0);
            if ((k & (nx - 1)) == 0) mesh[pk + nx] = T(0);      // the pad entry
        }
    }
    __syncthreads();

    T *Qx = static_cast<T *>(a.Qx), *Qy = static_cast<T *>(a.Qy);
    T *Px = static_cast<T *>(a.Px), *Py = static_cast<T *>(a.Py);
    T *qx = static_cast<T *>(a.qx), *qy = static_cast<T *>(a.qy);
    T *px = static_cast<T *>(a.px), *py = static_cast<T *>(a.py);
    const T *psi = static_cast<const T *>(a.psi);
    const T Lx = (T)a.Lx, Ly = (T)a.Ly, iLx = (T)a.inv_Lx, iLy = (T)a.inv_Ly;
    const T ihx = (T)a.inv_hx, ihy = (T)a.inv_hy;
    const T k1 = (T)a.k1, k2 = (T)a.k2, kd = (T)a.kd;
    const T cmx = T(nx) - T(0.5), cmy = T(ny) - T(0.5);
    Kahan<T> s_m{T(0), T(0)}, s_x{T(0), T(0)}, s_y{T(0), T(0)}, s_k{T(0), T(0)};

    // one particle per thread and turn; the next turn's particle is loaded
    // before this one is pushed, so its loads are in flight meanwhile
    auto load = [&](int64_t p, Part<T> &c) {
        c.x = Qx[p]; c.y = Qy[p]; c.vx = Px[p]; c.vy = Py[p]; c.w = psi[p];
        if (DEC) { c.sx = qx[p]; c.sy = qy[p]; c.rx = px[p]; c.ry = py[p]; }
        else { c.sx = c.sy = c.rx = c.ry = T(0); }
    };
    // lanes past the end of the particles carry empty deposit slots
    const int lognx = __ffs(nx) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t lane64 = threadIdx.x & 31;
    Part<T> cur;
    bool have = p < a.n;
    if (have) load(p, cur);
    for (; p - lane64 < a.n; p += stride) {
        Part<T> nxt;
        const bool nxt_have = p + stride < a.n;
        if (nxt_have) load(p + stride, nxt);
        T x = cur.x, y = cur.y, vx = cur.vx, vy = cur.vy, sx = cur.sx, sy = cur.sy, rx = cur.rx, ry = cur.ry;
        const T w = cur.w;
        const bool valid = have;
        cur = nxt;
        have = nxt_have;
        int dkey = -1;
        T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
        if (valid) {
        // grad phi_h and H_ik = d_k g_i at Q from the four corners of the cell
        T xi, eta;
        const int i = cell_of(x, ihx, cmx, xi), j = cell_of(y, ihy, cmy, eta);
        const int i1 = (i + 1 == nx) ? 0 : i + 1, j1 = (j + 1 == ny) ? 0 : j + 1;
        const T4 c00 = tab[j * rs + i], c10 = tab[j * rs + i1], c01 = tab[j1 * rs + i], c11 = tab[j1 * rs + i1];
        const T oe = T(1) - eta, ox = T(1) - xi;
        const T ex = ((c10.x - c00.x) * oe + (c11.x - c01.x) * eta) * ihx;
        const T ey = ((c01.x - c00.x) * ox + (c11.x - c10.x) * xi) * ihy;
        T hxx = T(0), hxy = T(0), hyx = T(0), hyy = T(0);
        if (DEC) {
            hxx = ((c10.y - c00.y) * oe + (c11.y - c01.y) * eta) * ihx;
            hxy = ((c01.y - c00.y) * ox + (c11.y - c10.y) * xi) * ihy;
            hyx = ((c10.z - c00.z) * oe + (c11.z - c01.z) * eta) * ihx;
            hyy = ((c01.z - c00.z) * ox + (c11.z - c10.z) * xi) * ihy;
        }
        // closing half-kick of the previous step
        vx -= k1 * ex;
        vy -= k1 * ey;
        if (DEC) {
            sx += k1 * (hxx * rx + hxy * ry);
            sy += k1 * (hyx * rx + hyy * ry);
        }
        if (DIAG) {
            s_m.add(w);
            s_x.add(w * vx + sx);
            s_y.add(w * vy + sy);
            s_k.add(T(0.5) * w * (vx * vx + vy * vy) + (sx * vx + sy * vy));
        }
        // opening half-kick of the next step
        vx -= k2 * ex;
        vy -= k2 * ey;
        if (DEC) {
            sx += k2 * (hxx * rx + hxy * ry);
            sy += k2 * (hyx * rx + hyy * ry);
        }
        // drift
        x = wrap(x + kd * vx, Lx, iLx);
        y = wrap(y + kd * vy, Ly, iLy);
        if (DEC) {
            rx -= kd * sx;
            ry -= kd * sy;
        }
        Qx[p] = x; Qy[p] = y; Px[p] = vx; Py[p] = vy;
        if (DEC) { qx[p] = sx; qy[p] = sy; px[p] = rx; py[p] = ry; }
        if (DEP) {
            // psi* N_c(Q) - p* . grad N_c(Q) for the four corners
            T u, v;
            const int di = cell_of(x, ihx, cmx, u), dj = cell_of(y, ihy, cmy, v);
            const T ou = T(1) - u, ov = T(1) - v;
            const T ax = DEC ? rx * ihx : T(0), ay = DEC ? ry * ihy : T(0);
            dkey = (dj << lognx) + di;
            d0 = w * ou * ov + ax * ov + ay * ou;
            d1 = w * u * ov - ax * ov + ay * u;
            d2 = w * ou * v + ax * v - ay * ou;
            d3 = w * u * v - ax * v - ay * u;
        }
        }
        if (DEP && dkey >= 0) {
            // one shared atomic per corner: the lattice start puts a warp's
            // lanes in neighbouring cells of a row, and a disordered plasma
            // spreads them, so aggregating lanes of one cell (which costs
            // shuffles on every particle) does not pay here
            const int di = dkey & (nx - 1), dj = dkey >> lognx;
            const int di1 = (di + 1) & (nx - 1), dj1 = (dj + 1) & (ny - 1);
            atomicAdd(mesh + dj * rs + di, d0);
            atomicAdd(mesh + dj * rs + di1, d1);
            atomicAdd(mesh + dj1 * rs + di, d2);
            atomicAdd(mesh + dj1 * rs + di1, d3);
        }
    }
    // every CTA has been scheduled by now: let the next pass launch early
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
    if (DEP) {
        for (int k = threadIdx.x; k < nn; k += blockDim.x) {
            const T v = mesh[(k >> lgx) * rs + (k & (nx - 1))];
            if (v != T(0)) atomicAdd(a.acc + k, to_fixed(v, a.fx_scale, a.err));
        }
    }
    if (DIAG) {
        const double m = block_sum(s_m.value(), s_red);
        const double mx = block_sum(s_x.value(), s_red);
        const double my = block_sum(s_y.value(), s_red);
        const double kk = block_sum(s_k.value(), s_red);
        if (threadIdx.x == 0) {
            atomicAdd(a.diag_acc + 0, m);
            atomicAdd(a.diag_acc + 1, mx);
            atomicAdd(a.diag_acc + 2, my);
            atomicAdd(a.diag_acc + 3, kk);
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (!a.tail) return;
        // the last CTA to finish (it sees every CTA's flush and partial sums)
        // writes the record and solves the new field; no wait on other CTAs
        __shared__ int s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(a.done, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        if ((a.tail & 1) && threadIdx.x == 0) write_record(a.rec);
        if (a.tail & 2) solve_tail_f32(a.solve, smem);
        if (threadIdx.x == 0) *a.done = 0u;
    }
}

// Bound of every partial sum of the deposit: sum psi* + 2 sum |p*_x|/hx +
// 2 sum |p*_y|/hy (FP64 atomics; only its binary exponent is used).
template <typename T>
__global__ void __launch_bounds__(256) k_bound2d(PassArgs2d a, double *out) {
    __shared__ double s_red[32];
    const T *psi = static_cast<const T *>(a.psi);
    const T *px = static_cast<const T *>(a.px), *py = static_cast<const T *>(a.py);
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride) {
        s += fabs((double)psi[p]);
        if (px) s += 2.0 * (fabs((double)px[p]) * a.inv_hx + fabs((double)py[p]) * a.inv_hy);
    }
    s = block_sum(s, s_red);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// ---------------------------------------------------------------------------
// Spectral solve
// ---------------------------------------------------------------------------
// In-place radix-2 DFT of n = 2^logn points already in bit-reversed order
// (sign -1 forward, +1 inverse; no normalisation).  All threads call it.
__device__ void fft_inplace(double2 *z, int n, const double2 *tw, int ntw, bool inverse) {
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1, step = ntw / len;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int g = b / half, pos = b - g * half;
            const int i0 = g * len + pos, i1 = i0 + half;
            double2 w = tw[pos * step];
            if (inverse) w.y = -w.y;
            const double2 u = z[i0], v = z[i1];
            const double2 t = make_double2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            z[i0] = make_double2(u.x + t.x, u.y + t.y);
            z[i1] = make_double2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_rows_fwd(SolveArgs2d s) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2 *z = reinterpret_cast<double2 *>(smem);
    const int j = blockIdx.x, nx = s.nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int k = j * nx + i;
        const long long q = (long long)s.acc[k];
        s.acc[k] = 0ull;
        const double b = (double)q * s.fx_inv;
        s.b[k] = b;
        z[bit_reverse(i, s.lognx)] = make_double2(b, 0.0);
    }
    if (j == 0 && threadIdx.x == 0) *s.W = 0.0;
    __syncthreads();
    fft_inplace(z, nx, s.tw, s.ntw, false);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) s.spec[j * nx + i] = z[i];
}

__global__ void __launch_bounds__(256) k_cols(SolveArgs2d s) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ny = s.ny, nx = s.nx, kx = blockIdx.x;
    double2 *z = reinterpret_cast<double2 *>(smem), *y = z + ny;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) z[bit_reverse(j, s.logny)] = s.spec[j * nx + kx];
    __syncthreads();
    fft_inplace(z, ny, s.tw, s.ntw, false);
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
        const double il = s.inv_lam[ky * nx + kx];
        const double2 v = z[ky];
        y[bit_reverse(ky, s.logny)] = make_double2(v.x * il, v.y * il);
    }
    __syncthreads();
    fft_inplace(y, ny, s.tw, s.ntw, true);
    for (int j = threadIdx.x; j < ny; j += blockDim.x) s.spec[j * nx + kx] = y[j];
}

__global__ void __launch_bounds__(256) k_rows_inv(SolveArgs2d s) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[32];
    double2 *z = reinterpret_cast<double2 *>(smem);
    const int j = blockIdx.x, nx = s.nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) z[bit_reverse(i, s.lognx)] = s.spec[j * nx + i];
    __syncthreads();
    fft_inplace(z, nx, s.tw, s.ntw, true);
    double e = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double phi = z[i].x * s.inv_nn;
        s.phi[j * nx + i] = phi;
        e += phi * s.b[j * nx + i];
    }
    e = block_sum(e, s_red);
    if (threadIdx.x == 0) {
        atomicAdd(s.W, 0.5 * e);
        if (!isfinite(e)) atomicOr(s.err, kErrNonFinite);
    }
}

// g_x(i,j) = (2/3) C_x(i,j) + (1/6)(C_x(i,j-1) + C_x(i,j+1)), C_x the central
// difference of Phi along x (the lumped projection of grad phi_h on a uniform
// bilinear mesh); g_y likewise across.
template <typename T>
__global__ void __launch_bounds__(256) k_table2d(SolveArgs2d s) {
    using T4 = typename V4<T>::type;
    const int nx = s.nx, ny = s.ny;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx * ny) return;
    const int i = k % nx, j = k / nx;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const double *P = s.phi;
    auto cx = [&](int r) { return (P[r * nx + ip] - P[r * nx + im]) * (0.5 * s.inv_hx); };
    auto cy = [&](int c) { return (P[jp * nx + c] - P[jm * nx + c]) * (0.5 * s.inv_hy); };
    const double gx = (2.0 / 3.0) * cx(j) + (1.0 / 6.0) * (cx(jm) + cx(jp));
    const double gy = (2.0 / 3.0) * cy(i) + (1.0 / 6.0) * (cy(im) + cy(ip));
    T4 t;
    t.x = (T)P[k];
    t.y = (T)gx;
    t.z = (T)gy;
    t.w = T(0);
    reinterpret_cast<T4 *>(s.table)[k] = t;
}

__global__ void k_record2d(RecordArgs2d r) {
    if (threadIdx.x == 0 && blockIdx.x == 0) write_record(r);
}

// ---------------------------------------------------------------------------
// Lattice initialisation: one thread per particle, cell integrals by the
// n^4 Gauss-Legendre rule in FP64 (nodes and weights on [-1, 1] in gl[0..n),
// gl[8..8+n)), stored in the state precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f0_lattice(const swpic2d_lattice &f, double x, double y, double vx, double vy) {
    return (1.0 + f.alpha * cos(f.kx * x + f.ky * y)) * exp(-(vx * vx + vy * vy) / (2.0 * f.vth * f.vth)) /
           (2.0 * M_PI * f.vth * f.vth);
}

template <typename T>
__global__ void __launch_bounds__(256) k_init_lattice2d(swpic2d_lattice f, double Lx, double Ly, const double *gl,
                                                        PassArgs2d a) {
    const int64_t n = (int64_t)f.nqx * f.nqy * f.nvx * f.nvy;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    // positions fastest: the lanes of a warp lie in neighbouring cells of one
    // row (distinct nodes, no shared-memory bank conflicts)
    const int i = (int)(p % f.nqx), j = (int)((p / f.nqx) % f.nqy);
    const int l = (int)((p / ((int64_t)f.nqx * f.nqy)) % f.nvy), k = (int)(p / ((int64_t)f.nqx * f.nqy * f.nvy));
    const double dx = Lx / f.nqx, dy = Ly / f.nqy, dvx = (f.vmax - f.vmin) / f.nvx, dvy = (f.vmax - f.vmin) / f.nvy;
    const double xc = (i + 0.5) * dx, yc = (j + 0.5) * dy;
    const double uc = f.vmin + (k + 0.5) * dvx, wc = f.vmin + (l + 0.5) * dvy;
    double sx = 0.0, sy = 0.0, tx = 0.0, ty = 0.0;
    if (f.decorate) {
        // f0 factors: (1 + alpha (cos kx x cos ky y - sin kx x sin ky y)) e(vx) e(vy) / (2 pi vth^2),
        // and each moment weight depends on one coordinate, so the n^4 rule is a
        // sum over (x, y) nodes times sums over the vx and vy nodes: the
        // transcendentals are taken per axis node, not per 4D node
        const int nq = f.quad_order;
        const double iv = 1.0 / (2.0 * f.vth * f.vth);
        double cxr[4], sxr[4], cys[4], sys_[4], pxr[4], pys[4];
        double bx = 0.0, by = 0.0, bqx = 0.0, bqy = 0.0;
        for (int r = 0; r < nq; ++r) {
            const double x = xc + 0.5 * dx * gl[r], y = yc + 0.5 * dy * gl[r];
            cxr[r] = cos(f.kx * x); sxr[r] = sin(f.kx * x);
            cys[r] = cos(f.ky * y); sys_[r] = sin(f.ky * y);
            pxr[r] = (Lx / (2.0 * M_PI)) * sin(2.0 * M_PI * (xc - x) / Lx);
            pys[r] = (Ly / (2.0 * M_PI)) * sin(2.0 * M_PI * (yc - y) / Ly);
            const double vx = uc + 0.5 * dvx * gl[r], vy = wc + 0.5 * dvy * gl[r];
            const double ex = gl[8 + r] * exp(-vx * vx * iv), ey = gl[8 + r] * exp(-vy * vy * iv);
            bx += ex; bqx += -ex * (uc - vx);
            by += ey; bqy += -ey * (wc - vy);
        }
        double a0 = 0.0, ax = 0.0, ay = 0.0;
        for (int r = 0; r < nq; ++r)
            for (int s = 0; s < nq; ++s) {
                const double F = gl[8 + r] * gl[8 + s] * (1.0 + f.alpha * (cxr[r] * cys[s] - sxr[r] * sys_[s]));
                a0 += F;
                ax += F * pxr[r];
                ay += F * pys[s];
            }
        const double K = 0.0625 * dx * dy * dvx * dvy / (2.0 * M_PI * f.vth * f.vth);
        sx = K * ax * bx * by;
        sy = K * ay * bx * by;
        tx = K * a0 * bqx * by;
        ty = K * a0 * bx * bqy;
    }
    static_cast<T *>(a.Qx)[p] = (T)xc;
    static_cast<T *>(a.Qy)[p] = (T)yc;
    static_cast<T *>(a.Px)[p] = (T)uc;
    static_cast<T *>(a.Py)[p] = (T)wc;
    const_cast<T *>(static_cast<const T *>(a.psi))[p] = (T)(f0_lattice(f, xc, yc, uc, wc) * dx * dy * dvx * dvy);
    if (a.qx) {
        static_cast<T *>(a.qx)[p] = (T)tx;
        static_cast<T *>(a.qy)[p] = (T)ty;
        static_cast<T *>(a.px)[p] = (T)sx;
        static_cast<T *>(a.py)[p] = (T)sy;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_init_lattice(int prec, const swpic2d_lattice &spec, double Lx, double Ly,
                                const double *gl, void *const st[9], cudaStream_t s) {
    PassArgs2d a{};
    a.Qx = st[0]; a.Qy = st[1]; a.Px = st[2]; a.Py = st[3];
    a.qx = st[4]; a.qy = st[5]; a.px = st[6]; a.py = st[7]; a.psi = st[8];
    const int64_t n = (int64_t)spec.nqx * spec.nqy * spec.nvx * spec.nvy;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (prec == SWPIC_F64) k_init_lattice2d<double><<<grid, 256, 0, s>>>(spec, Lx, Ly, gl, a);
    else k_init_lattice2d<float><<<grid, 256, 0, s>>>(spec, Lx, Ly, gl, a);
    return cudaGetLastError();
}
size_t pass_smem_bytes(int prec, int nx, int ny, bool deposit) {
    const size_t e = (prec == SWPIC_F64) ? 8 : 4, rows = (size_t)(nx + 1) * ny;   // padded rows
    return rows * 4 * e + (deposit ? rows * e : 0);
}

template <typename T>
static const void *pass_kernel_t(bool dec, bool dep, bool diag) {
    const int c = (dec ? 4 : 0) | (dep ? 2 : 0) | (diag ? 1 : 0);
    switch (c) {
    case 0: return (const void *)k_pass2d<T, false, false, false>;
    case 1: return (const void *)k_pass2d<T, false, false, true>;
    case 2: return (const void *)k_pass2d<T, false, true, false>;
    case 3: return (const void *)k_pass2d<T, false, true, true>;
    case 4: return (const void *)k_pass2d<T, true, false, false>;
    case 5: return (const void *)k_pass2d<T, true, false, true>;
    case 6: return (const void *)k_pass2d<T, true, true, false>;
    default: return (const void *)k_pass2d<T, true, true, true>;
    }
}

const void *pass_kernel(int prec, bool decorated, bool deposit, bool diag) {
    return prec == SWPIC_F64 ? pass_kernel_t<double>(decorated, deposit, diag)
                             : pass_kernel_t<float>(decorated, deposit, diag);
}

cudaError_t launch_pass(int prec, bool decorated, bool deposit, bool diag, const PassArgs2d &a, int grid,
                        int tpb, size_t smem, cudaStream_t s) {
    const void *fn = pass_kernel(prec, decorated, deposit, diag);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PassArgs2d copy = a;
    void *args[] = {&copy};
    // programmatic dependent launch: the next pass's CTAs become resident while
    // this one finishes (they wait for it in the kernel)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tpb);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_bound(int prec, const PassArgs2d &a, double *out, int grid, cudaStream_t s) {
    if (prec == SWPIC_F64) k_bound2d<double><<<grid, 256, 0, s>>>(a, out);
    else k_bound2d<float><<<grid, 256, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t launch_solve(int prec, const SolveArgs2d &a, cudaStream_t s, int64_t *launches) {
    const int tr = a.nx >= 256 ? 256 : (a.nx >= 64 ? a.nx / 2 : 32);
    const int tc = a.ny >= 256 ? 256 : (a.ny >= 64 ? a.ny / 2 : 32);
    k_rows_fwd<<<a.ny, tr, (size_t)a.nx * sizeof(double2), s>>>(a);
    k_cols<<<a.nx, tc, (size_t)2 * a.ny * sizeof(double2), s>>>(a);
    k_rows_inv<<<a.ny, tr, (size_t)a.nx * sizeof(double2), s>>>(a);
    const int nn = a.nx * a.ny;
    if (prec == SWPIC_F64) k_table2d<double><<<(nn + 255) / 256, 256, 0, s>>>(a);
    else k_table2d<float><<<(nn + 255) / 256, 256, 0, s>>>(a);
    *launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_record(const RecordArgs2d &a, cudaStream_t s) {
    k_record2d<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace swpic2d
