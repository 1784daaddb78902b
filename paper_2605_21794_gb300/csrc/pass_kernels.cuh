// The particle pass of the decorated-particle step (sm_103a), and the per-run
// field solve, done either by the last CTA of each run at the end of the
// depositing pass or by every CTA of the next pass at its start.
//
// Floating-point contraction is off for the translation units that include
// this header (pass.cu, pass64.cu: -fmad=false): every fused multiply-add is
// written as fma(), so each copy of the particle arithmetic (register-load and
// bulk-copy streams) rounds identically.
//
// One pass over the particles of every run does, per particle (Sec. 5,
// Eq. sw-evolution, with the canonical kick/drift split):
//   i      = clamp(floor(Q * nx/L), 0, nx-1)                       element of Q
//   P     -= c1 dt phi_h'_i ;  q* += c1 dt p* phi_h''(Q)           closing half-kick
//   [diag]  sum psi* P + q*,  sum psi* P^2/2 + q* P                 integer time
//   P     -= c2 dt phi_h'_i ;  q* += c2 dt p* phi_h''(Q)           opening half-kick
//   Q      = wrap(Q + cd dt P) ;  p* -= cd dt q*                    drift
//   [deposit] b_i += psi*(1 - xi) + p*/h,  b_{i+1} += psi* xi - p*/h  (Eq. rhs-assembly)
// with xi = Q nx/L - i of the drifted Q.  A full leapfrog step in one pass has
// c1 = c2 = 1/2, cd = 1: the two half-kicks with the same field are applied
// one after the other, so the pass is bit-for-bit the kick-drift-kick step.
//
// Deposit: each thread handles 16-byte vectors of consecutive particles.  When
// every lane of a warp finds all particles of its vector in one element, the
// lane first sums them; then lanes with equal elements in consecutive lanes are
// combined by a segmented shuffle reduction and one lane per segment adds the
// sum to the CTA's shared-memory mesh.  ATOMIC mode uses float/double shared
// atomics; DETERMINISTIC mode converts the (fixed-order) warp sums to 64-bit
// fixed point and uses integer atomics, which are associative, so the result
// does not depend on thread scheduling.  At the end of its particle range a
// CTA adds its mesh into the run's global int64 accumulator.
//
// The field solve removes the mean of b (Eq. neutrality / zero-mean test
// space), solves A Phi = btilde (Eq. lin-sys) by Gauss's law
//   e_j - e_{j-1} = btilde_j,  sum_j e_j = 0       (e_i = -phi_h' on element i)
// and builds the (phi_h', phi_h'') table.  Either the CTA that completes the
// last particles of a run (a completion counter, no spinning) does it at the
// end of the depositing pass and writes the table to global memory, or
// (PASS_FIELD_ACC) every CTA of the next pass does it at its start into its
// own shared-memory table while its first particle copies are in flight, so
// that no pass ends in a one-CTA solve; the accumulators rotate over three
// buffers so that the deposit being solved, the one being filled and the one
// being cleared are never the same.
#pragma once
#include <math.h>

#include "f32x2.cuh"
#include "swpic_internal.cuh"

namespace swpic {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
// The vector of particles one thread handles per array: two particles (8 bytes
// of FP32 state, 16 of FP64).  Two FP32 particles rather than four keep the
// FP32 push within 80 registers, so 24 warps fit an SM.  Vector ranges start
// on 16-byte boundaries (kAlignParticles) for the bulk copies.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float2; static constexpr int n = 2; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
template <typename T> struct AlignOf { static constexpr int n = 16 / (int)sizeof(T); };

__device__ __forceinline__ float flo(float x) { return floorf(x); }
__device__ __forceinline__ double flo(double x) { return floor(x); }

// A value the compiler must keep (or spill) rather than re-derive: under
// register pressure it would otherwise recompute loop-invariant values inside
// the particle loop, and conversions and FP64 arithmetic run on a narrow pipe
// on this GPU.
__device__ __forceinline__ float opaque(float x) {
    asm volatile("" : "+f"(x));
    return x;
}
__device__ __forceinline__ double opaque(double x) {
    asm volatile("" : "+d"(x));
    return x;
}

// cmax = nx - 1/2 bounds the element coordinate (see elem_index)
template <typename T> struct Geo { T L, inv_h, inv_L, dt, inv_h_lo, L_lo, cmax; };
__device__ __forceinline__ Geo<float> geo_of(const RunDev &r, float) {
    return {r.Lf, r.inv_hf, r.inv_Lf, r.dtf, r.inv_hf_lo, r.L_lo, opaque((float)r.nx - 0.5f)};
}
__device__ __forceinline__ Geo<double> geo_of(const RunDev &r, double) {
    return {r.L, r.inv_h, r.inv_L, r.dt, 0.0, 0.0, opaque((double)r.nx - 0.5)};
}

// Position inside element i, xi = Q nx/L - i.  The element index itself is
// decided by the single rounded product (the key definition); xi is formed
// as Q inv_h - i in one fused operation (the result is below 1, so it is
// rounded at the ulp of xi, not of Q nx/L), with the low part of nx/L added
// back, so an FP32 state does not see the ~nx ulp bias of fl32(nx/L) near
// Q = L.  fi is the element index as a float (p, the rounded product, is not
// needed).
__device__ __forceinline__ float xi_of(float Q, float p, float fi, const Geo<float> &G) {
    (void)p;
    return fmaf(Q, G.inv_h_lo, fmaf(Q, G.inv_h, -fi));
}
__device__ __forceinline__ double xi_of(double, double p, double fi, const Geo<double> &) {
    return p - fi;
}

// element of Q (see elem_index); p and fi are kept for xi_of
template <typename T>
__device__ __forceinline__ int elem_of(T Q, const Geo<T> &G, T &p, T &fi) {
    p = Q * G.inv_h;
    return elem_index_c(p, G.cmax, fi);
}

// Periodic wrap into [0, L); a value that rounds up to L maps to 0.
template <typename T>
__device__ __forceinline__ T wrap_pos(T Q, T L) {
    if (Q < T(0) || Q >= L) {
        T k = flo(Q / L);
        Q = Q - L * k;
        if (Q >= L) Q -= L;
        if (Q < T(0)) Q += L;
    }
    return Q;
}

// Drift with the periodic wrap, Q' = Q + kd P mod L.
// FP64: the domain length is the double L itself.
__device__ __forceinline__ double drift_wrap(double Q, double P, double kd, const Geo<double> &G) {
    return wrap_pos(fma(kd, P, Q), G.L);
}
// FP32: L is not a float; it is carried as L = L_hi + L_lo (L_hi = fl32(L)).
// Inside-test and shifts use both parts, and a crossing of L is formed from
// the unrounded sum, Q' = (Q - L_hi) + kd P - L_lo, so particles that wrap
// are not displaced by L - fl32(L) (which would bias the charge at the
// periodic node).  A value that can only round onto L moves to the wrapped
// side, as the FP32 rounding of the exact position does.
__device__ __forceinline__ bool inside_f32(float Q, const Geo<float> &G) {
    return Q >= 0.0f && (Q - G.L) < G.L_lo;        // Q - L_hi is exact near L
}
__device__ __forceinline__ float drift_wrap(float Q, float P, float kd, const Geo<float> &G) {
    const float q0 = fmaf(kd, P, Q);
    const float qa = fmaf(kd, P, Q - G.L) - G.L_lo;        // if it crossed L
    const float qb = (q0 + G.L) + G.L_lo;                   // if it crossed 0
    const bool in0 = inside_f32(q0, G) || q0 != q0;
    float Qn = in0 ? q0 : (q0 >= 0.0f ? qa : qb);           // selects, no divergent branch
    if (in0 || inside_f32(Qn, G)) return Qn;
    // several periods in one step, or a value that rounded onto the boundary
    const float k = floorf(Qn * G.inv_L);
    Qn = fmaf(-k, G.L_lo, fmaf(-k, G.L, Qn));
    if (Qn >= 0.0f && !inside_f32(Qn, G)) Qn = (Qn - G.L) - G.L_lo;
    if (Qn < 0.0f) Qn = (Qn + G.L) + G.L_lo;
    if (!inside_f32(Qn, G)) Qn = (Qn < 0.0f) ? 0.0f : (Qn - G.L) - G.L_lo;
    return Qn < 0.0f ? 0.0f : Qn;
}

// value * 2^k as an int64 bit pattern; out-of-range (or NaN) sets the error flag
__device__ __forceinline__ unsigned long long to_fixed(double x, double scale, int32_t *err) {
    double y = x * scale;
    if (!(fabs(y) < 4.0e18)) { atomicOr(err, kErrFixedOverflow); return 0ull; }
    return (unsigned long long)__double2ll_rn(y);
}
__device__ __forceinline__ unsigned long long to_fixed(float x, float scale, int32_t *err) {
    float y = x * (float)scale;   // exact: scale is a power of two
    if (!(fabsf(y) < 4.0e18f)) { atomicOr(err, kErrFixedOverflow); return 0ull; }
    return (unsigned long long)__float2ll_rn(y);
}

// ---------------------------------------------------------------------------
// block-wide helpers (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long warp_sum_ll(long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
static __device__ long long block_sum_ll(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_ll(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    long long t = 0;
    for (int k = 0; k < nw; ++k) t += sh[k];
    return t;
}
static __device__ double block_sum_d(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += sh[k];   // fixed order: deterministic
    return t;
}
// exclusive scan of one int64 per thread, in thread order
static __device__ long long block_exscan_ll(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    long long base = 0;
    for (int k = 0; k < w; ++k) base += sh[k];
    (void)nw;
    return base + inc - v;
}

// ---------------------------------------------------------------------------
// per-run field solve by one CTA.
//
// The charge arrives as int64 fixed point (acc_j = b_j 2^k).  Neutralisation
// and Gauss's law are exact in integers:
//   S = sum_j acc_j = q nx + rem (0 <= rem < nx),  bt_j = acc_j - q
//   e_int_j = sum_{i<=j} bt_i                       (exact prefix)
// so btilde_j = (bt_j - rem/nx) 2^-k and the element field, after the
// zero-sum gauge, is e_j = (e_int_j - mean(e_int)) 2^-k - (j + 1 - (nx+1)/2) rem/nx 2^-k.
// The table takes phi_h' = -e_j and the lumped phi'' (e_{j-1} - e_{j+1})/(2h)
// = -(bt_j + bt_{j+1}) 2^-k/(2h) straight from the integers (FP32 path: one
// rounding to float; FP64 path: FP64).  The accumulator is snapshot for
// read-out and zeroed for the next pass; W = (h/2) sum e^2 and E_amp are kept
// in FP64.  full = false: only the snapshot (swpic_deposit's read-out).
// ---------------------------------------------------------------------------
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        v += (__int128)(((unsigned __int128)ohi << 64) | (unsigned __int128)olo);
    }
    return v;
}

// Inputs of a run's diagnostic record, loaded by thread 0 into registers
// before the solve (their latency overlaps it); the record is written after
// the solve, with the field energy of the field this pass used (field_diag
// before the solve overwrites it).
struct DiagPre {
    long long step;
    int32_t count;
    double mass, mom, kin, W, Ea;
};
__device__ __forceinline__ void diag_preload(const PassArgs &a, int r, DiagPre &d) {
    d.step = a.steps[r];
    d.count = a.ring_count[r];
    d.mass = a.mass[r];
    d.mom = __ldcg(a.diag_acc + 2 * r);
    d.kin = __ldcg(a.diag_acc + 2 * r + 1);
    d.W = a.field_diag[2 * r];
    d.Ea = a.field_diag[2 * r + 1];
}
__device__ __forceinline__ void diag_write(const PassArgs &a, const RunDev &R, int r, const DiagPre &d) {
    double *rec = a.ring + ((size_t)r * a.ring_cap + (size_t)(d.count % a.ring_cap)) * kDiagWords;
    rec[0] = (double)d.step * R.dt;
    rec[1] = d.mass;
    rec[2] = d.mom;
    rec[3] = d.kin;
    rec[4] = d.W;
    rec[5] = d.kin + d.W;
    rec[6] = d.Ea;
    rec[7] = (double)d.step;
    a.ring_count[r] = d.count + 1;
    a.diag_acc[2 * r] = 0.0;
    a.diag_acc[2 * r + 1] = 0.0;
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}
__device__ __forceinline__ double i128_to_double(__int128 v) {
    return (double)(long long)(v >> 64) * 18446744073709551616.0 + (double)(unsigned long long)v;
}
// nearest float to a 64-bit integer (ties to even, as a conversion rounds),
// from integer operations only: the conversion instruction runs on the
// narrow FP64/conversion pipe of this GPU
__device__ __forceinline__ float ll_to_float(long long x) {
    const unsigned long long ax = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    if (ax == 0ull) return 0.0f;
    const int lz = __clzll((long long)ax);
    const unsigned long long m = ax << lz;                      // leading one at bit 63
    unsigned mant = (unsigned)(m >> 40);                        // 24 bits with the leading one
    const unsigned long long rest = m & 0xFFFFFFFFFFull, half = 0x8000000000ull;
    mant += (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
    const unsigned bits = ((unsigned)(190 - lz) << 23) + (mant - 0x800000u);   // a carry lifts the exponent
    return __uint_as_float(bits | (x < 0 ? 0x80000000u : 0u));
}

// One CTA, all its threads.  src (src_m: P2 midpoint loads) is the run's
// slice of a finished deposit; s_p is nx int64 of shared scratch.  The table
// goes to tab_sh (shared, when given) and, with globals, to the run's global
// table together with the snapshot, W, E_amp and the gauge; without globals
// nothing outside the CTA is written.  full = false: snapshot only
// (swpic_deposit's read-out).  The deposit itself is left as it is (the
// accumulators rotate between passes).
template <typename T, bool P2>
__device__ void solve_run(const PassArgs &a, const RunDev &R, int r, long long *s_p,
                          const unsigned long long *src, const unsigned long long *src_m,
                          typename Vec2<T>::type *tab_sh, bool globals, bool full) {
    using T2 = typename Vec2<T>::type;
    __shared__ long long sh_ll[34];
    __shared__ __int128 sh_q[2][32];
    const int nx = R.nx, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    long long *snap = a.snap + R.mesh_off;
    const int off = R.mesh_off;
    const int per = (nx + nt - 1) / nt;
    const int j0 = min(nx, tid * per), j1 = min(nx, j0 + per);
    // reference for the field energy: the last gauge mean
    const long long c = globals ? a.gauge[r] : 0ll;

    // 1. load (coalesced; a thread's loads are independent and unrolled, so
    //    the L2 round trips overlap), snapshot
#pragma unroll 8
    for (int j = tid; j < nx; j += nt) {
        const long long v = (long long)__ldcg(src + j);
        s_p[j] = v;
        if (globals) snap[j] = v;
    }
    if (!full) return;
    __syncthreads();
    // 2. one block scan of the chunk sums gives S = q nx + rem (0 <= rem < nx)
    //    and the exclusive prefix P of this thread's chunk
    long long tot = 0;
    for (int j = j0; j < j1; ++j) tot += s_p[j];
    long long inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh_ll[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long x = (lane < nw) ? sh_ll[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) sh_ll[lane] = x;                          // inclusive warp totals
        if (lane == nw - 1) {
            long long qq, rr;
            if ((nx & (nx - 1)) == 0) {                         // nx = 2^m: floor shift, low bits
                qq = x >> (__ffs(nx) - 1);
                rr = x & (long long)(nx - 1);
            } else {
                qq = x / nx;
                rr = x % nx;
                if (rr < 0) { rr += nx; qq -= 1; }
            }
            sh_ll[32] = qq;
            sh_ll[33] = rr;
        }
    }
    __syncthreads();
    const long long q = sh_ll[32], rem = sh_ll[33];
    long long P = ((warp > 0) ? sh_ll[warp - 1] : 0) + inc - tot;
    // 3. e_int_j = P_j - (j+1) q (exact Gauss prefix of btilde_j = acc_j - q),
    //    with the exact sums of e_int and of ((e_int - c) >> 8)^2 for the gauge
    //    and the field energy (one int128 block reduction for both)
    __int128 es = 0, e2 = 0;
    for (int j = j0; j < j1; ++j) {
        P += s_p[j];
        const long long e = P - (long long)(j + 1) * q;
        s_p[j] = e;
        es += (__int128)e;
        if (globals) {
            const long long e8 = (e - c) >> 8;                  // squares of 2^55 sum safely in int128
            e2 += (__int128)e8 * e8;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        es += shfl_xor_i128(es, o);
        if (globals) e2 += shfl_xor_i128(e2, o);    // globals is uniform over the CTA
    }
    __syncthreads();                                            // sh_ll reads above are done
    if (lane == 0) { sh_q[0][warp] = es; sh_q[1][warp] = e2; }
    __syncthreads();
    const double inv = R.fx_inv;
    // 4. gauge mean m = esum / nx as an integer part and a fraction: for
    //    nx = 2^m every thread takes it from the shift and the low bits of the
    //    exact sum; otherwise thread 0 refines a double estimate exactly.
    long long mean_i, mrem;
    const bool pow2 = (nx & (nx - 1)) == 0;
    if (pow2) {
        __int128 esum = 0;
        for (int w = 0; w < nw; ++w) esum += sh_q[0][w];
        mean_i = (long long)(esum >> (__ffs(nx) - 1));
        mrem = (long long)(esum & (__int128)(nx - 1));
    } else {
        if (tid == 0) {
            __int128 esum = 0;
            for (int w = 0; w < nw; ++w) esum += sh_q[0][w];
            long long mi = (long long)floor(i128_to_double(esum) * R.inv_nx);
            __int128 rr = esum - (__int128)mi * nx;
            while (rr < 0) { rr += nx; --mi; }
            while (rr >= nx) { rr -= nx; ++mi; }
            sh_ll[0] = mi;
            sh_ll[1] = (long long)rr;
        }
        __syncthreads();
        mean_i = sh_ll[0];
        mrem = sh_ll[1];
    }
    //    Thread 0 then computes the field energy about the reference while
    //    the other warps build the table: sum (e - m)^2 = sum (e - c)^2 -
    //    nx (m - c)^2 (no cancellation while c is near m), W = (h/2) sum e^2
    //    2^-2k, E_amp, in FP64 for either state precision (the sums are exact
    //    integers; only their conversion and the products round).
    if (globals && tid == 0) {
        __int128 e2sum = 0;
        for (int w = 0; w < nw; ++w) e2sum += sh_q[1][w];
        const double d8 = ((double)(mean_i - c) + (double)mrem * R.inv_nx) * (1.0 / 256.0);
        const double sc = inv * 256.0;                      // undo the >> 8
        double E2 = (i128_to_double(e2sum) - (double)nx * d8 * d8) * sc * sc;
        if (E2 < 0.0) E2 = 0.0;
        const double W = 0.5 * R.h * E2;
        a.field_diag[2 * r] = W;
        a.field_diag[2 * r + 1] = sqrt(E2 * R.inv_nx);
        if (!isfinite(W)) atomicOr(a.err + r, kErrNonFinite);
        a.gauge[r] = mean_i;
    }
    // the table nodes go to the threads after warp 0 while thread 0 forms the
    // energy (to all threads when there is one warp or no energy to form)
    const int tb = (globals && nt > 32) ? 32 : 0, nt2 = nt - tb;
    const int per2 = (nx + nt2 - 1) / nt2;
    const int t2 = tid - tb;
    const int k0 = (t2 < 0) ? nx : min(nx, t2 * per2), k1 = (t2 < 0) ? nx : min(nx, k0 + per2);
    // 5. the (phi_h', phi_h'') table.  P2: phi_h'(xi) = -e + beta (1 - 2 xi) with
    //    beta = (3/4) btilde_m, btilde_m = b_m - (2/3) S/nx (the midpoint load
    //    less its share of the uniform background), from exact integers
    T2 *tab = reinterpret_cast<T2 *>(a.table) + off;
    constexpr bool p2 = P2;
    double beta2 = 0.0;
    if (sizeof(T) == 4) {
        // FP32 table straight from the exact integers; the sub-quantum
        // gauge/remainder terms (< nx quanta) are below FP32 resolution
        // the FP32 units from the run parameters (rounded once on the host:
        // no FP64 conversions on this GPU's narrow FP64 pipe here)
        const float finv = R.fx_invf;                           // power of two: exact
        const float f_inv_h = R.inv_hf, f_half_inv_h = 0.5f * R.inv_hf;   // 0.5 scales exactly
        for (int j = k0; j < k1; ++j) {
            const int jm = (j == 0) ? nx - 1 : j - 1, jp = (j == nx - 1) ? 0 : j + 1;
            const long long ej_i = s_p[j], em_i = s_p[jm], ep_i = s_p[jp];
            const long long btj = (j == 0) ? ej_i : ej_i - em_i;
            T2 t;
            t.x = (T)(-(ll_to_float(ej_i - mean_i) * finv));
            if constexpr (p2) {
                const long long bm = (long long)__ldcg(src_m + j);
                const float beta = (0.25f * ll_to_float(3 * bm - 2 * q) - 0.5f * ll_to_float(rem) * R.inv_nxf) * finv;
                t.y = (T)beta;
                beta2 += (double)(beta * beta);
            } else if (a.d2_mode == SWPIC_D2_NODAL) {
                t.y = (T)(-ll_to_float(btj) * finv * f_inv_h);
            } else {
                t.y = (T)(ll_to_float(em_i - ep_i) * finv * f_half_inv_h);
            }
            if (tab_sh) tab_sh[j] = t;
            if (globals) tab[j] = t;
        }
    } else {
        const double mfrac = (double)mrem * R.inv_nx;
        const double rem_node = (double)rem * inv * R.inv_nx;
        const double cen = 0.5 * (double)(nx + 1);
        auto efield = [&](long long eint, int kk) {
            return ((double)(eint - mean_i) - mfrac) * inv - ((double)(kk + 1) - cen) * rem_node;
        };
        for (int j = k0; j < k1; ++j) {
            const int jm = (j == 0) ? nx - 1 : j - 1, jp = (j == nx - 1) ? 0 : j + 1;
            const long long ej_i = s_p[j], em_i = s_p[jm], ep_i = s_p[jp];
            const long long btj = (j == 0) ? ej_i : ej_i - em_i;
            T2 t;
            t.x = (T)(-efield(ej_i, j));
            if constexpr (p2) {
                const long long bm = (long long)__ldcg(src_m + j);
                const double beta = (0.25 * (double)(3 * bm - 2 * q) - 0.5 * (double)rem * R.inv_nx) * inv;
                t.y = (T)beta;
                beta2 += beta * beta;
            } else if (a.d2_mode == SWPIC_D2_NODAL) {
                t.y = (T)(-((double)btj * inv - rem_node) * R.inv_h);
            } else {
                t.y = (T)((efield(em_i, jm) - efield(ep_i, jp)) * (0.5 * R.inv_h));
            }
            if (tab_sh) tab_sh[j] = t;
            if (globals) tab[j] = t;
        }
    }
    if (p2 && globals) {
        // P2 field energy: (1/2) int phi'^2 = (h/2) sum (e^2 + beta^2/3); E_amp = (2W/L)^(1/2)
        __shared__ double sh_b[32];
        const double b2 = block_sum_d(beta2, sh_b);
        if (tid == 0) {
            const double W = a.field_diag[2 * r] + R.h * b2 / 6.0;
            a.field_diag[2 * r] = W;
            a.field_diag[2 * r + 1] = sqrt(2.0 * W * R.inv_nx / R.h);
            if (!isfinite(W)) atomicOr(a.err + r, kErrNonFinite);
        }
    }
}

// FP64 read-out of a run's mesh quantities from the integer snapshot (one CTA
// per run): b, btilde, E (zero-sum gauge) exactly as the solve defines them.
static __device__ void readout_run(const PassArgs &a, const RunDev &R, unsigned char *smem) {
    __shared__ long long sh_ll[32];
    __shared__ double sh_d[32];
    const int nx = R.nx, tid = threadIdx.x, nt = blockDim.x;
    long long *s_v = reinterpret_cast<long long *>(smem);
    const int per = (nx + nt - 1) / nt;
    const int j0 = min(nx, tid * per), j1 = min(nx, j0 + per);
    const long long *snap = a.snap + R.mesh_off;
    const int off = R.mesh_off;
    long long loc = 0;
    for (int j = j0; j < j1; ++j) { s_v[j] = snap[j]; loc += s_v[j]; }
    const long long S = block_sum_ll(loc, sh_ll);
    long long q = S / nx, rem = S % nx;
    if (rem < 0) { rem += nx; q -= 1; }
    const double inv = R.fx_inv;
    const double rem_node = (double)rem * inv / (double)nx;
    long long tot = 0;
    for (int j = j0; j < j1; ++j) tot += s_v[j] - q;
    long long p = block_exscan_ll(tot, sh_ll);
    double es = 0.0;
    for (int j = j0; j < j1; ++j) {
        const long long bt = s_v[j] - q;
        p += bt;
        a.b[off + j] = (double)s_v[j] * inv;
        a.btilde[off + j] = (double)bt * inv - rem_node;
        const double er = (double)p * inv - (double)(j + 1) * rem_node;
        a.efield[off + j] = er;
        es += er;
    }
    const double mean_e = block_sum_d(es, sh_d) / (double)nx;
    for (int j = j0; j < j1; ++j) a.efield[off + j] -= mean_e;
}

// ---------------------------------------------------------------------------
// per-thread state of a pass
// ---------------------------------------------------------------------------
template <typename T>
struct Kahan {
    T s, c;
    __device__ __forceinline__ void add(T x) {
        T y = x - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename T>
struct Thread {
    Kahan<T> mom, kin;     // diagnostics partials (integer-time P, q*)
};

template <typename T, int MODE>
__device__ __forceinline__ void mesh_add(int key, T a0, T a1, void *mesh, T scale, int32_t *err) {
    if (MODE == SWPIC_DEPOSIT_ATOMIC) {
        T *m = reinterpret_cast<T *>(mesh);
        atomicAdd(m + key, a0);
        atomicAdd(m + key + 1, a1);
    } else {
        unsigned long long *m = reinterpret_cast<unsigned long long *>(mesh);
        atomicAdd(m + key, to_fixed(a0, scale, err));
        atomicAdd(m + key + 1, to_fixed(a1, scale, err));
    }
}

// P2: one particle's midpoint load into the CTA's per-element mesh
template <typename T, int MODE>
__device__ __forceinline__ void mesh_m_add(int key, T v, void *mesh_m, T scale, int32_t *err) {
    if (MODE == SWPIC_DEPOSIT_ATOMIC) atomicAdd(reinterpret_cast<T *>(mesh_m) + key, v);
    else atomicAdd(reinterpret_cast<unsigned long long *>(mesh_m) + key, to_fixed(v, scale, err));
}

// Warp-aggregated deposit: lanes holding the same element in consecutive lanes
// form a segment; a segmented suffix sum (up to 5 shuffle steps, fixed order)
// gives the segment's first lane the segment total, and only that lane touches
// the shared mesh.  When no lane shares its element with the lane before (a
// disordered plasma) the shuffles are skipped and every lane adds its own
// value.  key < 0 marks an empty slot.  All 32 lanes must call this.  P2:
// the element's midpoint load am is combined alongside and added to the
// per-element mesh by the same lane.
template <typename T, int MODE, bool P2 = false>
__device__ __forceinline__ void warp_deposit(int key, T a0, T a1, void *mesh, T scale,
                                             int32_t *err, T am = T(0), void *mesh_m = nullptr) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(full, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(full, head);
    if (heads != full) {
        const unsigned above = (lane == 31) ? 0u : (heads & (0xffffffffu << (lane + 1)));
        const int seg_end = above ? (__ffs(above) - 2) : 31;
        // rounds only up to the longest segment (a uniform trip count): a disordered
        // warp with short segments skips most of the five shuffle rounds
        const int span = __reduce_max_sync(full, (unsigned)(seg_end - lane));   // longest segment - 1
#pragma unroll 1
        for (int off = 1; off <= span; off <<= 1) {
            const T b0 = __shfl_down_sync(full, a0, off);
            const T b1 = __shfl_down_sync(full, a1, off);
            T bm = T(0);
            if (P2) bm = __shfl_down_sync(full, am, off);
            if (lane + off <= seg_end) {
                a0 += b0;
                a1 += b1;
                if (P2) am += bm;
            }
        }
    }
    if (head && key >= 0) {
        mesh_add<T, MODE>(key, a0, a1, mesh, scale, err);
        if (P2) mesh_m_add<T, MODE>(key, am, mesh_m, scale, err);
    }
}

// Push one particle; returns its deposit (element of the drifted Q, weights of
// nodes key and key+1) in key/w0/w1 when DEP.
template <typename T, bool DEC, bool DEP, bool DIAG, int D2>
__device__ __forceinline__ void push_one(T &Q, T &P, T &qs, T &ps, const T w,
                                         const typename Vec2<T>::type *tab, const int nx,
                                         const Geo<T> &G, const T k1, const T k2, const T kd,
                                         T &dm, T &dk, int &key, T &w0, T &w1, T &wm) {
    T p0, f0;
    const int i = elem_of(Q, G, p0, f0);
    const auto f = tab[i];
    T d2 = T(0);
    T d1 = f.x;                                 // phi_h'(Q)
    if (D2 == SWPIC_D2_P2) {
        // P2: phi_h' = a + beta (1 - 2 xi), phi_h'' = -2 beta / h on the element
        const T xi = xi_of(Q, p0, f0, G);
        d1 = fma(f.y, T(1) - T(2) * xi, f.x);
        if (DEC) d2 = T(-2) * G.inv_h * f.y;
    } else if (DEC) {
        if (D2 == SWPIC_D2_NODAL) {
            const T xi = xi_of(Q, p0, f0, G);
            const T g1 = tab[i + 1 == nx ? 0 : i + 1].y;
            d2 = fma(xi, g1 - f.y, f.y);
        } else {
            d2 = f.y;
        }
    }
    // closing half-kick of the previous step
    P = fma(-k1, d1, P);
    if (DEC) qs = fma(k1 * ps, d2, qs);
    if (DIAG) {
        dm = DEC ? fma(w, P, qs) : w * P;                                 // momentum density
        dk = DEC ? fma(T(0.5) * w * P, P, qs * P) : T(0.5) * w * P * P;  // kinetic density
    }
    // opening half-kick of the next step
    P = fma(-k2, d1, P);
    if (DEC) qs = fma(k2 * ps, d2, qs);
    // drift
    Q = drift_wrap(Q, P, kd, G);
    if (DEC) ps = fma(-kd, qs, ps);
    if (DEP) {
        T p1, f1;
        key = elem_of(Q, G, p1, f1);
        const T xi = xi_of(Q, p1, f1, G);
        if (DEC) {
            const T dq = ps * G.inv_h;
            w0 = fma(w, T(1) - xi, dq);
            w1 = fma(w, xi, -dq);
        } else {
            w0 = w * (T(1) - xi);
            w1 = w * xi;
        }
        // P2: the vertex loads condense exactly to w0, w1 above; the midpoint
        // load psi* N_m(xi) - p* N_m'(xi), N_m = 4 xi (1 - xi), goes to its own
        // accumulator
        if (D2 == SWPIC_D2_P2) {
            wm = T(4) * w * xi * (T(1) - xi);
            if (DEC) wm = fma(-ps * G.inv_h, T(4) - T(8) * xi, wm);
        }
    }
}

// run r of a pass: from the kernel parameters when the pass has one run
__device__ __forceinline__ RunDev run_of(const PassArgs &a, int r) { return a.n_runs == 1 ? a.run0 : a.runs[r]; }

__device__ __forceinline__ int find_run(const RunDev *runs, int n_runs, int64_t idx) {
    int lo = 0, hi = n_runs - 1;
    while (lo < hi) {                // largest r with p0 <= idx
        int mid = (lo + hi + 1) >> 1;
        if (runs[mid].p0 <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Kick and drift coefficients of a pass for one run, c dt rounded once to T
// (opaque: the FP64 products are not to be recomputed per particle).
template <typename T>
__device__ __forceinline__ void step_coefficients(const PassArgs &a, const RunDev &R, T &k1, T &k2, T &kd) {
    k1 = opaque((T)(a.c1 * R.dt));
    k2 = opaque((T)(a.c2 * R.dt));
    kd = opaque((T)(a.cd * R.dt));
}

// Deposit slots of one 16-byte vector of particles: element and node weights.
template <typename T>
struct VecOut {
    static constexpr int n = Vec16<T>::n;
    int key[n];
    T w0[n], w1[n], wm[n];       // wm: P2 midpoint load (unused otherwise)
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int l = 0; l < n; ++l) { key[l] = -1; w0[l] = T(0); w1[l] = T(0); wm[l] = T(0); }
    }
};

// ---------------------------------------------------------------------------
// FP32 two-particle vectors in packed arithmetic.  Compute capability 10.x
// executes add, sub, mul and fma on a pair of FP32 values (.f32x2) as one
// instruction; each half is rounded exactly as the scalar operation would be,
// so the push below gives bit for bit the results of push_one on each
// particle (up to the sign of an exactly zero deposit weight), with half the
// FP32 instructions.  min, max and negation have no packed form: the clamps
// of the element index stay scalar, and negated operands are formed as 0 - x.
// ---------------------------------------------------------------------------
using namespace f32x2;

// element index of both halves of p = Q nx/L (see elem_index_c): clamp,
// 2^23 + p rounded down, bit pattern minus that of 2^23; fi = floor(p) as floats
__device__ __forceinline__ void elem2(f2p p, float cmax, int &i0, int &i1, f2p &fi) {
    float a, b;
    upk2(p, a, b);
    a = fminf(fmaxf(a, 0.0f), cmax);
    b = fminf(fmaxf(b, 0.0f), cmax);
    const f2p y = add2_rd(pk2(a, b), splat2(8388608.0f));
    fi = sub2(y, splat2(8388608.0f));
    float ya, yb;
    upk2(y, ya, yb);
    i0 = __float_as_int(ya) - 0x4B000000;
    i1 = __float_as_int(yb) - 0x4B000000;
}

template <bool DEC, bool DEP, bool DIAG, int D2>
__device__ __forceinline__ void push_vector_f2(float2 &q, float2 &p, float2 &x, float2 &y, const float2 &m,
                                               const float2 *s_tab, int nx, const Geo<float> &G, float k1,
                                               float k2, float kd, Thread<float> &th, VecOut<float> &o) {
    const f2p INVH = splat2(G.inv_h);
    f2p Q = pk2(q.x, q.y), P = pk2(p.x, p.y), W = pk2(m.x, m.y);
    f2p QS = DEC ? pk2(x.x, x.y) : 0ull, PS = DEC ? pk2(y.x, y.y) : 0ull;
    // gather at the old position: phi_h' and phi_h'' of the element
    int i0, i1;
    f2p FI;
    elem2(mul2(Q, INVH), G.cmax, i0, i1, FI);
    const float2 t0 = s_tab[i0], t1 = s_tab[i1];
    f2p D1 = pk2(t0.x, t1.x);
    f2p D2v = pk2(t0.y, t1.y);
    if (D2 == SWPIC_D2_P2) {
        // P2: phi_h' = a + beta (1 - 2 xi) and phi_h'' = -2 beta / h on the element
        const f2p XI = fma2(Q, splat2(G.inv_h_lo), fma2(Q, INVH, sub2(splat2(0.0f), FI)));
        const f2p BETA = D2v;
        D1 = fma2(BETA, sub2(splat2(1.0f), mul2(splat2(2.0f), XI)), D1);
        if (DEC) D2v = mul2(splat2(-2.0f * G.inv_h), BETA);
    }
    if (DEC && D2 == SWPIC_D2_NODAL) {
        // xi = Q nx/L - i with the low part of nx/L added back; phi'' linear in xi
        const f2p XI = fma2(Q, splat2(G.inv_h_lo), fma2(Q, INVH, sub2(splat2(0.0f), FI)));
        const float g0 = s_tab[i0 + 1 == nx ? 0 : i0 + 1].y, g1 = s_tab[i1 + 1 == nx ? 0 : i1 + 1].y;
        D2v = fma2(XI, sub2(pk2(g0, g1), D2v), D2v);
    }
    // closing half-kick of the previous step
    P = fma2(splat2(-k1), D1, P);
    if (DEC) QS = fma2(mul2(splat2(k1), PS), D2v, QS);
    if (DIAG) {
        const f2p DM = DEC ? fma2(W, P, QS) : mul2(W, P);
        const f2p WP = mul2(mul2(splat2(0.5f), W), P);
        const f2p DK = DEC ? fma2(WP, P, mul2(QS, P)) : mul2(WP, P);
        float a, b;
        upk2(DM, a, b);
        const float vm = a + b;
        upk2(DK, a, b);
        const float vk = a + b;
        th.mom.add(vm);
        th.kin.add(vk);
    }
    // opening half-kick of the next step
    P = fma2(splat2(-k2), D1, P);
    if (DEC) QS = fma2(mul2(splat2(k2), PS), D2v, QS);
    // drift, with the periodic wrap of each half (drift_wrap) when it leaves [0, L)
    const f2p Q0 = Q;
    Q = fma2(splat2(kd), P, Q);
    {
        float a, b, qa, qb, pa, pb;
        upk2(Q, a, b);
        // 0 <= q < L exactly  <=>  bits(q) < bits(Ltop) compared as unsigned (a
        // negative q has the sign bit set; Ltop is fl32(L), or the next float
        // above it when L lies above fl32(L))
        const float Ltop = (G.L_lo > 0.0f) ? __int_as_float(__float_as_int(G.L) + 1) : G.L;
        const unsigned lt = __float_as_uint(Ltop);
        if (__float_as_uint(a) >= lt || __float_as_uint(b) >= lt) {
            upk2(Q0, qa, qb);
            upk2(P, pa, pb);
            if (__float_as_uint(a) >= lt) a = drift_wrap(qa, pa, kd, G);
            if (__float_as_uint(b) >= lt) b = drift_wrap(qb, pb, kd, G);
            Q = pk2(a, b);
        }
    }
    if (DEC) PS = fma2(splat2(-kd), QS, PS);
    if (DEP) {
        f2p FK;
        elem2(mul2(Q, INVH), G.cmax, o.key[0], o.key[1], FK);
        const f2p XI = fma2(Q, splat2(G.inv_h_lo), fma2(Q, INVH, sub2(splat2(0.0f), FK)));
        f2p W0, W1;
        if (DEC) {
            const f2p DQ = mul2(PS, INVH);
            W0 = fma2(W, sub2(splat2(1.0f), XI), DQ);
            W1 = fma2(W, XI, sub2(splat2(0.0f), DQ));
        } else {
            W0 = mul2(W, sub2(splat2(1.0f), XI));
            W1 = mul2(W, XI);
        }
        upk2(W0, o.w0[0], o.w0[1]);
        upk2(W1, o.w1[0], o.w1[1]);
        if (D2 == SWPIC_D2_P2) {
            // the midpoint load psi* N_m(xi) - p* N_m'(xi), N_m = 4 xi (1 - xi)
            f2p WM = mul2(mul2(mul2(splat2(4.0f), W), XI), sub2(splat2(1.0f), XI));
            if (DEC)
                WM = fma2(mul2(sub2(splat2(0.0f), PS), INVH), sub2(splat2(4.0f), mul2(splat2(8.0f), XI)), WM);
            upk2(WM, o.wm[0], o.wm[1]);
        }
    }
    upk2(Q, q.x, q.y);
    upk2(P, p.x, p.y);
    if (DEC) {
        upk2(QS, x.x, x.y);
        upk2(PS, y.x, y.y);
    }
}

// Push the particles of one 16-byte vector in place; their diagnostics go to
// th (one compensated add per vector), their deposit slots to o.
template <typename T, bool DEC, bool DEP, bool DIAG, int D2>
__device__ __forceinline__ void push_vector(typename Vec16<T>::type &q, typename Vec16<T>::type &p,
                                            typename Vec16<T>::type &x, typename Vec16<T>::type &y,
                                            const typename Vec16<T>::type &m,
                                            const typename Vec2<T>::type *s_tab, int nx, const Geo<T> &G,
                                            T k1, T k2, T kd, Thread<T> &th, VecOut<T> &o) {
    if constexpr (sizeof(T) == 4) {
        // FP32: both particles of the vector in packed arithmetic
        push_vector_f2<DEC, DEP, DIAG, D2>(q, p, x, y, m, s_tab, nx, G, k1, k2, kd, th, o);
        return;
    }
    constexpr int VW = Vec16<T>::n;
    T *Q = reinterpret_cast<T *>(&q), *P = reinterpret_cast<T *>(&p);
    T *X = reinterpret_cast<T *>(&x), *Y = reinterpret_cast<T *>(&y);
    const T *M = reinterpret_cast<const T *>(&m);
    T vm = T(0), vk = T(0);
#pragma unroll
    for (int l = 0; l < VW; ++l) {
        T qs = DEC ? X[l] : T(0), ps = DEC ? Y[l] : T(0);
        T dm = T(0), dk = T(0);
        push_one<T, DEC, DEP, DIAG, D2>(Q[l], P[l], qs, ps, M[l], s_tab, nx, G, k1, k2, kd, dm, dk,
                                        o.key[l], o.w0[l], o.w1[l], o.wm[l]);
        if (DIAG) { vm += dm; vk += dk; }
        if (DEC) { X[l] = qs; Y[l] = ps; }
    }
    if (DIAG) { th.mom.add(vm); th.kin.add(vk); }
}


// Deposit one vector per lane.  Runs of equal elements inside the vector are
// summed in registers first (fixed order); the first run of every lane joins
// one warp-aggregated deposit (so a sorted or cold plasma, where whole
// vectors share an element, costs one shared atomic per segment of lanes and
// node, and with P2 one more for the element midpoint), later runs go to the
// mesh directly.  All lanes of the warp must call this.
template <typename T, int MODE, bool P2>
__device__ __forceinline__ void deposit_vector(const VecOut<T> &o, void *s_mesh, void *s_mesh_m, T scale,
                                               int32_t *err) {
    constexpr int VW = Vec16<T>::n;
    const int k0 = o.key[0];
    T s0 = o.w0[0], s1 = o.w1[0], sm = P2 ? o.wm[0] : T(0);
    bool first = true;
    int kr = -1;
    T r0 = T(0), r1 = T(0), rm = T(0);
#pragma unroll
    for (int l = 1; l < VW; ++l) {
        const int k = o.key[l];
        if (first && k == k0) {
            s0 += o.w0[l];
            s1 += o.w1[l];
            if (P2) sm += o.wm[l];
        } else {
            first = false;
            if (k == kr) {
                r0 += o.w0[l];
                r1 += o.w1[l];
                if (P2) rm += o.wm[l];
            } else {
                if (kr >= 0) {
                    mesh_add<T, MODE>(kr, r0, r1, s_mesh, scale, err);
                    if (P2) mesh_m_add<T, MODE>(kr, rm, s_mesh_m, scale, err);
                }
                kr = k;
                r0 = o.w0[l];
                r1 = o.w1[l];
                if (P2) rm = o.wm[l];
            }
        }
    }
    if (kr >= 0) {
        mesh_add<T, MODE>(kr, r0, r1, s_mesh, scale, err);
        if (P2) mesh_m_add<T, MODE>(kr, rm, s_mesh_m, scale, err);
    }
    warp_deposit<T, MODE, P2>(k0, s0, s1, s_mesh, scale, err, sm, s_mesh_m);
}

// One warp turn (both particle streams) covers 512 bytes of every array:
// 64 two-particle FP32 vectors or 32 FP64 vectors.
constexpr int kTurnBytes = 512;
template <typename T> struct TurnVecs {
    static constexpr int n = kTurnBytes / (int)sizeof(typename Vec16<T>::type);
};

template <typename T, bool DEC, int MODE, bool DEP, bool DIAG, int D2>
__device__ void process_segment(const PassArgs &a, const RunDev &R, int64_t s, int64_t e,
                                const typename Vec2<T>::type *s_tab, void *s_mesh, void *s_mesh_m, Thread<T> &th,
                                int32_t *err) {
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::n;
    const Geo<T> G = geo_of(R, T());
    const int nx = R.nx;
    T k1, k2, kd;
    step_coefficients(a, R, k1, k2, kd);
    const T scale = opaque((T)R.fx_scale);      // a power of two: exact in either type
    const bool wpsi = (a.flags & PASS_WRITE_PSI) != 0;
    // a half-kick without drift (the closing half-kick of a step) leaves Q and
    // p* as they are and does not write them back; a pass from the sort buffer
    // writes every array, and a pass with neither kick nor drift (the field of
    // a refreshed state) stores the wrapped positions
    const bool wdrift = a.cd != 0.0 || wpsi || (a.c1 == 0.0 && a.c2 == 0.0);
    const T *Qi = reinterpret_cast<const T *>(a.Qi), *Pi = reinterpret_cast<const T *>(a.Pi);
    const T *qsi = reinterpret_cast<const T *>(a.qsi), *psi = reinterpret_cast<const T *>(a.psi_i);
    const T *wi = reinterpret_cast<const T *>(a.wi);
    T *Qo = reinterpret_cast<T *>(a.Qo), *Po = reinterpret_cast<T *>(a.Po);
    T *qso = reinterpret_cast<T *>(a.qso), *pso = reinterpret_cast<T *>(a.pso);
    T *wo = reinterpret_cast<T *>(a.wo);

    // unaligned head / tail (less than 16 bytes of particles each): one particle per
    // thread, shared-memory atomics without aggregation
    auto scalar = [&](int64_t k) {
        T Q = Qi[k], P = Pi[k], w = wi[k];
        T qs = DEC ? qsi[k] : T(0), ps = DEC ? psi[k] : T(0);
        int key = -1;
        T w0 = T(0), w1 = T(0), wm = T(0), dm = T(0), dk = T(0);
        push_one<T, DEC, DEP, DIAG, D2>(Q, P, qs, ps, w, s_tab, nx, G, k1, k2, kd, dm, dk, key, w0, w1, wm);
        if (DIAG) { th.mom.add(dm); th.kin.add(dk); }
        if (wdrift) Qo[k] = Q;
        Po[k] = P;
        if (DEC) {
            qso[k] = qs;
            if (wdrift) pso[k] = ps;
        }
        if (wpsi) wo[k] = w;
        if (DEP) mesh_add<T, MODE>(key, w0, w1, s_mesh, scale, err);
        if (DEP && D2 == SWPIC_D2_P2) mesh_m_add<T, MODE>(key, wm, s_mesh_m, scale, err);
    };

    constexpr int A = AlignOf<T>::n;
    const int64_t vs = (s + A - 1) / A * A;
    const int64_t ve = e / A * A;
    if (vs >= ve) {
        for (int64_t k = s + threadIdx.x; k < e; k += blockDim.x) scalar(k);
        return;
    }
    for (int64_t k = s + threadIdx.x; k < vs; k += blockDim.x) scalar(k);
    const int64_t v0 = vs / VW, v1 = ve / VW;
    constexpr int U = TurnVecs<T>::n / 32;
    const int lane = threadIdx.x & 31;
    const int64_t step = (int64_t)U * blockDim.x;                // vectors per CTA iteration
    // warp w takes the N = TurnVecs<T>::n consecutive vectors v0 + k step + N w + [0, N)
    // in its k-th turn, lane l the vectors l, 32 + l, ... of them; the trip count is
    // warp-uniform and out-of-range lanes carry empty deposit slots.  A thread walks
    // its vectors in that order one at a time, and loads the next one before it
    // pushes the current one, so a vector's loads are always in flight.
    const int64_t vb0 = v0 + (int64_t)U * (threadIdx.x - lane);
    const int64_t nturn = (vb0 < v1) ? (v1 - vb0 + step - 1) / step : 0;
    const int64_t total = nturn * U;
    struct Vin { V q, p, x, y, m; };
    auto vec_of = [&](int64_t t) { return vb0 + (t / U) * step + 32 * (t % U) + lane; };
    auto load = [&](int64_t vv, Vin &c) {
        c.q = reinterpret_cast<const V *>(Qi)[vv];
        c.p = reinterpret_cast<const V *>(Pi)[vv];
        c.m = reinterpret_cast<const V *>(wi)[vv];
        if (DEC) {
            c.x = reinterpret_cast<const V *>(qsi)[vv];
            c.y = reinterpret_cast<const V *>(psi)[vv];
        }
    };
    Vin cur;
    bool cur_ok = total > 0 && vec_of(0) < v1;
    if (cur_ok) load(vec_of(0), cur);
    for (int64_t t = 0; t < total; ++t) {
        Vin nxt;
        const bool nxt_ok = t + 1 < total && vec_of(t + 1) < v1;
        if (nxt_ok) load(vec_of(t + 1), nxt);
        VecOut<T> o;
        if (cur_ok) {
            push_vector<T, DEC, DEP, DIAG, D2>(cur.q, cur.p, cur.x, cur.y, cur.m, s_tab, nx, G, k1, k2, kd, th, o);
            const int64_t vv = vec_of(t);
            if (wdrift) reinterpret_cast<V *>(Qo)[vv] = cur.q;
            reinterpret_cast<V *>(Po)[vv] = cur.p;
            if (DEC) {
                reinterpret_cast<V *>(qso)[vv] = cur.x;
                if (wdrift) reinterpret_cast<V *>(pso)[vv] = cur.y;
            }
            if (wpsi) reinterpret_cast<V *>(wo)[vv] = cur.m;
        } else {
            o.clear();
        }
        if (DEP) deposit_vector<T, MODE, D2 == SWPIC_D2_P2>(o, s_mesh, s_mesh_m, scale, err);
        cur = nxt;
        cur_ok = nxt_ok;
    }
    for (int64_t k = ve + threadIdx.x; k < e; k += blockDim.x) scalar(k);
}

// ---------------------------------------------------------------------------
// Bulk-copy (TMA) staged particle stream
// ---------------------------------------------------------------------------
// Every warp streams its own particles: in its k-th turn warp w handles the
// N = TurnVecs<T>::n consecutive vectors v0 + k (N/32) blockDim.x + N w
// + [0, N) of every array, lane l the vectors l, 32 + l, ... of them
// (the vectors the register-load loop gives its lanes, in the same order).
// Lane 0 copies them global -> shared with cp.async.bulk (one copy of at most
// N vectors per array, completion counted in bytes on the warp's
// mbarrier of that stage), S turns ahead; as soon as the lanes have read a
// stage into registers (__syncwarp) it is refilled with the turn S places
// further on, while the lanes push, store (plain stores) and deposit.  Warps
// never wait for each other, so one warp's shared atomics overlap another's
// arithmetic, and the copy engine keeps S turns per warp in flight without
// holding registers.
//
// Every wait is bounded (PassArgs::wait_limit_ns of wall time, 1 s unless a
// test shortens it); a wait that runs out sets kErrTimeout in the run's flag
// word, and the warp stops, waits (again bounded) for its copies in flight,
// and the CTA leaves the kernel after the segment.

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// true when the phase with this parity completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst_smem)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

template <typename T, int MODE>
__host__ __device__ __forceinline__ size_t mesh_bytes(int max_nx) {
    return (size_t)(max_nx + 1) * (MODE == SWPIC_DEPOSIT_ATOMIC ? sizeof(T) : sizeof(unsigned long long));
}
// node mesh plus, for P2, the per-element midpoint mesh; at least 8 bytes per
// node, since a pass that solves its field at its start uses the area as the
// solve's int64 scratch before it clears the mesh
template <typename T, int MODE, int D2>
__host__ __device__ __forceinline__ size_t mesh_bytes_all(int max_nx) {
    const size_t m = mesh_bytes<T, MODE>(max_nx) +
                     (D2 == SWPIC_D2_P2 ? (size_t)max_nx * (MODE == SWPIC_DEPOSIT_ATOMIC ? sizeof(T)
                                                                                   : sizeof(unsigned long long))
                                        : 0);
    const size_t scratch = (size_t)max_nx * sizeof(long long);
    return m > scratch ? m : scratch;
}

// Shared-memory layout of the pass: table | mesh | (bulk stream) mbarriers | stages.
__host__ __device__ __forceinline__ size_t round128(size_t x) { return (x + 127) / 128 * 128; }
__host__ __device__ __forceinline__ size_t bar_offset(size_t tab_bytes, size_t mesh_b) {
    return round128(tab_bytes + mesh_b);
}
__host__ __device__ __forceinline__ size_t stage_area_offset(size_t tab_bytes, size_t mesh_b, int nwarps, int S) {
    return bar_offset(tab_bytes, mesh_b) + round128((size_t)nwarps * S * sizeof(uint64_t));
}

// Pipeline bookkeeping of one warp; seq counts the warp's turns over the CTA's
// lifetime, so the stage of a turn is seq % S and its mbarrier parity (seq / S) & 1.
struct Pipe {
    unsigned char *base;     // this warp's S stages of n_arr x one turn (kTurnBytes per array)
    uint64_t *bar;           // this warp's S mbarriers
    int S;
    uint32_t seq;
    int pre;                 // turns of the next segment already issued (prefetched)
};

template <typename T, bool DEC, int MODE, bool DEP, bool DIAG, int D2>
__device__ bool process_segment_bulk(const PassArgs &a, const RunDev &R, int64_t s, int64_t e,
                                     const typename Vec2<T>::type *s_tab, void *s_mesh, void *s_mesh_m, Thread<T> &th,
                                     int32_t *err, Pipe &pp, int *s_abort, bool prefetch_only = false) {
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::n;
    constexpr int NA = DEC ? 5 : 3;                       // Q, P, w [, q*, p*]
    constexpr uint32_t ARR = TurnVecs<T>::n * sizeof(V);       // bytes per array in a stage
    const unsigned full = 0xffffffffu;
    const Geo<T> G = geo_of(R, T());
    const int nx = R.nx;
    T k1, k2, kd;
    step_coefficients(a, R, k1, k2, kd);
    const T scale = opaque((T)R.fx_scale);      // a power of two: exact in either type
    const bool wpsi = (a.flags & PASS_WRITE_PSI) != 0;
    // a half-kick without drift (the closing half-kick of a step) leaves Q and
    // p* as they are and does not write them back; a pass from the sort buffer
    // writes every array, and a pass with neither kick nor drift (the field of
    // a refreshed state) stores the wrapped positions
    const bool wdrift = a.cd != 0.0 || wpsi || (a.c1 == 0.0 && a.c2 == 0.0);
    const T *Qi = reinterpret_cast<const T *>(a.Qi), *Pi = reinterpret_cast<const T *>(a.Pi);
    const T *qsi = reinterpret_cast<const T *>(a.qsi), *psi = reinterpret_cast<const T *>(a.psi_i);
    const T *wi = reinterpret_cast<const T *>(a.wi);
    T *Qo = reinterpret_cast<T *>(a.Qo), *Po = reinterpret_cast<T *>(a.Po);
    T *qso = reinterpret_cast<T *>(a.qso), *pso = reinterpret_cast<T *>(a.pso);
    T *wo = reinterpret_cast<T *>(a.wo);
    const T *src[5] = {Qi, Pi, wi, qsi, psi};

    auto scalar = [&](int64_t k) {
        T Q = Qi[k], P = Pi[k], w = wi[k];
        T qs = DEC ? qsi[k] : T(0), ps = DEC ? psi[k] : T(0);
        int key = -1;
        T w0 = T(0), w1 = T(0), wm = T(0), dm = T(0), dk = T(0);
        push_one<T, DEC, DEP, DIAG, D2>(Q, P, qs, ps, w, s_tab, nx, G, k1, k2, kd, dm, dk, key, w0, w1, wm);
        if (DIAG) { th.mom.add(dm); th.kin.add(dk); }
        if (wdrift) Qo[k] = Q;
        Po[k] = P;
        if (DEC) {
            qso[k] = qs;
            if (wdrift) pso[k] = ps;
        }
        if (wpsi) wo[k] = w;
        if (DEP) mesh_add<T, MODE>(key, w0, w1, s_mesh, scale, err);
        if (DEP && D2 == SWPIC_D2_P2) mesh_m_add<T, MODE>(key, wm, s_mesh_m, scale, err);
    };

    constexpr int A = AlignOf<T>::n;
    const int64_t vs = (s + A - 1) / A * A;
    const int64_t ve = e / A * A;
    if (vs >= ve) {
        if (prefetch_only) return true;
        for (int64_t k = s + threadIdx.x; k < e; k += blockDim.x) scalar(k);
        return true;
    }
    if (!prefetch_only)
        for (int64_t k = s + threadIdx.x; k < vs; k += blockDim.x) scalar(k);

    const int64_t v0 = vs / VW, v1 = ve / VW;
    const int lane = threadIdx.x & 31;
    constexpr int U = TurnVecs<T>::n / 32;                      // vectors per lane and turn
    const int64_t wbase = v0 + (int64_t)U * (threadIdx.x - lane);   // first vector of this warp's turn 0
    const int64_t stride = (int64_t)U * blockDim.x;
    const int nturn = wbase < v1 ? (int)((v1 - wbase + stride - 1) / stride) : 0;
    const int S = pp.S;

    auto turn_vecs = [&](int k) -> int { return (int)min((int64_t)TurnVecs<T>::n, v1 - (wbase + (int64_t)k * stride)); };
    // test hook: the chosen warp leaves the stage of its first turn unarmed (no
    // arrival, no copy), so that stage's wait can only run out
    const bool stall = a.stall_warp >= 0 && pp.seq == 0 &&
                       (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) == a.stall_warp;
    auto issue = [&](int k) {            // lane 0 only
        const uint32_t q = pp.seq + (uint32_t)k;
        if (stall && q == 0) return;
        unsigned char *st = pp.base + (size_t)(q % S) * NA * ARR;
        uint64_t *bar = pp.bar + (q % S);
        const uint32_t nb = (uint32_t)turn_vecs(k) * (uint32_t)sizeof(V);
        mbar_arrive_expect_tx(bar, nb * NA);
        const int64_t gv = wbase + (int64_t)k * stride;
#pragma unroll
        for (int j = 0; j < NA; ++j) bulk_load(st + j * ARR, reinterpret_cast<const V *>(src[j]) + gv, nb, bar);
    };

    if (prefetch_only) {
        // the first turns only, issued before the CTA stages its table and
        // clears its mesh, so their latency overlaps that work
        if (lane == 0)
            for (int k = 0; k < S && k < nturn; ++k) issue(k);
        pp.pre = min(S, nturn);
        return true;
    }
    if (lane == 0)
        for (int k = pp.pre; k < S && k < nturn; ++k) issue(k);
    pp.pre = 0;
    int issued = min(S, nturn);
    bool ok = true;
    int k = 0;
    for (; k < nturn; ++k) {
        const uint32_t q = pp.seq + (uint32_t)k;
        const V *sv = reinterpret_cast<const V *>(pp.base + (size_t)(q % S) * NA * ARR);
        const bool arrived = mbar_wait_bounded(pp.bar + (q % S), (q / S) & 1u, a.wait_limit_ns);
        if (!__all_sync(full, arrived)) {
            if (lane == 0) { atomicOr(err, kErrTimeout); *s_abort = 1; }
            ok = false;
            break;
        }
        const int nv = turn_vecs(k);
        bool have[U];
        V qv[U], pv[U], mv[U], xv[U], yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = 32 * u + lane;
            have[u] = t < nv;
            if (have[u]) {
                qv[u] = sv[t];
                pv[u] = sv[TurnVecs<T>::n + t];
                mv[u] = sv[2 * TurnVecs<T>::n + t];
                if (DEC) { xv[u] = sv[3 * TurnVecs<T>::n + t]; yv[u] = sv[4 * TurnVecs<T>::n + t]; }
            }
        }
        __syncwarp();                    // the stage has been read: refill it
        if (k + S < nturn) {
            if (lane == 0) issue(k + S);
            ++issued;
        }
        // push both vectors of the turn first (their table loads and arithmetic
        // interleave), then store them, then deposit them
        VecOut<T> o[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (have[u]) {
                push_vector<T, DEC, DEP, DIAG, D2>(qv[u], pv[u], xv[u], yv[u], mv[u], s_tab, nx, G, k1, k2, kd,
                                                   th, o[u]);
            } else {
                o[u].clear();
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (have[u]) {
                const int64_t vv = wbase + (int64_t)k * stride + 32 * u + lane;
                if (wdrift) reinterpret_cast<V *>(Qo)[vv] = qv[u];
                reinterpret_cast<V *>(Po)[vv] = pv[u];
                if (DEC) {
                    reinterpret_cast<V *>(qso)[vv] = xv[u];
                    if (wdrift) reinterpret_cast<V *>(pso)[vv] = yv[u];
                }
                if (wpsi) reinterpret_cast<V *>(wo)[vv] = mv[u];
            }
        }
        if (DEP) {
#pragma unroll
            for (int u = 0; u < U; ++u) deposit_vector<T, MODE, D2 == SWPIC_D2_P2>(o[u], s_mesh, s_mesh_m, scale, err);
        }
    }
    if (!ok && lane == 0) {
        // drain: wait (bounded) for every copy still in flight into this warp's stages
        for (int u = k; u < issued; ++u) {
            const uint32_t qq = pp.seq + (uint32_t)u;
            mbar_wait_bounded(pp.bar + (qq % S), (qq / S) & 1u, a.wait_limit_ns);
        }
    }
    pp.seq += (uint32_t)issued;
    if (ok)         // same per-thread order as the register path: head, vectors, tail
        for (int64_t kk = ve + threadIdx.x; kk < e; kk += blockDim.x) scalar(kk);
    __syncthreads();
    return *s_abort == 0;
}

template <typename T, bool P2>
__device__ void finish_run(const PassArgs &a, const RunDev &R, int r, unsigned char *smem) {
    const uint32_t fl = a.flags;
    const bool diag = (fl & PASS_DIAG) != 0;
    DiagPre pre;
    if (diag && threadIdx.x == 0) diag_preload(a, r, pre);
    if (fl & PASS_SOLVE)
        solve_run<T, P2>(a, R, r, reinterpret_cast<long long *>(smem), a.acc + R.mesh_off, a.acc_m + R.mesh_off,
                         nullptr, true, true);
    if (threadIdx.x == 0) {
        if (diag) diag_write(a, R, r, pre);
        if (fl & PASS_COUNT_STEP) a.steps[r] += 1;
        a.run_done[r] = 0ull;
    }
}

template <typename T, bool DEC, int MODE, bool DEP, bool DIAG, int D2>
__device__ __forceinline__ void pass_body(const PassArgs &a) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_last, s_abort;
    __shared__ double s_red[64];
    T2 *s_tab = reinterpret_cast<T2 *>(smem);
    void *s_mesh = smem + (size_t)a.max_nx * sizeof(T2);
    // P2: the per-element midpoint mesh follows the node mesh (same element type)
    void *s_mesh_m = reinterpret_cast<unsigned char *>(s_mesh) + mesh_bytes<T, MODE>(a.max_nx);
    const bool bulk = a.stages >= 2;
    Pipe pp;
    {
        const size_t tb = (size_t)a.max_nx * sizeof(T2), mb = mesh_bytes_all<T, MODE, D2>(a.max_nx);
        const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
        constexpr size_t stage_bytes = (DEC ? 5 : 3) * TurnVecs<T>::n * sizeof(typename Vec16<T>::type);
        pp.S = a.stages;
        pp.seq = 0;
        pp.pre = 0;
        pp.bar = reinterpret_cast<uint64_t *>(smem + bar_offset(tb, mb)) + (size_t)w * pp.S;
        pp.base = smem + stage_area_offset(tb, mb, nw, pp.S) + (size_t)w * pp.S * stage_bytes;
    }
    if (threadIdx.x == 0) s_abort = 0;
    if (bulk && (threadIdx.x & 31) == 0) {
        for (int k = 0; k < pp.S; ++k) mbar_init(pp.bar + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Programmatic dependent launch: this grid may be scheduled while the
    // previous pass is still finishing; wait for that grid to complete (and
    // its writes to be visible) before touching any memory.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t c0 = (int64_t)blockIdx.x * a.chunk;
    const int64_t c1 = min(c0 + a.chunk, a.n_total);
    if (c0 >= c1) return;
    int r = find_run(a.runs, a.n_runs, c0);
    int64_t pos = c0;
    const bool last_work = (a.flags & (PASS_SOLVE | PASS_DIAG | PASS_COUNT_STEP)) != 0;
    if (bulk && a.prefetch && r < a.n_runs) {
        // issue the first segment's first bulk copies now, before the table is
        // staged and the mesh cleared (see process_segment_bulk)
        int rr = r;
        while (rr < a.n_runs && min(c1, run_of(a, rr).p1) <= pos) ++rr;
        if (rr < a.n_runs) {
            const RunDev R0 = run_of(a, rr);
            const T2 *tab0 = reinterpret_cast<const T2 *>(smem);
            Thread<T> th0;
            process_segment_bulk<T, DEC, MODE, DEP, DIAG, D2>(a, R0, pos, min(c1, R0.p1), tab0, s_mesh, s_mesh_m,
                                                              th0, a.err + rr, pp, &s_abort, true);
        }
    }
    while (pos < c1 && r < a.n_runs) {
        const RunDev R = run_of(a, r);
        const int64_t s = pos, e = min(c1, R.p1);
        if (s >= e) { ++r; continue; }
        const int nx = R.nx;
        const bool owner = s == R.p0;             // this CTA holds the run's first particle
        if (DEP && owner && a.acc_clr) {
            // the accumulator that the next depositing pass fills (no pass reads it now)
            for (int j = threadIdx.x; j < nx; j += blockDim.x) a.acc_clr[R.mesh_off + j] = 0ull;
            if (D2 == SWPIC_D2_P2)
                for (int j = threadIdx.x; j < nx; j += blockDim.x) a.acc_m_clr[R.mesh_off + j] = 0ull;
        }
        if (a.flags & PASS_FIELD_ACC) {
            // the field of the deposit the previous pass left, solved by every
            // CTA into its own table (the mesh area is the solve's scratch), so
            // that no pass ends in a one-CTA solve; the first bulk copies of the
            // segment are already in flight
            solve_run<T, D2 == SWPIC_D2_P2>(a, R, r, reinterpret_cast<long long *>(s_mesh), a.acc_src + R.mesh_off,
                                            a.acc_m_src + R.mesh_off, s_tab, owner, true);
            __syncthreads();
        } else {
            const T2 *gtab = reinterpret_cast<const T2 *>(a.table) + R.mesh_off;
            for (int j = threadIdx.x; j < nx; j += blockDim.x) s_tab[j] = gtab[j];
        }
        if (DEP) {
            if (MODE == SWPIC_DEPOSIT_ATOMIC) {
                T *m = reinterpret_cast<T *>(s_mesh);
                for (int j = threadIdx.x; j <= nx; j += blockDim.x) m[j] = T(0);
                if (D2 == SWPIC_D2_P2)
                    for (int j = threadIdx.x; j < nx; j += blockDim.x) reinterpret_cast<T *>(s_mesh_m)[j] = T(0);
            } else {
                unsigned long long *m = reinterpret_cast<unsigned long long *>(s_mesh);
                for (int j = threadIdx.x; j <= nx; j += blockDim.x) m[j] = 0ull;
                if (D2 == SWPIC_D2_P2)
                    for (int j = threadIdx.x; j < nx; j += blockDim.x)
                        reinterpret_cast<unsigned long long *>(s_mesh_m)[j] = 0ull;
            }
        }
        __syncthreads();
        Thread<T> th;
        th.mom = {T(0), T(0)};
        th.kin = {T(0), T(0)};
        if (bulk) {
            if (!process_segment_bulk<T, DEC, MODE, DEP, DIAG, D2>(a, R, s, e, s_tab, s_mesh, s_mesh_m, th, a.err + r,
                                                                  pp, &s_abort))
                return;      // a copy did not arrive: the run's flag says so
        } else {
            process_segment<T, DEC, MODE, DEP, DIAG, D2>(a, R, s, e, s_tab, s_mesh, s_mesh_m, th, a.err + r);
        }
        // every CTA has been scheduled by now: let the next pass launch early
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        if (DIAG) {
            // warp partials of the diagnostic sums first: their FP64 shuffle
            // chain overlaps the flush below
            const double m = warp_sum_d((double)th.mom.s + (double)(-th.mom.c));
            const double k = warp_sum_d((double)th.kin.s + (double)(-th.kin.c));
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            if (lane == 0) { s_red[w] = m; s_red[32 + w] = k; }
        }
        __syncthreads();
        if (DEP) {
            unsigned long long *gacc = a.acc + R.mesh_off;
            for (int j = threadIdx.x; j <= nx; j += blockDim.x) {
                const int node = (j == nx) ? 0 : j;
                if (MODE == SWPIC_DEPOSIT_ATOMIC) {
                    const T v = reinterpret_cast<T *>(s_mesh)[j];
                    if (v != T(0)) atomicAdd(gacc + node, to_fixed(v, (T)R.fx_scale, a.err + r));
                } else {
                    const unsigned long long v = reinterpret_cast<unsigned long long *>(s_mesh)[j];
                    if (v != 0ull) atomicAdd(gacc + node, v);
                }
            }
            if (D2 == SWPIC_D2_P2) {
                unsigned long long *gm = a.acc_m + R.mesh_off;
                for (int j = threadIdx.x; j < nx; j += blockDim.x) {
                    if (MODE == SWPIC_DEPOSIT_ATOMIC) {
                        const T v = reinterpret_cast<T *>(s_mesh_m)[j];
                        if (v != T(0)) atomicAdd(gm + j, to_fixed(v, (T)R.fx_scale, a.err + r));
                    } else {
                        const unsigned long long v = reinterpret_cast<unsigned long long *>(s_mesh_m)[j];
                        if (v != 0ull) atomicAdd(gm + j, v);
                    }
                }
            }
        }
        if (DIAG) {
            if (threadIdx.x == 0) {
                double sm = 0.0, sk = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sm += s_red[q]; sk += s_red[32 + q]; }
                atomicAdd(a.diag_acc + 2 * r, sm);
                atomicAdd(a.diag_acc + 2 * r + 1, sk);
            }
        }
        if (last_work) {
            // every thread's flush happens before the barrier; thread 0's fence
            // then orders all of them before its count (release, cumulative)
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned long long cnt = (unsigned long long)(e - s);
                const unsigned long long prev = atomicAdd(a.run_done + r, cnt);
                s_last = (prev + cnt == (unsigned long long)(R.p1 - R.p0)) ? 1 : 0;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                finish_run<T, D2 == SWPIC_D2_P2>(a, R, r, smem);
            }
        }
        __syncthreads();
        pos = e;
        ++r;
        while (r < a.n_runs && run_of(a, r).p1 <= pos) ++r;
    }
}

// FP32 state: at most 80 registers, so 24 warps (e.g. 3 x 256 or 6 x 128
// threads) fit an SM; FP64 state: the push needs the full 128 (<= 512 threads).
template <bool DEC, int MODE, bool DEP, bool DIAG, int D2>
__global__ void __maxnreg__(80) k_pass32(PassArgs a) {
    pass_body<float, DEC, MODE, DEP, DIAG, D2>(a);
}
template <bool DEC, int MODE, bool DEP, bool DIAG, int D2>
__global__ void __launch_bounds__(512) k_pass64(PassArgs a) {
    pass_body<double, DEC, MODE, DEP, DIAG, D2>(a);
}
template <typename T, bool DEC, int MODE, bool DEP, bool DIAG, int D2> struct PassKernel;
template <bool DEC, int MODE, bool DEP, bool DIAG, int D2>
struct PassKernel<float, DEC, MODE, DEP, DIAG, D2> {
    static constexpr auto fn = k_pass32<DEC, MODE, DEP, DIAG, D2>;
};
template <bool DEC, int MODE, bool DEP, bool DIAG, int D2>
struct PassKernel<double, DEC, MODE, DEP, DIAG, D2> {
    static constexpr auto fn = k_pass64<DEC, MODE, DEP, DIAG, D2>;
};

// Launch the pass variant for the pass flags (one kernel per flag combination).
template <typename T, bool DEC, int MODE>
inline cudaError_t launch_pass_t(const PassArgs &a, int grid, int tpb, size_t smem, cudaStream_t s) {
    const bool dep = (a.flags & PASS_DEPOSIT) != 0, diag = (a.flags & PASS_DIAG) != 0;
    const bool nodal = a.d2_mode == SWPIC_D2_NODAL;
#define SWPIC_LAUNCH(DEP, DIAG, D2)                                                               \
    do {                                                                                          \
        auto kern = PassKernel<T, DEC, MODE, DEP, DIAG, D2>::fn;                                  \
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                               (int)smem);                                        \
        if (err != cudaSuccess) return err;                                                       \
        cudaLaunchConfig_t cfg = {};                                                              \
        cudaLaunchAttribute attr[1];                                                              \
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                          \
        attr[0].val.programmaticStreamSerializationAllowed = 1;                                   \
        cfg.gridDim = dim3(grid);                                                                 \
        cfg.blockDim = dim3(tpb);                                                                 \
        cfg.dynamicSmemBytes = smem;                                                              \
        cfg.stream = s;                                                                           \
        cfg.attrs = attr;                                                                         \
        cfg.numAttrs = 1;                                                                         \
        return cudaLaunchKernelEx(&cfg, kern, a);                                                 \
    } while (0)
    if (a.d2_mode == SWPIC_D2_P2) {
        if (dep && diag) SWPIC_LAUNCH(true, true, SWPIC_D2_P2);
        if (dep) SWPIC_LAUNCH(true, false, SWPIC_D2_P2);
        if (diag) SWPIC_LAUNCH(false, true, SWPIC_D2_P2);
        SWPIC_LAUNCH(false, false, SWPIC_D2_P2);
    } else if (nodal) {
        if (dep && diag) SWPIC_LAUNCH(true, true, SWPIC_D2_NODAL);
        if (dep) SWPIC_LAUNCH(true, false, SWPIC_D2_NODAL);
        if (diag) SWPIC_LAUNCH(false, true, SWPIC_D2_NODAL);
        SWPIC_LAUNCH(false, false, SWPIC_D2_NODAL);
    } else {
        if (dep && diag) SWPIC_LAUNCH(true, true, SWPIC_D2_LUMPED);
        if (dep) SWPIC_LAUNCH(true, false, SWPIC_D2_LUMPED);
        if (diag) SWPIC_LAUNCH(false, true, SWPIC_D2_LUMPED);
        SWPIC_LAUNCH(false, false, SWPIC_D2_LUMPED);
    }
#undef SWPIC_LAUNCH
}

}  // namespace swpic
