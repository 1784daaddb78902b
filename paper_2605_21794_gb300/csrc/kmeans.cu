// Decorated particles from marker particles (Sec. 4.1-4.2 "Initialization",
// Alg. lumping_procedure, Eqs. psi-star and moment-def with the periodic c of
// the T^d subsection), on the GPU.
//
// k-means (Lloyd) in (q, p) with the minimum-image q difference:
//   assignment: every marker takes the nearest center; the decision is taken
//     in FP32 (dq = Qm - cq folded once into [-L/2, L/2), dp = Pm - cp,
//     d2 = dq*dq + dp*dp, each operation rounded; this file is compiled
//     without contraction), ties to the smaller cluster index;
//   update: psi-weighted member means, q unwrapped about the current center
//     and wrapped into [0, L); an empty cluster keeps its center.
// The member sums are exact: every term is a 64-bit fixed-point integer (a
// power-of-two unit per quantity, from the total weight, L and max |P|) added
// with integer atomics, so the means do not depend on the order of the atomics.
// Lumping: per non-empty cluster (in cluster order) psi* = sum psi; (Q, P) =
// the member nearest to the weighted mean (FP32 decision, ties to the smaller
// marker index, one 64-bit atomicMin of (d2 bits, index)); p* = sum psi (L/2pi)
// sin(2pi (Q - Qm)/L), q* = -sum psi (P - Pm) (FP64 atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "swpic_internal.cuh"

namespace swpic {
namespace {

constexpr int kCenterTile = 2048;   // centers staged in shared memory per pass over K
constexpr int kFixedBitsKm = 60;    // a sum bound maps to 2^60 units

__device__ __forceinline__ float fold_f(float d, float L, float half) {
    if (d >= half) return d - L;
    if (d < -half) return d + L;
    return d;
}
__device__ __forceinline__ double fold_d(double d, double L) {
    if (d >= 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}
// periodic wrap into [0, L); a value that rounds up to L maps to 0
__device__ __forceinline__ double wrap_d(double Q, double L) {
    double w = Q - L * floor(Q / L);
    if (w >= L) w -= L;
    if (w < 0.0) w += L;
    return w;
}

// nearest center of every marker
__global__ void k_km_assign(const double *Qm, const double *Pm, int64_t M, const double *cq,
                            const double *cp, int K, double L, int32_t *assign) {
    __shared__ float s_q[kCenterTile], s_p[kCenterTile];
    const float Lf = (float)L, half = (float)(0.5 * L);
    const int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = A < M;
    const float qf = live ? (float)Qm[A] : 0.0f, pf = live ? (float)Pm[A] : 0.0f;
    float best = INFINITY;
    int bi = 0;
    for (int k0 = 0; k0 < K; k0 += kCenterTile) {
        const int nk = min(kCenterTile, K - k0);
        __syncthreads();
        for (int j = threadIdx.x; j < nk; j += blockDim.x) {
            s_q[j] = (float)cq[k0 + j];
            s_p[j] = (float)cp[k0 + j];
        }
        __syncthreads();
        for (int j = 0; j < nk; ++j) {
            const float dq = fold_f(qf - s_q[j], Lf, half);
            const float dp = pf - s_p[j];
            const float d2 = dq * dq + dp * dp;
            if (d2 < best) { best = d2; bi = k0 + j; }
        }
    }
    if (live) assign[A] = bi;
}

struct Units {
    double w, q, p;        // 2^k of each sum
};

__device__ __forceinline__ unsigned long long fixed(double x, double unit) {
    return (unsigned long long)__double2ll_rn(x * unit);
}

// exact fixed-point member sums: w, w dq (about the center), w P
__global__ void k_km_accum(const double *Qm, const double *Pm, const double *wm, int64_t M,
                           const int32_t *assign, const double *cq, double L, Units u,
                           unsigned long long *sums) {
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M;
         A += (int64_t)gridDim.x * blockDim.x) {
        const int k = assign[A];
        const double w = wm[A];
        atomicAdd(sums + 3 * (int64_t)k, fixed(w, u.w));
        atomicAdd(sums + 3 * (int64_t)k + 1, fixed(w * fold_d(Qm[A] - cq[k], L), u.q));
        atomicAdd(sums + 3 * (int64_t)k + 2, fixed(w * Pm[A], u.p));
    }
}

// means from the sums; centers move to them (update) or the means are kept apart (lumping)
__global__ void k_km_means(const unsigned long long *sums, int K, double L, Units u, const double *cq,
                           const double *cp, double *mq, double *mp, double *wsum) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double sw = (double)(long long)sums[3 * k] / u.w;
    const double sq = (double)(long long)sums[3 * k + 1] / u.q;
    const double sp = (double)(long long)sums[3 * k + 2] / u.p;
    if (wsum) wsum[k] = sw;
    if (sw != 0.0) {
        mq[k] = wrap_d(cq[k] + sq / sw, L);
        mp[k] = sp / sw;
    } else {
        mq[k] = cq[k];
        mp[k] = cp[k];
    }
}

// (d2 bits, marker index) minimum per cluster: the member nearest to the mean
__global__ void k_lump_center(const double *Qm, const double *Pm, int64_t M, const int32_t *assign,
                              const double *mq, const double *mp, double L, unsigned long long *key) {
    const float Lf = (float)L, half = (float)(0.5 * L);
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M;
         A += (int64_t)gridDim.x * blockDim.x) {
        const int k = assign[A];
        const float dq = fold_f((float)Qm[A] - (float)mq[k], Lf, half);
        const float dp = (float)Pm[A] - (float)mp[k];
        const float d2 = dq * dq + dp * dp;
        const unsigned long long kv = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned long long)A;
        atomicMin(key + k, kv);
    }
}

// slot of every non-empty cluster (exclusive scan in cluster order, one CTA)
// and the particle's (Q, P, psi*)
__global__ void k_lump_slots(const unsigned long long *key, const double *wsum, int K, const double *Qm,
                             const double *Pm, int64_t *slot, double *Q, double *P, double *psi,
                             double *qs, double *ps, int64_t *n_out) {
    __shared__ int64_t sh[32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5;
    const int per = (K + nt - 1) / nt;
    const int j0 = min(K, tid * per), j1 = min(K, j0 + per);
    int64_t cnt = 0;
    for (int k = j0; k < j1; ++k) cnt += (key[k] != ~0ull) ? 1 : 0;
    int64_t inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    int64_t base = 0;
    for (int q = 0; q < w; ++q) base += sh[q];
    int64_t s = base + inc - cnt;
    for (int k = j0; k < j1; ++k) {
        if (key[k] == ~0ull) { slot[k] = -1; continue; }
        const int64_t A0 = (int64_t)(key[k] & 0xffffffffull);
        slot[k] = s;
        Q[s] = Qm[A0];
        P[s] = Pm[A0];
        psi[s] = wsum[k];
        qs[s] = 0.0;
        ps[s] = 0.0;
        ++s;
    }
    if (tid == nt - 1) *n_out = s;
}

__global__ void k_lump_moments(const double *Qm, const double *Pm, const double *wm, int64_t M,
                               const int32_t *assign, const int64_t *slot, double L, const double *Q,
                               const double *P, double *qs, double *ps) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M;
         A += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = slot[assign[A]];
        const double w = wm[A];
        atomicAdd(ps + s, w * (L / two_pi) * sin(two_pi * (Q[s] - Qm[A]) / L));
        atomicAdd(qs + s, -w * (P[s] - Pm[A]));
    }
}

// bounds for the fixed-point units: sum w, max |P|
__global__ void k_km_bounds(const double *Pm, const double *wm, int64_t M, double *wsum_total,
                            unsigned long long *pmax_bits) {
    double sw = 0.0;
    double pm = 0.0;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M;
         A += (int64_t)gridDim.x * blockDim.x) {
        sw += fabs(wm[A]);
        pm = fmax(pm, fabs(Pm[A]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(wsum_total, sw);
        atomicMax(pmax_bits, (unsigned long long)__double_as_longlong(pm));   // non-negative: bit order
    }
}

double unit_for(double bound) {
    int k = kFixedBitsKm;
    if (bound > 0.0) k = kFixedBitsKm - (int)std::ceil(std::log2(bound));
    return std::ldexp(1.0, std::max(-1000, std::min(1000, k)));
}

}  // namespace
}  // namespace swpic

using namespace swpic;

extern "C" swpic_status swpic_kmeans_lump(const double *Qm, const double *Pm, const double *wm, int64_t M,
                                          double *cq, double *cp, int32_t K, double L, int32_t n_iter,
                                          int32_t *assign, double *Q, double *P, double *qs, double *ps,
                                          double *psi, int64_t *n_out, swpic_stream stream) {
    if (M < 0 || K < 1 || n_iter < 0 || !(L > 0.0) || !std::isfinite(L) || !n_out) return SWPIC_EINVAL;
    if (M >= (int64_t)1 << 32) return SWPIC_EINVAL;              // marker index packs into 32 bits
    if (M > 0 && (!Qm || !Pm || !wm)) return SWPIC_EINVAL;
    if (!cq || !cp || !Q || !P || !qs || !ps || !psi) return SWPIC_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    *n_out = 0;
    if (M == 0) return SWPIC_OK;
    // work buffers: sums [K][3], keys [K], slots [K], means [K][2], wsum [K], assign (if not given),
    // bounds
    const size_t bytes = sizeof(unsigned long long) * 3 * K + sizeof(unsigned long long) * K +
                         sizeof(int64_t) * K + sizeof(double) * 3 * K + sizeof(int32_t) * (size_t)M +
                         sizeof(double) + sizeof(unsigned long long) + sizeof(int64_t) + 256;
    unsigned char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, bytes, s) != cudaSuccess) return SWPIC_ENOMEM;
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(buf);
    unsigned long long *key = sums + 3 * (size_t)K;
    int64_t *slot = reinterpret_cast<int64_t *>(key + K);
    double *mq = reinterpret_cast<double *>(slot + K), *mp = mq + K, *wsum = mp + K;
    double *wtot = wsum + K;
    unsigned long long *pmax = reinterpret_cast<unsigned long long *>(wtot + 1);
    int64_t *d_n = reinterpret_cast<int64_t *>(pmax + 1);
    int32_t *asg = assign ? assign : reinterpret_cast<int32_t *>(d_n + 1);

    auto fail = [&](swpic_status st) {
        cudaFreeAsync(buf, s);
        return st;
    };
    const int tpb = 256;
    const int gm = (int)std::min<int64_t>((M + tpb - 1) / tpb, 4096);
    const int ga = (int)((M + tpb - 1) / tpb);
    const int gk = (K + tpb - 1) / tpb;
    if (cudaMemsetAsync(wtot, 0, sizeof(double) + sizeof(unsigned long long), s) != cudaSuccess)
        return fail(SWPIC_ECUDA);
    k_km_bounds<<<gm, tpb, 0, s>>>(Pm, wm, M, wtot, pmax);
    double h_b[2];
    if (cudaMemcpyAsync(h_b, wtot, sizeof(h_b), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SWPIC_ECUDA);
    unsigned long long pbits;
    std::memcpy(&pbits, &h_b[1], sizeof(pbits));
    double pmaxv;
    std::memcpy(&pmaxv, &pbits, sizeof(pmaxv));
    if (!std::isfinite(h_b[0]) || !std::isfinite(pmaxv)) return fail(SWPIC_ENUMERIC);
    Units u;
    u.w = unit_for(h_b[0]);
    u.q = unit_for(h_b[0] * 0.5 * L);
    u.p = unit_for(h_b[0] * pmaxv);

    for (int it = 0; it <= n_iter; ++it) {
        k_km_assign<<<ga, tpb, 0, s>>>(Qm, Pm, M, cq, cp, K, L, asg);
        if (it == n_iter) break;
        if (cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * 3 * K, s) != cudaSuccess)
            return fail(SWPIC_ECUDA);
        k_km_accum<<<gm, tpb, 0, s>>>(Qm, Pm, wm, M, asg, cq, L, u, sums);
        k_km_means<<<gk, tpb, 0, s>>>(sums, K, L, u, cq, cp, mq, mp, nullptr);
        if (cudaMemcpyAsync(cq, mq, sizeof(double) * K, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(cp, mp, sizeof(double) * K, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(SWPIC_ECUDA);
    }
    // lumping: means about the final centers, nearest member, slots, moments
    if (cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * 3 * K, s) != cudaSuccess ||
        cudaMemsetAsync(key, 0xff, sizeof(unsigned long long) * K, s) != cudaSuccess)
        return fail(SWPIC_ECUDA);
    k_km_accum<<<gm, tpb, 0, s>>>(Qm, Pm, wm, M, asg, cq, L, u, sums);
    k_km_means<<<gk, tpb, 0, s>>>(sums, K, L, u, cq, cp, mq, mp, wsum);
    k_lump_center<<<gm, tpb, 0, s>>>(Qm, Pm, M, asg, mq, mp, L, key);
    k_lump_slots<<<1, 1024, 0, s>>>(key, wsum, K, Qm, Pm, slot, Q, P, psi, qs, ps, d_n);
    k_lump_moments<<<gm, tpb, 0, s>>>(Qm, Pm, wm, M, asg, slot, L, Q, P, qs, ps);
    if (cudaGetLastError() != cudaSuccess) return fail(SWPIC_ECUDA);
    if (cudaMemcpyAsync(n_out, d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SWPIC_ECUDA);
    cudaFreeAsync(buf, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? SWPIC_OK : SWPIC_ECUDA;
}
