// swpic_deposit_static: the charge deposit of one run without any device
// allocation.
//
// Who needs this: callers that cannot let a library allocate device memory,
// e.g. a host application that owns the whole device-memory budget through its
// own pool or allocator and forbids third-party cudaMalloc/cudaFree, or code
// that must not touch the allocator at all from a time-critical loop.  The
// regular path (swpic_create + swpic_deposit) allocates its accumulators when
// the context is created; this entry point instead keeps its scratch in
// file-scope device arrays of fixed size that exist as long as the library is
// loaded (every GPU that loads the library holds them until the process exits).
//
// Scratch: SWPIC_STATIC_NX_MAX (4096) int64 words for the fixed-point charge
// accumulator plus two doubles for the weight bound: 32 KB + 16 B per device.
//
// Arithmetic is the same as the context path's deposit: b_j = sum_a psi*_a
// phi_j(Q_a) - p*_a phi_j'(Q_a) on a periodic P1 mesh, positions wrapped into
// [0, L) first (in FP32 against L = fl32(L) + the low part, as the particle pass
// wraps), element decided by floor(Q nx/L) in the state's precision,
// per-thread contributions converted to 64-bit fixed point with a power-of-two
// scale fixed by sum |psi*| + 2 sum |p*|/h, and added exactly with integer
// atomics.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "swpic_internal.cuh"

namespace {

constexpr int kStaticNxMax = SWPIC_STATIC_NX_MAX;

// the scratch: it keeps the last call's contents; each call clears it first
static __device__ __align__(256) unsigned long long g_acc[kStaticNxMax];
static __device__ __align__(256) double g_bound[2];

struct StaticPtrs {
    unsigned long long *acc = nullptr;
    double *bound = nullptr;
};

std::mutex g_mu;
StaticPtrs g_ptrs[64];          // per device ordinal
bool g_ready[64] = {false};

__global__ void k_static_clear(unsigned long long *acc, double *bound, int nx) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= nx && j < kStaticNxMax; j += gridDim.x * blockDim.x)
        acc[j] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) { bound[0] = 0.0; bound[1] = 0.0; }
}

template <typename T>
__global__ void k_static_bound(const T *ps, const T *psi, int64_t n, double *bound) {
    double a = 0.0, b = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        a += fabs((double)psi[k]);
        if (ps) b += fabs((double)ps[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(bound, a);
        atomicAdd(bound + 1, b);
    }
}

// position inside the element whose index fi was decided from p = fl(q inv_h);
// in FP32 the rounding error of that product and the low part of nx/L are
// added back so xi is accurate to its own ulp
__device__ __forceinline__ float xi_t(float q, float p, float fi, float inv_h, float inv_h_lo) {
    return (p - fi) + fmaf(q, inv_h_lo, fmaf(q, inv_h, -p));
}
__device__ __forceinline__ double xi_t(double, double p, double fi, double, double) {
    return p - fi;
}

// Periodic wrap into [0, L).  FP64: Q - L floor(Q/L) with the round-up case
// (a result equal to L) mapped to 0.  FP32: L is not a float, so it is carried
// as L_hi + L_lo (L_hi = fl32(L)); a position is inside when Q >= 0 and
// Q - L_hi < L_lo (Q - L_hi is exact near L), and a position one period off is
// shifted with both parts, so wrapped particles are not moved by L - fl32(L).
__device__ __forceinline__ double wrap_t(double q, double L, double, double) {
    if (q >= 0.0 && q < L) return q;
    double w = __dsub_rn(q, __dmul_rn(L, floor(q / L)));     // unfused, as the pass rounds it
    if (w >= L) w -= L;
    if (w < 0.0) w += L;
    return w;
}
__device__ __forceinline__ bool inside_t(float q, float L_hi, float L_lo) {
    return q >= 0.0f && (q - L_hi) < L_lo;
}
__device__ __forceinline__ float wrap_t(float q, float L_hi, float L_lo, float inv_L) {
    if (inside_t(q, L_hi, L_lo) || q != q) return q;
    float w = (q >= 0.0f) ? (q - L_hi) - L_lo : (q + L_hi) + L_lo;   // one period off
    if (inside_t(w, L_hi, L_lo)) return w;
    const float k = floorf(w * inv_L);                                 // several periods
    w = fmaf(-k, L_lo, fmaf(-k, L_hi, w));
    if (w >= 0.0f && !inside_t(w, L_hi, L_lo)) w = (w - L_hi) - L_lo;
    if (w < 0.0f) w = (w + L_hi) + L_lo;
    if (!inside_t(w, L_hi, L_lo)) w = (w < 0.0f) ? 0.0f : (w - L_hi) - L_lo;
    return w < 0.0f ? 0.0f : w;
}

__device__ __forceinline__ double fixed_scale(const double *bound, double inv_h) {
    const double m = bound[0] + 2.0 * bound[1] * inv_h;
    int k = 58;
    if (m > 0.0) k = 58 - (int)ceil(log2(m));
    k = max(-1000, min(1000, k));
    return ldexp(1.0, k);
}

template <typename T>
__global__ void k_static_deposit(const T *Q, const T *ps, const T *psi, int64_t n, T inv_h, T inv_h_lo,
                                 T L_hi, T L_lo, T inv_L, int nx, const double *bound,
                                 unsigned long long *acc) {
    extern __shared__ unsigned long long s_mesh[];           // nx + 1 words
    for (int j = threadIdx.x; j <= nx; j += blockDim.x) s_mesh[j] = 0ull;
    __syncthreads();
    const double scale = fixed_scale(bound, (double)inv_h);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const T q = wrap_t(Q[k], L_hi, L_lo, inv_L);
        const T p = q * inv_h;
        T fi;
        const int i = swpic::elem_index(p, nx, fi);
        const T xi = xi_t(q, p, fi, inv_h, inv_h_lo);
        T w0 = psi[k] * (T(1) - xi), w1 = psi[k] * xi;
        if (ps) {
            const T dq = ps[k] * inv_h;
            w0 += dq;
            w1 -= dq;
        }
        atomicAdd(s_mesh + i, (unsigned long long)__double2ll_rn((double)w0 * scale));
        atomicAdd(s_mesh + i + 1, (unsigned long long)__double2ll_rn((double)w1 * scale));
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= nx; j += blockDim.x) {
        const unsigned long long v = s_mesh[j];
        if (v) atomicAdd(acc + (j == nx ? 0 : j), v);
    }
}

__global__ void k_static_finish(const unsigned long long *acc, const double *bound, double inv_h, int nx,
                                double *b) {
    const double inv = 1.0 / fixed_scale(bound, inv_h);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) b[j] = (double)(long long)acc[j] * inv;
}

// once per device, with that device current: the device addresses of the
// scratch arrays (their host-side names are not device addresses).  They are
// kept for the life of the process: a cudaDeviceReset unloads this code from
// the device, and the kept addresses are not valid after it.
swpic_status static_setup(StaticPtrs *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SWPIC_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        StaticPtrs p;
        if (cudaGetSymbolAddress((void **)&p.acc, g_acc) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&p.bound, g_bound) != cudaSuccess) {
            cudaGetLastError();          // this call's own error, reported by the status
            return SWPIC_ECUDA;
        }
        g_ptrs[dev] = p;
        g_ready[dev] = true;
    }
    *out = g_ptrs[dev];
    return SWPIC_OK;
}

}  // namespace

extern "C" swpic_status swpic_deposit_static(const void *Q, const void *ps, const void *psi, int64_t n,
                                             int32_t precision, double L, int32_t nx, double *b,
                                             swpic_stream stream) {
    if (nx < 2 || nx > kStaticNxMax) return SWPIC_EINVAL;        // beyond the static scratch
    if (!(L > 0.0) || !std::isfinite(L) || n < 0 || !b) return SWPIC_EINVAL;
    if (precision != SWPIC_F32 && precision != SWPIC_F64) return SWPIC_EINVAL;
    if (n > 0 && (!Q || !psi)) return SWPIC_EINVAL;
    // an error left pending by earlier work is reported, not cleared (it is
    // not this call's to consume); past this point every launch error is ours
    if (cudaPeekAtLastError() != cudaSuccess) return SWPIC_ECUDA;
    StaticPtrs p;
    swpic_status st = static_setup(&p);
    if (st != SWPIC_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double inv_h = (double)nx / L;
    k_static_clear<<<(nx + 256) / 256, 256, 0, s>>>(p.acc, p.bound, nx);
    if (cudaGetLastError() != cudaSuccess) return SWPIC_ECUDA;
    if (n > 0) {
        const int grid = (int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216);
        const size_t smem = (size_t)(nx + 1) * 8;
        if (precision == SWPIC_F64) {
            k_static_bound<double><<<grid, 256, 0, s>>>((const double *)ps, (const double *)psi, n, p.bound);
            if (cudaGetLastError() != cudaSuccess) return SWPIC_ECUDA;
            k_static_deposit<double><<<grid, 256, smem, s>>>((const double *)Q, (const double *)ps,
                                                             (const double *)psi, n, inv_h, 0.0, L, 0.0,
                                                             1.0 / L, nx, p.bound, p.acc);
        } else {
            k_static_bound<float><<<grid, 256, 0, s>>>((const float *)ps, (const float *)psi, n, p.bound);
            if (cudaGetLastError() != cudaSuccess) return SWPIC_ECUDA;
            const float hi = (float)inv_h, lo = (float)(inv_h - (double)hi);
            const float L_hi = (float)L, L_lo = (float)(L - (double)L_hi);
            k_static_deposit<float><<<grid, 256, smem, s>>>((const float *)Q, (const float *)ps,
                                                            (const float *)psi, n, hi, lo, L_hi, L_lo,
                                                            (float)(1.0 / L), nx, p.bound, p.acc);
        }
        if (cudaGetLastError() != cudaSuccess) return SWPIC_ECUDA;
    }
    k_static_finish<<<1, 256, 0, s>>>(p.acc, p.bound, inv_h, nx, b);
    return cudaGetLastError() == cudaSuccess ? SWPIC_OK : SWPIC_ECUDA;
}
