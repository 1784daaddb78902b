// a1 + a2: element keys and the stable counting sort of every run's particles
// by element (sm_103a).  No counterpart in the paper: its serial code needs no
// sort; on the GPU sorted particles give long same-element runs in the fused
// deposit and coherent table reads.
//
//   hist   : one CTA per chunk (a contiguous particle range inside one run)
//            counts its keys in shared memory -> cnt[run block][bin][chunk]
//   scan   : exclusive scan of the flat count array (bin-major inside each
//            run, runs in order) gives every (bin, chunk) its first output slot
//   scatter: one CTA per chunk walks its range in order, 256 particles at a
//            time; the stable rank of a particle among equal keys is
//              (running count of the bin in this chunk)
//            + (equal keys in earlier warps of the step)   [per-warp counts]
//            + (equal keys in earlier lanes of the warp)   [match.any + popc]
//            and all five arrays are copied to that slot.
#include "swpic_internal.cuh"

namespace swpic {

__device__ __forceinline__ float inv_h_of(const RunDev &r, float) { return r.inv_hf; }
__device__ __forceinline__ double inv_h_of(const RunDev &r, double) { return r.inv_h; }

template <typename T>
__device__ __forceinline__ int key_of(T Q, const RunDev &R) {
    T fi;
    return elem_index(Q * inv_h_of(R, T()), R.nx, fi);
}

__device__ __forceinline__ int find_run_s(const RunDev *runs, int n_runs, int64_t idx) {
    int lo = 0, hi = n_runs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (runs[mid].p0 <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void k_keys(const T *Q, const RunDev *runs, int n_runs, int64_t n, int32_t *keys) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int r = find_run_s(runs, n_runs, k);
        keys[k] = key_of(Q[k], runs[r]);
    }
}

template <typename T>
__global__ void __launch_bounds__(512) k_sort_hist(const T *Q, const RunDev *runs,
                                                   const SortChunk *chunks, int32_t *cnt) {
    extern __shared__ int32_t s_h[];
    const SortChunk c = chunks[blockIdx.x];
    const RunDev R = runs[c.run];
    const int nx = R.nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) s_h[j] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = c.start; base < c.end; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        const bool valid = k < c.end;
        const unsigned mask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const int key = key_of(Q[k], R);
            const unsigned peers = __match_any_sync(mask, key);
            if (lane == __ffs(peers) - 1) atomicAdd(&s_h[key], __popc(peers));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nx; j += blockDim.x)
        cnt[c.cnt_base + (int64_t)j * c.nch + c.local] = s_h[j];
}

// --- exclusive scan int32 -> int64 over n entries, tiles of 4096 -------------
constexpr int kScanTile = 4096;
constexpr int kScanThreads = 1024;

int64_t scan_block_count(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

__device__ int64_t block_incl_scan_i64(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t x = (lane < nw) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) sh[lane] = x;
    }
    __syncthreads();
    const int64_t base = (w > 0) ? sh[w - 1] : 0;
    if (total) *total = sh[nw - 1];
    return base + inc;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *cnt, int64_t n,
                                                              int64_t *block_sums) {
    __shared__ int64_t sh[32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int q = 0; q < kScanTile / kScanThreads; ++q) {
        const int64_t k = t0 + (int64_t)threadIdx.x * (kScanTile / kScanThreads) + q;
        if (k < n) s += cnt[k];
    }
    int64_t tot;
    block_incl_scan_i64(s, sh, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int64_t *block_sums, int64_t nb) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < nb; t0 += blockDim.x) {
        const int64_t k = t0 + threadIdx.x;
        const int64_t v = (k < nb) ? block_sums[k] : 0;
        int64_t tot;
        const int64_t inc = block_incl_scan_i64(v, sh, &tot);
        if (k < nb) block_sums[k] = carry + inc - v;   // exclusive
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t *cnt, int64_t n,
                                                            const int64_t *block_sums, int64_t *pos) {
    __shared__ int64_t sh[32];
    constexpr int PER = kScanTile / kScanThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * PER;
    int32_t v[PER];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        v[q] = (t0 + q < n) ? cnt[t0 + q] : 0;
        s += v[q];
    }
    const int64_t inc = block_incl_scan_i64(s, sh, nullptr);
    int64_t p = block_sums[blockIdx.x] + inc - s;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        if (t0 + q < n) pos[t0 + q] = p;
        p += v[q];
    }
}

// --- stable scatter -----------------------------------------------------------
constexpr int kScatterThreads = 256;
constexpr int kScatterWarps = kScatterThreads / 32;

template <typename T, bool DEC>
__global__ void __launch_bounds__(kScatterThreads) k_sort_scatter(
    const T *__restrict__ sQ, const T *__restrict__ sP, const T *__restrict__ sX,
    const T *__restrict__ sY, const T *__restrict__ sW, T *__restrict__ dQ, T *__restrict__ dP,
    T *__restrict__ dX, T *__restrict__ dY, T *__restrict__ dW, const RunDev *runs,
    const SortChunk *chunks, const int64_t *pos, int max_nx) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_run = reinterpret_cast<long long *>(smem);
    uint16_t *s_w = reinterpret_cast<uint16_t *>(smem + (size_t)max_nx * 8);
    const SortChunk c = chunks[blockIdx.x];
    const RunDev R = runs[c.run];
    const int nx = R.nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        s_run[j] = pos[c.cnt_base + (int64_t)j * c.nch + c.local];
#pragma unroll
        for (int w = 0; w < kScatterWarps; ++w) s_w[w * max_nx + j] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = c.start; base < c.end; base += kScatterThreads) {
        const int64_t k = base + threadIdx.x;
        const bool valid = k < c.end;
        T q = T(0), p = T(0), x = T(0), y = T(0), w = T(0);
        int key = 0;
        if (valid) {
            q = sQ[k]; p = sP[k]; w = sW[k];
            if (DEC) { x = sX[k]; y = sY[k]; }
            key = key_of(q, R);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0;
        int rank = 0, cnt = 0;
        if (valid) {
            peers = __match_any_sync(mask, key);
            rank = __popc(peers & lt);
            cnt = __popc(peers);
            if (rank == 0) s_w[warp * max_nx + key] = (uint16_t)cnt;
        }
        __syncthreads();
        long long dst = 0;
        if (valid) {
            int pre = 0;
            for (int v = 0; v < warp; ++v) pre += s_w[v * max_nx + key];
            dst = s_run[key] + pre + rank;
        }
        __syncthreads();
        if (valid && rank == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(s_run + key), (unsigned long long)cnt);
            s_w[warp * max_nx + key] = 0;
        }
        if (valid) {
            dQ[dst] = q; dP[dst] = p; dW[dst] = w;
            if (DEC) { dX[dst] = x; dY[dst] = y; }
        }
        __syncthreads();
    }
}

cudaError_t launch_keys(int prec, const void *Q, const RunDev *runs, int n_runs, int64_t n,
                        int32_t *keys, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (prec == SWPIC_F64) k_keys<double><<<grid, 256, 0, s>>>((const double *)Q, runs, n_runs, n, keys);
    else k_keys<float><<<grid, 256, 0, s>>>((const float *)Q, runs, n_runs, n, keys);
    return cudaGetLastError();
}

cudaError_t launch_sort_hist(int prec, const void *Q, const RunDev *runs, const SortChunk *chunks,
                             int n_chunks, int32_t *cnt, int max_nx, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_nx * 4;
    if (prec == SWPIC_F64)
        k_sort_hist<double><<<n_chunks, 512, smem, s>>>((const double *)Q, runs, chunks, cnt);
    else
        k_sort_hist<float><<<n_chunks, 512, smem, s>>>((const float *)Q, runs, chunks, cnt);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *cnt, int64_t *pos, int64_t n, int64_t *block_tmp,
                        int64_t n_blocks, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scan_reduce<<<(unsigned)n_blocks, kScanThreads, 0, s>>>(cnt, n, block_tmp);
    k_scan_top<<<1, kScanThreads, 0, s>>>(block_tmp, n_blocks);
    k_scan_down<<<(unsigned)n_blocks, kScanThreads, 0, s>>>(cnt, n, block_tmp, pos);
    return cudaGetLastError();
}

cudaError_t launch_sort_scatter(int prec, bool decorated, const void *const src[5], void *const dst[5],
                                const RunDev *runs, const SortChunk *chunks, int n_chunks,
                                const int64_t *pos, int max_nx, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_nx * 8 + (size_t)kScatterWarps * max_nx * 2;
#define SWPIC_SCATTER(T, DEC)                                                                      \
    do {                                                                                           \
        auto kern = k_sort_scatter<T, DEC>;                                                        \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                             (int)smem);                                           \
        if (e != cudaSuccess) return e;                                                            \
        kern<<<n_chunks, kScatterThreads, smem, s>>>(                                              \
            (const T *)src[0], (const T *)src[1], (const T *)src[2], (const T *)src[3],            \
            (const T *)src[4], (T *)dst[0], (T *)dst[1], (T *)dst[2], (T *)dst[3], (T *)dst[4],    \
            runs, chunks, pos, max_nx);                                                            \
        return cudaGetLastError();                                                                 \
    } while (0)
    if (prec == SWPIC_F64) {
        if (decorated) SWPIC_SCATTER(double, true);
        SWPIC_SCATTER(double, false);
    }
    if (decorated) SWPIC_SCATTER(float, true);
    SWPIC_SCATTER(float, false);
#undef SWPIC_SCATTER
}

}  // namespace swpic
