// Host side of the 1D particle pass: the launchers, the shared-memory layout
// sizes, and the per-run solve and read-out kernels (swpic_solve_field,
// swpic_deposit's read-out, the potential).  The kernels themselves are in
// pass_kernels.cuh; this file instantiates the FP32 variants and pass64.cu the
// FP64 ones (two translation units that compile in parallel).
#include "pass_kernels.cuh"

namespace swpic {

// solve every run (one CTA per run); used by swpic_solve_field / deposit read-out
template <typename T>
__global__ void __launch_bounds__(1024) k_solve_runs(PassArgs a, int full) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int r = blockIdx.x;
    if (r >= a.n_runs) return;
    const RunDev R = a.runs[r];
    if (full == 2) readout_run(a, R, smem);
    else if (a.d2_mode == SWPIC_D2_P2)
        solve_run<T, true>(a, R, r, reinterpret_cast<long long *>(smem), a.acc + R.mesh_off,
                           a.acc_m + R.mesh_off, nullptr, true, full != 0);
    else
        solve_run<T, false>(a, R, r, reinterpret_cast<long long *>(smem), a.acc + R.mesh_off,
                            a.acc_m + R.mesh_off, nullptr, true, full != 0);
}

// Phi from e: Phi_{j+1} = Phi_j - h e_j, then zero mean (one CTA per run)
__global__ void __launch_bounds__(1024) k_phi(const RunDev *runs, int n_runs, const double *efield,
                                              double *phi) {
    __shared__ double sh[32];
    const int r = blockIdx.x;
    if (r >= n_runs) return;
    const RunDev R = runs[r];
    const int nx = R.nx, nt = blockDim.x, tid = threadIdx.x;
    const int per = (nx + nt - 1) / nt;
    const int j0 = min(nx, tid * per), j1 = min(nx, j0 + per);
    const double *e = efield + R.mesh_off;
    double *ph = phi + R.mesh_off;
    // exclusive prefix of -h e (thread-serial + block scan of thread totals)
    double tot = 0.0;
    for (int j = j0; j < j1; ++j) tot += -R.h * e[j];
    const int lane = tid & 31, w = tid >> 5;
    double inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    double base = 0.0;
    for (int k = 0; k < w; ++k) base += sh[k];
    double p = base + inc - tot, s = 0.0;
    for (int j = j0; j < j1; ++j) { ph[j] = p; s += p; p += -R.h * e[j]; }
    __syncthreads();
    const double mean = block_sum_d(s, sh) / (double)nx;
    for (int j = j0; j < j1; ++j) ph[j] -= mean;
}

// ---------------------------------------------------------------------------
size_t solve_smem_bytes(int max_nx) { return (size_t)max_nx * 8; }

size_t pass_smem_bytes(int prec, int max_nx, int mode, bool decorated, int tpb, int stages, int d2_mode) {
    const size_t t2 = (prec == SWPIC_F64) ? 16 : 8;
    const size_t me = (mode == SWPIC_DEPOSIT_ATOMIC) ? ((prec == SWPIC_F64) ? 8 : 4) : 8;
    const size_t tb = (size_t)max_nx * t2,
                 mb0 = (size_t)(max_nx + 1) * me + (d2_mode == SWPIC_D2_P2 ? (size_t)max_nx * me : 0),
                 mb = mb0 > (size_t)max_nx * 8 ? mb0 : (size_t)max_nx * 8;     // as mesh_bytes_all
    size_t push = tb + mb;
    if (stages >= 2)
        push = stage_area_offset(tb, mb, tpb / 32, stages) +
               (size_t)stages * (decorated ? 5 : 3) * (size_t)(tpb / 32) * kTurnBytes;
    const size_t solve = solve_smem_bytes(max_nx);
    return push > solve ? push : solve;
}

cudaError_t launch_pass(int prec, bool decorated, int mode, const PassArgs &a, int grid, int tpb,
                        size_t smem, cudaStream_t s) {
    if (prec == SWPIC_F64) return launch_pass_f64(decorated, mode, a, grid, tpb, smem, s);
    if (decorated) {
        if (mode == SWPIC_DEPOSIT_ATOMIC) return launch_pass_t<float, true, 0>(a, grid, tpb, smem, s);
        return launch_pass_t<float, true, 1>(a, grid, tpb, smem, s);
    }
    if (mode == SWPIC_DEPOSIT_ATOMIC) return launch_pass_t<float, false, 0>(a, grid, tpb, smem, s);
    return launch_pass_t<float, false, 1>(a, grid, tpb, smem, s);
}

cudaError_t launch_solve_runs(int prec, const PassArgs &a, int tpb, size_t smem, cudaStream_t s) {
    // PASS_SOLVE: full solve; PASS_READOUT: FP64 read-out from the snapshot; else snapshot only
    const int full = (a.flags & PASS_READOUT) ? 2 : ((a.flags & PASS_SOLVE) ? 1 : 0);
    if (prec == SWPIC_F64) {
        cudaError_t err = cudaFuncSetAttribute(k_solve_runs<double>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k_solve_runs<double><<<a.n_runs, tpb, smem, s>>>(a, full);
    } else {
        cudaError_t err = cudaFuncSetAttribute(k_solve_runs<float>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k_solve_runs<float><<<a.n_runs, tpb, smem, s>>>(a, full);
    }
    return cudaGetLastError();
}

cudaError_t launch_phi(const RunDev *runs, int n_runs, const double *efield, double *phi, int max_nx,
                       cudaStream_t s) {
    (void)max_nx;
    k_phi<<<n_runs, 256, 0, s>>>(runs, n_runs, efield, phi);
    return cudaGetLastError();
}

}  // namespace swpic
