// The FP64 particle-pass variants, compiled in a translation unit of their own
// so that the pass variants build in parallel.
#include "pass_kernels.cuh"

namespace swpic {

cudaError_t launch_pass_f64(bool decorated, int mode, const PassArgs &a, int grid, int tpb, size_t smem,
                            cudaStream_t s) {
    if (decorated) {
        if (mode == SWPIC_DEPOSIT_ATOMIC) return launch_pass_t<double, true, 0>(a, grid, tpb, smem, s);
        return launch_pass_t<double, true, 1>(a, grid, tpb, smem, s);
    }
    if (mode == SWPIC_DEPOSIT_ATOMIC) return launch_pass_t<double, false, 0>(a, grid, tpb, smem, s);
    return launch_pass_t<double, false, 1>(a, grid, tpb, smem, s);
}

}  // namespace swpic
