// Internal declarations of the sm_103a decorated-particle kernels.
//
// Layout in HBM (all arrays device-resident):
//   particles  caller-owned SoA Q, P, q*, p*, psi* of T (float or double),
//              runs concatenated; run r owns [p0, p1)
//   acc        int64 fixed-point charge accumulator, one per mesh node of
//              every run (runs concatenated at mesh_off); zero between passes
//   table      (phi_h', phi_h'') per element as T2 (float2 / double2)
//   btilde, e  FP64 per node / per element, kept for read-out and diagnostics
//   per run    RunDev parameters, completion counters, diagnostics
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "swpic.h"

namespace swpic {

constexpr int kMaxNx = SWPIC_NX_MAX;
constexpr int kDiagWords = 8;        // t, mass, momentum, kinetic, field, H, E_amp, step

// error flags (bit mask in a device word)
constexpr int kErrFixedOverflow = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrTimeout = 4;       // a bounded device wait ran out

// Element of a position: clamp(floor(p), 0, nx - 1) of the rounded product
// p = fl(Q * nx/L), the definition shared by the pass, the sort keys and the
// static deposit.  It is formed without float -> int conversions (which run on
// the narrow FP64/conversion pipe of this GPU): after clamping p into
// [0, nx - 1/2] (NaN -> 0), the sum 2^m + p rounded toward -inf is exactly
// 2^m + floor(p) (m = 23 for float, 52 for double; p < nx <= 4096), so its bit
// pattern minus that of 2^m is the index, and the sum minus 2^m is floor(p)
// as a float (returned in fi).
// cmax = nx - 1/2 (exact in either type).
__device__ __forceinline__ int elem_index_c(float p, float cmax, float &fi) {
    const float c = fminf(fmaxf(p, 0.0f), cmax);
    const float y = __fadd_rd(c, 8388608.0f);
    fi = y - 8388608.0f;
    return __float_as_int(y) - 0x4B000000;
}
__device__ __forceinline__ int elem_index_c(double p, double cmax, double &fi) {
    const double c = fmin(fmax(p, 0.0), cmax);
    const double y = __dadd_rd(c, 4503599627370496.0);
    fi = y - 4503599627370496.0;
    return (int)(__double_as_longlong(y) - 0x4330000000000000ll);
}
template <typename T>
__device__ __forceinline__ int elem_index(T p, int nx, T &fi) {
    return elem_index_c(p, (T)nx - T(0.5), fi);
}

struct RunDev {
    int64_t p0, p1;          // particle range of the run
    double L, h, inv_h, dt;  // FP64 geometry; inv_h = nx / L
    double inv_L;
    double inv_nx;           // 1 / nx
    double fx_scale;         // fixed-point scale 2^k of the charge accumulator
    double fx_inv;           // 2^-k
    float Lf, inv_hf, inv_Lf, dtf;  // FP32 copies (rounded once from the FP64 values)
    float inv_hf_lo;         // (nx/L) - inv_hf, so Q nx/L = Q inv_hf + Q inv_hf_lo to ~2^-48
    float L_lo;              // L - Lf: the FP32 domain is [0, Lf + L_lo) in exact terms
    float hf, inv_nxf;       // FP32 h and 1/nx (diagnostics of FP32 runs)
    float fx_invf;           // (float) fx_inv, set with fx_scale (the FP32 table's unit)
    int32_t nx, mesh_off;
};

enum PassFlags : uint32_t {
    PASS_DEPOSIT = 1u,     // deposit the drifted (Q, p*) into acc
    PASS_SOLVE = 2u,       // last CTA of each run neutralises + solves + rebuilds tables
    PASS_DIAG = 4u,        // accumulate integer-time (P, q*) sums, last CTA writes a record
    PASS_WRITE_PSI = 8u,   // write psi* to the output arrays (input came from the sort buffer)
    PASS_COUNT_STEP = 16u, // last CTA advances the run's step counter
    PASS_READOUT = 32u,    // (solve kernel only) FP64 b, btilde, E from the snapshot
    PASS_FIELD_ACC = 64u,  // every CTA solves the field of acc_src at its start (no table load);
                           // the CTA holding a run's first particle also writes the run's
                           // table, snapshot, W, E_amp and gauge to global memory
};

struct PassArgs {
    const void *Qi, *Pi, *qsi, *psi_i, *wi;
    void *Qo, *Po, *qso, *pso, *wo;
    int64_t n_total;
    int64_t chunk;            // particles per CTA (multiple of the vector width)
    int32_t n_runs;
    int32_t d2_mode;
    int32_t max_nx;           // largest nx of the batch (shared-memory layout)
    int32_t stages;           // >= 2: bulk-copy pipeline with this many stages; else register loads
    const RunDev *runs;
    RunDev run0;              // runs[0] by value: a one-run pass reads its run from the
                              // kernel parameters instead of global memory
    double c1, c2, cd;        // closing kick, opening kick, drift: fractions of dt
    uint32_t flags;
    unsigned long long *acc;  // int64 bit patterns: deposit target (and the source of the
                              // last-CTA solve and of the solve kernel)
    const unsigned long long *acc_src;    // PASS_FIELD_ACC: the deposit of the current positions
    unsigned long long *acc_clr;          // depositing pass: zeroed by each run's first CTA
    const unsigned long long *acc_m_src;  // P2: midpoint loads beside acc_src
    unsigned long long *acc_m_clr;        // P2: beside acc_clr
    long long *snap;          // int64 snapshot of acc taken by the last solve (read-out)
    long long *gauge;         // [R] integer gauge mean of the last solve (reference of the next)
    unsigned long long *acc_m;  // P2: int64 bit patterns of the element-midpoint load (per element)
    void *table;              // T2 per element
    double *b, *btilde, *efield;
    unsigned long long *run_done;
    double *diag_acc;         // [R][2]: momentum, kinetic
    double *field_diag;       // [R][2]: W, E_amp of the field in `table`
    const double *mass;       // [R]
    long long *steps;         // [R]
    double *ring;             // [R][cap][kDiagWords]
    int32_t *ring_count;      // [R]
    int32_t ring_cap;
    int32_t *err;             // [R] per-run anomaly flags (kErr* bits)
    unsigned long long wait_limit_ns;   // bound of every mbarrier wait of the bulk-copy stream
    int32_t stall_warp;       // test hook: this warp (grid-wide index) never arms its first
                              // stage, so its first wait runs out; -1 = none
    int32_t prefetch;         // 1: issue a CTA's first bulk copies before it stages its table
};

// shared-memory bytes of the pass kernel / the per-run solve for a given max nx
size_t pass_smem_bytes(int prec, int max_nx, int mode, bool decorated, int tpb, int stages, int d2_mode);
size_t solve_smem_bytes(int max_nx);

// launchers (return cudaError_t of the launch)
cudaError_t launch_pass(int prec, bool decorated, int mode, const PassArgs &a, int grid, int tpb,
                        size_t smem, cudaStream_t s);
cudaError_t launch_solve_runs(int prec, const PassArgs &a, int tpb, size_t smem, cudaStream_t s);
// FP64 particle passes (pass64.cu)
cudaError_t launch_pass_f64(bool decorated, int mode, const PassArgs &a, int grid, int tpb, size_t smem,
                            cudaStream_t s);
cudaError_t launch_phi(const RunDev *runs, int n_runs, const double *efield, double *phi,
                       int max_nx, cudaStream_t s);

// sorting
struct SortChunk {
    int64_t start, end;   // particle range (inside one run)
    int64_t cnt_base;     // where this run's [bin][chunk] count block starts
    int32_t run, local;   // run index, chunk index inside the run
    int32_t nch;          // chunks of this run
    int32_t pad;
};
cudaError_t launch_sort_hist(int prec, const void *Q, const RunDev *runs, const SortChunk *chunks,
                             int n_chunks, int32_t *cnt, int max_nx, cudaStream_t s);
cudaError_t launch_scan(const int32_t *cnt, int64_t *pos, int64_t n, int64_t *block_tmp,
                        int64_t n_blocks, cudaStream_t s);
int64_t scan_block_count(int64_t n);
cudaError_t launch_sort_scatter(int prec, bool decorated, const void *const src[5], void *const dst[5],
                                const RunDev *runs, const SortChunk *chunks, int n_chunks,
                                const int64_t *pos, int max_nx, cudaStream_t s);
cudaError_t launch_keys(int prec, const void *Q, const RunDev *runs, int n_runs, int64_t n,
                        int32_t *keys, cudaStream_t s);

// initialisation
struct LatticeDev {
    int32_t nq, nv, n_terms, quad_order, decorate, pad;
    double vmin, vmax, alpha, kx;
    double amp[4], c0[4], c2[4], beta[4], u[4];
    double gx[5], gw[5];
};
cudaError_t launch_init_lattice(int prec, bool decorated, void *Q, void *P, void *qs, void *ps,
                                void *psi, int64_t p0, double L, const LatticeDev &lat,
                                const double *jx, const double *jv, cudaStream_t s);
cudaError_t launch_convert(int prec, const double *src, void *dst, int64_t n, cudaStream_t s);
// mass[r] = sum psi*, bound[2r] = sum |psi*|, bound[2r+1] = sum |p*| (FP64, fixed order)
cudaError_t launch_mass(int prec, const void *psi, const void *ps, const SortChunk *chunks,
                        int n_chunks, double *partials, int n_runs, double *mass, double *bound,
                        cudaStream_t s);

}  // namespace swpic
