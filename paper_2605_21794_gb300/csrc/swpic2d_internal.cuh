// Internal interface between the 2D2V host code (api2d.cu) and its kernels
// (pass2d.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "swpic2d.h"

namespace swpic2d {

constexpr int kErrOverflow = 1;     // a CTA's node sum left the fixed-point range
constexpr int kErrNonFinite = 2;    // non-finite charge or field energy

// Arguments of the spectral solve and of the node table.
struct SolveArgs2d {
    unsigned long long *acc;      // in: node loads (cleared on read)
    double *b;                    // out: node loads b (FP64)
    double2 *spec;                // nx*ny complex work array, row-major (j nx + i)
    double *phi;                  // out: zero-mean potential
    const double *inv_lam;        // 1 / symbol per mode (0 for the zero mode)
    const double2 *tw;            // exp(-2 pi i k / ntw), k < ntw/2
    double *W;                    // out: (1/2) Phi^T b
    void *table;                  // out: node table in the state precision
    int *err;
    double fx_inv, inv_hx, inv_hy, inv_nn;
    int nx, ny, lognx, logny, ntw;
    const float2 *twf;            // FP32 twiddles (the one-CTA FP32 solve)
    const float *inv_lamf;        // FP32 inverse symbol
    int fx_k;                     // fx_inv = 2^-fx_k
    long long *braw;              // FP32 solve: the integer node loads of the last update
};

struct RecordArgs2d {
    double *diag_acc;
    const double *W;
    double *rec;                  // 9 doubles per record
    int *err;
    double t, area;
    int64_t step;
};

// Arguments of one fused particle pass: closing half-kick (c1 dt), the
// diagnostics at the integer time, opening half-kick (c2 dt), drift (cd dt),
// deposit of the drifted charge into the fixed-point accumulator.
struct PassArgs2d {
    void *Qx, *Qy, *Px, *Py, *qx, *qy, *px, *py;
    const void *psi;
    int64_t n;
    const void *table;            // (Phi, g_x, g_y, 0) per node, state precision
    unsigned long long *acc;      // nx*ny fixed-point node loads
    double *diag_acc;             // mass, momentum x, y, kinetic (FP64 atomics)
    int *err;
    double Lx, Ly, inv_hx, inv_hy, inv_Lx, inv_Ly;
    double k1, k2, kd;            // c1 dt, c2 dt, cd dt
    double fx_scale;
    int nx, ny;
    // FP32 contexts: the last CTA to finish writes the diagnostic record
    // (tail bit 0) and solves the new field in FP32 (tail bit 1)
    int tail;
    unsigned int *done;           // CTAs finished in this pass
    RecordArgs2d rec;
    SolveArgs2d solve;
};

size_t pass_smem_bytes(int prec, int nx, int ny, bool deposit);
cudaError_t launch_pass(int prec, bool decorated, bool deposit, bool diag, const PassArgs2d &a, int grid,
                        int tpb, size_t smem, cudaStream_t s);
cudaError_t launch_solve(int prec, const SolveArgs2d &a, cudaStream_t s, int64_t *launches);
cudaError_t launch_record(const RecordArgs2d &a, cudaStream_t s);
cudaError_t launch_bound(int prec, const PassArgs2d &a, double *out, int grid, cudaStream_t s);
const void *pass_kernel(int prec, bool decorated, bool deposit, bool diag);
cudaError_t launch_init_lattice(int prec, const swpic2d_lattice &spec, double Lx, double Ly,
                                const double *gl, void *const st[9], cudaStream_t s);

}  // namespace swpic2d
