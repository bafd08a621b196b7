// Host-side launch table, one instance per number of fluids (each compiled
// in its own translation unit so the builds run in parallel).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "mfc_device.cuh"

namespace mfc {

// What the sweep does with its per-direction contribution t of cell c:
//   acc_in = 0: Lc = t;  acc_in = 1: Lc = rhs[c] + t;  acc_in = 2: Lc = rhsf[c] + t
//   out_kind = 0: rhs[c] = Lc
//   out_kind = 1: qout[c] = q[c] + dt Lc                       (RK3 stage 1)
//   out_kind = 2: qout[c] = rk_a qn[c] + rk_b (q[c] + dt Lc)   (RK3 stages 2, 3)
//   out_kind = 3: rhsf[c] = Lc
// The float accumulator (acc_in 2, out_kind 3) carries the sum of the
// directional contributions between the sweeps of the mixed-precision
// mode, whose contributions are float32 values; the stage update itself
// is float64 in every mode.
struct SweepArgs {
    const double* q;      // stage input (stencil source)
    double* rhs;          // accumulated right-hand side
    float* rhsf;          // float accumulator (mixed precision)
    const double* qn;     // q^n for out_kind 2 (may alias qout)
    double* qout;         // stage output for out_kind 1, 2
    const double* dt;     // device scalar
    double rk_a, rk_b;
    int acc_in, out_kind;
    int seg;              // cells per thread along the sweep axis
    int nseg;             // segments per line
    int* flag;            // non-physical flag
};

// Adjoint sweep: qbar[c] += (contribution of axis `dir` to (dL/dq)^T rbar)[c].
struct VjpArgs {
    const double* q;      // state at which L is linearised
    const double* rbar;   // adjoint of L (interior cells are read)
    double* qbar;         // accumulated (interior cells)
    int seg;              // cells per thread along the sweep axis
    int nseg;             // segments per line
};

// One chunk of lines of a split double-float sweep (mfc_split.cuh).
struct SplitChunk {
    int64_t line0, nl;  // lines [line0, line0 + nl) of the sweep direction
    double* E;          // the chunk's edge values: 2 N_q slots x (n + 2) cells x nl lines
};

struct LaunchFns {
    // One directional sweep of L(q); mode is MODE_EXACT for the exact
    // tables and MODE_FAST or MODE_MIXED for the others.
    cudaError_t (*sweep)(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s);
    // One directional sweep of the adjoint of L (see mfc_vjp.cuh).
    cudaError_t (*sweep_vjp)(const Consts& C, int dir, int mode, VjpArgs A, cudaStream_t s);
    // CFL minimum of dx_d / (|u_d| + c) into *minbits (atomicMin), in the
    // table's float64 arithmetic.
    cudaError_t (*cfl)(const Consts& C, const double* q, unsigned long long* minbits, int* flag, cudaStream_t s);
    // Viscous stress (mfc_visc.cuh): the cell velocities of q into vel
    // (ND fields of the mode's precision in the padded layout), then the
    // viscous right-hand side into rhs (float64) or rhsf (MODE_MIXED).
    cudaError_t (*viscous)(const Consts& C, int mode, const double* q, void* vel, double* rhs, float* rhsf,
                           cudaStream_t s);
    // Exact tables only: the primitive / conservative maps.
    cudaError_t (*prim_to_cons)(const Consts& C, const double* w, double* q, cudaStream_t s);
    cudaError_t (*cons_to_prim)(const Consts& C, const double* q, double* w, int* flag, cudaStream_t s);
    // MODE_DF tables only: one chunk of a split sweep, phase 0 the
    // reconstruction into K.E, phase 1 the Riemann solve and update from it.
    cudaError_t (*split_sweep)(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s);
};

// Exact tables (MODE_EXACT, built without FMA contraction) and fast tables
// (MODE_FAST, MODE_MIXED) for N_f = 1 .. 4.
const LaunchFns& launch_fns_exact_nf1();
const LaunchFns& launch_fns_exact_nf2();
const LaunchFns& launch_fns_exact_nf3();
const LaunchFns& launch_fns_exact_nf4();
const LaunchFns& launch_fns_fast_nf1();
const LaunchFns& launch_fns_fast_nf2();
const LaunchFns& launch_fns_fast_nf3();
const LaunchFns& launch_fns_fast_nf4();

// MODE_DF directional sweeps for N_f = 1 .. 4 (mfc_nf<NF>_df.cu).  The
// double-float mode's other entries (adjoint, CFL, viscous) are those of
// the fast tables, in MODE_FAST arithmetic.
cudaError_t sweep_df_nf1(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s);
cudaError_t sweep_df_nf2(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s);
cudaError_t sweep_df_nf3(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s);
cudaError_t sweep_df_nf4(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s);
cudaError_t split_df_nf1(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s);
cudaError_t split_df_nf2(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s);
cudaError_t split_df_nf3(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s);
cudaError_t split_df_nf4(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s);

// Cells per thread along a sweep of `n` cells with `nlines` lines.
int sweep_segment(int64_t n, int64_t nlines);

}  // namespace mfc
