// Launch wrappers.  Each translation unit mfc_nf<NF>_<exact|fast>.cu
// instantiates them for one number of fluids NF and one family of
// arithmetic modes (MODE_EXACT, compiled without FMA contraction; or
// MODE_FAST and MODE_MIXED).  ND (1..3) and the sweep direction are
// dispatched here to the kernel templates.
#pragma once

#include "mfc_fwd.cuh"
#include "mfc_launch.h"
#include "mfc_split.cuh"
#include "mfc_visc.cuh"
#include "mfc_vjp.cuh"

namespace mfc {

constexpr int kSweepBlock = 128;
// Below this many lines the per-thread march along x leaves the GPU idle
// (a 1D run is one line): the x sweep then runs one warp per segment.
constexpr int64_t kFewLines = 2048;
constexpr int kSweepVjpBlock = 64;

inline unsigned grid_for(int64_t threads, int block) {
    return (unsigned)((threads + block - 1) / block);
}

inline unsigned stride_grid(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Dynamic shared memory of the MODE_FAST march: the rings of sliding WENO5
// quantities, 7 doubles per field and thread (sweep_body).
template <int NF, int ND>
constexpr int slide_smem_bytes(int block) {
    return 7 * Lay<NF, ND>::NQ * 8 * block;
}

template <int NF, int ND, int DIR, int MODE>
void launch_sweep(unsigned grid, const Consts& C, const SweepArgs& A, cudaStream_t s) {
    if constexpr (MODE == MODE_MIXED) {
        sweep_kernel_mixed<NF, ND, DIR><<<grid, kSweepBlock, 0, s>>>(C, A);
    } else if constexpr (MODE == MODE_FAST) {
        constexpr int smem = slide_smem_bytes<NF, ND>(kSweepBlock);
        static const cudaError_t attr = cudaFuncSetAttribute(sweep_kernel<NF, ND, DIR, MODE>,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        (void)attr;
        sweep_kernel<NF, ND, DIR, MODE><<<grid, kSweepBlock, smem, s>>>(C, A);
    } else {
        sweep_kernel<NF, ND, DIR, MODE><<<grid, kSweepBlock, 0, s>>>(C, A);
    }
}

// y and z sweeps of the mixed mode with shared-memory staging
// (sweep_kernel_staged): 64-thread blocks, the rings in dynamic shared
// memory (under 48 KB for every N_f).
constexpr int kStagedBlock = 64;
template <int NF, int ND, int DIR>
void launch_sweep_staged(int64_t threads, const Consts& C, const SweepArgs& A, cudaStream_t s) {
    constexpr int smem_max = staged_smem_bytes<Lay<NF, ND>::NQ>(kStagedBlock, true);
    static_assert(smem_max <= 48 * 1024, "staged sweep rings must fit the default shared-memory limit");
    const int smem = staged_smem_bytes<Lay<NF, ND>::NQ>(kStagedBlock, A.out_kind == 2);
    // the largest shared-memory carveout, so that eight blocks' rings fit an SM
    static const cudaError_t carve = cudaFuncSetAttribute(
        sweep_kernel_staged<NF, ND, DIR>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    (void)carve;
    sweep_kernel_staged<NF, ND, DIR><<<grid_for(threads, kStagedBlock), kStagedBlock, smem, s>>>(C, A);
}

// x sweep, one warp per line segment (sweep_x_kernel): segments of at
// least 64 cells (32 when there are few lines), enough of them for ~32 warps
// per SM.
template <int NF, int ND, int MODE>
void launch_sweep_x(const Consts& C, SweepArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[1] * C.n[2];
    const int64_t n = C.n[0];
    int64_t nseg = (152LL * 32 + nlines - 1) / nlines;
    const int64_t minseg = nlines < kFewLines ? 32 : 64;
    const int64_t maxseg = (n + minseg - 1) / minseg;
    if (nseg > maxseg) nseg = maxseg;
    if (nseg < 1) nseg = 1;
    A.seg = (int)((n + nseg - 1) / nseg);
    A.nseg = (int)((n + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg * 32;
    sweep_x_kernel<NF, ND, MODE><<<grid_for(threads, kSweepBlock), kSweepBlock, 0, s>>>(C, A);
}

template <int NF, int ND, int DIR, int MODE>
void launch_sweep_vjp(unsigned grid, const Consts& C, const VjpArgs& A, cudaStream_t s) {
    sweep_vjp_kernel<NF, ND, DIR, MODE>
        <<<grid, kSweepVjpBlock, vjp_smem_bytes<NF, ND, MODE>(kSweepVjpBlock), s>>>(C, A);
}

// MODE_EXACT when EXACT, else MODE_FAST / MODE_MIXED as asked.
template <int NF, int ND, bool EXACT>
cudaError_t sweep_nd(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = grid_for(threads, kSweepBlock);
    auto go = [&](auto dirc) {
        constexpr int D = decltype(dirc)::value;
        // x sweeps run one warp per row in the mixed mode (float32 arithmetic
        // is cheap enough that the x march's strided loads bound it) and for
        // few lines (the march would leave most of the GPU idle)
        const bool few = nlines < kFewLines;
        if constexpr (EXACT) {
            if constexpr (D == 0) {
                if (few) {
                    launch_sweep_x<NF, ND, MODE_EXACT>(C, A, s);
                    return;
                }
            }
            launch_sweep<NF, ND, D, MODE_EXACT>(grid, C, A, s);
        } else {
            if (mode == MODE_MIXED) {
                if constexpr (D == 0)
                    launch_sweep_x<NF, ND, MODE_MIXED>(C, A, s);
                else
                    launch_sweep_staged<NF, ND, D>(threads, C, A, s);
            } else {
                if constexpr (D == 0) {
                    if (few) {
                        launch_sweep_x<NF, ND, MODE_FAST>(C, A, s);
                        return;
                    }
                }
                launch_sweep<NF, ND, D, MODE_FAST>(grid, C, A, s);
            }
        }
    };
    if (dir == 0) go(std::integral_constant<int, 0>());
    if constexpr (ND >= 2) if (dir == 1) go(std::integral_constant<int, 1>());
    if constexpr (ND >= 3) if (dir == 2) go(std::integral_constant<int, 2>());
    return cudaGetLastError();
}

// Fused MODE_DF sweeps, used by the allocation-free step (contexts run the
// split sweeps of mfc_split.cuh): the per-thread march in every direction
// and on every grid.
template <int NF, int ND>
cudaError_t sweep_df_nd(const Consts& C, int dir, SweepArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = grid_for(threads, kSweepBlock);
    if (dir == 0) launch_sweep<NF, ND, 0, MODE_DF>(grid, C, A, s);
    if constexpr (ND >= 2) if (dir == 1) launch_sweep<NF, ND, 1, MODE_DF>(grid, C, A, s);
    if constexpr (ND >= 3) if (dir == 2) launch_sweep<NF, ND, 2, MODE_DF>(grid, C, A, s);
    return cudaGetLastError();
}

template <int NF>
cudaError_t sweep_df(const Consts& C, int dir, int, SweepArgs A, cudaStream_t s) {
    switch (C.nd) {
        case 1: return sweep_df_nd<NF, 1>(C, dir, A, s);
        case 2: return sweep_df_nd<NF, 2>(C, dir, A, s);
        default: return sweep_df_nd<NF, 3>(C, dir, A, s);
    }
}

// One chunk of a split MODE_DF sweep (mfc_split.cuh); the segments are
// those of the whole direction, so both phases cut the lines alike.
template <int NF, int ND>
cudaError_t split_df_nd(const Consts& C, int dir, int phase, SweepArgs A, const SplitChunk& K, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = K.nl * A.nseg;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = grid_for(threads, kSweepBlock);
    auto go = [&](auto dirc) {
        constexpr int D = decltype(dirc)::value;
        if (phase == 0)
            recon_kernel_df<NF, ND, D><<<grid, kSweepBlock, 0, s>>>(C, A, K);
        else
            riemann_kernel_df<NF, ND, D><<<grid, kSweepBlock, 0, s>>>(C, A, K);
    };
    if (dir == 0) go(std::integral_constant<int, 0>());
    if constexpr (ND >= 2) if (dir == 1) go(std::integral_constant<int, 1>());
    if constexpr (ND >= 3) if (dir == 2) go(std::integral_constant<int, 2>());
    return cudaGetLastError();
}

template <int NF>
cudaError_t split_df(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s) {
    switch (C.nd) {
        case 1: return split_df_nd<NF, 1>(C, dir, phase, A, K, s);
        case 2: return split_df_nd<NF, 2>(C, dir, phase, A, K, s);
        default: return split_df_nd<NF, 3>(C, dir, phase, A, K, s);
    }
}

template <int NF, int ND, bool EXACT>
cudaError_t sweep_vjp_nd(const Consts& C, int dir, int mode, VjpArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = grid_for(threads, kSweepVjpBlock);
    auto go = [&](auto dirc) {
        constexpr int D = decltype(dirc)::value;
        if constexpr (EXACT) {
            launch_sweep_vjp<NF, ND, D, MODE_EXACT>(grid, C, A, s);
        } else {
            if (mode == MODE_MIXED)
                launch_sweep_vjp<NF, ND, D, MODE_MIXED>(grid, C, A, s);
            else if (mode == MODE_DF)
                launch_sweep_vjp<NF, ND, D, MODE_DF>(grid, C, A, s);
            else
                launch_sweep_vjp<NF, ND, D, MODE_FAST>(grid, C, A, s);
        }
    };
    if (dir == 0) go(std::integral_constant<int, 0>());
    if constexpr (ND >= 2) if (dir == 1) go(std::integral_constant<int, 1>());
    if constexpr (ND >= 3) if (dir == 2) go(std::integral_constant<int, 2>());
    return cudaGetLastError();
}

template <int NF, int ND, int MODE>
cudaError_t viscous_nd(const Consts& C, const double* q, void* vel, double* rhs, float* rhsf, cudaStream_t s) {
    using R = typename ModeT<MODE>::R;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    velocity_kernel<NF, ND, MODE><<<stride_grid(ncell, 256), 256, 0, s>>>(C, q, static_cast<R*>(vel));
    viscous_kernel<NF, ND, MODE><<<grid_for(ncell, 128), 128, 0, s>>>(C, q, static_cast<const R*>(vel), rhs, rhsf);
    return cudaGetLastError();
}

template <int NF, bool EXACT>
struct Launch {
    static cudaError_t sweep(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
        switch (C.nd) {
            case 1: return sweep_nd<NF, 1, EXACT>(C, dir, mode, A, s);
            case 2: return sweep_nd<NF, 2, EXACT>(C, dir, mode, A, s);
            default: return sweep_nd<NF, 3, EXACT>(C, dir, mode, A, s);
        }
    }
    static cudaError_t sweep_vjp(const Consts& C, int dir, int mode, VjpArgs A, cudaStream_t s) {
        switch (C.nd) {
            case 1: return sweep_vjp_nd<NF, 1, EXACT>(C, dir, mode, A, s);
            case 2: return sweep_vjp_nd<NF, 2, EXACT>(C, dir, mode, A, s);
            default: return sweep_vjp_nd<NF, 3, EXACT>(C, dir, mode, A, s);
        }
    }
    static cudaError_t viscous(const Consts& C, int mode, const double* q, void* vel, double* rhs, float* rhsf,
                               cudaStream_t s) {
        auto go = [&](auto modec) -> cudaError_t {
            constexpr int M = decltype(modec)::value;
            switch (C.nd) {
                case 1: return viscous_nd<NF, 1, M>(C, q, vel, rhs, rhsf, s);
                case 2: return viscous_nd<NF, 2, M>(C, q, vel, rhs, rhsf, s);
                default: return viscous_nd<NF, 3, M>(C, q, vel, rhs, rhsf, s);
            }
        };
        if constexpr (EXACT) return go(std::integral_constant<int, MODE_EXACT>());
        else if (mode == MODE_MIXED) return go(std::integral_constant<int, MODE_MIXED>());
        else return go(std::integral_constant<int, MODE_FAST>());
    }
    static cudaError_t cfl(const Consts& C, const double* q, unsigned long long* minbits, int* flag, cudaStream_t s) {
        const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
        const unsigned grid = stride_grid(ncell, 256);
        if constexpr (EXACT) {
            switch (C.nd) {
                case 1: cfl_kernel<NF, 1><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
                case 2: cfl_kernel<NF, 2><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
                default: cfl_kernel<NF, 3><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
            }
        } else {
            switch (C.nd) {
                case 1: cfl_fast_kernel<NF, 1><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
                case 2: cfl_fast_kernel<NF, 2><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
                default: cfl_fast_kernel<NF, 3><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
            }
        }
        return cudaGetLastError();
    }
    static cudaError_t p2c(const Consts& C, const double* w, double* q, cudaStream_t s) {
        const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
        const unsigned grid = stride_grid(ncell, 256);
        switch (C.nd) {
            case 1: prim_to_cons_kernel<NF, 1><<<grid, 256, 0, s>>>(C, w, q); break;
            case 2: prim_to_cons_kernel<NF, 2><<<grid, 256, 0, s>>>(C, w, q); break;
            default: prim_to_cons_kernel<NF, 3><<<grid, 256, 0, s>>>(C, w, q); break;
        }
        return cudaGetLastError();
    }
    static cudaError_t c2p(const Consts& C, const double* q, double* w, int* flag, cudaStream_t s) {
        const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
        const unsigned grid = stride_grid(ncell, 256);
        switch (C.nd) {
            case 1: cons_to_prim_kernel<NF, 1><<<grid, 256, 0, s>>>(C, q, w, flag); break;
            case 2: cons_to_prim_kernel<NF, 2><<<grid, 256, 0, s>>>(C, q, w, flag); break;
            default: cons_to_prim_kernel<NF, 3><<<grid, 256, 0, s>>>(C, q, w, flag); break;
        }
        return cudaGetLastError();
    }
    static const LaunchFns& fns() {
        static const LaunchFns f = {&sweep, &sweep_vjp, &cfl, &viscous, EXACT ? &p2c : nullptr,
                                    EXACT ? &c2p : nullptr};
        return f;
    }
};

}  // namespace mfc
