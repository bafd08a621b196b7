// Launch wrappers, instantiated once per number of fluids NF by
// mfc_nf<NF>.cu.  ND (1..3), the sweep direction and the precision are
// dispatched here to the kernel templates.
#pragma once

#include "mfc_fwd.cuh"
#include "mfc_launch.h"
#include "mfc_vjp.cuh"

namespace mfc {

constexpr int kSweepBlock = 128;
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

template <int NF, int ND>
cudaError_t sweep_nd(const Consts& C, int dir, int precision, SweepArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg;
    const unsigned grid = grid_for(threads, kSweepBlock);
    if (threads == 0) return cudaSuccess;
#define MFC_SWEEP(D)                                                                              \
    do {                                                                                          \
        if (precision == 0)                                                                       \
            sweep_kernel<NF, ND, D, double><<<grid, kSweepBlock, 0, s>>>(C, A);                   \
        else                                                                                      \
            sweep_kernel<NF, ND, D, float><<<grid, kSweepBlock, 0, s>>>(C, A);                    \
    } while (0)
    if (dir == 0) {
        MFC_SWEEP(0);
    } else if constexpr (ND >= 2) {
        if (dir == 1) {
            MFC_SWEEP(1);
        } else if constexpr (ND >= 3) {
            MFC_SWEEP(2);
        }
    }
#undef MFC_SWEEP
    return cudaGetLastError();
}

template <int NF, int ND>
cudaError_t sweep_vjp_nd(const Consts& C, int dir, int precision, VjpArgs A, cudaStream_t s) {
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[dir];
    A.seg = sweep_segment(C.n[dir], nlines);
    A.nseg = (int)((C.n[dir] + A.seg - 1) / A.seg);
    const int64_t threads = nlines * A.nseg;
    const unsigned grid = grid_for(threads, kSweepVjpBlock);
    if (threads == 0) return cudaSuccess;
#define MFC_SWEEP_VJP(D)                                                                          \
    do {                                                                                          \
        if (precision == 0)                                                                       \
            sweep_vjp_kernel<NF, ND, D, double><<<grid, kSweepVjpBlock, 0, s>>>(C, A);            \
        else                                                                                      \
            sweep_vjp_kernel<NF, ND, D, float><<<grid, kSweepVjpBlock, 0, s>>>(C, A);             \
    } while (0)
    if (dir == 0) {
        MFC_SWEEP_VJP(0);
    } else if constexpr (ND >= 2) {
        if (dir == 1) {
            MFC_SWEEP_VJP(1);
        } else if constexpr (ND >= 3) {
            MFC_SWEEP_VJP(2);
        }
    }
#undef MFC_SWEEP_VJP
    return cudaGetLastError();
}

template <int NF>
struct Launch {
    static cudaError_t sweep(const Consts& C, int dir, int precision, SweepArgs A, cudaStream_t s) {
        switch (C.nd) {
            case 1: return sweep_nd<NF, 1>(C, dir, precision, A, s);
            case 2: return sweep_nd<NF, 2>(C, dir, precision, A, s);
            default: return sweep_nd<NF, 3>(C, dir, precision, A, s);
        }
    }
    static cudaError_t sweep_vjp(const Consts& C, int dir, int precision, VjpArgs A, cudaStream_t s) {
        switch (C.nd) {
            case 1: return sweep_vjp_nd<NF, 1>(C, dir, precision, A, s);
            case 2: return sweep_vjp_nd<NF, 2>(C, dir, precision, A, s);
            default: return sweep_vjp_nd<NF, 3>(C, dir, precision, A, s);
        }
    }
    static cudaError_t cfl(const Consts& C, const double* q, unsigned long long* minbits, int* flag, cudaStream_t s) {
        const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
        const unsigned grid = stride_grid(ncell, 256);
        switch (C.nd) {
            case 1: cfl_kernel<NF, 1><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
            case 2: cfl_kernel<NF, 2><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
            default: cfl_kernel<NF, 3><<<grid, 256, 0, s>>>(C, q, minbits, flag); break;
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
        static const LaunchFns f = {&sweep, &cfl, &p2c, &c2p, &sweep_vjp};
        return f;
    }
};

}  // namespace mfc
