// Forward kernels: directional sweeps of L(q) with the fused Runge-Kutta
// stage update, the CFL reduction and the primitive/conservative maps.
#pragma once

#include "mfc_device.cuh"
#include "mfc_launch.h"

namespace mfc {

// One thread marches along one segment of one grid line parallel to axis
// DIR.  It keeps the primitive state of five consecutive cells in
// registers, reconstructs both edge values of every cell once with WENO5
// (so each face state is reconstructed exactly once), solves one HLLC
// problem per face, and finishes each cell as soon as both its faces are
// known.  Boundary cells are read through bc_source (no ghost layer is
// read).  Consecutive threads take consecutive lines; for DIR = 1, 2 those
// are consecutive x, so every load is coalesced.
//
// Positivity reading (the paper is silent): when either reconstructed
// state of a face is not a physical mixture, the face uses the states of
// its two cells (first-order reconstruction) instead.
template <int NF, int ND, int DIR, int MODE>
__device__ __forceinline__ void sweep_body(const Consts& C, const SweepArgs& A) {
    using L = Lay<NF, ND>;
    using R = typename ModeT<MODE>::R;
    constexpr int NQ = L::NQ;
    constexpr int TA = (DIR == 0) ? 1 : 0;
    constexpr int TB = (DIR == 2) ? 1 : 2;
    const int64_t nta = C.n[TA], ntb = C.n[TB];
    const int64_t nlines = nta * ntb;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= nlines * A.nseg) return;
    const int64_t line = tid % nlines;
    const int64_t seg = tid / nlines;
    const int64_t ia = line % nta, ib = line / nta;
    const int64_t base = C.origin + ia * C.stride[TA] + ib * C.stride[TB];
    const int64_t S = C.stride[DIR];
    const int64_t n = C.n[DIR];
    const int64_t s0 = seg * A.seg;
    const int64_t s1 = (s0 + A.seg < n) ? s0 + A.seg : n;
    const int bclo = C.bc_lo[DIR], bchi = C.bc_hi[DIR];
    const int variant = C.weno;
    const R eps = sizeof(R) == 8 ? R(C.eps) : R(C.epsf);
    const R inv_dx = sizeof(R) == 8 ? R(C.inv_dx[DIR]) : R(C.inv_dxf[DIR]);
    const double dx = C.dx[DIR];
    bool bad = false;

    R W[5][NQ];
    auto load_prim = [&](int64_t c, R* out) {
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * C.fstride);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE, R>(qc, out, C, bad);
    };

#pragma unroll
    for (int k = 0; k < 4; ++k) load_prim(s0 - 3 + k, W[k]);

    R WLprev[NQ], Fprev[NQ], uprev = R(0);
    const double dtv = (A.out_kind != 0) ? *A.dt : 0.0;

    for (int64_t m = s0 - 1; m <= s1; ++m) {
        load_prim(m + 2, W[4]);
        R WRm[NQ], WLm[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k)
            weno5_cell<MODE, R>(W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], variant, eps, WRm[k], WLm[k]);
        if (m >= s0) {
            // face m - 1/2: left state WLprev (cell m-1), right state WRm (cell m)
            if (!physical_state<NF, ND, R>(WLprev, C) || !physical_state<NF, ND, R>(WRm, C)) {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    WLprev[k] = W[1][k];
                    WRm[k] = W[2][k];
                }
            }
            R F[NQ], uf;
            hllc<NF, ND, DIR, MODE>(WLprev, WRm, C, F, uf, bad);
            if (m >= s0 + 1) {
                // finish cell m - 1 = window slot 1: faces m - 3/2 (Fprev) and m - 1/2 (F)
                const int64_t off = base + (m - 1) * S;
                const R du = uf - uprev;
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R t;
                    if constexpr (MODE == MODE_EXACT) {
                        t = (Fprev[k] - F[k]) / dx;
                        if (k >= L::A) t = t + W[1][k] * du / dx;
                    } else {
                        t = (Fprev[k] - F[k]) * inv_dx;
                        if (k >= L::A) t = t + W[1][k] * du * inv_dx;
                    }
                    const int64_t o = off + k * C.fstride;
                    double Lc;
                    if constexpr (MODE == MODE_MIXED) {
                        const float Lf = (A.acc_in == 2) ? A.rhsf[o] + t : t;
                        if (A.out_kind == 3) {
                            A.rhsf[o] = Lf;
                            continue;
                        }
                        Lc = double(Lf);
                    } else {
                        Lc = A.acc_in ? A.rhs[o] + double(t) : double(t);
                    }
                    if (A.out_kind == 0) {
                        A.rhs[o] = Lc;
                    } else if (A.out_kind == 1) {
                        A.qout[o] = A.q[o] + dtv * Lc;
                    } else {
                        A.qout[o] = A.rk_a * A.qn[o] + A.rk_b * (A.q[o] + dtv * Lc);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NQ; ++k) Fprev[k] = F[k];
            uprev = uf;
        }
#pragma unroll
        for (int k = 0; k < NQ; ++k) WLprev[k] = WLm[k];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int k = 0; k < NQ; ++k) W[s][k] = W[s + 1][k];
    }
    if (bad) atomicOr(A.flag, 1);
}

template <int NF, int ND, int DIR, int MODE>
__global__ void __launch_bounds__(128) sweep_kernel(const Consts C, const SweepArgs A) {
    sweep_body<NF, ND, DIR, MODE>(C, A);
}

// The mixed mode fits in 128 registers without spilling: four blocks per SM
// (16 warps) hide more of the latency of its float64 steps.
template <int NF, int ND, int DIR>
__global__ void __launch_bounds__(128, 4) sweep_kernel_mixed(const Consts C, const SweepArgs A) {
    sweep_body<NF, ND, DIR, MODE_MIXED>(C, A);
}

// Interior linear index -> element offset in the padded layout.
__device__ __forceinline__ int64_t interior_offset(const Consts& C, int64_t lin) {
    const int64_t i = lin % C.n[0];
    const int64_t j = (lin / C.n[0]) % C.n[1];
    const int64_t k = lin / (C.n[0] * C.n[1]);
    return C.origin + i * C.stride[0] + j * C.stride[1] + k * C.stride[2];
}

// CFL reduction: min over interior cells and active directions of
// dx_d / (|u_d| + c), c^2 = ((Gamma + 1) p + Pi)/(Gamma rho) (the mixture
// stiffened-gas sound speed).  Warp-shuffle min, block min in shared
// memory, then one atomicMin per block on the bit pattern of the positive
// double (ordered like the values).
template <int NF, int ND>
__global__ void __launch_bounds__(256) cfl_kernel(const Consts C, const double* q, unsigned long long* minbits,
                                                  int* flag) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    double m = __longlong_as_double(0x7ff0000000000000ULL);
    bool bad = false;
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = interior_offset(C, lin);
        double qc[NQ], w[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(q + off + f * C.fstride);
        cons_to_prim<NF, ND>(qc, w, C, bad);
        double rho = qc[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) rho = rho + qc[i];
        double Gamma, Pi;
        mixture<NF, double>(qc + L::A, C, Gamma, Pi);
        const double c2 = ((Gamma + 1.0) * w[L::E] + Pi) / (Gamma * rho);
        bad |= !(c2 > 0.0);
        const double cs = sqrt(c2);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double s = C.dx[d] / (fabs(w[L::MOM + d]) + cs);
            m = (s < m) ? s : m;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(0xffffffffu, m, o);
        m = (t < m) ? t : m;
    }
    __shared__ double wm[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wm[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = (lane < (int)(blockDim.x >> 5)) ? wm[lane] : __longlong_as_double(0x7ff0000000000000ULL);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, m, o);
            m = (t < m) ? t : m;
        }
        if (lane == 0) atomicMin(minbits, (unsigned long long)__double_as_longlong(m));
    }
    if (bad) atomicOr(flag, 1);
}

// The CFL reduction in the MODE_FAST arithmetic (MFC_FP64_FAST and
// MFC_MIXED): one refined reciprocal each for rho, Gamma and the largest
// (|u_d| + c)/dx_d of the cell, whose reciprocal is min_d dx_d/(|u_d| + c);
// float64 throughout, same reductions as cfl_kernel.
template <int NF, int ND>
__global__ void __launch_bounds__(256) cfl_fast_kernel(const Consts C, const double* q, unsigned long long* minbits,
                                                       int* flag) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    double m = __longlong_as_double(0x7ff0000000000000ULL);
    bool bad = false;
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = interior_offset(C, lin);
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(q + off + f * C.fstride);
        double rho = qc[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) rho = rho + qc[i];
        bad |= !(rho > 0.0);
        const double irho = rcp_nr(rho);
        double u[ND], ke = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            u[d] = qc[L::MOM + d] * irho;
            ke = fma(qc[L::MOM + d], u[d], ke);
        }
        double Gamma, Pi;
        mixture<NF, double>(qc + L::A, C, Gamma, Pi);
        const double iG = rcp_nr(Gamma);
        const double p = (qc[L::E] - 0.5 * ke - Pi) * iG;
        const double c2 = ((Gamma + 1.0) * p + Pi) * iG * irho;
        bad |= !(c2 > 0.0);
        const double cs = sqrt(c2);
        double smax = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) smax = fmax(smax, (fabs(u[d]) + cs) * C.inv_dx[d]);
        const double s = rcp_nr(smax);
        m = (s < m) ? s : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(0xffffffffu, m, o);
        m = (t < m) ? t : m;
    }
    __shared__ double wm[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wm[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = (lane < (int)(blockDim.x >> 5)) ? wm[lane] : __longlong_as_double(0x7ff0000000000000ULL);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, m, o);
            m = (t < m) ? t : m;
        }
        if (lane == 0) atomicMin(minbits, (unsigned long long)__double_as_longlong(m));
    }
    if (bad) atomicOr(flag, 1);
}

template <int NF, int ND>
__global__ void prim_to_cons_kernel(const Consts C, const double* w, double* q) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = interior_offset(C, lin);
        double wi[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) wi[f] = w[off + f * C.fstride];
        double rho = wi[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) rho = rho + wi[i];
        double u2 = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) u2 = u2 + wi[L::MOM + d] * wi[L::MOM + d];
        double Gamma, Pi;
        mixture<NF, double>(wi + L::A, C, Gamma, Pi);
#pragma unroll
        for (int i = 0; i < NF; ++i) q[off + i * C.fstride] = wi[i];
#pragma unroll
        for (int d = 0; d < ND; ++d) q[off + (L::MOM + d) * C.fstride] = rho * wi[L::MOM + d];
        q[off + L::E * C.fstride] = Gamma * wi[L::E] + Pi + 0.5 * rho * u2;
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) q[off + (L::A + j) * C.fstride] = wi[L::A + j];
    }
}

template <int NF, int ND>
__global__ void cons_to_prim_kernel(const Consts C, const double* q, double* w, int* flag) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    bool bad = false;
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = interior_offset(C, lin);
        double qc[NQ], wo[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = q[off + f * C.fstride];
        cons_to_prim<NF, ND>(qc, wo, C, bad);
#pragma unroll
        for (int f = 0; f < NQ; ++f) w[off + f * C.fstride] = wo[f];
    }
    if (bad) atomicOr(flag, 1);
}

}  // namespace mfc
