// The MODE_DF directional sweep as two kernels.  recon_kernel_df gives
// every cell of a chunk of lines both WENO5 edge values (double-float
// arithmetic on the float32 pipes, float64 c2p); riemann_kernel_df takes
// them from the scratch, solves one HLLC problem per face (float64) and
// finishes the cells as sweep_body does.  Each kernel needs about 155
// registers where the fused sweep needs 250, so three blocks per SM fit
// instead of two; launched on two streams in chunks of lines, the
// reconstruction of one chunk also runs beside the Riemann solve of the
// previous one, and blocks of both kernels share the SMs.  The operations
// are those of sweep_body<MODE_DF> on the same values; only the compiler's
// fused multiply-add contraction of the update may differ, so the two agree
// to rounding.
#pragma once

#include "mfc_device.cuh"
#include "mfc_launch.h"

namespace mfc {

// Edge value of cell c (-1 <= c <= n) of chunk line l: slot 2 k holds the
// left edge of field k (right state of face c - 1/2), slot 2 k + 1 the right
// edge (left state of face c + 1/2).
__device__ __forceinline__ int64_t edge_index(int slot, int64_t c, int64_t n, int64_t l, int64_t nl) {
    return ((int64_t)slot * (n + 2) + (c + 1)) * nl + l;
}

template <int NF, int ND, int DIR>
__global__ void __launch_bounds__(128) recon_kernel_df(const Consts C, const SweepArgs A, const SplitChunk K) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    constexpr int TA = (DIR == 0) ? 1 : 0;
    constexpr int TB = (DIR == 2) ? 1 : 2;
    const int64_t nta = C.n[TA];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= K.nl * A.nseg) return;
    const int64_t l = tid % K.nl;
    const int64_t line = K.line0 + l;
    const int64_t seg = tid / K.nl;
    const int64_t ia = line % nta, ib = line / nta;
    const int64_t base = C.origin + ia * C.stride[TA] + ib * C.stride[TB];
    const int64_t S = C.stride[DIR];
    const int64_t n = C.n[DIR];
    const int64_t s0 = seg * A.seg;
    const int64_t s1 = (s0 + A.seg < n) ? s0 + A.seg : n;
    // this segment's cells, and the ghost cells -1 and n at the ends of the line
    const int64_t c0 = (s0 == 0) ? -1 : s0;
    const int64_t c1 = (s1 == n) ? n : s1 - 1;
    const int bclo = C.bc_lo[DIR], bchi = C.bc_hi[DIR];
    const df64 eps_df(C.eps), ct_df(C.teno_ct);
    bool bad = false;

    double W[5][NQ];
    auto load_prim = [&](int64_t c, double* out) {
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * C.fstride);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE_DF, double>(qc, out, C, bad);
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) load_prim(c0 - 2 + k, W[k]);
    for (int64_t m = c0; m <= c1; ++m) {
        load_prim(m + 2, W[4]);
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const WenoEdges e = weno5_cell_df(W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], C.weno, eps_df, ct_df);
            K.E[edge_index(2 * k, m, n, l, K.nl)] = e.vl;
            K.E[edge_index(2 * k + 1, m, n, l, K.nl)] = e.vr;
            bad |= e.bad != 0;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int k = 0; k < NQ; ++k) W[s][k] = W[s + 1][k];
    }
    if (bad) atomicOr(A.flag, 1);
}

template <int NF, int ND, int DIR>
__global__ void __launch_bounds__(128) riemann_kernel_df(const Consts C, const SweepArgs A, const SplitChunk K) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    constexpr int TA = (DIR == 0) ? 1 : 0;
    constexpr int TB = (DIR == 2) ? 1 : 2;
    const int64_t nta = C.n[TA];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= K.nl * A.nseg) return;
    const int64_t l = tid % K.nl;
    const int64_t line = K.line0 + l;
    const int64_t seg = tid / K.nl;
    const int64_t ia = line % nta, ib = line / nta;
    const int64_t base = C.origin + ia * C.stride[TA] + ib * C.stride[TB];
    const int64_t S = C.stride[DIR];
    const int64_t n = C.n[DIR];
    const int64_t s0 = seg * A.seg;
    const int64_t s1 = (s0 + A.seg < n) ? s0 + A.seg : n;
    const int bclo = C.bc_lo[DIR], bchi = C.bc_hi[DIR];
    const double inv_dx = C.inv_dx[DIR];
    bool bad = false;

    // primitive state of cell c, as the reconstruction kernel computes it
    auto prim = [&](int64_t c, double* out) {
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * C.fstride);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE_DF, double>(qc, out, C, bad);
    };

    double WLprev[NQ], Fprev[NQ], uprev = 0.0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        WLprev[k] = K.E[edge_index(2 * k + 1, s0 - 1, n, l, K.nl)];
        Fprev[k] = 0.0;
    }
    const double dtv = (A.out_kind != 0) ? *A.dt : 0.0;

    for (int64_t m = s0; m <= s1; ++m) {
        // face m - 1/2: left state WLprev (cell m-1), right state WRm (cell m)
        double WRm[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) WRm[k] = K.E[edge_index(2 * k, m, n, l, K.nl)];
        MixState<double> mL = mix_state<NF, ND, MODE_DF, double>(WLprev, C);
        MixState<double> mR = mix_state<NF, ND, MODE_DF, double>(WRm, C);
        if (!physical_mix<NF, ND, double, MODE_DF>(WLprev, mL, C) || !physical_mix<NF, ND, double, MODE_DF>(WRm, mR, C)) {
            prim(m - 1, WLprev);
            prim(m, WRm);
            mL = mix_state<NF, ND, MODE_DF, double>(WLprev, C);
            mR = mix_state<NF, ND, MODE_DF, double>(WRm, C);
        }
        double F[NQ], uf;
        hllc<NF, ND, DIR, MODE_DF>(WLprev, WRm, mL, mR, C, F, uf, bad);
        if (m >= s0 + 1) {
            // finish cell m - 1: faces m - 3/2 (Fprev) and m - 1/2 (F)
            const int64_t off = base + (m - 1) * S;
            const double du = uf - uprev;
            // alpha rows: alpha div u, or (alpha + K) div u (Kapila); the
            // primitive volume fractions are the conserved ones
            double Kc = 0.0;
            if constexpr (NF == 2) {
                if (C.model == 1) {
                    double w1[NQ];
                    prim(m - 1, w1);
                    Kc = kapila_K<MODE_DF, double>(w1[L::E], w1[L::A], C);
                }
            }
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                double t = (Fprev[k] - F[k]) * inv_dx;
                if (k >= L::A) {
                    const double a = __ldg(A.q + off + k * C.fstride);
                    const double ac = (C.model == 1) ? a + Kc : a;
                    t = t + ac * du * inv_dx;
                }
                const int64_t o = off + k * C.fstride;
                const double Lc = A.acc_in ? A.rhs[o] + t : t;
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
        if (m < s1) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) WLprev[k] = K.E[edge_index(2 * k + 1, m, n, l, K.nl)];
        }
    }
    if (bad) atomicOr(A.flag, 1);
}

}  // namespace mfc
