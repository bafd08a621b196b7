// Device building blocks of the five-equation WENO5 / HLLC right-hand side
// (arXiv 2503.07953, Sec. 2-3).  Header-only; included by the kernel files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mfc {

constexpr int MAXF = 4;

// Everything a kernel needs to know about the grid, layout and fluids.
// Passed by value as a kernel parameter.
struct Consts {
    int nf, nd, nq;
    int weno;                 // 0 JS, 1 mapped, 2 Z
    int64_t n[3];             // interior cells per axis (1 on inactive axes)
    int64_t stride[3];        // element stride of one cell step along x, y, z
    int64_t fstride;          // elements per field
    int64_t origin;           // element offset of interior cell (0, 0, 0)
    int bc_lo[3], bc_hi[3];   // 0 periodic, 1 transmissive, 2 reflective
    double dx[3], inv_dx[3];
    double g[MAXF], h[MAXF];  // 1/(gamma_i - 1), gamma_i pi_i/(gamma_i - 1)
    float gf[MAXF], hf[MAXF];
    float inv_dxf[3];
    double eps;
    float epsf;
    double cfl;
};

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2 };
enum { WENO_JS = 0, WENO_M = 1, WENO_Z = 2 };

template <int NF, int ND>
struct Lay {
    static constexpr int NQ = 2 * NF + ND;
    static constexpr int MOM = NF;            // first momentum slot
    static constexpr int E = NF + ND;         // energy / pressure slot
    static constexpr int A = NF + ND + 1;     // first stored volume fraction
};

template <class R> __device__ __forceinline__ R coef_g(const Consts& C, int i);
template <> __device__ __forceinline__ double coef_g<double>(const Consts& C, int i) { return C.g[i]; }
template <> __device__ __forceinline__ float coef_g<float>(const Consts& C, int i) { return C.gf[i]; }
template <class R> __device__ __forceinline__ R coef_h(const Consts& C, int i);
template <> __device__ __forceinline__ double coef_h<double>(const Consts& C, int i) { return C.h[i]; }
template <> __device__ __forceinline__ float coef_h<float>(const Consts& C, int i) { return C.hf[i]; }

// Mixture rules (Sec. 2.1.1) with the stiffened-gas EOS (Sec. 2.2):
// Gamma = sum alpha_i/(gamma_i - 1), Pi = sum alpha_i gamma_i pi_i/(gamma_i - 1),
// with alpha_N = 1 - sum of the stored N-1 fractions.
template <int NF, class R>
__device__ __forceinline__ void mixture(const R* alpha, const Consts& C, R& Gamma, R& Pi) {
    R s = R(0);
#pragma unroll
    for (int j = 0; j < NF - 1; ++j) s = s + alpha[j];
    const R aN = R(1) - s;
    Gamma = aN * coef_g<R>(C, NF - 1);
    Pi = aN * coef_h<R>(C, NF - 1);
#pragma unroll
    for (int j = 0; j < NF - 1; ++j) {
        Gamma = Gamma + alpha[j] * coef_g<R>(C, j);
        Pi = Pi + alpha[j] * coef_h<R>(C, j);
    }
}

// Conservative -> primitive in float64 (a2).  Sets bad when rho <= 0.
template <int NF, int ND>
__device__ __forceinline__ void cons_to_prim(const double* q, double* w, const Consts& C, bool& bad) {
    using L = Lay<NF, ND>;
    double rho = q[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) rho = rho + q[i];
    bad |= !(rho > 0.0);
#pragma unroll
    for (int i = 0; i < NF; ++i) w[i] = q[i];
    double u2 = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        w[L::MOM + d] = q[L::MOM + d] / rho;
        u2 = u2 + w[L::MOM + d] * w[L::MOM + d];
    }
#pragma unroll
    for (int j = 0; j < NF - 1; ++j) w[L::A + j] = q[L::A + j];
    double Gamma, Pi;
    mixture<NF, double>(q + L::A, C, Gamma, Pi);
    const double ke = 0.5 * rho * u2;
    w[L::E] = (q[L::E] - ke - Pi) / Gamma;
}

// WENO5 values at both edges of the centre cell of f0..f4 (Sec. 3.2.1;
// candidate polynomials, smoothness indicators and ideal weights are the
// k = 3 uniform-grid case of Sec. 4.2.2).  vr: value at the right edge
// (left state of face c+1/2); vl: value at the left edge (right state of
// face c-1/2).  The smoothness indicators are shared by both edges.
template <class R>
__device__ __forceinline__ void weno5_edge_from_beta(const R* p, const R* beta, const R* d, int variant, R eps,
                                                     R& out) {
    R a[3], w[3];
    if (variant == WENO_Z) {
        const R tau = fabs(beta[0] - beta[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) a[r] = d[r] * (R(1) + tau / (beta[r] + eps));
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const R t = eps + beta[r];
            a[r] = d[r] / (t * t);
        }
    }
    const R s = a[0] + a[1] + a[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = a[r] / s;
    if (variant == WENO_M) {
        R gm[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            gm[r] = w[r] * (d[r] + d[r] * d[r] - R(3) * d[r] * w[r] + w[r] * w[r]) /
                    (d[r] * d[r] + w[r] * (R(1) - R(2) * d[r]));
        const R sm = gm[0] + gm[1] + gm[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) w[r] = gm[r] / sm;
    }
    out = w[0] * p[0] + w[1] * p[1] + w[2] * p[2];
}

template <class R>
__device__ __forceinline__ void weno5_cell(R f0, R f1, R f2, R f3, R f4, int variant, R eps, R& vl, R& vr) {
    const R c13 = R(13.0 / 12.0), c14 = R(0.25);
    R beta[3];
    {
        const R a0 = f0 - R(2) * f1 + f2, b0 = f0 - R(4) * f1 + R(3) * f2;
        const R a1 = f1 - R(2) * f2 + f3, b1 = f1 - f3;
        const R a2 = f2 - R(2) * f3 + f4, b2 = R(3) * f2 - R(4) * f3 + f4;
        beta[0] = c13 * (a0 * a0) + c14 * (b0 * b0);
        beta[1] = c13 * (a1 * a1) + c14 * (b1 * b1);
        beta[2] = c13 * (a2 * a2) + c14 * (b2 * b2);
    }
    {
        R p[3], d[3] = {R(0.1), R(0.6), R(0.3)};
        p[0] = (R(2) * f0 - R(7) * f1 + R(11) * f2) / R(6);
        p[1] = (-f1 + R(5) * f2 + R(2) * f3) / R(6);
        p[2] = (R(2) * f2 + R(5) * f3 - f4) / R(6);
        weno5_edge_from_beta(p, beta, d, variant, eps, vr);
    }
    {
        R p[3], d[3] = {R(0.3), R(0.6), R(0.1)};
        p[0] = (-f0 + R(5) * f1 + R(2) * f2) / R(6);
        p[1] = (R(2) * f1 + R(5) * f2 - f3) / R(6);
        p[2] = (R(11) * f2 - R(7) * f3 + R(2) * f4) / R(6);
        weno5_edge_from_beta(p, beta, d, variant, eps, vl);
    }
}

// HLLC flux across a face normal to axis DIR from reconstructed primitive
// states (Sec. 3.2.2).  Wave speeds min/max of u -/+ c over both sides
// (ties keep the left argument); S* from continuity of normal velocity and
// pressure; Toro's star states; S* >= 0 takes the left side.  The face
// velocity uf (u^{(x)} of Sec. 3.2.1) is u_K outside the fan and S* inside;
// the volume-fraction slots receive alpha_K uf.  bad is set when a squared
// sound speed is not positive.
template <int NF, int ND, int DIR, class R>
__device__ __forceinline__ void hllc(const R* WL, const R* WR, const Consts& C, R* F, R& uf, bool& bad) {
    using L = Lay<NF, ND>;
    R rho[2], un[2], p[2], E[2], c[2];
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        const R* w = K ? WR : WL;
        R r = w[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) r = r + w[i];
        R u2 = R(0);
#pragma unroll
        for (int e = 0; e < ND; ++e) u2 = u2 + w[L::MOM + e] * w[L::MOM + e];
        R Gamma, Pi;
        mixture<NF, R>(w + L::A, C, Gamma, Pi);
        rho[K] = r;
        un[K] = w[L::MOM + DIR];
        p[K] = w[L::E];
        E[K] = Gamma * p[K] + Pi + R(0.5) * r * u2;
        const R c2 = ((Gamma + R(1)) * p[K] + Pi) / (Gamma * r);
        bad |= !(c2 > R(0));
        c[K] = sqrt(c2);
    }
    const R aL = un[0] - c[0], aR = un[1] - c[1];
    const R SL = (aR < aL) ? aR : aL;
    const R bL = un[0] + c[0], bR = un[1] + c[1];
    const R SR = (bR > bL) ? bR : bL;
    const R Ss = (p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1])) /
                 (rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]));

    const bool left = Ss >= R(0);
    const R* w = left ? WL : WR;
    const R rK = left ? rho[0] : rho[1];
    const R uK = left ? un[0] : un[1];
    const R pK = left ? p[0] : p[1];
    const R EK = left ? E[0] : E[1];
    const R SK = left ? SL : SR;
    const bool star = left ? (SL < R(0)) : (SR > R(0));

#pragma unroll
    for (int i = 0; i < NF; ++i) F[i] = w[i] * uK;
#pragma unroll
    for (int e = 0; e < ND; ++e) {
        F[L::MOM + e] = rK * uK * w[L::MOM + e];
        if (e == DIR) F[L::MOM + e] = F[L::MOM + e] + pK;
    }
    F[L::E] = (EK + pK) * uK;
    if (star) {
        const R chi = (SK - uK) / (SK - Ss);
#pragma unroll
        for (int i = 0; i < NF; ++i) {
            const R Us = chi * w[i];
            F[i] = F[i] + SK * (Us - w[i]);
        }
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            const R Us = chi * rK * (e == DIR ? Ss : w[L::MOM + e]);
            F[L::MOM + e] = F[L::MOM + e] + SK * (Us - rK * w[L::MOM + e]);
        }
        const R Es = chi * rK * (EK / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
        F[L::E] = F[L::E] + SK * (Es - EK);
        uf = Ss;
    } else {
        uf = uK;
    }
#pragma unroll
    for (int j = 0; j < NF - 1; ++j) F[L::A + j] = w[L::A + j] * uf;
}

// Index of the interior cell that supplies the value of cell c along an
// axis with n cells (Sec. 3.3): periodic wrap, transmissive copy of the
// nearest cell, reflective mirror (flip = normal momentum changes sign).
__device__ __forceinline__ int64_t bc_source(int64_t c, int64_t n, int bclo, int bchi, bool& flip) {
    if (c < 0) {
        if (bclo == BC_PERIODIC) return c + n;
        if (bclo == BC_TRANSMISSIVE) return 0;
        flip = true;
        return -1 - c;
    }
    if (c >= n) {
        if (bchi == BC_PERIODIC) return c - n;
        if (bchi == BC_TRANSMISSIVE) return n - 1;
        flip = true;
        return 2 * n - 1 - c;
    }
    return c;
}

}  // namespace mfc
