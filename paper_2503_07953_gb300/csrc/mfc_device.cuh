// Device building blocks of the five-equation WENO5 / HLLC right-hand side
// (arXiv 2503.07953, Sec. 2-3).  Header-only; included by the kernel files.
//
// Every block is templated on an arithmetic mode:
//   MODE_EXACT  float64, every operation in the order of the defining
//               formula (IEEE division and square root; the translation
//               units that instantiate it are compiled without FMA
//               contraction), so results are reproducible bit for bit;
//   MODE_FAST   float64 with the divisions of the WENO weights folded into
//               one reciprocal per normalisation, reciprocals instead of
//               repeated divisions, and FMA contraction;
//   MODE_MIXED  the MODE_FAST formulas in float32 for reconstruction, the
//               Riemann solve and the per-direction flux difference;
//               conservative-to-primitive conversion stays float64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mfc {

constexpr int MAXF = 4;

enum { MODE_EXACT = 0, MODE_MIXED = 1, MODE_FAST = 2 };

template <int MODE> struct ModeT { using R = double; };
template <> struct ModeT<MODE_MIXED> { using R = float; };

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

// Reciprocal: in float64 the hardware approximation refined by two
// Newton-Raphson steps r <- r + r (1 - x r) (each step squares the
// relative error; the result is within a few ulps, not correctly rounded);
// in float32 the fast approximate instruction.
__device__ __forceinline__ double rcp_nr(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
template <class R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ double rcp<double>(double x) { return rcp_nr(x); }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

// Quotient by arithmetic mode: MODE_EXACT IEEE division; MODE_FAST a times
// the refined reciprocal of b; MODE_MIXED the fast float32 division.
template <int MODE> struct Arith {
    static __device__ __forceinline__ double quot(double a, double b) { return a * rcp_nr(b); }
};
template <> struct Arith<MODE_EXACT> {
    static __device__ __forceinline__ double quot(double a, double b) { return a / b; }
};
template <> struct Arith<MODE_MIXED> {
    static __device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
};

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

// Conservative -> primitive in float64 (a2): rho = sum alpha_i rho_i,
// u = (rho u)/rho, p = (rho E - 1/2 rho |u|^2 - Pi)/Gamma.  Sets bad when
// rho <= 0.
template <int NF, int ND, int MODE = MODE_EXACT>
__device__ __forceinline__ void cons_to_prim(const double* q, double* w, const Consts& C, bool& bad) {
    using L = Lay<NF, ND>;
    double rho = q[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) rho = rho + q[i];
    bad |= !(rho > 0.0);
#pragma unroll
    for (int i = 0; i < NF; ++i) w[i] = q[i];
    double u2 = 0.0;
    if constexpr (MODE == MODE_EXACT) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            w[L::MOM + d] = q[L::MOM + d] / rho;
            u2 = u2 + w[L::MOM + d] * w[L::MOM + d];
        }
    } else {
        const double irho = rcp_nr(rho);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            w[L::MOM + d] = q[L::MOM + d] * irho;
            u2 = u2 + w[L::MOM + d] * w[L::MOM + d];
        }
    }
#pragma unroll
    for (int j = 0; j < NF - 1; ++j) w[L::A + j] = q[L::A + j];
    double Gamma, Pi;
    mixture<NF, double>(q + L::A, C, Gamma, Pi);
    const double ke = 0.5 * rho * u2;
    w[L::E] = Arith<MODE>::quot(q[L::E] - ke - Pi, Gamma);
}

// Primitive state of one cell in the precision of the reconstruction.
// MODE_EXACT / MODE_FAST: cons_to_prim in float64.  MODE_MIXED: the
// cancelling part of the pressure recovery, rho E - Pi - |rho u|^2/(2 rho),
// is evaluated in float64 (Pi from the float64 volume fractions, the
// subtractions in float64); the kinetic energy, the velocities and the final
// division by Gamma, whose relative errors carry into p unamplified, in
// float32, as are the outputs.
template <int NF, int ND, int MODE, class R>
__device__ __forceinline__ void prim_for_recon(const double* q, R* out, const Consts& C, bool& bad) {
    using L = Lay<NF, ND>;
    if constexpr (MODE == MODE_MIXED) {
        float rho = float(q[0]);
#pragma unroll
        for (int i = 1; i < NF; ++i) rho += float(q[i]);
        bad |= !(rho > 0.0f);
        const float irho = __fdividef(1.0f, rho);
#pragma unroll
        for (int i = 0; i < NF; ++i) out[i] = float(q[i]);
        float ke = 0.0f;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const float m = float(q[L::MOM + d]);
            out[L::MOM + d] = m * irho;
            ke += m * out[L::MOM + d];
        }
        ke *= 0.5f;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) s = s + q[L::A + j];
        double Pi = (1.0 - s) * C.h[NF - 1];
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) Pi = Pi + q[L::A + j] * C.h[j];
        const double num = (q[L::E] - Pi) - double(ke);
        float Gamma = float(1.0 - s) * C.gf[NF - 1];
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) {
            out[L::A + j] = float(q[L::A + j]);
            Gamma += out[L::A + j] * C.gf[j];
        }
        out[L::E] = __fdividef(float(num), Gamma);
    } else {
        double w[Lay<NF, ND>::NQ];
        cons_to_prim<NF, ND, MODE>(q, w, C, bad);
#pragma unroll
        for (int f = 0; f < Lay<NF, ND>::NQ; ++f) out[f] = R(w[f]);
    }
}

// A primitive state is a physical mixture when rho > 0, Gamma > 0 and
// (Gamma + 1) p + Pi > 0 (so that c^2 > 0).
template <int NF, int ND, class R>
__device__ __forceinline__ bool physical_state(const R* w, const Consts& C) {
    using L = Lay<NF, ND>;
    R rho = w[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) rho = rho + w[i];
    R Gamma, Pi;
    mixture<NF, R>(w + L::A, C, Gamma, Pi);
    return rho > R(0) && Gamma > R(0) && (Gamma + R(1)) * w[L::E] + Pi > R(0);
}

// ---------------------------------------------------------------------------
// WENO5 (Sec. 3.2.1; candidate polynomials, smoothness indicators and ideal
// weights are the k = 3 uniform-grid case of Sec. 4.2.2).  weno5_cell gives
// the values at both edges of the centre cell of f0..f4: vr at the right
// edge (left state of face c+1/2), vl at the left edge (right state of face
// c-1/2).  The smoothness indicators are shared by both edges.
// ---------------------------------------------------------------------------

// Smoothness indicators.  float32 divides them and eps by sum(beta) (the
// weights depend only on ratios of eps + beta), with a relative floor of
// 1e-9 on eps that keeps every product in the weights inside the float
// range; scale receives the factor applied (1 in float64).
template <class R>
__device__ __forceinline__ void weno5_scaled_beta(R f0, R f1, R f2, R f3, R f4, R eps, R* b, R& e, R& scale) {
    const R c13 = R(13.0 / 12.0), c14 = R(0.25);
    const R a0 = f0 - R(2) * f1 + f2, g0 = f0 - R(4) * f1 + R(3) * f2;
    const R a1 = f1 - R(2) * f2 + f3, g1 = f1 - f3;
    const R a2 = f2 - R(2) * f3 + f4, g2 = R(3) * f2 - R(4) * f3 + f4;
    b[0] = c13 * (a0 * a0) + c14 * (g0 * g0);
    b[1] = c13 * (a1 * a1) + c14 * (g1 * g1);
    b[2] = c13 * (a2 * a2) + c14 * (g2 * g2);
    if constexpr (sizeof(R) == 8) {
        e = eps;
        scale = R(1);
    } else {
        scale = rcp<R>(b[0] + b[1] + b[2] + R(1e-30));
        b[0] *= scale;
        b[1] *= scale;
        b[2] *= scale;
        e = fmaxf(eps * scale, 1e-9f);
    }
}

// MODE_EXACT weights and value of one edge, in the order of the defining
// formulas: alpha_r = d_r/(eps + beta_r)^2 (JS, mapped) or
// d_r (1 + tau/(beta_r + eps)) (Z, q = 1, tau = |beta_0 - beta_2|),
// w = alpha/sum(alpha); mapped (Henrick 2005):
// g_r(w) = w (d + d^2 - 3 d w + w^2)/(d^2 + w (1 - 2 d)), omega = g/sum(g).
__device__ __forceinline__ double weno5_edge_exact(const double* p, const double* beta, const double* d,
                                                   int variant, double eps) {
    double a[3], w[3];
    if (variant == WENO_Z) {
        const double tau = fabs(beta[0] - beta[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) a[r] = d[r] * (1.0 + tau / (beta[r] + eps));
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double t = eps + beta[r];
            a[r] = d[r] / (t * t);
        }
    }
    const double s = a[0] + a[1] + a[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = a[r] / s;
    if (variant == WENO_M) {
        double gm[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            gm[r] = w[r] * (d[r] + d[r] * d[r] - 3.0 * d[r] * w[r] + w[r] * w[r]) /
                    (d[r] * d[r] + w[r] * (1.0 - 2.0 * d[r]));
        const double sm = gm[0] + gm[1] + gm[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) w[r] = gm[r] / sm;
    }
    return w[0] * p[0] + w[1] * p[1] + w[2] * p[2];
}

// MODE_FAST / MODE_MIXED weights of one edge: the same functions with one
// reciprocal per normalisation.  alpha_r = d_r / t_r^2 is multiplied
// through by t_0^2 t_1^2 t_2^2 (JS, mapped) and d_r (1 + tau / t_r) by
// t_0 t_1 t_2 (Z), so P_r holds the product over the other stencils; the
// mapped weights are normalised the same way.
template <class R>
__device__ __forceinline__ void weno5_edge_weights(const R* P, const R* d, int variant, R* om) {
    R a0 = d[0] * P[0], a1 = d[1] * P[1], a2 = d[2] * P[2];
    R inv = rcp<R>(a0 + a1 + a2);
    R w0 = a0 * inv, w1 = a1 * inv, w2 = a2 * inv;
    if (variant == WENO_M) {
        const R w[3] = {w0, w1, w2};
        R N[3], D[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            N[r] = w[r] * (d[r] * (R(1) + d[r]) + w[r] * (w[r] - R(3) * d[r]));
            D[r] = d[r] * d[r] + w[r] * (R(1) - R(2) * d[r]);
        }
        const R g0 = N[0] * (D[1] * D[2]), g1 = N[1] * (D[0] * D[2]), g2 = N[2] * (D[0] * D[1]);
        inv = rcp<R>(g0 + g1 + g2);
        w0 = g0 * inv;
        w1 = g1 * inv;
        w2 = g2 * inv;
    }
    om[0] = w0;
    om[1] = w1;
    om[2] = w2;
}

template <int MODE, class R>
__device__ __forceinline__ void weno5_cell(R f0, R f1, R f2, R f3, R f4, int variant, R eps, R& vl, R& vr) {
    if constexpr (MODE == MODE_EXACT) {
        const double c13 = 13.0 / 12.0, c14 = 0.25;
        double beta[3];
        const double a0 = f0 - 2.0 * f1 + f2, g0 = f0 - 4.0 * f1 + 3.0 * f2;
        const double a1 = f1 - 2.0 * f2 + f3, g1 = f1 - f3;
        const double a2 = f2 - 2.0 * f3 + f4, g2 = 3.0 * f2 - 4.0 * f3 + f4;
        beta[0] = c13 * (a0 * a0) + c14 * (g0 * g0);
        beta[1] = c13 * (a1 * a1) + c14 * (g1 * g1);
        beta[2] = c13 * (a2 * a2) + c14 * (g2 * g2);
        {
            const double d[3] = {0.1, 0.6, 0.3};
            const double p[3] = {(2.0 * f0 - 7.0 * f1 + 11.0 * f2) / 6.0, (-f1 + 5.0 * f2 + 2.0 * f3) / 6.0,
                                 (2.0 * f2 + 5.0 * f3 - f4) / 6.0};
            vr = weno5_edge_exact(p, beta, d, variant, eps);
        }
        {
            const double d[3] = {0.3, 0.6, 0.1};
            const double p[3] = {(-f0 + 5.0 * f1 + 2.0 * f2) / 6.0, (2.0 * f1 + 5.0 * f2 - f3) / 6.0,
                                 (11.0 * f2 - 7.0 * f3 + 2.0 * f4) / 6.0};
            vl = weno5_edge_exact(p, beta, d, variant, eps);
        }
    } else {
        R b[3], e, scale;
        weno5_scaled_beta(f0, f1, f2, f3, f4, eps, b, e, scale);
        R P[3];
        const R dR[3] = {R(0.1), R(0.6), R(0.3)}, dL[3] = {R(0.3), R(0.6), R(0.1)};
        R omR[3], omL[3];
        if (variant == WENO_Z) {
            const R tau = fabs(b[0] - b[2]);
            const R t0 = b[0] + e, t1 = b[1] + e, t2 = b[2] + e;
            P[0] = (t0 + tau) * (t1 * t2);
            P[1] = (t1 + tau) * (t0 * t2);
            P[2] = (t2 + tau) * (t0 * t1);
        } else {
            const R t0 = e + b[0], t1 = e + b[1], t2 = e + b[2];
            const R s0 = t0 * t0, s1 = t1 * t1, s2 = t2 * t2;
            P[0] = s1 * s2;
            P[1] = s0 * s2;
            P[2] = s0 * s1;
        }
        weno5_edge_weights(P, dR, variant, omR);
        weno5_edge_weights(P, dL, variant, omL);
        const R sixth = R(1.0 / 6.0);
        const R pr0 = (R(2) * f0 - R(7) * f1 + R(11) * f2) * sixth;
        const R pr1 = (-f1 + R(5) * f2 + R(2) * f3) * sixth;
        const R pr2 = (R(2) * f2 + R(5) * f3 - f4) * sixth;
        vr = omR[0] * pr0 + omR[1] * pr1 + omR[2] * pr2;
        const R pl0 = (-f0 + R(5) * f1 + R(2) * f2) * sixth;
        const R pl1 = (R(2) * f1 + R(5) * f2 - f3) * sixth;
        const R pl2 = (R(11) * f2 - R(7) * f3 + R(2) * f4) * sixth;
        vl = omL[0] * pl0 + omL[1] * pl1 + omL[2] * pl2;
    }
}

// HLLC flux across a face normal to axis DIR from reconstructed primitive
// states (Sec. 3.2.2).  Wave speeds min/max of u -/+ c over both sides
// (ties keep the left argument); S* from continuity of normal velocity and
// pressure; Toro's star states; S* >= 0 takes the left side.  The face
// velocity uf (u^{(x)} of Sec. 3.2.1) is u_K outside the fan and S* inside;
// the volume-fraction slots receive alpha_K uf.  bad is set when a squared
// sound speed is not positive.
template <int NF, int ND, int DIR, int MODE, class R = typename ModeT<MODE>::R>
__device__ __forceinline__ void hllc(const R* WL, const R* WR, const Consts& C, R* F, R& uf, bool& bad) {
    using L = Lay<NF, ND>;
    using A = Arith<MODE>;
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
        const R c2 = A::quot((Gamma + R(1)) * p[K] + Pi, Gamma * r);
        bad |= !(c2 > R(0));
        c[K] = sqrt(c2);
    }
    const R aL = un[0] - c[0], aR = un[1] - c[1];
    const R SL = (aR < aL) ? aR : aL;
    const R bL = un[0] + c[0], bR = un[1] + c[1];
    const R SR = (bR > bL) ? bR : bL;
    const R Ss = A::quot(p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1]),
                         rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]));

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
        const R chi = A::quot(SK - uK, SK - Ss);
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
        const R Es = chi * rK * (A::quot(EK, rK) + (Ss - uK) * (Ss + A::quot(pK, rK * (SK - uK))));
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
