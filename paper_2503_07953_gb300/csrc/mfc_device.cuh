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
//               conservative-to-primitive conversion stays float64;
//   MODE_DF     MODE_FAST with the WENO5 weights and candidate corrections
//               in double-float arithmetic (mfc_df64.cuh) on the float32
//               pipes; the Riemann solve and everything else stay in
//               MODE_FAST's float64, so both pipes work at once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mfc_df64.cuh"

namespace mfc {

constexpr int MAXF = 4;

enum { MODE_EXACT = 0, MODE_MIXED = 1, MODE_FAST = 2, MODE_DF = 3 };

// R: precision of the Riemann solve and flux difference; RW: precision of
// the primitive states the reconstruction reads.
template <int MODE> struct ModeT { using R = double; using RW = double; };
template <> struct ModeT<MODE_MIXED> { using R = float; using RW = float; };
template <> struct ModeT<MODE_DF> { using R = double; using RW = double; };

// Everything a kernel needs to know about the grid, layout and fluids.
// Passed by value as a kernel parameter.
struct Consts {
    int nf, nd, nq;
    int weno;                 // 0 JS, 1 mapped, 2 Z
    int64_t n[3];             // interior cells per axis (1 on inactive axes)
    int64_t stride[3];        // element stride of one cell step along x, y, z
    int64_t fstride;          // elements per field
    int64_t origin;           // element offset of interior cell (0, 0, 0)
    int bc_lo[3], bc_hi[3];   // 0 periodic, 1 transmissive, 2 reflective, 3 halo
    double dx[3], inv_dx[3];
    double g[MAXF], h[MAXF];  // 1/(gamma_i - 1), gamma_i pi_i/(gamma_i - 1)
    float gf[MAXF], hf[MAXF];
    double gd[MAXF], hd[MAXF];  // g_i - g_N, h_i - h_N (fast mixture rules)
    float gdf[MAXF], hdf[MAXF];
    float inv_dxf[3];
    double eps;
    float epsf;
    double teno_ct;           // TENO threshold C_T
    float teno_ctf;
    int model;                // 0: K = 0; 1: Kapila K div u (two fluids)
    int riemann;              // 0: HLLC; 1: HLL
    int low_mach;             // 0: none; 1: Thornber; 2: anti-dissipation pressure correction
    double gam[2], pinf[2];   // phasic gamma_i, pi_i of the two fluids (Kapila)
    float gamf[2], pinff[2];
    int viscous;              // 1 when some eta_i > 0 (Sec. 2.1.1 viscous stress)
    double eta[MAXF];         // phasic shear viscosities
    float etaf[MAXF];
    double cfl;
    int visc_dt;              // 1: the CFL dt also takes the explicit viscous limit
    double dx2min;            // min over active axes of dx_d^2
    double inv_dx2min;        // 1 / dx2min
};

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_HALO = 3 };
enum { WENO_JS = 0, WENO_M = 1, WENO_Z = 2, WENO_TENO = 3 };

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

// Reciprocal: in float64 the hardware approximation refined by one
// third-order step of the series 1/x = r / (1 - e) = r (1 + e + e^2 + ...),
// e = 1 - x r: r <- r + r (e + e^2), which cubes the relative error.  The
// approximation is within 2^-19.9 of 1/x (measured over 2^30 inputs of
// every exponent on GB300), so the result is within 2^-59 before its
// rounding: at most 1 ulp from the correctly rounded 1/x (same measurement).
// Three float64 operations, against four for two Newton-Raphson steps.  In
// float32 the fast approximate instruction.
__device__ __forceinline__ double rcp_nr(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
template <class R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ double rcp<double>(double x) { return rcp_nr(x); }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

// Sign tests and comparisons of float64 values on their bit patterns, with
// integer instructions: the float64 compare instructions occupy the float64
// pipe, which bounds the MODE_FAST and MODE_DF sweeps.  f64_pos, f64_neg and
// f64_nonneg equal x > 0, x < 0 and x >= 0 for every input, NaN included;
// f64_lt orders like a < b except that -0 is below +0 and NaN above +inf
// (it picks the sign of a zero in a minimum; NaN only arises in states that
// are reported non-physical).
__device__ __forceinline__ bool f64_pos(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b - 1ULL < 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool f64_neg(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) ^ 0x8000000000000000ULL;
    return b - 1ULL < 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool f64_nonneg(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b <= 0x7ff0000000000000ULL || b == 0x8000000000000000ULL;
}
__device__ __forceinline__ long long f64_key(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool f64_lt(double a, double b) { return f64_key(a) < f64_key(b); }

// The comparisons of the sweeps by arithmetic mode: on bit patterns for the
// float64 values of MODE_FAST and MODE_DF, the compare instructions
// otherwise (MODE_EXACT keeps the IEEE comparisons the oracle makes).
template <int MODE, class R> struct Cmp {
    static __device__ __forceinline__ bool pos(R x) { return x > R(0); }
    static __device__ __forceinline__ bool neg(R x) { return x < R(0); }
    static __device__ __forceinline__ bool nonneg(R x) { return x >= R(0); }
    static __device__ __forceinline__ bool lt(R a, R b) { return a < b; }
};
template <> struct Cmp<MODE_FAST, double> {
    static __device__ __forceinline__ bool pos(double x) { return f64_pos(x); }
    static __device__ __forceinline__ bool neg(double x) { return f64_neg(x); }
    static __device__ __forceinline__ bool nonneg(double x) { return f64_nonneg(x); }
    static __device__ __forceinline__ bool lt(double a, double b) { return f64_lt(a, b); }
};
template <> struct Cmp<MODE_DF, double> : Cmp<MODE_FAST, double> {};

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

// Phasic constant i of the precision R (float64 / float32 copies).
template <class R> __device__ __forceinline__ R phasic(const double* d, const float* f, int i);
template <> __device__ __forceinline__ double phasic<double>(const double* d, const float*, int i) { return d[i]; }
template <> __device__ __forceinline__ float phasic<float>(const double*, const float* f, int i) { return f[i]; }

// Kapila model, two fluids (Sec. 2.1.1): with Z_i = gamma_i (p + pi_i)
// (= rho_i c_i^2 of the phasic sound speeds),
//   K = (Z_2 - Z_1) / (Z_1/alpha_1 + Z_2/alpha_2)
// and the Wood mixture sound speed 1/(rho c^2) = alpha_1/Z_1 + alpha_2/Z_2,
// in the order of these formulas (MODE_EXACT) or with fast quotients.
template <int MODE, class R>
__device__ __forceinline__ R kapila_K(R p, R a1, const Consts& C) {
    using A = Arith<MODE>;
    const R Z1 = phasic<R>(C.gam, C.gamf, 0) * (p + phasic<R>(C.pinf, C.pinff, 0));
    const R Z2 = phasic<R>(C.gam, C.gamf, 1) * (p + phasic<R>(C.pinf, C.pinff, 1));
    const R a2 = R(1) - a1;
    return A::quot(Z2 - Z1, A::quot(Z1, a1) + A::quot(Z2, a2));
}

template <int MODE, class R>
__device__ __forceinline__ R wood_c2(R rho, R p, R a1, const Consts& C) {
    using A = Arith<MODE>;
    const R Z1 = phasic<R>(C.gam, C.gamf, 0) * (p + phasic<R>(C.pinf, C.pinff, 0));
    const R Z2 = phasic<R>(C.gam, C.gamf, 1) * (p + phasic<R>(C.pinf, C.pinff, 1));
    const R a2 = R(1) - a1;
    return A::quot(R(1), rho * (A::quot(a1, Z1) + A::quot(a2, Z2)));
}

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

// The same mixture rules with alpha_N eliminated: Gamma = g_N + sum_j
// alpha_j (g_j - g_N), Pi likewise, as fused multiply-adds (MODE_MIXED).
// The float64 modes keep the form above: with stiff fluids Pi ~ 1e9 is
// cancelled against p ~ 1e5 in the pressure recovery, and a different
// rounding of Pi shows up in the right-hand side at ~1e-11.
template <int NF, int MODE, class R>
__device__ __forceinline__ void mixture_mode(const R* alpha, const Consts& C, R& Gamma, R& Pi) {
    if constexpr (MODE != MODE_MIXED) {
        mixture<NF, R>(alpha, C, Gamma, Pi);
    } else if constexpr (sizeof(R) == 8) {
        Gamma = C.g[NF - 1];
        Pi = C.h[NF - 1];
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) {
            Gamma = fma(alpha[j], C.gd[j], Gamma);
            Pi = fma(alpha[j], C.hd[j], Pi);
        }
    } else {
        Gamma = C.gf[NF - 1];
        Pi = C.hf[NF - 1];
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) {
            Gamma = fmaf(alpha[j], C.gdf[j], Gamma);
            Pi = fmaf(alpha[j], C.hdf[j], Pi);
        }
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
    bad |= !Cmp<MODE, double>::pos(rho);
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
    mixture_mode<NF, MODE, double>(q + L::A, C, Gamma, Pi);
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
        // Pi = h_N + sum_j alpha_j (h_j - h_N): N_f - 1 fused multiply-adds
        // in float64; Gamma the same way in float32
        double Pi = C.h[NF - 1];
        float Gamma = C.gf[NF - 1];
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) {
            Pi = fma(q[L::A + j], C.hd[j], Pi);
            out[L::A + j] = float(q[L::A + j]);
            Gamma = fmaf(out[L::A + j], C.gdf[j], Gamma);
        }
        const double num = (q[L::E] - Pi) - double(ke);
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
// The mixture quantities of one primitive state that both the physical-state
// test and the Riemann solver use: rho, Gamma, Pi and num = (Gamma + 1) p + Pi
// (Gamma rho c^2 of the mixture stiffened gas), computed once per state.
template <class R>
struct MixState {
    R rho, G, P, num;
};

template <int NF, int ND, int MODE, class R>
__device__ __forceinline__ MixState<R> mix_state(const R* w, const Consts& C) {
    using L = Lay<NF, ND>;
    MixState<R> m;
    R rho = w[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) rho = rho + w[i];
    mixture_mode<NF, MODE, R>(w + L::A, C, m.G, m.P);
    m.rho = rho;
    m.num = (m.G + R(1)) * w[L::E] + m.P;
    return m;
}

template <int NF, int ND, class R, int MODE = MODE_EXACT>
__device__ __forceinline__ bool physical_mix(const R* w, const MixState<R>& m, const Consts& C) {
    using L = Lay<NF, ND>;
    using K = Cmp<MODE, R>;
    bool ok = K::pos(m.rho) && K::pos(m.G) && K::pos(m.num);
    if constexpr (NF == 2) {
        // Kapila: both phasic impedances gamma_i (p + pi_i) positive
        if (C.model == 1) ok = ok && w[L::E] + phasic<R>(C.pinf, C.pinff, 0) > R(0) &&
                               w[L::E] + phasic<R>(C.pinf, C.pinff, 1) > R(0);
    }
    return ok;
}

template <int NF, int ND, class R, int MODE = MODE_EXACT>
__device__ __forceinline__ bool physical_state(const R* w, const Consts& C) {
    return physical_mix<NF, ND, R, MODE>(w, mix_state<NF, ND, MODE, R>(w, C), C);
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
// TENO stencil selection of one edge (Sec. 4.2.2) in the MODE_EXACT order:
// gamma_r = d_r A_r^6, A_r = 1 + tau/(beta_r + eps), evaluated with
// A_r / max A; a stencil whose share chi_r of gamma is below C_T gets
// a_r = 0, the others a_r = d_r.
__device__ __forceinline__ void teno_select_exact(const double* beta, const double* d, double eps, double ct,
                                                  double* a) {
    const double tau = fabs(beta[0] - beta[2]);
    double A[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) A[r] = 1.0 + tau / (beta[r] + eps);
    double Am = (A[1] > A[0]) ? A[1] : A[0];
    Am = (A[2] > Am) ? A[2] : Am;
    double g[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double x = A[r] / Am;
        const double x2 = x * x;
        g[r] = d[r] * (x2 * x2 * x2);
    }
    const double sg = g[0] + g[1] + g[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) a[r] = (g[r] / sg < ct) ? 0.0 : d[r];
}

__device__ __forceinline__ double weno5_edge_exact(const double* p, const double* beta, const double* d,
                                                   int variant, double eps, double ct) {
    double a[3], w[3];
    if (variant == WENO_Z) {
        const double tau = fabs(beta[0] - beta[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) a[r] = d[r] * (1.0 + tau / (beta[r] + eps));
    } else if (variant == WENO_TENO) {
        teno_select_exact(beta, d, eps, ct, a);
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

// TENO weights of both edges in the MODE_FAST / MODE_MIXED arithmetic:
// x_r = A_r / max A with A_r = 1 + tau/(b_r + e) (one reciprocal per
// stencil and one for the maximum), gamma_r = d_r x_r^6 per edge, stencil r
// off when gamma_r < C_T sum gamma, weights d_r renormalised over the
// stencils that stay on.
template <class R>
__device__ __forceinline__ void teno_weights(const R* b, R e, R ct, const R* dR, const R* dL, R* omR, R* omL) {
    const R tau = fabs(b[0] - b[2]);
    R A[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) A[r] = R(1) + tau * rcp<R>(b[r] + e);
    R Am = (A[1] > A[0]) ? A[1] : A[0];
    Am = (A[2] > Am) ? A[2] : Am;
    const R iAm = rcp<R>(Am);
    R x6[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const R x = A[r] * iAm;
        const R x2 = x * x;
        x6[r] = x2 * x2 * x2;
    }
    const R* ds[2] = {dR, dL};
    R* oms[2] = {omR, omL};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const R* d = ds[s];
        const R g0 = d[0] * x6[0], g1 = d[1] * x6[1], g2 = d[2] * x6[2];
        const R lim = ct * (g0 + g1 + g2);
        const R a0 = (g0 < lim) ? R(0) : d[0];
        const R a1 = (g1 < lim) ? R(0) : d[1];
        const R a2 = (g2 < lim) ? R(0) : d[2];
        const R inv = rcp<R>(a0 + a1 + a2);
        oms[s][0] = a0 * inv;
        oms[s][1] = a1 * inv;
        oms[s][2] = a2 * inv;
    }
}

// MODE_DF: WENO5 of one cell in double-float arithmetic, the same
// smoothness indicators, candidate polynomials and weight functions as the
// float64 modes, written on the consecutive differences D_j = f_{j+1} - f_j
// of the stencil (taken in float64, then carried as double-float): the
// indicators depend only on differences, and each candidate value is
// f2 + (a combination of differences) / 6, because the candidate
// coefficients sum to one.  So constant data reconstruct exactly, and the
// double-float rounding applies to the corrections, not to the values.
// The weights depend only on ratios of t_r = eps + beta_r.  The t_r are
// scaled by the power of two that brings the largest into [1, 2) (exact)
// and floored at 2^-120; JS and mapped use u_r = t_min / t_r in (0, 1]
// (alpha_r = d_r u_r^2), Z and TENO use A_r = 1 + tau / t_r divided by
// max A, so no weight or normaliser leaves the normal float32 range where
// it matters.  The floor only moves weight between stencils whose
// indicators are below 2^-120 of the largest, and the candidates of two
// such stencils differ by at most (sqrt(beta_r) + sqrt(beta_s)) / 3 <
// 2^-60 sqrt(beta_max).  When every t_r is below 2^-120 (data flat to
// ~1e-18) the ideal weights are used, which is what alpha_r = d_r / eps^2
// gives.  e and cT are eps and C_T as double-float.  bad is set when an
// indicator overflows the float32 range (differences above ~1e18).  One call per field: not inlined, so a single
// copy of its code serves all fields from the instruction cache; the
// result is returned by value so that it stays in registers.
struct WenoEdges {
    double vl, vr;
    int bad;
};

static __device__ __noinline__ WenoEdges weno5_cell_df(double f0, double f1, double f2, double f3, double f4,
                                                       int variant, df64 e, df64 cT) {
    constexpr df64 c13(13.0 / 12.0), sixth(1.0 / 6.0), one(1.0);
    const df64 D01 = df_from_f64_bits(f1 - f0), D12 = df_from_f64_bits(f2 - f1);
    const df64 D23 = df_from_f64_bits(f3 - f2), D34 = df_from_f64_bits(f4 - f3);
    // smoothness indicators: beta_r = 13/12 a_r^2 + 1/4 g_r^2
    const df64 a0 = D12 - D01, g0 = df_mulf(D12, 3.0f) - D01;
    const df64 a1 = D23 - D12, g1 = D12 + D23;
    const df64 a2 = D34 - D23, g2 = D34 - df_mulf(D23, 3.0f);
    df64 t[3];
    t[0] = e + (c13 * (a0 * a0) + df_scale(g0 * g0, 0.25f));
    t[1] = e + (c13 * (a1 * a1) + df_scale(g1 * g1, 0.25f));
    t[2] = e + (c13 * (a2 * a2) + df_scale(g2 * g2, 0.25f));
    // 6 (candidate - f2) at the right (P) and left (Q) edges
    const df64 P[3] = {df_mulf(D12, 5.0f) - df_scale(D01, 2.0f), D12 + df_scale(D23, 2.0f),
                       df_scale(D23, 4.0f) - D34};
    const df64 Q[3] = {D01 - df_scale(D12, 4.0f), -(df_scale(D12, 2.0f) + D23),
                       df_scale(D34, 2.0f) - df_mulf(D23, 5.0f)};
    const double dR[3] = {0.1, 0.6, 0.3}, dL[3] = {0.3, 0.6, 0.1};
    // the weights of the (right, left) edges, stencil by stencil
    df64x2 om[3];
    const float th = fmaxf(fmaxf(t[0].hi, t[1].hi), t[2].hi);
    WenoEdges out;
    // an indicator that overflowed is inf or NaN, and so is the sum
    out.bad = !((t[0].hi + t[1].hi) + t[2].hi <= 0x1.fffffep127f);
    if (!(th >= 0x1p-120f)) {
#pragma unroll
        for (int r = 0; r < 3; ++r) om[r] = dfx2(dR[r], dL[r]);
    } else {
        int k = ((__float_as_int(th) >> 23) & 0xff) - 127;
        k = k > 126 ? 126 : k;
        const float s = __int_as_float((127 - k) << 23);
        df64 ts[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ts[r] = df_scale(t[r], s);
            if (ts[r].hi < 0x1p-120f) ts[r] = df64(0x1p-120f, 0.0f);
        }
        if (variant == WENO_Z || variant == WENO_TENO) {
            // A_r = 1 + tau / t_r with tau = |beta_0 - beta_2|, as B_r = A_r / max A
            const df64 tau = df_abs(df_scale(t[0], s) - df_scale(t[2], s));
            df64 B[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) B[r] = one + df_div(tau, ts[r]);
            df64 Am = (B[1] > B[0]) ? B[1] : B[0];
            Am = (B[2] > Am) ? B[2] : Am;
            const df64 iAm = df_div(one, Am);
#pragma unroll
            for (int r = 0; r < 3; ++r) B[r] = B[r] * iAm;
            if (variant == WENO_Z) {
                df64x2 x[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) x[r] = dfx2(dR[r], dL[r]) * dfx2(B[r], B[r]);
                const df64x2 inv = df_rcp((x[0] + x[1]) + x[2]);
#pragma unroll
                for (int r = 0; r < 3; ++r) om[r] = x[r] * inv;
            } else {
                // TENO: gamma_r = d_r B_r^6; stencil r off when gamma_r < C_T sum
                // gamma, the others at d_r renormalised
                df64 x6[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const df64 x2 = B[r] * B[r];
                    x6[r] = x2 * (x2 * x2);
                }
                df64 omR[3], omL[3];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const double* d = side ? dL : dR;
                    df64* os = side ? omL : omR;
                    const df64 y0 = df64(d[0]) * x6[0], y1 = df64(d[1]) * x6[1], y2 = df64(d[2]) * x6[2];
                    const df64 lim = cT * ((y0 + y1) + y2);
                    const df64 b0 = (y0 < lim) ? df64(0.0) : df64(d[0]);
                    const df64 b1 = (y1 < lim) ? df64(0.0) : df64(d[1]);
                    const df64 b2 = (y2 < lim) ? df64(0.0) : df64(d[2]);
                    const df64 inv = df_div(one, (b0 + b1) + b2);
                    os[0] = b0 * inv;
                    os[1] = b1 * inv;
                    os[2] = b2 * inv;
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) om[r] = dfx2(omR[r], omL[r]);
            }
        } else {
            // JS and mapped: alpha_r proportional to d_r (t_min / t_r)^2
            const float tmh = fminf(fminf(ts[0].hi, ts[1].hi), ts[2].hi);
            const df64 tmin = (ts[0].hi == tmh) ? ts[0] : ((ts[1].hi == tmh) ? ts[1] : ts[2]);
            df64 u2[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const df64 u = df_div(tmin, ts[r]);
                u2[r] = u * u;
            }
            // both edges at once, the right edge in lane x, the left in lane y
            df64x2 w[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) w[r] = dfx2(dR[r], dL[r]) * dfx2(u2[r], u2[r]);
            df64x2 inv = df_rcp((w[0] + w[1]) + w[2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) w[r] = w[r] * inv;
            if (variant == WENO_M) {
                // g_r(w) = w (d + d^2 - 3 d w + w^2) / (d^2 + w (1 - 2 d)), renormalised
                df64x2 N[3], D[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    N[r] = w[r] * (dfx2(dR[r] * (1.0 + dR[r]), dL[r] * (1.0 + dL[r])) +
                                   w[r] * (w[r] - dfx2(3.0 * dR[r], 3.0 * dL[r])));
                    D[r] = dfx2(dR[r] * dR[r], dL[r] * dL[r]) + w[r] * dfx2(1.0 - 2.0 * dR[r], 1.0 - 2.0 * dL[r]);
                }
                const df64x2 gm0 = N[0] * (D[1] * D[2]), gm1 = N[1] * (D[0] * D[2]), gm2 = N[2] * (D[0] * D[1]);
                inv = df_rcp((gm0 + gm1) + gm2);
                w[0] = gm0 * inv;
                w[1] = gm1 * inv;
                w[2] = gm2 * inv;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) om[r] = w[r];
        }
    }
    const df64x2 c = ((om[0] * dfx2(P[0], Q[0]) + om[1] * dfx2(P[1], Q[1])) + om[2] * dfx2(P[2], Q[2])) *
                     dfx2(sixth, sixth);
    const df64 cr = lane_x(c), cl = lane_y(c);
    out.vr = f2 + (f64_from_f32_bits(cr.hi) + f64_from_f32_bits(cr.lo));
    out.vl = f2 + (f64_from_f32_bits(cl.hi) + f64_from_f32_bits(cl.lo));
    return out;
}

// MODE_FAST WENO5 of one cell (JS, mapped and Z weights), arranged for few
// float64 operations.  With the consecutive differences D_j = f_{j+1} - f_j
// of the stencil, substencil r has the second difference a_r (a_0 = D12 -
// D01, a_1 = D23 - D12, a_2 = D34 - D23) and the first difference g_r
// (g_0 = 3 D12 - D01, g_1 = D12 + D23, g_2 = D34 - 3 D23), and the k = 3
// candidate polynomials and smoothness indicators of Sec. 4.2.2 become
//   4 beta_r = (13/3) a_r^2 + g_r^2,
//   12 (right-edge candidate_r - f2) = a_r + 3 s_r g_r,   s = (+1, +1, -1),
//   12 (left-edge candidate_r - f2)  = a_r - 3 s_r g_r.
// The weights depend only on ratios of eps + beta_r, so they are evaluated
// on t_r = 4 (eps + beta_r).  Each edge value is f2 + sum_r omega_r
// (candidate_r - f2), so constant data reconstruct exactly and the rounding
// of the weights only touches the correction.  Unnormalised weights: JS
// alpha_r = d_r prod_{s != r} t_s^2 (alpha_r = d_r / t_r^2 times the product
// of all t_s^2); mapped (Henrick 2005) g(w) = w (d + d^2 + w (w - 3 d)) /
// (d^2 + w (1 - 2 d)) of the normalised JS weights w, as numerator times the
// other two stencils' denominators; Z d_r (t_r + tau) prod_{s != r} t_s.
// The mapped weights of the two edges sum to within [5e-6, 3] each, so their
// normalisations share one reciprocal.
// The part of weno5_cell_fast64 that is not shared with the neighbouring
// cells: from the centre value f2, the differences D01 .. D34, the second
// differences a_r and the partial indicators A_r = (13/3) a_r^2 + 4 eps
// (which a march along a line carries over from the previous cell, shifted
// by one stencil).
__device__ __forceinline__ void weno5_fast64_core(double f2, double D01, double D12, double D23, double D34,
                                                  const double* a, const double* A, int variant, double& vl,
                                                  double& vr) {
    const double g[3] = {fma(3.0, D12, -D01), D12 + D23, fma(-3.0, D23, D34)};
    double t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = fma(g[r], g[r], A[r]);
    const double cR[3] = {fma(3.0, g[0], a[0]), fma(3.0, g[1], a[1]), fma(-3.0, g[2], a[2])};
    const double cL[3] = {fma(-3.0, g[0], a[0]), fma(-3.0, g[1], a[1]), fma(3.0, g[2], a[2])};
    double wR[3], wL[3], nR, nL;
    if (variant == WENO_Z) {
        const double tau = fabs(t[0] - t[2]);
        const double P0 = (t[0] + tau) * (t[1] * t[2]), P1 = (t[1] + tau) * (t[0] * t[2]);
        const double P2 = (t[2] + tau) * (t[0] * t[1]);
        const double m1 = 0.6 * P1;
        wR[0] = 0.1 * P0, wR[1] = m1, wR[2] = 0.3 * P2;
        wL[0] = 0.3 * P0, wL[1] = m1, wL[2] = 0.1 * P2;
    } else {
        const double s0 = t[0] * t[0], s1 = t[1] * t[1], s2 = t[2] * t[2];
        const double P0 = s1 * s2, P1 = s0 * s2, P2 = s0 * s1;
        const double m1 = 0.6 * P1;
        wR[0] = 0.1 * P0, wR[1] = m1, wR[2] = 0.3 * P2;
        wL[0] = 0.3 * P0, wL[1] = m1, wL[2] = 0.1 * P2;
    }
    nR = (wR[0] + wR[1]) + wR[2];
    nL = (wL[0] + wL[1]) + wL[2];
    double iR, iL;
    if (variant == WENO_M) {
        const double dR[3] = {0.1, 0.6, 0.3}, dL[3] = {0.3, 0.6, 0.1};
        double* ws[2] = {wR, wL};
        double* ns[2] = {&nR, &nL};
        const double* ds[2] = {dR, dL};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            double* w = ws[side];
            const double* d = ds[side];
            const double inv = rcp_nr(*ns[side]);
            double N[3], D[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double x = w[r] * inv;
                N[r] = x * fma(x, x - 3.0 * d[r], d[r] * (1.0 + d[r]));
                D[r] = fma(x, 1.0 - 2.0 * d[r], d[r] * d[r]);
            }
            w[0] = N[0] * (D[1] * D[2]);
            w[1] = N[1] * (D[0] * D[2]);
            w[2] = N[2] * (D[0] * D[1]);
            *ns[side] = (w[0] + w[1]) + w[2];
        }
        // 1 / (12 nR nL): nL / (12 nR nL) = 1 / (12 nR) and nR / (12 nR nL) = 1 / (12 nL)
        const double r = rcp_nr((12.0 * nR) * nL);
        iR = nL * r;
        iL = nR * r;
    } else {
        iR = rcp_nr(12.0 * nR);
        iL = rcp_nr(12.0 * nL);
    }
    const double sR = fma(wR[2], cR[2], fma(wR[1], cR[1], wR[0] * cR[0]));
    const double sL = fma(wL[2], cL[2], fma(wL[1], cL[1], wL[0] * cL[0]));
    vr = fma(iR, sR, f2);
    vl = fma(iL, sL, f2);
}

// (13/3) a^2 + 4 eps, the part of 4 (eps + beta_r) that depends on the
// second difference alone
__device__ __forceinline__ double weno5_fast64_A(double a, double e4) { return fma((13.0 / 3.0) * a, a, e4); }

__device__ __forceinline__ void weno5_cell_fast64(double f0, double f1, double f2, double f3, double f4, int variant,
                                                  double eps, double& vl, double& vr) {
    const double D01 = f1 - f0, D12 = f2 - f1, D23 = f3 - f2, D34 = f4 - f3;
    const double a[3] = {D12 - D01, D23 - D12, D34 - D23};
    const double e4 = 4.0 * eps;
    const double A[3] = {weno5_fast64_A(a[0], e4), weno5_fast64_A(a[1], e4), weno5_fast64_A(a[2], e4)};
    weno5_fast64_core(f2, D01, D12, D23, D34, a, A, variant, vl, vr);
}

// MODE_MIXED WENO5 of one cell (JS, mapped and Z weights) in float32: the
// formulation of weno5_cell_fast64 on consecutive differences, with the
// indicators divided by their sum and eps floored at 1e-9 of it (as
// weno5_scaled_beta does, so that every product of the weights stays inside
// the float32 range), and the right- and left-edge weights carried as the two
// lanes of float2 values: each paired add, multiply or fused multiply-add is
// one instruction for both edges (FADD2 / FMUL2 / FFMA2).
__device__ __forceinline__ float2 pair(float r, float l) { return make_float2(r, l); }

//
// Not inlined: one copy of its code serves the N_q fields of a cell from the
// instruction cache (inlined, the sweeps' loop bodies stalled on instruction
// fetch); the edge values come back in registers.
static __device__ __noinline__ float2 weno5_cell_mixed32(float f0, float f1, float f2, float f3, float f4,
                                                         int variant, float eps) {
    const float D01 = f1 - f0, D12 = f2 - f1, D23 = f3 - f2, D34 = f4 - f3;
    const float a[3] = {D12 - D01, D23 - D12, D34 - D23};
    const float g[3] = {fmaf(3.0f, D12, -D01), D12 + D23, fmaf(-3.0f, D23, D34)};
    float b[3];  // 4 beta_r
#pragma unroll
    for (int r = 0; r < 3; ++r) b[r] = fmaf((13.0f / 3.0f) * a[r], a[r], g[r] * g[r]);
    const float scale = __fdividef(1.0f, (b[0] + b[1]) + (b[2] + 4e-30f));
    const float e = fmaxf(4.0f * eps * scale, 1e-9f);
    float t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = fmaf(b[r], scale, e);
    float P[3];
    if (variant == WENO_Z) {
        const float tau = fabsf(t[0] - t[2]);
        P[0] = (t[0] + tau) * (t[1] * t[2]);
        P[1] = (t[1] + tau) * (t[0] * t[2]);
        P[2] = (t[2] + tau) * (t[0] * t[1]);
    } else {
        const float s0 = t[0] * t[0], s1 = t[1] * t[1], s2 = t[2] * t[2];
        P[0] = s1 * s2;
        P[1] = s0 * s2;
        P[2] = s0 * s1;
    }
    // (right, left) unnormalised weights: alpha_r = d_r P_r
    const float2 d0 = pair(0.1f, 0.3f), d1 = pair(0.6f, 0.6f), d2 = pair(0.3f, 0.1f);
    float2 w0 = __fmul2_rn(d0, pair(P[0], P[0]));
    float2 w1 = __fmul2_rn(d1, pair(P[1], P[1]));
    float2 w2 = __fmul2_rn(d2, pair(P[2], P[2]));
    float2 nrm = __fadd2_rn(__fadd2_rn(w0, w1), w2);
    float2 inv;
    if (variant == WENO_M) {
        // Henrick's map of the normalised JS weights x: numerator
        // x (d + d^2 + x (x - 3 d)) times the other stencils' denominators
        // d^2 + x (1 - 2 d)
        inv = pair(__fdividef(1.0f, nrm.x), __fdividef(1.0f, nrm.y));
        const float2 x0 = __fmul2_rn(w0, inv), x1 = __fmul2_rn(w1, inv), x2 = __fmul2_rn(w2, inv);
        const float2 N0 = __fmul2_rn(x0, __ffma2_rn(x0, __fadd2_rn(x0, pair(-0.3f, -0.9f)), pair(0.11f, 0.39f)));
        const float2 N1 = __fmul2_rn(x1, __ffma2_rn(x1, __fadd2_rn(x1, pair(-1.8f, -1.8f)), pair(0.96f, 0.96f)));
        const float2 N2 = __fmul2_rn(x2, __ffma2_rn(x2, __fadd2_rn(x2, pair(-0.9f, -0.3f)), pair(0.39f, 0.11f)));
        const float2 E0 = __ffma2_rn(x0, pair(0.8f, 0.4f), pair(0.01f, 0.09f));
        const float2 E1 = __ffma2_rn(x1, pair(-0.2f, -0.2f), pair(0.36f, 0.36f));
        const float2 E2 = __ffma2_rn(x2, pair(0.4f, 0.8f), pair(0.09f, 0.01f));
        w0 = __fmul2_rn(N0, __fmul2_rn(E1, E2));
        w1 = __fmul2_rn(N1, __fmul2_rn(E0, E2));
        w2 = __fmul2_rn(N2, __fmul2_rn(E0, E1));
        nrm = __fadd2_rn(__fadd2_rn(w0, w1), w2);
    }
    // 1 / (12 n) per edge
    inv = pair(__fdividef(1.0f, 12.0f * nrm.x), __fdividef(1.0f, 12.0f * nrm.y));
    // 12 (candidate_r - f2) of the (right, left) edges: a_r +- 3 s_r g_r
    const float2 c0 = __ffma2_rn(pair(3.0f, -3.0f), pair(g[0], g[0]), pair(a[0], a[0]));
    const float2 c1 = __ffma2_rn(pair(3.0f, -3.0f), pair(g[1], g[1]), pair(a[1], a[1]));
    const float2 c2 = __ffma2_rn(pair(-3.0f, 3.0f), pair(g[2], g[2]), pair(a[2], a[2]));
    const float2 sum = __ffma2_rn(w2, c2, __ffma2_rn(w1, c1, __fmul2_rn(w0, c0)));
    return __ffma2_rn(inv, sum, pair(f2, f2));  // (right edge, left edge)
}

// weno5_cell_mixed32 of two fields A and B at once (JS, mapped and Z
// weights): the per-field scalar steps (differences, indicators and their
// scaling, the products P_r) run as float2 instructions on the pair (A, B),
// and each field's edge-paired weights follow as in weno5_cell_mixed32, the
// two fields' chains interleaved.  Every lane performs the single-field
// function's operations with the same roundings (x - y as fma(y, -1, x) is
// the same rounded difference), so the results are bit for bit those of two
// weno5_cell_mixed32 calls.  Not inlined, like weno5_cell_mixed32.
struct WenoPair32 {
    float2 a, b;  // (right edge, left edge) of fields A and B
};

__device__ __forceinline__ float2 fsub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.0f, -1.0f), x); }

// The edge-paired weights and edge values of one field from its P_r, the
// differences' a_r and g_r, and the centre value f2.
__device__ __forceinline__ float2 weno5_mixed32_edges(float P0, float P1, float P2, float a0, float a1, float a2,
                                                      float g0, float g1, float g2, float f2, int variant) {
    const float2 d0 = pair(0.1f, 0.3f), d1 = pair(0.6f, 0.6f), d2 = pair(0.3f, 0.1f);
    float2 w0 = __fmul2_rn(d0, pair(P0, P0));
    float2 w1 = __fmul2_rn(d1, pair(P1, P1));
    float2 w2 = __fmul2_rn(d2, pair(P2, P2));
    float2 nrm = __fadd2_rn(__fadd2_rn(w0, w1), w2);
    float2 inv;
    if (variant == WENO_M) {
        inv = pair(__fdividef(1.0f, nrm.x), __fdividef(1.0f, nrm.y));
        const float2 x0 = __fmul2_rn(w0, inv), x1 = __fmul2_rn(w1, inv), x2 = __fmul2_rn(w2, inv);
        const float2 N0 = __fmul2_rn(x0, __ffma2_rn(x0, __fadd2_rn(x0, pair(-0.3f, -0.9f)), pair(0.11f, 0.39f)));
        const float2 N1 = __fmul2_rn(x1, __ffma2_rn(x1, __fadd2_rn(x1, pair(-1.8f, -1.8f)), pair(0.96f, 0.96f)));
        const float2 N2 = __fmul2_rn(x2, __ffma2_rn(x2, __fadd2_rn(x2, pair(-0.9f, -0.3f)), pair(0.39f, 0.11f)));
        const float2 E0 = __ffma2_rn(x0, pair(0.8f, 0.4f), pair(0.01f, 0.09f));
        const float2 E1 = __ffma2_rn(x1, pair(-0.2f, -0.2f), pair(0.36f, 0.36f));
        const float2 E2 = __ffma2_rn(x2, pair(0.4f, 0.8f), pair(0.09f, 0.01f));
        w0 = __fmul2_rn(N0, __fmul2_rn(E1, E2));
        w1 = __fmul2_rn(N1, __fmul2_rn(E0, E2));
        w2 = __fmul2_rn(N2, __fmul2_rn(E0, E1));
        nrm = __fadd2_rn(__fadd2_rn(w0, w1), w2);
    }
    inv = pair(__fdividef(1.0f, 12.0f * nrm.x), __fdividef(1.0f, 12.0f * nrm.y));
    const float2 c0 = __ffma2_rn(pair(3.0f, -3.0f), pair(g0, g0), pair(a0, a0));
    const float2 c1 = __ffma2_rn(pair(3.0f, -3.0f), pair(g1, g1), pair(a1, a1));
    const float2 c2 = __ffma2_rn(pair(-3.0f, 3.0f), pair(g2, g2), pair(a2, a2));
    const float2 sum = __ffma2_rn(w2, c2, __ffma2_rn(w1, c1, __fmul2_rn(w0, c0)));
    return __ffma2_rn(inv, sum, pair(f2, f2));
}

static __device__ __noinline__ WenoPair32 weno5_cells_mixed32_x2(float fa0, float fa1, float fa2, float fa3,
                                                                 float fa4, float fb0, float fb1, float fb2,
                                                                 float fb3, float fb4, int variant, float eps) {
    const float2 F0 = pair(fa0, fb0), F1 = pair(fa1, fb1), F2 = pair(fa2, fb2), F3 = pair(fa3, fb3),
                 F4 = pair(fa4, fb4);
    // -D01 (= f0 - f1, the same rounding as -(f1 - f0)), D12, D23, D34
    const float2 nD01 = fsub2(F0, F1), D12 = fsub2(F2, F1), D23 = fsub2(F3, F2), D34 = fsub2(F4, F3);
    const float2 a[3] = {__fadd2_rn(D12, nD01), fsub2(D23, D12), fsub2(D34, D23)};
    const float2 g[3] = {__ffma2_rn(pair(3.0f, 3.0f), D12, nD01), __fadd2_rn(D12, D23),
                         __ffma2_rn(pair(-3.0f, -3.0f), D23, D34)};
    float2 b[3];  // 4 beta_r
#pragma unroll
    for (int r = 0; r < 3; ++r)
        b[r] = __ffma2_rn(__fmul2_rn(pair(13.0f / 3.0f, 13.0f / 3.0f), a[r]), a[r], __fmul2_rn(g[r], g[r]));
    const float2 den = __fadd2_rn(__fadd2_rn(b[0], b[1]), __fadd2_rn(b[2], pair(4e-30f, 4e-30f)));
    const float2 scale = pair(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
    const float e4 = 4.0f * eps;
    const float2 e0 = __fmul2_rn(pair(e4, e4), scale);
    const float2 e = pair(fmaxf(e0.x, 1e-9f), fmaxf(e0.y, 1e-9f));
    float2 t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = __ffma2_rn(b[r], scale, e);
    float2 P[3];
    if (variant == WENO_Z) {
        const float2 dt = fsub2(t[0], t[2]);
        const float2 tau = pair(fabsf(dt.x), fabsf(dt.y));
        P[0] = __fmul2_rn(__fadd2_rn(t[0], tau), __fmul2_rn(t[1], t[2]));
        P[1] = __fmul2_rn(__fadd2_rn(t[1], tau), __fmul2_rn(t[0], t[2]));
        P[2] = __fmul2_rn(__fadd2_rn(t[2], tau), __fmul2_rn(t[0], t[1]));
    } else {
        const float2 s0 = __fmul2_rn(t[0], t[0]), s1 = __fmul2_rn(t[1], t[1]), s2 = __fmul2_rn(t[2], t[2]);
        P[0] = __fmul2_rn(s1, s2);
        P[1] = __fmul2_rn(s0, s2);
        P[2] = __fmul2_rn(s0, s1);
    }
    WenoPair32 out;
    out.a = weno5_mixed32_edges(P[0].x, P[1].x, P[2].x, a[0].x, a[1].x, a[2].x, g[0].x, g[1].x, g[2].x, fa2, variant);
    out.b = weno5_mixed32_edges(P[0].y, P[1].y, P[2].y, a[0].y, a[1].y, a[2].y, g[0].y, g[1].y, g[2].y, fb2, variant);
    return out;
}

// MODE_MIXED WENO5 of the NQ fields of a cell: f0..f4 the stencil (each
// [NQ]); vl, vr the left- and right-edge values.  Fields go two at a time
// through weno5_cells_mixed32_x2 (an odd last one through
// weno5_cell_mixed32); TENO field by field.
template <int NQ>
__device__ __forceinline__ void weno5_fields_mixed32(const float* f0, const float* f1, const float* f2,
                                                     const float* f3, const float* f4, int variant, float eps,
                                                     float ct, float* vl, float* vr);

template <int MODE, class R>
__device__ __forceinline__ void weno5_cell(R f0, R f1, R f2, R f3, R f4, int variant, R eps, R ct, R& vl, R& vr) {
    if constexpr (MODE == MODE_FAST) {
        if (variant != WENO_TENO) {
            weno5_cell_fast64(f0, f1, f2, f3, f4, variant, eps, vl, vr);
            return;
        }
    }
    if constexpr (MODE == MODE_DF) {
        // the double-float reconstruction (the adjoint sweeps recompute the
        // forward face states of a double-float step with it)
        const WenoEdges ed = weno5_cell_df(f0, f1, f2, f3, f4, variant, df64(double(eps)), df64(double(ct)));
        vl = ed.vl;
        vr = ed.vr;
        return;
    }
    if constexpr (MODE == MODE_MIXED) {
        if (variant != WENO_TENO) {
            const float2 v = weno5_cell_mixed32(f0, f1, f2, f3, f4, variant, eps);
            vr = v.x;
            vl = v.y;
            return;
        }
    }
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
            vr = weno5_edge_exact(p, beta, d, variant, eps, ct);
        }
        {
            const double d[3] = {0.3, 0.6, 0.1};
            const double p[3] = {(-f0 + 5.0 * f1 + 2.0 * f2) / 6.0, (2.0 * f1 + 5.0 * f2 - f3) / 6.0,
                                 (11.0 * f2 - 7.0 * f3 + 2.0 * f4) / 6.0};
            vl = weno5_edge_exact(p, beta, d, variant, eps, ct);
        }
    } else {
        R b[3], e, scale;
        weno5_scaled_beta(f0, f1, f2, f3, f4, eps, b, e, scale);
        R P[3];
        const R dR[3] = {R(0.1), R(0.6), R(0.3)}, dL[3] = {R(0.3), R(0.6), R(0.1)};
        R omR[3], omL[3];
        if (variant == WENO_TENO) {
            teno_weights(b, e, ct, dR, dL, omR, omL);
        } else {
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
        }
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

template <int NQ>
__device__ __forceinline__ void weno5_fields_mixed32(const float* f0, const float* f1, const float* f2,
                                                     const float* f3, const float* f4, int variant, float eps,
                                                     float ct, float* vl, float* vr) {
    if (variant == WENO_TENO) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) weno5_cell<MODE_MIXED, float>(f0[k], f1[k], f2[k], f3[k], f4[k], variant, eps, ct,
                                                                   vl[k], vr[k]);
        return;
    }
#pragma unroll
    for (int k = 0; k + 1 < NQ; k += 2) {
        const WenoPair32 w = weno5_cells_mixed32_x2(f0[k], f1[k], f2[k], f3[k], f4[k], f0[k + 1], f1[k + 1],
                                                    f2[k + 1], f3[k + 1], f4[k + 1], variant, eps);
        vr[k] = w.a.x;
        vl[k] = w.a.y;
        vr[k + 1] = w.b.x;
        vl[k + 1] = w.b.y;
    }
    if constexpr (NQ % 2 == 1) {
        const float2 v = weno5_cell_mixed32(f0[NQ - 1], f1[NQ - 1], f2[NQ - 1], f3[NQ - 1], f4[NQ - 1], variant, eps);
        vr[NQ - 1] = v.x;
        vl[NQ - 1] = v.y;
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
__device__ __forceinline__ void hllc(const R* WL0, const R* WR0, const MixState<R>& mL, const MixState<R>& mR,
                                     const Consts& C, R* F, R& uf, bool& bad) {
    using L = Lay<NF, ND>;
    using A = Arith<MODE>;
    constexpr int NQ = L::NQ;
    constexpr int UN = L::MOM + DIR;
    // sound speeds of the reconstructed states (independent of the velocity)
    R rho[2], un[2], p[2], E[2], c[2], Gm[2], Pm[2];
    const R* W0[2] = {WL0, WR0};
    const MixState<R>* M0[2] = {&mL, &mR};
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        const R* w = W0[K];
        const R r = M0[K]->rho;
        Gm[K] = M0[K]->G;
        Pm[K] = M0[K]->P;
        rho[K] = r;
        p[K] = w[L::E];
        R c2 = A::quot(M0[K]->num, Gm[K] * r);
        if constexpr (NF == 2) {
            if (C.model == 1) c2 = wood_c2<MODE, R>(r, p[K], w[L::A], C);
        }
        bad |= !Cmp<MODE, R>::pos(c2);
        c[K] = sqrt(c2);
    }
    // low-Mach corrections (Sec. 4.2.4): z = min(max(|u_L|/c_L, |u_R|/c_R), 1);
    // Thornber's modification pulls the normal velocities towards their mean
    R zlm = R(1);
    R WLm[NQ], WRm[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        WLm[k] = WL0[k];
        WRm[k] = WR0[k];
    }
    if (C.low_mach != 0) {
        const R uL = WL0[UN], uR = WR0[UN];
        const R aLz = A::quot(fabs(uL), c[0]), aRz = A::quot(fabs(uR), c[1]);
        const R zm = (aRz > aLz) ? aRz : aLz;
        zlm = (R(1) < zm) ? R(1) : zm;
        if (C.low_mach == 1) {
            const R mean = (uL + uR) / R(2);
            WLm[UN] = mean + zlm * (uL - uR) / R(2);
            WRm[UN] = mean + zlm * (uR - uL) / R(2);
        }
    }
    const R* WL = WLm;
    const R* WR = WRm;
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        const R* w = K ? WR : WL;
        R u2 = R(0);
#pragma unroll
        for (int e = 0; e < ND; ++e) u2 = u2 + w[L::MOM + e] * w[L::MOM + e];
        un[K] = w[UN];
        E[K] = Gm[K] * p[K] + Pm[K] + R(0.5) * rho[K] * u2;
    }
    using Kc = Cmp<MODE, R>;
    const R aL = un[0] - c[0], aR = un[1] - c[1];
    const R SL = Kc::lt(aR, aL) ? aR : aL;
    const R bL = un[0] + c[0], bR = un[1] + c[1];
    const R SR = Kc::lt(bL, bR) ? bR : bL;

    if (C.riemann == 1) {
        // HLL (Sec. 3.2.2): F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)
        // in the fan for every conserved component (U_alpha = alpha,
        // F_alpha = alpha u); the face velocity of alpha div u is the same
        // average of u
        R FK[2][NQ], UK[2][NQ];
#pragma unroll
        for (int K = 0; K < 2; ++K) {
            const R* w = K ? WR : WL;
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                FK[K][i] = w[i] * un[K];
                UK[K][i] = w[i];
            }
#pragma unroll
            for (int e = 0; e < ND; ++e) {
                FK[K][L::MOM + e] = rho[K] * un[K] * w[L::MOM + e];
                if (e == DIR) FK[K][L::MOM + e] = FK[K][L::MOM + e] + p[K];
                UK[K][L::MOM + e] = rho[K] * w[L::MOM + e];
            }
            FK[K][L::E] = (E[K] + p[K]) * un[K];
            UK[K][L::E] = E[K];
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) {
                FK[K][L::A + j] = w[L::A + j] * un[K];
                UK[K][L::A + j] = w[L::A + j];
            }
        }
        if (Kc::nonneg(SL)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) F[k] = FK[0][k];
            uf = un[0];
        } else if (!Kc::pos(SR)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) F[k] = FK[1][k];
            uf = un[1];
        } else {
#pragma unroll
            for (int k = 0; k < NQ; ++k)
                F[k] = A::quot(SR * FK[0][k] - SL * FK[1][k] + SL * SR * (UK[1][k] - UK[0][k]), SR - SL);
            uf = A::quot(SR * un[0] - SL * un[1], SR - SL);
        }
        return;
    }

    const R Ss = A::quot(p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1]),
                         rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]));

    const bool left = Kc::nonneg(Ss);
    const R* w = left ? WL : WR;
    const R rK = left ? rho[0] : rho[1];
    const R uK = left ? un[0] : un[1];
    const R pK = left ? p[0] : p[1];
    const R EK = left ? E[0] : E[1];
    const R SK = left ? SL : SR;
    const bool star = left ? Kc::neg(SL) : Kc::pos(SR);

    if constexpr (MODE != MODE_EXACT) {
        // The same star-state fluxes with one reciprocal.  With
        // B = S_K - S*, chi = (S_K - u_K)/B and dl = S_K (chi - 1) =
        // S_K (S* - u_K)/B (= chi S* - u_K):
        //   F*_K = F_K + S_K (U*_K - U_K) is (u_K + dl) U_K for the partial
        //   densities and the tangential momenta, p_K + rho_K (u_K^2 + S_K dl)
        //   for the normal momentum, and for the energy
        //   E*_K = chi rho_K (E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K))))
        //        = ((S_K - u_K)(E_K + rho_K (S* - u_K) S*) + (S* - u_K) p_K) / B.
        R m = uK, Fn, FE;
        if (star) {
            const R du = Ss - uK;
            const R iB = rcp<R>(SK - Ss);
            const R dl = SK * du * iB;
            m = uK + dl;
            Fn = fma(rK, fma(uK, uK, SK * dl), pK);
            const R Es = fma(du, pK, (SK - uK) * fma(rK * du, Ss, EK)) * iB;
            FE = fma(SK, Es - EK, (EK + pK) * uK);
        } else {
            Fn = fma(rK * uK, uK, pK);
            FE = (EK + pK) * uK;
        }
#pragma unroll
        for (int i = 0; i < NF; ++i) F[i] = w[i] * m;
        const R rm = rK * m;
#pragma unroll
        for (int e = 0; e < ND; ++e) F[L::MOM + e] = (e == DIR) ? Fn : rm * w[L::MOM + e];
        F[L::E] = FE;
        if (star && C.low_mach == 2) {
            // anti-dissipation pressure correction (Sec. 4.2.4)
            const R pd = A::quot(rho[0] * rho[1] * (SL - un[0]) * (SR - un[1]) * (un[1] - un[0]),
                                 rho[1] * (SR - un[1]) - rho[0] * (SL - un[0]));
            const R apc = (zlm - R(1)) * pd;
            F[UN] = F[UN] + apc;
            F[L::E] = F[L::E] + apc * Ss;
        }
        uf = star ? Ss : uK;
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) F[L::A + j] = w[L::A + j] * uf;
    } else {
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
            if (C.low_mach == 2) {
                // anti-dissipation pressure correction (Sec. 4.2.4)
                const R pd = A::quot(rho[0] * rho[1] * (SL - un[0]) * (SR - un[1]) * (un[1] - un[0]),
                                     rho[1] * (SR - un[1]) - rho[0] * (SL - un[0]));
                const R apc = (zlm - R(1)) * pd;
                F[UN] = F[UN] + apc;
                F[L::E] = F[L::E] + apc * Ss;
            }
            uf = Ss;
        } else {
            uf = uK;
        }
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) F[L::A + j] = w[L::A + j] * uf;
    }
}

// hllc with the mixture quantities of both states computed here.
template <int NF, int ND, int DIR, int MODE, class R = typename ModeT<MODE>::R>
__device__ __forceinline__ void hllc(const R* WL0, const R* WR0, const Consts& C, R* F, R& uf, bool& bad) {
    hllc<NF, ND, DIR, MODE, R>(WL0, WR0, mix_state<NF, ND, MODE, R>(WL0, C), mix_state<NF, ND, MODE, R>(WR0, C), C, F,
                               uf, bad);
}

// Index of the interior cell that supplies the value of cell c along an
// axis with n cells (Sec. 3.3): periodic wrap, transmissive copy of the
// nearest cell, reflective mirror (flip = normal momentum changes sign); a
// halo side supplies the ghost cell itself (the caller's copy of the
// neighbouring subdomain's cell).
__device__ __forceinline__ int64_t bc_source(int64_t c, int64_t n, int bclo, int bchi, bool& flip) {
    if (c < 0) {
        if (bclo == BC_HALO) return c;
        if (bclo == BC_PERIODIC) return c + n;
        if (bclo == BC_TRANSMISSIVE) return 0;
        flip = true;
        return -1 - c;
    }
    if (c >= n) {
        if (bchi == BC_HALO) return c;
        if (bchi == BC_PERIODIC) return c - n;
        if (bchi == BC_TRANSMISSIVE) return n - 1;
        flip = true;
        return 2 * n - 1 - c;
    }
    return c;
}

}  // namespace mfc
