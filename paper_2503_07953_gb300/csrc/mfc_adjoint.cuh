// Reverse-mode (adjoint) building blocks: the exact transposed derivatives
// of cons_to_prim, weno5_cell and hllc in mfc_device.cuh.  Every function
// recomputes the forward quantities it needs from its inputs and takes the
// same branches as the forward code (ties of min / max keep the left
// argument; d|x|/dx = +1 at 0), so the result is the derivative of the
// branch the forward pass takes.
#pragma once

#include "mfc_device.cuh"

namespace mfc {

// Division by one denominator b, possibly several times: IEEE a / b in
// MODE_EXACT; a times one reciprocal of b otherwise (rcp<R>).  div2 divides
// by b^2.  Only the reverse (bar) arithmetic and forward quantities that
// decide no branch go through it; the forward values that pick a branch
// (wave speeds, S*, the fallback test) are recomputed with the forward
// pass's own arithmetic.
template <int MODE, class R>
struct Recip {
    R b, ib;
    __device__ __forceinline__ explicit Recip(R x) : b(x) {
        if constexpr (MODE == MODE_EXACT) ib = R(0);
        else ib = rcp<R>(x);
    }
    __device__ __forceinline__ R div(R a) const {
        if constexpr (MODE == MODE_EXACT) return a / b;
        else return a * ib;
    }
    __device__ __forceinline__ R div2(R a) const {
        if constexpr (MODE == MODE_EXACT) return a / (b * b);
        else return a * ib * ib;
    }
};

// Partial derivatives of the Kapila K(p, alpha_1) (float64): with
// Z_i = gamma_i (p + pi_i), N = Z_2 - Z_1, D = Z_1/alpha_1 + Z_2/alpha_2,
// dK/dp = (N' D - N D') / D^2 and dK/dalpha_1 = -N (dD/dalpha_1) / D^2.
__device__ __forceinline__ void kapila_K_grad(double p, double a1, const Consts& C, double& dKdp, double& dKda) {
    const double g1 = C.gam[0], g2 = C.gam[1];
    const double Z1 = g1 * (p + C.pinf[0]), Z2 = g2 * (p + C.pinf[1]);
    const double a2 = 1.0 - a1;
    const double N = Z2 - Z1, D = Z1 / a1 + Z2 / a2;
    const double iD2 = 1.0 / (D * D);
    dKdp = ((g2 - g1) * D - N * (g1 / a1 + g2 / a2)) * iD2;
    dKda = -N * (-Z1 / (a1 * a1) + Z2 / (a2 * a2)) * iD2;
}

// q_bar += (dW/dq)^T W_bar for the conservative state q of one cell.
template <int NF, int ND, int MODE = MODE_EXACT>
__device__ __forceinline__ void cons_to_prim_adj(const double* q, const double* wbar, const Consts& C,
                                                 double* qbar) {
    using L = Lay<NF, ND>;
    constexpr int M = (MODE == MODE_EXACT) ? MODE_EXACT : MODE_FAST;  // float64 throughout
    double rho = q[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) rho = rho + q[i];
    const Recip<M, double> rr(rho);
    double u[ND];
    double u2 = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        u[d] = rr.div(q[L::MOM + d]);
        u2 = u2 + u[d] * u[d];
    }
    double Gamma, Pi;
    mixture_mode<NF, M, double>(q + L::A, C, Gamma, Pi);
    const Recip<M, double> rg(Gamma);
    const double ke = 0.5 * rho * u2;
    const double p = rg.div(q[L::E] - ke - Pi);
    // p = (E - ke - Pi) / Gamma
    const double pb = wbar[L::E];
    const double numb = rg.div(pb);
    const double Gb = rg.div(-pb * p);
    const double Pb = -numb;
    qbar[L::E] += numb;
    const double keb = -numb;
    double rhob = keb * 0.5 * u2;
    const double u2b = keb * 0.5 * rho;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const double ub = wbar[L::MOM + d] + u2b * 2.0 * u[d];
        qbar[L::MOM + d] += rr.div(ub);
        rhob -= rr.div(ub * u[d]);
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) qbar[i] += wbar[i] + rhob;
#pragma unroll
    for (int j = 0; j < NF - 1; ++j)
        qbar[L::A + j] += wbar[L::A + j] + Gb * (C.g[j] - C.g[NF - 1]) + Pb * (C.h[j] - C.h[NF - 1]);
}

// Adjoint of the nonlinear weights and the final sum of one edge:
// given p[3], beta[3], ideal weights d[3] and out_bar, add to p_bar and
// beta_bar.
template <int MODE, class R>
__device__ __forceinline__ void weno5_edge_adj(const R* p, const R* beta, const R* d, int variant, R eps, R outb,
                                               R* pb, R* betab) {
    R a[3], w[3], t[3], it[3];
    R tau = R(0);
    if (variant == WENO_Z) {
        tau = fabs(beta[0] - beta[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            t[r] = beta[r] + eps;
            const Recip<MODE, R> rt(t[r]);
            it[r] = rt.ib;
            a[r] = d[r] * (R(1) + rt.div(tau));
        }
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            t[r] = eps + beta[r];
            const Recip<MODE, R> rt(t[r]);
            it[r] = rt.ib;
            a[r] = rt.div2(d[r]);
        }
    }
    const R s = a[0] + a[1] + a[2];
    const Recip<MODE, R> rs(s);
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = rs.div(a[r]);
    R om[3], Nn[3], Dd[3], iD[3], gm[3];
    R sm = R(1), ism = R(1);
    if (variant == WENO_M) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Nn[r] = d[r] + d[r] * d[r] - R(3) * d[r] * w[r] + w[r] * w[r];
            Dd[r] = d[r] * d[r] + w[r] * (R(1) - R(2) * d[r]);
            const Recip<MODE, R> rd(Dd[r]);
            iD[r] = rd.ib;
            gm[r] = rd.div(w[r] * Nn[r]);
        }
        sm = gm[0] + gm[1] + gm[2];
        const Recip<MODE, R> rsm(sm);
        ism = rsm.ib;
#pragma unroll
        for (int r = 0; r < 3; ++r) om[r] = rsm.div(gm[r]);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) om[r] = w[r];
    }
    // division by a denominator whose reciprocal was taken above
    auto dv = [](R a_, R b_, R ib_) -> R {
        if constexpr (MODE == MODE_EXACT) return a_ / b_;
        else return a_ * ib_;
    };
    // out = sum om_r p_r
    R omb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        pb[r] += om[r] * outb;
        omb[r] = p[r] * outb;
    }
    R wb[3];
    if (variant == WENO_M) {
        // om_r = gm_r / sm
        const R dot = omb[0] * om[0] + omb[1] * om[1] + omb[2] * om[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const R gb = dv(omb[r] - dot, sm, ism);
            // gm = w N(w) / D(w), N' = -3 d + 2 w, D' = 1 - 2 d
            const R dN = R(-3) * d[r] + R(2) * w[r];
            const R dD = R(1) - R(2) * d[r];
            R dg;
            if constexpr (MODE == MODE_EXACT)
                dg = (Nn[r] + w[r] * dN) / Dd[r] - w[r] * Nn[r] * dD / (Dd[r] * Dd[r]);
            else
                dg = ((Nn[r] + w[r] * dN) - w[r] * Nn[r] * dD * iD[r]) * iD[r];
            wb[r] = gb * dg;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) wb[r] = omb[r];
    }
    // w_r = a_r / s
    const R dotw = wb[0] * w[0] + wb[1] * w[1] + wb[2] * w[2];
    R ab[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) ab[r] = rs.div(wb[r] - dotw);
    if (variant == WENO_Z) {
        R taub = R(0);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if constexpr (MODE == MODE_EXACT) {
                const R be = beta[r] + eps;
                taub += ab[r] * d[r] / be;
                betab[r] += -ab[r] * d[r] * tau / (be * be);
            } else {
                taub += ab[r] * d[r] * it[r];
                betab[r] += -ab[r] * d[r] * tau * it[r] * it[r];
            }
        }
        const R sg = (beta[0] - beta[2] >= R(0)) ? R(1) : R(-1);
        betab[0] += taub * sg;
        betab[2] -= taub * sg;
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) betab[r] += ab[r] * dv(R(-2) * a[r], t[r], it[r]);
    }
}

// Adjoint of weno5_cell_df with JS or mapped weights (MODE_DF): given the
// bars vlb, vrb of the left- and right-edge values, the bars of f0..f4, in
// double-float arithmetic on the float32 pipes, the two edges' weight
// computations paired in df64x2.  The forward quantities are recomputed with
// weno5_cell_df's operations, and the branch it takes is differentiated:
// the stencil of the smallest scaled indicator (t_min), the power-of-two
// scale (piecewise constant), indicators floored at 2^-120 and the flat
// branch with ideal weights (both constant).  With
// c = (sum_r omega_r P_r) / 6 and v = f2 + c per edge:
//   omega (mapped) = gm / sum gm,  gm_r = N_r prod_{s != r} D_s,
//   N = w (d (1 + d) + w (w - 3 d)),  D = d^2 + w (1 - 2 d),
//   w = a / sum a,  a_r = d_r u_r^2,  u_r = t_min / t_r,  t_r = s (eps + beta_r).
struct WenoBars {
    double b[5];
};

static __device__ __noinline__ WenoBars weno5_cell_adj_df(double f0, double f1, double f2, double f3, double f4,
                                                          double vlb, double vrb, int variant, df64 e) {
    constexpr df64 c13(13.0 / 12.0), sixth(1.0 / 6.0);
    const df64 D01 = df_from_f64_bits(f1 - f0), D12 = df_from_f64_bits(f2 - f1);
    const df64 D23 = df_from_f64_bits(f3 - f2), D34 = df_from_f64_bits(f4 - f3);
    const df64 a[3] = {D12 - D01, D23 - D12, D34 - D23};
    const df64 g[3] = {df_mulf(D12, 3.0f) - D01, D12 + D23, D34 - df_mulf(D23, 3.0f)};
    df64 t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = e + (c13 * (a[r] * a[r]) + df_scale(g[r] * g[r], 0.25f));
    const df64 P[3] = {df_mulf(D12, 5.0f) - df_scale(D01, 2.0f), D12 + df_scale(D23, 2.0f),
                       df_scale(D23, 4.0f) - D34};
    const df64 Q[3] = {D01 - df_scale(D12, 4.0f), -(df_scale(D12, 2.0f) + D23),
                       df_scale(D34, 2.0f) - df_mulf(D23, 5.0f)};
    const double dR[3] = {0.1, 0.6, 0.3}, dL[3] = {0.3, 0.6, 0.1};
    const df64x2 cb = dfx2(df_from_f64_bits(vrb), df_from_f64_bits(vlb)) * dfx2(sixth, sixth);
    df64x2 PQb[3];
    df64 ab[3] = {df64(0.0), df64(0.0), df64(0.0)}, gb[3] = {df64(0.0), df64(0.0), df64(0.0)};
    const float th = fmaxf(fmaxf(t[0].hi, t[1].hi), t[2].hi);
    if (!(th >= 0x1p-120f)) {
        // ideal weights: only the candidates carry bars
#pragma unroll
        for (int r = 0; r < 3; ++r) PQb[r] = cb * dfx2(dR[r], dL[r]);
    } else {
        int k = ((__float_as_int(th) >> 23) & 0xff) - 127;
        k = k > 126 ? 126 : k;
        const float sc = __int_as_float((127 - k) << 23);
        df64 ts[3];
        bool floored[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ts[r] = df_scale(t[r], sc);
            floored[r] = ts[r].hi < 0x1p-120f;
            if (floored[r]) ts[r] = df64(0x1p-120f, 0.0f);
        }
        const float tmh = fminf(fminf(ts[0].hi, ts[1].hi), ts[2].hi);
        const int rmin = (ts[0].hi == tmh) ? 0 : ((ts[1].hi == tmh) ? 1 : 2);
        const df64 tmin = ts[rmin];
        df64 u[3], its[3];
        df64x2 w[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            its[r] = df_div(df64(1.0), ts[r]);
            u[r] = tmin * its[r];
            const df64 u2 = u[r] * u[r];
            w[r] = dfx2(dR[r], dL[r]) * dfx2(u2, u2);
        }
        const df64x2 inv = df_rcp((w[0] + w[1]) + w[2]);
        df64x2 wn[3], om[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) om[r] = wn[r] = w[r] * inv;
        df64x2 Nn[3], Dd[3], inv2;
        if (variant == WENO_M) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                Nn[r] = wn[r] * (dfx2(dR[r] * (1.0 + dR[r]), dL[r] * (1.0 + dL[r])) +
                                 wn[r] * (wn[r] - dfx2(3.0 * dR[r], 3.0 * dL[r])));
                Dd[r] = dfx2(dR[r] * dR[r], dL[r] * dL[r]) + wn[r] * dfx2(1.0 - 2.0 * dR[r], 1.0 - 2.0 * dL[r]);
            }
            const df64x2 gm0 = Nn[0] * (Dd[1] * Dd[2]), gm1 = Nn[1] * (Dd[0] * Dd[2]), gm2 = Nn[2] * (Dd[0] * Dd[1]);
            inv2 = df_rcp((gm0 + gm1) + gm2);
            om[0] = gm0 * inv2;
            om[1] = gm1 * inv2;
            om[2] = gm2 * inv2;
        }
        // reverse: c = sum om_r PQ_r (times 1/6, in cb)
        df64x2 omb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            omb[r] = cb * dfx2(P[r], Q[r]);
            PQb[r] = cb * om[r];
        }
        df64x2 wb[3];
        if (variant == WENO_M) {
            // om = gm / sum gm
            const df64x2 dot = (omb[0] * om[0] + omb[1] * om[1]) + omb[2] * om[2];
            df64x2 gmb[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) gmb[r] = (omb[r] - dot) * inv2;
            // gm_r = N_r prod_{s != r} D_s
            const df64x2 Nb[3] = {gmb[0] * (Dd[1] * Dd[2]), gmb[1] * (Dd[0] * Dd[2]), gmb[2] * (Dd[0] * Dd[1])};
            const df64x2 gN[3] = {gmb[0] * Nn[0], gmb[1] * Nn[1], gmb[2] * Nn[2]};
            const df64x2 Db[3] = {gN[1] * Dd[2] + gN[2] * Dd[1], gN[0] * Dd[2] + gN[2] * Dd[0],
                                  gN[0] * Dd[1] + gN[1] * Dd[0]};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                // N' = d (1 + d) + w (3 w - 6 d), D' = 1 - 2 d
                const df64x2 dN = dfx2(dR[r] * (1.0 + dR[r]), dL[r] * (1.0 + dL[r])) +
                                  wn[r] * (wn[r] * dfx2(3.0, 3.0) - dfx2(6.0 * dR[r], 6.0 * dL[r]));
                wb[r] = Nb[r] * dN + Db[r] * dfx2(1.0 - 2.0 * dR[r], 1.0 - 2.0 * dL[r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) wb[r] = omb[r];
        }
        // wn = w / sum w,  w_r = d_r u_r^2 (both edges feed u_r)
        const df64x2 dotw = (wb[0] * wn[0] + wb[1] * wn[1]) + wb[2] * wn[2];
        df64 ub[3], tsb[3];
        df64 tminb(0.0);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const df64x2 x = ((wb[r] - dotw) * inv) * dfx2(dR[r], dL[r]);
            const df64 u2b = lane_x(x) + lane_y(x);
            ub[r] = df_scale(u2b * u[r], 2.0f);
            // u_r = t_min / ts_r
            tminb = tminb + ub[r] * its[r];
            tsb[r] = -((ub[r] * u[r]) * its[r]);
        }
        tsb[rmin] = tsb[rmin] + tminb;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const df64 tb = floored[r] ? df64(0.0) : df_scale(tsb[r], sc);
            // t_r = eps + 13/12 a_r^2 + 1/4 g_r^2
            ab[r] = tb * (c13 * df_scale(a[r], 2.0f));
            gb[r] = tb * df_scale(g[r], 0.5f);
        }
    }
    const df64 Pb[3] = {lane_x(PQb[0]), lane_x(PQb[1]), lane_x(PQb[2])};
    const df64 Qb[3] = {lane_y(PQb[0]), lane_y(PQb[1]), lane_y(PQb[2])};
    const df64 D01b = ((Qb[0] - df_scale(Pb[0], 2.0f)) - ab[0]) - gb[0];
    const df64 D12b = ((df_mulf(Pb[0], 5.0f) + Pb[1]) - (df_scale(Qb[0], 4.0f) + df_scale(Qb[1], 2.0f))) +
                      ((ab[0] + df_mulf(gb[0], 3.0f)) + (gb[1] - ab[1]));
    const df64 D23b = ((df_scale(Pb[1], 2.0f) + df_scale(Pb[2], 4.0f)) - (Qb[1] + df_mulf(Qb[2], 5.0f))) +
                      ((ab[1] + gb[1]) - (ab[2] + df_mulf(gb[2], 3.0f)));
    const df64 D34b = (df_scale(Qb[2], 2.0f) - Pb[2]) + (ab[2] + gb[2]);
    auto dbl = [](df64 x) { return f64_from_f32_bits(x.hi) + f64_from_f32_bits(x.lo); };
    const double e01 = dbl(D01b), e12 = dbl(D12b), e23 = dbl(D23b), e34 = dbl(D34b);
    WenoBars out;
    out.b[0] = -e01;
    out.b[1] = e01 - e12;
    out.b[2] = (e12 - e23) + (vrb + vlb);
    out.b[3] = e23 - e34;
    out.b[4] = e34;
    return out;
}

// Adjoint of weno5_cell_fast64 (JS, mapped and Z weights; MODE_FAST): the
// bars of f0..f4 given the bars vlb, vrb of the left- and right-edge values,
// in weno5_cell_fast64's own formulation, so that the indicators, the
// unnormalised weights and their products are formed once for both edges
// and each normalisation costs one reciprocal.  Per edge, with y_r the
// final unnormalised weights, n' = sum y, i = 1 / (12 n') and c_r the
// scaled candidate corrections (12 (candidate_r - f2)):
//   v = f2 + i sum_r y_r c_r,
//   y_bar_r = v_bar i (c_r - 12 i sum_s y_s c_s),  c_bar_r = v_bar i y_r;
// mapped: y_r = N_r D_s D_q ({r, s, q} = {0, 1, 2}) with N = x (x (x - 3 d)
// + d (1 + d)), D = x (1 - 2 d) + d^2, x = w / sum w, so
//   N_bar_r = y_bar_r D_s D_q,  D_bar_r = sum_{s != r} y_bar_s N_s D_q,
//   x_bar_r = N_bar_r (3 x^2 - 6 d x + d (1 + d)) + D_bar_r (1 - 2 d),
//   w_bar_r = (x_bar_r - sum_s x_bar_s x_s) / sum w;
// JS and Z: y = w.  Both edges' w are d_r P_r (d = (1, 6, 3)/10 right,
// (3, 6, 1)/10 left), so P_bar_r = dR_r w_bar^R_r + dL_r w_bar^L_r, and
// from P_r = prod_{s != r} t_s^2 (JS, mapped) or (t_r + tau) prod_{s != r}
// t_s, tau = |t_0 - t_2| (Z) to t_r = g_r^2 + (13/3) a_r^2 + 4 eps and the
// candidates c^R_r = a_r + 3 s_r g_r, c^L_r = a_r - 3 s_r g_r (s = +1, +1,
// -1), back to the consecutive differences and f.  The function has no
// branch but tau's sign (taken as the forward's |.| takes it: +1 at 0).
// Not inlined: one copy of its code serves the N_q fields from the
// instruction cache.
static __device__ __noinline__ WenoBars weno5_cell_adj_fast64(double f0, double f1, double f2, double f3,
                                                              double f4, double vlb, double vrb, int variant,
                                                              double eps) {
    const double D01 = f1 - f0, D12 = f2 - f1, D23 = f3 - f2, D34 = f4 - f3;
    const double a[3] = {D12 - D01, D23 - D12, D34 - D23};
    const double e4 = 4.0 * eps;
    const double g[3] = {fma(3.0, D12, -D01), D12 + D23, fma(-3.0, D23, D34)};
    double t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = fma(g[r], g[r], weno5_fast64_A(a[r], e4));
    const double cs[2][3] = {{fma(3.0, g[0], a[0]), fma(3.0, g[1], a[1]), fma(-3.0, g[2], a[2])},
                             {fma(-3.0, g[0], a[0]), fma(-3.0, g[1], a[1]), fma(3.0, g[2], a[2])}};
    const double ds[2][3] = {{0.1, 0.6, 0.3}, {0.3, 0.6, 0.1}};
    // unnormalised JS / Z weights d_r P_r
    double s[3], P[3], Q[3], tau = 0.0;
    if (variant == WENO_Z) {
        tau = fabs(t[0] - t[2]);
        Q[0] = t[1] * t[2];
        Q[1] = t[0] * t[2];
        Q[2] = t[0] * t[1];
#pragma unroll
        for (int r = 0; r < 3; ++r) P[r] = (t[r] + tau) * Q[r];
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) s[r] = t[r] * t[r];
        P[0] = s[1] * s[2];
        P[1] = s[0] * s[2];
        P[2] = s[0] * s[1];
    }
    const double m1 = 0.6 * P[1];
    double w[2][3] = {{0.1 * P[0], m1, 0.3 * P[2]}, {0.3 * P[0], m1, 0.1 * P[2]}};
    double y[2][3], n[2], iw[2] = {0.0, 0.0};
    double x[2][3], N[2][3], D[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        n[e] = (w[e][0] + w[e][1]) + w[e][2];
        if (variant == WENO_M) {
            const double* d = ds[e];
            iw[e] = rcp_nr(n[e]);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                x[e][r] = w[e][r] * iw[e];
                N[e][r] = x[e][r] * fma(x[e][r], x[e][r] - 3.0 * d[r], d[r] * (1.0 + d[r]));
                D[e][r] = fma(x[e][r], 1.0 - 2.0 * d[r], d[r] * d[r]);
            }
            y[e][0] = N[e][0] * (D[e][1] * D[e][2]);
            y[e][1] = N[e][1] * (D[e][0] * D[e][2]);
            y[e][2] = N[e][2] * (D[e][0] * D[e][1]);
            n[e] = (y[e][0] + y[e][1]) + y[e][2];
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) y[e][r] = w[e][r];
        }
    }
    double in[2];
    if (variant == WENO_M) {
        // the mapped sums lie within [5e-6, 3]: one reciprocal for both edges
        const double rr = rcp_nr((12.0 * n[0]) * n[1]);
        in[0] = n[1] * rr;
        in[1] = n[0] * rr;
    } else {
        in[0] = rcp_nr(12.0 * n[0]);
        in[1] = rcp_nr(12.0 * n[1]);
    }
    // reverse, edge by edge: bars of the candidates and of w
    const double vb[2] = {vrb, vlb};
    double cb[2][3], wb[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const double m = vb[e] * in[e];
        const double* c = cs[e];
        const double u = in[e] * fma(y[e][2], c[2], fma(y[e][1], c[1], y[e][0] * c[0]));
        const double mh = m * (12.0 * u);
        double yb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            yb[r] = fma(m, c[r], -mh);
            cb[e][r] = m * y[e][r];
        }
        if (variant == WENO_M) {
            const double* d = ds[e];
            const double* Ne = N[e];
            const double* De = D[e];
            const double Nb[3] = {yb[0] * (De[1] * De[2]), yb[1] * (De[0] * De[2]), yb[2] * (De[0] * De[1])};
            const double YN[3] = {yb[0] * Ne[0], yb[1] * Ne[1], yb[2] * Ne[2]};
            const double Db[3] = {fma(YN[1], De[2], YN[2] * De[1]), fma(YN[0], De[2], YN[2] * De[0]),
                                  fma(YN[0], De[1], YN[1] * De[0])};
            double xb[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double dN = fma(x[e][r], fma(3.0, x[e][r], -6.0 * d[r]), d[r] * (1.0 + d[r]));
                xb[r] = fma(Db[r], 1.0 - 2.0 * d[r], Nb[r] * dN);
            }
            const double dot = fma(xb[2], x[e][2], fma(xb[1], x[e][1], xb[0] * x[e][0]));
#pragma unroll
            for (int r = 0; r < 3; ++r) wb[e][r] = (xb[r] - dot) * iw[e];
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) wb[e][r] = yb[r];
        }
    }
    // w^R_r = dR_r P_r, w^L_r = dL_r P_r
    const double Pb[3] = {fma(0.1, wb[0][0], 0.3 * wb[1][0]), 0.6 * (wb[0][1] + wb[1][1]),
                          fma(0.3, wb[0][2], 0.1 * wb[1][2])};
    double tb[3];
    if (variant == WENO_Z) {
        // P_r = (t_r + tau) Q_r, Q_r = prod_{s != r} t_s
        const double PE[3] = {Pb[0] * (t[0] + tau), Pb[1] * (t[1] + tau), Pb[2] * (t[2] + tau)};
        tb[0] = fma(Pb[0], Q[0], fma(PE[1], t[2], PE[2] * t[1]));
        tb[1] = fma(Pb[1], Q[1], fma(PE[0], t[2], PE[2] * t[0]));
        tb[2] = fma(Pb[2], Q[2], fma(PE[0], t[1], PE[1] * t[0]));
        const double taub = fma(Pb[2], Q[2], fma(Pb[1], Q[1], Pb[0] * Q[0]));
        // tau = |t_0 - t_2|, d|z|/dz = +1 at 0
        const double sg = (f64_nonneg(t[0] - t[2])) ? taub : -taub;
        tb[0] += sg;
        tb[2] -= sg;
    } else {
        // P_0 = s_1 s_2, P_1 = s_0 s_2, P_2 = s_0 s_1, s_r = t_r^2
        const double sb[3] = {fma(Pb[1], s[2], Pb[2] * s[1]), fma(Pb[0], s[2], Pb[2] * s[0]),
                              fma(Pb[0], s[1], Pb[1] * s[0])};
#pragma unroll
        for (int r = 0; r < 3; ++r) tb[r] = (t[r] + t[r]) * sb[r];
    }
    // t_r = g_r^2 + (13/3) a_r^2 + 4 eps; c^R_r = a_r + 3 s_r g_r, c^L_r = a_r - 3 s_r g_r
    double ab[3], gb[3];
    const double sgn[3] = {3.0, 3.0, -3.0};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ab[r] = fma((26.0 / 3.0) * a[r], tb[r], cb[0][r] + cb[1][r]);
        gb[r] = fma(g[r] + g[r], tb[r], sgn[r] * (cb[0][r] - cb[1][r]));
    }
    // a_0 = D12 - D01, a_1 = D23 - D12, a_2 = D34 - D23;
    // g_0 = 3 D12 - D01, g_1 = D12 + D23, g_2 = D34 - 3 D23
    const double D01b = -(ab[0] + gb[0]);
    const double D12b = (ab[0] - ab[1]) + fma(3.0, gb[0], gb[1]);
    const double D23b = (ab[1] - ab[2]) + fma(-3.0, gb[2], gb[1]);
    const double D34b = ab[2] + gb[2];
    WenoBars out;
    out.b[0] = -D01b;
    out.b[1] = D01b - D12b;
    out.b[2] = (D12b - D23b) + (vrb + vlb);
    out.b[3] = D23b - D34b;
    out.b[4] = D34b;
    return out;
}

// Adjoint of weno5_cell_mixed32 (JS, mapped and Z weights; MODE_MIXED):
// weno5_cell_adj_fast64's reverse in float32, the two edges' weight
// arithmetic paired in float2 instructions as in the forward.  The forward
// evaluates the weights on t_r = b_r s + e, b_r = 4 beta_r, s = 1 / sum b,
// e = max(4 eps s, 1e-9), and the reverse differentiates that map too:
// dt_s/db_r = s (delta_rs - t_s + e_f) with e_f = e where the floor is taken
// and 0 where e = 4 eps s, so b_bar_r = s (t_bar_r - sum_s t_bar_s (t_s - e_f)).
struct WenoBars32 {
    float b[5];
};

static __device__ __noinline__ WenoBars32 weno5_cell_adj_mixed32(float f0, float f1, float f2, float f3, float f4,
                                                                 float vlb, float vrb, int variant, float eps) {
    const float D01 = f1 - f0, D12 = f2 - f1, D23 = f3 - f2, D34 = f4 - f3;
    const float a[3] = {D12 - D01, D23 - D12, D34 - D23};
    const float g[3] = {fmaf(3.0f, D12, -D01), D12 + D23, fmaf(-3.0f, D23, D34)};
    float b[3];  // 4 beta_r
#pragma unroll
    for (int r = 0; r < 3; ++r) b[r] = fmaf((13.0f / 3.0f) * a[r], a[r], g[r] * g[r]);
    const float scale = __fdividef(1.0f, (b[0] + b[1]) + (b[2] + 4e-30f));
    const float e0 = 4.0f * eps * scale;
    const bool floored = !(e0 > 1e-9f);
    const float e = fmaxf(e0, 1e-9f);
    float t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = fmaf(b[r], scale, e);
    float P[3], Q[3], s[3], tau = 0.0f;
    if (variant == WENO_Z) {
        tau = fabsf(t[0] - t[2]);
        Q[0] = t[1] * t[2];
        Q[1] = t[0] * t[2];
        Q[2] = t[0] * t[1];
#pragma unroll
        for (int r = 0; r < 3; ++r) P[r] = (t[r] + tau) * Q[r];
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) s[r] = t[r] * t[r];
        P[0] = s[1] * s[2];
        P[1] = s[0] * s[2];
        P[2] = s[0] * s[1];
    }
    // (right, left) pairs: ideal weights, unnormalised weights
    const float2 d[3] = {pair(0.1f, 0.3f), pair(0.6f, 0.6f), pair(0.3f, 0.1f)};
    float2 y[3], x[3], N[3], E[3], EE[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = __fmul2_rn(d[r], pair(P[r], P[r]));
    float2 nrm = __fadd2_rn(__fadd2_rn(y[0], y[1]), y[2]);
    float2 iw = pair(0.0f, 0.0f);
    if (variant == WENO_M) {
        iw = pair(__fdividef(1.0f, nrm.x), __fdividef(1.0f, nrm.y));
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = __fmul2_rn(y[r], iw);
        // N = x (x (x - 3 d) + d (1 + d)), E = x (1 - 2 d) + d^2
        N[0] = __fmul2_rn(x[0], __ffma2_rn(x[0], __fadd2_rn(x[0], pair(-0.3f, -0.9f)), pair(0.11f, 0.39f)));
        N[1] = __fmul2_rn(x[1], __ffma2_rn(x[1], __fadd2_rn(x[1], pair(-1.8f, -1.8f)), pair(0.96f, 0.96f)));
        N[2] = __fmul2_rn(x[2], __ffma2_rn(x[2], __fadd2_rn(x[2], pair(-0.9f, -0.3f)), pair(0.39f, 0.11f)));
        E[0] = __ffma2_rn(x[0], pair(0.8f, 0.4f), pair(0.01f, 0.09f));
        E[1] = __ffma2_rn(x[1], pair(-0.2f, -0.2f), pair(0.36f, 0.36f));
        E[2] = __ffma2_rn(x[2], pair(0.4f, 0.8f), pair(0.09f, 0.01f));
        EE[0] = __fmul2_rn(E[1], E[2]);
        EE[1] = __fmul2_rn(E[0], E[2]);
        EE[2] = __fmul2_rn(E[0], E[1]);
#pragma unroll
        for (int r = 0; r < 3; ++r) y[r] = __fmul2_rn(N[r], EE[r]);
        nrm = __fadd2_rn(__fadd2_rn(y[0], y[1]), y[2]);
    }
    const float2 in = pair(__fdividef(1.0f, 12.0f * nrm.x), __fdividef(1.0f, 12.0f * nrm.y));
    const float2 c[3] = {__ffma2_rn(pair(3.0f, -3.0f), pair(g[0], g[0]), pair(a[0], a[0])),
                         __ffma2_rn(pair(3.0f, -3.0f), pair(g[1], g[1]), pair(a[1], a[1])),
                         __ffma2_rn(pair(-3.0f, 3.0f), pair(g[2], g[2]), pair(a[2], a[2]))};
    // reverse: v = f2 + in sum_r y_r c_r per edge
    const float2 m = __fmul2_rn(pair(vrb, vlb), in);
    const float2 u = __fmul2_rn(in, __ffma2_rn(y[2], c[2], __ffma2_rn(y[1], c[1], __fmul2_rn(y[0], c[0]))));
    const float2 mh = __fmul2_rn(m, __fmul2_rn(pair(12.0f, 12.0f), u));
    const float2 nmh = pair(-mh.x, -mh.y);
    float2 yb[3], cb[3], wb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        yb[r] = __ffma2_rn(m, c[r], nmh);
        cb[r] = __fmul2_rn(m, y[r]);
    }
    if (variant == WENO_M) {
        const float2 YN[3] = {__fmul2_rn(yb[0], N[0]), __fmul2_rn(yb[1], N[1]), __fmul2_rn(yb[2], N[2])};
        const float2 Eb[3] = {__ffma2_rn(YN[1], E[2], __fmul2_rn(YN[2], E[1])),
                              __ffma2_rn(YN[0], E[2], __fmul2_rn(YN[2], E[0])),
                              __ffma2_rn(YN[0], E[1], __fmul2_rn(YN[1], E[0]))};
        // N' = x (3 x - 6 d) + d (1 + d); E' = 1 - 2 d
        const float2 m6d[3] = {pair(-0.6f, -1.8f), pair(-3.6f, -3.6f), pair(-1.8f, -0.6f)};
        const float2 d1d[3] = {pair(0.11f, 0.39f), pair(0.96f, 0.96f), pair(0.39f, 0.11f)};
        const float2 dE[3] = {pair(0.8f, 0.4f), pair(-0.2f, -0.2f), pair(0.4f, 0.8f)};
        float2 xb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float2 dN = __ffma2_rn(x[r], __ffma2_rn(pair(3.0f, 3.0f), x[r], m6d[r]), d1d[r]);
            xb[r] = __ffma2_rn(Eb[r], dE[r], __fmul2_rn(__fmul2_rn(yb[r], EE[r]), dN));
        }
        const float2 dot = __ffma2_rn(xb[2], x[2], __ffma2_rn(xb[1], x[1], __fmul2_rn(xb[0], x[0])));
#pragma unroll
        for (int r = 0; r < 3; ++r) wb[r] = __fmul2_rn(__fadd2_rn(xb[r], pair(-dot.x, -dot.y)), iw);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) wb[r] = yb[r];
    }
    // w^R_r = dR_r P_r, w^L_r = dL_r P_r
    float Pb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float2 q = __fmul2_rn(wb[r], d[r]);
        Pb[r] = q.x + q.y;
    }
    float tb[3];
    if (variant == WENO_Z) {
        const float PE[3] = {Pb[0] * (t[0] + tau), Pb[1] * (t[1] + tau), Pb[2] * (t[2] + tau)};
        tb[0] = fmaf(Pb[0], Q[0], fmaf(PE[1], t[2], PE[2] * t[1]));
        tb[1] = fmaf(Pb[1], Q[1], fmaf(PE[0], t[2], PE[2] * t[0]));
        tb[2] = fmaf(Pb[2], Q[2], fmaf(PE[0], t[1], PE[1] * t[0]));
        const float taub = fmaf(Pb[2], Q[2], fmaf(Pb[1], Q[1], Pb[0] * Q[0]));
        const float sg = (t[0] - t[2] >= 0.0f) ? taub : -taub;
        tb[0] += sg;
        tb[2] -= sg;
    } else {
        const float sb[3] = {fmaf(Pb[1], s[2], Pb[2] * s[1]), fmaf(Pb[0], s[2], Pb[2] * s[0]),
                             fmaf(Pb[0], s[1], Pb[1] * s[0])};
#pragma unroll
        for (int r = 0; r < 3; ++r) tb[r] = (t[r] + t[r]) * sb[r];
    }
    // t_s = b_s s + e
    const float ef = floored ? e : 0.0f;
    const float corr = fmaf(tb[2], t[2] - ef, fmaf(tb[1], t[1] - ef, tb[0] * (t[0] - ef)));
    float ab[3], gb[3];
    const float sgn[3] = {3.0f, 3.0f, -3.0f};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float bb = scale * (tb[r] - corr);
        // b_r = (13/3) a_r^2 + g_r^2; c^R_r = a_r + 3 s_r g_r, c^L_r = a_r - 3 s_r g_r
        ab[r] = fmaf((26.0f / 3.0f) * a[r], bb, cb[r].x + cb[r].y);
        gb[r] = fmaf(g[r] + g[r], bb, sgn[r] * (cb[r].x - cb[r].y));
    }
    const float D01b = -(ab[0] + gb[0]);
    const float D12b = (ab[0] - ab[1]) + fmaf(3.0f, gb[0], gb[1]);
    const float D23b = (ab[1] - ab[2]) + fmaf(-3.0f, gb[2], gb[1]);
    const float D34b = ab[2] + gb[2];
    WenoBars32 out;
    out.b[0] = -D01b;
    out.b[1] = D01b - D12b;
    out.b[2] = (D12b - D23b) + (vrb + vlb);
    out.b[3] = D23b - D34b;
    out.b[4] = D34b;
    return out;
}

// x != 0 for every x, NaN included; for float64 on the bit pattern (integer
// instructions, off the float64 pipe).
template <class R> __device__ __forceinline__ bool nonzero(R x) { return x != R(0); }
template <> __device__ __forceinline__ bool nonzero<double>(double x) {
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ULL;
}

// Adjoint of weno5_cell: given the bars of the right-edge value (vrb) and
// the left-edge value (vlb), write df to fb[0..4].
template <int MODE, class R>
__device__ __forceinline__ void weno5_cell_adj(const R* f, R vlb, R vrb, int variant, R eps, R ct, R* fb) {
    if constexpr (MODE == MODE_FAST) {
        if (variant != WENO_TENO) {
            if (!nonzero(vlb) && !nonzero(vrb)) {
#pragma unroll
                for (int i = 0; i < 5; ++i) fb[i] = R(0);
                return;
            }
            const WenoBars w = weno5_cell_adj_fast64(f[0], f[1], f[2], f[3], f[4], vlb, vrb, variant, eps);
#pragma unroll
            for (int i = 0; i < 5; ++i) fb[i] = w.b[i];
            return;
        }
    }
    if constexpr (MODE == MODE_MIXED) {
        if (variant != WENO_TENO) {
            if (vlb == R(0) && vrb == R(0)) {
#pragma unroll
                for (int i = 0; i < 5; ++i) fb[i] = R(0);
                return;
            }
            const WenoBars32 w = weno5_cell_adj_mixed32(f[0], f[1], f[2], f[3], f[4], vlb, vrb, variant, eps);
#pragma unroll
            for (int i = 0; i < 5; ++i) fb[i] = w.b[i];
            return;
        }
    }
    if constexpr (MODE == MODE_DF) {
        if (variant == WENO_JS || variant == WENO_M) {
            const WenoBars w = weno5_cell_adj_df(f[0], f[1], f[2], f[3], f[4], vlb, vrb, variant, df64(double(eps)));
#pragma unroll
            for (int i = 0; i < 5; ++i) fb[i] = w.b[i];
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) fb[i] = R(0);
    const R c13 = R(13.0 / 12.0), c14 = R(0.25);
    const R A0 = f[0] - R(2) * f[1] + f[2], B0 = f[0] - R(4) * f[1] + R(3) * f[2];
    const R A1 = f[1] - R(2) * f[2] + f[3], B1 = f[1] - f[3];
    const R A2 = f[2] - R(2) * f[3] + f[4], B2 = R(3) * f[2] - R(4) * f[3] + f[4];
    // indicators as the forward weights use them (scaled by `scale` in
    // float32); the weights depend only on ratios of eps + beta, so the bar
    // of the unscaled beta is the bar of the scaled one times the scale
    R beta[3], e, scale;
    weno5_scaled_beta(f[0], f[1], f[2], f[3], f[4], eps, beta, e, scale);
    R betab[3] = {R(0), R(0), R(0)};
    // TENO: the weights are piecewise constant in the indicators (a
    // stencil is on or off), so only the candidate values carry bars
    R omT[2][3];
    if (variant == WENO_TENO) {
        const R dR[3] = {R(0.1), R(0.6), R(0.3)}, dL[3] = {R(0.3), R(0.6), R(0.1)};
        if constexpr (MODE == MODE_EXACT) {
            const R* ds[2] = {dR, dL};
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                R a[3];
                teno_select_exact(beta, ds[s], e, ct, a);
                const R sa = a[0] + a[1] + a[2];
#pragma unroll
                for (int r = 0; r < 3; ++r) omT[s][r] = a[r] / sa;
            }
        } else {
            teno_weights(beta, e, ct, dR, dL, omT[0], omT[1]);
        }
    }
    const R sixth = R(1) / R(6);
    auto by6 = [&](R x) -> R {
        if constexpr (MODE == MODE_EXACT) return x / R(6);
        else return x * sixth;
    };
    if (vrb != R(0)) {
        R p[3], pb[3] = {R(0), R(0), R(0)};
        const R d[3] = {R(0.1), R(0.6), R(0.3)};
        p[0] = by6(R(2) * f[0] - R(7) * f[1] + R(11) * f[2]);
        p[1] = by6(-f[1] + R(5) * f[2] + R(2) * f[3]);
        p[2] = by6(R(2) * f[2] + R(5) * f[3] - f[4]);
        if (variant == WENO_TENO) {
#pragma unroll
            for (int r = 0; r < 3; ++r) pb[r] += omT[0][r] * vrb;
        } else {
            weno5_edge_adj<MODE, R>(p, beta, d, variant, e, vrb, pb, betab);
        }
        fb[0] += (R(2) * pb[0]) * sixth;
        fb[1] += (R(-7) * pb[0] - pb[1]) * sixth;
        fb[2] += (R(11) * pb[0] + R(5) * pb[1] + R(2) * pb[2]) * sixth;
        fb[3] += (R(2) * pb[1] + R(5) * pb[2]) * sixth;
        fb[4] += (-pb[2]) * sixth;
    }
    if (vlb != R(0)) {
        R p[3], pb[3] = {R(0), R(0), R(0)};
        const R d[3] = {R(0.3), R(0.6), R(0.1)};
        p[0] = by6(-f[0] + R(5) * f[1] + R(2) * f[2]);
        p[1] = by6(R(2) * f[1] + R(5) * f[2] - f[3]);
        p[2] = by6(R(11) * f[2] - R(7) * f[3] + R(2) * f[4]);
        if (variant == WENO_TENO) {
#pragma unroll
            for (int r = 0; r < 3; ++r) pb[r] += omT[1][r] * vlb;
        } else {
            weno5_edge_adj<MODE, R>(p, beta, d, variant, e, vlb, pb, betab);
        }
        fb[0] += (-pb[0]) * sixth;
        fb[1] += (R(5) * pb[0] + R(2) * pb[1]) * sixth;
        fb[2] += (R(2) * pb[0] + R(5) * pb[1] + R(11) * pb[2]) * sixth;
        fb[3] += (-pb[1] - R(7) * pb[2]) * sixth;
        fb[4] += (R(2) * pb[2]) * sixth;
    }
    betab[0] *= scale;
    betab[1] *= scale;
    betab[2] *= scale;
    // beta_r = c13 A_r^2 + c14 B_r^2
    const R a0 = R(2) * c13 * A0 * betab[0], b0 = R(2) * c14 * B0 * betab[0];
    const R a1 = R(2) * c13 * A1 * betab[1], b1 = R(2) * c14 * B1 * betab[1];
    const R a2 = R(2) * c13 * A2 * betab[2], b2 = R(2) * c14 * B2 * betab[2];
    fb[0] += a0 + b0;
    fb[1] += R(-2) * a0 - R(4) * b0 + a1 + b1;
    fb[2] += a0 + R(3) * b0 + R(-2) * a1 + a2 + R(3) * b2;
    fb[3] += a1 - b1 + R(-2) * a2 - R(4) * b2;
    fb[4] += a2 + b2;
}

// Adjoint of hllc (and of its HLL and low-Mach variants): given F_bar[NQ]
// and uf_bar, add to WLb, WRb.  Also returns the forward face velocity in
// uf_out.
template <int NF, int ND, int DIR, int MODE, class R = typename ModeT<MODE>::R>
__device__ __forceinline__ void hllc_adj(const R* WL0, const R* WR0, const Consts& C, const R* Fb, R ufb, R* WLb,
                                         R* WRb, R& uf_out) {
    using L = Lay<NF, ND>;
    using Q = Arith<MODE>;
    constexpr int NQ = L::NQ;
    constexpr int UN = L::MOM + DIR;
    // ---- forward recomputation ----
    // sound speeds (they do not depend on the velocity, so they are the same
    // before and after the low-Mach modification)
    R rho[2], un[2], p[2], E[2], c[2], G[2], P[2], u2[2], c2[2];
    const R* W0[2] = {WL0, WR0};
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        const R* w = W0[K];
        R r = w[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) r = r + w[i];
        mixture_mode<NF, MODE, R>(w + L::A, C, G[K], P[K]);
        rho[K] = r;
        p[K] = w[L::E];
        c2[K] = Q::quot((G[K] + R(1)) * p[K] + P[K], G[K] * r);
        if constexpr (NF == 2) {
            if (C.model == 1) c2[K] = wood_c2<MODE, R>(r, p[K], w[L::A], C);
        }
        c[K] = sqrt(c2[K]);
    }
    // low-Mach z = min(max(|u_L|/c_L, |u_R|/c_R), 1) and Thornber's velocities
    const R u0L = WL0[UN], u0R = WR0[UN];
    R zlm = R(1);
    bool zR = false, zclip = true;
    R aLz = R(0), aRz = R(0);
    if (C.low_mach != 0) {
        aLz = Q::quot(fabs(u0L), c[0]);
        aRz = Q::quot(fabs(u0R), c[1]);
        zR = aRz > aLz;
        const R zm = zR ? aRz : aLz;
        zclip = R(1) < zm;
        zlm = zclip ? R(1) : zm;
    }
    R WLm[NQ], WRm[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        WLm[k] = WL0[k];
        WRm[k] = WR0[k];
    }
    if (C.low_mach == 1) {
        const R mean = (u0L + u0R) / R(2);
        WLm[UN] = mean + zlm * (u0L - u0R) / R(2);
        WRm[UN] = mean + zlm * (u0R - u0L) / R(2);
    }
    const R* WL = WLm;
    const R* WR = WRm;
    const R* Wm[2] = {WL, WR};
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        const R* w = Wm[K];
        R s2 = R(0);
#pragma unroll
        for (int e = 0; e < ND; ++e) s2 = s2 + w[L::MOM + e] * w[L::MOM + e];
        u2[K] = s2;
        un[K] = w[UN];
        E[K] = G[K] * p[K] + P[K] + R(0.5) * rho[K] * s2;
    }
    const R aL = un[0] - c[0], aR = un[1] - c[1];
    const bool minR = aR < aL;
    const R SL = minR ? aR : aL;
    const R bL = un[0] + c[0], bR = un[1] + c[1];
    const bool maxR = bR > bL;
    const R SR = maxR ? bR : bL;

    // per-side bars: density, normal velocity, pressure, total energy, sound
    // speed, and the primitive slots read directly
    R rb[2] = {R(0), R(0)}, unb[2] = {R(0), R(0)}, pb[2] = {R(0), R(0)}, Eb[2] = {R(0), R(0)},
      cb[2] = {R(0), R(0)};
    R wbs[2][NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) wbs[0][k] = wbs[1][k] = R(0);
    R SLb = R(0), SRb = R(0), zb = R(0);

    if (C.riemann == 1) {
        // ---- HLL ----
        // physical fluxes and states of both sides (U_alpha = alpha, F_alpha = alpha u)
        R FK[2][NQ], UK[2][NQ];
#pragma unroll
        for (int K = 0; K < 2; ++K) {
            const R* w = Wm[K];
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
        R FKb[2][NQ], UKb[2][NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) FKb[0][k] = FKb[1][k] = UKb[0][k] = UKb[1][k] = R(0);
        if (SL >= R(0)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) FKb[0][k] = Fb[k];
            uf_out = un[0];
            unb[0] += ufb;
        } else if (SR <= R(0)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) FKb[1][k] = Fb[k];
            uf_out = un[1];
            unb[1] += ufb;
        } else {
            const Recip<MODE, R> rW(SR - SL);
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const R dU = UK[1][k] - UK[0][k];
                const R Fk = rW.div(SR * FK[0][k] - SL * FK[1][k] + SL * SR * dU);
                FKb[0][k] = rW.div(Fb[k] * SR);
                FKb[1][k] = rW.div(-Fb[k] * SL);
                UKb[1][k] = rW.div(Fb[k] * SL * SR);
                UKb[0][k] = -UKb[1][k];
                SRb += rW.div(Fb[k] * (FK[0][k] + SL * dU - Fk));
                SLb += rW.div(Fb[k] * (-FK[1][k] + SR * dU + Fk));
            }
            const R uf = rW.div(SR * un[0] - SL * un[1]);
            uf_out = uf;
            unb[0] += rW.div(ufb * SR);
            unb[1] -= rW.div(ufb * SL);
            SRb += rW.div(ufb * (un[0] - uf));
            SLb += rW.div(ufb * (uf - un[1]));
        }
        // F_K and U_K back to the side's variables
#pragma unroll
        for (int K = 0; K < 2; ++K) {
            const R* w = Wm[K];
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                wbs[K][i] += FKb[K][i] * un[K] + UKb[K][i];
                unb[K] += FKb[K][i] * w[i];
            }
#pragma unroll
            for (int e = 0; e < ND; ++e) {
                const R Fe = FKb[K][L::MOM + e], Ue = UKb[K][L::MOM + e];
                rb[K] += Fe * un[K] * w[L::MOM + e] + Ue * w[L::MOM + e];
                unb[K] += Fe * rho[K] * w[L::MOM + e];
                wbs[K][L::MOM + e] += Fe * rho[K] * un[K] + Ue * rho[K];
                if (e == DIR) pb[K] += Fe;
            }
            Eb[K] += FKb[K][L::E] * un[K] + UKb[K][L::E];
            pb[K] += FKb[K][L::E] * un[K];
            unb[K] += FKb[K][L::E] * (E[K] + p[K]);
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) {
                wbs[K][L::A + j] += FKb[K][L::A + j] * un[K] + UKb[K][L::A + j];
                unb[K] += FKb[K][L::A + j] * w[L::A + j];
            }
        }
    } else {
        // ---- HLLC ----
        const R num = p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1]);
        const R den = rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]);
        const R Ss = Q::quot(num, den);
        const bool left = Ss >= R(0);
        const int K = left ? 0 : 1;
        const R* w = left ? WL : WR;
        const R rK = rho[K], uK = un[K], pK = p[K], EK = E[K];
        const R SK = left ? SL : SR;
        const bool star = left ? (SL < R(0)) : (SR > R(0));
        const R uf = star ? Ss : uK;
        uf_out = uf;

        R* wb = wbs[K];
        R rKb = R(0), uKb = R(0), pKb = R(0), EKb = R(0), SKb = R(0), Ssb = R(0);
        R ufb_t = ufb;
        // alpha slots: F = alpha_K uf
#pragma unroll
        for (int j = 0; j < NF - 1; ++j) {
            wb[L::A + j] += Fb[L::A + j] * uf;
            ufb_t += Fb[L::A + j] * w[L::A + j];
        }
        if (star) {
            Ssb += ufb_t;
            if (C.low_mach == 2) {
                // anti-dissipation pressure correction: + (z - 1) p_d on the
                // normal momentum, + (z - 1) p_d S* on the energy
                const R A1 = SL - un[0], B1 = SR - un[1], dun = un[1] - un[0];
                const R Nn = rho[0] * rho[1] * A1 * B1 * dun;
                const R Dd = rho[1] * B1 - rho[0] * A1;
                const Recip<MODE, R> rDd(Dd);
                const R pd = rDd.div(Nn);
                const R apc = (zlm - R(1)) * pd;
                const R apcb = Fb[UN] + Fb[L::E] * Ss;
                Ssb += Fb[L::E] * apc;
                zb += apcb * pd;
                const R pdb = apcb * (zlm - R(1));
                const R Nnb = rDd.div(pdb);
                const R Ddb = rDd.div(-pdb * pd);
                rb[0] += Nnb * rho[1] * A1 * B1 * dun - Ddb * A1;
                rb[1] += Nnb * rho[0] * A1 * B1 * dun + Ddb * B1;
                const R A1b = Nnb * rho[0] * rho[1] * B1 * dun - Ddb * rho[0];
                const R B1b = Nnb * rho[0] * rho[1] * A1 * dun + Ddb * rho[1];
                const R dunb = Nnb * rho[0] * rho[1] * A1 * B1;
                SLb += A1b;
                unb[0] -= A1b + dunb;
                SRb += B1b;
                unb[1] += dunb - B1b;
            }
            const R A = SK - uK, B = SK - Ss;
            const R chi = Q::quot(A, B);
            const Recip<MODE, R> rB(B), rK_(rK);
            R chib = R(0);
            // energy
            const R Z = rK * (SK - uK);
            const Recip<MODE, R> rZ(Z);
            const R Y = Ss + rZ.div(pK);
            const R X = rK_.div(EK) + (Ss - uK) * Y;
            const R Es = chi * rK * X;
            SKb += Fb[L::E] * (Es - EK);
            const R Esb = Fb[L::E] * SK;
            EKb -= Fb[L::E] * SK;
            chib += Esb * rK * X;
            rKb += Esb * chi * X;
            const R Xb = Esb * chi * rK;
            EKb += rK_.div(Xb);
            rKb -= rK_.div2(Xb * EK);
            Ssb += Xb * Y;
            uKb -= Xb * Y;
            const R Yb = Xb * (Ss - uK);
            Ssb += Yb;
            pKb += rZ.div(Yb);
            const R Zb = rZ.div2(-Yb * pK);
            rKb += Zb * (SK - uK);
            SKb += Zb * rK;
            uKb -= Zb * rK;
            // momentum
#pragma unroll
            for (int e = 0; e < ND; ++e) {
                const R Fe = Fb[L::MOM + e];
                const R we = w[L::MOM + e];
                const R ve = (e == DIR) ? Ss : we;
                SKb += Fe * (chi * rK * ve - rK * we);
                chib += Fe * SK * rK * ve;
                rKb += Fe * SK * (chi * ve - we);
                if (e == DIR) {
                    Ssb += Fe * SK * chi * rK;
                    wb[L::MOM + e] -= Fe * SK * rK;
                } else {
                    wb[L::MOM + e] += Fe * SK * rK * (chi - R(1));
                }
            }
            // partial densities
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                SKb += Fb[i] * (chi - R(1)) * w[i];
                chib += Fb[i] * SK * w[i];
                wb[i] += Fb[i] * SK * (chi - R(1));
            }
            // chi = A / B
            const R Ab = rB.div(chib);
            const R Bb = rB.div(-chib * chi);
            SKb += Ab + Bb;
            uKb -= Ab;
            Ssb -= Bb;
        } else {
            uKb += ufb_t;
        }
        // physical flux of side K
#pragma unroll
        for (int i = 0; i < NF; ++i) {
            wb[i] += Fb[i] * uK;
            uKb += Fb[i] * w[i];
        }
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            const R Fe = Fb[L::MOM + e];
            rKb += Fe * uK * w[L::MOM + e];
            uKb += Fe * rK * w[L::MOM + e];
            wb[L::MOM + e] += Fe * rK * uK;
            if (e == DIR) pKb += Fe;
        }
        EKb += Fb[L::E] * uK;
        pKb += Fb[L::E] * uK;
        uKb += Fb[L::E] * (EK + pK);

        rb[K] += rKb;
        unb[K] += uKb;
        pb[K] += pKb;
        Eb[K] += EKb;
        if (left) SLb += SKb; else SRb += SKb;
        // Ss = num / den
        const Recip<MODE, R> rden(den);
        const R numb = rden.div(Ssb);
        const R denb = rden.div(-Ssb * Ss);
        pb[1] += numb;
        pb[0] -= numb;
        rb[0] += numb * un[0] * (SL - un[0]);
        unb[0] += numb * rho[0] * (SL - R(2) * un[0]);
        SLb += numb * rho[0] * un[0];
        rb[1] -= numb * un[1] * (SR - un[1]);
        unb[1] -= numb * rho[1] * (SR - R(2) * un[1]);
        SRb -= numb * rho[1] * un[1];
        rb[0] += denb * (SL - un[0]);
        SLb += denb * rho[0];
        unb[0] -= denb * rho[0];
        rb[1] -= denb * (SR - un[1]);
        SRb -= denb * rho[1];
        unb[1] += denb * rho[1];
    }
    // wave speeds
    if (minR) {
        unb[1] += SLb;
        cb[1] -= SLb;
    } else {
        unb[0] += SLb;
        cb[0] -= SLb;
    }
    if (maxR) {
        unb[1] += SRb;
        cb[1] += SRb;
    } else {
        unb[0] += SRb;
        cb[0] += SRb;
    }

    // bars of a side's primitive slots from a bar of its sound speed:
    // c = sqrt(c2), c2 = ((G + 1) p + P) / (G r), or Wood's
    // c2 = 1 / (r (a1/Z1 + a2/Z2)) for the Kapila model
    auto c_bar = [&](int S, R cbar, R* o) {
        const R* ws = W0[S];
        const R c2b = Recip<MODE, R>(R(2) * c[S]).div(cbar);
        bool wood = false;
        if constexpr (NF == 2) {
            if (C.model == 1) {
                wood = true;
                const R g1 = phasic<R>(C.gam, C.gamf, 0), g2 = phasic<R>(C.gam, C.gamf, 1);
                const R Z1 = g1 * (p[S] + phasic<R>(C.pinf, C.pinff, 0));
                const R Z2 = g2 * (p[S] + phasic<R>(C.pinf, C.pinff, 1));
                const R a1 = ws[L::A], a2 = R(1) - a1;
                const Recip<MODE, R> rZ1(Z1), rZ2(Z2);
                const R Dw = rZ1.div(a1) + rZ2.div(a2);
                const R Dwb = Recip<MODE, R>(Dw).div(-c2b * c2[S]);
                const R rbs = Recip<MODE, R>(rho[S]).div(-c2b * c2[S]);
#pragma unroll
                for (int i = 0; i < NF; ++i) o[i] += rbs;
                o[L::E] -= Dwb * (g1 * rZ1.div2(a1) + g2 * rZ2.div2(a2));
                o[L::A] += Dwb * (rZ1.div(R(1)) - rZ2.div(R(1)));
            }
        }
        if (!wood) {
            const R Dd = G[S] * rho[S];
            const Recip<MODE, R> rDd(Dd);
            const R Nnb = rDd.div(c2b);
            const R Ddb = rDd.div(-c2b * c2[S]);
            const R Gb = Nnb * p[S] + Ddb * rho[S];
            const R Pb = Nnb;
            o[L::E] += Nnb * (G[S] + R(1));
            const R rbs = Ddb * G[S];
#pragma unroll
            for (int i = 0; i < NF; ++i) o[i] += rbs;
#pragma unroll
            for (int j = 0; j < NF - 1; ++j)
                o[L::A + j] += Gb * (coef_g<R>(C, j) - coef_g<R>(C, NF - 1)) +
                               Pb * (coef_h<R>(C, j) - coef_h<R>(C, NF - 1));
        }
    };

    // bars of the (possibly modified) states
    R Wb[2][NQ];
#pragma unroll
    for (int S = 0; S < 2; ++S) {
        const R* ws = Wm[S];
        R* o = Wb[S];
#pragma unroll
        for (int k = 0; k < NQ; ++k) o[k] = wbs[S][k];
        c_bar(S, cb[S], o);
        // E = G p + P + 0.5 r u2
        const R Gb = Eb[S] * p[S];
        const R Pb = Eb[S];
        o[L::E] += pb[S] + Eb[S] * G[S];
        const R rbs = rb[S] + Eb[S] * R(0.5) * u2[S];
        const R u2b = Eb[S] * R(0.5) * rho[S];
#pragma unroll
        for (int e = 0; e < ND; ++e) o[L::MOM + e] += u2b * R(2) * ws[L::MOM + e];
        o[UN] += unb[S];
#pragma unroll
        for (int i = 0; i < NF; ++i) o[i] += rbs;
#pragma unroll
        for (int j = 0; j < NF - 1; ++j)
            o[L::A + j] += Gb * (coef_g<R>(C, j) - coef_g<R>(C, NF - 1)) + Pb * (coef_h<R>(C, j) - coef_h<R>(C, NF - 1));
    }
    // Thornber: the normal velocities of the modified states back to the
    // reconstructed ones, and their dependence on z
    if (C.low_mach == 1) {
        const R bL_ = Wb[0][UN], bR_ = Wb[1][UN];
        zb += bL_ * (u0L - u0R) / R(2) + bR_ * (u0R - u0L) / R(2);
        Wb[0][UN] = bL_ * (R(1) + zlm) / R(2) + bR_ * (R(1) - zlm) / R(2);
        Wb[1][UN] = bL_ * (R(1) - zlm) / R(2) + bR_ * (R(1) + zlm) / R(2);
    }
    // z = min(max(|u_L|/c_L, |u_R|/c_R), 1): the branch taken
    if (C.low_mach != 0 && !zclip) {
        const int S = zR ? 1 : 0;
        const R u0 = S ? u0R : u0L;
        const R sg = (u0 >= R(0)) ? R(1) : R(-1);
        const Recip<MODE, R> rc(c[S]);
        Wb[S][UN] += zb * sg * rc.div(R(1));
        c_bar(S, -zb * (S ? aRz : aLz) * rc.div(R(1)), Wb[S]);
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        WLb[k] += Wb[0][k];
        WRb[k] += Wb[1][k];
    }
}

}  // namespace mfc
