/*
 * Plain, slow FP64 CPU oracle for the five-equation
 * WENO5 / HLLC / TVD-RK3 finite-volume method of arXiv 2503.07953 (MFC 5.0).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (the CUDA library and its Python binding) never imports,
 * links or calls it, and this file shares no code, header, table or helper
 * with that path.
 *
 * Built twice from this one file: single-threaded (the tests), and with
 * OpenMP for the timing of the CPU baseline, where the loops over grid lines
 * and cells run on all host cores.  Each cell's arithmetic is the same in
 * both builds, so their results are identical bit for bit.
 *
 * Every numerical routine is templated on its scalar type:
 *   double  - the oracle proper;
 *   Dual    - forward-mode directional derivatives (JVPs) of the same code;
 *   Cnt     - a double that counts the floating-point operations it performs.
 *
 * What it computes (all citations are to the paper):
 *   * five-equation model, Sec. 2.1.1: partial densities alpha_i rho_i,
 *     mixture momentum rho u, total energy rho E and N_f - 1 volume
 *     fractions alpha_j, with alpha_N = 1 - sum_j alpha_j (mixture rules,
 *     Sec. 2.1.1); K = 0 (Allaire) or, for two fluids, the Kapila K div u
 *     term with the Wood mixture sound speed;
 *   * stiffened-gas EOS, Sec. 2.2: rho_i e_i = (p + gamma_i pi_i)/(gamma_i - 1),
 *     so rho e = Gamma p + Pi with Gamma = sum alpha_i/(gamma_i - 1) and
 *     Pi = sum alpha_i gamma_i pi_i/(gamma_i - 1);
 *   * finite-volume semi-discretisation, Sec. 3.1, Eq. (rhs), with
 *     h(q) = (0, ..., 0, -alpha) so that the alpha rows get + alpha div(u);
 *   * WENO5 reconstruction of the primitive variables with JS, mapped
 *     (Henrick) and Z weights, Sec. 3.2.1 and Sec. 4.2.2, and the
 *     fifth-order TENO stencil selection of Sec. 4.2.2;
 *   * HLLC and HLL approximate Riemann solvers, Sec. 3.2.2 (Toro), with the
 *     low-Mach corrections of Sec. 4.2.4 (Thornber's velocity modification,
 *     Chen's anti-dissipation pressure correction for HLLC);
 *   * the viscous stress T^v = 2 eta (D - tr(D) I/3) of Sec. 2.1.1 in the
 *     momentum and energy fluxes (optional: all eta_i = 0 is inviscid);
 *   * ghost cells by periodic wrap, zeroth-order extrapolation or mirror
 *     with negated normal momentum, Sec. 3.3;
 *   * third-order TVD Runge-Kutta, Sec. 3.4 (the same tableau as the
 *     q^{n+1} = q^n + h/6 (k1 + k2 + 4 k3) form of Sec. 4.2.3);
 *   * CFL time step dt = CFL * min over cells and directions of
 *     dx_d / (|u_d| + c) with the mixture sound speed.
 * Readings where the paper is silent are listed in the repository design
 * notes; each is restated at the routine that uses it.
 *
 * State layout used by this oracle (its own, independent of the GPU path):
 * interior cells only, C order [field][z][y][x], no ghost cells.  Field order:
 * alpha_1 rho_1 .. alpha_N rho_N, rho u_1 .. rho u_ndim, rho E,
 * alpha_1 .. alpha_{N-1}.  Primitive order: the same slots holding
 * alpha_i rho_i, u_d, p, alpha_j.
 */
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int MAXF = 4;
constexpr int MAXQ = 2 * MAXF + 3;

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2 };
enum { WENO_JS = 0, WENO_M = 1, WENO_Z = 2, WENO_TENO = 3 };

}  // namespace

extern "C" {
/* Problem description, mirrored field by field by the ctypes wrapper. */
typedef struct {
    int32_t ndim, nf;
    int32_t n[3];
    double lo[3], hi[3];
    int32_t bc_lo[3], bc_hi[3];
    double gamma[MAXF], pi_inf[MAXF];
    int32_t weno;
    double eps;
    double teno_ct;   /* TENO threshold C_T (weno = 3) */
    int32_t model;    /* 0: K = 0 (Allaire); 1: Kapila K div u, two fluids */
    int32_t riemann;  /* 0: HLLC; 1: HLL */
    int32_t low_mach; /* 0: none; 1: Thornber; 2: anti-dissipation pressure correction (HLLC) */
    double eta[MAXF]; /* shear viscosity of each fluid; all zero: inviscid */
    int32_t viscous_dt; /* 1: the CFL dt also respects the explicit viscous limit */
} oc_problem;
}

namespace {

/* ------------------------------------------------------------------ */
/* Scalar types                                                        */
/* ------------------------------------------------------------------ */

struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double x) : v(x), d(0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
    friend Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
    friend Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
    friend Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
    friend Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
    friend Dual operator/(Dual a, Dual b) {
        double r = a.v / b.v;
        return Dual(r, (a.d - r * b.d) / b.v);
    }
    friend bool operator<(Dual a, Dual b) { return a.v < b.v; }
    friend bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
    friend bool operator>(Dual a, Dual b) { return a.v > b.v; }
    friend bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
    friend Dual sqrt(Dual a) {
        double s = std::sqrt(a.v);
        return Dual(s, a.d / (2.0 * s));
    }
    /* d|x|/dx is taken as +1 at x = 0. */
    friend Dual fabs(Dual a) { return a.v >= 0 ? a : -a; }
    Dual& operator+=(Dual b) { return *this = *this + b; }
};

struct OpCounts {
    int64_t add, mul, div, sqrt, cmp;
};
OpCounts g_ops = {0, 0, 0, 0, 0};

struct Cnt {
    double v;
    Cnt() : v(0) {}
    Cnt(double x) : v(x) {}
    friend Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
    friend Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
    friend Cnt operator-(Cnt a) { return Cnt(-a.v); }
    friend Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
    friend Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
    friend bool operator<(Cnt a, Cnt b) { g_ops.cmp++; return a.v < b.v; }
    friend bool operator<=(Cnt a, Cnt b) { g_ops.cmp++; return a.v <= b.v; }
    friend bool operator>(Cnt a, Cnt b) { g_ops.cmp++; return a.v > b.v; }
    friend bool operator>=(Cnt a, Cnt b) { g_ops.cmp++; return a.v >= b.v; }
    friend Cnt sqrt(Cnt a) { g_ops.sqrt++; return Cnt(std::sqrt(a.v)); }
    friend Cnt fabs(Cnt a) { g_ops.cmp++; return Cnt(std::fabs(a.v)); }
    Cnt& operator+=(Cnt b) { return *this = *this + b; }
};

inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
inline double val(Cnt x) { return x.v; }

using std::fabs;
using std::sqrt;

/* min / max that keep the FIRST argument on a tie; the branch taken decides
 * which derivative a Dual carries. */
template <class T> inline T tmin(T a, T b) { return (b < a) ? b : a; }
template <class T> inline T tmax(T a, T b) { return (b > a) ? b : a; }
template <class T> inline T sq(T a) { return a * a; }

/* ------------------------------------------------------------------ */
/* Field layout and EOS coefficients                                   */
/* ------------------------------------------------------------------ */

struct Lay {
    int nf, nd;
    int nq() const { return 2 * nf + nd; }
    int rho(int i) const { return i; }
    int mom(int d) const { return nf + d; }
    int E() const { return nf + nd; }
    int alpha(int j) const { return nf + nd + 1 + j; }
};

/* Mixture-rule coefficients of Sec. 2.1.1 with the EOS of Sec. 2.2:
 * rho e = sum_i alpha_i (p + gamma_i pi_i)/(gamma_i - 1) = Gamma p + Pi,
 * Gamma = sum_i alpha_i g_i,  g_i = 1/(gamma_i - 1),
 * Pi    = sum_i alpha_i h_i,  h_i = gamma_i pi_i/(gamma_i - 1). */
struct Eos {
    int nf;
    int model, riemann, low_mach;
    double g[MAXF], h[MAXF], gam[MAXF], pinf[MAXF], eta[MAXF];
    bool viscous;
    explicit Eos(const oc_problem& P)
        : nf(P.nf), model(P.model), riemann(P.riemann), low_mach(P.low_mach), viscous(false) {
        for (int i = 0; i < nf; ++i) {
            g[i] = 1.0 / (P.gamma[i] - 1.0);
            h[i] = P.gamma[i] * P.pi_inf[i] / (P.gamma[i] - 1.0);
            gam[i] = P.gamma[i];
            pinf[i] = P.pi_inf[i];
            eta[i] = P.eta[i];
            if (P.eta[i] > 0.0) viscous = true;
        }
    }
    /* Gamma and Pi from the N_f - 1 stored volume fractions; the last one is
     * 1 - sum of the others (mixture rule sum alpha_i = 1). */
    template <class T> void mix(const T* alpha_stored, T& Gamma, T& Pi) const {
        T s = T(0.0);
        for (int j = 0; j < nf - 1; ++j) s = s + alpha_stored[j];
        T aN = T(1.0) - s;
        Gamma = aN * g[nf - 1];
        Pi = aN * h[nf - 1];
        for (int j = 0; j < nf - 1; ++j) {
            Gamma = Gamma + alpha_stored[j] * g[j];
            Pi = Pi + alpha_stored[j] * h[j];
        }
    }
};

int g_bad = 0; /* count of non-physical states met (rho <= 0 or c^2 <= 0 / NaN) */

inline void note_bad() {
#pragma omp atomic
    g_bad++;
}

/* Conservative -> primitive (a2): rho = sum alpha_i rho_i, u = (rho u)/rho,
 * p = (rho E - 1/2 rho |u|^2 - Pi)/Gamma. */
template <class T>
void cons_to_prim(const Lay& L, const Eos& eos, const T* q, T* w) {
    T rho = q[L.rho(0)];
    for (int i = 1; i < L.nf; ++i) rho = rho + q[L.rho(i)];
    if (!(val(rho) > 0.0)) note_bad();
    for (int i = 0; i < L.nf; ++i) w[L.rho(i)] = q[L.rho(i)];
    T u2 = T(0.0);
    for (int d = 0; d < L.nd; ++d) {
        w[L.mom(d)] = q[L.mom(d)] / rho;
        u2 = u2 + w[L.mom(d)] * w[L.mom(d)];
    }
    for (int j = 0; j < L.nf - 1; ++j) w[L.alpha(j)] = q[L.alpha(j)];
    T Gamma, Pi;
    eos.mix(q + L.alpha(0), Gamma, Pi);
    T ke = T(0.5) * rho * u2;
    w[L.E()] = (q[L.E()] - ke - Pi) / Gamma;
}

/* Primitive -> conservative: rho E = Gamma p + Pi + 1/2 rho |u|^2. */
template <class T>
void prim_to_cons(const Lay& L, const Eos& eos, const T* w, T* q) {
    T rho = w[L.rho(0)];
    for (int i = 1; i < L.nf; ++i) rho = rho + w[L.rho(i)];
    for (int i = 0; i < L.nf; ++i) q[L.rho(i)] = w[L.rho(i)];
    T u2 = T(0.0);
    for (int d = 0; d < L.nd; ++d) {
        q[L.mom(d)] = rho * w[L.mom(d)];
        u2 = u2 + w[L.mom(d)] * w[L.mom(d)];
    }
    for (int j = 0; j < L.nf - 1; ++j) q[L.alpha(j)] = w[L.alpha(j)];
    T Gamma, Pi;
    eos.mix(w + L.alpha(0), Gamma, Pi);
    q[L.E()] = Gamma * w[L.E()] + Pi + T(0.5) * rho * u2;
}

/* Mixture sound speed (reading: the mixture behaves as a stiffened gas with
 * 1/(gamma_m - 1) = Gamma and gamma_m pi_m/(gamma_m - 1) = Pi, so
 * c^2 = gamma_m (p + pi_m)/rho = ((Gamma + 1) p + Pi)/(Gamma rho); for one
 * fluid it is the phasic c_i of Sec. 2.1.1). */
template <class T> T sound_speed(T rho, T p, T Gamma, T Pi) {
    T c2 = ((Gamma + T(1.0)) * p + Pi) / (Gamma * rho);
    if (!(val(c2) > 0.0)) note_bad();
    return sqrt(c2);
}

/* Kapila model, two fluids (Sec. 2.1.1).  With the phasic sound speeds
 * c_i^2 = gamma_i (p + pi_i)/rho_i, rho_i c_i^2 = Z_i = gamma_i (p + pi_i)
 * needs no phasic density.
 *   K = (Z_2 - Z_1) / (Z_1/alpha_1 + Z_2/alpha_2)
 * (reading: the paper prints Z_2 + Z_1 in the numerator; K must vanish for
 * identical fluids, and the Kapila model has the difference), and the Wood
 * mixture sound speed, 1/(rho c^2) = alpha_1/Z_1 + alpha_2/Z_2 (reading:
 * the sound speed the Kapila model's characteristics carry, used for the
 * HLLC wave speeds and the CFL step of that model). */
template <class T> T kapila_K(const Eos& eos, T p, T a1) {
    T Z1 = T(eos.gam[0]) * (p + T(eos.pinf[0]));
    T Z2 = T(eos.gam[1]) * (p + T(eos.pinf[1]));
    T a2 = T(1.0) - a1;
    return (Z2 - Z1) / (Z1 / a1 + Z2 / a2);
}

template <class T> T wood_c2(const Eos& eos, T rho, T p, T a1) {
    T Z1 = T(eos.gam[0]) * (p + T(eos.pinf[0]));
    T Z2 = T(eos.gam[1]) * (p + T(eos.pinf[1]));
    T a2 = T(1.0) - a1;
    return T(1.0) / (rho * (a1 / Z1 + a2 / Z2));
}

/* Sound speed of the model: the mixture stiffened gas (K = 0) or Wood's
 * (Kapila). */
template <class T> T model_sound_speed(const Lay& L, const Eos& eos, const T* w, T rho, T Gamma, T Pi) {
    if (eos.model == 0) return sound_speed(rho, w[L.E()], Gamma, Pi);
    T c2 = wood_c2(eos, rho, w[L.E()], w[L.alpha(0)]);
    if (!(val(c2) > 0.0)) note_bad();
    return sqrt(c2);
}

/* A primitive state is a physical mixture when rho > 0, Gamma > 0 and
 * (Gamma + 1) p + Pi > 0 (so that c^2 > 0); for the Kapila model also
 * Z_i = gamma_i (p + pi_i) > 0 for both fluids (the Wood c^2 and K). */
template <class T> bool physical_state(const Lay& L, const Eos& eos, const T* w) {
    T rho = w[L.rho(0)];
    for (int i = 1; i < L.nf; ++i) rho = rho + w[L.rho(i)];
    T Gamma, Pi;
    eos.mix(w + L.alpha(0), Gamma, Pi);
    bool ok = val(rho) > 0.0 && val(Gamma) > 0.0 && val((Gamma + T(1.0)) * w[L.E()] + Pi) > 0.0;
    if (eos.model == 1)
        ok = ok && val(w[L.E()]) + eos.pinf[0] > 0.0 && val(w[L.E()]) + eos.pinf[1] > 0.0;
    return ok;
}

/* ------------------------------------------------------------------ */
/* WENO5 (Sec. 3.2.1, Sec. 4.2.2)                                      */
/* ------------------------------------------------------------------ */

/* Reconstruct the value at one edge of the centre cell of the five-cell
 * stencil f[0..4] = f_{c-2} .. f_{c+2}.  right_edge = true gives the left
 * state at face c+1/2, false the right state at face c-1/2.
 * Candidate stencils r = 0, 1, 2 are {c-2,c-1,c}, {c-1,c,c+1}, {c,c+1,c+2};
 * their third-order polynomials, the Jiang-Shu smoothness indicators and the
 * ideal weights (1/10, 6/10, 3/10) (mirrored for the other edge) are the
 * k = 3 uniform-grid case of the generic Lagrange / Delta-f construction of
 * Sec. 4.2.2.  Nonlinear weights: JS, alpha_r = d_r/(eps + beta_r)^2;
 * mapped (Henrick 2005, cited in Sec. 3.2.1), the JS weights pushed through
 * g_r(w) = w (d_r + d_r^2 - 3 d_r w + w^2)/(d_r^2 + w (1 - 2 d_r)) and
 * renormalised; Z (Sec. 4.2.2, q = 1), alpha_r = d_r (1 + tau/(beta_r + eps)),
 * tau = |beta_0 - beta_2|.  TENO (Sec. 4.2.2, K = 5: the same three
 * candidate stencils): gamma_r = d_r (1 + tau/(beta_r + eps))^6,
 * chi_r = gamma_r / sum gamma, delta_r = 0 if chi_r < C_T else 1,
 * omega_r = d_r delta_r / sum d delta.  Reading: chi is evaluated with
 * A_r = 1 + tau/(beta_r + eps) divided by the largest A (a factor common
 * to numerator and denominator), so that A^6 cannot overflow.
 * dbg (optional) receives p[3], beta[3], omega[3]. */
/* Jiang-Shu smoothness indicators of the three candidate stencils
 * (Sec. 4.2.2 with k = 3 on a uniform grid); shared by both edges. */
template <class T> void weno5_beta(const T* f, T* beta) {
    const T c13 = T(13.0 / 12.0), c14 = T(0.25);
    beta[0] = c13 * sq(f[0] - T(2.0) * f[1] + f[2]) + c14 * sq(f[0] - T(4.0) * f[1] + T(3.0) * f[2]);
    beta[1] = c13 * sq(f[1] - T(2.0) * f[2] + f[3]) + c14 * sq(f[1] - f[3]);
    beta[2] = c13 * sq(f[2] - T(2.0) * f[3] + f[4]) + c14 * sq(T(3.0) * f[2] - T(4.0) * f[3] + f[4]);
}

template <class T>
T weno5_edge(const T* f, bool right_edge, int variant, double eps, double ct, T* dbg = nullptr) {
    T p[3], beta[3], d[3];
    if (right_edge) {
        p[0] = (T(2.0) * f[0] - T(7.0) * f[1] + T(11.0) * f[2]) / T(6.0);
        p[1] = (-f[1] + T(5.0) * f[2] + T(2.0) * f[3]) / T(6.0);
        p[2] = (T(2.0) * f[2] + T(5.0) * f[3] - f[4]) / T(6.0);
        d[0] = T(0.1); d[1] = T(0.6); d[2] = T(0.3);
    } else {
        p[0] = (-f[0] + T(5.0) * f[1] + T(2.0) * f[2]) / T(6.0);
        p[1] = (T(2.0) * f[1] + T(5.0) * f[2] - f[3]) / T(6.0);
        p[2] = (T(11.0) * f[2] - T(7.0) * f[3] + T(2.0) * f[4]) / T(6.0);
        d[0] = T(0.3); d[1] = T(0.6); d[2] = T(0.1);
    }
    weno5_beta(f, beta);

    T a[3], w[3];
    if (variant == WENO_Z) {
        T tau = fabs(beta[0] - beta[2]);
        for (int r = 0; r < 3; ++r) a[r] = d[r] * (T(1.0) + tau / (beta[r] + T(eps)));
    } else if (variant == WENO_TENO) {
        T tau = fabs(beta[0] - beta[2]);
        T A[3];
        for (int r = 0; r < 3; ++r) A[r] = T(1.0) + tau / (beta[r] + T(eps));
        T Am = tmax(tmax(A[0], A[1]), A[2]);
        T g[3];
        for (int r = 0; r < 3; ++r) {
            T x = A[r] / Am;
            T x2 = x * x;
            g[r] = d[r] * (x2 * x2 * x2);
        }
        T sg = g[0] + g[1] + g[2];
        for (int r = 0; r < 3; ++r) {
            T chi = g[r] / sg;
            a[r] = (chi < T(ct)) ? T(0.0) : d[r];
        }
    } else {
        for (int r = 0; r < 3; ++r) a[r] = d[r] / sq(T(eps) + beta[r]);
    }
    T s = a[0] + a[1] + a[2];
    for (int r = 0; r < 3; ++r) w[r] = a[r] / s;
    if (variant == WENO_M) {
        T gm[3];
        for (int r = 0; r < 3; ++r)
            gm[r] = w[r] * (d[r] + d[r] * d[r] - T(3.0) * d[r] * w[r] + w[r] * w[r]) /
                    (d[r] * d[r] + w[r] * (T(1.0) - T(2.0) * d[r]));
        T sm = gm[0] + gm[1] + gm[2];
        for (int r = 0; r < 3; ++r) w[r] = gm[r] / sm;
    }
    if (dbg) {
        for (int r = 0; r < 3; ++r) { dbg[r] = p[r]; dbg[3 + r] = beta[r]; dbg[6 + r] = w[r]; }
    }
    return w[0] * p[0] + w[1] * p[1] + w[2] * p[2];
}

/* ------------------------------------------------------------------ */
/* HLLC (Sec. 3.2.2)                                                   */
/* ------------------------------------------------------------------ */

/* HLLC flux across a face with normal along axis d, from the reconstructed
 * primitive states WL, WR.  Readings (the paper gives the structure only):
 *  - wave speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R);
 *  - S* from continuity of normal velocity and pressure across the contact;
 *  - star states U*_K = chi_K (alpha_i rho_i, rho S* / rho u_t,
 *    rho [E/rho + (S* - u)(S* + p/(rho (S_K - u)))]), chi_K = (S_K - u)/(S_K - S*),
 *    and F*_K = F_K + S_K (U*_K - U_K) (Toro);
 *  - side: S* >= 0 takes the left (F_L if S_L >= 0, else F*_L), S* < 0 the
 *    right (F_R if S_R <= 0, else F*_R);
 *  - face velocity u_f = u_K outside the fan, S* inside it (the u^{(x)} of
 *    Sec. 3.2.1); volume-fraction "flux" alpha_f u_f with alpha_f from the
 *    side taken.
 * F receives N_q entries (the alpha slots hold alpha_f u_f); uf the face
 * velocity. */
template <class T>
void hllc(const Lay& L, const Eos& eos, int d, const T* WL0, const T* WR0, T* F, T& uf) {
    /* Thornber's low-Mach correction (Sec. 4.2.4): the normal velocities of
     * the two states are pulled towards their mean by z = min(max(|u_L|/c_L,
     * |u_R|/c_R), 1) before the solve; reading: the modified states replace
     * the reconstructed ones everywhere in the solver (wave speeds, fluxes,
     * star states, total energies). */
    T WLm[MAXQ], WRm[MAXQ];
    for (int k = 0; k < L.nq(); ++k) { WLm[k] = WL0[k]; WRm[k] = WR0[k]; }
    T zlm = T(1.0);
    if (eos.low_mach != 0) {
        T cs[2];
        const T* W0[2] = {WL0, WR0};
        for (int K = 0; K < 2; ++K) {
            T r = W0[K][L.rho(0)];
            for (int i = 1; i < L.nf; ++i) r = r + W0[K][L.rho(i)];
            T Gamma, Pi;
            eos.mix(W0[K] + L.alpha(0), Gamma, Pi);
            cs[K] = model_sound_speed(L, eos, W0[K], r, Gamma, Pi);
        }
        T uL = WL0[L.mom(d)], uR = WR0[L.mom(d)];
        zlm = tmin(tmax(fabs(uL) / cs[0], fabs(uR) / cs[1]), T(1.0));
        if (eos.low_mach == 1) {
            T mean = (uL + uR) / T(2.0);
            WLm[L.mom(d)] = mean + zlm * (uL - uR) / T(2.0);
            WRm[L.mom(d)] = mean + zlm * (uR - uL) / T(2.0);
        }
    }
    const T* WL = WLm;
    const T* WR = WRm;
    const T* W[2] = {WL, WR};
    T rho[2], un[2], p[2], E[2], c[2];
    for (int K = 0; K < 2; ++K) {
        const T* w = W[K];
        T r = w[L.rho(0)];
        for (int i = 1; i < L.nf; ++i) r = r + w[L.rho(i)];
        T u2 = T(0.0);
        for (int e = 0; e < L.nd; ++e) u2 = u2 + w[L.mom(e)] * w[L.mom(e)];
        T Gamma, Pi;
        eos.mix(w + L.alpha(0), Gamma, Pi);
        rho[K] = r;
        un[K] = w[L.mom(d)];
        p[K] = w[L.E()];
        E[K] = Gamma * p[K] + Pi + T(0.5) * r * u2;
        c[K] = model_sound_speed(L, eos, w, r, Gamma, Pi);
    }
    T SL = tmin(un[0] - c[0], un[1] - c[1]);
    T SR = tmax(un[0] + c[0], un[1] + c[1]);
    if (eos.riemann == 1) {
        /* HLL (Sec. 3.2.2): one averaged state between S_L and S_R,
         * F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) for every
         * conserved component, the alpha slots with U = alpha, F = alpha u.
         * Reading: the face velocity of the alpha div u term is the same
         * average of u, (S_R u_L - S_L u_R)/(S_R - S_L), so that a uniform
         * alpha stays uniform. */
        T FK[2][MAXQ], UK[2][MAXQ];
        for (int K = 0; K < 2; ++K) {
            const T* w = W[K];
            for (int i = 0; i < L.nf; ++i) { FK[K][L.rho(i)] = w[L.rho(i)] * un[K]; UK[K][L.rho(i)] = w[L.rho(i)]; }
            for (int e = 0; e < L.nd; ++e) {
                FK[K][L.mom(e)] = rho[K] * un[K] * w[L.mom(e)];
                if (e == d) FK[K][L.mom(e)] = FK[K][L.mom(e)] + p[K];
                UK[K][L.mom(e)] = rho[K] * w[L.mom(e)];
            }
            FK[K][L.E()] = (E[K] + p[K]) * un[K];
            UK[K][L.E()] = E[K];
            for (int j = 0; j < L.nf - 1; ++j) {
                FK[K][L.alpha(j)] = w[L.alpha(j)] * un[K];
                UK[K][L.alpha(j)] = w[L.alpha(j)];
            }
        }
        if (SL >= T(0.0)) {
            for (int k = 0; k < L.nq(); ++k) F[k] = FK[0][k];
            uf = un[0];
        } else if (SR <= T(0.0)) {
            for (int k = 0; k < L.nq(); ++k) F[k] = FK[1][k];
            uf = un[1];
        } else {
            for (int k = 0; k < L.nq(); ++k)
                F[k] = (SR * FK[0][k] - SL * FK[1][k] + SL * SR * (UK[1][k] - UK[0][k])) / (SR - SL);
            uf = (SR * un[0] - SL * un[1]) / (SR - SL);
        }
        return;
    }
    T Ss = (p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1])) /
           (rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]));

    int K;
    T SK;
    bool star;
    if (Ss >= T(0.0)) {
        K = 0; SK = SL; star = SL < T(0.0);
    } else {
        K = 1; SK = SR; star = SR > T(0.0);
    }
    const T* w = W[K];
    /* physical flux of side K */
    for (int i = 0; i < L.nf; ++i) F[L.rho(i)] = w[L.rho(i)] * un[K];
    for (int e = 0; e < L.nd; ++e) {
        F[L.mom(e)] = rho[K] * un[K] * w[L.mom(e)];
        if (e == d) F[L.mom(e)] = F[L.mom(e)] + p[K];
    }
    F[L.E()] = (E[K] + p[K]) * un[K];
    if (star) {
        T chi = (SK - un[K]) / (SK - Ss);
        for (int i = 0; i < L.nf; ++i) {
            T Us = chi * w[L.rho(i)];
            F[L.rho(i)] = F[L.rho(i)] + SK * (Us - w[L.rho(i)]);
        }
        for (int e = 0; e < L.nd; ++e) {
            T Us = chi * rho[K] * (e == d ? Ss : w[L.mom(e)]);
            F[L.mom(e)] = F[L.mom(e)] + SK * (Us - rho[K] * w[L.mom(e)]);
        }
        T Es = chi * rho[K] * (E[K] / rho[K] + (Ss - un[K]) * (Ss + p[K] / (rho[K] * (SK - un[K]))));
        F[L.E()] = F[L.E()] + SK * (Es - E[K]);
        if (eos.low_mach == 2) {
            /* anti-dissipation pressure correction (Sec. 4.2.4) inside the fan:
             * p_d = rho_L rho_R (S_L - u_L)(S_R - u_R)(u_R - u_L) /
             *       (rho_R (S_R - u_R) - rho_L (S_L - u_L)),
             * + (z - 1) p_d on the normal momentum, + (z - 1) p_d S* on the energy */
            T pd = rho[0] * rho[1] * (SL - un[0]) * (SR - un[1]) * (un[1] - un[0]) /
                   (rho[1] * (SR - un[1]) - rho[0] * (SL - un[0]));
            T apc = (zlm - T(1.0)) * pd;
            F[L.mom(d)] = F[L.mom(d)] + apc;
            F[L.E()] = F[L.E()] + apc * Ss;
        }
        uf = Ss;
    } else {
        uf = un[K];
    }
    for (int j = 0; j < L.nf - 1; ++j) F[L.alpha(j)] = w[L.alpha(j)] * uf;
}

/* ------------------------------------------------------------------ */
/* Ghost cells (Sec. 3.3)                                              */
/* ------------------------------------------------------------------ */

/* Map index i along axis ax (possibly outside [0, n)) to the interior cell
 * whose value the ghost cell carries.  Periodic: wrap.  Transmissive
 * (zeroth-order extrapolation): the nearest interior cell.  Reflective
 * (symmetry / slip wall): the mirror image, with the normal momentum
 * negated (flip toggled). */
inline int bc_map(const oc_problem& P, int ax, int i, bool& flip) {
    int n = P.n[ax];
    if (i < 0) {
        switch (P.bc_lo[ax]) {
            case BC_PERIODIC: return i + n;
            case BC_TRANSMISSIVE: return 0;
            default: flip = !flip; return -1 - i;
        }
    }
    if (i >= n) {
        switch (P.bc_hi[ax]) {
            case BC_PERIODIC: return i - n;
            case BC_TRANSMISSIVE: return n - 1;
            default: flip = !flip; return 2 * n - 1 - i;
        }
    }
    return i;
}

struct Idx {
    int c[3];
};

inline int64_t lin(const oc_problem& P, int i, int j, int k) {
    return ((int64_t)k * P.n[1] + j) * P.n[0] + i;
}

/* Whole-domain storage: the conservative state of every interior cell. */
template <class T> struct FullView {
    const oc_problem* P;
    const T* q;
    int64_t ncell;
    void load(int64_t c, T* out) const {
        int nq = 2 * P->nf + P->ndim;
        for (int f = 0; f < nq; ++f) out[f] = q[f * ncell + c];
    }
};

/* Sparse storage: the conservative state of a set of interior cells. */
template <class T> struct MapView {
    const oc_problem* P;
    const std::unordered_map<int64_t, std::array<T, MAXQ>>* m;
    void load(int64_t c, T* out) const {
        const auto& a = m->at(c);
        int nq = 2 * P->nf + P->ndim;
        for (int f = 0; f < nq; ++f) out[f] = a[f];
    }
};

/* Conservative state of cell (i,j,k) where at most one index lies outside the
 * domain (a ghost cell along that axis). */
template <class T, class View>
void fetch(const View& V, const Lay& L, int i, int j, int k, T* out) {
    const oc_problem& P = *V.P;
    int idx[3] = {i, j, k};
    bool flip[3] = {false, false, false};
    for (int ax = 0; ax < 3; ++ax) idx[ax] = bc_map(P, ax, idx[ax], flip[ax]);
    V.load(lin(P, idx[0], idx[1], idx[2]), out);
    for (int ax = 0; ax < L.nd; ++ax)
        if (flip[ax]) out[L.mom(ax)] = -out[L.mom(ax)];
}

/* Flux and face velocity at the face between cell c and c + e_ax.  The six
 * cells c-2 .. c+3 along ax are converted to primitives, the left state is
 * reconstructed from c-2..c+2 and the right state from c-1..c+3, and the
 * HLLC solver gives the flux. */
template <class T, class View>
void face_flux(const View& V, const Lay& L, const Eos& eos, int ax, const int* c, T* F, T& uf) {
    const oc_problem& P = *V.P;
    T W[6][MAXQ], q[MAXQ];
    for (int m = 0; m < 6; ++m) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[ax] += m - 2;
        fetch<T>(V, L, cc[0], cc[1], cc[2], q);
        cons_to_prim(L, eos, q, W[m]);
    }
    T WL[MAXQ], WR[MAXQ], f[5];
    for (int k = 0; k < L.nq(); ++k) {
        for (int m = 0; m < 5; ++m) f[m] = W[m][k];
        WL[k] = weno5_edge(f, true, P.weno, P.eps, P.teno_ct);
        for (int m = 0; m < 5; ++m) f[m] = W[m + 1][k];
        WR[k] = weno5_edge(f, false, P.weno, P.eps, P.teno_ct);
    }
    /* Positivity reading (the paper is silent): if either reconstructed
     * state is not a physical mixture, the face falls back to first-order
     * reconstruction, i.e. the states of its two cells. */
    if (!physical_state(L, eos, WL) || !physical_state(L, eos, WR)) {
        for (int k = 0; k < L.nq(); ++k) {
            WL[k] = W[2][k];
            WR[k] = W[3][k];
        }
    }
    hllc(L, eos, ax, WL, WR, F, uf);
}

inline double dx_of(const oc_problem& P, int ax) { return (P.hi[ax] - P.lo[ax]) / P.n[ax]; }

/* Contribution of direction ax to the right-hand side of cell c, Eq. (rhs):
 * (F_{c-1/2} - F_{c+1/2})/dx, plus alpha_c (u_{c+1/2} - u_{c-1/2})/dx for the
 * volume-fraction rows (the -h(q) div u term with h = (0,..,0,-alpha)); the
 * Kapila model adds K_c (u_{c+1/2} - u_{c-1/2})/dx to the alpha_1 row
 * (alpha_1_t + u . grad alpha_1 = K div u, Sec. 2.1.1), K_c from the cell's
 * own pressure and volume fraction (Kc = 0 for K = 0). */
template <class T>
void cell_term(const Lay& L, double dx, const T* Fm, T um, const T* Fp, T up, const T* qc, T Kc, bool kapila,
               T* t) {
    for (int k = 0; k < L.nq(); ++k) t[k] = (Fm[k] - Fp[k]) / T(dx);
    for (int j = 0; j < L.nf - 1; ++j) {
        int k = L.alpha(j);
        if (kapila)
            t[k] = t[k] + (qc[k] + Kc) * (up - um) / T(dx);
        else
            t[k] = t[k] + qc[k] * (up - um) / T(dx);
    }
}

/* K of cell state qc (conservative) for the Kapila model. */
template <class T> T cell_K(const Lay& L, const Eos& eos, const T* qc) {
    if (eos.model == 0) return T(0.0);
    T w[MAXQ];
    cons_to_prim(L, eos, qc, w);
    return kapila_K(eos, w[L.E()], w[L.alpha(0)]);
}

/* ------------------------------------------------------------------ */
/* Viscous stress (Sec. 2.1.1)                                         */
/* ------------------------------------------------------------------ */

/* T^v = 2 eta (D - tr(D) I/3) with D = (grad u + (grad u)^T)/2, i.e.
 *   T_ab = eta (d_a u_b + d_b u_a) - 2/3 eta (div u) delta_ab,
 * enters the momentum flux as -T and the energy flux as -T.u (Sec. 2.1.1).
 * Readings (the paper states neither):
 *   - mixture viscosity eta = sum_i alpha_i eta_i, alpha_N = 1 - sum_j alpha_j;
 *   - the stress is evaluated on each face by second-order central
 *     differences of the cell velocities u = (rho u)/rho: on the face
 *     between cells A = c and B = c + e_ax,
 *       d_ax u_b = (u_b(B) - u_b(A)) / dx_ax,
 *       d_t u_b  = ((u_b(A + e_t) - u_b(A - e_t)) + (u_b(B + e_t) - u_b(B - e_t))) / (4 dx_t),  t != ax,
 *     the face velocity and the face volume fractions being the means of
 *     A's and B's;
 *   - ghost cells as for the inviscid flux (a reflective wall mirrors the
 *     velocity with its normal component negated, i.e. a slip wall).
 * The viscous right-hand side of a cell sums (G_{c-1/2} - G_{c+1/2})/dx over
 * the directions in axis order, G being the viscous flux; it is the value
 * L(q) starts from, the inviscid directional terms being added to it. */
template <class T, class View>
void cell_velocity(const View& V, const Lay& L, const int* c, T* q, T* u) {
    fetch<T>(V, L, c[0], c[1], c[2], q);
    T rho = q[L.rho(0)];
    for (int i = 1; i < L.nf; ++i) rho = rho + q[L.rho(i)];
    for (int d = 0; d < L.nd; ++d) u[d] = q[L.mom(d)] / rho;
}

template <class T, class View>
void viscous_face_flux(const View& V, const Lay& L, const Eos& eos, int ax, const int* c, T* G) {
    const oc_problem& P = *V.P;
    const int nd = L.nd;
    int A[3] = {c[0], c[1], c[2]}, B[3] = {c[0], c[1], c[2]};
    B[ax] += 1;
    T qA[MAXQ], qB[MAXQ], uA[3], uB[3], tmp[MAXQ];
    cell_velocity(V, L, A, qA, uA);
    cell_velocity(V, L, B, qB, uB);
    T g[3][3];  // g[a][b] = d_a u_b on the face
    for (int b = 0; b < nd; ++b) g[ax][b] = (uB[b] - uA[b]) / T(dx_of(P, ax));
    for (int t = 0; t < nd; ++t) {
        if (t == ax) continue;
        int Ap[3] = {A[0], A[1], A[2]}, Am[3] = {A[0], A[1], A[2]};
        int Bp[3] = {B[0], B[1], B[2]}, Bm[3] = {B[0], B[1], B[2]};
        Ap[t] += 1;
        Am[t] -= 1;
        Bp[t] += 1;
        Bm[t] -= 1;
        T uAp[3], uAm[3], uBp[3], uBm[3];
        cell_velocity(V, L, Ap, tmp, uAp);
        cell_velocity(V, L, Am, tmp, uAm);
        cell_velocity(V, L, Bp, tmp, uBp);
        cell_velocity(V, L, Bm, tmp, uBm);
        for (int b = 0; b < nd; ++b)
            g[t][b] = ((uAp[b] - uAm[b]) + (uBp[b] - uBm[b])) / T(4.0 * dx_of(P, t));
    }
    T div = g[0][0];
    for (int d = 1; d < nd; ++d) div = div + g[d][d];
    T s = T(0.0), af[MAXF];
    for (int j = 0; j < L.nf - 1; ++j) {
        af[j] = (qA[L.alpha(j)] + qB[L.alpha(j)]) * T(0.5);
        s = s + af[j];
    }
    T eta = (T(1.0) - s) * T(eos.eta[L.nf - 1]);
    for (int j = 0; j < L.nf - 1; ++j) eta = eta + af[j] * T(eos.eta[j]);
    for (int k = 0; k < L.nq(); ++k) G[k] = T(0.0);
    T work = T(0.0);
    for (int b = 0; b < nd; ++b) {
        T Tab = eta * (g[ax][b] + g[b][ax]);
        if (b == ax) Tab = Tab - T(2.0 / 3.0) * eta * div;
        const T uf = (uA[b] + uB[b]) * T(0.5);
        work = (b == 0) ? Tab * uf : work + Tab * uf;
        G[L.mom(b)] = -Tab;
    }
    G[L.E()] = -work;
}

template <class T, class View>
void viscous_cell(const View& V, const Lay& L, const Eos& eos, const int* c, T* Vc) {
    const oc_problem& P = *V.P;
    for (int k = 0; k < L.nq(); ++k) Vc[k] = T(0.0);
    for (int ax = 0; ax < P.ndim; ++ax) {
        T Gm[MAXQ], Gp[MAXQ];
        int cm[3] = {c[0], c[1], c[2]};
        cm[ax] -= 1;
        viscous_face_flux(V, L, eos, ax, cm, Gm);
        viscous_face_flux(V, L, eos, ax, c, Gp);
        for (int k = 0; k < L.nq(); ++k) Vc[k] = Vc[k] + (Gm[k] - Gp[k]) / T(dx_of(P, ax));
    }
}

/* Right-hand side L(q) on every interior cell. */
template <class T>
void rhs_full(const oc_problem& P, const T* q, T* Lout) {
    Lay L{P.nf, P.ndim};
    Eos eos(P);
    const int nq = L.nq();
    const int64_t ncell = (int64_t)P.n[0] * P.n[1] * P.n[2];
    FullView<T> V{&P, q, ncell};
    for (int64_t i = 0; i < (int64_t)nq * ncell; ++i) Lout[i] = T(0.0);
    if (eos.viscous) {
#pragma omp parallel for schedule(static)
        for (int64_t cl = 0; cl < ncell; ++cl) {
            int c[3] = {(int)(cl % P.n[0]), (int)((cl / P.n[0]) % P.n[1]), (int)(cl / ((int64_t)P.n[0] * P.n[1]))};
            T Vc[MAXQ];
            viscous_cell(V, L, eos, c, Vc);
            for (int f = 0; f < nq; ++f) Lout[f * ncell + cl] = Vc[f];
        }
    }
    for (int ax = 0; ax < P.ndim; ++ax) {
        const int n = P.n[ax];
        const double dx = dx_of(P, ax);
        /* iterate over the lines along ax (each line writes only its own cells) */
        const int t1 = (ax == 0) ? 1 : 0, t2 = (ax == 2) ? 1 : 2;
        const int64_t nlines = (int64_t)P.n[t1] * P.n[t2];
#pragma omp parallel for schedule(static)
        for (int64_t line = 0; line < nlines; ++line) {
            std::vector<std::array<T, MAXQ>> F(n + 1);
            std::vector<T> uf(n + 1);
            int c[3];
            c[t1] = (int)(line % P.n[t1]);
            c[t2] = (int)(line / P.n[t1]);
            for (int s = -1; s < n; ++s) { /* face s+1/2, stored at s+1 */
                c[ax] = s;
                face_flux(V, L, eos, ax, c, F[s + 1].data(), uf[s + 1]);
            }
            for (int s = 0; s < n; ++s) {
                c[ax] = s;
                int64_t cl = lin(P, c[0], c[1], c[2]);
                T qc[MAXQ], t[MAXQ];
                V.load(cl, qc);
                T Kc = cell_K(L, eos, qc);
                cell_term(L, dx, F[s].data(), uf[s], F[s + 1].data(), uf[s + 1], qc, Kc, eos.model == 1, t);
                for (int k = 0; k < nq; ++k) Lout[k * ncell + cl] = Lout[k * ncell + cl] + t[k];
            }
        }
    }
}

/* Right-hand side at a single interior cell (both faces per direction are
 * computed by face_flux exactly as rhs_full does, so the result is bitwise
 * identical to rhs_full at that cell). */
template <class T, class View>
void rhs_cell(const View& V, const Lay& L, const Eos& eos, const int* c, T* Lc) {
    const oc_problem& P = *V.P;
    if (eos.viscous)
        viscous_cell(V, L, eos, c, Lc);
    else
        for (int k = 0; k < L.nq(); ++k) Lc[k] = T(0.0);
    T qc[MAXQ];
    fetch<T>(V, L, c[0], c[1], c[2], qc);
    T Kc = cell_K(L, eos, qc);
    for (int ax = 0; ax < P.ndim; ++ax) {
        T Fm[MAXQ], Fp[MAXQ], um, up, t[MAXQ];
        int cm[3] = {c[0], c[1], c[2]};
        cm[ax] -= 1;
        face_flux(V, L, eos, ax, cm, Fm, um);
        face_flux(V, L, eos, ax, c, Fp, up);
        cell_term(L, dx_of(P, ax), Fm, um, Fp, up, qc, Kc, eos.model == 1, t);
        for (int k = 0; k < L.nq(); ++k) Lc[k] = Lc[k] + t[k];
    }
}

/* ------------------------------------------------------------------ */
/* TVD-RK3 (Sec. 3.4)                                                  */
/* ------------------------------------------------------------------ */

/* Shu-Osher form:
 *   q1 = qn + dt L(qn)
 *   q2 = 3/4 qn + 1/4 (q1 + dt L(q1))
 *   q^{n+1} = 1/3 qn + 2/3 (q2 + dt L(q2)). */
const double RK_A2 = 0.75, RK_B2 = 0.25, RK_A3 = 1.0 / 3.0, RK_B3 = 2.0 / 3.0;

template <class T, class RhsFn>
void rk3_generic(int64_t n, T* q, double dt, RhsFn rhs) {
    std::vector<T> q1(n), q2(n), Lb(n);
    rhs(q, Lb.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) q1[i] = q[i] + T(dt) * Lb[i];
    rhs(q1.data(), Lb.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) q2[i] = T(RK_A2) * q[i] + T(RK_B2) * (q1[i] + T(dt) * Lb[i]);
    rhs(q2.data(), Lb.data());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) q[i] = T(RK_A3) * q[i] + T(RK_B3) * (q2[i] + T(dt) * Lb[i]);
}

template <class T> void rk3_step(const oc_problem& P, T* q, double dt) {
    const int nq = 2 * P.nf + P.ndim;
    const int64_t n = (int64_t)nq * P.n[0] * P.n[1] * P.n[2];
    rk3_generic(n, q, dt, [&](const T* in, T* out) { rhs_full(P, in, out); });
}

/* CFL time step: CFL * min over interior cells and active directions of
 * dx_d / (|u_d| + c) (the paper states the CFL form of neither). */
template <class T> double cfl_dt(const oc_problem& P, const T* q, double cfl) {
    Lay L{P.nf, P.ndim};
    Eos eos(P);
    const int nq = L.nq();
    const int64_t ncell = (int64_t)P.n[0] * P.n[1] * P.n[2];
    FullView<T> V{&P, q, ncell};
    double m = INFINITY;
    /* a minimum: the same value whatever the order of the cells */
#pragma omp parallel for schedule(static) reduction(min : m)
    for (int64_t c = 0; c < ncell; ++c) {
        T qc[MAXQ], w[MAXQ];
        V.load(c, qc);
        cons_to_prim(L, eos, qc, w);
        T rho = qc[L.rho(0)];
        for (int i = 1; i < L.nf; ++i) rho = rho + qc[L.rho(i)];
        T Gamma, Pi;
        eos.mix(qc + L.alpha(0), Gamma, Pi);
        T cs = model_sound_speed(L, eos, w, rho, Gamma, Pi);
        for (int ax = 0; ax < P.ndim; ++ax) {
            T s = T(dx_of(P, ax)) / (fabs(w[L.mom(ax)]) + cs);
            m = std::min(m, val(s));
        }
        /* Reading (the paper states no viscous time-step bound): with
         * viscous_dt, also the explicit limit of the momentum diffusion,
         * rho min_d dx_d^2 / (2 ndim eta), eta the mixture viscosity
         * (1 - sum_j alpha_j) eta_N + sum_j alpha_j eta_j of the cell. */
        if (P.viscous_dt && eos.viscous) {
            T sa = T(0.0);
            for (int j = 0; j < L.nf - 1; ++j) sa = sa + qc[L.alpha(j)];
            T eta = (T(1.0) - sa) * T(eos.eta[L.nf - 1]);
            for (int j = 0; j < L.nf - 1; ++j) eta = eta + qc[L.alpha(j)] * T(eos.eta[j]);
            if (val(eta) > 0.0) {
                double dx2 = dx_of(P, 0) * dx_of(P, 0);
                for (int ax = 1; ax < P.ndim; ++ax) dx2 = std::min(dx2, dx_of(P, ax) * dx_of(P, ax));
                T s = rho * T(dx2) / (T(2.0 * P.ndim) * eta);
                m = std::min(m, val(s));
            }
        }
        (void)nq;
    }
    return cfl * m;
}

int check_problem(const oc_problem* P) {
    if (!P) return -1;
    if (P->ndim < 1 || P->ndim > 3 || P->nf < 1 || P->nf > MAXF) return -1;
    for (int ax = 0; ax < 3; ++ax) {
        if (ax < P->ndim) {
            if (P->n[ax] < 1) return -1;
            if (!(P->hi[ax] > P->lo[ax])) return -1;
            for (int s = 0; s < 2; ++s) {
                int bc = s ? P->bc_hi[ax] : P->bc_lo[ax];
                if (bc < 0 || bc > 2) return -1;
                if (bc != BC_TRANSMISSIVE && P->n[ax] < 3) return -1;
            }
            if ((P->bc_lo[ax] == BC_PERIODIC) != (P->bc_hi[ax] == BC_PERIODIC)) return -1;
        } else if (P->n[ax] != 1) {
            return -1;
        }
    }
    for (int i = 0; i < P->nf; ++i)
        if (!(P->gamma[i] > 1.0) || !(P->pi_inf[i] >= 0.0)) return -1;
    if (P->weno < 0 || P->weno > 3 || !(P->eps > 0.0)) return -1;
    if (P->weno == WENO_TENO && !(P->teno_ct > 0.0 && P->teno_ct < 1.0)) return -1;
    if (P->model < 0 || P->model > 1 || (P->model == 1 && P->nf != 2)) return -1;
    if (P->riemann < 0 || P->riemann > 1 || P->low_mach < 0 || P->low_mach > 2) return -1;
    if (P->low_mach == 2 && P->riemann != 0) return -1;
    for (int i = 0; i < P->nf; ++i)
        if (!(P->eta[i] >= 0.0) || !std::isfinite(P->eta[i])) return -1;
    if (P->viscous_dt != 0 && P->viscous_dt != 1) return -1;
    return 0;
}

inline int64_t ncells(const oc_problem* P) { return (int64_t)P->n[0] * P->n[1] * P->n[2]; }
inline int nfields(const oc_problem* P) { return 2 * P->nf + P->ndim; }

}  // namespace

/* ------------------------------------------------------------------ */
/* C entry points (ctypes)                                             */
/* ------------------------------------------------------------------ */
extern "C" {

/* Threads the loops over lines and cells use: 1 in the single-threaded
 * build, the OpenMP default (all host cores, or OMP_NUM_THREADS) otherwise. */
int oc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oc_nfields(const oc_problem* P) { return check_problem(P) ? -1 : nfields(P); }

int oc_prim_to_cons(const oc_problem* P, const double* w, double* q) {
    if (check_problem(P)) return -1;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    int64_t nc = ncells(P);
    for (int64_t c = 0; c < nc; ++c) {
        double wi[MAXQ], qo[MAXQ];
        for (int k = 0; k < L.nq(); ++k) wi[k] = w[k * nc + c];
        prim_to_cons(L, eos, wi, qo);
        for (int k = 0; k < L.nq(); ++k) q[k * nc + c] = qo[k];
    }
    return 0;
}

int oc_cons_to_prim(const oc_problem* P, const double* q, double* w) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    int64_t nc = ncells(P);
    for (int64_t c = 0; c < nc; ++c) {
        double qi[MAXQ], wo[MAXQ];
        for (int k = 0; k < L.nq(); ++k) qi[k] = q[k * nc + c];
        cons_to_prim(L, eos, qi, wo);
        for (int k = 0; k < L.nq(); ++k) w[k * nc + c] = wo[k];
    }
    return g_bad;
}

/* Returns dt (> 0), or -1 on a bad problem. */
double oc_dt(const oc_problem* P, const double* q, double cfl) {
    if (check_problem(P)) return -1.0;
    return cfl_dt(*P, q, cfl);
}

/* L(q) on every interior cell.  Returns the number of non-physical states met. */
int oc_rhs(const oc_problem* P, const double* q, double* Lout) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    rhs_full(*P, q, Lout);
    return g_bad;
}

/* The viscous part of L(q) alone (zero when every eta_i is 0). */
int oc_viscous_rhs(const oc_problem* P, const double* q, double* Vout) {
    if (check_problem(P)) return -1;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    const int64_t nc = ncells(P);
    FullView<double> V{P, q, nc};
    for (int k = 0; k < P->n[2]; ++k)
        for (int j = 0; j < P->n[1]; ++j)
            for (int i = 0; i < P->n[0]; ++i) {
                int c[3] = {i, j, k};
                double Vc[MAXQ];
                viscous_cell(V, L, eos, c, Vc);
                for (int f = 0; f < L.nq(); ++f) Vout[f * nc + lin(*P, i, j, k)] = Vc[f];
            }
    return 0;
}

/* One RK3 step in place with the given dt. */
int oc_rk3_step(const oc_problem* P, double* q, double dt) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    rk3_step(*P, q, dt);
    return g_bad;
}

/* nsteps RK3 steps in place.  dt_in (nullable): fixed per-step dt; else the
 * CFL dt of each step's initial state.  dt_out (nullable) receives the dts. */
int oc_rk3_run(const oc_problem* P, double* q, int nsteps, double cfl, const double* dt_in, double* dt_out) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = dt_in ? dt_in[s] : cfl_dt(*P, q, cfl);
        if (dt_out) dt_out[s] = dt;
        rk3_step(*P, q, dt);
    }
    return g_bad;
}

/* Forward-mode derivative of L: dL = (dL/dq) dq. */
int oc_rhs_jvp(const oc_problem* P, const double* q, const double* dq, double* Lout, double* dL) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    int64_t n = (int64_t)nfields(P) * ncells(P);
    std::vector<Dual> qd(n), Ld(n);
    for (int64_t i = 0; i < n; ++i) qd[i] = Dual(q[i], dq[i]);
    rhs_full(*P, qd.data(), Ld.data());
    for (int64_t i = 0; i < n; ++i) {
        if (Lout) Lout[i] = Ld[i].v;
        dL[i] = Ld[i].d;
    }
    return g_bad;
}

/* Forward-mode derivative of one RK3 step at fixed dt, in place on (q, dq). */
int oc_rk3_step_jvp(const oc_problem* P, double* q, double* dq, double dt) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    int64_t n = (int64_t)nfields(P) * ncells(P);
    std::vector<Dual> qd(n);
    for (int64_t i = 0; i < n; ++i) qd[i] = Dual(q[i], dq[i]);
    rk3_step(*P, qd.data(), dt);
    for (int64_t i = 0; i < n; ++i) {
        q[i] = qd[i].v;
        dq[i] = qd[i].d;
    }
    return g_bad;
}

/* One RK3 step evaluated only at the listed cells, through their domain of
 * dependence: stage 3 at the cell needs q2 on its stencil, stage 2 there
 * needs q1 on theirs.  cells holds (i, j, k) triples; out receives
 * ncell_out x nfields values (cell-major).  Same arithmetic as oc_rk3_step. */
int oc_rk3_step_sampled(const oc_problem* P, const double* q, double dt, int64_t nsample,
                        const int64_t* cells, double* out) {
    if (check_problem(P)) return -1;
    g_bad = 0;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    const int nq = L.nq();
    const int64_t nc = ncells(P);
    FullView<double> V0{P, q, nc};
    auto decode = [&](int64_t c, int* ijk) {
        ijk[0] = (int)(c % P->n[0]);
        ijk[1] = (int)((c / P->n[0]) % P->n[1]);
        ijk[2] = (int)(c / ((int64_t)P->n[0] * P->n[1]));
    };
    /* cells the right-hand side of the cells in S reads: +-3 along each
     * axis, and with viscosity the cells one step along two axes */
    auto closure = [&](const std::unordered_set<int64_t>& S) {
        std::unordered_set<int64_t> R = S;
        for (int64_t c : S) {
            int ijk[3];
            decode(c, ijk);
            for (int ax = 0; ax < P->ndim; ++ax)
                for (int m = -3; m <= 3; ++m) {
                    int id[3] = {ijk[0], ijk[1], ijk[2]};
                    bool fl = false;
                    id[ax] = bc_map(*P, ax, id[ax] + m, fl);
                    R.insert(lin(*P, id[0], id[1], id[2]));
                }
            if (eos.viscous)
                for (int a = 0; a < P->ndim; ++a)
                    for (int b = a + 1; b < P->ndim; ++b)
                        for (int sa = -1; sa <= 1; sa += 2)
                            for (int sb = -1; sb <= 1; sb += 2) {
                                int id[3] = {ijk[0], ijk[1], ijk[2]};
                                bool fl = false;
                                id[a] = bc_map(*P, a, id[a] + sa, fl);
                                id[b] = bc_map(*P, b, id[b] + sb, fl);
                                R.insert(lin(*P, id[0], id[1], id[2]));
                            }
        }
        return R;
    };
    for (int64_t s = 0; s < nsample; ++s) {
        int tgt[3] = {(int)cells[3 * s], (int)cells[3 * s + 1], (int)cells[3 * s + 2]};
        for (int ax = 0; ax < 3; ++ax)
            if (tgt[ax] < 0 || tgt[ax] >= P->n[ax]) return -1;
        std::unordered_set<int64_t> S3 = {lin(*P, tgt[0], tgt[1], tgt[2])};
        auto S2 = closure(S3);
        auto S1 = closure(S2);
        std::unordered_map<int64_t, std::array<double, MAXQ>> m1, m2;
        for (int64_t c : S1) {
            int ijk[3];
            decode(c, ijk);
            double Lc[MAXQ], qc[MAXQ];
            rhs_cell(V0, L, eos, ijk, Lc);
            V0.load(c, qc);
            std::array<double, MAXQ> a{};
            for (int k = 0; k < nq; ++k) a[k] = qc[k] + dt * Lc[k];
            m1[c] = a;
        }
        MapView<double> V1{P, &m1};
        for (int64_t c : S2) {
            int ijk[3];
            decode(c, ijk);
            double Lc[MAXQ], qc[MAXQ];
            rhs_cell(V1, L, eos, ijk, Lc);
            V0.load(c, qc);
            std::array<double, MAXQ> a{};
            for (int k = 0; k < nq; ++k) a[k] = RK_A2 * qc[k] + RK_B2 * (m1[c][k] + dt * Lc[k]);
            m2[c] = a;
        }
        MapView<double> V2{P, &m2};
        {
            double Lc[MAXQ], qc[MAXQ];
            int64_t c = *S3.begin();
            rhs_cell(V2, L, eos, tgt, Lc);
            V0.load(c, qc);
            for (int k = 0; k < nq; ++k) out[s * nq + k] = RK_A3 * qc[k] + RK_B3 * (m2[c][k] + dt * Lc[k]);
        }
    }
    return g_bad;
}

/* Floating-point operations of one RK3 step (incl. the CFL dt when cfl > 0),
 * as the oracle performs them: counts = {add/sub, mul, div, sqrt, cmp}. */
int oc_rk3_step_count(const oc_problem* P, const double* q, double dt, int64_t* counts) {
    if (check_problem(P)) return -1;
    int64_t n = (int64_t)nfields(P) * ncells(P);
    std::vector<Cnt> qc(n);
    for (int64_t i = 0; i < n; ++i) qc[i] = Cnt(q[i]);
    g_ops = {0, 0, 0, 0, 0};
    rk3_step(*P, qc.data(), dt);
    counts[0] = g_ops.add; counts[1] = g_ops.mul; counts[2] = g_ops.div;
    counts[3] = g_ops.sqrt; counts[4] = g_ops.cmp;
    return 0;
}

/* Operation counts of each building block, one call each, on the given cell
 * states (conservative qa, qb of two neighbouring cells; the face uses qa as
 * the left and qb as the right primitive state after conversion):
 * row 0 cons_to_prim, row 1 one WENO5 edge value, row 2 HLLC, row 3 the cell
 * term of one direction, row 4 one RK3 stage update of one cell (the costlier
 * stage form a*qn + b*(q + dt*L)), row 5 the CFL quantity of one cell,
 * row 6 the smoothness indicators of one five-cell stencil (shared by the
 * two edge values of a cell), row 7 the physical-state test of both
 * reconstructed states of one face.  out: 8 rows x 5 counts. */
int oc_block_counts(const oc_problem* P, const double* qa, const double* qb, int64_t* out) {
    if (check_problem(P)) return -1;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    const int nq = L.nq();
    Cnt a[MAXQ], b[MAXQ], wa[MAXQ], wb[MAXQ], F[MAXQ], uf;
    for (int k = 0; k < nq; ++k) { a[k] = Cnt(qa[k]); b[k] = Cnt(qb[k]); }
    auto take = [&](int row) {
        out[row * 5 + 0] = g_ops.add; out[row * 5 + 1] = g_ops.mul; out[row * 5 + 2] = g_ops.div;
        out[row * 5 + 3] = g_ops.sqrt; out[row * 5 + 4] = g_ops.cmp;
        g_ops = {0, 0, 0, 0, 0};
    };
    g_ops = {0, 0, 0, 0, 0};
    cons_to_prim(L, eos, a, wa);
    take(0);
    cons_to_prim(L, eos, b, wb);
    g_ops = {0, 0, 0, 0, 0};
    Cnt f[5] = {wa[0], wb[0], wa[0], wb[0], wa[0]};
    weno5_edge(f, true, P->weno, P->eps, P->teno_ct);
    take(1);
    hllc(L, eos, 0, wa, wb, F, uf);
    take(2);
    Cnt t[MAXQ];
    cell_term(L, 1.0, F, uf, F, uf, a, Cnt(0.0), false, t);
    take(3);
    for (int k = 0; k < nq; ++k) t[k] = Cnt(RK_A2) * a[k] + Cnt(RK_B2) * (b[k] + Cnt(1e-3) * F[k]);
    take(4);
    {
        Cnt rho = a[L.rho(0)];
        for (int i = 1; i < L.nf; ++i) rho = rho + a[L.rho(i)];
        Cnt Gamma, Pi;
        eos.mix(a + L.alpha(0), Gamma, Pi);
        Cnt cs = sound_speed(rho, wa[L.E()], Gamma, Pi);
        for (int ax = 0; ax < P->ndim; ++ax) {
            Cnt s = Cnt(1.0) / (fabs(wa[L.mom(ax)]) + cs);
            (void)s;
        }
    }
    take(5);
    Cnt bt[3];
    weno5_beta(f, bt);
    take(6);
    physical_state(L, eos, wa);
    physical_state(L, eos, wb);
    take(7);
    return 0;
}

/* One WENO5 stencil, for pinning the constants and weights:
 * out[0..2] candidate values at the right edge, [3..5] beta, [6..8] weights,
 * [9] right-edge value; [10..12] candidates at the left edge, [13..15]
 * weights, [16] left-edge value. */
void oc_weno5_detail(int variant, double eps, double ct, const double* f, double* out) {
    double dbg[9];
    out[9] = weno5_edge(f, true, variant, eps, ct, dbg);
    for (int i = 0; i < 9; ++i) out[i] = dbg[i];
    out[16] = weno5_edge(f, false, variant, eps, ct, dbg);
    for (int i = 0; i < 3; ++i) { out[10 + i] = dbg[i]; out[13 + i] = dbg[6 + i]; }
}

/* HLLC flux for one face from primitive states (N_q each) along axis dir. */
int oc_hllc_face(const oc_problem* P, int dir, const double* WL, const double* WR, double* F, double* uf) {
    if (check_problem(P) || dir < 0 || dir >= P->ndim) return -1;
    g_bad = 0;
    Lay L{P->nf, P->ndim};
    Eos eos(*P);
    double u;
    hllc(L, eos, dir, WL, WR, F, u);
    *uf = u;
    return g_bad;
}

/* The RK3 combination applied to the scalar linear ODE y' = lambda y. */
double oc_rk3_linear(double lambda, double y0, double dt) {
    double y = y0;
    rk3_generic(1, &y, dt, [&](const double* in, double* out) { out[0] = lambda * in[0]; });
    return y;
}

}  /* extern "C" */
