// Viscous stress of the five-equation model (Sec. 2.1.1):
//   T = 2 eta (D - tr(D) I/3),  D = (grad u + (grad u)^T)/2,
// i.e. T_ab = eta (d_a u_b + d_b u_a) - 2/3 eta (div u) delta_ab, entering
// the momentum flux as -T and the energy flux as -T.u.  The mixture
// viscosity is eta = sum_i alpha_i eta_i (alpha_N = 1 - sum of the stored
// fractions).  The stress is evaluated on each face by second-order central
// differences of the cell velocities: on the face between A = c and
// B = c + e_ax,
//   d_ax u_b = (u_b(B) - u_b(A)) / dx_ax,
//   d_t u_b  = ((u_b(A + e_t) - u_b(A - e_t)) + (u_b(B + e_t) - u_b(B - e_t))) / (4 dx_t),  t != ax,
// with the face velocity and volume fractions the means of A's and B's.
// Ghost cells follow the inviscid rules (a reflective wall mirrors the
// velocity with its normal component negated).
//
// Two kernels per evaluation of L.  velocity_kernel stores u = (rho u)/rho
// of every interior cell, in the mode's precision, in a scratch with the
// state's padded layout.  viscous_kernel gives each interior cell
//   V_c = sum over the axes, in axis order, of (G_{c-1/2} - G_{c+1/2}) / dx,
// G being the viscous flux, and stores it (every row; only the momentum and
// energy rows are non-zero) as the value the directional sweeps then
// accumulate onto: rhs in float64, the float accumulator in the mixed mode.
// MODE_EXACT follows the defining formulas operation by operation (IEEE
// division, no contraction); MODE_FAST multiplies by reciprocals of the
// spacings; MODE_MIXED works in float32.  Each face flux is evaluated by
// both cells that share it; the velocities come through L1 / L2.
#pragma once

#include "mfc_device.cuh"

namespace mfc {

template <int NF, int ND, int MODE>
__global__ void __launch_bounds__(256) velocity_kernel(const Consts C, const double* __restrict__ q,
                                                       typename ModeT<MODE>::R* __restrict__ vel) {
    using L = Lay<NF, ND>;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = lin % C.n[0];
        const int64_t j = (lin / C.n[0]) % C.n[1];
        const int64_t k = lin / (C.n[0] * C.n[1]);
        const int64_t off = C.origin + i * C.stride[0] + j * C.stride[1] + k * C.stride[2];
        if constexpr (MODE == MODE_MIXED) {
            float rho = float(__ldg(q + off));
#pragma unroll
            for (int f = 1; f < NF; ++f) rho = rho + float(__ldg(q + off + f * C.fstride));
            const float irho = rcp<float>(rho);
#pragma unroll
            for (int d = 0; d < ND; ++d)
                vel[d * C.fstride + off] = float(__ldg(q + off + (L::MOM + d) * C.fstride)) * irho;
        } else {
            double rho = __ldg(q + off);
#pragma unroll
            for (int f = 1; f < NF; ++f) rho = rho + __ldg(q + off + f * C.fstride);
            if constexpr (MODE == MODE_EXACT) {
#pragma unroll
                for (int d = 0; d < ND; ++d) vel[d * C.fstride + off] = __ldg(q + off + (L::MOM + d) * C.fstride) / rho;
            } else {
                const double irho = rcp_nr(rho);
#pragma unroll
                for (int d = 0; d < ND; ++d) vel[d * C.fstride + off] = __ldg(q + off + (L::MOM + d) * C.fstride) * irho;
            }
        }
    }
}

// Phasic viscosity i in the precision R.
template <class R> __device__ __forceinline__ R eta_of(const Consts& C, int i);
template <> __device__ __forceinline__ double eta_of<double>(const Consts& C, int i) { return C.eta[i]; }
template <> __device__ __forceinline__ float eta_of<float>(const Consts& C, int i) { return C.etaf[i]; }

template <int NF, int ND, int MODE>
__global__ void __launch_bounds__(128) viscous_kernel(const Consts C, const double* __restrict__ q,
                                                      const typename ModeT<MODE>::R* __restrict__ vel,
                                                      double* __restrict__ rhs, float* __restrict__ rhsf) {
    using L = Lay<NF, ND>;
    using R = typename ModeT<MODE>::R;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];

    // offset of cell (c0, c1, c2) after the ghost rules, and the axes whose
    // reflection negates the velocity component along them
    auto source = [&](const int64_t* cc, bool* fl) -> int64_t {
        int64_t o = C.origin;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            fl[a] = false;
            int64_t id = cc[a];
            if (a < ND) id = bc_source(id, C.n[a], C.bc_lo[a], C.bc_hi[a], fl[a]);
            o += id * C.stride[a];
        }
        return o;
    };
    auto vel_at = [&](const int64_t* cc, R* u, int64_t& o) {
        bool fl[3];
        o = source(cc, fl);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const R v = vel[d * C.fstride + o];
            u[d] = fl[d] ? -v : v;
        }
    };
    auto quot = [&](R a, int ax, bool four) -> R {
        if constexpr (MODE == MODE_EXACT) {
            return four ? a / (4.0 * C.dx[ax]) : a / C.dx[ax];
        } else if constexpr (MODE == MODE_FAST) {
            return a * (four ? 0.25 * C.inv_dx[ax] : C.inv_dx[ax]);
        } else {
            return a * (four ? 0.25f * C.inv_dxf[ax] : C.inv_dxf[ax]);
        }
    };
    // viscous flux G (rows: momenta 0..ND-1, energy ND) on the face between
    // A and A + e_ax
    auto face = [&](int ax, const int64_t* A, R* G) {
        int64_t B[3] = {A[0], A[1], A[2]};
        B[ax] += 1;
        R uA[ND], uB[ND];
        int64_t oA, oB;
        vel_at(A, uA, oA);
        vel_at(B, uB, oB);
        R gax[ND];  // d_ax u_b
#pragma unroll
        for (int b = 0; b < ND; ++b) gax[b] = quot(uB[b] - uA[b], ax, false);
        R gtax[3], gtt[3];  // d_t u_ax and d_t u_t, t != ax
#pragma unroll
        for (int t = 0; t < ND; ++t) {
            if (t == ax) continue;
            int64_t Ap[3] = {A[0], A[1], A[2]}, Am[3] = {A[0], A[1], A[2]};
            int64_t Bp[3] = {B[0], B[1], B[2]}, Bm[3] = {B[0], B[1], B[2]};
            Ap[t] += 1;
            Am[t] -= 1;
            Bp[t] += 1;
            Bm[t] -= 1;
            R uAp[ND], uAm[ND], uBp[ND], uBm[ND];
            int64_t o;
            vel_at(Ap, uAp, o);
            vel_at(Am, uAm, o);
            vel_at(Bp, uBp, o);
            vel_at(Bm, uBm, o);
            gtax[t] = quot((uAp[ax] - uAm[ax]) + (uBp[ax] - uBm[ax]), t, true);
            gtt[t] = quot((uAp[t] - uAm[t]) + (uBp[t] - uBm[t]), t, true);
        }
        R div = (ax == 0) ? gax[0] : gtt[0];
#pragma unroll
        for (int a = 1; a < ND; ++a) div = div + ((a == ax) ? gax[a] : gtt[a]);
        R eta;
        if constexpr (NF == 1) {
            eta = eta_of<R>(C, 0);
        } else {
            R af[NF - 1];
            R s = R(0);
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) {
                const R a = R(__ldg(q + oA + (L::A + j) * C.fstride));
                const R b = R(__ldg(q + oB + (L::A + j) * C.fstride));
                af[j] = (a + b) * R(0.5);
                s = s + af[j];
            }
            eta = (R(1) - s) * eta_of<R>(C, NF - 1);
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) eta = eta + af[j] * eta_of<R>(C, j);
        }
        R work = R(0);
#pragma unroll
        for (int b = 0; b < ND; ++b) {
            R Tab = eta * (gax[b] + ((b == ax) ? gax[ax] : gtax[b]));
            if (b == ax) Tab = Tab - R(2.0 / 3.0) * eta * div;
            const R uf = (uA[b] + uB[b]) * R(0.5);
            work = (b == 0) ? Tab * uf : work + Tab * uf;
            G[b] = -Tab;
        }
        G[ND] = -work;
    };

    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c[3] = {lin % C.n[0], (lin / C.n[0]) % C.n[1], lin / (C.n[0] * C.n[1])};
        R V[ND + 1];
#pragma unroll
        for (int r = 0; r <= ND; ++r) V[r] = R(0);
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) {
            R Gm[ND + 1], Gp[ND + 1];
            int64_t cm[3] = {c[0], c[1], c[2]};
            cm[ax] -= 1;
            face(ax, cm, Gm);
            face(ax, c, Gp);
#pragma unroll
            for (int r = 0; r <= ND; ++r) V[r] = V[r] + quot(Gm[r] - Gp[r], ax, false);
        }
        const int64_t off = C.origin + c[0] * C.stride[0] + c[1] * C.stride[1] + c[2] * C.stride[2];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const R v = (k >= L::MOM && k <= L::E) ? V[k - L::MOM] : R(0);
            if constexpr (MODE == MODE_MIXED)
                rhsf[off + k * C.fstride] = v;
            else
                rhs[off + k * C.fstride] = v;
        }
    }
}

}  // namespace mfc
