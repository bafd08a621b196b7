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
    using RW = typename ModeT<MODE>::RW;
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
    const R ct = sizeof(R) == 8 ? R(C.teno_ct) : R(C.teno_ctf);
    const R inv_dx = sizeof(R) == 8 ? R(C.inv_dx[DIR]) : R(C.inv_dxf[DIR]);
    const double dx = C.dx[DIR];
    const df64 eps_df(C.eps), ct_df(C.teno_ct);
    bool bad = false;

    RW W[5][NQ];
    auto load_prim = [&](int64_t c, RW* out) {
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * C.fstride);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE, RW>(qc, out, C, bad);
    };

#pragma unroll
    for (int k = 0; k < 4; ++k) load_prim(s0 - 3 + k, W[k]);

    // MODE_FAST with JS, mapped or Z weights: the differences D_j, second
    // differences a_r and partial indicators A_r of a cell's stencil
    // (weno5_fast64_core) are the previous cell's shifted by one, so each
    // thread keeps three D, two a and two A per field in shared-memory rings
    // ([slot][field][thread]) and computes only those of the new cell; the
    // values are those weno5_cell_fast64 would compute, bit for bit.
    constexpr bool kSlide = MODE == MODE_FAST;
    const bool slide = kSlide && variant != WENO_TENO;
    extern __shared__ double slide_ring[];
    auto RD = [&](int slot, int k) -> double& { return slide_ring[(slot * NQ + k) * blockDim.x + threadIdx.x]; };
    auto RA = [&](int slot, int k) -> double& { return slide_ring[((3 + slot) * NQ + k) * blockDim.x + threadIdx.x]; };
    auto RB = [&](int slot, int k) -> double& { return slide_ring[((5 + slot) * NQ + k) * blockDim.x + threadIdx.x]; };
    int d0 = 0, d1 = 1, d2 = 2, p0 = 0, p1 = 1;  // ring slots of D01, D12, D23 and of a0, a1
    const double e4 = 4.0 * C.eps;
    if constexpr (kSlide) {
        if (slide) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const double D01 = double(W[1][k]) - double(W[0][k]), D12 = double(W[2][k]) - double(W[1][k]);
                const double D23 = double(W[3][k]) - double(W[2][k]);
                const double a0 = D12 - D01, a1 = D23 - D12;
                RD(0, k) = D01;
                RD(1, k) = D12;
                RD(2, k) = D23;
                RA(0, k) = a0;
                RA(1, k) = a1;
                RB(0, k) = weno5_fast64_A(a0, e4);
                RB(1, k) = weno5_fast64_A(a1, e4);
            }
        }
    }

    R WLprev[NQ], Fprev[NQ], uprev = R(0);
    const double dtv = (A.out_kind != 0) ? *A.dt : 0.0;

    for (int64_t m = s0 - 1; m <= s1; ++m) {
        if constexpr (MODE == MODE_MIXED) {
            // the float32 march is bound by the latency of its loads: bring
            // the state two cells ahead of the window, and the accumulator and
            // q^n of the cell finished two iterations later, into L2 now
            const int64_t cpf = m + 4;
            if (cpf < n) {
                const double* pq = A.q + base + cpf * S;
#pragma unroll
                for (int f = 0; f < NQ; ++f) asm volatile("prefetch.global.L2 [%0];" ::"l"(pq + f * C.fstride));
            }
            const int64_t co = m + 1;
            if (co >= s0 && co < s1) {
                const int64_t oo = base + co * S;
                if (A.acc_in == 2) {
#pragma unroll
                    for (int f = 0; f < NQ; ++f)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(A.rhsf + oo + f * C.fstride));
                }
                if (A.out_kind == 2) {
#pragma unroll
                    for (int f = 0; f < NQ; ++f)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(A.qn + oo + f * C.fstride));
                }
            }
        }
        load_prim(m + 2, W[4]);
        R WRm[NQ], WLm[NQ];
        if constexpr (kSlide) {
            if (slide) {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    const double D01 = RD(d0, k), D12 = RD(d1, k), D23 = RD(d2, k);
                    const double D34 = double(W[4][k]) - double(W[3][k]);
                    const double a[3] = {RA(p0, k), RA(p1, k), D34 - D23};
                    const double Ab[3] = {RB(p0, k), RB(p1, k), weno5_fast64_A(a[2], e4)};
                    weno5_fast64_core(double(W[2][k]), D01, D12, D23, D34, a, Ab, variant, WRm[k], WLm[k]);
                    // the new cell's values replace the oldest
                    RD(d0, k) = D34;
                    RA(p0, k) = a[2];
                    RB(p0, k) = Ab[2];
                }
                const int t = d0;
                d0 = d1;
                d1 = d2;
                d2 = t;
                p0 ^= 1;
                p1 ^= 1;
            }
        }
        if (!(kSlide && slide)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                if constexpr (MODE == MODE_DF) {
                    const WenoEdges e = weno5_cell_df(W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], variant, eps_df,
                                                      ct_df);
                    WRm[k] = e.vl;
                    WLm[k] = e.vr;
                    bad |= e.bad != 0;
                } else if constexpr (MODE != MODE_MIXED) {
                    weno5_cell<MODE, R>(W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], variant, eps, ct, WRm[k],
                                        WLm[k]);
                }
            }
            if constexpr (MODE == MODE_MIXED) weno5_fields_mixed32<NQ>(W[0], W[1], W[2], W[3], W[4], variant, eps, ct,
                                                                       WRm, WLm);
        }
        if (m >= s0) {
            // face m - 1/2: left state WLprev (cell m-1), right state WRm (cell m)
            MixState<R> mL = mix_state<NF, ND, MODE, R>(WLprev, C), mR = mix_state<NF, ND, MODE, R>(WRm, C);
            if (!physical_mix<NF, ND, R, MODE>(WLprev, mL, C) || !physical_mix<NF, ND, R, MODE>(WRm, mR, C)) {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    WLprev[k] = R(W[1][k]);
                    WRm[k] = R(W[2][k]);
                }
                mL = mix_state<NF, ND, MODE, R>(WLprev, C);
                mR = mix_state<NF, ND, MODE, R>(WRm, C);
            }
            R F[NQ], uf;
            hllc<NF, ND, DIR, MODE>(WLprev, WRm, mL, mR, C, F, uf, bad);
            if (m >= s0 + 1) {
                // finish cell m - 1 = window slot 1: faces m - 3/2 (Fprev) and m - 1/2 (F)
                const int64_t off = base + (m - 1) * S;
                const R du = uf - uprev;
                // alpha rows: alpha div u, or (alpha + K) div u (Kapila)
                R Kc = R(0);
                if constexpr (NF == 2) {
                    if (C.model == 1) Kc = kapila_K<MODE, R>(R(W[1][L::E]), R(W[1][L::A]), C);
                }
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R t;
                    const R ac = (k >= L::A && C.model == 1) ? R(W[1][k]) + Kc : R(W[1][k]);
                    if constexpr (MODE == MODE_EXACT) {
                        t = (Fprev[k] - F[k]) / dx;
                        if (k >= L::A) t = t + ac * du / dx;
                    } else {
                        t = (Fprev[k] - F[k]) * inv_dx;
                        if (k >= L::A) t = t + ac * du * inv_dx;
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

// Asynchronous global -> shared copies of 4 or 8 bytes (cp.async), their
// commit groups and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// float -> double, exact.  The conversion instruction issues to the float64
// pipe, which the stage updates of the staged sweep already load heavily, so
// normal floats and zeros are widened with integer instructions on the bit
// pattern instead (sign; exponent + 1023 - 127; mantissa shifted into the top
// of the 52-bit field); subnormal, infinite and NaN inputs take the
// conversion instruction.
__device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e - 1u < 254u)
        return __hiloint2double((int)((b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + 0x38000000u)), (int)(b << 29));
    if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return double(f);
}

// Shared memory of the staged mixed sweep, per thread: a ring of kStageQ
// slots of the conservative state of one cell, then one slot of the
// accumulator (float) of the cell being finished and, for a stage update
// that reads q^n, one slot of its q^n; each value at [slot][field][thread].
// Eight 64-thread blocks fit an SM with or without the q^n slot.
constexpr int kStageQ = 5;
template <int NQ>
constexpr int staged_smem_bytes(int block, bool with_qn) {
    return block * (kStageQ * NQ * 8 + NQ * 4 + (with_qn ? NQ * 8 : 0));
}

// The y and z sweeps of the mixed mode with their global loads staged
// through shared memory.  Each thread marches its line segment exactly as
// sweep_body<MODE_MIXED> does (same arithmetic in the same order, so the
// results are identical); its loads are asynchronous copies into per-thread
// shared memory, in two kinds of commit group: S(g), the state of cell
// s0 - 3 + g (the window's new cell when g >= 4), issued at the top of the
// iteration before the one that converts it; and U(g), the accumulator and
// q^n of cell s0 - 6 + g (the cell finished in iteration g), issued at the end
// of iteration g - 1 into the single slot the update of that iteration has
// just read.  Iteration g waits for S(g) before its reconstruction and for
// U(g) before its update, so the latency of the loads (L2 or HBM) overlaps
// the reconstruction and Riemann solve instead of stalling them.  The copies
// of a warp are contiguous along x.  The state of the finished cell, needed
// by the stage update, is still in the state ring (group g - 3).
template <int NF, int ND, int DIR>
__device__ __forceinline__ void sweep_body_staged(const Consts& C, const SweepArgs& A) {
    using L = Lay<NF, ND>;
    using R = float;
    constexpr int NQ = L::NQ;
    constexpr int TA = 0;
    constexpr int TB = (DIR == 2) ? 1 : 2;
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int bd = blockDim.x, tx = threadIdx.x;
    double* ringQ = reinterpret_cast<double*>(stage_raw);
    float* slotF = reinterpret_cast<float*>(ringQ + kStageQ * NQ * bd);
    double* slotN = reinterpret_cast<double*>(slotF + NQ * bd);  // 8-byte aligned: bd is even
    auto Q = [&](int slot, int f) -> double* { return ringQ + (slot * NQ + f) * bd + tx; };
    auto QN = [&](int f) -> double* { return slotN + f * bd + tx; };
    auto RF = [&](int f) -> float* { return slotF + f * bd + tx; };

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
    const R eps = C.epsf, ct = C.teno_ctf, inv_dx = C.inv_dxf[DIR];
    const bool acc = A.acc_in == 2, upd2 = A.out_kind == 2;
    bool bad = false;

    const int64_t G = (s1 - s0) + 6;
    int64_t issued = 0;
    // S(issued): the state of cell s0 - 3 + issued into its ring slot
    auto issue_state = [&]() {
        if (issued < G) {
            const int slot = (int)(issued % kStageQ);
            bool flip = false;
            const int64_t cc = bc_source(s0 - 3 + issued, n, bclo, bchi, flip);
            const double* p = A.q + base + cc * S;
#pragma unroll
            for (int f = 0; f < NQ; ++f) cp_async8(Q(slot, f), p + f * C.fstride);
        }
        cp_async_commit();
        ++issued;
    };
    // U(g): the accumulator and q^n of cell s0 - 6 + g (empty group outside the segment)
    auto issue_update = [&](int64_t g) {
        const int64_t u = s0 - 6 + g;
        if (u >= s0 && u < s1) {
            const int64_t o = base + u * S;
            if (acc) {
#pragma unroll
                for (int f = 0; f < NQ; ++f) cp_async4(RF(f), A.rhsf + o + f * C.fstride);
            }
            if (upd2) {
#pragma unroll
                for (int f = 0; f < NQ; ++f) cp_async8(QN(f), A.qn + o + f * C.fstride);
            }
        }
        cp_async_commit();
    };
    // primitive state of the cell of group g, from its ring slot
    auto prim_of = [&](int64_t g, R* out) {
        bool flip = false;
        bc_source(s0 - 3 + g, n, bclo, bchi, flip);
        const int slot = (int)(g % kStageQ);
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = *Q(slot, f);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE_MIXED, R>(qc, out, C, bad);
    };

    issue_state();  // S(0); one state group is always in flight ahead of the one in use
    R W[5][NQ];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        issue_state();
        cp_async_wait<1>();
        prim_of(k, W[k]);
    }
    issue_update(4);  // U(4) (empty: no cell is finished in the first iterations)

    R WLprev[NQ], Fprev[NQ], uprev = R(0);
    const double dtv = (A.out_kind != 0) ? *A.dt : 0.0;

    for (int64_t m = s0 - 1; m <= s1; ++m) {
        const int64_t g = m + 5 - s0;
        issue_state();          // S(g + 1)
        cp_async_wait<2>();     // S(g) done; U(g) and S(g + 1) may be in flight
        prim_of(g, W[4]);
        R WRm[NQ], WLm[NQ];
        weno5_fields_mixed32<NQ>(W[0], W[1], W[2], W[3], W[4], variant, eps, ct, WRm, WLm);
        if (m >= s0) {
            MixState<R> mL = mix_state<NF, ND, MODE_MIXED, R>(WLprev, C), mR = mix_state<NF, ND, MODE_MIXED, R>(WRm, C);
            if (!physical_mix<NF, ND, R, MODE_MIXED>(WLprev, mL, C) || !physical_mix<NF, ND, R, MODE_MIXED>(WRm, mR, C)) {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    WLprev[k] = W[1][k];
                    WRm[k] = W[2][k];
                }
                mL = mix_state<NF, ND, MODE_MIXED, R>(WLprev, C);
                mR = mix_state<NF, ND, MODE_MIXED, R>(WRm, C);
            }
            R F[NQ], uf;
            hllc<NF, ND, DIR, MODE_MIXED>(WLprev, WRm, mL, mR, C, F, uf, bad);
            if (m >= s0 + 1) {
                // finish cell m - 1 (window slot 1); its accumulator and q^n are
                // in the update slot (U(g)), its state in state slot g - 3
                cp_async_wait<1>();     // U(g) done; S(g + 1) may be in flight
                const int64_t off = base + (m - 1) * S;
                const int qs = (int)((g - 3) % kStageQ);
                const R du = uf - uprev;
                R Kc = R(0);
                if constexpr (NF == 2) {
                    if (C.model == 1) Kc = kapila_K<MODE_MIXED, R>(W[1][L::E], W[1][L::A], C);
                }
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R t = (Fprev[k] - F[k]) * inv_dx;
                    const R ac = (k >= L::A && C.model == 1) ? W[1][k] + Kc : W[1][k];
                    if (k >= L::A) t = t + ac * du * inv_dx;
                    const int64_t o = off + k * C.fstride;
                    const float Lf = acc ? *RF(k) + t : t;
                    if (A.out_kind == 3) {
                        A.rhsf[o] = Lf;
                        continue;
                    }
                    // the widening off the float64 pipe pays where the three-term update
                    // loads that pipe; the one-term update (q1 = q + dt L) keeps the instruction
                    const double Lc = upd2 ? f64_of_f32(Lf) : double(Lf);
                    const double qc = *Q(qs, k);
                    if (A.out_kind == 0) {
                        A.rhs[o] = Lc;
                    } else if (A.out_kind == 1) {
                        A.qout[o] = qc + dtv * Lc;
                    } else {
                        A.qout[o] = A.rk_a * *QN(k) + A.rk_b * (qc + dtv * Lc);
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
        issue_update(g + 1);  // U(g + 1) into the slot this iteration's update has read
    }
    cp_async_wait<0>();
    if (bad) atomicOr(A.flag, 1);
}

// Eight 64-thread blocks per SM (16 warps) at 128 registers, the rings of
// eight blocks fitting an SM; fewer warps left the march's dependency stalls
// exposed (8 warps: issue active 36-39 %).
template <int NF, int ND, int DIR>
__global__ void __launch_bounds__(64, 8) sweep_kernel_staged(const Consts C, const SweepArgs A) {
    sweep_body_staged<NF, ND, DIR>(C, A);
}

// Value of neighbour lane + off (|off| <= 2) in the sequence formed by the
// previous, current and next 32-cell chunks held by the warp (p, c, nx).
template <class R>
__device__ __forceinline__ R chunk_neighbour(R p, R c, R nx, int lane, int off) {
    const int src = (lane + off) & 31;
    const R inside = __shfl_sync(0xffffffffu, c, src);
    const R outside = __shfl_sync(0xffffffffu, off < 0 ? p : nx, src);
    return (lane + off >= 0 && lane + off < 32) ? inside : outside;
}

// x-direction sweep with one warp per line segment.  The warp walks the
// segment in 32-cell chunks, lane l holding cell c = c0 + l: the primitive
// state of every cell is computed once, the five-cell WENO stencil comes
// from warp shuffles of the previous / current / next chunk, lane l solves
// the face c - 1/2 (left state: the right edge value of lane l - 1) and
// finishes cell c - 1 from its own face and lane l - 1's.  Loads and stores
// along x are contiguous across the warp (the per-thread march of
// sweep_body reads 32 rows at once along x and depends on L1 to keep them).
// Same arithmetic, in the same order, as sweep_body.
template <int NF, int ND, int MODE>
__device__ __forceinline__ void sweep_x_body(const Consts& C, const SweepArgs& A) {
    using L = Lay<NF, ND>;
    using R = typename ModeT<MODE>::R;
    constexpr int NQ = L::NQ;
    const int lane = threadIdx.x & 31;
    const int64_t nlines = C.n[1] * C.n[2];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nlines * A.nseg) return;  // whole warps only
    const int64_t line = warp % nlines;
    const int64_t seg = warp / nlines;
    const int64_t ia = line % C.n[1], ib = line / C.n[1];
    const int64_t base = C.origin + ia * C.stride[1] + ib * C.stride[2];
    const int64_t S = C.stride[0];
    const int64_t n = C.n[0];
    const int64_t s0 = seg * A.seg;
    const int64_t s1 = (s0 + A.seg < n) ? s0 + A.seg : n;
    const int bclo = C.bc_lo[0], bchi = C.bc_hi[0];
    const int variant = C.weno;
    const R eps = sizeof(R) == 8 ? R(C.eps) : R(C.epsf);
    const R ct = sizeof(R) == 8 ? R(C.teno_ct) : R(C.teno_ctf);
    const R inv_dx = sizeof(R) == 8 ? R(C.inv_dx[0]) : R(C.inv_dxf[0]);
    const double dx = C.dx[0];
    const double dtv = (A.out_kind == 1 || A.out_kind == 2) ? *A.dt : 0.0;
    bool bad = false;

    // cells outside [-3, n + 2] are never needed; clamping keeps the lanes
    // past the end of a segment on valid addresses
    auto load_prim = [&](int64_t c, R* out) {
        const bool need = c >= s0 - 3 && c <= s1 + 2;
        c = c < -3 ? -3 : (c > n + 2 ? n + 2 : c);
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * C.fstride);
        if (flip) qc[L::MOM] = -qc[L::MOM];
        bool b = false;
        prim_for_recon<NF, ND, MODE, R>(qc, out, C, b);
        bad |= need && b;
    };
    // the mixed mode brings the chunk after the next into L1 one iteration
    // before load_prim reads it (the same clamped, boundary-mapped cells), so
    // that its loads do not wait on L2 or HBM
    auto prefetch_l1 = [&](int64_t c) {
        c = c < -3 ? -3 : (c > n + 2 ? n + 2 : c);
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
#pragma unroll
        for (int f = 0; f < NQ; ++f) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + f * C.fstride));
    };

    int64_t c0 = s0 - 1;
    R Wp[NQ], Wc[NQ], Wn[NQ];
    // lanes 30, 31 of the chunk before the first: cells s0 - 3, s0 - 2
    load_prim(c0 - 32 + (lane < 30 ? 30 : lane), Wp);
    load_prim(c0 + lane, Wc);
    load_prim(c0 + 32 + lane, Wn);
    if constexpr (MODE == MODE_MIXED) {
        if (c0 + 32 <= s1) prefetch_l1(c0 + 64 + lane);
    }
    R VRp[NQ], Fp[NQ], ufp = R(0);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        VRp[k] = Wp[k];
        Fp[k] = R(0);
    }

    while (c0 <= s1) {
        const int64_t c = c0 + lane;
        R VL[NQ], VR[NQ], Wm1[NQ];
        if constexpr (MODE == MODE_MIXED) {
            // fields two at a time (weno5_cells_mixed32_x2), an odd last one alone
            if (variant != WENO_TENO) {
#pragma unroll
                for (int k = 0; k < NQ; k += 2) {
                    const int k1 = (k + 1 < NQ) ? k + 1 : k;
                    R fm2[2], fm1[2], fp1[2], fp2[2];
                    const int nh = (k + 1 < NQ) ? 2 : 1;
#pragma unroll
                    for (int h = 0; h < nh; ++h) {
                        const int kk = h ? k1 : k;
                        fm2[h] = chunk_neighbour(Wp[kk], Wc[kk], Wn[kk], lane, -2);
                        fm1[h] = chunk_neighbour(Wp[kk], Wc[kk], Wn[kk], lane, -1);
                        fp1[h] = chunk_neighbour(Wp[kk], Wc[kk], Wn[kk], lane, 1);
                        fp2[h] = chunk_neighbour(Wp[kk], Wc[kk], Wn[kk], lane, 2);
                    }
                    if (k + 1 < NQ) {
                        const WenoPair32 w = weno5_cells_mixed32_x2(fm2[0], fm1[0], Wc[k], fp1[0], fp2[0], fm2[1],
                                                                    fm1[1], Wc[k1], fp1[1], fp2[1], variant, eps);
                        VR[k] = w.a.x;
                        VL[k] = w.a.y;
                        VR[k1] = w.b.x;
                        VL[k1] = w.b.y;
                    } else {
                        const float2 v = weno5_cell_mixed32(fm2[0], fm1[0], Wc[k], fp1[0], fp2[0], variant, eps);
                        VR[k] = v.x;
                        VL[k] = v.y;
                    }
                    Wm1[k] = fm1[0];
                    if (k + 1 < NQ) Wm1[k1] = fm1[1];
                }
            } else {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    const R fm2 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, -2);
                    const R fm1 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, -1);
                    const R fp1 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, 1);
                    const R fp2 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, 2);
                    weno5_cell<MODE, R>(fm2, fm1, Wc[k], fp1, fp2, variant, eps, ct, VL[k], VR[k]);
                    Wm1[k] = fm1;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const R fm2 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, -2);
                const R fm1 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, -1);
                const R fp1 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, 1);
                const R fp2 = chunk_neighbour(Wp[k], Wc[k], Wn[k], lane, 2);
                weno5_cell<MODE, R>(fm2, fm1, Wc[k], fp1, fp2, variant, eps, ct, VL[k], VR[k]);
                Wm1[k] = fm1;
            }
        }
        // face c - 1/2: left state = right edge value of cell c - 1
        R WL[NQ], WR[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            WL[k] = chunk_neighbour(VRp[k], VR[k], VR[k], lane, -1);
            WR[k] = VL[k];
        }
        const bool face = c >= s0 && c <= s1;
        MixState<R> mL = mix_state<NF, ND, MODE, R>(WL, C), mR = mix_state<NF, ND, MODE, R>(WR, C);
        if (!physical_mix<NF, ND, R, MODE>(WL, mL, C) || !physical_mix<NF, ND, R, MODE>(WR, mR, C)) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                WL[k] = Wm1[k];
                WR[k] = Wc[k];
            }
            mL = mix_state<NF, ND, MODE, R>(WL, C);
            mR = mix_state<NF, ND, MODE, R>(WR, C);
        }
        R F[NQ], uf;
        bool fb = false;
        hllc<NF, ND, 0, MODE>(WL, WR, mL, mR, C, F, uf, fb);
        bad |= face && fb;
        // finish cell c - 1 from faces c - 3/2 (lane - 1) and c - 1/2 (own)
        const R ufm = chunk_neighbour(ufp, uf, uf, lane, -1);
        const bool out = c - 1 >= s0 && c - 1 < s1;
        const int64_t off = base + (c - 1) * S;
        const R du = uf - ufm;
        R Kc = R(0);
        if constexpr (NF == 2) {
            if (C.model == 1) Kc = kapila_K<MODE, R>(Wm1[L::E], Wm1[L::A], C);
        }
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const R Fm = chunk_neighbour(Fp[k], F[k], F[k], lane, -1);
            R t;
            const R ac = (k >= L::A && C.model == 1) ? Wm1[k] + Kc : Wm1[k];
            if constexpr (MODE == MODE_EXACT) {
                t = (Fm - F[k]) / dx;
                if (k >= L::A) t = t + ac * du / dx;
            } else {
                t = (Fm - F[k]) * inv_dx;
                if (k >= L::A) t = t + ac * du * inv_dx;
            }
            if (!out) continue;
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
        // next chunk
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            Wp[k] = Wc[k];
            Wc[k] = Wn[k];
            VRp[k] = VR[k];
            Fp[k] = F[k];
        }
        ufp = uf;
        c0 += 32;
        if (c0 <= s1) load_prim(c0 + 32 + lane, Wn);
        if constexpr (MODE == MODE_MIXED) {
            if (c0 + 32 <= s1) prefetch_l1(c0 + 64 + lane);
        }
    }
    if (bad) atomicOr(A.flag, 1);
}

template <int NF, int ND, int MODE>
__global__ void __launch_bounds__(128, (MODE == MODE_MIXED ? 5 : 1)) sweep_x_kernel(const Consts C, const SweepArgs A) {
    sweep_x_body<NF, ND, MODE>(C, A);
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
        double c2;
        if constexpr (NF == 2) {
            c2 = (C.model == 1) ? wood_c2<MODE_EXACT, double>(rho, w[L::E], w[L::A], C)
                                : ((Gamma + 1.0) * w[L::E] + Pi) / (Gamma * rho);
        } else {
            c2 = ((Gamma + 1.0) * w[L::E] + Pi) / (Gamma * rho);
        }
        bad |= !(c2 > 0.0);
        const double cs = sqrt(c2);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double s = C.dx[d] / (fabs(w[L::MOM + d]) + cs);
            m = (s < m) ? s : m;
        }
        if (C.visc_dt) {
            // explicit viscous limit rho min_d dx_d^2 / (2 ndim eta), eta the
            // mixture viscosity (1 - sum alpha_j) eta_N + sum alpha_j eta_j
            double sa = 0.0;
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) sa = sa + qc[L::A + j];
            double eta = (1.0 - sa) * C.eta[NF - 1];
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) eta = eta + qc[L::A + j] * C.eta[j];
            if (eta > 0.0) {
                const double s = rho * C.dx2min / ((2.0 * ND) * eta);
                m = (s < m) ? s : m;
            }
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
// MFC_MIXED): one refined reciprocal each for rho and Gamma per cell; the
// largest (|u_d| + c)/dx_d over the block's cells is reduced first and its
// reciprocal, min dx_d/(|u_d| + c), taken once per block.  The maxima of these
// non-negative doubles and the sign tests run on bit patterns with integer
// instructions (off the float64 pipe that bounds this kernel); a non-physical
// state gives NaN, which orders above every finite value here, is ignored by
// the final minimum (NaN's pattern is above +inf's) and is reported by the
// flag.  float64 throughout.
template <int NF, int ND>
__global__ void __launch_bounds__(256) cfl_fast_kernel(const Consts C, const double* q, unsigned long long* minbits,
                                                       int* flag) {
    using L = Lay<NF, ND>;
    constexpr int NQ = L::NQ;
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    long long mb = 0;  // bit pattern of the largest (|u_d| + c)/dx_d so far (+0.0)
    bool bad = false;
    auto bmax = [](long long a, double v) {
        const long long b = __double_as_longlong(v);
        return b > a ? b : a;
    };
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < ncell;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = interior_offset(C, lin);
        double qc[NQ];
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(q + off + f * C.fstride);
        double rho = qc[0];
#pragma unroll
        for (int i = 1; i < NF; ++i) rho = rho + qc[i];
        bad |= !f64_pos(rho);
        const double irho = rcp_nr(rho);
        double u[ND], ke = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            u[d] = qc[L::MOM + d] * irho;
            ke = fma(qc[L::MOM + d], u[d], ke);
        }
        double Gamma, Pi;
        mixture_mode<NF, MODE_FAST, double>(qc + L::A, C, Gamma, Pi);
        const double iG = rcp_nr(Gamma);
        const double p = (qc[L::E] - 0.5 * ke - Pi) * iG;
        double c2 = ((Gamma + 1.0) * p + Pi) * iG * irho;
        if constexpr (NF == 2) {
            if (C.model == 1) c2 = wood_c2<MODE_FAST, double>(rho, p, qc[L::A], C);
        }
        bad |= !f64_pos(c2);
        const double cs = sqrt(c2);
#pragma unroll
        for (int d = 0; d < ND; ++d) mb = bmax(mb, (fabs(u[d]) + cs) * C.inv_dx[d]);
        if (C.visc_dt) {
            // the viscous limit's reciprocal, 2 ndim eta / (rho min_d dx_d^2)
            double eta = C.eta[NF - 1];
#pragma unroll
            for (int j = 0; j < NF - 1; ++j) eta = fma(qc[L::A + j], C.eta[j] - C.eta[NF - 1], eta);
            mb = bmax(mb, (2.0 * ND) * eta * irho * C.inv_dx2min);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_down_sync(0xffffffffu, mb, o);
        mb = t > mb ? t : mb;
    }
    __shared__ long long wm[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wm[wid] = mb;
    __syncthreads();
    if (wid == 0) {
        mb = (lane < (int)(blockDim.x >> 5)) ? wm[lane] : 0LL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long t = __shfl_down_sync(0xffffffffu, mb, o);
            mb = t > mb ? t : mb;
        }
        if (lane == 0) {
            // min dx_d/(|u_d| + c) of the block (+inf when every maximum is 0)
            const double m = mb == 0 ? __longlong_as_double(0x7ff0000000000000LL) : rcp_nr(__longlong_as_double(mb));
            atomicMin(minbits, (unsigned long long)__double_as_longlong(m));
        }
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
