// Adjoint sweep: one directional contribution of (dL/dq)^T rbar.
#pragma once

#include "mfc_adjoint.cuh"
#include "mfc_device.cuh"
#include "mfc_launch.h"

namespace mfc {

// One thread owns the cells [s0, s1) of one line along axis DIR and gathers
// every contribution to them (no atomics): it recomputes the forward states
// of the faces s0 - 5/2 .. s1 + 3/2 and runs, face by face, the adjoint of
// the flux difference and alpha div(u) term, of HLLC and of WENO5; the
// primitive-state bars of a cell are complete three faces after its own and
// are then pulled back through conservative-to-primitive and added to
// qbar.  Contributions to ghost cells are folded into the interior cell the
// ghost copies (normal momentum negated across a reflective wall); for a
// periodic axis the segments that own the copied cells collect those
// contributions in a short pass over the far end of the line first.
// Dynamic shared memory of one sweep_vjp_kernel block (the rings of the
// float32 mode; none for the float64 modes).
template <int NF, int ND, int MODE>
constexpr size_t vjp_smem_bytes(int block) {
    return MODE == MODE_MIXED ? size_t(16 * Lay<NF, ND>::NQ + 8) * block * sizeof(float) : 0;
}

// The float32 mode is bound by latency, not by a pipe: it asks for seven
// blocks per SM (128 registers, a few spilled; its rings allow seven), where
// the unconstrained 251 registers left four (six blocks at 167 registers
// measure the same).  The double-float mode asks for six (168 registers,
// its spills staying in L1), 3 % faster than four at 255; the float64
// modes are bound by the float64 pipe and keep the compiler's choice.
template <int NF, int ND, int DIR, int MODE>
__global__ void __launch_bounds__(64, (MODE == MODE_MIXED ? 7 : (MODE == MODE_DF ? 6 : 1)))
    sweep_vjp_kernel(const Consts C, const VjpArgs A) {
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
    const int64_t fs = C.fstride;
    const int64_t n = C.n[DIR];
    const int64_t s0 = seg * A.seg;
    const int64_t s1 = (s0 + A.seg < n) ? s0 + A.seg : n;
    const int bclo = C.bc_lo[DIR], bchi = C.bc_hi[DIR];
    const bool periodic = bclo == BC_PERIODIC;
    const int variant = C.weno;
    const R eps = sizeof(R) == 8 ? R(C.eps) : R(C.epsf);
    const R ct = sizeof(R) == 8 ? R(C.teno_ct) : R(C.teno_ctf);
    const R inv_dx = R(C.inv_dx[DIR]);

    // rings indexed by cell & 7 (face & 7 for the face velocities): forward
    // primitive states, their bars, forward face velocities.  The float32
    // mode keeps them in shared memory, interleaved by thread so that a warp
    // touches 32 consecutive words (vjp_smem_bytes); the float64 modes in
    // local memory.
    constexpr bool kSmem = MODE == MODE_MIXED;
    extern __shared__ unsigned char vjp_smem[];
    R* const sm = reinterpret_cast<R*>(vjp_smem);
    const int tix = threadIdx.x, bdim = blockDim.x;
    R Wr_l[kSmem ? 1 : 8][NQ];
    R acc_l[kSmem ? 1 : 8][NQ];
    R ufr_l[kSmem ? 1 : 8];
    auto WR = [&](int64_t slot, int k) -> R& {
        if constexpr (kSmem) return sm[((slot & 7) * NQ + k) * bdim + tix];
        else return Wr_l[slot & 7][k];
    };
    auto ACC = [&](int64_t slot, int k) -> R& {
        if constexpr (kSmem) return sm[((8 + (slot & 7)) * NQ + k) * bdim + tix];
        else return acc_l[slot & 7][k];
    };
    auto UFR = [&](int64_t slot) -> R& {
        if constexpr (kSmem) return sm[(16 * NQ + (slot & 7)) * bdim + tix];
        else return ufr_l[slot & 7];
    };
    R ext_lo[3][NQ];   // periodic: bars of ghosts n..n+2, i.e. of cells 0..2
    R ext_hi[3][NQ];   // periodic: bars of ghosts -3..-1, i.e. of cells n-3..n-1
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < NQ; ++k) ext_lo[a][k] = ext_hi[a][k] = R(0);

    auto load_prim = [&](int64_t c, R* out) {
        bool flip = false;
        const int64_t cc = bc_source(c, n, bclo, bchi, flip);
        const double* p = A.q + base + cc * S;
        double qc[NQ];
        bool bad = false;
#pragma unroll
        for (int f = 0; f < NQ; ++f) qc[f] = __ldg(p + f * fs);
        if (flip) qc[L::MOM + DIR] = -qc[L::MOM + DIR];
        prim_for_recon<NF, ND, MODE, R>(qc, out, C, bad);
    };
    auto load_ring = [&](int64_t c) {
        R w[NQ];
        load_prim(c, w);
#pragma unroll
        for (int k = 0; k < NQ; ++k) WR(c, k) = w[k];
    };
    auto rbar = [&](int64_t c, int k) -> R {
        return (c >= 0 && c < n) ? R(__ldg(A.rbar + base + c * S + k * fs)) : R(0);
    };

    // pass 0: periodic, segments owning cells 0..2: contributions of the far
    //         end to ghosts n..n+2 (copies of cells 0..2);
    // pass 1: periodic, segments owning cells n-3..n-1: contributions of the
    //         near end to ghosts -3..-1 (copies of cells n-3..n-1);
    // pass 2: the faces and cells that touch the segment itself.
    // Each pass runs j over [jb, je]: face j (= j+1/2) is processed for
    // j <= fmax, the WENO adjoint of cell j for cmin <= j <= cmax, and cell
    // j-3 is finished in pass 2.
    for (int pass = 0; pass < 3; ++pass) {
        int64_t jb, je, fmax, cmin, cmax;
        if (pass == 0) {
            if (!(periodic && s0 < 3)) continue;
            jb = n - 3; je = n; fmax = n - 1; cmin = n - 2; cmax = n;
        } else if (pass == 1) {
            if (!(periodic && s1 > n - 3)) continue;
            jb = -1; je = 1; fmax = 1; cmin = -1; cmax = 1;
        } else {
            jb = (s0 - 3 > -1) ? s0 - 3 : -1;
            je = s1 + 2;
            cmin = (jb == -1) ? -1 : jb + 1;
            // a non-periodic segment owning one of cells n-3..n-1 also collects
            // the mirrored / copied contributions of ghosts n..n+2
            const bool ext = !periodic && s1 >= n - 2;
            fmax = ext ? n - 1 : ((s1 + 1 < n - 1) ? s1 + 1 : n - 1);
            cmax = ext ? n : ((s1 + 1 < n) ? s1 + 1 : n);
        }
        // contributions to cell x, routed according to the pass
        auto sink = [&](int64_t x, int k, R v) {
            if (pass == 0) {
                if (x >= n && x < n + 3) ext_lo[x - n][k] += v;
            } else if (pass == 1) {
                if (x >= -3 && x < 0) ext_hi[x + 3][k] += v;
            } else if (x >= 0 && x < n) {
                ACC(x, k) += v;
            } else if (!periodic) {
                bool flip = false;
                const int64_t img = bc_source(x, n, bclo, bchi, flip);
                ACC(img, k) += (flip && k == L::MOM + DIR) ? -v : v;
            }
        };
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < NQ; ++k) ACC(s, k) = R(0);
        for (int64_t c = jb - 2; c <= jb + 2; ++c) load_ring(c);
        // forward left state of face jb (right edge of cell jb)
        R WLcur[NQ], WRbprev[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            R vl, vr;
            weno5_cell<MODE, R>(WR(jb - 2, k), WR(jb - 1, k), WR(jb, k), WR(jb + 1, k), WR(jb + 2, k), variant, eps,
                                ct, vl, vr);
            WLcur[k] = vr;
            WRbprev[k] = R(0);
        }
        for (int64_t j = jb; j <= je; ++j) {
            const bool face = (j >= -1) && (j <= fmax);
            const bool cellw = (j >= cmin) && (j <= cmax);
            if (face) load_ring(j + 3);  // j + 3 <= n + 2
#pragma unroll
            for (int k = 0; k < NQ; ++k) ACC(j + 3, k) = R(0);
            R WLb[NQ], WRb[NQ], WLnext[NQ];
#pragma unroll
            for (int k = 0; k < NQ; ++k) WLb[k] = WRb[k] = R(0);
            if (face) {
                // forward right state of face j (left edge of cell j+1), and left state of face j+1
                R WRj[NQ];
#pragma unroll
                for (int k = 0; k < NQ; ++k)
                    weno5_cell<MODE, R>(WR(j - 1, k), WR(j, k), WR(j + 1, k), WR(j + 2, k), WR(j + 3, k), variant, eps,
                                        ct, WRj[k], WLnext[k]);
                // first-order fallback of the forward pass at a non-physical face
                const bool first_order =
                    !physical_state<NF, ND, R, MODE>(WLcur, C) || !physical_state<NF, ND, R, MODE>(WRj, C);
                if (first_order) {
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        WLcur[k] = WR(j, k);
                        WRj[k] = WR(j + 1, k);
                    }
                }
                // bars of the face flux and face velocity from rbar of cells j and j+1
                R Fb[NQ];
#pragma unroll
                for (int k = 0; k < NQ; ++k) Fb[k] = (rbar(j + 1, k) - rbar(j, k)) * inv_dx;
                R ufb = R(0);
                // the alpha rows' coefficient of div u: alpha, or alpha + K (Kapila)
                R Kj = R(0), Kj1 = R(0);
                if constexpr (NF == 2) {
                    if (C.model == 1) {
                        Kj = kapila_K<MODE, R>(WR(j, L::E), WR(j, L::A), C);
                        Kj1 = kapila_K<MODE, R>(WR(j + 1, L::E), WR(j + 1, L::A), C);
                    }
                }
#pragma unroll
                for (int a = 0; a < NF - 1; ++a) {
                    const int k = L::A + a;
                    ufb += (rbar(j, k) * (WR(j, k) + Kj) - rbar(j + 1, k) * (WR(j + 1, k) + Kj1)) * inv_dx;
                }
                R uf;
                hllc_adj<NF, ND, DIR, MODE>(WLcur, WRj, C, Fb, ufb, WLb, WRb, uf);
                UFR(j) = uf;
                if (first_order) {
                    // the face states are the cell states themselves
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        if (nonzero(WLb[k])) sink(j, k, WLb[k]);
                        if (nonzero(WRb[k])) sink(j + 1, k, WRb[k]);
                        WLb[k] = WRb[k] = R(0);
                    }
                }
            } else {
                UFR(j) = R(0);
#pragma unroll
                for (int k = 0; k < NQ; ++k) WLnext[k] = R(0);
            }
            if (cellw) {
                // adjoint of the WENO5 reconstruction of cell j: right edge = face j (WLb),
                // left edge = face j-1 (WRbprev)
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R f[5], fb[5];
#pragma unroll
                    for (int m = 0; m < 5; ++m) f[m] = WR(j - 2 + m, k);
                    weno5_cell_adj<MODE, R>(f, WRbprev[k], WLb[k], variant, eps, ct, fb);
#pragma unroll
                    for (int m = 0; m < 5; ++m)
                        if (nonzero(fb[m])) sink(j - 2 + m, k, fb[m]);
                }
            }
            // finish cell j-3
            const int64_t c = j - 3;
            if (pass == 2 && c >= s0 && c < s1) {
                const int64_t off = base + c * S;
                double qc[NQ], wb[NQ], qb[NQ];
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    qc[k] = __ldg(A.q + off + k * fs);
                    double v = double(ACC(c, k));
                    if (periodic && c < 3) v += double(ext_lo[c][k]);
                    if (periodic && c >= n - 3) v += double(ext_hi[c - (n - 3)][k]);
                    wb[k] = v;
                    qb[k] = 0.0;
                }
                // alpha_c (u_{c+1/2} - u_{c-1/2}) / dx, and for the Kapila model
                // K_c(p_c, alpha_c) (u_{c+1/2} - u_{c-1/2}) / dx
                const double du = double(UFR(c)) - double(UFR(c - 1));
                if constexpr (NF == 2) {
                    if (C.model == 1) {
                        double w[NQ];
                        bool b = false;
                        cons_to_prim<NF, ND, (MODE == MODE_EXACT ? MODE_EXACT : MODE_FAST)>(qc, w, C, b);
                        double dKdp, dKda;
                        kapila_K_grad(w[L::E], w[L::A], C, dKdp, dKda);
                        const double Kb = double(rbar(c, L::A)) * du * double(inv_dx);
                        wb[L::E] += Kb * dKdp;
                        wb[L::A] += Kb * dKda;
                    }
                }
                cons_to_prim_adj<NF, ND, MODE>(qc, wb, C, qb);
#pragma unroll
                for (int a = 0; a < NF - 1; ++a) {
                    const int k = L::A + a;
                    qb[k] += double(rbar(c, k)) * du * double(inv_dx);
                }
#pragma unroll
                for (int k = 0; k < NQ; ++k) A.qbar[off + k * fs] += qb[k];
            }
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                WRbprev[k] = WRb[k];
                WLcur[k] = WLnext[k];
            }
        }
    }
}

}  // namespace mfc
