// C ABI of the library (declared in include/mfc.h): argument checking,
// scratch ownership and the launch sequences of L(q), the RK3 step and the
// adjoints.  All numerical work runs in the kernels of mfc_fwd.cuh and
// mfc_vjp.cuh.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

#include "../../include/mfc.h"
#include "mfc_launch.h"

namespace {

thread_local std::string g_init_error;

struct DevScalars {
    unsigned long long minbits;  // CFL minimum (bit pattern of a positive double)
    double dt;                   // dt of the current step
    int flag;                    // non-physical state seen
    int pad;
};

}  // namespace

struct mfc_ctx {
    mfc_grid grid;
    mfc_eos eos;
    mfc_opts opts;
    mfc::Consts C;
    const mfc::LaunchFns* exact;  // CFL, maps and the MFC_FP64 sweeps
    const mfc::LaunchFns* fns;    // the sweeps of the chosen precision
    int mode;                     // mfc::MODE_* of the sweeps
    int device;
    int64_t total;        // doubles in a state-sized buffer
    double* q1 = nullptr;  // RK stage 1
    double* q2 = nullptr;  // RK stage 2
    double* r = nullptr;   // accumulated right-hand side
    // adjoint scratch (allocated on first use)
    double* a1 = nullptr;
    double* a2 = nullptr;
    double* a3 = nullptr;
    // x <-> y transposed copies for the x adjoint sweep (allocated on first use)
    double* t1 = nullptr;
    double* t2 = nullptr;
    double* t3 = nullptr;
    // cell velocities for the viscous stress (allocated at init when some eta_i > 0)
    double* vel = nullptr;
    // staging of host-resident states (mfc_rk3_step_batch_host; allocated on first use):
    // two device states, a dt per state, and the upload / download copy streams
    double* h[2] = {nullptr, nullptr};
    double* hdt = nullptr;
    int32_t hdt_cap = 0;
    cudaStream_t up = nullptr;
    cudaStream_t down = nullptr;
    cudaEvent_t ev_start = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_out[2] = {nullptr, nullptr};
    // split double-float sweeps (MFC_DF64; created at init): the stream that
    // runs the reconstructions, its fork event, a ring of edge-value buffers
    // with an event per slot for "filled" and "read", lines per chunk per axis
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_filled[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_read[3] = {nullptr, nullptr, nullptr};
    double* ebuf[3] = {nullptr, nullptr, nullptr};
    int64_t chunk_lines[3] = {0, 0, 0};
    DevScalars* scal = nullptr;
    std::string err;
};

namespace mfc {

int sweep_segment(int64_t n, int64_t nlines) {
    // Aim for ~8 resident 128-thread blocks per SM on 152 SMs; longer
    // segments amortise the 6-cell halo, shorter ones fill the GPU.
    const int64_t target = 152LL * 1024;
    int64_t seg = (n * nlines + target - 1) / target;
    if (seg < 16) seg = 16;
    if (seg > 64) seg = 64;
    if (seg > n) seg = n;
    if (seg < 1) seg = 1;
    return (int)seg;
}

}  // namespace mfc

namespace {

__global__ void set_scalars_kernel(DevScalars* s, double dt) {
    s->minbits = 0x7ff0000000000000ULL;  // +inf
    s->dt = dt;
}

__global__ void finalize_dt_kernel(DevScalars* s, double cfl, double* dt_out) {
    const double m = __longlong_as_double((long long)s->minbits);
    s->dt = cfl * m;
    if (dt_out) *dt_out = s->dt;
}

__global__ void copy_dt_kernel(const DevScalars* s, double* dt_out) { *dt_out = s->dt; }

// dst = src (add = 0) or dst += src (add = 1) with the x and y axes of the
// interior swapped and the fields of the x and y momenta swapped: cell
// (i, j, k) of src (layout Cs) goes to cell (j, i, k) of dst (layout Cd).
// 32 x 32 tiles through shared memory, so that both sides are read and
// written along their own fastest axis.
__global__ void __launch_bounds__(256) transpose_xy_kernel(const mfc::Consts Cs, const mfc::Consts Cd,
                                                           const double* src, double* dst, int add, int mom0) {
    __shared__ double tile[32][33];
    const int64_t nx = Cs.n[0], ny = Cs.n[1];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int64_t kf = blockIdx.z;  // field * nz + k
    const int64_t k = kf % Cs.n[2];
    const int f = (int)(kf / Cs.n[2]);
    const int fd = (f == mom0) ? mom0 + 1 : ((f == mom0 + 1) ? mom0 : f);
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + tx, j = j0 + r;
        if (i < nx && j < ny)
            tile[r][tx] = src[f * Cs.fstride + Cs.origin + i * Cs.stride[0] + j * Cs.stride[1] + k * Cs.stride[2]];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + tx, i = i0 + r;  // dst cell (j, i, k)
        if (i < nx && j < ny) {
            double* p = dst + fd * Cd.fstride + Cd.origin + j * Cd.stride[0] + i * Cd.stride[1] + k * Cd.stride[2];
            *p = add ? *p + tile[tx][r] : tile[tx][r];
        }
    }
}

// out = a x + b y + c z on the interior cells of every field (y, z may be
// null when their coefficient is 0).  Element-wise, so out may alias x, y or z.
__global__ void lincomb_kernel(const mfc::Consts C, double* out, double a, const double* x, double b,
                               const double* y, double c, const double* z) {
    const int64_t ncell = C.n[0] * C.n[1] * C.n[2];
    const int64_t total = ncell * C.nq;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / ncell, lin = t - f * ncell;
        const int64_t i = lin % C.n[0];
        const int64_t j = (lin / C.n[0]) % C.n[1];
        const int64_t k = lin / (C.n[0] * C.n[1]);
        const int64_t o = C.origin + i * C.stride[0] + j * C.stride[1] + k * C.stride[2] + f * C.fstride;
        double v = a * x[o];
        if (y) v += b * y[o];
        if (z) v += c * z[o];
        out[o] = v;
    }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

mfc_status fail(mfc_ctx* ctx, mfc_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

mfc_status cuda_fail(mfc_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, MFC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::string check_description(const mfc_grid* g, const mfc_eos* e, const mfc_opts* o) {
    if (!g || !e || !o) return "null description pointer";
    if (g->ndim < 1 || g->ndim > 3) return "ndim must be 1, 2 or 3";
    if (g->ghost < 0 || g->ghost > 64) return "ghost must be in [0, 64]";
    for (int a = 0; a < 3; ++a) {
        if (a < g->ndim) {
            if (g->n[a] < 1) return "every active axis needs n >= 1";
            if (!(g->hi[a] > g->lo[a]) || !std::isfinite(g->hi[a] - g->lo[a])) return "need lo < hi on active axes";
            for (int s = 0; s < 2; ++s) {
                const int bc = s ? g->bc_hi[a] : g->bc_lo[a];
                if (bc < 0 || bc > 3) return "unknown boundary condition";
                if (bc != MFC_BC_TRANSMISSIVE && g->n[a] < 3) return "periodic / reflective / halo axes need n >= 3";
                if (bc == MFC_BC_HALO && g->ghost < 3) return "a halo side needs ghost >= 3";
            }
            if ((g->bc_lo[a] == MFC_BC_PERIODIC) != (g->bc_hi[a] == MFC_BC_PERIODIC))
                return "periodic must be set on both ends of an axis";
        } else if (g->n[a] != 1) {
            return "inactive axes must have n = 1";
        }
    }
    const double cells = (double)g->n[0] * (double)g->n[1] * (double)g->n[2];
    if (cells > 4.0e12) return "grid too large";
    if (e->nfluids < 1 || e->nfluids > 4) return "nfluids must be 1 .. 4";
    for (int i = 0; i < e->nfluids; ++i) {
        if (!(e->gamma[i] > 1.0) || !std::isfinite(e->gamma[i])) return "gamma must be > 1";
        if (!(e->pi_inf[i] >= 0.0) || !std::isfinite(e->pi_inf[i])) return "pi_inf must be >= 0";
        if (!(e->eta[i] >= 0.0) || !std::isfinite(e->eta[i])) return "eta must be >= 0";
    }
    if (o->precision != MFC_FP64 && o->precision != MFC_MIXED && o->precision != MFC_FP64_FAST &&
        o->precision != MFC_DF64)
        return "unknown precision";
    if (o->weno < 0 || o->weno > 3) return "unknown WENO variant";
    if (o->weno == 3 && !(o->teno_ct > 0.0 && o->teno_ct < 1.0)) return "teno_ct must be in (0, 1)";
    if (o->model < 0 || o->model > 1) return "unknown model";
    if (o->model == 1 && e->nfluids != 2) return "the Kapila model needs nfluids = 2";
    if (o->riemann < 0 || o->riemann > 1) return "unknown Riemann solver";
    if (o->low_mach < 0 || o->low_mach > 2) return "unknown low-Mach correction";
    if (o->low_mach == 2 && o->riemann != 0) return "the anti-dissipation pressure correction needs HLLC";
    if (!(o->weno_eps > 0.0) || !std::isfinite(o->weno_eps)) return "weno_eps must be > 0";
    if (!(o->cfl > 0.0) || !std::isfinite(o->cfl)) return "cfl must be > 0";
    if (o->viscous_dt != 0 && o->viscous_dt != 1) return "viscous_dt must be 0 or 1";
    return "";
}

bool has_halo(const mfc_grid* g) {
    for (int a = 0; a < g->ndim; ++a)
        if (g->bc_lo[a] == MFC_BC_HALO || g->bc_hi[a] == MFC_BC_HALO) return true;
    return false;
}

void make_consts(const mfc_grid* g, const mfc_eos* e, const mfc_opts* o, mfc::Consts& C, int64_t& total) {
    std::memset(&C, 0, sizeof(C));
    C.nf = e->nfluids;
    C.nd = g->ndim;
    C.nq = 2 * C.nf + C.nd;
    C.weno = o->weno;
    int64_t np[3];
    for (int a = 0; a < 3; ++a) {
        C.n[a] = g->n[a];
        np[a] = g->n[a] + (a < g->ndim ? 2 * (int64_t)g->ghost : 0);
        C.bc_lo[a] = a < g->ndim ? g->bc_lo[a] : MFC_BC_TRANSMISSIVE;
        C.bc_hi[a] = a < g->ndim ? g->bc_hi[a] : MFC_BC_TRANSMISSIVE;
        C.dx[a] = a < g->ndim ? (g->hi[a] - g->lo[a]) / (double)g->n[a] : 1.0;
        C.inv_dx[a] = 1.0 / C.dx[a];
        C.inv_dxf[a] = (float)C.inv_dx[a];
    }
    C.stride[0] = 1;
    C.stride[1] = np[0];
    C.stride[2] = np[0] * np[1];
    C.fstride = np[0] * np[1] * np[2];
    C.origin = 0;
    for (int a = 0; a < g->ndim; ++a) C.origin += (int64_t)g->ghost * C.stride[a];
    for (int i = 0; i < e->nfluids; ++i) {
        C.g[i] = 1.0 / (e->gamma[i] - 1.0);
        C.h[i] = e->gamma[i] * e->pi_inf[i] / (e->gamma[i] - 1.0);
        C.gf[i] = (float)C.g[i];
        C.hf[i] = (float)C.h[i];
    }
    for (int i = 0; i < e->nfluids; ++i) {
        C.gd[i] = C.g[i] - C.g[e->nfluids - 1];
        C.hd[i] = C.h[i] - C.h[e->nfluids - 1];
        C.gdf[i] = (float)C.gd[i];
        C.hdf[i] = (float)C.hd[i];
    }
    C.eps = o->weno_eps;
    // float32 WENO rescales eps with the indicators and floors it (mfc_device.cuh)
    C.epsf = (float)o->weno_eps;
    C.teno_ct = o->weno == 3 ? o->teno_ct : 0.0;
    C.teno_ctf = (float)C.teno_ct;
    C.model = o->model;
    C.riemann = o->riemann;
    C.low_mach = o->low_mach;
    for (int i = 0; i < 2; ++i) {
        C.gam[i] = i < e->nfluids ? e->gamma[i] : 0.0;
        C.pinf[i] = i < e->nfluids ? e->pi_inf[i] : 0.0;
        C.gamf[i] = (float)C.gam[i];
        C.pinff[i] = (float)C.pinf[i];
    }
    C.viscous = 0;
    for (int i = 0; i < 4; ++i) {
        C.eta[i] = i < e->nfluids ? e->eta[i] : 0.0;
        C.etaf[i] = (float)C.eta[i];
        if (C.eta[i] > 0.0) C.viscous = 1;
    }
    C.cfl = o->cfl;
    C.visc_dt = (o->viscous_dt != 0 && C.viscous) ? 1 : 0;
    C.dx2min = C.dx[0] * C.dx[0];
    for (int a = 1; a < g->ndim; ++a) C.dx2min = (C.dx[a] * C.dx[a] < C.dx2min) ? C.dx[a] * C.dx[a] : C.dx2min;
    C.inv_dx2min = 1.0 / C.dx2min;
    total = C.fstride * C.nq;
}

const mfc::LaunchFns* exact_fns_for(int nf) {
    switch (nf) {
        case 1: return &mfc::launch_fns_exact_nf1();
        case 2: return &mfc::launch_fns_exact_nf2();
        case 3: return &mfc::launch_fns_exact_nf3();
        default: return &mfc::launch_fns_exact_nf4();
    }
}

const mfc::LaunchFns* fast_fns_for(int nf) {
    switch (nf) {
        case 1: return &mfc::launch_fns_fast_nf1();
        case 2: return &mfc::launch_fns_fast_nf2();
        case 3: return &mfc::launch_fns_fast_nf3();
        default: return &mfc::launch_fns_fast_nf4();
    }
}

// The MFC_DF64 tables: the fast table with the double-float sweeps.
mfc::LaunchFns with_df_sweep(const mfc::LaunchFns& fast,
                             cudaError_t (*sweep)(const mfc::Consts&, int, int, mfc::SweepArgs, cudaStream_t),
                             cudaError_t (*split)(const mfc::Consts&, int, int, mfc::SweepArgs, mfc::SplitChunk,
                                                  cudaStream_t)) {
    mfc::LaunchFns f = fast;
    f.sweep = sweep;
    f.split_sweep = split;
    return f;
}

const mfc::LaunchFns* df_fns_for(int nf) {
    static const mfc::LaunchFns t1 = with_df_sweep(mfc::launch_fns_fast_nf1(), &mfc::sweep_df_nf1, &mfc::split_df_nf1);
    static const mfc::LaunchFns t2 = with_df_sweep(mfc::launch_fns_fast_nf2(), &mfc::sweep_df_nf2, &mfc::split_df_nf2);
    static const mfc::LaunchFns t3 = with_df_sweep(mfc::launch_fns_fast_nf3(), &mfc::sweep_df_nf3, &mfc::split_df_nf3);
    static const mfc::LaunchFns t4 = with_df_sweep(mfc::launch_fns_fast_nf4(), &mfc::sweep_df_nf4, &mfc::split_df_nf4);
    switch (nf) {
        case 1: return &t1;
        case 2: return &t2;
        case 3: return &t3;
        default: return &t4;
    }
}

// Sweep table and arithmetic mode of a precision.
void select_precision(int precision, int nf, const mfc::LaunchFns*& fns, int& mode) {
    switch (precision) {
        case MFC_FP64: fns = exact_fns_for(nf); mode = mfc::MODE_EXACT; break;
        case MFC_MIXED: fns = fast_fns_for(nf); mode = mfc::MODE_MIXED; break;
        case MFC_DF64: fns = df_fns_for(nf); mode = mfc::MODE_DF; break;
        default: fns = fast_fns_for(nf); mode = mfc::MODE_FAST; break;
    }
}

// dt into ctx->scal->dt: the given value, or the CFL dt of q.
mfc_status eval_dt(mfc_ctx* ctx, const double* q, double dt, cudaStream_t s) {
    cudaError_t e;
    set_scalars_kernel<<<1, 1, 0, s>>>(ctx->scal, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "set scalars");
    if (dt > 0.0) return MFC_OK;
    if ((e = ctx->fns->cfl(ctx->C, q, &ctx->scal->minbits, &ctx->scal->flag, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "cfl kernel");
    finalize_dt_kernel<<<1, 1, 0, s>>>(ctx->scal, ctx->C.cfl, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "finalize dt");
    return MFC_OK;
}

constexpr int kSplitSlots = 3;

// Lines per chunk of a split sweep along `dir`: chunks of about four
// 128-thread blocks per SM of either kernel (measured on the 256^3
// shock-bubble: 158.6 M cell-updates/s; 151.6 M with two blocks per SM and
// 107.8 M with one, where chunks are smaller and more of their tails show).
int64_t split_chunk_lines(const mfc::Consts& C, int dir) {
    const int64_t n = C.n[dir];
    const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int64_t seg = mfc::sweep_segment(n, nlines);
    const int64_t nseg = (n + seg - 1) / seg;
    int64_t chunks = nlines * nseg / (152LL * 128 * 4);
    if (chunks < 1) chunks = 1;
    if (chunks > 16) chunks = 16;
    return (nlines + chunks - 1) / chunks;
}

// Stream, events and edge-value ring of the split MFC_DF64 sweeps.
mfc_status create_split(mfc_ctx* ctx) {
    const mfc::Consts& C = ctx->C;
    size_t doubles = 0;
    for (int d = 0; d < C.nd; ++d) {
        ctx->chunk_lines[d] = split_chunk_lines(C, d);
        const size_t need = (size_t)2 * C.nq * (size_t)(C.n[d] + 2) * (size_t)ctx->chunk_lines[d];
        if (need > doubles) doubles = need;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < kSplitSlots && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ctx->ev_filled[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_read[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->ebuf[i], doubles * sizeof(double));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? MFC_ERR_ALLOC : MFC_ERR_CUDA;
    }
    return MFC_OK;
}

void destroy_split(mfc_ctx* ctx) {
    for (int i = 0; i < kSplitSlots; ++i) {
        if (ctx->ebuf[i]) cudaFree(ctx->ebuf[i]);
        if (ctx->ev_filled[i]) cudaEventDestroy(ctx->ev_filled[i]);
        if (ctx->ev_read[i]) cudaEventDestroy(ctx->ev_read[i]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->side) cudaStreamDestroy(ctx->side);
}

// The directional sweeps of one evaluation of L in MFC_DF64, split: for each
// direction and chunk of lines, the reconstruction on ctx->side into a slot
// of the ring, then the Riemann solve and update from it on s.  A slot is
// refilled only after the Riemann kernel that read it (3 chunks earlier)
// is done; the reconstructions start after everything queued on s before
// this call.  Same SweepArgs as the fused sweeps of eval_L.
mfc_status eval_L_split(mfc_ctx* ctx, const double* qin, double* rhs, int out_kind, const double* qn,
                        double* qout, double a, double b, cudaStream_t s) {
    const mfc::Consts& C = ctx->C;
    cudaError_t e = cudaEventRecord(ctx->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "split sweep: fork");
    if (C.viscous) {
        e = ctx->fns->viscous(C, ctx->mode, qin, ctx->vel, rhs, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "viscous kernels");
    }
    int64_t j = 0;
    for (int d = 0; d < C.nd; ++d) {
        mfc::SweepArgs A;
        std::memset(&A, 0, sizeof(A));
        A.q = qin;
        A.rhs = rhs;
        A.acc_in = (d == 0 && !C.viscous) ? 0 : 1;
        A.out_kind = d == C.nd - 1 ? out_kind : 0;
        A.qn = qn;
        A.qout = qout;
        A.dt = &ctx->scal->dt;
        A.rk_a = a;
        A.rk_b = b;
        A.flag = &ctx->scal->flag;
        const int64_t nlines = C.n[0] * C.n[1] * C.n[2] / C.n[d];
        const int64_t per = ctx->chunk_lines[d];
        for (int64_t l0 = 0; l0 < nlines; l0 += per, ++j) {
            const int slot = (int)(j % kSplitSlots);
            mfc::SplitChunk K;
            K.line0 = l0;
            K.nl = (nlines - l0 < per) ? nlines - l0 : per;
            K.E = ctx->ebuf[slot];
            if (j >= kSplitSlots && (e = cudaStreamWaitEvent(ctx->side, ctx->ev_read[slot], 0)) != cudaSuccess)
                return cuda_fail(ctx, e, "split sweep: slot wait");
            if ((e = ctx->fns->split_sweep(C, d, 0, A, K, ctx->side)) != cudaSuccess)
                return cuda_fail(ctx, e, "reconstruction kernel");
            if ((e = cudaEventRecord(ctx->ev_filled[slot], ctx->side)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, ctx->ev_filled[slot], 0)) != cudaSuccess)
                return cuda_fail(ctx, e, "split sweep: join");
            if ((e = ctx->fns->split_sweep(C, d, 1, A, K, s)) != cudaSuccess)
                return cuda_fail(ctx, e, "riemann kernel");
            if ((e = cudaEventRecord(ctx->ev_read[slot], s)) != cudaSuccess)
                return cuda_fail(ctx, e, "split sweep: slot record");
        }
    }
    return MFC_OK;
}

// All directional sweeps of one evaluation of L(qin), after the viscous
// kernels when some eta_i > 0 (their result is the starting value of the
// accumulation).  out_kind 0 writes L into rhs; 1 and 2 fuse the RK stage
// update into the last sweep.  The
// mixed mode sums the directions in a float accumulator that aliases the
// scratch buffer ctx->r (first half; rhs may be ctx->r itself only when
// out_kind is 1 or 2, where rhs is not written).
mfc_status eval_L(mfc_ctx* ctx, const double* qin, double* rhs, int out_kind, const double* qn, double* qout,
                  double a, double b, cudaStream_t s) {
    if (ctx->side) return eval_L_split(ctx, qin, rhs, out_kind, qn, qout, a, b, s);
    const bool mixed = ctx->mode == mfc::MODE_MIXED;
    float* accf = reinterpret_cast<float*>(ctx->r);
    if (ctx->C.viscous) {
        // the viscous right-hand side is the value the sweeps accumulate onto
        cudaError_t e = ctx->fns->viscous(ctx->C, ctx->mode, qin, ctx->vel, rhs, accf, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "viscous kernels");
    }
    for (int d = 0; d < ctx->C.nd; ++d) {
        mfc::SweepArgs A;
        std::memset(&A, 0, sizeof(A));
        A.q = qin;
        A.rhs = rhs;
        A.rhsf = accf;
        const bool last = d == ctx->C.nd - 1;
        A.acc_in = (d == 0 && !ctx->C.viscous) ? 0 : (mixed ? 2 : 1);
        A.out_kind = last ? out_kind : (mixed ? 3 : 0);
        A.qn = qn;
        A.qout = qout;
        A.dt = &ctx->scal->dt;
        A.rk_a = a;
        A.rk_b = b;
        A.flag = &ctx->scal->flag;
        cudaError_t e = ctx->fns->sweep(ctx->C, d, ctx->mode, A, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep kernel");
    }
    return MFC_OK;
}

const double RK_A2 = 0.75, RK_B2 = 0.25, RK_A3 = 1.0 / 3.0, RK_B3 = 2.0 / 3.0;

mfc_status rk3_once(mfc_ctx* ctx, double* q, double dt, double* dt_used, cudaStream_t s) {
    mfc_status st = eval_dt(ctx, q, dt, s);
    if (st != MFC_OK) return st;
    if ((st = eval_L(ctx, q, ctx->r, 1, nullptr, ctx->q1, 0.0, 1.0, s)) != MFC_OK) return st;
    if ((st = eval_L(ctx, ctx->q1, ctx->r, 2, q, ctx->q2, RK_A2, RK_B2, s)) != MFC_OK) return st;
    if ((st = eval_L(ctx, ctx->q2, ctx->r, 2, q, q, RK_A3, RK_B3, s)) != MFC_OK) return st;
    if (dt_used) {
        copy_dt_kernel<<<1, 1, 0, s>>>(ctx->scal, dt_used);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy dt");
    }
    return MFC_OK;
}

mfc_status lincomb(mfc_ctx* ctx, double* out, double a, const double* x, double b, const double* y, double c,
                   const double* z, cudaStream_t s) {
    const int64_t total = ctx->C.n[0] * ctx->C.n[1] * ctx->C.n[2] * ctx->C.nq;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    lincomb_kernel<<<(unsigned)blocks, 256, 0, s>>>(ctx->C, out, a, x, b, y, c, z);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MFC_OK : cuda_fail(ctx, e, "lincomb kernel");
}

// qbar += (dL/dq)^T rbar: one adjoint sweep per direction.
// The constants of the same grid with the x and y axes swapped.
mfc::Consts transposed_xy(const mfc::Consts& C) {
    mfc::Consts T = C;
    std::swap(T.n[0], T.n[1]);
    std::swap(T.bc_lo[0], T.bc_lo[1]);
    std::swap(T.bc_hi[0], T.bc_hi[1]);
    std::swap(T.dx[0], T.dx[1]);
    std::swap(T.inv_dx[0], T.inv_dx[1]);
    std::swap(T.inv_dxf[0], T.inv_dxf[1]);
    // padded extents: x of T is y of C and vice versa (ghost width g on both)
    const int64_t px = C.stride[1], py = C.stride[2] / C.stride[1];
    const int64_t g = (px - C.n[0]) / 2;
    T.stride[0] = 1;
    T.stride[1] = py;
    T.stride[2] = C.stride[2];
    T.origin = g * T.stride[0] + g * T.stride[1] + (C.origin - g * C.stride[0] - g * C.stride[1]);
    return T;
}

mfc_status ensure_transpose_scratch(mfc_ctx* ctx) {
    if (ctx->t1) return MFC_OK;
    const size_t bytes = (size_t)ctx->total * sizeof(double);
    if (cudaMalloc(&ctx->t1, bytes) != cudaSuccess || cudaMalloc(&ctx->t2, bytes) != cudaSuccess ||
        cudaMalloc(&ctx->t3, bytes) != cudaSuccess) {
        cudaGetLastError();
        for (double** p : {&ctx->t1, &ctx->t2, &ctx->t3}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        return fail(ctx, MFC_ERR_ALLOC, "device allocation of the adjoint transpose scratch failed");
    }
    return MFC_OK;
}

mfc_status transpose_xy(mfc_ctx* ctx, const mfc::Consts& Cs, const mfc::Consts& Cd, const double* src, double* dst,
                        int add, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((Cs.n[0] + 31) / 32), (unsigned)((Cs.n[1] + 31) / 32),
                    (unsigned)(Cs.n[2] * Cs.nq));
    transpose_xy_kernel<<<grid, block, 0, s>>>(Cs, Cd, src, dst, add, Cs.nf);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MFC_OK : cuda_fail(ctx, e, "transpose kernel");
}

// qbar += (dL/dq)^T rbar: one adjoint sweep per direction.  In 2D and 3D
// the x sweep runs as a y sweep on x <-> y transposed copies of q, rbar and
// its own bar: the per-thread march along x reads 32 rows at once and
// thrashes L1, the y march reads rows whole (the result is the same
// arithmetic on the same values).
mfc_status eval_L_vjp(mfc_ctx* ctx, const double* q, const double* rbar, double* qbar, cudaStream_t s) {
    const mfc::Consts& C = ctx->C;
    for (int d = 0; d < C.nd; ++d) {
        mfc::VjpArgs A;
        std::memset(&A, 0, sizeof(A));
        cudaError_t e;
        if (d == 0 && C.nd >= 2) {
            mfc_status st = ensure_transpose_scratch(ctx);
            if (st != MFC_OK) return st;
            const mfc::Consts T = transposed_xy(C);
            if ((st = transpose_xy(ctx, C, T, q, ctx->t1, 0, s)) != MFC_OK) return st;
            if ((st = transpose_xy(ctx, C, T, rbar, ctx->t2, 0, s)) != MFC_OK) return st;
            if ((e = cudaMemsetAsync(ctx->t3, 0, (size_t)ctx->total * sizeof(double), s)) != cudaSuccess)
                return cuda_fail(ctx, e, "clear transposed bar");
            A.q = ctx->t1;
            A.rbar = ctx->t2;
            A.qbar = ctx->t3;
            if ((e = ctx->fns->sweep_vjp(T, 1, ctx->mode, A, s)) != cudaSuccess)
                return cuda_fail(ctx, e, "adjoint sweep kernel");
            if ((st = transpose_xy(ctx, T, C, ctx->t3, qbar, 1, s)) != MFC_OK) return st;
            continue;
        }
        A.q = q;
        A.rbar = rbar;
        A.qbar = qbar;
        if ((e = ctx->fns->sweep_vjp(C, d, ctx->mode, A, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "adjoint sweep kernel");
    }
    return MFC_OK;
}

mfc_status ensure_adjoint_scratch(mfc_ctx* ctx) {
    if (ctx->a1) return MFC_OK;
    const size_t bytes = (size_t)ctx->total * sizeof(double);
    if (cudaMalloc(&ctx->a1, bytes) != cudaSuccess || cudaMalloc(&ctx->a2, bytes) != cudaSuccess ||
        cudaMalloc(&ctx->a3, bytes) != cudaSuccess) {
        cudaGetLastError();
        for (double** p : {&ctx->a1, &ctx->a2, &ctx->a3}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        return fail(ctx, MFC_ERR_ALLOC, "device allocation of the adjoint scratch failed");
    }
    return MFC_OK;
}

mfc_status read_flag(mfc_ctx* ctx, cudaStream_t s) {
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, &ctx->scal->flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read flag");
    if (flag) {
        e = cudaMemsetAsync(&ctx->scal->flag, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear flag");
        return fail(ctx, MFC_ERR_NONPHYSICAL, "non-physical state (rho <= 0 or c^2 <= 0) met on the device");
    }
    return MFC_OK;
}

// Device staging for mfc_rk3_step_batch_host: two state buffers, copy
// streams that do not synchronise with the legacy default stream, and
// events without timing.  dts holds the dt of every state of one call.
void release_host_staging(mfc_ctx* ctx) {
    for (double*& p : ctx->h) {
        if (p) cudaFree(p);
        p = nullptr;
    }
    for (cudaEvent_t* ev : {&ctx->ev_start, &ctx->ev_in[0], &ctx->ev_in[1], &ctx->ev_done[0], &ctx->ev_done[1],
                            &ctx->ev_out[0], &ctx->ev_out[1]}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    for (cudaStream_t* st : {&ctx->up, &ctx->down}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
}

mfc_status ensure_host_staging(mfc_ctx* ctx, int32_t count) {
    const size_t bytes = (size_t)ctx->total * sizeof(double);
    if (!ctx->h[0]) {
        bool ok = cudaMalloc(&ctx->h[0], bytes) == cudaSuccess && cudaMalloc(&ctx->h[1], bytes) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->up, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->down, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < 2; ++k)
            ok = cudaEventCreateWithFlags(&ctx->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->ev_out[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            release_host_staging(ctx);
            return fail(ctx, MFC_ERR_ALLOC, "creating the host staging buffers, streams or events failed");
        }
    }
    if (count > ctx->hdt_cap) {
        if (ctx->hdt) cudaFree(ctx->hdt);
        ctx->hdt = nullptr;
        ctx->hdt_cap = 0;
        const int32_t cap = count < 64 ? 64 : count;
        if (cudaMalloc(&ctx->hdt, (size_t)cap * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, MFC_ERR_ALLOC, "device allocation of the dt array failed");
        }
        ctx->hdt_cap = cap;
    }
    return MFC_OK;
}

// Enqueue the pipelined batch (see mfc_rk3_step_batch_host).  State b
// uses staging buffer b % 2: its upload waits for the download of state
// b - 2 from the same buffer, its step (on s) waits for the upload, and
// its download waits for the step.
mfc_status enqueue_batch_host(mfc_ctx* ctx, int32_t count, const double* const* q_in, double* const* q_out,
                              double dt, cudaStream_t s) {
    const size_t bytes = (size_t)ctx->total * sizeof(double);
    cudaError_t e;
    if ((e = cudaEventRecord(ctx->ev_start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->up, ctx->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->down, ctx->ev_start, 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "batch start");
    for (int32_t b = 0; b < count; ++b) {
        const int k = b & 1;
        double* buf = ctx->h[k];
        if (b >= 2 && (e = cudaStreamWaitEvent(ctx->up, ctx->ev_out[k], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "upload wait");
        if ((e = cudaMemcpyAsync(buf, q_in[b], bytes, cudaMemcpyHostToDevice, ctx->up)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_in[k], ctx->up)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, ctx->ev_in[k], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "upload");
        mfc_status st = rk3_once(ctx, buf, dt, ctx->hdt + b, s);
        if (st != MFC_OK) return st;
        if ((e = cudaEventRecord(ctx->ev_done[k], s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->down, ctx->ev_done[k], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(q_out[b], buf, bytes, cudaMemcpyDeviceToHost, ctx->down)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_out[k], ctx->down)) != cudaSuccess)
            return cuda_fail(ctx, e, "download");
    }
    return MFC_OK;
}

#define MFC_CHECK_CTX(ctx)                  \
    do {                                    \
        if (!(ctx)) return MFC_ERR_ARG;     \
    } while (0)

}  // namespace

extern "C" {

mfc_status mfc_init(const mfc_grid* grid, const mfc_eos* eos, const mfc_opts* opts, mfc_ctx** out) {
    if (!out) {
        g_init_error = "null output pointer";
        return MFC_ERR_ARG;
    }
    *out = nullptr;
    const std::string why = check_description(grid, eos, opts);
    if (!why.empty()) {
        g_init_error = why;
        return MFC_ERR_ARG;
    }
    bool viscous = false;
    for (int i = 0; i < eos->nfluids; ++i) viscous = viscous || eos->eta[i] > 0.0;
    if (viscous && has_halo(grid)) {
        g_init_error = "halo sides (MFC_BC_HALO) are not supported with viscosity";
        return MFC_ERR_UNSUPPORTED;
    }
    mfc_ctx* ctx = new (std::nothrow) mfc_ctx();
    if (!ctx) {
        g_init_error = "host allocation failed";
        return MFC_ERR_ALLOC;
    }
    ctx->grid = *grid;
    ctx->eos = *eos;
    ctx->opts = *opts;
    make_consts(grid, eos, opts, ctx->C, ctx->total);
    ctx->exact = exact_fns_for(eos->nfluids);
    select_precision(opts->precision, eos->nfluids, ctx->fns, ctx->mode);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        g_init_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        delete ctx;
        return MFC_ERR_CUDA;
    }
    const size_t bytes = (size_t)ctx->total * sizeof(double);
    if (cudaMalloc(&ctx->q1, bytes) != cudaSuccess || cudaMalloc(&ctx->q2, bytes) != cudaSuccess ||
        cudaMalloc(&ctx->r, bytes) != cudaSuccess || cudaMalloc(&ctx->scal, sizeof(DevScalars)) != cudaSuccess) {
        cudaGetLastError();
        g_init_error = "device allocation of the scratch buffers failed";
        mfc_destroy(ctx);
        return MFC_ERR_ALLOC;
    }
    if (ctx->C.viscous && cudaMalloc(&ctx->vel, (size_t)ctx->C.nd * ctx->C.fstride * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        g_init_error = "device allocation of the velocity scratch failed";
        mfc_destroy(ctx);
        return MFC_ERR_ALLOC;
    }
    if (ctx->mode == mfc::MODE_DF) {
        const mfc_status st = create_split(ctx);
        if (st != MFC_OK) {
            g_init_error = "creating the split double-float sweep's stream, events or edge-value buffers failed";
            mfc_destroy(ctx);
            return st;
        }
    }
    if ((e = cudaMemset(ctx->scal, 0, sizeof(DevScalars))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        g_init_error = std::string("initialising scalars: ") + cudaGetErrorString(e);
        mfc_destroy(ctx);
        return MFC_ERR_CUDA;
    }
    g_init_error.clear();
    *out = ctx;
    return MFC_OK;
}

mfc_status mfc_destroy(mfc_ctx* ctx) {
    if (!ctx) return MFC_OK;
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
    for (double* p : {ctx->q1, ctx->q2, ctx->r, ctx->a1, ctx->a2, ctx->a3, ctx->t1, ctx->t2, ctx->t3, ctx->hdt,
                      ctx->vel})
        if (p) cudaFree(p);
    release_host_staging(ctx);
    destroy_split(ctx);
    if (ctx->scal) cudaFree(ctx->scal);
    delete ctx;
    return MFC_OK;
}

int64_t mfc_field_stride(const mfc_ctx* ctx) { return ctx ? ctx->C.fstride : -1; }

int32_t mfc_num_fields(const mfc_ctx* ctx) { return ctx ? ctx->C.nq : -1; }

mfc_status mfc_prim_to_cons(mfc_ctx* ctx, const double* w, double* q, void* stream) {
    MFC_CHECK_CTX(ctx);
    if (!w || !q) return fail(ctx, MFC_ERR_ARG, "null buffer");
    DeviceGuard guard(ctx->device);
    cudaError_t e = ctx->exact->prim_to_cons(ctx->C, w, q, (cudaStream_t)stream);
    return e == cudaSuccess ? MFC_OK : cuda_fail(ctx, e, "prim_to_cons");
}

mfc_status mfc_cons_to_prim(mfc_ctx* ctx, const double* q, double* w, void* stream) {
    MFC_CHECK_CTX(ctx);
    if (!w || !q) return fail(ctx, MFC_ERR_ARG, "null buffer");
    DeviceGuard guard(ctx->device);
    cudaError_t e = ctx->exact->cons_to_prim(ctx->C, q, w, &ctx->scal->flag, (cudaStream_t)stream);
    return e == cudaSuccess ? MFC_OK : cuda_fail(ctx, e, "cons_to_prim");
}

mfc_status mfc_compute_dt(mfc_ctx* ctx, const double* q, double* dt_out, void* stream) {
    MFC_CHECK_CTX(ctx);
    if (!q || !dt_out) return fail(ctx, MFC_ERR_ARG, "null buffer");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    mfc_status st = eval_dt(ctx, q, 0.0, s);
    if (st != MFC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(dt_out, &ctx->scal->dt, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy dt");
    return read_flag(ctx, s);
}

mfc_status mfc_rhs(mfc_ctx* ctx, const double* q, double* rhs, void* stream) {
    MFC_CHECK_CTX(ctx);
    if (!q || !rhs) return fail(ctx, MFC_ERR_ARG, "null buffer");
    if (q == rhs) return fail(ctx, MFC_ERR_ARG, "rhs must not alias q");
    DeviceGuard guard(ctx->device);
    return eval_L(ctx, q, rhs, 0, nullptr, nullptr, 0.0, 0.0, (cudaStream_t)stream);
}

#define MFC_REFUSE_HALO(ctx)                                                                              \
    do {                                                                                                  \
        if (has_halo(&(ctx)->grid))                                                                       \
            return fail(ctx, MFC_ERR_UNSUPPORTED,                                                         \
                        "a context with halo sides steps stage by stage (mfc_rk3_stage), the halos "      \
                        "refreshed between stages");                                                     \
    } while (0)

mfc_status mfc_rk3_step(mfc_ctx* ctx, double* q, double dt, double* dt_used, void* stream) {
    MFC_CHECK_CTX(ctx);
    MFC_REFUSE_HALO(ctx);
    if (!q) return fail(ctx, MFC_ERR_ARG, "null buffer");
    if (!std::isfinite(dt)) return fail(ctx, MFC_ERR_ARG, "dt must be finite");
    DeviceGuard guard(ctx->device);
    return rk3_once(ctx, q, dt, dt_used, (cudaStream_t)stream);
}

mfc_status mfc_rk3_stage(mfc_ctx* ctx, int32_t stage, const double* q_in, const double* q_n, double* q_out,
                         double dt, void* stream) {
    MFC_CHECK_CTX(ctx);
    if (stage < 1 || stage > 3) return fail(ctx, MFC_ERR_ARG, "stage must be 1, 2 or 3");
    if (!q_in || !q_out || (stage > 1 && !q_n)) return fail(ctx, MFC_ERR_ARG, "null buffer");
    if (q_out == q_in) return fail(ctx, MFC_ERR_ARG, "q_out must not alias q_in");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, MFC_ERR_ARG, "a stage needs the step's dt > 0");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    mfc_status st = eval_dt(ctx, q_in, dt, s);
    if (st != MFC_OK) return st;
    if (stage == 1) return eval_L(ctx, q_in, ctx->r, 1, nullptr, q_out, 0.0, 1.0, s);
    if (stage == 2) return eval_L(ctx, q_in, ctx->r, 2, q_n, q_out, RK_A2, RK_B2, s);
    return eval_L(ctx, q_in, ctx->r, 2, q_n, q_out, RK_A3, RK_B3, s);
}

mfc_status mfc_rk3_run(mfc_ctx* ctx, double* q, int32_t nsteps, double dt, double* dt_log, void* stream) {
    MFC_CHECK_CTX(ctx);
    MFC_REFUSE_HALO(ctx);
    if (!q || nsteps < 0) return fail(ctx, MFC_ERR_ARG, "null buffer or negative step count");
    if (!std::isfinite(dt)) return fail(ctx, MFC_ERR_ARG, "dt must be finite");
    DeviceGuard guard(ctx->device);
    for (int32_t i = 0; i < nsteps; ++i) {
        mfc_status st = rk3_once(ctx, q, dt, dt_log ? dt_log + i : nullptr, (cudaStream_t)stream);
        if (st != MFC_OK) return st;
    }
    return MFC_OK;
}

mfc_status mfc_rk3_step_batch_host(mfc_ctx* ctx, int32_t count, const double* const* q_in, double* const* q_out,
                                   double dt, double* dt_used, void* stream) {
    MFC_CHECK_CTX(ctx);
    MFC_REFUSE_HALO(ctx);
    if (count < 0) return fail(ctx, MFC_ERR_ARG, "negative state count");
    if (count == 0) return MFC_OK;
    if (!q_in || !q_out) return fail(ctx, MFC_ERR_ARG, "null pointer array");
    for (int32_t b = 0; b < count; ++b)
        if (!q_in[b] || !q_out[b]) return fail(ctx, MFC_ERR_ARG, "null host buffer");
    if (!std::isfinite(dt)) return fail(ctx, MFC_ERR_ARG, "dt must be finite");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    mfc_status st = ensure_host_staging(ctx, count);
    if (st != MFC_OK) return st;
    st = enqueue_batch_host(ctx, count, q_in, q_out, dt, s);
    // drain all three streams whatever happened, so that no copy into or
    // out of the caller's host buffers is in flight after the return
    cudaError_t e1 = cudaStreamSynchronize(ctx->up);
    cudaError_t e2 = cudaStreamSynchronize(ctx->down);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (st != MFC_OK) return st;
    if (e1 != cudaSuccess) return cuda_fail(ctx, e1, "upload stream");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "download stream");
    if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "step stream");
    if (dt_used) {
        cudaError_t e = cudaMemcpy(dt_used, ctx->hdt, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dt read-back");
    }
    return read_flag(ctx, s);
}

mfc_status mfc_rhs_vjp(mfc_ctx* ctx, const double* q, const double* rhs_bar, double* q_bar, void* stream) {
    MFC_CHECK_CTX(ctx);
    MFC_REFUSE_HALO(ctx);
    if (!q || !rhs_bar || !q_bar) return fail(ctx, MFC_ERR_ARG, "null buffer");
    if (q_bar == q || q_bar == rhs_bar) return fail(ctx, MFC_ERR_ARG, "q_bar must not alias q or rhs_bar");
    if (ctx->C.viscous) return fail(ctx, MFC_ERR_UNSUPPORTED, "the adjoint of the viscous term is not implemented");
    DeviceGuard guard(ctx->device);
    return eval_L_vjp(ctx, q, rhs_bar, q_bar, (cudaStream_t)stream);
}

mfc_status mfc_rk3_step_vjp(mfc_ctx* ctx, const double* q_n, double dt, const double* qnp1_bar, double* qn_bar,
                            void* stream) {
    MFC_CHECK_CTX(ctx);
    MFC_REFUSE_HALO(ctx);
    if (!q_n || !qnp1_bar || !qn_bar) return fail(ctx, MFC_ERR_ARG, "null buffer");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, MFC_ERR_ARG, "the adjoint needs the step's dt > 0");
    if (qn_bar == q_n || qnp1_bar == q_n) return fail(ctx, MFC_ERR_ARG, "bars must not alias q_n");
    if (ctx->C.viscous) return fail(ctx, MFC_ERR_UNSUPPORTED, "the adjoint of the viscous term is not implemented");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    mfc_status st = ensure_adjoint_scratch(ctx);
    if (st != MFC_OK) return st;
    // recompute the stages q1, q2 of the forward step at the same dt
    if ((st = eval_dt(ctx, q_n, dt, s)) != MFC_OK) return st;
    if ((st = eval_L(ctx, q_n, ctx->r, 1, nullptr, ctx->q1, 0.0, 1.0, s)) != MFC_OK) return st;
    if ((st = eval_L(ctx, ctx->q1, ctx->r, 2, q_n, ctx->q2, RK_A2, RK_B2, s)) != MFC_OK) return st;
    const double* g3 = qnp1_bar;
    double *b2 = ctx->a1, *r = ctx->a2, *b1 = ctx->a3;
    // q^{n+1} = 1/3 q^n + 2/3 (q2 + dt L(q2))
    if ((st = lincomb(ctx, b2, RK_B3, g3, 0.0, nullptr, 0.0, nullptr, s)) != MFC_OK) return st;
    if ((st = lincomb(ctx, r, RK_B3 * dt, g3, 0.0, nullptr, 0.0, nullptr, s)) != MFC_OK) return st;
    if ((st = eval_L_vjp(ctx, ctx->q2, r, b2, s)) != MFC_OK) return st;
    // q2 = 3/4 q^n + 1/4 (q1 + dt L(q1))
    if ((st = lincomb(ctx, b1, RK_B2, b2, 0.0, nullptr, 0.0, nullptr, s)) != MFC_OK) return st;
    if ((st = lincomb(ctx, r, RK_B2 * dt, b2, 0.0, nullptr, 0.0, nullptr, s)) != MFC_OK) return st;
    if ((st = eval_L_vjp(ctx, ctx->q1, r, b1, s)) != MFC_OK) return st;
    // q1 = q^n + dt L(q^n)
    if ((st = lincomb(ctx, qn_bar, RK_A3, g3, RK_A2, b2, 1.0, b1, s)) != MFC_OK) return st;
    if ((st = lincomb(ctx, r, dt, b1, 0.0, nullptr, 0.0, nullptr, s)) != MFC_OK) return st;
    return eval_L_vjp(ctx, q_n, r, qn_bar, s);
}

mfc_status mfc_check(mfc_ctx* ctx, void* stream) {
    MFC_CHECK_CTX(ctx);
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pending CUDA error");
    return read_flag(ctx, (cudaStream_t)stream);
}

const char* mfc_last_error(const mfc_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free RK3 step.  Its scratch (the two stage states, the
// right-hand-side accumulator and the dt / flag scalars) is a file-scope
// device array, so the call needs no context and allocates no device memory.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoallocScalarDoubles = 32;  // 256 bytes in front of the state buffers
static __device__ __align__(256) double g_noalloc_scratch[MFC_NOALLOC_SCRATCH_DOUBLES];

constexpr int kNoallocMaxDevices = 64;
// Device address of the array on each device, looked up by the first call on
// that device.  Concurrent first calls may both look it up; they store the
// same value.
std::atomic<double*> g_noalloc_ptr[kNoallocMaxDevices] = {};

// dt_used = NaN when the step met a non-physical state (the flag the step's
// kernels set), so that a caller without a context can still see it.
__global__ void flag_to_dt_kernel(const DevScalars* s, double* dt_out) {
    if (s->flag) *dt_out = __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace

extern "C" mfc_status mfc_rk3_step_noalloc(const mfc_grid* grid, const mfc_eos* eos, const mfc_opts* opts,
                                           double* q, double dt, double* dt_used, void* stream) {
    const std::string why = check_description(grid, eos, opts);
    if (!why.empty()) {
        g_init_error = why;
        return MFC_ERR_ARG;
    }
    if (!q || !std::isfinite(dt)) {
        g_init_error = "null state or non-finite dt";
        return MFC_ERR_ARG;
    }
    if (has_halo(grid)) {
        g_init_error = "the allocation-free step has no halo exchange between its stages";
        return MFC_ERR_UNSUPPORTED;
    }
    mfc_ctx ctx;
    make_consts(grid, eos, opts, ctx.C, ctx.total);
    if (ctx.C.viscous) {
        g_init_error = "the allocation-free step has no scratch for the viscous stress";
        return MFC_ERR_UNSUPPORTED;
    }
    if (kNoallocScalarDoubles + 3 * ctx.total > (int64_t)MFC_NOALLOC_SCRATCH_DOUBLES) {
        g_init_error = "state too large for the allocation-free step: 3 x (padded cells x fields) + 32 must not "
                       "exceed MFC_NOALLOC_SCRATCH_DOUBLES";
        return MFC_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        g_init_error = "no usable current CUDA device";
        return MFC_ERR_CUDA;
    }
    // once per device, with that device current: the device address of the array
    double* base = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!base) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            g_init_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return MFC_ERR_CUDA;
        }
        base = static_cast<double*>(p);
        g_noalloc_ptr[dev].store(base, std::memory_order_release);
    }
    ctx.grid = *grid;
    ctx.eos = *eos;
    ctx.opts = *opts;
    ctx.device = dev;
    ctx.exact = exact_fns_for(eos->nfluids);
    select_precision(opts->precision, eos->nfluids, ctx.fns, ctx.mode);
    ctx.scal = reinterpret_cast<DevScalars*>(base);
    ctx.q1 = base + kNoallocScalarDoubles;
    ctx.q2 = ctx.q1 + ctx.total;
    ctx.r = ctx.q2 + ctx.total;
    cudaStream_t s = (cudaStream_t)stream;
    // the non-physical flag is the only scratch value read before it is written
    e = cudaMemsetAsync(&ctx.scal->flag, 0, sizeof(int), s);
    if (e != cudaSuccess) {
        g_init_error = std::string("clearing the flag: ") + cudaGetErrorString(e);
        return MFC_ERR_CUDA;
    }
    const mfc_status st = rk3_once(&ctx, q, dt, dt_used, s);
    if (st != MFC_OK) {
        g_init_error = ctx.err;
        return st;
    }
    if (dt_used) {
        flag_to_dt_kernel<<<1, 1, 0, s>>>(ctx.scal, dt_used);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            g_init_error = std::string("flag kernel: ") + cudaGetErrorString(e);
            return MFC_ERR_CUDA;
        }
    }
    return MFC_OK;
}
