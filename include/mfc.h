/*
 * mfc.h - C ABI of the GB300 (sm_103a) library for the finite-volume
 * right-hand side of the five-equation diffuse-interface model of
 * arXiv 2503.07953 (MFC 5.0), time-stepped with third-order TVD Runge-Kutta.
 *
 * What the library computes (citations are to the paper):
 *   state q per cell (Sec. 2.1.1): alpha_1 rho_1 .. alpha_N rho_N,
 *     rho u_1 .. rho u_ndim, rho E, alpha_1 .. alpha_{N-1}
 *     (alpha_N = 1 - sum of the others, mixture rules of Sec. 2.1.1);
 *   EOS: stiffened gas per fluid (Sec. 2.2);
 *   L(q): Eq. (rhs) of Sec. 3.1 - per direction, conservative-to-primitive
 *     conversion, WENO5 reconstruction of the primitive variables
 *     (Sec. 3.2.1 / Sec. 4.2.2), HLLC flux and face velocity (Sec. 3.2.2),
 *     flux difference plus alpha div(u) for the volume-fraction rows;
 *   ghost cells: periodic, transmissive (zeroth-order extrapolation) or
 *     reflective (mirror, normal momentum negated) (Sec. 3.3);
 *   time step: third-order TVD Runge-Kutta (Sec. 3.4) with
 *     dt = CFL * min over cells and directions of dx_d / (|u_d| + c).
 * The adjoint entry points (mfc_rhs_vjp, mfc_rk3_step_vjp) have no
 * counterpart in the paper: they are the exact transposed derivatives of
 * mfc_rhs and mfc_rk3_step at fixed dt.
 *
 * Memory layout.  Every state-shaped buffer (q, rhs, w, q_bar, ...) is a
 * DEVICE pointer to float64, structure-of-arrays, C order
 *     [field][nz + 2g][ny + 2g][nx + 2g]
 * where g = grid.ghost on each active axis and inactive axes have extent 1
 * and no ghost layer.  mfc_field_stride() returns the doubles per field.
 * The library reads and writes interior cells only; ghost entries of caller
 * buffers are never read and never written (boundary values are produced by
 * index remapping inside the kernels).
 *
 * Ownership.  The caller owns every buffer passed in.  The library owns its
 * scratch buffers (allocated by mfc_init, and on the first adjoint call for
 * the adjoint's extra scratch) and frees them in mfc_destroy.
 *
 * Execution.  Calls are asynchronous on the given CUDA stream
 * (a cudaStream_t passed as void*, NULL = legacy default stream) unless a
 * HOST output pointer is documented, in which case the call synchronises
 * that stream.  A context may be used by one stream at a time.
 *
 * Errors.  Every call returns an mfc_status.  Argument errors are detected
 * on the host before any launch (MFC_ERR_ARG).  Kernels that meet a
 * non-physical state (mixture density <= 0, or a squared sound speed <= 0 or
 * NaN) set a device flag; it is reported as MFC_ERR_NONPHYSICAL (and
 * cleared) by the next call that synchronises: mfc_compute_dt and
 * mfc_check.  mfc_last_error() describes the last failure.  No exception
 * crosses the ABI.
 */
#ifndef MFC_H
#define MFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MFC_OK = 0,
    MFC_ERR_ARG = -1,          /* invalid argument (checked on the host) */
    MFC_ERR_ALLOC = -2,        /* device allocation failed */
    MFC_ERR_CUDA = -3,         /* a CUDA runtime call or launch failed */
    MFC_ERR_NONPHYSICAL = -4,  /* rho <= 0 or c^2 <= 0 / NaN met on the device */
    MFC_ERR_UNSUPPORTED = -5   /* valid but not supported by this build */
} mfc_status;

/* Boundary conditions (Sec. 3.3): periodic wrap, transmissive (zeroth-order
 * extrapolation) and reflective (mirror with the normal momentum negated)
 * are applied by the library; their ghost cells in the caller's buffers are
 * neither read nor written.  MFC_BC_HALO is the side of a subdomain of a
 * domain decomposition (the paper's block decomposition with one halo
 * exchange per Runge-Kutta stage, Sec. 4.3): the ghost cells of that side
 * hold the neighbouring subdomain's cells, which the caller writes before
 * every evaluation of L (grid.ghost >= 3), and the library reads them as
 * cells.  A context with a halo side steps with mfc_rk3_stage, the caller
 * refreshing the halos of each stage's input; mfc_rk3_step, mfc_rk3_run,
 * mfc_rk3_step_batch_host, mfc_rk3_step_noalloc and the adjoints return
 * MFC_ERR_UNSUPPORTED for it, as does mfc_init with viscosity. */
typedef enum { MFC_BC_PERIODIC = 0, MFC_BC_TRANSMISSIVE = 1, MFC_BC_REFLECTIVE = 2, MFC_BC_HALO = 3 } mfc_bc;

/* MFC_FP64: everything in float64, every operation in the order of the
 *   defining formula with IEEE division and square root and no fused
 *   multiply-add, so results are reproducible bit for bit (and equal to a
 *   plain CPU evaluation of the same formulas).
 * MFC_FP64_FAST: float64 with the WENO weight divisions folded into one
 *   reciprocal per normalisation, other divisions as products with a
 *   reciprocal refined to a few ulps, and fused multiply-adds; agrees with
 *   MFC_FP64 to rounding.
 * MFC_MIXED: WENO5 reconstruction, HLLC and the per-direction flux
 *   differences (and their sum over directions) in float32; the
 *   cancelling part of the conservative-to-primitive conversion, the
 *   Runge-Kutta stage update and the CFL reduction in float64 (the CFL
 *   reduction with the MFC_FP64_FAST arithmetic).
 * MFC_DF64: MFC_FP64_FAST with the WENO5 reconstruction (smoothness
 *   indicators, weights, candidate values) in double-float arithmetic: pairs
 *   of float32 values with a 48-bit significand, evaluated on the float32
 *   pipes, which on GB300 run 64 times as many operations per clock as the
 *   float64 pipe.  Everything else (conservative-to-primitive conversion,
 *   HLLC, flux differences, stage update, CFL reduction) is the
 *   MFC_FP64_FAST float64 arithmetic.  The reconstruction is carried on
 *   the stencil's consecutive differences, so constant data reconstruct
 *   exactly.  Agrees with MFC_FP64 to rounding (the same 1e-11 bar as
 *   MFC_FP64_FAST).  Primitive values must keep the smoothness indicators
 *   inside the float32 range (differences across a stencil below ~1e18);
 *   an overflow is reported as MFC_ERR_NONPHYSICAL.  The adjoint entry
 *   points of an MFC_DF64 context recompute the RK stages with the
 *   double-float sweeps; their adjoint sweeps recompute the double-float
 *   face states and run the reverse of WENO5 in double-float arithmetic as
 *   well (JS and mapped weights; Z and TENO in the MFC_FP64_FAST
 *   arithmetic), the reverse of HLLC and of the pressure recovery in the
 *   MFC_FP64_FAST arithmetic. */
typedef enum { MFC_FP64 = 0, MFC_MIXED = 1, MFC_FP64_FAST = 2, MFC_DF64 = 3 } mfc_precision;

/* WENO weights: Jiang-Shu, mapped (Henrick; Sec. 3.2.1), Z with q = 1 (Sec. 4.2.2),
 * and fifth-order TENO (Sec. 4.2.2): the same three candidate stencils, each
 * switched off when its share chi_r = gamma_r / sum gamma of
 * gamma_r = d_r (1 + tau/(beta_r + eps))^6 is below the threshold C_T, the
 * others weighted by their ideal weights renormalised. */
typedef enum { MFC_WENO_JS = 0, MFC_WENO_M = 1, MFC_WENO_Z = 2, MFC_WENO_TENO = 3 } mfc_weno;

/* Uniform Cartesian grid.  n[d] interior cells on [lo[d], hi[d]] for
 * d < ndim (n[d] = 1 for d >= ndim).  ghost >= 0 is the padding of the
 * buffer layout on each active axis (MFC uses 3 for WENO5).  Periodic must
 * be set on both ends of an axis; periodic and reflective axes need n >= 3. */
typedef struct {
    int32_t ndim;          /* 1, 2 or 3 */
    int64_t n[3];
    double lo[3], hi[3];
    int32_t ghost;
    int32_t bc_lo[3], bc_hi[3];  /* mfc_bc */
} mfc_grid;

/* Stiffened-gas fluids (Sec. 2.2): gamma_i > 1, pi_inf_i >= 0.
 * eta_i >= 0: shear viscosity of fluid i.  When some eta_i > 0 the fluxes
 * carry the viscous stress of Sec. 2.1.1, T = 2 eta (D - tr(D) I/3) with
 * D = (grad u + (grad u)^T)/2 (momentum flux -T, energy flux -T.u), the
 * mixture viscosity being eta = sum_i alpha_i eta_i.  The stress is taken on
 * each face by second-order central differences of the cell velocities
 * (normal derivative across the face; tangential derivatives the mean of
 * the two cells' centred differences; face velocity and volume fractions
 * the means of the two cells').  The CFL dt is the convective one unless
 * opts.viscous_dt = 1, which adds the explicit viscous limit (the paper
 * states none; the usual bound of an explicit step of the momentum
 * diffusion): dt = CFL min over cells of min(min_d dx_d / (|u_d| + c),
 * rho min_d dx_d^2 / (2 ndim eta)), eta the cell's mixture viscosity
 * (cells with eta = 0 have no viscous bound).  Without it, the viscous limit
 * is the caller's to respect (pass dt > 0).  With viscosity the adjoints and mfc_rk3_step_noalloc
 * return MFC_ERR_UNSUPPORTED.  All eta_i = 0 is the inviscid method, bit
 * for bit. */
typedef struct {
    int32_t nfluids;       /* 1 .. 4 */
    double gamma[4];
    double pi_inf[4];
    double eta[4];
} mfc_eos;

/* Volume-fraction equation (Sec. 2.1.1): alpha_t + u . grad alpha = K div u.
 * MFC_MODEL_K0: K = 0 (the model of Allaire et al.); the sound speed is that
 *   of the mixture stiffened gas, c^2 = ((Gamma + 1) p + Pi)/(Gamma rho).
 * MFC_MODEL_KAPILA: two fluids; K = (Z_2 - Z_1)/(Z_1/alpha_1 + Z_2/alpha_2)
 *   with Z_i = gamma_i (p + pi_i) = rho_i c_i^2, evaluated per cell, and the
 *   Wood sound speed 1/(rho c^2) = alpha_1/Z_1 + alpha_2/Z_2 in the HLLC wave
 *   speeds and the CFL step.  States with p + pi_i <= 0 for either fluid are
 *   non-physical (first-order fallback at faces, MFC_ERR_NONPHYSICAL in cells). */
typedef enum { MFC_MODEL_K0 = 0, MFC_MODEL_KAPILA = 1 } mfc_model;

/* Approximate Riemann solver (Sec. 3.2.2).  HLLC: Toro's three-wave solver;
 * the face velocity of the alpha div u term is u_L / S* / S* / u_R.  HLL:
 * one averaged state between S_L and S_R, F = (S_R F_L - S_L F_R + S_L S_R
 * (U_R - U_L)) / (S_R - S_L), the volume fraction with U = alpha and
 * F = alpha u, and the face velocity the same average of u. */
typedef enum { MFC_RIEMANN_HLLC = 0, MFC_RIEMANN_HLL = 1 } mfc_riemann;

/* Low-Mach corrections (Sec. 4.2.4), with z = min(max(|u_L|/c_L, |u_R|/c_R), 1)
 * on the face-normal velocities.  THORNBER: the two normal velocities are
 * replaced by (u_L + u_R)/2 +- z (u_L - u_R)/2 before the solve (both solvers).
 * APC (HLLC only): (z - 1) p_d is added to the normal momentum flux and
 * (z - 1) p_d S* to the energy flux inside the fan, with
 * p_d = rho_L rho_R (S_L - u_L)(S_R - u_R)(u_R - u_L) / (rho_R (S_R - u_R) - rho_L (S_L - u_L)). */
typedef enum { MFC_LOW_MACH_NONE = 0, MFC_LOW_MACH_THORNBER = 1, MFC_LOW_MACH_APC = 2 } mfc_low_mach;

typedef struct {
    int32_t precision;     /* mfc_precision */
    int32_t weno;          /* mfc_weno */
    double weno_eps;       /* > 0: epsilon of the nonlinear weights (1e-40 for M and Z, 1e-6 for JS) */
    double cfl;            /* > 0: Courant number used when a step is asked for dt <= 0 */
    double teno_ct;        /* TENO threshold C_T in (0, 1) (MFC_WENO_TENO only; 1e-6 is customary) */
    int32_t model;         /* mfc_model */
    int32_t riemann;       /* mfc_riemann */
    int32_t low_mach;      /* mfc_low_mach */
    int32_t viscous_dt;    /* 1: the CFL dt also respects the explicit viscous limit (see mfc_eos); 0: convective only */
} mfc_opts;

typedef struct mfc_ctx mfc_ctx;

/* Validate the description, derive the constants and allocate the scratch
 * (three state-sized float64 buffers) on the current CUDA device.  An
 * MFC_DF64 context also creates a second CUDA stream, six events and three
 * edge-value buffers of 2 N_q (n_d + 2) x (lines per chunk) doubles (about
 * 0.2 of a state buffer each at 256^3): its sweeps run split into a
 * reconstruction kernel on that stream and a Riemann kernel on the caller's
 * stream, joined by events, so the calls stay ordered on the caller's stream
 * and can be captured in a CUDA graph.
 * *out receives the context (NULL on failure). */
mfc_status mfc_init(const mfc_grid* grid, const mfc_eos* eos, const mfc_opts* opts, mfc_ctx** out);

/* Free the context and its scratch (synchronises the device first).  NULL is a no-op. */
mfc_status mfc_destroy(mfc_ctx* ctx);

/* Doubles per field of a state-sized buffer (padded layout), or -1. */
int64_t mfc_field_stride(const mfc_ctx* ctx);

/* Number of fields N_q = 2 N_f + ndim, or -1. */
int32_t mfc_num_fields(const mfc_ctx* ctx);

/* Primitive (alpha_i rho_i, u_d, p, alpha_j) -> conservative state:
 * rho u = rho * u, rho E = Gamma p + Pi + 1/2 rho |u|^2 (Sec. 2.1.1, 2.2). */
mfc_status mfc_prim_to_cons(mfc_ctx* ctx, const double* w, double* q, void* stream);

/* Conservative -> primitive: p = (rho E - 1/2 rho |u|^2 - Pi)/Gamma. */
mfc_status mfc_cons_to_prim(mfc_ctx* ctx, const double* q, double* w, void* stream);

/* CFL time step of state q: CFL * min over cells and axes of
 * dx_d / (|u_d| + c), in the context's float64 arithmetic (MFC_FP64: the
 * formula as written, bit for bit).  dt_out is a HOST pointer; the call
 * synchronises the stream and returns MFC_ERR_NONPHYSICAL if the flag was
 * set. */
mfc_status mfc_compute_dt(mfc_ctx* ctx, const double* q, double* dt_out, void* stream);

/* rhs = L(q) on every interior cell (Eq. (rhs)). */
mfc_status mfc_rhs(mfc_ctx* ctx, const double* q, double* rhs, void* stream);

/* One TVD-RK3 step in place (Sec. 3.4):
 *   q1 = q + dt L(q); q2 = 3/4 q + 1/4 (q1 + dt L(q1));
 *   q <- 1/3 q + 2/3 (q2 + dt L(q2)).
 * dt > 0 is used as given; dt <= 0 asks for the CFL dt of q, computed on the
 * device without a host round trip.  dt_used (nullable) is a DEVICE pointer
 * to one double that receives the dt of this step. */
mfc_status mfc_rk3_step(mfc_ctx* ctx, double* q, double dt, double* dt_used, void* stream);

/* One stage of the TVD-RK3 step (Sec. 3.4) on caller buffers, for callers
 * that act between the stages (a domain decomposition refreshes the halo
 * cells of each stage's input, MFC_BC_HALO):
 *   stage 1: q_out = q_in + dt L(q_in)                       (q_n unused, may be NULL)
 *   stage 2: q_out = 3/4 q_n + 1/4 (q_in + dt L(q_in))
 *   stage 3: q_out = 1/3 q_n + 2/3 (q_in + dt L(q_in))
 * dt > 0 is the step's time step, the same for its three stages (for a
 * decomposed domain: the minimum over the subdomains of mfc_compute_dt).
 * The three stages in order, on q_in = q, q1, q2 with q_out = q1, q2, q and
 * q_n = q, give exactly mfc_rk3_step at that dt.  All pointers are DEVICE
 * buffers in the context's layout; q_out may alias q_n but not q_in.  Only
 * interior cells of q_out are written. */
mfc_status mfc_rk3_stage(mfc_ctx* ctx, int32_t stage, const double* q_in, const double* q_n, double* q_out,
                         double dt, void* stream);

/* nsteps RK3 steps in place, each with its own CFL dt (dt <= 0) or the
 * fixed dt.  dt_log (nullable) is a DEVICE array of nsteps doubles. */
mfc_status mfc_rk3_run(mfc_ctx* ctx, double* q, int32_t nsteps, double dt, double* dt_log, void* stream);

/* One mfc_rk3_step (Sec. 3.4) of each of `count` independent states held
 * in HOST memory, with the copies overlapped with the steps.  q_in[b] and
 * q_out[b] are host buffers of mfc_num_fields() x mfc_field_stride()
 * doubles in the layout above (ghost entries are copied through
 * unchanged); state b is read from q_in[b], stepped, and written to
 * q_out[b].  q_in and q_out are host arrays of count pointers.
 *
 * The context stages the states through two device states of its own
 * (allocated on the first call: twice the state size) on two copy streams
 * of its own: while state b is stepped on `stream`, state b+1 is uploaded
 * and state b-1 downloaded.  Uploads run in the order of b, downloads too.
 * So a host buffer may be read as several q_in[b] and written as several
 * q_out[b] (it ends holding the last), and q_out[b] may be q_in[b]; a
 * buffer written as q_out[b] must not be read as q_in[b'] for b' != b.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the
 * copies overlap the steps; pageable memory gives the same results with
 * the copies serialised.
 *
 * dt as for mfc_rk3_step, per state (dt <= 0: each state's own CFL dt).
 * dt_used (nullable) is a HOST array of count doubles.  The call returns
 * when every result is in host memory, with `stream` synchronised, and
 * reports a non-physical state as mfc_check does.  count == 0 does
 * nothing; a null array or element, count < 0 or a non-finite dt is
 * MFC_ERR_ARG before any copy. */
mfc_status mfc_rk3_step_batch_host(mfc_ctx* ctx, int32_t count, const double* const* q_in, double* const* q_out,
                                   double dt, double* dt_used, void* stream);

/* Adjoint of mfc_rhs: q_bar += (dL/dq)^T rhs_bar, interior cells.  rhs_bar
 * and q_bar are state-sized device buffers; q_bar must not alias q or
 * rhs_bar.  Non-smooth points (min/max of wave speeds, the HLLC side, |.|
 * of WENO-Z) take the derivative of the branch the forward pass takes. */
mfc_status mfc_rhs_vjp(mfc_ctx* ctx, const double* q, const double* rhs_bar, double* q_bar, void* stream);

/* Adjoint of one mfc_rk3_step at the fixed dt > 0:
 * qn_bar = (d q^{n+1} / d q^n)^T qnp1_bar (overwritten, interior cells).
 * Recomputes the two intermediate stages from q_n.  qn_bar may alias
 * qnp1_bar; neither may alias q_n. */
mfc_status mfc_rk3_step_vjp(mfc_ctx* ctx, const double* q_n, double dt, const double* qnp1_bar,
                            double* qn_bar, void* stream);

/* Allocation-free variant of mfc_rk3_step, for callers that cannot
 * allocate device memory: code that runs while another component owns the
 * device's memory budget, code that must not take the device-wide
 * synchronisation cudaMalloc and cudaFree imply, or a caller that keeps a
 * fixed footprint.  (The paper has no counterpart: it is a property of
 * this library, not of the method.)
 *
 * Same arguments and results as creating a context with grid / eos / opts
 * and calling mfc_rk3_step, without the context: the step's scratch (two
 * stage states, the right-hand side and the dt / flag scalars) is a
 * file-scope device array of MFC_NOALLOC_SCRATCH_DOUBLES doubles (64 MiB)
 * that every GPU loading the library holds until the process exits.  The
 * state may hold at most (MFC_NOALLOC_SCRATCH_DOUBLES - 32) / 3 doubles
 * (padded cells x fields); larger grids return MFC_ERR_ARG.  q and dt_used
 * are DEVICE pointers, as for mfc_rk3_step.
 *
 * No cudaMalloc, cudaFree or other allocating routine is called.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array, which keeps
 * the last call's contents: calls that overlap on the GPU (concurrent
 * streams, several host threads) race and must be serialised by the
 * caller.  A non-physical state met during the step (rho <= 0 or c^2 <= 0,
 * reported as MFC_ERR_NONPHYSICAL by the context calls) is reported here
 * through dt_used, which then holds NaN; with dt_used = NULL it is not
 * reported.  The cached address belongs to the device's current context: a
 * device reset (cudaDeviceReset) invalidates it, so this call must not be
 * used on a device after its reset.  Errors: mfc_last_error(NULL). */
#define MFC_NOALLOC_SCRATCH_DOUBLES 8388608
mfc_status mfc_rk3_step_noalloc(const mfc_grid* grid, const mfc_eos* eos, const mfc_opts* opts, double* q,
                                double dt, double* dt_used, void* stream);

/* Synchronise the stream; report (and clear) the non-physical-state flag. */
mfc_status mfc_check(mfc_ctx* ctx, void* stream);

/* Message of the last failure on this context ("" if none).  With a NULL
 * context: the last mfc_init failure of this thread. */
const char* mfc_last_error(const mfc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MFC_H */
