/*
 * nbp.h -- C ABI of the GB300 nested block preconditioned solver.
 *
 * Solves A x = b for the block tangent
 *
 *        A = [[A_sp + sum_k r_k a^k a^kT , B],
 *             [C                          , D]]
 *
 * of the P1-P1 VMS / generalized-alpha Navier-Stokes discretisation (paper
 * Sec. 2.5: definitions of A, B, C, D and of the resistance term
 * K = alpha_f gamma dt sum_k m^k a^k a^kT; Sec. 3: the block system) with an
 * outer flexible GMRES preconditioned by the Schur complement reduction
 * P_SCR (Sec. 3.1, Algorithm 3), whose Schur complement S = D - C A^{-1} B is
 * applied matrix-free (Algorithm 2) and preconditioned by AMG on
 * S_hat = D - C diag(A)^{-1} B (Sec. 3.1).
 *
 * Conventions for every entry point:
 *   - Unknowns are ordered x = [x_v (3N, node-interleaved u,v,w); x_p (N)].
 *   - Unless stated otherwise, vector arguments are DEVICE pointers owned by
 *     the caller, and all work is ordered on the stream given to nbp_create.
 *     Entry points return after the stream has been synchronised, except where
 *     stated.
 *   - Every entry point returns an nbp_status; on error nbp_last_error()
 *     gives a one-line message.  No entry point aborts the process.
 *   - The library owns the context and all device memory it allocates (with
 *     cudaMallocAsync on the context stream); nbp_destroy releases it.
 */
#ifndef NBP_H
#define NBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbp_ctx nbp_ctx;   /* opaque, library-owned */

typedef enum {
    NBP_OK = 0,
    NBP_ERR_INVALID = 1,      /* bad argument, malformed sparse structure, NaN input */
    NBP_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the call) */
    NBP_ERR_OOM = 3,          /* device allocation failed */
    NBP_NOT_CONVERGED = 4,    /* solve ended at n_max; x and info are still filled */
    NBP_ERR_BREAKDOWN = 5,    /* zero Givens denominator with a nonzero residual */
    NBP_ERR_NAN = 6,          /* NaN/Inf met in the iteration */
    NBP_ERR_TIMEOUT = 7,      /* a bounded device wait ran out */
    NBP_ERR_STATE = 8         /* call order violated (e.g. solve before setup) */
} nbp_status;

/* Inputs of nbp_create.  All arrays are DEVICE pointers owned by the caller;
 * they are read (copied) during nbp_create only.
 *   A: block CSR with 3x3 row-major blocks, N block rows (velocity nodes).
 *   B: block CSR with 3x1 blocks (velocity row dofs x pressure column), N block rows.
 *   C: block CSR with 1x3 blocks (pressure row x velocity column dofs), N rows.
 *   D: CSR, N x N.
 *   Column indices must be sorted and unique within each row; rowptr[0] = 0.
 *   Outlet k (0 <= k < n_out) is the sparse vector a^k over velocity dofs
 *   0..3N-1 with entries out_idx/out_val[out_ptr[k] .. out_ptr[k+1]-1]
 *   (indices unique within one outlet).  r[k] (host or device, see flag) is
 *   the coefficient r_k multiplying a^k a^kT in A, i.e. the paper's
 *   alpha_f gamma dt m^k (Sec. 2.5); out_ptr is a DEVICE array. */
typedef struct {
    int32_t n_nodes;
    const int32_t *a_rowptr, *a_col; const double *a_val;
    const int32_t *b_rowptr, *b_col; const double *b_val;
    const int32_t *c_rowptr, *c_col; const double *c_val;
    const int32_t *d_rowptr, *d_col; const double *d_val;
    int32_t n_out;
    const int32_t *out_ptr, *out_idx; const double *out_val;
    const double *r;          /* HOST array of n_out weights */
} nbp_system;

/* Solver settings (paper Sec. 3.1: delta^r, delta^r_A, delta^r_S, delta^r_I,
 * delta^a, m, m_A, m_S, n_max).  Defaults from nbp_default_options():
 * rtol 1e-8, rtol_A 1e-3, rtol_S 1e-2, rtol_I 1e-2, atol 1e-50,
 * m = m_A = m_S = nmax = nmax_A = nmax_S = 200, AMG P_A and P_S with a
 * K-cycle on the S_hat hierarchy, device-driven Krylov loops. */
typedef struct {
    double rtol, rtol_A, rtol_S, rtol_I, atol;
    int32_t m, m_A, m_S, nmax, nmax_A, nmax_S;
    int32_t precision;      /* 0 FP64 everywhere; 1 FP32 inner (values, vectors, basis);
                               2 BF16 inner matrix values with FP32 vectors/accumulation;
                               3 FP32 inner operators (A, B, C, D) and Krylov bases with
                               BF16 values in the two AMG hierarchies only (smoothers,
                               residuals and coarse levels of the preconditioners);
                               4 as 3, with A applied with BF16 values inside the inner
                               A-solves of Algorithm 2 (the S-apply's A^{-1}, tolerance
                               rtol_I; the rank-one term stays FP64 there too).
                               The outer FGMRES, Givens update, true residual and the
                               rank-one term stay FP64 in every mode.  Modes 2-4 need
                               nbp_setup run with one of modes 2-4 (all build every copy). */
    int32_t pc_A;           /* 0 AMG V-cycle, 1 point Jacobi diag(A)^{-1} */
    int32_t pc_S;           /* 0 AMG on S_hat, 1 none */
    int32_t variant;        /* 0 P_SCR (Algorithm 3); 1 upper block-triangular [[A,B],[0,S]];
                               2 SIMPLE (Sec. 3.2: S replaced by S_hat, diag(A)^{-1} B in the
                               upper factor, no inner solver) */
    int32_t amg_max_levels; /* default 5 */
    int32_t amg_coarse_max; /* default 300 block rows */
    int32_t cheb_degree;    /* default 2 */
    double theta;           /* aggregation strength threshold, default 0.0064 */
    int32_t amg_cycle;      /* 0 V-cycle on both hierarchies; 1 (default) K-cycle on the
                               coarse levels of AMG(S_hat); 2 K-cycle on both.  Takes
                               effect at nbp_setup. */
    int32_t amg_kdepth;     /* K-cycle on coarse levels 1..amg_kdepth (default 2), V-cycles
                               below */
    int32_t cheb_degree_S;  /* Chebyshev degree of the AMG(S_hat) smoother, default 1
                               (cheb_degree, default 2, is that of AMG(A)) */
    int32_t device_loop;    /* 1 (default): the whole nested solve is one CUDA graph whose
                               GMRES loops are graph WHILE nodes driven on the device (one
                               launch per solve, captured at the first solve and kept;
                               nbp_batch_solve then runs every instance in one launch);
                               0: the host drives the Krylov loops, reading one status per
                               iteration.  Needs m_A >= nmax_A and m_S >= nmax_S (inner
                               solves in one cycle) and variant 0 or 1; otherwise, or while
                               profiling, the host-driven loop runs.  Same kernels, same
                               arithmetic; the fused Gram-Schmidt kernel of the device loop
                               splits its sums over one fixed grid for every basis length, so
                               results differ from the host loop at rounding level. */
    int32_t cheb_degree_I;  /* Chebyshev degree of the AMG(A) cycle that preconditions the
                               inner A-solves of Algorithm 2 (the S-apply's A^{-1}, solved only
                               to rtol_I), default 1; cheb_degree (default 2) in the A-solves of
                               Algorithm 3 */
    int32_t gs_passes_I;    /* Gram-Schmidt passes per Arnoldi step in those inner A-solves:
                               1 (default, classical Gram-Schmidt) or 2 (CGS2, as in every
                               other solve) */
} nbp_options;

typedef struct {
    int32_t outer_iters;
    int64_t A_iters, S_iters, I_iters;          /* intermediate A, S, inner A iterations */
    int64_t n_A_solves, n_I_solves, n_S_solves;
    double rel_res_est, rel_res_true;           /* outer estimate and FP64 true residual */
    double setup_s, solve_s;                    /* wall seconds of the last setup / solve */
    int32_t status;
} nbp_info;

void nbp_default_options(nbp_options *opt);

/* Copies the system to device memory owned by the context; validates the
 * sparse structure on the device (monotone row pointers, column indices in
 * range and sorted, finite values).  `stream` is a cudaStream_t (NULL for the
 * legacy default stream).  The current CUDA device at this call is used for
 * the life of the context.  Errors: NBP_ERR_INVALID, NBP_ERR_CUDA, NBP_ERR_OOM. */
nbp_status nbp_create(nbp_ctx **ctx, const nbp_system *sys, const nbp_options *opt, void *stream);

/* Builds, on the device: the aggregation AMG hierarchy of A_sp, S_hat =
 * D - C diag(A)^{-1} B (diag(A) includes the rank-one terms), the AMG
 * hierarchy of S_hat, and the FP32/BF16 value copies the precision mode
 * needs.  Time is reported in info.setup_s of the next solve. */
nbp_status nbp_setup(nbp_ctx *ctx);

/* Numeric re-setup after new values on the same patterns (nbp_set_values,
 * nbp_set_resistances; the Newton tangents of a time step, Sec. 2.5): both
 * AMG hierarchies, S_hat and the value copies are rebuilt from the current
 * values on the aggregate maps of the last nbp_setup -- Galerkin operators,
 * block-diagonal inverses, Chebyshev bounds and coarsest inverses all new,
 * only the aggregation (the most expensive part of the setup) is kept, and
 * with it the number of levels.  The options' theta and level limits are
 * those of that nbp_setup.  Errors: NBP_ERR_STATE (no earlier nbp_setup),
 * NBP_ERR_INVALID (a singular diagonal block), NBP_ERR_CUDA, NBP_ERR_OOM. */
nbp_status nbp_setup_numeric(nbp_ctx *ctx);

/* Replaces the n_out weights r_k (HOST array).  S_hat depends on them through
 * diag(A); call nbp_setup again before solving if P_S should track them. */
nbp_status nbp_set_resistances(nbp_ctx *ctx, const double *r);

/* Nested solve (paper Sec. 3): outer FGMRES(m) preconditioned by P_SCR
 * (Algorithm 3) to ||b - A x|| <= max(rtol ||b||, atol), x_0 = 0.  b, x:
 * DEVICE arrays of 4N doubles.  `opt` may be NULL (context options).  The
 * true residual is recomputed in FP64 before returning.  Returns NBP_OK,
 * NBP_NOT_CONVERGED (x filled), or an error. */
nbp_status nbp_solve(nbp_ctx *ctx, const double *b, double *x, const nbp_options *opt, nbp_info *info);

/* Same as nbp_solve with HOST b and x (copied in and out on the context
 * stream inside the call). */
nbp_status nbp_solve_host(nbp_ctx *ctx, const double *b_host, double *x_host, const nbp_options *opt,
                          nbp_info *info);

/* Adjoint of the nested solve: lambda = A^{-T} g by the same nested method on
 * the transposed tangent [[A^T, C^T], [B^T, D^T]] (whose Schur complement is
 * S^T, so Algorithms 2 and 3 apply unchanged), then dL/db = lambda and
 * dL/dr_k = -(lambda_v . a^k)(a^k . x_v) because dA/dr_k = a^k a^kT (Sec. 2.5).
 * g, x, lambda: DEVICE arrays of 4N doubles; dL_dr: HOST array of n_out.
 * The transposed hierarchy is built on the first call (and after setup). */
nbp_status nbp_adjoint(nbp_ctx *ctx, const double *g, const double *x, double *lambda, double *dL_dr,
                       nbp_info *info);

nbp_status nbp_destroy(nbp_ctx *ctx);
const char *nbp_last_error(const nbp_ctx *ctx);

/* ---- steps of the method, exposed for parity tests and benchmarks ---- */

/* y = A x = A_sp x + sum_k r_k a^k (a^kT x) (Sec. 2.5).  x, y: DEVICE, 3N
 * doubles.  precision 0 uses FP64 values; 1/2 use the FP32/BF16 value copies
 * made by nbp_setup with FP32 vectors (x, y are then float*). */
nbp_status nbp_apply_A(nbp_ctx *ctx, const void *x, void *y, int32_t precision);

/* y = [[A, B], [C, D]] x in FP64 (the outer operator of Sec. 3). */
nbp_status nbp_apply_full(nbp_ctx *ctx, const double *x, double *y);

/* Algorithm 2: y = D x_p - C A^{-1} B x_p with the inner GMRES(m_A) + P_A to
 * rtol_I.  x_p, y: DEVICE, N doubles.  Needs nbp_setup. */
nbp_status nbp_apply_S(nbp_ctx *ctx, const double *xp, double *y);

/* Algorithm 3: y = P_SCR^{-1} s.  s, y: DEVICE, 4N doubles.  Needs nbp_setup. */
nbp_status nbp_apply_pscr(nbp_ctx *ctx, const double *s, double *y);

/* GMRES(m_A) + P_A on A y = s to relative tolerance rtol (Sec. 3.1).
 * s, y: DEVICE, 3N doubles.  *iters receives the iteration count. */
nbp_status nbp_solve_A(nbp_ctx *ctx, const double *s, double *y, double rtol, int32_t *iters);

/* One AMG V(1,1)-cycle, x = M^{-1} b, on the hierarchy of A_sp (which = 0,
 * 3N doubles) or of S_hat (which = 1, N doubles).  DEVICE arrays. */
nbp_status nbp_vcycle(nbp_ctx *ctx, int32_t which, const double *b, double *x);

/* Hierarchy introspection (after nbp_setup).  nbp_amg_level_sizes returns the
 * number of levels; rows/nnz (HOST arrays of length >= levels) get the block
 * rows and stored blocks of each level.  nbp_amg_level_get copies level l to
 * HOST arrays: rowptr (rows+1), col (nnz), val (nnz*bs*bs doubles), the
 * aggregate map to level l+1 (rows; -1 = left out) and rho, the upper end of
 * the level's Chebyshev interval (AMG(A): min of the Gershgorin bound of
 * D_b^{-1} A and 1.1 x the spectral radius of a 20-step Arnoldi Hessenberg
 * matrix; AMG(S_hat): the Gershgorin bound), any of which may be NULL. */
int32_t nbp_amg_level_sizes(nbp_ctx *ctx, int32_t which, int32_t *rows, int64_t *nnz, int32_t max_levels);
nbp_status nbp_amg_level_get(nbp_ctx *ctx, int32_t which, int32_t l, int32_t *rowptr, int32_t *col, double *val,
                             int32_t *agg, double *rho);

/* S_hat after nbp_setup: nnz, then its CSR copied to HOST arrays. */
int64_t nbp_shat_nnz(nbp_ctx *ctx);
nbp_status nbp_shat_get(nbp_ctx *ctx, int32_t *rowptr, int32_t *col, double *val);

/* Per-kernel device-time accounting of the last solve: total milliseconds and
 * algorithmic bytes of the SpMV family and of the Arnoldi (CGS2) kernels,
 * measured with CUDA events on the context stream when `enable` was set by
 * nbp_profile(ctx, 1) before the solve. */
typedef struct {
    double spmv_ms, spmv_bytes, arnoldi_ms, arnoldi_bytes;
    double a0_ms, a0_bytes;     /* the fine-level A product (A_sp + rank-one) alone */
    double cheb0_ms, cheb0_bytes; /* fine-level Chebyshev steps of the AMG(A) cycle */
    double vcycle_ms;
    int64_t spmv_launches, arnoldi_launches, a0_launches, cheb0_launches;
    int64_t kernel_launches;    /* every kernel this library launched in the last call */
    double host_wait_s;         /* host time blocked in per-iteration status reads */
    int64_t host_syncs;         /* number of those reads */
} nbp_profile_info;
nbp_status nbp_profile(nbp_ctx *ctx, int32_t enable);
nbp_status nbp_profile_get(nbp_ctx *ctx, nbp_profile_info *out);
/* Per-kernel breakdown of the last profiled call as a JSON object
 * {"tag": [launches, total ms, algorithmic bytes]}; tags name the matrix
 * (A, B, C, D, HA<level>, HS<level>), the epilogue and the kernel chosen.  The
 * string is owned by the context and valid until its next profiled call. */
const char *nbp_profile_report(const nbp_ctx *ctx);

/* ---- batched solves (many independent tangents of uneven size) ----
 * One context and one CUDA stream per instance; nbp_batch_setup and
 * nbp_batch_solve drive the instances from a pool of host threads so that
 * their kernels overlap on the GPU.  With opt->device_loop = 1 the solve is
 * one CUDA graph holding every instance's device-driven nested solve as a
 * parallel branch, captured once and launched once per call.  systems: HOST array of `count` nbp_system
 * (each with its own DEVICE arrays, copied during the call).  b, x: HOST arrays
 * of `count` DEVICE pointers (4 N_i doubles each); infos: HOST array of
 * `count` (may be NULL).  Returns NBP_OK when every instance converged, else
 * the first error (nbp_batch_last_error names the instance) or
 * NBP_NOT_CONVERGED.  Each solve is the nested method of nbp_solve. */
typedef struct nbp_batch nbp_batch;
nbp_status nbp_batch_create(nbp_batch **batch, int32_t count, const nbp_system *systems, const nbp_options *opt);
nbp_status nbp_batch_setup(nbp_batch *batch);
nbp_status nbp_batch_solve(nbp_batch *batch, const double *const *b, double *const *x, const nbp_options *opt,
                           nbp_info *infos);
int32_t nbp_batch_size(const nbp_batch *batch);
nbp_status nbp_batch_destroy(nbp_batch *batch);
const char *nbp_batch_last_error(const nbp_batch *batch);

/* ---- allocation-free variant (no counterpart in the paper) ----
 * y = A x = A_sp x + sum_k r_k a^k (a^kT x) like nbp_apply_A (precision 0),
 * but without a context and without allocating any memory, for callers that
 * cannot call cudaMalloc: code running after a framework has frozen its
 * memory pool, real-time or embedded callers that forbid allocation once they
 * are running, and callers that hold no library context.  The per-outlet inner
 * products live in a fixed device array inside the library (8 KiB on every
 * GPU that loads it, held until the process exits), so n_out is limited to
 * 1024; larger n_out, negative sizes or null pointers return NBP_ERR_INVALID
 * before anything is launched.  The call allocates nothing and frees nothing.
 * Arrays (all DEVICE, caller-owned): A in block CSR with 3x3 row-major blocks
 * (N = n_nodes block rows, sorted in-range columns: they are not validated
 * here), outlet k as out_idx/out_val[out_ptr[k] .. out_ptr[k+1]-1] over
 * velocity dofs with indices unique within one outlet, r (n_out weights), x
 * and y (3N doubles).  Work is queued on `stream` and the call returns
 * without synchronising; NBP_ERR_CUDA reports a failed launch.  Every call
 * looks up the device address of the fixed array on the current device (no
 * address is cached, so a device reset between calls is safe); the first
 * call on a device also sets up the library's device code there, so make
 * that first call before any stream capture.  A call launches three kernels
 * whatever n_out (one kernel adds every outlet's terms, in ascending k).
 * Every call shares the array: each call overwrites the entries it uses
 * before reading them, and calls that overlap on the GPU (on unordered
 * streams) race on it. */
nbp_status nbp_apply_A_noalloc(int32_t n_nodes, const int32_t *a_rowptr, const int32_t *a_col, const double *a_val,
                               int32_t n_out, const int32_t *out_ptr, const int32_t *out_idx, const double *out_val,
                               const double *r, const double *x, double *y, void *stream);

/* ------------------------------------------------------------ RCR outlets
 * Three-element Windkessel (RCR) outlet model, paper Sec. 2.1 (RCR circuit
 * equations): dPi^k/dt = -Pi^k / (R_d^k C^k) + Q^k / C^k and
 * P^k = R_p^k Q^k + Pi^k + P_d^k, with Pi^k the pressure drop across the
 * distal resistor and Q^k the flow through outlet k.  Parameters and the
 * state at t_n of n_out outlets, each a DEVICE array of n_out doubles owned
 * by the caller (read during the call only). */
typedef struct {
    const double *Rp, *C, *Rd;  /* proximal resistance, compliance, distal resistance (> 0) */
    const double *Pd;           /* distal reference pressure P_d at t_{n+1} */
    const double *Pi_n, *Q_n;   /* Pi and Q at t_n */
    double eps_abs, eps_rel;    /* difference step eps = max(eps_abs, eps_rel |Q_{n+1}|) for m^k;
                                   Sec. 2.5 fixes 1e-8 and 1e-5 (non-negative, not both zero) */
} nbp_rcr;

/* One time step of n_out RCR outlets (Algorithm 1): Pi from t_n to
 * t_{n+1} = t_n + dt in nts equal substeps of the four-stage Runge-Kutta
 * scheme, with Q linear in time from Q_n to Q_np1; P_np1 = R_p Q_np1 +
 * Pi_{n+1} + P_d.  m^k = dP_{n+1}/dQ_{n+1} by the central difference
 * quotient of Sec. 2.5 (two more steps at Q_np1 +- eps/2).  Q_np1: DEVICE
 * array of n_out flows; outputs P_np1, Pi_np1, m: DEVICE arrays of n_out
 * doubles, each may be NULL.  One thread per outlet, queued on `stream`
 * (NULL: legacy default stream); returns without synchronising.  Errors:
 * NBP_ERR_INVALID (n_out < 0, nts < 1, dt <= 0, a missing parameter
 * array), NBP_ERR_CUDA (launch).  Explicit RK4 needs dt / nts below about
 * 2.8 R_d C for stability; the caller picks nts. */
nbp_status nbp_rcr_step(int32_t n_out, const nbp_rcr *p, const double *Q_np1, double dt, int32_t nts,
                        double *P_np1, double *Pi_np1, double *m, void *stream);

/* Flow rates through the context's outlets, Q^k = a^k . v (Sec. 2.5: Q^k is
 * the integral of v . n over outlet k and a^k_{Ai} the integral of N_A n_i,
 * the outlet vectors given to nbp_create).  v: DEVICE array of the 3N
 * velocity dofs; Q: DEVICE array of n_out doubles.  Fixed-order
 * reductions (bitwise repeatable).  Synchronises the context stream.
 * Errors: NBP_ERR_INVALID (null pointer), NBP_ERR_CUDA. */
nbp_status nbp_outlet_flows(nbp_ctx *ctx, const double *v, double *Q);

/* The outlet coupling of one Newton iteration (Sec. 2.5): Q_{n+1}^k =
 * a^k . v_np1, the RCR step and m^k as in nbp_rcr_step, and the context's
 * rank-one weights set to r_k = scale m^k (scale = alpha_f gamma dt gives
 * the matrix K of Sec. 2.5), all on the device: Q and m make no host round
 * trip before the weights are in place.  p describes the context's n_out
 * outlets in order.  Outputs (DEVICE, n_out doubles each, may be NULL):
 * Q_np1, P_np1, Pi_np1, m.  Like nbp_set_resistances, S_hat keeps the
 * weights of the last nbp_setup (call it again if P_S should track them).
 * Synchronises the context stream.  Errors: NBP_ERR_INVALID, NBP_ERR_NAN
 * (a non-finite m^k; the weights are then left unchanged), NBP_ERR_CUDA. */
nbp_status nbp_rcr_update(nbp_ctx *ctx, const nbp_rcr *p, const double *v_np1, double dt, int32_t nts, double scale,
                          double *Q_np1, double *P_np1, double *Pi_np1, double *m);

/* --------------------------------------------- tangent values in place
 * Replaces the values of A, B, C, D (DEVICE arrays in the layout and on the
 * pattern given to nbp_create: 9, 3, 3, 1 values per entry), e.g. with the
 * tangent of a new Newton iteration.  Copies them, drops every copy built
 * from the old values (precision copies, sliced-ELL layouts, AMG, S_hat, the
 * transposed context of the adjoint): call nbp_setup again before solving.
 * No paper counterpart as an entry point (the tangent is reassembled every
 * iteration in Sec. 2.5, step 8).  Errors: NBP_ERR_INVALID (null array, a
 * non-finite value: nothing is replaced), NBP_ERR_CUDA. */
nbp_status nbp_set_values(nbp_ctx *ctx, const double *a_val, const double *b_val, const double *c_val,
                          const double *d_val);

/* ------------------------------------ VMS residual, tangent, Newton step
 * On-device assembly for the P1-P1 residual-based VMS formulation with
 * generalized-alpha time stepping (paper Sec. 2.3-2.5):
 *   residual  R_m = R_m^vol + R_m^bc + R_m^bf and R_p (Sec. 2.3, B_m^vol,
 *             B_m^bc, B_m^bf, B_p), fine scales v', p' and tau_M, tau_C, G
 *             as defined there; the outlet traction is R_m^bc = sum_k P_k a^k
 *             with the context's outlet vectors a^k;
 *   tangent   A = F (+ K, kept as the context's rank-one term), B, C, D of
 *             Sec. 2.5: the exact derivative of the residual with respect to
 *             (vdot_{n+1}, pdot_{n+1}), with tau_M and tau_C held fixed.
 * Readings: P1 elements (the viscous second derivatives in v' vanish), no
 * body force, degree-2 4-point rule on tets and the 3-point rule at the
 * barycentric points (2/3, 1/6, 1/6) on outlet triangles; a Dirichlet node
 * prescribes all three velocity components: its momentum residual rows are
 * zero, its tangent rows and columns in A keep the diagonal entry only, its
 * B rows and C columns are zero, and Newton increments leave it unchanged.
 * Unknowns as in nbp_solve: x = [v (3N, node-interleaved); p (N)]. */
typedef struct nbp_vms nbp_vms;

typedef struct {
    int32_t n_nodes;          /* must equal the context's N */
    int32_t n_tets, n_tris;
    const double *X;          /* HOST, 3N node coordinates */
    const int32_t *tets;      /* HOST, 4 node ids per tet (any vertex order) */
    const int32_t *tris;      /* HOST, 3 node ids per Neumann (outlet) triangle, ordered so that
                                 (x1 - x0) x (x2 - x0) points out of the domain */
    const uint8_t *dir;       /* HOST, N flags: 1 = velocity prescribed (Dirichlet) */
} nbp_mesh;

typedef struct {
    double rho, mu;           /* density, dynamic viscosity */
    double dt;                /* time step Delta t_n */
    double rho_inf;           /* generalized-alpha spectral radius (Sec. 2.4.1), in [0, 1] */
    double beta;              /* backflow coefficient (0.2 in Sec. 2.3) */
    double CI, CT;            /* 36 and 4 for linear tets (Sec. 2.3) */
    int32_t tangent_fp32;     /* 1: tangent arithmetic in FP32 (written as FP64 values); 0: FP64 */
} nbp_vms_params;

/* Binds a mesh to a context (its pattern must contain every pair of nodes
 * sharing a tet or an outlet triangle; A, B, C, D share one pattern).  Host
 * arrays are copied; the gather maps (node -> incident elements, pattern
 * slot -> element blocks, ascending element order) are built on the host
 * once.  The handle uses the context's stream and must be destroyed before
 * the context.  Errors: NBP_ERR_INVALID (sizes, node ids, parameters, a pair
 * absent from the pattern, a degenerate element: |det| of a tet at most 1e-12
 * of its longest edge cubed, twice the area of a triangle at most 1e-12 of
 * its longest edge squared), NBP_ERR_OOM, NBP_ERR_CUDA. */
nbp_status nbp_vms_create(nbp_vms **vms, nbp_ctx *ctx, const nbp_mesh *mesh, const nbp_vms_params *par);

/* The host step of nbp_vms_create, on HOST arrays and without any device
 * work: for n_el elements of w = 4 (tets) or 3 (triangles) nodes each (el),
 * inc_ptr (n_nodes + 1) / inc (w n_el) list for every node the entries
 * w e + a of the elements e having it as local node a, ascending e; and
 * slot_ptr (nnz + 1) / slot_src (w^2 n_el) list for every pattern slot
 * (row A, column B of rowptr/col) the entries w^2 e + w a + b with
 * el[e][a] = A and el[e][b] = B, ascending e.  No paper counterpart (the
 * deterministic assembly order).  Errors: NBP_ERR_INVALID (bad arguments, a
 * node id out of range, a pair absent from the pattern), NBP_ERR_OOM. */
nbp_status nbp_vms_maps(int32_t n_nodes, const int32_t *rowptr, const int32_t *col, int32_t n_el, int32_t w,
                        const int32_t *el, int32_t *inc_ptr, int32_t *inc, int32_t *slot_ptr, int32_t *slot_src);
nbp_status nbp_vms_destroy(nbp_vms *vms);

/* R (DEVICE, 4N) at vd = vdot_{n+alpha_m} (3N), v = v_{n+alpha_f} (3N),
 * p = p_{n+alpha_f} (N), outlet pressures P (DEVICE, n_out; may be NULL
 * without outlets), tau evaluated at vtau (DEVICE 3N, NULL: v).  Every row is
 * a fixed-order sum (bitwise repeatable).  Synchronises the context stream.
 * Errors: NBP_ERR_INVALID, NBP_ERR_CUDA. */
nbp_status nbp_vms_residual(nbp_vms *vms, const double *vd, const double *v, const double *p, const double *vtau,
                            const double *P, double *R);

/* Tangent values on the context's pattern (DEVICE a_val 9 nnz, b_val 3 nnz,
 * c_val 3 nnz, d_val nnz) at the same state as nbp_vms_residual.  Does not
 * touch the context (see nbp_set_values).  Synchronises the context stream.
 * Errors: NBP_ERR_INVALID, NBP_ERR_CUDA. */
nbp_status nbp_vms_tangent(nbp_vms *vms, const double *vd, const double *v, const double *p, const double *vtau,
                           double *a_val, double *b_val, double *c_val, double *d_val);

typedef struct {
    double tol_R, tol_A;      /* stopping rule ||R_(l)|| / ||R_(0)|| <= tol_R or ||R_(l)|| <= tol_A (1e-6 in Sec. 2.5) */
    int32_t l_max;            /* corrector iterations (20 in Sec. 2.5) */
    int32_t nts;              /* RK4 substeps of the outlet model per time step */
    int32_t pc_rebuild;       /* preconditioner of the nested solves (AMG(A), S_hat, AMG(S_hat)):
                                 0 built from every tangent; 1 from the first tangent of this
                                 step only; 2 the one the context holds (from nbp_setup or an
                                 earlier step) is kept, one is built only if there is none;
                                 3 rebuilt from every tangent by nbp_setup_numeric (new values
                                 on the held aggregates); 4 the same from the first tangent of
                                 this step only.  Modes 2-4 build one in full when the context
                                 holds none.  A kept preconditioner acts on the new tangent's
                                 operators (their sliced and precision copies are refreshed): a
                                 lagged preconditioner changes the path of each solve, not its
                                 solution.  A caller rebuilding every k steps passes 1 (or 4) on
                                 those steps and 2 on the others. */
} nbp_newton_opts;

typedef struct {
    int32_t iters;            /* tangent solves made */
    int32_t converged;        /* the stopping rule was met */
    int32_t unconverged_solves; /* nested solves that stopped at their iteration limit */
    double res0, res;         /* ||R_(0)|| (at the predictor) and the last ||R|| */
    int64_t outer_iters, A_iters, S_iters, I_iters;   /* summed over the solves */
    double residual_s, tangent_s, setup_s, solve_s, total_s;   /* wall seconds per phase */
    int32_t setups;           /* full preconditioner builds made in this step */
    int32_t numeric_setups;   /* numeric re-setups (pc_rebuild 3, 4) made in this step */
} nbp_newton_info;

/* One time step by the predictor multi-corrector of Sec. 2.5: predictor
 * y = y_n, ydot = (gamma - 1) / gamma ydot_n; then per corrector l: outlet
 * flows Q^k = a^k . v, the RCR step and m^k (Algorithm 1 and the difference
 * quotient, as nbp_rcr_step; rcr->Q_n is ignored: Q_n is computed from y_n),
 * the alpha stages, the residual with P_{n+alpha_f} = (1 - alpha_f) P_n +
 * alpha_f P_{n+1} (P_n = R_p Q_n + Pi_n + P_d), the stopping rule, the
 * tangent installed in the context with r_k = alpha_f gamma dt m^k, a new
 * nbp_setup, the nested solve of [[A, B], [C, D]] dydot = -R with the
 * context's options, and ydot += dydot, y += gamma dt dydot.  ||R_(0)|| is
 * the residual at the predictor (reading).  y_n, yd_n: DEVICE 4N inputs;
 * y, yd: DEVICE 4N outputs (distinct from the inputs); Pi_np1: DEVICE n_out
 * (may be NULL): Pi^k at t_{n+1} from the accepted state.  rcr: the outlet
 * parameters (DEVICE arrays, as nbp_rcr_step; may be NULL without outlets).
 * The context's values and weights are left at the last tangent.  Returns
 * NBP_OK when the stopping rule is met, NBP_NOT_CONVERGED after l_max
 * corrector solves (y, yd hold the last iterate).  Errors: NBP_ERR_INVALID,
 * NBP_ERR_NAN (non-finite residual or m^k), the nested solve's errors,
 * NBP_ERR_CUDA. */
nbp_status nbp_newton_step(nbp_vms *vms, const nbp_rcr *rcr, const double *y_n, const double *yd_n, double *y,
                           double *yd, double *Pi_np1, const nbp_newton_opts *opts, nbp_newton_info *info);

#ifdef __cplusplus
}
#endif
#endif /* NBP_H */
