/*
 * bri.h -- C ABI of the GB300 (sm_103a) Brillouin-kernel overlap library.
 *
 * Operator definitions follow Duerr & Koutsou, "On the suitability of the
 * Brillouin action as a kernel to the overlap procedure", arXiv:1701.00726:
 *
 *   D_bri = sum_mu gamma_mu nabla^iso_mu - (1/2) Delta^bri + m0
 *           - (c_SW/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}          (Eq. def_bril)
 *   D_wil = sum_mu gamma_mu nabla^std_mu - (1/2) Delta^std + m0 - clover
 *                                                                   (Eq. def_wils)
 *   D_ov  = rho [1 + gamma5 f_nn(H)],  H = gamma5 D_K(m0 = -rho)    (Eq. def_over)
 *           with the kernel D_K = D_bri (default) or D_wil (bri_set_kernel)
 *   f_nn(x) = x [c0 + sum_i w_i / (x^2 + sigma_i)]                  (Eq. KLnn_parfrac)
 *
 * with a = 1.  Conventions shared by every call:
 *
 *   dims[4]   = {Lx, Ly, Lz, Lt}; site n = x + Lx*(y + Ly*(z + Lz*t)); V = Lx*Ly*Lz*Lt.
 *   gauge U   = [V][mu=0..3 (x,y,z,t)][3][3] complex128 (re, im interleaved),
 *               device memory; U_mu(n) transports from n+mu to n.
 *   spinors   = [rhs][V][spin 4][colour 3] complex, interleaved (re, im), device
 *               memory, complex128 when the precision is BRI_PREC_F64 (or
 *               BRI_PREC_DW) and complex64 (float) for BRI_PREC_F32 /
 *               BRI_PREC_F32_BF16.
 *   gamma basis: chiral, gamma_k = [[0,-i s_k],[i s_k,0]], gamma_4 = [[0,1],[1,0]],
 *               gamma5 = diag(1,1,-1,-1) (App. C counts gamma products as free
 *               permutations in this basis).
 *   offsets   : the 81 hypercube offsets d in {-1,0,1}^4 are numbered
 *               nu-1 = (d_x+1) + 3(d_y+1) + 9(d_z+1) + 27(d_t+1); nu and 82-nu
 *               are opposite and only nu = 1..40 are stored (App. C).
 *
 * Ownership: every array argument is caller-owned; the library never frees
 * or retains caller memory.  The context owns the off-axis links, the clover
 * field and solver workspaces.  All device work is issued on the context's
 * stream; calls return once the work is enqueued unless documented otherwise
 * (solvers synchronise the stream to test convergence).
 *
 * Errors: functions return BRI_OK (0), BRI_NOT_CONVERGED (1, output written)
 * or a negative code; bri_last_error() gives a thread-local message.
 */
#ifndef BRI_H
#define BRI_H

#ifdef __cplusplus
extern "C" {
#endif

#define BRI_OK 0
#define BRI_NOT_CONVERGED 1
#define BRI_ERR_INVALID (-1)   /* bad argument (size, pointer, precision, order) */
#define BRI_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define BRI_ERR_OOM (-3)       /* device allocation failed */
#define BRI_ERR_NOLINKS (-4)   /* bri_build_links has not been called */
#define BRI_ERR_NONFINITE (-5) /* a solver met a NaN/Inf in a reduction */

/* Operator precision (spinor storage / link storage / accumulation). */
#define BRI_PREC_F64 0       /* complex128 spinors, FP64 links, FP64 arithmetic */
#define BRI_PREC_F32 1       /* complex64 spinors, FP32 links, FP32 accumulation */
#define BRI_PREC_F32_BF16 2  /* complex64 spinors, BF16-stored links, FP32 accumulation */
#define BRI_PREC_DW 3        /* bri_apply only: complex128 spinors in and out, the FP64 links and clover
                                split into double-word FP32 pairs, double-word FP32 arithmetic
                                (error-free transformations: ~48-bit significands on the FP32 pipe) */

/* bri_create flags */
#define BRI_ANTIPERIODIC_T 1 /* antiperiodic time direction (sign of U_t on the last slice) */

/* Kernel operator of the overlap solvers (bri_set_kernel) */
#define BRI_KERNEL_BRILLOUIN 0 /* D_bri, Eq. def_bril (the default) */
#define BRI_KERNEL_WILSON 1    /* D_wil, Eq. def_wils */

/* Kenney-Laub family for kl_coeffs / solvers */
#define BRI_KL_DIAGONAL 0 /* f_nn = g_{2n+1}: constant term + n shifts (Tab. 5) */
#define BRI_KL_UPPER 1    /* f_{n-1,n} = g_{2n}: n shifts, no constant (Tab. 6) */

#define BRI_MAX_SHIFTS 32

typedef struct bri_ctx bri_ctx;

/* Solver statistics (per call; per-rhs entries for rhs < 64). */
typedef struct bri_stats {
  int iterations;          /* multi-shift CG iterations (max over rhs) */
  int matvecs;             /* applications of the kernel operator D or D^dagger */
  int matvecs_f64;         /* of which in FP64 (double-word FP32 applications count in
                              matvecs only) */
  int refinements;         /* mixed precision: outer refinement rounds */
  int n_shifts;            /* number of shifts solved */
  double max_true_residual;/* max over rhs and shifts of ||b-(A+s_i)x_i||/||b|| (FP64),
                              filled when want_true_residual != 0 */
  double shift_residual[BRI_MAX_SHIFTS]; /* per shift, max over rhs */
  int want_true_residual;  /* input: compute FP64 true residuals per shift */
  int maxiter;             /* input: iteration cap (0 = default 20000) */
  double seconds;          /* wall time of the call */
  double phase_seconds[4]; /* main multi-shift solve, FP64-class residuals, corrections, final D */
} bri_stats;

/* Create a context for one lattice.  dims: {Lx,Ly,Lz,Lt}, each >= 2.
 * flags: BRI_ANTIPERIODIC_T or 0.  stream: a cudaStream_t (NULL = legacy
 * default stream).  Allocates nothing large until bri_build_links. */
int bri_create(bri_ctx** ctx, const int dims[4], int flags, void* stream);
void bri_destroy(bri_ctx* ctx);
int bri_set_stream(bri_ctx* ctx, void* stream);

/* Select the kernel operator D_K of the overlap solvers of this context
 * (sign_apply_multishift, overlap_apply, overlap_apply_batch, overlap_solve,
 * overlap_grad, sign_apply_multishift_noalloc): BRI_KERNEL_BRILLOUIN (default)
 * or BRI_KERNEL_WILSON.  The paper compares both kernels inside the overlap
 * (Eqs. def_wils, def_bril inside Eq. def_over; Secs. 5-8).  Both use the same
 * clover coefficient and, for the Wilson kernel, the thin links. */
int bri_set_kernel(bri_ctx* ctx, int kernel);

/* Build the 40 stored path-averaged off-axis links W_nu(n), nu = 1..40
 * (App. C: the average over the k! shortest paths of the link products, no
 * SU(3) back-projection) in FP64, FP32 and BF16 storage, the thin-link copy
 * used by wils_apply and, when c_sw != 0, the clover term
 * -(c_sw/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu} with F the traceless
 * anti-Hermitian part of the four-leaf clover divided by 8i.
 * U: device, [V][4][3][3] complex128, read once; may be freed afterwards. */
int bri_build_links(bri_ctx* ctx, const double* U, double c_sw);

/* Export the stored links in the App. C layout [V][40][3][3] complex128
 * (device pointer W, caller-allocated, 5760 bytes per site). */
int bri_get_links(bri_ctx* ctx, double* W);

/* y = D_bri x (dagger = 0) or D_bri^dagger x = gamma5 D_bri gamma5 x
 * (dagger = 1) for nrhs right-hand sides, at bare mass m0 (Eq. def_bril;
 * App. C: y(n) = sum over the 81 offsets of W_d(n) M_d x(n+d) with real
 * stencil weights).  prec selects spinor dtype and link storage; with
 * BRI_PREC_DW (complex128 in and out) the operator runs in double-word FP32
 * arithmetic (relative error ~1e-15, the FP64 operator's accuracy class) and
 * the call allocates two double-word work vectors of nrhs right-hand sides
 * (stream-ordered) plus, on first use after bri_build_links, the double-word
 * link and clover copies (5760 + 576 bytes per site).  x and y must not
 * alias. */
int bri_apply(bri_ctx* ctx, void* y, const void* x, int nrhs, double m0, int dagger, int prec);

/* y = D_wil x or D_wil^dagger x (Eq. def_wils): 9-point stencil over the thin
 * links plus the same clover term. */
int wils_apply(bri_ctx* ctx, void* y, const void* x, int nrhs, double m0, int dagger, int prec);

/* Host-only: Kenney-Laub partial-fraction coefficients (Eq. KLnn_parfrac, Tab. 5;
 * kind BRI_KL_UPPER: Tab. 6) of f(x/scale) = x [c0 + sum_i w_i/(x^2+sigma_i)],
 * i = 0..n-1, shifts increasing.  Writes n entries into w and sigma. */
int kl_coeffs(int n, int kind, double scale, double* c0, double* w, double* sigma);

/* y = gamma5 f(H) x = D r(D^dagger D) x, H = gamma5 D_K(m0 = -rho), with
 * r(s) = c0 + sum_i w_i/(s+sigma_i) evaluated by one multi-shift CG
 * (Sec. 3.3, Sec. 4.1) to relative residual tol on every shift.
 * x, y: device complex128 [nrhs][V][4][3].  prec: BRI_PREC_F64 (all FP64) or
 * BRI_PREC_F32 / BRI_PREC_F32_BF16 (FP32 inner solve with FP32 or BF16 links
 * and FP64-accumulated solutions, FP64 reductions, defect-correction refinement
 * to tol on FP64-class residuals: the double-word FP32 operator of
 * BRI_PREC_DW for the Brillouin kernel wherever its error bound, 1e-13 of the
 * solution's norm, stays below 5 % of tol ||b||, else FP64).  kind selects
 * the Kenney-Laub family.  st may be NULL. */
int sign_apply_multishift(bri_ctx* ctx, void* y, const void* x, int nrhs, int n, int kind,
                          double rho, double scale, double tol, int prec, bri_stats* st);

/* y = (1 - am/(2 rho)) rho (x + gamma5 f(H) x) + am x: the massless overlap
 * (am = 0, Eq. def_over) or its traditional massive form
 * (Eq. def_mass_traditional).  Same arguments as sign_apply_multishift. */
int overlap_apply(bri_ctx* ctx, void* y, const void* x, int nrhs, int n, int kind,
                  double rho, double am, double scale, double tol, int prec, bri_stats* st);

/* Batched overlap application over several independent lattices (e.g. gauge
 * fields of uneven volume; the multi-rhs trick of App. C extended across
 * lattices): the same result as overlap_apply on
 * each context.  The multi-shift phase of every lattice and right-hand side
 * runs as one system table: each stencil launch walks a device-side work list
 * of (lattice, right-hand side, 128-site block) items, the CG scalars and
 * convergence flags of every system stay in device memory, and the iterations
 * run inside one CUDA graph whose conditional WHILE node repeats the
 * iteration until every system has converged (or reached the iteration cap),
 * with no host polling.  For the mixed precisions the FP64-class residuals, FP32
 * corrections and the final application then run per lattice, concurrently
 * on the contexts' own streams.  At most 32 contexts, all on the current
 * device, each with the Brillouin kernel; ys[i], xs[i]: device complex128
 * [nrhs[i]][V_i][4][3]; st: NULL or an array of nctx statistics.  Returns the
 * worst per-lattice code. */
int overlap_apply_batch(bri_ctx* const* ctxs, int nctx, void* const* ys, const void* const* xs, const int* nrhs,
                        int n, int kind, double rho, double am, double scale, double tol, int prec, bri_stats* st);

/* Massive overlap solve D_m x = b (Secs. 4.2-4.4) with cascaded
 * preconditioning (Sec. 8, Eqs. cascaded_one, cascaded_two): solves
 * (D_ov + mt) x = bt, mt = am/(1 - am/(2 rho)), with bt of the traditional
 * form (complete = 0, Eq. upshot_traditional) or of the complete form
 * (complete = 1, Eq. upshot_complete), D_ov of Kenney-Laub order n_outer, by
 * right-preconditioned BiCGstab to relative residual tol.  n_inner > 0 adds
 * the cascade: the preconditioner is an inexact solve (relative 1e-2) with the
 * order-n_inner operator, itself preconditioned by an inexact solve with the
 * kernel D_{-rho} + (1 + mt/rho); n_inner = 0 runs unpreconditioned.
 * x, b: device complex128 [nrhs][V][4][3], x overwritten (initial guess 0).
 * st (may be NULL): iterations = outer BiCGstab iterations (max over rhs),
 * refinements = inner iterations (sum), matvecs = kernel applications,
 * max_true_residual = final FP64 relative residual of the outer system. */
int overlap_solve(bri_ctx* ctx, void* x, const void* b, int nrhs, int n_outer, int n_inner, int kind,
                  double rho, double am, int complete, double tol, int prec, bri_stats* st);

/* Adjoint of overlap_apply for L = sum_r Re <eta_r, D_m psi_r>,
 * D_m = (1 - am/(2 rho)) D_ov + am (Eqs. def_over, def_mass_traditional;
 * Sec. 9: with a fixed-order rational the inner derivative is explicit).
 * Writes g_psi = D_m^dagger eta = gamma5 D_m gamma5 eta ([nrhs][V][4][3]
 * complex128) and g_U = dL/dU for the thin links given to bri_build_links
 * ([V][4][3][3] complex128), with the conventions dL = Re<g_psi, dpsi> and
 * dL = Re sum tr(g_U^dagger dU) (those of PyTorch's complex autograd).  The
 * derivative runs through the multi-shift solves (x_i for psi and z_i for
 * D^dagger eta, same shifts; g_psi reuses the z_i) and the path-averaged link
 * construction (App. C) -- for the Wilson kernel the thin links directly --
 * and, when the links were built with c_sw != 0, through the clover term (its
 * four-leaf field strength).  prec as for overlap_apply (solves); the force
 * and link back-propagation run in FP64. */
int overlap_grad(bri_ctx* ctx, void* g_psi, void* g_U, const void* eta, const void* psi, int nrhs, int n,
                 int kind, double rho, double am, double scale, double tol, int prec, bri_stats* st);

/* The FP64 sign-function solve of sign_apply_multishift (prec BRI_PREC_F64)
 * without any device allocation, for callers that cannot call cudaMalloc at
 * apply time (device memory fully reserved by their own pool, or loops where
 * an implicitly synchronising allocation is not acceptable).  There is no
 * counterpart in the paper; it is a deployment convenience.
 *
 * All solver workspace comes from one 32 MiB static device array that every
 * device loading the library holds until exit.  Limit: V * nrhs * (2n + 3) *
 * 192 bytes plus 64 KB + 4 KB * nrhs + 8 B * nrhs * ceil(V / 64) + 512 B of
 * state and reduction partials must fit in it (e.g. 8^4 with
 * nrhs = 1 and n <= 19, or 4^4 with nrhs <= 16 at n = 16); larger problems
 * are rejected with BRI_ERR_INVALID and a message.  The array's device address
 * is looked up (cudaGetSymbolAddress) by bri_build_links on the device that is
 * current then, which under lazy module loading is also when its 32 MiB are
 * committed; a call on a device where no links were built does that set-up
 * itself and should then come before any stream capture.  Every call reuses
 * the same array and leaves its contents behind;
 * the solver initialises everything it reads, but two calls whose work
 * overlaps on one device (other streams or host threads) race on it.
 * x, y: device complex128 [nrhs][V][4][3]; st may be NULL (true residuals are
 * not computed here). */
int sign_apply_multishift_noalloc(bri_ctx* ctx, void* y, const void* x, int nrhs, int n, int kind,
                                  double rho, double scale, double tol, bri_stats* st);

/* Profiling (tracing) of the stencil kernels.  When enabled, every launch of
 * the Brillouin (op 0) or Wilson (op 1) stencil, including those issued inside
 * the solvers, is bracketed by CUDA events on the context stream.
 * bri_profile_read synchronises those events and returns, for one operator and
 * precision, the launches, summed kernel milliseconds and site x rhs units
 * processed since the previous read, then resets the counters. */
int bri_profile_enable(bri_ctx* ctx, int enable);
int bri_profile_read(bri_ctx* ctx, int op, int prec, long long* launches, double* ms, double* site_rhs);

/* Quality diagnostics of the massless overlap operator D = D_ov of
 * Kenney-Laub order n (Sec. 5): for each of the nrhs vectors eta (device
 * complex128 [nrhs][V][4][3]) writes the normality defect
 * ||(D D^dagger - D^dagger D) eta|| (Sec. 5.1) and the Ginsparg-Wilson defect
 * ||(D gamma5 + gamma5 D - (1/rho) D gamma5 D) eta|| (Sec. 5.2, Eq.
 * ginswils_one) into the host arrays normality[nrhs] and gw[nrhs]
 * (absolute 2-norms; the paper normalises eta to 1).  Uses D^dagger =
 * gamma5 D gamma5: two overlap applications to 2 nrhs vectors.  The context's
 * kernel, kind, rho, tol and prec as for overlap_apply; st may be NULL. */
int overlap_quality(bri_ctx* ctx, const void* eta, int nrhs, int n, int kind, double rho, double tol, int prec,
                    double* normality, double* gw, bri_stats* st);

/* Locality of the massless overlap operator (Sec. 5.3): zeta = D_ov eta for
 * nrhs sources eta (device complex128 [nrhs][V][4][3]) supported on the site
 * src, and per source the sum of |zeta(x)| (spin-colour 2-norm) over the sites
 * x with Euclidean distance |x - src|^2 = b (minimal periodic image) into the
 * host array profile[nrhs][nbins], and the number of such sites into counts[nbins]
 * (distances with |x - src|^2 >= nbins are left out).  The profile is summed
 * with atomic additions, so its last bits may differ between runs. */
int overlap_locality(bri_ctx* ctx, const void* eta, int nrhs, int src, int n, int kind, double rho, double tol,
                     int prec, int nbins, double* profile, int* counts, bri_stats* st);

/* Nested Kenney-Laub iterate D^(k) of the shifted kernel (Sec. 4.1):
 * X = D_K(m0 = -rho), Y_1 = X r_{n1}(X^dagger X), Y_j = Y_{j-1} r_{nj}(Y_{j-1}^dagger Y_{j-1})
 * with the diagonal rationals of orders orders[0..levels-1] (host array), and
 * y = D^(k) x = rho (x + Y_k x), k = levels (1..4).  Level 1 is overlap_apply
 * of order n1; each further level is a multi-shift solve whose operator
 * applications are solves of the level below (FP64 throughout, relative
 * residual tol at every level).  By the nesting of the principal Pade maps,
 * orders {1, 1} give the same operator as order 4 (g_3 o g_3 = g_9 = f_44).
 * x, y: device complex128 [nrhs][V][4][3]; st may be NULL. */
int overlap_nested_apply(bri_ctx* ctx, void* y, const void* x, int nrhs, int levels, const int* orders, double rho,
                         double tol, bri_stats* st);

/* Free-field quark dispersion relations (Sec. 2, App. A): for npts spatial
 * momenta p (host, [npts][3], lattice units) and quark masses am (host,
 * [npts]) writes the energies aE (host, [npts]) of the free Wilson
 * (kernel = BRI_KERNEL_WILSON) or Brillouin (BRI_KERNEL_BRILLOUIN) operator,
 * or, with overlap != 0, of the overlap operator built on that kernel with
 * the exact sign function at parameter rho.  E is the smallest positive zero
 * of the free propagator's denominator after p4 -> iE (the transcendental
 * equations of App. A), one GPU thread per point: scanned from E = 0 in steps
 * of 2e-3 up to E = 8, then bisected to full FP64 precision; NaN where no zero
 * lies below E = 8.  Allocates a small device buffer; synchronises stream. */
int bri_dispersion(int kernel, int overlap, double rho, int npts, const double* p, const double* am, double* energy,
                   void* stream);

/* Measured fused-multiply-add throughput of this GPU, the ALU roofline of the
 * stencils (App. C counts the matvec in flops; it runs on CUDA cores).  kind:
 * 0 = FP64 FMA, 1 = FP32 FMA, 2 = paired FP32 FMA (fma.rn.f32x2).  A grid of
 * 8 blocks per SM, each thread advancing eight independent FMA chains, timed
 * with CUDA events on stream (best of three launches after one warm-up).
 * Writes TFLOP/s (2 flops per FMA) and the kernel milliseconds; allocates a
 * small output buffer; synchronises the stream. */
int bri_fma_probe(int kind, void* stream, double* tflops, double* ms);

/* Process-wide number of CUDA kernels this library has launched so far. */
long long bri_kernel_launches(void);

/* Process-wide number of device allocations this library has made so far
 * (link and clover storage, solver workspaces).  Diagnostic: the
 * allocation-free entry point leaves it unchanged. */
long long bri_device_allocations(void);

/* Thread-local description of the last error (never NULL). */
const char* bri_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BRI_H */
