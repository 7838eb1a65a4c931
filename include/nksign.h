/*
 * nksign -- nested Krylov-Ritz evaluation of sgn(A) b for A = gamma5 D_w(mu)
 * (Bloch & Heybrock, "A nested Krylov subspace method to compute the sign
 * function of large complex matrices", 2009), on one NVIDIA GB300 (sm_103a).
 *
 * C ABI. Plain pointers and sizes only; no C++ or PyTorch types cross it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: dims = {Lx, Ly, Lz, Lt}; site s = x + Lx*(y + Ly*(z + Lz*t)), V = Lx*Ly*Lz*Lt.
 * Spinor vectors: 12*V complex numbers, complex = two doubles (re, im)
 *   interleaved; element 12*s + 3*spin + colour.  A block of n vectors is
 *   stored vector after vector (vector r starts at element r*12*V).
 * Links: U_{x,+nu} in SU(3) for nu = 0,1,2,3 = x,y,z,t, layout
 *   [t][z][y][x][nu][3][3] complex doubles (row-major 3x3).
 * Gamma matrices (the paper leaves the basis open, Sec. 2): chiral basis,
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]],
 *   gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
 * Boundary conditions: periodic in x, y, z; in t antiperiodic (a factor -1 on
 *   every hop that crosses the t boundary) unless created with
 *   bc_t_antiperiodic = 0 (then periodic).
 * Wilson-Dirac operator (Sec. 2):
 *   D_w(mu) = 1 - kappa sum_{i=1..3}(T_i^+ + T_i^-) - kappa(e^{mu} T_4^+ + e^{-mu} T_4^-),
 *   (T_nu^{+-})_{yx} = (1 +- gamma_nu) U_{x,+-nu} delta_{y,x+-nu},
 *   U_{x,-nu} = U^dagger_{x-nu,+nu}, kappa = 1/(8 + 2 m_w).
 *
 * Pointers: entry points without the _dev suffix take HOST pointers, which
 * the library copies; the caller keeps ownership.  Entry points with the _dev
 * suffix take DEVICE pointers (of the context's device) and a cudaStream_t
 * passed as void* (NULL = legacy default stream); they are asynchronous with
 * respect to the host unless stated otherwise, and the caller keeps ownership.
 * The context owns all other device memory (links, Krylov bases, scratch),
 * allocated on first use and kept until nk_destroy.
 *
 * Errors: every int-returning call returns NK_OK (0) or a negative NK_E*
 * code; nk_last_error() then holds a one-line message.  A context is not
 * thread-safe: one host thread at a time.
 */
#ifndef NKSIGN_H
#define NKSIGN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NK_OK 0
#define NK_EINVAL (-1)      /* bad argument: odd k or l, l > k, bad dims, ... */
#define NK_ENOMEM (-2)      /* device allocation failed */
#define NK_EBREAKDOWN (-3)  /* two-sided Lanczos serious breakdown (App. B) */
#define NK_ENOTCONV (-4)    /* adaptive k: tolerance not met at k_max */
#define NK_ERHI (-5)        /* Roberts-Higham iteration did not converge */
#define NK_ECUDA (-6)       /* CUDA runtime error */
#define NK_ETIMEOUT (-7)    /* a bounded device-side wait ran out: the streaming kernels of the
                               outer recurrence wait at most one second for the bulk copies of
                               each tile into shared memory; that RHS is failed (the RHi
                               clusters synchronise with hardware cluster barriers) */
#define NK_ESTATE (-8)      /* call out of order (e.g. no links loaded) */

/* Solve flags (bitwise or). */
#define NK_FP64 0x0u        /* every stencil application in FP64 */
#define NK_MIXED 0x1u       /* two-float stencil for the first j0 outer steps, FP32 after; FP64
                               recurrence (nk_set_precision) */
#define NK_DOUBLE_PASS 0x2u /* regenerate V_k in a second pass instead of storing it (Sec. 4.4) */
#define NK_NO_GRAPH 0x10u   /* launch kernel by kernel instead of replaying a CUDA graph */
#define NK_ASYNC 0x40u      /* nk_sign_apply_dev / nk_overlap_apply_dev with tol = 0: enqueue the
                               solve and return without waiting; nk_wait collects its outcome.
                               One pending solve per context (its workspace); two contexts on two
                               streams keep two batches in flight.  Until nk_wait, the calls that
                               write the context's workspace, links or deflation vectors (the
                               solves, nk_load_links(_dev), nk_set_deflation, nk_eigs_smallest,
                               nk_autotune, nk_outer_lanczos_dev, nk_inner_sign, nk_features,
                               nk_predict_sizes, nk_overlap_solve) return NK_ESTATE. */
#define NK_SHARED_P 0x80u   /* one p for the whole batch (Eq. popt with z_min and z_max of A taken as
                               the extremes of the per-RHS estimates over the batch: every RHS
                               shares A), instead of one per RHS; p > 0 overrides both */
#define NK_PROFILE 0x20u    /* kernel by kernel, with CUDA events around every launch; fills
                               nk_stats.t_class_ms / n_class (implies NK_NO_GRAPH) */
#define NK_PREFIX_FP64 0x100u /* with NK_MIXED: the outer steps before j0 apply the FP64 stencil
                               instead of the two-float one (nk_set_precision) */
#define NK_EPS_EST 0x200u   /* also estimate the error of every result as in Sec. 3: apply the
                               method a second time to the result, x~ = approx(approx(x)), and
                               report eps = |x~ - x| / (2 |x|) per RHS in nk_stats.eps_sgn2
                               (doubles the work; nk_sign_apply(_dev) only, not with NK_ASYNC) */
#define NK_PREDICT 0x400u   /* with tol > 0: predict (k, l) with the predictor given to
                               nk_set_predictor from source 0 of the batch (nk_predict_sizes),
                               start the adaptive checks at k_pred - 2 NK_ADAPT_STEP with
                               l = min(2 ceil(0.75 l_pred), k_pred, 256) (k stays the maximum);
                               if the tolerance is not met by k with that l, the solve is
                               repeated once with the caller's l from the default start */

#define NK_MAX_RHS 12

/* Kernel classes of a solve, for nk_stats.t_class_ms / n_class. */
#define NK_CLASS_DSLASH 0     /* FP32 Wilson stencil A v (and A^dagger w), multi-RHS (in the
                                 optional two-float recurrence fused with its step 1) */
#define NK_CLASS_DSLASH_DF 1  /* two-float (about 48-bit) stencil fused with the FP64
                                 r = Av - c v_prev and the H(j,j) reduction */
#define NK_CLASS_STEP2 2      /* the FP64 recurrence kernels: step 1 after an FP32 stencil
                                 (r = Av - c v_prev, H(j,j)) and step 2 (r -= H(j,j) v,
                                 beta / delta, stencil input copies) */
#define NK_CLASS_DSLASH64 3   /* FP64 stencil fused with the FP64 step 1 */
#define NK_CLASS_INNER 4    /* p estimate, LU of p H_k, inner Lanczos */
#define NK_CLASS_RHI 5      /* Roberts-Higham iteration */
#define NK_CLASS_LIFT 6     /* V_l s and |x| V_k c */
#define NK_CLASS_OTHER 7    /* layout conversion, norms */
#define NK_CLASS_STEP2_DF 8 /* step 2 of the FP32-stencil steps of NK_MIXED (two-float) */
#define NK_NCLASS 9

typedef struct nk_ctx nk_ctx;

/* Per-solve statistics (all optional to read). */
typedef struct nk_stats {
    int n_rhs;
    int k_used;                        /* outer Krylov size used (largest over the RHS) */
    int k_rhs[NK_MAX_RHS];             /* outer Krylov size used per RHS (adaptive k) */
    int checks;                        /* adaptive k: convergence checks made */
    int ell_used;                      /* inner Krylov size used */
    int rhi_iters[NK_MAX_RHS];         /* Roberts-Higham iterations per RHS */
    int status[NK_MAX_RHS];            /* NK_OK or NK_E* per RHS */
    double p[NK_MAX_RHS];              /* preconditioning factor used (Eq. precond) */
    double z_min[NK_MAX_RHS];          /* spectral estimates behind p (Eq. popt) */
    double z_max[NK_MAX_RHS];
    double xnorm[NK_MAX_RHS];          /* |x| of each source */
    double t_total_ms;                 /* device time of the whole solve (CUDA events) */
    int launches;                      /* kernels this library launched for the solve */
    double t_class_ms[NK_NCLASS];      /* NK_PROFILE: summed device time per kernel class */
    int n_class[NK_NCLASS];            /* NK_PROFILE: launches per kernel class */
    /* Device time split as in the paper's timings (Sec. 3, Sec. 4.3), from CUDA
     * events between the phases of every solve: construction of the outer
     * basis (App. A / B), the inner part (p, LU of p H_k, inner Lanczos, RHi;
     * App. C steps 3-5) and the lift (step 6; with NK_DOUBLE_PASS it includes
     * the second basis construction).  Adaptive k sums its chunks. */
    double t_basis_ms, t_inner_ms, t_lift_ms;
    double eps_sgn2[NK_MAX_RHS];       /* NK_EPS_EST: |x~ - x| / (2|x|) per RHS (Sec. 3), else 0 */
    int k_pred, ell_pred;              /* NK_PREDICT: the predicted sizes, else 0 */
    int predict_fallback;              /* NK_PREDICT: 1 if the solve was repeated with the caller's l */
    int defl_m;                        /* LR deflation: eigenpairs deflated (nk_set_deflation) */
    double defl_gap;                   /* and the deflation gap Delta = max |lambda_i| (Sec. 3) */
} nk_stats;

/* Create a context for a lattice of dims[4] = {Lx, Ly, Lz, Lt} (each >= 2;
 * Lt even when antiperiodic is not required).  Selects the current CUDA
 * device.  *out receives the context. */
int nk_create_lattice(const int dims[4], int bc_t_antiperiodic, nk_ctx** out);

/* Load links from HOST memory, layout [t][z][y][x][nu][3][3] complex double
 * (18*4*V doubles).  Copies them, keeps an FP64 master and an FP32 copy on
 * the device (the FP32 copy is what the mixed-precision stencil reads). */
int nk_load_links(nk_ctx* ctx, const double* U);

/* Same from DEVICE memory (stream-ordered on `stream`). */
int nk_load_links_dev(nk_ctx* ctx, const double* U_dev, void* stream);

/* Set the chemical potential mu (Sec. 2; mu = 0 gives the Hermitian case and
 * the Lanczos recurrence, mu != 0 the two-sided recurrence) and the Wilson
 * mass m_w (kappa = 1/(8 + 2 m_w); requires 8 + 2 m_w > 0). */
int nk_set_mu_mw(nk_ctx* ctx, double mu, double m_w);

/* Precision schedule for NK_MIXED (the outer recurrence, App. A/B): outer
 * steps j < j0 apply the stencil in two-float arithmetic (about 48 bits, on
 * the FP32 pipe; FP32 links hi + lo) or, with NK_PREFIX_FP64, in FP64; steps
 * j >= j0 in FP32 (input vector, links and arithmetic FP32, including the
 * scale 1/|q_j| of the stencil output).  j0 < 0 selects the default k/4.
 * The recurrence itself (the updates of r and l, their inner products and
 * accumulation, the basis V_k) runs in FP64, and so do H_k, p, the LU of
 * p H_k, the inner Lanczos, RHi and the lift; nk_set_df_recurrence can move
 * the recurrence from a given step on to two-float arithmetic instead. */
int nk_set_precision(nk_ctx* ctx, int j0);

/* Optional two-float recurrence for NK_MIXED: from outer step j1 on the
 * updates of r and l, their inner products and the basis columns run in
 * two-float arithmetic (about 48 bits, on the FP32 pipe) on rings of the
 * newest three vectors, and the lift sums in two-float arithmetic.  j1 < 0
 * (the default) keeps the whole recurrence in FP64.  Takes effect with the
 * next solve. */
int nk_set_df_recurrence(nk_ctx* ctx, int j1);

/* LR deflation (App. C steps 1 and 6; Sec. 3).  m critical eigenpairs of A
 * (the paper deflates those of smallest modulus; the largest deflated
 * |lambda| is the deflation gap Delta): lambda[2 i], lambda[2 i + 1] = re, im
 * of lambda_i; R (HOST, m vectors in the ABI spinor layout, vector i at
 * element 12 V i) the right eigenvectors r_i; L the left eigenvectors l_i
 * with <l_i, r_j> = delta_ij, or NULL for Hermitian A (mu = 0: l_i = r_i).
 * Every following solve of this context projects its sources,
 *   x_minus = b - sum_i <l_i, b> r_i,
 * runs the nested method on x_minus, and adds sum_i sgn(Re lambda_i) <l_i, b> r_i
 * (Eq. sgnz) to the result; nk_overlap_apply applies b + gamma5 y to the whole.
 * Computing the eigenpairs is the caller's one-off initialisation (Sec. 3:
 * "performed once in an initialization step").  The eigenpairs must belong
 * to the current (mu, m_w) and links.  m = 0 switches deflation off.  Copies
 * the vectors (m <= NK_MAX_DEFL).  Blocks. */
#define NK_MAX_DEFL 256
int nk_set_deflation(nk_ctx* ctx, int m, const double* lambda, const double* R, const double* L);

/* The m eigenpairs of A = gamma5 D_w(mu) of smallest |lambda|: the critical
 * eigenpairs that LR deflation removes (App. C step 1; Sec. 3 computes them
 * once, as an initialisation, and deflates those of smallest modulus).  A
 * Lanczos eigensolver on the device: k steps of the FP64 recurrence of App. A
 * (mu = 0) or App. B (two-sided) from the start vector b (HOST, ABI spinor
 * layout, nonzero) with both bases V_k and W_k kept; the eigenvalues of the
 * tridiagonal H_k by the QL iteration; as candidates the 2 m + 8 distinct
 * ones nearest zero (finite-precision Lanczos repeats a converged eigenvalue:
 * up to 3 copies form one cluster); per cluster the right (and left)
 * eigenvectors of H_k spanning its invariant subspace (block inverse
 * iteration) and the refined combinations of them whose last component
 * vanishes, lifted through the bases (Ritz vectors); the true residuals
 * |A r - theta r| / |r| and |A^dagger l - theta^* l| / |l| (FP64 stencil),
 * and per cluster the candidate of least residual on each side; the returned
 * eigenvalue is the Rayleigh quotient <l, A r> (<l, r> = 1) where its
 * residuals are not larger than those of H_k's eigenvalue (H_k's is good to
 * about the residual, the quotient to about the product of the left and
 * right residuals), else H_k's.
 * Unrestarted: the small eigenvalues need k large enough for them to
 * converge (several hundred on the small lattices of the tests; k = 12 V
 * exhausts the space).
 *   k     even, >= 2 m + 2; the workspace holds 2 (k + 1) vectors of 12 V,
 *         and 2 (48 + m) + 1 more of temporary device memory
 *   tol   residual bound for a returned pair
 * Returns, for the found <= m converged candidates nearest zero, in order of
 * |theta|: lambda (HOST, 2 m doubles: re, im), R (HOST, m vectors of 12 V
 * complex, ABI layout, |r_i| = 1), L (HOST, the same, <l_i, r_i> = 1; at
 * mu = 0 L may be NULL, else it receives r_i), resid (HOST, m, or NULL:
 * the larger of the right and left residuals);
 * these are the arguments of nk_set_deflation.  NK_OK when found = m,
 * NK_ENOTCONV when fewer converged (the found ones are returned),
 * NK_EBREAKDOWN on a Lanczos breakdown before step k.  Blocks; allocates its
 * temporary device memory per call (a one-off initialisation). */
int nk_eigs_smallest(nk_ctx* ctx, const double* b, int k, int m, double tol, double* lambda, double* R, double* L,
                     double* resid, int* found);

/* Multi-level nesting (Sec. 4.5).  A solve's l argument is the size l_1 of the
 * first nested level; nk_set_nesting adds n_deeper levels below it with sizes
 * ells[0] = l_2 >= l_3 >= ... (even, >= 2; a level larger than the one above
 * is clipped to it), n_deeper <= NK_MAX_LEVELS - 1.  Level i + 1 repeats App. C
 * steps 3-4 on the Ritz matrix H_{l_i} of level i: p_{i+1} by Eq. popt from
 * H_{l_i} (one per RHS), the LU of p_{i+1} H_{l_i}, and l_{i+1} steps of the
 * (two-sided) Lanczos recurrence with H_{l_i}' from e_1.  RHi runs on the
 * deepest Ritz matrix only, and the result is lifted back through every
 * level: y = |b| V_k V_{l_1} ... V_{l_n} sgn(H_{l_n}) e_1.  n_deeper = 0 (the
 * default) is the single nesting of Eq. nested.  Applies to the solves and to
 * nk_inner_sign of this context from the next call on. */
#define NK_MAX_LEVELS 6
int nk_set_nesting(nk_ctx* ctx, int n_deeper, const int* ells);

/* Adaptive k: the outer size at the first convergence check (even; 0 selects
 * NK_ADAPT_FIRST(l)).  A predicted k (nk_predict_sizes) minus two check
 * intervals goes here, so that a good prediction costs three checks. */
int nk_set_adapt_start(nk_ctx* ctx, int k_first);

/*
 * Launch shape of the outer recurrence (batching of the RHS and the
 * autotuner; a property of the implementation, not of the method).
 *  stencil_threads  lattice sites per CTA of the fused stencil kernel, one
 *                   thread per site and vector: 64, 128 or 256;
 *  stencil_order    0: consecutive CTAs take all vectors (RHS and, for mu != 0,
 *                   both sides) of one block of sites, so the links of those
 *                   sites are read from HBM once and then from L2;
 *                   1: consecutive CTAs take the site blocks of one vector;
 *  step2_blocks     CTAs per RHS of the step-2 and norm kernels (grid-stride),
 *                   1..4096; also the number of partial sums of their
 *                   deterministic reductions;
 *  stencil_split    threads per site of the fused stencil: 1, or 3 (one per
 *                   colour: each projects the neighbour spinors and forms one
 *                   colour row, with a third of the accumulators);
 *  early_threads, early_order, early_split
 *                   the stencil shape of the two-float steps before j0 in
 *                   NK_MIXED mode (unused in NK_FP64 mode).
 * A shape belongs to (n_rhs, sidedness of the current mu (mu != 0), the
 * NK_MIXED bit of flags).  Different shapes sum in different orders, so
 * results differ at rounding level; one shape is bitwise reproducible.
 * Unset shapes use 128 / 0 / min(ceil(12 V / 2048), 608 / n_rhs) / 128 / 0 / 1 / 1.
 */
typedef struct nk_launch {
    int stencil_threads;
    int stencil_order;
    int step2_blocks;
    int early_threads;
    int early_order;
    int stencil_split;
    int early_split;
} nk_launch;
int nk_set_launch(nk_ctx* ctx, int n_rhs, unsigned flags, const nk_launch* shape);
int nk_get_launch(nk_ctx* ctx, int n_rhs, unsigned flags, nk_launch* shape);
/* Tunes the launch shape on a synthetic constant source: after 8 outer steps,
 * 50 repetitions of one outer step (fused stencil, then step 2, as in a
 * solve; best of 3 rounds) are timed with CUDA events for each candidate -- the 3 x 2 x 2
 * stencil shapes with the FP32 stencil (NK_MIXED) or the FP64 one; in NK_MIXED mode
 * the same shapes with the two-float stencil (early_threads, early_order);
 * then step2_blocks in {b/2, b, 2b, 4b, 8b} (b the default) with the fastest
 * late stencil shape.  Keeps the fastest of each (written to *best, and the
 * time of one late outer step to *ms_per_step; both nullable).
 * cache_path (nullable): a text file of lines
 *   nk_launch Lx Ly Lz Lt n_rhs two_sided mixed threads order blocks
 *             early_threads early_order split early_split ms_per_step
 * read first (a matching line is used without timing) and appended to after
 * timing.  Blocks. */
int nk_autotune(nk_ctx* ctx, int n_rhs, unsigned flags, const char* cache_path, nk_launch* best,
                double* ms_per_step);

/*
 * y = sgn(A) b by the nested Krylov-Ritz method (Eq. nested; App. C steps
 * 2-6 without deflation):
 *   outer (two-sided) Lanczos of size k (App. A / B) -> V_k, H_k;
 *   p from Eq. popt (power / inverse iteration with H_k) unless p > 0 given;
 *   LU of p H_k (gttrf form, App. C step 3);
 *   inner (two-sided) Lanczos of size l with H_k' = [pH_k + (pH_k)^{-1}]/2 and
 *   e_1 (Eq. precond, App. C step 4) -> V_l, H_l;
 *   Roberts-Higham iteration on H_l (Eq. Roberts, App. C step 5);
 *   y = |b| V_k V_l sgn(H_l) e_1 (App. C step 6).
 * b, y: HOST arrays of n_rhs vectors (1 <= n_rhs <= NK_MAX_RHS), each solved
 * independently (own recurrence coefficients) but batched through one
 * stencil launch per step.  k, l even (Fig. 7 caption), 2 <= l <= k, k <= 1536, l <= 256.
 * tol = 0: fixed k.  tol > 0: adaptive k (the paper fixes k; this stopping
 * rule is the library's): k is the maximum, the outer recurrence is
 * checked every NK_ADAPT_STEP steps from NK_ADAPT_FIRST(l) on (or from
 * nk_set_adapt_start), each check computes c = V_l sgn(H_l) e_1 from the
 * current H_k, and a RHS stops growing k once |c - c_prev| <= tol |c| at two
 * consecutive checks (its result is taken at that k); a RHS that never
 * meets it uses k_max and gets status NK_ENOTCONV (its result is still
 * written).  Adaptive solves are launched kernel by kernel.  flags: NK_FP64
 * or NK_MIXED, optionally NK_DOUBLE_PASS (fixed k only) / NK_NO_GRAPH.  st
 * may be NULL.  Blocks until y is written.  Returns NK_EBREAKDOWN / NK_ERHI /
 * NK_ENOTCONV when any RHS failed (st->status says which; the other RHS are
 * still valid). */
#define NK_ADAPT_STEP 64
#define NK_ADAPT_FIRST(l) ((((l) + 63) / 64) * 64)
int nk_sign_apply(nk_ctx* ctx, const double* b, int n_rhs, int k, int ell, double tol,
                  double p, unsigned flags, double* y, nk_stats* st);

/* Same with DEVICE b and y, stream-ordered on `stream`; returns once the
 * solve has completed (it reads the per-RHS status back). */
int nk_sign_apply_dev(nk_ctx* ctx, const double* b_dev, int n_rhs, int k, int ell, double tol,
                      double p, unsigned flags, double* y_dev, nk_stats* st, void* stream);

/* Overlap operator D_ov(mu) b = b + gamma5 sgn(gamma5 D_w(mu)) b (Eq. Dovmu),
 * one sign evaluation per call; arguments as nk_sign_apply with p automatic. */
int nk_overlap_apply(nk_ctx* ctx, const double* b, int n_rhs, int k, int ell, double tol,
                     unsigned flags, double* y, nk_stats* st);
int nk_overlap_apply_dev(nk_ctx* ctx, const double* b_dev, int n_rhs, int k, int ell,
                         double tol, unsigned flags, double* y_dev, nk_stats* st, void* stream);

/* Overlap inversion (the consumer the paper's Sec. 3 names: f(A) x "needed
 * by iterative inverters"): x = (D_ov(mu) + mass)^{-1} b by conjugate
 * gradients on the normal equations M^dagger M x = M^dagger b, M = D_ov(mu) +
 * mass (mass >= 0: the library's shift; mass = 0 is Eq. Dovmu itself).  Every
 * iteration applies M (nk_overlap_apply) and M^dagger = gamma5 (D_ov(-mu) +
 * mass) gamma5 (A(mu)^dagger = A(-mu)), each through the nested sign function
 * with (k, l, tol_sign, flags) as nk_sign_apply (and the deflation of the
 * context, with left and right eigenvectors exchanged for -mu).  Stops when
 * |M^dagger (b - M x)| <= tol_cg |M^dagger b| for every RHS, or after maxit
 * iterations (NK_ENOTCONV; x is still written).  b, x HOST arrays of n_rhs
 * vectors; iters and resid (nullable, n_rhs entries) receive the iterations
 * and the final relative residual of the normal equations per RHS.  The
 * sign function's own error bounds the attainable residual.  Blocks. */
int nk_overlap_solve(nk_ctx* ctx, const double* b, int n_rhs, int k, int ell, double tol_sign, unsigned flags,
                     double mass, double tol_cg, int maxit, double* x, int* iters, double* resid);

/* Waits for the pending NK_ASYNC solve of the context and returns its result
 * code; st (nullable) receives its statistics.  NK_OK if none is pending. */
int nk_wait(nk_ctx* ctx, nk_stats* st);

/* The Wilson stencil alone: out_r = A in_r (dagger = 0) or A^dagger in_r
 * (dagger = 1; A^dagger = gamma5 D_w(-mu)) for n_vec DEVICE vectors in the
 * ABI layout (n_vec <= 24).  precision = 64 computes in FP64 with the FP64
 * links; 48 in two-float arithmetic (about 48 bits); 32 rounds the input to
 * FP32 and computes with the FP32 links through nk_stencil32_dev's kernel
 * (output FP64).
 * Stream-ordered, asynchronous. */
int nk_dslash_dev(nk_ctx* ctx, const double* in_dev, double* out_dev, int n_vec, int dagger,
                  int precision, void* stream);

/* The multi-RHS FP32 stencil alone, in its native layout: for the 2 n_rhs
 * DEVICE vectors of in_dev (FP32, 16-byte aligned), out_r = A in_r for
 * r < n_rhs and out_r = A^dagger in_r for n_rhs <= r < 2 n_rhs, with the FP32
 * links (1 <= n_rhs <= NK_MAX_RHS).  Layout of each vector: the "pair layout"
 * [6][V] of four floats, entry i of site s holding spin-colour components
 * 2i and 2i + 1 (component = 3 spin + colour) as (re, im, re, im); vector r
 * starts at float 24 V r.  One launch applies the stencil to all 2 n_rhs
 * vectors, each link read once per block of sites.  This is the stencil of
 * the late outer steps of NK_MIXED (there fused with the first half of the
 * Lanczos step).  Stream-ordered, asynchronous. */
int nk_stencil32_dev(nk_ctx* ctx, const float* in_dev, float* out_dev, int n_rhs, void* stream);

/* The outer recurrence alone (App. A for mu = 0, App. B otherwise): k steps
 * from each of n_rhs DEVICE sources b_dev; writes H_k of each RHS as
 * three HOST arrays of complex doubles, alpha[r*k + j] = H(j,j),
 * beta[r*k + j] = H(j+1,j), gamma[r*k + j] = H(j,j+1) (j < k-1), and |b_r|
 * to xnorm[r].  flags: NK_FP64 or NK_MIXED.  Blocks. */
int nk_outer_lanczos_dev(nk_ctx* ctx, const double* b_dev, int n_rhs, int k, unsigned flags,
                         double* alpha, double* beta, double* gamma, double* xnorm,
                         void* stream);

/* The inner half (App. C steps 3-5 and the product V_l s) for n_rhs given
 * tridiagonal Ritz matrices (HOST arrays in the nk_outer_lanczos_dev layout):
 * c_r = V_l sgn(H_l) e_1 as complex doubles in the HOST array c[r*k + i].
 * hermitian = 1 uses the real Lanczos path (H real symmetric), 0 the
 * two-sided one.  p > 0 fixes p; p == 0 estimates it per RHS (Eq. popt);
 * p < 0 estimates one p for the batch (as NK_SHARED_P).  Needs a
 * context only for its device and scratch memory.  Blocks. */
int nk_inner_sign(nk_ctx* ctx, const double* alpha, const double* beta, const double* gamma,
                  int n_rhs, int k, int ell, double p, int hermitian, double* c,
                  nk_stats* st);

/*
 * Learned subspace sizes.  The paper chooses k and l by hand (Sec. 4.2-4.3);
 * this predictor is the library's: a 16 -> 64 -> 64 -> 2 perceptron (tanh,
 * tanh, linear; FP32) from NK_MLP_IN features of the operator and source to
 * (log2 k, log2 l) reaching a tolerance, trained on runs of the method
 * itself.  Forward pass, backward pass (mean squared error of the
 * standardised outputs) and Adam updates are CUDA kernels.  Host arrays;
 * the calls block.  Parameter layout: W1[64][16], b1[64], W2[64][64], b2[64],
 * W3[2][64], b3[2] (row = output unit).
 */
#define NK_MLP_IN 16
#define NK_MLP_HIDDEN 64
#define NK_MLP_OUT 2
#define NK_MLP_PARAMS (64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2)
typedef struct nk_mlp nk_mlp;
/* Glorot-uniform weights from `seed` (splitmix64), zero biases, identity
 * standardisation.  Uses the current CUDA device. */
int nk_mlp_create(unsigned long long seed, nk_mlp** out);
/* Standardisation: inputs x -> (x - xmu)/xsd, targets y -> (y - ymu)/ysd. */
int nk_mlp_set_norm(nk_mlp* m, const float* xmu, const float* xsd, const float* ymu, const float* ysd);
int nk_mlp_get_params(nk_mlp* m, float* params);          /* NK_MLP_PARAMS floats */
int nk_mlp_set_params(nk_mlp* m, const float* params);    /* also resets the Adam state */
/* Loss and gradient (w.r.t. the parameters) for n <= 256 samples X[n][16], Y[n][2]. */
int nk_mlp_loss_grad(nk_mlp* m, const float* X, const float* Y, int n, float* loss, float* grad);
/* Decoupled weight decay of the Adam steps (w -= lr wd w per step), in [0, 1);
 * 0 (the default) is plain Adam. */
int nk_mlp_set_weight_decay(nk_mlp* m, float wd);
/* `epochs` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on n <= 256
 * samples; loss_hist (nullable) receives the loss before each step. */
int nk_mlp_train(nk_mlp* m, const float* X, const float* Y, int n, int epochs, float lr, float* loss_hist);
/* Predictions Y[n][2] (de-standardised) for X[n][16]. */
int nk_mlp_forward(nk_mlp* m, const float* X, int n, float* Y);
const char* nk_mlp_last_error(const nk_mlp* m);
void nk_mlp_destroy(nk_mlp* m);

/* The NK_MLP_IN predictor features of one DEVICE source b_dev (ABI layout):
 *  0 mu, 1 m_w, 2 log10 V, 3 mean plaquette (1/3) Re tr U_mu(x)^+ U_nu(x+mu)^+
 *  U_mu(x+nu) U_nu(x) (gauge invariant in the hop convention of Sec. 2),
 *  then from 32 steps of the outer recurrence (App. A / B, FP64 stencil) and
 *  the inner part on H_32 (l = 32):
 *  4 log10 z_min, 5 log10 z_max, 6 log10(z_max / z_min), 7 log10 p (Eq. popt),
 *  8 mean Re H(j,j), 9 std Re H(j,j), 10 max |Im H(j,j)|, 11 mean |H(j+1,j)|,
 *  12 std |H(j+1,j)|, 13 least-squares slope of log|H(j+1,j)| over j,
 *  14 log10(|c_24..31| / |c|) of c = V_l sgn(H_l) e_1, 15 RHi iterations.
 * Blocks. */
int nk_features(nk_ctx* ctx, const double* b_dev, float* features, void* stream);

/* Predicted sizes for one DEVICE source: features -> predictor -> k (even,
 * clamped to [64, k_max]) and l (even, clamped to [16, min(k, 256)]). */
int nk_predict_sizes(nk_ctx* ctx, nk_mlp* m, const double* b_dev, int k_max, int* k, int* ell, void* stream);

/* The predictor that NK_PREDICT solves of this context use (NULL: none).  The
 * context does not own it: keep it alive while such solves run. */
int nk_set_predictor(nk_ctx* ctx, nk_mlp* m);

/* No-allocation variant of nk_inner_sign (the paper has no counterpart: this
 * is a deployment entry point, not a step of the method).  For callers that
 * must not allocate device memory -- code running where cudaMalloc is
 * forbidden or unsafe, such as inside another framework's memory budget or a
 * process whose allocator it does not own.  It computes the same c_r =
 * V_l sgn(H_l) e_1 as nk_inner_sign (p > 0 fixed, p == 0 one estimate per
 * RHS, p < 0 one p for the batch), but all inputs and outputs are DEVICE
 * arrays owned by the caller (alpha_dev, beta_dev, gamma_dev, c_dev in the
 * nk_outer_lanczos_dev layout, complex doubles [r*k + j]) and every other
 * buffer it needs lives in one static device array of the library (about
 * 5.9 MB, held by every GPU that loads the library until the process exits).
 * It calls no cudaMalloc/cudaFree and needs no context.
 * Limits: n_rhs <= NK_NOALLOC_MAX_RHS, k <= NK_NOALLOC_MAX_K,
 * l <= NK_NOALLOC_MAX_ELL; larger sizes return NK_EINVAL with a message.
 * The first call on each device looks up the array's device address and sets
 * kernel attributes.  The array is shared by all calls and keeps the previous call's contents, so
 * calls whose GPU work overlaps (other streams, other host threads) race on
 * it.  Stream-ordered on `stream`; returns after the stream has finished the
 * call (it reads the per-RHS status back).  err (may be NULL) receives a
 * one-line message of err_len bytes at most. */
#define NK_NOALLOC_MAX_RHS 2
#define NK_NOALLOC_MAX_K 1024
#define NK_NOALLOC_MAX_ELL 128
int nk_inner_sign_noalloc(const double* alpha_dev, const double* beta_dev, const double* gamma_dev,
                          int n_rhs, int k, int ell, double p, int hermitian, double* c_dev,
                          void* stream, char* err, size_t err_len);

/* Message of the last failed call on this context (never NULL). */
const char* nk_last_error(const nk_ctx* ctx);

/* Release every device resource of the context.  NULL is a no-op. */
void nk_destroy(nk_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* NKSIGN_H */
