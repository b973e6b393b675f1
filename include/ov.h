/*
 * ov.h -- C ABI of the GB300 two-sided Lanczos sgn(H) b library and its
 * gauge-force vector-Jacobian product.
 *
 * Method: M. Puhr, P. Buividovich, "A numerical method to compute derivatives
 * of functions of large complex matrices and its application to the overlap
 * Dirac operator at finite chemical potential", arXiv:1604.08057.
 *
 *   H(mu) = gamma5 D_w(mu)                                   (Sec. 1, Eq. overlap)
 *   D_w(mu) = 1 - kappa sum_{i<=3}(G_i^+ + G_i^-)
 *                - kappa (e^{mu} G_4^+ + e^{-mu} G_4^-)       (App. A, Eq. WD_op)
 *   (G_nu^+)_{x,y} = (1 + gamma_nu) U_nu(x) delta_{x+nu,y}
 *   (G_nu^-)_{x,y} = (1 - gamma_nu) U_nu(x-nu)^dagger delta_{x-nu,y}   (Eq. WD_G)
 *   kappa = 1 / (2 m_w + 8)
 *
 * Conventions shared by every entry point:
 *   - Lattice dims[4] = {Nx, Ny, Nz, Nt}; site index ((t*Nz + z)*Ny + y)*Nx + x;
 *     periodic boundary conditions in all four directions.
 *   - gamma matrices: Euclidean chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma5 = diag(1,1,-1,-1).
 *   - All array arguments are DEVICE pointers to interleaved complex128
 *     (re, im doubles), caller-owned, 16-byte aligned:
 *       links  U[V][4][3][3]  (direction order x, y, z, t; U[..][a][b] row a col b)
 *       spinor psi[V][4][3]   (spin, colour)
 *       n sources are stored back to back: psi[nsrc][V][4][3].
 *   - Every call is ordered on the context's CUDA stream and returns only
 *     after the stream has finished the call's work; the return value is 0
 *     on success or a negative OV_ERR_* code.  No exception crosses the ABI.
 *   - The context owns all device workspace; it grows on demand and is
 *     released by ov_context_destroy.  A context is used by one host thread
 *     at a time.
 */
#ifndef OV_H
#define OV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define OV_OK                  0
#define OV_ERR_INVALID_ARG    -1  /* a null pointer, a non-positive size, k out of range */
#define OV_ERR_OOM            -2  /* device workspace could not be allocated */
#define OV_ERR_BREAKDOWN      -3  /* Lanczos breakdown: |omega| <= 1e-14 ||r|| ||s|| */
#define OV_ERR_SIGN_ILLPOSED  -4  /* k x k Newton sign did not converge or hit a singular iterate */
#define OV_ERR_CUDA           -5  /* a CUDA runtime call failed */
#define OV_ERR_NONFINITE      -6  /* a NaN or Inf appeared in a recurrence coefficient */
#define OV_ERR_SCRATCH_LIMIT  -7  /* the problem does not fit the fixed scratch of ov_apply_H_noalloc */
#define OV_ERR_TIMEOUT        -8  /* a device-side wait between blocks ran past its limit (2 s); the
                                     blocks stop and the context stays usable */
#define OV_ERR_NOCONV         -9  /* an iteration did not converge: the Ritz values of the run
                                     diagnostics, or ov_overlap_solve within maxit */

/* Precision of lattice vectors, links and stencil arithmetic.
 * OV_FP64 : everything in FP64.
 * OV_MIXED: links, basis vectors and stencils in FP32; dot products accumulated
 *           with compensated (Dot2) FP32 arithmetic per thread and FP64 across
 *           threads; recurrence coefficients, re-biorthogonalisation
 *           coefficients, the k x k sign and its Frechet adjoint in FP64. */
#define OV_FP64  0
#define OV_MIXED 1

typedef struct {
  int32_t precision;   /* OV_FP64 or OV_MIXED */
  int32_t rebiorth;    /* 0: none; 1: every step; P > 1: at the two steps j = 0, 1 (mod P) */
  int32_t passes;      /* classical Gram-Schmidt passes per re-biorthogonalisation (1 or 2) */
  int32_t segment;     /* 0: keep all k basis vectors in device memory.  S > 0: two-pass TSL
                        * (Sec. 4.1) with segment replay: the recurrence keeps a window of
                        * S + 2 basis vectors, checkpoints its state every S steps, and
                        * recomputes each segment bit for bit when x = V_k y, g_y = V_k^dag xbar
                        * and the reverse sweep need its vectors.  Requires rebiorth = 0 (every
                        * projection reads the whole basis); not for the block TSL. */
  int32_t dense;       /* k x k inversions of the Newton sign (Gauss-Jordan, partial pivoting):
                        * 0: one cooperative launch per inversion where the problems' rows fit
                        * in shared memory (rows stay on chip for all k elimination steps; the
                        * steps are separated by bounded inter-block waits), else 1;
                        * 1: one launch per elimination step, replayed as a CUDA graph.
                        * Both give bitwise identical results.  The m x m matrices of the nested
                        * stage (options.nested) always use form 1. */
  int32_t diagnostics; /* 0: none.  1: after the forward recurrence of ov_tsl_sign, ov_tsl_sign_vjp,
                        * ov_tsl_sign_fwd and ov_tsl_batch, measure (a) the loss of
                        * biorthogonality of the stored bases, sampled on the last pair of basis
                        * vectors: max over i < k of |w_i^dag v_k|, |v_i^dag w_k| and of
                        * |w_k^dag v_k - 1| (one dot-product sweep over both bases; not with
                        * segments), and (b) the Ritz values, the eigenvalues of T_k (host,
                        * ov_tridiag_eigenvalues), and return OV_ERR_SIGN_ILLPOSED, with info
                        * filled, when min |Re lambda(T_k)| <= 1e-14 ||T_k||_inf (sgn is not
                        * defined on the imaginary axis, Sec. 2 Eq. spectral_form). */
  int32_t newton;      /* rules of the scaled Newton iteration for the k x k sign (Higham,
                        * "Functions of Matrices", ch. 5; the Frechet adjoint reuses the forward's
                        * scalings): 0 (default): Frobenius-norm scaling
                        * g = (||X^{-1}||_F / ||X||_F)^{1/2} and a stop one iteration after the
                        * quadratic model s_{i+1} ~ s_i^3 / s_{i-1}^2 predicts a relative step
                        * <= 1e-12; 1: determinant scaling |det X|^{-1/k} and a stop when the
                        * relative step is <= 1e-14 or no longer halves.  Scaling ends once the
                        * step is below 1e-2 in both. */
  int32_t basis_memory; /* where the Krylov bases V_k, W_k live: 0 (default) device memory;
                        * 1 pinned host memory mapped into the device address space, read and
                        * written by the kernels over the CPU-GPU link (NVLink-C2C on a GB300),
                        * for bases larger than device memory.  Same kernels and results, bit
                        * for bit, with any re-biorthogonalisation schedule. */
  int32_t graphs;      /* 1 (the default when ov_context_create gets no options): when a call
                        * on the context repeats the previous call's shape, buffers and schedule
                        * (k, sources, lattice, mu, m_w, options), its forward Lanczos sweep and
                        * its reverse sweep are captured as CUDA graphs, and later calls with that
                        * shape replay them, which removes the host's per-kernel launch cost (the
                        * sweeps launch ~10 kernels per step); results are bit for bit those of
                        * direct launches.  Not used while per-kernel profiling or a fault
                        * injection is active, or with segments.  0: direct launches. */
  int32_t gemm;        /* complex k x k products of the Frechet adjoint's iteration (Theorem 1;
                        * also the block forward mode of ov_block_tsl_sign / ov_tsl_sign_jvp):
                        * 0 (default): on the BF16 tensor cores for 128 <= k <= 1024, by an exact
                        * splitting of each FP64 operand into ten 7-bit integer digits below a
                        * per-row (left factor) or per-column (right factor) power-of-two scale
                        * (Ozaki scheme; the 55 digit products with p + q <= 11, summed exactly
                        * in integers, at most two FP64 roundings per real product: error per
                        * entry <~ 4u (|L||R|)_ij + 12 k 2^-70 max_l |L_il| max_l |R_lj|, the
                        * size of FP64 rounding for lines spanning up to ~2^17 in magnitude),
                        * else FP64 arithmetic; 1: FP64 arithmetic always; 2: the tensor-core
                        * form wherever k <= 1024.  Needs ~930 k^2 bytes of device workspace
                        * (0.6 GB at k = 800). */
  int32_t nested;      /* k x k sign of the forward passes (ov_tsl_sign and everything built on it:
                        * ov_tsl_eps, ov_overlap_apply, ov_overlap_solve, the deflated forms; the
                        * block TSL of ov_block_tsl_sign / ov_tsl_sign_jvp / ov_block_tsl_eps):
                        * 0 (default) sgn(T_k) e_1 by the scaled Newton iteration on T_k;
                        * m in 1..OV_NESTED_MAX: the nested TSL with one nesting level and inner
                        * Krylov size m (Sec. 4.1, inner size 100 there), sgn(T_k) e_1 ~
                        * Q_m sgn(H_m) e_1 from m Arnoldi steps on S = (T_k + T_k^{-1})/2 started
                        * at e_1 (sgn(S) = sgn(T_k): z -> (z + 1/z)/2 keeps the sign of Re z), see
                        * ov_tridiag_sign_nested.  O(k^2 m) work instead of O(k^3) per Newton
                        * iteration; an approximation of the full result whose error falls with m.
                        * The reverse mode (ov_tsl_sign_vjp, ov_tsl_sign_fwd, ov_tsl_batch,
                        * ov_u1_current) differentiates the full k x k sign and returns
                        * OV_ERR_INVALID_ARG while nested > 0.  Needs 16 k^2 bytes of device
                        * workspace per source for S. */
} ov_options;

#define OV_NESTED_MAX 1024   /* largest inner Krylov size of options.nested */

typedef struct {
  int32_t k_reached;        /* Lanczos steps completed */
  int32_t newton_iters;     /* Newton iterations of the k x k sign (forward) */
  int32_t newton_iters_adj; /* Newton iterations of the Frechet adjoint (VJP only) */
  int32_t reserved;
  double  min_abs_re_ritz;  /* with options.diagnostics: min over sources and Ritz values of
                               |Re lambda(T_k)|; else 0 */
  double  t_ms[8];          /* phase times (ms).  ov_tsl_sign: 0 forward Krylov, 1 k x k sign,
                               2 combine.  ov_tsl_sign_vjp: 0 forward Krylov, 1 g_y = V^dag xbar,
                               2 k x k sign and Frechet adjoint, 3 combine, 4 reverse sweep and
                               force.  Others unused. */
  double  biorth_loss;      /* with options.diagnostics: the sampled loss of biorthogonality
                               (max over sources; -1 with segments); else 0 */
  double  t_norm;           /* with options.diagnostics: max over sources of ||T_k||_inf; else 0 */
} ov_tsl_info;

typedef struct ov_context ov_context;

/* Create a context bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current CUDA device.  `opt` may be NULL (FP64, rebiorth 1,
 * 2 passes).  *ctx receives the handle. */
int ov_context_create(ov_context **ctx, const ov_options *opt, void *stream);
int ov_context_destroy(ov_context *ctx);
int ov_context_set_options(ov_context *ctx, const ov_options *opt);

/* out = H(mu) in (dagger = 0) or H(mu)^dagger in (dagger != 0) for nsrc
 * sources; H^dagger = gamma5 D_w(-mu) (gamma5-hermiticity of Eq. WD_op).
 * in and out must not overlap.  Arithmetic in the context's precision. */
int ov_apply_H(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
               int32_t nsrc, const void *in, void *out, int32_t dagger);

/* x ~ sgn(H(mu)) b by k steps of two-sided Lanczos (Sec. 1 and 2, the TSL of
 * Bloch et al.), one independent Krylov recurrence per source:
 *   v_1 = w_1 = b/||b||; T_k tridiagonal; x = ||b|| V_k sgn(T_k) e_1.
 * 2 <= k <= 4096.  info may be NULL. */
int ov_tsl_sign(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                int32_t nsrc, const void *b, int32_t k, void *x, ov_tsl_info *info);

/* Vector-Jacobian product of the k-step TSL map: with L = sum_src Re <xbar, x>,
 *   dU[V][4][3][3] (device, complex128) = dL/dRe U + i dL/dIm U   (all 9 entries
 *                                          independent, no SU(3) projection)
 *   *dmu (host double)                   = dL/dmu.
 * The forward pass is recomputed; the reverse sweep differentiates every step
 * of it, including the re-biorthogonalisation, and the k x k sign through its
 * Frechet adjoint, taken from the Theorem-1 block matrix by Newton iteration.
 * x (device, may be NULL) receives the forward result.  info may be NULL. */
int ov_tsl_sign_vjp(ov_context *ctx, const int32_t dims[4], const void *U, double mu,
                    double m_w, int32_t nsrc, const void *b, int32_t k, const void *xbar,
                    void *x, void *dU, double *dmu, ov_tsl_info *info);

/* Reverse mode in two calls, for callers that need x first and the gradient
 * later (an autograd framework): ov_tsl_sign_fwd computes x as ov_tsl_sign
 * does and returns a tape that keeps what the reverse mode needs (the bases or,
 * with options.segment, the segment checkpoints; the recurrence coefficients;
 * every inverse of the Newton iteration of each source's k x k sign: about
 * 48 k^2 complex doubles per source).  ov_tsl_sign_vjp_tape then computes dU
 * and dmu for a cotangent xbar exactly as ov_tsl_sign_vjp would, without
 * repeating the forward recurrence or the Newton iteration; a tape may serve
 * several cotangents.  The tape owns its device memory until ov_tape_destroy;
 * it runs on ctx's stream and must not outlive ctx.  Arguments and errors as
 * ov_tsl_sign / ov_tsl_sign_vjp; on error no tape is returned. */
typedef struct ov_tape ov_tape;
int ov_tsl_sign_fwd(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                    int32_t nsrc, const void *b, int32_t k, void *x, ov_tsl_info *info, ov_tape **tape);
int ov_tsl_sign_vjp_tape(ov_tape *tape, const void *xbar, void *dU, double *dmu, ov_tsl_info *info);
int ov_tape_destroy(ov_tape *tape);

/* One problem of an uneven batch: the arguments of ov_tsl_sign (xbar = NULL)
 * or of ov_tsl_sign_vjp (xbar != NULL) for one lattice, mu and k, and its
 * outputs: info and status (OV_OK or the call's error code). */
typedef struct {
  int32_t dims[4];
  const void *U;
  double mu, m_w;
  int32_t nsrc;
  const void *b;
  int32_t k;
  const void *xbar;           /* NULL: forward only */
  void *x;                    /* forward result (may be NULL with xbar) */
  void *dU;                   /* with xbar: link gradient */
  double *dmu;                /* with xbar: host double */
  ov_tsl_info info;           /* out */
  int32_t status;             /* out */
} ov_problem;

/* Uneven batch (problems on different lattices, mu and k; not in the paper,
 * which treats one problem at a time): the problems run concurrently on
 * nworkers (1..16) worker contexts, each with its own stream and workspace,
 * owned by ctx and kept for later batches; a problem runs exactly as the
 * corresponding single call on a context with ctx's options and tuned stencil
 * variants, so its results equal that call's bit for bit.  The most expensive
 * problems (V k^2 nsrc, VJP twice the forward) are started first.  Work on
 * ctx's stream before the call is ordered before the problems, and the
 * problems before later work on it.  Each worker context allocates workspace
 * for the largest problem it runs.  Returns OV_OK, or the status of the first
 * failed problem in batch order (every problem's status is in probs[i].status). */
int ov_tsl_batch(ov_context *ctx, int32_t nprob, ov_problem *probs, int32_t nworkers);

/* Launch-shape autotuner.  Times every compiled variant of the two stencil
 * kernels -- ov_apply_H (sources per thread x threads per block) and the
 * TSL step's H/H^dagger pair (both products sharing each link load in one
 * thread, or computed one after the other, x threads per block) -- on this
 * lattice, nsrc sources and the context's precision, and keeps the fastest
 * of each in the context for later calls (a variant replaces variant 0, or an
 * earlier pick, only when it is more than 2% faster: variants reduce in
 * different block sizes, so results differ between them at rounding level).
 * U is as in ov_apply_H; the spinor data used for timing is internal
 * scratch.  rep may be NULL. */
typedef struct {
  int32_t apply_variant;    /* chosen variant of the ov_apply_H stencil */
  int32_t pair_variant;     /* chosen variant of the TSL stencil pair */
  int32_t n_apply, n_pair;  /* number of variants timed */
  float apply_us[16];       /* device microseconds per launch, per variant (apply variants 9, 10,
                               11 stage 1, 2 or 4 z-planes of the FP32 input in shared memory) */
  float pair_us[16];
} ov_tune_report;
int ov_autotune(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                int32_t nsrc, ov_tune_report *rep);
/* Select the stencil variants by number for the context's precision (0 is
 * the default; out-of-range numbers are rejected).  For tests and for
 * reusing a tuning result. */
int ov_set_stencil_variants(ov_context *ctx, int32_t apply_variant, int32_t pair_variant);

/* Theorem 1 (Sec. 2, Eq. func_derivative_1): k-step TSL on the block matrix
 *   B = [[H, dH], [0, H]],   dH = d/dt H(U + t E, mu + t m_dir) at t = 0,
 * started from the block vector (top, bottom); out_top and out_bottom receive
 * the two halves of the approximation of sgn(B) (top, bottom), which are
 *   sgn(H) top + (d sgn(H)) bottom   and   sgn(H) bottom.
 * top, bottom, out_top, out_bottom: device arrays of nsrc spinor fields each
 * (complex128, user layout); top may be NULL (zero).  E: device array shaped
 * like U (complex128; NULL for a pure mu direction).  The left Krylov space
 * starts from w_1 proportional to (top + bottom, bottom) with w_1^dag v_1 = 1
 * (the paper does not state it; with w_1 = v_1 = (0, b)/||b|| the left space
 * stays in the lower half and the upper half is not a derivative).  Internal
 * fields are twice as long as in ov_tsl_sign; the re-biorthogonalisation
 * options apply to them.  Errors as ov_tsl_sign. */
int ov_block_tsl_sign(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                      int32_t nsrc, const void *top, const void *bottom, int32_t k, const void *E,
                      double m_dir, void *out_top, void *out_bottom, ov_tsl_info *info);

/* Directional derivative by Theorem 1: ov_block_tsl_sign from (0, b), so
 * dx ~ (d sgn(H)) b along (E, m_dir) and x ~ sgn(H) b. */
int ov_tsl_sign_jvp(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                    int32_t nsrc, const void *b, int32_t k, const void *E, double m_dir, void *dx,
                    void *x, ov_tsl_info *info);

/* Deflation (Sec. 3).  l eigen-triples of H(U, mu) are supplied by the caller:
 * lam (host double[2l], complex interleaved), R and L (device arrays of l
 * spinor fields each, complex128 user layout: right and left eigenvectors,
 * H R_i = lambda_i R_i, L_i^dag H = lambda_i L_i^dag, L_i^dag R_j = delta_ij).
 * The library computes no eigenvectors (the paper obtains them by Arnoldi).
 *
 * ov_tsl_sign_deflated: standard deflation of sgn(H) b,
 *   x = TSL_k(H, Pbar b) + sum_i sgn(Re lambda_i) R_i (L_i^dag b),
 *   Pbar b = b - sum_i R_i (L_i^dag b)
 * (the k-step TSL of ov_tsl_sign on the projected source; b and x: device
 * arrays of nsrc spinor fields).  An eigenvalue with Re lambda_i = 0 exactly
 * is rejected (OV_ERR_SIGN_ILLPOSED).  l = 0 is the plain ov_tsl_sign.  Other
 * errors as ov_tsl_sign; OV_ERR_INVALID_ARG for l < 0, l > 4096, a null or
 * misaligned array (R, L may be NULL only when l = 0). */
int ov_tsl_sign_deflated(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                         int32_t nsrc, const void *b, int32_t k, int32_t l, const double *lam,
                         const void *R, const void *L, void *x, ov_tsl_info *info);

/* Eigen-triples for the deflation from the last forward pass on this context
 * (ov_tsl_sign or ov_tsl_sign_vjp with the same dims, the same k and
 * precision, no segments; the bases V_k, W_k and T_k are still held): the
 * Ritz triples of source src.  The eigenvalues theta of T_k
 * (ov_tridiag_eigenvalues) are taken in order of |theta| (the paper deflates
 * the eigenvalues smallest in absolute value); for up to 2 lmax + 8 of them the
 * right and left eigenvectors y, z of T_k (ov_tridiag_eigenvector, scaled to
 * z^dag y = 1) give R = V_k y and L = W_k z (then L^dag R = 1 while the bases
 * are biorthogonal), and the residual ||H R - theta R|| / ||R|| is computed
 * with one application of H.  Those with residual <= tol are written, in
 * |theta| order: l_out (host) their number (<= lmax), lam (host
 * double[2 lmax]) their theta, R and L (device arrays of lmax spinor fields,
 * complex128 user layout) the vectors, resid (host double[lmax], may be NULL)
 * the residuals.  The paper computes the eigen-triples by Arnoldi (ARPACK);
 * Ritz triples of the TSL's own Krylov space are this library's source (the
 * converged ones are eigen-triples to the stated residual).  U, mu, m_w: as
 * in the forward pass.  Returns OV_OK, OV_ERR_INVALID_ARG (no matching
 * forward pass, lmax < 1, tol <= 0, src out of range), OV_ERR_NOCONV. */
int ov_tsl_ritz_triples(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w, int32_t src,
                        int32_t k, int32_t lmax, double tol, int32_t *l_out, double *lam, void *R, void *L,
                        double *resid);

/* Eigen-triples of H(U, mu) smallest in |lambda|, for the deflation (the
 * paper obtains them by ARPACK's Arnoldi): shift-and-invert Arnoldi, m steps on
 * H^{-1} and m steps on H^{-dag} from the caller's start vector (device, one
 * spinor field), each inversion by conjugate gradients on the normal
 * equations to relative residual tol in at most maxit steps, classical
 * Gram-Schmidt twice per step; the eigenpairs of each m x m Hessenberg matrix
 * (ov_hessenberg_eigen) with the largest |mu| give lambda = 1/mu and the Ritz
 * vectors.  Right and left are paired by eigenvalue (within 1e-6 |lambda|) and
 * L scaled to L^dag R = 1.  Outputs up to l triples in order of |lambda|:
 * l_out (host), lam (host double[2l]), R, L (device arrays of l spinor fields,
 * complex128 user layout), resid (host double[l], may be NULL: ||H R -
 * lambda R|| / ||R||).  FP64 whatever the context's precision.  Needs
 * m >= l (m = 4l to 8l is typical), m <= 1024.  Returns OV_OK, OV_ERR_NOCONV
 * (an inner solve missed tol; results still written), OV_ERR_INVALID_ARG,
 * OV_ERR_NONFINITE. */
int ov_eigen_smallest(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w, int32_t l,
                      int32_t m, const void *start, double tol, int32_t maxit, int32_t *l_out, double *lam,
                      void *R, void *L, double *resid);

/* Eigenvalue and eigenvector derivatives for the generalised deflation (App.
 * B; computed, as App. E does, by shifted inversions), FP64 whatever the
 * context's precision: for the eigen-triples (lam, R, L) of H(U, mu) as in
 * ov_tsl_sign_deflated and the direction (E, m_dir) of ov_block_tsl_sign,
 *   dlambda_i = L_i^dag dH R_i,
 *   (lambda_i - H) dR_i = (1 - R_i L_i^dag)(dH - dlambda_i) R_i,
 *   (conj lambda_i - H^dag) dL_i = (1 - L_i R_i^dag)(dH^dag - conj dlambda_i) L_i,
 * each solved by conjugate gradients on the normal equations (CG on
 * A A^dag with A = lambda_i - H, the paper's App. E choice) to relative
 * residual tol in at most maxit CG steps (two applications of H each), then
 * normalised by L_i^dag dR_i = 0, dL_i^dag R_i = 0.
 * dlam (host double[2l]), dR, dL (device arrays of l spinor fields), resid
 * (host double[2l], may be NULL: the right and left solves' final relative
 * residuals).  Accuracy needs the eigen-triples to be accurate and the
 * eigenvalue separated from the others (the shifted operator's smallest
 * singular value on the complement is about the gap; CG needs about
 * ||H|| / gap steps per digit).  Returns OV_OK,
 * OV_ERR_NOCONV (a solve missed tol; everything is still written),
 * OV_ERR_INVALID_ARG, OV_ERR_NONFINITE. */
int ov_eigen_derivatives(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                         const void *E, double m_dir, int32_t l, const double *lam, const void *R, const void *L,
                         double tol, int32_t maxit, double *dlam, void *dR, void *dL, double *resid);

/* ov_tsl_sign_jvp_deflated: the generalised deflation of Theorem 1's block
 * matrix B = [[H, dH], [0, H]] (Sec. 3, Eqs. x_final, xinv_final,
 * projector_1, final_res), dH along (E, m_dir) as in ov_block_tsl_sign, for
 * the start (0, b): with a_i = L_i^dag b and c_i = dL_i^dag b,
 *   (top', bottom') = (-sum_i (R_i c_i + dR_i a_i), b - sum_i R_i a_i),
 *   (dx, x) = ov_block_tsl_sign(top', bottom')
 *             + sum_i sgn(Re lambda_i) (R_i c_i + dR_i a_i, R_i a_i),
 * the mixing term d sgn(lambda_i) of Eq. final_res being zero.  dR, dL:
 * device arrays of l spinor fields, the derivatives of the eigenvectors along
 * the same direction, normalised by L_i^dag dR_i = 0 and dL_i^dag R_i = 0
 * (App. B).  dx ~ (d sgn(H)) b and x ~ sgn(H) b.  Errors as
 * ov_tsl_sign_deflated and ov_block_tsl_sign. */
int ov_tsl_sign_jvp_deflated(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                             int32_t nsrc, const void *b, int32_t k, const void *E, double m_dir, int32_t l,
                             const double *lam, const void *R, const void *L, const void *dR, const void *dL,
                             void *dx, void *x, ov_tsl_info *info);

/* A-posteriori error estimates of Sec. 4.1.  The sign is applied twice, each
 * time by its own k-step TSL (the second starts from the first's result), and
 * eps[src] (host array of nsrc doubles) receives per source
 *   ov_tsl_eps:        ||sgn(H)^2 b - b|| / (2 ||b||)                (Eq. error_est)
 *   ov_block_tsl_eps:  ||sgn(B)^2 (0, b) - (0, b)|| / (2 ||b||)       (Eq. bA_error_est)
 * with B, E and m_dir as in ov_block_tsl_sign.  The norms are reduced on the
 * device in FP64.  info: k_reached is the smaller, newton_iters the larger of
 * the two runs, t_ms their sums.  Errors as ov_tsl_sign. */
int ov_tsl_eps(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w, int32_t nsrc,
               const void *b, int32_t k, double *eps, ov_tsl_info *info);
int ov_block_tsl_eps(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                     int32_t nsrc, const void *b, int32_t k, const void *E, double m_dir, double *eps,
                     ov_tsl_info *info);

/* Recurrence coefficients of source `src` from the last ov_tsl_sign or
 * ov_tsl_sign_vjp call on this context (k must equal that call's k), copied
 * to HOST arrays: alpha[2k] and beta[2k] interleaved complex, delta[k].
 * alpha_j = T[j][j], beta_j = T[j-1][j], delta_j = T[j][j-1] (0-based j,
 * beta_0 = delta_0 = 0). */
int ov_tsl_coefficients(ov_context *ctx, int32_t src, int32_t k, double *alpha, double *beta,
                        double *delta);

/* Live per-kernel timing.  While enabled, every kernel launch of the library
 * is bracketed by CUDA events on the context's stream and its device time is
 * added to the kind's total when the enclosing call returns.  Kinds: */
#define OV_KIND_STENCIL_PAIR  0  /* TSL step: v_j, w_j, p = H v_j, q = H^dag w_j, alpha_j */
#define OV_KIND_UPDATE        1  /* three-term update r, s and omega */
#define OV_KIND_PROJ_DOTS     2  /* Gram-Schmidt coefficients (dots against the bases + reduction) */
#define OV_KIND_PROJ_UPDATE   3  /* Gram-Schmidt update (basis combination) */
#define OV_KIND_COMBINE       4  /* x = V y and g_y = V^dag xbar */
#define OV_KIND_DENSE         5  /* k x k Newton sign and Frechet adjoint: inverses, updates */
#define OV_KIND_REV_SCALAR    6  /* reverse-sweep dots and scalar steps */
#define OV_KIND_REV_STENCIL   7  /* reverse-sweep stencil pair (H^dag g_p, H g_q) */
#define OV_KIND_FORCE         8  /* link-gradient contraction and dmu */
#define OV_KIND_APPLY_H       9  /* ov_apply_H stencil */
#define OV_KIND_LAYOUT       10  /* layout conversion (complex128 <-> internal) */
#define OV_KIND_DENSE_GEMM   11  /* k x k products of the block Frechet iteration */
#define OV_NKIND             12
int ov_profile_enable(ov_context *ctx, int32_t enable);
/* Self-test of the bounded inter-block wait used by the cooperative k x k
 * inversion (an implementation detail with no counterpart in the paper): two
 * blocks wait on a counter that nothing increments; the first gives up after
 * limit_ns (1 .. 1e8 ns) and flags it, the second, with a 100x longer limit,
 * must leave through that flag.  Returns OV_ERR_TIMEOUT when both left as
 * designed (*elapsed_ms = device time of the launch), OV_ERR_CUDA otherwise.
 * No GPU state outlives the call. */
int ov_selftest_wait(ov_context *ctx, uint64_t limit_ns, double *elapsed_ms);
/* Restrict the timing to the kinds whose bit (1 << OV_KIND_*) is set in
 * kind_mask (all kinds by default): each timed launch group costs two event
 * records on the stream, so a caller timing one kernel kind inside a long run
 * can leave the others untimed. */
int ov_profile_select(ov_context *ctx, uint32_t kind_mask);
/* Totals since the last reset for `kind`: number of timed launches and summed
 * device milliseconds.  reset != 0 clears all kinds after reading. */
int ov_profile_read(ov_context *ctx, int32_t kind, int64_t *launches, double *ms, int32_t reset);
/* Number of kernels this context has launched since it was created. */
int64_t ov_launch_count(ov_context *ctx);

/* Allocation-free H(mu) psi.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory when they apply the
 * operator (a framework allocator that already owns the device memory, an
 * inner loop that cannot afford the device synchronisation of cudaMalloc and
 * cudaFree, a plug-in whose host forbids allocations after start-up).
 * Same operator, arguments and layouts as ov_apply_H, always in FP64, but
 * without a context: the work is enqueued on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and the call returns without waiting for it.
 * Workspace: one file-scope device array of OV_NOALLOC_SCRATCH_BYTES, which
 * every GPU that loads the library holds until the process exits; the call
 * allocates and frees nothing.  It needs (72 V + 2 nsrc ceil64(24 V)) * 8
 * bytes (ceil64 rounds up to a multiple of 64) and returns
 * OV_ERR_SCRATCH_LIMIT when that exceeds the array (nsrc above 4096 is
 * OV_ERR_INVALID_ARG).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  The cached address belongs to the device's
 * primary context: after cudaDeviceReset it is stale, so do not use this
 * entry point in a process that resets a device it has already called it
 * on.  A launch error left pending by earlier work on the calling thread is
 * cleared on entry (cudaGetLastError), so OV_ERR_CUDA always refers to this
 * call's own launches.  All calls share
 * the one array: calls whose work overlaps on the GPU (different streams, or
 * different host threads on one device) race and corrupt each other's
 * results; calls ordered on one stream are safe. */
#define OV_NOALLOC_SCRATCH_BYTES (32u << 20)
int ov_apply_H_noalloc(const int32_t dims[4], const void *U, double mu, double m_w, int32_t nsrc,
                       const void *in, void *out, int32_t dagger, void *stream);

/* Overlap Dirac operator (Sec. 1, Eq. overlap, lattice spacing 1):
 *   dagger = 0: out = D_ov b = b + gamma5 sgn(H(mu)) b
 *   dagger = 1: out = D_ov^dagger b = b + sgn(H(-mu)) gamma5 b
 * (H(mu)^dagger = H(-mu) by gamma5-hermiticity of Eq. WD_op; sgn(H)^dagger =
 * sgn(H^dagger) since sgn(lambda) = sgn(Re lambda) is real), the sign applied
 * by the k-step TSL of ov_tsl_sign with the context's options.  b and out:
 * nsrc spinor fields (device, complex128, user layout); out may equal b.
 * info as ov_tsl_sign (of the TSL run).  Errors as ov_tsl_sign. */
int ov_overlap_apply(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                     int32_t nsrc, const void *b, int32_t k, int32_t dagger, void *out, ov_tsl_info *info);

/* Solve D_ov x = rhs (dagger = 0) or D_ov^dagger x = rhs (dagger = 1) for each of
 * nsrc right-hand sides by restarted GMRES(30) from x = 0, each operator
 * application an ov_overlap_apply with k TSL steps.  The k-step TSL is linear in
 * its vector only up to its approximation error, which bounds the attainable
 * residual.  Stops when ||rhs - D_ov x|| <= tol ||rhs|| (the true residual,
 * recomputed at every restart) or after maxit applications; *iters (largest
 * count over the sources) and *resid (largest final relative residual) may be
 * NULL.  Returns OV_ERR_NOCONV when a source ends above tol (x holds the last
 * iterate), else the errors of ov_tsl_sign. */
int ov_overlap_solve(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w,
                     int32_t nsrc, const void *rhs, int32_t k, int32_t dagger, double tol, int32_t maxit,
                     void *x, int32_t *iters, double *resid);

/* Stochastic estimator of the U(1) vector currents (Sec. 4.3, Eq. lat_vec_cur)
 *   j_{x,nu} = Tr(D_ov^{-1} dD_ov/dTheta_{x,nu})
 * over nnoise noise vectors eta (device, nnoise spinor fields, complex128; Z2
 * noise in the paper): for each, chi = D_ov^{-dagger} eta by ov_overlap_solve
 * (tol, maxit), then eta^dagger D_ov^{-1} (dD_ov/dTheta) eta =
 * <gamma5 chi, d(sgn(H) eta)/dTheta> for all links at once from one forward TSL
 * and two reverse sweeps (the VJP of ov_tsl_sign_vjp with cotangents gamma5 chi
 * and i gamma5 chi), where Theta enters as U_nu(x) -> e^{i Theta_{x,nu}} U_nu(x).
 * j: device array [V][4] of complex128 (direction order x, y, z, t), the mean
 * over the noise vectors.  trace_mu (host double[2], may be NULL): the same
 * estimator of Tr(D_ov^{-1} dD_ov/dmu) (real, imaginary part).  The divergence
 * sum_nu (j_{x,nu} - j_{x-nu,nu}) of the exact trace vanishes (Eq.
 * divergence_def); the estimator reaches it on average.  Errors as
 * ov_overlap_solve. */
int ov_u1_current(ov_context *ctx, const int32_t dims[4], const void *U, double mu, double m_w, int32_t nnoise,
                  const void *eta, int32_t k, double tol, int32_t maxit, void *j, double *trace_mu,
                  ov_tsl_info *info);

/* The k x k stage of the TSL on one tridiagonal T, on the device: y = beta0 f,
 * with f = sgn(T) e_1 by the scaled Newton iteration on T when m = 0 (the
 * stage of ov_tsl_sign without nesting), or, for m > 0, the nested
 * approximation of Sec. 4.1 (one nesting level, inner Krylov size m):
 *   S = (T + T^{-1})/2 (dense; T^{-1} from an LU of T with partial pivoting),
 *   m steps of Arnoldi on S from e_1 (classical Gram-Schmidt twice),
 *   S Q_m = Q_m H_m + h q e_m^T,  f = Q_m sgn(H_m) e_1,
 * sgn(H_m) by the same Newton iteration; m >= k, or a Krylov space of S that
 * closes early (a residual <= 1e-14 ||S q_j||), gives f = sgn(T) e_1 up to
 * rounding.  Host arrays as ov_tsl_coefficients writes them: alpha[2k],
 * beta[2k] interleaved complex (alpha_j = T[j][j], beta_j = T[j-1][j],
 * beta_0 unused), delta[k] (delta_j = T[j][j-1], delta_0 unused); y (host
 * double[2k], interleaved complex); newton_iters (may be NULL) receives the
 * Newton iteration count.  Uses the context's workspace and stream; of the
 * options only newton applies, and dense for m = 0 (the nested form inverts
 * its m x m matrices in the step form, which is faster at these sizes and
 * gives the same bits).  2 <= k <= 4096,
 * 0 <= m <= OV_NESTED_MAX.  Returns OV_OK, OV_ERR_INVALID_ARG,
 * OV_ERR_SIGN_ILLPOSED (T singular, a non-finite entry, or the Newton
 * iteration failed), OV_ERR_OOM, OV_ERR_CUDA. */
int ov_tridiag_sign_nested(ov_context *ctx, int32_t k, const double *alpha, const double *beta,
                           const double *delta, int32_t m, double beta0, double *y, int32_t *newton_iters);

/* Eigenvalues of one TSL tridiagonal T_k (the Ritz values), on the host: no
 * GPU and no context needed.  Host arrays as ov_tsl_coefficients writes them:
 * alpha[2k] and beta[2k] interleaved complex (alpha_j = T[j][j],
 * beta_j = T[j-1][j], beta_0 unused), delta[k] (delta_j = T[j][j-1]).  The
 * off-diagonal pairs must satisfy |beta_j| = |delta_j| (the TSL's split of
 * omega); eig[2k] receives the eigenvalues, interleaved complex, unordered.
 * Method: diagonal similarity to a complex-symmetric tridiagonal and implicit
 * QL iteration with complex-orthogonal rotations, O(k^2).  Returns OV_OK,
 * OV_ERR_INVALID_ARG, OV_ERR_NONFINITE (a non-finite entry) or OV_ERR_NOCONV
 * (no convergence, or a rotation that would break down). */
int ov_tridiag_eigenvalues(int32_t k, const double *alpha, const double *beta, const double *delta,
                           double *eig);

/* One eigenvector of the same T_k, on the host: the right eigenvector
 * (T_k y = theta y; left = 0) or the left one (z^dag T_k = theta z^dag, i.e.
 * T_k^dag z = conj(theta) z; left = 1) for the eigenvalue theta (host
 * double[2]), by three steps of inverse iteration with a pivoted tridiagonal
 * solve (Wilkinson, The Algebraic Eigenvalue Problem, ch. 9), O(k).  vec
 * (host double[2k], interleaved complex) receives it with unit 2-norm.  theta
 * should be an eigenvalue of T_k to working accuracy (e.g. from
 * ov_tridiag_eigenvalues); a nearby value gives the eigenvector of the nearest
 * eigenvalue.  Returns OV_OK, OV_ERR_INVALID_ARG, OV_ERR_NONFINITE or
 * OV_ERR_NOCONV (a solve overflowed). */
int ov_tridiag_eigenvector(int32_t k, const double *alpha, const double *beta, const double *delta,
                           const double *theta, int32_t left, double *vec);

/* Eigenvalues (and, with vecs non-NULL, right eigenvectors) of a complex upper
 * Hessenberg matrix on the host: h (host double[2 m^2], row-major,
 * interleaved complex; entries below the subdiagonal must be zero), eig (host
 * double[2m]), vecs (host double[2 m^2], row-major, column i the unit
 * eigenvector of eig[i]).  Implicit single-shift QR with Wilkinson and
 * exceptional shifts (Golub and Van Loan, Matrix Computations, ch. 7.5), then
 * three steps of inverse iteration per eigenvector with a pivoted LU; O(m^3),
 * for the Arnoldi matrices of ov_eigen_smallest.  Returns OV_OK,
 * OV_ERR_INVALID_ARG (m out of 1..4096, not Hessenberg), OV_ERR_NONFINITE,
 * OV_ERR_NOCONV. */
int ov_hessenberg_eigen(int32_t m, const double *h, double *eig, double *vecs);

/* One complex k x k product of the kind the Frechet adjoint's iteration forms
 * (Theorem 1: X_i^{-H} E X_i^{-H} and sgn(T)^H E sgn(T)^H):
 * C = op(A) op(B), op = identity (flag 0) or conjugate transpose (flag 1).
 * A, B, C: device arrays of k x k complex128, row-major, interleaved
 * (re, im), 16-byte aligned; C must not overlap A or B.  mode 1: FP64
 * arithmetic; mode 2: the BF16 tensor-core form of options.gemm (exact digit
 * splitting; k <= 1024).  Runs on the context's stream and returns when the
 * product is complete.  Returns OV_OK, OV_ERR_INVALID_ARG (k < 1, mode not 1
 * or 2, mode 2 with k > 1024, a null or misaligned pointer), OV_ERR_OOM
 * (workspace) or OV_ERR_CUDA (a launch or cuBLAS failure). */
int ov_kk_gemm(ov_context *ctx, const void *A, int32_t hA, const void *B, int32_t hB, void *C, int32_t k,
               int32_t mode);

/* Host-side fault injection for tests of error propagation (no GPU fault is
 * caused: the library writes an ordinary value, or fails an allocation, on
 * the host's initiative).  One-shot: the injection fires once in the next
 * call that reaches it on this context, then clears.  The paper has no
 * counterpart.  Kinds: */
#define OV_INJECT_NONE        0
#define OV_INJECT_BREAKDOWN   1  /* after the three-term update of Lanczos step `step` (0-based),
                                    source 0 is flagged as broken down, as the update kernel flags
                                    |omega| <= 1e-14 ||r|| ||s||; the call returns OV_ERR_BREAKDOWN */
#define OV_INJECT_NONFINITE   2  /* after the stencil of step `step`, alpha_step of source 0 is set
                                    to NaN; the update kernel then flags a non-finite omega and the
                                    call returns OV_ERR_NONFINITE */
#define OV_INJECT_OOM         3  /* the workspace allocation after the next `step` successful ones
                                    fails as cudaMalloc would; the call returns OV_ERR_OOM and the
                                    context stays usable */
int ov_debug_inject(ov_context *ctx, int32_t kind, int32_t step);

/* Human-readable text for a status code (static storage). */
const char *ov_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* OV_H */
