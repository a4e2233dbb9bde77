/*
 * rsrr.h -- C ABI of the GB300 resolvent-sampling Rayleigh-Ritz (RSRR) library.
 *
 * The library computes the hot path of RSRR (Xiao, Meng, Zhang, Zheng,
 * arXiv:1510.07522) on one CUDA device:
 *
 *   rsrr_create_nep  T(z) = sum_i f_i(z) A_i over one sparsity pattern (Eq. eq-Z-expr)
 *   rsrr_sample      S_hat = [T(z_0)^{-1} U, ..., T(z_{N-1})^{-1} U]     (Eq. eq-hatS,
 *                    Algorithm 2 Steps 1-2) by band LU + L-column solves
 *   rsrr_project     truncated SVD of S_hat (Algorithm 2 Step 3), then
 *                    P_i = S^H A_i S                                      (Eq. eq-Zs-expr)
 *   rsrr_solve       modified block Sakurai-Sugiura on T_S(z) = sum_i f_i(z) P_i
 *                    (Algorithm 1) and the back-map v = S g (Algorithm 2 Step 5)
 *
 * Conventions shared by every call:
 *   - Complex numbers are interleaved (re, im) pairs of doubles.
 *   - Matrices are column-major.  Vectors and matrices that the caller passes or
 *     receives are in the caller's row ordering; the band ordering the library
 *     chooses internally is invisible.
 *   - Host pointers unless a flag says otherwise.  Every input is copied before
 *     the call returns; the caller keeps ownership of all its buffers.
 *   - Every call is synchronous with respect to the host: when it returns, its
 *     device work on the handle's stream has completed.
 *   - Return value 0 on success, a negative RSRR_E* code on failure; the text of
 *     the last failure on the calling thread is available from rsrr_last_error().
 *   - One handle must not be used by two host threads at the same time.
 */
#ifndef RSRR_H
#define RSRR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define RSRR_OK              0
#define RSRR_EINVAL         -1  /* bad argument (size, pointer, kind, flag)               */
#define RSRR_ENOMEM         -2  /* device allocation failed or exceeds the memory budget  */
#define RSRR_ESINGULAR      -3  /* exactly zero pivot in some T(z_j): z_j is an eigenvalue */
#define RSRR_ENOTCONVERGED  -4  /* iterative refinement did not reach the tolerance       */
#define RSRR_ENONFINITE     -5  /* NaN or Inf in the inputs or in a result                */
#define RSRR_ETIMEOUT       -6  /* a bounded device-side wait gave up                     */
#define RSRR_ECUDA          -7  /* a CUDA runtime call failed                             */
#define RSRR_EORDER         -8  /* calls out of order (sample -> project -> solve)        */
#define RSRR_EUNSUPPORTED   -9  /* the problem's band is wider than the band kernels take */

/* ---- scalar functions f_i of T(z) = sum_i f_i(z) A_i (Eq. eq-Z-expr) ----------------- */
typedef enum {
    RSRR_F_CONST = 0,       /* f = 1                                                     */
    RSRR_F_Z = 1,           /* f = z                                                     */
    RSRR_F_Z2 = 2,          /* f = z^2                                                   */
    RSRR_F_ISQRT_SHIFT = 3, /* f = i sqrt(z - p0); p1 = 0: principal root,
                               p1 = 1: continued branch -sqrt(p0 - z), holomorphic off
                               [p0, +inf) (gun-type problems, Section 7.2)               */
    RSRR_F_EXP_DELAY = 4,   /* f = exp(-p0 z)                                            */
    RSRR_F_RATIONAL = 5,    /* f = p0 z / (z + p1)  (Biot / loaded-string terms)         */
    RSRR_F_CALLBACK = 6,    /* f and f' from the caller's function `cb` (any analytic f) */
    RSRR_F_CHEBYSHEV = 7    /* f = tau_m((2z - p1 - p2) / (p2 - p1)), the Chebyshev polynomial
                               of the first kind of degree m = p0 (an integer, 0..1024) on the
                               interval [p1, p2], p1 < p2 (Section 6.2, Eq. eq-T-interp)   */
} rsrr_fkind;

/* Caller-supplied scalar function (RSRR_F_CALLBACK): for k < m, write f(z_k) and f'(z_k) to
 * f_reim[2k..2k+1] and df_reim[2k..2k+1] (z_reim[2k] + i z_reim[2k+1]).  It must be analytic
 * inside and on the contour (Section 6: T(z) = sum_i f_i(z) A_i); f' is used by the winding
 * number (Eq. eq-ncs).  Called on the host, from the thread that runs rsrr_sample / rsrr_solve,
 * for as long as the handle lives. */
typedef void (*rsrr_fn_cb)(void* user, int64_t m, const double* z_reim, double* f_reim, double* df_reim);

typedef struct {
    int32_t kind;           /* an rsrr_fkind                                             */
    int32_t reserved;       /* must be 0                                                 */
    double p[4];            /* parameters, meaning per kind above                        */
    rsrr_fn_cb cb;          /* RSRR_F_CALLBACK: the function; otherwise ignored (NULL)   */
    void* user;             /* passed to cb unchanged                                    */
} rsrr_fn;

/* The contour C enclosing the wanted eigenvalues, and the quadrature rule on it.
 *   RSRR_CONTOUR_ELLIPSE    phi(t) = gamma + a cos t + i b sin t (Eq. eq-contour); N points at the
 *                           trapezoid nodes t_j = 2 pi (j + 1/2) / N (Eq. eq-Ap-num).
 *   RSRR_CONTOUR_RECTANGLE  the rectangle gamma + [-a, a] + i [-b, b], run counter-clockwise from
 *                           its lower-left corner (bottom, right, top, left side), with a
 *                           Gauss-Legendre rule on each side (Section 7.2, the gun example).  N is
 *                           even; each horizontal side gets side_nodes points and each vertical
 *                           side N/2 - side_nodes (the paper's "10-5" for N = 30 is side_nodes =
 *                           10 when a > b).  side_nodes = 0 splits in proportion to the side
 *                           lengths; rsrr_solve always splits its N_S points that way.
 * A zero-initialised struct with gamma, a, b set is an ellipse. */
#define RSRR_CONTOUR_ELLIPSE   0
#define RSRR_CONTOUR_RECTANGLE 1
typedef struct {
    double gamma_re, gamma_im;  /* centre                                                  */
    double a, b;                /* semi-axes (ellipse) or half-sides (rectangle), both > 0  */
    int32_t shape;              /* RSRR_CONTOUR_ELLIPSE or RSRR_CONTOUR_RECTANGLE           */
    int32_t side_nodes;         /* rectangle: points per horizontal side (0 = proportional) */
} rsrr_contour;

/* precision of the sample solves (rsrr_sample) */
#define RSRR_FP64     0  /* complex128 band LU and solves                                */
#define RSRR_C64_IR   1  /* complex64 band LU and solves, FP64 residual and refinement   */
/* flag OR-ed into precision: keep refining every point while its worst eta still halves per
 * sweep (working accuracy), not only until eta <= tol; acceptance is still eta <= tol */
#define RSRR_REFINE_FULL 0x100

/* flags of rsrr_create_nep */
#define RSRR_NATURAL_ORDER 0x1u  /* keep the caller's ordering (skip the band reordering) */
#define RSRR_DENSE_LU      0x2u  /* factor every sampling point with the dense LU, whatever the
                                    band (otherwise chosen when the band is wider than 768 or
                                    than 2n/5 for n >= 128) */
#define RSRR_AUTOTUNE      0x8u  /* before the first sampling, time the sampler strategies on one
                                    sampling point and keep the fastest that meets the tolerance:
                                    band LU on the tensor cores, band LU on the CUDA cores, the
                                    dense LU, or the iterative sampler (GMRES preconditioned by the
                                    factor of the band part holding all but 1e-12 of the weight of
                                    T(z_0)); decisions are cached process-wide per size bucket
                                    (rsrr_info.tune_*).  Overrides the flags and the band
                                    preconditioner set before that sampling. */
#define RSRR_BAND_CUDA_CORES 0x4u  /* complex64 band LU on the CUDA cores for every band (otherwise
                                    bands with 32 <= kl <= 224 run their trailing updates on the
                                    tensor cores, with the forward solve on the stored
                                    inv(L11), L21 inv(L11) panel blocks) */

typedef struct rsrr_nep_s* rsrr_nep;

/* ---- rsrr_create_nep ------------------------------------------------------------------
 * Build a handle for T(z) = sum_{i<J} f_i(z) A_i (Eq. eq-Z-expr, Section 6).
 *   n         order of T (n >= 1)
 *   J         number of terms (1 <= J <= 16)
 *   rowptr    [n+1] CSR row pointers of the union pattern of all A_i (rowptr[0] = 0)
 *   colind    [nnz] column indices, each row's entries strictly increasing
 *   vals_reim [J][nnz][2] values of A_i on the union pattern (zeros where A_i has none)
 *   f         [J] the functions f_i
 *   flags     0, or RSRR_NATURAL_ORDER, RSRR_DENSE_LU, RSRR_BAND_CUDA_CORES, RSRR_AUTOTUNE
 *   stream    cudaStream_t on which all device work of this handle runs (NULL = default)
 *   out       receives the handle
 * The library picks a row/column ordering (reverse Cuthill-McKee, or the natural one if
 * its band is no wider) and uploads the pattern and values to the device.
 * Errors: EINVAL (bad sizes/pattern/kind), ENONFINITE (NaN/Inf value), ENOMEM, ECUDA. */
int rsrr_create_nep(int64_t n, int32_t J, const int64_t* rowptr, const int32_t* colind,
                    const double* vals_reim, const rsrr_fn* f, uint32_t flags,
                    void* stream, rsrr_nep* out);

/* ---- rsrr_create_nep_tz ---------------------------------------------------------------
 * A handle for a T(z) known only through its values (Section 6: T need not be affine, e.g. a
 * BEM matrix whose entries depend on z through the kernel).  The library calls
 *   tz(user, m, z_reim, vals_reim)
 * on the host to get T(z_k) on the fixed pattern for m points at once:
 *   z_reim    [m][2] the points
 *   vals_reim [m][nnz][2] to fill, entry order of rowptr/colind (the caller's ordering)
 * It is called for the sampling points (rsrr_sample), the Chebyshev points
 * (rsrr_project_chebyshev) and the eigenvalues (the residuals of rsrr_solve), from the thread
 * that makes those calls, for as long as the handle lives.  Such a handle is projected with
 * rsrr_project_chebyshev only (there are no A_i for rsrr_project or rsrr_project_moments).
 * Arguments otherwise as rsrr_create_nep.
 * Errors: EINVAL (NULL tz, bad pattern), ENOMEM, ECUDA; later calls report ENONFINITE if tz
 *         returns a non-finite value. */
typedef void (*rsrr_tz_cb)(void* user, int64_t m, const double* z_reim, double* vals_reim);
int rsrr_create_nep_tz(int64_t n, const int64_t* rowptr, const int32_t* colind, rsrr_tz_cb tz, void* user,
                       uint32_t flags, void* stream, rsrr_nep* out);

/* ---- rsrr_sample ----------------------------------------------------------------------
 * Algorithm 2, Steps 1-2: for j = 0..N-1, z_j = phi(2 pi (j + 1/2) / N), factor T(z_j)
 * by LU with partial pivoting (band LU, or dense LU when the band is too wide to pay: see
 * RSRR_DENSE_LU) and solve T(z_j) X_j = U; S_hat = [X_0 ... X_{N-1}] (Eq. eq-hatS,
 * n x N*L) stays on the device.
 *   C          contour
 *   N, L       sampling points (1..4096) and probing columns (1..256)
 *   U_reim     [L][n][2] the probing matrix U (n x L, column-major, caller ordering);
 *              NULL reuses the U of the previous rsrr_sample on this handle (same n, L)
 *   precision  RSRR_FP64 or RSRR_C64_IR, optionally | RSRR_REFINE_FULL
 *   tol        backward-error target per column,
 *              eta = ||u - T x||_2 / (||T||_1 ||x||_2 + ||u||_2) <= tol  (e.g. 1e-10)
 *   max_refine refinement sweeps allowed in RSRR_C64_IR (ignored for RSRR_FP64), 0..100; after
 *              rsrr_set_band_preconditioner the budget of Krylov iterations, 0..100000
 * Errors: EINVAL, ESINGULAR (a zero pivot: some z_j is an eigenvalue),
 *         ENOTCONVERGED (eta > tol after max_refine sweeps, or > tol in FP64),
 *         ENONFINITE, ENOMEM, ECUDA. */
int rsrr_sample(rsrr_nep h, const rsrr_contour* C, int32_t N, int32_t L,
                const double* U_reim, int32_t precision, double tol, int32_t max_refine);

/* ---- rsrr_set_band_preconditioner -----------------------------------------------------
 * An iterative sampler for NEPs whose full band is too wide to factor but whose dominant part
 * is banded (Section 7.3 solves such systems iteratively: GMRES preconditioned by an incomplete
 * factorisation).  With band >= 0, the following rsrr_sample / rsrr_sample_points /
 * rsrr_sample_batch calls factor only the entries of T(z_j) with |i - j| <= band (in the
 * handle's ordering: pass RSRR_NATURAL_ORDER at creation to keep the caller's) and solve
 * T(z_j) X = U by restarted flexible GMRES in FP64 (restart length up to 30, fewer when device
 * memory is short), right-preconditioned by that factor (complex64 in RSRR_C64_IR, complex128 in
 * RSRR_FP64), starting from X = M^{-1} U.  Every (point, column) system iterates until its
 * residual estimate gives eta <= tol / 2 (eta ~ 2e-16 with RSRR_REFINE_FULL); max_refine is the
 * budget of preconditioned products over all restarts, after which a column with eta > tol fails
 * the call with ENOTCONVERGED.  band = -1 turns it off (the default: the full band, or the dense
 * LU).  It overrides RSRR_DENSE_LU.
 * Errors: EINVAL (NULL handle, band < -1 or >= n). */
int rsrr_set_band_preconditioner(rsrr_nep h, int32_t band);

/* ---- rsrr_sample_points ---------------------------------------------------------------
 * rsrr_sample at sampling points the caller chooses.  The sampling scheme needs only the
 * solutions T(z_j)^{-1} U at some points z_j (Eq. eq-hatS): nothing ties them to a quadrature
 * rule on the contour, and points inside the contour can serve too (Section 3.2).  The contour C
 * is still the one Algorithm 1 integrates over in rsrr_solve.
 *   C           contour used by rsrr_solve (and for nothing else here)
 *   N, z_reim   the N sampling points, [N][2] (re, im); none may be an eigenvalue
 *   L, U_reim, precision, tol, max_refine   as in rsrr_sample
 * rsrr_project_moments refuses a handle sampled this way (its weights are the contour's).
 * Errors: as rsrr_sample; EINVAL also for a NULL or non-finite point. */
int rsrr_sample_points(rsrr_nep h, const rsrr_contour* C, int32_t N, const double* z_reim, int32_t L,
                       const double* U_reim, int32_t precision, double tol, int32_t max_refine);

/* ---- rsrr_sample_batch ----------------------------------------------------------------
 * rsrr_sample on `count` handles in one call (Algorithm 2, Steps 1-2 for a batch of NEPs).
 * The points of every NEP that takes the dense LU go into one persistent launch (one CTA per
 * point at a time, largest n first, each CTA in a memory slot of its own) on the stream of the
 * first such handle, ordered after the work already queued on the other handles' streams;
 * banded NEPs run one after another on the band path, each on its own stream.  Each handle
 * afterwards holds its own S_hat, exactly as after its own rsrr_sample, and goes on to
 * rsrr_project / rsrr_solve independently (on its own stream, so several can run at once).
 * Returns after all of it has completed.
 *   hs          [count] distinct handles, all created on the same device
 *   C, N, L     [count] contour, sampling points and probing columns per handle
 *   U_reim      [count] probing matrices as in rsrr_sample (an entry, or U_reim itself, may
 *               be NULL to reuse each handle's resident U)
 *   precision, tol, max_refine   as in rsrr_sample, shared by all handles
 * Errors: as rsrr_sample (the first failing handle's); EINVAL also for mixed devices or a
 * repeated handle.  After an error no handle of the batch counts as sampled. */
int rsrr_sample_batch(rsrr_nep* hs, int32_t count, const rsrr_contour* C, const int32_t* N,
                      const int32_t* L, const double* const* U_reim, int32_t precision,
                      double tol, int32_t max_refine);

/* ---- rsrr_project ---------------------------------------------------------------------
 * Algorithm 2 Step 3 and Eq. eq-Zs-expr: S_hat = Q R (Householder, FP64), R = W Sigma
 * Y^H (one-sided Jacobi, FP64); keep the k_S singular values sigma_k > delta sigma_1;
 * S = Q W[:, :k_S]; P_i = S^H A_i S for every term.  Requires a successful rsrr_sample.
 *   delta   truncation threshold (the paper uses 1e-14)
 *   k_S_out receives k_S
 * Errors: EORDER, EINVAL, ENOMEM, ECUDA, ENONFINITE. */
int rsrr_project(rsrr_nep h, double delta, int32_t* k_S_out);

/* ---- rsrr_project_moments -------------------------------------------------------------
 * rsrr_project with the moment scheme of SSRR (Section 3.1) in place of the sampling scheme:
 * Step 3 factors M_hat = [M_0 ... M_{K'-1}] (Eq. eq-hatM), the quadrature moments
 * M_alpha = sum_i w_i zeta_i^alpha T(z_i)^{-1} U of the samples already on the device
 * (Eq. eq-malpha-qud, trapezoid weights w_i = phi'(theta_i) / (i N) of the contour), i.e.
 * M_hat = S_hat D Z (Eq. eq-hatMS).  zeta_i = (z_i - gamma) / max(a, b): the shifted and scaled
 * monomials span the same space as z_i^alpha.  Everything after (truncation at delta, P_i,
 * rsrr_solve) is unchanged, so the two schemes can be compared on the same samples.
 *   Kp       moment order K', 1 <= K' <= N (K' = N spans the same space as S_hat when Z has
 *            full rank)
 * Errors: as rsrr_project; EINVAL for K' outside 1..N. */
int rsrr_project_moments(rsrr_nep h, int32_t Kp, double delta, int32_t* k_S_out);

/* ---- rsrr_project_chebyshev ------------------------------------------------------------
 * rsrr_project (Step 3: S from the truncated SVD), then the reduced NEP is replaced by its
 * Chebyshev interpolant of degree d on the real interval [x_lo, x_hi] (Section 6.2,
 * Eqs. eq-T-interp, eq-Ts-interp, eq-Ts-coefs):
 *   x_k = c + r cos(theta_k), theta_k = (k + 1/2) pi / (d + 1), k = 0..d, c, r the interval's
 *   centre and half-width;  P_hat_j = (2 / (d + 1)) sum_k [S^H T(x_k) S] cos(j theta_k), with
 *   P_hat_0 halved (the standard first-kind interpolant: it reproduces every polynomial of
 *   degree <= d);  T_S(z) ~ sum_j P_hat_j tau_j((z - c) / r).
 * rsrr_solve then runs Algorithm 1 on this polynomial NEP; its residuals ||T(lambda) v|| are
 * still those of the true T.  rsrr_get_projected returns the d + 1 matrices P_hat_j and
 * rsrr_info.red_terms is d + 1.  Useful when T is costly to project term by term (a BEM
 * matrix) or has many terms; the interpolation error decays exponentially in d when T is
 * holomorphic near the interval.
 *   d           degree, 0 <= d <= 256
 *   x_lo, x_hi  the interval, x_lo < x_hi (typically the contour's extent on the real axis)
 * For a handle from rsrr_create_nep_tz, S^H T(x_k) S is formed from the values T(x_k)
 * (SpMM, then ZGEMM), exactly as Eq. eq-Ts-coefs writes it.
 * Errors: as rsrr_project; EINVAL for bad d or interval, ENONFINITE if some f_i (or T) is
 *         not finite at a Chebyshev point. */
int rsrr_project_chebyshev(rsrr_nep h, int32_t d, double x_lo, double x_hi, double delta, int32_t* k_S_out);

/* ---- rsrr_solve -----------------------------------------------------------------------
 * Algorithm 1 on T_S(z) = sum_i f_i(z) P_i with the same contour as rsrr_sample:
 * moments A_alpha (Eq. eq-Ap-num, rho = max(a, b)), block Hankel H, H^< (Eq. eq-HH),
 * SVD of H, nbar from the winding number (Eq. eq-ncs) and the singular-value gap
 * (Eq. eq-gap, gaps over the whole SVD), A = V_0^H H^< W_0 Sigma_0^{-1} (Eq. eq-A), its
 * eigenpairs, lambda = rho lambda' + gamma, g (Eq. eq-eigens); then v = S g / ||S g||
 * (Algorithm 2 Step 5) and the residual ||T(lambda) v||_2 (||v|| = 1, Section 7.1).
 * The quadrature is the contour's rule with N_S points (trapezoid on an ellipse,
 * Gauss-Legendre on a rectangle's sides, split in proportion to the side lengths).
 * Only eigenvalues strictly inside the contour are returned, sorted by |lambda|.
 *   N_S, K      quadrature points (even for a rectangle) and Hankel block count (the paper:
 *               500..1000, 2..8)
 *   tol_gap     gap acceptance threshold (the paper: 1e3)
 *   cap         capacity of the output arrays
 *   lambda_reim [cap][2] eigenvalues
 *   V_reim      [cap][n][2] unit eigenvectors (caller ordering), or NULL
 *   resid       [cap] residuals ||T(lambda) v||_2, or NULL
 *   nC_out      receives the number of eigenvalues returned (<= cap)
 * Errors: EORDER, EINVAL (cap too small: nC_out still holds the count), ESINGULAR
 *         (T_S(z) singular at a quadrature point), ENOMEM, ECUDA, ENONFINITE. */
int rsrr_solve(rsrr_nep h, int32_t N_S, int32_t K, double tol_gap, int32_t cap,
               double* lambda_reim, double* V_reim, double* resid, int32_t* nC_out);

/* ---- rsrr_zgemm (diagnostics) ----------------------------------------------------------
 * The library's complex GEMM on caller device memory, C = alpha op(A) op(B) + beta C for each
 * of `batch` problems (column-major, complex128 as [2] doubles; op 0 = as stored, 1 =
 * transpose, 2 = conjugate transpose; sA, sB, sC element strides between problems).  It is
 * the GEMM the projection and the reduced solve use, exported to test its two paths against a
 * reference: path 0 = chosen by shape (as inside the library), 1 = FP64 on the CUDA cores,
 * 2 = FP64-accurate emulation on the tensor cores (exact BF16 digit products with FP32
 * accumulation, combined in FP64) for any shape.  Runs on `stream` (NULL = default) and
 * returns after the work is queued, or after it finished for path 2.  The paper has no
 * counterpart (it leaves dense algebra to its host libraries).
 * Errors: EINVAL (bad sizes, op or path), ENOMEM, ETIMEOUT (a tensor-core wait gave up), ECUDA. */
int rsrr_zgemm(int32_t path, int32_t opA, int32_t opB, int32_t M, int32_t N, int32_t K, const double* alpha_reim,
               const void* A, int64_t lda, int64_t sA, const void* B, int64_t ldb, int64_t sB,
               const double* beta_reim, void* C, int64_t ldc, int64_t sC, int32_t batch, void* stream);

/* ---- rsrr_zinv_batch (diagnostics) -----------------------------------------------------
 * The reduced solve's matrix inverse on caller device memory: A (batch x [k][k], column-major,
 * complex128 as [2] doubles, consecutive matrices) is replaced by its inverse, computed by
 * blocked Gauss-Jordan elimination with partial pivoting (Algorithm 1 needs T_S(z_j)^{-1} in
 * full for the moments of Eq. eq-Ap-num).  Its rank-b updates run on rsrr_zgemm's `path` (as
 * there).  info (device, batch int32) is zeroed here and set to 1 for a matrix that met an
 * exactly zero pivot column (its result is then meaningless).  Runs on `stream` (NULL = the
 * default stream) and returns after the work finished.
 * Errors: EINVAL (bad sizes or path), EUNSUPPORTED (k above the panel limit, about 1600),
 *         ENOMEM, ETIMEOUT, ECUDA. */
int rsrr_zinv_batch(int32_t path, int32_t k, int32_t batch, void* A, int32_t* info, void* stream);

/* ---- introspection (tests, diagnostics) ------------------------------------------------ */
typedef struct {
    int64_t n, nnz;
    int32_t J, N, L;
    int32_t kl, ku;             /* band of the chosen ordering                             */
    int32_t natural_order;      /* 1 if the caller's ordering was kept                     */
    int32_t precision;
    int32_t refine_sweeps;      /* refinement sweeps run by the last rsrr_sample           */
    int32_t k_S;                /* after rsrr_project, else -1                             */
    int32_t nbar;               /* after rsrr_solve (before the inside filter), else -1    */
    int32_t n_winding, n_gap;   /* after rsrr_solve: the two counts (n_gap -1: no gap)     */
    double winding_re, winding_im;
    double max_eta;             /* max backward error over all N*L columns                 */
    double ms_sample, ms_project, ms_solve;  /* device time of the last calls              */
    int64_t device_bytes;       /* device memory held by the handle                        */
    double ms_factor;           /* device time of the LU launches of the last rsrr_sample (after
                                   rsrr_sample_batch: of all dense-LU launches of the batch)   */
    double ms_trsv;             /* device time of its triangular-solve launches              */
    int32_t factor_launches;    /* LU launches in the last rsrr_sample                       */
    int32_t trsv_launches;      /* forward + backward solve launches in the last rsrr_sample */
    int32_t rows_kept;          /* rows of R kept by rsrr_project's early-stopped QR         */
    int32_t jacobi_sweeps_project, jacobi_sweeps_solve;  /* sweeps of the two Jacobi SVDs  */
    double ms_project_qr, ms_project_svd, ms_project_basis, ms_project_gemm;  /* rsrr_project parts */
    double ms_solve_inverse, ms_solve_svd, ms_solve_extract;  /* rsrr_solve parts: reduced inverses
                                   with moments and traces; Hankel SVD; count, eig, back-map */
    double ms_zgemm;            /* device time of the FP64 complex GEMMs of the last project + solve */
    double zgemm_gflop;         /* their algorithmic work, 8 M N K per product, in GFLOP          */
    int32_t dense_lu;           /* 1 if the last rsrr_sample factored with the dense LU            */
    int32_t red_terms;          /* terms of the reduced NEP: J, or d + 1 after
                                   rsrr_project_chebyshev                                   */
    int32_t proj_cols;          /* columns of the matrix the last projection factored: N*L
                                   (rsrr_project) or K'*L (rsrr_project_moments)                 */
    double ms_zgemm_tc;         /* the part of ms_zgemm spent in the tensor-core emulation       */
    double zgemm_tc_gflop;      /* and its algorithmic work (8 M N K per product), GFLOP        */
    double ms_jacobi;           /* device time of the one-sided Jacobi sweeps (project + solve)  */
    double jacobi_gflop;        /* their algorithmic work: per sweep and column pair of an mb-row
                                   matrix, 40 mb real flops (+ 24 k for the accumulated rotations) */
    int32_t band_lu_tc;         /* 1 if the last rsrr_sample ran the complex64 band LU with its
                                   trailing updates on the tensor cores (kl in [32, 224])     */
    int32_t tune_strategy;      /* RSRR_AUTOTUNE's choice: 0 band LU (tensor cores), 1 band LU
                                   (CUDA cores), 2 dense LU, 3 iterative sampler; -1 untuned */
    int32_t tune_band;          /* the iterative sampler's band half-width it chose, else -1   */
    int32_t tune_cached;        /* 1 if the choice came from the cache of a similar NEP        */
    int32_t iterative_band;     /* the band preconditioner in force (-1: direct solves)       */
} rsrr_info;

int rsrr_get_info(rsrr_nep h, rsrr_info* out);
/* Column blocks j0..j1-1 of S_hat, n x (j1-j0)*L, caller ordering, into host memory. */
int rsrr_get_samples(rsrr_nep h, int32_t j0, int32_t j1, double* out_reim);
/* Backward errors eta of all N*L columns (column jL + l is point j, probe l). */
int rsrr_get_eta(rsrr_nep h, double* out);
/* The min(n, proj_cols) singular values of S_hat (or M_hat after rsrr_project_moments),
 * descending. */
int rsrr_get_sigma(rsrr_nep h, double* out);
/* The orthonormal basis S, n x k_S, caller ordering (after rsrr_project). */
int rsrr_get_basis(rsrr_nep h, double* out_reim);
/* The projected matrices P_i, [J][k_S][k_S] column-major (after rsrr_project). */
int rsrr_get_projected(rsrr_nep h, double* out_reim);
/* The singular values of H, K*k_S of them, descending (after rsrr_solve). */
int rsrr_get_hankel_sigma(rsrr_nep h, double* out);

/* ---- rsrr_band_solve_noalloc --------------------------------------------------------------
 * The paper has no counterpart: this is a deployment variant of the band LU and solves that
 * rsrr_sample runs per sampling point, for callers that cannot allocate device memory (a
 * process that hands all device memory to its own allocator up front, or a loop that must not
 * pay for an allocation).  It allocates nothing: the factor scratch (L panel blocks, row
 * permutations, pivots, status) lives in one file-scope device array of
 * RSRR_NOALLOC_SCRATCH_BYTES, which every device that loads the library holds until exit.
 *   n, kl, ku  order and bandwidths of A (0 <= kl, ku < n)
 *   ab_reim    DEVICE pointer, A in general-band layout, complex128 interleaved, column-major
 *              with leading dimension 2 kl + ku + 1, A(i, c) at row kl + ku + i - c; the top kl
 *              rows (pivoting fill) must be zero on entry.  Overwritten: rows <= the diagonal
 *              hold U of P A = L U (partial pivoting by |re| + |im|).
 *   L, b_reim  DEVICE pointer to the n x L right-hand sides (complex128, column-major),
 *              overwritten by the solution X of A X = B.
 *   stream     cudaStream_t for the work (NULL = default stream); returns after it completes.
 * The first call on a device looks up the scratch array's address (cudaGetSymbolAddress, with
 * that device current) and caches it; make that first call before any stream capture.  All
 * calls on a device share the array and leave their contents in it; calls whose GPU work
 * overlaps race on it.  Errors: EINVAL (bad arguments, or the factor scratch of this band
 * would exceed RSRR_NOALLOC_SCRATCH_BYTES), ESINGULAR (zero pivot), ECUDA, EUNSUPPORTED
 * (band too wide for the shared-memory panels). */
#define RSRR_NOALLOC_SCRATCH_BYTES (32u << 20)
int rsrr_band_solve_noalloc(int64_t n, int32_t kl, int32_t ku, double* ab_reim, int32_t L, double* b_reim,
                            void* stream);

/* ---- rsrr_selftest_bounded_wait (diagnostics) ---------------------------------------------
 * The paper has no counterpart.  Every device-side wait of this library (the grid barrier of its
 * cooperative kernels, the mbarrier waits of its tensor-core pipelines) gives up after a bounded
 * number of polls, records the failure and lets the kernel return, and the call that launched it
 * reports RSRR_ETIMEOUT.  This call runs one such wait with a short poll limit (well under a
 * second) on a condition the host arranged, so that a test can check that chain without faulting
 * or hanging the device:
 *   kind 0  a grid barrier (2 CTAs, cooperative launch) whose arrival count starts where no CTA
 *           can complete it: returns RSRR_ETIMEOUT
 *   kind 1  an mbarrier wait on a phase that nothing arrives at: returns RSRR_ETIMEOUT
 *   kind 2  the same grid barrier from a zero count: returns RSRR_OK
 *   kind 3  the same mbarrier wait after its one expected arrival: returns RSRR_OK
 *   stream  cudaStream_t for the work (NULL = default); returns after it completes.
 * The device context stays usable after every kind.  Errors: EINVAL (kind), ENOMEM, ECUDA. */
int rsrr_selftest_bounded_wait(int32_t kind, void* stream);

/* Diagnostics: the largest number of bytes the library's device allocations (the current
 * device's default stream-ordered memory pool) have held at once since the last reset; reset != 0
 * starts a new measurement after reading.  Negative RSRR_E* code on failure. */
int64_t rsrr_device_peak_bytes(int32_t reset);

/* Number of CUDA kernels this library has launched in the process so far (all handles). */
int64_t rsrr_kernel_launches(void);

void rsrr_destroy(rsrr_nep h);
const char* rsrr_last_error(void);
/* Library version string. */
const char* rsrr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RSRR_H */
