// rsrr_solve: Algorithm 1 (modified block Sakurai-Sugiura) on T_S(z) = sum_i f_i(z) P_i, then
// Algorithm 2 Step 5 (v = S g) and the residuals ||T(lambda) v|| (Section 7.1), FP64.
//
//   moments   A_alpha = 1/(i N_S) sum_j w_j^alpha phi'(theta_j) T_S(z_j)^{-1},
//             w_j = (z_j - gamma)/rho, rho = max(a, b)                       (Eq. eq-Ap-num)
//             T_S(z_j)^{-1}: blocked Gauss-Jordan elimination with partial pivoting, batched
//             over the points, its rank-bb updates on the ZGEMM (zinv.cu); for k_S too large
//             for its panels, a dense LU on the band kernels (kl = ku = k_S-1) solved against I.
//             The weighted sums are one ZGEMM.
//   winding   1/(i N_S) sum_j phi'_j tr(T_S(z_j)^{-1} T_S'(z_j))            (Eq. eq-ncs)
//   Hankel    H, H^< from A_0..A_{2K-1}                                      (Eq. eq-HH)
//   SVD of H  one-sided Jacobi with accumulated rotations                  (Eq. eq-svdH)
//   count     gap argmax over the whole SVD if >= tol_gap (Eq. eq-gap), combined with the
//             winding number as Section 4.3 suggests (see the comments at the decision)
//   A         V_0^H H^< W_0 Sigma_0^{-1}, eig by Hessenberg + shifted QR     (Eq. eq-A)
//   pairs     lambda = rho lambda' + gamma, g = H_r W_0 Sigma_0^{-1} g'     (Eq. eq-eigens)
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "band.cuh"
#include "dense.cuh"
#include "internal.h"

namespace rsrr {

namespace {

// T_S(z_j) = sum_i F[j][i] P_i into dense-band storage (ldab rows, kv = 2(k-1)).
__global__ void assemble_reduced_kernel(const c128* P, int J, int k, const c128* F, int j0, int kv, int ldab,
                                        c128* ab, int64_t ab_stride) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    if (idx >= (int64_t)k * k) return;
    const int r = (int)(idx % k), c = (int)(idx / k);
    const c128* f = F + (int64_t)(j0 + pt) * J;
    c128 v = czero<double>();
    for (int i = 0; i < J; ++i) cfma(v, f[i], P[(int64_t)i * k * k + idx]);
    ab[pt * ab_stride + (int64_t)(kv + r - c) + (int64_t)c * ldab] = v;
}

// T_S(z_j) = sum_i F[j][i] P_i, dense column-major (k x k per point).
__global__ void assemble_reduced_dense_kernel(const c128* P, int J, int k, const c128* F, int j0, c128* X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    const int64_t kk = (int64_t)k * k;
    if (idx >= kk) return;
    const c128* f = F + (int64_t)(j0 + pt) * J;
    c128 v = czero<double>();
    for (int i = 0; i < J; ++i) cfma(v, f[i], P[(int64_t)i * kk + idx]);
    X[pt * kk + idx] = v;
}

__global__ void identity_batch_kernel(c128* X, int k, int npts) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    X[(int64_t)blockIdx.y * k * k + idx] = (idx % k == idx / k) ? mk<double>(1.0, 0.0) : czero<double>();
}

__global__ void transpose_terms_kernel(const c128* P, int k, int J, c128* Pt) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (idx >= (int64_t)k * k) return;
    const int r = (int)(idx % k), c = (int)(idx / k);
    Pt[(int64_t)i * k * k + c + (int64_t)r * k] = P[(int64_t)i * k * k + idx];
}

// H (or H^<) from the moments: block (r, c) = A_{r + c + shift}
__global__ void hankel_kernel(const c128* mom, int k, int K, int shift, c128* H) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t dim = (int64_t)K * k;
    if (idx >= dim * dim) return;
    const int64_t gr = idx % dim, gc = idx / dim;
    const int br = (int)(gr / k), bc = (int)(gc / k);
    const int r = (int)(gr % k), c = (int)(gc % k);
    H[idx] = mom[(int64_t)(br + bc + shift) * k * k + r + (int64_t)c * k];
}

__global__ void scale_cols_kernel(c128* X, int64_t rows, int cols, int64_t ld, const double* s, int invert) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    const double f = invert ? 1.0 / s[c] : s[c];
    X[r + c * ld] = cscale(X[r + c * ld], f);
}

__global__ void scale_rows_kernel(c128* X, int rows, int cols, int64_t ld, const double* s) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    X[r + c * ld] = cscale(X[r + c * ld], 1.0 / s[r]);
}

__global__ void gather_cols_kernel(const c128* X, int64_t rows, int64_t ld, const int* cols, int nc, c128* Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * nc) return;
    const int64_t r = idx % rows, c = idx / rows;
    Y[idx] = X[r + (int64_t)cols[c] * ld];
}

// r_t = sum_i F[t][i] (Y_i)[:, t] for each column t (Y_i = M_i G, stacked with stride sY)
__global__ void combine_terms_kernel(const c128* Y, int64_t rows, int ncol, int J, int64_t sY, const c128* F,
                                     c128* R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * ncol) return;
    const int t = (int)(idx / rows);
    c128 v = czero<double>();
    for (int i = 0; i < J; ++i) cfma(v, F[(int64_t)t * J + i], Y[(int64_t)i * sY + idx]);
    R[idx] = v;
}

// ||T(lambda_t) v_t|| through the CSR: one thread per (row, pair), atomics into out[t]
__global__ void csr_residual_kernel(const int64_t* rowptr, const int32_t* colind, const c128* vals, int64_t nnz,
                                    int64_t n, int J, const c128* F, const c128* V, int npair, double* out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    double s = 0.0;
    if (r < n) {
        c128 acc = czero<double>();
        const c128* f = F + (int64_t)t * J;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            c128 tv = czero<double>();
            for (int i = 0; i < J; ++i) cfma(tv, f[i], vals[(int64_t)i * nnz + e]);
            cfma(acc, tv, V[colind[e] + (int64_t)t * n]);
        }
        s = cnorm2(acc);
    }
    for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[t], s);
}

// ------------------------------------------------------------------------------------------
// Eigenpairs of a small complex matrix A (n x n, column-major, global memory), one CTA:
// Householder reduction to Hessenberg form, single-shift QR with Wilkinson shifts and
// deflation (Givens rotations), eigenvectors of the triangular Schur factor by back
// substitution, back-transformed by the accumulated unitary Z.  Writes lam[n], X[n x n]
// (unit columns).  status: 0 ok, 1 no convergence.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) small_eig_kernel(c128* A, int n, c128* Z, c128* vtmp, c128* lam,
                                                        c128* X, int* status) {
    const int tid = threadIdx.x;
    __shared__ c128 s_c, s_s, s_tau;
    __shared__ int s_flag;
#define Am(i, j) A[(i) + (int64_t)(j) * n]
#define Zm(i, j) Z[(i) + (int64_t)(j) * n]
    for (int idx = tid; idx < n * n; idx += 256) Z[idx] = (idx % n == idx / n) ? mk<double>(1.0, 0.0) : czero<double>();
    __syncthreads();
    // Hessenberg reduction
    for (int j = 0; j + 2 < n; ++j) {
        // reflector from A[j+1:n, j]
        double xs = 0.0;
        for (int i = j + 2 + tid; i < n; i += 256) xs += cnorm2(Am(i, j));
        xs = block_sum_all(xs);
        if (tid == 0) {
            const c128 al = Am(j + 1, j);
            if (xs == 0.0 && al.im == 0.0) {
                s_tau = czero<double>();
                s_flag = 1;
            } else {
                const double beta = -copysign(sqrt(al.re * al.re + al.im * al.im + xs), al.re);
                s_tau = mk<double>((beta - al.re) / beta, -al.im / beta);
                s_c = crecip(mk<double>(al.re - beta, al.im));
                s_s = mk<double>(beta, 0.0);
                s_flag = 0;
            }
        }
        __syncthreads();
        if (s_flag) continue;
        for (int i = tid; i < n; i += 256) vtmp[i] = (i < j + 1) ? czero<double>() : (i == j + 1 ? mk<double>(1.0, 0.0) : Am(i, j) * s_c);
        __syncthreads();
        if (tid == 0) Am(j + 1, j) = s_s;
        for (int i = j + 2 + tid; i < n; i += 256) Am(i, j) = czero<double>();
        __syncthreads();
        const c128 tau = s_tau;
        // A <- H^H A (columns j+1..n-1), H = I - tau v v^H
        for (int c = j + 1 + tid; c < n; c += 256) {
            c128 w = czero<double>();
            for (int i = j + 1; i < n; ++i) cfma_conj(w, vtmp[i], Am(i, c));
            const c128 f = cconj(tau) * w;
            for (int i = j + 1; i < n; ++i) cfms(Am(i, c), vtmp[i], f);
        }
        __syncthreads();
        // A <- A H (rows 0..n-1), Z <- Z H
        for (int r = tid; r < 2 * n; r += 256) {
            c128* M = (r < n) ? A : Z;
            const int rr = (r < n) ? r : r - n;
            c128 w = czero<double>();
            for (int i = j + 1; i < n; ++i) cfma(w, M[rr + (int64_t)i * n], vtmp[i]);
            const c128 f = w * tau;
            for (int i = j + 1; i < n; ++i) cfms(M[rr + (int64_t)i * n], f, cconj(vtmp[i]));
        }
        __syncthreads();
    }
    // shifted QR on the Hessenberg matrix, active window [lo, hi]
    int hi = n - 1, iter = 0, total = 0;
    const double eps = 1.1102230246251565e-16;
    while (hi > 0) {
        // deflation check (thread 0 decides, everyone follows)
        if (tid == 0) {
            int l = hi;
            while (l > 0) {
                const double sub = cabs1(Am(l, l - 1));
                const double dd = cabs1(Am(l, l)) + cabs1(Am(l - 1, l - 1));
                if (sub <= eps * (dd == 0.0 ? 1.0 : dd)) { Am(l, l - 1) = czero<double>(); break; }
                --l;
            }
            s_flag = l;
        }
        __syncthreads();
        const int lo = s_flag;
        __syncthreads();  // everyone has read s_flag before thread 0 may write it again
        if (lo == hi) { --hi; iter = 0; continue; }
        if (++total > 60 * n) { if (tid == 0) *status = 1; return; }
        ++iter;
        // Wilkinson shift from the trailing 2x2 (exceptional shift every 10 iterations)
        c128 mu;
        {
            const c128 a = Am(hi - 1, hi - 1), b = Am(hi - 1, hi), c = Am(hi, hi - 1), d = Am(hi, hi);
            if (iter % 10 == 0) {
                mu = d + mk<double>(0.75 * cabs1(c), 0.0);
            } else {
                const c128 tr2 = cscale(a + d, 0.5);
                const c128 det = a * d - b * c;
                const c128 disc = tr2 * tr2 - det;
                // complex sqrt from |disc| and the half-angle formulas
                const double r = sqrt(disc.re * disc.re + disc.im * disc.im);
                double sr = sqrt(fmax(0.0, 0.5 * (r + disc.re)));
                double si = sqrt(fmax(0.0, 0.5 * (r - disc.re)));
                if (disc.im < 0) si = -si;
                const c128 sq = mk<double>(sr, si);
                const c128 m1 = tr2 + sq, m2 = tr2 - sq;
                mu = (cnorm2(m1 - d) < cnorm2(m2 - d)) ? m1 : m2;
            }
        }
        // implicit single-shift QR sweep on [lo, hi] by Givens rotations
        for (int k = lo; k < hi; ++k) {
            if (tid == 0) {
                c128 x, y;
                if (k == lo) { x = Am(lo, lo) - mu; y = Am(lo + 1, lo); }
                else { x = Am(k, k - 1); y = Am(k + 1, k - 1); }
                const double nx = sqrt(cnorm2(x)), ny = sqrt(cnorm2(y));
                const double nr = sqrt(nx * nx + ny * ny);
                if (nr == 0.0) { s_c = mk<double>(1.0, 0.0); s_s = czero<double>(); }
                else {
                    // G = [c s; -conj(s) c] with c real: G [x; y] = [r; 0]
                    const double c = nx / nr;
                    const c128 ph = (nx == 0.0) ? mk<double>(1.0, 0.0) : cscale(x, 1.0 / nx);
                    const c128 s = cscale(ph * cconj(y), 1.0 / nr);
                    s_c = mk<double>(c, 0.0);
                    s_s = s;
                }
            }
            __syncthreads();
            const double c = s_c.re;
            const c128 s = s_s;
            // rows k, k+1 from the left (columns from max(lo, k-1))
            for (int col = max(lo, k - 1) + tid; col < n; col += 256) {
                const c128 u = Am(k, col), v = Am(k + 1, col);
                Am(k, col) = cscale(u, c) + s * v;
                Am(k + 1, col) = cscale(v, c) - cconj(s) * u;
            }
            __syncthreads();
            // columns k, k+1 from the right (rows up to min(hi, k+2)), and Z
            const int rmax = min(hi, k + 2);
            for (int r = tid; r <= rmax + n; r += 256) {
                if (r <= rmax) {
                    const c128 u = Am(r, k), v = Am(r, k + 1);
                    Am(r, k) = cscale(u, c) + cconj(s) * v;
                    Am(r, k + 1) = cscale(v, c) - s * u;
                } else {
                    const int rr = r - rmax - 1;
                    if (rr < n) {
                        const c128 u = Zm(rr, k), v = Zm(rr, k + 1);
                        Zm(rr, k) = cscale(u, c) + cconj(s) * v;
                        Zm(rr, k + 1) = cscale(v, c) - s * u;
                    }
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // eigenvalues and eigenvectors of the triangular Schur form, back-transformed by Z
    for (int k = tid; k < n; k += 256) lam[k] = Am(k, k);
    __syncthreads();
    const double small = 1e-300;
    for (int k = tid; k < n; k += 256) {
        // y = eigenvector of upper-triangular T for lambda_k, stored in column k of X (scratch)
        c128* y = X + (int64_t)k * n;
        for (int i = 0; i < n; ++i) y[i] = czero<double>();
        y[k] = mk<double>(1.0, 0.0);
        const c128 lk = Am(k, k);
        double tnorm = 0.0;
        for (int i = 0; i <= k; ++i) tnorm = fmax(tnorm, cabs1(Am(i, i)));
        for (int i = k - 1; i >= 0; --i) {
            c128 s = czero<double>();
            for (int j = i + 1; j <= k; ++j) cfma(s, Am(i, j), y[j]);
            c128 den = Am(i, i) - lk;
            if (cabs1(den) < eps * fmax(tnorm, small)) den = mk<double>(eps * fmax(tnorm, small), 0.0);
            y[i] = czero<double>() - s * crecip(den);
        }
    }
    __syncthreads();
    // X <- Z Y (in place per column is not possible: use vtmp as one column of workspace each)
    for (int k = 0; k < n; ++k) {
        for (int r = tid; r < n; r += 256) {
            c128 s = czero<double>();
            for (int j = 0; j <= k; ++j) cfma(s, Zm(r, j), X[j + (int64_t)k * n]);
            vtmp[r] = s;
        }
        __syncthreads();
        double nn = 0.0;
        for (int r = tid; r < n; r += 256) nn += cnorm2(vtmp[r]);
        nn = block_sum_all(nn);
        const double inv = nn > 0 ? 1.0 / sqrt(nn) : 1.0;
        for (int r = tid; r < n; r += 256) X[r + (int64_t)k * n] = cscale(vtmp[r], inv);
        __syncthreads();
    }
    if (tid == 0) *status = 0;
#undef Am
#undef Zm
}

int alloc_zero(c128** p, size_t n, cudaStream_t s) {
    RSRR_TRY(dalloc_n(p, n, s));
    if (cudaMemsetAsync(*p, 0, n * sizeof(c128), s) != cudaSuccess) return set_error(RSRR_ECUDA, "memset");
    return RSRR_OK;
}

}  // namespace

int solve_run(rsrr_nep h, int N_S, int K, double tol_gap, int cap, double* lambda_reim, double* V_reim,
              double* resid, int32_t* nC_out) {
    cudaStream_t st = h->stream;
    cudaEvent_t ev[4];
    for (auto& e : ev) cudaEventCreate(&e);
    struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]); } } evg{ev};
    cudaEventRecord(ev[0], st);
    for (double& x : h->ms_solve_parts) x = 0.0;
    zgemm_profile_begin();
    jacobi_profile_begin();
    struct ZpGuard {
        rsrr_nep h;
        ~ZpGuard() {
            zgemm_profile_end(&h->ms_zgemm_solve, &h->zgemm_flops_solve, &h->ms_zgemm_tc_solve, &h->zgemm_tc_flops_solve);
            jacobi_profile_end(&h->ms_jacobi_solve, &h->jacobi_flops_solve);
        }
    } zpg{h};
    // J, fns: the reduced NEP's terms (T's own, or Chebyshev polynomials); the final residual
    // uses T itself (h->J, h->fns, the CSR values)
    const int k = h->kS, J = h->red_J;
    const std::vector<rsrr_fn>& fns = h->red_fns;
    const int64_t n = h->n;
    *nC_out = 0;
    h->nbar = 0;
    h->n_winding = 0;
    h->n_gap = -1;
    h->winding = 0;
    h->sigma_H.clear();
    if (k <= 0) return RSRR_OK;
    const double rho = std::max(h->C.a, h->C.b);
    const zd gamma(h->C.gamma_re, h->C.gamma_im);
    std::vector<zd> z, wq;
    contour_rule(h->C, N_S, &z, &wq);
    std::vector<c128> F((size_t)N_S * J), dF((size_t)N_S * J), Wt((size_t)N_S * 2 * K);
    for (int j = 0; j < N_S; ++j) {
        for (int i = 0; i < J; ++i) {
            zd v, d;
            eval_fn(fns[i], z[j], &v, &d);
            if (!std::isfinite(std::abs(v)) || !std::isfinite(std::abs(d)))
                return set_error(RSRR_ENONFINITE, "f_i is not finite at a quadrature point");
            F[(size_t)j * J + i] = fromstd(v);
            dF[(size_t)j * J + i] = fromstd(d);
        }
        const zd w = (z[j] - gamma) / rho;
        zd p = wq[j];
        for (int al = 0; al < 2 * K; ++al) {
            Wt[(size_t)j + (size_t)al * N_S] = fromstd(p);  // N_S x 2K, column al
            p *= w;
        }
    }
    const int64_t kk = (int64_t)k * k;
    // The inverses: blocked Gauss-Jordan (zinv.cu) while a k-row panel fits shared memory, else
    // the band LU and solve kernels on dense band storage (kl = ku = k - 1) against I.
    const bool gje = zinv_block(k) > 0;
    BandDims d{};
    size_t ab_e = 0, lp_e = 0, perm_e = 0, per_pt = 0;
    if (gje) {
        per_pt = zinv_bytes_per_matrix(k) + 64;
    } else {
        RSRR_TRY(pick_dims(k, k - 1, k - 1, false, &d));
        ab_e = (size_t)d.ldab * k;
        lp_e = (size_t)d.npanels * d.ldp * d.nb;
        perm_e = (size_t)d.npanels * d.ldp;
        per_pt = (ab_e + lp_e + kk) * sizeof(c128) + perm_e * 4 + (size_t)k * 4 + 64;
    }
    size_t free_b = 0, total_b = 0;
    RSRR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    // Points factored at once: as many as fit 60 % of the free memory and a fixed 24 GiB (so that
    // a caller can bound the request's footprint: at most max(per_pt, 24 GiB) here), spread
    // evenly over the chunks.
    const int64_t fit = std::min<int64_t>((int64_t)(0.6 * free_b), (int64_t)24 << 30) / (int64_t)per_pt;
    const int64_t nchunk = ceil_div((int64_t)N_S, std::max<int64_t>(1, fit));
    const int chunk = (int)ceil_div((int64_t)N_S, nchunk);

    c128 *dFt = nullptr, *dWt = nullptr, *ab = nullptr, *lp = nullptr, *X = nullptr, *mom = nullptr,
         *Pt = nullptr, *trc = nullptr, *H = nullptr, *Hl = nullptr, *Jm = nullptr, *V0 = nullptr, *W0 = nullptr,
         *T1 = nullptr, *Am = nullptr, *Zs = nullptr, *vt = nullptr, *lam_d = nullptr, *Xe = nullptr,
         *G = nullptr, *Hr = nullptr, *T2 = nullptr, *PG = nullptr, *RG = nullptr, *Fl = nullptr, *Vfull = nullptr,
         *Tz = nullptr;
    int32_t *perm = nullptr, *ipiv = nullptr, *info = nullptr, *cols = nullptr, *est = nullptr;
    double *sig = nullptr, *rn = nullptr, *sigs = nullptr, *sigsafe = nullptr;
    int rc = RSRR_OK;
    auto cleanup = [&]() {
        for (void* p : {(void*)dFt, (void*)dWt, (void*)ab, (void*)lp, (void*)X, (void*)mom, (void*)Pt, (void*)trc,
                        (void*)H, (void*)Hl, (void*)Jm, (void*)V0, (void*)W0, (void*)T1, (void*)Am, (void*)Zs,
                        (void*)vt, (void*)lam_d, (void*)Xe, (void*)G, (void*)Hr, (void*)T2, (void*)PG, (void*)RG,
                        (void*)Fl, (void*)Vfull, (void*)Tz, (void*)perm, (void*)ipiv, (void*)info, (void*)cols, (void*)est,
                        (void*)sig, (void*)rn, (void*)sigs, (void*)sigsafe})
            dfree(p, st);
    };
#define TRYC(expr) do { rc = (expr); if (rc != RSRR_OK) { cleanup(); return rc; } } while (0)
#define CUDAC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return set_error(RSRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)

    TRYC(dalloc_n(&dFt, F.size(), st));
    CUDAC(cudaMemcpyAsync(dFt, F.data(), F.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
    TRYC(dalloc_n(&dWt, Wt.size(), st));
    CUDAC(cudaMemcpyAsync(dWt, Wt.data(), Wt.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
    if (!gje) {
        TRYC(dalloc(reinterpret_cast<void**>(&ab), ab_e * sizeof(c128) * chunk, st));
        TRYC(dalloc(reinterpret_cast<void**>(&lp), lp_e * sizeof(c128) * chunk, st));
        TRYC(dalloc_n(&perm, perm_e * chunk, st));
        TRYC(dalloc_n(&ipiv, (size_t)k * chunk, st));
    }
    TRYC(dalloc_n(&X, (size_t)kk * chunk, st));
    TRYC(dalloc_n(&info, (size_t)chunk, st));
    TRYC(alloc_zero(&mom, (size_t)2 * K * kk, st));
    TRYC(dalloc_n(&Pt, (size_t)J * kk, st));
    TRYC(dalloc_n(&trc, (size_t)N_S * J, st));
    {
        dim3 g((unsigned)ceil_div(kk, 256), J);
        { transpose_terms_kernel<<<g, 256, 0, st>>>(h->d_P, k, J, Pt); note_launch(); }
    }
    // ---- moments and traces, chunk by chunk ------------------------------------------------------
    for (int j0 = 0; j0 < N_S; j0 += chunk) {
        const int np = std::min(chunk, N_S - j0);
        dim3 ga((unsigned)ceil_div(kk, 256), np);
        std::vector<int32_t> hinfo(np);
        if (gje) {
            { assemble_reduced_dense_kernel<<<ga, 256, 0, st>>>(h->d_P, J, k, dFt, j0, X); note_launch(); }
            CUDAC(cudaMemsetAsync(info, 0, (size_t)np * 4, st));
            TRYC(zinv_batch(X, k, np, info, st));
            CUDAC(cudaMemcpyAsync(hinfo.data(), info, np * 4, cudaMemcpyDeviceToHost, st));
        } else {
            CUDAC(cudaMemsetAsync(ab, 0, ab_e * sizeof(c128) * np, st));
            { assemble_reduced_kernel<<<ga, 256, 0, st>>>(h->d_P, J, k, dFt, j0, d.kv, d.ldab, ab, (int64_t)ab_e); note_launch(); }
            FactorArgs<double> fa{d, ab, (int64_t)ab_e, lp, (int64_t)lp_e, perm, (int64_t)perm_e, ipiv, info};
            TRYC(launch_factor<double>(fa, np, st));
            CUDAC(cudaMemcpyAsync(hinfo.data(), info, np * 4, cudaMemcpyDeviceToHost, st));
            { identity_batch_kernel<<<ga, 256, 0, st>>>(X, k, np); note_launch(); }
            SolveArgs<double> sa{d, ab, (int64_t)ab_e, lp, (int64_t)lp_e, perm, (int64_t)perm_e, X, kk, k, nullptr};
            TRYC(launch_fwd<double>(sa, np, st));
            TRYC(launch_bwd<double>(sa, np, st));
        }
        CUDAC(cudaStreamSynchronize(st));
        for (int t = 0; t < np; ++t)
            if (hinfo[t]) { cleanup(); return set_error(RSRR_ESINGULAR, "T_S(z) is singular at a quadrature point"); }
        // moments: [k^2 x 2K] += [k^2 x np] * Wt[j0:j0+np, :]
        Zgemm gm;
        gm.opA = OP_N; gm.opB = OP_N; gm.M = (int)kk; gm.N = 2 * K; gm.K = np;
        gm.A = X; gm.lda = kk; gm.B = dWt + j0; gm.ldb = N_S; gm.C = mom; gm.ldc = kk;
        gm.beta = mk<double>(1.0, 0.0); gm.ksplit = 1;
        TRYC(zgemm(gm, st));
        // traces tr(X_j P_i) = vec(X_j)^T vec(P_i^T): [np x J]
        Zgemm gt;
        gt.opA = OP_T; gt.opB = OP_N; gt.M = np; gt.N = J; gt.K = (int)kk;
        gt.A = X; gt.lda = kk; gt.B = Pt; gt.ldb = kk; gt.C = trc + j0; gt.ldc = N_S;
        TRYC(zgemm(gt, st));
    }
    cudaEventRecord(ev[1], st);  // inverses, moments, traces done
    std::vector<c128> htr((size_t)N_S * J);
    CUDAC(cudaMemcpyAsync(htr.data(), trc, htr.size() * sizeof(c128), cudaMemcpyDeviceToHost, st));
    CUDAC(cudaStreamSynchronize(st));
    zd wind = 0.0;
    for (int j = 0; j < N_S; ++j) {
        zd t = 0.0;
        for (int i = 0; i < J; ++i) t += tostd(dF[(size_t)j * J + i]) * tostd(htr[(size_t)j + (size_t)i * N_S]);
        wind += t * wq[j];
    }
    h->winding = wind;
    // ---- Hankel matrices and the SVD of H ------------------------------------------------------
    const int D = K * k;
    const int64_t DD = (int64_t)D * D;
    TRYC(dalloc_n(&H, (size_t)DD, st));
    TRYC(dalloc_n(&Hl, (size_t)DD, st));
    TRYC(dalloc_n(&Jm, (size_t)DD, st));
    { hankel_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(mom, k, K, 0, H); note_launch(); }
    { hankel_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(mom, k, K, 1, Hl); note_launch(); }
    { identity_batch_kernel<<<dim3((unsigned)ceil_div(DD, 256), 1), 256, 0, st>>>(Jm, D, 1); note_launch(); }
    int sweeps = 0;
    double hmax = 0.0, hfro2 = 0.0;
    {
        TRYC(dalloc_n(&sig, (size_t)D, st));
        column_norms(H, D, D, D, sig, st);
        std::vector<double> cn(D);
        CUDAC(cudaMemcpyAsync(cn.data(), sig, D * 8, cudaMemcpyDeviceToHost, st));
        CUDAC(cudaStreamSynchronize(st));
        for (double x : cn) {
            hmax = std::max(hmax, x);
            hfro2 += x * x;
        }
        dfree(sig, st);
        sig = nullptr;
    }
    // Columns at the rounding-noise level of H (a few u ||H||_F: the moments carry errors of
    // that size) resolve no singular value and never settle, so they are not rotated.
    const double hfloor = std::max(1e-16 * hmax, 4.0 * 1.1102230246251565e-16 * std::sqrt(hfro2));
    TRYC(jacobi_svd_preconditioned(H, D, Jm, st, hfloor, 1e-12, &sweeps));
    h->jacobi_sweeps_solve = sweeps;
    cudaEventRecord(ev[2], st);  // Hankel SVD done
    TRYC(dalloc_n(&sig, (size_t)D, st));
    column_norms(H, D, D, D, sig, st);
    std::vector<double> sv(D);
    CUDAC(cudaMemcpyAsync(sv.data(), sig, D * 8, cudaMemcpyDeviceToHost, st));
    CUDAC(cudaStreamSynchronize(st));
    std::vector<int> ord(D);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return sv[x] > sv[y]; });
    h->sigma_H.resize(D);
    for (int i = 0; i < D; ++i) h->sigma_H[i] = sv[ord[i]];
    // ---- the count ----------------------------------------------------------------------------
    const int n_w = (int)std::lround(wind.real());
    int n_g = -1;
    {
        double best = 0.0;
        for (int i = 0; i + 1 < D; ++i) {
            const double gap = h->sigma_H[i] / std::max(h->sigma_H[i + 1], 1e-300);
            if (gap > best) { best = gap; n_g = i + 1; }
        }
        if (best < tol_gap) n_g = -1;
    }
    h->n_winding = n_w;
    h->n_gap = n_g;
    TRYC(dalloc_n(&cols, (size_t)D, st));
    CUDAC(cudaMemcpyAsync(cols, ord.data(), D * 4, cudaMemcpyHostToDevice, st));
    TRYC(dalloc_n(&V0, (size_t)DD, st));
    TRYC(dalloc_n(&W0, (size_t)DD, st));
    TRYC(dalloc_n(&T1, (size_t)DD, st));
    TRYC(dalloc_n(&Am, (size_t)D * D, st));
    TRYC(dalloc_n(&Zs, (size_t)D * D, st));
    TRYC(dalloc_n(&vt, (size_t)D, st));
    TRYC(dalloc_n(&lam_d, (size_t)D, st));
    TRYC(dalloc_n(&Xe, (size_t)D * D, st));
    TRYC(dalloc_n(&G, (size_t)k * D, st));
    TRYC(dalloc_n(&Hr, (size_t)k * D, st));
    TRYC(dalloc_n(&T2, (size_t)D * D, st));
    TRYC(dalloc_n(&est, 1, st));
    // V (left singular vectors, sorted, normalised) and W = J (sorted)
    { gather_cols_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(H, D, D, cols, D, V0); note_launch(); }
    { gather_cols_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(Jm, D, D, cols, D, W0); note_launch(); }
    std::vector<double> sv_sorted(h->sigma_H);
    TRYC(dalloc_n(&sigs, (size_t)D, st));
    CUDAC(cudaMemcpyAsync(sigs, sv_sorted.data(), D * 8, cudaMemcpyHostToDevice, st));
    std::vector<double> sv_safe(sv_sorted);
    for (double& x : sv_safe) x = x > 0 ? x : 1.0;
    TRYC(dalloc_n(&sigsafe, (size_t)D, st));
    CUDAC(cudaMemcpyAsync(sigsafe, sv_safe.data(), D * 8, cudaMemcpyHostToDevice, st));
    { scale_cols_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(V0, D, D, D, sigsafe, 1); note_launch(); }
    // H_r = [A_0 ... A_{K-1}] (k x D): the first k rows of H in the original (unrotated) form
    {
        // mom holds A_alpha as k x k blocks consecutively: [A_0 | A_1 | ...] is exactly k x (2K k)
        CUDAC(cudaMemcpyAsync(Hr, mom, (size_t)k * D * sizeof(c128), cudaMemcpyDeviceToDevice, st));
    }

    // extract(nb): eigenvalues (host) and g = H_r W_0 Sigma_0^{-1} g' in G (k x nb, device)
    std::vector<zd> lam_h;
    auto extract = [&](int nb) -> int {
        lam_h.clear();
        if (nb <= 0) return RSRR_OK;
        Zgemm a1;  // T1 = H^< W_0
        a1.opA = OP_N; a1.opB = OP_N; a1.M = D; a1.N = nb; a1.K = D;
        a1.A = Hl; a1.lda = D; a1.B = W0; a1.ldb = D; a1.C = T1; a1.ldc = D;
        RSRR_TRY(zgemm(a1, st));
        Zgemm a2;  // A = V_0^H T1, then columns / sigma
        a2.opA = OP_C; a2.opB = OP_N; a2.M = nb; a2.N = nb; a2.K = D;
        a2.A = V0; a2.lda = D; a2.B = T1; a2.ldb = D; a2.C = Am; a2.ldc = nb;
        RSRR_TRY(zgemm(a2, st));
        { scale_cols_kernel<<<(unsigned)ceil_div((int64_t)nb * nb, 256), 256, 0, st>>>(Am, nb, nb, nb, sigsafe, 1); note_launch(); }
        { small_eig_kernel<<<1, 256, 0, st>>>(Am, nb, Zs, vt, lam_d, Xe, est); note_launch(); }
        RSRR_CUDA(cudaGetLastError());
        int hst = 0;
        std::vector<c128> lh(nb);
        RSRR_CUDA(cudaMemcpyAsync(&hst, est, 4, cudaMemcpyDeviceToHost, st));
        RSRR_CUDA(cudaMemcpyAsync(lh.data(), lam_d, nb * sizeof(c128), cudaMemcpyDeviceToHost, st));
        RSRR_CUDA(cudaStreamSynchronize(st));
        if (hst) return set_error(RSRR_ENOTCONVERGED, "QR iteration for eig(A) did not converge");
        for (int t = 0; t < nb; ++t) lam_h.push_back(rho * tostd(lh[t]) + gamma);
        { scale_rows_kernel<<<(unsigned)ceil_div((int64_t)nb * nb, 256), 256, 0, st>>>(Xe, nb, nb, nb, sigsafe); note_launch(); }
        Zgemm b1;  // T2 = W_0 (Sigma_0^{-1} g')
        b1.opA = OP_N; b1.opB = OP_N; b1.M = D; b1.N = nb; b1.K = nb;
        b1.A = W0; b1.lda = D; b1.B = Xe; b1.ldb = nb; b1.C = T2; b1.ldc = D;
        RSRR_TRY(zgemm(b1, st));
        Zgemm b2;  // G = H_r T2
        b2.opA = OP_N; b2.opB = OP_N; b2.M = k; b2.N = nb; b2.K = D;
        b2.A = Hr; b2.lda = k; b2.B = T2; b2.ldb = D; b2.C = G; b2.ldc = k;
        RSRR_TRY(zgemm(b2, st));
        return RSRR_OK;
    };
    // max over pairs of ||T_S(lambda) g|| / ||g|| for the pairs currently in (lam_h, G)
    TRYC(dalloc_n(&PG, (size_t)J * k * D, st));
    TRYC(dalloc_n(&RG, (size_t)k * D, st));
    TRYC(dalloc_n(&Fl, (size_t)D * std::max(J, h->J), st));
    TRYC(dalloc_n(&rn, (size_t)2 * D, st));
    auto coef_upload = [&](const std::vector<zd>& lams, const std::vector<rsrr_fn>& fs) -> int {
        const int nf = (int)fs.size();
        std::vector<c128> fl(lams.size() * nf);
        for (size_t t = 0; t < lams.size(); ++t)
            for (int i = 0; i < nf; ++i) {
                zd v, dv;
                eval_fn(fs[i], lams[t], &v, &dv);
                fl[t * nf + i] = fromstd(v);
            }
        if (!fl.empty())
            RSRR_CUDA(cudaMemcpyAsync(Fl, fl.data(), fl.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
        return RSRR_OK;
    };
    auto reduced_residual = [&](int nb, double* out) -> int {
        *out = 0.0;
        if (nb <= 0) return RSRR_OK;
        RSRR_TRY(coef_upload(lam_h, fns));
        Zgemm gp;
        gp.opA = OP_N; gp.opB = OP_N; gp.M = k; gp.N = nb; gp.K = k;
        gp.A = h->d_P; gp.lda = k; gp.sA = kk; gp.B = G; gp.ldb = k; gp.sB = 0;
        gp.C = PG; gp.ldc = k; gp.sC = (int64_t)k * nb; gp.batch = J;
        RSRR_TRY(zgemm(gp, st));
        { combine_terms_kernel<<<(unsigned)ceil_div((int64_t)k * nb, 256), 256, 0, st>>>(PG, k, nb, J,
                                                                                      (int64_t)k * nb, Fl, RG); note_launch(); }
        column_norms(RG, k, nb, k, rn, st);
        column_norms(G, k, nb, k, rn + D, st);
        std::vector<double> hr(2 * D);
        RSRR_CUDA(cudaMemcpyAsync(hr.data(), rn, 2 * D * 8, cudaMemcpyDeviceToHost, st));
        RSRR_CUDA(cudaStreamSynchronize(st));
        for (int t = 0; t < nb; ++t) *out = std::max(*out, hr[t] / std::max(hr[D + t], 1e-300));
        return RSRR_OK;
    };
    // Section 4.3: the winding number and the gap rule should agree; when they do not, both
    // candidate sets are computed and the one with the smaller reduced residual is kept.  A
    // winding count of zero means no eigenvalue inside the contour.
    int nbar;
    if (n_w <= 0) nbar = 0;
    else if (n_g < 0 || n_g == n_w) nbar = n_w;
    else {
        double rw = 0, rg = 0;
        TRYC(extract(std::min(n_w, D)));
        TRYC(reduced_residual(std::min(n_w, D), &rw));
        TRYC(extract(std::min(n_g, D)));
        TRYC(reduced_residual(std::min(n_g, D), &rg));
        nbar = (rg < rw) ? n_g : n_w;
    }
    nbar = std::min(nbar, D);
    h->nbar = nbar;
    TRYC(extract(nbar));
    // keep eigenvalues strictly inside the contour, sorted by |lambda|
    std::vector<int> keep;
    for (int t = 0; t < nbar; ++t)
        if (inside_contour(h->C, lam_h[t])) keep.push_back(t);
    std::stable_sort(keep.begin(), keep.end(), [&](int x, int y) { return std::abs(lam_h[x]) < std::abs(lam_h[y]); });
    const int nk = (int)keep.size();
    *nC_out = nk;
    if (nk > cap) { cleanup(); return set_error(RSRR_EINVAL, "cap too small for the eigenvalues found"); }
    if (nk > 0) {
        // v = S g (normalised), residual ||T(lambda) v||
        CUDAC(cudaMemcpyAsync(cols, keep.data(), nk * 4, cudaMemcpyHostToDevice, st));
        { gather_cols_kernel<<<(unsigned)ceil_div((int64_t)k * nk, 256), 256, 0, st>>>(G, k, k, cols, nk, RG); note_launch(); }
        TRYC(dalloc_n(&Vfull, (size_t)n * nk, st));
        Zgemm gv;
        gv.opA = OP_N; gv.opB = OP_N; gv.M = (int)n; gv.N = nk; gv.K = k;
        gv.A = h->d_Q; gv.lda = n; gv.B = RG; gv.ldb = k; gv.C = Vfull; gv.ldc = n; gv.ksplit = 1;
        TRYC(zgemm(gv, st));
        column_norms(Vfull, (int)n, nk, n, rn, st);
        { scale_cols_kernel<<<(unsigned)ceil_div(n * nk, 256), 256, 0, st>>>(Vfull, n, nk, n, rn, 1); note_launch(); }
        std::vector<zd> lk(nk);
        for (int t = 0; t < nk; ++t) lk[t] = lam_h[keep[t]];
        const c128* tvals = h->d_vals;
        int tJ = h->J;
        if (h->tz) {
            // T(lambda_t) from the caller's values: nk terms with coefficients F = I
            TRYC(tz_values(h, lk, &Tz));
            tvals = Tz;
            tJ = nk;
            std::vector<c128> eye((size_t)nk * nk, czero<double>());
            for (int t = 0; t < nk; ++t) eye[(size_t)t * nk + t] = mk<double>(1.0, 0.0);
            dfree(Fl, st);
            Fl = nullptr;
            TRYC(dalloc_n(&Fl, eye.size(), st));
            CUDAC(cudaMemcpyAsync(Fl, eye.data(), eye.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
        } else {
            TRYC(coef_upload(lk, h->fns));
        }
        CUDAC(cudaMemsetAsync(rn, 0, nk * 8, st));
        dim3 gr((unsigned)ceil_div(n, 128), nk);
        { csr_residual_kernel<<<gr, 128, 0, st>>>(h->d_rowptr, h->d_colind, tvals, h->nnz, n, tJ, Fl, Vfull, nk, rn); note_launch(); }
        std::vector<double> hres(nk);
        CUDAC(cudaMemcpyAsync(hres.data(), rn, nk * 8, cudaMemcpyDeviceToHost, st));
        std::vector<c128> hv;
        if (V_reim) {
            hv.resize((size_t)n * nk);
            CUDAC(cudaMemcpyAsync(hv.data(), Vfull, hv.size() * sizeof(c128), cudaMemcpyDeviceToHost, st));
        }
        CUDAC(cudaStreamSynchronize(st));
        for (int t = 0; t < nk; ++t) {
            lambda_reim[2 * t] = lk[t].real();
            lambda_reim[2 * t + 1] = lk[t].imag();
            if (resid) resid[t] = std::sqrt(hres[t]);
            if (V_reim)
                for (int64_t r = 0; r < n; ++r) {
                    const c128 v = hv[(size_t)(r + (int64_t)t * n)];
                    const int64_t ro = h->ord.perm[r];
                    V_reim[2 * (ro + (int64_t)t * n)] = v.re;
                    V_reim[2 * (ro + (int64_t)t * n) + 1] = v.im;
                }
        }
    }
    cudaEventRecord(ev[3], st);
    CUDAC(cudaStreamSynchronize(st));
    for (int i = 0; i < 3; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
        h->ms_solve_parts[i] = t;
    }
    cleanup();
#undef TRYC
#undef CUDAC
    return RSRR_OK;
}

}  // namespace rsrr
