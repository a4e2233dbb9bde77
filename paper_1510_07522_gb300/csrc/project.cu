// rsrr_project: Algorithm 2 Step 3 (truncated SVD of S_hat, keep sigma_k > delta sigma_1)
// and Eq. eq-Zs-expr (P_i = S^H A_i S), all in FP64 on the device.
//
//   1. Householder QR of S_hat (n x m, m = N L) in panels of 32 columns.  The point blocks are
//      taken in bit-reversed order (0, N/2, N/4, 3N/4, ...) so early columns sample the whole
//      contour.  Each panel is factored by one cooperative kernel (two grid barriers per
//      column); the trailing matrix is updated with the compact WY form by three ZGEMMs.
//      After every panel the remaining trailing block is measured (Frobenius norm, then a
//      power-iteration estimate of its 2-norm with a safety factor of 3); once its 2-norm is
//      below 10% of delta * sigma_1 (sigma_1 from a power-iteration lower bound of ||S_hat||_2,
//      so the rule errs on the side of keeping rows), or below the rounding noise of S_hat
//      (at most 30% of delta * sigma_1), the remaining rows of R are dropped: by Weyl's
//      inequality they move no singular value by more than that, so the truncation only
//      differs from the full SVD for sigma that close to the threshold.
//   2. A second QR, of R_keep^H (m x k'), keeps only its k' x k' triangle R2; one-sided Jacobi
//      on R2 with the rotations accumulated gives R2^H = J Sigma W^H, and the left singular
//      vectors of R_keep = R2^H Q2^H are the columns of J.
//   3. S = Q [J(:, 1:k_S); 0] by applying the panels' reflectors in reverse, after one
//      Newton-Schulz step on J(:, 1:k_S) against the rounding its rotations accumulated.
//   4. P_i = S^H (A_i S): CSR SpMM, then ZGEMM.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dense.cuh"
#include "internal.h"

namespace rsrr {

namespace {

constexpr int kPB = 32;  // panel width

struct PanelArgs {
    c128* A;
    int64_t lda;
    int n, kb, bw;
    c128* tau;
    c128* T;       // bw x bw, column-major
    double* part;  // [G]
    c128* alpha;   // [1]
    c128* part2;   // [G][kPB]
    c128* part3;   // [G][kPB*kPB]
    c128* Y;       // [kPB*kPB]
    GridBar gb;
};

__global__ void __launch_bounds__(256) hqr_panel_kernel(PanelArgs a) {
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = 8;
    const int rows = a.n - a.kb;
    const int per = (rows + G - 1) / G;
    const int r0 = min(a.n, a.kb + g * per), r1 = min(a.n, r0 + per);
    __shared__ c128 s_w[kPB];
    __shared__ c128 s_tau, s_scal;
    __shared__ int s_ident;
    const int cend = a.kb + a.bw;
    for (int j = 0; j < a.bw; ++j) {
        const int c = a.kb + j, d = c;
        c128* col = a.A + (int64_t)c * a.lda;
        // phase 1: partial squared norm below the diagonal, and alpha
        double ss = 0.0;
        for (int i = max(r0, d + 1) + tid; i < r1; i += 256) ss += cnorm2(col[i]);
        ss = block_sum_all(ss);
        if (tid == 0) {
            a.part[g] = ss;
            if (d >= r0 && d < r1) *a.alpha = col[d];
        }
        if (!grid_sync(a.gb)) return;
        // phase 2: reflector (LAPACK zlarfg convention: real beta), scale own rows, partial dots
        double xs = 0.0;
        for (int t = tid; t < G; t += 256) xs += a.part[t];
        xs = block_sum_all(xs);
        if (tid == 0) {
            const c128 al = *a.alpha;
            if (xs == 0.0 && al.im == 0.0) {
                s_ident = 1;
                s_tau = czero<double>();
                s_scal = mk<double>(1.0, 0.0);
            } else {
                const double beta = -copysign(sqrt(al.re * al.re + al.im * al.im + xs), al.re);
                s_ident = 0;
                s_tau = mk<double>((beta - al.re) / beta, -al.im / beta);
                s_scal = crecip(mk<double>(al.re - beta, al.im));
                if (d >= r0 && d < r1) col[d] = mk<double>(beta, 0.0);
            }
            if (g == 0) a.tau[c] = s_tau;
        }
        __syncthreads();
        const bool ident = s_ident != 0;
        if (!ident) {
            const c128 sc = s_scal;
            for (int i = max(r0, d + 1) + tid; i < r1; i += 256) col[i] = col[i] * sc;
        }
        __syncthreads();
        for (int cc = c + 1 + warp; cc < cend; cc += NW) {
            const c128* x = a.A + (int64_t)cc * a.lda;
            c128 w = czero<double>();
            for (int i = max(r0, d) + lane; i < r1; i += 32) {
                const c128 v = (i == d) ? mk<double>(1.0, 0.0) : col[i];
                cfma_conj(w, v, x[i]);
            }
            for (int off = 16; off; off >>= 1) {
                w.re += __shfl_down_sync(0xffffffffu, w.re, off);
                w.im += __shfl_down_sync(0xffffffffu, w.im, off);
            }
            if (lane == 0) a.part2[(int64_t)g * kPB + (cc - a.kb)] = w;
        }
        if (!grid_sync(a.gb)) return;
        // phase 3: A[i, cc] -= conj(tau) v_i w_cc on own rows
        for (int cc = c + 1 + warp; cc < cend; cc += NW) {
            c128 w = czero<double>();
            for (int t = lane; t < G; t += 32) w = w + a.part2[(int64_t)t * kPB + (cc - a.kb)];
            for (int off = 16; off; off >>= 1) {
                w.re += __shfl_down_sync(0xffffffffu, w.re, off);
                w.im += __shfl_down_sync(0xffffffffu, w.im, off);
            }
            if (lane == 0) s_w[cc - a.kb] = w;
        }
        __syncthreads();
        if (!ident) {
            const c128 ct = cconj(s_tau);
            const int nc = cend - (c + 1);
            const int lo = max(r0, d);
            const int nr = max(0, r1 - lo);
            for (int idx = tid; idx < nr * nc; idx += 256) {
                const int i = lo + idx % nr, cc = c + 1 + idx / nr;
                const c128 v = (i == d) ? mk<double>(1.0, 0.0) : col[i];
                cfms(a.A[i + (int64_t)cc * a.lda], ct * v, s_w[cc - a.kb]);
            }
        }
        __syncthreads();
    }
    // compact WY factor: T upper triangular with I - V T V^H = H_0 ... H_{bw-1}
    const int bw = a.bw;
    for (int e = tid; e < bw * bw; e += 256) {
        const int p = e % bw, q = e / bw;
        c128 s = czero<double>();
        if (p < q) {
            for (int i = max(r0, a.kb + q); i < r1; ++i) {
                const c128 vp = (i == a.kb + p) ? mk<double>(1.0, 0.0) : a.A[i + (int64_t)(a.kb + p) * a.lda];
                const c128 vq = (i == a.kb + q) ? mk<double>(1.0, 0.0) : a.A[i + (int64_t)(a.kb + q) * a.lda];
                cfma_conj(s, vp, vq);
            }
        }
        a.part3[(int64_t)g * kPB * kPB + e] = s;
    }
    if (!grid_sync(a.gb)) return;
    if (tid == 0) {
        for (int e = g; e < bw * bw; e += G) {
            c128 s = czero<double>();
            for (int t = 0; t < G; ++t) s = s + a.part3[(int64_t)t * kPB * kPB + e];
            a.Y[e] = s;
        }
    }
    if (!grid_sync(a.gb)) return;
    if (g == 0) {
        for (int q = 0; q < bw; ++q) {
            const c128 tq = a.tau[a.kb + q];
            if (tid < q) {
                c128 s = czero<double>();
                for (int l = tid; l < q; ++l) cfma(s, a.T[tid + l * bw], a.Y[l + q * bw]);
                a.T[tid + q * bw] = czero<double>() - tq * s;
            }
            if (tid == 0) a.T[q + q * bw] = tq;
            for (int i = q + 1 + tid; i < bw; i += 256) a.T[i + q * bw] = czero<double>();
            __syncthreads();
        }
    }
}

// explicit V block: rows kb..n-1 of the panel, unit diagonal, zeros above
__global__ void extract_v_kernel(const c128* A, int64_t lda, int n, int kb, int bw, c128* V, int64_t ldv) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows = n - kb;
    if (idx >= rows * bw) return;
    const int i = (int)(idx % rows), t = (int)(idx / rows);
    const int gi = kb + i, col = kb + t;
    c128 v = czero<double>();
    if (gi == col) v = mk<double>(1.0, 0.0);
    else if (gi > col) v = A[gi + (int64_t)col * lda];
    V[i + (int64_t)t * ldv] = v;
}

// B = R_keep^H: B[c, r] = conj(A[r, c]) for r <= c (rows r < kk), zero below the diagonal of R
__global__ void rkeep_h_kernel(const c128* A, int64_t lda, int m, int kk, c128* B) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * kk) return;
    const int c = (int)(idx % m), r = (int)(idx / m);
    B[c + (int64_t)r * m] = (r <= c) ? cconj(A[r + (int64_t)c * lda]) : czero<double>();
}

__global__ void gather_blocks_kernel(const c128* S, int64_t n, int L, const int* order, int m, c128* A) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * m) return;
    const int64_t r = idx % n, c = idx / n;
    const int blk = (int)(c / L), l = (int)(c % L);
    A[idx] = S[r + ((int64_t)order[blk] * L + l) * n];
}

__global__ void init_y_kernel(const c128* J, int kk, const int* cols, int kS, int64_t n, c128* Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * kS) return;
    const int64_t r = idx % n, c = idx / n;
    Y[idx] = (r < kk) ? J[r + (int64_t)cols[c] * kk] : czero<double>();
}

__global__ void identity_kernel(c128* J, int k) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    J[idx] = (idx % k == idx / k) ? mk<double>(1.0, 0.0) : czero<double>();
}

// Y_i = A_i X for every term (CSR of the union pattern with the term's values)
__global__ void spmm_terms_kernel(const int64_t* rowptr, const int32_t* colind, const c128* vals, int64_t nnz,
                                  int64_t n, const c128* X, int k, c128* Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int term = blockIdx.y;
    if (idx >= n * k) return;
    const int64_t r = idx % n, c = idx / n;
    const c128* v = vals + (int64_t)term * nnz;
    c128 acc = czero<double>();
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) cfma(acc, v[e], X[colind[e] + c * n]);
    Y[(int64_t)term * n * k + idx] = acc;
}

std::vector<int> bit_reversed_order(int N) {
    int bits = 0;
    while ((1 << bits) < N) ++bits;
    std::vector<int> idx(N);
    std::iota(idx.begin(), idx.end(), 0);
    auto rev = [&](int x) {
        int r = 0;
        for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
        return r;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return rev(a) < rev(b); });
    return idx;
}

// Householder QR of A (rows x cols, ld lda) in place: R in the upper triangle, the
// reflectors below it, T factors of each panel in Tall.  When stop2 >= 0 the factorisation
// stops after the first panel whose remaining trailing block has squared Frobenius norm
// <= stop2.  Returns the number of rows of R produced in *kk and panels in *npan.
struct HqrWork {
    c128 *V = nullptr, *W = nullptr, *W2 = nullptr, *tau = nullptr, *Tall = nullptr, *alpha = nullptr,
         *part2 = nullptr, *part3 = nullptr, *Yb = nullptr;
    double *part = nullptr, *dnorm = nullptr;
    c128 *px = nullptr, *py = nullptr;
    unsigned* bar = nullptr;
    int G = 0;
    cudaStream_t st = nullptr;
    int alloc(int64_t rows, int cols, int kmax, cudaStream_t s) {
        st = s;
        int dev = 0, nsm = 0, occ = 0;
        RSRR_CUDA(cudaGetDevice(&dev));
        RSRR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        RSRR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hqr_panel_kernel, 256, 0));
        if (occ < 1) return set_error(RSRR_ECUDA, "panel kernel cannot be resident");
        G = nsm;
        const int np = (int)ceil_div(kmax, kPB);
        RSRR_TRY(dalloc_n(&V, (size_t)rows * kPB, s));
        RSRR_TRY(dalloc_n(&W, (size_t)kPB * cols, s));
        RSRR_TRY(dalloc_n(&W2, (size_t)kPB * cols, s));
        RSRR_TRY(dalloc_n(&tau, (size_t)kmax, s));
        RSRR_TRY(dalloc_n(&Tall, (size_t)np * kPB * kPB, s));
        RSRR_TRY(dalloc_n(&alpha, 1, s));
        RSRR_TRY(dalloc_n(&part, (size_t)G, s));
        RSRR_TRY(dalloc_n(&part2, (size_t)G * kPB, s));
        RSRR_TRY(dalloc_n(&part3, (size_t)G * kPB * kPB, s));
        RSRR_TRY(dalloc_n(&Yb, (size_t)kPB * kPB, s));
        RSRR_TRY(dalloc_n(&bar, kGridBarWords, s));
        RSRR_TRY(dalloc_n(&dnorm, 1, s));
        RSRR_TRY(dalloc_n(&px, (size_t)cols, s));
        RSRR_TRY(dalloc_n(&py, (size_t)rows, s));
        RSRR_CUDA(cudaMemsetAsync(bar, 0, kGridBarWords * sizeof(unsigned), s));
        return RSRR_OK;
    }
    ~HqrWork() {
        for (void* p : {(void*)V, (void*)W, (void*)W2, (void*)tau, (void*)Tall, (void*)alpha, (void*)part2,
                        (void*)part3, (void*)Yb, (void*)part, (void*)dnorm, (void*)bar, (void*)px, (void*)py})
            dfree(p, st);
    }
};

int block_norm2_est(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, int iters, c128* x, c128* y,
                    double* dn, cudaStream_t st, double* est);

// stop_norm >= 0: stop after the first panel whose remaining trailing block has 2-norm at most
// stop_norm, tested by the Frobenius norm (an upper bound) or, once that is within
// sqrt(min(rows, cols)) of the target, by three times a power-iteration estimate.
int householder_qr(c128* A, int64_t rows, int cols, int64_t lda, HqrWork& w, double stop_norm, int* kk_out,
                   int* npan_out) {
    cudaStream_t st = w.st;
    const int kmax = (int)std::min<int64_t>(rows, cols);
    int kk = 0, npan = 0;
    for (int kb = 0; kb < kmax; kb += kPB) {
        const int bw = std::min(kPB, kmax - kb);
        PanelArgs pa{A, lda, (int)rows, kb, bw, w.tau, w.Tall + (int64_t)npan * kPB * kPB, w.part, w.alpha,
                     w.part2, w.part3, w.Yb, grid_bar_at(w.bar)};
        void* args[] = {&pa};
        RSRR_CUDA(cudaLaunchCooperativeKernel((void*)hqr_panel_kernel, w.G, 256, args, 0, st));
        note_launch();
        ++npan;
        kk = kb + bw;
        const int mt = cols - kk;
        if (mt > 0) {
            { extract_v_kernel<<<(unsigned)ceil_div((rows - kb) * bw, 256), 256, 0, st>>>(A, lda, (int)rows, kb, bw, w.V, rows); note_launch(); }
            Zgemm g1;
            g1.opA = OP_C; g1.opB = OP_N; g1.M = bw; g1.N = mt; g1.K = (int)(rows - kb);
            g1.A = w.V; g1.lda = rows; g1.B = A + kb + (int64_t)kk * lda; g1.ldb = lda; g1.C = w.W; g1.ldc = kPB;
            RSRR_TRY(zgemm(g1, st));
            Zgemm g2;
            g2.opA = OP_C; g2.opB = OP_N; g2.M = bw; g2.N = mt; g2.K = bw;
            g2.A = w.Tall + (int64_t)(npan - 1) * kPB * kPB; g2.lda = bw; g2.B = w.W; g2.ldb = kPB; g2.C = w.W2;
            g2.ldc = kPB;
            RSRR_TRY(zgemm(g2, st));
            Zgemm g3;
            g3.opA = OP_N; g3.opB = OP_N; g3.M = (int)(rows - kb); g3.N = mt; g3.K = bw;
            g3.alpha = mk<double>(-1.0, 0.0); g3.beta = mk<double>(1.0, 0.0);
            g3.A = w.V; g3.lda = rows; g3.B = w.W2; g3.ldb = kPB; g3.C = A + kb + (int64_t)kk * lda; g3.ldc = lda;
            g3.ksplit = 1;
            RSRR_TRY(zgemm(g3, st));
        }
        int berr = 0;
        double tn2 = 0.0;
        if (stop_norm >= 0.0) {
            RSRR_CUDA(cudaMemsetAsync(w.dnorm, 0, 8, st));
            block_norm2(A, lda, kk, (int)rows, kk, cols, w.dnorm, st);
            RSRR_CUDA(cudaMemcpyAsync(&tn2, w.dnorm, 8, cudaMemcpyDeviceToHost, st));
        }
        RSRR_CUDA(cudaMemcpyAsync(&berr, w.bar + kGridBarErrWord, 4, cudaMemcpyDeviceToHost, st));
        RSRR_CUDA(cudaStreamSynchronize(st));
        if (berr) return set_error(RSRR_ETIMEOUT, "grid barrier gave up in the panel kernel");
        if (!std::isfinite(tn2)) return set_error(RSRR_ENONFINITE, "non-finite QR");
        if (stop_norm >= 0.0 && kk < kmax) {
            const double fro = sqrt(tn2);
            if (fro <= stop_norm) break;
            const double dimf = sqrt((double)std::min<int64_t>(rows - kk, cols - kk));
            if (fro <= stop_norm * dimf) {
                double est = 0.0;
                RSRR_TRY(block_norm2_est(A, lda, kk, (int)rows, kk, cols, 12, w.px, w.py, w.dnorm, st, &est));
                if (3.0 * est <= stop_norm) break;
            }
        }
    }
    *kk_out = kk;
    *npan_out = npan;
    return RSRR_OK;
}

// y = A x for the block rows [r0, r1) x cols [c0, c1) (one thread per row)
// Y (n x ncols, leading dimension n) <- Q Y with Q = H_0 H_1 ... from the reflectors that
// householder_qr left in A (npan panels, kmax columns): the panels in reverse, each as
// Y -= V (T (V^H Y)) with two work blocks Z, Z2 of kPB x ncols.
int apply_q(const c128* A, int64_t n, int npan, int kmax, HqrWork& hw, c128* Y, int ncols, c128* Z, c128* Z2,
            cudaStream_t st) {
    for (int p = npan - 1; p >= 0; --p) {
        const int kb = p * kPB, bw = std::min(kPB, kmax - kb);
        { extract_v_kernel<<<(unsigned)ceil_div((n - kb) * bw, 256), 256, 0, st>>>(A, n, (int)n, kb, bw, hw.V, n); note_launch(); }
        Zgemm g1;
        g1.opA = OP_C; g1.opB = OP_N; g1.M = bw; g1.N = ncols; g1.K = (int)(n - kb);
        g1.A = hw.V; g1.lda = n; g1.B = Y + kb; g1.ldb = n; g1.C = Z; g1.ldc = kPB;
        RSRR_TRY(zgemm(g1, st));
        Zgemm g2;
        g2.opA = OP_N; g2.opB = OP_N; g2.M = bw; g2.N = ncols; g2.K = bw;
        g2.A = hw.Tall + (int64_t)p * kPB * kPB; g2.lda = bw; g2.B = Z; g2.ldb = kPB; g2.C = Z2; g2.ldc = kPB;
        RSRR_TRY(zgemm(g2, st));
        Zgemm g3;
        g3.opA = OP_N; g3.opB = OP_N; g3.M = (int)(n - kb); g3.N = ncols; g3.K = bw;
        g3.alpha = mk<double>(-1.0, 0.0); g3.beta = mk<double>(1.0, 0.0);
        g3.A = hw.V; g3.lda = n; g3.B = Z2; g3.ldb = kPB; g3.C = Y + kb; g3.ldc = n; g3.ksplit = 1;
        RSRR_TRY(zgemm(g3, st));
    }
    return RSRR_OK;
}

__global__ void gemv_n_kernel(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, const c128* x, c128* y) {
    const int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r1) return;
    c128 acc = czero<double>();
    // unrolled so that the loads of several columns are in flight; the sum keeps its order
#pragma unroll 8
    for (int c = c0; c < c1; ++c) cfma(acc, A[i + (int64_t)c * lda], x[c - c0]);
    y[i - r0] = acc;
}
// x = A^H y for the same block (one warp per column); also accumulates ||x||^2 into *nrm
__global__ void gemv_c_kernel(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, const c128* y, c128* x,
                              double* nrm) {
    const int c = c0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= c1) return;
    c128 acc = czero<double>();
#pragma unroll 8
    for (int i = r0 + lane; i < r1; i += 32) cfma_conj(acc, A[i + (int64_t)c * lda], y[i - r0]);
    for (int off = 16; off; off >>= 1) {
        acc.re += __shfl_down_sync(0xffffffffu, acc.re, off);
        acc.im += __shfl_down_sync(0xffffffffu, acc.im, off);
    }
    if (lane == 0) {
        x[c - c0] = acc;
        atomicAdd(nrm, cnorm2(acc));
    }
}
__global__ void scale_vec_kernel(c128* x, int n, const double* nrm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = cscale(x[i], 1.0 / sqrt(fmax(*nrm, 1e-300)));
}
__global__ void seed_vec_kernel(c128* x, int n) {  // fixed pseudo-random start vector
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned h = 2166136261u ^ (unsigned)i;
    h *= 16777619u; h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
    x[i] = mk<double>(((h & 0xffff) / 65536.0) - 0.5, ((h >> 16) / 65536.0) - 0.5);
}

// Power-iteration estimate of the 2-norm of the block (a lower bound that converges from
// below; the caller applies a safety factor).
int block_norm2_est(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, int iters, c128* x, c128* y,
                    double* dn, cudaStream_t st, double* est) {
    const int nr = r1 - r0, nc = c1 - c0;
    *est = 0.0;
    if (nr <= 0 || nc <= 0) return RSRR_OK;
    { seed_vec_kernel<<<(unsigned)ceil_div(nc, 256), 256, 0, st>>>(x, nc); note_launch(); }
    double prev = 0.0, cur = 0.0;
    for (int it = 0; it < iters; ++it) {
        { gemv_n_kernel<<<(unsigned)ceil_div(nr, 128), 128, 0, st>>>(A, lda, r0, r1, c0, c1, x, y); note_launch(); }
        RSRR_CUDA(cudaMemsetAsync(dn, 0, 8, st));
        { gemv_c_kernel<<<(unsigned)ceil_div(nc, 8), 256, 0, st>>>(A, lda, r0, r1, c0, c1, y, x, dn); note_launch(); }
        double h2 = 0.0;
        RSRR_CUDA(cudaMemcpyAsync(&h2, dn, 8, cudaMemcpyDeviceToHost, st));
        { scale_vec_kernel<<<(unsigned)ceil_div(nc, 256), 256, 0, st>>>(x, nc, dn); note_launch(); }
        RSRR_CUDA(cudaStreamSynchronize(st));
        // x had unit norm (after the first step): ||A^H A x|| -> sigma_max^2
        cur = (it == 0) ? 0.0 : sqrt(sqrt(h2));
        if (it >= 2 && cur <= 1.02 * prev) { prev = cur; break; }
        prev = cur;
    }
    *est = prev;
    return RSRR_OK;
}

// upper triangle (rows < k, cols < k) of a factored matrix into a dense k x k matrix
__global__ void upper_kernel(const c128* A, int64_t lda, int k, c128* R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    const int r = (int)(idx % k), c = (int)(idx / k);
    R[idx] = (r <= c) ? A[r + (int64_t)c * lda] : czero<double>();
}

}  // namespace

namespace {
struct PhaseClock {  // device time between successive marks on one stream
    cudaStream_t s;
    cudaEvent_t e[8];
    int k = 0;
    explicit PhaseClock(cudaStream_t st) : s(st) { for (auto& x : e) cudaEventCreate(&x); }
    ~PhaseClock() { for (auto& x : e) cudaEventDestroy(x); }
    void mark() { if (k < 8) cudaEventRecord(e[k++], s); }
    double ms(int i) {  // between mark i and i+1
        if (i + 1 >= k) return 0.0;
        cudaEventSynchronize(e[i + 1]);
        float t = 0.f;
        cudaEventElapsedTime(&t, e[i], e[i + 1]);
        return t;
    }
};
}  // namespace

int project_run(rsrr_nep h, double delta) {
    cudaStream_t st = h->stream;
    PhaseClock pc(st);
    pc.mark();
    zgemm_profile_begin();
    jacobi_profile_begin();
    const int64_t n = h->n;
    const int N = h->N, L = h->L, J = h->J;
    const int Kp = h->moment_order;
    const int m = Kp > 0 ? Kp * L : N * L;
    const int kmax = (int)std::min<int64_t>(n, m);
    h->proj_cols = m;
    dfree(h->d_Q, st);
    dfree(h->d_P, st);
    h->d_Q = nullptr;
    h->d_P = nullptr;
    h->red_fns = h->fns;  // the reduced NEP keeps T's own functions: P_i = S^H A_i S
    h->red_J = h->tz ? 0 : J;  // a tz handle has no A_i: its reduced NEP comes from chebyshev_reduce

    c128 *A = nullptr, *V = nullptr, *W = nullptr, *W2 = nullptr, *tau = nullptr, *Tall = nullptr,
         *alpha = nullptr, *part2 = nullptr, *part3 = nullptr, *Yb = nullptr, *B = nullptr, *Jm = nullptr,
         *Ybuf = nullptr, *Z = nullptr, *Z2 = nullptr, *AY = nullptr, *Eg = nullptr, *Jn = nullptr;
    double *part = nullptr, *dnorm = nullptr, *colnrm = nullptr;
    unsigned* bar = nullptr;
    int *order_d = nullptr, *cols_d = nullptr;
    int rc = RSRR_OK;
    auto cleanup = [&]() {
        double zm, zf;
        zgemm_profile_end(&zm, &zf);
        jacobi_profile_end(&zm, &zf);
        for (void* p : {(void*)A, (void*)V, (void*)W, (void*)W2, (void*)tau, (void*)Tall, (void*)alpha,
                        (void*)part2, (void*)part3, (void*)Yb, (void*)B, (void*)Jm, (void*)Ybuf, (void*)Z,
                        (void*)Z2, (void*)AY, (void*)Eg, (void*)Jn, (void*)part, (void*)dnorm, (void*)colnrm, (void*)bar,
                        (void*)order_d, (void*)cols_d})
            dfree(p, st);
    };
#define TRYC(expr) do { rc = (expr); if (rc != RSRR_OK) { cleanup(); return rc; } } while (0)
#define CUDAC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return set_error(RSRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)

    int dev = 0, nsm = 0, occ = 0;
    CUDAC(cudaGetDevice(&dev));
    CUDAC(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDAC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hqr_panel_kernel, 256, 0));
    if (occ < 1) { cleanup(); return set_error(RSRR_ECUDA, "panel kernel cannot be resident"); }

    TRYC(dalloc_n(&A, (size_t)n * m, st));
    if (Kp > 0) {
        // ---- SSRR moment scheme (Eqs. eq-malpha-qud, eq-hatM, eq-hatMS): M_hat = S_hat D Z ------
        // Column block alpha is sum_i w_i zeta_i^alpha X_i with the contour rule's weights w_i of
        // (1 / 2 pi i) oint dz (trapezoid on the ellipse: phi'(theta_i) / (i N); Gauss-Legendre on
        // a rectangle's sides) and zeta_i = (z_i - gamma) / rho, rho = max(a, b) (a change of
        // polynomial basis: the same span as z_i^alpha, better scaled).
        // D Z is block diagonal in the probe index, so it is one NL x K'L matrix and one ZGEMM.
        std::vector<zd> z, wq;
        contour_rule(h->C, N, &z, &wq, h->C.side_nodes);
        const zd gamma(h->C.gamma_re, h->C.gamma_im);
        const double rho = std::max(h->C.a, h->C.b);
        std::vector<c128> Wt((size_t)N * L * m, czero<double>());
        for (int i = 0; i < N; ++i) {
            const zd wi = wq[i], zeta = (z[i] - gamma) / rho;
            zd p = wi;
            for (int al = 0; al < Kp; ++al, p *= zeta)
                for (int l = 0; l < L; ++l) Wt[(size_t)(i * L + l) + (size_t)(al * L + l) * N * L] = fromstd(p);
        }
        TRYC(dalloc_n(&Z, Wt.size(), st));
        CUDAC(cudaMemcpyAsync(Z, Wt.data(), Wt.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
        Zgemm gm;
        gm.opA = OP_N; gm.opB = OP_N; gm.M = (int)n; gm.N = m; gm.K = N * L;
        gm.A = h->d_S; gm.lda = n; gm.B = Z; gm.ldb = N * L; gm.C = A; gm.ldc = n;
        gm.ksplit = 1;
        TRYC(zgemm(gm, st));
        CUDAC(cudaStreamSynchronize(st));
        dfree(Z, st);
        Z = nullptr;
    } else {
        // ---- work copy of S_hat with point blocks in bit-reversed order --------------------------
        std::vector<int> order = bit_reversed_order(N);
        TRYC(dalloc_n(&order_d, (size_t)N, st));
        CUDAC(cudaMemcpyAsync(order_d, order.data(), N * 4, cudaMemcpyHostToDevice, st));
        { gather_blocks_kernel<<<(unsigned)ceil_div(n * m, 256), 256, 0, st>>>(h->d_S, n, L, order_d, m, A); note_launch(); }
    }
    // reference size for the stopping rule: max column norm of S_hat (<= sigma_1)
    TRYC(dalloc_n(&colnrm, (size_t)m, st));
    column_norms(A, (int)n, m, n, colnrm, st);
    std::vector<double> cn(m);
    CUDAC(cudaMemcpyAsync(cn.data(), colnrm, m * 8, cudaMemcpyDeviceToHost, st));
    CUDAC(cudaStreamSynchronize(st));
    const double smax = *std::max_element(cn.begin(), cn.end());
    if (!std::isfinite(smax)) { cleanup(); return set_error(RSRR_ENONFINITE, "non-finite sample matrix"); }

    // ---- Householder QR with early termination -----------------------------------------------
    // stop once the trailing block's 2-norm is below 0.1 delta sigma_1 (or the noise level
    // below): dropping it moves no
    // singular value by more than a tenth of the truncation level (Weyl).  sigma_1 is taken
    // from a power-iteration estimate of ||S_hat||_2 (a lower bound, so the rule stays safe).
    HqrWork hw;
    TRYC(hw.alloc(n, m, kmax, st));
    double s1_est = 0.0;
    TRYC(block_norm2_est(A, n, 0, (int)n, 0, m, 30, hw.px, hw.py, hw.dnorm, st, &s1_est));
    const double sref = std::max(smax, s1_est);
    // The stop level is raised to the rounding noise of S_hat itself when that is higher, up
    // to 0.3 delta sigma_1: in FP64 the trailing block of the QR levels off near u ||S_hat||_F
    // (measured: a plateau at 0.7-0.9e-15 sigma_1 on the damped QEP, just under 0.1 delta
    // sigma_1, so the stop point swung by hundreds of rows with the rounding), and rows at that
    // level resolve no singular value.  Dropping a block of norm <= 0.3 delta sigma_1 still moves
    // no singular value by more than that (Weyl).
    double fro2 = 0.0;
    for (double c : cn) fro2 += c * c;
    const double noise = std::min(8.0 * 1.1102230246251565e-16 * std::sqrt(fro2), 0.3 * delta * sref);
    int kk = 0, npan = 0;
    TRYC(householder_qr(A, n, m, n, hw, std::max(0.1 * delta * sref, noise), &kk, &npan));
    pc.mark();  // QR done
    // ---- SVD of R_keep (kk x m) ---------------------------------------------------------------
    // R_keep^H = Q2 R2 (a second QR, only R2 kept), so R_keep = R2^H Q2^H and the left singular
    // vectors of R_keep are those of R2^H.  One-sided Jacobi on the columns of R2 with the
    // rotations accumulated: R2 J = W orthogonal => R2^H = J Sigma (W Sigma^{-1})^H.
    TRYC(dalloc_n(&B, (size_t)m * kk, st));
    { rkeep_h_kernel<<<(unsigned)ceil_div((int64_t)m * kk, 256), 256, 0, st>>>(A, n, m, kk, B); note_launch(); }
    c128* R2 = nullptr;
    {
        HqrWork hw2;
        TRYC(hw2.alloc(m, kk, std::min(m, kk), st));
        int kk2 = 0, np2 = 0;
        TRYC(householder_qr(B, m, kk, m, hw2, -1.0, &kk2, &np2));
        TRYC(dalloc_n(&R2, (size_t)kk * kk, st));
        const int kr = std::min(m, kk);
        CUDAC(cudaMemsetAsync(R2, 0, (size_t)kk * kk * sizeof(c128), st));
        { upper_kernel<<<(unsigned)ceil_div((int64_t)kk * kk, 256), 256, 0, st>>>(B, m, kk, R2); note_launch(); }
        (void)kr;
    }
    TRYC(dalloc_n(&Jm, (size_t)kk * kk, st));
    { identity_kernel<<<(unsigned)ceil_div((int64_t)kk * kk, 256), 256, 0, st>>>(Jm, kk); note_launch(); }
    int sweeps = 0;
    // Columns below 0.3 delta sigma_1 are rounding noise of R2 (its entries carry errors of
    // ~u sigma_1, so such columns never settle): they are not rotated.  A rotation against a
    // column of norm eps moves any other column by O(eps), and such columns stay below the
    // truncation level.  Kept-subspace accuracy needs pairs orthogonal to ~1e-10 only.  (An
    // absolute cut on the inner product, |<a, b>| < c sigma_1^2, stops rotating pairs of small
    // columns before their norms separate and miscounts the singular values near delta sigma_1,
    // so pairs are judged only relative to their own norms.)
    TRYC(jacobi_orthogonalize(R2, kk, kk, Jm, st, 40, &sweeps, 0.3 * delta * sref, 1e-10, 0.0));
    h->jacobi_sweeps_project = sweeps;
    h->rows_kept = kk;
    dfree(colnrm, st);
    colnrm = nullptr;
    TRYC(dalloc_n(&colnrm, (size_t)kk, st));
    column_norms(R2, kk, kk, kk, colnrm, st);
    dfree(R2, st);
    std::vector<double> sv(kk);
    CUDAC(cudaMemcpyAsync(sv.data(), colnrm, kk * 8, cudaMemcpyDeviceToHost, st));
    CUDAC(cudaStreamSynchronize(st));
    std::vector<int> idx(kk);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return sv[x] > sv[y]; });
    h->sigma.assign((size_t)std::min<int64_t>(n, m), 0.0);
    for (int i = 0; i < kk; ++i) h->sigma[i] = sv[idx[i]];
    const double s1 = kk ? h->sigma[0] : 0.0;
    int kS = 0;
    while (kS < kk && h->sigma[kS] > delta * s1) ++kS;
    if (s1 == 0.0) kS = 0;
    h->kS = kS;

    pc.mark();  // SVD done
    // ---- S = Q [J(:, idx[:kS]); 0] ------------------------------------------------------------
    if (kS > 0) {
        TRYC(dalloc_n(&cols_d, (size_t)kS, st));
        CUDAC(cudaMemcpyAsync(cols_d, idx.data(), kS * 4, cudaMemcpyHostToDevice, st));
        TRYC(dalloc_n(&Ybuf, (size_t)n * kS, st));
        { init_y_kernel<<<(unsigned)ceil_div(n * kS, 256), 256, 0, st>>>(Jm, kk, cols_d, kS, n, Ybuf); note_launch(); }
        // J is a product of many thousands of plane rotations, and its columns drift from
        // orthonormal by about sqrt(rotations) u each (1e-13 in the 2-norm after tens of sweeps
        // over a few hundred columns).  One Newton-Schulz step, J <- J (I - E / 2) with
        // E = J^H J - I, makes them orthonormal to O(|E|^2) and leaves span(J) unchanged.
        TRYC(dalloc_n(&Eg, (size_t)kS * kS, st));
        { identity_kernel<<<(unsigned)ceil_div((int64_t)kS * kS, 256), 256, 0, st>>>(Eg, kS); note_launch(); }
        Zgemm ge;
        ge.opA = OP_C; ge.opB = OP_N; ge.M = kS; ge.N = kS; ge.K = kk;
        ge.beta = mk<double>(-1.0, 0.0);
        ge.A = Ybuf; ge.lda = n; ge.B = Ybuf; ge.ldb = n; ge.C = Eg; ge.ldc = kS;
        TRYC(zgemm(ge, st));
        TRYC(dalloc_n(&Jn, (size_t)kk * kS, st));
        CUDAC(cudaMemcpy2DAsync(Jn, (size_t)kk * sizeof(c128), Ybuf, (size_t)n * sizeof(c128), (size_t)kk * sizeof(c128),
                                kS, cudaMemcpyDeviceToDevice, st));
        Zgemm gn;
        gn.M = kk; gn.N = kS; gn.K = kS;
        gn.alpha = mk<double>(-0.5, 0.0); gn.beta = mk<double>(1.0, 0.0);
        gn.A = Ybuf; gn.lda = n; gn.B = Eg; gn.ldb = kS; gn.C = Jn; gn.ldc = kk; gn.ksplit = 1;
        TRYC(zgemm(gn, st));
        CUDAC(cudaMemcpy2DAsync(Ybuf, (size_t)n * sizeof(c128), Jn, (size_t)kk * sizeof(c128), (size_t)kk * sizeof(c128),
                                kS, cudaMemcpyDeviceToDevice, st));
        TRYC(dalloc_n(&Z, (size_t)kPB * kS, st));
        TRYC(dalloc_n(&Z2, (size_t)kPB * kS, st));
        TRYC(apply_q(A, n, npan, kmax, hw, Ybuf, kS, Z, Z2, st));
        pc.mark();  // basis done
        if (h->tz) {  // no A_i: rsrr_project_chebyshev forms the reduced NEP from T(x_k)
            h->d_Q = Ybuf;
            Ybuf = nullptr;
            pc.mark();
            CUDAC(cudaStreamSynchronize(st));
            for (int i = 0; i < 4; ++i) h->ms_project_parts[i] = pc.ms(i);
            zgemm_profile_end(&h->ms_zgemm_project, &h->zgemm_flops_project, &h->ms_zgemm_tc_project,
                              &h->zgemm_tc_flops_project);
            jacobi_profile_end(&h->ms_jacobi_project, &h->jacobi_flops_project);
            cleanup();
            return RSRR_OK;
        }
        // ---- P_i = S^H (A_i S) ---------------------------------------------------------------
        TRYC(dalloc_n(&AY, (size_t)J * n * kS, st));
        dim3 gs((unsigned)ceil_div(n * kS, 256), J);
        { spmm_terms_kernel<<<gs, 256, 0, st>>>(h->d_rowptr, h->d_colind, h->d_vals, h->nnz, n, Ybuf, kS, AY); note_launch(); }
        TRYC(dalloc_n(&h->d_P, (size_t)J * kS * kS, st));
        Zgemm gp;
        gp.opA = OP_C; gp.opB = OP_N; gp.M = kS; gp.N = kS; gp.K = (int)n;
        gp.A = Ybuf; gp.lda = n; gp.sA = 0; gp.B = AY; gp.ldb = n; gp.sB = n * kS;
        gp.C = h->d_P; gp.ldc = kS; gp.sC = (int64_t)kS * kS; gp.batch = J;
        TRYC(zgemm(gp, st));
        h->d_Q = Ybuf;
        Ybuf = nullptr;
        pc.mark();  // projection done
    }
    CUDAC(cudaStreamSynchronize(st));
    for (int i = 0; i < 4; ++i) h->ms_project_parts[i] = pc.ms(i);
    zgemm_profile_end(&h->ms_zgemm_project, &h->zgemm_flops_project, &h->ms_zgemm_tc_project,
                      &h->zgemm_tc_flops_project);
    jacobi_profile_end(&h->ms_jacobi_project, &h->jacobi_flops_project);
    cleanup();
#undef TRYC
#undef CUDAC
    return RSRR_OK;
}

// ---------------------------------------------------------------------------------------------
// Section 6.2 (Eqs. eq-T-interp, eq-Ts-interp, eq-Ts-coefs): the reduced NEP replaced by its
// degree-d Chebyshev interpolant on [lo, hi].  With T = sum_i f_i A_i, S^H T(x_k) S is
// sum_i f_i(x_k) P_i, so P_hat_j = sum_i W[i][j] P_i with W[i][j] = sum_k f_i(x_k) c_kj and
// c_kj = (2 / (d + 1)) cos(j theta_k) (halved for j = 0): one ZGEMM of the k_S^2 x J matrix of
// the P_i against the J x (d + 1) matrix W.
// ---------------------------------------------------------------------------------------------
// A tz handle has no P_i: Q_k = S^H T(x_k) S is formed from T's values at the Chebyshev points
// (SpMM, batched ZGEMM), then P_hat_j = sum_k c_kj Q_k is one more ZGEMM, as Eq. eq-Ts-coefs.
int chebyshev_reduce_tz(rsrr_nep h, int d, double lo, double hi) {
    cudaStream_t st = h->stream;
    const int k = h->kS, m = d + 1;
    const int64_t n = h->n, kk = (int64_t)k * k;
    const double pi = 3.14159265358979323846, c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    std::vector<zd> x(m);
    std::vector<c128> Cm((size_t)m * m);
    for (int kx = 0; kx < m; ++kx) {
        const double th = (kx + 0.5) * pi / m;
        x[kx] = zd(c + r * std::cos(th), 0.0);
        for (int j = 0; j < m; ++j)
            Cm[(size_t)kx + (size_t)j * m] = mk<double>((2.0 / m) * std::cos(j * th) * (j == 0 ? 0.5 : 1.0), 0.0);
    }
    std::vector<rsrr_fn> fns(m);
    for (int j = 0; j < m; ++j) {
        fns[j] = rsrr_fn{};
        fns[j].kind = RSRR_F_CHEBYSHEV;
        fns[j].p[0] = j;
        fns[j].p[1] = lo;
        fns[j].p[2] = hi;
    }
    if (k > 0) {
        c128 *vals = nullptr, *AY = nullptr, *Q = nullptr, *Cd = nullptr, *Pn = nullptr;
        auto release = [&]() { for (c128* p : {vals, AY, Q, Cd}) dfree(p, st); };
        int rc = tz_values(h, x, &vals);
        if (rc == RSRR_OK) rc = dalloc_n(&AY, (size_t)m * n * k, st);
        if (rc == RSRR_OK) rc = dalloc_n(&Q, (size_t)m * kk, st);
        if (rc == RSRR_OK) rc = dalloc_n(&Cd, Cm.size(), st);
        if (rc == RSRR_OK) rc = dalloc_n(&Pn, (size_t)m * kk, st);
        if (rc != RSRR_OK) { release(); dfree(Pn, st); return rc; }
        cudaMemcpyAsync(Cd, Cm.data(), Cm.size() * sizeof(c128), cudaMemcpyHostToDevice, st);
        dim3 gs((unsigned)ceil_div(n * k, 256), m);
        { spmm_terms_kernel<<<gs, 256, 0, st>>>(h->d_rowptr, h->d_colind, vals, h->nnz, n, h->d_Q, k, AY); note_launch(); }
        Zgemm gq;  // Q_k = S^H (T(x_k) S)
        gq.opA = OP_C; gq.opB = OP_N; gq.M = k; gq.N = k; gq.K = (int)n;
        gq.A = h->d_Q; gq.lda = n; gq.sA = 0; gq.B = AY; gq.ldb = n; gq.sB = n * k;
        gq.C = Q; gq.ldc = k; gq.sC = kk; gq.batch = m;
        rc = zgemm(gq, st);
        if (rc == RSRR_OK) {
            Zgemm gc;  // P_hat = [Q_0 .. Q_d] C
            gc.M = (int)kk; gc.N = m; gc.K = m;
            gc.A = Q; gc.lda = kk; gc.B = Cd; gc.ldb = m; gc.C = Pn; gc.ldc = kk; gc.ksplit = 1;
            rc = zgemm(gc, st);
        }
        if (rc == RSRR_OK && cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_error(RSRR_ECUDA, "Chebyshev coefficients");
        release();
        if (rc != RSRR_OK) { dfree(Pn, st); return rc; }
        dfree(h->d_P, st);
        h->d_P = Pn;
    }
    h->red_fns = fns;
    h->red_J = m;
    return RSRR_OK;
}

int chebyshev_reduce(rsrr_nep h, int d, double lo, double hi) {
    if (h->tz) return chebyshev_reduce_tz(h, d, lo, hi);
    cudaStream_t st = h->stream;
    const int J = h->J, k = h->kS, m = d + 1;
    const double pi = 3.14159265358979323846, c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    std::vector<zd> W((size_t)J * m, zd(0.0, 0.0));
    for (int kx = 0; kx < m; ++kx) {
        const double th = (kx + 0.5) * pi / m, x = c + r * std::cos(th);
        for (int i = 0; i < J; ++i) {
            zd f, df;
            eval_fn(h->fns[i], zd(x, 0.0), &f, &df);
            if (!std::isfinite(std::abs(f)))
                return set_error(RSRR_ENONFINITE, "f_i is not finite at a Chebyshev point");
            for (int j = 0; j < m; ++j) {
                const double cj = (2.0 / m) * std::cos(j * th) * (j == 0 ? 0.5 : 1.0);
                W[(size_t)i + (size_t)j * J] += f * cj;
            }
        }
    }
    std::vector<rsrr_fn> fns(m);
    for (int j = 0; j < m; ++j) {
        fns[j] = rsrr_fn{};
        fns[j].kind = RSRR_F_CHEBYSHEV;
        fns[j].p[0] = j;
        fns[j].p[1] = lo;
        fns[j].p[2] = hi;
    }
    if (k > 0) {
        const int64_t kk = (int64_t)k * k;
        c128 *Wd = nullptr, *Pn = nullptr;
        RSRR_TRY(dalloc_n(&Wd, (size_t)J * m, st));
        int rc = dalloc_n(&Pn, (size_t)kk * m, st);
        if (rc != RSRR_OK) { dfree(Wd, st); return rc; }
        std::vector<c128> Wh(W.size());
        for (size_t e = 0; e < W.size(); ++e) Wh[e] = fromstd(W[e]);
        cudaMemcpyAsync(Wd, Wh.data(), Wh.size() * sizeof(c128), cudaMemcpyHostToDevice, st);
        Zgemm g;
        g.M = (int)kk; g.N = m; g.K = J;
        g.A = h->d_P; g.lda = kk; g.B = Wd; g.ldb = J; g.C = Pn; g.ldc = kk; g.ksplit = 1;
        rc = zgemm(g, st);
        if (rc == RSRR_OK && cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_error(RSRR_ECUDA, "Chebyshev coefficients");
        dfree(Wd, st);
        if (rc != RSRR_OK) { dfree(Pn, st); return rc; }
        dfree(h->d_P, st);
        h->d_P = Pn;
    }
    h->red_fns = fns;
    h->red_J = m;
    return RSRR_OK;
}

// ---------------------------------------------------------------------------------------------
// One-sided Jacobi SVD of a square D x D matrix H with a QR preconditioner (after Drmac and
// Veselic): the columns of H are put in order of decreasing norm, H P = Q R by Householder QR, and
// the one-sided Jacobi runs on X = R^H with its rotations accumulated, X J = W = U Sigma.  Then
// H = (Q J) Sigma (P U)^H.  The graded triangular factor converges in fewer sweeps than H itself
// (on the Hankel matrices of the reduced solve, 16 -> 12 sweeps in a replay of the same rotations).
// On return H holds (Q J) Sigma and Jr the right singular vectors P U: the same contract as a plain
// one-sided Jacobi of H with the rotations accumulated into Jr, which the callers' extraction uses.
// Columns below `floor` are not rotated (their right vectors come out as zero).
// ---------------------------------------------------------------------------------------------
namespace {
__global__ void permute_cols_kernel(const c128* src, int D, const int* perm, c128* dst) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)D * D) return;
    const int64_t r = idx % D, c = idx / D;
    dst[idx] = src[r + (int64_t)perm[c] * D];
}
// H[:, j] = Y[:, j] sigma_j;  Jr[perm[i], j] = W[i, j] / sigma_j  (zero where sigma_j is zero)
__global__ void svd_finish_kernel(const c128* W, const c128* Y, const double* sig, const int* perm, int D, c128* H,
                                  c128* Jr) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)D * D) return;
    const int64_t i = idx % D, j = idx / D;
    const double sj = sig[j], inv = sj > 0.0 ? 1.0 / sj : 0.0;
    H[idx] = cscale(Y[idx], sj);
    Jr[perm[i] + j * (int64_t)D] = cscale(W[idx], inv);
}
}  // namespace

int jacobi_svd_preconditioned(c128* H, int D, c128* Jr, cudaStream_t st, double floor, double conv, int* sweeps) {
    if (sweeps) *sweeps = 0;
    if (D < 2) return jacobi_orthogonalize(H, D, D, Jr, st, 40, sweeps, floor, conv, 0.0);
    const int64_t DD = (int64_t)D * D;
    c128 *A = nullptr, *X = nullptr, *Z = nullptr, *Z2 = nullptr;
    double* sig = nullptr;
    int* perm_d = nullptr;
    int rc = RSRR_OK;
    auto release = [&]() {
        for (void* q : {(void*)A, (void*)X, (void*)Z, (void*)Z2, (void*)sig, (void*)perm_d}) dfree(q, st);
    };
#define TRYR(expr) do { rc = (expr); if (rc != RSRR_OK) { release(); return rc; } } while (0)
    TRYR(dalloc_n(&A, (size_t)DD, st));
    TRYR(dalloc_n(&X, (size_t)DD, st));
    TRYR(dalloc_n(&Z, (size_t)kPB * D, st));
    TRYR(dalloc_n(&Z2, (size_t)kPB * D, st));
    TRYR(dalloc_n(&sig, (size_t)D, st));
    TRYR(dalloc_n(&perm_d, (size_t)D, st));
    // columns in order of decreasing norm
    column_norms(H, D, D, D, sig, st);
    std::vector<double> hn(D);
    if (cudaMemcpyAsync(hn.data(), sig, (size_t)D * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { release(); return set_error(RSRR_ECUDA, "column norms"); }
    std::vector<int> perm(D);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return hn[a] > hn[b]; });
    cudaMemcpyAsync(perm_d, perm.data(), (size_t)D * 4, cudaMemcpyHostToDevice, st);
    { permute_cols_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(H, D, perm_d, A); note_launch(); }
    // H P = Q R
    HqrWork hw;
    TRYR(hw.alloc(D, D, D, st));
    int kk = 0, npan = 0;
    TRYR(householder_qr(A, D, D, D, hw, -1.0, &kk, &npan));
    // X = R^H, then the Jacobi with the rotations accumulated into Jr (used as J here)
    { rkeep_h_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(A, D, D, D, X); note_launch(); }
    { identity_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(Jr, D); note_launch(); }
    TRYR(jacobi_orthogonalize(X, D, D, Jr, st, 40, sweeps, floor, conv, 0.0));
    // left singular vectors Q J (in place of J), sigma_j = |W_j|, right vectors P W Sigma^{-1}
    TRYR(apply_q(A, D, npan, kk, hw, Jr, D, Z, Z2, st));
    column_norms(X, D, D, D, sig, st);
    // the reflectors are no longer needed: A takes Q J while Jr receives the right vectors
    if (cudaMemcpyAsync(A, Jr, (size_t)DD * sizeof(c128), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        release();
        return set_error(RSRR_ECUDA, "copy of Q J");
    }
    { svd_finish_kernel<<<(unsigned)ceil_div(DD, 256), 256, 0, st>>>(X, A, sig, perm_d, D, H, Jr); note_launch(); }
    if (cudaStreamSynchronize(st) != cudaSuccess) { release(); return set_error(RSRR_ECUDA, "preconditioned Jacobi"); }
#undef TRYR
    release();
    return rc;
}

}  // namespace rsrr
