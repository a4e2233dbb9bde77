// Restarted flexible GMRES for the sample solves T(z_j) x = u of the iterative sampler
// (Algorithm 2, Step 2 done iteratively, as the paper does for its largest problems: GMRES with
// an incomplete factorisation as preconditioner, Section 7.3).
//
// Every (sampling point, probing column) pair is one system; all of them advance together.
// Vectors are FP64.  The preconditioner M^{-1} is the band LU of the band part of T(z_j)
// (complex64 or complex128), applied by the band solve kernels; because a complex64 solve of an
// FP64 vector is not exactly a fixed linear map, the flexible variant keeps the preconditioned
// vectors Z_k = M^{-1} V_k and forms x = x_0 + Z y.  Orthogonalisation is classical Gram-Schmidt
// applied twice (two batched dot-product / update passes per step), the small least-squares
// problem is updated with complex Givens rotations, one thread per system.
//
// Layout: the vector of system s = point * L + column is contiguous, at offset s * n of a block
// of np * L * n values (the same layout as the samples X and the work array of the solves).
#include <cmath>
#include <vector>

#include "krylov.cuh"

namespace rsrr {

namespace {

constexpr int KT = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    }
    return v;  // valid in thread 0
}

// W = U - T X (residual) or W = T Z (product), per point, CSR rows (one thread per row, all
// L columns).  U == nullptr selects the product.
__global__ void k_csr_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                             const c128* __restrict__ tvals, int64_t nnz, int64_t n, int L,
                             const c128* __restrict__ U, const c128* __restrict__ X, c128* __restrict__ W) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    if (r >= n) return;
    const c128* tv = tvals + (int64_t)pt * nnz;
    const int64_t k0 = rowptr[r], k1 = rowptr[r + 1];
    for (int l = 0; l < L; ++l) {
        const int64_t off = ((int64_t)pt * L + l) * n;
        c128 acc = U ? U[r + (int64_t)l * n] : czero<double>();
        for (int64_t k = k0; k < k1; ++k) {
            if (U) cfms(acc, tv[k], X[off + colind[k]]);
            else cfma(acc, tv[k], X[off + colind[k]]);
        }
        W[off + r] = acc;
    }
}

// h[s * ldh + i] = <V_i, W> over system s (grid: systems x nv)
__global__ void k_dot_kernel(const c128* __restrict__ V, int64_t vstride, const c128* __restrict__ W, int64_t n,
                             c128* __restrict__ h, int ldh) {
    __shared__ double red[32];
    const int64_t s = blockIdx.x;
    const int i = blockIdx.y;
    const c128* v = V + (int64_t)i * vstride + s * n;
    const c128* w = W + s * n;
    c128 acc = czero<double>();
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) cfma_conj(acc, v[r], w[r]);
    const double re = block_sum(acc.re, red);
    __syncthreads();
    const double im = block_sum(acc.im, red);
    if (threadIdx.x == 0) h[s * ldh + i] = mk<double>(re, im);
}

// W -= sum_{i < nv} h_i V_i
__global__ void k_axpy_kernel(const c128* __restrict__ V, int64_t vstride, int nv, const c128* __restrict__ h, int ldh,
                              c128* __restrict__ W, int64_t n, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t s = e / n;
    c128 w = W[e];
    for (int i = 0; i < nv; ++i) cfms(w, h[s * ldh + i], V[(int64_t)i * vstride + e]);
    W[e] = w;
}

__global__ void k_norm_kernel(const c128* __restrict__ W, int64_t n, double* __restrict__ nrm) {
    __shared__ double red[32];
    const int64_t s = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += cnorm2(W[s * n + r]);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) nrm[s] = sqrt(acc);
}

// Vout = W / nrm (a zero vector stays zero: the Krylov space is exhausted for that system)
__global__ void k_scale_kernel(const c128* __restrict__ W, const double* __restrict__ nrm, c128* __restrict__ Vout,
                               int64_t n, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const double a = nrm[e / n];
    Vout[e] = a > 0.0 ? cscale(W[e], 1.0 / a) : czero<double>();
}

template <typename R>
__global__ void k_down_kernel(const c128* __restrict__ V, cplx<R>* __restrict__ B, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) B[e] = ccast<R>(V[e]);
}
template <typename R>
__global__ void k_up_kernel(const cplx<R>* __restrict__ B, c128* __restrict__ Z, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) Z[e] = ccast<double>(B[e]);
}

// g = beta e_1, target from ||x|| and ||u||, per system
__global__ void k_start_kernel(int S, int m, int L, const double* __restrict__ beta, double* __restrict__ res,
                               c128* __restrict__ g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    for (int i = 0; i <= m; ++i) g[(int64_t)s * (m + 1) + i] = czero<double>();
    g[(int64_t)s * (m + 1)] = mk<double>(beta[s], 0.0);
    res[s] = beta[s];
}

// Column k of the Hessenberg matrix (h1 + h2 from the two Gram-Schmidt passes, nrm below the
// diagonal), the earlier rotations applied to it, a new rotation that zeroes its subdiagonal,
// applied to g as well; res = |g_{k+1}|, the residual norm of the current iterate.
__global__ void k_givens_kernel(int k, int m, int S, const c128* __restrict__ h1, const c128* __restrict__ h2, int ldh,
                                const double* __restrict__ nrm, c128* __restrict__ H, double* __restrict__ cs,
                                c128* __restrict__ sn, c128* __restrict__ g, double* __restrict__ res) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    c128* Hk = H + (int64_t)s * (m + 1) * m + (int64_t)k * (m + 1);
    for (int i = 0; i <= k; ++i) Hk[i] = h1[(int64_t)s * ldh + i] + h2[(int64_t)s * ldh + i];
    c128 sub = mk<double>(nrm[s], 0.0);
    double* c = cs + (int64_t)s * m;
    c128* sv = sn + (int64_t)s * m;
    for (int j = 0; j < k; ++j) {
        const c128 a = Hk[j], b = Hk[j + 1];
        Hk[j] = cscale(a, c[j]) + sv[j] * b;
        Hk[j + 1] = cscale(b, c[j]) - cconj(sv[j]) * a;
    }
    const c128 a = Hk[k];
    const double aa = sqrt(cnorm2(a)), bb = sqrt(cnorm2(sub));
    double cc;
    c128 ss, rho;
    if (bb == 0.0) {
        cc = 1.0;
        ss = czero<double>();
        rho = a;
    } else if (aa == 0.0) {
        cc = 0.0;
        ss = mk<double>(1.0, 0.0);
        rho = sub;
    } else {
        const double r = hypot(aa, bb);
        const c128 ph = cscale(a, 1.0 / aa);  // a / |a|
        cc = aa / r;
        ss = cscale(ph * cconj(sub), 1.0 / r);
        rho = cscale(ph, r);
    }
    c[k] = cc;
    sv[k] = ss;
    Hk[k] = rho;
    Hk[k + 1] = czero<double>();
    c128* gs = g + (int64_t)s * (m + 1);
    const c128 gk = gs[k];
    gs[k] = cscale(gk, cc);
    gs[k + 1] = czero<double>() - cconj(ss) * gk;
    res[s] = sqrt(cnorm2(gs[k + 1]));
}

// y = R^{-1} g with R the leading kk x kk block of the rotated Hessenberg matrix
__global__ void k_backsolve_kernel(int kk, int m, int S, const c128* __restrict__ H, const c128* __restrict__ g,
                                   c128* __restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const c128* Hs = H + (int64_t)s * (m + 1) * m;
    c128* ys = y + (int64_t)s * m;
    for (int i = kk - 1; i >= 0; --i) {
        c128 v = g[(int64_t)s * (m + 1) + i];
        for (int j = i + 1; j < kk; ++j) cfms(v, Hs[(int64_t)j * (m + 1) + i], ys[j]);
        const c128 d = Hs[(int64_t)i * (m + 1) + i];
        ys[i] = cis_zero(d) ? czero<double>() : v * crecip(d);
    }
}

// X += sum_{j < kk} y_j Z_j
__global__ void k_xupdate_kernel(const c128* __restrict__ Z, int64_t vstride, int kk, const c128* __restrict__ y, int m,
                                 c128* __restrict__ X, int64_t n, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t s = e / n;
    c128 x = X[e];
    for (int j = 0; j < kk; ++j) cfma(x, y[s * m + j], Z[(int64_t)j * vstride + e]);
    X[e] = x;
}

// target_s = tau (||T||_1 ||x_s|| + ||u_s||): the residual that gives eta <= tau for the x of
// the cycle's start (x changes little within a cycle once it is close)
__global__ void k_target_kernel(int S, int L, double tau, const double* __restrict__ xn, const double* __restrict__ un2,
                                const double* __restrict__ normT, double* __restrict__ target) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    target[s] = tau * (normT[s / L] * xn[s] + sqrt(un2[s % L]));
}

// per point: 1 while some column is above its target
__global__ void k_active_kernel(int np, int L, const double* __restrict__ res, const double* __restrict__ target,
                                int32_t* __restrict__ active, int32_t* __restrict__ count) {
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= np) return;
    int a = 0;
    for (int l = 0; l < L; ++l) a |= !(res[(int64_t)pt * L + l] <= target[(int64_t)pt * L + l]);
    active[pt] = a;
    if (a) atomicAdd(count, 1);
}

unsigned blocks(int64_t total, int t = KT) { return (unsigned)((total + t - 1) / t); }

}  // namespace

int krylov_restart(int64_t n, int64_t systems, size_t free_bytes) {
    // V: m + 1 vectors, Z: m vectors, one system block each; at most 40 % of free memory
    const double per = (double)systems * (double)n * sizeof(c128);
    int m = (int)std::min<double>(30.0, (0.4 * (double)free_bytes / per - 1.0) / 2.0);
    return m;
}

template <typename R>
int krylov_solve(const KrylovArgs<R>& a, int* iters_out) {
    cudaStream_t st = a.st;
    const int64_t n = a.n, S = (int64_t)a.np * a.L, total = S * n;
    const int m = a.m, np = a.np, L = a.L;
    *iters_out = 0;
    if (m < 2) return set_error(RSRR_ENOMEM, "iterative sampler: too little device memory for a Krylov space");
    const int64_t vstride = total;
    c128 *V = nullptr, *Z = nullptr, *W = nullptr, *H = nullptr, *sn = nullptr, *g = nullptr, *h1 = nullptr,
         *h2 = nullptr, *y = nullptr;
    double *nrm = nullptr, *res = nullptr, *cs = nullptr, *xn = nullptr, *target = nullptr;
    int32_t *active = nullptr, *count = nullptr;
    int rc = RSRR_OK;
    auto cleanup = [&]() {
        for (void* p : {(void*)V, (void*)Z, (void*)W, (void*)H, (void*)sn, (void*)g, (void*)h1, (void*)h2, (void*)y,
                        (void*)nrm, (void*)res, (void*)cs, (void*)xn, (void*)target, (void*)active, (void*)count})
            dfree(p, st);
    };
#define KTRY(expr) do { rc = (expr); if (rc != RSRR_OK) { cleanup(); return rc; } } while (0)
#define KCUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return set_error(RSRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)
    KTRY(dalloc_n(&V, (size_t)(m + 1) * total, st));
    KTRY(dalloc_n(&Z, (size_t)m * total, st));
    KTRY(dalloc_n(&W, (size_t)total, st));
    KTRY(dalloc_n(&H, (size_t)S * (m + 1) * m, st));
    KTRY(dalloc_n(&cs, (size_t)S * m, st));
    KTRY(dalloc_n(&sn, (size_t)S * m, st));
    KTRY(dalloc_n(&g, (size_t)S * (m + 1), st));
    KTRY(dalloc_n(&h1, (size_t)S * (m + 1), st));
    KTRY(dalloc_n(&h2, (size_t)S * (m + 1), st));
    KTRY(dalloc_n(&y, (size_t)S * m, st));
    KTRY(dalloc_n(&nrm, (size_t)S, st));
    KTRY(dalloc_n(&res, (size_t)S, st));
    KTRY(dalloc_n(&xn, (size_t)S, st));
    KTRY(dalloc_n(&target, (size_t)S, st));
    KTRY(dalloc_n(&active, (size_t)np, st));
    KTRY(dalloc_n(&count, 1, st));
    const dim3 gc((unsigned)blocks(n, 128), np);
    int iters = 0;
    bool done = false;
    std::vector<int32_t> hcount(1);
    while (!done) {
        // ---- cycle start: r = u - T x, beta, v_0, g = beta e_1, targets --------------------------
        { k_csr_kernel<<<gc, 128, 0, st>>>(a.rowptr, a.colind, a.tvals, a.nnz, n, L, a.U, a.X, W); note_launch(); }
        { k_norm_kernel<<<(unsigned)S, KT, 0, st>>>(W, n, nrm); note_launch(); }
        { k_norm_kernel<<<(unsigned)S, KT, 0, st>>>(a.X, n, xn); note_launch(); }
        { k_scale_kernel<<<blocks(total), KT, 0, st>>>(W, nrm, V, n, total); note_launch(); }
        { k_start_kernel<<<blocks(S), KT, 0, st>>>((int)S, m, L, nrm, res, g); note_launch(); }
        { k_target_kernel<<<blocks(S), KT, 0, st>>>((int)S, L, a.tau, xn, a.un2, a.normT, target); note_launch(); }
        KCUDA(cudaMemsetAsync(count, 0, 4, st));
        { k_active_kernel<<<blocks(np), KT, 0, st>>>(np, L, res, target, active, count); note_launch(); }
        KCUDA(cudaMemcpyAsync(hcount.data(), count, 4, cudaMemcpyDeviceToHost, st));
        KCUDA(cudaStreamSynchronize(st));
        if (hcount[0] == 0 || iters >= a.max_iter) break;
        int kk = 0;
        for (int k = 0; k < m && iters < a.max_iter; ++k) {
            // z_k = M^{-1} v_k (the solves skip points whose columns all meet their targets)
            { k_down_kernel<R><<<blocks(total), KT, 0, st>>>(V + (int64_t)k * vstride, a.B, total); note_launch(); }
            KTRY(a.precond(active));
            { k_up_kernel<R><<<blocks(total), KT, 0, st>>>(a.B, Z + (int64_t)k * vstride, total); note_launch(); }
            // w = T z_k, orthogonalised against v_0..v_k twice
            { k_csr_kernel<<<gc, 128, 0, st>>>(a.rowptr, a.colind, a.tvals, a.nnz, n, L, nullptr,
                                               Z + (int64_t)k * vstride, W); note_launch(); }
            { k_dot_kernel<<<dim3((unsigned)S, k + 1), KT, 0, st>>>(V, vstride, W, n, h1, m + 1); note_launch(); }
            { k_axpy_kernel<<<blocks(total), KT, 0, st>>>(V, vstride, k + 1, h1, m + 1, W, n, total); note_launch(); }
            { k_dot_kernel<<<dim3((unsigned)S, k + 1), KT, 0, st>>>(V, vstride, W, n, h2, m + 1); note_launch(); }
            { k_axpy_kernel<<<blocks(total), KT, 0, st>>>(V, vstride, k + 1, h2, m + 1, W, n, total); note_launch(); }
            { k_norm_kernel<<<(unsigned)S, KT, 0, st>>>(W, n, nrm); note_launch(); }
            { k_scale_kernel<<<blocks(total), KT, 0, st>>>(W, nrm, V + (int64_t)(k + 1) * vstride, n, total); note_launch(); }
            { k_givens_kernel<<<blocks(S), KT, 0, st>>>(k, m, (int)S, h1, h2, m + 1, nrm, H, cs, sn, g, res); note_launch(); }
            ++iters;
            kk = k + 1;
            KCUDA(cudaMemsetAsync(count, 0, 4, st));
            { k_active_kernel<<<blocks(np), KT, 0, st>>>(np, L, res, target, active, count); note_launch(); }
            KCUDA(cudaMemcpyAsync(hcount.data(), count, 4, cudaMemcpyDeviceToHost, st));
            KCUDA(cudaStreamSynchronize(st));
            if (hcount[0] == 0) break;
        }
        // ---- x += Z y ------------------------------------------------------------------------
        { k_backsolve_kernel<<<blocks(S), KT, 0, st>>>(kk, m, (int)S, H, g, y); note_launch(); }
        { k_xupdate_kernel<<<blocks(total), KT, 0, st>>>(Z, vstride, kk, y, m, a.X, n, total); note_launch(); }
        if (iters >= a.max_iter) done = true;
    }
    KCUDA(cudaStreamSynchronize(st));
    cleanup();
#undef KTRY
#undef KCUDA
    *iters_out = iters;
    return RSRR_OK;
}

template int krylov_solve<float>(const KrylovArgs<float>&, int*);
template int krylov_solve<double>(const KrylovArgs<double>&, int*);

}  // namespace rsrr
