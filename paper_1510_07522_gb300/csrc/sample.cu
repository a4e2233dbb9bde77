// rsrr_sample: Algorithm 2 Steps 1-2 (Eq. eq-hatS) on the device.
//
// For every sampling point z_j of the contour:
//   assemble T(z_j) = sum_i f_i(z_j) A_i into band storage        (Eq. eq-Z-expr)
//   factor T(z_j) = P L U (band LU, partial pivoting)           (band.cu)
//   X_j = U^{-1} L^{-1} P U_probe                                (band.cu)
//   FP64 residual R = U_probe - T(z_j) X_j from the CSR values, normwise backward error
//   eta = ||r|| / (||T||_1 ||x|| + ||u||) per column; in complex64 mode, refinement sweeps
//   X_j += (LU)^{-1} R until eta <= tol.
// All points of a chunk run concurrently (one CTA per point); chunks are sized so the
// factors fit in free device memory.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "band.cuh"
#include "band_tc.cuh"
#include "dense_lu.cuh"
#include "internal.h"
#include "krylov.cuh"

namespace rsrr {

namespace {

// T values of each point on the CSR pattern (FP64) and the band image (precision R).
template <typename R>
__global__ void assemble_kernel(const c128* __restrict__ vals, int J, int64_t nnz,
                                const int32_t* __restrict__ rowidx, const int32_t* __restrict__ colind,
                                const c128* __restrict__ F, int j0, int kl, int ku, int ldab,
                                c128* __restrict__ tvals, cplx<R>* __restrict__ ab, int64_t ab_stride) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    if (k >= nnz) return;
    const c128* f = F + (int64_t)(j0 + pt) * J;
    c128 v = czero<double>();
    for (int i = 0; i < J; ++i) cfma(v, f[i], vals[(int64_t)i * nnz + k]);
    tvals[(int64_t)pt * nnz + k] = v;
    if (ab) {  // entries outside the factored band (an incomplete factorisation) are left out
        const int r = rowidx[k], c = colind[k];
        if (r - c <= kl && c - r <= ku)
            ab[pt * ab_stride + (int64_t)(kl + ku + r - c) + (int64_t)c * ldab] = ccast<R>(v);
    }
}

// ||T(z_j)||_1: column sums of |T_rc| (atomics), then the maximum.
__global__ void colsum_kernel(const c128* __restrict__ tvals, int64_t nnz, const int32_t* __restrict__ colind,
                              int64_t n, double* __restrict__ colsum) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    if (k >= nnz) return;
    const c128 v = tvals[(int64_t)pt * nnz + k];
    atomicAdd(&colsum[(int64_t)pt * n + colind[k]], sqrt(cnorm2(v)));
}

__global__ void max_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    const int pt = blockIdx.x;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[(int64_t)pt * n + i]);
    __shared__ double red[32];
    for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) out[pt] = m;
    }
}

// B_j = U (converted to precision R) for every point of the chunk.
template <typename R>
__global__ void broadcast_rhs_kernel(const c128* __restrict__ U, int64_t nl, cplx<R>* __restrict__ B) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nl) return;
    B[(int64_t)blockIdx.y * nl + k] = ccast<R>(U[k]);
}

// X = B (first solve) or X += B (refinement), X in FP64.
template <typename R>
__global__ void accumulate_kernel(c128* __restrict__ X, const cplx<R>* __restrict__ B, int64_t nl,
                                  int add, const int32_t* __restrict__ active) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = blockIdx.y;
    if (k >= nl || (active && !active[pt])) return;
    const c128 b = ccast<double>(B[(int64_t)pt * nl + k]);
    c128& x = X[(int64_t)pt * nl + k];
    x = add ? x + b : b;
}

// R = U - T X in FP64 (CSR rows, one thread per row, all L columns); R goes to B in
// precision R; per-column ||r||^2 and ||x||^2 accumulate in rn2 / xn2.
template <typename R>
__global__ void residual_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                const c128* __restrict__ tvals, int64_t nnz, int64_t n, int L,
                                const c128* __restrict__ U, const c128* __restrict__ X,
                                cplx<R>* __restrict__ B, double* __restrict__ rn2, double* __restrict__ xn2,
                                const int32_t* __restrict__ active) {
    const int pt = blockIdx.y;
    if (active && !active[pt]) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = r < n;
    const c128* tv = tvals + (int64_t)pt * nnz;
    const c128* Xp = X + (int64_t)pt * n * L;
    cplx<R>* Bp = B + (int64_t)pt * n * L;
    const int64_t k0 = valid ? rowptr[r] : 0, k1 = valid ? rowptr[r + 1] : 0;
    for (int l = 0; l < L; ++l) {
        double sr = 0.0, sx = 0.0;
        if (valid) {
            c128 acc = U[r + (int64_t)l * n];
            for (int64_t k = k0; k < k1; ++k) cfms(acc, tv[k], Xp[colind[k] + (int64_t)l * n]);
            if (B) Bp[r + (int64_t)l * n] = ccast<R>(acc);
            sr = cnorm2(acc);
            sx = cnorm2(Xp[r + (int64_t)l * n]);
        }
        for (int off = 16; off; off >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, off);
            sx += __shfl_down_sync(0xffffffffu, sx, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&rn2[(int64_t)pt * L + l], sr);
            atomicAdd(&xn2[(int64_t)pt * L + l], sx);
        }
    }
}

// eta per column.  A point stays active (gets another refinement sweep) while its worst eta is
// above the target (tol, or 0 when refining to working accuracy) and fell at least twofold in
// the last sweep; a point still above tol that stopped improving is counted as stagnated.
// counters: [0] active, [1] non-finite, [2] stagnated.
__global__ void eta_kernel(const double* __restrict__ rn2, const double* __restrict__ xn2,
                           const double* __restrict__ un2, const double* __restrict__ normT, int npts, int L,
                           double tol, double target, double* __restrict__ eta, int32_t* __restrict__ active,
                           double* __restrict__ prev_max, int32_t* __restrict__ counters, int first) {
    const int pt = blockIdx.x;
    if (!first && !active[pt]) return;  // residual not recomputed for this point
    double mx = 0.0;
    int nonfinite = 0;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const double e = sqrt(rn2[pt * L + l]) / (normT[pt] * sqrt(xn2[pt * L + l]) + sqrt(un2[l]));
        eta[(int64_t)pt * L + l] = e;
        if (!isfinite(e)) nonfinite = 1;
        mx = fmax(mx, e);
    }
    for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if (threadIdx.x == 0) {
        if (nonfinite) atomicOr(&counters[1], 1);
        int act = 0;
        const bool improving = first || mx < 0.5 * prev_max[pt];
        if (!(mx <= target) && improving) act = 1;
        else if (!(mx <= tol)) atomicAdd(&counters[2], 1);
        prev_max[pt] = mx;
        active[pt] = act;
        if (act) atomicAdd(&counters[0], 1);
    }
}

__global__ void column_norm2_kernel(const c128* __restrict__ U, int64_t n, double* __restrict__ out) {
    const int l = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += cnorm2(U[i + (int64_t)l * n]);
    __shared__ double red[32];
    for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) out[l] = s;
    }
}

__global__ void gather_rows_kernel(const c128* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                                   int cols, c128* __restrict__ dst) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * cols) return;
    const int64_t r = k % n, c = k / n;
    dst[k] = src[perm[r] + c * n];
}

}  // namespace

int pick_dims(int64_t n, int64_t kl, int64_t ku, bool is_c64, BandDims* d) {
    if (kl > 2048 || ku > 2048) return set_error(RSRR_EUNSUPPORTED, "band too wide for the band kernels");
    d->n = (int)n;
    d->kl = (int)kl;
    d->ku = (int)ku;
    d->kv = d->kl + d->ku;
    d->ldab = 2 * d->kl + d->ku + 1;
    const size_t es = is_c64 ? sizeof(cplx<float>) : sizeof(cplx<double>);
    const size_t limit = 220 * 1024;
    const int64_t ubw = std::min<int64_t>(d->kv, n - 1);  // U's bandwidth cannot exceed n - 1
    for (int nb : {32, 16, 8, 4}) {
        d->nb = nb;
        d->ldp = (int)ceil_div(nb + d->kl, 32) * 32;
        size_t s = 2 * ((size_t)d->ldp * nb * es + (size_t)d->ldp * 4) + 16 * 32 * 4 * es;
        if (s <= limit) break;
        if (nb == 4) return set_error(RSRR_EUNSUPPORTED, "band too wide for shared-memory panels");
    }
    // backward blocks: prefer two staging buffers (copy-ahead), else one
    d->bwd_nbuf = 0;
    for (int nbuf : {2, 1}) {
        for (int nbb : {32, 16, 8, 4}) {
            d->nbb = nbb;
            d->ldb = (int)ceil_div(nbb + ubw, 32) * 32;
            size_t s = (size_t)nbuf * d->ldb * nbb * es + 16 * 32 * 2 * es + 32 * es;
            if (s <= limit && (nbuf == 1 || nbb >= 8)) { d->bwd_nbuf = nbuf; break; }
        }
        if (d->bwd_nbuf) break;
    }
    if (!d->bwd_nbuf) return set_error(RSRR_EUNSUPPORTED, "band too wide for shared-memory blocks");
    {
        const size_t one = (size_t)d->ldp * d->nb * es + (size_t)d->ldp * 4;
        d->fwd_nbuf = (2 * one + 16 * 32 * 2 * es <= limit) ? 2 : 1;
    }
    d->npanels = (int)ceil_div(n, d->nb);
    return RSRR_OK;
}

namespace {

// Event pair around a group of launches on the stream; elapsed time is read after the next
// stream synchronisation.
struct EvPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EvPair() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~EvPair() { cudaEventDestroy(a); cudaEventDestroy(b); }
    void start(cudaStream_t s) { cudaEventRecord(a, s); }
    void stop(cudaStream_t s) { cudaEventRecord(b, s); }
    double ms() { float t = 0.f; cudaEventElapsedTime(&t, a, b); return t; }
};

// The complex64 band LU runs on the tensor cores (band_tc.cu) when its band suits them
// (kl in [32, 224]), unless the handle was created with RSRR_BAND_CUDA_CORES.
template <typename R>
bool use_band_tc(rsrr_nep h, int64_t n, int64_t kl, int64_t ku) {
    return sizeof(R) == 4 && !h->band_cuda_cores && band_tc_eligible(n, kl, ku);
}
template <typename R>
int factor_any(bool tc, const FactorArgs<R>& a, int np, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (tc) return launch_factor_tc(a, np, st);
    }
    return launch_factor<R>(a, np, st);
}
// The tensor-core factor's solves take at most 64 right-hand sides per launch: more run as
// column blocks (each a separate set of systems with the same factors).
template <typename R, typename F>
int by_column_blocks(const SolveArgs<R>& a, F&& launch) {
    for (int c0 = 0; c0 < a.L; c0 += 64) {
        SolveArgs<R> b = a;
        b.x = a.x + (int64_t)c0 * a.d.n;
        b.L = std::min(64, a.L - c0);
        RSRR_TRY(launch(b));
    }
    return RSRR_OK;
}
template <typename R>
int fwd_any(bool tc, const SolveArgs<R>& a, int np, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (tc) return by_column_blocks(a, [&](const SolveArgs<R>& b) { return launch_fwd_tc(b, np, st); });
    }
    return launch_fwd<R>(a, np, st);
}
template <typename R>
int bwd_any(bool tc, const SolveArgs<R>& a, int np, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (tc && band_bwd_tc_fits(a.d))
            return by_column_blocks(a, [&](const SolveArgs<R>& b) { return launch_bwd_tc(b, np, st); });
    }
    return launch_bwd<R>(a, np, st);
}

template <typename R>
int sample_impl(rsrr_nep h, const std::vector<c128>& F, int max_refine) {
    cudaStream_t st = h->stream;
    const int64_t n = h->n, nnz = h->nnz;
    const int N = h->N, L = h->L, J = h->J;
    BandDims d;
    int64_t kl = h->ord.kl, ku = h->ord.ku;
    if (h->precond_band >= 0) {  // factor the band part only; the refinement iterates with the full T
        kl = std::min<int64_t>(kl, h->precond_band);
        ku = std::min<int64_t>(ku, h->precond_band);
    }
    const bool tc = use_band_tc<R>(h, n, kl, ku);
    if (tc) RSRR_TRY(pick_dims_tc(n, kl, ku, &d));
    else RSRR_TRY(pick_dims(n, kl, ku, sizeof(R) == 4, &d));
    const int64_t nl = n * L;
    // per-point footprint
    const size_t es = sizeof(cplx<R>);
    const size_t ab_b = (size_t)(tc ? tc_ab_stride(d) : (int64_t)d.ldab * n) * es;
    const size_t lp_b = (size_t)d.npanels * d.ldp * d.nb * es;
    const size_t perm_b = (size_t)d.npanels * d.ldp * 4;
    const size_t per_pt = ab_b + lp_b + perm_b + (size_t)n * 4 + (size_t)nl * es + (size_t)nnz * 16 +
                          (size_t)n * 8 + 256;
    size_t free_b = 0, total_b = 0;
    RSRR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = (size_t)(0.8 * (double)free_b);
    int chunk = (int)std::min<int64_t>(N, std::max<int64_t>(1, budget / per_pt));
    if ((size_t)chunk * per_pt > budget) return set_error(RSRR_ENOMEM, "one sampling point does not fit in device memory");

    c128* dF = nullptr;
    RSRR_TRY(dalloc_n(&dF, F.size(), st));
    RSRR_CUDA(cudaMemcpyAsync(dF, F.data(), F.size() * sizeof(c128), cudaMemcpyHostToDevice, st));
    cplx<R>*ab = nullptr, *lp = nullptr, *B = nullptr;
    int32_t *perm = nullptr, *ipiv = nullptr, *info = nullptr, *active = nullptr, *counters = nullptr;
    c128* tvals = nullptr;
    double *colsum = nullptr, *normT = nullptr, *rn2 = nullptr, *xn2 = nullptr, *un2 = nullptr,
           *prev_max = nullptr;
    int rc = RSRR_OK;
    auto cleanup = [&]() {
        dfree(dF, st); dfree(ab, st); dfree(lp, st); dfree(B, st); dfree(perm, st); dfree(ipiv, st);
        dfree(info, st); dfree(active, st); dfree(counters, st); dfree(tvals, st); dfree(colsum, st);
        dfree(normT, st); dfree(rn2, st); dfree(xn2, st); dfree(un2, st); dfree(prev_max, st);
    };
#define TRYC(expr) do { rc = (expr); if (rc != RSRR_OK) { cleanup(); return rc; } } while (0)
#define CUDAC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return set_error(RSRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)
    TRYC(dalloc(reinterpret_cast<void**>(&ab), ab_b * chunk, st));
    TRYC(dalloc(reinterpret_cast<void**>(&lp), lp_b * chunk, st));
    TRYC(dalloc_n(&B, (size_t)nl * chunk, st));
    TRYC(dalloc_n(&perm, (size_t)d.npanels * d.ldp * chunk, st));
    TRYC(dalloc_n(&ipiv, (size_t)n * chunk, st));
    TRYC(dalloc_n(&info, (size_t)chunk, st));
    TRYC(dalloc_n(&active, (size_t)chunk, st));
    TRYC(dalloc_n(&counters, 4, st));
    TRYC(dalloc_n(&prev_max, (size_t)chunk, st));
    TRYC(dalloc_n(&tvals, (size_t)nnz * chunk, st));
    TRYC(dalloc_n(&colsum, (size_t)n * chunk, st));
    TRYC(dalloc_n(&normT, (size_t)chunk, st));
    TRYC(dalloc_n(&rn2, (size_t)L * chunk, st));
    TRYC(dalloc_n(&xn2, (size_t)L * chunk, st));
    TRYC(dalloc_n(&un2, (size_t)L, st));
    h->ms_factor = h->ms_trsv = 0;
    h->factor_launches = h->trsv_launches = 0;
    h->band_tc_used = tc;
    EvPair evf, evs;
    { column_norm2_kernel<<<L, 256, 0, st>>>(h->d_U, n, un2); note_launch(); }

    int max_sweeps = 0;
    bool singular = false, nonfinite = false, notconv = false;
    for (int j0 = 0; j0 < N; j0 += chunk) {
        const int np = std::min(chunk, N - j0);
        c128* X = h->d_S + (int64_t)j0 * nl;
        double* eta = h->d_eta + (int64_t)j0 * L;
        CUDAC(cudaMemsetAsync(ab, 0, ab_b * np, st));
        {
            dim3 g((unsigned)ceil_div(nnz, 256), np);
            { assemble_kernel<R><<<g, 256, 0, st>>>(h->d_vals, J, nnz, h->d_rowidx, h->d_colind, dF, j0, d.kl, d.ku,
                                                  d.ldab, tvals, ab, (int64_t)(ab_b / es)); note_launch(); }
            CUDAC(cudaGetLastError());
            CUDAC(cudaMemsetAsync(colsum, 0, (size_t)n * np * 8, st));
            { colsum_kernel<<<g, 256, 0, st>>>(tvals, nnz, h->d_colind, n, colsum); note_launch(); }
            { max_kernel<<<np, 256, 0, st>>>(colsum, n, normT); note_launch(); }
        }
        FactorArgs<R> fa{d, ab, (int64_t)(ab_b / es), lp, (int64_t)(lp_b / es), perm,
                         (int64_t)d.npanels * d.ldp, ipiv, info};
        evf.start(st);
        TRYC(factor_any<R>(tc, fa, np, st));
        evf.stop(st);
        std::vector<int32_t> hinfo(np);
        CUDAC(cudaMemcpyAsync(hinfo.data(), info, np * 4, cudaMemcpyDeviceToHost, st));
        CUDAC(cudaStreamSynchronize(st));
        h->ms_factor += evf.ms();
        h->factor_launches += 1;
        bool timeout = false;
        for (int k = 0; k < np; ++k) {
            if (hinfo[k] > 0) singular = true;
            if (hinfo[k] < 0) timeout = true;
        }
        if (timeout) {
            cleanup();
            return set_error(RSRR_ETIMEOUT, "band LU: a tensor-core wait gave up");
        }
        if (singular) break;
        SolveArgs<R> sa{d, ab, (int64_t)(ab_b / es), lp, (int64_t)(lp_b / es), perm,
                        (int64_t)d.npanels * d.ldp, B, nl, L, nullptr};
        {
            dim3 g((unsigned)ceil_div(nl, 256), np);
            { broadcast_rhs_kernel<R><<<g, 256, 0, st>>>(h->d_U, nl, B); note_launch(); }
        }
        evs.start(st);
        TRYC(fwd_any<R>(tc, sa, np, st));
        TRYC(bwd_any<R>(tc, sa, np, st));
        evs.stop(st);
        bool trsv_pending = true;
        h->trsv_launches += 2;
        {
            dim3 g((unsigned)ceil_div(nl, 256), np);
            { accumulate_kernel<R><<<g, 256, 0, st>>>(X, B, nl, 0, nullptr); note_launch(); }
        }
        if (h->precond_band >= 0) {
            // Iterative sampler: flexible GMRES from X = M^{-1} U, preconditioned by the factor of
            // the band part of T(z_j) (krylov.cu); max_refine counts preconditioned products.
            size_t fb = 0, tbytes = 0;
            CUDAC(cudaMemGetInfo(&fb, &tbytes));
            KrylovArgs<R> ka;
            ka.st = st;
            ka.n = n;
            ka.nnz = nnz;
            ka.np = np;
            ka.L = L;
            ka.rowptr = h->d_rowptr;
            ka.colind = h->d_colind;
            ka.tvals = tvals;
            ka.U = h->d_U;
            ka.X = X;
            ka.normT = normT;
            ka.un2 = un2;
            ka.tau = h->refine_full ? 2e-16 : 0.5 * h->tol;
            ka.m = krylov_restart(n, (int64_t)np * L, fb);
            ka.max_iter = max_refine;
            ka.B = B;
            ka.precond = [&](const int32_t* act) {
                SolveArgs<R> s2 = sa;
                s2.active = act;
                int r = fwd_any<R>(tc, s2, np, st);
                if (r == RSRR_OK) r = bwd_any<R>(tc, s2, np, st);
                h->trsv_launches += 2;
                return r;
            };
            int kit = 0;
            TRYC(krylov_solve<R>(ka, &kit));
            max_sweeps = std::max(max_sweeps, kit);
            // backward errors of the result; every column must meet tol
            CUDAC(cudaMemsetAsync(rn2, 0, (size_t)L * np * 8, st));
            CUDAC(cudaMemsetAsync(xn2, 0, (size_t)L * np * 8, st));
            CUDAC(cudaMemsetAsync(counters, 0, 16, st));
            dim3 g((unsigned)ceil_div(n, 128), np);
            { residual_kernel<R><<<g, 128, 0, st>>>(h->d_rowptr, h->d_colind, tvals, nnz, n, L, h->d_U, X, B, rn2, xn2,
                                                  nullptr); note_launch(); }
            { eta_kernel<<<np, 32, 0, st>>>(rn2, xn2, un2, normT, np, L, h->tol, h->tol, eta, active, prev_max,
                                          counters, 1); note_launch(); }
            int32_t hc[4];
            std::vector<double> he((size_t)np * L);
            CUDAC(cudaMemcpyAsync(hc, counters, 16, cudaMemcpyDeviceToHost, st));
            CUDAC(cudaMemcpyAsync(he.data(), eta, he.size() * 8, cudaMemcpyDeviceToHost, st));
            CUDAC(cudaStreamSynchronize(st));
            if (trsv_pending) { h->ms_trsv += evs.ms(); trsv_pending = false; }
            if (hc[1]) { nonfinite = true; break; }
            for (double e : he) if (!(e <= h->tol)) notconv = true;
            if (notconv) break;
            continue;
        }
        int sweeps = 0;
        for (;;) {
            CUDAC(cudaMemsetAsync(rn2, 0, (size_t)L * np * 8, st));
            CUDAC(cudaMemsetAsync(xn2, 0, (size_t)L * np * 8, st));
            CUDAC(cudaMemsetAsync(counters, 0, 16, st));
            dim3 g((unsigned)ceil_div(n, 128), np);
            { residual_kernel<R><<<g, 128, 0, st>>>(h->d_rowptr, h->d_colind, tvals, nnz, n, L, h->d_U, X, B, rn2, xn2,
                                                  sweeps == 0 ? nullptr : active); note_launch(); }
            { eta_kernel<<<np, 32, 0, st>>>(rn2, xn2, un2, normT, np, L, h->tol, h->refine_full ? 0.0 : h->tol,
                                          eta, active, prev_max, counters, sweeps == 0 ? 1 : 0); note_launch(); }
            int32_t hc[4];
            CUDAC(cudaMemcpyAsync(hc, counters, 16, cudaMemcpyDeviceToHost, st));
            CUDAC(cudaStreamSynchronize(st));
            if (trsv_pending) { h->ms_trsv += evs.ms(); trsv_pending = false; }
            if (hc[1]) { nonfinite = true; break; }
            if (hc[2]) { notconv = true; break; }
            if (hc[0] == 0) break;
            if (sweeps >= max_refine) {
                // out of sweeps: fine if every column already meets tol (possible in full mode)
                std::vector<double> he((size_t)np * L);
                CUDAC(cudaMemcpyAsync(he.data(), eta, he.size() * 8, cudaMemcpyDeviceToHost, st));
                CUDAC(cudaStreamSynchronize(st));
                for (double e : he) if (!(e <= h->tol)) notconv = true;
                break;
            }
            sa.active = active;
            evs.start(st);
            TRYC(fwd_any<R>(tc, sa, np, st));
            TRYC(bwd_any<R>(tc, sa, np, st));
            evs.stop(st);
            trsv_pending = true;
            h->trsv_launches += 2;
            dim3 ga((unsigned)ceil_div(nl, 256), np);
            { accumulate_kernel<R><<<ga, 256, 0, st>>>(X, B, nl, 1, active); note_launch(); }
            sa.active = nullptr;
            ++sweeps;
        }
        max_sweeps = std::max(max_sweeps, sweeps);
        if (nonfinite || notconv) break;
    }
    CUDAC(cudaStreamSynchronize(st));
    cleanup();
#undef TRYC
#undef CUDAC
    h->refine_sweeps = max_sweeps;
    if (singular) return set_error(RSRR_ESINGULAR, "zero pivot: a sampling point is an eigenvalue of T");
    if (nonfinite) return set_error(RSRR_ENONFINITE, "non-finite backward error in a sample solve");
    if (notconv) return set_error(RSRR_ENOTCONVERGED, "sample solves did not reach the backward-error tolerance");
    return RSRR_OK;
}

// ---------------------------------------------------------------------------------------------
// Dense sampling of a set of NEPs (dense_lu.cu): every point of every NEP is one job of a single
// persistent launch that assembles, factors, solves and refines the point in a per-CTA memory
// slot (largest n first), so uneven NEPs share the GPU with no host round trip between stages.
// ---------------------------------------------------------------------------------------------
template <typename R>
int sample_dense_set(const std::vector<rsrr_nep>& hs, const std::vector<c128*>& dF, int max_refine) {
    if (hs.empty()) return RSRR_OK;
    cudaStream_t st = hs[0]->stream;
    const int nh = (int)hs.size();
    int n_max = 0, L_max = 0;
    int64_t total_points = 0;
    for (rsrr_nep h : hs) {
        n_max = std::max<int>(n_max, (int)h->n);
        L_max = std::max<int>(L_max, h->L);
        total_points += h->N;
        h->refine_sweeps = 0;
    }
    // jobs, largest n first
    std::vector<DenseSampleJob> jobs;
    jobs.reserve((size_t)total_points);
    std::vector<int> order(nh);
    for (int i = 0; i < nh; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->n > hs[b]->n; });
    for (int i : order)
        for (int j = 0; j < hs[i]->N; ++j) jobs.push_back(DenseSampleJob{i, j});
    const int njobs = (int)jobs.size();
    // CTAs: one per SM at most, and no more slots than the free memory holds
    size_t free_b = 0, total_b = 0;
    RSRR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t per_cta = dense_slot_bytes<R>(n_max, L_max) + dense_image_bytes<R>(n_max);
    const size_t budget = (size_t)(0.8 * (double)free_b);
    const int grid = (int)std::min<size_t>((size_t)dense_sample_grid(njobs), budget / per_cta);
    if (grid < 1) return set_error(RSRR_ENOMEM, "one dense sampling slot does not fit in device memory");

    std::vector<DenseNep> neps(nh);
    std::vector<double*> un2(nh, nullptr);
    std::vector<int32_t*> status(nh, nullptr), sweeps(nh, nullptr);
    DenseNep* d_neps = nullptr;
    DenseSampleJob* d_jobs = nullptr;
    int32_t* d_next = nullptr;
    void* d_slots = nullptr;
    void* d_img = nullptr;
    auto cleanup = [&]() {
        for (int i = 0; i < nh; ++i) { dfree(un2[i], st); dfree(status[i], st); dfree(sweeps[i], st); }
        dfree(d_neps, st); dfree(d_jobs, st); dfree(d_next, st); dfree(d_slots, st); dfree(d_img, st);
    };
#define TRYD(expr) do { int rc_ = (expr); if (rc_ != RSRR_OK) { cleanup(); return rc_; } } while (0)
#define CUDAD(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cleanup(); return set_error(RSRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); } } while (0)
    for (int i = 0; i < nh; ++i) {
        rsrr_nep h = hs[i];
        TRYD(dalloc_n(&un2[i], (size_t)h->L, st));
        TRYD(dalloc_n(&status[i], (size_t)h->N, st));
        TRYD(dalloc_n(&sweeps[i], (size_t)h->N, st));
        { column_norm2_kernel<<<(unsigned)h->L, 256, 0, st>>>(h->d_U, h->n, un2[i]); note_launch(); }
        CUDAD(cudaGetLastError());
        DenseNep& E = neps[i];
        E.n = (int32_t)h->n;
        E.J = h->J;
        E.L = h->L;
        E.N = h->N;
        E.nnz = h->nnz;
        E.rowptr = h->d_rowptr;
        E.colind = h->d_colind;
        E.rowidx = h->d_rowidx;
        E.vals = h->d_vals;
        E.F = dF[i];
        E.U = h->d_U;
        E.un2 = un2[i];
        E.S = h->d_S;
        E.eta = h->d_eta;
        E.status = status[i];
        E.sweeps = sweeps[i];
    }
    TRYD(dalloc_n(&d_neps, (size_t)nh, st));
    TRYD(dalloc_n(&d_jobs, (size_t)njobs, st));
    TRYD(dalloc_n(&d_next, 1, st));
    TRYD(dalloc(&d_slots, (size_t)grid * dense_slot_bytes<R>(n_max, L_max), st));
    if (dense_image_bytes<R>(n_max)) TRYD(dalloc(&d_img, (size_t)grid * dense_image_bytes<R>(n_max), st));
    CUDAD(cudaMemcpyAsync(d_neps, neps.data(), neps.size() * sizeof(DenseNep), cudaMemcpyHostToDevice, st));
    CUDAD(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(DenseSampleJob), cudaMemcpyHostToDevice, st));
    DenseSampleCfg cfg;
    cfg.tol = hs[0]->tol;
    cfg.target = hs[0]->refine_full ? 0.0 : hs[0]->tol;
    cfg.max_refine = max_refine;
    EvPair ev;
    ev.start(st);
    TRYD(launch_dense_sample<R>(d_neps, d_jobs, njobs, n_max, L_max, grid, d_slots, d_img, d_next, cfg, st));
    ev.stop(st);
    bool singular = false, timeout = false, nonfinite = false, notconv = false;
    for (int i = 0; i < nh; ++i) {
        std::vector<int32_t> hst(hs[i]->N), hsw(hs[i]->N);
        CUDAD(cudaMemcpyAsync(hst.data(), status[i], hst.size() * 4, cudaMemcpyDeviceToHost, st));
        CUDAD(cudaMemcpyAsync(hsw.data(), sweeps[i], hsw.size() * 4, cudaMemcpyDeviceToHost, st));
        CUDAD(cudaStreamSynchronize(st));
        for (int j = 0; j < hs[i]->N; ++j) {
            if (hst[j] > 0) singular = true;
            if (hst[j] == -1) timeout = true;
            if (hst[j] == -2) nonfinite = true;
            if (hst[j] == -3) notconv = true;
            hs[i]->refine_sweeps = std::max(hs[i]->refine_sweeps, hsw[j]);
        }
    }
    const double ms = ev.ms();
    for (rsrr_nep h : hs) {  // one launch serves the whole set: each handle reports it
        h->ms_factor = ms;
        h->ms_trsv = 0;
        h->factor_launches = 1;
        h->trsv_launches = 0;
    }
    cleanup();
#undef TRYD
#undef CUDAD
    if (timeout) return set_error(RSRR_ETIMEOUT, "dense LU: a tensor-core wait timed out");
    if (singular) return set_error(RSRR_ESINGULAR, "zero pivot: a sampling point is an eigenvalue of T");
    if (nonfinite) return set_error(RSRR_ENONFINITE, "non-finite backward error in a sample solve");
    if (notconv) return set_error(RSRR_ENOTCONVERGED, "sample solves did not reach the backward-error tolerance");
    return RSRR_OK;
}

}  // namespace

// Coefficient table F (host FP64), the probing matrix on the device (permuted to the band
// ordering) and S_hat storage for the sampling set up on h.
int sample_prepare(rsrr_nep h, const double* U_reim, std::vector<c128>* Fout) {
    cudaStream_t st = h->stream;
    const int64_t n = h->n;
    const int N = h->N, L = h->L;
    std::vector<zd> z;
    if (h->points.empty()) contour_rule(h->C, N, &z, nullptr, h->C.side_nodes);
    else z = h->points;
    std::vector<c128>& F = *Fout;
    if (h->tz) {
        // T known by its values: T(z_j) for every sampling point become the J = N terms, F = I
        c128* v = nullptr;
        RSRR_TRY(tz_values(h, z, &v));
        dfree(h->d_vals, st);
        h->d_vals = v;
        h->J = N;
        F.assign((size_t)N * N, czero<double>());
        for (int j = 0; j < N; ++j) F[(size_t)j * N + j] = mk<double>(1.0, 0.0);
    } else {
        // coefficient table F[j][i] = f_i(z_j) (host FP64)
        const int J = h->J;
        F.assign((size_t)N * J, czero<double>());
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < J; ++i) {
                zd v, dv;
                eval_fn(h->fns[i], z[j], &v, &dv);
                if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
                    return set_error(RSRR_ENONFINITE, "f_i(z_j) is not finite (a sampling point at a pole?)");
                F[(size_t)j * J + i] = fromstd(v);
            }
    }
    // probing matrix: upload and permute to the band ordering
    if (U_reim) {
        if (h->d_U && h->U_L != L) { dfree(h->d_U, st); h->d_U = nullptr; }
        if (!h->d_U) RSRR_TRY(dalloc_n(&h->d_U, (size_t)n * L, st));
        c128* raw = nullptr;
        RSRR_TRY(dalloc_n(&raw, (size_t)n * L, st));
        RSRR_CUDA(cudaMemcpyAsync(raw, U_reim, (size_t)n * L * sizeof(c128), cudaMemcpyHostToDevice, st));
        { gather_rows_kernel<<<(unsigned)ceil_div(n * L, 256), 256, 0, st>>>(raw, h->d_perm, n, L, h->d_U); note_launch(); }
        RSRR_CUDA(cudaGetLastError());
        dfree(raw, st);
        h->U_L = L;
    } else if (!h->d_U || h->U_L != L) {
        return set_error(RSRR_EINVAL, "U_reim is NULL but no probing matrix with this L is resident");
    }
    const size_t cols = (size_t)N * L;
    if (h->S_cols_cap < cols) {
        dfree(h->d_S, st);
        dfree(h->d_eta, st);
        h->d_S = nullptr;
        h->d_eta = nullptr;
        h->S_cols_cap = 0;
        RSRR_TRY(dalloc_n(&h->d_S, cols * n, st));
        RSRR_TRY(dalloc_n(&h->d_eta, cols, st));
        h->S_cols_cap = cols;
    }
    return RSRR_OK;
}

bool use_dense(const rsrr_nep h) {
    if (h->precond_band >= 0) return false;
    const int64_t n = h->n, kl = h->ord.kl, ku = h->ord.ku;
    return h->force_dense || kl > 768 || ku > 768 || (n >= 128 && 5 * (kl + ku) > 2 * n);
}

namespace {
template <typename R>
int dense_run(const std::vector<rsrr_nep>& hs, const std::vector<std::vector<c128>>& Fs, int max_refine) {
    std::vector<c128*> dF(hs.size(), nullptr);
    cudaStream_t st = hs.empty() ? nullptr : hs[0]->stream;
    int rc = RSRR_OK;
    for (size_t i = 0; i < hs.size() && rc == RSRR_OK; ++i) {
        rc = dalloc_n(&dF[i], Fs[i].size(), st);
        if (rc == RSRR_OK) {
            cudaError_t e = cudaMemcpyAsync(dF[i], Fs[i].data(), Fs[i].size() * sizeof(c128), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) rc = set_error(RSRR_ECUDA, std::string("cudaMemcpyAsync(F): ") + cudaGetErrorString(e));
        }
    }
    if (rc == RSRR_OK) rc = sample_dense_set<R>(hs, dF, max_refine);
    for (c128* p : dF) dfree(p, st);
    return rc;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// Sampler autotuner (handles created with RSRR_AUTOTUNE).  Before a handle's first sampling, the
// candidate strategies for its T(z_j) solves are timed on one sampling point (z_0) with the call's
// own precision, tolerance and budget, and the fastest that meets the tolerance is kept:
//   band LU on the tensor cores (when the band suits them), band LU on the CUDA cores, the dense
//   LU, and the iterative sampler (flexible GMRES preconditioned by the factor of a band part,
//   the half-width p holding all but 1e-12 of the Frobenius weight of T(z_0)).
// A dense point is timed only for n <= 2048; above that its time is extrapolated with n^3 from
// the last dense measurement.  Decisions are cached process-wide per size bucket (n, kl, ku in
// steps of 25 %, J, precision, ordering), so a batch of similar NEPs tunes once.
// ---------------------------------------------------------------------------------------------
namespace {
struct TuneKey {
    int nb, klb, kub, J, prec, natural;
    bool operator<(const TuneKey& o) const {
        return std::tie(nb, klb, kub, J, prec, natural) < std::tie(o.nb, o.klb, o.kub, o.J, o.prec, o.natural);
    }
};
std::mutex g_tune_mx;
std::map<TuneKey, std::pair<int, int>> g_tune;   // -> (strategy, band)
double g_dense_ms_per_n3 = 0.0;                  // last dense trial: ms / n^3

int size_bucket(int64_t x) { return x <= 0 ? -1 : (int)std::floor(std::log((double)x) / std::log(1.25)); }

// weight of T(z_0) per |row - col| offset (device atomics), then the smallest half-width holding
// all but `frac` of it
__global__ void offset_weight_kernel(const c128* __restrict__ vals, int J, int64_t nnz, const int32_t* __restrict__ rowidx,
                                     const int32_t* __restrict__ colind, const c128* __restrict__ F,
                                     double* __restrict__ w) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    c128 v = czero<double>();
    for (int i = 0; i < J; ++i) cfma(v, F[i], vals[(int64_t)i * nnz + k]);
    atomicAdd(&w[abs(rowidx[k] - colind[k])], cnorm2(v));
}

int dominant_band(rsrr_nep h, const c128* F0, double frac, int64_t* band) {
    cudaStream_t st = h->stream;
    const int64_t n = h->n;
    double* w = nullptr;
    c128* dF = nullptr;
    RSRR_TRY(dalloc_n(&w, (size_t)n, st));
    int rc = dalloc_n(&dF, (size_t)h->J, st);
    std::vector<double> hw((size_t)n);
    if (rc == RSRR_OK && (cudaMemsetAsync(w, 0, (size_t)n * 8, st) != cudaSuccess ||
                          cudaMemcpyAsync(dF, F0, (size_t)h->J * sizeof(c128), cudaMemcpyHostToDevice, st) != cudaSuccess))
        rc = set_error(RSRR_ECUDA, "autotune: copies");
    if (rc == RSRR_OK) {
        offset_weight_kernel<<<(unsigned)ceil_div(h->nnz, 256), 256, 0, st>>>(h->d_vals, h->J, h->nnz, h->d_rowidx,
                                                                             h->d_colind, dF, w);
        note_launch();
        if (cudaMemcpyAsync(hw.data(), w, (size_t)n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_error(RSRR_ECUDA, "autotune: offset weights");
    }
    dfree(w, st);
    dfree(dF, st);
    RSRR_TRY(rc);
    double total = 0.0;
    for (double x : hw) total += x;
    double acc = 0.0;
    int64_t p = 0;
    for (; p < n; ++p) {
        acc += hw[p];
        if (total - acc <= frac * total) break;
    }
    *band = p;
    return RSRR_OK;
}

enum { TUNE_BAND_TC = 0, TUNE_BAND_CC = 1, TUNE_DENSE = 2, TUNE_ITER = 3 };

void apply_strategy(rsrr_nep h, int strategy, int band) {
    h->precond_band = strategy == TUNE_ITER ? band : -1;
    h->band_cuda_cores = strategy == TUNE_BAND_CC;
    h->force_dense = strategy == TUNE_DENSE;
}

// Time of one sampling point (z_0) with a strategy, in ms; +inf if it fails or does not converge.
double trial_ms(rsrr_nep h, const std::vector<c128>& F0, int strategy, int band, int max_refine) {
    const int N0 = h->N, pb = h->precond_band;
    const bool cc = h->band_cuda_cores, fd = h->force_dense;
    apply_strategy(h, strategy, band);
    h->N = 1;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h->stream);
    int rc;
    if (strategy == TUNE_DENSE) {
        std::vector<rsrr_nep> hs{h};
        std::vector<std::vector<c128>> Fs{F0};
        rc = h->precision == RSRR_FP64 ? dense_run<double>(hs, Fs, max_refine) : dense_run<float>(hs, Fs, max_refine);
    } else {
        rc = h->precision == RSRR_FP64 ? sample_impl<double>(h, F0, max_refine) : sample_impl<float>(h, F0, max_refine);
    }
    cudaEventRecord(b, h->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->N = N0;
    h->precond_band = pb;
    h->band_cuda_cores = cc;
    h->force_dense = fd;
    return rc == RSRR_OK ? (double)ms : INFINITY;
}

int autotune(rsrr_nep h, const std::vector<c128>& F, int max_refine) {
    if (!h->autotune || h->tuned || h->tz) return RSRR_OK;
    const int64_t n = h->n, kl = h->ord.kl, ku = h->ord.ku;
    const TuneKey key{size_bucket(n), size_bucket(kl), size_bucket(ku), h->J, h->precision | (h->refine_full ? 0x100 : 0),
                      h->ord.natural ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mx);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            int64_t band = it->second.second;
            if (it->second.first == TUNE_ITER) RSRR_TRY(dominant_band(h, F.data(), 1e-12, &band));
            apply_strategy(h, it->second.first, (int)band);
            h->tuned = true;
            h->tune_cached = true;
            h->tune_strategy = it->second.first;
            h->tune_band = (int)band;
            return RSRR_OK;
        }
    }
    const std::vector<c128> F0(F.begin(), F.begin() + h->J);
    double best = INFINITY;
    int best_s = -1, best_band = -1;
    auto consider = [&](int s, int band, double ms) {
        if (ms < best) { best = ms; best_s = s; best_band = band; }
    };
    const bool band_ok = kl <= 2048 && ku <= 2048;
    if (band_ok) {
        if (h->precision != RSRR_FP64 && band_tc_eligible(n, kl, ku))
            consider(TUNE_BAND_TC, -1, trial_ms(h, F0, TUNE_BAND_TC, -1, max_refine));
        consider(TUNE_BAND_CC, -1, trial_ms(h, F0, TUNE_BAND_CC, -1, max_refine));
    }
    if (n <= 2048) {
        const double ms = trial_ms(h, F0, TUNE_DENSE, -1, max_refine);
        if (std::isfinite(ms)) g_dense_ms_per_n3 = ms / ((double)n * n * n);
        consider(TUNE_DENSE, -1, ms);
    } else if (g_dense_ms_per_n3 > 0.0) {
        consider(TUNE_DENSE, -1, g_dense_ms_per_n3 * (double)n * n * n);
    } else if (!band_ok) {
        consider(TUNE_DENSE, -1, 1e30);  // the only direct option left
    }
    int64_t p = 0;
    RSRR_TRY(dominant_band(h, F0.data(), 1e-12, &p));
    if (p < std::min(kl, ku) && p < n - 1)
        consider(TUNE_ITER, (int)p, trial_ms(h, F0, TUNE_ITER, (int)p, max_refine));
    if (best_s < 0) best_s = band_ok ? TUNE_BAND_CC : TUNE_DENSE;
    apply_strategy(h, best_s, best_band);
    h->tuned = true;
    h->tune_cached = false;
    h->tune_strategy = best_s;
    h->tune_band = best_band;
    std::lock_guard<std::mutex> lk(g_tune_mx);
    g_tune[key] = {best_s, best_band};
    return RSRR_OK;
}
}  // namespace

int sample_run(rsrr_nep h, const double* U_reim, int max_refine) {
    std::vector<std::vector<c128>> F(1);
    RSRR_TRY(sample_prepare(h, U_reim, &F[0]));
    RSRR_TRY(autotune(h, F[0], max_refine));
    h->dense_used = use_dense(h);
    if (h->dense_used) {
        std::vector<rsrr_nep> hs{h};
        return h->precision == RSRR_FP64 ? dense_run<double>(hs, F, max_refine) : dense_run<float>(hs, F, max_refine);
    }
    if (h->precision == RSRR_FP64) return sample_impl<double>(h, F[0], max_refine);
    return sample_impl<float>(h, F[0], max_refine);
}

// Several NEPs in one call: the dense ones share one fused dense launch, the banded ones run one
// after another on the band path, each on its own stream.  All handles use one precision.
int sample_batch_run(const std::vector<rsrr_nep>& hs, const std::vector<const double*>& U, int max_refine) {
    std::vector<std::vector<c128>> F(hs.size());
    for (size_t i = 0; i < hs.size(); ++i) RSRR_TRY(sample_prepare(hs[i], U[i], &F[i]));
    for (size_t i = 0; i < hs.size(); ++i) RSRR_TRY(autotune(hs[i], F[i], max_refine));
    std::vector<rsrr_nep> dh;
    std::vector<std::vector<c128>> dFs;
    for (size_t i = 0; i < hs.size(); ++i) {
        hs[i]->dense_used = use_dense(hs[i]);
        if (hs[i]->dense_used) {
            dh.push_back(hs[i]);
            dFs.push_back(F[i]);
        }
    }
    const bool fp64 = hs[0]->precision == RSRR_FP64;
    if (!dh.empty()) {
        // The dense NEPs share one launch on the first one's stream: it waits for the work already
        // queued on the other handles' streams (their probing matrices and S_hat storage), and
        // those streams wait for it in turn.
        cudaStream_t s0 = dh[0]->stream;
        cudaEvent_t ev = nullptr;
        RSRR_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        int rc = RSRR_OK;
        for (rsrr_nep h : dh) {
            if (h->stream == s0 || rc != RSRR_OK) continue;
            if (cudaEventRecord(ev, h->stream) != cudaSuccess || cudaStreamWaitEvent(s0, ev, 0) != cudaSuccess)
                rc = set_error(RSRR_ECUDA, "rsrr_sample_batch: stream ordering failed");
        }
        if (rc == RSRR_OK) rc = fp64 ? dense_run<double>(dh, dFs, max_refine) : dense_run<float>(dh, dFs, max_refine);
        if (cudaEventRecord(ev, s0) == cudaSuccess)
            for (rsrr_nep h : dh)
                if (h->stream != s0) cudaStreamWaitEvent(h->stream, ev, 0);
        cudaEventDestroy(ev);
        RSRR_TRY(rc);
    }
    for (size_t i = 0; i < hs.size(); ++i) {
        if (use_dense(hs[i])) continue;
        RSRR_TRY(fp64 ? sample_impl<double>(hs[i], F[i], max_refine) : sample_impl<float>(hs[i], F[i], max_refine));
    }
    for (rsrr_nep h : hs) RSRR_CUDA(cudaStreamSynchronize(h->stream));
    return RSRR_OK;
}

}  // namespace rsrr
