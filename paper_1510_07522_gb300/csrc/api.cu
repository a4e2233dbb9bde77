// C ABI entry points (rsrr.h): handle life cycle, rsrr_sample, introspection.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "internal.h"

namespace rsrr {
int sample_run(rsrr_nep h, const double* U_reim, int max_refine);
int sample_batch_run(const std::vector<rsrr_nep>& hs, const std::vector<const double*>& U, int max_refine);
int project_run(rsrr_nep h, double delta);
int chebyshev_reduce(rsrr_nep h, int d, double lo, double hi);
int solve_run(rsrr_nep h, int N_S, int K, double tol_gap, int cap, double* lambda_reim, double* V_reim,
              double* resid, int32_t* nC_out);

int tz_values(rsrr_nep_s* h, const std::vector<zd>& z, c128** d_vals) {
    const int64_t m = (int64_t)z.size(), nnz = h->nnz;
    *d_vals = nullptr;
    if (m == 0) return RSRR_OK;
    std::vector<double> zr(2 * m), raw((size_t)2 * m * nnz, 0.0);
    for (int64_t k = 0; k < m; ++k) {
        zr[2 * k] = z[k].real();
        zr[2 * k + 1] = z[k].imag();
    }
    h->tz(h->tz_user, m, zr.data(), raw.data());
    std::vector<c128> pv((size_t)m * nnz);
    for (int64_t k = 0; k < m; ++k)
        for (int64_t e = 0; e < nnz; ++e) {
            const double* v = raw.data() + 2 * (k * nnz + h->vsrc[e]);
            if (!std::isfinite(v[0]) || !std::isfinite(v[1]))
                return set_error(RSRR_ENONFINITE, "T(z) from the tz callback is not finite");
            pv[(size_t)k * nnz + e] = mk<double>(v[0], v[1]);
        }
    RSRR_TRY(dalloc_n(d_vals, pv.size(), h->stream));
    if (cudaMemcpyAsync(*d_vals, pv.data(), pv.size() * sizeof(c128), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        dfree(*d_vals, h->stream);
        *d_vals = nullptr;
        return set_error(RSRR_ECUDA, "upload of T(z) values");
    }
    return RSRR_OK;
}

namespace {
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

struct Timer {
    rsrr_nep h;
    explicit Timer(rsrr_nep hh) : h(hh) { cudaEventRecord(h->ev0, h->stream); }
    double stop() {
        cudaEventRecord(h->ev1, h->stream);
        cudaEventSynchronize(h->ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        return ms;
    }
};
}  // namespace
}  // namespace rsrr

using namespace rsrr;

extern "C" {

const char* rsrr_last_error(void) { return rsrr::last_error(); }
const char* rsrr_version(void) { return "rsrr-gb300 0.1 (sm_103a)"; }
int64_t rsrr_kernel_launches(void) { return rsrr::launches_total(); }

int64_t rsrr_device_peak_bytes(int32_t reset) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return rsrr::set_error(RSRR_ECUDA, "cudaGetDevice failed");
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess)
        return rsrr::set_error(RSRR_ECUDA, "no default memory pool");
    uint64_t high = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess)
        return rsrr::set_error(RSRR_ECUDA, "cudaMemPoolGetAttribute failed");
    if (reset) {
        uint64_t zero = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    return (int64_t)high;
}

}  // extern "C"

namespace {
// Shared by rsrr_create_nep (J terms with values) and rsrr_create_nep_tz (J = 0, tz given).
int create_impl(int64_t n, int32_t J, const int64_t* rowptr, const int32_t* colind,
                const double* vals_reim, const rsrr_fn* f, rsrr_tz_cb tz, void* tz_user, uint32_t flags,
                void* stream, rsrr_nep* out) {
    if (!out) return set_error(RSRR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX - 1) return set_error(RSRR_EINVAL, "n out of range");
    if (tz ? J != 0 : (J < 1 || J > 16)) return set_error(RSRR_EINVAL, "J must be in 1..16");
    if (!rowptr || !colind || (!tz && (!vals_reim || !f))) return set_error(RSRR_EINVAL, "NULL input array");
    if (flags & ~(RSRR_NATURAL_ORDER | RSRR_DENSE_LU | RSRR_BAND_CUDA_CORES | RSRR_AUTOTUNE))
        return set_error(RSRR_EINVAL, "unknown flag bits");
    if (rowptr[0] != 0) return set_error(RSRR_EINVAL, "rowptr[0] must be 0");
    for (int64_t r = 0; r < n; ++r) {
        if (rowptr[r + 1] < rowptr[r]) return set_error(RSRR_EINVAL, "rowptr not monotone");
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            if (colind[k] < 0 || colind[k] >= n) return set_error(RSRR_EINVAL, "column index out of range");
            if (k > rowptr[r] && colind[k] <= colind[k - 1])
                return set_error(RSRR_EINVAL, "column indices of a row must be strictly increasing");
        }
    }
    const int64_t nnz = rowptr[n];
    if (nnz < 1 || nnz > (int64_t)INT32_MAX) return set_error(RSRR_EINVAL, "nnz out of range");
    for (int i = 0; i < J; ++i) RSRR_TRY(check_fn(f[i]));
    for (int64_t k = 0; k < 2 * nnz * J; ++k)
        if (!std::isfinite(vals_reim[k])) return set_error(RSRR_ENONFINITE, "non-finite matrix value");

    auto* h = new rsrr_nep_s();
    cudaGetDevice(&h->device);
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    h->n = n;
    h->nnz = nnz;
    h->J = J;
    if (J) h->fns.assign(f, f + J);
    h->tz = tz;
    h->tz_user = tz_user;
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        delete h;
        return set_error(RSRR_ECUDA, "cudaEventCreate failed");
    }
    choose_ordering(n, rowptr, colind, (flags & RSRR_NATURAL_ORDER) != 0, &h->ord);
    h->force_dense = (flags & RSRR_DENSE_LU) != 0;
    h->band_cuda_cores = (flags & RSRR_BAND_CUDA_CORES) != 0;
    h->autotune = (flags & RSRR_AUTOTUNE) != 0;
    // permuted CSR (rows in new order, columns renumbered and sorted) and values
    std::vector<int64_t> prow(n + 1, 0);
    std::vector<int32_t> pcol(nnz), prowidx(nnz);
    std::vector<int64_t> src(nnz);
    {
        std::vector<std::pair<int32_t, int64_t>> tmp;
        int64_t pos = 0;
        for (int64_t rn = 0; rn < n; ++rn) {
            const int64_t ro = h->ord.perm[rn];
            tmp.clear();
            for (int64_t k = rowptr[ro]; k < rowptr[ro + 1]; ++k) tmp.emplace_back(h->ord.iperm[colind[k]], k);
            std::sort(tmp.begin(), tmp.end());
            for (auto& pr : tmp) {
                pcol[pos] = pr.first;
                prowidx[pos] = (int32_t)rn;
                src[pos] = pr.second;
                ++pos;
            }
            prow[rn + 1] = pos;
        }
    }
    h->vsrc = src;
    std::vector<c128> pv((size_t)J * nnz);
    h->normA.assign(J, 0.0);
    for (int i = 0; i < J; ++i) {
        double s2 = 0.0;
        for (int64_t k = 0; k < nnz; ++k) {
            const double* v = vals_reim + 2 * ((int64_t)i * nnz + src[k]);
            pv[(size_t)i * nnz + k] = mk<double>(v[0], v[1]);
            s2 += v[0] * v[0] + v[1] * v[1];
        }
        h->normA[i] = std::sqrt(s2);
    }
    DeviceGuard g(h->device);
    cudaStream_t st = h->stream;
    int rc = RSRR_OK;
    if ((rc = dalloc_n(&h->d_rowptr, n + 1, st)) || (rc = dalloc_n(&h->d_colind, nnz, st)) ||
        (rc = dalloc_n(&h->d_rowidx, nnz, st)) || (J && (rc = dalloc_n(&h->d_vals, (size_t)J * nnz, st))) ||
        (rc = dalloc_n(&h->d_perm, n, st))) {
        rsrr_destroy(h);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_rowptr, prow.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_colind, pcol.data(), nnz * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_rowidx, prowidx.data(), nnz * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && J) e = cudaMemcpyAsync(h->d_vals, pv.data(), pv.size() * sizeof(c128), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_perm, h->ord.perm.data(), n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        rsrr_destroy(h);
        return set_error(RSRR_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    h->device_bytes = (n + 1) * 8 + nnz * 8 + (int64_t)pv.size() * 16 + n * 4;
    *out = h;
    return RSRR_OK;
}
}  // namespace

extern "C" {

int rsrr_create_nep(int64_t n, int32_t J, const int64_t* rowptr, const int32_t* colind,
                    const double* vals_reim, const rsrr_fn* f, uint32_t flags, void* stream,
                    rsrr_nep* out) {
    if (!vals_reim || !f) return set_error(RSRR_EINVAL, "NULL input array");
    return create_impl(n, J, rowptr, colind, vals_reim, f, nullptr, nullptr, flags, stream, out);
}

int rsrr_create_nep_tz(int64_t n, const int64_t* rowptr, const int32_t* colind, rsrr_tz_cb tz, void* user,
                       uint32_t flags, void* stream, rsrr_nep* out) {
    if (!tz) return set_error(RSRR_EINVAL, "tz is NULL");
    return create_impl(n, 0, rowptr, colind, nullptr, nullptr, tz, user, flags, stream, out);
}

namespace {
// N < 0: the contour serves rsrr_solve only (its own N_S is checked there).
int check_contour(const rsrr_contour* C, int32_t N) {
    if (!(C->a > 0) || !(C->b > 0) || !std::isfinite(C->gamma_re) || !std::isfinite(C->gamma_im) ||
        !std::isfinite(C->a) || !std::isfinite(C->b))
        return set_error(RSRR_EINVAL, "bad contour");
    if (C->shape != RSRR_CONTOUR_ELLIPSE && C->shape != RSRR_CONTOUR_RECTANGLE)
        return set_error(RSRR_EINVAL, "unknown contour shape");
    if (C->shape == RSRR_CONTOUR_RECTANGLE) {
        if (N >= 0 && (N < 4 || N % 2)) return set_error(RSRR_EINVAL, "a rectangle needs an even N >= 4");
        if (C->side_nodes < 0 || (N >= 0 && C->side_nodes > N / 2 - 1))
            return set_error(RSRR_EINVAL, "side_nodes must be in 0..N/2-1");
    } else if (C->side_nodes != 0) {
        return set_error(RSRR_EINVAL, "side_nodes is for rectangles only");
    }
    return RSRR_OK;
}

int check_sample_args(rsrr_nep h, const rsrr_contour* C, int32_t N, int32_t L, int32_t precision, double tol,
                      int32_t max_refine, bool own_points = false) {
    if (!h || !C) return set_error(RSRR_EINVAL, "NULL handle or contour");
    if (N < 1 || N > 4096 || L < 1 || L > 256) return set_error(RSRR_EINVAL, "N or L out of range");
    RSRR_TRY(check_contour(C, own_points ? -1 : N));
    const int mode = precision & 0xff;
    if ((mode != RSRR_FP64 && mode != RSRR_C64_IR) || (precision & ~(0xff | RSRR_REFINE_FULL)))
        return set_error(RSRR_EINVAL, "unknown precision or flag");
    // max_refine: refinement sweeps (direct factor), or Krylov iterations (iterative sampler)
    if (!(tol > 0) || max_refine < 0 || max_refine > (h->precond_band >= 0 ? 100000 : 100))
        return set_error(RSRR_EINVAL, "bad tol or max_refine");
    if ((int64_t)N * L * h->n > (int64_t)1 << 34) return set_error(RSRR_ENOMEM, "S_hat too large");
    return RSRR_OK;
}

void begin_sample(rsrr_nep h, const rsrr_contour* C, int32_t N, int32_t L, int32_t precision, double tol) {
    h->C = *C;
    h->points.clear();
    h->N = N;
    h->L = L;
    h->precision = precision & 0xff;
    h->refine_full = (precision & RSRR_REFINE_FULL) != 0;
    h->tol = tol;
    h->sampled = h->projected = false;
    h->kS = -1;
    h->nbar = -1;
}

int finish_sample(rsrr_nep h) {
    std::vector<double> eta((size_t)h->N * h->L);
    RSRR_CUDA(cudaMemcpy(eta.data(), h->d_eta, eta.size() * 8, cudaMemcpyDeviceToHost));
    h->max_eta = 0;
    for (double e : eta) h->max_eta = std::max(h->max_eta, e);
    h->sampled = true;
    return RSRR_OK;
}
}  // namespace

int rsrr_sample(rsrr_nep h, const rsrr_contour* C, int32_t N, int32_t L, const double* U_reim,
                int32_t precision, double tol, int32_t max_refine) {
    RSRR_TRY(check_sample_args(h, C, N, L, precision, tol, max_refine));
    DeviceGuard g(h->device);
    begin_sample(h, C, N, L, precision, tol);
    Timer t(h);
    int rc = sample_run(h, U_reim, max_refine);
    h->ms_sample = t.stop();
    if (rc != RSRR_OK) return rc;
    return finish_sample(h);
}

int rsrr_sample_points(rsrr_nep h, const rsrr_contour* C, int32_t N, const double* z_reim, int32_t L,
                       const double* U_reim, int32_t precision, double tol, int32_t max_refine) {
    RSRR_TRY(check_sample_args(h, C, N, L, precision, tol, max_refine, true));
    if (!z_reim) return set_error(RSRR_EINVAL, "rsrr_sample_points: NULL point array");
    std::vector<zd> pts(N);
    for (int32_t j = 0; j < N; ++j) {
        pts[j] = zd(z_reim[2 * j], z_reim[2 * j + 1]);
        if (!std::isfinite(pts[j].real()) || !std::isfinite(pts[j].imag()))
            return set_error(RSRR_EINVAL, "rsrr_sample_points: non-finite point");
    }
    DeviceGuard g(h->device);
    begin_sample(h, C, N, L, precision, tol);
    h->points = pts;
    Timer t(h);
    int rc = sample_run(h, U_reim, max_refine);
    h->ms_sample = t.stop();
    if (rc != RSRR_OK) return rc;
    return finish_sample(h);
}

int rsrr_sample_batch(rsrr_nep* hs, int32_t count, const rsrr_contour* C, const int32_t* N, const int32_t* L,
                      const double* const* U_reim, int32_t precision, double tol, int32_t max_refine) {
    if (!hs || !C || !N || !L || count < 1 || count > 65536)
        return set_error(RSRR_EINVAL, "rsrr_sample_batch: NULL array or count out of range");
    for (int32_t i = 0; i < count; ++i) {
        RSRR_TRY(check_sample_args(hs[i], &C[i], N[i], L[i], precision, tol, max_refine));
        if (hs[i]->device != hs[0]->device)
            return set_error(RSRR_EINVAL, "rsrr_sample_batch: all handles must be on one device");
        for (int32_t k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return set_error(RSRR_EINVAL, "rsrr_sample_batch: a handle appears twice");
    }
    DeviceGuard g(hs[0]->device);
    std::vector<rsrr_nep> v(hs, hs + count);
    std::vector<const double*> U(count, nullptr);
    for (int32_t i = 0; i < count; ++i) {
        begin_sample(hs[i], &C[i], N[i], L[i], precision, tol);
        U[i] = U_reim ? U_reim[i] : nullptr;
    }
    Timer t(hs[0]);
    int rc = sample_batch_run(v, U, max_refine);
    const double ms = t.stop();
    for (rsrr_nep h : v) h->ms_sample = ms;
    if (rc != RSRR_OK) return rc;
    for (rsrr_nep h : v) RSRR_TRY(finish_sample(h));
    return RSRR_OK;
}

int rsrr_project(rsrr_nep h, double delta, int32_t* k_S_out) {
    if (!h) return set_error(RSRR_EINVAL, "NULL handle");
    if (!h->sampled) return set_error(RSRR_EORDER, "rsrr_project needs a successful rsrr_sample");
    if (!(delta >= 0) || !(delta < 1)) return set_error(RSRR_EINVAL, "delta must be in [0, 1)");
    if (h->tz && !h->tz_basis_only)
        return set_error(RSRR_EINVAL, "a handle of rsrr_create_nep_tz is projected with rsrr_project_chebyshev");
    DeviceGuard g(h->device);
    h->projected = false;
    Timer t(h);
    int rc = project_run(h, delta);
    h->ms_project = t.stop();
    if (rc != RSRR_OK) return rc;
    h->projected = true;
    if (k_S_out) *k_S_out = h->kS;
    return RSRR_OK;
}

int rsrr_project_chebyshev(rsrr_nep h, int32_t d, double x_lo, double x_hi, double delta, int32_t* k_S_out) {
    if (!h) return set_error(RSRR_EINVAL, "NULL handle");
    if (d < 0 || d > 256 || !std::isfinite(x_lo) || !std::isfinite(x_hi) || !(x_lo < x_hi))
        return set_error(RSRR_EINVAL, "Chebyshev degree must be in 0..256 and x_lo < x_hi");
    h->tz_basis_only = true;
    const int rp = rsrr_project(h, delta, k_S_out);
    h->tz_basis_only = false;
    RSRR_TRY(rp);
    DeviceGuard g(h->device);
    const int rc = chebyshev_reduce(h, d, x_lo, x_hi);
    if (rc != RSRR_OK) h->projected = false;
    return rc;
}

int rsrr_project_moments(rsrr_nep h, int32_t Kp, double delta, int32_t* k_S_out) {
    if (!h) return set_error(RSRR_EINVAL, "NULL handle");
    if (!h->sampled) return set_error(RSRR_EORDER, "rsrr_project_moments needs a successful rsrr_sample");
    if (Kp < 1 || Kp > h->N) return set_error(RSRR_EINVAL, "moment order K' must be in 1..N");
    if (!h->points.empty())
        return set_error(RSRR_EINVAL, "the moment scheme needs the contour's quadrature nodes, not rsrr_sample_points");
    h->moment_order = Kp;
    const int rc = rsrr_project(h, delta, k_S_out);
    h->moment_order = 0;
    return rc;
}

int rsrr_solve(rsrr_nep h, int32_t N_S, int32_t K, double tol_gap, int32_t cap, double* lambda_reim,
               double* V_reim, double* resid, int32_t* nC_out) {
    if (!h) return set_error(RSRR_EINVAL, "NULL handle");
    if (!h->projected) return set_error(RSRR_EORDER, "rsrr_solve needs a successful rsrr_project");
    if (h->red_J < 1) return set_error(RSRR_EORDER, "no reduced NEP (a tz handle needs rsrr_project_chebyshev)");
    if (N_S < 4 || N_S > 100000 || K < 1 || K > 64 || !(tol_gap > 1) || cap < 0 || !nC_out ||
        (cap > 0 && !lambda_reim))
        return set_error(RSRR_EINVAL, "bad rsrr_solve arguments");
    if (h->C.shape == RSRR_CONTOUR_RECTANGLE && N_S % 2)
        return set_error(RSRR_EINVAL, "a rectangular contour needs an even N_S");
    DeviceGuard g(h->device);
    Timer t(h);
    int rc = solve_run(h, N_S, K, tol_gap, cap, lambda_reim, V_reim, resid, nC_out);
    h->ms_solve = t.stop();
    return rc;
}

int rsrr_set_band_preconditioner(rsrr_nep h, int32_t band) {
    if (!h) return set_error(RSRR_EINVAL, "NULL handle");
    if (band < -1 || band >= h->n) return set_error(RSRR_EINVAL, "band must be -1 (off) or in 0..n-1");
    h->precond_band = band;
    return RSRR_OK;
}

int rsrr_zgemm(int32_t path, int32_t opA, int32_t opB, int32_t M, int32_t N, int32_t K, const double* alpha_reim,
               const void* A, int64_t lda, int64_t sA, const void* B, int64_t ldb, int64_t sB,
               const double* beta_reim, void* C, int64_t ldc, int64_t sC, int32_t batch, void* stream) {
    if (path < 0 || path > 2 || opA < 0 || opA > 2 || opB < 0 || opB > 2 || M < 0 || N < 0 || K < 0 || batch < 1 ||
        !alpha_reim || !beta_reim || !A || !B || !C)
        return set_error(RSRR_EINVAL, "rsrr_zgemm: bad argument");
    const int64_t rowsA = opA == OP_N ? M : K, rowsB = opB == OP_N ? K : N;
    if (lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB) || ldc < std::max<int64_t>(1, M))
        return set_error(RSRR_EINVAL, "rsrr_zgemm: leading dimension too small");
    Zgemm g;
    g.opA = opA; g.opB = opB; g.M = M; g.N = N; g.K = K;
    g.alpha = mk<double>(alpha_reim[0], alpha_reim[1]);
    g.beta = mk<double>(beta_reim[0], beta_reim[1]);
    g.A = static_cast<const c128*>(A); g.lda = lda; g.sA = sA;
    g.B = static_cast<const c128*>(B); g.ldb = ldb; g.sB = sB;
    g.C = static_cast<c128*>(C); g.ldc = ldc; g.sC = sC; g.batch = batch;
    const int prev = zgemm_get_path();
    zgemm_set_path(path);
    const int rc = zgemm(g, reinterpret_cast<cudaStream_t>(stream));
    zgemm_set_path(prev);
    return rc;
}

int rsrr_zinv_batch(int32_t path, int32_t k, int32_t batch, void* A, int32_t* info, void* stream) {
    if (path < 0 || path > 2 || k < 1 || batch < 1 || !A || !info)
        return set_error(RSRR_EINVAL, "rsrr_zinv_batch: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(info, 0, (size_t)batch * 4, st) != cudaSuccess)
        return set_error(RSRR_ECUDA, "rsrr_zinv_batch: memset");
    const int prev = zgemm_get_path();
    zgemm_set_path(path);
    int rc = zinv_batch(static_cast<c128*>(A), k, batch, info, st);
    zgemm_set_path(prev);
    if (rc == RSRR_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = set_error(RSRR_ECUDA, "rsrr_zinv_batch");
    return rc;
}

int rsrr_get_info(rsrr_nep h, rsrr_info* o) {
    if (!h || !o) return set_error(RSRR_EINVAL, "NULL argument");
    std::memset(o, 0, sizeof(*o));
    o->n = h->n;
    o->nnz = h->nnz;
    o->J = h->J;
    o->N = h->N;
    o->L = h->L;
    o->kl = (int32_t)h->ord.kl;
    o->ku = (int32_t)h->ord.ku;
    o->natural_order = h->ord.natural ? 1 : 0;
    o->precision = h->precision;
    o->refine_sweeps = h->refine_sweeps;
    o->k_S = h->kS;
    o->nbar = h->nbar;
    o->n_winding = h->n_winding;
    o->n_gap = h->n_gap;
    o->winding_re = h->winding.real();
    o->winding_im = h->winding.imag();
    o->max_eta = h->max_eta;
    o->ms_sample = h->ms_sample;
    o->ms_project = h->ms_project;
    o->ms_solve = h->ms_solve;
    o->device_bytes = h->device_bytes;
    o->ms_factor = h->ms_factor;
    o->ms_trsv = h->ms_trsv;
    o->factor_launches = h->factor_launches;
    o->trsv_launches = h->trsv_launches;
    o->rows_kept = h->rows_kept;
    o->jacobi_sweeps_project = h->jacobi_sweeps_project;
    o->jacobi_sweeps_solve = h->jacobi_sweeps_solve;
    o->ms_project_qr = h->ms_project_parts[0];
    o->ms_project_svd = h->ms_project_parts[1];
    o->ms_project_basis = h->ms_project_parts[2];
    o->ms_project_gemm = h->ms_project_parts[3];
    o->ms_solve_inverse = h->ms_solve_parts[0];
    o->ms_solve_svd = h->ms_solve_parts[1];
    o->ms_solve_extract = h->ms_solve_parts[2];
    o->ms_zgemm = h->ms_zgemm_project + h->ms_zgemm_solve;
    o->zgemm_gflop = (h->zgemm_flops_project + h->zgemm_flops_solve) * 1e-9;
    o->dense_lu = h->dense_used ? 1 : 0;
    o->band_lu_tc = (h->band_tc_used && !h->dense_used) ? 1 : 0;
    o->tune_strategy = h->tuned ? h->tune_strategy : -1;
    o->tune_band = h->tuned ? h->tune_band : -1;
    o->tune_cached = h->tune_cached ? 1 : 0;
    o->iterative_band = h->precond_band;
    o->proj_cols = h->proj_cols;
    o->red_terms = h->red_J;
    o->ms_zgemm_tc = h->ms_zgemm_tc_project + h->ms_zgemm_tc_solve;
    o->zgemm_tc_gflop = (h->zgemm_tc_flops_project + h->zgemm_tc_flops_solve) * 1e-9;
    o->ms_jacobi = h->ms_jacobi_project + h->ms_jacobi_solve;
    o->jacobi_gflop = (h->jacobi_flops_project + h->jacobi_flops_solve) * 1e-9;
    return RSRR_OK;
}

int rsrr_get_samples(rsrr_nep h, int32_t j0, int32_t j1, double* out_reim) {
    if (!h || !out_reim) return set_error(RSRR_EINVAL, "NULL argument");
    if (!h->sampled) return set_error(RSRR_EORDER, "no samples");
    if (j0 < 0 || j1 > h->N || j0 >= j1) return set_error(RSRR_EINVAL, "bad point range");
    DeviceGuard g(h->device);
    const int64_t n = h->n, cols = (int64_t)(j1 - j0) * h->L;
    std::vector<c128> tmp((size_t)(n * cols));
    RSRR_CUDA(cudaMemcpy(tmp.data(), h->d_S + (int64_t)j0 * h->L * n, tmp.size() * sizeof(c128),
                         cudaMemcpyDeviceToHost));
    for (int64_t c = 0; c < cols; ++c)
        for (int64_t r = 0; r < n; ++r) {
            const c128 v = tmp[(size_t)(r + c * n)];
            const int64_t ro = h->ord.perm[r];
            out_reim[2 * (ro + c * n)] = v.re;
            out_reim[2 * (ro + c * n) + 1] = v.im;
        }
    return RSRR_OK;
}

int rsrr_get_eta(rsrr_nep h, double* out) {
    if (!h || !out) return set_error(RSRR_EINVAL, "NULL argument");
    if (!h->sampled) return set_error(RSRR_EORDER, "no samples");
    DeviceGuard g(h->device);
    RSRR_CUDA(cudaMemcpy(out, h->d_eta, (size_t)h->N * h->L * 8, cudaMemcpyDeviceToHost));
    return RSRR_OK;
}

int rsrr_get_sigma(rsrr_nep h, double* out) {
    if (!h || !out) return set_error(RSRR_EINVAL, "NULL argument");
    if (!h->projected) return set_error(RSRR_EORDER, "no projection");
    std::copy(h->sigma.begin(), h->sigma.end(), out);
    return RSRR_OK;
}

int rsrr_get_basis(rsrr_nep h, double* out_reim) {
    if (!h || !out_reim) return set_error(RSRR_EINVAL, "NULL argument");
    if (!h->projected) return set_error(RSRR_EORDER, "no projection");
    DeviceGuard g(h->device);
    const int64_t n = h->n;
    std::vector<c128> tmp((size_t)(n * h->kS));
    if (!tmp.empty())
        RSRR_CUDA(cudaMemcpy(tmp.data(), h->d_Q, tmp.size() * sizeof(c128), cudaMemcpyDeviceToHost));
    for (int64_t c = 0; c < h->kS; ++c)
        for (int64_t r = 0; r < n; ++r) {
            const c128 v = tmp[(size_t)(r + c * n)];
            const int64_t ro = h->ord.perm[r];
            out_reim[2 * (ro + c * n)] = v.re;
            out_reim[2 * (ro + c * n) + 1] = v.im;
        }
    return RSRR_OK;
}

int rsrr_get_projected(rsrr_nep h, double* out_reim) {
    if (!h || !out_reim) return set_error(RSRR_EINVAL, "NULL argument");
    if (!h->projected) return set_error(RSRR_EORDER, "no projection");
    DeviceGuard g(h->device);
    const size_t cnt = (size_t)h->red_J * h->kS * h->kS;
    if (cnt) RSRR_CUDA(cudaMemcpy(out_reim, h->d_P, cnt * sizeof(c128), cudaMemcpyDeviceToHost));
    return RSRR_OK;
}

int rsrr_get_hankel_sigma(rsrr_nep h, double* out) {
    if (!h || !out) return set_error(RSRR_EINVAL, "NULL argument");
    if (h->nbar < 0) return set_error(RSRR_EORDER, "no reduced solve");
    std::copy(h->sigma_H.begin(), h->sigma_H.end(), out);
    return RSRR_OK;
}

void rsrr_destroy(rsrr_nep h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStream_t st = h->stream;
    dfree(h->d_rowptr, st);
    dfree(h->d_colind, st);
    dfree(h->d_rowidx, st);
    dfree(h->d_vals, st);
    dfree(h->d_perm, st);
    dfree(h->d_U, st);
    dfree(h->d_S, st);
    dfree(h->d_eta, st);
    dfree(h->d_Q, st);
    dfree(h->d_P, st);
    cudaStreamSynchronize(st);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

}  // extern "C"
