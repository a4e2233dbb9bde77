// Host-side parts of the RSRR library: error state, the scalar functions f_i(z) of
// T(z) = sum_i f_i(z) A_i (Eq. eq-Z-expr), contour nodes, and the band-reducing ordering.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>

#include "internal.h"

namespace rsrr {

// ---- error state -----------------------------------------------------------------------
static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
const char* last_error() { return g_last_error.c_str(); }

// ---- launch counter ------------------------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
void note_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ---- stream-ordered allocation -----------------------------------------------------------
int dalloc(void** p, size_t bytes, cudaStream_t s) {
    static thread_local int configured_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        configured_device = dev;
    }
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(RSRR_ENOMEM, "device allocation of " + std::to_string(bytes) +
                                          " bytes failed: " + cudaGetErrorString(e));
    }
    return RSRR_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---- scalar functions ----------------------------------------------------------------------
int check_fn(const rsrr_fn& f) {
    if (f.kind < RSRR_F_CONST || f.kind > RSRR_F_CHEBYSHEV)
        return set_error(RSRR_EINVAL, "unknown function kind " + std::to_string(f.kind));
    if (f.kind == RSRR_F_CALLBACK && !f.cb) return set_error(RSRR_EINVAL, "RSRR_F_CALLBACK without a function");
    for (double v : f.p)
        if (!std::isfinite(v)) return set_error(RSRR_ENONFINITE, "non-finite function parameter");
    if (f.kind == RSRR_F_ISQRT_SHIFT && f.p[1] != 0.0 && f.p[1] != 1.0)
        return set_error(RSRR_EINVAL, "sqrt branch flag must be 0 or 1");
    if (f.kind == RSRR_F_CHEBYSHEV &&
        (f.p[0] < 0 || f.p[0] > 1024 || f.p[0] != std::floor(f.p[0]) || !(f.p[1] < f.p[2])))
        return set_error(RSRR_EINVAL, "Chebyshev kind needs an integer degree 0..1024 and p1 < p2");
    return RSRR_OK;
}

void eval_fn(const rsrr_fn& f, zd z, zd* val, zd* deriv) {
    const zd I(0.0, 1.0);
    switch (f.kind) {
        case RSRR_F_CONST: *val = 1.0; *deriv = 0.0; break;
        case RSRR_F_Z: *val = z; *deriv = 1.0; break;
        case RSRR_F_Z2: *val = z * z; *deriv = 2.0 * z; break;
        case RSRR_F_ISQRT_SHIFT:
            if (f.p[1] == 0.0) {  // i sqrt(z - s), principal root
                zd r = std::sqrt(z - f.p[0]);
                *val = I * r;
                *deriv = 0.5 * I / r;
            } else {              // continued branch: i sqrt(z - s) := -sqrt(s - z)
                zd r = std::sqrt(f.p[0] - z);
                *val = -r;
                *deriv = 0.5 / r;
            }
            break;
        case RSRR_F_EXP_DELAY: {
            zd e = std::exp(-f.p[0] * z);
            *val = e;
            *deriv = -f.p[0] * e;
            break;
        }
        case RSRR_F_RATIONAL: {
            zd d = z + f.p[1];
            *val = f.p[0] * z / d;
            *deriv = f.p[0] * f.p[1] / (d * d);
            break;
        }
        case RSRR_F_CALLBACK: {
            const double zr[2] = {z.real(), z.imag()};
            double fr[2] = {0.0, 0.0}, dr[2] = {0.0, 0.0};
            f.cb(f.user, 1, zr, fr, dr);
            *val = zd(fr[0], fr[1]);
            *deriv = zd(dr[0], dr[1]);
            break;
        }
        case RSRR_F_CHEBYSHEV: {
            // three-term recurrences tau_{k+1} = 2x tau_k - tau_{k-1} and, differentiated,
            // tau'_{k+1} = 2 tau_k + 2x tau'_k - tau'_{k-1}, at x = (2z - p1 - p2) / (p2 - p1)
            const int m = (int)f.p[0];
            const double w = f.p[2] - f.p[1];
            const zd x = (2.0 * z - (f.p[1] + f.p[2])) / w;
            zd t0 = 1.0, t1 = x, d0 = 0.0, d1 = 1.0;
            if (m == 0) { *val = 1.0; *deriv = 0.0; break; }
            for (int k = 1; k < m; ++k) {
                const zd t2 = 2.0 * x * t1 - t0, d2 = 2.0 * t1 + 2.0 * x * d1 - d0;
                t0 = t1; t1 = t2; d0 = d1; d1 = d2;
            }
            *val = t1;
            *deriv = d1 * (2.0 / w);
            break;
        }
        default: *val = 0.0; *deriv = 0.0;
    }
}

// m-point Gauss-Legendre rule on [-1, 1], nodes increasing: Newton's method on P_m from the
// asymptotic first guesses cos(pi (k + 3/4) / (m + 1/2)), P_m and P_m' by the three-term
// recurrence; w_k = 2 / ((1 - x_k^2) P_m'(x_k)^2).
void gauss_legendre(int m, std::vector<double>* x, std::vector<double>* w) {
    x->assign(m, 0.0);
    w->assign(m, 0.0);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < (m + 1) / 2; ++k) {
        double t = std::cos(pi * (k + 0.75) / (m + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 1; j < m; ++j) {
                const double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p1 = t; p0 = 1.0; }
            dp = m * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) <= 4e-16 * std::fabs(t) + 1e-300) break;
        }
        // one more evaluation at the converged node for the weight
        double p0 = 1.0, p1 = t;
        for (int j = 1; j < m; ++j) {
            const double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = (m == 1) ? 1.0 : m * (t * p1 - p0) / (t * t - 1.0);
        const double wk = 2.0 / ((1.0 - t * t) * dp * dp);
        (*x)[m - 1 - k] = t;
        (*x)[k] = -t;
        (*w)[m - 1 - k] = wk;
        (*w)[k] = wk;
    }
    if (m % 2 == 1) (*x)[m / 2] = 0.0;
}

void rectangle_split(const rsrr_contour& C, int N, int side_nodes, int* nh, int* nv) {
    const int half = N / 2;
    int h = side_nodes > 0 ? side_nodes : (int)std::lround(half * C.a / (C.a + C.b));
    h = std::min(std::max(h, 1), half - 1);
    *nh = h;
    *nv = half - h;
}

void contour_rule(const rsrr_contour& C, int N, std::vector<zd>* z, std::vector<zd>* w, int side_nodes) {
    z->resize(N);
    if (w) w->resize(N);
    const double pi = 3.14159265358979323846;
    const zd gamma(C.gamma_re, C.gamma_im);
    if (C.shape != RSRR_CONTOUR_RECTANGLE) {
        // trapezoid rule in t on phi(t): (1 / 2 pi i) oint g dz ~ sum_j phi'(t_j) g(z_j) / (i N)
        for (int j = 0; j < N; ++j) {
            const double t = 2.0 * pi * (j + 0.5) / N;
            (*z)[j] = gamma + zd(C.a * std::cos(t), C.b * std::sin(t));
            if (w) (*w)[j] = zd(-C.a * std::sin(t), C.b * std::cos(t)) / (zd(0.0, 1.0) * (double)N);
        }
        return;
    }
    int nh = 0, nv = 0;
    rectangle_split(C, N, side_nodes, &nh, &nv);
    const zd corner[4] = {gamma + zd(-C.a, -C.b), gamma + zd(C.a, -C.b), gamma + zd(C.a, C.b),
                          gamma + zd(-C.a, C.b)};
    int j = 0;
    for (int side = 0; side < 4; ++side) {
        const zd P = corner[side], Q = corner[(side + 1) % 4], half = 0.5 * (Q - P);
        std::vector<double> x, om;
        gauss_legendre(side % 2 == 0 ? nh : nv, &x, &om);
        for (size_t k = 0; k < x.size(); ++k, ++j) {
            (*z)[j] = P + half * (x[k] + 1.0);
            if (w) (*w)[j] = om[k] * half / zd(0.0, 2.0 * pi);
        }
    }
}

bool inside_contour(const rsrr_contour& C, zd z) {
    const zd d = z - zd(C.gamma_re, C.gamma_im);
    if (C.shape == RSRR_CONTOUR_RECTANGLE) return std::fabs(d.real()) < C.a && std::fabs(d.imag()) < C.b;
    const double q = std::pow(d.real() / C.a, 2) + std::pow(d.imag() / C.b, 2);
    return q < 1.0 && std::isfinite(q);
}

// ---- ordering --------------------------------------------------------------------------------
void band_of(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* iperm,
             int64_t* kl, int64_t* ku) {
    int64_t l = 0, u = 0;
    for (int64_t r = 0; r < n; ++r) {
        int64_t rn = iperm ? iperm[r] : r;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            int64_t cn = iperm ? iperm[colind[k]] : colind[k];
            l = std::max(l, rn - cn);
            u = std::max(u, cn - rn);
        }
    }
    *kl = l;
    *ku = u;
}

// Reverse Cuthill-McKee on the symmetrised pattern; each connected component starts from a
// pseudo-peripheral node found by repeated breadth-first searches (George-Liu).
static void rcm(int64_t n, const std::vector<int64_t>& adjp, const std::vector<int32_t>& adj,
                std::vector<int32_t>* order) {
    std::vector<int32_t> deg(n);
    for (int64_t v = 0; v < n; ++v) deg[v] = (int32_t)(adjp[v + 1] - adjp[v]);
    std::vector<char> done(n, 0);
    std::vector<int32_t> level(n, -1);
    order->clear();
    order->reserve(n);
    auto bfs_last_level = [&](int32_t s, int32_t* ecc, std::vector<int32_t>* last) {
        std::vector<int32_t> touched{s};
        level[s] = 0;
        size_t head = 0;
        int32_t maxl = 0;
        while (head < touched.size()) {
            int32_t v = touched[head++];
            for (int64_t k = adjp[v]; k < adjp[v + 1]; ++k) {
                int32_t w = adj[k];
                if (level[w] < 0 && !done[w]) {
                    level[w] = level[v] + 1;
                    maxl = std::max(maxl, level[w]);
                    touched.push_back(w);
                }
            }
        }
        last->clear();
        for (int32_t v : touched)
            if (level[v] == maxl) last->push_back(v);
        for (int32_t v : touched) level[v] = -1;
        *ecc = maxl;
    };
    for (int64_t s0 = 0; s0 < n; ++s0) {
        if (done[s0]) continue;
        int32_t s = (int32_t)s0, ecc = 0;
        std::vector<int32_t> last;
        bfs_last_level(s, &ecc, &last);
        for (int it = 0; it < 8; ++it) {
            int32_t best = last[0];
            for (int32_t v : last)
                if (deg[v] < deg[best]) best = v;
            int32_t ecc2;
            std::vector<int32_t> last2;
            bfs_last_level(best, &ecc2, &last2);
            if (ecc2 <= ecc) break;
            s = best;
            ecc = ecc2;
            last.swap(last2);
        }
        // Cuthill-McKee from s
        size_t head = order->size();
        order->push_back(s);
        done[s] = 1;
        std::vector<int32_t> nb;
        while (head < order->size()) {
            int32_t v = (*order)[head++];
            nb.clear();
            for (int64_t k = adjp[v]; k < adjp[v + 1]; ++k)
                if (!done[adj[k]]) { nb.push_back(adj[k]); done[adj[k]] = 1; }
            std::stable_sort(nb.begin(), nb.end(),
                             [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
            order->insert(order->end(), nb.begin(), nb.end());
        }
    }
    std::reverse(order->begin(), order->end());
}

void choose_ordering(int64_t n, const int64_t* rowptr, const int32_t* colind, bool force_natural,
                     Ordering* out) {
    int64_t kl0, ku0;
    band_of(n, rowptr, colind, nullptr, &kl0, &ku0);
    out->perm.resize(n);
    out->iperm.resize(n);
    std::iota(out->perm.begin(), out->perm.end(), 0);
    std::iota(out->iperm.begin(), out->iperm.end(), 0);
    out->kl = kl0;
    out->ku = ku0;
    out->natural = true;
    if (force_natural || n <= 2) return;
    // symmetrised adjacency without the diagonal
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
            if (colind[k] != r) { cnt[r + 1]++; cnt[colind[k] + 1]++; }
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    std::vector<int32_t> adj(cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
            if (colind[k] != r) { adj[fill[r]++] = colind[k]; adj[fill[colind[k]]++] = (int32_t)r; }
    std::vector<int64_t> adjp(n + 1);
    std::vector<int32_t> adju;
    adju.reserve(adj.size());
    adjp[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        std::sort(adj.begin() + cnt[v], adj.begin() + cnt[v + 1]);
        auto e = std::unique(adj.begin() + cnt[v], adj.begin() + cnt[v + 1]);
        adju.insert(adju.end(), adj.begin() + cnt[v], e);
        adjp[v + 1] = (int64_t)adju.size();
    }
    std::vector<int32_t> order;
    rcm(n, adjp, adju, &order);
    std::vector<int32_t> iperm(n);
    for (int64_t i = 0; i < n; ++i) iperm[order[i]] = (int32_t)i;
    int64_t kl1, ku1;
    band_of(n, rowptr, colind, iperm.data(), &kl1, &ku1);
    if (kl1 + ku1 < kl0 + ku0) {
        out->perm = order;
        out->iperm = iperm;
        out->kl = kl1;
        out->ku = ku1;
        out->natural = false;
    }
}

}  // namespace rsrr
