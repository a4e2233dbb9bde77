// Dense FP64 complex kernels: tiled ZGEMM, bounded grid barrier, one-sided Jacobi.
#include <algorithm>
#include <cstring>
#include <vector>

#include "dense.cuh"

namespace rsrr {

// ---------------------------------------------------------------------------------------------
// ZGEMM: 64 x 64 output tile per CTA, K in steps of 8, 256 threads each owning a 4 x 4 grid of
// outputs spaced 16 apart.  FP64 FMA throughput bounds it on this part; the tiling keeps the
// operands in shared memory so global traffic is (M + N) K / 64 elements per tile.
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int BK = 8;

// Tile BM x BN, NT = BM BN / 16 threads as TY x TX = (BM/4) x (BN/4), each owning a 4 x 4 grid
// of outputs spaced TY rows and TX columns apart.  64 x 64 for general shapes, 32 x 128 when
// M <= 32, 32 x 32 (64 threads) when those give too few CTAs to fill the GPU.  Every output
// accumulates over k in the same order whatever the tile.
template <int OPA, int OPB, int BM, int BN>
__global__ void __launch_bounds__(BM * BN / 16) zgemm_kernel(Zgemm g, int kchunk) {
    constexpr int TY = BM / 4, TX = BN / 4, NT = TY * TX;
    static_assert(BM * BK % NT == 0 && BN * BK % NT == 0, "tile loads");
    __shared__ c128 As[BK][BM + 1];
    __shared__ c128 Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int bm = blockIdx.x * BM, bn = blockIdx.y * BN;
    const int bz = blockIdx.z, b = bz / g.ksplit, ks = bz % g.ksplit;
    const c128* A = g.A + b * g.sA;
    const c128* B = g.B + b * g.sB;
    c128* C = g.C + b * g.sC;
    const int k_begin = ks * kchunk, k_end = min(g.K, k_begin + kchunk);
    c128 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = czero<double>();
    for (int k0 = k_begin; k0 < k_end; k0 += BK) {
#pragma unroll
        for (int r = 0; r < BM * BK / NT; ++r) {
            const int idx = tid + NT * r;
            int i, k;
            if (OPA == OP_N) { i = idx % BM; k = idx / BM; } else { k = idx % BK; i = idx / BK; }
            const int gi = bm + i, gk = k0 + k;
            c128 v = czero<double>();
            if (gi < g.M && gk < k_end) {
                v = (OPA == OP_N) ? A[gi + (int64_t)gk * g.lda] : A[gk + (int64_t)gi * g.lda];
                if (OPA == OP_C) v.im = -v.im;
            }
            As[k][i] = v;
        }
#pragma unroll
        for (int r = 0; r < BN * BK / NT; ++r) {
            const int idx = tid + NT * r;
            int j, k;
            if (OPB == OP_N) { k = idx % BK; j = idx / BK; } else { j = idx % BN; k = idx / BN; }
            const int gj = bn + j, gk = k0 + k;
            c128 w = czero<double>();
            if (gj < g.N && gk < k_end) {
                w = (OPB == OP_N) ? B[gk + (int64_t)gj * g.ldb] : B[gj + (int64_t)gk * g.ldb];
                if (OPB == OP_C) w.im = -w.im;
            }
            Bs[k][j] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            c128 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + TY * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + TX * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], bb[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = bm + ty + TY * i;
        if (gi >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = bn + tx + TX * j;
            if (gj >= g.N) continue;
            c128* c = C + gi + (int64_t)gj * g.ldc;
            const c128 v = g.alpha * acc[i][j];
            if (g.ksplit > 1) {
                atomicAdd(&c->re, v.re);
                atomicAdd(&c->im, v.im);
            } else if (g.beta.re == 0.0 && g.beta.im == 0.0) {
                *c = v;
            } else {
                *c = v + g.beta * (*c);
            }
        }
    }
}

__global__ void scale_kernel(c128* C, int M, int N, int64_t ldc, int64_t sC, c128 beta) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (idx >= (int64_t)M * N) return;
    const int64_t i = idx % M, j = idx / M;
    c128* c = C + b * sC + i + j * ldc;
    *c = (beta.re == 0.0 && beta.im == 0.0) ? czero<double>() : beta * (*c);
}
}  // namespace

template <int BM, int BN>
int zgemm_shape(Zgemm g, cudaStream_t s) {
    const int tm = (int)ceil_div(g.M, BM), tn = (int)ceil_div(g.N, BN);
    if (g.ksplit <= 0) {
        const int64_t tiles = (int64_t)tm * tn * g.batch;
        int ks = 1;
        while (tiles * ks < 2 * 152 && (int64_t)g.K / (ks * 2) >= 256) ks *= 2;
        g.ksplit = ks;
    }
    int kchunk = (int)ceil_div(ceil_div(g.K, g.ksplit), BK) * BK;
    g.ksplit = (int)ceil_div(g.K, kchunk);
    if (g.ksplit > 1) {
        dim3 grid((unsigned)ceil_div((int64_t)g.M * g.N, 256), g.batch);
        { scale_kernel<<<grid, 256, 0, s>>>(g.C, g.M, g.N, g.ldc, g.sC, g.beta); note_launch(); }
    }
    if constexpr (BM * BN > 32 * 32) {
        // too few tiles and no K split: 32 x 32 tiles give up to four times the CTAs
        if (g.ksplit == 1 && (int64_t)tm * tn * g.batch < 2 * 152) return zgemm_shape<32, 32>(g, s);
    }
    dim3 grid(tm, tn, g.batch * g.ksplit);
#define ZG(a, b) { zgemm_kernel<a, b, BM, BN><<<grid, BM * BN / 16, 0, s>>>(g, kchunk); note_launch(); }
    if (g.opA == OP_N && g.opB == OP_N) ZG(OP_N, OP_N)
    else if (g.opA == OP_N && g.opB == OP_T) ZG(OP_N, OP_T)
    else if (g.opA == OP_N && g.opB == OP_C) ZG(OP_N, OP_C)
    else if (g.opA == OP_T && g.opB == OP_N) ZG(OP_T, OP_N)
    else if (g.opA == OP_C && g.opB == OP_N) ZG(OP_C, OP_N)
    else if (g.opA == OP_C && g.opB == OP_C) ZG(OP_C, OP_C)
    else if (g.opA == OP_T && g.opB == OP_T) ZG(OP_T, OP_T)
    else if (g.opA == OP_T && g.opB == OP_C) ZG(OP_T, OP_C)
    else if (g.opA == OP_C && g.opB == OP_T) ZG(OP_C, OP_T)
    else return set_error(RSRR_EINVAL, "zgemm: unsupported op combination");
#undef ZG
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

// ZGEMM accounting for the calling host thread: device time (events around each call) and
// algorithmic flops 8 M N K per product, between zgemm_profile_begin and zgemm_profile_end.
namespace {
struct ZgemmProfile {
    bool on = false;
    double flops = 0.0, flops_tc = 0.0;
    struct Ev { cudaEvent_t a, b; bool tc; };
    std::vector<Ev> ev;
};
thread_local ZgemmProfile g_zprof;
struct JacobiProfile {
    bool on = false;
    double flops = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
thread_local JacobiProfile g_jprof;
double drain_events(std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& ev) {
    double t = 0.0;
    for (auto& e : ev) {
        float x = 0.f;
        cudaEventSynchronize(e.second);
        cudaEventElapsedTime(&x, e.first, e.second);
        t += x;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    ev.clear();
    return t;
}
}  // namespace

void zgemm_profile_begin() {
    g_zprof.on = true;
    g_zprof.flops = g_zprof.flops_tc = 0.0;
    g_zprof.ev.clear();
}

void zgemm_profile_end(double* ms, double* flops, double* ms_tc, double* flops_tc) {
    double t = 0.0, t_tc = 0.0;
    for (auto& e : g_zprof.ev) {
        float x = 0.f;
        cudaEventSynchronize(e.b);
        cudaEventElapsedTime(&x, e.a, e.b);
        t += x;
        if (e.tc) t_tc += x;
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    g_zprof.ev.clear();
    g_zprof.on = false;
    *ms = t;
    *flops = g_zprof.flops;
    if (ms_tc) *ms_tc = t_tc;
    if (flops_tc) *flops_tc = g_zprof.flops_tc;
}

void jacobi_profile_begin() {
    g_jprof.on = true;
    g_jprof.flops = 0.0;
    g_jprof.ev.clear();
}

void jacobi_profile_end(double* ms, double* flops) {
    *ms = drain_events(g_jprof.ev);
    *flops = g_jprof.flops;
    g_jprof.on = false;
}

static int zgemm_dispatch(const Zgemm& g0, cudaStream_t s);

namespace {
thread_local int g_zpath = 0;
}
void zgemm_set_path(int path) { g_zpath = path; }
int zgemm_get_path() { return g_zpath; }

int zgemm(const Zgemm& g0, cudaStream_t s) {
    if (!g_zprof.on || g0.M <= 0 || g0.N <= 0 || g0.K <= 0 || g0.batch <= 0) return zgemm_dispatch(g0, s);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    const int rc = zgemm_dispatch(g0, s);
    cudaEventRecord(b, s);
    const bool tc = g_zpath == 2 || (g_zpath == 0 && !g0.fp64 && zgemm_tc_fits(g0));
    g_zprof.ev.push_back({a, b, tc});
    const double f = 8.0 * g0.M * (double)g0.N * g0.K * g0.batch;
    g_zprof.flops += f;
    if (tc) g_zprof.flops_tc += f;
    return rc;
}

static int zgemm_dispatch(const Zgemm& g0, cudaStream_t s) {
    Zgemm g = g0;
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return RSRR_OK;
    if (g.K <= 0) {
        dim3 grid((unsigned)ceil_div((int64_t)g.M * g.N, 256), g.batch);
        { scale_kernel<<<grid, 256, 0, s>>>(g.C, g.M, g.N, g.ldc, g.sC, g.beta); note_launch(); }
        RSRR_CUDA(cudaGetLastError());
        return RSRR_OK;
    }
    if (g_zpath == 2 || (g_zpath == 0 && !g.fp64 && zgemm_tc_fits(g))) return zgemm_tc(g, s);
    if (g.M <= 32) return zgemm_shape<32, 128>(g, s);
    return zgemm_shape<64, 64>(g, s);
}

// ---------------------------------------------------------------------------------------------
// Norms
// ---------------------------------------------------------------------------------------------
namespace {
__device__ double block_sum(double v) {
    __shared__ double red[32];
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    }
    return r;  // valid in thread 0
}

__global__ void colnorm_kernel(const c128* B, int mb, int64_t ld, double* out) {
    const int c = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < mb; i += blockDim.x) s += cnorm2(B[i + (int64_t)c * ld]);
    s = block_sum(s);
    if (threadIdx.x == 0) out[c] = sqrt(s);
}

__global__ void blocknorm_kernel(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, double* out) {
    const int64_t rows = r1 - r0;
    const int64_t total = rows * (c1 - c0);
    double s = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + idx % rows, j = c0 + idx / rows;
        s += cnorm2(A[i + j * lda]);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}
}  // namespace

void column_norms(const c128* B, int mb, int k, int64_t ld, double* out, cudaStream_t s) {
    if (k > 0) { colnorm_kernel<<<k, 256, 0, s>>>(B, mb, ld, out); note_launch(); }
}

void block_norm2(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, double* out, cudaStream_t s) {
    if (r1 <= r0 || c1 <= c0) return;
    const int64_t total = (int64_t)(r1 - r0) * (c1 - c0);
    const int blocks = (int)std::min<int64_t>(4 * 152, ceil_div(total, 256));
    { blocknorm_kernel<<<blocks, 256, 0, s>>>(A, lda, r0, r1, c0, c1, out); note_launch(); }
}

// ---------------------------------------------------------------------------------------------
// One-sided Jacobi.  A sweep is one cooperative kernel over the round-robin rounds, one CTA per
// column pair, each pair ordered after the two pairs of the previous round that held its columns.
// A pair is rotated when its inner product is above tol relative to the column norms and both
// columns are above an absolute floor: columns below the floor are rounding noise, and rotating
// them against anything changes no column above the floor by more than the floor itself.
//
// The squared column norms live in a small array: computed once at the start of the sweep and
// recomputed from the rotated entries by the CTA that rotates a pair, so they are always the sums
// a fresh pass over the stored columns would give.  A pair then costs one complex inner product
// (4 FP64 fused multiply-adds a row) when it is not rotated, nothing when a column is below the
// floor, and the columns it rotates are held in registers between the two passes.
// ---------------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ int rr_pos(int k, int r, int n) {  // player at seat k in round r
    return k == 0 ? 0 : ((k - 1 + r) % (n - 1)) + 1;
}

struct JacobiArgs {
    c128* B;
    int mb, kk, npad;
    c128* J;
    double tol, floor2, abs_g;
    double* nrm2;  // squared column norms of B (kk entries)
    int* ver;      // rounds each column has finished in this sweep (kk entries, zero at launch)
    int* jver;     // rounds whose rotation of J's column is done (kk entries, zero at launch)
    unsigned long long* max_off;
    int* rotations;  // [0] pairs rotated, [1] pairs whose inner product was formed
    GridBar gb;      // the barrier after the norms; its error word also records a wait that gave up
};

// Two block-wide sums; every thread gets both, summed in the same order (two CTA barriers).  The
// per-warp partials are combined by a shuffle tree in every warp (log2 of the warp count FP64
// additions a thread), not by a loop over them: FP64 issue slots are the scarce resource here.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double red2_[2][32];
    for (int off = 16; off; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red2_[0][w] = a; red2_[1][w] = b; }
    __syncthreads();
    double s0 = lane < nw ? red2_[0][lane] : 0.0, s1 = lane < nw ? red2_[1][lane] : 0.0;
    for (int off = nw >> 1; off; off >>= 1) {  // nw is a power of two
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    a = __shfl_sync(0xffffffffu, s0, 0);
    b = __shfl_sync(0xffffffffu, s1, 0);
}

constexpr int kJacThreads = 256;
// Columns are read past L1: between rounds they are rewritten by CTAs on other SMs.
__device__ __forceinline__ c128 ldcg_c(const c128* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk<double>(v.x, v.y);
}
constexpr int kJacCache = 3;  // rows per thread kept in registers (columns up to 768 rows)

__device__ __forceinline__ void jac_norm_acc(double& acc, c128 x) { acc = fma(x.re, x.re, fma(x.im, x.im, acc)); }
// conj(x) y accumulated into (gr, gi)
__device__ __forceinline__ void jac_dot_acc(double& gr, double& gi, c128 x, c128 y) {
    gr = fma(x.re, y.re, fma(x.im, y.im, gr));
    gi = fma(x.re, y.im, fma(-x.im, y.re, gi));
}
// (x, y) <- (c x - sp y, s x + cp y): the rotation with the phase folded into the two complex
// coefficients (12 FP64 operations a row)
__device__ __forceinline__ void jac_rotate(c128& x, c128& y, double c, double s, c128 sp, c128 cp) {
    const c128 nx = mk<double>(fma(-sp.re, y.re, fma(sp.im, y.im, c * x.re)),
                               fma(-sp.re, y.im, fma(-sp.im, y.re, c * x.im)));
    const c128 ny = mk<double>(fma(cp.re, y.re, fma(-cp.im, y.im, s * x.re)),
                               fma(cp.re, y.im, fma(cp.im, y.re, s * x.im)));
    x = nx;
    y = ny;
}

// One column pair (p, q) of a round, p < q < kk; every thread of the CTA takes the same branches.
// Rotates the pair's columns of B and stores their norms; returns whether it rotated, with the
// rotation in (c, s, sp, cp) for J's columns, which the caller rotates after releasing B's.
// The rotation of the CTA's current pair (c, s, s e^{-i phi}, c e^{-i phi}): written by thread 0,
// read by every thread for B's columns and, after B's release, for J's.
__shared__ double jac_spar[6];

__device__ __forceinline__ bool jac_pair(const JacobiArgs& a, int p, int q) {
    const int tid = threadIdx.x;
    const double al = __ldcg(a.nrm2 + p), be = __ldcg(a.nrm2 + q);
    if (fmin(al, be) <= a.floor2) return false;
    c128* bp = a.B + (int64_t)p * a.mb;
    c128* bq = a.B + (int64_t)q * a.mb;
    c128 xc[kJacCache], yc[kJacCache];
    double gr = 0.0, gi = 0.0;
#pragma unroll
    for (int u = 0; u < kJacCache; ++u) {
        const int r = tid + kJacThreads * u;
        xc[u] = yc[u] = czero<double>();
        if (r < a.mb) {
            xc[u] = ldcg_c(bp + r);
            yc[u] = ldcg_c(bq + r);
            jac_dot_acc(gr, gi, xc[u], yc[u]);
        }
    }
    for (int r = tid + kJacThreads * kJacCache; r < a.mb; r += kJacThreads)
        jac_dot_acc(gr, gi, ldcg_c(bp + r), ldcg_c(bq + r));
    block_sum2(gr, gi);
    // the decision and the rotation are computed once, by thread 0, and shared
    __shared__ int s_act;
    if (tid == 0) {
        atomicAdd(a.rotations + 1, 1);
        int act = 0;
        const double g = sqrt(gr * gr + gi * gi);
        if (g > a.abs_g) {
            const double off = g / sqrt(al * be);
            atomicMax(a.max_off, (unsigned long long)__double_as_longlong(off));
            if (off > a.tol) {
                const double ig = 1.0 / g;
                const c128 ph = mk<double>(gr * ig, -gi * ig);  // e^{-i phi}, phi = arg(conj(b_p) b_q)
                const double zeta = (be - al) * (0.5 * ig);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                jac_spar[0] = c;
                jac_spar[1] = sn;
                jac_spar[2] = ph.re * sn;
                jac_spar[3] = ph.im * sn;
                jac_spar[4] = ph.re * c;
                jac_spar[5] = ph.im * c;
                act = 1;
            }
        }
        s_act = act;
    }
    __syncthreads();
    if (!s_act) return false;
    // (b_p, b_q) <- (c b_p - s e^{-i phi} b_q, s b_p + c e^{-i phi} b_q)
    const double c = jac_spar[0], s = jac_spar[1];
    const c128 sp = mk<double>(jac_spar[2], jac_spar[3]), cp = mk<double>(jac_spar[4], jac_spar[5]);
    double an = 0.0, bn = 0.0;
#pragma unroll
    for (int u = 0; u < kJacCache; ++u) {
        const int r = tid + kJacThreads * u;
        if (r < a.mb) {
            jac_rotate(xc[u], yc[u], c, s, sp, cp);
            bp[r] = xc[u];
            bq[r] = yc[u];
            jac_norm_acc(an, xc[u]);
            jac_norm_acc(bn, yc[u]);
        }
    }
    for (int r = tid + kJacThreads * kJacCache; r < a.mb; r += kJacThreads) {
        c128 x = ldcg_c(bp + r), y = ldcg_c(bq + r);
        jac_rotate(x, y, c, s, sp, cp);
        bp[r] = x;
        bq[r] = y;
        jac_norm_acc(an, x);
        jac_norm_acc(bn, y);
    }
    block_sum2(an, bn);
    if (tid == 0) {
        a.nrm2[p] = an;
        a.nrm2[q] = bn;
        atomicAdd(a.rotations, 1);
    }
    return true;
}

// Thread 0 waits until column c has finished `target` rounds.  Bounded: after the spin limit, or
// once another CTA has reported a timeout, it records the failure and returns false.
__device__ __forceinline__ bool jac_wait(const int* ver, int c, int target, int* err) {
    const volatile int* v = ver + c;
    long long spins = 0;
    unsigned backoff = 16;
    while (*v < target) {
        if (++spins > (1LL << 24) || *(volatile int*)err != 0) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(backoff);
        if (backoff < 256) backoff <<= 1;
    }
    return true;
}

__global__ void __launch_bounds__(kJacThreads, 3) jacobi_sweep_kernel(JacobiArgs a) {
    // One CTA per column pair (CTAs take the pairs in order, see below), so every round spreads its
    // FP64 work over all SMs.  The rounds are not separated by grid barriers: a pair of round r
    // starts as soon as both of its columns have come out of round r - 1 (a per-column count of
    // finished rounds), so a slow pair holds up only the pairs that need its columns.  The pairs,
    // their order and every value are those of the barrier-separated sweep.
    const int tid = threadIdx.x;
    __shared__ int s_ok;
    for (int c = blockIdx.x; c < a.kk; c += gridDim.x) {
        const c128* bc = a.B + (int64_t)c * a.mb;
        double s = 0.0, unused = 0.0;
        for (int r = tid; r < a.mb; r += kJacThreads) jac_norm_acc(s, ldcg_c(bc + r));
        block_sum2(s, unused);
        if (tid == 0) a.nrm2[c] = s;
    }
    if (!grid_sync(a.gb)) return;
    // The pairs of all rounds are numbered g = round * (npad / 2) + i and dealt out in that order.
    // A pair releases its columns of B (and their norms) to the next round as soon as they are
    // rotated; it then rotates its columns of J, once the previous round's rotation of them is done
    // (jver), and releases those.  With more CTAs than pairs in a round, CTAs start pairs of the next
    // round while J's rotations of this one run.  Every wait is on a smaller g (or the same g's B
    // part), every CTA takes its pairs in increasing g and all are resident (cooperative launch), so
    // the smallest unfinished step can always proceed.  The arithmetic is that of the sweep with a
    // grid barrier between rounds.
    const int ppr = a.npad / 2;
    const int64_t npairs = (int64_t)(a.npad - 1) * ppr;
    for (int64_t gi = blockIdx.x; gi < npairs; gi += gridDim.x) {
        const int round = (int)(gi / ppr), i = (int)(gi % ppr);
        int p = rr_pos(i, round, a.npad), q = rr_pos(a.npad - 1 - i, round, a.npad);
        if (p > q) { const int t = p; p = q; q = t; }
        const bool real_pair = q < a.kk;  // q == kk is the padding column of an odd count
        if (tid == 0) {
            const bool ok = jac_wait(a.ver, p, round, a.gb.err) && (!real_pair || jac_wait(a.ver, q, round, a.gb.err));
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        const bool rot = real_pair && jac_pair(a, p, q);
        __syncthreads();  // every store of B and of the norms issued
        if (tid == 0) {
            __threadfence();
            atomicExch(a.ver + p, round + 1);
            if (real_pair) atomicExch(a.ver + q, round + 1);
        }
        if (a.J) {
            if (tid == 0) {
                const bool ok = jac_wait(a.jver, p, round, a.gb.err) &&
                                (!real_pair || jac_wait(a.jver, q, round, a.gb.err));
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            if (rot) {
                const double c = jac_spar[0], sn = jac_spar[1];
                const c128 sp = mk<double>(jac_spar[2], jac_spar[3]), cp = mk<double>(jac_spar[4], jac_spar[5]);
                c128* jp = a.J + (int64_t)p * a.kk;
                c128* jq = a.J + (int64_t)q * a.kk;
                for (int r = tid; r < a.kk; r += kJacThreads) {
                    c128 x = ldcg_c(jp + r), y = ldcg_c(jq + r);
                    jac_rotate(x, y, c, sn, sp, cp);
                    jp[r] = x;
                    jq[r] = y;
                }
            }
            __syncthreads();  // every store of J issued
            if (tid == 0) {
                __threadfence();
                atomicExch(a.jver + p, round + 1);
                if (real_pair) atomicExch(a.jver + q, round + 1);
            }
        }
    }
}
}  // namespace

namespace {
// out[:, i] = in[:, perm[i]] for the k columns of an m-row matrix (leading dimension m).
__global__ void gather_cols_kernel(const c128* __restrict__ in, int m, int k, const int* __restrict__ perm,
                                   c128* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * k) return;
    const int64_t r = idx % m, c = idx / m;
    out[idx] = in[r + (int64_t)perm[c] * m];
}
}  // namespace

int jacobi_orthogonalize(c128* B, int mb, int k, c128* J, cudaStream_t s, int max_sweeps, int* sweeps_out,
                         double abs_floor, double conv, double abs_inner) {
    if (sweeps_out) *sweeps_out = 0;
    if (k < 2) return RSRR_OK;
    const int npad = k + (k & 1);
    int dev = 0, nsm = 0, occ = 0;
    RSRR_CUDA(cudaGetDevice(&dev));
    RSRR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RSRR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_sweep_kernel, kJacThreads, 0));
    if (occ < 1) return set_error(RSRR_ECUDA, "jacobi kernel cannot be resident");
    // as many CTAs as are resident (up to 4 per SM), also when that is more than a round's npad / 2
    // pairs: the surplus starts the next round's pairs while this round's J rotations finish
    const int G = (int)std::min<int64_t>((int64_t)nsm * std::min(occ, 4), (int64_t)(npad - 1) * (npad / 2));
    unsigned long long* dmax = nullptr;
    int* drot = nullptr;
    unsigned* bar = nullptr;
    double* dn2 = nullptr;
    int* dver = nullptr;
    int* djver = nullptr;
    double* dnrm = nullptr;
    int* dperm = nullptr;
    c128* tmp = nullptr;
    auto cleanup = [&]() {
        dfree(dn2, s);
        dfree(dver, s);
        dfree(djver, s);
        dfree(dmax, s);
        dfree(drot, s);
        dfree(bar, s);
        dfree(dnrm, s);
        dfree(dperm, s);
        dfree(tmp, s);
    };
    int rc = RSRR_OK;
#define JTRY(expr) do { rc = (expr); if (rc != RSRR_OK) { cleanup(); return rc; } } while (0)
    JTRY(dalloc_n(&dn2, (size_t)k, s));
    JTRY(dalloc_n(&dver, (size_t)k, s));
    JTRY(dalloc_n(&djver, (size_t)k, s));
    JTRY(dalloc_n(&dmax, 1, s));
    JTRY(dalloc_n(&drot, 2, s));
    JTRY(dalloc_n(&bar, kGridBarWords, s));
    // Before each sweep the columns (and J's with them) are put in order of decreasing norm: the
    // round-robin pairs then meet in an order that converges in fewer sweeps, and the caller,
    // which sorts the final column norms itself, sees no difference.
    JTRY(dalloc_n(&dnrm, (size_t)k, s));
    JTRY(dalloc_n(&dperm, (size_t)k, s));
    JTRY(dalloc_n(&tmp, (size_t)mb * k + (J ? (size_t)k * k : 0), s));
    if (cudaMemsetAsync(bar, 0, kGridBarWords * sizeof(unsigned), s) != cudaSuccess)
        JTRY(set_error(RSRR_ECUDA, "jacobi: clearing the grid barrier"));
#undef JTRY
    JacobiArgs ja{B, mb, k, npad, J, sqrt((double)mb) * 1.1102230246251565e-16, abs_floor * abs_floor, abs_inner,
                  dn2, dver, djver, dmax, drot, grid_bar_at(bar)};
    std::vector<double> hn(k);
    std::vector<int> order(k);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        column_norms(B, mb, k, mb, dnrm, s);
        if (cudaMemcpyAsync(hn.data(), dnrm, (size_t)k * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(RSRR_ECUDA, "jacobi norms"); break; }
        for (int i = 0; i < k; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hn[a] > hn[b]; });
        bool sorted = true;
        for (int i = 0; i < k && sorted; ++i) sorted = order[i] == i;
        if (!sorted) {
            if (cudaMemcpyAsync(dperm, order.data(), (size_t)k * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
                rc = set_error(RSRR_ECUDA, "jacobi: column order upload");
                break;
            }
            { gather_cols_kernel<<<(unsigned)ceil_div((int64_t)mb * k, 256), 256, 0, s>>>(B, mb, k, dperm, tmp); note_launch(); }
            cudaError_t ce = cudaMemcpyAsync(B, tmp, (size_t)mb * k * sizeof(c128), cudaMemcpyDeviceToDevice, s);
            if (J && ce == cudaSuccess) {
                c128* tj = tmp + (size_t)mb * k;
                { gather_cols_kernel<<<(unsigned)ceil_div((int64_t)k * k, 256), 256, 0, s>>>(J, k, k, dperm, tj); note_launch(); }
                ce = cudaMemcpyAsync(J, tj, (size_t)k * k * sizeof(c128), cudaMemcpyDeviceToDevice, s);
            }
            if (ce != cudaSuccess) { rc = set_error(RSRR_ECUDA, "jacobi: column reorder"); break; }
        }
        if (cudaMemsetAsync(dmax, 0, 8, s) != cudaSuccess || cudaMemsetAsync(drot, 0, 8, s) != cudaSuccess ||
            cudaMemsetAsync(dver, 0, (size_t)k * sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(djver, 0, (size_t)k * sizeof(int), s) != cudaSuccess) {
            rc = set_error(RSRR_ECUDA, "jacobi: clearing the sweep counters");
            break;
        }
        void* args[] = {&ja};
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (g_jprof.on) {
            cudaEventCreate(&ea);
            cudaEventCreate(&eb);
            cudaEventRecord(ea, s);
        }
        cudaError_t e = cudaLaunchCooperativeKernel((void*)jacobi_sweep_kernel, G, kJacThreads, args, 0, s);
        note_launch();
        if (g_jprof.on) {
            cudaEventRecord(eb, s);
            g_jprof.ev.emplace_back(ea, eb);
        }
        if (e != cudaSuccess) { rc = set_error(RSRR_ECUDA, cudaGetErrorString(e)); break; }
        int hrot[2] = {0, 0}, herr = 0;
        unsigned long long hmax = 0;
        if (cudaMemcpyAsync(hrot, drot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&herr, bar + kGridBarErrWord, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&hmax, dmax, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(RSRR_ECUDA, "jacobi sync"); break; }
        if (herr) { rc = set_error(RSRR_ETIMEOUT, "a wait in the Jacobi sweep gave up"); break; }
        // the sweep's work: the column norms (4 real flops a row), one complex inner product for
        // every pair formed (8 a row), and for every rotated pair the rotation of both columns of
        // B and J (24 a row each) and the two new norms (8 a row)
        if (g_jprof.on)
            g_jprof.flops += 4.0 * mb * k + 8.0 * mb * hrot[1] + hrot[0] * (32.0 * mb + (J ? 24.0 * k : 0.0));
        double off;
        std::memcpy(&off, &hmax, 8);
        // converged: no rotation left, or every pair above the floor orthogonal to `conv` (the
        // remaining effect on the singular values is of second order in that number)
        if (hrot[0] == 0 || off <= conv) { ++sweep; break; }
    }
    cleanup();
    if (sweeps_out) *sweeps_out = sweep;
    return rc;
}

}  // namespace rsrr
