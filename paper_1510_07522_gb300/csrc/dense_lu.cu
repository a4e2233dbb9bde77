// Dense complex LU with partial pivoting, one CTA per sampling point, and its block solves.
//
// Factorisation of one point (right-looking, panels of NB = 64 columns):
//   1. panel: the m x 64 panel is factored as two 32-column leaves (left leaf, its
//      interchanges and L11^{-1} applied to the right half, rank-32 update of the right half,
//      right leaf, its interchanges applied back to the left half).  A leaf is column-by-
//      column getf2 (pivot by cabs1 = |re| + |im|, lowest row on ties).  Panels of at most
//      ~380 (complex64) / ~190 (complex128) rows are staged in shared memory, taller ones are
//      factored in place in global memory.
//   2. the panel's 64 interchanges are composed into one permutation of the <= 128 rows they
//      touch; inv(L11) and inv(U11) of the diagonal block are formed once.
//   3. trailing rows: per block of columns, the touched rows are gathered, permuted, and the
//      64 pivot rows become U12 = inv(L11) * (permuted rows)  (one small product).
//   4. trailing update A22 -= L21 * U12: 128 x 128 (complex64) or 64 x 64 (complex128) tiles,
//      L21 tiles double-buffered in shared memory by cp.async, U12 block resident, each
//      thread holding an 8 x 8 (4 x 4) block of the tile in registers.
// The update is the dense contraction that carries (8/3) n^3 real flops per point; steps 1-3
// are O(n^2 NB).
#include <algorithm>
#include <climits>
#include <string>

#include <cuda_bf16.h>

#include "dense_lu.cuh"
#include "tc.cuh"

namespace rsrr {

namespace {
using namespace tc;

constexpr int NB = kDenseNB;
constexpr int NBP = NB + 1;  // padded row length of the diagonal-block arrays in shared memory
constexpr int NT = kDenseThreads;
constexpr int NW = NT / 32;
constexpr unsigned FULL = 0xffffffffu;

// Barrier of the NT worker threads (warps 0..7).  The complex64 factor kernel adds a ninth warp
// that feeds the tensor cores and never takes part in the workers' barriers.
__device__ __forceinline__ void wsync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

template <typename R> struct DTile;
template <> struct DTile<float> { static constexpr int TM = 128, TN = 128; };  // trailing rows only
template <> struct DTile<double> { static constexpr int TM = 64, TN = 64, MI = 4, MJ = 4; };

template <typename R>
constexpr size_t gemm_smem() {
    return (2 * (size_t)NB * DTile<R>::TM + (size_t)NB * (DTile<R>::TN + 1)) * sizeof(cplx<R>);
}
template <typename R>
constexpr size_t rows_smem() {
    return ((size_t)NB * NBP + (size_t)2 * NB * DTile<R>::TN) * sizeof(cplx<R>);
}
template <typename R>
constexpr size_t inverse_smem() {
    return (size_t)3 * NB * NBP * sizeof(cplx<R>);
}
// Tensor-core trailing update (complex64): an L21 tile of 128 rows and a U12 block of 128
// columns, each as six BF16 arrays (re hi, mid, lo; im hi, mid, lo) with K = 64 (one 128-byte
// row) in the swizzled K-major layout the MMA reads; +1024 B to align the operand base.
constexpr uint32_t TC_ROWS = 128, TC_COLS = 128;
constexpr uint32_t TC_SPLIT = 3;                                     // bf16 pieces per FP32 value
constexpr uint32_t TC_ARR = 2 * TC_SPLIT;                           // arrays per operand
constexpr uint32_t TC_A_BYTES = TC_ARR * TC_ROWS * NB * 2;          // 96 KB
constexpr uint32_t TC_B_BYTES = TC_ARR * TC_COLS * NB * 2;          // 96 KB
constexpr uint32_t TC_A_FLOATS = TC_A_BYTES / 4, TC_B_FLOATS = TC_B_BYTES / 4;  // image sizes in 4-byte words
constexpr uint32_t TC_TMEM_COLS = 512;               // two accumulator buffers of (128 re + 128 im) columns
constexpr size_t tc_smem() { return (size_t)TC_A_BYTES + TC_B_BYTES + 1024; }

template <typename R>
constexpr size_t factor_smem() {
    return std::max(sizeof(R) == 4 ? tc_smem() : gemm_smem<R>(), std::max(rows_smem<R>(), inverse_smem<R>()));
}

struct DShared {
    double2 u12[32 * 32];  // U12 of the panel's left leaf (32 x 32, complex64 or complex128)
    int piv[NB];        // panel pivots, relative to the panel's first row
    int rows[2 * NB];   // composed interchanges: row rows[e] receives row src[e]
    int src[2 * NB];
    int cnt;
    int res;
    int info;
    int job;
    int red_i[NW];
    double red_v[NW];
};

template <typename R>
__device__ __forceinline__ cplx<R>* sh_u12(DShared& sh) { return reinterpret_cast<cplx<R>*>(sh.u12); }

// ------------------------------------------------------------------------------------------
// cp.async element copies (src_bytes = 0 fills zeros; the source must still be a valid address)
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void cp_elem(cplx<R>* smem, const cplx<R>* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(cplx<R>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Row of the largest cabs1 in col[c..m) (lowest row on ties; c if every entry is NaN).
template <typename R>
__device__ int col_argmax(const cplx<R>* col, int c, int m, DShared& sh) {
    double best = -1.0;
    int bi = INT_MAX;
    for (int r = c + (int)threadIdx.x; r < m; r += NT) {
        const double a = (double)cabs1(col[r]);
        if (a > best) { best = a; bi = r; }
    }
    for (int off = 16; off; off >>= 1) {
        const double ob = __shfl_down_sync(FULL, best, off);
        const int oi = __shfl_down_sync(FULL, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh.red_v[w] = best; sh.red_i[w] = bi; }
    wsync();
    if (w == 0) {
        best = lane < NW ? sh.red_v[lane] : -1.0;
        bi = lane < NW ? sh.red_i[lane] : INT_MAX;
        for (int off = 16; off; off >>= 1) {
            const double ob = __shfl_down_sync(FULL, best, off);
            const int oi = __shfl_down_sync(FULL, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) sh.res = (bi == INT_MAX) ? c : bi;
    }
    wsync();
    return sh.res;
}

// getf2 on the m x w block P (leading dimension ld): pivots piv[c] relative to row 0.
template <typename R>
__device__ void leaf_factor(cplx<R>* P, int64_t ld, int m, int w, int* piv, int col_base, DShared& sh) {
    for (int c = 0; c < w; ++c) {
        cplx<R>* colc = P + (int64_t)c * ld;
        const int p = col_argmax(colc, c, m, sh);
        if (threadIdx.x == 0) piv[c] = p;
        if (p != c)
            for (int q = threadIdx.x; q < w; q += NT) {
                cplx<R>* cq = P + (int64_t)q * ld;
                const cplx<R> t = cq[c];
                cq[c] = cq[p];
                cq[p] = t;
            }
        wsync();
        const cplx<R> pv = colc[c];
        const bool zero = cis_zero(pv);
        if (zero && threadIdx.x == 0 && sh.info == 0) sh.info = col_base + c + 1;
        const cplx<R> rp = zero ? czero<R>() : crecip(pv);
        // U row c of the leaf in shared memory (read by every thread); each row's entries are
        // loaded in chunks before any is stored, so a tall leaf in global memory pays the memory
        // latency once per chunk instead of once per column.
        cplx<R>* urow = sh_u12<R>(sh);
        if ((int)threadIdx.x < w) urow[threadIdx.x] = P[c + (int64_t)threadIdx.x * ld];
        wsync();
        constexpr int QL = sizeof(R) == 4 ? 16 : 8;
        for (int r = c + 1 + (int)threadIdx.x; r < m; r += NT) {
            cplx<R> l = colc[r];
            if (!zero) {
                l = l * rp;
                colc[r] = l;
            }
            for (int q0 = c + 1; q0 < w; q0 += QL) {
                cplx<R> x[QL];
#pragma unroll
                for (int j = 0; j < QL; ++j)
                    x[j] = (q0 + j < w) ? P[r + (int64_t)(q0 + j) * ld] : czero<R>();
#pragma unroll
                for (int j = 0; j < QL; ++j)
                    if (q0 + j < w) {
                        cfms(x[j], l, urow[q0 + j]);
                        P[r + (int64_t)(q0 + j) * ld] = x[j];
                    }
            }
        }
        wsync();
    }
}

// Factor the m x nbk panel P as two leaves of 32 columns; sh.piv[0..nbk) relative to row 0,
// with every interchange applied to all nbk columns.
template <typename R>
__device__ void panel_factor(cplx<R>* P, int64_t ld, int m, int nbk, int col_base, DShared& sh) {
    const int w1 = min(32, nbk);
    leaf_factor(P, ld, m, w1, sh.piv, col_base, sh);
    if (nbk <= w1) return;
    const int w2 = nbk - w1;  // w1 == 32 from here on
    cplx<R>* Rt = P + (int64_t)w1 * ld;
    for (int q = threadIdx.x; q < w2; q += NT) {  // left interchanges on the right half
        cplx<R>* cq = Rt + (int64_t)q * ld;
        for (int c = 0; c < w1; ++c) {
            const int p = sh.piv[c];
            if (p != c) {
                const cplx<R> t = cq[c];
                cq[c] = cq[p];
                cq[p] = t;
            }
        }
    }
    wsync();
    for (int q = threadIdx.x; q < w2; q += NT) {  // U12 = L11^{-1} (top 32 rows of the right half)
        cplx<R>* cq = Rt + (int64_t)q * ld;
        for (int r = 1; r < w1; ++r) {
            cplx<R> acc = cq[r];
            for (int s = 0; s < r; ++s) cfms(acc, P[r + (int64_t)s * ld], cq[s]);
            cq[r] = acc;
        }
    }
    wsync();
    // A22 -= L21 U12 (K = 32): U12 (32 x w2) is staged in shared memory (the caller's buffer
    // past the panel when the panel itself is staged there); each row loads its L21 part and a
    // chunk of its A22 part before storing anything.
    cplx<R>* u12 = sh_u12<R>(sh);
    for (int idx = threadIdx.x; idx < 32 * w2; idx += NT) {
        const int s = idx % 32, q = idx / 32;
        u12[q * 32 + s] = Rt[s + (int64_t)q * ld];
    }
    wsync();
    constexpr int QC = sizeof(R) == 4 ? 16 : 8;  // A22 columns per chunk
    for (int r = w1 + (int)threadIdx.x; r < m; r += NT) {
        cplx<R> lrow[32];
#pragma unroll
        for (int s = 0; s < 32; ++s) lrow[s] = P[r + (int64_t)s * ld];
        for (int q0 = 0; q0 < w2; q0 += QC) {
            cplx<R> x[QC];
#pragma unroll
            for (int j = 0; j < QC; ++j)
                x[j] = (q0 + j < w2) ? Rt[r + (int64_t)(q0 + j) * ld] : czero<R>();
#pragma unroll
            for (int j = 0; j < QC; ++j) {
                if (q0 + j < w2) {
                    const cplx<R>* uq = u12 + (q0 + j) * 32;
#pragma unroll
                    for (int s = 0; s < 32; ++s) cfms(x[j], lrow[s], uq[s]);
                    Rt[r + (int64_t)(q0 + j) * ld] = x[j];
                }
            }
        }
    }
    wsync();
    leaf_factor(Rt + w1, ld, m - w1, w2, sh.piv + w1, col_base + w1, sh);
    if ((int)threadIdx.x < w2) sh.piv[w1 + threadIdx.x] += w1;
    wsync();
    for (int q = threadIdx.x; q < w1; q += NT) {  // right interchanges on the left half
        cplx<R>* cq = P + (int64_t)q * ld;
        for (int c = w1; c < nbk; ++c) {
            const int p = sh.piv[c];
            if (p != c) {
                const cplx<R> t = cq[c];
                cq[c] = cq[p];
                cq[p] = t;
            }
        }
    }
    wsync();
}

// Compose the panel's interchanges (applied in order t = 0..nbk-1) into one permutation of the
// rows they touch.  Entries 0..nbk-1 are the diagonal rows; further entries are pivot rows
// below the panel's diagonal block.  Warp 0 does it; everyone waits.
__device__ void compose_swaps(int nbk, DShared& sh) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int t = lane; t < nbk; t += 32) { sh.rows[t] = t; sh.src[t] = t; }
        __syncwarp();
        int cnt = nbk;
        for (int t = 0; t < nbk; ++t) {
            const int p = sh.piv[t];
            if (p == t) continue;
            int e = -1;
            if (p < nbk) {
                e = p;
            } else {
                for (int base = nbk; base < cnt && e < 0; base += 32) {
                    const int idx = base + lane;
                    const unsigned hit = __ballot_sync(FULL, idx < cnt && sh.rows[idx] == p);
                    if (hit) e = base + __ffs(hit) - 1;
                }
                if (e < 0) {
                    e = cnt;
                    if (lane == 0) { sh.rows[e] = p; sh.src[e] = p; }
                    ++cnt;
                }
            }
            __syncwarp();
            if (lane == 0) {
                const int a = sh.src[t];
                sh.src[t] = sh.src[e];
                sh.src[e] = a;
            }
            __syncwarp();
        }
        if (lane == 0) sh.cnt = cnt;
    }
    wsync();
}

// inv(L11) and inv(U11) of the nbk x nbk diagonal block of P; shared layout (r, c) at r * NBP + c:
// sm[0 ..) = inv(L11), then inv(U11), then a copy of the block (its padding column holds 1/U(r,r)).
// Both go to ginv (column-major, leading dimension NB, zero outside nbk x nbk).
template <typename R>
__device__ void diag_inverses(const cplx<R>* P, int64_t ld, int nbk, cplx<R>* sm, cplx<R>* ginv) {
    cplx<R>* iL = sm;
    cplx<R>* iU = sm + NB * NBP;
    cplx<R>* T = sm + 2 * NB * NBP;
    const cplx<R> one = mk<R>(R(1), R(0));
    for (int idx = threadIdx.x; idx < nbk * nbk; idx += NT) {
        const int r = idx % nbk, c = idx / nbk;
        T[r * NBP + c] = P[r + (int64_t)c * ld];
    }
    wsync();
    for (int r = threadIdx.x; r < nbk; r += NT) {
        const cplx<R> d = T[r * NBP + r];
        T[r * NBP + NB] = cis_zero(d) ? czero<R>() : crecip(d);
    }
    wsync();
    const int t = threadIdx.x;
    if (t < nbk) {
        for (int r = 0; r < nbk; ++r) {
            iL[r * NBP + t] = (r == t) ? one : czero<R>();
            iU[r * NBP + t] = czero<R>();
        }
        for (int r = t + 1; r < nbk; ++r) {  // column t of inv(L11): unit lower forward substitution
            cplx<R> a0 = czero<R>(), a1 = czero<R>();
            int s = t;
            for (; s + 1 < r; s += 2) {
                cfms(a0, T[r * NBP + s], iL[s * NBP + t]);
                cfms(a1, T[r * NBP + s + 1], iL[(s + 1) * NBP + t]);
            }
            if (s < r) cfms(a0, T[r * NBP + s], iL[s * NBP + t]);
            iL[r * NBP + t] = a0 + a1;
        }
        iU[t * NBP + t] = T[t * NBP + NB];
        for (int r = t - 1; r >= 0; --r) {  // column t of inv(U11): backward substitution
            cplx<R> a0 = czero<R>(), a1 = czero<R>();
            int s = r + 1;
            for (; s + 1 <= t; s += 2) {
                cfma(a0, T[r * NBP + s], iU[s * NBP + t]);
                cfma(a1, T[r * NBP + s + 1], iU[(s + 1) * NBP + t]);
            }
            if (s <= t) cfma(a0, T[r * NBP + s], iU[s * NBP + t]);
            const cplx<R> acc = a0 + a1;
            iU[r * NBP + t] = mk<R>(-acc.re, -acc.im) * T[r * NBP + NB];
        }
    }
    wsync();
    for (int idx = threadIdx.x; idx < NB * NB; idx += NT) {
        const int r = idx % NB, c = idx / NB;
        const bool in = r < nbk && c < nbk;
        ginv[idx] = in ? iL[r * NBP + c] : czero<R>();
        ginv[NB * NB + idx] = in ? iU[r * NBP + c] : czero<R>();
    }
    wsync();
}

// Trailing columns, rows of the panel: apply the composed interchanges and form
// U12 = inv(L11) * (pivot rows), block of TN columns at a time.  sm[0..NB*NBP) = inv(L11).
template <typename R>
__device__ void trailing_rows(cplx<R>* A, int64_t lda, int n, int k0, cplx<R>* sm, const DShared& sh) {
    constexpr int TN = DTile<R>::TN;
    const cplx<R>* iL = sm;
    cplx<R>* g = sm + NB * NBP;  // gathered rows, g[col * 2NB + e]
    const int cnt = sh.cnt, extra = cnt - NB;
    for (int c0 = k0 + NB; c0 < n; c0 += TN) {
        const int nc = min(TN, n - c0);
        for (int idx = threadIdx.x; idx < cnt * nc; idx += NT) {
            const int e = idx % cnt, col = idx / cnt;
            g[col * 2 * NB + e] = A[(int64_t)(k0 + sh.src[e]) + (int64_t)(c0 + col) * lda];
        }
        wsync();
        for (int idx = threadIdx.x; idx < extra * nc; idx += NT) {
            const int e = NB + idx % extra, col = idx / extra;
            A[(int64_t)(k0 + sh.rows[e]) + (int64_t)(c0 + col) * lda] = g[col * 2 * NB + e];
        }
        {
            const int t = threadIdx.x % NB, grp = threadIdx.x / NB;
            for (int col = grp; col < nc; col += NT / NB) {
                const cplx<R>* gc = g + col * 2 * NB;
                cplx<R> a0 = czero<R>(), a1 = czero<R>();
                int s = 0;
                for (; s + 1 <= t; s += 2) {
                    cfma(a0, iL[t * NBP + s], gc[s]);
                    cfma(a1, iL[t * NBP + s + 1], gc[s + 1]);
                }
                if (s <= t) cfma(a0, iL[t * NBP + s], gc[s]);
                A[(int64_t)(k0 + t) + (int64_t)(c0 + col) * lda] = a0 + a1;
            }
        }
        wsync();
    }
}

// A22 -= L21 * U12 over rows and columns [k0 + NB, n).
template <typename R>
__device__ void trailing_update(cplx<R>* A, int64_t lda, int n, int k0, cplx<R>* sm) {
    using T = DTile<R>;
    constexpr int TM = T::TM, TN = T::TN, MI = T::MI, MJ = T::MJ, TNP = TN + 1;
    cplx<R>* As = sm;                 // [2][NB][TM]
    cplx<R>* Bs = sm + 2 * NB * TM;   // [NB][TNP]
    const int tid = threadIdx.x, ty = tid % 16, tx = tid / 16;
    const int r_begin = k0 + NB;
    const int ntiles = (n - r_begin + TM - 1) / TM;
    const cplx<R>* L21 = A + (int64_t)k0 * lda;  // panel columns
    auto load_a = [&](cplx<R>* buf, int i0) {
        for (int idx = tid; idx < NB * TM; idx += NT) {
            const int r = idx % TM, k = idx / TM;
            const bool ok = i0 + r < n;
            cp_elem(&buf[k * TM + r], ok ? L21 + (i0 + r) + (int64_t)k * lda : A, ok);
        }
    };
    for (int c0 = r_begin; c0 < n; c0 += TN) {
        const int ce = min(n, c0 + TN);
        for (int idx = tid; idx < NB * TN; idx += NT) {
            const int k = idx % NB, c = idx / NB;
            const bool ok = c0 + c < ce;
            cp_elem(&Bs[k * TNP + c], ok ? A + (k0 + k) + (int64_t)(c0 + c) * lda : A, ok);
        }
        load_a(As, r_begin);
        cp_commit();
        for (int t = 0; t < ntiles; ++t) {
            const int i0 = r_begin + t * TM;
            if (t + 1 < ntiles) load_a(As + ((t + 1) & 1) * NB * TM, i0 + TM);
            cp_commit();
            cplx<R> acc[MI][MJ];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < MJ; ++j) {
                    const int r = i0 + ty + 16 * i, c = c0 + tx + 16 * j;
                    acc[i][j] = (r < n && c < ce) ? A[r + (int64_t)c * lda] : czero<R>();
                }
            cp_wait<1>();
            wsync();
            const cplx<R>* Ab = As + (t & 1) * NB * TM;
#pragma unroll 2
            for (int k = 0; k < NB; ++k) {
                cplx<R> a[MI], b[MJ];
#pragma unroll
                for (int i = 0; i < MI; ++i) a[i] = Ab[k * TM + ty + 16 * i];
#pragma unroll
                for (int j = 0; j < MJ; ++j) b[j] = Bs[k * TNP + tx + 16 * j];
#pragma unroll
                for (int i = 0; i < MI; ++i)
#pragma unroll
                    for (int j = 0; j < MJ; ++j) cfms(acc[i][j], a[i], b[j]);
            }
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < MJ; ++j) {
                    const int r = i0 + ty + 16 * i, c = c0 + tx + 16 * j;
                    if (r < n && c < ce) A[r + (int64_t)c * lda] = acc[i][j];
                }
            wsync();
        }
        cp_wait<0>();
        wsync();
    }
}

// ------------------------------------------------------------------------------------------
// Complex64 trailing update on the tensor cores (tcgen05, kind::f16 with BF16 operands).
//
// A22 -= L21 U12 in real arithmetic is four real products (Lr Ur, -Li Ui into the real part;
// Lr Ui, Li Ur into the imaginary part).  Each FP32 operand x is split into three BF16 pieces
// x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m): 24 significant bits), and a
// product is taken as the six piece products of order >= 2^-16 (hh, hm, mh, hl, mm, lh) with
// FP32 accumulation in tensor memory: FP32-level accuracy (what is dropped is ~2^-24 relative).
// The FP64 refinement of the sample solves sits on top as for the CUDA-core path.  Against a
// two-piece TF32 split (three products) this is the same tensor time, but the operands take
// 12 instead of 16 bytes per complex value, which lets a 128 x 128 step fit in shared memory:
// N = 128 per MMA keeps the operand reads per MMA within the shared-memory bandwidth.
//
// Per panel the operands are split once into "images" in global memory whose bytes are exactly
// the shared-memory layout the MMA reads (K-major, 128-byte swizzle, K = 64 = one 128-byte row):
// one 96 KB image per 128-row tile of L21 and one per 128-column block of U12.  For each L21
// tile the MMA issuer (thread 0) bulk-copies the tile, then walks the U12 blocks through one smem
// buffer and two TMEM accumulator pairs: while all 8 warps run the epilogue of block t (C
// prefetched from global memory, TMEM -> registers, C -= D), thread 0 refills the buffer with
// block t+1 and issues its MMAs.  Every wait is bounded; a timeout marks the job failed.
// ------------------------------------------------------------------------------------------
struct TcShared {
    // 0: L21 tile; 1: U12 buffer; 2: command to the producer warp; 3 + b: epilogue of accumulator
    // pair b done (one arrival per worker warp); 5 + b: MMAs into accumulator pair b done
    uint64_t bar[7];
    uint32_t tmem;       // tensor-memory base address
    int fail;            // set by any thread whose bounded wait ran out
    int stop;            // the workers' common view of `fail`, written by worker thread 0 between barriers
    int cmd;             // 1: run a trailing update with the parameters below, 2: exit
    int n, k0;
    int64_t lda;
    const float* imgA;
    const float* imgB;
};
struct TcPhase {
    uint32_t a = 0, b = 0, go = 0, e[2] = {0, 0}, d[2] = {0, 0};
};

__device__ __forceinline__ bool failed(const TcShared& ts) { return *(const volatile int*)&ts.fail != 0; }

// Write the six BF16 pieces of (re, im) at (row r, k) of an operand image with `rows` rows:
// array q (0..2 re hi/mid/lo, 3..5 im hi/mid/lo) occupies rows * 64 elements.
__device__ __forceinline__ void put_split(__nv_bfloat16* t, int r, int k, int rows, float re, float im) {
    const uint32_t at = sw128_index16(r, k), stride = (uint32_t)rows * NB;
    float x[2] = {re, im};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x[c]);
        const float r1 = x[c] - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
        t[(3 * c + 0) * stride + at] = h;
        t[(3 * c + 1) * stride + at] = m;
        t[(3 * c + 2) * stride + at] = l;
    }
}


// L21 (rows k0+NB.., panel columns) -> one image per 128-row tile; rows past n are zero.
__device__ void emit_a_image(const c64* A, int64_t lda, int n, int k0, float* img) {
    const int r_begin = k0 + NB, m = n - r_begin;
    const int rows_pad = (m + TC_ROWS - 1) / TC_ROWS * TC_ROWS;
    for (int idx = threadIdx.x; idx < rows_pad * NB; idx += NT) {
        const int rr = idx % rows_pad, k = idx / rows_pad;
        c64 v = czero<float>();
        if (rr < m) v = A[(int64_t)(r_begin + rr) + (int64_t)(k0 + k) * lda];
        put_split(reinterpret_cast<__nv_bfloat16*>(img + (size_t)(rr / TC_ROWS) * TC_A_FLOATS), rr % TC_ROWS, k,
                  TC_ROWS, v.re, v.im);
    }
}
// U12 (panel rows, columns k0+NB..) -> one image per 128-column block; columns past n are zero.
__device__ void emit_b_image(const c64* A, int64_t lda, int n, int k0, float* img) {
    const int c_begin = k0 + NB, m = n - c_begin;
    const int cols_pad = (m + TC_COLS - 1) / TC_COLS * TC_COLS;
    for (int idx = threadIdx.x; idx < cols_pad * NB; idx += NT) {
        const int k = idx % NB, cc = idx / NB;
        c64 v = czero<float>();
        if (cc < m) v = A[(int64_t)(k0 + k) + (int64_t)(c_begin + cc) * lda];
        put_split(reinterpret_cast<__nv_bfloat16*>(img + (size_t)(cc / TC_COLS) * TC_B_FLOATS), cc % TC_COLS, k,
                  TC_COLS, v.re, v.im);
    }
}

// All MMAs of one (L21 tile, U12 block) step into the accumulator pair at TMEM column dt:
// re part at dt, im part at dt + 128.  Descriptors are built once; an offset of o bytes inside
// an operand buffer is + (o >> 4) on the descriptor (no carry: the buffers lie below 256 KB).
__device__ __forceinline__ void tc_issue(uint64_t adesc, uint64_t bdesc, uint32_t dt) {
    // kind::f16: F32 accumulate, BF16 A and B, K-major both, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((TC_COLS >> 3) << 17) | ((TC_ROWS >> 4) << 24);
    const int pa[4] = {0, 1, 0, 1}, pb[4] = {0, 1, 1, 0}, pd[4] = {0, 0, 128, 128}, ng[4] = {0, 1, 0, 0};
    const int sa[6] = {0, 0, 1, 0, 1, 2}, sb[6] = {0, 1, 0, 2, 1, 0};  // hh hm mh hl mm lh
    uint32_t acc_r = 0, acc_i = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t id = idesc | (ng[p] ? (1u << 13) : 0u);  // negate A for -Li Ui
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            const uint32_t qa = pa[p] * TC_SPLIT + sa[s], qb = pb[p] * TC_SPLIT + sb[s];
#pragma unroll
            for (int ks = 0; ks < NB / 16; ++ks) {
                const uint32_t ao = qa * TC_ROWS * NB * 2 + ks * 32;
                const uint32_t bo = qb * TC_COLS * NB * 2 + ks * 32;
                uint32_t& acc = pd[p] ? acc_i : acc_r;
                tc_mma(dt + pd[p], adesc + (ao >> 4), bdesc + (bo >> 4), id, acc);
                acc = 1;
            }
        }
    }
}

// C -= D for one 128 x 128 step: warp w reads TMEM lanes 32 (w % 4).., complex columns 64 (w / 4)..
// in two chunks of 32.  `v` holds a chunk of C values, loaded before the TMEM data is waited for.
__device__ __forceinline__ void tc_load_c(const c64* A, int64_t lda, int n, int i0, int c0, int chunk, c64* v) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const int row = i0 + 32 * q + lane, cb = c0 + half * 64 + chunk * 32;
#pragma unroll
    for (int c = 0; c < 32; ++c)
        v[c] = (row < n && cb + c < n) ? A[row + (int64_t)(cb + c) * lda] : czero<float>();
}
__device__ __forceinline__ void tc_store_c(c64* A, int64_t lda, int n, int i0, int c0, int chunk, uint32_t tbuf,
                                           const c64* v) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const uint32_t ta = tbuf + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * 64 + chunk * 32);
    const int row = i0 + 32 * q + lane, cb = c0 + half * 64 + chunk * 32;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float dr[16], di[16];
        tc_ld16(ta + h * 16, dr);
        tc_ld16(ta + 128 + h * 16, di);
        tc_wait_ld();
        if (row < n) {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int col = cb + h * 16 + c;
                if (col < n) A[row + (int64_t)col * lda] = mk<float>(v[h * 16 + c].re - dr[c], v[h * 16 + c].im - di[c]);
            }
        }
    }
}

// Worker side (warps 0..7) of one panel's trailing update: hand the parameters to the producer
// warp, then for every (L21 tile, U12 block) step in order: prefetch C, wait for the step's
// MMAs, read the accumulators, release them to the producer, write C back.
__device__ void trailing_update_tc(c64* A, int64_t lda, int n, int k0, const float* imgA, const float* imgB,
                                   TcShared& ts, TcPhase& ph) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int r_begin = k0 + NB, m = n - r_begin;
    const int ncb = (m + TC_COLS - 1) / TC_COLS, steps = (m + TC_ROWS - 1) / TC_ROWS * ncb;
    if (tid == 0) {
        ts.n = n;
        ts.k0 = k0;
        ts.lda = lda;
        ts.imgA = imgA;
        ts.imgB = imgB;
        ts.cmd = 1;
        mbar_arrive(&ts.bar[2]);  // release: the producer reads the parameters after its wait
    }
    c64 v[32];
    for (int g = 0; g < steps && !failed(ts); ++g) {
        const int b = g & 1;
        const int i0 = r_begin + (g / ncb) * TC_ROWS, c0 = r_begin + (g % ncb) * TC_COLS;
        const uint32_t tb = ts.tmem + b * 256;
        tc_load_c(A, lda, n, i0, c0, 0, v);
        if (!mbar_wait(&ts.bar[5 + b], ph.d[b])) ts.fail = 1;
        ph.d[b] ^= 1;
        tc_fence_after();
        tc_store_c(A, lda, n, i0, c0, 0, tb, v);
        tc_load_c(A, lda, n, i0, c0, 1, v);
        tc_store_c(A, lda, n, i0, c0, 1, tb, v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ts.bar[3 + b]);
    }
    wsync();  // warps may leave the loop at different steps after a timeout; all meet here
    if (tid == 0) ts.stop = failed(ts) ? 1 : 0;
    wsync();
}

// Producer warp (warp 8; lane 0 issues): per trailing update, bulk-copy each L21 tile and U12
// block into shared memory and issue the step's MMAs into accumulator pair g % 2 once the
// workers have released it.  Runs until the exit command.
__device__ void tc_producer(unsigned char* smem_raw, TcShared& ts) {
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sB = base + TC_A_BYTES;
    const uint64_t adesc = sw128_desc(smem_u32(base)), bdesc = sw128_desc(smem_u32(sB));
    const bool leader = (threadIdx.x & 31) == 0;
    uint32_t pa = 0, pb = 0, pgo = 0, pm[2] = {0, 0}, pe[2] = {0, 0};
    auto wait = [&](uint64_t* bar, uint32_t& par) {
        if (!failed(ts) && !mbar_wait(bar, par)) ts.fail = 1;
        par ^= 1;
    };
    for (;;) {
        // the command barrier completes once per command; the workers factor a panel in between,
        // so one bounded wait may run out: retry a bounded number of times, then give up
        int got = 0;
        if (leader)
            for (int tries = 0; tries < 64 && !got; ++tries) got = mbar_wait(&ts.bar[2], pgo) ? 1 : 0;
        got = __shfl_sync(FULL, got, 0);  // one decision for the whole warp
        if (!got) {
            ts.fail = 1;
            return;
        }
        pgo ^= 1;
        if (*(volatile int*)&ts.cmd != 1) break;
        const int n = *(volatile int*)&ts.n, k0 = *(volatile int*)&ts.k0;
        const float* imgA = *(const float* volatile*)&ts.imgA;
        const float* imgB = *(const float* volatile*)&ts.imgB;
        const int r_begin = k0 + NB, m = n - r_begin;
        const int ncb = (m + TC_COLS - 1) / TC_COLS, steps = (m + TC_ROWS - 1) / TC_ROWS * ncb;
        for (int g = 0; g < steps; ++g) {
            const int rt = g / ncb, t = g % ncb, b = g & 1;
            if (g > 0) wait(&ts.bar[5 + ((g - 1) & 1)], pm[(g - 1) & 1]);  // the operand buffers are free
            if (leader && !failed(ts)) {
                if (t == 0) {
                    mbar_expect_tx(&ts.bar[0], TC_A_BYTES);
                    for (int c = 0; c < 6; ++c)
                        bulk_g2s(base + c * (TC_A_BYTES / 6), imgA + (size_t)rt * TC_A_FLOATS + c * (TC_A_FLOATS / 6),
                                 TC_A_BYTES / 6, &ts.bar[0]);
                }
                mbar_expect_tx(&ts.bar[1], TC_B_BYTES);
                const float* src = imgB + (size_t)t * TC_B_FLOATS;
                for (int c = 0; c < 6; ++c)
                    bulk_g2s(sB + c * (TC_B_BYTES / 6), src + c * (TC_B_FLOATS / 6), TC_B_BYTES / 6, &ts.bar[1]);
                if (t + 1 < ncb) prefetch_l2(src + TC_B_FLOATS, TC_B_BYTES);
                else if ((rt + 1) * TC_ROWS < m) prefetch_l2(imgA + (size_t)(rt + 1) * TC_A_FLOATS, TC_A_BYTES);
            }
            __syncwarp();
            if (t == 0) wait(&ts.bar[0], pa);
            wait(&ts.bar[1], pb);
            if (g >= 2) wait(&ts.bar[3 + b], pe[b]);  // the workers have read accumulator pair b
            tc_fence_after();
            if (leader) {
                if (!failed(ts)) tc_issue(adesc, bdesc, ts.tmem + b * 256);
                tc_commit(&ts.bar[5 + b]);
            }
            __syncwarp();
        }
        // consume the completions not waited for above, so every barrier's phase stays in step
        if (steps > 0) wait(&ts.bar[5 + ((steps - 1) & 1)], pm[(steps - 1) & 1]);
        if (steps > 1) wait(&ts.bar[3 + ((steps - 2) & 1)], pe[(steps - 2) & 1]);
        if (steps > 0) wait(&ts.bar[3 + ((steps - 1) & 1)], pe[(steps - 1) & 1]);
    }
}

template <typename R>
__device__ void factor_one(const DenseJob<R>& J, cplx<R>* sm, DShared& sh, float* img, size_t img_b, TcShared* ts,
                           TcPhase* ph) {
    const int n = J.n;
    const int64_t lda = J.lda;
    cplx<R>* A = J.a;
    const int cap_rows = (int)(factor_smem<R>() / (NB * sizeof(cplx<R>)));
    for (int p = 0, k0 = 0; k0 < n; ++p, k0 += NB) {
        const int nbk = min(NB, n - k0), m = n - k0;
        cplx<R>* Pg = A + k0 + (int64_t)k0 * lda;
        if (m <= cap_rows) {
            for (int idx = threadIdx.x; idx < m * nbk; idx += NT) {
                const int r = idx % m, c = idx / m;
                sm[r + c * m] = Pg[r + (int64_t)c * lda];
            }
            wsync();
            panel_factor(sm, (int64_t)m, m, nbk, k0, sh);
            for (int idx = threadIdx.x; idx < m * nbk; idx += NT) {
                const int r = idx % m, c = idx / m;
                Pg[r + (int64_t)c * lda] = sm[r + c * m];
            }
            wsync();
        } else {
            panel_factor(Pg, lda, m, nbk, k0, sh);
        }
        if ((int)threadIdx.x < nbk) J.ipiv[k0 + threadIdx.x] = k0 + sh.piv[threadIdx.x];
        compose_swaps(nbk, sh);
        int32_t* sw = J.swaps + (int64_t)p * kDenseSwapInts;
        if (threadIdx.x == 0) sw[0] = sh.cnt;
        for (int i = threadIdx.x; i < 2 * NB; i += NT) {
            sw[1 + i] = i < sh.cnt ? sh.rows[i] : 0;
            sw[1 + 2 * NB + i] = i < sh.cnt ? sh.src[i] : 0;
        }
        diag_inverses(Pg, lda, nbk, sm, J.inv + (int64_t)p * 2 * NB * NB);
        if (k0 + nbk < n) {
            trailing_rows(A, lda, n, k0, sm, sh);
            if constexpr (sizeof(R) == 4) {
                emit_a_image(A, lda, n, k0, img);
                emit_b_image(A, lda, n, k0, img + img_b);
                // the images (global) and the shared buffers were last touched through the generic
                // proxy; the bulk copies and MMAs that follow go through the async proxy
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                wsync();
                trailing_update_tc(A, lda, n, k0, img, img + img_b, *ts, *ph);
                if (ts->stop) {  // uniform: written by thread 0 between two worker barriers
                    if (threadIdx.x == 0) sh.info = -1;
                    break;
                }
            } else {
                trailing_update(A, lda, n, k0, sm);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Solves.  x (n x L, leading dimension n) <- A^{-1} x.  Forward: per panel, the composed
// interchanges, y = inv(L11) x_top, x_below -= L21 y.  Backward: per panel from the last,
// y = inv(U11) x_top, x_above -= U01 y.  Right-hand sides in groups of LG columns.
// ------------------------------------------------------------------------------------------
constexpr int LG = 32;  // right-hand-side columns per pass over the factor
template <typename R> struct SolveChunk;
template <> struct SolveChunk<float> { static constexpr int LC = 8; };
template <> struct SolveChunk<double> { static constexpr int LC = 4; };

template <typename R>
constexpr size_t solve_smem() {
    return ((size_t)NB * NBP + (size_t)2 * NB * LG + (size_t)NB * LG) * sizeof(cplx<R>);
}

// x[r, l] -= sum_k Ablk[r + k lda] y[k * LP + l]  for r in [r0, r1), l < lg
template <typename R>
__device__ void solve_update(const cplx<R>* __restrict__ Ablk, int64_t lda, int r0, int r1, int nbk,
                             const cplx<R>* y, int LP, int lg, cplx<R>* __restrict__ x, int64_t ldx) {
    constexpr int LC = SolveChunk<R>::LC;
    for (int l0 = 0; l0 < lg; l0 += LC) {
        for (int r = r0 + (int)threadIdx.x; r < r1; r += NT) {
            cplx<R> acc[LC];
#pragma unroll
            for (int l = 0; l < LC; ++l) acc[l] = (l0 + l < lg) ? x[r + (int64_t)(l0 + l) * ldx] : czero<R>();
#pragma unroll 8
            for (int k = 0; k < nbk; ++k) {
                const cplx<R> a = Ablk[r + (int64_t)k * lda];
#pragma unroll
                for (int l = 0; l < LC; ++l) cfms(acc[l], a, y[k * LP + l0 + l]);
            }
#pragma unroll
            for (int l = 0; l < LC; ++l)
                if (l0 + l < lg) x[r + (int64_t)(l0 + l) * ldx] = acc[l];
        }
    }
}

// x <- A^{-1} x for one factored point (all J.L columns), by the NT worker threads.
// smem: solve_smem<R>() bytes; rows/src/cnt: 2 NB + 2 NB + 1 ints of shared scratch.
template <typename R>
__device__ void solve_one(const DenseJob<R>& J, unsigned char* smem, int* s_rows, int* s_src, int* s_cnt) {
    constexpr int LC = SolveChunk<R>::LC;
    cplx<R>* sinv = reinterpret_cast<cplx<R>*>(smem);  // (r, c) at r * NBP + c
    cplx<R>* g = sinv + NB * NBP;                      // [2 NB][LG]
    cplx<R>* y = g + 2 * NB * LG;                      // [NB][LP]
    const int n = J.n;
    const int np = (int)dense_panels(n);
    const int64_t lda = J.lda;
    for (int l_begin = 0; l_begin < J.L; l_begin += LG) {
        const int lg = min(LG, J.L - l_begin);
        const int LP = (lg + LC - 1) / LC * LC;
        cplx<R>* x = J.x + (int64_t)l_begin * n;
        for (int idx = threadIdx.x; idx < NB * LP; idx += NT) y[idx] = czero<R>();
        wsync();
        for (int p = 0; p < np; ++p) {  // forward
            const int k0 = p * NB, nbk = min(NB, n - k0);
            const int32_t* sw = J.swaps + (int64_t)p * kDenseSwapInts;
            const cplx<R>* gi = J.inv + (int64_t)p * 2 * NB * NB;
            if (threadIdx.x == 0) *s_cnt = sw[0];
            for (int i = threadIdx.x; i < 2 * NB; i += NT) {
                s_rows[i] = sw[1 + i];
                s_src[i] = sw[1 + 2 * NB + i];
            }
            for (int idx = threadIdx.x; idx < nbk * nbk; idx += NT) {
                const int r = idx % nbk, c = idx / nbk;
                sinv[r * NBP + c] = gi[r + c * NB];
            }
            wsync();
            const int cnt = *s_cnt;
            for (int idx = threadIdx.x; idx < cnt * lg; idx += NT) {
                const int e = idx % cnt, l = idx / cnt;
                g[e * LG + l] = x[k0 + s_src[e] + (int64_t)l * n];
            }
            wsync();
            const int extra = cnt - nbk;
            for (int idx = threadIdx.x; idx < extra * lg; idx += NT) {
                const int e = nbk + idx % extra, l = idx / extra;
                x[k0 + s_rows[e] + (int64_t)l * n] = g[e * LG + l];
            }
            for (int idx = threadIdx.x; idx < nbk * lg; idx += NT) {
                const int t = idx % nbk, l = idx / nbk;
                cplx<R> acc = czero<R>();
                for (int s = 0; s <= t; ++s) cfma(acc, sinv[t * NBP + s], g[s * LG + l]);
                y[t * LP + l] = acc;
                x[k0 + t + (int64_t)l * n] = acc;
            }
            wsync();
            if (k0 + nbk < n) solve_update(J.a + (int64_t)k0 * lda, lda, k0 + nbk, n, nbk, y, LP, lg, x, n);
            wsync();
        }
        for (int p = np - 1; p >= 0; --p) {  // backward
            const int k0 = p * NB, nbk = min(NB, n - k0);
            const cplx<R>* gi = J.inv + (int64_t)p * 2 * NB * NB + NB * NB;
            for (int idx = threadIdx.x; idx < nbk * nbk; idx += NT) {
                const int r = idx % nbk, c = idx / nbk;
                sinv[r * NBP + c] = gi[r + c * NB];
            }
            for (int idx = threadIdx.x; idx < nbk * lg; idx += NT) {
                const int t = idx % nbk, l = idx / nbk;
                g[t * LG + l] = x[k0 + t + (int64_t)l * n];
            }
            wsync();
            for (int idx = threadIdx.x; idx < nbk * lg; idx += NT) {
                const int t = idx % nbk, l = idx / nbk;
                cplx<R> acc = czero<R>();
                for (int s = t; s < nbk; ++s) cfma(acc, sinv[t * NBP + s], g[s * LG + l]);
                y[t * LP + l] = acc;
                x[k0 + t + (int64_t)l * n] = acc;
            }
            wsync();
            if (k0 > 0) solve_update(J.a + (int64_t)k0 * lda, lda, 0, k0, nbk, y, LP, lg, x, n);
            wsync();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Fused dense sampling.  Per job (point j of NEP E), in the CTA's slot:
//   zero the matrix, scatter T(z_j) = sum_i f_i(z_j) A_i (precision R) and the FP64 column
//   sums |T| (for ||T||_1); factor; x = U; solve; X = x in S_hat (FP64); then
//   r = U - T X in FP64 from the CSR values (T recomputed from the f_i), eta per column,
//   and refinement X += (LU)^{-1} r while the stopping rule of the band path asks for it.
// ------------------------------------------------------------------------------------------
constexpr int kMaxL = 256;

struct SampleShared {
    double rn2[kMaxL], xn2[kMaxL];
    double red[NW];
    double normT, mx;
    int action;
};

template <typename R>
struct Slot {
    cplx<R>* a;
    cplx<R>* x;
    int32_t* ipiv;
    cplx<R>* inv;
    int32_t* swaps;
    double* colsum;
};

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R>
__host__ __device__ inline size_t slot_bytes(int n_max, int L_max) {
    const size_t np = (size_t)dense_panels(n_max);
    return align256((size_t)n_max * n_max * sizeof(cplx<R>)) + align256((size_t)n_max * L_max * sizeof(cplx<R>)) +
           align256((size_t)n_max * 4) + align256(np * 2 * NB * NB * sizeof(cplx<R>)) +
           align256(np * kDenseSwapInts * 4) + align256((size_t)n_max * 8);
}

template <typename R>
__device__ Slot<R> slot_at(unsigned char* base, int n_max, int L_max) {
    const size_t np = (size_t)dense_panels(n_max);
    Slot<R> t;
    unsigned char* p = base;
    t.a = reinterpret_cast<cplx<R>*>(p);
    p += align256((size_t)n_max * n_max * sizeof(cplx<R>));
    t.x = reinterpret_cast<cplx<R>*>(p);
    p += align256((size_t)n_max * L_max * sizeof(cplx<R>));
    t.ipiv = reinterpret_cast<int32_t*>(p);
    p += align256((size_t)n_max * 4);
    t.inv = reinterpret_cast<cplx<R>*>(p);
    p += align256(np * 2 * NB * NB * sizeof(cplx<R>));
    t.swaps = reinterpret_cast<int32_t*>(p);
    p += align256(np * kDenseSwapInts * 4);
    t.colsum = reinterpret_cast<double*>(p);
    return t;
}

// Block-wide max of one double per thread (workers only); every worker gets the result.
__device__ double worker_max(double v, SampleShared& ss) {
    for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, off));
    if ((threadIdx.x & 31) == 0) ss.red[threadIdx.x >> 5] = v;
    wsync();
    double m = ss.red[0];
    for (int w = 1; w < NW; ++w) m = fmax(m, ss.red[w]);
    wsync();
    return m;
}

// r = U - T X (FP64, T from the CSR values and f_i(z_j)); x = r in precision R; per-column
// ||r||^2 and ||X||^2 into ss.rn2 / ss.xn2.
template <typename R>
__device__ void residual_one(const DenseNep& E, int j, const c128* X, cplx<R>* x, SampleShared& ss) {
    constexpr int LC = 8;
    const int n = E.n, L = E.L, J = E.J;
    const int64_t nnz = E.nnz;
    const c128* f = E.F + (int64_t)j * J;
    for (int l = threadIdx.x; l < L; l += NT) ss.rn2[l] = ss.xn2[l] = 0.0;
    wsync();
    for (int l0 = 0; l0 < L; l0 += LC) {
        double pr[LC], px[LC];
#pragma unroll
        for (int l = 0; l < LC; ++l) pr[l] = px[l] = 0.0;
        for (int r = threadIdx.x; r < n; r += NT) {
            c128 acc[LC];
#pragma unroll
            for (int l = 0; l < LC; ++l) acc[l] = (l0 + l < L) ? E.U[r + (int64_t)(l0 + l) * n] : czero<double>();
            for (int64_t k = E.rowptr[r]; k < E.rowptr[r + 1]; ++k) {
                c128 t = czero<double>();
                for (int i = 0; i < J; ++i) cfma(t, f[i], E.vals[(int64_t)i * nnz + k]);
                const int64_t c = E.colind[k];
#pragma unroll
                for (int l = 0; l < LC; ++l)
                    if (l0 + l < L) cfms(acc[l], t, X[c + (int64_t)(l0 + l) * n]);
            }
#pragma unroll
            for (int l = 0; l < LC; ++l)
                if (l0 + l < L) {
                    x[r + (int64_t)(l0 + l) * n] = ccast<R>(acc[l]);
                    pr[l] += cnorm2(acc[l]);
                    px[l] += cnorm2(X[r + (int64_t)(l0 + l) * n]);
                }
        }
#pragma unroll
        for (int l = 0; l < LC; ++l) {
            double a = pr[l], b = px[l];
            for (int off = 16; off; off >>= 1) {
                a += __shfl_down_sync(FULL, a, off);
                b += __shfl_down_sync(FULL, b, off);
            }
            if ((threadIdx.x & 31) == 0 && l0 + l < L) {
                atomicAdd(&ss.rn2[l0 + l], a);
                atomicAdd(&ss.xn2[l0 + l], b);
            }
        }
    }
    wsync();
}

template <typename R>
__device__ void sample_one(const DenseNep& E, int j, const Slot<R>& sl, cplx<R>* sm, DShared& sh, SampleShared& ss,
                           float* img, size_t img_b, TcShared* ts, TcPhase* ph, const DenseSampleCfg& cfg) {
    const int n = E.n, L = E.L, J = E.J;
    const int64_t nnz = E.nnz, nl = (int64_t)n * L;
    cplx<R>* A = sl.a;
    // assemble T(z_j) (precision R) and its FP64 column sums
    {
        const int64_t nn = (int64_t)n * n;
        for (int64_t idx = threadIdx.x; idx < nn; idx += NT) A[idx] = czero<R>();
        for (int c = threadIdx.x; c < n; c += NT) sl.colsum[c] = 0.0;
        wsync();
        const c128* f = E.F + (int64_t)j * J;
        for (int64_t k = threadIdx.x; k < nnz; k += NT) {
            c128 t = czero<double>();
            for (int i = 0; i < J; ++i) cfma(t, f[i], E.vals[(int64_t)i * nnz + k]);
            const int c = E.colind[k];
            A[E.rowidx[k] + (int64_t)c * n] = ccast<R>(t);
            atomicAdd(&sl.colsum[c], sqrt(cnorm2(t)));
        }
        wsync();
        double m = 0.0;
        for (int c = threadIdx.x; c < n; c += NT) m = fmax(m, sl.colsum[c]);
        m = worker_max(m, ss);
        if (threadIdx.x == 0) ss.normT = m;
    }
    DenseJob<R> Jb;
    Jb.a = A;
    Jb.lda = n;
    Jb.n = n;
    Jb.L = L;
    Jb.ipiv = sl.ipiv;
    Jb.inv = sl.inv;
    Jb.swaps = sl.swaps;
    Jb.x = sl.x;
    if (threadIdx.x == 0) sh.info = 0;
    wsync();
    factor_one(Jb, sm, sh, img, img_b, ts, ph);
    wsync();
    const int info = sh.info;
    if (info != 0) {
        if (threadIdx.x == 0) {
            E.status[j] = info;
            E.sweeps[j] = 0;
        }
        wsync();
        return;
    }
    c128* X = E.S + (int64_t)j * nl;
    for (int64_t idx = threadIdx.x; idx < nl; idx += NT) sl.x[idx] = ccast<R>(E.U[idx]);
    wsync();
    unsigned char* smb = reinterpret_cast<unsigned char*>(sm);
    solve_one(Jb, smb, sh.rows, sh.src, &sh.cnt);
    for (int64_t idx = threadIdx.x; idx < nl; idx += NT) X[idx] = ccast<double>(sl.x[idx]);
    wsync();
    double prev = 0.0;
    int sweeps = 0;
    for (;;) {
        residual_one(E, j, X, sl.x, ss);
        // backward error per column and the decision (one thread decides, all follow)
        double mx = 0.0;
        int nonfinite = 0;
        for (int l = threadIdx.x; l < L; l += NT) {
            const double e = sqrt(ss.rn2[l]) / (ss.normT * sqrt(ss.xn2[l]) + sqrt(E.un2[l]));
            E.eta[(int64_t)j * L + l] = e;
            if (!isfinite(e)) nonfinite = 1;
            mx = fmax(mx, e);
        }
        mx = worker_max(nonfinite ? INFINITY : mx, ss);
        if (threadIdx.x == 0) {
            int action;                                          // 0 done, 1 refine, < 0 failed
            const bool improving = sweeps == 0 || mx < 0.5 * prev;
            if (!isfinite(mx)) action = -2;
            else if (!(mx <= cfg.target) && improving) action = sweeps >= cfg.max_refine ? (mx <= cfg.tol ? 0 : -3) : 1;
            else action = (mx <= cfg.tol) ? 0 : -3;
            ss.action = action;
        }
        prev = mx;
        wsync();
        const int action = ss.action;
        if (action != 1) {
            if (threadIdx.x == 0) {
                E.status[j] = action;
                E.sweeps[j] = sweeps;
            }
            break;
        }
        solve_one(Jb, smb, sh.rows, sh.src, &sh.cnt);
        for (int64_t idx = threadIdx.x; idx < nl; idx += NT) X[idx] = X[idx] + ccast<double>(sl.x[idx]);
        wsync();
        ++sweeps;
    }
    wsync();
}

// Complex64 launches NT + 32 threads: warps 0..7 work, warp 8 feeds the tensor cores;
// complex128 launches NT.  CTA b uses slot b and (complex64) image block b.
template <typename R>
__global__ void __launch_bounds__(sizeof(R) == 4 ? NT + 32 : NT, 1)
    dense_sample_kernel(const DenseNep* __restrict__ neps, const DenseSampleJob* __restrict__ jobs, int njobs,
                        int n_max, int L_max, unsigned char* slots, size_t slot_stride, float* img, size_t img_stride,
                        size_t img_b, int32_t* __restrict__ next, DenseSampleCfg cfg) {
    extern __shared__ __align__(16) unsigned char dense_smem[];
    cplx<R>* sm = reinterpret_cast<cplx<R>*>(dense_smem);
    __shared__ DShared sh;
    __shared__ SampleShared ss;
    __shared__ __align__(8) TcShared ts;
    TcPhase ph;
    constexpr bool tc = sizeof(R) == 4;
    if (tc) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < 7; ++i) mbar_init(&ts.bar[i], i == 3 || i == 4 ? NT / 32 : 1);
            ts.fail = 0;
            ts.stop = 0;
            ts.cmd = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(&ts.tmem)), "r"(TC_TMEM_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x >= NT) tc_producer(dense_smem, ts);
    }
    if (threadIdx.x < NT) {
        const Slot<R> sl = slot_at<R>(slots + (size_t)blockIdx.x * slot_stride, n_max, L_max);
        float* my_img = img ? img + (size_t)blockIdx.x * img_stride : nullptr;
        for (;;) {
            if (threadIdx.x == 0) sh.job = (tc && ts.stop) ? njobs : atomicAdd(next, 1);  // no new job after a timeout
            wsync();
            const int jb = sh.job;
            if (jb >= njobs) break;
            const DenseSampleJob job = jobs[jb];
            sample_one<R>(neps[job.nep], job.j, sl, sm, sh, ss, my_img, img_b, &ts, &ph, cfg);
        }
        if (tc && threadIdx.x == 0) {
            ts.cmd = 2;
            mbar_arrive(&ts.bar[2]);
        }
    }
    if (tc) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ts.tmem), "r"(TC_TMEM_COLS)
                         : "memory");
    }
}

// Opt a kernel into its dynamic shared memory.  The attribute is per function and process-wide,
// so it is set to the largest allowed value rather than to this launch's size: host threads
// launching the same kernel concurrently never lower it under one another.
template <typename K>
int set_smem(K kernel, size_t bytes, const char* name) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    if (bytes + fa.sharedSizeBytes > (size_t)optin)
        return set_error(RSRR_EUNSUPPORTED, std::string(name) + ": shared memory " + std::to_string(bytes) +
                                                " + " + std::to_string(fa.sharedSizeBytes) + " exceeds " +
                                                std::to_string(optin));
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess)
        return set_error(RSRR_ECUDA, std::string(name) + ": cudaFuncSetAttribute: " + cudaGetErrorString(e));
    return RSRR_OK;
}

int sm_count() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

}  // namespace

int dense_sample_grid(int njobs) { return std::max(1, std::min(njobs, sm_count())); }

template <typename R>
size_t dense_slot_bytes(int n_max, int L_max) {
    return slot_bytes<R>(n_max, L_max);
}

template <typename R>
size_t dense_image_bytes(int n_max) {
    if (sizeof(R) != 4) return 0;
    const size_t tiles = (size_t)(n_max + TC_ROWS - 1) / TC_ROWS, blocks = (size_t)(n_max + TC_COLS - 1) / TC_COLS;
    return (tiles * TC_A_FLOATS + blocks * TC_B_FLOATS) * 4;
}

template <typename R>
int launch_dense_sample(const DenseNep* d_neps, const DenseSampleJob* d_jobs, int njobs, int n_max, int L_max,
                        int grid, void* d_slots, void* d_img, int32_t* d_next, DenseSampleCfg cfg, cudaStream_t s) {
    if (njobs <= 0) return RSRR_OK;
    if (L_max > kMaxL) return set_error(RSRR_EINVAL, "dense sampling: L above 256");
    if (sizeof(R) == 4 && !d_img) return set_error(RSRR_EINVAL, "dense sampling: operand images missing");
    const size_t sm = std::max(factor_smem<R>(), solve_smem<R>());
    RSRR_TRY(set_smem(dense_sample_kernel<R>, sm, "dense_sample_kernel"));
    RSRR_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int32_t), s));
    const int threads = sizeof(R) == 4 ? NT + 32 : NT;
    const size_t img_stride = dense_image_bytes<R>(n_max) / 4;
    const size_t img_b = sizeof(R) == 4 ? (size_t)((n_max + TC_ROWS - 1) / TC_ROWS) * TC_A_FLOATS : 0;
    {
        dense_sample_kernel<R><<<grid, threads, sm, s>>>(d_neps, d_jobs, njobs, n_max, L_max,
                                                         static_cast<unsigned char*>(d_slots),
                                                         dense_slot_bytes<R>(n_max, L_max), static_cast<float*>(d_img),
                                                         img_stride, img_b, d_next, cfg);
        note_launch();
    }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template size_t dense_slot_bytes<float>(int, int);
template size_t dense_slot_bytes<double>(int, int);
template size_t dense_image_bytes<float>(int);
template size_t dense_image_bytes<double>(int);
template int launch_dense_sample<float>(const DenseNep*, const DenseSampleJob*, int, int, int, int, void*, void*,
                                        int32_t*, DenseSampleCfg, cudaStream_t);
template int launch_dense_sample<double>(const DenseNep*, const DenseSampleJob*, int, int, int, int, void*, void*,
                                         int32_t*, DenseSampleCfg, cudaStream_t);

}  // namespace rsrr
