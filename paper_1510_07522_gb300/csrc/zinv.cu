// Batched in-place inverse of dense complex128 matrices by blocked Gauss-Jordan elimination with
// partial pivoting: the N_S inverses T_S(z_j)^{-1} of the reduced solve (Algorithm 1, the moments
// of Eq. eq-Ap-num need the whole inverse at every quadrature point).
//
// Per block column J = [jb, jb + bb) of the in-place matrix M (k x k, column-major):
//   1. panel (CUDA cores, one CTA per matrix): LU with partial pivoting (cabs1, lowest row on
//      ties) of a copy of rows jb..k-1 of the block column, in shared memory; it picks the bb
//      pivot rows, which are swapped into rows J across the whole matrix.  With D = M_JJ after
//      the swaps (its LU is the top of the panel), D^{-1} = U11^{-1} L11^{-1}.
//      E = M_:J with rows J cleared is kept, then M_:J is set to [0; I], and
//      W = D^{-1} M_J: (b x k) is written into rows J of M and into a separate buffer.
//   2. trailing update (one batched ZGEMM over all matrices, K = bb):  M -= E W.
//      Rows J are left as W (E is zero there); the other rows get M_O: - M_OJ D^{-1} M_J:, and
//      the pivot columns become -M_OJ D^{-1} (rows O) and D^{-1} (rows J): the Gauss-Jordan step.
// After the last block the row interchanges, applied to whole rows throughout, are undone on the
// columns in reverse order: inv(A) = inv(P A) P.
//
// The elimination costs k^3 complex multiply-adds per matrix, as LU plus an inverse from the
// factors does; nearly all of it is in the ZGEMMs (k x k x bb each), which take the FP64-accurate
// tensor-core emulation when the batch is large enough.  The panels are FP64 CUDA-core work of
// order k^2 bb per matrix.
#include <algorithm>

#include "dense.cuh"

namespace rsrr {

namespace {

constexpr int kZiThreads = 512;
constexpr int kZiWarps = kZiThreads / 32;
constexpr unsigned FULLM = 0xffffffffu;
constexpr size_t kZiSmemMax = 225 * 1024;

size_t panel_smem(int rows, int bb) { return (size_t)rows * bb * sizeof(c128) + (size_t)32 * 32 * sizeof(c128); }

__global__ void __launch_bounds__(kZiThreads) zinv_panel_kernel(c128* X, int k, int jb, int bb, int b, int32_t* piv,
                                                               c128* E, c128* Wb, int32_t* info) {
    extern __shared__ __align__(16) unsigned char zi_raw[];
    __shared__ double s_best[kZiWarps];
    __shared__ int s_pos[kZiWarps];
    __shared__ int s_piv[32];
    __shared__ int s_sing;
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t kk = (int64_t)k * k;
    c128* Xm = X + (int64_t)t * kk;
    c128* Et = E + (int64_t)t * k * b;
    c128* Wt = Wb + (int64_t)t * b * k;
    const int rows = k - jb;
    c128* P = reinterpret_cast<c128*>(zi_raw);  // [bb][rows], column-major
    c128* Di = P + (size_t)rows * bb;           // [32][32] D^{-1}, column-major
    if (tid == 0) s_sing = 0;
    for (int idx = tid; idx < rows * bb; idx += kZiThreads) {
        const int r = idx % rows, c = idx / rows;
        P[idx] = Xm[(int64_t)(jb + r) + (int64_t)(jb + c) * k];
    }
    __syncthreads();

    // ---- LU with partial pivoting of the panel copy ------------------------------------------
    for (int i = 0; i < bb; ++i) {
        double best = -1.0;
        int pos = rows;
        for (int r = i + tid; r < rows; r += kZiThreads) {
            const double a = cabs1(P[r + (int64_t)i * rows]);
            if (a > best) { best = a; pos = r; }
        }
        for (int off = 16; off; off >>= 1) {
            const double ob = __shfl_down_sync(FULLM, best, off);
            const int op = __shfl_down_sync(FULLM, pos, off);
            if (ob > best || (ob == best && op < pos)) { best = ob; pos = op; }
        }
        if (lane == 0) { s_best[warp] = best; s_pos[warp] = pos; }
        __syncthreads();
        if (warp == 0) {
            best = lane < kZiWarps ? s_best[lane] : -1.0;
            pos = lane < kZiWarps ? s_pos[lane] : rows;
            for (int off = 16; off; off >>= 1) {
                const double ob = __shfl_down_sync(FULLM, best, off);
                const int op = __shfl_down_sync(FULLM, pos, off);
                if (ob > best || (ob == best && op < pos)) { best = ob; pos = op; }
            }
            if (lane == 0) {
                // an exactly zero (or non-finite) column: singular; keep going with the diagonal
                // entry so that the launch stays well defined, the caller reports the point
                if (!(best > 0.0) || pos >= rows) { s_sing = 1; pos = i; }
                s_piv[i] = pos;
            }
        }
        __syncthreads();
        const int p = s_piv[i];
        if (p != i && tid < bb) {
            const c128 tmp = P[i + (int64_t)tid * rows];
            P[i + (int64_t)tid * rows] = P[p + (int64_t)tid * rows];
            P[p + (int64_t)tid * rows] = tmp;
        }
        __syncthreads();
        const c128 d = P[i + (int64_t)i * rows];
        const c128 dinv = cis_zero(d) ? mk<double>(1.0, 0.0) : crecip(d);
        for (int r = i + 1 + tid; r < rows; r += kZiThreads) P[r + (int64_t)i * rows] = P[r + (int64_t)i * rows] * dinv;
        __syncthreads();
        const int nr = rows - i - 1, nc = bb - i - 1;
        for (int idx = tid; idx < nr * nc; idx += kZiThreads) {
            const int r = i + 1 + idx % nr, c = i + 1 + idx / nr;
            cfms(P[r + (int64_t)c * rows], P[r + (int64_t)i * rows], P[i + (int64_t)c * rows]);
        }
        __syncthreads();
    }

    // ---- the interchanges on whole rows of M, the kept block column E, M_:J = [0; I] -----------
    if (tid < bb) piv[(int64_t)t * k + jb + tid] = jb + s_piv[tid];
    for (int c = tid; c < k; c += kZiThreads) {
        c128* col = Xm + (int64_t)c * k + jb;
        for (int i = 0; i < bb; ++i) {
            const int p = s_piv[i];
            if (p != i) {
                const c128 tmp = col[i];
                col[i] = col[p];
                col[p] = tmp;
            }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < k * bb; idx += kZiThreads) {
        const int r = idx % k, c = idx / k;
        c128* xp = Xm + r + (int64_t)(jb + c) * k;
        Et[r + (int64_t)c * k] = (r >= jb && r < jb + bb) ? czero<double>() : *xp;
        *xp = (r == jb + c) ? mk<double>(1.0, 0.0) : czero<double>();
    }

    // ---- D^{-1} = U11^{-1} L11^{-1}: column c solves D x = e_c (lane = row) --------------------
    for (int c = warp; c < bb; c += kZiWarps) {
        c128 y = (lane == c) ? mk<double>(1.0, 0.0) : czero<double>();
        for (int i = c; i < bb - 1; ++i) {  // unit lower
            const c128 yi = shfl(y, i);
            if (lane > i && lane < bb) cfms(y, P[lane + (int64_t)i * rows], yi);
        }
        for (int i = bb - 1; i >= 0; --i) {  // upper
            if (lane == i) {
                const c128 u = P[i + (int64_t)i * rows];
                y = y * (cis_zero(u) ? mk<double>(1.0, 0.0) : crecip(u));
            }
            const c128 xi = shfl(y, i);
            if (lane < i) cfms(y, P[lane + (int64_t)i * rows], xi);
        }
        if (lane < bb) Di[lane + c * 32] = y;
    }
    __syncthreads();

    // ---- W = D^{-1} M_J: (rows J hold the swapped pivot rows, their J columns the identity) ----
    for (int c = warp; c < k; c += kZiWarps) {
        c128* xp = Xm + (int64_t)c * k + jb;
        const c128 xv = lane < bb ? xp[lane] : czero<double>();
        c128 acc = czero<double>();
        for (int s = 0; s < bb; ++s) {
            const c128 xs = shfl(xv, s);
            if (lane < bb) cfma(acc, Di[lane + s * 32], xs);
        }
        if (lane < bb) {
            xp[lane] = acc;
            Wt[lane + (int64_t)c * b] = acc;
        }
    }
    if (tid == 0 && s_sing) info[t] = 1;
}

// inv(A) = inv(P A) P: the interchanges of rows i <-> piv[i], undone on the columns from the last.
__global__ void zinv_unpermute_kernel(c128* X, int k, const int32_t* piv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (r >= k) return;
    c128* Xm = X + (int64_t)t * k * k;
    const int32_t* pv = piv + (int64_t)t * k;
    for (int i = k - 1; i >= 0; --i) {
        const int p = pv[i];
        if (p != i) {
            const c128 tmp = Xm[r + (int64_t)i * k];
            Xm[r + (int64_t)i * k] = Xm[r + (int64_t)p * k];
            Xm[r + (int64_t)p * k] = tmp;
        }
    }
}

}  // namespace

int zinv_block(int k) {
    for (int b : {32, 16, 8})
        if (panel_smem(k, std::min(b, k)) <= kZiSmemMax) return b;
    return 0;
}

size_t zinv_bytes_per_matrix(int k) {
    const int b = std::max(1, zinv_block(k));
    // M, E, W, pivots, and the emulated ZGEMM's digit images of E and W (about 3 KB per row)
    return (size_t)k * k * sizeof(c128) + (size_t)2 * k * b * sizeof(c128) + (size_t)k * 4 + (size_t)3072 * k + 256;
}

int zinv_batch(c128* X, int k, int batch, int32_t* info, cudaStream_t st) {
    const int b = zinv_block(k);
    if (b == 0) return set_error(RSRR_EUNSUPPORTED, "zinv_batch: matrix too large for shared-memory panels");
    if (k < 1 || batch < 1) return set_error(RSRR_EINVAL, "zinv_batch: empty problem");
    c128 *E = nullptr, *Wb = nullptr;
    int32_t* piv = nullptr;
    auto release = [&]() {
        dfree(E, st);
        dfree(Wb, st);
        dfree(piv, st);
    };
    int rc = RSRR_OK;
    if ((rc = dalloc_n(&E, (size_t)batch * k * b, st)) || (rc = dalloc_n(&Wb, (size_t)batch * b * k, st)) ||
        (rc = dalloc_n(&piv, (size_t)batch * k, st))) {
        release();
        return rc;
    }
    static bool attr_set = false;  // the same value every time
    if (!attr_set) {
        cudaFuncSetAttribute(zinv_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZiSmemMax);
        attr_set = true;
    }
    for (int jb = 0; jb < k && rc == RSRR_OK; jb += b) {
        const int bb = std::min(b, k - jb);
        { zinv_panel_kernel<<<batch, kZiThreads, panel_smem(k - jb, bb), st>>>(X, k, jb, bb, b, piv, E, Wb, info); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) {
            rc = set_error(RSRR_ECUDA, "zinv_panel_kernel launch");
            break;
        }
        Zgemm g;
        g.opA = OP_N; g.opB = OP_N; g.M = k; g.N = k; g.K = bb;
        g.alpha = mk<double>(-1.0, 0.0);
        g.beta = mk<double>(1.0, 0.0);
        g.A = E; g.lda = k; g.sA = (int64_t)k * b;
        g.B = Wb; g.ldb = b; g.sB = (int64_t)b * k;
        g.C = X; g.ldc = k; g.sC = (int64_t)k * k;
        g.batch = batch;
        rc = zgemm(g, st);
    }
    if (rc == RSRR_OK) {
        dim3 g((unsigned)ceil_div(k, 256), (unsigned)batch);
        { zinv_unpermute_kernel<<<g, 256, 0, st>>>(X, k, piv); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) rc = set_error(RSRR_ECUDA, "zinv_unpermute_kernel launch");
    }
    release();
    return rc;
}

}  // namespace rsrr
