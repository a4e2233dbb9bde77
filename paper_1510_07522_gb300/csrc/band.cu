// Band LU factorisation and blocked triangular solves (see band.cuh for the storage).
//
// Factorisation, per panel of nb columns starting at k0 (right-looking, blocked):
//   A. the panel's (nb + kl) x nb row block is staged in shared memory and factored with
//      partial pivoting by cabs1 = |re| + |im| (ties: lowest row), swapping whole panel rows
//      so the multipliers end in final pivot order; U11 goes back to the band array, the
//      whole block to lp, the composed row permutation to perm;
//   B. every trailing column the panel reaches (at most kv of them) gets, in one pass by
//      one warp for a group of CG columns: the panel's row permutation, U12 = L11^{-1} A12,
//      and A22 -= L21 U12.  Rows are spread over lanes (row q on lane q % 32) and processed
//      in chunks, so registers do not grow with the bandwidth.
// The forward solve reuses step B verbatim on the right-hand-side columns; the backward
// solve runs the same routine in reversed row order with a non-unit diagonal.
#include "band.cuh"

namespace rsrr {

namespace {

// ------------------------------------------------------------------------------------------
// Column accessors for apply_block (row q is relative to the block; c < CG within a group).
// ------------------------------------------------------------------------------------------
template <typename R, int CG>
struct TrailingCols {          // band columns c0 .. c0+CG-1 (< ce), rows k0 + q
    cplx<R>* ab;
    int ldab, kv, k0, c0, ce;
    __device__ __forceinline__ bool ok(int q, int c) const {
        int col = c0 + c, i = k0 + q;
        return col < ce && i >= col - kv;
    }
    __device__ __forceinline__ cplx<R>* ptr(int q, int c) const {
        int col = c0 + c, i = k0 + q;
        return ab + (int64_t)(kv + i - col) + (int64_t)col * ldab;
    }
    __device__ __forceinline__ cplx<R> load(int q, int c) const { return ok(q, c) ? *ptr(q, c) : czero<R>(); }
    __device__ __forceinline__ void store(int q, int c, cplx<R> v) const { if (ok(q, c)) *ptr(q, c) = v; }
};

template <typename R, int CG>
struct RhsCols {               // right-hand-side columns r0 .. r0+CG-1 (< L), rows row0 +/- q
    cplx<R>* x;
    int n, L, r0, row0, dir;   // dir = +1: row = row0 + q; dir = -1: row = row0 - q
    __device__ __forceinline__ cplx<R>* ptr(int q, int c) const {
        return x + (int64_t)(row0 + dir * q) + (int64_t)(r0 + c) * n;
    }
    __device__ __forceinline__ cplx<R> load(int q, int c) const { return (r0 + c < L) ? *ptr(q, c) : czero<R>(); }
    __device__ __forceinline__ void store(int q, int c, cplx<R> v) const { if (r0 + c < L) *ptr(q, c) = v; }
};

// ------------------------------------------------------------------------------------------
// One warp applies a factored block to CG columns:
//   rows 0..nbe-1   : triangular solve with the block's diagonal part (unit or not)
//   rows nbe..m-1   : x -= Blk[q, 0:nbe] * x[0:nbe]
// With a permutation, row q first takes the value of row perm[q]; for q >= nbe the source
// is q itself or a row < nbe (pivot rows only move up, displaced rows only move down), so the
// displaced values come from the slot-0 originals kept in registers.
// Blk, perm, invd are in shared memory; rows of Blk at or beyond m are never read.
// ------------------------------------------------------------------------------------------
template <typename R, int CG, int CH, bool UNIT, class Acc>
__device__ __forceinline__ void apply_block(const cplx<R>* __restrict__ Blk, int ld, int nbe, int m,
                                            const int* __restrict__ perm,
                                            const cplx<R>* __restrict__ invd,
                                            cplx<R>* __restrict__ ustash, const Acc& acc, int lane) {
    cplx<R> orig[CG], x0[CG];
    const bool v0 = lane < m;
#pragma unroll
    for (int c = 0; c < CG; ++c) orig[c] = v0 ? acc.load(lane, c) : czero<R>();
    int src0 = (perm && v0) ? perm[lane] : lane;
#pragma unroll
    for (int c = 0; c < CG; ++c) {
        cplx<R> sv = shfl(orig[c], src0 & 31);
        x0[c] = !v0 ? czero<R>() : (src0 < 32 ? sv : acc.load(src0, c));
    }
    // triangular part
    for (int t = 0; t < nbe; ++t) {
        if (!UNIT && lane == t) {
            const cplx<R> r = invd[t];
#pragma unroll
            for (int c = 0; c < CG; ++c) x0[c] = x0[c] * r;
        }
        cplx<R> u[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) u[c] = shfl(x0[c], t);
        if (lane > t && lane < nbe) {
            const cplx<R> l = Blk[lane + t * ld];
#pragma unroll
            for (int c = 0; c < CG; ++c) cfms(x0[c], l, u[c]);
        }
    }
    if (lane < nbe) {
#pragma unroll
        for (int c = 0; c < CG; ++c) ustash[lane * CG + c] = x0[c];
    }
    __syncwarp();
    if (lane >= nbe && v0) {
        for (int t = 0; t < nbe; ++t) {
            const cplx<R> l = Blk[lane + t * ld];
#pragma unroll
            for (int c = 0; c < CG; ++c) cfms(x0[c], l, ustash[t * CG + c]);
        }
    }
    if (v0) {
#pragma unroll
        for (int c = 0; c < CG; ++c) acc.store(lane, c, x0[c]);
    }
    // remaining rows, CH slots of 32 at a time
    for (int base = 32; base < m; base += 32 * CH) {
        cplx<R> x[CH][CG];
#pragma unroll
        for (int s = 0; s < CH; ++s) {
            const int q = base + 32 * s + lane;
            const bool vq = q < m;
            const int src = (perm && vq) ? perm[q] : q;
#pragma unroll
            for (int c = 0; c < CG; ++c) {
                cplx<R> sv = shfl(orig[c], src & 31);
                x[s][c] = !vq ? czero<R>() : (src < 32 ? sv : acc.load(q, c));
            }
        }
        for (int t = 0; t < nbe; ++t) {
            cplx<R> u[CG];
#pragma unroll
            for (int c = 0; c < CG; ++c) u[c] = ustash[t * CG + c];
#pragma unroll
            for (int s = 0; s < CH; ++s) {
                const int q = base + 32 * s + lane;
                const cplx<R> l = (q < m) ? Blk[q + t * ld] : czero<R>();
#pragma unroll
                for (int c = 0; c < CG; ++c) cfms(x[s][c], l, u[c]);
            }
        }
#pragma unroll
        for (int s = 0; s < CH; ++s) {
            const int q = base + 32 * s + lane;
            if (q < m) {
#pragma unroll
                for (int c = 0; c < CG; ++c) acc.store(q, c, x[s][c]);
            }
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// Factorisation kernel: one CTA per sampling point.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kLuThreads) band_factor_kernel(FactorArgs<R> a) {
    constexpr int CG = BandTraits<R>::CG, CH = BandTraits<R>::CH;
    constexpr int NW = kLuThreads / 32;
    const BandDims d = a.d;
    const int pt = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    cplx<R>* ab = a.ab + pt * a.ab_stride;
    cplx<R>* lp = a.lp + pt * a.lp_stride;
    int32_t* permg = a.perm + pt * a.perm_stride;
    int32_t* ipiv = a.ipiv + (int64_t)pt * d.n;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);
    int* psm = reinterpret_cast<int*>(P + (size_t)d.ldp * d.nb);
    cplx<R>* ust = reinterpret_cast<cplx<R>*>(psm + d.ldp);
    __shared__ int s_piv;
    __shared__ int s_info;
    if (tid == 0) s_info = 0;

    const int kv = d.kv, kl = d.kl, ldab = d.ldab, ldp = d.ldp, nb = d.nb, n = d.n;
    for (int p = 0; p < d.npanels; ++p) {
        const int k0 = p * nb;
        const int nbe = min(nb, n - k0);
        const int m = min(nb + kl, n - k0);
        // ---- A: stage and factor the panel -------------------------------------------
        for (int idx = tid; idx < ldp * nb; idx += kLuThreads) {
            const int q = idx % ldp, t = idx / ldp;
            cplx<R> v = czero<R>();
            const int dq = q - t;
            if (t < nbe && q < m && dq <= kl && dq >= -kv)
                v = ab[(int64_t)(kv + dq) + (int64_t)(k0 + t) * ldab];
            P[idx] = v;
        }
        for (int q = tid; q < ldp; q += kLuThreads) psm[q] = q;
        __syncthreads();
        for (int jj = 0; jj < nbe; ++jj) {
            const int last = min(jj + kl, m - 1);
            if (warp == 0) {
                R best = R(-1);
                int bi = jj;
                for (int q = jj + lane; q <= last; q += 32) {
                    const R v = cabs1(P[q + jj * ldp]);
                    if (v > best) { best = v; bi = q; }
                }
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    const R ob = __shfl_down_sync(0xffffffffu, best, off);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) s_piv = bi;
            }
            __syncthreads();
            const int pv = s_piv;
            if (pv != jj) {
                for (int t = tid; t < nb; t += kLuThreads) {
                    const cplx<R> tmp = P[jj + t * ldp];
                    P[jj + t * ldp] = P[pv + t * ldp];
                    P[pv + t * ldp] = tmp;
                }
                if (tid == 0) { const int tmp = psm[jj]; psm[jj] = psm[pv]; psm[pv] = tmp; }
            }
            __syncthreads();
            const cplx<R> piv = P[jj + jj * ldp];
            if (tid == 0) {
                ipiv[k0 + jj] = k0 + pv;
                if (cis_zero(piv) && s_info == 0) s_info = k0 + jj + 1;
            }
            if (!cis_zero(piv)) {
                const cplx<R> rp = crecip(piv);
                for (int q = jj + 1 + tid; q <= last; q += kLuThreads) P[q + jj * ldp] = P[q + jj * ldp] * rp;
                __syncthreads();
                const int nr = last - jj, nc = nbe - 1 - jj;
                for (int idx = tid; idx < nr * nc; idx += kLuThreads) {
                    const int q = jj + 1 + idx % nr, c = jj + 1 + idx / nr;
                    cfms(P[q + c * ldp], P[q + jj * ldp], P[jj + c * ldp]);
                }
            }
            __syncthreads();
        }
        // U11 back to the band, the whole block to lp, the permutation to perm
        for (int idx = tid; idx < nb * nb; idx += kLuThreads) {
            const int q = idx % nb, t = idx / nb;
            if (t < nbe && q <= t && t - q <= kv)
                ab[(int64_t)(kv + q - t) + (int64_t)(k0 + t) * ldab] = P[q + t * ldp];
        }
        cplx<R>* lpb = lp + (int64_t)p * ldp * nb;
        for (int idx = tid; idx < ldp * nb; idx += kLuThreads) lpb[idx] = P[idx];
        for (int q = tid; q < ldp; q += kLuThreads) permg[(int64_t)p * ldp + q] = psm[q];
        // ---- B: trailing columns ------------------------------------------------------
        const int cb = k0 + nbe, ce = min(n, k0 + nbe + kv);
        const int ntask = (ce - cb + CG - 1) / CG;
        for (int task = warp; task < ntask; task += NW) {
            TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
            apply_block<R, CG, CH, true>(P, ldp, nbe, m, psm, nullptr, ust + warp * 32 * CG, acc, lane);
        }
        __syncthreads();
    }
    if (tid == 0) a.info[pt] = s_info;
}

// ------------------------------------------------------------------------------------------
// Forward solve: X <- L^{-1} P X panel by panel, one CTA per point, one warp per CG columns.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kSolveThreads) band_fwd_kernel(SolveArgs<R> a) {
    constexpr int CG = BandTraits<R>::CG, CH = BandTraits<R>::CH;
    constexpr int NW = kSolveThreads / 32;
    const BandDims d = a.d;
    const int pt = blockIdx.x;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const cplx<R>* lp = a.lp + pt * a.lp_stride;
    const int32_t* permg = a.perm + pt * a.perm_stride;
    cplx<R>* x = a.x + pt * a.x_stride;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);
    int* psm = reinterpret_cast<int*>(P + (size_t)d.ldp * d.nb);
    cplx<R>* ust = reinterpret_cast<cplx<R>*>(psm + d.ldp);
    const int ldp = d.ldp, nb = d.nb, n = d.n;
    const int ntask = (a.L + CG - 1) / CG;
    for (int p = 0; p < d.npanels; ++p) {
        const int k0 = p * nb;
        const int nbe = min(nb, n - k0);
        const int m = min(nb + d.kl, n - k0);
        const cplx<R>* lpb = lp + (int64_t)p * ldp * nb;
        for (int idx = tid; idx < ldp * nb; idx += kSolveThreads) P[idx] = lpb[idx];
        for (int q = tid; q < ldp; q += kSolveThreads) psm[q] = permg[(int64_t)p * ldp + q];
        __syncthreads();
        for (int task = warp; task < ntask; task += NW) {
            RhsCols<R, CG> acc{x, n, a.L, task * CG, k0, +1};
            apply_block<R, CG, CH, true>(P, ldp, nbe, m, psm, nullptr, ust + warp * 32 * CG, acc, lane);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Backward solve: X <- U^{-1} X from the last block up.  Rows are taken in reversed order
// (block row k0+nbe-1 first), which turns U's block into a lower-triangular one.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kSolveThreads) band_bwd_kernel(SolveArgs<R> a) {
    constexpr int CG = BandTraits<R>::CG, CH = BandTraits<R>::CH;
    constexpr int NW = kSolveThreads / 32;
    const BandDims d = a.d;
    const int pt = blockIdx.x;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const cplx<R>* ab = a.ab + pt * a.ab_stride;
    cplx<R>* x = a.x + pt * a.x_stride;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* Ub = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* invd = Ub + (size_t)d.ldb * d.nbb;
    cplx<R>* ust = invd + 32;
    const int ldb = d.ldb, nbb = d.nbb, n = d.n, kv = d.kv, ldab = d.ldab;
    const int nblk = (n + nbb - 1) / nbb;
    const int ntask = (a.L + CG - 1) / CG;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int k0 = bk * nbb;
        const int nbe = min(nbb, n - k0);
        const int m = nbe + min(kv, k0);
        const int top = k0 + nbe - 1;  // reversed origin
        for (int idx = tid; idx < ldb * nbb; idx += kSolveThreads) {
            const int q = idx % ldb, t = idx / ldb;
            cplx<R> v = czero<R>();
            if (q < m && t < nbe) {
                const int i = top - q, c = top - t;
                if (i <= c && c - i <= kv) v = ab[(int64_t)(kv + i - c) + (int64_t)c * ldab];
            }
            Ub[idx] = v;
        }
        for (int t = tid; t < nbe; t += kSolveThreads) {
            const int c = top - t;
            invd[t] = crecip(ab[(int64_t)kv + (int64_t)c * ldab]);
        }
        __syncthreads();
        for (int task = warp; task < ntask; task += NW) {
            RhsCols<R, CG> acc{x, n, a.L, task * CG, top, -1};
            apply_block<R, CG, CH, false>(Ub, ldb, nbe, m, nullptr, invd, ust + warp * 32 * CG, acc, lane);
        }
        __syncthreads();
    }
}

}  // namespace

template <typename R>
int launch_factor(const FactorArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = factor_smem_bytes<R>(a.d);
    RSRR_CUDA(cudaFuncSetAttribute(band_factor_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { band_factor_kernel<R><<<npts, kLuThreads, sm, s>>>(a); note_launch(); }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template <typename R>
int launch_fwd(const SolveArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = fwd_smem_bytes<R>(a.d);
    RSRR_CUDA(cudaFuncSetAttribute(band_fwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { band_fwd_kernel<R><<<npts, kSolveThreads, sm, s>>>(a); note_launch(); }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template <typename R>
int launch_bwd(const SolveArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = bwd_smem_bytes<R>(a.d);
    RSRR_CUDA(cudaFuncSetAttribute(band_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { band_bwd_kernel<R><<<npts, kSolveThreads, sm, s>>>(a); note_launch(); }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template int launch_factor<float>(const FactorArgs<float>&, int, cudaStream_t);
template int launch_factor<double>(const FactorArgs<double>&, int, cudaStream_t);
template int launch_fwd<float>(const SolveArgs<float>&, int, cudaStream_t);
template int launch_fwd<double>(const SolveArgs<double>&, int, cudaStream_t);
template int launch_bwd<float>(const SolveArgs<float>&, int, cudaStream_t);
template int launch_bwd<double>(const SolveArgs<double>&, int, cudaStream_t);

}  // namespace rsrr
