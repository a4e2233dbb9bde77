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
#include <cooperative_groups.h>

#include "band.cuh"

namespace rsrr {

namespace {

// ------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async), used to stage the next block of a solve
// while the current one is applied.  src_bytes = 0 fills the destination with zeros.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
template <typename R>
__device__ __forceinline__ void cp_async_elem(cplx<R>* smem, const cplx<R>* gmem, bool valid) {
    if (sizeof(cplx<R>) == 16) cp_async_16(smem, gmem, valid ? 16 : 0);
    else cp_async_8(smem, gmem, valid ? 8 : 0);
}

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
// Factorisation kernel: one CTA per sampling point, with look-ahead.
//   warps 0..3  (panel team): factor panel p+1 into the second shared buffer
//   warps 4..15 (update team): during step p first update the columns of panel p+1, signal
//                the panel team (named barrier 2: the team waits, the update warps arrive),
//                then update the rest of step p's trailing columns.
// Step p ends with a CTA-wide barrier, after which panel p+1 is complete in its buffer.
// Barrier ids: 0 = __syncthreads, 1 = panel team only (128 threads), 2 = lead signal (512).
// Every thread reaches each barrier exactly once per step, whatever the sizes.
// ------------------------------------------------------------------------------------------
constexpr int kPanelWarps = 4;
constexpr int kUpdateWarps = kLuThreads / 32 - kPanelWarps;

__device__ __forceinline__ void team_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kPanelWarps * 32) : "memory"); }
__device__ __forceinline__ void lead_wait() { asm volatile("bar.sync 2, %0;" ::"n"(kLuThreads) : "memory"); }
__device__ __forceinline__ void lead_arrive() { asm volatile("bar.arrive 2, %0;" ::"n"(kLuThreads) : "memory"); }

// Panel factorisation by the panel team (kPanelWarps warps), two team barriers per column:
//   S: rows jj and pv swapped in every panel column but jj; column jj gets the pivot and the
//      multipliers (one thread owns rows jj and pv of that column, so no value is read after
//      another thread overwrote it); the pivot value comes from the search warp.
//   R: rank-1 update, warp w owning columns jj+1+w, jj+1+w+W, ... and lanes owning rows; warp 0
//      owns column jj+1, updates it first and then searches the next pivot in it.
// Multipliers stay in final pivot order (whole panel rows are swapped).
template <typename R>
__device__ __forceinline__ void pivot_search(const cplx<R>* P, int ldp, int col, int first, int last, int lane,
                                             int* s_piv, cplx<R>* s_pval) {
    R best = R(-1);
    int bi = first;
    for (int q = first + lane; q <= last; q += 32) {
        const R v = cabs1(P[q + col * ldp]);
        if (v > best) { best = v; bi = q; }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const R ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
        *s_piv = bi;
        *s_pval = P[bi + col * ldp];
    }
}

template <typename R>
__device__ void factor_panel(const FactorArgs<R>& a, cplx<R>* ab, cplx<R>* lp, int32_t* permg, int32_t* ipiv,
                             int p, cplx<R>* P, int* psm, int* s_piv, cplx<R>* s_pval, int* s_info) {
    constexpr int PT = kPanelWarps * 32;
    const BandDims& d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kv = d.kv, kl = d.kl, ldab = d.ldab, ldp = d.ldp, nb = d.nb, n = d.n;
    const int k0 = p * nb;
    const int nbe = min(nb, n - k0);
    const int m = min(nb + kl, n - k0);
    // stage the panel with cp.async (every load in flight at once; zero fill outside the band)
    for (int t = warp; t < nb; t += kPanelWarps) {  // one warp per column: no index division
        const int col = k0 + t;
        for (int q = lane; q < ldp; q += 32) {
            const int dq = q - t;
            const bool valid = t < nbe && q < m && dq <= kl && dq >= -kv;
            const cplx<R>* src = valid ? ab + (int64_t)(kv + dq) + (int64_t)col * ldab : ab;
            cp_async_elem<R>(P + q + t * ldp, src, valid);
        }
    }
    cp_async_commit();
    for (int q = tid; q < ldp; q += PT) psm[q] = q;
    cp_async_wait<0>();
    team_sync();
    if (warp == 0) pivot_search(P, ldp, 0, 0, min(kl, m - 1), lane, s_piv, s_pval);
    team_sync();
    for (int jj = 0; jj < nbe; ++jj) {
        const int last = min(jj + kl, m - 1);
        const int pv = *s_piv;
        const cplx<R> piv = *s_pval;
        const bool nz = !cis_zero(piv);
        const cplx<R> rp = nz ? crecip(piv) : czero<R>();
        // ---- S: swap (columns != jj) and column jj (pivot + multipliers) --------------------
        if (pv != jj) {
            for (int t = tid; t < nb; t += PT) {
                if (t == jj) continue;
                const cplx<R> tmp = P[jj + t * ldp];
                P[jj + t * ldp] = P[pv + t * ldp];
                P[pv + t * ldp] = tmp;
            }
        }
        for (int q = jj + tid; q <= last; q += PT) {
            if (q == jj) {
                const cplx<R> old = P[jj + jj * ldp];
                P[jj + jj * ldp] = piv;
                if (pv != jj) P[pv + jj * ldp] = nz ? old * rp : old;
            } else if (q != pv && nz) {
                P[q + jj * ldp] = P[q + jj * ldp] * rp;
            }
        }
        if (tid == 0) {
            if (pv != jj) { const int tmp = psm[jj]; psm[jj] = psm[pv]; psm[pv] = tmp; }
            ipiv[k0 + jj] = k0 + pv;
            if (!nz && *s_info == 0) *s_info = k0 + jj + 1;
        }
        team_sync();
        // ---- R: rank-1 update of columns jj+1..nbe-1 ----------------------------------------
        if (nz) {
            for (int c = jj + 1 + warp; c < nbe; c += kPanelWarps) {
                const cplx<R> u = P[jj + c * ldp];
                if (!cis_zero(u))
                    for (int q = jj + 1 + lane; q <= last; q += 32) cfms(P[q + c * ldp], P[q + jj * ldp], u);
                if (c == jj + 1) {  // warp 0: the next pivot column is complete
                    __syncwarp();
                    pivot_search(P, ldp, jj + 1, jj + 1, min(jj + 1 + kl, m - 1), lane, s_piv, s_pval);
                }
            }
        } else if (warp == 0 && jj + 1 < nbe) {
            pivot_search(P, ldp, jj + 1, jj + 1, min(jj + 1 + kl, m - 1), lane, s_piv, s_pval);
        }
        team_sync();
    }
    for (int t = warp; t < nbe; t += kPanelWarps) {  // U11 back to the band
        for (int q = lane; q <= t; q += 32)
            if (t - q <= kv) ab[(int64_t)(kv + q - t) + (int64_t)(k0 + t) * ldab] = P[q + t * ldp];
    }
    cplx<R>* lpb = lp + (int64_t)p * ldp * nb;
    for (int idx = tid; idx < ldp * nb; idx += PT) lpb[idx] = P[idx];
    for (int q = tid; q < ldp; q += PT) permg[(int64_t)p * ldp + q] = psm[q];
}

template <typename R>
__global__ void __launch_bounds__(kLuThreads) band_factor_kernel(FactorArgs<R> a) {
    constexpr int CG = BandTraits<R>::CG, CH = BandTraits<R>::CH;
    const BandDims d = a.d;
    const int pt = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    cplx<R>* ab = a.ab + pt * a.ab_stride;
    cplx<R>* lp = a.lp + pt * a.lp_stride;
    int32_t* permg = a.perm + pt * a.perm_stride;
    int32_t* ipiv = a.ipiv + (int64_t)pt * d.n;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int blk = d.ldp * d.nb;
    cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);                 // [2][blk]
    int* psm = reinterpret_cast<int*>(P + 2 * (size_t)blk);            // [2][ldp]
    cplx<R>* ust = reinterpret_cast<cplx<R>*>(psm + 2 * (size_t)d.ldp);  // [kUpdateWarps][32*CG]
    __shared__ int s_piv;
    __shared__ int s_info;
    __shared__ cplx<R> s_pval;
    if (tid == 0) s_info = 0;
    __syncthreads();

    const int kv = d.kv, ldab = d.ldab, ldp = d.ldp, nb = d.nb, n = d.n;
    if (warp < kPanelWarps) factor_panel<R>(a, ab, lp, permg, ipiv, 0, P, psm, &s_piv, &s_pval, &s_info);
    __syncthreads();
    for (int p = 0; p < d.npanels; ++p) {
        const int k0 = p * nb;
        const int nbe = min(nb, n - k0);
        const int m = min(nb + d.kl, n - k0);
        const int buf = p & 1;
        const int cb = k0 + nbe, ce = min(n, k0 + nbe + kv);
        const int ntask = max(0, (ce - cb + CG - 1) / CG);
        const bool has_next = p + 1 < d.npanels;
        const int nlead = has_next ? min(ntask, (nb + CG - 1) / CG) : 0;
        if (warp >= kPanelWarps) {
            const int uw = warp - kPanelWarps;
            cplx<R>* Pb = P + (size_t)buf * blk;
            int* pb = psm + (size_t)buf * ldp;
            for (int task = uw; task < nlead; task += kUpdateWarps) {
                TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
                apply_block<R, CG, CH, true>(Pb, ldp, nbe, m, pb, nullptr, ust + uw * 32 * CG, acc, lane);
            }
            __threadfence_block();
            lead_arrive();
            for (int task = nlead + uw; task < ntask; task += kUpdateWarps) {
                TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
                apply_block<R, CG, CH, true>(Pb, ldp, nbe, m, pb, nullptr, ust + uw * 32 * CG, acc, lane);
            }
        } else {
            lead_wait();
            if (has_next)
                factor_panel<R>(a, ab, lp, permg, ipiv, p + 1, P + (size_t)(buf ^ 1) * blk, psm + (size_t)(buf ^ 1) * ldp,
                                &s_piv, &s_pval, &s_info);
        }
        __syncthreads();
    }
    if (tid == 0) a.info[pt] = s_info;
}

// ------------------------------------------------------------------------------------------
// Cluster variant: two CTAs (one thread-block cluster) per sampling point, so a batch of N
// points keeps 2N SMs busy.
//   CTA 0: panel team (warps 0..3) + update team (warps 4..15), exactly as above; its update
//          warps do the lead tasks (columns of the next panel) and a share of the rest.
//   CTA 1: 16 update warps; at the start of each step it copies the finished panel block and
//          its permutation from CTA 0's shared memory (distributed shared memory), then does
//          the remaining share of the trailing columns.
// Each step ends with a cluster barrier (release/acquire), which also orders both CTAs'
// updates of the band in global memory before the next step reads them.  Every thread of
// both CTAs reaches it exactly once per step and once after the prologue.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kLuThreads) band_factor_cluster_kernel(FactorArgs<R> a) {
    namespace cg = cooperative_groups;
    constexpr int CG = BandTraits<R>::CG, CH = BandTraits<R>::CH;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const BandDims d = a.d;
    const int pt = blockIdx.x / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    cplx<R>* ab = a.ab + pt * a.ab_stride;
    cplx<R>* lp = a.lp + pt * a.lp_stride;
    int32_t* permg = a.perm + pt * a.perm_stride;
    int32_t* ipiv = a.ipiv + (int64_t)pt * d.n;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int blk = d.ldp * d.nb;
    cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);                 // [2][blk]
    int* psm = reinterpret_cast<int*>(P + 2 * (size_t)blk);            // [2][ldp]
    cplx<R>* ust = reinterpret_cast<cplx<R>*>(psm + 2 * (size_t)d.ldp);  // per update warp
    __shared__ int s_piv;
    __shared__ int s_info;
    __shared__ cplx<R> s_pval;
    if (tid == 0) s_info = 0;
    __syncthreads();

    const int kv = d.kv, ldab = d.ldab, ldp = d.ldp, nb = d.nb, n = d.n;
    if (rank == 0 && warp < kPanelWarps) factor_panel<R>(a, ab, lp, permg, ipiv, 0, P, psm, &s_piv, &s_pval, &s_info);
    cluster.sync();
    for (int p = 0; p < d.npanels; ++p) {
        const int k0 = p * nb;
        const int nbe = min(nb, n - k0);
        const int m = min(nb + d.kl, n - k0);
        const int buf = p & 1;
        const int cb = k0 + nbe, ce = min(n, k0 + nbe + kv);
        const int ntask = max(0, (ce - cb + CG - 1) / CG);
        const bool has_next = p + 1 < d.npanels;
        const int nlead = has_next ? min(ntask, (nb + CG - 1) / CG) : 0;
        const int rest = ntask - nlead;
        const int n1 = (rest * 3) / 5;  // CTA 1's share of the non-lead columns
        cplx<R>* Pb = P + (size_t)buf * blk;
        int* pb = psm + (size_t)buf * ldp;
        if (rank == 1) {
            // copy panel p (block and permutation) from CTA 0's shared memory
            const cplx<R>* rP = cluster.map_shared_rank(Pb, 0);
            const int* rpb = cluster.map_shared_rank(pb, 0);
            for (int idx = tid; idx < blk; idx += kLuThreads) Pb[idx] = rP[idx];
            for (int q = tid; q < ldp; q += kLuThreads) pb[q] = rpb[q];
            __syncthreads();
            for (int task = nlead + warp; task < nlead + n1; task += kLuThreads / 32) {
                TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
                apply_block<R, CG, CH, true>(Pb, ldp, nbe, m, pb, nullptr, ust + warp * 32 * CG, acc, lane);
            }
        } else if (warp >= kPanelWarps) {
            const int uw = warp - kPanelWarps;
            for (int task = uw; task < nlead; task += kUpdateWarps) {
                TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
                apply_block<R, CG, CH, true>(Pb, ldp, nbe, m, pb, nullptr, ust + uw * 32 * CG, acc, lane);
            }
            __threadfence_block();
            lead_arrive();
            for (int task = nlead + n1 + uw; task < ntask; task += kUpdateWarps) {
                TrailingCols<R, CG> acc{ab, ldab, kv, k0, cb + task * CG, ce};
                apply_block<R, CG, CH, true>(Pb, ldp, nbe, m, pb, nullptr, ust + uw * 32 * CG, acc, lane);
            }
        } else {
            lead_wait();
            if (has_next)
                factor_panel<R>(a, ab, lp, permg, ipiv, p + 1, P + (size_t)(buf ^ 1) * blk, psm + (size_t)(buf ^ 1) * ldp,
                                &s_piv, &s_pval, &s_info);
        }
        cluster.sync();
    }
    if (rank == 0 && tid == 0) a.info[pt] = s_info;
}

// ------------------------------------------------------------------------------------------
// Forward solve: X <- L^{-1} P X panel by panel, one CTA per point, one warp per CG columns.
// The next panel's L block and permutation are staged with cp.async while the current one
// is applied (two buffers when they fit in shared memory).
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kSolveThreads) band_fwd_kernel(SolveArgs<R> a) {
    constexpr int CG = SolveTraits<R>::CG, CH = SolveTraits<R>::CH;
    constexpr int NW = kSolveThreads / 32;
    const BandDims d = a.d;
    const int pt = blockIdx.x / a.split, part = blockIdx.x % a.split;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const cplx<R>* lp = a.lp + pt * a.lp_stride;
    const int32_t* permg = a.perm + pt * a.perm_stride;
    const int c_lo = (int)((int64_t)a.L * part / a.split), c_hi = (int)((int64_t)a.L * (part + 1) / a.split);
    cplx<R>* x = a.x + pt * a.x_stride + (int64_t)c_lo * d.n;
    const int Lp = c_hi - c_lo;
    const int ldp = d.ldp, nb = d.nb, n = d.n, nbuf = d.fwd_nbuf;
    const int blk = ldp * nb;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);
    int* psm = reinterpret_cast<int*>(P + (size_t)nbuf * blk);
    cplx<R>* ust = reinterpret_cast<cplx<R>*>(psm + (size_t)nbuf * ldp);
    auto stage = [&](int p, int buf) {
        const char* src = reinterpret_cast<const char*>(lp + (int64_t)p * blk);
        char* dst = reinterpret_cast<char*>(P + (size_t)buf * blk);
        const int nch = blk * (int)sizeof(cplx<R>) / 16;
        for (int c = tid; c < nch; c += kSolveThreads) cp_async_16(dst + 16 * c, src + 16 * c, 16);
        const char* ps = reinterpret_cast<const char*>(permg + (int64_t)p * ldp);
        char* pd = reinterpret_cast<char*>(psm + (size_t)buf * ldp);
        for (int c = tid; c < ldp / 4; c += kSolveThreads) cp_async_16(pd + 16 * c, ps + 16 * c, 16);
        cp_async_commit();
    };
    const int ntask = (Lp + CG - 1) / CG;
    stage(0, 0);
    for (int p = 0; p < d.npanels; ++p) {
        const int k0 = p * nb;
        const int nbe = min(nb, n - k0);
        const int m = min(nb + d.kl, n - k0);
        const bool ahead = nbuf == 2 && p + 1 < d.npanels;
        if (ahead) {
            stage(p + 1, (p + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int buf = nbuf == 2 ? (p & 1) : 0;
        for (int task = warp; task < ntask; task += NW) {
            RhsCols<R, CG> acc{x, n, Lp, task * CG, k0, +1};
            apply_block<R, CG, CH, true>(P + (size_t)buf * blk, ldp, nbe, m, psm + (size_t)buf * ldp, nullptr,
                                         ust + warp * 32 * CG, acc, lane);
        }
        __syncthreads();
        if (nbuf == 1 && p + 1 < d.npanels) stage(p + 1, 0);
    }
}

// ------------------------------------------------------------------------------------------
// Backward solve: X <- U^{-1} X from the last block up.  Rows are taken in reversed order
// (block row k0+nbe-1 first), which turns U's block into a lower-triangular one.  The next
// block's U entries are gathered from the band array with cp.async (zero-filled outside the
// band) while the current block is applied.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kSolveThreads) band_bwd_kernel(SolveArgs<R> a) {
    constexpr int CG = SolveTraits<R>::CG, CH = SolveTraits<R>::CH;
    constexpr int NW = kSolveThreads / 32;
    const BandDims d = a.d;
    const int pt = blockIdx.x / a.split, part = blockIdx.x % a.split;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const cplx<R>* ab = a.ab + pt * a.ab_stride;
    const int c_lo = (int)((int64_t)a.L * part / a.split), c_hi = (int)((int64_t)a.L * (part + 1) / a.split);
    cplx<R>* x = a.x + pt * a.x_stride + (int64_t)c_lo * d.n;
    const int Lp = c_hi - c_lo;
    const int ldb = d.ldb, nbb = d.nbb, n = d.n, kv = d.kv, ldab = d.ldab, nbuf = d.bwd_nbuf;
    const int blk = ldb * nbb;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* Ub = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* invd = Ub + (size_t)nbuf * blk;
    cplx<R>* ust = invd + 32;
    const int nblk = (n + nbb - 1) / nbb;
    auto stage = [&](int bk, int buf) {
        const int k0 = bk * nbb;
        const int nbe = min(nbb, n - k0);
        const int m = nbe + min(kv, k0);
        const int top = k0 + nbe - 1;
        cplx<R>* dst = Ub + (size_t)buf * blk;
        for (int idx = tid; idx < blk; idx += kSolveThreads) {
            const int q = idx % ldb, t = idx / ldb;
            const int i = top - q, c = top - t;
            const bool valid = q < m && t < nbe && i <= c && c - i <= kv;
            const cplx<R>* src = valid ? ab + (int64_t)(kv + i - c) + (int64_t)c * ldab : ab;
            cp_async_elem<R>(dst + idx, src, valid);
        }
        cp_async_commit();
    };
    const int ntask = (Lp + CG - 1) / CG;
    stage(nblk - 1, 0);
    for (int bk = nblk - 1, it = 0; bk >= 0; --bk, ++it) {
        const int k0 = bk * nbb;
        const int nbe = min(nbb, n - k0);
        const int m = nbe + min(kv, k0);
        const int top = k0 + nbe - 1;
        const bool ahead = nbuf == 2 && bk > 0;
        if (ahead) {
            stage(bk - 1, (it + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int buf = nbuf == 2 ? (it & 1) : 0;
        cplx<R>* U = Ub + (size_t)buf * blk;
        for (int t = tid; t < nbe; t += kSolveThreads) invd[t] = crecip(U[t + t * ldb]);
        __syncthreads();
        for (int task = warp; task < ntask; task += NW) {
            RhsCols<R, CG> acc{x, n, Lp, task * CG, top, -1};
            apply_block<R, CG, CH, false>(U, ldb, nbe, m, nullptr, invd, ust + warp * 32 * CG, acc, lane);
        }
        __syncthreads();
        if (nbuf == 1 && bk > 0) stage(bk - 1, 0);
    }
}

}  // namespace

namespace {
// Opt a kernel into `sm` bytes of dynamic shared memory, with a readable error when the
// request plus the kernel's static shared memory exceeds the device's per-block limit.
template <typename K>
int set_smem(K kernel, size_t sm, const char* name) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    if (sm + fa.sharedSizeBytes > (size_t)optin)
        return set_error(RSRR_EUNSUPPORTED, std::string(name) + ": shared memory " + std::to_string(sm) + " + " +
                                                std::to_string(fa.sharedSizeBytes) + " exceeds " + std::to_string(optin));
    // The attribute is per function and process-wide: set it to the largest allowed value (not
    // to this launch's size), so that host threads launching the same kernel with different
    // sizes never lower it under one another's launch.
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess)
        return set_error(RSRR_ECUDA, std::string(name) + ": cudaFuncSetAttribute(" + std::to_string(sm) + ", static " +
                                         std::to_string(fa.sharedSizeBytes) + ", optin " + std::to_string(optin) +
                                         "): " + cudaGetErrorString(e));
    return RSRR_OK;
}
}  // namespace

// CTAs per point for the solves: two when the doubled grid still fits one wave, so the
// right-hand-side columns of a point are shared by two SMs.
int solve_split(int npts, int L) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (L >= 2 && 2 * npts <= nsm) ? 2 : 1;
}

template <typename R>
int launch_factor(const FactorArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = factor_smem_bytes<R>(a.d);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (2 * npts <= nsm) {  // few points: two SMs per point
        RSRR_TRY(set_smem(band_factor_cluster_kernel<R>, sm, "band_factor_cluster_kernel"));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * npts, 1, 1);
        cfg.blockDim = dim3(kLuThreads, 1, 1);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        RSRR_CUDA(cudaLaunchKernelEx(&cfg, band_factor_cluster_kernel<R>, a));
        note_launch();
        return RSRR_OK;
    }
    RSRR_TRY(set_smem(band_factor_kernel<R>, sm, "band_factor_kernel"));
    { band_factor_kernel<R><<<npts, kLuThreads, sm, s>>>(a); note_launch(); }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template <typename R>
int launch_fwd(const SolveArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = fwd_smem_bytes<R>(a.d, a.d.fwd_nbuf);
    RSRR_TRY(set_smem(band_fwd_kernel<R>, sm, "band_fwd_kernel"));
    SolveArgs<R> b = a;
    b.split = solve_split(npts, a.L);
    { band_fwd_kernel<R><<<npts * b.split, kSolveThreads, sm, s>>>(b); note_launch(); }
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

template <typename R>
int launch_bwd(const SolveArgs<R>& a, int npts, cudaStream_t s) {
    const size_t sm = bwd_smem_bytes<R>(a.d, a.d.bwd_nbuf);
    RSRR_TRY(set_smem(band_bwd_kernel<R>, sm, "band_bwd_kernel"));
    SolveArgs<R> b = a;
    b.split = solve_split(npts, a.L);
    { band_bwd_kernel<R><<<npts * b.split, kSolveThreads, sm, s>>>(b); note_launch(); }
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
