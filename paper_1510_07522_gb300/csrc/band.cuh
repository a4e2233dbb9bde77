// Blocked complex band LU with partial pivoting and the blocked triangular solves that use
// its factors (Algorithm 2, Step 2: Y_i = T(z_i)^{-1} U).  One CTA owns one sampling point.
//
// Storage of one point's factorisation:
//   ab    general-band array, column-major, ldab = 2 kl + ku + 1, A(i, c) at
//         ab[(kv + i - c) + c * ldab] with kv = kl + ku.  On exit the rows i <= c of each
//         column hold U (upper bandwidth kv once pivoting fill is counted).
//   lp    one (ldp x nb) block per panel of nb columns: the panel after factorisation with
//         its rows in final pivot order (unit lower L11 and L21 below the diagonal), so a
//         solve applies a panel's row permutation once and then two dense products.
//   perm  per panel, ldp entries: final position q of the panel's row block holds the row
//         that started at relative position perm[q].
//   ipiv  LAPACK-style pivot rows (absolute, 0-based) for reporting.
#pragma once

#include "common.cuh"

namespace rsrr {

struct BandDims {
    int n = 0, kl = 0, ku = 0, kv = 0;
    int ldab = 0;
    int nb = 0;    // panel width of the factorisation (<= 32)
    int ldp = 0;   // rows of a panel block: multiple of 32, >= nb + kl
    int npanels = 0;
    int nbb = 0;   // block width of the backward solve (<= 32)
    int ldb = 0;   // rows of a backward block: multiple of 32, >= nbb + kv
    int fwd_nbuf = 1, bwd_nbuf = 1;  // staging buffers of the solves (2 = copy-ahead)
};

template <typename R>
struct FactorArgs {
    BandDims d;
    cplx<R>* ab;
    int64_t ab_stride;
    cplx<R>* lp;
    int64_t lp_stride;
    int32_t* perm;
    int64_t perm_stride;
    int32_t* ipiv;   // [pts][n]
    int32_t* info;   // [pts] first zero pivot column (1-based), 0 if none
};

template <typename R>
struct SolveArgs {
    BandDims d;
    const cplx<R>* ab;
    int64_t ab_stride;
    const cplx<R>* lp;
    int64_t lp_stride;
    const int32_t* perm;
    int64_t perm_stride;
    cplx<R>* x;       // [pts][L][n] right-hand sides, overwritten by the solution
    int64_t x_stride;
    int L;
    const int32_t* active;  // [pts] 0 = skip this point (already converged); may be null
    int split = 1;          // CTAs per point; CTA r of a point takes a contiguous share of the columns
};

template <typename R> struct BandTraits;
template <> struct BandTraits<float> { static constexpr int CG = 4; static constexpr int CH = 4; };
template <> struct BandTraits<double> { static constexpr int CG = 2; static constexpr int CH = 4; };
// The solves give each warp fewer right-hand-side columns (more warps share a block), which
// shortens the per-block critical path of the serial triangular part.
template <typename R> struct SolveTraits;
template <> struct SolveTraits<float> { static constexpr int CG = 1; static constexpr int CH = 4; };
template <> struct SolveTraits<double> { static constexpr int CG = 1; static constexpr int CH = 4; };

constexpr int kLuThreads = 512;
constexpr int kSolveThreads = 512;

template <typename R>
size_t factor_smem_bytes(const BandDims& d) {  // two panel buffers (look-ahead) + per-warp stash
    return 2 * ((size_t)d.ldp * d.nb * sizeof(cplx<R>) + (size_t)d.ldp * sizeof(int)) +
           (size_t)(kLuThreads / 32) * 32 * BandTraits<R>::CG * sizeof(cplx<R>) + 64;
}
template <typename R>
size_t fwd_smem_bytes(const BandDims& d, int nbuf) {
    return (size_t)nbuf * ((size_t)d.ldp * d.nb * sizeof(cplx<R>) + (size_t)d.ldp * sizeof(int)) +
           (size_t)(kSolveThreads / 32) * 32 * SolveTraits<R>::CG * sizeof(cplx<R>) + 64;
}
template <typename R>
size_t bwd_smem_bytes(const BandDims& d, int nbuf) {
    return (size_t)nbuf * d.ldb * d.nbb * sizeof(cplx<R>) + (size_t)32 * sizeof(cplx<R>) +
           (size_t)(kSolveThreads / 32) * 32 * SolveTraits<R>::CG * sizeof(cplx<R>) + 64;
}

// Panel sizes for a band of (kl, ku) that fit the shared-memory budget.
int pick_dims(int64_t n, int64_t kl, int64_t ku, bool is_c64, BandDims* d);

template <typename R>
int launch_factor(const FactorArgs<R>& a, int npts, cudaStream_t s);
template <typename R>
int launch_fwd(const SolveArgs<R>& a, int npts, cudaStream_t s);
template <typename R>
int launch_bwd(const SolveArgs<R>& a, int npts, cudaStream_t s);

}  // namespace rsrr
