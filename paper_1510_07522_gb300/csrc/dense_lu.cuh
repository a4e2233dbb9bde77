// Dense complex LU with partial pivoting and the triangular solves that use it, for sampling
// points whose T(z_j) has no usable band (Algorithm 2, Step 2: Y_j = T(z_j)^{-1} U, with T
// dense or with a band as wide as n, e.g. the time-delay NEPs whose delay term is a random
// sparse matrix).
//
// One CTA owns one sampling point for the whole factorisation: a persistent launch hands out
// points largest-first from a device counter, so a batch of uneven problems (many NEPs of
// different n, all their points) runs in one launch without cross-CTA synchronisation.
//
// Storage of one point:
//   a      n x n column-major, leading dimension lda.  On exit the upper triangle holds U and
//          the strict lower triangle the multipliers of L, panel by panel: the rows of panel
//          p's multipliers are in the order reached after panel p's own interchanges (later
//          interchanges are applied to the right-hand side during the solve, not to stored L).
//   ipiv   LAPACK-style pivot rows (absolute, 0-based).
//   swaps  per panel of kDenseNB columns: the panel's interchanges composed into one
//          permutation of the rows it touches: count c, then rows[2 NB], then src[2 NB]; row
//          k0 + rows[e] receives the contents of row k0 + src[e].  Entries 0..nbk-1 are the
//          panel's own diagonal rows.
//   inv    per panel: inv(L11) and inv(U11) of its nbk x nbk diagonal block (column-major,
//          leading dimension kDenseNB), so each block solve is one small product.
#pragma once

#include "common.cuh"

namespace rsrr {

constexpr int kDenseNB = 64;        // panel width (K depth of the trailing update)
constexpr int kDenseThreads = 256;  // threads per CTA (one CTA per point)
constexpr int kDenseSwapInts = 1 + 4 * kDenseNB;

__host__ __device__ inline int64_t dense_panels(int64_t n) { return (n + kDenseNB - 1) / kDenseNB; }

template <typename R>
struct DenseJob {
    cplx<R>* a;              // [n][lda] column-major
    int64_t lda;
    int32_t n;
    int32_t L;               // right-hand sides (solve)
    int32_t* ipiv;           // [n]
    int32_t* info;           // [1]: first zero pivot (1-based), 0 if none
    cplx<R>* inv;            // [npanels][2][NB * NB]
    int32_t* swaps;          // [npanels][kDenseSwapInts]
    cplx<R>* x;              // [L][n] right-hand sides, overwritten by the solution (solve)
    const int32_t* active;   // solve: the point is skipped when *active == 0 (may be null)
};

// Device bytes of the per-point work arrays besides a, x and ipiv.
template <typename R>
inline size_t dense_aux_bytes(int64_t n) {
    return (size_t)dense_panels(n) * (2 * kDenseNB * kDenseNB * sizeof(cplx<R>) + kDenseSwapInts * 4);
}

// Factor every job (any order of sizes; the launcher expects them sorted largest first so
// the last CTAs to finish hold the smallest points).  d_next: one int32 of device scratch.
// Complex64 runs the trailing updates on the tensor cores and needs d_img: device scratch of
// dense_factor_grid(njobs) * dense_image_floats(n_max) floats (n_max = the largest job's n);
// complex128 ignores it.  A job whose tensor-core waits time out gets *info = -1.
template <typename R>
int dense_factor_grid(int njobs);
template <typename R>
size_t dense_image_floats(int n_max);
template <typename R>
int launch_dense_factor(const DenseJob<R>* d_jobs, int njobs, int n_max, int32_t* d_next, float* d_img,
                        cudaStream_t s);
// X = A^{-1} X for every job (forward with the composed interchanges, then backward).
template <typename R>
int launch_dense_solve(const DenseJob<R>* d_jobs, int njobs, int maxL, cudaStream_t s);

}  // namespace rsrr
