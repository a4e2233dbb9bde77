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

// The factor and solve of one point (one CTA's slot).
template <typename R>
struct DenseJob {
    cplx<R>* a;              // [n][lda] column-major
    int64_t lda;
    int32_t n;
    int32_t L;               // right-hand sides (solve)
    int32_t* ipiv;           // [n]
    cplx<R>* inv;            // [npanels][2][NB * NB]
    int32_t* swaps;          // [npanels][kDenseSwapInts]
    cplx<R>* x;              // [L][n] right-hand sides, overwritten by the solution (solve)
};

// ---- fused dense sampling: one persistent launch for all points of a set of NEPs --------------
// Each CTA takes (NEP, point) jobs largest n first and, in a memory slot of its own, assembles
// T(z_j), factors it, solves T X = U, computes the FP64 residual and backward error and refines
// until the stopping rule of the band path holds, writing X into the NEP's S_hat.
struct DenseNep {
    int32_t n, J, L, N;
    int64_t nnz;
    const int64_t* rowptr;   // CSR of the union pattern (band ordering)
    const int32_t* colind;
    const int32_t* rowidx;
    const c128* vals;        // [J][nnz]
    const c128* F;           // [N][J] f_i(z_j)
    const c128* U;           // [L][n] probing matrix (band ordering)
    const double* un2;       // [L] squared column norms of U
    c128* S;                 // [N][L][n] S_hat
    double* eta;             // [N][L] backward errors
    int32_t* status;         // [N] 0 ok, > 0 first zero pivot (1-based), -1 tensor-core timeout,
                             //     -2 non-finite backward error, -3 tolerance not reached
    int32_t* sweeps;         // [N] refinement sweeps
};
struct DenseSampleJob {
    int32_t nep, j;
};
struct DenseSampleCfg {
    double tol;              // acceptance: eta <= tol per column
    double target;           // keep refining while eta > target and still halving (0 = working accuracy)
    int32_t max_refine;
};

// Device bytes of one CTA's slot for n <= n_max, L <= L_max.
template <typename R>
size_t dense_slot_bytes(int n_max, int L_max);
// Largest CTA count worth launching for njobs jobs (one per SM at most).
int dense_sample_grid(int njobs);
// Device bytes of one CTA's tensor-core operand images (complex64; 0 for complex128).
template <typename R>
size_t dense_image_bytes(int n_max);
// d_slots: grid * dense_slot_bytes; d_img: grid * dense_image_bytes; d_next: one int32.
template <typename R>
int launch_dense_sample(const DenseNep* d_neps, const DenseSampleJob* d_jobs, int njobs, int n_max, int L_max,
                        int grid, void* d_slots, void* d_img, int32_t* d_next, DenseSampleCfg cfg, cudaStream_t s);

}  // namespace rsrr
