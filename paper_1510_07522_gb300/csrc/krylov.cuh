// Restarted flexible GMRES for the sample solves of the iterative sampler (krylov.cu).
#pragma once

#include <functional>

#include "common.cuh"

namespace rsrr {

template <typename R>
struct KrylovArgs {
    cudaStream_t st;
    int64_t n, nnz;
    int np, L;
    const int64_t* rowptr;    // CSR of T(z_j) on the union pattern (band ordering)
    const int32_t* colind;
    const c128* tvals;        // [np][nnz] values of T(z_j)
    const c128* U;            // [L][n] probing matrix
    c128* X;                  // [np][L][n] in: starting samples, out: refined samples
    const double* normT;      // [np] ||T(z_j)||_1
    const double* un2;        // [L] ||u_l||^2
    double tau;               // stop a system once ||r|| <= tau (||T||_1 ||x|| + ||u||)
    int m;                    // restart length
    int max_iter;             // preconditioned products in all (over restarts)
    cplx<R>* B;               // [np][L][n] the preconditioner's work array
    std::function<int(const int32_t* active)> precond;  // B <- M^{-1} B for the active points
};

// Restart length that fits about 40 % of `free_bytes` (at most 30); < 2 when nothing fits.
int krylov_restart(int64_t n, int64_t systems, size_t free_bytes);

// Runs cycles of FGMRES(m) from the samples in X until every system meets its target or
// max_iter preconditioned products were spent; *iters_out receives their count.  The caller
// checks the backward errors of the result itself.
template <typename R>
int krylov_solve(const KrylovArgs<R>& a, int* iters_out);

}  // namespace rsrr
