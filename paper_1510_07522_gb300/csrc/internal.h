// Internal declarations of the RSRR library: the handle, host-side ordering and
// coefficient evaluation, and the launch wrappers of each device stage.
#pragma once

#include <complex>
#include <vector>

#include "common.cuh"

namespace rsrr {

using zd = std::complex<double>;

// ---- host: scalar functions f_i and their derivatives (Eq. eq-Z-expr, Eq. eq-ncs) -----
int check_fn(const rsrr_fn& f);
void eval_fn(const rsrr_fn& f, zd z, zd* val, zd* deriv);

// ---- host: contour nodes (Eq. eq-contour, Eq. eq-Ap-num) --------------------------------
// Nodes z_j and weights w_j of the contour's rule: (1 / 2 pi i) oint g(z) dz ~ sum_j w_j g(z_j).
// side_nodes: points per horizontal side of a rectangle (0 = in proportion to the side lengths).
void contour_rule(const rsrr_contour& C, int N, std::vector<zd>* z, std::vector<zd>* w, int side_nodes = 0);
void gauss_legendre(int m, std::vector<double>* x, std::vector<double>* w);
// strictly inside C (Algorithm 1 keeps only those eigenvalues)
bool inside_contour(const rsrr_contour& C, zd z);

// ---- host: band-reducing ordering ---------------------------------------------------------
struct Ordering {
    std::vector<int32_t> perm;   // perm[new] = old
    std::vector<int32_t> iperm;  // iperm[old] = new
    int64_t kl = 0, ku = 0;
    bool natural = true;
};
void band_of(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* iperm,
             int64_t* kl, int64_t* ku);
void choose_ordering(int64_t n, const int64_t* rowptr, const int32_t* colind, bool force_natural,
                     Ordering* out);

// ---- device stage launchers ----------------------------------------------------------------
struct SampleWork;  // defined in sample.cu

}  // namespace rsrr
struct rsrr_nep_s;
namespace rsrr {
// T(z_k) values of a tz handle for m points, permuted to the device's entry order and uploaded
// to *d_vals ([m][nnz], allocated here, freed by the caller).
int tz_values(rsrr_nep_s* h, const std::vector<zd>& z, c128** d_vals);

}  // namespace rsrr

struct rsrr_nep_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // problem (permuted ordering on the device)
    int64_t n = 0, nnz = 0;
    int32_t J = 0;
    std::vector<rsrr_fn> fns;
    rsrr::Ordering ord;
    int64_t* d_rowptr = nullptr;   // [n+1]
    int32_t* d_colind = nullptr;   // [nnz]
    int32_t* d_rowidx = nullptr;   // [nnz] row of each entry
    rsrr::c128* d_vals = nullptr;  // [J][nnz]
    int32_t* d_perm = nullptr;     // [n] perm[new] = old
    bool force_dense = false;      // RSRR_DENSE_LU: factor every point with the dense LU
    bool band_cuda_cores = false;  // RSRR_BAND_CUDA_CORES: no tensor-core band LU
    bool autotune = false;         // RSRR_AUTOTUNE: the sampler strategy is timed and chosen
    bool tuned = false, tune_cached = false;
    int tune_strategy = -1, tune_band = -1;
    int32_t precond_band = -1;     // >= 0: factor only |i - j| <= precond_band of T(z_j) and iterate
    bool dense_used = false;       // the last rsrr_sample factored densely
    bool band_tc_used = false;     // the last rsrr_sample ran the tensor-core band LU
    std::vector<double> normA;     // ||A_i||_F
    rsrr_tz_cb tz = nullptr;       // T known by its values (rsrr_create_nep_tz): the library calls
    void* tz_user = nullptr;       // tz for T(z) at the points it needs; d_vals then holds T(z_j)
                                   // of the sampling points as J = N "terms" with F = I
    std::vector<int64_t> vsrc;     // device entry e holds the caller's entry vsrc[e]
    bool tz_basis_only = false;    // rsrr_project_chebyshev's inner rsrr_project on a tz handle

    // sampling state
    int32_t N = 0, L = 0, precision = 0;
    std::vector<std::complex<double>> points;  // caller's sampling points (empty: the contour's nodes)
    bool refine_full = false;
    rsrr_contour C{};
    double tol = 0;
    int32_t refine_sweeps = 0;
    double max_eta = 0;
    bool sampled = false;
    rsrr::c128* d_U = nullptr;     // [L][n] permuted probing matrix
    int32_t U_L = 0;
    rsrr::c128* d_S = nullptr;     // [N*L][n] S_hat (permuted rows)
    double* d_eta = nullptr;       // [N*L]
    size_t S_cols_cap = 0;

    // projection state
    int32_t moment_order = 0;      // > 0: the next rsrr_project uses K' quadrature moments (SSRR)
    int32_t proj_cols = 0;         // columns of the matrix the last projection factored
    bool projected = false;
    int32_t kS = -1;
    rsrr::c128* d_Q = nullptr;     // [kS][n] orthonormal basis S (permuted rows)
    rsrr::c128* d_P = nullptr;     // [red_J][kS][kS]
    std::vector<rsrr_fn> red_fns;  // functions of the reduced NEP T_S(z) = sum_i red_fns[i](z) P_i:
    int32_t red_J = 0;             // fns (rsrr_project) or Chebyshev polynomials (rsrr_project_chebyshev)
    std::vector<double> sigma;     // singular values of S_hat

    // reduced solve state
    int32_t nbar = -1, n_winding = 0, n_gap = -1;
    std::complex<double> winding{0, 0};
    std::vector<double> sigma_H;

    double ms_sample = 0, ms_project = 0, ms_solve = 0;
    double ms_factor = 0, ms_trsv = 0;
    int32_t factor_launches = 0, trsv_launches = 0;
    int32_t rows_kept = 0, jacobi_sweeps_project = 0, jacobi_sweeps_solve = 0;
    double ms_project_parts[4] = {0, 0, 0, 0};
    double ms_solve_parts[3] = {0, 0, 0};
    double ms_zgemm_project = 0, zgemm_flops_project = 0, ms_zgemm_solve = 0, zgemm_flops_solve = 0;
    double ms_zgemm_tc_project = 0, zgemm_tc_flops_project = 0, ms_zgemm_tc_solve = 0, zgemm_tc_flops_solve = 0;
    double ms_jacobi_project = 0, jacobi_flops_project = 0, ms_jacobi_solve = 0, jacobi_flops_solve = 0;
    int64_t device_bytes = 0;
};
