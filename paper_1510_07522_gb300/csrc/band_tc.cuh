// Complex64 band LU with the trailing updates on the tensor cores (tcgen05) and TMA-staged
// panels, and the forward solve that uses its stored panel blocks (Algorithm 2, Step 2:
// Y_j = T(z_j)^{-1} U for every sampling point).  One CTA owns one sampling point.
//
// Storage of one point's factorisation (band layout as in band.cuh; ldab is chosen so that the
// band can be addressed as a dense matrix by TMA, see pick_dims_tc):
//   ab    on exit the rows i <= c of each column hold U (upper bandwidth kv).
//   lp    one (256 x 32) block per panel, column-major: rows 0..31 hold inv(L11) strictly below
//         the diagonal and inv(U11) on and above it; rows 32..m-1 hold W = L21 inv(L11).  With
//         them the forward solve of a panel is y = inv(L11) x'_top, x'_below -= W x'_top (x' the
//         permuted block rows), and the backward solve's diagonal block is a product too.
//   perm  per panel, 256 entries, as in band.cuh.
//   ipiv  LAPACK-style pivot rows (absolute, 0-based).
#pragma once

#include "band.cuh"

namespace rsrr {

constexpr int kTcNB = 32;     // panel width: the K depth of the trailing-update MMAs
constexpr int kTcLDP = 256;   // panel rows: nb + kl <= 256, two 128-row MMA tiles
constexpr int kTcMaxKl = kTcLDP - kTcNB;

// True when the tensor-core factorisation takes this band (complex64, kl in [32, 224]).
bool band_tc_eligible(int64_t n, int64_t kl, int64_t ku);
// Dimensions for the tensor-core path: nb = 32, ldp = 256, ku padded so that kv = kl + ku is
// even, ldab odd (so (ldab - 1) * 8 bytes, the TMA row stride, is a multiple of 16).
int pick_dims_tc(int64_t n, int64_t kl, int64_t ku, BandDims* d);
// Elements between the band arrays of consecutive points (ldab * n rounded up to 32).
int64_t tc_ab_stride(const BandDims& d);

int launch_factor_tc(const FactorArgs<float>& a, int npts, cudaStream_t s);
// Solves take at most 64 right-hand sides per launch (EINVAL beyond).
int launch_fwd_tc(const SolveArgs<float>& a, int npts, cudaStream_t s);
// Backward solve with U in the band and the stored inv(U11) blocks.  Its shared memory holds a
// window of kv + 64 solved rows (16 right-hand sides) and a ring of TMA-loaded U12 chunks (8
// buffers up to kv ~ 480, 4 up to ~990, 2 up to ~1250: band_bwd_tc_fits); beyond that the
// CUDA-core backward solve (band.cuh) takes the same storage.  (The sampler sends bands with
// ku > 768 to the dense LU, so it uses the eight- and four-buffer plans.)
bool band_bwd_tc_fits(const BandDims& d);
int launch_bwd_tc(const SolveArgs<float>& a, int npts, cudaStream_t s);

}  // namespace rsrr
