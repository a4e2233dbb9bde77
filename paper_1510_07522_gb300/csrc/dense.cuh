// Dense FP64 complex building blocks for the projection and reduced-solve stages.
#pragma once

#include "common.cuh"

namespace rsrr {

enum { OP_N = 0, OP_T = 1, OP_C = 2 };

// C = alpha op(A) op(B) + beta C for `batch` independent problems (strided).  With ksplit > 1
// the K range is cut into slices whose products are added to C atomically (beta is applied
// first by a separate pass).  op(A) is M x K, op(B) is K x N, all column-major.
struct Zgemm {
    int opA = OP_N, opB = OP_N;
    int M = 0, N = 0, K = 0;
    c128 alpha{1, 0}, beta{0, 0};
    const c128* A = nullptr;
    int64_t lda = 0, sA = 0;
    const c128* B = nullptr;
    int64_t ldb = 0, sB = 0;
    c128* C = nullptr;
    int64_t ldc = 0, sC = 0;
    int batch = 1;
    int ksplit = 0;  // 0 = choose
    bool fp64 = false;  // FP64 CUDA cores even where the tensor-core emulation would be chosen
};
int zgemm(const Zgemm& g, cudaStream_t s);
// In-place inverses of `batch` dense k x k complex128 matrices (column-major, stride k^2) by
// blocked Gauss-Jordan elimination with partial pivoting (zinv.cu); info[t] (zeroed by the
// caller) is set to 1 where matrix t met an exactly zero pivot column.  zinv_block(k) is the block
// width, 0 when a k-row panel does not fit shared memory (EUNSUPPORTED).
int zinv_block(int k);
size_t zinv_bytes_per_matrix(int k);
int zinv_batch(c128* X, int k, int batch, int32_t* info, cudaStream_t st);
// FP64-accurate ZGEMM on the tensor cores (exact BF16 digit products, see zgemm_tc.cu), and
// the shapes for which zgemm() takes it.  zgemm_path: 0 = by shape, 1 = FP64 CUDA cores only,
// 2 = tensor cores for every shape (per host thread; for tests and measurements).
int zgemm_tc(const Zgemm& g, cudaStream_t s);
bool zgemm_tc_fits(const Zgemm& g);
void zgemm_set_path(int path);
int zgemm_get_path();
// Accounting of the ZGEMMs issued by this host thread between the two calls.
void zgemm_profile_begin();
void zgemm_profile_end(double* ms, double* flops, double* ms_tc = nullptr, double* flops_tc = nullptr);
// Accounting of the one-sided Jacobi sweeps (device time of the sweep kernels, algorithmic flops).
void jacobi_profile_begin();
void jacobi_profile_end(double* ms, double* flops);
// One-sided Jacobi SVD of a square D x D matrix with a QR preconditioner (project.cu): on return H
// holds U Sigma and Jr the right singular vectors, as jacobi_orthogonalize(H, ..., Jr) would give.
int jacobi_svd_preconditioned(c128* H, int D, c128* Jr, cudaStream_t st, double floor, double conv, int* sweeps);

// Sum of v over a CTA (blockDim a multiple of 32, <= 1024); every thread gets the result.
// Four block-wide sums at once (two CTA barriers instead of eight); every thread gets them.
__device__ __forceinline__ void block_sum4(double& a, double& b, double& c, double& d) {
    __shared__ double red4_[4][33];
    for (int off = 16; off; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
        d += __shfl_down_sync(0xffffffffu, d, off);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { red4_[0][w] = a; red4_[1][w] = b; red4_[2][w] = c; red4_[3][w] = d; }
    __syncthreads();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < nw; ++i)
        for (int j = 0; j < 4; ++j) s[j] += red4_[j][i];
    a = s[0];
    b = s[1];
    c = s[2];
    d = s[3];
}

__device__ __forceinline__ double block_sum_all(double v) {
    __shared__ double red_[33];
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red_[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = (threadIdx.x < (blockDim.x >> 5)) ? red_[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
        if (threadIdx.x == 0) red_[32] = r;
    }
    __syncthreads();
    return red_[32];
}

// Device-wide barrier for cooperative kernels.  Every wait is bounded: after the spin limit
// the barrier records a timeout in *err and returns false, and the kernel returns.
struct GridBar {
    unsigned* count;
    unsigned* gen;
    int* err;
    long long spin_limit;  // polls before a wait gives up (2^24 with backoff: about a second)
};
// The three words sit on separate 128-byte lines: the arrival atomics on `count` must not
// queue behind hundreds of CTAs polling `gen` in the same L2 line.
constexpr int kGridBarWords = 96;  // allocation size in unsigned words
inline GridBar grid_bar_at(unsigned* base, long long spin_limit = 1LL << 24) {
    return GridBar{base, base + 32, reinterpret_cast<int*>(base + 64), spin_limit};
}
constexpr int kGridBarErrWord = 64;
__device__ __forceinline__ bool grid_sync(const GridBar& gb) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = gb.gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(gb.count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(gb.count, 0u);
            __threadfence();
            atomicAdd(gb.gen, 1u);
        } else {
            long long spins = 0;
            unsigned backoff = 8;
            while (*vgen == g) {
                if (++spins > gb.spin_limit) {  // bounded: give up, report, return
                    atomicExch(gb.err, 1);
                    ok = 0;
                    break;
                }
                // short backoff from the first miss, so that a few hundred pollers do not
                // saturate the line the releasing CTA has to write
                __nanosleep(backoff);
                if (backoff < 128) backoff <<= 1;
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int*)gb.err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}


// One-sided (Hestenes) Jacobi on the k columns of B (mb x k, ld mb), accumulating the
// rotations into J (k x k, ld k, initialised to I by the caller when wanted; may be null).
// Sweeps stop once every pair of columns above abs_floor has |<b_p, b_q>| / (|b_p| |b_q|) <=
// conv (singular values are then exact to second order in conv); columns below abs_floor are
// not rotated, nor are pairs with |<b_p, b_q>| <= abs_inner (absolute).
int jacobi_orthogonalize(c128* B, int mb, int k, c128* J, cudaStream_t s, int max_sweeps, int* sweeps_out,
                         double abs_floor, double conv, double abs_inner);

// Column 2-norms of B (mb x k) into out[k] (device).
void column_norms(const c128* B, int mb, int k, int64_t ld, double* out, cudaStream_t s);

// Frobenius norm squared of the block rows [r0, r1) x cols [c0, c1) of A (ld lda), added
// atomically to *out (device, caller zeroes it).
void block_norm2(const c128* A, int64_t lda, int r0, int r1, int c0, int c1, double* out, cudaStream_t s);

}  // namespace rsrr
