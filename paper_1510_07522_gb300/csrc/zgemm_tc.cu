// FP64-accurate complex GEMM on the tensor cores: C = alpha op(A) op(B) + beta C.
//
// This part runs FP64 at about 1.2 TFLOP/s and BF16 MMAs at about 1.8 PFLOP/s, so the large
// ZGEMMs of the projection (the trailing updates of the Householder QR of S_hat, the basis,
// S^H (A_i S)) are emulated with exact integer pieces (the splitting idea of Ozaki et al.):
//
//  1. Real form.  With a = op(A) (M x K) and b = op(B) (K x N) complex, K2 = K rounded up to 32:
//       A' (2M x 2 K2) = [[Re a, -Im a], [Im a, Re a]],   B' (2 K2 x N) = [[Re b], [Im b]],
//     so A' B' = [[Re ab], [Im ab]].  A tile holds 64 complex rows: their real parts in rows
//     0..63 and their imaginary parts in rows 64..127.
//  2. Exact digits.  Row i of a is scaled by 2^(55 - E_i), E_i the binary exponent of its largest
//     |Re|, |Im| (so every scaled value is below 2^55 in magnitude), rounded to an integer X and
//     written as X = sum_{s<8} d_s 128^(7-s) with d_1..d_7 balanced in [-64, 63] and |d_0| <= 64.
//     Column j of b likewise with F_j.  Every digit is exact in BF16.
//  3. Exact products.  A digit product is at most 2^12; the products of one diagonal q = s + t
//     (at most 8 pairs) summed over 512 consecutive K' terms stay below 2^24, so the tensor cores
//     accumulate them exactly in FP32: one TMEM accumulator per diagonal q = 0..7 (pairs with
//     s + t >= 8 weigh below 2^-56 of the leading term and are not formed: 36 of 64 pairs).
//  4. FP64 combination.  After each 512-term chunk the diagonal sums (exact integers) are combined
//     four at a time in int64 and added to an FP64 accumulator with weights 2^(7 (14 - q)); at
//     the end the tile is scaled by 2^(E_i + F_j - 110)
//     and alpha, beta are applied.  The error is of the order of K' 2^-53 max_k |a_ik| max_k |b_kj|,
//     the same size as an FP64 GEMM's normwise bound.
//
// Kernels: row and column maxima (atomicMax on the bit patterns of non-negative doubles), the
// digit images of A' and B' in the MMA's shared-memory layout (K-major, 128-byte swizzle, one
// 64-term slab per 128-byte row; 8 digit planes per slab), and the GEMM over 128 x 32 output
// tiles (and K ranges when split): a producer warp that bulk-copies each slab's 160 KB of digit
// planes and issues its 32 MMAs (one per A plane and K step, N up to 256, covering the 36 digit
// pairs), and four warps that drain the diagonal accumulators (two TMEM buffers, so the MMAs of
// the next chunk overlap the drain) and write C.  The CTAs are persistent (one per SM, each
// walking its share of the tiles): the next tile's copies and MMAs run under the current tile's
// drain, scaling and stores.
// Every wait is bounded; a timeout is reported through an error word and the call fails.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "dense.cuh"
#include "tc.cuh"

namespace rsrr {
namespace {
using namespace tc;

constexpr int OZ_D = 8;                      // digits per value, 7 bits each
constexpr int OZ_ROWS = 128;                 // real rows per tile (64 complex rows)
constexpr int OZ_CROWS = 64;
constexpr int OZ_COLS = 32;                  // output columns per tile
constexpr int OZ_KS = 64;                    // K' terms per slab (one swizzled 128-byte row)
constexpr int OZ_CHUNK = 8;                  // slabs per exact FP32 accumulation (512 terms)
constexpr uint32_t OZ_A_PLANE = OZ_ROWS * OZ_KS * 2;   // 16 KB
constexpr uint32_t OZ_B_PLANE = OZ_COLS * OZ_KS * 2;   // 4 KB
constexpr uint32_t OZ_A_BYTES = OZ_D * OZ_A_PLANE;     // 128 KB per (tile, slab)
constexpr uint32_t OZ_B_BYTES = OZ_D * OZ_B_PLANE;     // 32 KB
constexpr int OZ_EPI_WARPS = 8;                        // two per TMEM lane group: 16 columns each
constexpr int OZ_THREADS = (OZ_EPI_WARPS + 1) * 32;   // + one producer warp
constexpr uint32_t OZ_TMEM_COLS = 512;                 // 2 buffers x 8 diagonals x 32 columns
// Each slab is consumed in two pieces: digit planes 0..3 of A' with all 8 planes of B' (the 26
// pairs with s <= 3), then planes 4..7 of A' (the 10 pairs with s >= 4, which need B' planes 0..3
// only).  Two A slots (one per half) and two B slots let the next piece's copy run under the
// current piece's MMAs.
constexpr uint32_t OZ_A_HALF = OZ_A_BYTES / 2;          // 64 KB
constexpr int OZ_XCOLS = OZ_COLS;                       // output columns per exchange round
constexpr size_t OZ_XBYTES = (size_t)OZ_ROWS * (OZ_XCOLS + 1) * 8;
constexpr size_t OZ_SMEM = 2 * OZ_A_HALF + 2 * OZ_B_BYTES + OZ_XBYTES + 1024;

// ---- maxima ----------------------------------------------------------------------------------
// out[b][u] = max over v < V of max(|Re|, |Im|) of X(u, v) = base[b*sb + u*su + v*sv], as the bit
// pattern of a non-negative double (monotone as an unsigned integer).
__global__ void oz_max_contig_u(const c128* X, int64_t sv, int64_t sb, int U, int V, int vch,
                                unsigned long long* out) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.z;
    if (u >= U) return;
    const int v0 = blockIdx.y * vch, v1 = min(V, v0 + vch);
    const c128* p = X + b * sb + u;
    double m = 0.0;
    for (int v = v0; v < v1; ++v) {
        const c128 x = p[(int64_t)v * sv];
        m = fmax(m, fmax(fabs(x.re), fabs(x.im)));
    }
    if (v1 > v0) atomicMax(out + (int64_t)b * U + u, (unsigned long long)__double_as_longlong(m));
}
__global__ void oz_max_contig_v(const c128* X, int64_t su, int64_t sb, int U, int V, int vch,
                                unsigned long long* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, b = blockIdx.z;
    const int u = blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= U) return;
    const int v0 = blockIdx.y * vch, v1 = min(V, v0 + vch);
    const c128* p = X + b * sb + (int64_t)u * su;
    double m = 0.0;
    for (int v = v0 + lane; v < v1; v += 32) m = fmax(m, fmax(fabs(p[v].re), fabs(p[v].im)));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && v1 > v0) atomicMax(out + (int64_t)b * U + u, (unsigned long long)__double_as_longlong(m));
}

// The FP64 pipe of this part issues two operations per clock per SM, the integer pipe 64: the
// exponent reads, the fixed-point digits and the conversions of the exact integer sums below are
// integer operations on the bit patterns, with the FP64 library call only on the rare subnormal
// or out-of-range path.

// E with m = f 2^E, f in [0.5, 1) (frexp's exponent) of the non-negative double with bits `bits`.
__device__ __forceinline__ int oz_exp(unsigned long long bits) {
    const int ev = (int)((bits >> 52) & 0x7ff);
    if (ev != 0) return ev - 1022;
    const double m = __longlong_as_double((long long)bits);
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    return e;
}

// llrint(v 2^(55 - E)) for |v| < 2^E (round to nearest, ties to even), from the bits of v.
__device__ __forceinline__ long long oz_fixed(double v, int E) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ev = (int)((bits >> 52) & 0x7ff);
    if (ev == 0) return llrint(ldexp(v, 55 - E));  // zero or subnormal
    const unsigned long long m = (bits & ((1ull << 52) - 1)) | (1ull << 52);  // |v| = m 2^(ev - 1075)
    const int sh = ev - 1075 + 55 - E;  // <= 2 since |v| < 2^E
    unsigned long long q;
    if (sh >= 0) {
        q = m << sh;
    } else if (sh <= -54) {
        q = 0;  // below one half
    } else {
        const int r = -sh;
        q = m >> r;
        const unsigned long long rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    return (bits >> 63) ? -(long long)q : (long long)q;
}

// Digits of v * 2^(55 - E) (|v| < 2^E): d[0] most significant.
__device__ __forceinline__ void oz_digits(double v, int E, float* d) {
    long long X = oz_fixed(v, E);
#pragma unroll
    for (int s = OZ_D - 1; s >= 1; --s) {
        int r = (int)(X & 127);
        if (r >= 64) r -= 128;
        d[s] = (float)r;
        X = (X - r) >> 7;
    }
    d[0] = (float)X;
}

// The double nearest to t (ties to even), |t| < 2^126.
__device__ __forceinline__ double oz_i128_to_double(__int128 t) {
    if (t == 0) return 0.0;
    const bool neg = t < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long m;
    if (msb <= 52) {
        m = lo << (52 - msb);
    } else {
        const int r = msb - 52;
        m = (unsigned long long)(u >> r);
        const unsigned __int128 rem = u & (((unsigned __int128)1 << r) - 1), half = (unsigned __int128)1 << (r - 1);
        if (rem > half || (rem == half && (m & 1))) {
            ++m;
            if (m == (1ull << 53)) {
                m >>= 1;
                ++msb;
            }
        }
    }
    const unsigned long long out = ((unsigned long long)(msb + 1023) << 52) | (m & ((1ull << 52) - 1)) |
                                   (neg ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)out);
}

// x 2^s, exact: the exponent field moves by s (ldexp where the result would leave the normal range).
__device__ __forceinline__ double oz_scale2(double x, int s) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ev = (int)((bits >> 52) & 0x7ff);
    if (ev == 0 || ev + s <= 0 || ev + s >= 2047) return ldexp(x, s);
    return __longlong_as_double((long long)(bits + ((unsigned long long)(long long)s << 52)));
}

__device__ __forceinline__ uint4 oz_pack8(const float* v, float sign) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(sign * v[2 * e], sign * v[2 * e + 1]);
    return *reinterpret_cast<uint4*>(h);
}

// Operand element access: op 0 = as stored (row u, column v at u + v*ld), 1 = transpose,
// 2 = conjugate transpose, 3 = conjugate (no transpose).
__device__ __forceinline__ c128 oz_at(const c128* X, int64_t ld, int op, int u, int v) {
    c128 x = (op == 0 || op == 3) ? X[u + (int64_t)v * ld] : X[v + (int64_t)u * ld];
    if (op >= 2) x.im = -x.im;
    return x;
}

// ---- digit images -----------------------------------------------------------------------------
// A': one thread per (complex row i, 8 consecutive k).  Image of batch b, row tile rt, slab sl
// at byte (b * MT * nslab + rt * nslab + sl) * OZ_A_BYTES, plane s at + s * OZ_A_PLANE.
__global__ void oz_slice_a(const c128* A, int64_t lda, int64_t sA, int op, int M, int K, int K2, int MT, int nslab,
                           const unsigned long long* rmax, uint8_t* img) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.z, kgroups = K2 / 8;
    const int64_t rows = (int64_t)MT * OZ_CROWS;
    if (t >= rows * kgroups) return;
    // consecutive threads take consecutive rows when op(A)'s rows are contiguous in memory (op 0,
    // 3), else consecutive k groups of one row: the reads are coalesced either way, and in the second
    // case the image stores too (eight threads fill a 128-byte row of a digit plane)
    const bool kfast = op == 1 || op == 2;
    const int i = kfast ? (int)(t / kgroups) : (int)(t % rows);
    const int k0 = kfast ? (int)(t % kgroups) * 8 : (int)(t / rows) * 8;
    const c128* Ab = A + b * sA;
    const int E = i < M ? oz_exp(rmax[(int64_t)b * M + i]) : 0;
    c128 x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        x[e] = (i < M && k < K) ? oz_at(Ab, lda, op, i, k) : czero<double>();
    }
    const int rt = i / OZ_CROWS, rl = i % OZ_CROWS;
    uint8_t* base = img + ((size_t)b * MT * nslab + (size_t)rt * nslab) * OZ_A_BYTES;
    // k' = k0 (first half) and K2 + k0 (second half); re row: (Re, -Im), im row: (Im, Re)
    uint8_t* lo = base + (size_t)(k0 / OZ_KS) * OZ_A_BYTES;
    uint8_t* hi = base + (size_t)((K2 + k0) / OZ_KS) * OZ_A_BYTES;
    const uint32_t re_lo = sw128_index16(rl, k0 % OZ_KS) * 2, im_lo = sw128_index16(rl + OZ_CROWS, k0 % OZ_KS) * 2;
    const uint32_t re_hi = sw128_index16(rl, (K2 + k0) % OZ_KS) * 2;
    const uint32_t im_hi = sw128_index16(rl + OZ_CROWS, (K2 + k0) % OZ_KS) * 2;
#pragma unroll
    for (int part = 0; part < 2; ++part) {  // 0: Re digits, 1: Im digits
        float d[8][OZ_D];
#pragma unroll
        for (int e = 0; e < 8; ++e) oz_digits(part == 0 ? x[e].re : x[e].im, E, d[e]);
#pragma unroll
        for (int sidx = 0; sidx < OZ_D; ++sidx) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = d[e][sidx];
            const size_t po = (size_t)sidx * OZ_A_PLANE;
            if (part == 0) {
                *reinterpret_cast<uint4*>(lo + po + re_lo) = oz_pack8(v, 1.f);
                *reinterpret_cast<uint4*>(hi + po + im_hi) = oz_pack8(v, 1.f);
            } else {
                *reinterpret_cast<uint4*>(hi + po + re_hi) = oz_pack8(v, -1.f);
                *reinterpret_cast<uint4*>(lo + po + im_lo) = oz_pack8(v, 1.f);
            }
        }
    }
}

// B': one thread per (column j, 8 consecutive k); rows of the K-major operand are columns j.
__global__ void oz_slice_b(const c128* B, int64_t ldb, int64_t sB, int op, int N, int K, int K2, int NTt, int nslab,
                           const unsigned long long* cmax, uint8_t* img) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.z, kgroups = K2 / 8;
    const int64_t cols = (int64_t)NTt * OZ_COLS;
    if (t >= cols * kgroups) return;
    // as for A': k groups fastest when a column of op(B) is contiguous (op 0, 3)
    const bool kfast = op == 0 || op == 3;
    const int j = kfast ? (int)(t / kgroups) : (int)(t % cols);
    const int k0 = kfast ? (int)(t % kgroups) * 8 : (int)(t / cols) * 8;
    const c128* Bb = B + b * sB;
    const int F = j < N ? oz_exp(cmax[(int64_t)b * N + j]) : 0;
    c128 x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        x[e] = (j < N && k < K) ? oz_at(Bb, ldb, op, k, j) : czero<double>();
    }
    const int ct = j / OZ_COLS, cl = j % OZ_COLS;
    uint8_t* base = img + ((size_t)b * NTt * nslab + (size_t)ct * nslab) * OZ_B_BYTES;
#pragma unroll
    for (int part = 0; part < 2; ++part) {  // Re digits at k' = k0, Im digits at k' = K2 + k0
        const int kp = part == 0 ? k0 : K2 + k0;
        uint8_t* slab = base + (size_t)(kp / OZ_KS) * OZ_B_BYTES;
        const uint32_t at = sw128_index16(cl, kp % OZ_KS) * 2;
        float d[8][OZ_D];
#pragma unroll
        for (int e = 0; e < 8; ++e) oz_digits(part == 0 ? x[e].re : x[e].im, F, d[e]);
#pragma unroll
        for (int sidx = 0; sidx < OZ_D; ++sidx) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = d[e][sidx];
            *reinterpret_cast<uint4*>(slab + (size_t)sidx * OZ_B_PLANE + at) = oz_pack8(v, 1.f);
        }
    }
}

__global__ void oz_scale_c(c128* C, int M, int N, int64_t ldc, int64_t sC, c128 beta) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * N) return;
    c128* c = C + blockIdx.y * sC + idx % M + (idx / M) * ldc;
    *c = (beta.re == 0.0 && beta.im == 0.0) ? czero<double>() : beta * (*c);
}

// ---- the GEMM -------------------------------------------------------------------------------
struct OzArgs {
    const uint8_t* imgA;
    const uint8_t* imgB;
    const unsigned long long* rmax;  // [batch][M]
    const unsigned long long* cmax;  // [batch][N]
    c128* C;
    int64_t cs_i, cs_j, sC;          // C(i, j) of batch b at C + b*sC + i*cs_i + j*cs_j
    int M, N, MT, NTt, nslab, nchunk, cper, ksplit;
    int ntiles;                      // MT * NTt * batch * ksplit; CTA c takes tiles c, c + grid, ...
    c128 alpha, beta;                // beta applies when ksplit == 1 (else C was scaled before)
    int* err;
};

struct OzShared {
    // 0 + h: piece of half h loaded; 2 + h: its MMAs done; 4 + b: chunk's MMAs into TMEM buffer b
    // done; 6 + b: buffer b drained
    uint64_t bar[8];
    uint32_t tmem;
    int fail;
};

__device__ __forceinline__ void oz_epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(OZ_EPI_WARPS * 32) : "memory"); }

// Tile t of the launch: column tile ct (fastest), row tile rt, then batch b and K range ks.
struct OzTile {
    int rt, ct, b, ks, S0, S1;
};
__device__ __forceinline__ OzTile oz_tile(const OzArgs& a, int t) {
    OzTile o;
    o.ct = t % a.NTt;
    const int r = t / a.NTt;
    o.rt = r % a.MT;
    const int z = r / a.MT;
    o.b = z / a.ksplit;
    o.ks = z % a.ksplit;
    const int c0 = o.ks * a.cper, c1 = min(a.nchunk, c0 + a.cper);
    o.S0 = c0 * OZ_CHUNK;
    o.S1 = min(a.nslab, c1 * OZ_CHUNK);
    return o;
}

// Persistent: each CTA walks a contiguous range of tiles.  The producer's pieces (half slabs) and
// the epilogue's chunks are numbered across the CTA's tiles, so the copies and MMAs of the next
// tile run while the epilogue warps drain and store the current one (two TMEM buffers, two A
// slots, two B slots).  With a single slab (K' <= 64) consecutive tiles of the same row tile keep
// A' in shared memory and load only their 32 KB of B'.  All tiles of a CTA have the same number
// of pieces: the launch uses K splits only with one tile per CTA.
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(OzArgs a) {
    extern __shared__ uint8_t oz_dyn[];
    __shared__ OzShared sh;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_dyn) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                   // two A halves of 64 KB
    uint8_t* sB = smem + 2 * OZ_A_HALF;   // two B slabs of 32 KB
    double* xs = reinterpret_cast<double*>(sB + 2 * OZ_B_BYTES);  // [OZ_ROWS][OZ_XCOLS + 1] exchange
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int tbeg = (int)((int64_t)a.ntiles * blockIdx.x / G), tend = (int)((int64_t)a.ntiles * (blockIdx.x + 1) / G);
    const int ntl = tend - tbeg;  // tiles of this CTA
    const OzTile t0 = oz_tile(a, tbeg);
    const int P = 2 * max(0, t0.S1 - t0.S0);      // pieces per tile
    const int nch = (t0.S1 - t0.S0 + OZ_CHUNK - 1) / OZ_CHUNK;  // chunks per tile

    if (threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) mbar_init(&sh.bar[i], (i >= 6) ? OZ_EPI_WARPS : 1);
        sh.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sh.tmem)), "r"(OZ_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem;

    if (warp == OZ_EPI_WARPS) {
        // ---- producer: copies and MMAs (one thread) ----
        if (lane == 0) {
            // kind::f16: F32 accumulate, BF16 A and B, K-major both, M = 128; N is set per MMA
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((OZ_ROWS >> 4) << 24);
            const uint64_t adesc = sw128_desc(smem_u32(sA)), bdesc = sw128_desc(smem_u32(sB));
            const int total = ntl * P;
            auto load = [&](int gp) {
                const int lt = gp / P;
                const OzTile tt = oz_tile(a, tbeg + lt);
                const int w = gp % P, sl = tt.S0 + w / 2, half = w & 1;
                bool needA = true;
                if (P == 2 && lt > 0) {  // one slab: A' stays while the row tile and batch do
                    const OzTile tp = oz_tile(a, tbeg + lt - 1);
                    needA = tp.rt != tt.rt || tp.b != tt.b;
                }
                const uint8_t* gA = a.imgA + ((size_t)tt.b * a.MT * a.nslab + (size_t)tt.rt * a.nslab) * OZ_A_BYTES;
                const uint8_t* gB = a.imgB + ((size_t)tt.b * a.NTt * a.nslab + (size_t)tt.ct * a.nslab) * OZ_B_BYTES;
                uint64_t* full = &sh.bar[half];
                const uint32_t bytes = (needA ? OZ_A_HALF : 0u) + (half == 0 ? OZ_B_BYTES : 0u);
                if (bytes == 0) {
                    mbar_arrive(full);  // nothing to copy: complete the phase
                    return;
                }
                mbar_expect_tx(full, bytes);
                if (needA) bulk_g2s(sA + half * OZ_A_HALF, gA + (size_t)sl * OZ_A_BYTES + half * OZ_A_HALF, OZ_A_HALF, full);
                if (half == 0)
                    bulk_g2s(sB + ((gp / 2) & 1) * OZ_B_BYTES, gB + (size_t)sl * OZ_B_BYTES, OZ_B_BYTES, full);
            };
            uint32_t use[2] = {0, 0};
            bool ok = true;
            if (total > 0) load(0);
            if (total > 1) load(1);
            for (int gp = 0; gp < total && ok; ++gp) {
                const int lt = gp / P, w = gp % P, ls = w / 2, half = w & 1;  // ls: slab within the tile
                const int cl = ls / OZ_CHUNK, buf = (lt * nch + cl) & 1;
                const bool chunk_first = half == 0 && ls % OZ_CHUNK == 0;
                const bool chunk_last = half == 1 && (ls + 1 == P / 2 || (ls + 1) % OZ_CHUNK == 0);
                if (chunk_first && use[buf] > 0 && !mbar_wait(&sh.bar[6 + buf], (use[buf] - 1) & 1)) { ok = false; break; }
                if (!mbar_wait(&sh.bar[half], (uint32_t)(gp / 2) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dbuf = tmem + (uint32_t)buf * (OZ_D * OZ_COLS);
                const uint32_t a_base = (uint32_t)half * OZ_A_HALF, b_base = (uint32_t)((gp / 2) & 1) * OZ_B_BYTES;
                // One MMA per A plane s and K step: B planes 0..7-s are consecutive 32-row blocks of
                // one K-major operand of N = 32 (8 - s) rows, and the product's column block t lands
                // on TMEM columns 32 (s + t), the accumulator of diagonal q = s + t.
                const int s_lo = half == 0 ? 0 : 4;
#pragma unroll 1
                for (int s = s_lo; s < s_lo + 4; ++s) {
                    const uint32_t n_s = (uint32_t)OZ_COLS * (OZ_D - s);
                    const uint32_t id = idesc | ((n_s >> 3) << 17);
                    const uint32_t ds = dbuf + (uint32_t)s * OZ_COLS;
#pragma unroll
                    for (int kk = 0; kk < OZ_KS / 16; ++kk) {
                        const uint32_t ao = a_base + (uint32_t)(s - s_lo) * OZ_A_PLANE + kk * 32;
                        const uint32_t bo = b_base + kk * 32;
                        const uint32_t acc = (chunk_first && s == 0 && kk == 0) ? 0u : 1u;
                        tc_mma(ds, adesc + (ao >> 4), bdesc + (bo >> 4), id, acc);
                    }
                }
                tc_commit(&sh.bar[2 + half]);
                if (chunk_last) {
                    tc_commit(&sh.bar[4 + buf]);
                    ++use[buf];
                }
                // refill: piece gp + 1 goes into the slot piece gp - 1 used, once its MMAs are done
                if (gp >= 1 && gp + 1 < total) {
                    if (!mbar_wait(&sh.bar[2 + ((gp - 1) & 1)], (uint32_t)((gp - 1) / 2) & 1)) { ok = false; break; }
                    load(gp + 1);
                }
            }
            if (!ok) {  // the epilogue warps see the flag after their own bounded wait and stop
                atomicExch(a.err, 1);
                *(volatile int*)&sh.fail = 1;
            }
            // let every issued MMA finish before the CTA frees tensor memory (the last commit
            // tracks all of them); when a wait gave up, also every copy still in flight
            if (total > 0) mbar_wait(&sh.bar[2 + ((total - 1) & 1)], (uint32_t)((total - 1) / 2) & 1);
        }
    } else {
        // ---- epilogue warps: drain the diagonal sums of each chunk, then scale and store ----
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (the rows it may access) and the 16 columns
        // 16 (w / 4) .. + 15 of every diagonal
        const int lg = warp & 3, hc = warp >> 2;
        const uint32_t lane_base = (uint32_t)(lg * 32) << 16;
        const int r = lg * 32 + lane, il = r % OZ_CROWS;
        // a real alpha of +-1 (the trailing updates' -1) is a sign on the scaled sums
        const bool alpha_pm1 = a.alpha.im == 0.0 && fabs(a.alpha.re) == 1.0;
        const unsigned long long sgn = (alpha_pm1 && a.alpha.re < 0.0) ? (1ull << 63) : 0ull;
        const bool beta0 = a.beta.re == 0.0 && a.beta.im == 0.0, beta1 = a.beta.re == 1.0 && a.beta.im == 0.0;
        uint32_t use[2] = {0, 0};
        bool stop = false;
        for (int lt = 0; lt < ntl && !stop; ++lt) {
            const OzTile tt = oz_tile(a, tbeg + lt);
            double acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.0;
            for (int c = 0; c < nch; ++c) {
                const int buf = (lt * nch + c) & 1;
                bool got = false;
                for (int tries = 0; tries < 4 && !got; ++tries) {
                    got = mbar_wait(&sh.bar[4 + buf], use[buf] & 1);
                    if (!got && *(volatile int*)&sh.fail) break;
                }
                got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                if (!got) {
                    if (lane == 0) {
                        atomicExch(a.err, 1);
                        *(volatile int*)&sh.fail = 1;
                    }
                    stop = true;
                    break;
                }
                ++use[buf];
                tc_fence_after();
                const uint32_t dbuf = tmem + lane_base + (uint32_t)buf * (OZ_D * OZ_COLS) + 16u * hc;
                // The diagonal sums are integers below 2^24: four consecutive ones combine exactly
                // in an int64 (below 2^46), the two groups in an int128.
#pragma unroll
                for (int h8 = 0; h8 < 2; ++h8) {  // two groups of 8 columns (register budget)
                    float v[OZ_D][8];
#pragma unroll
                    for (int q = 0; q < OZ_D; ++q) tc_ld8(dbuf + (uint32_t)q * OZ_COLS + 8u * h8, v[q]);
                    tc_wait_ld();
                    if (h8 == 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sh.bar[6 + buf]);  // the values are in registers
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        long long g[2];
#pragma unroll
                        for (int hq = 0; hq < 2; ++hq) {
                            const int q0 = 4 * hq;
                            g[hq] = ((long long)__float2int_rn(v[q0][j]) << 21) + ((long long)__float2int_rn(v[q0 + 1][j]) << 14) +
                                    ((long long)__float2int_rn(v[q0 + 2][j]) << 7) + (long long)__float2int_rn(v[q0 + 3][j]);
                        }
                        // weights: diagonal q carries 2^(7 (14 - q)); g[0] is in units of q = 3, g[1] of
                        // q = 7, so the chunk's exact sum is 2^49 (g[0] 2^28 + g[1]); acc in units of 2^49
                        const __int128 t = ((__int128)g[0] << 28) + (__int128)g[1];
                        acc[8 * h8 + j] += oz_i128_to_double(t);
                    }
                }
            }
            // every epilogue warp takes the same decision (the flag is read between two barriers)
            oz_epi_sync();
            const bool failed_now = *(volatile int*)&sh.fail != 0 || stop;
            oz_epi_sync();
            if (failed_now) { stop = true; break; }
            // scale, exchange re/im halves through shared memory, combine with alpha, beta, store
            const int i = tt.rt * OZ_CROWS + il;
            const int E = i < a.M ? oz_exp(a.rmax[(int64_t)tt.b * a.M + i]) : 0;
            // column exponents: lane j reads column j's, the others take it by shuffle
            const int jl = tt.ct * OZ_COLS + lane;
            const int Fl = jl < a.N ? oz_exp(a.cmax[(int64_t)tt.b * a.N + jl]) : 0;
            c128* Cb = a.C + tt.b * a.sC;
#pragma unroll
            for (int jx = 0; jx < 16; ++jx) {
                const int j = 16 * hc + jx;
                const int F = __shfl_sync(0xffffffffu, Fl, j);
                const double y = oz_scale2(acc[jx], E + F - 61);
                xs[r * (OZ_XCOLS + 1) + j] = __longlong_as_double(__double_as_longlong(y) ^ (long long)sgn);
            }
            // this thread's C entries, all loads in flight before any use
            constexpr int kPer = OZ_CROWS * OZ_XCOLS / (OZ_EPI_WARPS * 32);
            c128 cold[kPer];
            const bool need_c = a.ksplit == 1 && !beta0;
#pragma unroll
            for (int it = 0; it < kPer; ++it) {
                const int e = threadIdx.x + it * OZ_EPI_WARPS * 32, il2 = e % OZ_CROWS, jx = e / OZ_CROWS;
                const int i2 = tt.rt * OZ_CROWS + il2, j2 = tt.ct * OZ_COLS + jx;
                cold[it] = (need_c && i2 < a.M && j2 < a.N) ? Cb[(int64_t)i2 * a.cs_i + (int64_t)j2 * a.cs_j]
                                                           : czero<double>();
            }
            oz_epi_sync();
#pragma unroll
            for (int it = 0; it < kPer; ++it) {
                const int e = threadIdx.x + it * OZ_EPI_WARPS * 32, il2 = e % OZ_CROWS, jx = e / OZ_CROWS;
                const int i2 = tt.rt * OZ_CROWS + il2, j2 = tt.ct * OZ_COLS + jx;
                if (i2 >= a.M || j2 >= a.N) continue;
                const c128 p = mk<double>(xs[il2 * (OZ_XCOLS + 1) + jx], xs[(il2 + OZ_CROWS) * (OZ_XCOLS + 1) + jx]);
                const c128 v = alpha_pm1 ? p : a.alpha * p;
                c128* cp = Cb + (int64_t)i2 * a.cs_i + (int64_t)j2 * a.cs_j;
                if (a.ksplit > 1) {
                    atomicAdd(&cp->re, v.re);
                    atomicAdd(&cp->im, v.im);
                } else if (beta0) {
                    *cp = v;
                } else if (beta1) {
                    *cp = v + cold[it];
                } else {
                    *cp = v + a.beta * cold[it];
                }
            }
            oz_epi_sync();  // the exchange buffer is reused by the next tile
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
    }
}
}  // namespace

// Element strides of op(X) (row u, column v) for the maxima: op 0/3 -> (1, ld), op 1/2 -> (ld, 1).
static void oz_strides(int op, int64_t ld, int64_t* su, int64_t* sv) {
    if (op == 0 || op == 3) { *su = 1; *sv = ld; } else { *su = ld; *sv = 1; }
}

static int oz_max(const c128* X, int64_t ld, int64_t sb, int op, int U, int V, int batch, unsigned long long* out,
                  cudaStream_t s) {
    int64_t su, sv;
    oz_strides(op, ld, &su, &sv);
    const int vch = 2048;
    const unsigned gy = (unsigned)ceil_div(V, vch);
    if (su == 1) {
        dim3 g((unsigned)ceil_div(U, 128), gy, batch);
        { oz_max_contig_u<<<g, 128, 0, s>>>(X, sv, sb, U, V, vch, out); note_launch(); }
    } else {
        dim3 g((unsigned)ceil_div(U, 8), gy, batch);
        { oz_max_contig_v<<<g, 256, 0, s>>>(X, su, sb, U, V, vch, out); note_launch(); }
    }
    return RSRR_OK;
}

// Worth it when the FP64 GEMM would take a while.  A thin output side (the moments' 2K columns,
// the traces' J columns) wastes most of a 32-column tile, but the FP64 kernel wastes more of
// its 64 x 64 tile on such shapes (measured 0.05-0.07 TFLOP/s on the moments and traces).  The
// QR updates of an 800-column Hankel matrix (0.17 GFLOP each) ran at 0.2 TFLOP/s on the FP64
// kernel: from 0.1 GFLOP on, the emulation's fixed costs (five launches, one host wait) are paid.
bool zgemm_tc_fits(const Zgemm& g) {
    const double work = 8.0 * g.M * (double)g.N * g.K * g.batch;
    return work >= 1e8 && g.K >= 16;
}

int zgemm_tc(const Zgemm& g0, cudaStream_t s) {
    Zgemm g = g0;
    // orientation: the 32-column tile side goes to the smaller output side; computing C^T =
    // op(B)^T op(A)^T swaps the operands (transposes the ops) and the output strides
    // operand codes: 0 as stored, 1 transpose, 2 conjugate transpose, 3 conjugate
    int64_t cs_i = 1, cs_j = g.ldc;
    auto tr = [](int op) { return op == 0 ? 1 : op == 1 ? 0 : op == 2 ? 3 : 2; };
    auto code = [](int op) { return op == OP_N ? 0 : op == OP_T ? 1 : 2; };
    int opA = code(g.opA), opB = code(g.opB);
    const c128 *A = g.A, *B = g.B;
    int64_t lda = g.lda, ldb = g.ldb, sA = g.sA, sB = g.sB;
    int M = g.M, N = g.N;
    if (g.N > g.M) {
        const int nA = tr(opB), nB = tr(opA);
        std::swap(A, B);
        std::swap(lda, ldb);
        std::swap(sA, sB);
        std::swap(M, N);
        opA = nA;
        opB = nB;
        std::swap(cs_i, cs_j);
    }
    const int K = g.K, batch = g.batch;
    const int K2 = (int)ceil_div(K, 32) * 32, nslab = 2 * K2 / OZ_KS, nchunk = (int)ceil_div(nslab, OZ_CHUNK);
    const int MT = (int)ceil_div(M, OZ_CROWS), NTt = (int)ceil_div(N, OZ_COLS);
    const int64_t tiles = (int64_t)MT * NTt * batch;
    int ksplit = 1;
    if (tiles < 2 * 152) ksplit = (int)std::min<int64_t>(nchunk, ceil_div(2 * 152, tiles));
    const int cper = (int)ceil_div(nchunk, ksplit);
    ksplit = (int)ceil_div(nchunk, cper);

    unsigned long long *rmax = nullptr, *cmax = nullptr;
    uint8_t *imgA = nullptr, *imgB = nullptr;
    int* err = nullptr;
    int rc = RSRR_OK;
    auto release = [&]() {
        for (void* p : {(void*)rmax, (void*)cmax, (void*)imgA, (void*)imgB, (void*)err}) dfree(p, s);
    };
    const size_t bytesA = (size_t)batch * MT * nslab * OZ_A_BYTES, bytesB = (size_t)batch * NTt * nslab * OZ_B_BYTES;
    if ((rc = dalloc_n(&rmax, (size_t)batch * M, s)) || (rc = dalloc_n(&cmax, (size_t)batch * N, s)) ||
        (rc = dalloc_n(&imgA, bytesA, s)) || (rc = dalloc_n(&imgB, bytesB, s)) || (rc = dalloc_n(&err, 1, s))) {
        release();
        return rc;
    }
    cudaMemsetAsync(rmax, 0, (size_t)batch * M * 8, s);
    cudaMemsetAsync(cmax, 0, (size_t)batch * N * 8, s);
    cudaMemsetAsync(err, 0, 4, s);
    oz_max(A, lda, sA, opA, M, K, batch, rmax, s);
    // columns of op(B) are the rows of op(B)^T
    oz_max(B, ldb, sB, tr(opB), N, K, batch, cmax, s);
    {
        const int64_t na = (int64_t)MT * OZ_CROWS * (K2 / 8), nb = (int64_t)NTt * OZ_COLS * (K2 / 8);
        { oz_slice_a<<<dim3((unsigned)ceil_div(na, 128), 1, batch), 128, 0, s>>>(A, lda, sA, opA, M, K, K2, MT, nslab, rmax, imgA); note_launch(); }
        { oz_slice_b<<<dim3((unsigned)ceil_div(nb, 128), 1, batch), 128, 0, s>>>(B, ldb, sB, opB, N, K, K2, NTt, nslab, cmax, imgB); note_launch(); }
    }
    if (ksplit > 1) {
        // C = beta C first; the K ranges then add alpha op(A) op(B) atomically
        dim3 gsc((unsigned)ceil_div((int64_t)g.M * g.N, 256), batch);
        { oz_scale_c<<<gsc, 256, 0, s>>>(g.C, g.M, g.N, g.ldc, g.sC, g.beta); note_launch(); }
    }
    static bool attr_set = false;  // same value every time: concurrent callers cannot lower it
    if (!attr_set) {
        cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
        attr_set = true;
    }
    // one CTA per SM walking a contiguous range of tiles (the next tile's copies and MMAs under
    // the current tile's epilogue); with K split, one CTA per tile (the ranges differ in length)
    const int ntiles = MT * NTt * batch * ksplit;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int G = ksplit == 1 ? std::min(ntiles, std::max(1, nsm)) : ntiles;
    OzArgs oa{imgA, imgB, rmax, cmax, g.C, cs_i, cs_j, g.sC, M, N, MT, NTt, nslab, nchunk, cper, ksplit,
              ntiles, g.alpha, g.beta, err};
    { oz_gemm_kernel<<<G, OZ_THREADS, OZ_SMEM, s>>>(oa); note_launch(); }
    rc = cudaGetLastError() == cudaSuccess ? RSRR_OK : set_error(RSRR_ECUDA, "tensor-core ZGEMM launch");
    int herr = 0;
    if (rc == RSRR_OK) {
        cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = set_error(RSRR_ECUDA, "tensor-core ZGEMM");
        else if (herr) rc = set_error(RSRR_ETIMEOUT, "tensor-core ZGEMM: a bounded wait gave up");
    }
    release();
    return rc;
}

}  // namespace rsrr
