// Complex64 band LU with partial pivoting whose trailing updates run on the tensor cores, and
// the forward solve with its panel blocks (Algorithm 2, Step 2).  Layout in band_tc.cuh.
//
// Per panel of nb = 32 columns starting at k0 (right-looking, one CTA per sampling point):
//   1. The (32 + kl) x 32 panel is staged by one TMA load: the band, read as the dense matrix
//      D(x, c) = ab[x + c (ldab - 1)] with x = kv + i, is a 2D tensor (rows x = kv + i, columns c),
//      and the panel is one rectangular box of it.  Entries outside the band are cleared after
//      the load.  The panel team (4 warps) factors it with cabs1 partial pivoting (lowest row on
//      ties), swapping whole panel rows.
//   2. The panel team forms X = [inv(L11); W], W = L21 inv(L11) (row-wise substitutions with
//      L11), and inv(U11) in the upper triangle of the top block, and stores X for the solves.
//   3. The trailing update of the at most kv columns to the right, in chunks of 64 columns:
//        x'  = the chunk's block rows in pivot order (the displaced rows below the panel take the
//              original top rows, as getrf's interchanges do);
//        D   = X x'_top                (256 x 32 times 32 x N, tcgen05 MMAs into tensor memory)
//        rows 0..31 of the block  <- D (that is U12 = inv(L11) x'_top)
//        rows 32..m-1             <- x'_below - D (that is A22 - L21 U12).
//      The product is complex and runs as four real products, each FP32 operand split into three
//      BF16 pieces (h + m + l, 24 significant bits) and the six piece products of order >= 2^-16
//      accumulated in FP32 (kind::f16): FP32-level accuracy, the FP64 refinement of the sample
//      solves sits on top.  The operand images are written to shared memory in the layout the
//      MMA reads (K-major, 128-byte swizzle): X once per panel (two 128-row tiles), x'_top per
//      chunk (double-buffered).
//   Warp roles: warps 0..7 gather x'_top, write its image and run the epilogue (tensor memory ->
//   registers, C -= D into the band); warp 8 issues the MMAs (two tensor-memory buffers, so the
//   next chunk's MMAs run under the current chunk's epilogue); warps 9..12 factor the next panel
//   as soon as the first chunk (the next panel's own columns) is written back (look-ahead).
//   Every mbarrier wait is bounded; a timeout marks the point failed (info = -1).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string>

#include "band_tc.cuh"
#include "tc.cuh"

namespace rsrr {

namespace {
using namespace tc;

constexpr int NB = kTcNB;
constexpr int LDP = kTcLDP;
constexpr int MT = 128;              // rows of one MMA tile
constexpr int NCH = 64;              // columns per trailing chunk (the first chunk has 32)
constexpr int kUW = 8;               // update warps (gather + image + MMA issue + epilogue)
constexpr int kPW0 = kUW;            // first panel warp
constexpr int kPWn = 8;              // panel warps: one panel row per thread
constexpr int kThreads = (kUW + kPWn) * 32;
constexpr int kUT = kUW * 32;
constexpr int kPT = kPWn * 32;
constexpr unsigned FULL = 0xffffffffu;

// shared memory (offsets from the 1024-byte aligned base)
constexpr int A_TILE = 3 * MT * 128;           // 3 swizzle atoms (6 planes x 32 k) per 128-row tile
constexpr int OFF_B = 2 * A_TILE;
constexpr int B_BUF = 3 * NCH * 128;
constexpr int OFF_P = OFF_B + 2 * B_BUF;
constexpr int P_BYTES = LDP * NB * 8;
constexpr int OFF_PERM = OFF_P + P_BYTES;      // perm of the panel being applied, then of the next
constexpr int OFF_DISP = OFF_PERM + 2 * LDP * 4;
constexpr int SMEM_BYTES = OFF_DISP + 2 * 32 * 4 + 1024;
constexpr uint32_t TMEM_COLS = 512;            // two buffers x two tiles x (re, im) x 64 columns

struct TcbShared {
    uint64_t accfull[2];   // the MMAs into a tensor-memory buffer are complete (one tcgen05.commit per tile)
    uint64_t tma;          // the panel's TMA load
    uint32_t tmem;
    int fail;              // a bounded wait ran out
    int info;              // first zero pivot column (1-based)
    int nd;                // displaced rows of the panel being applied
    int nd_next;
    float pbest[1][kPWn];  // per panel warp: best cabs1 of the pivot search and its position
    int ppos[1][kPWn];
    c64 urow[NB];          // the pivot row of the current column
    c64 dinv[NB];          // 1 / U11(j, j)
};

__device__ __forceinline__ bool failed(const TcbShared& S) { return *(const volatile int*)&S.fail != 0; }
__device__ __forceinline__ void usync() { asm volatile("bar.sync 1, %0;" ::"n"(kUT) : "memory"); }
__device__ __forceinline__ void psync() { asm volatile("bar.sync 2, %0;" ::"n"(kPT) : "memory"); }
__device__ __forceinline__ void lead_wait() { asm volatile("bar.sync 3, %0;" ::"n"(kUT + kPT) : "memory"); }
__device__ __forceinline__ void lead_arrive() { asm volatile("bar.arrive 3, %0;" ::"n"(kUT + kPT) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait that sleeps between polls (from the second one), so that waiting warps leave the
// issue slots to the warps that share their scheduler; gives up after ~2^18 polls (~0.1 s).
__device__ __forceinline__ bool wait_backoff(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < (1u << 18); ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(it < 8 ? 32 : 256);
    }
    return false;
}
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, TcbShared& S) {
    if (failed(S)) return false;
    if (wait_backoff(bar, parity)) return true;
    S.fail = 1;
    return false;
}

// Byte offset of (row r, plane q, k < 32) in an operand image of R rows: plane q lies in swizzle
// atom q / 2 (R rows of 128 bytes), at byte 64 (q % 2) + 2 k of its row, 16-byte chunks permuted by
// the 128-byte swizzle (chunk index XOR r mod 8).
__device__ __forceinline__ uint32_t img_off(int R, int r, int q, int k) {
    const uint32_t chunk = ((uint32_t)(((q & 1) << 2) | (k >> 3))) ^ (uint32_t)(r & 7);
    return (uint32_t)(q >> 1) * (uint32_t)R * 128u + (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u +
           chunk * 16u + (uint32_t)(k & 7) * 2u;
}
// x = h + m + l with h, m, l in BF16 (24 significant bits together), as raw 16-bit patterns.
__device__ __forceinline__ void split3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const __nv_bfloat16 bl = __float2bfloat16_rn(r1 - __bfloat162float(bm));
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}
// One complex value at (r, k) of an image: planes 0..2 = re pieces, 3..5 = im pieces.
__device__ __forceinline__ void put_elem(unsigned char* img, int R, int r, int k, c64 v) {
    uint32_t p0, p1, p2, p3, p4, p5;
    split3(v.re, p0, p1, p2);
    split3(v.im, p3, p4, p5);
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 0, k)) = (unsigned short)p0;
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 1, k)) = (unsigned short)p1;
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 2, k)) = (unsigned short)p2;
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 3, k)) = (unsigned short)p3;
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 4, k)) = (unsigned short)p4;
    *reinterpret_cast<unsigned short*>(img + img_off(R, r, 5, k)) = (unsigned short)p5;
}
// Eight consecutive k (8 g .. 8 g + 7) of row r: six 16-byte stores, packed in registers.
__device__ __forceinline__ void put_row8(unsigned char* img, int R, int r, int g, const c64* v) {
    uint32_t w[6][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        uint32_t a0, a1, a2, a3, a4, a5, b0, b1, b2, b3, b4, b5;
        split3(v[e].re, a0, a1, a2);
        split3(v[e].im, a3, a4, a5);
        split3(v[e + 1].re, b0, b1, b2);
        split3(v[e + 1].im, b3, b4, b5);
        w[0][e >> 1] = a0 | (b0 << 16);
        w[1][e >> 1] = a1 | (b1 << 16);
        w[2][e >> 1] = a2 | (b2 << 16);
        w[3][e >> 1] = a3 | (b3 << 16);
        w[4][e >> 1] = a4 | (b4 << 16);
        w[5][e >> 1] = a5 | (b5 << 16);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        *reinterpret_cast<uint4*>(img + img_off(R, r, q, 8 * g)) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)) : "memory");
}

// The MMAs of one chunk for one 128-row tile i: D_i = X_i x'_top, N columns, into tensor-memory
// buffer `tb` (tile i: re at tb + 128 i, im at tb + 128 i + 64).  Real products (X_re x_re,
// -X_im x_im) into re and (X_re x_im, X_im x_re) into im, six BF16 piece products each, two
// K = 16 steps.
__device__ __forceinline__ void issue_tile(uint32_t a_base, uint32_t b_base, uint32_t tb, int N, int i) {
    // descriptors differ only in the start-address field (address >> 4, below 2^14 for the whole
    // shared window), so each is the base descriptor plus a constant
    const uint64_t ad0 = sw128_desc(a_base + i * A_TILE), bd0 = sw128_desc(b_base);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
    const int pa[4] = {0, 1, 0, 1}, pb[4] = {0, 1, 1, 0}, pd[4] = {0, 0, 64, 64}, ng[4] = {0, 1, 0, 0};
    const int sa[6] = {0, 0, 1, 0, 1, 2}, sb[6] = {0, 1, 0, 2, 1, 0};
    uint32_t acc_r = 0, acc_i = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t id = idesc | (ng[p] ? (1u << 13) : 0u);
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            const int qa = pa[p] * 3 + sa[s], qb = pb[p] * 3 + sb[s];
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t ao = (qa >> 1) * MT * 128 + (qa & 1) * 64 + ks * 32;
                const uint32_t bo = (qb >> 1) * NCH * 128 + (qb & 1) * 64 + ks * 32;
                uint32_t& acc = pd[p] ? acc_i : acc_r;
                tc_mma(tb + i * 128 + pd[p], ad0 + (ao >> 4), bd0 + (bo >> 4), id, acc);
                acc = 1;
            }
        }
    }
}

struct Geo {  // one step of the factorisation (panel p applied to its trailing columns)
    int k0, nbe, m, cb, ce, ncols, nch;
    __device__ Geo(int p, int n, int kl, int kv) {
        k0 = p * NB;
        nbe = min(NB, n - k0);
        m = min(NB + kl, n - k0);
        cb = k0 + nbe;
        ce = min(n, cb + kv);
        ncols = max(0, ce - cb);
        nch = ncols == 0 ? 0 : 1 + (max(0, ncols - NB) + NCH - 1) / NCH;
    }
    // chunk t: first column c0 and width w (chunk 0 is the next panel's 32 columns)
    __device__ void chunk(int t, int& c0, int& w) const {
        if (t == 0) { c0 = cb; w = min(NB, ncols); }
        else { c0 = cb + NB + (t - 1) * NCH; w = min(NCH, ce - c0); }
    }
};

// ------------------------------------------------------------------------------------------
// Panel team (kPT = 256 threads, barrier id 2): stage panel pn by TMA, factor it with one panel
// row per thread held in registers, write U11 / pivots / permutation, form X and store it.
//
// Rows are not moved during the factorisation: each thread keeps the logical position `pos` of
// its row, and an interchange of positions jj and pv only swaps two labels.  Per column jj:
//   the candidates (positions >= jj) reduce (cabs1, then lowest position) within each warp, the
//   warp results through shared memory (first barrier); the pivot row's thread publishes its row;
//   after the second barrier every row below scales its multiplier and applies the rank-1
//   update in registers.  Rows further than kl below the diagonal are structurally zero in the
//   column, so taking them as candidates changes neither the pivot nor the tie rule.
// ------------------------------------------------------------------------------------------
__device__ void panel_step(const CUtensorMap* tmap, const FactorArgs<float>& a, c64* ab, c64* lp, int32_t* permg,
                           int32_t* ipiv, int pn, unsigned char* base, TcbShared& S, uint32_t& ph_tma) {
    const BandDims& d = a.d;
    const int ptid = threadIdx.x - kPW0 * 32, lane = ptid & 31, pw = ptid >> 5;
    const int n = d.n, kl = d.kl, kv = d.kv, ldab = d.ldab;
    const int k0 = pn * NB, nbe = min(NB, n - k0), m = min(NB + kl, n - k0);
    c64* P = reinterpret_cast<c64*>(base + OFF_P);
    int* psm = reinterpret_cast<int*>(base + OFF_PERM) + LDP;  // the next panel's permutation
    int* dq = reinterpret_cast<int*>(base + OFF_DISP);
    // 1. stage: one box of LDP x NB of the band's dense view
    if (ptid == 0 && !failed(S)) {
        mbar_expect_tx(&S.tma, (uint32_t)P_BYTES);
        tma_load_3d(P, tmap, kv + k0, k0, (int)blockIdx.x, &S.tma);
    }
    wait_or_fail(&S.tma, ph_tma, S);
    ph_tma ^= 1;
    // My row (block row q = ptid) in registers.  Entries outside the band, past the matrix or past
    // the panel's columns are zero; a column t >= nbe (last panel only) gets a unit diagonal so
    // that the inverses below are the identity there.
    const int q = ptid;
    c64 r[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const c64 v = P[q + t * LDP];
        r[t] = (t >= nbe) ? ((q == t) ? mk<float>(1.f, 0.f) : czero<float>())
                          : ((q < m && q - t <= kl) ? v : czero<float>());
    }
    int pos = q;
    psync();  // every row read before the buffer is rewritten below
    // 2. factor (the column loop is unrolled: the row stays in registers, indexed statically)
#pragma unroll
    for (int jj = 0; jj < NB; ++jj) {
        if (jj < nbe) {
            float v = (pos >= jj) ? cabs1(r[jj]) : -1.f;
            int pp = pos;
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const float ov = __shfl_down_sync(FULL, v, off);
                const int op = __shfl_down_sync(FULL, pp, off);
                if (ov > v || (ov == v && op < pp)) { v = ov; pp = op; }
            }
            if (lane == 0) {
                S.pbest[0][pw] = v;
                S.ppos[0][pw] = pp;
            }
            psync();
            float bv = S.pbest[0][0];
            int bp = S.ppos[0][0];
#pragma unroll
            for (int w2 = 1; w2 < kPWn; ++w2) {
                const float ov = S.pbest[0][w2];
                const int op = S.ppos[0][w2];
                if (ov > bv || (ov == bv && op < bp)) { bv = ov; bp = op; }
            }
            if (pos == bp) {  // the pivot row: publish it
#pragma unroll
                for (int t = jj; t < NB; ++t) S.urow[t] = r[t];
                ipiv[k0 + jj] = k0 + bp;
                if (cis_zero(r[jj]) && S.info == 0) S.info = k0 + jj + 1;
            }
            if (pos == jj) pos = bp;
            else if (pos == bp) pos = jj;
            psync();
            const c64 piv = S.urow[jj];
            if (pos > jj && !cis_zero(piv)) {
                const c64 l = r[jj] * crecip(piv);
                r[jj] = l;
                if (!cis_zero(l)) {
#pragma unroll
                    for (int c = jj + 1; c < NB; ++c) cfms(r[c], l, S.urow[c]);
                }
            }
        }
    }
    // 3. the factored panel in pivot order, the permutation, U11 to the band
#pragma unroll
    for (int t = 0; t < NB; ++t) P[pos + t * LDP] = r[t];
    psm[pos] = q;
    permg[(int64_t)pn * LDP + pos] = q;
    if (pos < nbe) {
#pragma unroll
        for (int t = 0; t < NB; ++t)
            if (t >= pos && t < nbe) ab[(int64_t)(kv + pos - t) + (int64_t)(k0 + t) * ldab] = r[t];
        S.dinv[pos] = crecip(P[pos + pos * LDP]);  // (a runtime index into r would put r in local memory)
    } else if (pos < NB) {
        S.dinv[pos] = mk<float>(1.f, 0.f);
    }
    psync();
    // displaced rows of the next application (positions >= nbe whose row started in the top
    // block): at most nbe of them
    if (pw == 0) {
        int cnt = 0;
        for (int base_q = nbe; base_q < m; base_q += 32) {
            const int qq = base_q + lane;
            const bool disp = qq < m && psm[qq] != qq;
            const unsigned bal = __ballot_sync(FULL, disp);
            if (disp) {
                const int slot = cnt + __popc(bal & ((1u << lane) - 1u));
                if (slot < 32) dq[32 + slot] = qq;
            }
            cnt += __popc(bal);
        }
        if (lane == 0) S.nd_next = min(cnt, 32);
    }
    // 4. inv(L11) (warp 1) and inv(U11) (warp 2) in place in the top block: inv(L11) strictly below
    //    the diagonal, inv(U11) on and above it.  Both are column sweeps with lane = row:
    //      inv(L11), column j from 31 down: x_i = -(L_ij + sum_{j<t<i} inv(L)_it L_tj), i > j
    //      (the columns right of j are final, column j itself is still L's);
    //      inv(U11), column j from 0 up: x_i = -(sum_{i<=t<j} inv(U)_it U_tj) / U_jj, i < j, and
    //      x_j = 1 / U_jj (the columns left of j are final, column j itself is still U's).
    //    Each lane computes its entry before the warp writes the column.
    if (pw == 1) {
        const int i = lane;
        for (int j = NB - 2; j >= 0; --j) {
            c64 x = czero<float>();
            if (i > j) {
                x = P[i + j * LDP];
                for (int t = j + 1; t < i; ++t) cfma(x, P[i + t * LDP], P[t + j * LDP]);
                x = mk<float>(-x.re, -x.im);
            }
            __syncwarp();
            if (i > j) P[i + j * LDP] = x;
            __syncwarp();
        }
    } else if (pw == 2) {
        const int i = lane;
        for (int j = 0; j < NB; ++j) {
            c64 x = czero<float>();
            if (i < j) {
                for (int t = i; t < j; ++t) cfma(x, P[i + t * LDP], P[t + j * LDP]);
                x = mk<float>(-x.re, -x.im) * S.dinv[j];
            }
            __syncwarp();
            if (i < j) P[i + j * LDP] = x;
            else if (i == j) P[i + j * LDP] = S.dinv[j];
            __syncwarp();
        }
    }
    psync();
    // 5. W = L21 inv(L11): the row at position pos >= nbe, eight columns at a time (a short loop:
    //    straight-line code this size would not stay in the instruction cache)
    if (pos >= nbe && pos < m) {
        for (int jb = 0; jb < NB; jb += 8) {
            c64 acc[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] = P[pos + (jb + e) * LDP];  // unit diagonal of inv(L11)
            for (int t = jb + 1; t < NB; ++t) {
                const c64 lt = P[pos + t * LDP];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (t > jb + e) cfma(acc[e], lt, P[t + (jb + e) * LDP]);
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) P[pos + (jb + e) * LDP] = acc[e];
        }
    }
    psync();
    c64* lpb = lp + (int64_t)pn * LDP * NB;
    for (int idx = ptid; idx < LDP * NB; idx += kPT) lpb[idx] = P[idx];
}

// ------------------------------------------------------------------------------------------
// Update team, one chunk: gather x'_top (and write the displaced rows back), its image.
// Warp uw takes columns uw, uw + 8, ...; lane = k.
// ------------------------------------------------------------------------------------------
__device__ void gather_chunk(c64* ab, const BandDims& d, const Geo& G, int c0, int w, unsigned char* bimg,
                             const int* perm, const int* dq, int nd) {
    constexpr int CPW = NCH / kUW;  // columns per warp
    const int lane = threadIdx.x & 31, uw = threadIdx.x >> 5;
    const int kv = d.kv, ldab = d.ldab, k0 = G.k0;
    const int i = k0 + perm[lane];
    const int drow = lane < nd ? dq[lane] : 0;
    const int s = k0 + (lane < nd ? perm[drow] : 0);  // the original top row that moves down to drow
    c64 v[CPW], dv[CPW];
#pragma unroll
    for (int e = 0; e < CPW; ++e) {  // every load in flight before any store
        const int j = uw + e * kUW, c = c0 + j;
        const bool valid = j < w;
        v[e] = (valid && i >= c - kv) ? ab[(int64_t)(kv + i - c) + (int64_t)c * ldab] : czero<float>();
        dv[e] = (valid && lane < nd && s >= c - kv) ? ab[(int64_t)(kv + s - c) + (int64_t)c * ldab] : czero<float>();
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < CPW; ++e) {
        const int j = uw + e * kUW, c = c0 + j;
        if (j < w && lane < nd) ab[(int64_t)(kv + k0 + drow - c) + (int64_t)c * ldab] = dv[e];
        put_elem(bimg, NCH, j, lane, v[e]);
    }
}

// Epilogue of one chunk: warp uw reads tensor-memory lanes 32 (uw % 4).. of tile uw / 4, i.e.
// block rows q = 128 (uw / 4) + 32 (uw % 4) + lane, 16 columns at a time (the C values are loaded
// before the accumulators are read).
__device__ void epilogue_chunk(c64* ab, const BandDims& d, const Geo& G, int c0, int w, int N, uint32_t tb,
                               uint64_t* accfull, uint32_t parity, TcbShared& S) {
    const int lane = threadIdx.x & 31, uw = threadIdx.x >> 5;
    const int kv = d.kv, ldab = d.ldab;
    const int tile = uw >> 2, quarter = uw & 3;
    const int q = tile * MT + quarter * 32 + lane;
    const int row = G.k0 + q;
    const bool is_u = q < G.nbe, is_c = !is_u && q < G.m;
    const uint32_t ta = tb + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tile * 128);
    bool ok = true;
    for (int h = 0; h < N; h += 16) {
        c64 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int col = c0 + h + c;
            v[c] = (is_c && h + c < w) ? ab[(int64_t)(kv + row - col) + (int64_t)col * ldab] : czero<float>();
        }
        if (h == 0) {
            ok = wait_or_fail(accfull, parity, S);
            tc_fence_after();
        }
        float dr[16], di[16];
        tc_ld16(ta + h, dr);
        tc_ld16(ta + 64 + h, di);
        tc_wait_ld();
        if (ok) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int cc = h + e;
                const int col = c0 + cc;
                if (cc < w) {
                    const int64_t at = (int64_t)(kv + row - col) + (int64_t)col * ldab;
                    if (is_c) ab[at] = mk<float>(v[e].re - dr[e], v[e].im - di[e]);
                    else if (is_u && row >= col - kv) ab[at] = mk<float>(dr[e], di[e]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    band_factor_tc_kernel(const __grid_constant__ CUtensorMap tmap, FactorArgs<float> a) {
    extern __shared__ __align__(16) unsigned char tcb_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tcb_raw + 1023) & ~(uintptr_t)1023);
    __shared__ TcbShared S;
    const BandDims d = a.d;
    const int pt = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    c64* ab = a.ab + pt * a.ab_stride;
    c64* lp = a.lp + pt * a.lp_stride;
    int32_t* permg = a.perm + pt * a.perm_stride;
    int32_t* ipiv = a.ipiv + (int64_t)pt * d.n;
    c64* P = reinterpret_cast<c64*>(base + OFF_P);
    int* perm_cur = reinterpret_cast<int*>(base + OFF_PERM);
    int* perm_next = perm_cur + LDP;
    int* dq = reinterpret_cast<int*>(base + OFF_DISP);  // displaced rows: [0..31] current, [32..63] next

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) mbar_init(&S.accfull[i], 2);
        mbar_init(&S.tma, 1);
        S.fail = 0;
        S.info = 0;
        S.nd = S.nd_next = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == kPW0 && lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap) : "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    uint32_t ph_tma = 0;
    if (warp >= kPW0) panel_step(&tmap, a, ab, lp, permg, ipiv, 0, base, S, ph_tma);
    __syncthreads();

    const uint32_t a_base = smem_u32(base), b_base = smem_u32(base + OFF_B);
    int g = 0;  // chunks issued before this step (tensor-memory and image buffers alternate with it)
    for (int p = 0; p < d.npanels; ++p) {
        const Geo G(p, d.n, d.kl, d.kv);
        // ---- the panel's X to its operand image, its permutation and displaced rows current ----
        for (int it = tid; it < LDP * 4; it += kThreads) {
            const int r = it & (LDP - 1), gq = it >> 8;
            c64 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int t = 8 * gq + e;
                // rows of the top block hold inv(U11) on and above the diagonal (for the solves):
                // the operand takes inv(L11) there, unit diagonal and zeros above it
                c64 val = (r < G.m) ? P[r + t * LDP] : czero<float>();
                if (r < G.nbe && t >= r) val = (t == r) ? mk<float>(1.f, 0.f) : czero<float>();
                v[e] = val;
            }
            put_row8(base + (r >> 7) * A_TILE, MT, r & (MT - 1), gq, v);
        }
        for (int q = tid; q < LDP; q += kThreads) perm_cur[q] = perm_next[q];
        if (tid < 32) dq[tid] = dq[32 + tid];  // the list of this panel; the panel team fills [32..] next
        if (tid == 0) S.nd = S.nd_next;
        fence_async_smem();
        __syncthreads();
        const int nd = S.nd;

        if (warp < kUW) {
            // ---- update team: image of chunk t + 1 and its MMAs, then the epilogue of chunk t -----
            // Warps 0 and 4 issue the MMAs of tile 0 and tile 1 right after the team barrier that
            // follows the image writes; the epilogues of the buffer's previous chunk were complete
            // (tensor-memory loads waited for) before that barrier.
            auto produce = [&](int t) {
                int c0, w;
                G.chunk(t, c0, w);
                gather_chunk(ab, d, G, c0, w, base + OFF_B + ((g + t) & 1) * B_BUF, perm_cur, dq, nd);
                fence_async_smem();
            };
            auto issue = [&](int t) {
                int c0, w;
                G.chunk(t, c0, w);
                const int N = (w + 15) & ~15;
                const int b = (g + t) & 1;
                tc_fence_after();
                if ((warp & 3) == 0 && lane == 0) {
                    if (!failed(S)) issue_tile(a_base, b_base + b * B_BUF, S.tmem + b * 256, N, warp >> 2);
                    tc_commit(&S.accfull[b]);
                }
                __syncwarp();
            };
            if (G.nch > 0) produce(0);
            tc_fence_before();
            usync();
            if (G.nch > 0) issue(0);
            for (int t = 0; t < G.nch; ++t) {
                if (t + 1 < G.nch) produce(t + 1);
                tc_fence_before();
                usync();  // image t + 1 written; displaced rows of chunk t visible to every epilogue warp
                if (t + 1 < G.nch) issue(t + 1);
                int c0, w;
                G.chunk(t, c0, w);
                const int N = (w + 15) & ~15;
                const int gg = g + t, b = gg & 1;
                epilogue_chunk(ab, d, G, c0, w, N, S.tmem + b * 256, &S.accfull[b], (gg >> 1) & 1, S);
                if (t == 0) {
                    fence_async_global();  // the next panel's columns, read next by TMA
                    __threadfence_block();
                    lead_arrive();
                }
            }
        } else if (p + 1 < d.npanels) {
            // ---- panel team: the next panel, once its columns are updated --------------------
            lead_wait();
            panel_step(&tmap, a, ab, lp, permg, ipiv, p + 1, base, S, ph_tma);
        }
        g += G.nch;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (failed(S)) break;
    }
    // drain: the last commits of each buffer (bounded), so tensor memory is idle before it is freed
    if (warp == 0 && g > 0) {
        for (int b = 0; b < 2; ++b) {
            const int uses = (g - b + 1) / 2;  // chunks that used buffer b
            if (uses > 0) wait_backoff(&S.accfull[b], (uses - 1) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(TMEM_COLS) : "memory");
    if (tid == 0) a.info[pt] = failed(S) ? -1 : S.info;
}

// ------------------------------------------------------------------------------------------
// Forward solve with the X blocks: per panel, x' = the block rows in pivot order, then
//   x[k0 + q] = sum_{t <= q} inv(L11)[q, t] x'_t       (q < nbe, unit diagonal)
//   x[k0 + q] = x'_q - sum_t W[q, t] x'_t              (nbe <= q < m).
// The next panel's X block is bulk-copied into the second buffer while the current one is used.
// One CTA per (point, share of the right-hand-side columns).  A bounded wait that gives up marks
// the point's solution non-finite (the caller's residual check then reports it).
// ------------------------------------------------------------------------------------------
constexpr int kFwdThreads = 512;
constexpr int kFwdLC = 4;  // right-hand-side columns per thread

__global__ void __launch_bounds__(kFwdThreads) band_fwd_tc_kernel(SolveArgs<float> a) {
    extern __shared__ __align__(16) unsigned char fwd_raw[];
    const BandDims d = a.d;
    const int pt = blockIdx.x / a.split, part = blockIdx.x % a.split;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x;
    const c64* lp = a.lp + pt * a.lp_stride;
    const int32_t* permg = a.perm + pt * a.perm_stride;
    const int c_lo = (int)((int64_t)a.L * part / a.split), c_hi = (int)((int64_t)a.L * (part + 1) / a.split);
    c64* x = a.x + pt * a.x_stride + (int64_t)c_lo * d.n;
    const int Lp = c_hi - c_lo, n = d.n;
    c64* Xb = reinterpret_cast<c64*>(fwd_raw);                               // [2][LDP * NB]
    c64* xt = Xb + 2 * LDP * NB;                                             // [NB][Lmax] x'_top
    c64* xo = xt + NB * 32;                                                  // [NB][Lmax] original top
    int* pm = reinterpret_cast<int*>(xo + NB * 32);                          // [2][LDP]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_fail;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto stage = [&](int p, int buf) {
        if (tid == 0) {
            mbar_expect_tx(&bar[buf], (uint32_t)(P_BYTES + LDP * 4));
            bulk_g2s(Xb + (size_t)buf * LDP * NB, lp + (int64_t)p * LDP * NB, (uint32_t)P_BYTES, &bar[buf]);
            bulk_g2s(pm + buf * LDP, permg + (int64_t)p * LDP, (uint32_t)(LDP * 4), &bar[buf]);
        }
    };
    uint32_t ph[2] = {0, 0};
    stage(0, 0);
    for (int p = 0; p < d.npanels; ++p) {
        const int buf = p & 1;
        const int k0 = p * NB, nbe = min(NB, n - k0), m = min(NB + d.kl, n - k0);
        if (p + 1 < d.npanels) stage(p + 1, buf ^ 1);  // that buffer was released by the last barrier
        if (!mbar_wait(&bar[buf], ph[buf])) s_fail = 1;
        ph[buf] ^= 1;
        const c64* X = Xb + (size_t)buf * LDP * NB;
        const int* perm = pm + buf * LDP;
        // original top rows, then the permuted top rows
        for (int idx = tid; idx < NB * Lp; idx += kFwdThreads) {
            const int k = idx % NB, l = idx / NB;
            xo[k * 32 + l] = (k < m) ? x[(int64_t)(k0 + k) + (int64_t)l * n] : czero<float>();
        }
        __syncthreads();
        for (int idx = tid; idx < NB * Lp; idx += kFwdThreads) {
            const int k = idx % NB, l = idx / NB;
            const int s = perm[k];
            xt[k * 32 + l] = (k >= m) ? czero<float>() : (s < NB ? xo[s * 32 + l] : x[(int64_t)(k0 + s) + (int64_t)l * n]);
        }
        __syncthreads();
        // rows: thread -> (row q, group of kFwdLC columns); consecutive threads take consecutive rows
        const int ngroups = (Lp + kFwdLC - 1) / kFwdLC;
        for (int it = tid; it < LDP * ngroups; it += kFwdThreads) {
            const int q = it % LDP, lg = it / LDP;
            if (q >= m) continue;
            const int l0 = lg * kFwdLC;
            c64 acc[kFwdLC];
            if (q < nbe) {
#pragma unroll
                for (int c = 0; c < kFwdLC; ++c) acc[c] = (l0 + c < Lp) ? xt[q * 32 + l0 + c] : czero<float>();
                for (int t = 0; t < q; ++t) {
                    const c64 lv = X[q + t * LDP];
#pragma unroll
                    for (int c = 0; c < kFwdLC; ++c) cfma(acc[c], lv, xt[t * 32 + l0 + c]);
                }
            } else {
                const int s = perm[q];
#pragma unroll
                for (int c = 0; c < kFwdLC; ++c)
                    acc[c] = (l0 + c < Lp) ? (s != q ? xo[s * 32 + l0 + c] : x[(int64_t)(k0 + q) + (int64_t)(l0 + c) * n])
                                           : czero<float>();
#pragma unroll 8
                for (int t = 0; t < nbe; ++t) {
                    const c64 wv = X[q + t * LDP];
#pragma unroll
                    for (int c = 0; c < kFwdLC; ++c) cfms(acc[c], wv, xt[t * 32 + l0 + c]);
                }
            }
#pragma unroll
            for (int c = 0; c < kFwdLC; ++c)
                if (l0 + c < Lp) x[(int64_t)(k0 + q) + (int64_t)(l0 + c) * n] = acc[c];
        }
        __syncthreads();
        // every thread reads the flag between two barriers, so all of them leave together
        const int stop = s_fail;
        __syncthreads();
        if (stop) break;
    }
    if (s_fail) {
        // let the copies in flight land (bounded), then mark this share of the solution non-finite
        if (tid == 0) {
            mbar_wait(&bar[0], ph[0], 1u << 16);
            mbar_wait(&bar[1], ph[1], 1u << 16);
        }
        const float nan = __int_as_float(0x7fc00000);
        for (int64_t idx = tid; idx < (int64_t)Lp * n; idx += kFwdThreads) x[idx] = mk<float>(nan, nan);
    }
}

// ------------------------------------------------------------------------------------------
// Backward solve with U in the band and inv(U11) from the stored blocks: per panel, from the
// last one up,
//   r = x_blk - U12 x_right        (U12: the block's rows of U right of its diagonal block, at most
//                                   kv columns; x_right: the rows already solved)
//   x_blk = inv(U11) r
// U12 is a rectangle of the band's dense view (rows x = kv + k0 .. + 31, columns c), so it
// arrives by TMA in chunks of 32 x 64 into a ring of nbuf shared-memory buffers; thread 0 keeps
// the ring nbuf - 1 chunks ahead of the consumers, across panel boundaries.  Entries of a chunk
// right of a row's band (c > row + kv) are never used.  The solved rows a panel needs (the kv
// rows below it) stay in a circular window of shared memory (row c at c mod wrows, 16 columns).
// U12 x_right is tiled over the threads: lane q = block row, warp w = (column group w % 4 of four
// right-hand sides, quarter w / 4 of each chunk's 64 columns); the four quarters' partial sums are
// added at the end of the panel.  Per step a thread loads one U entry and four window entries
// (broadcast) for four complex multiply-adds.
// One CTA per (point, share of at most 16 right-hand sides).  A bounded wait that gives up marks
// the point's solution non-finite (the caller's residual check then reports it).
// ------------------------------------------------------------------------------------------
constexpr int kBwdThreads = 512;
constexpr int kBwdCh = 64;                                  // U12 columns per chunk
constexpr uint32_t kBwdChBytes = kBwdCh * NB * 8;           // 16 KB
constexpr int kBwdMaxBuf = 8;
constexpr int kBwdCols = 16;                                // right-hand sides per CTA
constexpr int kBwdPartLd = 18;                              // row stride of the partial sums (16-byte rows)

__global__ void __launch_bounds__(kBwdThreads)
    band_bwd_tc_kernel(const __grid_constant__ CUtensorMap umap, SolveArgs<float> a, int wrows, int nbuf) {
    extern __shared__ __align__(16) unsigned char bwd_raw[];
    __shared__ __align__(8) uint64_t fb[kBwdMaxBuf];
    __shared__ int s_fail;
    const BandDims d = a.d;
    const int pt = blockIdx.x / a.split, part = blockIdx.x % a.split;
    if (a.active && !a.active[pt]) return;
    const int tid = threadIdx.x, q = tid & 31, w = tid >> 5, cg = w & 3, ks = w >> 2;
    const c64* lp = a.lp + pt * a.lp_stride;
    const int c_lo = (int)((int64_t)a.L * part / a.split), c_hi = (int)((int64_t)a.L * (part + 1) / a.split);
    c64* x = a.x + pt * a.x_stride + (int64_t)c_lo * d.n;
    const int Lp = c_hi - c_lo, n = d.n, kv = d.kv;
    // [nbuf][kBwdCh][32] U12 chunks (TMA box layout), 1024-byte aligned (the size includes the slack)
    c64* ub = reinterpret_cast<c64*>(bwd_raw + ((1024u - (smem_u32(bwd_raw) & 1023u)) & 1023u));
    c64* win = ub + (size_t)nbuf * kBwdCh * 32;         // [wrows][16]
    c64* ui = win + (size_t)wrows * kBwdCols;           // [32][33] inv(U11)
    c64* pr = ui + 32 * 33;                             // [4][32][kBwdPartLd] partial sums, then r
    const bool grp = 4 * cg < Lp;                       // this thread's column group holds a right-hand side
    auto chunks_of = [&](int p) {
        const int k0 = p * NB, cb = k0 + min(NB, n - k0), c_end = min(n, k0 + NB + kv);
        return cb < c_end ? (c_end - cb + kBwdCh - 1) / kBwdCh : 0;
    };
    // producer state (thread 0): the next chunk to load
    int pp = d.npanels - 1, pc = 0;
    auto issue_next = [&](int slot) {
        while (pp >= 0 && pc >= chunks_of(pp)) { --pp; pc = 0; }
        if (pp < 0) return;
        const int k0 = pp * NB, cb = k0 + min(NB, n - k0);
        mbar_expect_tx(&fb[slot], kBwdChBytes);
        tma_load_3d(ub + (size_t)slot * kBwdCh * 32, &umap, kv + k0, cb + pc * kBwdCh, pt, &fb[slot]);
        ++pc;
    };
    if (tid == 0) {
        for (int i = 0; i < nbuf; ++i) mbar_init(&fb[i], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&umap) : "memory");
    }
    // the last chunk of a panel can reach columns whose window slots were never written
    for (int idx = tid; idx < wrows * kBwdCols; idx += kBwdThreads) win[idx] = czero<float>();
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < nbuf; ++i) issue_next(i);
    int g = 0;  // chunks consumed
    for (int p = d.npanels - 1; p >= 0; --p) {
        const int k0 = p * NB, nbe = min(NB, n - k0), cb = k0 + nbe, row = k0 + q;
        for (int idx = tid; idx < NB * NB; idx += kBwdThreads) {
            const int qq = idx % NB, j = idx / NB;
            ui[qq * 33 + j] = (qq <= j && j < nbe) ? lp[(int64_t)p * LDP * NB + qq + (int64_t)j * LDP] : czero<float>();
        }
        const int nch = chunks_of(p);
        c64 acc[4] = {czero<float>(), czero<float>(), czero<float>(), czero<float>()};
        // this row's band ends at column row + kv (and the matrix at n - 1)
        const int c_stop = min(n, row + kv + 1);
        for (int ch = 0; ch < nch; ++ch, ++g) {
            const int slot = g % nbuf;
            if (!mbar_wait(&fb[slot], (uint32_t)((g / nbuf) & 1))) s_fail = 1;
            const c64* u = ub + (size_t)slot * kBwdCh * 32;
            const int c0 = cb + ch * kBwdCh;
            if (grp && q < nbe && !s_fail) {
                const int j0 = ks * (kBwdCh / 4), j1 = min(j0 + kBwdCh / 4, c_stop - c0);
                int sw = (c0 + j0) % wrows;
                for (int j = j0; j < j1; ++j) {
                    const c64 uv = u[j * 32 + q];
                    const float4* wp = reinterpret_cast<const float4*>(win + (size_t)sw * kBwdCols + 4 * cg);
                    const float4 w01 = wp[0], w23 = wp[1];
                    cfms(acc[0], uv, mk<float>(w01.x, w01.y));
                    cfms(acc[1], uv, mk<float>(w01.z, w01.w));
                    cfms(acc[2], uv, mk<float>(w23.x, w23.y));
                    cfms(acc[3], uv, mk<float>(w23.z, w23.w));
                    if (++sw == wrows) sw = 0;
                }
            }
            __syncthreads();  // the slot is free again
            if (tid == 0 && !s_fail) issue_next(slot);
        }
        {
            float4* pp4 = reinterpret_cast<float4*>(pr + ((size_t)ks * 32 + q) * kBwdPartLd + 4 * cg);
            pp4[0] = make_float4(acc[0].re, acc[0].im, acc[1].re, acc[1].im);
            pp4[1] = make_float4(acc[2].re, acc[2].im, acc[3].re, acc[3].im);
        }
        __syncthreads();
        // r = x_blk - sum of the quarters (thread: row q, right-hand side w)
        if (w < Lp && q < nbe) {
            c64 r = x[row + (int64_t)w * n];
            for (int s2 = 0; s2 < 4; ++s2) r = r + pr[((size_t)s2 * 32 + q) * kBwdPartLd + w];
            pr[(size_t)q * kBwdPartLd + w] = r;
        }
        __syncthreads();
        if (w < Lp && q < nbe) {
            c64 sacc = czero<float>();
            for (int j = q; j < nbe; ++j) cfma(sacc, ui[q * 33 + j], pr[(size_t)j * kBwdPartLd + w]);
            x[row + (int64_t)w * n] = sacc;
            win[(size_t)(row % wrows) * kBwdCols + w] = sacc;
        }
        __syncthreads();
        // every thread reads the flag between two barriers, so all of them leave together
        const int stop = s_fail;
        __syncthreads();
        if (stop) break;
    }
    if (s_fail) {
        // let the loads in flight land (bounded) before the block's shared memory is released,
        // then mark this share of the solution non-finite
        if (tid == 0)
            for (int i = 0; i < nbuf; ++i) mbar_wait(&fb[(g + i) % nbuf], (uint32_t)(((g + i) / nbuf) & 1), 1u << 16);
        const float nan = __int_as_float(0x7fc00000);
        for (int64_t idx = tid; idx < (int64_t)Lp * n; idx += kBwdThreads) x[idx] = mk<float>(nan, nan);
    }
}

}  // namespace

// ---- host side -------------------------------------------------------------------------------

bool band_tc_eligible(int64_t n, int64_t kl, int64_t ku) {
    return n >= 2 * kTcNB && kl >= 32 && kl <= kTcMaxKl && ku >= 1 && kl + ku + 1 <= 2048;
}

int pick_dims_tc(int64_t n, int64_t kl, int64_t ku, BandDims* d) {
    if (!band_tc_eligible(n, kl, ku)) return set_error(RSRR_EUNSUPPORTED, "band not suited to the tensor-core LU");
    const int64_t ku2 = ku + ((kl + ku) & 1);  // kv even: the TMA row coordinate kv + k0 is 16-byte aligned
    // the backward solve is the CUDA-core one: its block sizes as for any complex64 band
    RSRR_TRY(pick_dims(n, kl, ku2, true, d));
    d->n = (int)n;
    d->kl = (int)kl;
    d->ku = (int)ku2;
    d->kv = d->kl + d->ku;
    int ldab = 2 * d->kl + d->ku + 1;
    if ((ldab & 1) == 0) ++ldab;  // (ldab - 1) * 8 bytes, the TMA column stride, a multiple of 16
    d->ldab = ldab;
    d->nb = kTcNB;
    d->ldp = kTcLDP;
    d->npanels = (int)ceil_div(n, kTcNB);
    d->fwd_nbuf = 2;
    return RSRR_OK;
}

int64_t tc_ab_stride(const BandDims& d) { return ((int64_t)d.ldab * d.n + 31) / 32 * 32; }

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The band arrays of npts points as one 3D tensor of 8-byte elements: x = kv + i (the row's slot in
// its column shifted by the column), y = column, z = point.  Element (x, y, z) sits at
// ab + z * stride + x + y * (ldab - 1); every in-extent element lies inside point z's array.
int band_tensor_map(CUtensorMap* map, const c64* ab, int64_t stride, int npts, const BandDims& d, int box_x, int box_y) {
    auto fn = encode_fn();
    if (!fn) return set_error(RSRR_ECUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[3] = {(cuuint64_t)d.n + (cuuint64_t)d.ldab - 1, (cuuint64_t)d.n, (cuuint64_t)npts};
    cuuint64_t strides[2] = {(cuuint64_t)(d.ldab - 1) * 8u, (cuuint64_t)stride * 8u};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<c64*>(ab), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(RSRR_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return RSRR_OK;
}

template <typename K>
int set_smem_max(K kernel, size_t sm, const char* name) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    if (sm + fa.sharedSizeBytes > (size_t)optin)
        return set_error(RSRR_EUNSUPPORTED, std::string(name) + ": shared memory " + std::to_string(sm) + " + " +
                                                std::to_string(fa.sharedSizeBytes) + " exceeds " + std::to_string(optin));
    // process-wide attribute: the largest allowed value, so concurrent launches never lower it
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return set_error(RSRR_ECUDA, std::string(name) + ": " + cudaGetErrorString(e));
    return RSRR_OK;
}

int solve_split_tc(int npts, int L) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (L >= 2 && 2 * npts <= nsm) ? 2 : 1;
}
}  // namespace

int launch_factor_tc(const FactorArgs<float>& a, int npts, cudaStream_t s) {
    const BandDims& d = a.d;
    if (d.nb != kTcNB || d.ldp != kTcLDP || (d.kv & 1) || !(d.ldab & 1) || (a.ab_stride & 1) ||
        (reinterpret_cast<uintptr_t>(a.ab) & 15))
        return set_error(RSRR_EINVAL, "launch_factor_tc: band layout not prepared for TMA");
    CUtensorMap map;
    RSRR_TRY(band_tensor_map(&map, a.ab, a.ab_stride, npts, d, kTcLDP, kTcNB));
    RSRR_TRY(set_smem_max(band_factor_tc_kernel, SMEM_BYTES, "band_factor_tc_kernel"));
    band_factor_tc_kernel<<<npts, kThreads, SMEM_BYTES, s>>>(map, a);
    note_launch();
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

namespace {
int bwd_window_rows(const BandDims& d) { return (d.kv + 2 * NB + 31) / 32 * 32; }  // >= kv + 64 solved rows
size_t bwd_smem(const BandDims& d, int nbuf) {
    return (size_t)nbuf * kBwdChBytes + (size_t)bwd_window_rows(d) * kBwdCols * sizeof(c64) +
           (size_t)32 * 33 * sizeof(c64) + (size_t)4 * 32 * kBwdPartLd * sizeof(c64) + 1024;
}
constexpr size_t kBwdSmemMax = 224 * 1024;
int bwd_nbuf(const BandDims& d) {
    for (int nb : {kBwdMaxBuf, 4, 2})
        if (bwd_smem(d, nb) <= kBwdSmemMax) return nb;
    return 0;
}
}  // namespace

bool band_bwd_tc_fits(const BandDims& d) { return bwd_nbuf(d) > 0; }

int launch_bwd_tc(const SolveArgs<float>& a, int npts, cudaStream_t s) {
    if (a.L > 64) return set_error(RSRR_EINVAL, "launch_bwd_tc: at most 64 right-hand sides");
    const int nbuf = bwd_nbuf(a.d);
    if (!nbuf) return set_error(RSRR_EINVAL, "launch_bwd_tc: band too wide for the solved-row window");
    if ((a.d.kv & 1) || (a.ab_stride & 1) || (reinterpret_cast<uintptr_t>(a.ab) & 15))
        return set_error(RSRR_EINVAL, "launch_bwd_tc: band layout not prepared for TMA");
    const int wrows = bwd_window_rows(a.d);
    const size_t sm = bwd_smem(a.d, nbuf);
    CUtensorMap map;
    RSRR_TRY(band_tensor_map(&map, a.ab, a.ab_stride, npts, a.d, NB, kBwdCh));
    RSRR_TRY(set_smem_max(band_bwd_tc_kernel, sm, "band_bwd_tc_kernel"));
    SolveArgs<float> b = a;
    b.split = a.L > kBwdCols ? 2 : solve_split_tc(npts, a.L);
    if ((a.L + b.split - 1) / b.split > kBwdCols) b.split = (a.L + kBwdCols - 1) / kBwdCols;
    band_bwd_tc_kernel<<<npts * b.split, kBwdThreads, sm, s>>>(map, b, wrows, nbuf);
    note_launch();
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

int launch_fwd_tc(const SolveArgs<float>& a, int npts, cudaStream_t s) {
    if (a.L > 64) return set_error(RSRR_EINVAL, "launch_fwd_tc: at most 64 right-hand sides");
    const size_t sm = (size_t)2 * P_BYTES + (size_t)2 * NB * 32 * sizeof(c64) + (size_t)2 * LDP * 4;
    RSRR_TRY(set_smem_max(band_fwd_tc_kernel, sm, "band_fwd_tc_kernel"));
    SolveArgs<float> b = a;
    b.split = a.L > 32 ? 2 : solve_split_tc(npts, a.L);
    if ((a.L + b.split - 1) / b.split > 32) return set_error(RSRR_EINVAL, "launch_fwd_tc: too many columns per CTA");
    band_fwd_tc_kernel<<<npts * b.split, kFwdThreads, sm, s>>>(b);
    note_launch();
    RSRR_CUDA(cudaGetLastError());
    return RSRR_OK;
}

}  // namespace rsrr
