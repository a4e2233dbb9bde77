// rsrr_band_solve_noalloc: the band LU and the two triangular solves of rsrr_sample for one
// banded system, with every piece of scratch in a fixed file-scope device array instead of
// memory allocated per call.
//
// Who needs it: processes that reserve all device memory up front for their own allocator
// (a library cudaMalloc there either fails or escapes the process's memory budget), and
// latency-bound loops that must not pay for an allocation, which can synchronise the device.
// The caller provides the band matrix and the right-hand sides in device memory; this file
// provides the rest from `g_noalloc_scratch`.
//
// Contract:
//   - scratch is at most RSRR_NOALLOC_SCRATCH_BYTES; larger problems are rejected (EINVAL);
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that first call
//     before any stream capture;
//   - every call on a device shares the one array and leaves its contents behind; nothing in
//     it has to start at zero (each call writes every scratch entry before reading it);
//   - calls whose GPU work overlaps (different streams or host threads) race on the array.
#include <mutex>

#include "band.cuh"
#include "internal.h"

namespace rsrr {

namespace {
constexpr size_t kScratchBytes = (size_t)RSRR_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = 0;
    RSRR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(RSRR_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(RSRR_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RSRR_OK;
}
}  // namespace

}  // namespace rsrr

using namespace rsrr;

extern "C" int rsrr_band_solve_noalloc(int64_t n, int32_t kl, int32_t ku, double* ab_reim, int32_t L,
                                       double* b_reim, void* stream) {
    if (n < 1 || n > (int64_t)INT32_MAX / 2 || kl < 0 || ku < 0 || kl >= n || ku >= n || L < 1 || L > 4096 ||
        !ab_reim || !b_reim)
        return set_error(RSRR_EINVAL, "rsrr_band_solve_noalloc: bad size or NULL pointer");
    BandDims d;
    RSRR_TRY(pick_dims(n, kl, ku, false, &d));
    const size_t lp_b = round_up((size_t)d.npanels * d.ldp * d.nb * sizeof(c128));
    const size_t perm_b = round_up((size_t)d.npanels * d.ldp * sizeof(int32_t));
    const size_t ipiv_b = round_up((size_t)n * sizeof(int32_t));
    const size_t info_b = 256;
    if (lp_b + perm_b + ipiv_b + info_b > kScratchBytes)
        return set_error(RSRR_EINVAL, "rsrr_band_solve_noalloc: the factor scratch of this band exceeds "
                                      "RSRR_NOALLOC_SCRATCH_BYTES");
    void* base = nullptr;
    RSRR_TRY(scratch_address(&base));
    unsigned char* p = static_cast<unsigned char*>(base);
    c128* lp = reinterpret_cast<c128*>(p);
    int32_t* perm = reinterpret_cast<int32_t*>(p + lp_b);
    int32_t* ipiv = reinterpret_cast<int32_t*>(p + lp_b + perm_b);
    int32_t* info = reinterpret_cast<int32_t*>(p + lp_b + perm_b + ipiv_b);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    c128* ab = reinterpret_cast<c128*>(ab_reim);
    c128* x = reinterpret_cast<c128*>(b_reim);
    FactorArgs<double> fa{d, ab, 0, lp, 0, perm, 0, ipiv, info};
    RSRR_TRY(launch_factor<double>(fa, 1, st));
    int32_t hinfo = 0;
    RSRR_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RSRR_CUDA(cudaStreamSynchronize(st));
    if (hinfo) return set_error(RSRR_ESINGULAR, "rsrr_band_solve_noalloc: zero pivot");
    SolveArgs<double> sa{d, ab, 0, lp, 0, perm, 0, x, 0, L, nullptr};
    RSRR_TRY(launch_fwd<double>(sa, 1, st));
    RSRR_TRY(launch_bwd<double>(sa, 1, st));
    RSRR_CUDA(cudaStreamSynchronize(st));
    return RSRR_OK;
}
