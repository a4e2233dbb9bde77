// Self-test of the failure path of the library's bounded device-side waits.  The paper has no
// counterpart.  Every wait a kernel of this library makes on another CTA or on the tensor-core
// pipeline (the grid barrier of the cooperative kernels, the mbarrier waits of the tcgen05
// pipelines) gives up after a bounded number of polls, records the failure and returns, and the
// host maps the record to RSRR_ETIMEOUT.  This entry point makes such a wait run out on purpose,
// with a short poll limit and a condition that the host arranged never to hold, so that a test
// can check the whole chain -- the wait gives up, the kernel returns, the context stays usable,
// the status reaches the caller -- without faulting or hanging the device.
#include "dense.cuh"
#include "internal.h"
#include "tc.cuh"

namespace rsrr {
namespace {

// Every CTA enters the grid barrier once; `result` counts the CTAs that saw it complete.
__global__ void selftest_grid_kernel(GridBar gb, int* result) {
    const bool ok = grid_sync(gb);
    if (threadIdx.x == 0 && ok) atomicAdd(result, 1);
}

// Thread 0 waits for phase 0 of an mbarrier that expects one arrival.  With `arrive` set, the
// thread arrives first (the wait then completes at once); otherwise nothing ever arrives.
__global__ void selftest_mbar_kernel(int arrive, uint32_t limit, int* result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) tc::mbar_arrive(&bar);
        result[0] = tc::mbar_wait(&bar, 0, limit) ? 1 : 0;
    }
}

}  // namespace
}  // namespace rsrr

using namespace rsrr;

extern "C" int rsrr_selftest_bounded_wait(int32_t kind, void* stream) {
    if (kind < 0 || kind > 3) return set_error(RSRR_EINVAL, "rsrr_selftest_bounded_wait: kind is 0..3");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    constexpr int kCtas = 2;
    unsigned* bar = nullptr;
    int* result = nullptr;
    int rc = dalloc_n(&bar, kGridBarWords, st);
    if (rc == RSRR_OK) rc = dalloc_n(&result, 1, st);
    auto done = [&](int code) {
        cudaStreamSynchronize(st);
        dfree(bar, st);
        dfree(result, st);
        return code;
    };
    if (rc != RSRR_OK) return done(rc);
    if (cudaMemsetAsync(bar, 0, kGridBarWords * sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(result, 0, sizeof(int), st) != cudaSuccess)
        return done(set_error(RSRR_ECUDA, "rsrr_selftest_bounded_wait: memset"));
    int herr = 0, hres = 0;
    if (kind == 0 || kind == 2) {
        if (kind == 0) {
            // an arrival count no CTA can complete: the releasing CTA is the one that finds
            // gridDim.x - 1 arrivals before its own, which never happens from this start
            const unsigned far = 0x40000000u;
            if (cudaMemcpyAsync(bar, &far, sizeof(unsigned), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return done(set_error(RSRR_ECUDA, "rsrr_selftest_bounded_wait: copy"));
        }
        GridBar gb = grid_bar_at(bar, 4096);  // ~0.5 ms of polling with backoff
        void* args[] = {&gb, &result};
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)selftest_grid_kernel, dim3(kCtas), dim3(64),
                                                          args, 0, st);
        note_launch();
        if (e != cudaSuccess)
            return done(set_error(RSRR_ECUDA, std::string("rsrr_selftest_bounded_wait: ") + cudaGetErrorString(e)));
        if (cudaMemcpyAsync(&herr, bar + kGridBarErrWord, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return done(set_error(RSRR_ECUDA, "rsrr_selftest_bounded_wait: copy back"));
    } else {
        selftest_mbar_kernel<<<1, 32, 0, st>>>(kind == 3 ? 1 : 0, 1u << 16, result);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return done(set_error(RSRR_ECUDA, "rsrr_selftest_bounded_wait: launch"));
    }
    if (cudaMemcpyAsync(&hres, result, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return done(set_error(RSRR_ECUDA, "rsrr_selftest_bounded_wait: copy back"));
    const cudaError_t se = cudaStreamSynchronize(st);
    if (se != cudaSuccess) return done(set_error(RSRR_ECUDA, std::string("rsrr_selftest_bounded_wait: ") + cudaGetErrorString(se)));
    if (kind == 0 || kind == 2) {
        if (herr) return done(set_error(RSRR_ETIMEOUT, "grid barrier: a bounded wait gave up"));
        if (hres != kCtas) return done(set_error(RSRR_ECUDA, "grid barrier: completed for only some CTAs"));
        return done(RSRR_OK);
    }
    if (!hres) return done(set_error(RSRR_ETIMEOUT, "mbarrier: a bounded wait gave up"));
    return done(RSRR_OK);
}
