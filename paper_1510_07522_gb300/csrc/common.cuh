// Shared device/host utilities of the RSRR library: complex arithmetic, error state,
// stream-ordered allocation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>

#include "rsrr.h"

namespace rsrr {

// ---------------------------------------------------------------------------------------
// Complex numbers as (re, im) pairs with natural alignment (8 B for c64, 16 B for c128),
// so a value moves in one vector load/store.
// ---------------------------------------------------------------------------------------
template <typename R>
struct __align__(2 * sizeof(R)) cplx {
    R re, im;
};
using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { cplx<R> c; c.re = a; c.im = b; return c; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> czero() { return mk<R>(R(0), R(0)); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cscale(cplx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cconj(cplx<R> a) { return mk<R>(a.re, -a.im); }
template <typename R>
__host__ __device__ __forceinline__ R cabs1(cplx<R> a) { return fabs(a.re) + fabs(a.im); }
template <typename R>
__host__ __device__ __forceinline__ R cnorm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
template <typename R>
__host__ __device__ __forceinline__ bool cis_zero(cplx<R> a) { return a.re == R(0) && a.im == R(0); }
// acc -= a * b  (two fused multiply-adds per real component)
template <typename R>
__host__ __device__ __forceinline__ void cfms(cplx<R>& acc, cplx<R> a, cplx<R> b) {
    acc.re = fma(-a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cfma_conj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
// 1 / a by Smith's scaled division (avoids overflow in |a|^2).
template <typename R>
__host__ __device__ __forceinline__ cplx<R> crecip(cplx<R> a) {
    if (fabs(a.re) >= fabs(a.im)) {
        R r = a.im / a.re, d = a.re + a.im * r;
        return mk<R>(R(1) / d, -r / d);
    } else {
        R r = a.re / a.im, d = a.re * r + a.im;
        return mk<R>(r / d, R(-1) / d);
    }
}
template <typename To, typename From>
__host__ __device__ __forceinline__ cplx<To> ccast(cplx<From> a) { return mk<To>((To)a.re, (To)a.im); }

template <typename R>
__device__ __forceinline__ cplx<R> shfl(cplx<R> v, int src) {
    return mk<R>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

inline std::complex<double> tostd(c128 a) { return {a.re, a.im}; }
inline c128 fromstd(std::complex<double> a) { return mk<double>(a.real(), a.imag()); }

// ---------------------------------------------------------------------------------------
// Error state (thread-local last message) and check macros.
// ---------------------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
const char* last_error();

#define RSRR_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::rsrr::set_error(RSRR_ECUDA, std::string(#call) + ": " +              \
                                                     cudaGetErrorString(e_));             \
    } while (0)

#define RSRR_TRY(expr)             \
    do {                           \
        int r_ = (expr);           \
        if (r_ != RSRR_OK) return r_; \
    } while (0)

// Process-wide count of kernels this library has launched (diagnostics, benchmarks).
void note_launch(int count = 1);
int64_t launches_total();

// Stream-ordered device allocation from the current device's default pool.  The pool keeps
// freed blocks (release threshold raised once per device), so repeated handles reuse memory.
int dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <typename T>
int dalloc_n(T** p, size_t count, cudaStream_t s) {
    return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace rsrr
