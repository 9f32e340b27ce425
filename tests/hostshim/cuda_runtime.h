/* Test-only stand-in for <cuda_runtime.h>: lets the CPU tests compile the
 * library's device arithmetic headers (gks_device.cuh, lr2.cuh) with a host
 * compiler.  The function qualifiers are dropped; the packed two-lane FP32
 * operations are the per-lane IEEE operations their CUDA documentation
 * states (round to nearest); the single-precision fast exponential and the
 * reciprocal square roots are the C library's functions (the device ones
 * differ in the last bits, which the FP32 tests' tolerance covers).  Nothing
 * in the product includes this file. */
#pragma once
#include <cmath>

#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __noinline__

struct float2 {
    float x, y;
};
inline float2 make_float2(float a, float b) { return float2{a, b}; }
inline float2 __fadd2_rn(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
inline float2 __fmul2_rn(float2 a, float2 b) { return float2{a.x * b.x, a.y * b.y}; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return float2{std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline float __expf(float x) { return std::exp(x); }

/* Declarations that let the kernel headers parse on the host; the CPU tests
 * call only their arithmetic (no kernel, no launch, no device query). */
#include <cstring>
#define __shared__ static
#define __align__(n) __attribute__((aligned(n)))
using std::isfinite;
using std::isnan;
#define __launch_bounds__(...)
struct gks_host_dim3 {
    unsigned x, y, z;
};
static const gks_host_dim3 threadIdx{0, 0, 0}, blockIdx{0, 0, 0}, blockDim{1, 1, 1}, gridDim{1, 1, 1};
inline void __syncthreads() {}
inline int atomicOr(int *p, int v)
{
    const int o = *p;
    *p = o | v;
    return o;
}
template <typename T> inline T atomicMax(T *p, T v)
{
    const T o = *p;
    if (v > o) *p = v;
    return o;
}
template <typename T> inline T atomicAdd(T *p, T v)
{
    const T o = *p;
    *p = o + v;
    return o;
}
inline unsigned __cvta_generic_to_shared(const void *) { return 0u; }
inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b)
{
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline long long __double_as_longlong(double x)
{
    long long r;
    std::memcpy(&r, &x, 8);
    return r;
}
inline double __longlong_as_double(long long x)
{
    double r;
    std::memcpy(&r, &x, 8);
    return r;
}
typedef int cudaError_t;
static const cudaError_t cudaSuccess = 0;
struct cudaFuncAttributes {
    size_t sharedSizeBytes;
};
enum gks_host_attr {
    cudaDevAttrMaxSharedMemoryPerMultiprocessor,
    cudaDevAttrReservedSharedMemoryPerBlock,
    cudaDevAttrMultiProcessorCount,
    cudaFuncAttributePreferredSharedMemoryCarveout,
    cudaFuncAttributeMaxDynamicSharedMemorySize
};
template <typename F> inline cudaError_t cudaFuncGetAttributes(cudaFuncAttributes *a, F) { a->sharedSizeBytes = 0; return 0; }
template <typename F> inline cudaError_t cudaFuncSetAttribute(F, int, int) { return 0; }
inline cudaError_t cudaGetDevice(int *d) { *d = 0; return 0; }
inline cudaError_t cudaDeviceGetAttribute(int *v, int, int) { *v = 0; return 0; }
inline cudaError_t cudaGetLastError() { return 0; }
