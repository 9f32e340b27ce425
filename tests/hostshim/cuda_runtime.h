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
