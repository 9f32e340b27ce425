/*
 * Left/right lane pairs for the FP32 gas-kinetic flux.
 *
 * The flux evaluates the same formulas for the two initial Maxwellians of a
 * face (their half-space moments, transverse moments, micro-slopes and slope
 * moments).  LR holds one value of each side, lane 0 left and lane 1 right,
 * and its arithmetic issues the packed two-lane FP32 instructions
 * (add / mul / fma .rn.f32x2): one instruction for both sides, per-lane
 * results identical to the scalar round-to-nearest operations.  The product
 * is lazy (LRProd), so that a * b + c, a * b - c and c - a * b become one
 * packed fused multiply-add, as the scalar code's contraction would give.
 * Transcendentals and divisions run per lane.
 */
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace gks {

struct LRProd;

struct LR {
    float2 v;
    LR() = default;
    __device__ __forceinline__ LR(float2 x) : v(x) {}
    __device__ __forceinline__ LR(float l, float r) : v(make_float2(l, r)) {}
    template <typename T, std::enable_if_t<std::is_arithmetic_v<T>, int> = 0>
    __device__ __forceinline__ LR(T s) : v(make_float2((float)s, (float)s))
    {
    }
    __device__ __forceinline__ LR(const LRProd &p);
    __device__ __forceinline__ float l() const { return v.x; }
    __device__ __forceinline__ float r() const { return v.y; }
    /* left + right */
    __device__ __forceinline__ float sum() const { return v.x + v.y; }
};

struct LRProd {
    float2 a, b;
};

namespace lr {
__device__ __forceinline__ float2 neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 eval(const LRProd &p) { return mul(p.a, p.b); }
} // namespace lr

__device__ __forceinline__ LR::LR(const LRProd &p) : v(lr::eval(p)) {}

/* products (lazy) */
__device__ __forceinline__ LRProd operator*(LR a, LR b) { return LRProd{a.v, b.v}; }
__device__ __forceinline__ LRProd operator*(const LRProd &p, LR b) { return LRProd{lr::eval(p), b.v}; }
__device__ __forceinline__ LRProd operator*(LR a, const LRProd &p) { return LRProd{a.v, lr::eval(p)}; }
__device__ __forceinline__ LRProd operator*(const LRProd &p, const LRProd &q) { return LRProd{lr::eval(p), lr::eval(q)}; }

/* sums: a product meeting an addend becomes one fused multiply-add */
__device__ __forceinline__ LR operator+(LR a, LR b) { return LR(lr::add(a.v, b.v)); }
__device__ __forceinline__ LR operator-(LR a, LR b) { return LR(lr::fma(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ LR operator+(const LRProd &p, LR c) { return LR(lr::fma(p.a, p.b, c.v)); }
__device__ __forceinline__ LR operator+(LR c, const LRProd &p) { return LR(lr::fma(p.a, p.b, c.v)); }
__device__ __forceinline__ LR operator-(const LRProd &p, LR c) { return LR(lr::fma(p.a, p.b, lr::neg(c.v))); }
__device__ __forceinline__ LR operator-(LR c, const LRProd &p) { return LR(lr::fma(lr::neg(p.a), p.b, c.v)); }
__device__ __forceinline__ LR operator+(const LRProd &p, const LRProd &q) { return LR(lr::fma(p.a, p.b, lr::eval(q))); }
__device__ __forceinline__ LR operator-(const LRProd &p, const LRProd &q)
{
    return LR(lr::fma(lr::neg(q.a), q.b, lr::eval(p)));
}
__device__ __forceinline__ LR operator-(LR a) { return LR(lr::neg(a.v)); }
__device__ __forceinline__ LRProd operator-(const LRProd &p) { return LRProd{lr::neg(p.a), p.b}; }

__device__ __forceinline__ LR &operator+=(LR &a, LR b) { return a = a + b; }
__device__ __forceinline__ LR &operator+=(LR &a, const LRProd &p) { return a = a + p; }
__device__ __forceinline__ LR &operator-=(LR &a, LR b) { return a = a - b; }
__device__ __forceinline__ LR &operator-=(LR &a, const LRProd &p) { return a = a - p; }
__device__ __forceinline__ LR &operator*=(LR &a, LR b) { return a = LR(a * b); }

/* per-lane division (the build's FP32 division) */
__device__ __forceinline__ LR operator/(LR a, LR b) { return LR(a.v.x / b.v.x, a.v.y / b.v.y); }

} // namespace gks
