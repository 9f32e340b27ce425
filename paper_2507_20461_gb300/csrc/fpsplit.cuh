/*
 * Exact FP32 <-> FP64 conversions of the mixed-precision update, done on the
 * integer pipe.
 *
 * The stage-2 update of the mixed-precision path (W in FP64, its FP32 shadow
 * hi + lo) widens the double-float increment to FP64 and splits the new W
 * back into two floats: five conversions and three FP64 additions per
 * variable.  On GB300 conversions to and from FP64 issue to the FP64 pipe,
 * which retires about two operations per clock per SM, so they, not HBM,
 * bound that kernel.  The functions below compute the same bits from the
 * IEEE-754 encodings with integer operations (and one int -> float
 * conversion and one exact FP32 product for the low part), and hand the
 * values outside their range to the hardware conversion:
 *   widen(x)       = (double)x              for every float;
 *   split(w, h, l) : h = (float)w, l = (float)(w - (double)h)  for every double
 * with round-to-nearest-even throughout, bit for bit.  Fast ranges: widen,
 * normal floats and zeros; split, 2^-74 <= |w| < 2^127 and zeros.
 *
 * Host and device code alike (the host build is what the CPU tests check
 * against the compiler's own conversions).
 */
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define GKS_HD __host__ __device__ __forceinline__
#define GKS_HD_COLD static __host__ __device__ __noinline__
#else
#define GKS_HD inline
#define GKS_HD_COLD static inline
#endif

namespace gks {
namespace fps {

GKS_HD uint32_t fbits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}
GKS_HD float bitsf(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}
GKS_HD uint64_t dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}
GKS_HD double bitsd(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

/* exponent biases: FP64 1023, FP32 127 */
constexpr uint32_t kRebias = 1023 - 127;

} // namespace fps

/* The hardware conversions, for the values outside the fast ranges: behind a
 * call, so that the compiler cannot if-convert them into every element's
 * instruction stream (they issue to the FP64 pipe). */
GKS_HD_COLD double widen_hw(float x) { return (double)x; }
GKS_HD_COLD void split_hw(double w, float &h, float &l)
{
    h = (float)w;
    l = (float)(w - (double)h);
}

/* (double)x.  A normal float's 8-bit exponent and 23-bit fraction move into
 * the 11-bit exponent (rebased) and the top of the 52-bit fraction; zeros
 * keep their sign.  Subnormals, infinities and NaNs go to the hardware. */
GKS_HD double widen(float x)
{
    const uint32_t u = fps::fbits(x);
    const uint32_t a = u & 0x7fffffffu;
    if (a - 0x00800000u >= 0x7f000000u && a != 0) return widen_hw(x);
    const uint32_t hi = (u & 0x80000000u) | (a ? (a >> 3) + (fps::kRebias << 20) : 0u);
    return fps::bitsd(((uint64_t)hi << 32) | (uint64_t)(u << 29));
}

/* h = (float)w and l = (float)(w - (double)h), round-to-nearest-even.
 * Rounding w's 52-bit fraction to 23 bits is an integer add on the magnitude's
 * encoding (a carry into the exponent is the round-up to the next binade),
 * then a mask; the masked encoding is (double)h, and its distance from w's in
 * units of w's last place, R (|R| <= 2^28), is w - (double)h exactly.  So
 * l = (float)R * 2^(e - 52) with e the exponent of w: one rounding in the
 * int -> float conversion, then an exact product by a power of two (a
 * normal float while e >= -74). */
GKS_HD void split(double w, float &h, float &l)
{
    const uint64_t b = fps::dbits(w);
    const uint64_t a = b & 0x7fffffffffffffffull;
    const uint32_t e = (uint32_t)(a >> 52); /* biased FP64 exponent */
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    if (e - 949u <= 1149u - 949u) { /* 2^-74 <= |w| < 2^127 */
        const uint64_t r = a + 0x0fffffffull + ((a >> 29) & 1u);
        const uint64_t m = r & ~0x1fffffffull;
        h = fps::bitsf(sign | ((uint32_t)(m >> 29) - (fps::kRebias << 23)));
        const int32_t R = (int32_t)(int64_t)(a - m);
        l = (float)(sign ? -R : R) * fps::bitsf((e - 948u) << 23); /* R = 0 gives +0, as w - w does */
        return;
    }
    if (a == 0) {
        h = fps::bitsf(sign);
        l = 0.f;
        return;
    }
    split_hw(w, h, l);
}

} // namespace gks
