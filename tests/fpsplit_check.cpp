// Host check of the integer-pipe FP32 <-> FP64 conversions (csrc/fpsplit.cuh)
// against the compiler's own conversions, bit for bit.
//   widen: every one of the 2^32 float encodings;
//   split: the boundaries of the fast range, rounding ties and carries, and
//          random encodings over the whole exponent range.
// Prints "ok <cases>" or the first mismatch; exit status 0 only when all agree.
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <random>

#include "fpsplit.cuh"

static uint64_t bits_d(double x)
{
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
}
static uint32_t bits_f(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
}
static double from_bits(uint64_t u)
{
    double x;
    std::memcpy(&x, &u, 8);
    return x;
}

static long checked = 0;

static bool same_d(double a, double b) { return bits_d(a) == bits_d(b) || (a != a && b != b); }
static bool same_f(float a, float b) { return bits_f(a) == bits_f(b) || (a != a && b != b); }

static bool check_split(uint64_t enc)
{
    const double w = from_bits(enc);
    float h, l;
    gks::split(w, h, l);
    const float H = (float)w;
    const float L = (float)(w - (double)H);
    ++checked;
    if (!same_f(h, H) || !same_f(l, L)) {
        std::printf("split mismatch w=%016" PRIx64 " h=%08x/%08x l=%08x/%08x\n", enc, bits_f(h), bits_f(H), bits_f(l),
                    bits_f(L));
        return false;
    }
    return true;
}

int main()
{
    for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
        float x;
        const uint32_t v = (uint32_t)u;
        std::memcpy(&x, &v, 4);
        if (!same_d(gks::widen(x), (double)x)) {
            std::printf("widen mismatch x=%08x\n", v);
            return 1;
        }
    }
    checked += 1l << 32;

    // every exponent, both signs, fractions at and around the rounding
    // boundaries (ties to even and odd, the carry into the exponent)
    const uint64_t fr[] = {0,          1,          0x0fffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull,
                           0x30000000ull, 0x2fffffffull, 0x30000001ull, 0xfffffffffffffull, 0xffffff0000000ull,
                           0xfffffefffffffull, 0xffffff7ffffffull, 0xffffff8000000ull, 0xffffffa000000ull};
    for (uint64_t s = 0; s < 2; ++s)
        for (uint64_t e = 0; e < 2048; ++e)
            for (uint64_t f : fr)
                if (!check_split((s << 63) | (e << 52) | f)) return 1;

    std::mt19937_64 rng(20461);
    for (int i = 0; i < 20000000; ++i) {
        uint64_t u = rng();
        if (i & 1) { // keep the exponent near the working range
            const uint64_t e = 900 + (rng() % 300);
            u = (u & 0x800fffffffffffffull) | (e << 52);
        }
        if (!check_split(u)) return 1;
    }
    std::printf("ok %ld\n", checked);
    return 0;
}
