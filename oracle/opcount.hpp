/*
 * Operation-counting scalar type for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * The oracle's C source is compiled as C++ with every floating-point type
 * replaced by `ocn` (oracle/opcount.py does the replacement).  An ocn carries
 * its value (in long double, so the oracle's branches take their usual
 * course) and the identity of the arithmetic node that produced it.  Each
 * new node is counted once:
 *   - common subexpressions are shared: an operation on operands it has
 *     already combined in the same way (commutative operands in either
 *     order) returns the earlier node and counts nothing, so a quantity the
 *     oracle recomputes (a cell's cubic for each of its faces, a half-space
 *     moment for every term that needs it) counts once;
 *   - constants are folded: an operation whose operands are all constants
 *     (scheme constants, Gauss points, the time step, the grid spacing) is a
 *     constant, and x * 1, x + 0, x * 0, x / 1 and negation cost nothing.
 * This is the arithmetic an optimising compiler would keep of the oracle's
 * straight-line code.  Categories: add/sub, mul, div, and the
 * transcendentals exp, erfc, sqrt, tanh counted separately; integer powers
 * are expanded into the multiplications of binary exponentiation; abs, min
 * and max are counted apart and are not flops.  A fused multiply-add is a
 * mul and an add (2 flops).
 */
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <unordered_map>

namespace opc {

enum Op : uint32_t { ADD = 1, SUB, MUL, DIV, NEG, EXP, ERFC, SQRT, TANH, ABS, MIN, MAX };

struct Key {
    uint64_t a, b;
    uint32_t op;
    bool operator==(const Key &o) const { return a == o.a && b == o.b && op == o.op; }
};
struct KeyHash {
    size_t operator()(const Key &k) const
    {
        uint64_t h = k.a * 0x9E3779B97F4A7C15ull ^ (k.b + 0x632BE59BD9B4E019ull + (h_rot(k.a)));
        return (size_t)(h ^ (h >> 29) ^ ((uint64_t)k.op << 58));
    }
    static uint64_t h_rot(uint64_t x) { return (x << 17) | (x >> 47); }
};

struct Counters {
    uint64_t add, mul, div, exp, erfc, sqrt, tanh, absminmax;
};

inline Counters &counters()
{
    static Counters c;
    return c;
}
inline std::unordered_map<Key, uint64_t, KeyHash> &table()
{
    static std::unordered_map<Key, uint64_t, KeyHash> t;
    return t;
}
inline uint64_t &next_id()
{
    static uint64_t n = 1;
    return n;
}
/* constants are keyed by their value: one key per distinct value */
inline std::unordered_map<uint64_t, uint64_t> &const_keys()
{
    static std::unordered_map<uint64_t, uint64_t> t;
    return t;
}
/* start a fresh count (forget the shared nodes too) */
inline void reset()
{
    counters() = Counters{};
    table().clear();
}

} // namespace opc

struct ocn {
    long double v;
    uint64_t id; /* 0: a constant whose value is v */
    ocn() = default;
    template <typename T, std::enable_if_t<std::is_arithmetic_v<T>, int> = 0> ocn(T x) : v((long double)x), id(0) {}
    template <typename T, std::enable_if_t<std::is_arithmetic_v<T>, int> = 0> explicit operator T() const
    {
        return (T)v;
    }
    bool konst() const { return id == 0; }
    /* a fresh input value (a node that no operation produced) */
    static ocn input(long double x)
    {
        ocn r;
        r.v = x;
        r.id = opc::next_id()++;
        return r;
    }
};

namespace opc {

inline uint64_t okey(const ocn &x)
{
    if (x.id) return x.id;
    const double d = (double)x.v;
    uint64_t b;
    std::memcpy(&b, &d, sizeof b);
    auto &t = const_keys();
    auto it = t.find(b);
    if (it != t.end()) return it->second;
    const uint64_t k = (1ull << 63) | (uint64_t)t.size();
    t.emplace(b, k);
    return k;
}

inline ocn node(Op op, const ocn &a, const ocn &b, long double val)
{
    uint64_t ka = okey(a), kb = (op == NEG || op >= EXP) ? 0 : okey(b);
    if ((op == ADD || op == MUL || op == MIN || op == MAX) && ka > kb) std::swap(ka, kb);
    const Key k{ka, kb, (uint32_t)op};
    auto &t = table();
    auto it = t.find(k);
    ocn r;
    r.v = val;
    if (it != t.end()) {
        r.id = it->second;
        return r;
    }
    r.id = next_id()++;
    t.emplace(k, r.id);
    Counters &c = counters();
    switch (op) {
    case ADD:
    case SUB: ++c.add; break;
    case MUL: ++c.mul; break;
    case DIV: ++c.div; break;
    case EXP: ++c.exp; break;
    case ERFC: ++c.erfc; break;
    case SQRT: ++c.sqrt; break;
    case TANH: ++c.tanh; break;
    case ABS:
    case MIN:
    case MAX: ++c.absminmax; break;
    case NEG: break; /* a sign flip is free */
    }
    return r;
}

inline ocn neg(const ocn &a)
{
    if (a.konst()) return ocn(-a.v);
    return node(NEG, a, ocn(0), -a.v);
}

} // namespace opc

inline ocn operator-(const ocn &a) { return opc::neg(a); }
inline ocn operator+(const ocn &a) { return a; }

inline ocn operator+(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v + b.v);
    if (a.konst() && a.v == 0) return b;
    if (b.konst() && b.v == 0) return a;
    return opc::node(opc::ADD, a, b, a.v + b.v);
}
inline ocn operator-(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v - b.v);
    if (b.konst() && b.v == 0) return a;
    if (a.konst() && a.v == 0) return opc::neg(b);
    return opc::node(opc::SUB, a, b, a.v - b.v);
}
inline ocn operator*(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v * b.v);
    if ((a.konst() && a.v == 0) || (b.konst() && b.v == 0)) return ocn(0);
    if (a.konst() && a.v == 1) return b;
    if (b.konst() && b.v == 1) return a;
    if (a.konst() && a.v == -1) return opc::neg(b);
    if (b.konst() && b.v == -1) return opc::neg(a);
    return opc::node(opc::MUL, a, b, a.v * b.v);
}
inline ocn operator/(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v / b.v);
    if (a.konst() && a.v == 0) return ocn(0);
    if (b.konst() && b.v == 1) return a;
    if (b.konst() && b.v == -1) return opc::neg(a);
    return opc::node(opc::DIV, a, b, a.v / b.v);
}
inline ocn &operator+=(ocn &a, const ocn &b) { return a = a + b; }
inline ocn &operator-=(ocn &a, const ocn &b) { return a = a - b; }
inline ocn &operator*=(ocn &a, const ocn &b) { return a = a * b; }
inline ocn &operator/=(ocn &a, const ocn &b) { return a = a / b; }

inline bool operator<(const ocn &a, const ocn &b) { return a.v < b.v; }
inline bool operator>(const ocn &a, const ocn &b) { return a.v > b.v; }
inline bool operator<=(const ocn &a, const ocn &b) { return a.v <= b.v; }
inline bool operator>=(const ocn &a, const ocn &b) { return a.v >= b.v; }
inline bool operator==(const ocn &a, const ocn &b) { return a.v == b.v; }
inline bool operator!=(const ocn &a, const ocn &b) { return a.v != b.v; }

#define OPC_UNARY(NAME, OP, FN)                                                                                        \
    inline ocn NAME(const ocn &a)                                                                                      \
    {                                                                                                                  \
        if (a.konst()) return ocn(FN(a.v));                                                                            \
        return opc::node(opc::OP, a, ocn(0), FN(a.v));                                                                 \
    }
OPC_UNARY(exp, EXP, std::exp)
OPC_UNARY(expl, EXP, std::exp)
OPC_UNARY(erfc, ERFC, std::erfc)
OPC_UNARY(erfcl, ERFC, std::erfc)
OPC_UNARY(sqrt, SQRT, std::sqrt)
OPC_UNARY(sqrtl, SQRT, std::sqrt)
OPC_UNARY(tanh, TANH, std::tanh)
OPC_UNARY(tanhl, TANH, std::tanh)
OPC_UNARY(fabs, ABS, std::fabs)
OPC_UNARY(fabsl, ABS, std::fabs)
#undef OPC_UNARY

inline ocn fmin(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v < b.v ? a.v : b.v);
    return opc::node(opc::MIN, a, b, a.v < b.v ? a.v : b.v);
}
inline ocn fmax(const ocn &a, const ocn &b)
{
    if (a.konst() && b.konst()) return ocn(a.v > b.v ? a.v : b.v);
    return opc::node(opc::MAX, a, b, a.v > b.v ? a.v : b.v);
}

/* x^k for an integer k >= 0 by binary exponentiation (the multiplications
 * a program computing the power would do) */
inline ocn powl(const ocn &x, const ocn &k)
{
    const long double kv = k.v;
    const long n = (long)kv;
    if (!k.konst() || (long double)n != kv || n < 0) return ocn(std::pow(x.v, kv)); /* not used by the oracle */
    ocn r(1.0L), b = x;
    for (long e = n; e > 0; e >>= 1) {
        if (e & 1) r = r * b;
        if (e > 1) b = b * b;
    }
    return r;
}
inline ocn pow(const ocn &x, const ocn &k) { return powl(x, k); }

inline bool isfinite(const ocn &a) { return std::isfinite(a.v); }
inline bool isnan(const ocn &a) { return std::isnan(a.v); }
