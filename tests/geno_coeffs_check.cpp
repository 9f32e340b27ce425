// Host build of the generated reconstruction code (csrc/geno_coeffs.cuh)
// for the CPU tests: reads cases from stdin, prints the results, one case
// per line.
//   geno_coeffs_check fit M          per case nd data values      -> nc coefficients
//   geno_coeffs_check eval M D S G   per case nc coefficients     -> 1 + M values
//   geno_coeffs_check ind M          per case nc coefficients     -> IS^H, IS^tau
//   geno_coeffs_check p7             per case 8 values (w, d)     -> value, derivative
// The first number on stdin is the case count.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#define __host__
#define __device__
#define __forceinline__ inline
#include "geno_coeffs.cuh"

static std::vector<double> read_n(int n)
{
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i)
        if (std::scanf("%lf", &v[i]) != 1) std::exit(2);
    return v;
}

static void print(const double *v, int n)
{
    for (int i = 0; i < n; ++i) std::printf("%.17g%c", v[i], i + 1 < n ? ' ' : '\n');
}

template <int M> static void eval_case(int d, int s, int g, const double *c, double *o)
{
    if constexpr (M == 2) {
        if (d == 0) (s ? CubicEval<double, 2, 0, 1>::run(g, c, o) : CubicEval<double, 2, 0, 0>::run(g, c, o));
        else (s ? CubicEval<double, 2, 1, 1>::run(g, c, o) : CubicEval<double, 2, 1, 0>::run(g, c, o));
    } else {
        if (d == 0) (s ? CubicEval<double, 3, 0, 1>::run(g, c, o) : CubicEval<double, 3, 0, 0>::run(g, c, o));
        else if (d == 1) (s ? CubicEval<double, 3, 1, 1>::run(g, c, o) : CubicEval<double, 3, 1, 0>::run(g, c, o));
        else (s ? CubicEval<double, 3, 2, 1>::run(g, c, o) : CubicEval<double, 3, 2, 0>::run(g, c, o));
    }
}

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    int ncase = 0;
    if (std::scanf("%d", &ncase) != 1) return 2;
    const char *mode = argv[1];
    if (!std::strcmp(mode, "p7")) {
        for (int k = 0; k < ncase; ++k) {
            const std::vector<double> x = read_n(8);
            double out[2];
            p7_face<double>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], out[0], out[1]);
            print(out, 2);
        }
        return 0;
    }
    if (argc < 3) return 2;
    const int m = std::atoi(argv[2]);
    const int nc = m == 2 ? GENO_NC2 : GENO_NC3, nd = m == 2 ? GENO_ND2 : GENO_ND3;
    for (int k = 0; k < ncase; ++k) {
        if (!std::strcmp(mode, "fit")) {
            const std::vector<double> d = read_n(nd);
            double c[GENO_NC3];
            if (m == 2) cubic2d_fit<double>(d.data(), c);
            else cubic3d_fit<double>(d.data(), c);
            print(c, nc);
        } else if (!std::strcmp(mode, "eval")) {
            const int d = std::atoi(argv[3]), s = std::atoi(argv[4]), g = std::atoi(argv[5]);
            const std::vector<double> c = read_n(nc);
            double o[4];
            if (m == 2) eval_case<2>(d, s, g, c.data(), o);
            else eval_case<3>(d, s, g, c.data(), o);
            print(o, 1 + m);
        } else if (!std::strcmp(mode, "ind")) {
            const std::vector<double> c = read_n(nc);
            double o[2];
            if (m == 2) cubic2d_indicators<double>(c.data(), o[0], o[1]);
            else cubic3d_indicators<double>(c.data(), o[0], o[1]);
            print(o, 2);
        } else {
            return 2;
        }
    }
    return 0;
}
