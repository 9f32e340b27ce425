// Host build of the library's double-float arithmetic and stage constants
// (csrc/kernels.cuh: df_two_sum, df_fast_two_sum, df_mul, df_add,
// two_sum_acc, make_updc) for the CPU tests, through the test-only CUDA
// stand-in in tests/hostshim.  Results are printed as hexadecimal floats so
// that the test can check them exactly.
//   dfloat_check twosum      stdin: n, then n pairs a b (floats)   -> s e
//   dfloat_check acc         stdin: n, len, then n sequences        -> s e
//   dfloat_check mul         stdin: n, then n quads khi klo xhi xlo -> hi lo
//   dfloat_check updc dt cw                                         -> 5 x (hi lo)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

#include "kernels.cuh"

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    const char *mode = argv[1];
    if (!std::strcmp(mode, "updc")) {
        const gks::UpdC u = gks::make_updc(std::atof(argv[2]), std::atof(argv[3]));
        for (int k = 0; k < 5; ++k) std::printf("%a %a\n", (double)u.k[k].hi, (double)u.k[k].lo);
        return 0;
    }
    int n = 0;
    if (std::scanf("%d", &n) != 1) return 2;
    if (!std::strcmp(mode, "acc")) {
        int len = 0;
        if (std::scanf("%d", &len) != 1) return 2;
        for (int c = 0; c < n; ++c) {
            float s = 0.f, e = 0.f;
            for (int i = 0; i < len; ++i) {
                double x;
                if (std::scanf("%lf", &x) != 1) return 2;
                gks::two_sum_acc(s, e, (float)x);
            }
            std::printf("%a %a\n", (double)s, (double)e);
        }
        return 0;
    }
    for (int c = 0; c < n; ++c) {
        if (!std::strcmp(mode, "twosum")) {
            double a, b;
            if (std::scanf("%lf %lf", &a, &b) != 2) return 2;
            const gks::F2 r = gks::df_two_sum((float)a, (float)b);
            const float hi = std::fabs((float)a) >= std::fabs((float)b) ? (float)a : (float)b;
            const float lo = hi == (float)a ? (float)b : (float)a;
            const gks::F2 f = gks::df_fast_two_sum(hi, lo);
            std::printf("%a %a %a %a\n", (double)r.hi, (double)r.lo, (double)f.hi, (double)f.lo);
        } else if (!std::strcmp(mode, "mul")) {
            double a, b, x, y;
            if (std::scanf("%lf %lf %lf %lf", &a, &b, &x, &y) != 4) return 2;
            const gks::F2 r = gks::df_mul(gks::F2{(float)a, (float)b}, gks::F2{(float)x, (float)y});
            const gks::F2 s = gks::df_add(gks::F2{(float)a, (float)b}, gks::F2{(float)x, (float)y});
            std::printf("%a %a %a %a\n", (double)r.hi, (double)r.lo, (double)s.hi, (double)s.lo);
        } else {
            return 2;
        }
    }
    return 0;
}
