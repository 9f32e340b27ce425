// Host build of the library's per-cell GENO blend (csrc/kernels.cuh,
// blend_cubic) for the CPU tests, through the test-only CUDA stand-in in
// tests/hostshim.  Arguments: M limiter prec (0 double, 1 float).  stdin: the
// case count, then per case the cross data d in the kernel's layout (cell
// units): d[q(1+M)] = W_q - W_0, d[q(1+M)+1+a] = dW_q/dxi_a, then the own
// dW/dxi_a, q = 2e + (side > 0).  stdout per case: the blended cubic's
// coefficients in the generated code's monomial order.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#include "kernels.cuh"

template <typename R, int M> static void run(const gks::KP &P, const double *in)
{
    constexpr int ND = gks::Cubic<R, M>::ND, NC = gks::Cubic<R, M>::NC;
    R d[ND], b[NC];
    for (int i = 0; i < ND; ++i) d[i] = (R)in[i];
    gks::blend_cubic<R, M>(P, d, b);
    for (int k = 0; k < NC; ++k) std::printf("%.17g%c", (double)b[k], k + 1 < NC ? ' ' : '\n');
}

int main(int argc, char **argv)
{
    if (argc < 4) return 2;
    const int m = std::atoi(argv[1]), limiter = std::atoi(argv[2]), prec = std::atoi(argv[3]);
    gks::KP P{};
    P.gamma = 1.4;
    P.h = 1.0;
    P.ih = 1.0;
    P.C = 20.0;
    P.itanhC = 1.0 / std::tanh(20.0);
    P.eps = 1e-15;
    P.C0 = 8.0;
    P.adm = 0.3;
    P.d0 = 0.85;
    P.ct = 1e-6;
    P.limiter = limiter;
    P.fp.c1 = 0.05;
    P.fp.c2 = 1.0;
    gks::finalize_kp(P);
    int ncase = 0;
    if (std::scanf("%d", &ncase) != 1) return 2;
    const int nd = m == 2 ? GENO_ND2 : GENO_ND3;
    double in[64];
    for (int k = 0; k < ncase; ++k) {
        for (int i = 0; i < nd; ++i)
            if (std::scanf("%lf", &in[i]) != 1) return 2;
        if (m == 2) (prec ? run<float, 2>(P, in) : run<double, 2>(P, in));
        else (prec ? run<float, 3>(P, in) : run<double, 3>(P, in));
    }
    return 0;
}
