// Host build of the library's 1D compact reconstruction (csrc/kernels.cuh,
// recon1d_face: p^7, the three sub-stencil quadratics of each side and the
// GENO / WENO-Z / TENO blend) for the CPU tests, through the test-only CUDA
// stand-in in tests/hostshim.  Arguments: n bc limiter prec (0 double,
// 1 float).  stdin: W[3][n] then G[3][n] (physical units, cell size 1/n).
// stdout: per face f = 0..n one line, st[side][v][value, d/dx] (12 numbers).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>

#include "kernels.cuh"

template <typename R> static void run(const gks::KP &P, const double *W, const double *G, int n)
{
    for (int f = 0; f <= n; ++f) {
        R st[2][3][2], cw[2][3];
        gks::recon1d_face<R>(P, W, G, f, st, cw);
        for (int s = 0; s < 2; ++s)
            for (int v = 0; v < 3; ++v)
                for (int c = 0; c < 2; ++c) std::printf("%.17g%c", (double)st[s][v][c], (s == 1 && v == 2 && c == 1) ? '\n' : ' ');
    }
}

int main(int argc, char **argv)
{
    if (argc < 5) return 2;
    const int n = std::atoi(argv[1]), bc = std::atoi(argv[2]), limiter = std::atoi(argv[3]), prec = std::atoi(argv[4]);
    gks::KP P{};
    P.n[0] = n;
    P.n[1] = P.n[2] = 1;
    gks::set_bcs(P, bc);
    P.ncell = n;
    P.gamma = 1.4;
    P.h = 1.0 / n;
    P.ih = n;
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
    std::vector<double> W(3 * n), G(3 * n);
    for (double &x : W)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (double &x : G)
        if (std::scanf("%lf", &x) != 1) return 2;
    if (prec) run<float>(P, W.data(), G.data(), n);
    else run<double>(P, W.data(), G.data(), n);
    return 0;
}
