// Host build of the library's mixed-precision stage update (csrc/kernels.cuh,
// update_item<float, M, S>: exact face sums, double-float stage combination,
// the FP64 state and its FP32 shadow) for the CPU tests, through the
// test-only CUDA stand-in in tests/hostshim.  Arguments: nx ny nz h dt (nz = 0:
// 2D).  stdin: W[nv][cells] (FP64), then the face sums of stage 1,
// ff1[3][nv][faces], and of stage 2, ff2[3][nv][faces] (FP32 values; faces:
// all x faces, then y faces, then z faces).
// stdout, hexadecimal floats, one array per line: after stage 1 the shadow
// s1.hi, s1.lo, s1.g and the accumulator pair acc; after stage 2 W, s0.hi,
// s0.lo, s0.g; then the status word.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>

#include "kernels.cuh"

template <typename T> static void print(const std::vector<T> &v)
{
    for (size_t i = 0; i < v.size(); ++i) std::printf("%a%c", (double)v[i], i + 1 < v.size() ? ' ' : '\n');
}

template <int M> static int run(gks::KP &P, double dt)
{
    constexpr int NV = M + 2;
    const long nc = P.ncell, nf = P.nftot;
    std::vector<double> W(NV * nc);
    std::vector<float> ff1(3 * NV * nf), ff2(3 * NV * nf);
    for (double &x : W)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (auto *ff : {&ff1, &ff2})
        for (float &x : *ff) {
            double d;
            if (std::scanf("%lf", &d) != 1) return 2;
            x = (float)d;
        }
    std::vector<float> h0(NV * nc), l0(NV * nc), g0(M * NV * nc), h1(NV * nc), l1(NV * nc), g1(M * NV * nc),
        acc(2 * NV * nc);
    for (long i = 0; i < NV * nc; ++i) gks::split(W[i], h0[i], l0[i]);
    const gks::Shadow s0{h0.data(), l0.data(), g0.data()}, s1{h1.data(), l1.data(), g1.data()};
    const gks::UpdC uc = gks::make_updc(dt, gks::updc_cw(P, M));
    int status = 0;
    for (long c = 0; c < nc; ++c)
        gks::update_item<float, M, 1>(P, ff1.data(), dt, W.data(), nullptr, nullptr, nullptr, (double *)acc.data(), s0,
                                      s1, &status, c, uc);
    print(h1), print(l1), print(g1), print(acc);
    for (long c = 0; c < nc; ++c)
        gks::update_item<float, M, 2>(P, ff2.data(), dt, W.data(), nullptr, nullptr, nullptr, (double *)acc.data(), s0,
                                      s1, &status, c, uc);
    print(W), print(h0), print(l0), print(g0);
    std::printf("%d\n", status);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 6) return 2;
    const int n[3] = {std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3])};
    const int m = n[2] > 0 ? 3 : 2;
    const double h = std::atof(argv[4]), dt = std::atof(argv[5]);
    gks::KP P{};
    long ncell = 1, next = 1;
    for (int a = 0; a < 3; ++a) {
        P.n[a] = a < m ? n[a] : 1;
        P.ext[a] = a < m ? n[a] + 2 : 1;
        ncell *= P.n[a];
        next *= P.ext[a];
    }
    P.ncell = ncell;
    P.next = next;
    long off = 0;
    for (int d = 0; d < m; ++d) {
        long f = 1;
        for (int a = 0; a < m; ++a) f *= (a == d) ? P.n[a] + 1 : P.n[a];
        P.nface[d] = f;
        P.foff[d] = off;
        off += f;
    }
    P.nftot = off;
    P.h = h;
    P.ih = 1.0 / h;
    P.gamma = 1.4;
    P.C = 20.0;
    P.itanhC = 1.0 / std::tanh(20.0);
    P.eps = 1e-15;
    P.C0 = 8.0;
    P.adm = 0.3;
    P.fp.c1 = 0.05;
    P.fp.c2 = 1.0;
    gks::finalize_kp(P);
    return m == 2 ? run<2>(P, dt) : run<3>(P, dt);
}
