// Host build of the library's mixed-precision stage update (csrc/kernels.cuh,
// update_item<float, 2, S>: exact face sums, double-float stage combination,
// the FP64 state and its FP32 shadow) for the CPU tests, through the
// test-only CUDA stand-in in tests/hostshim.  Arguments: nx ny h dt.  stdin:
// W[4][cells] (FP64), then the face sums of stage 1, ff1[3][4][faces], and of
// stage 2, ff2[3][4][faces] (FP32 values; faces: all x faces, then y faces).
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

int main(int argc, char **argv)
{
    if (argc < 5) return 2;
    const int nx = std::atoi(argv[1]), ny = std::atoi(argv[2]);
    const double h = std::atof(argv[3]), dt = std::atof(argv[4]);
    gks::KP P{};
    P.n[0] = nx;
    P.n[1] = ny;
    P.n[2] = 1;
    P.ncell = (long)nx * ny;
    P.nface[0] = (long)(nx + 1) * ny;
    P.nface[1] = (long)nx * (ny + 1);
    P.foff[0] = 0;
    P.foff[1] = P.nface[0];
    P.nftot = P.nface[0] + P.nface[1];
    P.ext[0] = nx + 2;
    P.ext[1] = ny + 2;
    P.ext[2] = 1;
    P.next = (long)(nx + 2) * (ny + 2);
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
    const long nc = P.ncell, nf = P.nftot;
    std::vector<double> W(4 * nc);
    std::vector<float> ff1(12 * nf), ff2(12 * nf);
    for (double &x : W)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (auto *ff : {&ff1, &ff2})
        for (float &x : *ff) {
            double d;
            if (std::scanf("%lf", &d) != 1) return 2;
            x = (float)d;
        }
    std::vector<float> h0(4 * nc), l0(4 * nc), g0(8 * nc), h1(4 * nc), l1(4 * nc), g1(8 * nc), acc(8 * nc);
    for (long i = 0; i < 4 * nc; ++i) gks::split(W[i], h0[i], l0[i]);
    const gks::Shadow s0{h0.data(), l0.data(), g0.data()}, s1{h1.data(), l1.data(), g1.data()};
    const gks::UpdC uc = gks::make_updc(dt, gks::updc_cw(P, 2));
    int status = 0;
    for (long c = 0; c < nc; ++c)
        gks::update_item<float, 2, 1>(P, ff1.data(), dt, W.data(), nullptr, nullptr, nullptr, (double *)acc.data(), s0,
                                      s1, &status, c, uc);
    print(h1), print(l1), print(g1), print(acc);
    for (long c = 0; c < nc; ++c)
        gks::update_item<float, 2, 2>(P, ff2.data(), dt, W.data(), nullptr, nullptr, nullptr, (double *)acc.data(), s0,
                                      s1, &status, c, uc);
    print(W), print(h0), print(l0), print(g0);
    std::printf("%d\n", status);
    return 0;
}
