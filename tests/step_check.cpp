// Host build of the library's FP64 step (csrc/kernels.cuh: cell_poly_item,
// face_flux_item, update_item, the per-item functions of the GPU kernels) for
// the CPU tests, through the test-only CUDA stand-in in tests/hostshim: the
// two stages of one step run item by item in plain loops.  Arguments:
// M n0 n1 n2 h bc limiter [mu] (mu > 0: the Navier-Stokes flux).  stdin: dt,
// W[nv][cells], G[M][nv][cells].
// stdout: W then G after the step (one line each), then the status word.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>

#include "kernels.cuh"

template <int M, bool NS> static int step(gks::KP &P, double dt, std::vector<double> &W, std::vector<double> &G)
{
    constexpr int NV = M + 2, NC = gks::Cubic<double, M>::NC, NG = (M == 2) ? 2 : 4;
    const long nc = P.ncell;
    std::vector<double> Ws(W.size()), Gs(G.size()), Acc(W.size()), B((size_t)NV * NC * P.next),
        ff((size_t)3 * NV * NG * P.nftot);
    int status = 0;
    gks::UpdC uc{};
    const gks::Shadow none{nullptr, nullptr, nullptr};
    for (int stage = 1; stage <= 2; ++stage) {
        const gks::Src<double> src{stage == 1 ? W.data() : Ws.data(), stage == 1 ? G.data() : Gs.data()};
        for (long t = 0; t < P.next; ++t) gks::cell_poly_item<double, M>(P, src, B.data(), t);
        for (long t = 0; t < P.nface[0] * NG; ++t)
            gks::face_flux_item<double, M, 0, true, NS>(P, src, B.data(), dt, nullptr, ff.data(), &status, t);
        for (long t = 0; t < P.nface[1] * NG; ++t)
            gks::face_flux_item<double, M, 1, true, NS>(P, src, B.data(), dt, nullptr, ff.data(), &status, t);
        if constexpr (M == 3)
            for (long t = 0; t < P.nface[2] * NG; ++t)
                gks::face_flux_item<double, M, 2, true, NS>(P, src, B.data(), dt, nullptr, ff.data(), &status, t);
        for (long c = 0; c < nc; ++c) {
            if (stage == 1)
                gks::update_item<double, M, 1>(P, ff.data(), dt, W.data(), G.data(), Ws.data(), Gs.data(), Acc.data(),
                                               none, none, &status, c, uc);
            else
                gks::update_item<double, M, 2>(P, ff.data(), dt, W.data(), G.data(), Ws.data(), Gs.data(), Acc.data(),
                                               none, none, &status, c, uc);
        }
    }
    return status;
}

int main(int argc, char **argv)
{
    if (argc < 8) return 2;
    const double mu = argc > 8 ? std::atof(argv[8]) : 0.0;
    const int m = std::atoi(argv[1]);
    const int n[3] = {std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4])};
    const double h = std::atof(argv[5]);
    const int bc = std::atoi(argv[6]), limiter = std::atoi(argv[7]);
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
    for (int a = 0; a < 3; ++a) P.bcs[a][0] = P.bcs[a][1] = a < m ? bc : 0;
    P.limiter = limiter;
    P.h = h;
    P.ih = 1.0 / h;
    P.gamma = 1.4;
    P.C = 20.0;
    P.itanhC = 1.0 / std::tanh(20.0);
    P.eps = 1e-15;
    P.C0 = 8.0;
    P.adm = 0.3;
    P.d0 = 0.85;
    P.ct = 1e-6;
    P.fp.gamma = 1.4;
    P.fp.c1 = 0.05;
    P.fp.c2 = 1.0;
    P.fp.mu = mu;
    gks::finalize_kp(P);
    double dt;
    if (std::scanf("%lf", &dt) != 1) return 2;
    std::vector<double> W((size_t)(m + 2) * ncell), G((size_t)m * (m + 2) * ncell);
    for (double &x : W)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (double &x : G)
        if (std::scanf("%lf", &x) != 1) return 2;
    const int st = m == 2 ? (mu > 0 ? step<2, true>(P, dt, W, G) : step<2, false>(P, dt, W, G))
                          : (mu > 0 ? step<3, true>(P, dt, W, G) : step<3, false>(P, dt, W, G));
    for (size_t i = 0; i < W.size(); ++i) std::printf("%.17g%c", W[i], i + 1 < W.size() ? ' ' : '\n');
    for (size_t i = 0; i < G.size(); ++i) std::printf("%.17g%c", G[i], i + 1 < G.size() ? ' ' : '\n');
    std::printf("%d\n", st);
    return 0;
}
