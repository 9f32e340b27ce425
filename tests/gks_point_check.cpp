// Host build of the library's gas-kinetic flux at one interface point
// (csrc/gks_device.cuh, gks_point) for the CPU tests, through the test-only
// CUDA stand-in in tests/hostshim.  stdin: the case count, then per case
//   M NS prec gamma c1 c2 mu dt  Wl[M+2] Wr[M+2] dWl[M][M+2] dWr[M][M+2]
// (prec 0: double, 1: float, the FP32 path with the left/right lane pairs).
// stdout per case: status (1 = admissible) then F, dF/dt, W(dt/2).
#include <cstdio>
#include <cstdlib>
#include <initializer_list>

#include "gks_device.cuh"

template <typename R, int M, bool NS>
static void run(double gamma, double c1, double c2, double mu, double dt, const double *in)
{
    constexpr int NV = M + 2;
    gks::FluxParams fp{};
    fp.mu = mu;
    gks::fill_flux(fp, gamma, c1, c2);
    R Wl[NV], Wr[NV], dWl[M][NV], dWr[M][NV], F[NV], Ft[NV], Wh[NV];
    for (int b = 0; b < NV; ++b) {
        Wl[b] = (R)in[b];
        Wr[b] = (R)in[NV + b];
    }
    for (int e = 0; e < M; ++e)
        for (int b = 0; b < NV; ++b) {
            dWl[e][b] = (R)in[2 * NV + e * NV + b];
            dWr[e][b] = (R)in[2 * NV + M * NV + e * NV + b];
        }
    const bool ok = gks::gks_point<R, M, NS>(fp, (R)dt, Wl, Wr, dWl, dWr, F, Ft, Wh);
    std::printf("%d", ok ? 1 : 0);
    for (const R *q : {F, Ft, Wh})
        for (int b = 0; b < NV; ++b) std::printf(" %.17g", (double)q[b]);
    std::printf("\n");
}

template <int M> static void dispatch(int ns, int prec, double g, double c1, double c2, double mu, double dt, const double *in)
{
    if (prec == 0) ns ? run<double, M, true>(g, c1, c2, mu, dt, in) : run<double, M, false>(g, c1, c2, mu, dt, in);
    else ns ? run<float, M, true>(g, c1, c2, mu, dt, in) : run<float, M, false>(g, c1, c2, mu, dt, in);
}

int main()
{
    int ncase = 0;
    if (std::scanf("%d", &ncase) != 1) return 2;
    for (int k = 0; k < ncase; ++k) {
        int m, ns, prec;
        double g, c1, c2, mu, dt;
        if (std::scanf("%d %d %d %lf %lf %lf %lf %lf", &m, &ns, &prec, &g, &c1, &c2, &mu, &dt) != 8) return 2;
        const int nv = m + 2, n = 2 * nv + 2 * m * nv;
        double in[2 * 5 + 2 * 3 * 5];
        for (int i = 0; i < n; ++i)
            if (std::scanf("%lf", &in[i]) != 1) return 2;
        if (m == 1) dispatch<1>(ns, prec, g, c1, c2, mu, dt, in);
        else if (m == 2) dispatch<2>(ns, prec, g, c1, c2, mu, dt, in);
        else dispatch<3>(ns, prec, g, c1, c2, mu, dt, in);
    }
    return 0;
}
