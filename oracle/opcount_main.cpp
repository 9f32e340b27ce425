/*
 * Main program of the op-counting build of the oracle (TEST INFRASTRUCTURE ONLY).
 * oracle/opcount.py translates geno_gks_oracle.c to the counting scalar
 * (opcount.hpp) as oracle_ocn.inc and compiles this file with it.
 *
 * Usage (inputs as little-endian doubles on stdin, one JSON line per count):
 *   opcount selftest
 *   opcount gks  m ncases gamma c1 c2 tau_mode mu     per case Wl, Wr, dWl, dWr, dt
 *   opcount step|flux|recon dim n0 n1 n2 h dt gamma bc limiter    W, G of the grid
 *   opcount cell dim ncells limiter                   per cell the or_genomd_cell input
 *   opcount ncstep order n h dt gamma bc              W of a 1D grid (non-compact GENO, HLLC, RK4)
 * Data values enter as inputs (fresh nodes); the scheme constants, h and dt
 * as constants.
 */
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "opcount.hpp"
#include "oracle_ocn.inc"

namespace {

std::vector<double> read_doubles(size_t n)
{
    std::vector<double> v(n);
    if (n && std::fread(v.data(), sizeof(double), n, stdin) != n) {
        std::fprintf(stderr, "short input\n");
        std::exit(2);
    }
    return v;
}

std::vector<ocn> inputs(const std::vector<double> &v)
{
    std::vector<ocn> r(v.size());
    for (size_t i = 0; i < v.size(); ++i) r[i] = ocn::input(v[i]);
    return r;
}

void print_counts(const char *what, long units, const char *extra = "")
{
    const opc::Counters &c = opc::counters();
    std::printf("{\"what\": \"%s\", \"units\": %ld, \"add\": %llu, \"mul\": %llu, \"div\": %llu, \"exp\": %llu, "
                "\"erfc\": %llu, \"sqrt\": %llu, \"tanh\": %llu, \"absminmax\": %llu%s}\n",
                what, units, (unsigned long long)c.add, (unsigned long long)c.mul, (unsigned long long)c.div,
                (unsigned long long)c.exp, (unsigned long long)c.erfc, (unsigned long long)c.sqrt,
                (unsigned long long)c.tanh, (unsigned long long)c.absminmax, extra);
}

or_cfg make_cfg(int dim, const int *n, double h, double gamma, int bc, int limiter)
{
    or_cfg c;
    std::memset(&c, 0, sizeof c);
    c.dim = dim;
    for (int a = 0; a < 3; ++a) c.n[a] = n[a];
    c.h = h;
    c.gamma = gamma;
    c.bc = bc;
    c.C = 20.0;
    c.eps = 1e-15;
    c.C0 = 8.0;
    c.c1_tau = 0.05;
    c.c2_tau = 1.0;
    c.limiter = limiter;
    c.tau_mode = 0;
    c.adm_delta = 0.3;
    c.mu = 0.0;
    for (int s = 0; s < 6; ++s) c.bcs[s] = bc;
    c.ao_d0 = 0.85;
    c.teno_ct = 1e-6;
    return c;
}

void selftest()
{
    const ocn a = ocn::input(1.3), b = ocn::input(-0.7), c = ocn::input(2.1);
    opc::reset();
    { volatile long double r = (a * b + c).v; (void)r; }
    print_counts("a*b+c", 1); /* 1 mul, 1 add */
    opc::reset();
    { const ocn x = a + b, y = b + a; volatile long double r = (x * y).v; (void)r; }
    print_counts("(a+b)*(b+a)", 1); /* 1 add, 1 mul: the sum is shared */
    opc::reset();
    { volatile long double r = powl(a, ocn(7)).v; (void)r; }
    print_counts("a^7", 1); /* 4 mul */
    opc::reset();
    { volatile long double r = (a * 1.0 + 0.0 - 0.0 * b).v; (void)r; }
    print_counts("a*1+0-0*b", 1); /* nothing */
    opc::reset();
    { const ocn e1 = exp(a), e2 = exp(a); volatile long double r = (e1 + e2).v; (void)r; }
    print_counts("exp(a)+exp(a)", 1); /* 1 exp, 1 add */
    opc::reset();
    { volatile long double r = ((ocn(2.0) * ocn(3.0)) * a / ocn(-1.0)).v; (void)r; }
    print_counts("(2*3)*a/-1", 1); /* 1 mul */
    opc::reset();
    { volatile long double r = (fabs(a - b) / (a + b) + sqrt(c) + erfc(c) + tanh(c)).v; (void)r; }
    print_counts("|a-b|/(a+b)+sqrt+erfc+tanh", 1); /* 2 add + 3 add, 1 div, 1 sqrt, 1 erfc, 1 tanh, 1 abs */
}

} // namespace

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    const std::string mode = argv[1];
    if (mode == "selftest") {
        selftest();
        return 0;
    }
    if (mode == "gks") {
        const int m = std::atoi(argv[2]), ncase = std::atoi(argv[3]);
        const double gamma = std::atof(argv[4]), c1 = std::atof(argv[5]), c2 = std::atof(argv[6]);
        const int tau_mode = std::atoi(argv[7]);
        const double mu = std::atof(argv[8]);
        const int nv = m + 2;
        for (int k = 0; k < ncase; ++k) {
            const std::vector<double> d = read_doubles(2 * nv + 2 * m * nv + 1);
            opc::reset();
            std::vector<ocn> x = inputs(std::vector<double>(d.begin(), d.end() - 1));
            const ocn dt = d.back();
            ocn F[5], Ft[5], Wh[5];
            const int r = or_gks_point(m, gamma, c1, c2, tau_mode, mu, dt, x.data(), x.data() + nv, x.data() + 2 * nv,
                                       x.data() + 2 * nv + m * nv, F, Ft, Wh);
            print_counts("gks_point", 1, r ? ", \"status\": 1" : ", \"status\": 0");
        }
        return 0;
    }
    if (mode == "step" || mode == "flux" || mode == "recon") {
        const int dim = std::atoi(argv[2]);
        const int n[3] = {std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5])};
        const double h = std::atof(argv[6]), dt = std::atof(argv[7]), gamma = std::atof(argv[8]);
        const int bc = std::atoi(argv[9]), limiter = std::atoi(argv[10]);
        const or_cfg c = make_cfg(dim, n, h, gamma, bc, limiter);
        const long cells = (long)n[0] * n[1] * n[2];
        const int nv = dim + 2, ng = dim == 1 ? 1 : (dim == 2 ? 2 : 4);
        std::vector<ocn> W = inputs(read_doubles((size_t)nv * cells));
        std::vector<ocn> G = inputs(read_doubles((size_t)dim * nv * cells));
        const long nft = or_face_total(&c);
        opc::reset();
        int r;
        if (mode == "step") {
            r = or_step(&c, dt, W.data(), G.data());
        } else if (mode == "flux") {
            std::vector<ocn> out((size_t)3 * nv * ng * nft);
            r = or_flux(&c, dt, W.data(), G.data(), out.data());
        } else {
            std::vector<ocn> out((size_t)2 * nv * (dim + 1) * ng * nft);
            r = or_reconstruct(&c, W.data(), G.data(), out.data());
        }
        char extra[128];
        std::snprintf(extra, sizeof extra, ", \"faces\": %ld, \"gauss_points\": %ld, \"status\": %d", nft,
                      nft * ng, r);
        print_counts(mode.c_str(), cells, extra);
        return 0;
    }
    if (mode == "ncstep") {
        const int order = std::atoi(argv[2]);
        const int n[3] = {std::atoi(argv[3]), 1, 1};
        const double h = std::atof(argv[4]), dt = std::atof(argv[5]), gamma = std::atof(argv[6]);
        const int bc = std::atoi(argv[7]);
        const or_cfg c = make_cfg(1, n, h, gamma, bc, 0);
        std::vector<ocn> W = inputs(read_doubles((size_t)3 * n[0]));
        opc::reset();
        const int r = or_nc_step(&c, order, dt, W.data());
        char extra[64];
        std::snprintf(extra, sizeof extra, ", \"status\": %d", r);
        print_counts("ncstep", n[0], extra);
        return 0;
    }
    if (mode == "cell") {
        const int dim = std::atoi(argv[2]), ncell = std::atoi(argv[3]), limiter = std::atoi(argv[4]);
        const int n[3] = {4, 4, 4};
        const or_cfg c = make_cfg(dim, n, 1.0, 1.4, 0, limiter);
        const int nin = 1 + dim + 2 * dim * (1 + dim);
        for (int k = 0; k < ncell; ++k) {
            const std::vector<double> d = read_doubles(nin);
            opc::reset();
            std::vector<ocn> x = inputs(d);
            ocn out[64];
            const int r = or_genomd_cell(&c, x.data(), out);
            print_counts("genomd_cell", 1, r < 0 ? ", \"status\": 1" : ", \"status\": 0");
        }
        return 0;
    }
    return 2;
}
