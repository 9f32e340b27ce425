/*
 * Oracle for the compact gas-kinetic scheme (GKS) with GENO reconstruction
 * (Zhao & Xu, "A generalized ENO reconstruction in compact GKS for
 * compressible flow simulations", arXiv 2507.20461).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 restatement of
 * the method, used by the test-suite, the smoke check and the CPU baseline of
 * the benchmark to check the CUDA library.  The product path never calls it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is written the direct way:
 *   - every reconstruction polynomial is obtained by solving its moment
 *     conditions (square systems, or constrained least squares through the
 *     normal equations) in long double, per call;
 *   - smoothness indicators are integrals of squared derivatives evaluated by
 *     exact monomial integration;
 *   - every velocity-space integral of the gas-kinetic flux is formed by
 *     multiplying velocity polynomials term by term and integrating each
 *     monomial against the (half-space) Maxwellian;
 *   - micro-slopes are solved from the moment matrix <psi psi^T> by Gaussian
 *     elimination.
 *
 * Where the paper is silent (it defers the GKS flux and the two-stage
 * fourth-order time stepping to earlier work, Sec. 2) the readings used are:
 *   R1  conservative variables, component-wise GENO;
 *   R2  1D: S_2 (centred on the reconstruction cell) carries d = C0 = 8;
 *   R3  1D: the right interface state mirrors the left one about the face;
 *   R4  derivatives are blended with the same chi and omega as values;
 *   R5  multi-D on Cartesian cells: cubic p^3 from the face-neighbour cross by
 *       least squares (neighbour averages, neighbour averaged gradients and
 *       the own averaged gradient, unit weights in cell units) with the own
 *       average as a hard constraint; linear sub-polynomials on {cell, face
 *       neighbour} by least squares with the own average exact; every
 *       multi-index counted once in IS^H; r = 3, d_k = 1; in 3D the cubic
 *       omits xi eta zeta, which the face-neighbour data cannot determine;
 *   R6  GKS: BGK solution with the initial state built from the left/right
 *       states and their slopes, one equilibrium slope per direction taken
 *       from the mean of the left/right derivatives; the numerical collision
 *       time tau_n = C1 dt + C2 |pl - pr| / (pl + pr) dt enters only the
 *       exponential relaxation, the physical one (0 for the Euler equations)
 *       the Chapman-Enskog terms (C1 = 0.05, C2 = 1); for the Navier-Stokes
 *       equations the physical one is mu / p0 (Prandtl number 1) and is added
 *       to tau_n;
 *   R7  two-stage fourth-order update with F and dF/dt recovered from the
 *       time-integrated fluxes over dt/2 and dt; the cell-averaged gradients
 *       are refreshed from the interface states at dt/2 of each stage
 *       (Eq. slope, Gauss theorem);
 *   R8  boundary types per side; transmissive ghosts are the even extension
 *       (normal gradient negated),
 *       reflective ghosts also negate the normal momentum (an odd component),
 *       no-slip walls negate every momentum component; no wall face
 *       carries mass or energy flux (walls are at rest and adiabatic; at a
 *       no-slip wall the mirrored states alone leave a truncation-size mass
 *       flux through the tangential transport terms, at a slip wall one of
 *       the size of the rounding asymmetry of the two sides),
 *       periodic ghosts wrap;
 *   R14 WENO-Z / TENO variants (Sec. 5.1): the same candidates as GENO (the
 *       high-order polynomial with indicator IS^H, and the sub-stencil
 *       polynomials) in the adaptive-order combination
 *       (w0/d0) q^H + sum_k (w_k - (w0/d0) d_k) p_k with d0 = 0.85 and the
 *       sub-stencils sharing 1 - d0 as GENO's low-order weights do;
 *       tau_Z = IS^tau;
 *   R16 1D non-compact GENO (5th / 6th order, Sec. 4.1): the sub-stencil
 *       centred on the reconstruction cell carries d = C0; IS^tau takes the
 *       outer-left, outer-right and centred sub-stencils (6th order: S_1,
 *       S_4, S_2; the printed S_1..S_3 never see the stencil's last cell and
 *       leave chi = 1 across a jump there); HLLC with the
 *       Davis wave-speed bounds; classical RK4; the fallback of R9 and the
 *       wall fluxes of R8 as for the compact scheme;
 *   R9  a reconstructed interface state whose density or pressure is not
 *       above 0.3 times that of its cell average falls back to the cell
 *       average with zero slopes.
 *
 * Layouts (row-major, x fastest):
 *   W[v][k][j][i]          nv = dim + 2 conservative variables (rho, rho u.., rho E)
 *   G[d][v][k][j][i]       physical derivative d/dx_d of W
 *   faces of direction d:  extent n_d + 1 along d, n_e across; all x faces,
 *                          then y faces, then z faces
 *   face_states[side][v][c][g][face]  side 0 = minus cell, 1 = plus cell;
 *                          c = 0 value, 1 + e = d/dx_e (global axes)
 *   face_flux[q][v][g][face]  q = 0 flux F (time average over the step,
 *                          recovered at t^n), 1 dF/dt, 2 interface W(dt/2)
 * Gauss points: 1D one; 2D two at t = -/+ 1/(2 sqrt 3) (cell units, weights 1/2);
 * 3D 2x2 with index g = a + 2 b, a for the lower tangential axis.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NONPHYSICAL (-4)

typedef struct {
    int dim;
    int n[3];
    double h;
    double gamma;
    int bc; /* 0 periodic, 1 transmissive, 2 reflective (slip), 3 no-slip wall */
    double C;      /* path-function steepness, Eq. HLP-weight: 20 */
    double eps;    /* Eq. HLP-sp: 1e-15 */
    double C0;     /* central sub-stencil weight, Sec. 3.3: 8 */
    double c1_tau; /* R6 */
    double c2_tau; /* R6 */
    int limiter;   /* 0 GENO, 1 linear (chi = 1), 2 WENO-Z, 3 TENO (R14) */
    int tau_mode;  /* 0: Euler (physical tau = 0); 1: tau = tau_n (plain BGK);
                      2: Navier-Stokes, physical tau = mu / p0, tau_n = tau + ... */
    double adm_delta; /* R9 admissibility fraction: 0.3 */
    double mu;     /* dynamic viscosity for tau_mode 2 */
    int bcs[6];    /* per side (x lo, x hi, y lo, y hi, z lo, z hi), same codes
                      as bc, which they replace */
    double ao_d0;  /* R14: linear weight of the high-order candidate: 0.85 */
    double teno_ct; /* TENO cut-off C_T (Sec. 5.1): 1e-6 */
} or_cfg;

/* ------------------------------------------------------------------ */
/* Small dense solver: Gaussian elimination with partial pivoting.      */
/* ------------------------------------------------------------------ */
static int solve_ld(int n, long double *A, long double *b)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0L) return -1;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                long double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t;
            }
            long double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            long double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0L) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        long double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Spatial polynomials in cell units (cell 0 = [-1/2, 1/2]^m).          */
/* Monomials xi^a eta^b zeta^c of total degree <= deg.                   */
/* ------------------------------------------------------------------ */
#define SP_MAXMON 120 /* degree 7 in 1D: 8; degree 3 in 3D: 20; squares need more */
typedef struct { int m; int nmon; int e[SP_MAXMON][3]; } monset;

static void monset_build(monset *s, int m, int deg)
{
    s->m = m; s->nmon = 0;
    for (int t = 0; t <= deg; ++t)
        for (int a = t; a >= 0; --a)
            for (int b = t - a; b >= 0; --b) {
                int c = t - a - b;
                if (m < 2 && b) continue;
                if (m < 3 && c) continue;
                /* xi eta zeta: every average and averaged gradient of it over
                 * the seven-cell face-neighbour cross vanishes, so the compact
                 * 3D stencil cannot see it; the 3D cubic space omits it */
                if (a == 1 && b == 1 && c == 1) continue;
                s->e[s->nmon][0] = a; s->e[s->nmon][1] = b; s->e[s->nmon][2] = c;
                s->nmon++;
            }
}

static long double ipow(long double x, int k)
{
    long double r = 1.0L;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

/* average of xi^k over the unit cell centred at integer offset c */
static long double avg1(int k, int c)
{
    return (ipow(c + 0.5L, k + 1) - ipow(c - 0.5L, k + 1)) / (k + 1);
}

/* average over cell `off` of the monomial with exponents e, differentiated once along axis `dax` (-1: none) */
static long double mon_avg(const int e[3], const int off[3], int m, int dax)
{
    int ee[3] = {e[0], e[1], e[2]};
    long double f = 1.0L;
    if (dax >= 0) {
        if (ee[dax] == 0) return 0.0L;
        f = ee[dax];
        ee[dax] -= 1;
    }
    for (int a = 0; a < m; ++a) f *= avg1(ee[a], off[a]);
    return f;
}

static long double mon_eval(const int e[3], const long double x[3], int m, int dax)
{
    int ee[3] = {e[0], e[1], e[2]};
    long double f = 1.0L;
    if (dax >= 0) {
        if (ee[dax] == 0) return 0.0L;
        f = ee[dax];
        ee[dax] -= 1;
    }
    for (int a = 0; a < m; ++a) f *= ipow(x[a], ee[a]);
    return f;
}

/* A moment condition of a reconstruction: the average over cell `off` of p
 * (dax = -1) or of dp/dxi_dax equals `val`. */
typedef struct { int off[3]; int dax; long double val; } cond;

/* Square fit: as many monomials as conditions (1D stencils, Sec. 4.2). */
static int fit_square(const monset *s, int nc, const cond *cs, long double *coef)
{
    long double A[SP_MAXMON * SP_MAXMON];
    if (nc != s->nmon) return -1;
    for (int r = 0; r < nc; ++r) {
        for (int k = 0; k < nc; ++k) A[r * nc + k] = mon_avg(s->e[k], cs[r].off, s->m, cs[r].dax);
        coef[r] = cs[r].val;
    }
    return solve_ld(nc, A, coef);
}

/* Constrained least squares: average over cell 0 equals W0 exactly; the
 * remaining conditions in the least-squares sense with unit weights (R5).
 * Basis: phi_k = mon_k - avg_0(mon_k) for every non-constant monomial. */
static int fit_lsq(const monset *s, int nc, const cond *cs, long double W0, long double *coef)
{
    int nu = s->nmon - 1; /* monomial 0 is the constant */
    long double A[64 * 24], N[24 * 24], rhs[24];
    if (nu > 24 || nc > 64) return -1;
    for (int r = 0; r < nc; ++r) {
        int zero[3] = {0, 0, 0};
        for (int k = 0; k < nu; ++k) {
            long double v = mon_avg(s->e[k + 1], cs[r].off, s->m, cs[r].dax);
            if (cs[r].dax < 0) v -= mon_avg(s->e[k + 1], zero, s->m, -1);
            A[r * nu + k] = v;
        }
    }
    for (int a = 0; a < nu; ++a) {
        for (int b = 0; b < nu; ++b) {
            long double t = 0.0L;
            for (int r = 0; r < nc; ++r) t += A[r * nu + a] * A[r * nu + b];
            N[a * nu + b] = t;
        }
        long double t = 0.0L;
        for (int r = 0; r < nc; ++r) {
            long double d = cs[r].val - ((cs[r].dax < 0) ? W0 : 0.0L);
            t += A[r * nu + a] * d;
        }
        rhs[a] = t;
    }
    if (solve_ld(nu, N, rhs)) return -1;
    /* back to monomial coefficients */
    int zero[3] = {0, 0, 0};
    long double c0 = W0;
    for (int k = 0; k < nu; ++k) {
        coef[k + 1] = rhs[k];
        c0 -= rhs[k] * mon_avg(s->e[k + 1], zero, s->m, -1);
    }
    coef[0] = c0;
    return 0;
}

static long double poly_eval(const monset *s, const long double *coef, const long double x[3], int dax)
{
    long double v = 0.0L;
    for (int k = 0; k < s->nmon; ++k) v += coef[k] * mon_eval(s->e[k], x, s->m, dax);
    return v;
}

/* Integral over cell 0 of the square of the derivative D^l p, multi-index l. */
static long double int_sq_deriv(const monset *s, const long double *coef, const int l[3])
{
    /* derivative polynomial as a list of (coefficient, exponents) */
    long double dc[SP_MAXMON];
    int de[SP_MAXMON][3];
    int nd = 0;
    for (int k = 0; k < s->nmon; ++k) {
        long double f = coef[k];
        int e[3] = {s->e[k][0], s->e[k][1], s->e[k][2]};
        int ok = 1;
        for (int a = 0; a < 3 && ok; ++a)
            for (int t = 0; t < l[a]; ++t) {
                if (e[a] == 0) { ok = 0; break; }
                f *= e[a];
                e[a] -= 1;
            }
        if (!ok || f == 0.0L) continue;
        dc[nd] = f; de[nd][0] = e[0]; de[nd][1] = e[1]; de[nd][2] = e[2]; nd++;
    }
    long double r = 0.0L;
    int zero[3] = {0, 0, 0};
    for (int p = 0; p < nd; ++p)
        for (int q = 0; q < nd; ++q) {
            int e[3] = {de[p][0] + de[q][0], de[p][1] + de[q][1], de[p][2] + de[q][2]};
            r += dc[p] * dc[q] * mon_avg(e, zero, s->m, -1);
        }
    return r;
}

/* Smoothness indicator sum_{lo <= |l| <= hi} int (D^l p)^2 over cell 0, in
 * cell units, each multi-index once (Eq. IS-highorder-1; the h-powers cancel
 * against the cell-unit derivatives). */
static long double smooth_ind(const monset *s, const long double *coef, int lo, int hi)
{
    long double r = 0.0L;
    for (int t = lo; t <= hi; ++t)
        for (int a = t; a >= 0; --a)
            for (int b = t - a; b >= 0; --b) {
                int c = t - a - b;
                if (s->m < 2 && b) continue;
                if (s->m < 3 && c) continue;
                int l[3] = {a, b, c};
                r += int_sq_deriv(s, coef, l);
            }
    return r;
}

/* ------------------------------------------------------------------ */
/* GENO path function and weights (Sec. 3).                              */
/* ------------------------------------------------------------------ */
/* Eq. HLP-sp and Eq. HLP-weight */
static long double geno_chi(long double ISt, long double ISH, long double ISL, int r, long double eps, long double C)
{
    long double aH = 1.0L + powl(ISt / (ISH + eps), r);
    long double aL = 1.0L + powl(ISt / (ISL + eps), r);
    long double alpha = 2.0L * aH / (aH + aL);
    return tanhl(C * alpha) / tanhl(C);
}

/* WENO-Z weights (Eq. wgt-WENO-Z) or TENO weights (Eq. wgt-TENO-1 with the
 * exponent 7, Eq. wgt-TENO-2 with the cut-off C_T) over the candidates
 * k = 0 (the high-order polynomial, indicator IS^H) and k = 1..K (the
 * sub-stencil polynomials), linear weights d[0..K], tau_Z = IS^tau (R14).
 * Returns the normalised nonlinear weights w[0..K]. */
static void ao_weights(int limiter, int K, const long double *d, const long double *IS, long double tau,
                       long double eps, long double ct, long double *w)
{
    long double wt[8], s = 0.0L;
    if (limiter == 2) {
        for (int k = 0; k <= K; ++k) wt[k] = d[k] * (1.0L + tau / (IS[k] + eps));
    } else {
        long double g[8], gs = 0.0L;
        for (int k = 0; k <= K; ++k) { g[k] = powl(1.0L / (IS[k] + eps), 7); gs += g[k]; }
        for (int k = 0; k <= K; ++k) wt[k] = (g[k] / gs <= ct) ? 0.0L : d[k];
    }
    for (int k = 0; k <= K; ++k) s += wt[k];
    for (int k = 0; k <= K; ++k) w[k] = wt[k] / s;
}

/* ------------------------------------------------------------------ */
/* 1D eighth-order compact GENO reconstruction (Sec. 4.2).               */
/* Reconstruction cell at offset 0 in the arrays w[-2..2], d[-2..2]       */
/* (averages and cell-unit averaged derivatives h W_x, index +2 shift).  */
/* side 0: left state at xi = +1/2 with S0 = {-1..2}, S1 = {-1,0} (plus   */
/* the derivative on -1), S2 = {-1,0,1}, S3 = {0,1,2}.  side 1: mirror.   */
/* ------------------------------------------------------------------ */
typedef struct { double val, der, chi, IS[3], ISH, ISL, ISt; } geno1d_out;

static int geno1d(const double *w5, const double *d5, int side, const or_cfg *cfg, geno1d_out *o)
{
    int sg = side ? -1 : 1; /* offsets are mirrored for the right state */
    monset s7, s2;
    monset_build(&s7, 1, 7);
    monset_build(&s2, 1, 2);
    long double x[3] = {0.5L * sg, 0, 0};
#define W_AT(o_) ((long double)w5[(o_) + 2])
#define D_AT(o_) ((long double)d5[(o_) + 2])
    /* p^7 on S0 = {-1, 0, 1, 2} (mirrored for side 1): averages and averaged derivatives */
    cond c7[8];
    int k = 0;
    for (int q = -1; q <= 2; ++q) {
        int o_ = sg * q;
        c7[k].off[0] = o_; c7[k].off[1] = c7[k].off[2] = 0; c7[k].dax = -1; c7[k].val = W_AT(o_); k++;
        c7[k].off[0] = o_; c7[k].off[1] = c7[k].off[2] = 0; c7[k].dax = 0;
        c7[k].val = D_AT(o_); k++;
    }
    long double a7[8];
    if (fit_square(&s7, 8, c7, a7)) return -1;
    long double pH = poly_eval(&s7, a7, x, -1);
    long double pHd = poly_eval(&s7, a7, x, 0);

    /* three quadratics */
    cond cq[3][3];
    /* S1: average and averaged derivative on -1, average on 0 */
    cq[0][0] = (cond){{-sg, 0, 0}, -1, W_AT(-sg)};
    cq[0][1] = (cond){{-sg, 0, 0}, 0, D_AT(-sg)};
    cq[0][2] = (cond){{0, 0, 0}, -1, W_AT(0)};
    /* S2: averages on -1, 0, 1 (central) */
    for (int q = 0; q < 3; ++q) cq[1][q] = (cond){{sg * (q - 1), 0, 0}, -1, W_AT(sg * (q - 1))};
    /* S3: averages on 0, 1, 2 */
    for (int q = 0; q < 3; ++q) cq[2][q] = (cond){{sg * q, 0, 0}, -1, W_AT(sg * q)};
#undef W_AT
#undef D_AT
    long double aq[3][3], IS[3], pv[3], pd[3];
    for (int j = 0; j < 3; ++j) {
        if (fit_square(&s2, 3, cq[j], aq[j])) return -1;
        IS[j] = smooth_ind(&s2, aq[j], 1, 2);
        pv[j] = poly_eval(&s2, aq[j], x, -1);
        pd[j] = poly_eval(&s2, aq[j], x, 0);
    }
    long double eps = cfg->eps;
    long double ISH = IS[0], ISL = IS[0];
    for (int j = 1; j < 3; ++j) { if (IS[j] > ISH) ISH = IS[j]; if (IS[j] < ISL) ISL = IS[j]; } /* Eq. IS-highorder-2, Eq. HLP-IS-loworder-2 */
    long double ISt = fabsl((IS[1] + IS[2]) / 2.0L - IS[0]); /* Eq. 6th-compact-path */
    long double chi = (cfg->limiter == 1) ? 1.0L : geno_chi(ISt, ISH, ISL, 2, eps, cfg->C);
    long double d[3] = {1.0L, cfg->C0, 1.0L}, wt[3], ws = 0.0L;
    for (int j = 0; j < 3; ++j) { wt[j] = d[j] / ((IS[j] + eps) * (IS[j] + eps)); ws += wt[j]; } /* Eq. HLP-q-loworder */
    long double qL = 0.0L, qLd = 0.0L;
    for (int j = 0; j < 3; ++j) { qL += wt[j] / ws * pv[j]; qLd += wt[j] / ws * pd[j]; }
    o->val = (double)(chi * pH + (1.0L - chi) * qL); /* Eq. 8th-compact-HLP */
    o->der = (double)(chi * pHd + (1.0L - chi) * qLd);
    if (cfg->limiter >= 2) {
        /* R14: R = (w0/d0) p^7 + sum_k (w_k - (w0/d0) d_k) p_k, the sub-stencils
         * sharing 1 - d0 in GENO's low-order proportions (1, C0, 1) */
        long double d0 = cfg->ao_d0, dd[4] = {d0, 0, 0, 0}, I4[4] = {ISH, IS[0], IS[1], IS[2]}, w[4];
        for (int j = 0; j < 3; ++j) dd[j + 1] = (1.0L - d0) * d[j] / (cfg->C0 + 2.0L);
        ao_weights(cfg->limiter, 3, dd, I4, ISt, eps, cfg->teno_ct, w);
        chi = w[0] / d0;
        long double v = chi * pH, dv = chi * pHd;
        for (int j = 0; j < 3; ++j) { v += (w[j + 1] - chi * dd[j + 1]) * pv[j]; dv += (w[j + 1] - chi * dd[j + 1]) * pd[j]; }
        o->val = (double)v;
        o->der = (double)dv;
    }
    o->chi = (double)chi;
    for (int j = 0; j < 3; ++j) o->IS[j] = (double)IS[j];
    o->ISH = (double)ISH; o->ISL = (double)ISL; o->ISt = (double)ISt;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Multi-D compact GENO on Cartesian cells (Sec. 4.3, reading R5).       */
/* data: W0; D0[m] own averaged gradient (cell units); for neighbour     */
/* q = 2 e + (s>0): Wn[q], Dn[q][m].  Output: the blended cubic.          */
/* ------------------------------------------------------------------ */
typedef struct { long double coef[20]; double chi, ISH, ISL, ISt, IS[6]; } genomd_out;

static int genomd(int m, double W0, const double *D0, const double *Wn, const double (*Dn)[3], const or_cfg *cfg,
                  genomd_out *o)
{
    monset s3, s1;
    monset_build(&s3, m, 3);
    monset_build(&s1, m, 1);
    cond cs[32];
    memset(cs, 0, sizeof cs);
    int nc = 0;
    for (int e = 0; e < m; ++e)
        for (int sgn = 0; sgn < 2; ++sgn) {
            int q = 2 * e + sgn;
            int off[3] = {0, 0, 0};
            off[e] = sgn ? 1 : -1;
            cs[nc] = (cond){{off[0], off[1], off[2]}, -1, Wn[q]}; nc++;
            for (int a = 0; a < m; ++a) { cs[nc] = (cond){{off[0], off[1], off[2]}, a, Dn[q][a]}; nc++; }
        }
    for (int a = 0; a < m; ++a) { cs[nc] = (cond){{0, 0, 0}, a, D0[a]}; nc++; }
    long double c3[20];
    if (fit_lsq(&s3, nc, cs, W0, c3)) return -1;

    /* linear polynomials on {cell, face neighbour} */
    long double c1[6][4], IS[6];
    int k0 = 2 * m;
    for (int q = 0; q < k0; ++q) {
        int e = q / 2, sgn = q % 2;
        int off[3] = {0, 0, 0};
        off[e] = sgn ? 1 : -1;
        cond cl[4];
        int ncl = 0;
        cl[ncl++] = (cond){{off[0], off[1], off[2]}, -1, Wn[q]};
        for (int a = 0; a < m; ++a) cl[ncl++] = (cond){{off[0], off[1], off[2]}, a, Dn[q][a]};
        if (fit_lsq(&s1, ncl, cl, W0, c1[q])) return -1;
        IS[q] = smooth_ind(&s1, c1[q], 1, 1);
    }
    long double ISH = smooth_ind(&s3, c3, 1, 3);   /* Eq. IS-highorder-1 */
    long double ISHt = smooth_ind(&s3, c3, 1, 2);  /* auxiliary indicator, |l| <= 2 */
    long double ISt = fabsl(ISH - ISHt);           /* Eq. IS-tau */
    long double smin = IS[0], smax = IS[0], ssum = 0.0L;
    for (int q = 0; q < k0; ++q) { ssum += IS[q]; if (IS[q] < smin) smin = IS[q]; if (IS[q] > smax) smax = IS[q]; }
    long double ISL = (ssum - smin - smax) / (k0 - 2); /* Eq. HLP-IS-loworder-3 */
    long double eps = cfg->eps;
    long double chi = (cfg->limiter == 1) ? 1.0L : geno_chi(ISt, ISH, ISL, 3, eps, cfg->C);
    long double wt[6], ws = 0.0L;
    for (int q = 0; q < k0; ++q) { wt[q] = 1.0L / ((IS[q] + eps) * (IS[q] + eps)); ws += wt[q]; }
    /* blended polynomial in the cubic's monomial basis; the linear
     * monomials come first after the constant (monset ordering by degree) */
    for (int k = 0; k < s3.nmon; ++k) o->coef[k] = chi * c3[k];
    if (cfg->limiter >= 2) {
        /* R14: (w0/d0) p^3 + sum_q (w_q - (w0/d0) d_q) p_q, the 2m linear
         * polynomials sharing 1 - d0 equally */
        long double d0 = cfg->ao_d0, dd[7], I7[7], w[7];
        dd[0] = d0; I7[0] = ISH;
        for (int q = 0; q < k0; ++q) { dd[q + 1] = (1.0L - d0) / k0; I7[q + 1] = IS[q]; }
        ao_weights(cfg->limiter, k0, dd, I7, ISt, eps, cfg->teno_ct, w);
        chi = w[0] / d0;
        for (int k = 0; k < s3.nmon; ++k) o->coef[k] = chi * c3[k];
        for (int q = 0; q < k0; ++q)
            for (int k = 0; k < s1.nmon; ++k) o->coef[k] += (w[q + 1] - chi * dd[q + 1]) * c1[q][k];
    } else {
        for (int q = 0; q < k0; ++q)
            for (int k = 0; k < s1.nmon; ++k) o->coef[k] += (1.0L - chi) * wt[q] / ws * c1[q][k];
    }
    o->chi = (double)chi; o->ISH = (double)ISH; o->ISL = (double)ISL; o->ISt = (double)ISt;
    for (int q = 0; q < k0; ++q) o->IS[q] = (double)IS[q];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Velocity-space polynomials and Maxwellian moments (GKS, reading R6).  */
/* A term is c * u^a v^b w^c (xi^2)^d; the Maxwellian                     */
/*   g = rho (lam/pi)^((K+m)/2) exp(-lam (|u - U|^2 + xi^2))              */
/* has m translational and K internal degrees of freedom.                */
/* ------------------------------------------------------------------ */
#define VP_MAX 160
typedef struct { int n; double c[VP_MAX]; unsigned char e[VP_MAX][4]; } vpoly;
typedef struct { int m; double rho, U[3], lam, K; } maxw;

static void vp_zero(vpoly *p) { p->n = 0; }

static void vp_add(vpoly *p, double c, int a, int b, int cc, int d)
{
    if (c == 0.0) return;
    for (int k = 0; k < p->n; ++k)
        if (p->e[k][0] == a && p->e[k][1] == b && p->e[k][2] == cc && p->e[k][3] == d) { p->c[k] += c; return; }
    if (p->n >= VP_MAX) abort();
    p->c[p->n] = c; p->e[p->n][0] = a; p->e[p->n][1] = b; p->e[p->n][2] = cc; p->e[p->n][3] = d; p->n++;
}

static void vp_mul(const vpoly *x, const vpoly *y, vpoly *out)
{
    vpoly r; vp_zero(&r);
    for (int i = 0; i < x->n; ++i)
        for (int j = 0; j < y->n; ++j)
            vp_add(&r, x->c[i] * y->c[j], x->e[i][0] + y->e[j][0], x->e[i][1] + y->e[j][1],
                   x->e[i][2] + y->e[j][2], x->e[i][3] + y->e[j][3]);
    *out = r;
}

/* psi_a: 1, u, v, w (first m), 1/2(|u|^2 + xi^2) */
static void vp_psi(int m, int a, vpoly *p)
{
    vp_zero(p);
    if (a == 0) { vp_add(p, 1.0, 0, 0, 0, 0); return; }
    if (a <= m) { vp_add(p, 1.0, a == 1, a == 2, a == 3, 0); return; }
    vp_add(p, 0.5, 2, 0, 0, 0);
    if (m >= 2) vp_add(p, 0.5, 0, 2, 0, 0);
    if (m >= 3) vp_add(p, 0.5, 0, 0, 2, 0);
    vp_add(p, 0.5, 0, 0, 0, 1);
}

/* velocity component k (0 = normal u, 1 = v, 2 = w) as a polynomial */
static void vp_vel(int k, vpoly *p)
{
    vp_zero(p);
    vp_add(p, 1.0, k == 0, k == 1, k == 2, 0);
}

/* a = sum_b s_b psi_b */
static void vp_from_coef(int m, const double *s, vpoly *p)
{
    vp_zero(p);
    for (int b = 0; b < m + 2; ++b) {
        vpoly q; vp_psi(m, b, &q);
        for (int k = 0; k < q.n; ++k) vp_add(p, s[b] * q.c[k], q.e[k][0], q.e[k][1], q.e[k][2], q.e[k][3]);
    }
}

/* Full-space moments E[u^n] of a normal variable with mean U and variance
 * 1/(2 lam): E[u^{n+2}] = U E[u^{n+1}] + (n+1)/(2 lam) E[u^n]. */
static double mom_full(int n, double U, double lam)
{
    double a = 1.0, b = U;
    if (n == 0) return a;
    for (int k = 0; k + 1 < n; ++k) { double c = U * b + (k + 1) / (2.0 * lam) * a; a = b; b = c; }
    return b;
}

/* Half-space moments int_{u>0} (or u<0) u^n sqrt(lam/pi) exp(-lam (u-U)^2) du.
 * n = 0: erfc(-/+ sqrt(lam) U)/2; n = 1: U m0 +/- exp(-lam U^2) / (2 sqrt(pi lam));
 * the same recursion as the full-space moments (integration by parts). */
double or_mom_half(int n, double U, double lam, int sign)
{
    double sl = sqrt(lam);
    double a, b;
    if (sign > 0) {
        a = 0.5 * erfc(-sl * U);
        b = U * a + 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    } else {
        a = 0.5 * erfc(sl * U);
        b = U * a - 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    }
    if (n == 0) return a;
    for (int k = 0; k + 1 < n; ++k) { double c = U * b + (k + 1) / (2.0 * lam) * a; a = b; b = c; }
    return b;
}

/* E[(xi^2)^d] for K internal degrees of freedom of variance 1/(2 lam) each */
static double mom_xi(int d, double K, double lam)
{
    double r = 1.0;
    for (int i = 0; i < d; ++i) r *= (K + 2.0 * i) / (2.0 * lam);
    return r;
}

/* <p> = (1/rho) int p g; half = +1 / -1 restricts the normal velocity u */
static double vp_moment(const vpoly *p, const maxw *g, int half)
{
    double r = 0.0;
    for (int k = 0; k < p->n; ++k) {
        int a = p->e[k][0], b = p->e[k][1], c = p->e[k][2], d = p->e[k][3];
        double t = p->c[k];
        t *= half ? or_mom_half(a, g->U[0], g->lam, half) : mom_full(a, g->U[0], g->lam);
        if (b) t *= mom_full(b, g->U[1], g->lam);
        if (c) t *= mom_full(c, g->U[2], g->lam);
        if (d) t *= mom_xi(d, g->K, g->lam);
        r += t;
    }
    return r;
}

static int to_maxw(int m, double gamma, const double *W, maxw *g)
{
    g->m = m;
    g->rho = W[0];
    double ke = 0.0;
    for (int a = 0; a < 3; ++a) g->U[a] = 0.0;
    for (int a = 0; a < m; ++a) { g->U[a] = W[1 + a] / W[0]; ke += g->U[a] * g->U[a]; }
    double p = (gamma - 1.0) * (W[m + 1] - 0.5 * W[0] * ke);
    g->lam = W[0] / (2.0 * p);
    g->K = 2.0 / (gamma - 1.0) - m; /* N - m internal degrees, N = 2/(gamma-1) in total */
    if (!(W[0] > 0.0) || !(p > 0.0)) return -1;
    return 0;
}

/* Solve <a psi> = rhs for a = sum s_b psi_b with the moment matrix <psi_a psi_b>. */
static int slope_solve(const maxw *g, const double *rhs, double *s)
{
    int nv = g->m + 2;
    long double A[25], b[5];
    for (int i = 0; i < nv; ++i) {
        vpoly pi; vp_psi(g->m, i, &pi);
        for (int j = 0; j < nv; ++j) {
            vpoly pj, pp; vp_psi(g->m, j, &pj);
            vp_mul(&pi, &pj, &pp);
            A[i * nv + j] = vp_moment(&pp, g, 0);
        }
        b[i] = rhs[i];
    }
    if (solve_ld(nv, A, b)) return -1;
    for (int i = 0; i < nv; ++i) s[i] = (double)b[i];
    return 0;
}

/* <X psi_a> and <X u psi_a> for every a, against Maxwellian g (half-space flag) */
static void vp_mom_psi(const vpoly *X, const maxw *g, int half, int with_u, double *out)
{
    vpoly u; vp_vel(0, &u);
    vpoly Xu;
    if (with_u) vp_mul(X, &u, &Xu); else Xu = *X;
    for (int a = 0; a < g->m + 2; ++a) {
        vpoly pa, t; vp_psi(g->m, a, &pa);
        vp_mul(&Xu, &pa, &t);
        out[a] = vp_moment(&t, g, half);
    }
}

/* One interface Gauss point in the face frame (velocity component 0 and
 * derivative axis 0 are along the face normal).  dWl[e][a]: derivative of
 * W_a along face axis e on the left, physical units. */
static int gks_point(int m, double gamma, double c1, double c2, int tau_mode, double mu, double dt, const double *Wl,
                     const double *Wr, double dWl[3][5], double dWr[3][5], double *F, double *Ft, double *Wh)
{
    int nv = m + 2;
    maxw gl, gr, g0;
    if (to_maxw(m, gamma, Wl, &gl) || to_maxw(m, gamma, Wr, &gr)) return -1;
    /* equilibrium state at the interface: kinetic collision of the two sides */
    double W0[5] = {0, 0, 0, 0, 0};
    vpoly one; vp_zero(&one); vp_add(&one, 1.0, 0, 0, 0, 0);
    double ml[5], mr[5];
    vp_mom_psi(&one, &gl, +1, 0, ml);
    vp_mom_psi(&one, &gr, -1, 0, mr);
    for (int a = 0; a < nv; ++a) W0[a] = gl.rho * ml[a] + gr.rho * mr[a];
    if (to_maxw(m, gamma, W0, &g0)) return -1;

    /* micro-slopes along each face axis and the spatial part T = sum_e s_e * vel_e */
    vpoly Tl, Tr, T0;
    vp_zero(&Tl); vp_zero(&Tr); vp_zero(&T0);
    for (int e = 0; e < m; ++e) {
        double rl[5], rr[5], r0[5], sl[5], sr[5], s0[5];
        for (int a = 0; a < nv; ++a) {
            rl[a] = dWl[e][a] / gl.rho;
            rr[a] = dWr[e][a] / gr.rho;
            r0[a] = 0.5 * (dWl[e][a] + dWr[e][a]) / g0.rho;
        }
        if (slope_solve(&gl, rl, sl) || slope_solve(&gr, rr, sr) || slope_solve(&g0, r0, s0)) return -1;
        vpoly pl, pr, p0, ve, t;
        vp_from_coef(m, sl, &pl); vp_from_coef(m, sr, &pr); vp_from_coef(m, s0, &p0);
        vp_vel(e, &ve);
        vp_mul(&pl, &ve, &t); for (int k = 0; k < t.n; ++k) vp_add(&Tl, t.c[k], t.e[k][0], t.e[k][1], t.e[k][2], t.e[k][3]);
        vp_mul(&pr, &ve, &t); for (int k = 0; k < t.n; ++k) vp_add(&Tr, t.c[k], t.e[k][0], t.e[k][1], t.e[k][2], t.e[k][3]);
        vp_mul(&p0, &ve, &t); for (int k = 0; k < t.n; ++k) vp_add(&T0, t.c[k], t.e[k][0], t.e[k][1], t.e[k][2], t.e[k][3]);
    }
    /* time coefficients from the compatibility condition <(T + A) psi> = 0 */
    double rhs[5], sA[5];
    vpoly Al, Ar, A0;
    vp_mom_psi(&Tl, &gl, 0, 0, rhs); for (int a = 0; a < nv; ++a) rhs[a] = -rhs[a];
    if (slope_solve(&gl, rhs, sA)) return -1;
    vp_from_coef(m, sA, &Al);
    vp_mom_psi(&Tr, &gr, 0, 0, rhs); for (int a = 0; a < nv; ++a) rhs[a] = -rhs[a];
    if (slope_solve(&gr, rhs, sA)) return -1;
    vp_from_coef(m, sA, &Ar);
    vp_mom_psi(&T0, &g0, 0, 0, rhs); for (int a = 0; a < nv; ++a) rhs[a] = -rhs[a];
    if (slope_solve(&g0, rhs, sA)) return -1;
    vp_from_coef(m, sA, &A0);

    /* numerical collision time tau_n (exponential relaxation only) and the
     * physical collision time tau of the Chapman-Enskog terms: 0 for the
     * Euler equations, tau_n for the plain BGK solution */
    double pl = Wl[0] / (2.0 * gl.lam), pr = Wr[0] / (2.0 * gr.lam);
    double tn = c1 * dt + c2 * fabs(pl - pr) / (pl + pr) * dt;
    double tau = (tau_mode == 1) ? tn : 0.0;
    if (tau_mode == 2) {
        /* Navier-Stokes: the physical collision time from the interface
         * equilibrium, tau = mu / p0 (Prandtl number 1), enters both */
        tau = mu / (g0.rho / (2.0 * g0.lam));
        tn += tau;
    }

    /* the velocity moments the flux and interface state need */
    double e0u[5], eTu[5], eAu[5], fl[5], fr[5], flT[5], frT[5], flA[5], frA[5];
    vp_mom_psi(&one, &g0, 0, 1, e0u);
    vp_mom_psi(&T0, &g0, 0, 1, eTu);
    vp_mom_psi(&A0, &g0, 0, 1, eAu);
    vp_mom_psi(&one, &gl, +1, 1, fl);
    vp_mom_psi(&one, &gr, -1, 1, fr);
    vp_mom_psi(&Tl, &gl, +1, 1, flT);
    vp_mom_psi(&Tr, &gr, -1, 1, frT);
    vp_mom_psi(&Al, &gl, +1, 1, flA);
    vp_mom_psi(&Ar, &gr, -1, 1, frA);

    /* f(0,t) = (1-e) g0 + ((t+tau) e - tau) T0 g0 + (t - tau + tau e) A0 g0
     *        + e [(1 - (t+tau) T_l - tau A_l) H(u) g_l + (1 - (t+tau) T_r - tau A_r) H(-u) g_r],
     * e = exp(-t/tau_n); q0..q5 are the time integrals of the six coefficients */
    double Fi[2][5];
    for (int s = 0; s < 2; ++s) {
        double d = s ? dt : 0.5 * dt;
        double e = (tn > 0.0) ? exp(-d / tn) : 0.0;
        double ite = tn * tn - tn * (d + tn) * e; /* int_0^d t e dt */
        double ie = tn * (1.0 - e);               /* int_0^d e dt */
        double q0 = d - ie;
        double q1 = ite + tau * ie - tau * d;
        double q2 = 0.5 * d * d - tau * d + tau * ie;
        double q3 = ie;
        double q4 = ite + tau * ie;
        double q5 = tau * ie;
        for (int a = 0; a < nv; ++a)
            Fi[s][a] = g0.rho * (q0 * e0u[a] + q1 * eTu[a] + q2 * eAu[a]) + q3 * (gl.rho * fl[a] + gr.rho * fr[a]) -
                       q4 * (gl.rho * flT[a] + gr.rho * frT[a]) - q5 * (gl.rho * flA[a] + gr.rho * frA[a]);
    }
    for (int a = 0; a < nv; ++a) {
        F[a] = (4.0 * Fi[0][a] - Fi[1][a]) / dt;
        Ft[a] = 4.0 * (Fi[1][a] - 2.0 * Fi[0][a]) / (dt * dt);
    }
    /* interface state W(t) = int psi f(0, t), t = dt/2 */
    double e0[5], eT[5], eA[5], hl[5], hr[5], hlT[5], hrT[5], hlA[5], hrA[5];
    vp_mom_psi(&one, &g0, 0, 0, e0);
    vp_mom_psi(&T0, &g0, 0, 0, eT);
    vp_mom_psi(&A0, &g0, 0, 0, eA);
    vp_mom_psi(&one, &gl, +1, 0, hl);
    vp_mom_psi(&one, &gr, -1, 0, hr);
    vp_mom_psi(&Tl, &gl, +1, 0, hlT);
    vp_mom_psi(&Tr, &gr, -1, 0, hrT);
    vp_mom_psi(&Al, &gl, +1, 0, hlA);
    vp_mom_psi(&Ar, &gr, -1, 0, hrA);
    double t = 0.5 * dt;
    double et = (tn > 0.0) ? exp(-t / tn) : 0.0;
    for (int a = 0; a < nv; ++a)
        Wh[a] = (1.0 - et) * g0.rho * e0[a] + ((t + tau) * et - tau) * g0.rho * eT[a] +
                (t - tau + tau * et) * g0.rho * eA[a] + et * (gl.rho * hl[a] + gr.rho * hr[a]) -
                (t + tau) * et * (gl.rho * hlT[a] + gr.rho * hrT[a]) - tau * et * (gl.rho * hlA[a] + gr.rho * hrA[a]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid helpers: ghost cells by index mapping (reading R8).              */
/* ------------------------------------------------------------------ */
static long cells(const or_cfg *c) { return (long)c->n[0] * c->n[1] * c->n[2]; }

/* Fetch W and G of the (possibly ghost) cell (i, j, k); G in cell units
 * (h * grad W).  Returns the sign-adjusted copy. */
static void fetch(const or_cfg *c, const double *W, const double *G, int i, int j, int k, double *w, double (*g)[5])
{
    int m = c->dim, nv = m + 2;
    int idx[3] = {i, j, k};
    /* per axis: parity of the mirrors crossed, and of the crossings that
     * negate the normal momentum (reflective, no-slip) and the tangential
     * momenta (no-slip) */
    int mir[3] = {0, 0, 0}, odd_n[3] = {0, 0, 0}, odd_t[3] = {0, 0, 0};
    for (int a = 0; a < m; ++a) {
        int n = c->n[a];
        int x = idx[a];
        int lo = c->bcs[2 * a], hi = c->bcs[2 * a + 1];
        if (lo == 0) {
            x %= n; if (x < 0) x += n;
        } else {
            while (x < 0 || x >= n) {
                int t;
                if (x < 0) { x = -1 - x; t = lo; }
                else { x = 2 * n - 1 - x; t = hi; }
                mir[a] ^= 1;
                if (t >= 2) odd_n[a] ^= 1;
                if (t == 3) odd_t[a] ^= 1;
            }
        }
        idx[a] = x;
    }
    long nc = cells(c);
    long cell = ((long)idx[2] * c->n[1] + idx[1]) * c->n[0] + idx[0];
    for (int v = 0; v < nv; ++v) {
        /* mirror image: even extension of every variable (transmissive); a
         * reflective wall also negates the momentum normal to it, a no-slip
         * wall every momentum component (R8) */
        double sv = 1.0;
        for (int a = 0; a < m; ++a) {
            if (v == 1 + a && odd_n[a]) sv = -sv;
            if (v >= 1 && v <= m && v != 1 + a && odd_t[a]) sv = -sv;
        }
        w[v] = sv * W[v * nc + cell];
        for (int a = 0; a < m; ++a) {
            double x = sv * G[(a * nv + v) * nc + cell] * c->h;
            g[a][v] = mir[a] ? -x : x;
        }
    }
}

static long face_count(const or_cfg *c, int d)
{
    long r = 1;
    for (int a = 0; a < c->dim; ++a) r *= (a == d) ? (c->n[a] + 1) : c->n[a];
    return r;
}

static long face_total(const or_cfg *c)
{
    long r = 0;
    for (int d = 0; d < c->dim; ++d) r += face_count(c, d);
    return r;
}

static int ngauss(int m) { return m == 1 ? 1 : (m == 2 ? 2 : 4); }

/* tangential Gauss coordinates (cell units) of point g on a face normal to d */
static void gauss_pt(int m, int d, int g, long double x[3])
{
    const long double s = 0.5L / sqrtl(3.0L);
    int t[2], nt = 0;
    for (int a = 0; a < m; ++a) if (a != d) t[nt++] = a;
    x[0] = x[1] = x[2] = 0.0L;
    if (nt >= 1) x[t[0]] = (g & 1) ? s : -s;
    if (nt >= 2) x[t[1]] = (g & 2) ? s : -s;
}

/* Reading R9: a reconstructed interface state whose density or pressure is
 * not above adm_delta times that of its reconstruction cell's average is
 * replaced by the cell average with zero slopes. */
static double pressure(int m, double gamma, const double *w)
{
    double ke = 0.0;
    for (int a = 0; a < m; ++a) ke += w[1 + a] * w[1 + a];
    return (gamma - 1.0) * (w[m + 1] - 0.5 * ke / w[0]);
}
static int admissible(int m, double gamma, double delta, const double *w, const double *wc)
{
    if (!(w[0] > delta * wc[0])) return 0;
    return pressure(m, gamma, w) > delta * pressure(m, gamma, wc);
}

static int check_cfg(const or_cfg *c)
{
    if (c->dim < 1 || c->dim > 3) return OR_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (a < c->dim && c->n[a] < 1) return OR_ERR_ARG;
        if (a >= c->dim && c->n[a] != 1) return OR_ERR_ARG;
    }
    if (!(c->h > 0.0) || !(c->gamma > 1.0)) return OR_ERR_ARG;
    for (int a = 0; a < c->dim; ++a) {
        int lo = c->bcs[2 * a], hi = c->bcs[2 * a + 1];
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return OR_ERR_ARG;
        if ((lo == 0) != (hi == 0)) return OR_ERR_ARG; /* periodic pairs */
    }
    if (c->tau_mode == 2 && !(c->mu >= 0.0)) return OR_ERR_ARG;
    if (!(c->adm_delta >= 0.0) || c->adm_delta >= 1.0) return OR_ERR_ARG;
    if (c->limiter < 0 || c->limiter > 3) return OR_ERR_ARG;
    if (c->limiter >= 2 && (!(c->ao_d0 > 0.0) || !(c->ao_d0 < 1.0) || !(c->teno_ct > 0.0) || !(c->teno_ct < 1.0)))
        return OR_ERR_ARG;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Interface states at every face Gauss point.                           */
/* ------------------------------------------------------------------ */
static int recon_all(const or_cfg *c, const double *W, const double *G, double *out)
{
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nft = face_total(c);
    int err = 0;
    if (m == 1) {
        int n = c->n[0];
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int f = 0; f <= n; ++f) {
            /* face f lies between cells f-1 and f; left reconstruction cell f-1 */
            for (int side = 0; side < 2; ++side) {
                int rc = side ? f : f - 1;
                double val[5] = {0}, der[5] = {0}, wc[5] = {0};
                for (int v = 0; v < nv; ++v) {
                    double w5[5], d5[5];
                    for (int q = -2; q <= 2; ++q) {
                        double w[5], g[3][5];
                        fetch(c, W, G, rc + q, 0, 0, w, g);
                        w5[q + 2] = w[v]; d5[q + 2] = g[0][v];
                    }
                    wc[v] = w5[2];
                    geno1d_out o;
                    if (geno1d(w5, d5, side, c, &o)) { err |= 1; continue; }
                    val[v] = o.val;
                    der[v] = o.der / c->h;
                }
                if (!admissible(1, c->gamma, c->adm_delta, val, wc))
                    for (int v = 0; v < nv; ++v) { val[v] = wc[v]; der[v] = 0.0; }
                for (int v = 0; v < nv; ++v) {
                    out[((long)(side * nv + v) * 2 + 0) * nft + f] = val[v];
                    out[((long)(side * nv + v) * 2 + 1) * nft + f] = der[v];
                }
            }
        }
        return err ? OR_ERR_ARG : OR_OK;
    }
    long off = 0;
    for (int d = 0; d < m; ++d) {
        long nf = face_count(c, d);
        int ext[3] = {c->n[0], c->n[1], c->n[2]};
        ext[d] += 1;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
        for (long f = 0; f < nf; ++f) {
            int idx[3] = {(int)(f % ext[0]), (int)((f / ext[0]) % ext[1]), (int)(f / ((long)ext[0] * ext[1]))};
            for (int side = 0; side < 2; ++side) {
                int ci[3] = {idx[0], idx[1], idx[2]};
                if (side == 0) ci[d] -= 1;
                double w[5], g[3][5];
                fetch(c, W, G, ci[0], ci[1], ci[2], w, g);
                double wn[6][5], gn[6][3][5];
                for (int e = 0; e < m; ++e)
                    for (int s = 0; s < 2; ++s) {
                        int cj[3] = {ci[0], ci[1], ci[2]};
                        cj[e] += s ? 1 : -1;
                        fetch(c, W, G, cj[0], cj[1], cj[2], wn[2 * e + s], gn[2 * e + s]);
                    }
                monset s3;
                monset_build(&s3, m, 3);
                double val[4][5], der[4][3][5];
                for (int v = 0; v < nv; ++v) {
                    double D0[3], Wn[6], Dn[6][3];
                    for (int a = 0; a < m; ++a) D0[a] = g[a][v];
                    for (int q = 0; q < 2 * m; ++q) {
                        Wn[q] = wn[q][v];
                        for (int a = 0; a < m; ++a) Dn[q][a] = gn[q][a][v];
                    }
                    genomd_out o;
                    if (genomd(m, w[v], D0, Wn, Dn, c, &o)) { err |= 1; continue; }
                    for (int gp = 0; gp < ng; ++gp) {
                        long double x[3];
                        gauss_pt(m, d, gp, x);
                        x[d] = side ? -0.5L : 0.5L;
                        val[gp][v] = (double)poly_eval(&s3, o.coef, x, -1);
                        for (int a = 0; a < m; ++a) der[gp][a][v] = (double)(poly_eval(&s3, o.coef, x, a) / c->h);
                    }
                }
                for (int gp = 0; gp < ng; ++gp) {
                    if (!admissible(m, c->gamma, c->adm_delta, val[gp], w))
                        for (int v = 0; v < nv; ++v) {
                            val[gp][v] = w[v];
                            for (int a = 0; a < m; ++a) der[gp][a][v] = 0.0;
                        }
                    for (int v = 0; v < nv; ++v) {
                        long base = (long)(side * nv + v) * (m + 1);
                        out[((base + 0) * ng + gp) * nft + off + f] = val[gp][v];
                        for (int a = 0; a < m; ++a) out[((base + 1 + a) * ng + gp) * nft + off + f] = der[gp][a][v];
                    }
                }
            }
        }
        off += nf;
    }
    return err ? OR_ERR_ARG : OR_OK;
}

/* Face-frame axis order for a face normal to d: d first, then the others ascending. */
static void face_axes(int m, int d, int ax[3])
{
    int k = 0;
    ax[k++] = d;
    for (int a = 0; a < m; ++a) if (a != d) ax[k++] = a;
}

static int flux_all(const or_cfg *c, double dt, const double *fs, double *out)
{
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nft = face_total(c);
    int err = 0;
    long off = 0;
    for (int d = 0; d < m; ++d) {
        long nf = face_count(c, d);
        int ax[3];
        face_axes(m, d, ax);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
        for (long f = 0; f < nf; ++f) {
            for (int gp = 0; gp < ng; ++gp) {
                double Wlr[2][5], dW[2][3][5];
                for (int side = 0; side < 2; ++side)
                    for (int v = 0; v < nv; ++v) {
                        /* rotate: face-frame variable of global variable v */
                        int fv = v;
                        if (v >= 1 && v <= m) { for (int k = 0; k < m; ++k) if (ax[k] == v - 1) fv = 1 + k; }
                        long base = (long)(side * nv + v) * (m + 1);
                        Wlr[side][fv] = fs[((base + 0) * ng + gp) * nft + off + f];
                        for (int k = 0; k < m; ++k)
                            dW[side][k][fv] = fs[((base + 1 + ax[k]) * ng + gp) * nft + off + f];
                    }
                double F[5], Ft[5], Wh[5];
                if (gks_point(m, c->gamma, c->c1_tau, c->c2_tau, c->tau_mode, c->mu, dt, Wlr[0], Wlr[1], dW[0], dW[1], F, Ft, Wh)) {
                    err |= 1; continue;
                }
                /* walls (R8), slip or no-slip, at rest and adiabatic: neither
                 * mass nor energy crosses them; only the momentum flux
                 * (pressure and stress) is kept */
                {
                    long e0 = c->n[0] + (d == 0), e1 = c->n[1] + (d == 1);
                    long pos = (d == 0) ? f % e0 : (d == 1) ? (f / e0) % e1 : f / (e0 * e1);
                    int wall = (pos == 0) ? c->bcs[2 * d] : (pos == c->n[d]) ? c->bcs[2 * d + 1] : -1;
                    if (wall >= 2) F[0] = F[nv - 1] = Ft[0] = Ft[nv - 1] = 0.0;
                }
                for (int v = 0; v < nv; ++v) {
                    int fv = v;
                    if (v >= 1 && v <= m) { for (int k = 0; k < m; ++k) if (ax[k] == v - 1) fv = 1 + k; }
                    out[((long)(0 * nv + v) * ng + gp) * nft + off + f] = F[fv];
                    out[((long)(1 * nv + v) * ng + gp) * nft + off + f] = Ft[fv];
                    out[((long)(2 * nv + v) * ng + gp) * nft + off + f] = Wh[fv];
                }
            }
        }
        off += nf;
    }
    return err ? OR_ERR_NONPHYSICAL : OR_OK;
}

/* ------------------------------------------------------------------ */
/* 1D non-compact GENO with the HLLC flux and classical RK4 (Sec. 4.1,   */
/* Sec. 2; reading R16).                                                 */
/* ------------------------------------------------------------------ */
/* Left value at the face x_{j+1/2} of cell j from the averages u[i] at
 * offsets i - 2 (i = 0..5).  order 5: p^4 on {-2..2}, quadratics on
 * {-2,-1,0}, {-1,0,1}, {0,1,2}; order 6: p^5 on {-2..3}, quadratics on
 * {-2,-1,0}, {-1,0,1}, cubics on {-1..2}, {0..3}.  IS_k: sum over the
 * derivative orders 1..deg of int (d^l p_k)^2 on cell j (cell units);
 * IS^H = max IS_k (Eq. IS-highorder-2), IS^L = min IS_k
 * (Eq. HLP-IS-loworder-2), IS^tau = |(IS_first + IS_last)/2 - IS_2|
 * (Eq. 6th-noncompact-path, R16), r = 2; the sub-stencil centred on cell j,
 * {-1,0,1}, carries d = C0. */
static int nc_left_ex(const or_cfg *cfg, int order, const long double *u, long double *val, double *info);

static int nc_left(const or_cfg *cfg, int order, const long double *u, long double *val)
{
    return nc_left_ex(cfg, order, u, val, NULL);
}

/* info (optional): qH, chi, p_k[4], IS_k[4] */
static int nc_left_ex(const or_cfg *cfg, int order, const long double *u, long double *val, double *info)
{
    static const int off5[3][4] = {{-2, -1, 0}, {-1, 0, 1}, {0, 1, 2}};
    static const int off6[4][4] = {{-2, -1, 0}, {-1, 0, 1}, {-1, 0, 1, 2}, {0, 1, 2, 3}};
    static const int deg5[3] = {2, 2, 2}, deg6[4] = {2, 2, 3, 3};
    int nbig = (order == 5) ? 5 : 6, ksub = (order == 5) ? 3 : 4;
    monset sH, sk[4];
    monset_build(&sH, 1, nbig - 1);
    cond c[6];
    for (int i = 0; i < nbig; ++i) c[i] = (cond){{i - 2, 0, 0}, -1, u[i]};
    long double aH[8];
    if (fit_square(&sH, nbig, c, aH)) return -1;
    long double x[3] = {0.5L, 0, 0};
    long double qH = poly_eval(&sH, aH, x, -1);
    long double pk[4], IS[4];
    for (int k = 0; k < ksub; ++k) {
        int deg = (order == 5) ? deg5[k] : deg6[k];
        const int *off = (order == 5) ? off5[k] : off6[k];
        monset_build(&sk[k], 1, deg);
        cond ck[4];
        for (int i = 0; i <= deg; ++i) ck[i] = (cond){{off[i], 0, 0}, -1, u[off[i] + 2]};
        long double a[8];
        if (fit_square(&sk[k], deg + 1, ck, a)) return -1;
        pk[k] = poly_eval(&sk[k], a, x, -1);
        IS[k] = smooth_ind(&sk[k], a, 1, deg);
    }
    long double ISH = IS[0], ISL = IS[0];
    for (int k = 1; k < ksub; ++k) { if (IS[k] > ISH) ISH = IS[k]; if (IS[k] < ISL) ISL = IS[k]; }
    /* IS^tau from the outer-left, the outer-right and the centred
     * sub-stencil: S_1, S_3, S_2 in 5th order (Eq. 6th-noncompact-path);
     * in 6th order S_1, S_4, S_2, since S_1..S_3 leave the stencil's last
     * cell unseen (R16) */
    long double ISt = fabsl((IS[0] + IS[ksub - 1]) / 2.0L - IS[1]);
    long double eps = cfg->eps;
    long double chi = (cfg->limiter == 1) ? 1.0L : geno_chi(ISt, ISH, ISL, 2, eps, cfg->C);
    long double ws = 0.0L, qL = 0.0L, wt[4];
    for (int k = 0; k < ksub; ++k) {
        long double d = (k == 1) ? cfg->C0 : 1.0L;
        wt[k] = d / ((IS[k] + eps) * (IS[k] + eps)); /* Eq. HLP-q-loworder */
        ws += wt[k];
    }
    for (int k = 0; k < ksub; ++k) qL += wt[k] / ws * pk[k];
    *val = chi * qH + (1.0L - chi) * qL; /* Eq. 6th-noncompact-HLP */
    if (info) {
        info[0] = (double)qH;
        info[1] = (double)chi;
        for (int k = 0; k < 4; ++k) {
            info[2 + k] = (k < ksub) ? (double)pk[k] : 0.0;
            info[6 + k] = (k < ksub) ? (double)IS[k] : 0.0;
        }
    }
    return 0;
}

/* one left value from six averages (offsets -2..3): out = val, qH, chi, p[4], IS[4] */
int or_nc_point(const or_cfg *c, int order, const double *u6, double *out)
{
    if (order != 5 && order != 6) return OR_ERR_ARG;
    long double u[6], val;
    for (int i = 0; i < 6; ++i) u[i] = u6[i];
    if (nc_left_ex(c, order, u, &val, out + 1)) return OR_ERR_ARG;
    out[0] = (double)val;
    return OR_OK;
}

/* Face states of every face f = 0..n (between cells f-1 and f):
 * st[side][v][f], side 0 left, 1 right; the right state mirrors the stencil
 * about the face; an inadmissible state falls back to its cell average (R9). */
static int nc_states(const or_cfg *c, int order, const double *W, double *st)
{
    int n = c->n[0], nv = 3;
    long nf = n + 1;
    double *Gz = (double *)calloc((size_t)nv * n, sizeof(double));
    if (!Gz) return OR_ERR_ARG;
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (long f = 0; f < nf; ++f) {
        double w6[2][6][3], g[3][5];
        for (int i = 0; i < 6; ++i) {
            fetch(c, W, Gz, (int)f - 3 + i, 0, 0, w6[0][i], g); /* cells f-3..f+2, cell f-1 at i = 2 */
            fetch(c, W, Gz, (int)f + 2 - i, 0, 0, w6[1][i], g); /* mirrored: cell f at i = 2 */
        }
        for (int side = 0; side < 2; ++side) {
            double s3[3] = {0};
            for (int v = 0; v < nv; ++v) {
                long double u[6], val;
                for (int i = 0; i < 6; ++i) u[i] = w6[side][i][v];
                if (nc_left(c, order, u, &val)) { err |= 1; val = 0.0L; }
                s3[v] = (double)val;
            }
            if (!admissible(1, c->gamma, c->adm_delta, s3, w6[side][2]))
                for (int v = 0; v < nv; ++v) s3[v] = w6[side][2][v];
            for (int v = 0; v < nv; ++v) st[((long)side * nv + v) * nf + f] = s3[v];
        }
    }
    free(Gz);
    return err ? OR_ERR_ARG : OR_OK;
}

/* HLLC flux (Toro) with the Davis wave-speed bounds
 * SL = min(uL - cL, uR - cR), SR = max(uL + cL, uR + cR) (reading R16) */
static int hllc(double gamma, const double *L, const double *R, double *F)
{
    double rl = L[0], ul = L[1] / rl, pl = (gamma - 1.0) * (L[2] - 0.5 * rl * ul * ul);
    double rr = R[0], ur = R[1] / rr, pr = (gamma - 1.0) * (R[2] - 0.5 * rr * ur * ur);
    if (!(rl > 0.0) || !(rr > 0.0) || !(pl > 0.0) || !(pr > 0.0)) return -1;
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double SL = fmin(ul - cl, ur - cr), SR = fmax(ul + cl, ur + cr);
    double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur));
    double FL[3] = {rl * ul, rl * ul * ul + pl, ul * (L[2] + pl)};
    double FR[3] = {rr * ur, rr * ur * ur + pr, ur * (R[2] + pr)};
    if (0.0 <= SL) {
        for (int v = 0; v < 3; ++v) F[v] = FL[v];
    } else if (0.0 <= Ss) {
        double k = rl * (SL - ul) / (SL - Ss);
        double Us[3] = {k, k * Ss, k * (L[2] / rl + (Ss - ul) * (Ss + pl / (rl * (SL - ul))))};
        for (int v = 0; v < 3; ++v) F[v] = FL[v] + SL * (Us[v] - L[v]);
    } else if (0.0 <= SR) {
        double k = rr * (SR - ur) / (SR - Ss);
        double Us[3] = {k, k * Ss, k * (R[2] / rr + (Ss - ur) * (Ss + pr / (rr * (SR - ur))))};
        for (int v = 0; v < 3; ++v) F[v] = FR[v] + SR * (Us[v] - R[v]);
    } else {
        for (int v = 0; v < 3; ++v) F[v] = FR[v];
    }
    return 0;
}

/* HLLC fluxes F[v][f] of every face; walls carry no mass or energy flux (R8) */
static int nc_fluxes(const or_cfg *c, int order, const double *W, double *F)
{
    int n = c->n[0];
    long nf = n + 1;
    double *st = (double *)malloc(sizeof(double) * 2 * 3 * nf);
    if (!st) return OR_ERR_ARG;
    int r = nc_states(c, order, W, st);
    int err = 0;
    if (!r) {
        for (long f = 0; f < nf; ++f) {
            double L[3], R[3], Fv[3];
            for (int v = 0; v < 3; ++v) { L[v] = st[v * nf + f]; R[v] = st[(3 + v) * nf + f]; }
            if (hllc(c->gamma, L, R, Fv)) { err = 1; break; }
            int wall = (f == 0) ? c->bcs[0] : (f == n) ? c->bcs[1] : -1;
            if (wall >= 2) Fv[0] = Fv[2] = 0.0;
            for (int v = 0; v < 3; ++v) F[v * nf + f] = Fv[v];
        }
    }
    free(st);
    return r ? r : (err ? OR_ERR_NONPHYSICAL : OR_OK);
}

int or_nc_reconstruct(const or_cfg *c, int order, const double *W, double *st)
{
    if (check_cfg(c) || c->dim != 1 || (order != 5 && order != 6)) return OR_ERR_ARG;
    return nc_states(c, order, W, st);
}

int or_nc_flux(const or_cfg *c, int order, const double *W, double *F)
{
    if (check_cfg(c) || c->dim != 1 || (order != 5 && order != 6)) return OR_ERR_ARG;
    return nc_fluxes(c, order, W, F);
}

/* classical four-stage fourth-order Runge-Kutta step with
 * L(U)_j = -(F_{j+1/2} - F_{j-1/2}) / h */
int or_nc_step(const or_cfg *c, int order, double dt, double *W)
{
    if (check_cfg(c) || c->dim != 1 || (order != 5 && order != 6) || !(dt > 0.0)) return OR_ERR_ARG;
    int n = c->n[0];
    long nf = n + 1;
    double *F = (double *)malloc(sizeof(double) * 3 * nf);
    double *U = (double *)malloc(sizeof(double) * 3 * n);
    double *K = (double *)malloc(sizeof(double) * 4 * 3 * n);
    int r = OR_ERR_ARG;
    if (!F || !U || !K) goto done;
    static const double a[4] = {0.0, 0.5, 0.5, 1.0}, b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int s = 0; s < 4; ++s) {
        for (long i = 0; i < 3L * n; ++i) U[i] = W[i] + (s ? a[s] * dt * K[(s - 1) * 3 * n + i] : 0.0);
        r = nc_fluxes(c, order, U, F);
        if (r) goto done;
        for (int v = 0; v < 3; ++v)
            for (int j = 0; j < n; ++j) K[s * 3 * n + v * n + j] = -(F[v * nf + j + 1] - F[v * nf + j]) / c->h;
    }
    for (int v = 0; v < 3; ++v)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int s = 0; s < 4; ++s) acc += b[s] * K[s * 3 * n + v * n + j];
            W[v * n + j] += dt * acc;
        }
    for (int j = 0; j < n; ++j) {
        double w[3] = {W[j], W[n + j], W[2 * n + j]};
        if (!(w[0] > 0.0) || !(pressure(1, c->gamma, w) > 0.0)) { r = OR_ERR_NONPHYSICAL; goto done; }
    }
    r = OR_OK;
done:
    free(F); free(U); free(K);
    return r;
}

/* ------------------------------------------------------------------ */
/* Public oracle entry points (ctypes).                                  */
/* ------------------------------------------------------------------ */
long or_face_total(const or_cfg *c) { return check_cfg(c) ? -1 : face_total(c); }

int or_reconstruct(const or_cfg *c, const double *W, const double *G, double *face_states)
{
    if (check_cfg(c)) return OR_ERR_ARG;
    return recon_all(c, W, G, face_states);
}

int or_flux(const or_cfg *c, double dt, const double *W, const double *G, double *face_flux)
{
    if (check_cfg(c) || !(dt > 0.0)) return OR_ERR_ARG;
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nft = face_total(c);
    double *fs = (double *)malloc(sizeof(double) * 2 * nv * (m + 1) * ng * nft);
    if (!fs) return OR_ERR_ARG;
    int r = recon_all(c, W, G, fs);
    if (!r) r = flux_all(c, dt, fs, face_flux);
    free(fs);
    return r;
}

/* Face index (within the full face list) of the face of cell (i,j,k) on side s of axis d. */
static long face_of(const or_cfg *c, int d, int i, int j, int k, int s)
{
    int ext[3] = {c->n[0], c->n[1], c->n[2]};
    ext[d] += 1;
    int idx[3] = {i, j, k};
    idx[d] += s;
    long off = 0;
    for (int a = 0; a < d; ++a) off += face_count(c, a);
    return off + ((long)idx[2] * ext[1] + idx[1]) * ext[0] + idx[0];
}

/* One stage's face quantities -> divergence D(q)_j = sum_d sum_g w_g (q(+d face) - q(-d face)) */
static double face_div(const or_cfg *c, const double *ff, int q, int v, int i, int j, int k)
{
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nft = face_total(c);
    double wg = 1.0 / ng, r = 0.0;
    for (int d = 0; d < m; ++d) {
        long fp = face_of(c, d, i, j, k, 1), fm = face_of(c, d, i, j, k, 0);
        for (int g = 0; g < ng; ++g)
            r += wg * (ff[((long)(q * nv + v) * ng + g) * nft + fp] - ff[((long)(q * nv + v) * ng + g) * nft + fm]);
    }
    return r;
}

static double face_diff_dir(const or_cfg *c, const double *ff, int q, int v, int d, int i, int j, int k)
{
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nft = face_total(c);
    double wg = 1.0 / ng, r = 0.0;
    long fp = face_of(c, d, i, j, k, 1), fm = face_of(c, d, i, j, k, 0);
    for (int g = 0; g < ng; ++g)
        r += wg * (ff[((long)(q * nv + v) * ng + g) * nft + fp] - ff[((long)(q * nv + v) * ng + g) * nft + fm]);
    return r;
}

/* One two-stage fourth-order step (reading R7), in place on W and G. */
int or_step(const or_cfg *c, double dt, double *W, double *G)
{
    if (check_cfg(c) || !(dt > 0.0)) return OR_ERR_ARG;
    int m = c->dim, nv = m + 2, ng = ngauss(m);
    long nc = cells(c), nft = face_total(c);
    long ffsz = (long)3 * nv * ng * nft;
    double *f1 = (double *)malloc(sizeof(double) * ffsz);
    double *f2 = (double *)malloc(sizeof(double) * ffsz);
    double *Ws = (double *)malloc(sizeof(double) * nv * nc);
    double *Gs = (double *)malloc(sizeof(double) * m * nv * nc);
    int r = OR_ERR_ARG;
    double h = c->h;
    if (!f1 || !f2 || !Ws || !Gs) goto done;
    /* stage 1 from (W^n, G^n) */
    r = or_flux(c, dt, W, G, f1);
    if (r) goto done;
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < nc; ++cell) {
        int i = (int)(cell % c->n[0]), j = (int)((cell / c->n[0]) % c->n[1]), k = (int)(cell / ((long)c->n[0] * c->n[1]));
        for (int v = 0; v < nv; ++v) {
            Ws[v * nc + cell] = W[v * nc + cell] - 0.5 * dt / h * face_div(c, f1, 0, v, i, j, k) -
                                dt * dt / 8.0 / h * face_div(c, f1, 1, v, i, j, k);
            for (int d = 0; d < m; ++d) Gs[(d * nv + v) * nc + cell] = face_diff_dir(c, f1, 2, v, d, i, j, k) / h;
        }
    }
    /* stage 2 from (W*, G*) */
    r = or_flux(c, dt, Ws, Gs, f2);
    if (r) goto done;
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < nc; ++cell) {
        int i = (int)(cell % c->n[0]), j = (int)((cell / c->n[0]) % c->n[1]), k = (int)(cell / ((long)c->n[0] * c->n[1]));
        for (int v = 0; v < nv; ++v) {
            W[v * nc + cell] = W[v * nc + cell] - dt / h * face_div(c, f1, 0, v, i, j, k) -
                               dt * dt / 6.0 / h * (face_div(c, f1, 1, v, i, j, k) + 2.0 * face_div(c, f2, 1, v, i, j, k));
            for (int d = 0; d < m; ++d) G[(d * nv + v) * nc + cell] = face_diff_dir(c, f2, 2, v, d, i, j, k) / h;
        }
    }
    /* physical admissibility of the result */
    for (long cell = 0; cell < nc; ++cell) {
        double rho = W[cell], ke = 0.0;
        for (int a = 0; a < m; ++a) ke += W[(1 + a) * nc + cell] * W[(1 + a) * nc + cell];
        double p = (c->gamma - 1.0) * (W[(m + 1) * nc + cell] - 0.5 * ke / rho);
        if (!(rho > 0.0) || !(p > 0.0)) { r = OR_ERR_NONPHYSICAL; break; }
    }
done:
    free(f1); free(f2); free(Ws); free(Gs);
    return r;
}

/* max over cells and axes of |u_d| + c (the CFL time step uses h / this) */
double or_max_wavespeed(const or_cfg *c, const double *W)
{
    int m = c->dim;
    long nc = cells(c);
    double s = 0.0;
    for (long cell = 0; cell < nc; ++cell) {
        double rho = W[cell], ke = 0.0;
        for (int a = 0; a < m; ++a) ke += W[(1 + a) * nc + cell] * W[(1 + a) * nc + cell];
        double p = (c->gamma - 1.0) * (W[(m + 1) * nc + cell] - 0.5 * ke / rho);
        double cs = sqrt(c->gamma * p / rho);
        for (int a = 0; a < m; ++a) {
            double v = fabs(W[(1 + a) * nc + cell] / rho) + cs;
            if (v > s) s = v;
        }
    }
    return s;
}

/* max over cells of mu / rho (viscous time step) */
double or_max_kin_viscosity(const or_cfg *c, const double *W)
{
    long nc = cells(c);
    double s = 0.0;
    for (long cell = 0; cell < nc; ++cell) {
        double v = c->mu / W[cell];
        if (v > s) s = v;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Internals exposed for the pins.                                        */
/* ------------------------------------------------------------------ */
/* 1D GENO at one interface: w5/d5 = averages / cell-unit derivatives of the
 * cells at offsets -2..2 around the reconstruction cell.  out[0..8] =
 * value, derivative (cell units), chi, IS1, IS2, IS3, ISH, ISL, IStau. */
int or_geno1d_point(const or_cfg *c, const double *w5, const double *d5, int side, double *out)
{
    geno1d_out o;
    if (geno1d(w5, d5, side, c, &o)) return OR_ERR_ARG;
    out[0] = o.val; out[1] = o.der; out[2] = o.chi;
    out[3] = o.IS[0]; out[4] = o.IS[1]; out[5] = o.IS[2];
    out[6] = o.ISH; out[7] = o.ISL; out[8] = o.ISt;
    return OR_OK;
}

/* Multi-D GENO for one cell.  in: W0, D0[m], then for q = 0..2m-1 (q = 2e +
 * (side > 0)): Wn[q], Dn[q][0..m-1].  out: monomial coefficients of the
 * blended cubic (ordering by total degree, then exponents descending in x,
 * then y), then chi, ISH, ISL, IStau, IS[0..2m-1].  Returns the number of
 * monomials. */
int or_genomd_cell(const or_cfg *c, const double *in, double *out)
{
    int m = c->dim;
    double W0 = in[0], D0[3], Wn[6], Dn[6][3];
    for (int a = 0; a < m; ++a) D0[a] = in[1 + a];
    for (int q = 0; q < 2 * m; ++q) {
        Wn[q] = in[1 + m + q * (1 + m)];
        for (int a = 0; a < m; ++a) Dn[q][a] = in[1 + m + q * (1 + m) + 1 + a];
    }
    genomd_out o;
    if (genomd(m, W0, D0, Wn, Dn, c, &o)) return OR_ERR_ARG;
    monset s3;
    monset_build(&s3, m, 3);
    for (int k = 0; k < s3.nmon; ++k) out[k] = (double)o.coef[k];
    out[s3.nmon + 0] = o.chi; out[s3.nmon + 1] = o.ISH; out[s3.nmon + 2] = o.ISL; out[s3.nmon + 3] = o.ISt;
    for (int q = 0; q < 2 * m; ++q) out[s3.nmon + 4 + q] = o.IS[q];
    return s3.nmon;
}

/* Monomial exponents of the multi-D cubic basis (3 ints per monomial). */
int or_monomials(int m, int deg, int *e)
{
    monset s;
    monset_build(&s, m, deg);
    for (int k = 0; k < s.nmon; ++k) { e[3 * k] = s.e[k][0]; e[3 * k + 1] = s.e[k][1]; e[3 * k + 2] = s.e[k][2]; }
    return s.nmon;
}

/* Flux at one face point in the face frame; dWl/dWr are [m][nv] row-major. */
int or_gks_point(int m, double gamma, double c1, double c2, int tau_mode, double mu, double dt, const double *Wl,
                 const double *Wr, const double *dWl, const double *dWr, double *F, double *Ft, double *Wh)
{
    double a[3][5], b[3][5];
    int nv = m + 2;
    for (int e = 0; e < m; ++e)
        for (int v = 0; v < nv; ++v) { a[e][v] = dWl[e * nv + v]; b[e][v] = dWr[e * nv + v]; }
    return gks_point(m, gamma, c1, c2, tau_mode, mu, dt, Wl, Wr, a, b, F, Ft, Wh) ? OR_ERR_NONPHYSICAL : OR_OK;
}

/* Micro-slope solve <a psi> = rhs against the Maxwellian of W (pin P7). */
int or_slope_solve(int m, double gamma, const double *W, const double *rhs, double *s)
{
    maxw g;
    if (to_maxw(m, gamma, W, &g)) return OR_ERR_NONPHYSICAL;
    return slope_solve(&g, rhs, s) ? OR_ERR_ARG : OR_OK;
}

/* <psi_a psi_b> moment matrix of the Maxwellian of W, normalised by rho. */
int or_moment_matrix(int m, double gamma, const double *W, double *M)
{
    maxw g;
    if (to_maxw(m, gamma, W, &g)) return OR_ERR_NONPHYSICAL;
    int nv = m + 2;
    for (int i = 0; i < nv; ++i) {
        vpoly pi; vp_psi(m, i, &pi);
        for (int j = 0; j < nv; ++j) {
            vpoly pj, pp; vp_psi(m, j, &pj);
            vp_mul(&pi, &pj, &pp);
            M[i * nv + j] = vp_moment(&pp, &g, 0);
        }
    }
    return OR_OK;
}
