/*
 * Kernels of one stage of the compact GKS with GENO reconstruction
 * (arXiv 2507.20461, Sec. 2-4), templated on the dimension M and on the
 * reconstruction/flux precision R (double, or float with FP64 accumulation).
 *
 * Stage pipeline on uniform grids (cell size h, nv = M + 2 variables):
 *   1D   face1d        one thread per face: p^7 on {j-1..j+2} (shared by both
 *                      sides), the three sub-stencil quadratics of each side,
 *                      GENO blend, admissibility fallback, GKS flux.
 *   M-D  cell_poly     one thread per cell (plus the ghost ring): least-squares
 *                      cubic, linear sub-polynomials, GENO blend -> blended
 *                      cubic coefficients B[v][k].
 *        face_flux     one thread per (face, Gauss point) of one direction:
 *                      both interface states from B, admissibility fallback,
 *                      GKS flux, F / dF/dt / W(dt/2) to the face arrays.
 *   all  update        one thread per cell: FP64 two-stage update of the
 *                      averages (Eq. semifvs) and of the averaged gradients by
 *                      the Gauss theorem (Eq. slope).
 * Ghost cells are index mappings (periodic wrap, or transmissive even
 * extension with the normal derivative negated); no padded copies exist.
 */
#pragma once
#include <cstdint>

#include "fpsplit.cuh"
#include "geno_coeffs.cuh"
#include "gks_device.cuh"

namespace gks {

enum StatusBits : int { ST_RHO = 1, ST_P = 2, ST_NAN = 4, ST_FLUX = 8 };

/* Division of 32-bit unsigned integers by a divisor fixed at launch:
 * q = floor(n / d) = floor(M n / 2^64) with M = ceil(2^64 / d), exact for all
 * n, d < 2^32 (Lemire, Kaser and Kurz, "Faster remainder by direct
 * computation", 2019, Theorem 1); M = 0 marks d = 1.  Replaces the 64-bit
 * divisions of the index decompositions (a long instruction sequence each). */
struct FDiv {
    unsigned d;
    unsigned long long M;
};

inline FDiv make_fdiv(unsigned d)
{
    FDiv f;
    f.d = d;
    f.M = (d <= 1) ? 0ull : (~0ull / d + 1ull);
    return f;
}

__device__ __forceinline__ unsigned fdiv(const FDiv &f, unsigned n)
{
    return f.M ? (unsigned)__umul64hi(f.M, (unsigned long long)n) : n;
}

/* q = n / d, returns n % d */
__device__ __forceinline__ unsigned fdivmod(const FDiv &f, unsigned n, unsigned &q)
{
    q = fdiv(f, n);
    return n - q * f.d;
}

struct KP {
    int n[3];
    int bcs[3][2]; /* per axis, low / high side: 0 periodic (both sides),
                      1 transmissive, 2 reflective (slip), 3 no-slip wall */
    int limiter; /* 0 GENO, 1 linear, 2 WENO-Z, 3 TENO */
    long ncell;
    long nface[3];
    long foff[3];
    long nftot;
    int ext[3]; /* extended box: n + 2 along the active axes */
    long next;
    double h, ih, gamma;
    double C, itanhC, eps, C0, adm;
    double d0, ct; /* WENO-Z / TENO: linear weight of the high-order candidate, TENO cut-off */
    FluxParams fp;
    /* FP32 copies for the mixed-precision kernels (fill with finalize_kp) */
    float fh, fih, fgm1, fC, fitanhC, feps, fC0, fadm, fd0, fct;
    /* index decompositions (fill with finalize_kp; every index space of a
     * launch is below 2^32): cells per axis, extended box, per face
     * direction its two leading extents and its face count */
    FDiv dn[3], dext[2], dface[3][2], dnf[3];
};

/* the same boundary type on every side */
inline void set_bcs(KP &P, int bc)
{
    for (int a = 0; a < 3; ++a) P.bcs[a][0] = P.bcs[a][1] = bc;
}

/* derived fields of a parameter block whose double fields are set */
inline void finalize_kp(KP &P)
{
    fill_flux(P.fp, P.gamma, P.fp.c1, P.fp.c2);
    P.fh = (float)P.h;
    P.fih = (float)P.ih;
    P.fgm1 = (float)(P.gamma - 1.0);
    P.fC = (float)P.C;
    P.fitanhC = (float)P.itanhC;
    P.feps = (float)P.eps;
    P.fC0 = (float)P.C0;
    P.fd0 = (float)P.d0;
    P.fct = (float)P.ct;
    for (int a = 0; a < 3; ++a) P.dn[a] = make_fdiv((unsigned)P.n[a]);
    P.dext[0] = make_fdiv((unsigned)P.ext[0]);
    P.dext[1] = make_fdiv((unsigned)P.ext[1]);
    for (int d = 0; d < 3; ++d) {
        P.dface[d][0] = make_fdiv((unsigned)(P.n[0] + (d == 0)));
        P.dface[d][1] = make_fdiv((unsigned)(P.n[1] + (d == 1)));
        P.dnf[d] = make_fdiv((unsigned)(P.nface[d] > 0 ? P.nface[d] : 1));
    }
    P.fadm = (float)P.adm;
}

/* FP32 shadow of a state (mixed precision, 2D/3D): hi = float(W),
 * lo = float(W - hi) (so neighbour differences keep FP64-level accuracy),
 * g = float(grad W).  hi/lo: nv x cells, g: M x nv x cells. */
struct Shadow {
    float *hi, *lo, *g;
};

/* What the reconstruction and flux kernels read of a stage's input state:
 * the FP64 arrays (R = double) or the FP32 shadow (R = float).  Indices:
 * v * ncell + cell for averages, (a * nv + v) * ncell + cell for gradients. */
template <typename R> struct Src;
template <> struct Src<double> {
    const double *W, *G;
    __device__ __forceinline__ double w0(long i) const { return W[i]; }
    __device__ __forceinline__ double delta(long iq, long i0) const { return W[iq] - W[i0]; }
    /* (sq W[iq]) - (s0 W[i0]) for mirror signs sq, s0 = +-1 */
    __device__ __forceinline__ double delta_signed(long iq, int sq, long i0, int s0) const
    {
        return (sq > 0 ? W[iq] : -W[iq]) - (s0 > 0 ? W[i0] : -W[i0]);
    }
    __device__ __forceinline__ double grad(long i) const { return G[i]; }
};
template <> struct Src<float> {
    const float *hi, *lo, *g;
    __device__ __forceinline__ float w0(long i) const { return hi[i]; }
    __device__ __forceinline__ float delta(long iq, long i0) const { return (hi[iq] - hi[i0]) + (lo[iq] - lo[i0]); }
    __device__ __forceinline__ float delta_signed(long iq, int sq, long i0, int s0) const
    {
        const float hq = sq > 0 ? hi[iq] : -hi[iq], lq = sq > 0 ? lo[iq] : -lo[iq];
        const float h0 = s0 > 0 ? hi[i0] : -hi[i0], l0 = s0 > 0 ? lo[i0] : -lo[i0];
        return (hq - h0) + (lq - l0);
    }
    __device__ __forceinline__ float grad(long i) const { return g[i]; }
};

__device__ __forceinline__ void split_store(double w, float *hi, float *lo, long i)
{
    float a, b;
    split(w, a, b);
    hi[i] = a;
    lo[i] = b;
}

/* Mirror bits of one crossing of a wall of type t (ghost cells are mirror
 * images): bit 0 the mirror itself (derivatives along the axis change sign),
 * bit 1 the momentum normal to the wall is odd (reflective and no-slip),
 * bit 2 the tangential momenta are odd (no-slip). */
__device__ __forceinline__ int wall_bits(int t) { return t == 1 ? 1 : (t == 2 ? 3 : 7); }

/* index of the (possibly ghost) cell i along an axis of n cells with
 * boundary types lo / hi; flip accumulates the mirror bits (several
 * crossings on grids thinner than the stencil) */
__device__ __forceinline__ int map_idx(int i, int n, int lo, int hi, int &flip)
{
    if (i >= 0 && i < n) return i;
    if (lo == 0) {
        i %= n;
        if (i < 0) i += n;
        return i;
    }
    while (i < 0 || i >= n) {
        if (i < 0) { i = -1 - i; flip ^= wall_bits(lo); }
        if (i >= n) { i = 2 * n - 1 - i; flip ^= wall_bits(hi); }
    }
    return i;
}

/* Sign of variable v in a mirrored ghost cell: a reflective (slip) wall
 * negates the momentum component normal to it, a no-slip wall every momentum
 * component; every other variable (and everything under a transmissive
 * boundary) is mirrored evenly.  The derivative along axis a carries this
 * sign times -1 if the ghost is mirrored across axis a (flip bit 0). */
template <int M>
__device__ __forceinline__ int ghost_sign(const KP &P, const int *flip, int v)
{
    int s = 1;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        if (v == 1 + a) {
            if (flip[a] & 2) s = -s;
        } else if (v >= 1 && v <= M) {
            if (flip[a] & 4) s = -s;
        }
    }
    return s;
}

/* the signs of a (ghost) cell packed in one word: bit v set if variable v
 * is negated, bit 8 + a set if the cell is mirrored across axis a (its
 * derivatives along a change sign on top of that) */
template <int M>
__device__ __forceinline__ unsigned ghost_mask(const KP &P, const int *flip)
{
    unsigned m = 0;
#pragma unroll
    for (int v = 0; v < M + 2; ++v)
        if (ghost_sign<M>(P, flip, v) < 0) m |= 1u << v;
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (flip[a] & 1) m |= 1u << (8 + a);
    return m;
}

/* linear cell index and the mirror flips of a (ghost) cell */
template <int M>
__device__ __forceinline__ long cell_lin(const KP &P, int i, int j, int k, int *flip)
{
    flip[0] = flip[1] = flip[2] = 0;
    const int ii = map_idx(i, P.n[0], P.bcs[0][0], P.bcs[0][1], flip[0]);
    const int jj = (M >= 2) ? map_idx(j, P.n[1], P.bcs[1][0], P.bcs[1][1], flip[1]) : 0;
    const int kk = (M >= 3) ? map_idx(k, P.n[2], P.bcs[2][0], P.bcs[2][1], flip[2]) : 0;
    return ((long)kk * P.n[1] + jj) * P.n[0] + ii;
}

template <typename R>
__device__ __forceinline__ R chi_of(const KP &P, R ISt, R ISH, R ISL, int r)
{
    const R eps = pick<R>(P.eps, P.feps);
    R xH = ISt / (ISH + eps), xL = ISt / (ISL + eps);
    R pH = xH * xH, pL = xL * xL;
    if (r == 3) { pH *= xH; pL *= xL; }
    const R aH = R(1) + pH, aL = R(1) + pL;
    const R alpha = R(2) * aH / (aH + aL);
    return RT<R>::tanh_(pick<R>(P.C, P.fC) * alpha) * pick<R>(P.itanhC, P.fitanhC);
}

/* WENO-Z (limiter 2, Eq. wgt-WENO-Z) or TENO (limiter 3, Eq. wgt-TENO-1 with
 * the exponent 7 and Eq. wgt-TENO-2) weights over K + 1 candidates: 0 is
 * the high-order polynomial (indicator IS^H), 1..K the sub-stencil
 * polynomials; linear weights d, tau_Z = IS^tau.  TENO's (1/(IS + eps))^7 is
 * taken relative to the smallest indicator, (IS_min + eps) / (IS_k + eps) to
 * the 7th, which leaves the normalised gamma_k unchanged and keeps FP32 from
 * overflowing. */
template <typename R, int K>
__device__ __forceinline__ void ao_weights(const KP &P, const R *d, const R *IS, R tau, R *w)
{
    const R eps = pick<R>(P.eps, P.feps);
    R s = R(0);
    if (P.limiter == 2) {
#pragma unroll
        for (int k = 0; k <= K; ++k) {
            w[k] = d[k] * (R(1) + tau / (IS[k] + eps));
            s += w[k];
        }
    } else {
        R m = IS[0];
#pragma unroll
        for (int k = 1; k <= K; ++k) m = fmin(m, IS[k]);
        R g[K + 1], gs = R(0);
#pragma unroll
        for (int k = 0; k <= K; ++k) {
            const R r = (m + eps) / (IS[k] + eps);
            const R r2 = r * r;
            g[k] = r2 * r2 * r2 * r;
            gs += g[k];
        }
        const R cut = pick<R>(P.ct, P.fct) * gs;
#pragma unroll
        for (int k = 0; k <= K; ++k) {
            w[k] = (g[k] <= cut) ? R(0) : d[k];
            s += w[k];
        }
    }
    const R is = R(1) / s;
#pragma unroll
    for (int k = 0; k <= K; ++k) w[k] *= is;
}

template <typename R, int M>
__device__ __forceinline__ bool admissible(const R *w, const R *wc, R gm1, R delta)
{
    R ke = R(0), kc = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        ke += w[1 + a] * w[1 + a];
        kc += wc[1 + a] * wc[1 + a];
    }
    if (!(w[0] > delta * wc[0])) return false;
    const R p = gm1 * (w[M + 1] - R(0.5) * ke / w[0]);
    const R pc = gm1 * (wc[M + 1] - R(0.5) * kc / wc[0]);
    return p > delta * pc;
}

/* ------------------------------------------------------------------ */
/* 1D: reconstruction + flux per face                                  */
/* ------------------------------------------------------------------ */
/* GENO blend of one side.  a[k][0..1] = (a1, a2) of the sub-stencil
 * quadratics S1, S2 (central), S3 about the reconstruction cell; pv/pd =
 * their values/derivatives at the face; qv/qd = p^7 at the face.  All in cell
 * units relative to the reconstruction cell's average. */
template <typename R>
__device__ __forceinline__ void geno1d_blend(const KP &P, const R (*a)[2], const R *pv, const R *pd, R qv, R qd, R &val,
                                             R &der)
{
    R IS[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) IS[k] = a[k][0] * a[k][0] + R(13.0 / 3.0) * a[k][1] * a[k][1];
    const R ISH = fmax(IS[0], fmax(IS[1], IS[2]));
    const R ISL = fmin(IS[0], fmin(IS[1], IS[2]));
    const R ISt = RT<R>::abs_(R(0.5) * (IS[1] + IS[2]) - IS[0]);
    if (P.limiter >= 2) {
        /* WENO-Z / TENO in the adaptive-order combination:
         * (w0/d0) q^H + sum_k (w_k - (w0/d0) d_k) p_k, the sub-stencils sharing
         * 1 - d0 in GENO's low-order proportions (1, C0, 1) */
        const R d0 = pick<R>(P.d0, P.fd0), C0 = pick<R>(P.C0, P.fC0);
        const R dl = (R(1) - d0) / (C0 + R(2));
        const R d[4] = {d0, dl, dl * C0, dl};
        const R I4[4] = {ISH, IS[0], IS[1], IS[2]};
        R w[4];
        ao_weights<R, 3>(P, d, I4, ISt, w);
        const R chi = w[0] / d0;
        val = chi * qv;
        der = chi * qd;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R ck = w[k + 1] - chi * d[k + 1];
            val += ck * pv[k];
            der += ck * pd[k];
        }
        return;
    }
    const R chi = P.limiter ? R(1) : chi_of<R>(P, ISt, ISH, ISL, 2);
    const R eps = pick<R>(P.eps, P.feps);
    const R w0 = R(1) / ((IS[0] + eps) * (IS[0] + eps));
    const R w1 = pick<R>(P.C0, P.fC0) / ((IS[1] + eps) * (IS[1] + eps));
    const R w2 = R(1) / ((IS[2] + eps) * (IS[2] + eps));
    const R iws = R(1) / (w0 + w1 + w2);
    const R lv = (w0 * pv[0] + w1 * pv[1] + w2 * pv[2]) * iws;
    const R ld = (w0 * pd[0] + w1 * pd[1] + w2 * pd[2]) * iws;
    val = chi * qv + (R(1) - chi) * lv;
    der = chi * qd + (R(1) - chi) * ld;
}

/* states[side][v][c]: c = 0 value, 1 physical derivative */
template <typename R>
__device__ __forceinline__ void recon1d_face(const KP &P, const double *__restrict__ W, const double *__restrict__ G, int f,
                                             R (*st)[3][2], R (*cw)[3])
{
    double w[4][3], d[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int flip[3];
        const long c = cell_lin<1>(P, f - 2 + q, 0, 0, flip);
        const double sg = (flip[0] & 1) ? -P.h : P.h;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const double sv = (double)ghost_sign<1>(P, flip, v);
            w[q][v] = sv * W[v * P.ncell + c];
            d[q][v] = sv * G[v * P.ncell + c] * sg;
        }
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        /* left: reconstruction cell j = f-1 (index 1), deltas relative to it */
        const R wm1 = R(w[0][v] - w[1][v]), w1 = R(w[2][v] - w[1][v]), w2 = R(w[3][v] - w[1][v]);
        R qv, qd;
        p7_face<R>(wm1, R(0), w1, w2, R(d[0][v]), R(d[1][v]), R(d[2][v]), R(d[3][v]), qv, qd);
        {
            const R dm1 = R(d[0][v]);
            R a[3][2], pv[3], pd[3];
            a[0][1] = -(wm1 + dm1);
            a[0][0] = -R(2) * wm1 - dm1;
            a[1][0] = R(0.5) * (w1 - wm1);
            a[1][1] = R(0.5) * (w1 + wm1);
            a[2][1] = R(0.5) * (w2 - R(2) * w1);
            a[2][0] = R(0.5) * (R(4) * w1 - w2);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pv[k] = R(0.5) * a[k][0] + a[k][1] * R(1.0 / 6.0);
                pd[k] = a[k][0] + a[k][1];
            }
            R val, der;
            geno1d_blend<R>(P, a, pv, pd, qv, qd, val, der);
            st[0][v][0] = R(w[1][v]) + val;
            st[0][v][1] = der * pick<R>(P.ih, P.fih);
            cw[0][v] = R(w[1][v]);
        }
        /* right: reconstruction cell j+1 = f (index 2), mirrored stencils */
        {
            const R dj = R(w[2][v] - w[1][v]);
            const R um2 = R(w[0][v] - w[2][v]), um1 = R(w[1][v] - w[2][v]), u1 = R(w[3][v] - w[2][v]);
            const R d1 = R(d[3][v]);
            R a[3][2], pv[3], pd[3];
            a[0][1] = d1 - u1;
            a[0][0] = R(2) * u1 - d1;
            a[1][0] = R(0.5) * (u1 - um1);
            a[1][1] = R(0.5) * (u1 + um1);
            a[2][1] = R(0.5) * (um2 - R(2) * um1);
            a[2][0] = R(0.5) * (um2 - R(4) * um1);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pv[k] = -R(0.5) * a[k][0] + a[k][1] * R(1.0 / 6.0);
                pd[k] = a[k][0] - a[k][1];
            }
            R val, der;
            geno1d_blend<R>(P, a, pv, pd, qv - dj, qd, val, der);
            st[1][v][0] = R(w[2][v]) + val;
            st[1][v][1] = der * pick<R>(P.ih, P.fih);
            cw[1][v] = R(w[2][v]);
        }
    }
}

/* FLUX = false: write the interface states face_states[side][v][c][face] (double).
 * FLUX = true : write ff[q][v][face] (R), q = F, dF/dt, W(dt/2). */
template <typename R, bool FLUX, bool NS = false>
__global__ void __launch_bounds__(128) face1d_kernel(KP P, const double *__restrict__ W, const double *__restrict__ G,
                                                     const double *__restrict__ dtp, double *__restrict__ fs,
                                                     R *__restrict__ ff, int *__restrict__ status)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > P.n[0]) return;
    R st[2][3][2], cw[2][3];
    recon1d_face<R>(P, W, G, f, st, cw);
    const R gm1 = pick<R>(P.fp.gm1, P.fgm1);
    R Wl[3], Wr[3], dWl[1][3], dWr[1][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        R s[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) s[v] = st[side][v][0];
        const bool ok = admissible<R, 1>(s, cw[side], gm1, pick<R>(P.adm, P.fadm));
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const R val = ok ? st[side][v][0] : cw[side][v];
            const R der = ok ? st[side][v][1] : R(0);
            if (side == 0) { Wl[v] = val; dWl[0][v] = der; }
            else { Wr[v] = val; dWr[0][v] = der; }
        }
    }
    if (!FLUX) {
        const long nf = P.nftot;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            fs[((long)(0 * 3 + v) * 2 + 0) * nf + f] = (double)Wl[v];
            fs[((long)(0 * 3 + v) * 2 + 1) * nf + f] = (double)dWl[0][v];
            fs[((long)(1 * 3 + v) * 2 + 0) * nf + f] = (double)Wr[v];
            fs[((long)(1 * 3 + v) * 2 + 1) * nf + f] = (double)dWr[0][v];
        }
        return;
    }
    R F[3], Ft[3], Wh[3];
    const R dt = R(dtp[0]);
    if (!gks_point<R, 1, NS>(P.fp, dt, Wl, Wr, dWl, dWr, F, Ft, Wh)) {
        atomicOr(status, ST_FLUX);
#pragma unroll
        for (int v = 0; v < 3; ++v) F[v] = Ft[v] = Wh[v] = R(0);
    }
    /* walls (slip or no-slip) are at rest and adiabatic: neither mass nor energy crosses them */
    if ((f == 0 && P.bcs[0][0] >= 2) || (f == P.n[0] && P.bcs[0][1] >= 2)) F[0] = F[2] = Ft[0] = Ft[2] = R(0);
    const long nf = P.nftot;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        ff[(0 * 3 + v) * nf + f] = F[v];
        ff[(1 * 3 + v) * nf + f] = Ft[v];
        ff[(2 * 3 + v) * nf + f] = Wh[v];
    }
}

/* ------------------------------------------------------------------ */
/* multi-D: blended GENO cubic per cell                                 */
/* ------------------------------------------------------------------ */
template <typename R, int M> struct Cubic;
template <typename R> struct Cubic<R, 2> {
    static constexpr int NC = GENO_NC2, ND = GENO_ND2;
    __device__ __forceinline__ static void fit(const R *d, R *c) { cubic2d_fit<R>(d, c); }
    __device__ __forceinline__ static void ind(const R *c, R &h, R &t) { cubic2d_indicators<R>(c, h, t); }
};
template <typename R> struct Cubic<R, 3> {
    static constexpr int NC = GENO_NC3, ND = GENO_ND3;
    __device__ __forceinline__ static void fit(const R *d, R *c) { cubic3d_fit<R>(d, c); }
    __device__ __forceinline__ static void ind(const R *c, R &h, R &t) { cubic3d_indicators<R>(c, h, t); }
};

/* thread -> extended cell (-1..n along every active axis); false for corner
 * cells (two or more ghost coordinates) that no face needs */
template <int M>
__device__ __forceinline__ bool ext_cell(const KP &P, long t, int &i, int &j, int &k)
{
    unsigned q0, q1;
    i = (int)fdivmod(P.dext[0], (unsigned)t, q0) - 1;
    j = (M >= 2) ? (int)fdivmod(P.dext[1], q0, q1) - 1 : 0;
    k = (M >= 3) ? (int)q1 - 1 : 0;
    int out = (i < 0 || i >= P.n[0]);
    if (M >= 2) out += (j < 0 || j >= P.n[1]);
    if (M >= 3) out += (k < 0 || k >= P.n[2]);
    return out <= 1;
}

/* The blended GENO cubic of one variable of one cell (Sec. 3, Sec. 4.3 on
 * Cartesian cells): the least-squares cubic from the cross data d (neighbour
 * differences and cell-unit gradients, Cubic<R, M>::fit order), its
 * indicators, the 2m linear sub-polynomials and the path function, blended
 * into one cubic b = chi p^3 + (1 - chi) sum_k w_k p_k (coefficient M-1-a
 * multiplies xi_a); WENO-Z / TENO in the adaptive-order combination. */
template <typename R, int M>
__device__ __forceinline__ void blend_cubic(const KP &P, const R *d, R *b)
{
    constexpr int NC = Cubic<R, M>::NC;
    R c[NC];
    Cubic<R, M>::fit(d, c);
    /* blended cubic: chi c, plus lin on the linear monomials */
    R chi = R(1), lin[M];
#pragma unroll
    for (int a = 0; a < M; ++a) lin[a] = R(0);
    if (P.limiter != 1) {
        R ISH, ISt;
        Cubic<R, M>::ind(c, ISH, ISt);
        /* linear sub-polynomials on {cell, neighbour q}: g_e = (s dW + D_e)/2, g_t = D_t */
        R IS[2 * M], g[2 * M][M];
#pragma unroll
        for (int q = 0; q < 2 * M; ++q) {
            const int e = q / 2;
            const R s = (q & 1) ? R(1) : R(-1);
            R sum = R(0);
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const R D = d[q * (1 + M) + 1 + a];
                g[q][a] = (a == e) ? R(0.5) * (s * d[q * (1 + M)] + D) : D;
                sum += g[q][a] * g[q][a];
            }
            IS[q] = sum;
        }
        if (P.limiter == 0) {
            R smin = IS[0], smax = IS[0], ssum = R(0);
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                smin = fmin(smin, IS[q]);
                smax = fmax(smax, IS[q]);
                ssum += IS[q];
            }
            const R ISL = (ssum - smin - smax) * R(1.0 / (2 * M - 2));
            chi = chi_of<R>(P, ISt, ISH, ISL, 3);
            const R eps = pick<R>(P.eps, P.feps);
            R ws = R(0);
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                const R wq = R(1) / ((IS[q] + eps) * (IS[q] + eps));
                ws += wq;
#pragma unroll
                for (int a = 0; a < M; ++a) lin[a] += wq * g[q][a];
            }
            const R iws = R(1) / ws;
#pragma unroll
            for (int a = 0; a < M; ++a) lin[a] = (R(1) - chi) * (lin[a] * iws);
        } else {
            /* WENO-Z / TENO, adaptive-order combination: (w0/d0) p^3 +
             * sum_q (w_q - (w0/d0) d_q) p_q, the 2m linear polynomials
             * sharing 1 - d0 equally */
            const R d0 = pick<R>(P.d0, P.fd0), dq = (R(1) - d0) * R(1.0 / (2 * M));
            R d[2 * M + 1], I[2 * M + 1], w[2 * M + 1];
            d[0] = d0;
            I[0] = ISH;
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                d[q + 1] = dq;
                I[q + 1] = IS[q];
            }
            ao_weights<R, 2 * M>(P, d, I, ISt, w);
            chi = w[0] / d0;
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                const R cq = w[q + 1] - chi * dq;
#pragma unroll
                for (int a = 0; a < M; ++a) lin[a] += cq * g[q][a];
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < NC; ++kk) {
        b[kk] = chi * c[kk];
        if (kk < M) b[kk] += lin[M - 1 - kk];
    }
}

template <typename R, int M>
__device__ __forceinline__ void cell_poly_item(const KP &P, const Src<R> &src, R *__restrict__ B, long t)
{
    constexpr int NV = M + 2, NC = Cubic<R, M>::NC, ND = Cubic<R, M>::ND;
    int i, j, k;
    if (!ext_cell<M>(P, t, i, j, k)) return;
    /* the seven (five) cells of the cross: own first, then q = 2 e + (side > 0);
     * their ghost signs packed one word per cell (ghost_mask) */
    long cl[2 * M + 1];
    unsigned sm[2 * M + 1];
    /* a cell whose whole cross lies inside the grid needs no ghost mapping */
    bool inner = i >= 1 && i + 1 < P.n[0];
    if (M >= 2) inner = inner && j >= 1 && j + 1 < P.n[1];
    if (M >= 3) inner = inner && k >= 1 && k + 1 < P.n[2];
    if (inner) {
        const long st[3] = {1, (long)P.n[0], (long)P.n[0] * P.n[1]};
        cl[0] = ((long)k * P.n[1] + j) * P.n[0] + i;
        sm[0] = 0;
#pragma unroll
        for (int q = 0; q < 2 * M; ++q) {
            cl[1 + q] = cl[0] + ((q & 1) ? st[q / 2] : -st[q / 2]);
            sm[1 + q] = 0;
        }
    } else {
        int fl[3];
        cl[0] = cell_lin<M>(P, i, j, k, fl);
        sm[0] = ghost_mask<M>(P, fl);
#pragma unroll
        for (int q = 0; q < 2 * M; ++q) {
            int o[3] = {i, j, k};
            o[q / 2] += (q & 1) ? 1 : -1;
            cl[1 + q] = cell_lin<M>(P, o[0], o[1], o[2], fl);
            sm[1 + q] = ghost_mask<M>(P, fl);
        }
    }
    /* a cross with no mirrored cell (every cell away from non-periodic
     * boundaries) reads its data without the sign selects; the values are
     * those of the general path with every sign +1 */
    unsigned anyflip = 0;
#pragma unroll
    for (int q = 0; q <= 2 * M; ++q) anyflip |= sm[q];
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
        R d[ND];
        const R hr = pick<R>(P.h, P.fh);
        if (anyflip == 0) {
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                d[q * (1 + M)] = R(src.delta(v * P.ncell + cl[1 + q], v * P.ncell + cl[0]));
#pragma unroll
                for (int a = 0; a < M; ++a) d[q * (1 + M) + 1 + a] = src.grad((a * NV + v) * P.ncell + cl[1 + q]) * hr;
            }
#pragma unroll
            for (int a = 0; a < M; ++a) d[2 * M * (1 + M) + a] = src.grad((a * NV + v) * P.ncell + cl[0]) * hr;
        } else {
            const int s0v = ((sm[0] >> v) & 1u) ? -1 : 1;
#pragma unroll
            for (int q = 0; q < 2 * M; ++q) {
                const unsigned mq = sm[1 + q];
                const int sq = ((mq >> v) & 1u) ? -1 : 1;
                d[q * (1 + M)] = R(src.delta_signed(v * P.ncell + cl[1 + q], sq, v * P.ncell + cl[0], s0v));
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    const R g = src.grad((a * NV + v) * P.ncell + cl[1 + q]) * hr;
                    d[q * (1 + M) + 1 + a] = (((mq >> v) ^ (mq >> (8 + a))) & 1u) ? -g : g;
                }
            }
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const R g = src.grad((a * NV + v) * P.ncell + cl[0]) * hr;
                d[2 * M * (1 + M) + a] = (((sm[0] >> v) ^ (sm[0] >> (8 + a))) & 1u) ? -g : g;
            }
        }
        R b[NC];
        blend_cubic<R, M>(P, d, b);
        const long base = (long)v * NC;
#pragma unroll
        for (int kk = 0; kk < NC; ++kk) B[(base + kk) * P.next + t] = b[kk];
    }
}

template <typename R, int M>
__global__ void __launch_bounds__(128) cell_poly_kernel(KP P, Src<R> src, R *__restrict__ B)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < P.next) cell_poly_item<R, M>(P, src, B, t);
}

template <int M>
__device__ __forceinline__ long ext_lin(const KP &P, int i, int j, int k)
{
    long r = i + 1;
    if (M >= 2) r += (long)(j + 1) * P.ext[0];
    if (M >= 3) r += (long)(k + 1) * P.ext[0] * P.ext[1];
    return r;
}

/* The FP32 flux's staging buffer: one per dimension, shared by the
 * directions (a kernel that runs several directions, such as the batched
 * flux, holds one buffer, not one per direction). */
template <int M> __device__ __forceinline__ float *flux_stage()
{
    constexpr int NV = M + 2, NG = (M == 2) ? 2 : 4;
    __shared__ __align__(16) float buf[2 * NV * Cubic<float, M>::NC * (128 / NG)];
    return buf;
}

/* one (face, Gauss point) of direction D.  FLUX = false writes the states
 * face_states[side][v][c][g][face] (double, global axes); FLUX = true the
 * fluxes ff[q][v][g][face] (R, global momentum order). */
template <typename R, int M, int D, bool FLUX, bool NS = false, bool FSUM = false>
__device__ __forceinline__ void face_flux_item(const KP &P, const Src<R> &src, const R *__restrict__ B, double dtv,
                                               double *__restrict__ fs, R *__restrict__ ff, int *__restrict__ status,
                                               long t)
{
    constexpr int NV = M + 2, NC = Cubic<R, M>::NC, NG = (M == 2) ? 2 : 4;
    const long nf = P.nface[D];
    /* FP32: each aligned group of 128 items is one block of 4 warps; its NG
     * consecutive warps take the NG Gauss points of the same 32 faces, so the
     * Gauss point is warp-uniform (the per-point evaluation does not diverge)
     * and the two cells' coefficients are shared through L1.  Items past the
     * last face (the index space is rounded up to whole groups) compute a
     * valid face and write nothing.  FP64: one Gauss point per half of the
     * index space. */
    constexpr bool gfast = sizeof(R) == sizeof(float);
    const unsigned tu = (unsigned)t;
    int g;
    long fl;
    if constexpr (gfast) {
        g = (int)((tu >> 5) % NG);
        fl = (long)(tu >> 7) * (128 / NG) + (long)(((tu & 127u) >> 5) / NG) * 32 + (long)(tu & 31u);
    } else {
        g = (int)fdiv(P.dnf[D], tu);
        fl = t - (long)g * nf;
    }
    const bool valid = fl < nf && g < NG;
    /* a masked item evaluates the last face; in FP32 it keeps its warp's
     * Gauss point (always < NG), which also places it in the face sums'
     * shared tile below */
    if (!valid) {
        fl = nf - 1;
        if constexpr (!gfast) g = 0;
    }
    int idx[3];
    unsigned q0, q1;
    idx[0] = (int)fdivmod(P.dface[D][0], (unsigned)fl, q0);
    idx[1] = (M >= 2) ? (int)fdivmod(P.dface[D][1], q0, q1) : 0;
    idx[2] = (M >= 3) ? (int)q1 : 0;
    const R gm1 = pick<R>(P.fp.gm1, P.fgm1);
    /* FP32: the blended coefficients of the two cells of the block's faces
     * are staged in shared memory, stage[side][v * NC + k][face in block].
     * Each face's NG threads copy a share of its 2 NV NC values with cp.async
     * (all copies in flight at once, each value read once per face instead
     * of once per Gauss point, no registers held while they land); the face
     * sums below reuse the buffer. */
    constexpr int FB = 128 / NG, NVC = NV * NC;
    float *stage = nullptr;
    if constexpr (gfast) stage = flux_stage<M>();
    const int fb = (int)((((unsigned)threadIdx.x >> 5) / NG) * 32 + (threadIdx.x & 31u));
    if constexpr (gfast) {
        constexpr int PARTS = NG / 2, PER = NVC / PARTS;
        static_assert(NVC % PARTS == 0, "the copies split evenly over a side's threads");
        const int side = g & 1, part = g >> 1;
        int ci[3] = {idx[0], idx[1], idx[2]};
        if (side == 0) ci[D] -= 1;
        const float *sp = (const float *)B + (long)(part * PER) * P.next + ext_lin<M>(P, ci[0], ci[1], ci[2]);
        unsigned dp = (unsigned)__cvta_generic_to_shared(stage) + 4u * (unsigned)((side * NVC + part * PER) * FB + fb);
        __syncthreads(); /* a previous item's readers of the buffer are done */
#pragma unroll 10
        for (int k = 0; k < PER; ++k) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dp), "l"(sp) : "memory");
            sp += P.next;
            dp += 4u * FB;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
    }
    /* interface states, global axes: st[side][v][c], c = 0 value, 1 + e d/dx_e */
    R st[2][NV][M + 1], cw[2][NV];
    /* a face inside the grid has two real cells: no ghost mapping, no signs */
    const bool inner = idx[D] > 0 && idx[D] < P.n[D];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        int ci[3] = {idx[0], idx[1], idx[2]};
        if (side == 0) ci[D] -= 1;
        int flip[3] = {0, 0, 0};
        const long cl = inner ? ((long)ci[2] * P.n[1] + ci[1]) * P.n[0] + ci[0] : cell_lin<M>(P, ci[0], ci[1], ci[2], flip);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R c[NC], out[M + 1];
            if constexpr (gfast) {
#pragma unroll
                for (int kk = 0; kk < NC; ++kk) c[kk] = stage[(side * NVC + v * NC + kk) * FB + fb];
            } else {
                const long ce = ext_lin<M>(P, ci[0], ci[1], ci[2]);
#pragma unroll
                for (int kk = 0; kk < NC; ++kk) c[kk] = B[((long)v * NC + kk) * P.next + ce];
            }
            if (side == 0) CubicEval<R, M, D, 1>::run(g, c, out);
            else CubicEval<R, M, D, 0>::run(g, c, out);
            R w0 = R(src.w0(v * P.ncell + cl));
            if (!inner) w0 *= R(ghost_sign<M>(P, flip, v));
            cw[side][v] = w0;
            st[side][v][0] = w0 + out[0];
#pragma unroll
            for (int a = 0; a < M; ++a) st[side][v][1 + a] = out[1 + a] * pick<R>(P.ih, P.fih);
        }
        R s[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] = st[side][v][0];
        if (!admissible<R, M>(s, cw[side], gm1, pick<R>(P.adm, P.fadm))) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                st[side][v][0] = cw[side][v];
#pragma unroll
                for (int a = 0; a < M; ++a) st[side][v][1 + a] = R(0);
            }
        }
    }
    const long nft = P.nftot, face = P.foff[D] + fl;
    if (!FLUX) {
        if (!valid) return;
#pragma unroll
        for (int side = 0; side < 2; ++side)
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int c = 0; c < M + 1; ++c)
                    fs[(((long)(side * NV + v) * (M + 1) + c) * NG + g) * nft + face] = (double)st[side][v][c];
        return;
    }
    /* face frame: axis order (D, then the others ascending) */
    constexpr int A1 = (D == 0) ? 1 : 0;
    constexpr int A2 = (D == 2) ? 1 : 2;
    const int ax[3] = {D, A1, A2};
    R Wl[NV], Wr[NV], dWl[M][NV], dWr[M][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        /* face-frame variable index fv of global variable v */
        int fv = v;
        if (v >= 1 && v <= M) {
#pragma unroll
            for (int kk = 0; kk < M; ++kk)
                if (ax[kk] == v - 1) fv = 1 + kk;
        }
        Wl[fv] = st[0][v][0];
        Wr[fv] = st[1][v][0];
#pragma unroll
        for (int kk = 0; kk < M; ++kk) {
            dWl[kk][fv] = st[0][v][1 + ax[kk]];
            dWr[kk][fv] = st[1][v][1 + ax[kk]];
        }
    }
    R F[NV], Ft[NV], Wh[NV];
    const R dt = R(dtv);
    if (!gks_point<R, M, NS>(P.fp, dt, Wl, Wr, dWl, dWr, F, Ft, Wh)) {
        atomicOr(status, ST_FLUX);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = Ft[v] = Wh[v] = R(0);
    }
    /* walls (slip or no-slip) are at rest and adiabatic: neither mass nor
     * energy crosses them (exactly, whatever the rounding of the two sides) */
    if ((idx[D] == 0 && P.bcs[D][0] >= 2) || (idx[D] == P.n[D] && P.bcs[D][1] >= 2))
        F[0] = F[NV - 1] = Ft[0] = Ft[NV - 1] = R(0);
    if constexpr (FSUM) {
        /* step path in FP32: sum the face's NG Gauss points (the NG warps of
         * its group, through shared memory; every thread of the block takes
         * part) in the order (F0 + F1) [+ (F2 + F3)], and store one value per
         * face and quantity, ff[q][v][face] (q = F, dF/dt, W(dt/2)) */
        static_assert(gfast, "face sums need the warp-group mapping");
        static_assert(3 * NV * 128 <= 2 * NVC * FB, "the face sums fit in the staging buffer");
        R(*xs)[128] = reinterpret_cast<R(*)[128]>(stage);
        const int lt = threadIdx.x;
        __syncthreads(); /* every thread has read its coefficients */
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            xs[v][lt] = F[v];
            xs[NV + v][lt] = Ft[v];
            xs[2 * NV + v][lt] = Wh[v];
        }
        __syncthreads();
        const int l0 = lt - g * 32; /* this face's Gauss point 0 */
#pragma unroll
        for (int q = 0; q < 3 * NV; ++q) {
            R a = xs[q][l0] + xs[q][l0 + 32];
            if constexpr (NG == 4) a = a + (xs[q][l0 + 64] + xs[q][l0 + 96]);
            if (q < NV) F[q] = a;
            else if (q < 2 * NV) Ft[q - NV] = a;
            else Wh[q - 2 * NV] = a;
        }
        __syncthreads();
        if (g == 0 && valid) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                int fv = v;
                if (v >= 1 && v <= M) {
#pragma unroll
                    for (int kk = 0; kk < M; ++kk)
                        if (ax[kk] == v - 1) fv = 1 + kk;
                }
                ff[(long)(0 * NV + v) * nft + face] = F[fv];
                ff[(long)(1 * NV + v) * nft + face] = Ft[fv];
                ff[(long)(2 * NV + v) * nft + face] = Wh[fv];
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            int fv = v;
            if (v >= 1 && v <= M) {
#pragma unroll
                for (int kk = 0; kk < M; ++kk)
                    if (ax[kk] == v - 1) fv = 1 + kk;
            }
            if (!valid) continue;
            ff[((long)(0 * NV + v) * NG + g) * nft + face] = F[fv];
            ff[((long)(1 * NV + v) * NG + g) * nft + face] = Ft[fv];
            ff[((long)(2 * NV + v) * NG + g) * nft + face] = Wh[fv];
        }
    }
}

/* 128 threads.  Blocks per SM asked of the FP32 flux, measured with the
 * warp-group mapping: 2D 8 (64 registers; 1.7% faster than 7, 4.5% than 6),
 * 3D 7 (72 registers; 6.8% faster than 8), Navier-Stokes 5 (more live
 * moments; 3.4% faster than 4 and 6).  The FP64 flux is bound by the FP64
 * pipe and keeps its registers. */
template <typename R, int M, bool NS> constexpr int flux_blocks_per_sm()
{
    return sizeof(R) == sizeof(float) ? (NS ? 5 : (M == 2 ? 8 : 7)) : 1;
}

template <typename R, int M, int D, bool FLUX, bool NS = false, bool FSUM = false>
__global__ void __launch_bounds__(128, (flux_blocks_per_sm<R, M, NS>())) face_flux_kernel(KP P, Src<R> src, const R *__restrict__ B,
                                                        const double *__restrict__ dtp, double *__restrict__ fs,
                                                        R *__restrict__ ff, int *__restrict__ status)
{
    constexpr int NG = (M == 2) ? 2 : 4;
    /* 128 threads per block.  FP32: the grid covers whole 128-item groups
     * (ceil(nface / (128 / NG)) blocks) and every thread runs the item, which
     * masks the items past the last face (its face sums synchronise the
     * block).  FP64: one thread per (face, Gauss point). */
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sizeof(R) == sizeof(float) || t < P.nface[D] * NG)
        face_flux_item<R, M, D, FLUX, NS, FSUM>(P, src, B, FLUX ? dtp[0] : 0.0, fs, ff, status, t);
}

/* Shared-memory carveout of a kernel with static shared memory: the smallest
 * share of the SM's unified L1/shared storage that still holds `blocks`
 * resident blocks (the CUDA driver rounds the preference up to the next supported
 * capacity; the default can hold fewer blocks than the launch bounds ask
 * for), so the rest stays L1.  Set once per kernel; a refusal leaves the
 * default. */
template <typename K> inline void smem_carveout_for(K kernel, int blocks)
{
    cudaFuncAttributes fa;
    int dev = 0, maxsm = 0, rsv = 0;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess || maxsm <= 0) {
        (void)cudaGetLastError();
        return;
    }
    const long need = (long)blocks * (long)(fa.sharedSizeBytes + rsv);
    long pct = (need * 100 + maxsm - 1) / maxsm;
    if (pct > 100) pct = 100;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)pct) != cudaSuccess)
        (void)cudaGetLastError();
}

/* once per instantiation, before its first launch */
template <typename R, int M, int D, bool FLUX, bool NS = false, bool FSUM = false> inline void face_flux_prepare()
{
    static const bool done = (smem_carveout_for(face_flux_kernel<R, M, D, FLUX, NS, FSUM>, flux_blocks_per_sm<R, M, NS>()), true);
    (void)done;
}

/* ------------------------------------------------------------------ */
/* FP64 stage update                                                   */
/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* Double-float arithmetic in FP32 (a value is hi + lo, |lo| <= ulp(hi)/2 */
/* after normalisation): TwoSum (Knuth), FastTwoSum (Dekker) and TwoProd  */
/* by fused multiply-add give the rounding errors of FP32 additions and   */
/* products exactly, so sums and products carry about 48 bits.            */
/* ------------------------------------------------------------------ */
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 df_two_sum(float a, float b)
{
    const float s = a + b;
    const float z = s - a;
    return F2{s, (a - (s - z)) + (b - z)};
}

/* requires |a| >= |b| (or a == 0) */
__device__ __forceinline__ F2 df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return F2{s, b - (s - a)};
}

__device__ __forceinline__ F2 df_mul(F2 k, F2 x)
{
    const float p = k.hi * x.hi;
    float e = fmaf(k.hi, x.hi, -p);
    e = fmaf(k.hi, x.lo, e);
    e = fmaf(k.lo, x.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ F2 df_add(F2 a, F2 b)
{
    const F2 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ F2 df_split(double x)
{
    const float h = (float)x;
    return F2{h, (float)(x - (double)h)};
}

/* the stage constants of the mixed-precision update as double-floats:
 * with S the exact face sum of a cell and cw = 1 / (h NG),
 *   stage 1: W* - W = k0 S(F) + k1 S(Ft),  Acc = k2 S(F) + k3 S(Ft);
 *   stage 2: W^{n+1} - W = Acc + k4 S(Ft*) */
struct UpdC {
    F2 k[5];
};

__device__ __forceinline__ UpdC make_updc(double dt, double cw)
{
    UpdC u;
    u.k[0] = df_split(-0.5 * dt * cw);
    u.k[1] = df_split(-0.125 * dt * dt * cw);
    u.k[2] = df_split(-dt * cw);
    u.k[3] = df_split(-dt * dt / 6.0 * cw);
    u.k[4] = df_split(-dt * dt / 3.0 * cw);
    return u;
}

/* The stage constants live in a 10-float device buffer, written once per
 * time step by the kernel that sets dt, so the update kernel (one cell per
 * thread) neither recomputes them per block in FP64 nor waits on a barrier
 * for them.  The fused stage kernels compute them once per strip, which
 * their rows amortise. */
__device__ __forceinline__ void store_updc(float *p, const UpdC &u)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        p[2 * k] = u.k[k].hi;
        p[2 * k + 1] = u.k[k].lo;
    }
}
__device__ __forceinline__ UpdC load_updc(const float *__restrict__ p)
{
    UpdC u;
#pragma unroll
    for (int k = 0; k < 5; ++k) u.k[k] = F2{p[2 * k], p[2 * k + 1]};
    return u;
}
/* the Gauss-point weight of a face sum over the cell size: 1 / (h NG) */
__host__ __device__ __forceinline__ double updc_cw(const KP &P, int dim) { return P.ih / (dim == 3 ? 4 : 2); }

/* s + e += x exactly up to the rounding of e (Knuth's TwoSum, FP32 adds
 * only, so nothing can be contracted or reassociated) */
__device__ __forceinline__ void two_sum_acc(float &s, float &e, float x)
{
    const float t = s + x;
    const float z = t - s;
    e += (s - (t - z)) + (x - z);
    s = t;
}

template <int M>
__device__ __forceinline__ long face_of(const KP &P, int d, int i, int j, int k, int s)
{
    int e0 = P.n[0] + (d == 0), e1 = P.n[1] + (d == 1);
    int idx[3] = {i, j, k};
    idx[d] += s;
    return P.foff[d] + ((long)idx[2] * e1 + idx[1]) * e0 + idx[0];
}

/* The mixed-precision stage update of one cell from the FP32 face sums over
 * the Gauss points, fsum(q, v, d, plus): q = 0 F, 1 dF/dt, 2 W(dt/2) of
 * variable v on the cell's face of direction d (plus = 1 the upper face).
 * A cell adds its faces' fluxes exactly (double-float accumulation), so each
 * face's flux leaves one cell and enters the other without a rounding of its
 * own, and the stage combination runs in double-float FP32 arithmetic (about
 * 48 bits; GB300's FP64 rate is 1/64 of FP32).  Stage 1 writes the next
 * input directly as its FP32 shadow s1 (= s0 + increment) and keeps Acc as a
 * float pair acc[2][nv][cell]; stage 2 adds its increment to the FP64 state W
 * and re-splits W into s0, so the shadow never drifts from W.  The sums of
 * the averages are conserved to FP64 rounding.  Gradients (not conserved)
 * come from FP32 differences of the interface states and live in the shadow
 * only (Eq. slope).  mixed_update_var updates variable v (nc cells, fih =
 * 1/h in FP32) and returns its new FP32 value; mixed_update_cell all
 * variables and the admissibility flags. */
template <int M, int STAGE, typename FaceSum>
__device__ __forceinline__ float mixed_update_var(long nc, float fih, const FaceSum &fsum, const UpdC &uc,
                                                 double *__restrict__ W, float *__restrict__ acc, const Shadow &s0,
                                                 const Shadow &s1, long cell, int v)
{
    constexpr int NV = M + 2, NG = (M == 2) ? 2 : 4;
    const float gw = fih / NG;
    const Shadow &so = (STAGE == 1) ? s1 : s0;
    float sF = 0.f, eF = 0.f, sT = 0.f, eT = 0.f;
#pragma unroll
    for (int d = 0; d < M; ++d) {
        if (STAGE == 1) {
            two_sum_acc(sF, eF, fsum(0, v, d, 1));
            two_sum_acc(sF, eF, -fsum(0, v, d, 0));
        }
        two_sum_acc(sT, eT, fsum(1, v, d, 1));
        two_sum_acc(sT, eT, -fsum(1, v, d, 0));
        so.g[(d * NV + v) * nc + cell] = (fsum(2, v, d, 1) - fsum(2, v, d, 0)) * gw;
    }
    const F2 ST{sT, eT};
    if (STAGE == 1) {
        const F2 SF{sF, eF};
        const F2 dW = df_add(df_mul(uc.k[0], SF), df_mul(uc.k[1], ST));
        const F2 A = df_add(df_mul(uc.k[2], SF), df_mul(uc.k[3], ST));
        acc[v * nc + cell] = A.hi;
        acc[(NV + v) * nc + cell] = A.lo;
        const F2 w = df_add(F2{s0.hi[v * nc + cell], s0.lo[v * nc + cell]}, dW);
        so.hi[v * nc + cell] = w.hi;
        so.lo[v * nc + cell] = w.lo;
        return w.hi;
    } else {
        const F2 dW = df_add(F2{acc[v * nc + cell], acc[(NV + v) * nc + cell]}, df_mul(uc.k[4], ST));
        const double w = (W[v * nc + cell] + widen(dW.hi)) + widen(dW.lo);
        W[v * nc + cell] = w;
        float wh, wl;
        split(w, wh, wl);
        so.hi[v * nc + cell] = wh;
        so.lo[v * nc + cell] = wl;
        return wh;
    }
}

/* admissibility flags of a new state from the FP32 values of its variables */
template <int M> __device__ __forceinline__ void mixed_state_flags(const KP &P, const float *wn, int *__restrict__ status)
{
    float ke = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) ke += wn[1 + a] * wn[1 + a];
    const float p = P.fgm1 * (wn[M + 1] - 0.5f * ke / wn[0]);
    int st = 0;
    if (!(wn[0] > 0.f)) st |= ST_RHO;
    if (!(p > 0.f)) st |= ST_P;
    if (!isfinite(p) || !isfinite(wn[0])) st |= ST_NAN;
    if (st) atomicOr(status, st);
}

template <int M, int STAGE, typename FaceSum>
__device__ __forceinline__ void mixed_update_cell(const KP &P, const FaceSum &fsum, const UpdC &uc,
                                                  double *__restrict__ W, float *__restrict__ acc, const Shadow &s0,
                                                  const Shadow &s1, int *__restrict__ status, long cell)
{
    constexpr int NV = M + 2;
    float wn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) wn[v] = mixed_update_var<M, STAGE>(P.ncell, P.fih, fsum, uc, W, acc, s0, s1, cell, v);
    mixed_state_flags<M>(P, wn, status);
}

/* STAGE 1: Ws = W - dt/2 L(F) - dt^2/8 L(Ft), Gs = Gauss(W(dt/2)), Acc = -dt L(F) - dt^2/6 L(Ft)
 * STAGE 2: W += Acc - dt^2/3 L(Ft*),        G  = Gauss(W*(dt/2))
 * with L(q)_j = (1/h) sum_d sum_g w_g (q(+d face) - q(-d face)). */
template <typename R, int M, int STAGE>
__device__ __forceinline__ void update_item(const KP &P, const R *__restrict__ ff, double dt, double *__restrict__ W,
                                            double *__restrict__ G, double *__restrict__ Ws, double *__restrict__ Gs,
                                            double *__restrict__ Acc, const Shadow &s0, const Shadow &s1,
                                            int *__restrict__ status, long cell, const UpdC &uc)
{
    constexpr int NV = M + 2, NG = (M == 1) ? 1 : ((M == 2) ? 2 : 4);
    if constexpr (sizeof(R) == sizeof(float) && M >= 2) {
        /* mixed precision: the face values are per-face FP32 sums over the
         * Gauss points (ff[q][v][face]); see mixed_update_cell */
        unsigned q0, q1;
        const int i = (int)fdivmod(P.dn[0], (unsigned)cell, q0);
        const int j = (int)fdivmod(P.dn[1], q0, q1);
        const int k = (M >= 3) ? (int)q1 : 0;
        const long nft = P.nftot;
        long fp[M], fm[M];
#pragma unroll
        for (int d = 0; d < M; ++d) {
            fp[d] = face_of<M>(P, d, i, j, k, 1);
            fm[d] = face_of<M>(P, d, i, j, k, 0);
        }
        /* face sums ff[q][v][face] of the cell's faces */
        auto fsum = [&](int q, int v, int d, int plus) -> float {
            return ff[(long)(q * NV + v) * nft + (plus ? fp[d] : fm[d])];
        };
        mixed_update_cell<M, STAGE>(P, fsum, uc, W, (float *)Acc, s0, s1, status, cell);
        return;
    }
    unsigned q0, q1 = 0;
    const int i = (int)fdivmod(P.dn[0], (unsigned)cell, q0);
    const int j = (M >= 2) ? (int)fdivmod(P.dn[1], q0, q1) : 0;
    const int k = (M >= 3) ? (int)q1 : 0;
    const double ih = P.ih, wg = 1.0 / NG;
    const long nft = P.nftot;
    long fp[M], fm[M];
#pragma unroll
    for (int d = 0; d < M; ++d) {
        fp[d] = face_of<M>(P, d, i, j, k, 1);
        fm[d] = face_of<M>(P, d, i, j, k, 0);
    }
    double Wn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double DF = 0.0, DFt = 0.0;
#pragma unroll
        for (int d = 0; d < M; ++d) {
            double Dh = 0.0;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const long o0 = ((long)(0 * NV + v) * NG + g) * nft, o1 = ((long)(1 * NV + v) * NG + g) * nft,
                           o2 = ((long)(2 * NV + v) * NG + g) * nft;
                DF += (double)ff[o0 + fp[d]] - (double)ff[o0 + fm[d]];
                DFt += (double)ff[o1 + fp[d]] - (double)ff[o1 + fm[d]];
                Dh += (double)ff[o2 + fp[d]] - (double)ff[o2 + fm[d]];
            }
            double *Gout = (STAGE == 1) ? Gs : G;
            Gout[(d * NV + v) * P.ncell + cell] = Dh * wg * ih;
        }
        DF *= wg * ih;
        DFt *= wg * ih;
        if (STAGE == 1) {
            Ws[v * P.ncell + cell] = W[v * P.ncell + cell] - 0.5 * dt * DF - dt * dt * 0.125 * DFt;
            Acc[v * P.ncell + cell] = -dt * DF - dt * dt / 6.0 * DFt;
            Wn[v] = Ws[v * P.ncell + cell];
        } else {
            const double w = W[v * P.ncell + cell] + Acc[v * P.ncell + cell] - dt * dt / 3.0 * DFt;
            W[v * P.ncell + cell] = w;
            Wn[v] = w;
        }
    }
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) ke += Wn[1 + a] * Wn[1 + a];
    const double p = (P.gamma - 1.0) * (Wn[M + 1] - 0.5 * ke / Wn[0]);
    int st = 0;
    if (!(Wn[0] > 0.0)) st |= ST_RHO;
    if (!(p > 0.0)) st |= ST_P;
    if (!isfinite(p) || !isfinite(Wn[0])) st |= ST_NAN;
    if (st) atomicOr(status, st);
}

template <typename R, int M, int STAGE>
__global__ void __launch_bounds__(256) update_kernel(KP P, const R *__restrict__ ff, const double *__restrict__ dtp,
                                                    double *__restrict__ W, double *__restrict__ G,
                                                    double *__restrict__ Ws, double *__restrict__ Gs,
                                                    double *__restrict__ Acc, Shadow s0, Shadow s1,
                                                    int *__restrict__ status, const float *__restrict__ updc)
{
    /* the mixed-precision stage constants of this time step (FP64 path: unused) */
    UpdC uc;
    if constexpr (sizeof(R) == sizeof(float) && M >= 2) uc = load_updc(updc);
    const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell < P.ncell) update_item<R, M, STAGE>(P, ff, dtp[0], W, G, Ws, Gs, Acc, s0, s1, status, cell, uc);
}

/* FP64 gradients from the FP32 shadow (mixed precision keeps the gradients
 * in the shadow only; this fills G when the state is read) */
static __global__ void widen_grad_kernel(const float *__restrict__ g, double *__restrict__ G, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        G[i] = (double)g[i];
}

/* FP32 shadow of the FP64 state (after the state is set) */
template <int M>
__global__ void shadow_kernel(KP P, const double *__restrict__ W, const double *__restrict__ G, Shadow s)
{
    constexpr int NV = M + 2;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += (long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            split_store(W[v * P.ncell + c], s.hi, s.lo, v * P.ncell + c);
#pragma unroll
            for (int a = 0; a < M; ++a) s.g[(a * NV + v) * P.ncell + c] = (float)G[(a * NV + v) * P.ncell + c];
        }
    }
}

/* ------------------------------------------------------------------ */
/* CFL time step on the device                                         */
/* ------------------------------------------------------------------ */
/* max over cells of max_d |u_d| + c, read from the FP64 state (T = double)
 * or from its FP32 shadow (T = float) */
template <int M, typename T>
__global__ void wavespeed_kernel(KP P, const T *__restrict__ W, unsigned long long *__restrict__ smax)
{
    T s = T(0), ir = T(0); /* max |u_d| + c and max 1 / rho */
    const T gam = pick<T>(P.gamma, (float)(P.fgm1 + 1.0f));
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += (long)gridDim.x * blockDim.x) {
        const T rho = W[c];
        T ke = T(0), um = T(0);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const T u = W[(1 + a) * P.ncell + c] / rho;
            ke += u * u;
            um = fmax(um, fabs(u));
        }
        const T p = (gam - T(1)) * (W[(M + 1) * P.ncell + c] - T(0.5) * rho * ke);
        s = fmax(s, um + sqrt(gam * p / rho));
        ir = fmax(ir, T(1) / rho);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        ir = fmax(ir, __shfl_xor_sync(0xffffffffu, ir, o));
    }
    __shared__ T red[2][32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s;
        red[1][threadIdx.x >> 5] = ir;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < (blockDim.x >> 5);
        s = in ? red[0][threadIdx.x] : T(0);
        ir = in ? red[1][threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
            ir = fmax(ir, __shfl_xor_sync(0xffffffffu, ir, o));
        }
        /* non-negative doubles order like their bit patterns; NaN is caught on the host */
        const double sd = (double)s, id = (double)ir;
        if (threadIdx.x == 0) {
            atomicMax(smax, (unsigned long long)__double_as_longlong(isnan(sd) ? 1e300 : sd));
            atomicMax(smax + 1, (unsigned long long)__double_as_longlong(isnan(id) ? 1e300 : id));
        }
    }
}

/* dt = cfl h / max(|u_d| + c), and with viscosity mu > 0 also at most
 * cfl h^2 / (2 (m - 1) nu_max), nu_max = mu max(1 / rho) (Sec. 6; the factor
 * 2 (m - 1) is taken as 2 in 1D) */
static __global__ void dt_from_speed_kernel(const unsigned long long *__restrict__ smax, double cfl_h, double visc,
                                            double *__restrict__ dtp, float *__restrict__ updc, double cw)
{
    const double s = __longlong_as_double((long long)smax[0]);
    double dt = cfl_h / s;
    if (visc > 0.0) {
        const double nu = visc * __longlong_as_double((long long)smax[1]);
        dt = fmin(dt, cfl_h / nu);
    }
    dtp[0] = dt;
    if (updc) store_updc(updc, make_updc(dt, cw));
}

/* a time step given by the caller (and, with updc, its stage constants) */
static __global__ void set_dt_kernel(double *__restrict__ dtp, double dt, float *__restrict__ updc, double cw)
{
    dtp[0] = dt;
    if (updc) store_updc(updc, make_updc(dt, cw));
}

} // namespace gks
