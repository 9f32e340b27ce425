/*
 * Gas-kinetic interface flux for the Euler and Navier-Stokes equations
 * (device code).
 *
 * The paper (Sec. 2) takes the flux from the time-dependent gas distribution
 * function of the GKS and defers its formulas to earlier work; this is the
 * BGK solution at an interface Gauss point in the face frame (velocity
 * component 0 and derivative axis 0 along the face normal):
 *
 *   f(0,t) = (1-e) g0 + t e (T0 g0) + t (A0 g0)
 *          + e [ (1 - t T_l) H(u) g_l + (1 - t T_r) H(-u) g_r ],   e = exp(-t/tau_n),
 *
 * with T = sum_e a_e u_e the spatial micro-slopes (left, right, and the
 * equilibrium one from the mean of the left/right derivatives), A0 the
 * equilibrium time slope from the compatibility condition, the physical
 * collision time 0 (Euler) in the Chapman-Enskog terms and the numerical one
 * tau_n = C1 dt + C2 |pl - pr| / (pl + pr) dt in the relaxation factor.
 *
 * Closed forms used here (all exact rearrangements of the velocity
 * integrals):
 *   rho0 <u psi>_0        = Euler flux of W0;
 *   rho0 <T0 psi>_0       = sum_e dF_e/dx_e(W0) = -dW0/dt;
 *   rho0 <A0 u psi>_0     = dF_n/dt = F_n'(W0) dW0/dt;
 *   time integrals over [0, d]: int (1-e) = d - ie, int t e = ite,
 *     ie = tau_n (1 - e_d), ite = tau_n^2 - tau_n (d + tau_n) e_d.
 * With the integrated fluxes over dt/2 and dt, F = (4 F(dt/2) - F(dt)) / dt
 * and dF/dt = 4 (F(dt) - 2 F(dt/2)) / dt^2 reduce to
 *   F  = F0 + (4 ie_h - ie_1)/dt (Fk - F0) + (4 ite_h - ite_1)/dt (FT0 - FTk),
 *   Ft = FA0 + 4 (ie_1 - 2 ie_h)/dt^2 (Fk - F0) + 4 (ite_1 - 2 ite_h)/dt^2 (FT0 - FTk),
 * and the interface state W(dt/2) = W0 + t (1 - e_t) dW0/dt - t e_t WTk.
 *
 * Navier-Stokes (Sec. 2, viscous flux of the same scheme; Prandtl number 1):
 * the general BGK solution with physical collision time tau > 0,
 *   f(0,t) = (1-e) g0 + ((t+tau) e - tau) T0 g0 + (t - tau + tau e) A0 g0
 *          + e [ (1 - (t+tau) T_l - tau A_l) H(u) g_l + (same, r) H(-u) g_r ],
 * tau = mu / p0 and e = exp(-t/(tau_n + tau)); A_l, A_r the time slopes of
 * the two initial states from their own compatibility conditions.  The tau
 * terms of the integrals add tau (cF1 D - V) to F, tau cT1 D to Ft and
 * -tau e_t (WTk + WAk) to W(dt/2), with V = rho0 <u psi (T0 + A0)>_0 and
 * D = V - FTk - FAk (FAk, WAk: the two half-space moments of A_l, A_r).
 *
 * The FP32 Euler flux evaluates the left and the right Maxwellian together
 * on lane pairs (lr2.cuh: one packed two-lane instruction for both sides);
 * the arithmetic of each lane is the scalar code's.
 */
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "lr2.cuh"

namespace gks {

template <typename R> struct RT;
template <> struct RT<double> {
    __device__ static double erfc_(double x) { return erfc(x); }
    __device__ static double exp_(double x) { return exp(x); }
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double rsqrt_(double x) { return rsqrt(x); }
    __device__ static double tanh_(double x) { return tanh(x); }
    __device__ static double abs_(double x) { return fabs(x); }
};
/* FP32: the exponentials of the flux (the half-space moments' exp(-lambda
 * U^2) and the relaxation factor) take the hardware exponential (__expf,
 * about 2 + 1.2 |x| ulp); both multiply terms that vanish as |x| grows, and
 * the 2048^2 mixed step is 1.3% shorter */
template <> struct RT<float> {
    __device__ static float erfc_(float x) { return erfcf(x); }
    __device__ static float exp_(float x) { return __expf(x); }
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ static float tanh_(float x) { return tanhf(x); }
    __device__ static float abs_(float x) { return fabsf(x); }
};

/* left/right pairs: the transcendentals per lane */
template <> struct RT<LR> {
    __device__ static LR erfc_(LR x) { return LR(erfcf(x.l()), erfcf(x.r())); }
    __device__ static LR exp_(LR x) { return LR(__expf(x.l()), __expf(x.r())); }
    __device__ static LR sqrt_(LR x) { return LR(sqrtf(x.l()), sqrtf(x.r())); }
    __device__ static LR rsqrt_(LR x) { return LR(rsqrtf(x.l()), rsqrtf(x.r())); }
};

/* x > 0 (every lane of a pair) */
__device__ __forceinline__ bool positive(double x) { return x > 0.0; }
__device__ __forceinline__ bool positive(float x) { return x > 0.f; }
__device__ __forceinline__ bool positive(LR x) { return x.l() > 0.f && x.r() > 0.f; }

/* Primitive description of a Maxwellian: density, velocity, pressure,
 * 1/(2 lambda) = p/rho, lambda = rho/(2p), and 1/rho (each reciprocal taken
 * once per Maxwellian and shared by every moment and slope of it). */
template <typename R, int M> struct Prim {
    R rho, U[3], p, i2l, lam, inv; /* i2l = 1 / (2 lambda), inv = 1 / rho */
};

template <typename R, int M>
__device__ __forceinline__ bool to_prim(const R *W, R gm1, Prim<R, M> &P)
{
    P.rho = W[0];
    const R inv = R(1) / W[0];
    R ke = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) P.U[a] = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        P.U[a] = W[1 + a] * inv;
        ke += P.U[a] * W[1 + a];
    }
    P.p = gm1 * (W[M + 1] - R(0.5) * ke);
    P.i2l = P.p * inv;
    P.lam = R(0.5) / P.i2l;
    P.inv = inv;
    return positive(W[0]) && positive(P.p);
}

/* Moments of a Maxwellian: u-moments (full or half space), full v, w moments,
 * and <xi^2>, <xi^4> of the K internal degrees of freedom. */
template <typename R, int M> struct Mom {
    R u[7];
    R v[6];
    R w[6];
    R xi[3];
};

template <typename R, int N>
__device__ __forceinline__ void full_moments(R U, R i2l, R *m)
{
    m[0] = R(1);
    m[1] = U;
#pragma unroll
    for (int k = 0; k + 2 < N; ++k) m[k + 2] = U * m[k + 1] + R(k + 1) * i2l * m[k];
}

/* half-space u moments: s = +1 integrates u > 0, -1 integrates u < 0 */
template <typename R, int N>
__device__ __forceinline__ void half_moments(R U, R lam, R i2l, R s, R *m)
{
    const R isl = RT<R>::rsqrt_(lam); /* 1 / sqrt(lambda) */
    const R x = lam * isl * U;        /* sqrt(lambda) U */
    m[0] = R(0.5) * RT<R>::erfc_(-s * x);
    /* exp(-lambda U^2) / (2 sqrt(pi lambda)) */
    m[1] = U * m[0] + s * R(0.5) * RT<R>::exp_(-x * x) * R(0.56418958354775628) * isl;
#pragma unroll
    for (int k = 0; k + 2 < N; ++k) m[k + 2] = U * m[k + 1] + R(k + 1) * i2l * m[k];
}

template <typename R, int M>
__device__ __forceinline__ void tangential_and_internal(const Prim<R, M> &P, R K, Mom<R, M> &T)
{
    if constexpr (M >= 2) full_moments<R, 6>(P.U[1], P.i2l, T.v);
    if constexpr (M >= 3) full_moments<R, 6>(P.U[2], P.i2l, T.w);
    T.xi[0] = R(1);
    T.xi[1] = K * P.i2l;
    T.xi[2] = K * (K + R(2)) * P.i2l * P.i2l;
}

/* <u^a v^b w^c xi^(2d)> */
template <typename R, int M, int A, int B, int C, int D>
__device__ __forceinline__ R mono(const Mom<R, M> &T)
{
    static_assert(A <= 6 && B <= 5 && C <= 5 && D <= 2, "moment order");
    R r = T.u[A];
    if constexpr (M >= 2 && B > 0) r *= T.v[B];
    if constexpr (M >= 3 && C > 0) r *= T.w[C];
    if constexpr (D > 0) r *= T.xi[D];
    return r;
}

/* <s u^A v^B w^C xi^(2D)> for s = s0 + s1 u (+ s2 v + s3 w) + sE (|u|^2 + xi^2)/2 */
template <typename R, int M, int A, int B, int C, int D>
__device__ __forceinline__ R mom_s(const Mom<R, M> &T, const R *s)
{
    R r = s[0] * mono<R, M, A, B, C, D>(T) + s[1] * mono<R, M, A + 1, B, C, D>(T);
    R e = mono<R, M, A + 2, B, C, D>(T) + mono<R, M, A, B, C, D + 1>(T);
    if constexpr (M >= 2) {
        r += s[2] * mono<R, M, A, B + 1, C, D>(T);
        e += mono<R, M, A, B + 2, C, D>(T);
    }
    if constexpr (M >= 3) {
        r += s[3] * mono<R, M, A, B, C + 1, D>(T);
        e += mono<R, M, A, B, C + 2, D>(T);
    }
    return r + R(0.5) * s[M + 1] * e;
}

/* out[b] += <psi_b u^A v^B w^C s> for every b */
template <typename R, int M, int A, int B, int C>
__device__ __forceinline__ void psi_mom_s(const Mom<R, M> &T, const R *s, R *out)
{
    out[0] += mom_s<R, M, A, B, C, 0>(T, s);
    out[1] += mom_s<R, M, A + 1, B, C, 0>(T, s);
    if constexpr (M >= 2) out[2] += mom_s<R, M, A, B + 1, C, 0>(T, s);
    if constexpr (M >= 3) out[3] += mom_s<R, M, A, B, C + 1, 0>(T, s);
    R e = mom_s<R, M, A + 2, B, C, 0>(T, s) + mom_s<R, M, A, B, C, 1>(T, s);
    if constexpr (M >= 2) e += mom_s<R, M, A, B + 2, C, 0>(T, s);
    if constexpr (M >= 3) e += mom_s<R, M, A, B, C + 2, 0>(T, s);
    out[M + 1] += R(0.5) * e;
}

/* <v^A w^B (S^2)^P> over the transverse variables, S^2 = v^2 + w^2 + xi^2
 * (w absent for M = 2, v and w for M = 1), P = 0, 1, 2; the factors are
 * independent Maxwellian moments. */
template <typename R, int M, int A, int B, int P>
__device__ __forceinline__ R tv(const Mom<R, M> &T)
{
    auto V = [&](int k) -> R {
        if constexpr (M >= 2) return T.v[k];
        else return k == 0 ? R(1) : R(0);
    };
    auto Wm = [&](int k) -> R {
        if constexpr (M >= 3) return T.w[k];
        else return k == 0 ? R(1) : R(0);
    };
    const R X1 = T.xi[1], X2 = T.xi[2];
    if constexpr (P == 0) {
        return V(A) * Wm(B);
    } else if constexpr (P == 1) {
        R r = V(A) * Wm(B) * X1;
        if constexpr (M >= 2) r += V(A + 2) * Wm(B);
        if constexpr (M >= 3) r += V(A) * Wm(B + 2);
        return r;
    } else {
        R r = V(A) * Wm(B) * X2;
        if constexpr (M >= 2) r += V(A + 4) * Wm(B) + R(2) * V(A + 2) * Wm(B) * X1;
        if constexpr (M >= 3) r += V(A) * Wm(B + 4) + R(2) * V(A) * Wm(B + 2) * X1 + R(2) * V(A + 2) * Wm(B + 2);
        return r;
    }
}

/* Moments of the slope term T = sum_e u_e (s_e . psi) of one Maxwellian:
 * Wo[b] = <psi_b T> (if Wo) and Fo[b] = <u psi_b T> (if Fo), the u-moments
 * of T taken from Tm (half or full space).  T is split by powers of u,
 *   T = T0 + u T1 + u^2 T2 + u^3 T3 (coefficients in the transverse v, w, xi),
 * the transverse expectations <T_n>, <v_r T_n>, <S^2 T_n> are tabulated once,
 * and every psi moment is a short dot product with the u-moments:
 *   <u^K psi_0 T> = sum_n U_(n+K) <T_n>,  <u^K psi_1 T> = sum_n U_(n+1+K) <T_n>,
 *   <u^K v_r T> = sum_n U_(n+K) <v_r T_n>,
 *   <u^K psi_E T> = 1/2 sum_n (U_(n+2+K) <T_n> + U_(n+K) <S^2 T_n>). */
template <typename R, int M>
__device__ __forceinline__ void slope_moments(const Mom<R, M> &Tm, const R (*s)[M + 2], R *Wo, R *Fo)
{
    constexpr int NT = M - 1; /* tangential axes */
    constexpr int NTa = NT > 0 ? NT : 1;
    /* transverse tables: E1[t] = <v_t>, E2[t][u] = <v_t v_u>, E3[r][t][u],
     * E1S[t] = <v_t S^2>, E2S[r][t] = <v_r v_t S^2>, E1S4[t] = <v_t S^4> */
    R E1[NTa], E2[NTa][NTa], E3[NTa][NTa][NTa], E1S[NTa], E2S[NTa][NTa], E1S4[NTa];
    const R P2 = tv<R, M, 0, 0, 1>(Tm), P4 = tv<R, M, 0, 0, 2>(Tm);
    if constexpr (M == 2) {
        E1[0] = tv<R, M, 1, 0, 0>(Tm);
        E2[0][0] = tv<R, M, 2, 0, 0>(Tm);
        E3[0][0][0] = tv<R, M, 3, 0, 0>(Tm);
        E1S[0] = tv<R, M, 1, 0, 1>(Tm);
        E2S[0][0] = tv<R, M, 2, 0, 1>(Tm);
        E1S4[0] = tv<R, M, 1, 0, 2>(Tm);
    } else if constexpr (M == 3) {
        E1[0] = tv<R, M, 1, 0, 0>(Tm);
        E1[1] = tv<R, M, 0, 1, 0>(Tm);
        E2[0][0] = tv<R, M, 2, 0, 0>(Tm);
        E2[0][1] = E2[1][0] = tv<R, M, 1, 1, 0>(Tm);
        E2[1][1] = tv<R, M, 0, 2, 0>(Tm);
        const R vvv = tv<R, M, 3, 0, 0>(Tm), vvw = tv<R, M, 2, 1, 0>(Tm), vww = tv<R, M, 1, 2, 0>(Tm),
                www = tv<R, M, 0, 3, 0>(Tm);
        E3[0][0][0] = vvv;
        E3[0][0][1] = E3[0][1][0] = E3[1][0][0] = vvw;
        E3[0][1][1] = E3[1][0][1] = E3[1][1][0] = vww;
        E3[1][1][1] = www;
        E1S[0] = tv<R, M, 1, 0, 1>(Tm);
        E1S[1] = tv<R, M, 0, 1, 1>(Tm);
        E2S[0][0] = tv<R, M, 2, 0, 1>(Tm);
        E2S[0][1] = E2S[1][0] = tv<R, M, 1, 1, 1>(Tm);
        E2S[1][1] = tv<R, M, 0, 2, 1>(Tm);
        E1S4[0] = tv<R, M, 1, 0, 2>(Tm);
        E1S4[1] = tv<R, M, 0, 1, 2>(Tm);
    }
    /* coefficient polynomials: q_e = s_e,E / 2; a_t = s_0,(1+t) + s_t,1 */
    const R q0 = R(0.5) * s[0][M + 1];
    R A[4], Bt[NTa][4], Cn[4];
    A[3] = q0;
    Cn[3] = q0 * P2;
    A[2] = s[0][1];
    Cn[2] = s[0][1] * P2;
    A[1] = s[0][0] + q0 * P2;
    Cn[1] = s[0][0] * P2 + q0 * P4;
    A[0] = R(0);
    Cn[0] = R(0);
#pragma unroll
    for (int r = 0; r < NT; ++r) {
        Bt[r][3] = q0 * E1[r];
        Bt[r][2] = s[0][1] * E1[r];
        Bt[r][1] = s[0][0] * E1[r] + q0 * E1S[r];
        Bt[r][0] = R(0);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const R qt = R(0.5) * s[1 + t][M + 1];
        const R at = s[0][2 + t] + s[1 + t][1];
        A[2] += qt * E1[t];
        Cn[2] += qt * E1S[t];
        A[1] += at * E1[t];
        Cn[1] += at * E1S[t];
        A[0] += s[1 + t][0] * E1[t] + qt * E1S[t];
        Cn[0] += s[1 + t][0] * E1S[t] + qt * E1S4[t];
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            A[0] += s[1 + t][2 + u] * E2[t][u];
            Cn[0] += s[1 + t][2 + u] * E2S[t][u];
        }
#pragma unroll
        for (int r = 0; r < NT; ++r) {
            Bt[r][2] += qt * E2[r][t];
            Bt[r][1] += at * E2[r][t];
            Bt[r][0] += s[1 + t][0] * E2[r][t] + qt * E2S[r][t];
#pragma unroll
            for (int u = 0; u < NT; ++u) Bt[r][0] += s[1 + t][2 + u] * E3[r][t][u];
        }
    }
    const R *U = Tm.u;
#pragma unroll
    for (int K = 0; K < 2; ++K) {
        R *o = K ? Fo : Wo;
        if (!o) continue;
        R o0 = R(0), o1 = R(0), oE = R(0);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            o0 += U[n + K] * A[n];
            o1 += U[n + 1 + K] * A[n];
            oE += U[n + 2 + K] * A[n] + U[n + K] * Cn[n];
        }
        o[0] = o0;
        o[1] = o1;
#pragma unroll
        for (int r = 0; r < NT; ++r) {
            R b = R(0);
#pragma unroll
            for (int n = 0; n < 4; ++n) b += U[n + K] * Bt[r][n];
            o[2 + r] = b;
        }
        o[M + 1] = R(0.5) * oE;
    }
}

/* Micro-slope a (coefficients on 1, u, v, w, (|u|^2+xi^2)/2) with <a psi> = r,
 * closed form through the peculiar velocity c = u - U:
 * <c_i a> = alpha_i / (2 lambda), and the two scalar moments give alpha_1, alpha_E. */
template <typename R, int M>
__device__ __forceinline__ void slope(const Prim<R, M> &P, R Ntot, R c8N, const R *r, R *a)
{
    R sv[3], Us = R(0), U2 = R(0);
    const R s0 = r[0];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        sv[i] = r[1 + i] - P.U[i] * s0;
        Us += P.U[i] * sv[i];
        U2 += P.U[i] * P.U[i];
    }
    const R sE = r[M + 1] - R(0.5) * U2 * s0 - Us;
    const R lam = P.lam;
    const R aE = c8N * lam * lam * sE - R(2) * lam * s0; /* c8N = 8 / Ntot */
    const R a1 = s0 - aE * Ntot * R(0.5) * P.i2l;
    R aU = R(0);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const R al = R(2) * lam * sv[i];
        aU += al * P.U[i];
        a[1 + i] = al - aE * P.U[i];
    }
    a[0] = a1 - aU + R(0.5) * aE * U2;
    a[M + 1] = aE;
}

/* Euler flux along face axis e of the state (P, W) */
template <typename R, int M>
__device__ __forceinline__ void euler_flux(const Prim<R, M> &P, const R *W, int e, R *F)
{
    const R ue = P.U[e];
    F[0] = W[1 + e];
#pragma unroll
    for (int i = 0; i < M; ++i) F[1 + i] = W[1 + i] * ue + (i == e ? P.p : R(0));
    F[M + 1] = ue * (W[M + 1] + P.p);
}

/* dF_e for a variation dW of the conservative variables (Jacobian-vector product) */
template <typename R, int M>
__device__ __forceinline__ void euler_dflux(const Prim<R, M> &P, const R *W, R gm1, int e, const R *dW, R *dF)
{
    const R inv = P.inv;
    R dU[3], UdU = R(0), U2 = R(0);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        dU[i] = (dW[1 + i] - P.U[i] * dW[0]) * inv;
        UdU += P.U[i] * dU[i];
        U2 += P.U[i] * P.U[i];
    }
    const R dp = gm1 * (dW[M + 1] - R(0.5) * U2 * dW[0] - P.rho * UdU);
    dF[0] = dW[1 + e];
#pragma unroll
    for (int i = 0; i < M; ++i) dF[1 + i] = dW[1 + i] * P.U[e] + W[1 + i] * dU[e] + (i == e ? dp : R(0));
    dF[M + 1] = dU[e] * (W[M + 1] + P.p) + P.U[e] * (dW[M + 1] + dp);
}

/* Flux constants, precomputed on the host in both precisions so that an
 * FP32 kernel issues no FP64 instruction for them (fill with fill_flux). */
struct FluxParams {
    double gamma, c1, c2;
    double gm1, Ntot, c8N; /* gamma - 1, 2 / (gamma - 1), 8 / Ntot */
    double mu;             /* dynamic viscosity (Navier-Stokes flux only) */
    float fgm1, fNtot, fc8N, fc1, fc2, fmu;
};

/* the constant in the precision R */
template <typename R> __host__ __device__ __forceinline__ R pick(double d, float f)
{
    if constexpr (sizeof(R) == sizeof(float)) return f;
    else return d;
}

inline void fill_flux(FluxParams &fp, double gamma, double c1, double c2)
{
    fp.gamma = gamma;
    fp.c1 = c1;
    fp.c2 = c2;
    fp.gm1 = gamma - 1.0;
    fp.Ntot = 2.0 / (gamma - 1.0);
    fp.c8N = 8.0 / fp.Ntot;
    fp.fgm1 = (float)fp.gm1;
    fp.fNtot = (float)fp.Ntot;
    fp.fc8N = (float)fp.c8N;
    fp.fc1 = (float)c1;
    fp.fc2 = (float)c2;
    fp.fmu = (float)fp.mu;
}

/* Returns false (and leaves outputs untouched) when a state is not admissible.
 * NS = false: the Euler flux (physical collision time 0 in the Chapman-Enskog
 * terms).  NS = true: the Navier-Stokes flux with Prandtl number 1, physical
 * collision time tau = mu / p0 of the interface equilibrium, added to the
 * numerical one in the relaxation factor. */
template <typename R, int M, bool NS = false>
__device__ __forceinline__ bool gks_point(const FluxParams &fp, R dt, const R *Wl, const R *Wr, const R (*dWl)[M + 2],
                                          const R (*dWr)[M + 2], R *F, R *Ft, R *Wh)
{
    constexpr int NV = M + 2;
    const R gm1 = pick<R>(fp.gm1, fp.fgm1);
    const R Ntot = pick<R>(fp.Ntot, fp.fNtot);
    const R c8N = pick<R>(fp.c8N, fp.fc8N);
    const R K = Ntot - R(M);
    /* The two initial Maxwellians' part: the equilibrium state W0 and its
     * flux Fk from the kinetic collision of the two half streams, and the
     * density-weighted slope moments of the two sides, WTs = rho_l <psi T_l>_l
     * + rho_r <psi T_r>_r and FTs the same with u.  The FP32 Euler flux takes
     * both sides at once on left/right lane pairs (packed two-lane
     * instructions); the Navier-Stokes terms below need each side apart. */
    R W0[NV], Fk[NV], WTs[NV], FTs[NV], pl, pr;
    Prim<R, M> Pl, Pr;
    Mom<R, M> Tl, Tr;
    if constexpr (std::is_same_v<R, float> && !NS) {
        Prim<LR, M> Q;
        {
            LR Wq[NV];
#pragma unroll
            for (int b = 0; b < NV; ++b) Wq[b] = LR(Wl[b], Wr[b]);
            if (!to_prim<LR, M>(Wq, LR(gm1), Q)) return false;
        }
        pl = Q.p.l();
        pr = Q.p.r();
        Mom<LR, M> T;
        half_moments<LR, 7>(Q.U[0], Q.lam, Q.i2l, LR(1.f, -1.f), T.u);
        tangential_and_internal<LR, M>(Q, LR(K), T);
        {
            LR e = T.xi[1];
            if constexpr (M >= 2) e += T.v[2];
            if constexpr (M >= 3) e += T.w[2];
            const LR ru0 = Q.rho * T.u[0], ru1 = Q.rho * T.u[1];
            W0[0] = ru0.sum();
            W0[1] = ru1.sum();
            Fk[0] = W0[1];
            Fk[1] = LR(Q.rho * T.u[2]).sum();
#pragma unroll
            for (int i = 1; i < M; ++i) {
                W0[1 + i] = LR(ru0 * Q.U[i]).sum();
                Fk[1 + i] = LR(ru1 * Q.U[i]).sum();
            }
            W0[M + 1] = R(0.5) * LR(Q.rho * (T.u[2] + T.u[0] * e)).sum();
            Fk[M + 1] = R(0.5) * LR(Q.rho * (T.u[3] + T.u[1] * e)).sum();
        }
        LR sq[M][NV];
#pragma unroll
        for (int e = 0; e < M; ++e) {
            LR rq[NV];
#pragma unroll
            for (int b = 0; b < NV; ++b) rq[b] = LR(dWl[e][b], dWr[e][b]) * Q.inv;
            slope<LR, M>(Q, LR(Ntot), LR(c8N), rq, sq[e]);
        }
        LR WT[NV], FT[NV];
        slope_moments<LR, M>(T, sq, WT, FT);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            WTs[b] = LR(Q.rho * WT[b]).sum();
            FTs[b] = LR(Q.rho * FT[b]).sum();
        }
    } else {
        if (!to_prim<R, M>(Wl, gm1, Pl) || !to_prim<R, M>(Wr, gm1, Pr)) return false;
        pl = Pl.p;
        pr = Pr.p;
        half_moments<R, 7>(Pl.U[0], Pl.lam, Pl.i2l, R(1), Tl.u);
        half_moments<R, 7>(Pr.U[0], Pr.lam, Pr.i2l, R(-1), Tr.u);
        tangential_and_internal<R, M>(Pl, K, Tl);
        tangential_and_internal<R, M>(Pr, K, Tr);
        R el = Tl.xi[1], er = Tr.xi[1];
        if constexpr (M >= 2) { el += Tl.v[2]; er += Tr.v[2]; }
        if constexpr (M >= 3) { el += Tl.w[2]; er += Tr.w[2]; }
        W0[0] = Pl.rho * Tl.u[0] + Pr.rho * Tr.u[0];
        W0[1] = Pl.rho * Tl.u[1] + Pr.rho * Tr.u[1];
        Fk[0] = W0[1];
        Fk[1] = Pl.rho * Tl.u[2] + Pr.rho * Tr.u[2];
#pragma unroll
        for (int i = 1; i < M; ++i) {
            W0[1 + i] = Pl.rho * Tl.u[0] * Pl.U[i] + Pr.rho * Tr.u[0] * Pr.U[i];
            Fk[1 + i] = Pl.rho * Tl.u[1] * Pl.U[i] + Pr.rho * Tr.u[1] * Pr.U[i];
        }
        W0[M + 1] = R(0.5) * (Pl.rho * (Tl.u[2] + Tl.u[0] * el) + Pr.rho * (Tr.u[2] + Tr.u[0] * er));
        Fk[M + 1] = R(0.5) * (Pl.rho * (Tl.u[3] + Tl.u[1] * el) + Pr.rho * (Tr.u[3] + Tr.u[1] * er));
        R sl[M][NV], sr[M][NV];
        const R il = Pl.inv, ir = Pr.inv;
#pragma unroll
        for (int e = 0; e < M; ++e) {
            R rl[NV], rr[NV];
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                rl[b] = dWl[e][b] * il;
                rr[b] = dWr[e][b] * ir;
            }
            slope<R, M>(Pl, Ntot, c8N, rl, sl[e]);
            slope<R, M>(Pr, Ntot, c8N, rr, sr[e]);
        }
        R FTl[NV], FTr[NV], WTl[NV], WTr[NV];
        slope_moments<R, M>(Tl, sl, WTl, FTl);
        slope_moments<R, M>(Tr, sr, WTr, FTr);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            WTs[b] = Pl.rho * WTl[b] + Pr.rho * WTr[b];
            FTs[b] = Pl.rho * FTl[b] + Pr.rho * FTr[b];
        }
    }

    /* equilibrium state */
    Prim<R, M> P0;
    Mom<R, M> T0;
    if (!to_prim<R, M>(W0, gm1, P0)) return false;
    full_moments<R, 7>(P0.U[0], P0.i2l, T0.u);
    tangential_and_internal<R, M>(P0, K, T0);

    /* micro-slopes of the equilibrium along every face axis */
    R s0[M][NV], dW0[M][NV];
    {
        const R i0 = P0.inv;
#pragma unroll
        for (int e = 0; e < M; ++e) {
            R r0[NV];
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                dW0[e][b] = R(0.5) * (dWl[e][b] + dWr[e][b]);
                r0[b] = dW0[e][b] * i0;
            }
            slope<R, M>(P0, Ntot, c8N, r0, s0[e]);
        }
    }
    /* dW0/dt = -sum_e dF_e/dx_e, dF_n/dt, Euler flux of W0 */
    R W0t[NV], FA0[NV], F0[NV];
    {
#pragma unroll
        for (int b = 0; b < NV; ++b) W0t[b] = R(0);
#pragma unroll
        for (int e = 0; e < M; ++e) {
            R d[NV];
            euler_dflux<R, M>(P0, W0, gm1, e, dW0[e], d);
#pragma unroll
            for (int b = 0; b < NV; ++b) W0t[b] -= d[b];
        }
        euler_dflux<R, M>(P0, W0, gm1, 0, W0t, FA0);
        euler_flux<R, M>(P0, W0, 0, F0);
    }
    /* moments carrying the equilibrium's spatial slopes */
    R FT0[NV];
    slope_moments<R, M>(T0, s0, nullptr, FT0);

    /* collision times and time integrals */
    R tn = pick<R>(fp.c1, fp.fc1) * dt + pick<R>(fp.c2, fp.fc2) * RT<R>::abs_(pl - pr) / (pl + pr) * dt;
    /* Navier-Stokes only: the time slopes A of the two initial states, each
     * from its own compatibility condition <psi (sum_e a_e u_e + A) g> = 0,
     * i.e. the Euler time derivative of that side's state; their half-space
     * moments carry the physical collision time tau */
    R tau = R(0), FA[NV], WA[NV];
    if constexpr (NS) {
        tau = pick<R>(fp.mu, fp.fmu) / P0.p;
        tn += tau;
        R Wlt[NV], Wrt[NV];
#pragma unroll
        for (int b = 0; b < NV; ++b) Wlt[b] = Wrt[b] = FA[b] = WA[b] = R(0);
#pragma unroll
        for (int e = 0; e < M; ++e) {
            R d[NV];
            euler_dflux<R, M>(Pl, Wl, gm1, e, dWl[e], d);
#pragma unroll
            for (int b = 0; b < NV; ++b) Wlt[b] -= d[b];
            euler_dflux<R, M>(Pr, Wr, gm1, e, dWr[e], d);
#pragma unroll
            for (int b = 0; b < NV; ++b) Wrt[b] -= d[b];
        }
        R Al[NV], Ar[NV];
        {
            const R il = Pl.inv, ir = Pr.inv;
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                Wlt[b] *= il;
                Wrt[b] *= ir;
            }
        }
        slope<R, M>(Pl, Ntot, c8N, Wlt, Al);
        slope<R, M>(Pr, Ntot, c8N, Wrt, Ar);
        R fl[NV], fr[NV], hl[NV], hr[NV];
#pragma unroll
        for (int b = 0; b < NV; ++b) fl[b] = fr[b] = hl[b] = hr[b] = R(0);
        psi_mom_s<R, M, 1, 0, 0>(Tl, Al, fl);
        psi_mom_s<R, M, 1, 0, 0>(Tr, Ar, fr);
        psi_mom_s<R, M, 0, 0, 0>(Tl, Al, hl);
        psi_mom_s<R, M, 0, 0, 0>(Tr, Ar, hr);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            FA[b] = Pl.rho * fl[b] + Pr.rho * fr[b];
            WA[b] = Pl.rho * hl[b] + Pr.rho * hr[b];
        }
    }
    const R hdt = R(0.5) * dt;
    R eh = R(0), e1 = R(0);
    if (tn > R(0)) {
        eh = RT<R>::exp_(-hdt / tn);
        e1 = eh * eh; /* exp(-dt/tn) */
    }
    const R ie_h = tn * (R(1) - eh), ie_1 = tn * (R(1) - e1);
    const R ite_h = tn * tn - tn * (hdt + tn) * eh, ite_1 = tn * tn - tn * (dt + tn) * e1;
    const R idt = R(1) / dt;
    const R cF1 = (R(4) * ie_h - ie_1) * idt, cF2 = (R(4) * ite_h - ite_1) * idt;
    const R cT1 = R(4) * (ie_1 - R(2) * ie_h) * idt * idt, cT2 = R(4) * (ite_1 - R(2) * ite_h) * idt * idt;
#pragma unroll
    for (int b = 0; b < NV; ++b) {
        const R dk = Fk[b] - F0[b];
        const R dT = P0.rho * FT0[b] - FTs[b];
        F[b] = F0[b] + cF1 * dk + cF2 * dT;
        Ft[b] = FA0[b] + cT1 * dk + cT2 * dT;
        Wh[b] = W0[b] + hdt * (R(1) - eh) * W0t[b] - hdt * eh * WTs[b];
        if constexpr (NS) {
            /* the tau terms of the time integrals: with V = <u psi (T0 + A0) g0>
             * (the equilibrium's viscous part) and D = V - (left + right
             * half-space <u psi (T + A) g>), F gains tau (cF1 D - V) and Ft
             * gains tau cT1 D; the interface state gains -tau e (the two
             * sides' half-space <psi (T + A) g>), since <psi (T0 + A0) g0> = 0 */
            const R V = P0.rho * FT0[b] + FA0[b];
            const R D = V - FTs[b] - FA[b];
            F[b] += tau * (cF1 * D - V);
            Ft[b] += tau * cT1 * D;
            Wh[b] -= tau * eh * (WTs[b] + WA[b]);
        }
    }
    return true;
}

} // namespace gks
