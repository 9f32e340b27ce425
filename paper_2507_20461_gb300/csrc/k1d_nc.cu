/* 1D non-compact GENO schemes (Sec. 4.1): 5th order (the 5th-order WENO
 * stencils) and 6th order (six-cell stencil symmetric about the face), with
 * the HLLC flux and classical four-stage RK4 (Sec. 2).  FP64.
 *
 * Face f (0..n) lies between cells f-1 and f.  The left state is
 * reconstructed in cell f-1 from the averages at offsets -2..3; the right
 * state in cell f from the mirrored stencil, so both use the same map
 * (nc5_left / nc6_left, generated in exact arithmetic). */
#include "internal.h"

namespace gks {

namespace {

/* GENO blend of the left value from averages relative to the reconstruction
 * cell (u[2] = 0): chi qH + (1 - chi) sum_k omega_k p_k, with IS^H = max,
 * IS^L = min, IS^tau = |(IS_first + IS_last)/2 - IS_2|, r = 2, and d = C0 on the
 * sub-stencil centred on the cell (index 1). */
template <int ORDER>
__device__ __forceinline__ double nc_value(const KP &P, const double *u)
{
    constexpr int K = (ORDER == 5) ? 3 : 4;
    double qH, p[K], IS[K];
    if constexpr (ORDER == 5) nc5_left<double>(u, qH, p, IS);
    else nc6_left<double>(u, qH, p, IS);
    if (P.limiter == 1) return qH;
    double ISH = IS[0], ISL = IS[0];
#pragma unroll
    for (int k = 1; k < K; ++k) {
        ISH = fmax(ISH, IS[k]);
        ISL = fmin(ISL, IS[k]);
    }
    /* outer-left, outer-right and centred sub-stencils (6th order: S_1, S_4,
     * S_2; S_1..S_3 would never see the stencil's last cell) */
    const double ISt = fabs(0.5 * (IS[0] + IS[K - 1]) - IS[1]);
    const double chi = chi_of<double>(P, ISt, ISH, ISL, 2);
    double ws = 0.0, ql = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double w = ((k == 1) ? P.C0 : 1.0) / ((IS[k] + P.eps) * (IS[k] + P.eps));
        ws += w;
        ql += w * p[k];
    }
    return chi * qH + (1.0 - chi) * (ql / ws);
}

/* HLLC flux (Toro) with the Davis wave-speed bounds; false if a state is
 * not admissible */
__device__ __forceinline__ bool hllc(double gamma, const double *L, const double *R, double *F)
{
    const double rl = L[0], ul = L[1] / rl, pl = (gamma - 1.0) * (L[2] - 0.5 * rl * ul * ul);
    const double rr = R[0], ur = R[1] / rr, pr = (gamma - 1.0) * (R[2] - 0.5 * rr * ur * ur);
    if (!(rl > 0.0) || !(rr > 0.0) || !(pl > 0.0) || !(pr > 0.0)) return false;
    const double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    const double SL = fmin(ul - cl, ur - cr), SR = fmax(ul + cl, ur + cr);
    const double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur));
    if (0.0 <= SL) {
        F[0] = rl * ul;
        F[1] = rl * ul * ul + pl;
        F[2] = ul * (L[2] + pl);
    } else if (0.0 <= Ss) {
        const double k = rl * (SL - ul) / (SL - Ss);
        const double Us[3] = {k, k * Ss, k * (L[2] / rl + (Ss - ul) * (Ss + pl / (rl * (SL - ul))))};
        const double FL[3] = {rl * ul, rl * ul * ul + pl, ul * (L[2] + pl)};
#pragma unroll
        for (int v = 0; v < 3; ++v) F[v] = FL[v] + SL * (Us[v] - L[v]);
    } else if (0.0 <= SR) {
        const double k = rr * (SR - ur) / (SR - Ss);
        const double Us[3] = {k, k * Ss, k * (R[2] / rr + (Ss - ur) * (Ss + pr / (rr * (SR - ur))))};
        const double FR[3] = {rr * ur, rr * ur * ur + pr, ur * (R[2] + pr)};
#pragma unroll
        for (int v = 0; v < 3; ++v) F[v] = FR[v] + SR * (Us[v] - R[v]);
    } else {
        F[0] = rr * ur;
        F[1] = rr * ur * ur + pr;
        F[2] = ur * (R[2] + pr);
    }
    return true;
}

/* FLUX = false: face states fs[side][v][c][face] (c = 0 value, 1 derivative,
 * which this scheme does not reconstruct: 0).  FLUX = true: ff[q][v][face]
 * with q = 0 the HLLC flux and q = 1, 2 zero (no time derivative, no
 * interface state). */
template <int ORDER, bool FLUX>
__global__ void __launch_bounds__(128) nc_face_kernel(KP P, const double *__restrict__ W, double *__restrict__ fs,
                                                      double *__restrict__ ff, int *__restrict__ status)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > P.n[0]) return;
    const long nf = P.nftot;
    double st[2][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        double w[6][3];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            int flip[3];
            const int cell = side ? f + 2 - i : f - 3 + i;
            const long c = cell_lin<1>(P, cell, 0, 0, flip);
#pragma unroll
            for (int v = 0; v < 3; ++v) w[i][v] = (double)ghost_sign<1>(P, flip, v) * W[v * P.ncell + c];
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            double u[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) u[i] = w[i][v] - w[2][v];
            st[side][v] = w[2][v] + nc_value<ORDER>(P, u);
        }
        if (!admissible<double, 1>(st[side], w[2], P.fp.gm1, P.adm)) {
#pragma unroll
            for (int v = 0; v < 3; ++v) st[side][v] = w[2][v];
        }
    }
    if (!FLUX) {
#pragma unroll
        for (int side = 0; side < 2; ++side)
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                fs[((long)(side * 3 + v) * 2 + 0) * nf + f] = st[side][v];
                fs[((long)(side * 3 + v) * 2 + 1) * nf + f] = 0.0;
            }
        return;
    }
    double F[3];
    if (!hllc(P.gamma, st[0], st[1], F)) {
        atomicOr(status, ST_FLUX);
        F[0] = F[1] = F[2] = 0.0;
    }
    /* walls are at rest and adiabatic: no mass or energy flux */
    if ((f == 0 && P.bcs[0][0] >= 2) || (f == P.n[0] && P.bcs[0][1] >= 2)) F[0] = F[2] = 0.0;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        ff[(long)(0 * 3 + v) * nf + f] = F[v];
        ff[(long)(1 * 3 + v) * nf + f] = 0.0;
        ff[(long)(2 * 3 + v) * nf + f] = 0.0;
    }
}

/* classical RK4 with L(U)_j = -(F_{j+1/2} - F_{j-1/2}) / h:
 *   stage 1: Acc = L(U0),   U1 = U0 + dt/2 L(U0)
 *   stage 2: Acc += 2 L(U1), U2 = U0 + dt/2 L(U1)
 *   stage 3: Acc += 2 L(U2), U3 = U0 + dt L(U2)
 *   stage 4: U0 += dt/6 (Acc + L(U3)) */
__global__ void __launch_bounds__(256) nc_rk_kernel(KP P, int stage, const double *__restrict__ dtp,
                                                    const double *__restrict__ ff, double *__restrict__ W0,
                                                    double *__restrict__ Ws, double *__restrict__ Acc,
                                                    int *__restrict__ status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n[0]) return;
    const double dt = dtp[0];
    const long nf = P.nftot, nc = P.ncell;
    double out[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const double L = -(ff[(long)v * nf + j + 1] - ff[(long)v * nf + j]) * P.ih;
        const long i = (long)v * nc + j;
        if (stage == 1) {
            Acc[i] = L;
            out[v] = Ws[i] = W0[i] + 0.5 * dt * L;
        } else if (stage == 2) {
            Acc[i] += 2.0 * L;
            out[v] = Ws[i] = W0[i] + 0.5 * dt * L;
        } else if (stage == 3) {
            Acc[i] += 2.0 * L;
            out[v] = Ws[i] = W0[i] + dt * L;
        } else {
            out[v] = W0[i] = W0[i] + dt / 6.0 * (Acc[i] + L);
        }
    }
    const double p = P.fp.gm1 * (out[2] - 0.5 * out[1] * out[1] / out[0]);
    int st = 0;
    if (!(out[0] > 0.0)) st |= ST_RHO;
    if (!(p > 0.0)) st |= ST_P;
    if (!isfinite(p) || !isfinite(out[0])) st |= ST_NAN;
    if (st) atomicOr(status, st);
}

} // namespace

cudaError_t nc_launch_faces(gks_ctx *c, int input, double *fs_dev, bool flux)
{
    const KP &P = c->kp;
    const double *W = input ? c->Ws : c->W;
    const unsigned nb = blocks_for(P.n[0] + 1);
    double *ff = (double *)c->ff;
    ProfScope ps(c, GKS_KC_FACE);
    if (c->order == 5) {
        if (flux) nc_face_kernel<5, true><<<nb, kBlock, 0, c->stream>>>(P, W, nullptr, ff, c->status);
        else nc_face_kernel<5, false><<<nb, kBlock, 0, c->stream>>>(P, W, fs_dev, nullptr, c->status);
    } else {
        if (flux) nc_face_kernel<6, true><<<nb, kBlock, 0, c->stream>>>(P, W, nullptr, ff, c->status);
        else nc_face_kernel<6, false><<<nb, kBlock, 0, c->stream>>>(P, W, fs_dev, nullptr, c->status);
    }
    return cudaGetLastError();
}

cudaError_t nc_launch_step(gks_ctx *c)
{
    for (int stage = 1; stage <= 4; ++stage) {
        cudaError_t e = nc_launch_faces(c, stage > 1, nullptr, true);
        if (e != cudaSuccess) return e;
        ProfScope ps(c, GKS_KC_UPDATE);
        nc_rk_kernel<<<blocks_for(c->kp.n[0], 256), 256, 0, c->stream>>>(c->kp, stage, c->dt, (const double *)c->ff, c->W,
                                                                         c->Ws, c->Acc, c->status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace gks
