/* Launch wrappers of the stage kernels for one dimension M; included by the
 * per-dimension translation units k1d.cu, k2d.cu, k3d.cu. */
#pragma once
#include "internal.h"

namespace gks {

template <typename R> Src<R> stage_src(gks_ctx *c, int input);
template <> inline Src<double> stage_src<double>(gks_ctx *c, int input)
{
    return input ? Src<double>{c->Ws, c->Gs} : Src<double>{c->W, c->G};
}
template <> inline Src<float> stage_src<float>(gks_ctx *c, int input)
{
    const Shadow &s = input ? c->s1 : c->s0;
    return Src<float>{s.hi, s.lo, s.g};
}

/* flux = false: interface states into fs_dev; flux = true: fluxes per Gauss
 * point into c->ff, or (sums, FP32 multi-D step path) per-face sums over the
 * Gauss points */
template <typename R, int M>
static cudaError_t flux_impl(gks_ctx *c, int input, double *fs_dev, bool flux, bool sums = false)
{
    const KP &P = c->kp;
    R *ff = (R *)c->ff;
    const double *W = input ? c->Ws : c->W;
    const double *G = input ? c->Gs : c->G;
    if constexpr (M == 1) {
        if (c->order != 8) return nc_launch_faces(c, input, fs_dev, flux);
        const unsigned nb = blocks_for(P.n[0] + 1);
        ProfScope ps(c, GKS_KC_FACE);
        if (flux && P.fp.mu > 0.0) face1d_kernel<R, true, true><<<nb, kBlock, 0, c->stream>>>(P, W, G, c->dt, nullptr, ff, c->status);
        else if (flux) face1d_kernel<R, true><<<nb, kBlock, 0, c->stream>>>(P, W, G, c->dt, nullptr, ff, c->status);
        else face1d_kernel<R, false><<<nb, kBlock, 0, c->stream>>>(P, W, G, c->dt, fs_dev, nullptr, c->status);
    } else {
        constexpr int NG = (M == 2) ? 2 : 4;
        R *B = (R *)c->B;
        const Src<R> src = stage_src<R>(c, input);
        {
            ProfScope ps(c, GKS_KC_RECON);
            cell_poly_kernel<R, M><<<blocks_for(P.next), kBlock, 0, c->stream>>>(P, src, B);
        }
        for (int d = 0; d < M; ++d) {
            const unsigned nb = blocks_for(P.nface[d] * NG);
            ProfScope ps(c, GKS_KC_FACE);
#define GKS_FACE(D)                                                                                           \
    if (d == D) {                                                                                             \
        if constexpr (sizeof(R) == sizeof(float)) {                                                           \
            if (flux && sums && P.fp.mu > 0.0)                                                                \
                { face_flux_prepare<R, M, D, true, true, true>(); face_flux_kernel<R, M, D, true, true, true><<<nb, kBlock, 0, c->stream>>>(P, src, B, c->dt, nullptr, ff, c->status); } \
            else if (flux && sums)                                                                            \
                { face_flux_prepare<R, M, D, true, false, true>(); face_flux_kernel<R, M, D, true, false, true><<<nb, kBlock, 0, c->stream>>>(P, src, B, c->dt, nullptr, ff, c->status); } \
        }                                                                                                     \
        if (flux && !(sizeof(R) == sizeof(float) && sums)) {                                                 \
            if (P.fp.mu > 0.0) { face_flux_prepare<R, M, D, true, true>(); face_flux_kernel<R, M, D, true, true><<<nb, kBlock, 0, c->stream>>>(P, src, B, c->dt, nullptr, ff, c->status); } \
            else { face_flux_prepare<R, M, D, true>(); face_flux_kernel<R, M, D, true><<<nb, kBlock, 0, c->stream>>>(P, src, B, c->dt, nullptr, ff, c->status); } \
        }                                                                                                     \
        if (!flux) { face_flux_prepare<R, M, D, false>(); face_flux_kernel<R, M, D, false><<<nb, kBlock, 0, c->stream>>>(P, src, B, c->dt, fs_dev, nullptr, c->status); } \
    }
            GKS_FACE(0)
            GKS_FACE(1)
            if constexpr (M == 3) { GKS_FACE(2) }
#undef GKS_FACE
        }
    }
    return cudaGetLastError();
}

template <int M> cudaError_t launch_states(gks_ctx *c, int input, double *fs_dev)
{
    return c->precision ? flux_impl<float, M>(c, input, fs_dev, false) : flux_impl<double, M>(c, input, fs_dev, false);
}

template <int M> cudaError_t launch_flux(gks_ctx *c, int input, bool sums)
{
    return c->precision ? flux_impl<float, M>(c, input, nullptr, true, sums)
                        : flux_impl<double, M>(c, input, nullptr, true, sums);
}

template <typename R, int M> static cudaError_t update_impl(gks_ctx *c, int stage)
{
    const KP &P = c->kp;
    const unsigned nb = blocks_for(P.ncell, 256);
    const R *ff = (const R *)c->ff;
    ProfScope ps(c, GKS_KC_UPDATE);
    if (stage == 1)
        update_kernel<R, M, 1><<<nb, 256, 0, c->stream>>>(P, ff, c->dt, c->W, c->G, c->Ws, c->Gs, c->Acc, c->s0, c->s1,
                                                          c->status, c->updc);
    else
        update_kernel<R, M, 2><<<nb, 256, 0, c->stream>>>(P, ff, c->dt, c->W, c->G, c->Ws, c->Gs, c->Acc, c->s0, c->s1,
                                                          c->status, c->updc);
    return cudaGetLastError();
}

template <int M> cudaError_t launch_update(gks_ctx *c, int stage)
{
    return c->precision ? update_impl<float, M>(c, stage) : update_impl<double, M>(c, stage);
}

template <int M> cudaError_t launch_wavespeed(gks_ctx *c, double cfl)
{
    cudaError_t e = cudaMemsetAsync(c->smax, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    long want = (c->kp.ncell + 255) / 256;
    long cap = (long)nsm * 8;
    const unsigned nb = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    ProfScope ps(c, GKS_KC_DT);
    if (c->shadows) wavespeed_kernel<M, float><<<nb, 256, 0, c->stream>>>(c->kp, c->s0.hi, c->smax);
    else wavespeed_kernel<M, double><<<nb, 256, 0, c->stream>>>(c->kp, c->W, c->smax);
    if (cfl > 0.0) {
        /* viscous limit cfl h^2 / (2 (m - 1) nu): passed as the factor
         * 2 (m - 1) mu / h that turns max(1 / rho) into the rate cfl h / dt */
        const double visc = c->kp.fp.mu > 0.0 ? 2.0 * (M > 1 ? M - 1 : 1) * c->kp.fp.mu / c->h : 0.0;
        dt_from_speed_kernel<<<1, 1, 0, c->stream>>>(c->smax, cfl * c->h, visc, c->dt, c->shadows ? c->updc : nullptr,
                                                     updc_cw(c->kp, M));
    }
    return cudaGetLastError();
}

template <int M> cudaError_t launch_shadow(gks_ctx *c)
{
    if (!c->shadows) return cudaSuccess;
    const long want = (c->kp.ncell + 255) / 256;
    shadow_kernel<M><<<(unsigned)(want < 4096 ? (want > 0 ? want : 1) : 4096), 256, 0, c->stream>>>(c->kp, c->W, c->G,
                                                                                                   c->s0);
    return cudaGetLastError();
}

#define GKS_INSTANTIATE(M)                                                                                \
    template cudaError_t launch_states<M>(gks_ctx *, int, double *);                                      \
    template cudaError_t launch_flux<M>(gks_ctx *, int, bool);                                            \
    template cudaError_t launch_update<M>(gks_ctx *, int);                                                \
    template cudaError_t launch_wavespeed<M>(gks_ctx *, double);                                          \
    template cudaError_t launch_shadow<M>(gks_ctx *);

} // namespace gks
