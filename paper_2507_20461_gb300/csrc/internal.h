/* Internal host-side declarations of libgenogks (not part of the C ABI). */
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdio>

#include "../../include/genogks.h"
#include "kernels.cuh"

struct gks_ctx {
    int dim, nv, ng, precision, order;
    int n[3];
    double h, gamma;
    gks_opts_t opts;
    gks::KP kp;
    cudaStream_t stream;
    /* state and stage buffers (FP64) */
    double *W, *G, *Ws, *Gs, *Acc;
    /* mixed precision, 2D/3D: FP32 shadows of the step's input state (s0) and
     * of the stage-1 output (s1) that the reconstruction and flux read */
    gks::Shadow s0, s1;
    int shadows;
    /* 2D mixed precision with the fused stage kernel (opts.stage_kernels == 1) */
    int fused;
    /* mixed precision: the steps keep the gradients in s0.g only; G is
     * filled from it when the state is read */
    int g_stale;
    /* device scalars */
    double *dt;
    float *updc; /* mixed precision: the stage constants of the current dt (UpdC, 10 floats) */
    unsigned long long *smax;
    int *status;
    /* reconstruction coefficients (multi-D) and face quantities, in the
     * reconstruction precision */
    void *B;
    void *ff;
    size_t B_elems, ff_elems;
    /* all of the above live in one workspace */
    void *ws;
    size_t ws_bytes;
    int own_ws;
    /* lazily allocated staging buffer for host-side outputs */
    double *stage_out;
    size_t stage_bytes;
    /* kernel profiler: event pairs around launches while enabled */
    int prof_on;
    int prof_n;
    cudaEvent_t *prof_ev;  /* 2 * kProfCap events */
    int *prof_cls;
    long prof_launches[8];
    double prof_ms[8];
    char err[256];
};

namespace gks {

constexpr int kProfCap = 4096;

/* flush recorded event pairs into the per-class totals (synchronises) */
inline void prof_flush(gks_ctx *c)
{
    for (int i = 0; i < c->prof_n; ++i) {
        float ms = 0.f;
        cudaEventSynchronize(c->prof_ev[2 * i + 1]);
        cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]);
        c->prof_ms[c->prof_cls[i]] += ms;
        c->prof_launches[c->prof_cls[i]] += 1;
    }
    c->prof_n = 0;
}

/* brackets one kernel launch of class cls with events on the handle's stream */
struct ProfScope {
    gks_ctx *c;
    int slot;
    ProfScope(gks_ctx *cc, int cls) : c(cc), slot(-1)
    {
        if (!c->prof_on) return;
        if (c->prof_n == kProfCap) prof_flush(c);
        slot = c->prof_n++;
        c->prof_cls[slot] = cls;
        cudaEventRecord(c->prof_ev[2 * slot], c->stream);
    }
    ~ProfScope()
    {
        if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
    }
};

/* per-dimension launchers (k1d.cu, k2d.cu, k3d.cu) */
/* input: 0 = the step's input state (W, G), 1 = the stage-1 output (W*, G*) */
template <int M> cudaError_t launch_states(gks_ctx *c, int input, double *fs_dev);
/* sums: the step path (FP32 multi-D: per-face Gauss sums, read by the update);
 * false: per-Gauss-point fluxes (gks_flux) */
template <int M> cudaError_t launch_flux(gks_ctx *c, int input, bool sums);
template <int M> cudaError_t launch_update(gks_ctx *c, int stage);
template <int M> cudaError_t launch_wavespeed(gks_ctx *c, double cfl);
template <int M> cudaError_t launch_shadow(gks_ctx *c);
/* 1D non-compact schemes (order 5 or 6): face states / HLLC fluxes of the
 * stage input (input 0: W, 1: Ws), and one classical RK4 step */
cudaError_t nc_launch_faces(gks_ctx *c, int input, double *fs_dev, bool flux);
cudaError_t nc_launch_step(gks_ctx *c);
/* 2D mixed precision: one stage (1 or 2) as one fused kernel */
cudaError_t launch_fused2d(gks_ctx *c, int stage);

inline int ngauss(int m) { return m == 1 ? 1 : (m == 2 ? 2 : 4); }
inline int ncubic(int m) { return m == 2 ? GENO_NC2 : (m == 3 ? GENO_NC3 : 0); }

constexpr int kBlock = 128;
inline unsigned blocks_for(long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

} // namespace gks
