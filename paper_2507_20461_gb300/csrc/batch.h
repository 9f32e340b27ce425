/* Batched 2D mode: many independent grids of uneven sizes advanced by
 * persistent kernels over tile work lists, one step captured in a CUDA graph.
 * Internal declarations (the C ABI is in include/genogks.h). */
#pragma once
#include "internal.h"

namespace gks {

/* per-grid device descriptor: parameters and buffer bases */
struct GridDesc {
    KP P;
    double *W, *G, *Ws, *Gs, *Acc;
    void *B, *ff;
    Shadow s0, s1; /* FP32 shadows (mixed precision only) */
};

/* a contiguous range [begin, end) of one kernel's index space on one grid;
 * kind = face direction for the flux kernel.  For the fused stage kernel a
 * tile is one strip: columns kind .. kind + strip width - 1, rows begin ..
 * end - 1. */
struct Tile {
    int grid;
    int kind;
    long begin, end;
};

enum BatchKernel { BK_SPEED = 0, BK_POLY = 1, BK_FLUX = 2, BK_UPDATE = 3, BK_STAGE = 4, BK_COUNT = 5 };

/* strip width of the fused stage kernel (columns per tile) */
constexpr int kStageStrip = 62;

struct LaunchShape {
    int block;   /* threads per block */
    long tile;   /* items per tile */
    int blocks;  /* persistent blocks (grid size) */
};

struct BatchLaunch {
    const GridDesc *gd;         /* device */
    const Tile *tiles;
    int ntiles;
    double *dt;                 /* per grid */
    unsigned long long *smax;   /* per grid */
    int *status;                /* per grid: status[g] */
    const KP *common;           /* host: the scheme constants every grid shares */
    int *queue;                 /* device: work counters of the fused stage kernel (one per stage) */
};

template <typename R> cudaError_t batch_speed(const BatchLaunch &L, const LaunchShape &S, cudaStream_t st);
template <typename R> cudaError_t batch_poly(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st);
template <typename R> cudaError_t batch_flux(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st);
template <typename R> cudaError_t batch_update(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st);
/* mixed precision: one stage of every grid as one persistent fused kernel
 * over a strip list (a work counter hands out the strips) */
cudaError_t batch_stage(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st);
cudaError_t batch_dt(const GridDesc *gd, int nb, double cfl, const unsigned long long *smax, double *dt, cudaStream_t st);
cudaError_t batch_shadow(const GridDesc &g, cudaStream_t st);
/* FP64 gradients of grid g from its FP32 shadow (mixed precision) */
cudaError_t batch_widen_grad(const GridDesc &g, cudaStream_t st);
int batch_occupancy(int kernel, int precision, int block);

} // namespace gks
