/* Persistent batched kernels of the 2D compact GKS: every block walks the tile
 * list (grid-stride over tiles), every thread walks the items of its tile.
 * The per-item arithmetic is the single-grid kernels' (kernels.cuh). */
#include "batch.h"
#include "fused2d.cuh"

namespace gks {

template <typename R> __device__ __forceinline__ Src<R> stage_src_of(const GridDesc &g, int stage);
template <> __device__ __forceinline__ Src<double> stage_src_of<double>(const GridDesc &g, int stage)
{
    return stage == 1 ? Src<double>{g.W, g.G} : Src<double>{g.Ws, g.Gs};
}
template <> __device__ __forceinline__ Src<float> stage_src_of<float>(const GridDesc &g, int stage)
{
    const Shadow &s = stage == 1 ? g.s0 : g.s1;
    return Src<float>{s.hi, s.lo, s.g};
}

template <typename R>
__global__ void __launch_bounds__(256) bk_speed(const GridDesc *__restrict__ gd, const Tile *__restrict__ tiles, int ntiles,
                                                unsigned long long *__restrict__ smax)
{
    __shared__ double red[8];
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile T = tiles[ti];
        const KP &P = gd[T.grid].P;
        /* the FP64 state, or its FP32 shadow in mixed precision */
        const R *W;
        if constexpr (sizeof(R) == sizeof(float)) W = gd[T.grid].s0.hi;
        else W = gd[T.grid].W;
        const R gam = R(P.gamma);
        R sr = R(0);
        for (long c = T.begin + threadIdx.x; c < T.end; c += blockDim.x) {
            const R rho = W[c];
            const R u = W[P.ncell + c] / rho, v = W[2 * P.ncell + c] / rho;
            const R p = (gam - R(1)) * (W[3 * P.ncell + c] - R(0.5) * rho * (u * u + v * v));
            sr = fmax(sr, fmax(fabs(u), fabs(v)) + sqrt(gam * p / rho));
        }
        double s = (double)sr;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
            atomicMax(&smax[T.grid], (unsigned long long)__double_as_longlong(isnan(m) ? 1e300 : m));
        }
        __syncthreads();
    }
}

__global__ void bk_dt(const GridDesc *__restrict__ gd, int nb, double cfl, const unsigned long long *__restrict__ smax,
                      double *__restrict__ dt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) dt[b] = cfl * gd[b].P.h / __longlong_as_double((long long)smax[b]);
}

template <typename R>
__global__ void __launch_bounds__(128) bk_poly(const GridDesc *__restrict__ gd, const Tile *__restrict__ tiles, int ntiles,
                                               int stage)
{
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile T = tiles[ti];
        const GridDesc &g = gd[T.grid];
        const Src<R> src = stage_src_of<R>(g, stage);
        for (long t = T.begin + threadIdx.x; t < T.end; t += blockDim.x) cell_poly_item<R, 2>(g.P, src, (R *)g.B, t);
    }
}

/* same register cap as the single-grid 2D FP32 flux (8 blocks of 128 per SM) */
template <typename R>
__global__ void __launch_bounds__(128, (flux_blocks_per_sm<R, 2, false>())) bk_flux(const GridDesc *__restrict__ gd, const Tile *__restrict__ tiles, int ntiles,
                                               int stage, const double *__restrict__ dt, int *__restrict__ status)
{
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile T = tiles[ti];
        const GridDesc &g = gd[T.grid];
        const Src<R> src = stage_src_of<R>(g, stage);
        const double dtv = dt[T.grid];
        /* FP32: per-face Gauss sums, as the single-grid step path (tiles are
         * whole 128-item groups, so every thread runs the same iterations and
         * t mod 128 is its thread index) */
        constexpr bool fsum = sizeof(R) == sizeof(float);
        if (T.kind == 0) {
            for (long t = T.begin + threadIdx.x; t < T.end; t += blockDim.x)
                face_flux_item<R, 2, 0, true, false, fsum>(g.P, src, (const R *)g.B, dtv, nullptr, (R *)g.ff, status + T.grid, t);
        } else {
            for (long t = T.begin + threadIdx.x; t < T.end; t += blockDim.x)
                face_flux_item<R, 2, 1, true, false, fsum>(g.P, src, (const R *)g.B, dtv, nullptr, (R *)g.ff, status + T.grid, t);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) bk_update(const GridDesc *__restrict__ gd, const Tile *__restrict__ tiles, int ntiles,
                                                 int stage, const double *__restrict__ dt, int *__restrict__ status)
{
    __shared__ UpdC uc;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile T = tiles[ti];
        const GridDesc &g = gd[T.grid];
        const double dtv = dt[T.grid];
        if constexpr (sizeof(R) == sizeof(float)) {
            /* the tile's grid's stage constants (the tile loop is uniform over the block) */
            __syncthreads();
            if (threadIdx.x == 0) uc = make_updc(dtv, g.P.ih / 2);
            __syncthreads();
        }
        for (long c = T.begin + threadIdx.x; c < T.end; c += blockDim.x) {
            if (stage == 1)
                update_item<R, 2, 1>(g.P, (const R *)g.ff, dtv, g.W, g.G, g.Ws, g.Gs, g.Acc, g.s0, g.s1, status + T.grid, c, uc);
            else
                update_item<R, 2, 2>(g.P, (const R *)g.ff, dtv, g.W, g.G, g.Ws, g.Gs, g.Acc, g.s0, g.s1, status + T.grid, c, uc);
        }
    }
}

/* Mixed precision: one stage of every grid in one persistent launch.  Each
 * block takes the next strip of the list from a work counter (strips ordered
 * by size, largest first) and runs the fused reconstruction -> flux ->
 * update sweep (fused2d_strip) of it, until the list is done.  The grids
 * share every scheme constant and boundary type, so the kernel takes one
 * parameter block (its geometry fields unused) as a launch parameter, and
 * per strip only the grid's geometry, state pointers and time step. */
constexpr int kStageThreads = 256, kStageMinBlocks = 2;

template <int STAGE>
__global__ void __launch_bounds__(kStageThreads, kStageMinBlocks)
    bk_stage(const KP P, const GridDesc *__restrict__ gd, const Tile *__restrict__ tiles, int ntiles,
             const double *__restrict__ dt, int *__restrict__ queue, int *__restrict__ status)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ UpdC uc;
    __shared__ int next;
    for (;;) {
        __syncthreads(); /* every thread has read `next`; the previous strip is done with uc and the rings */
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int ti = next;
        if (ti >= ntiles) break;
        const Tile T = tiles[ti];
        const GridDesc &g = gd[T.grid];
        const FusedGeo geo{g.P.n[0], g.P.n[1], g.P.ncell, g.P.ih, g.P.fh, g.P.fih};
        /* the shadows' lo and g planes follow hi at 4 and 8 planes of cells */
        const long nc = geo.nc;
        float *const h0 = g.s0.hi, *const h1 = g.s1.hi;
        const Shadow s0{h0, h0 + 4 * nc, h0 + 8 * nc}, s1{h1, h1 + 4 * nc, h1 + 8 * nc};
        fused2d_strip<STAGE, false, kStageStrip, kStageThreads>(P, geo, s0, s1, g.W, (float *)g.Acc, dt[T.grid],
                                                               status + T.grid, T.kind, (int)T.begin, (int)(T.end - T.begin),
                                                               smem, uc);
    }
}

/* the dynamic shared memory opt-in of both stage kernels, once */
cudaError_t stage_prepare()
{
    using Strip = SweepStrip<kStageStrip>;
    static const cudaError_t prep = [] {
        cudaError_t e = cudaFuncSetAttribute(bk_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Strip::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bk_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Strip::SMEM);
        for (auto k : {bk_stage<1>, bk_stage<2>})
            if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
                (void)cudaGetLastError();
        return e;
    }();
    return prep;
}

cudaError_t batch_stage(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st)
{
    using Strip = SweepStrip<kStageStrip>;
    const cudaError_t prep = stage_prepare();
    if (prep != cudaSuccess) return prep;
    if (S.block != kStageThreads) return cudaErrorInvalidConfiguration;
    if (L.ntiles < 1) return cudaSuccess;
    int *q = L.queue + (stage - 1);
    cudaError_t e = cudaMemsetAsync(q, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (stage == 1)
        bk_stage<1><<<S.blocks, kStageThreads, Strip::SMEM, st>>>(*L.common, L.gd, L.tiles, L.ntiles, L.dt, q, L.status);
    else
        bk_stage<2><<<S.blocks, kStageThreads, Strip::SMEM, st>>>(*L.common, L.gd, L.tiles, L.ntiles, L.dt, q, L.status);
    return cudaGetLastError();
}

template <typename R> cudaError_t batch_speed(const BatchLaunch &L, const LaunchShape &S, cudaStream_t st)
{
    bk_speed<R><<<S.blocks, S.block, 0, st>>>(L.gd, L.tiles, L.ntiles, L.smax);
    return cudaGetLastError();
}
template <typename R> cudaError_t batch_poly(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st)
{
    bk_poly<R><<<S.blocks, S.block, 0, st>>>(L.gd, L.tiles, L.ntiles, stage);
    return cudaGetLastError();
}
template <typename R> cudaError_t batch_flux(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st)
{
    if (S.block != 128) return cudaErrorInvalidConfiguration; /* the face mapping's group size */
    bk_flux<R><<<S.blocks, S.block, 0, st>>>(L.gd, L.tiles, L.ntiles, stage, L.dt, L.status);
    return cudaGetLastError();
}
template <typename R> cudaError_t batch_update(const BatchLaunch &L, const LaunchShape &S, int stage, cudaStream_t st)
{
    bk_update<R><<<S.blocks, S.block, 0, st>>>(L.gd, L.tiles, L.ntiles, stage, L.dt, L.status);
    return cudaGetLastError();
}
cudaError_t batch_shadow(const GridDesc &g, cudaStream_t st)
{
    const long want = (g.P.ncell + 255) / 256;
    shadow_kernel<2><<<(unsigned)(want < 4096 ? (want > 0 ? want : 1) : 4096), 256, 0, st>>>(g.P, g.W, g.G, g.s0);
    return cudaGetLastError();
}

cudaError_t batch_widen_grad(const GridDesc &g, cudaStream_t st)
{
    const long n = 2L * 4 * g.P.ncell;
    const long want = (n + 255) / 256;
    widen_grad_kernel<<<(unsigned)(want < 4096 ? (want > 0 ? want : 1) : 4096), 256, 0, st>>>(g.s0.g, g.G, n);
    return cudaGetLastError();
}

cudaError_t batch_dt(const GridDesc *gd, int nb, double cfl, const unsigned long long *smax, double *dt, cudaStream_t st)
{
    bk_dt<<<(nb + 127) / 128, 128, 0, st>>>(gd, nb, cfl, smax, dt);
    return cudaGetLastError();
}

/* resident blocks per SM of one kernel class at a block size */
int batch_occupancy(int kernel, int precision, int block)
{
    int n = 0;
    switch (kernel) {
    case BK_SPEED:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, precision ? bk_speed<float> : bk_speed<double>, block, 0);
        break;
    case BK_POLY:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bk_poly<double>, block, 0);
        break;
    case BK_FLUX:
        smem_carveout_for(bk_flux<double>, flux_blocks_per_sm<double, 2, false>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bk_flux<double>, block, 0);
        break;
    case BK_STAGE:
        /* the opt-in to the dynamic shared memory, then the occupancy with it */
        if (stage_prepare() == cudaSuccess)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bk_stage<1>, kStageThreads, SweepStrip<kStageStrip>::SMEM);
        else
            (void)cudaGetLastError();
        break;
    default:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bk_update<double>, block, 0);
        break;
    }
    return n;
}

#define GKS_BATCH_INST(R)                                                                             \
    template cudaError_t batch_speed<R>(const BatchLaunch &, const LaunchShape &, cudaStream_t);       \
    template cudaError_t batch_poly<R>(const BatchLaunch &, const LaunchShape &, int, cudaStream_t);   \
    template cudaError_t batch_flux<R>(const BatchLaunch &, const LaunchShape &, int, cudaStream_t);   \
    template cudaError_t batch_update<R>(const BatchLaunch &, const LaunchShape &, int, cudaStream_t);
template cudaError_t batch_speed<float>(const BatchLaunch &, const LaunchShape &, cudaStream_t);
GKS_BATCH_INST(double)

} // namespace gks
