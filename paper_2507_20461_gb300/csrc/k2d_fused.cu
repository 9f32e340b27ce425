/* Launcher of the fused 2D mixed-precision stage kernel (fused2d.cuh). */
#include "fused2d.cuh"
#include "internal.h"

namespace gks {

namespace {

/* strips of 62 columns swept by 256 threads (both phases one full round),
 * 3 blocks per SM (80 registers), chunks of 32 rows */
constexpr int kTX = 62, kNT = 256, kMinBlocks = 3, kRows = 32;
using Strip = SweepStrip<kTX>;

template <int STAGE, bool NS> cudaError_t fused_launch(gks_ctx *c)
{
    auto kernel = fused2d_stage_kernel<STAGE, NS, kTX, kNT, kMinBlocks>;
    /* dynamic shared memory above 48 KB needs the opt-in, once per kernel */
    static const cudaError_t prep = [&] {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Strip::SMEM);
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
            (void)cudaGetLastError();
        return e;
    }();
    if (prep != cudaSuccess) return prep;
    const dim3 grid((unsigned)((c->kp.n[0] + kTX - 1) / kTX), (unsigned)((c->kp.n[1] + kRows - 1) / kRows));
    ProfScope ps(c, GKS_KC_STAGE);
    kernel<<<grid, kNT, Strip::SMEM, c->stream>>>(c->kp, c->s0, c->s1, c->W, (float *)c->Acc, c->dt, c->status,
                                                  kRows);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_fused2d(gks_ctx *c, int stage)
{
    const bool ns = c->kp.fp.mu > 0.0;
    if (stage == 1) return ns ? fused_launch<1, true>(c) : fused_launch<1, false>(c);
    return ns ? fused_launch<2, true>(c) : fused_launch<2, false>(c);
}

} // namespace gks
