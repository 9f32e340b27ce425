/* gks_flux_2d_static: the 2D FP64 interface-flux computation (the same
 * kernels as gks_flux) for callers that cannot allocate device memory.
 *
 * Who needs it: code that runs where cudaMalloc is not available or not
 * allowed - inside a host callback or a plugin that must not own memory,
 * in a process whose allocator is owned by another framework, or in a
 * latency-critical loop where an allocation (and its implicit device
 * synchronisation) is not acceptable.  Those callers pass their own input
 * and output buffers; the only scratch this call needs (the per-cell GENO
 * coefficients, the time step and a status word) lives in one file-scope
 * device array that every GPU loading this library holds until exit.
 *
 * The array is shared by every call on a device and keeps the previous
 * call's contents; calls that overlap on the GPU (different streams, or
 * different host threads without ordering) race on it.
 */
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

/* maximum (nx + 2) * (ny + 2): the cells plus their one-cell ghost ring */
constexpr long kMaxExtCells = 14400;
constexpr int kNC = GENO_NC2;
/* coefficient block (4 variables x kNC doubles per extended cell), then
 * 256 bytes for the time step and the status word */
constexpr size_t kCoefBytes = sizeof(double) * 4 * kNC * kMaxExtCells;
constexpr size_t kScratchBytes = kCoefBytes + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

/* device address of g_scratch on the current device (looked up once per device) */
int scratch_address(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GKS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return GKS_ERR_CUDA;
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return GKS_OK;
}

} // namespace

extern "C" int gks_flux_2d_static(int nx, int ny, double h, double gamma, gks_bc_t bc, const gks_opts_t *opts,
                                  const double *W, const double *G, double dt, double *face_flux, void *stream)
{
    if (nx < 1 || ny < 1 || !(h > 0.0) || !std::isfinite(h) || !(gamma > 1.0) || !std::isfinite(gamma))
        return GKS_ERR_ARG;
    /* larger grids do not fit the static scratch (widened before adding, so
     * sides near INT_MAX cannot wrap) */
    if (((long)nx + 2) * ((long)ny + 2) > kMaxExtCells) return GKS_ERR_ARG;
    if (bc != GKS_BC_PERIODIC && bc != GKS_BC_TRANSMISSIVE && bc != GKS_BC_REFLECTIVE && bc != GKS_BC_NOSLIP)
        return GKS_ERR_ARG;
    if (!W || !G || !face_flux) return GKS_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return GKS_ERR_ARG;
    gks_opts_t o;
    gks_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 0 || o.mu != 0.0) return GKS_ERR_UNSUPPORTED;
    if (o.limiter < 0 || o.limiter > 3) return GKS_ERR_ARG;
    if (o.limiter >= 2 && (!(o.ao_d0 > 0.0) || !(o.ao_d0 < 1.0) || !(o.teno_ct > 0.0) || !(o.teno_ct < 1.0)))
        return GKS_ERR_ARG;
    /* the scheme constants geno_gks_create accepts, and no others */
    if (!(o.C > 0.0) || !(o.eps > 0.0) || !(o.C0 > 0.0) || !(o.c1_tau >= 0.0) || !(o.c2_tau >= 0.0) ||
        !(o.adm_delta >= 0.0) || !(o.adm_delta < 1.0) || !std::isfinite(o.C) || !std::isfinite(o.C0) ||
        !std::isfinite(o.c1_tau) || !std::isfinite(o.c2_tau))
        return GKS_ERR_ARG;

    unsigned char *base = nullptr;
    int r = scratch_address(&base);
    if (r) return r;
    double *B = (double *)base;
    double *dtp = (double *)(base + kCoefBytes);
    int *status = (int *)(base + kCoefBytes + 64);
    cudaStream_t s = (cudaStream_t)stream;

    gks::KP P;
    std::memset(&P, 0, sizeof(P));
    P.n[0] = nx;
    P.n[1] = ny;
    P.n[2] = 1;
    P.ext[0] = nx + 2;
    P.ext[1] = ny + 2;
    P.ext[2] = 1;
    P.ncell = (long)nx * ny;
    P.next = (long)(nx + 2) * (ny + 2);
    P.nface[0] = (long)(nx + 1) * ny;
    P.nface[1] = (long)nx * (ny + 1);
    P.foff[1] = P.nface[0];
    P.nftot = P.nface[0] + P.nface[1];
    gks::set_bcs(P, (int)bc);
    P.limiter = o.limiter;
    P.h = h;
    P.ih = 1.0 / h;
    P.gamma = gamma;
    P.C = o.C;
    P.itanhC = 1.0 / std::tanh(o.C);
    P.eps = o.eps;
    P.C0 = o.C0;
    P.adm = o.adm_delta;
    P.d0 = o.ao_d0;
    P.ct = o.teno_ct;
    P.fp.gamma = gamma;
    P.fp.c1 = o.c1_tau;
    P.fp.c2 = o.c2_tau;
    gks::finalize_kp(P);

    /* the status word must start at zero; the coefficients are fully rewritten */
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        gks::set_dt_kernel<<<1, 1, 0, s>>>(dtp, dt, nullptr, 0.0);
        const gks::Src<double> src{W, G};
        gks::face_flux_prepare<double, 2, 0, true>();
        gks::face_flux_prepare<double, 2, 1, true>();
        gks::cell_poly_kernel<double, 2><<<gks::blocks_for(P.next), gks::kBlock, 0, s>>>(P, src, B);
        gks::face_flux_kernel<double, 2, 0, true>
            <<<gks::blocks_for(P.nface[0] * 2), gks::kBlock, 0, s>>>(P, src, B, dtp, nullptr, face_flux, status);
        gks::face_flux_kernel<double, 2, 1, true>
            <<<gks::blocks_for(P.nface[1] * 2), gks::kBlock, 0, s>>>(P, src, B, dtp, nullptr, face_flux, status);
        e = cudaGetLastError();
    }
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GKS_ERR_CUDA;
    if (st) return GKS_ERR_NONPHYSICAL;
    return GKS_OK;
}
