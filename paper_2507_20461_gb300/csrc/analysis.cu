/* geno_linearity: the nonlinear weights of the reconstruction evaluated on
 * given indicator sets, by the same device functions the reconstruction
 * kernels call (chi_of for GENO, ao_weights for WENO-Z / TENO).  It exposes
 * the paper's analysis of how much of the high-order linear reconstruction
 * each method keeps (Sec. 3.1-3.2, Sec. 5.1-5.2) on the GPU's own arithmetic,
 * in FP64 or FP32. */
#include <cmath>
#include <cstring>

#include "internal.h"

namespace {

template <typename R, int K>
__global__ void linearity_kernel(gks::KP P, int r, long n, const double *__restrict__ IS, const double *__restrict__ tau,
                                 double *__restrict__ chi)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        R I[K + 1];
#pragma unroll
        for (int k = 0; k <= K; ++k) I[k] = R(IS[i * (K + 1) + k]);
        const R t = R(tau[i]);
        R out = R(1);
        if (P.limiter == 0) {
            R hi = I[0], lo = I[0];
#pragma unroll
            for (int k = 1; k <= K; ++k) {
                hi = fmax(hi, I[k]);
                lo = fmin(lo, I[k]);
            }
            out = gks::chi_of<R>(P, t, hi, lo, r);
        } else if (P.limiter >= 2) {
            R d[K + 1], w[K + 1];
#pragma unroll
            for (int k = 0; k <= K; ++k) d[k] = R(1) / R(K + 1);
            gks::ao_weights<R, K>(P, d, I, t, w);
            out = w[0] / d[0];
#pragma unroll
            for (int k = 1; k <= K; ++k) out = fmin(out, w[k] / d[k]);
        }
        chi[i] = (double)out;
    }
}

template <typename R>
cudaError_t launch(const gks::KP &P, int r, int k, long n, const double *IS, const double *tau, double *chi,
                   cudaStream_t s)
{
    const long want = (n + 255) / 256;
    const unsigned nb = (unsigned)(want < 1024 ? (want > 0 ? want : 1) : 1024);
    switch (k) {
#define GKS_LIN(KK)                                                                                  \
    case KK + 1: linearity_kernel<R, KK><<<nb, 256, 0, s>>>(P, r, n, IS, tau, chi); break;
        GKS_LIN(1) GKS_LIN(2) GKS_LIN(3) GKS_LIN(4) GKS_LIN(5) GKS_LIN(6) GKS_LIN(7)
#undef GKS_LIN
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace

extern "C" int geno_linearity(const gks_opts_t *opts, int limiter, int r, int k, long n, const double *IS,
                              const double *tau, double *chi, void *stream)
{
    if (limiter < 0 || limiter > 3 || (r != 2 && r != 3) || k < 2 || k > 8 || n < 0) return GKS_ERR_ARG;
    if (n > 0 && (!IS || !tau || !chi)) return GKS_ERR_ARG;
    gks_opts_t o;
    gks_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) return GKS_ERR_ARG;
    if (!(o.C > 0.0) || !(o.eps > 0.0) || !(o.teno_ct > 0.0) || !(o.teno_ct < 1.0)) return GKS_ERR_ARG;
    if (n == 0) return GKS_OK;
    gks::KP P;
    std::memset(&P, 0, sizeof(P));
    P.limiter = limiter;
    P.gamma = 1.4;
    P.C = o.C;
    P.itanhC = 1.0 / std::tanh(o.C);
    P.eps = o.eps;
    P.C0 = o.C0;
    P.d0 = o.ao_d0;
    P.ct = o.teno_ct;
    gks::finalize_kp(P);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = o.precision ? launch<float>(P, r, k, n, IS, tau, chi, s) : launch<double>(P, r, k, n, IS, tau, chi, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}
