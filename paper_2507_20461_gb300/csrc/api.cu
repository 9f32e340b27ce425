/* C ABI of libgenogks: handle lifetime, state transfer, and the step driver.
 * The numerics are in kernels.cuh / gks_device.cuh; see include/genogks.h
 * for the contract of every entry point. */
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "internal.h"

namespace {

thread_local char g_create_err[256] = "";

int fail(gks_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(gks_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, GKS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t W, G, Ws, Gs, Acc, small, B, ff, sh0, sh1, total;
    size_t B_elems, ff_elems;
    int shadows;
};

bool grid_ok(const gks_grid_t *g, double *h)
{
    if (!g || g->dim < 1 || g->dim > 3) return false;
    double hh = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a < g->dim) {
            if (g->n[a] < 1 || g->n[a] > (1 << 24)) return false;
            const double ha = (g->hi[a] - g->lo[a]) / g->n[a];
            if (!(ha > 0.0) || !std::isfinite(ha)) return false;
            if (a == 0) hh = ha;
            else if (std::fabs(ha - hh) > 1e-12 * hh) return false;
        } else if (g->n[a] != 1) {
            return false;
        }
    }
    if (h) *h = hh;
    return true;
}

long face_count(const gks_grid_t *g)
{
    long r = 0;
    for (int d = 0; d < g->dim; ++d) {
        long f = 1;
        for (int a = 0; a < g->dim; ++a) f *= (a == d) ? (g->n[a] + 1) : g->n[a];
        r += f;
    }
    return r;
}

Layout layout(const gks_grid_t *g, int precision)
{
    Layout L{};
    const int m = g->dim, nv = m + 2, ng = gks::ngauss(m);
    long ncell = 1, next = 1;
    for (int a = 0; a < m; ++a) {
        ncell *= g->n[a];
        next *= g->n[a] + 2;
    }
    const size_t rs = precision ? sizeof(float) : sizeof(double);
    L.B_elems = (m >= 2) ? (size_t)nv * gks::ncubic(m) * next : 0;
    L.ff_elems = (size_t)3 * nv * ng * face_count(g);
    size_t off = 0;
    L.W = off; off = align_up(off + sizeof(double) * nv * ncell);
    L.G = off; off = align_up(off + sizeof(double) * m * nv * ncell);
    L.Ws = off; off = align_up(off + sizeof(double) * nv * ncell);
    L.Gs = off; off = align_up(off + sizeof(double) * m * nv * ncell);
    L.Acc = off; off = align_up(off + sizeof(double) * nv * ncell);
    L.small = off; off = align_up(off + 256);
    L.B = off; off = align_up(off + rs * L.B_elems);
    L.ff = off; off = align_up(off + rs * L.ff_elems);
    /* FP32 shadows (mixed precision, 2D/3D): hi, lo (nv x cells), g (m x nv x cells) */
    L.shadows = (precision == 1 && m >= 2);
    const size_t shb = L.shadows ? sizeof(float) * (size_t)(2 + m) * nv * ncell : 0;
    L.sh0 = off; off = align_up(off + shb);
    L.sh1 = off; off = align_up(off + shb);
    L.total = off;
    return L;
}

int sync_status(gks_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    return st;
}

int stage_buffer(gks_ctx *c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return GKS_OK;
    if (c->stage_out) cudaFree(c->stage_out);
    c->stage_out = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&c->stage_out, bytes);
    if (e != cudaSuccess) return fail(c, GKS_ERR_OOM, "staging buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
    c->stage_bytes = bytes;
    return GKS_OK;
}

__global__ void widen_kernel(const float *__restrict__ in, double *__restrict__ out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

cudaError_t run_flux(gks_ctx *c, int input, bool sums)
{
    switch (c->dim) {
    case 1: return gks::launch_flux<1>(c, input, sums);
    case 2: return gks::launch_flux<2>(c, input, sums);
    default: return gks::launch_flux<3>(c, input, sums);
    }
}

cudaError_t run_shadow(gks_ctx *c)
{
    switch (c->dim) {
    case 1: return gks::launch_shadow<1>(c);
    case 2: return gks::launch_shadow<2>(c);
    default: return gks::launch_shadow<3>(c);
    }
}

cudaError_t run_update(gks_ctx *c, int stage)
{
    switch (c->dim) {
    case 1: return gks::launch_update<1>(c, stage);
    case 2: return gks::launch_update<2>(c, stage);
    default: return gks::launch_update<3>(c, stage);
    }
}

cudaError_t run_wavespeed(gks_ctx *c, double cfl)
{
    switch (c->dim) {
    case 1: return gks::launch_wavespeed<1>(c, cfl);
    case 2: return gks::launch_wavespeed<2>(c, cfl);
    default: return gks::launch_wavespeed<3>(c, cfl);
    }
}

/* both stages with the time step already in c->dt */
int two_stages(gks_ctx *c)
{
    cudaError_t e;
    if (c->shadows) c->g_stale = 1;
    if (c->dim == 1 && c->order != 8) {
        if ((e = gks::nc_launch_step(c)) != cudaSuccess) return cuda_fail(c, e, "RK4 step");
        return GKS_OK;
    }
    if (c->fused) {
        if ((e = gks::launch_fused2d(c, 1)) != cudaSuccess) return cuda_fail(c, e, "stage 1");
        if ((e = gks::launch_fused2d(c, 2)) != cudaSuccess) return cuda_fail(c, e, "stage 2");
        return GKS_OK;
    }
    if ((e = run_flux(c, 0, true)) != cudaSuccess) return cuda_fail(c, e, "stage 1 flux");
    if ((e = run_update(c, 1)) != cudaSuccess) return cuda_fail(c, e, "stage 1 update");
    if ((e = run_flux(c, 1, true)) != cudaSuccess) return cuda_fail(c, e, "stage 2 flux");
    if ((e = run_update(c, 2)) != cudaSuccess) return cuda_fail(c, e, "stage 2 update");
    return GKS_OK;
}

} // namespace

extern "C" {

void gks_default_opts(gks_opts_t *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = 0;
    o->limiter = 0;
    o->C = 20.0;
    o->eps = 1e-15;
    o->C0 = 8.0;
    o->c1_tau = 0.05;
    o->c2_tau = 1.0;
    o->adm_delta = 0.3;
    o->ao_d0 = 0.85;
    o->teno_ct = 1e-6;
}

size_t gks_workspace_bytes(const gks_grid_t *grid, int precision)
{
    if (!grid_ok(grid, nullptr) || (precision != 0 && precision != 1)) return 0;
    return layout(grid, precision).total;
}

long gks_face_count(const gks_grid_t *grid)
{
    if (!grid_ok(grid, nullptr)) return -1;
    return face_count(grid);
}

int geno_gks_create(const gks_grid_t *grid, double gamma, int order, gks_bc_t bc, const gks_opts_t *opts,
                    gks_handle_t *out)
{
    const gks_bc_t sides[6] = {bc, bc, bc, bc, bc, bc};
    return geno_gks_create_sides(grid, gamma, order, sides, opts, out);
}

int geno_gks_create_sides(const gks_grid_t *grid, double gamma, int order, const gks_bc_t *bc, const gks_opts_t *opts,
                          gks_handle_t *out)
{
    if (!out) return fail(nullptr, GKS_ERR_ARG, "out is NULL");
    *out = nullptr;
    double h = 0.0;
    if (!grid_ok(grid, &h)) return fail(nullptr, GKS_ERR_ARG, "invalid grid (dim 1..3, n >= 1, equal cell size)");
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(nullptr, GKS_ERR_ARG, "gamma must be > 1");
    if (!bc) return fail(nullptr, GKS_ERR_ARG, "boundary conditions are NULL");
    for (int a = 0; a < grid->dim; ++a) {
        for (int sd = 0; sd < 2; ++sd) {
            const gks_bc_t b = bc[2 * a + sd];
            if (b != GKS_BC_PERIODIC && b != GKS_BC_TRANSMISSIVE && b != GKS_BC_REFLECTIVE && b != GKS_BC_NOSLIP)
                return fail(nullptr, GKS_ERR_ARG, "unknown boundary condition on side %d", 2 * a + sd);
        }
        if ((bc[2 * a] == GKS_BC_PERIODIC) != (bc[2 * a + 1] == GKS_BC_PERIODIC))
            return fail(nullptr, GKS_ERR_ARG, "axis %d: periodic on one side only", a);
    }
    const int want = (grid->dim == 1) ? 8 : 4;
    const bool noncompact = grid->dim == 1 && (order == 5 || order == 6);
    if (order != want && !noncompact)
        return fail(nullptr, GKS_ERR_UNSUPPORTED, "order %d is not provided in %dD (use %d%s)", order, grid->dim, want,
                    grid->dim == 1 ? ", or 5 / 6 for the non-compact schemes" : "");
    gks_opts_t o;
    gks_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) return fail(nullptr, GKS_ERR_ARG, "precision must be 0 or 1");
    if (o.limiter < 0 || o.limiter > 3) return fail(nullptr, GKS_ERR_ARG, "limiter must be 0..3");
    if (o.stage_kernels != 0 && o.stage_kernels != 1) return fail(nullptr, GKS_ERR_ARG, "stage_kernels must be 0 or 1");
    if (o.limiter >= 2 && (!(o.ao_d0 > 0.0) || !(o.ao_d0 < 1.0) || !(o.teno_ct > 0.0) || !(o.teno_ct < 1.0)))
        return fail(nullptr, GKS_ERR_ARG, "ao_d0 and teno_ct must lie in (0, 1)");
    if (!(o.C > 0.0) || !(o.eps > 0.0) || !(o.C0 > 0.0) || !(o.c1_tau >= 0.0) || !(o.c2_tau >= 0.0) ||
        !(o.adm_delta >= 0.0) || !(o.adm_delta < 1.0))
        return fail(nullptr, GKS_ERR_ARG, "invalid scheme constants");
    if (!(o.mu >= 0.0) || !std::isfinite(o.mu)) return fail(nullptr, GKS_ERR_ARG, "viscosity mu must be finite and >= 0");
    if (noncompact && (o.precision != 0 || o.mu != 0.0 || o.limiter > 1))
        return fail(nullptr, GKS_ERR_UNSUPPORTED, "the non-compact schemes run in FP64, inviscid, with limiter 0 or 1");

    gks_ctx *c = new (std::nothrow) gks_ctx;
    if (!c) return fail(nullptr, GKS_ERR_OOM, "host allocation");
    std::memset(c, 0, sizeof(*c));
    c->dim = grid->dim;
    c->nv = grid->dim + 2;
    c->ng = gks::ngauss(grid->dim);
    c->precision = o.precision;
    c->order = order;
    for (int a = 0; a < 3; ++a) c->n[a] = grid->n[a];
    c->h = h;
    c->gamma = gamma;
    c->opts = o;
    c->stream = (cudaStream_t)o.stream;

    const Layout L = layout(grid, o.precision);
    if (o.workspace) {
        if (o.workspace_bytes < L.total || ((size_t)o.workspace & 255)) {
            delete c;
            return fail(nullptr, GKS_ERR_OOM, "workspace needs %zu bytes, 256-byte aligned", L.total);
        }
        c->ws = o.workspace;
        c->own_ws = 0;
    } else {
        cudaError_t e = cudaMalloc(&c->ws, L.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, GKS_ERR_OOM, "cudaMalloc of %zu bytes: %s", L.total, cudaGetErrorString(e));
        }
        c->own_ws = 1;
    }
    c->ws_bytes = L.total;
    char *base = (char *)c->ws;
    c->W = (double *)(base + L.W);
    c->G = (double *)(base + L.G);
    c->Ws = (double *)(base + L.Ws);
    c->Gs = (double *)(base + L.Gs);
    c->Acc = (double *)(base + L.Acc);
    c->dt = (double *)(base + L.small);
    c->updc = (float *)(base + L.small + 16);
    c->smax = (unsigned long long *)(base + L.small + 64);
    c->status = (int *)(base + L.small + 128);
    c->B = base + L.B;
    c->ff = base + L.ff;
    c->shadows = L.shadows;
    if (L.shadows) {
        const size_t nvc = (size_t)c->nv;
        long nc = 1;
        for (int a = 0; a < grid->dim; ++a) nc *= grid->n[a];
        float *s0 = (float *)(base + L.sh0), *s1 = (float *)(base + L.sh1);
        c->s0 = gks::Shadow{s0, s0 + nvc * nc, s0 + 2 * nvc * nc};
        c->s1 = gks::Shadow{s1, s1 + nvc * nc, s1 + 2 * nvc * nc};
    }
    c->B_elems = L.B_elems;
    c->ff_elems = L.ff_elems;
    c->fused = (L.shadows && grid->dim == 2 && o.stage_kernels == 1) ? 1 : 0;

    gks::KP &P = c->kp;
    std::memset(&P, 0, sizeof(P));
    long ncell = 1, next = 1;
    for (int a = 0; a < 3; ++a) {
        P.n[a] = grid->n[a];
        P.ext[a] = (a < grid->dim) ? grid->n[a] + 2 : 1;
        ncell *= grid->n[a];
        next *= P.ext[a];
    }
    P.ncell = ncell;
    P.next = next;
    long off = 0;
    for (int d = 0; d < grid->dim; ++d) {
        long f = 1;
        for (int a = 0; a < grid->dim; ++a) f *= (a == d) ? (grid->n[a] + 1) : grid->n[a];
        P.nface[d] = f;
        P.foff[d] = off;
        off += f;
    }
    P.nftot = off;
    /* the kernels decompose indices in 32-bit arithmetic; the FP32 flux
     * rounds its (face, Gauss point) index space up to whole 128-item groups */
    bool fits = next < (1L << 32) && ncell < (1L << 32);
    for (int d = 0; d < grid->dim; ++d)
        fits = fits && (P.nface[d] * gks::ngauss(grid->dim) + 127) / 128 * 128 < (1L << 32);
    if (!fits) {
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return fail(nullptr, GKS_ERR_UNSUPPORTED, "grid too large (an index space reaches 2^32)");
    }
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd) P.bcs[a][sd] = (a < grid->dim) ? (int)bc[2 * a + sd] : 0;
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
    P.fp.mu = o.mu;
    gks::finalize_kp(P);

    cudaError_t e = cudaMemsetAsync(c->ws, 0, L.total, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        int r = cuda_fail(nullptr, e, "workspace clear");
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return r;
    }
    *out = c;
    return GKS_OK;
}

int gks_set_state(gks_handle_t c, const double *W, const double *G, int on_device)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!W || !G) return fail(c, GKS_ERR_ARG, "W and G are required");
    const size_t nW = (size_t)c->nv * c->kp.ncell, nG = (size_t)c->dim * nW;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(c->W, W, nW * sizeof(double), k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->G, G, nG * sizeof(double), k, c->stream);
    if (e == cudaSuccess) e = run_shadow(c);
    c->g_stale = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
    c->err[0] = 0;
    return GKS_OK;
}

int gks_get_state(gks_handle_t c, double *W, double *G, int on_device)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    const size_t nW = (size_t)c->nv * c->kp.ncell, nG = (size_t)c->dim * nW;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (G && c->g_stale) {
        gks::widen_grad_kernel<<<gks::blocks_for((long)nG, 256) > 4096 ? 4096 : gks::blocks_for((long)nG, 256), 256, 0,
                                 c->stream>>>(c->s0.g, c->G, (long)nG);
        e = cudaGetLastError();
        if (e == cudaSuccess) c->g_stale = 0;
    }
    if (e == cudaSuccess && W) e = cudaMemcpyAsync(W, c->W, nW * sizeof(double), k, c->stream);
    if (e == cudaSuccess && G) e = cudaMemcpyAsync(G, c->G, nG * sizeof(double), k, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
    const int st = sync_status(c);
    if (st < 0) return st;
    if (st) return fail(c, GKS_ERR_NONPHYSICAL, "non-physical state (status bits 0x%x)", st);
    return GKS_OK;
}

int geno_reconstruct(gks_handle_t c, double *fs, int on_device)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!fs) return fail(c, GKS_ERR_ARG, "face_states is NULL");
    const size_t n = (size_t)2 * c->nv * (c->dim + 1) * c->ng * c->kp.nftot;
    double *dst = fs;
    if (!on_device) {
        int r = stage_buffer(c, n * sizeof(double));
        if (r) return r;
        dst = c->stage_out;
    }
    cudaError_t e;
    switch (c->dim) {
    case 1: e = gks::launch_states<1>(c, 0, dst); break;
    case 2: e = gks::launch_states<2>(c, 0, dst); break;
    default: e = gks::launch_states<3>(c, 0, dst); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "reconstruct");
    if (!on_device) {
        e = cudaMemcpyAsync(fs, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "reconstruct copy");
    }
    const int st = sync_status(c);
    return st < 0 ? st : GKS_OK;
}

int gks_flux(gks_handle_t c, double dt, double *out, int on_device)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!out) return fail(c, GKS_ERR_ARG, "face_flux is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, GKS_ERR_ARG, "dt must be finite and > 0");
    gks::set_dt_kernel<<<1, 1, 0, c->stream>>>(c->dt, dt, c->shadows ? c->updc : nullptr, gks::updc_cw(c->kp, c->dim));
    cudaError_t e = run_flux(c, 0, false);
    if (e != cudaSuccess) return cuda_fail(c, e, "flux");
    const size_t n = c->ff_elems;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->precision == 0) {
        e = cudaMemcpyAsync(out, c->ff, n * sizeof(double), k, c->stream);
    } else {
        double *dst = out;
        if (!on_device) {
            int r = stage_buffer(c, n * sizeof(double));
            if (r) return r;
            dst = c->stage_out;
        }
        widen_kernel<<<gks::blocks_for((long)n, 256) > 4096 ? 4096 : gks::blocks_for((long)n, 256), 256, 0,
                       c->stream>>>((const float *)c->ff, dst, n);
        e = cudaGetLastError();
        if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, n * sizeof(double), k, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "flux copy");
    const int st = sync_status(c);
    if (st < 0) return st;
    if (st & GKS_ST_FLUX) return fail(c, GKS_ERR_NONPHYSICAL, "a face state was not admissible (status 0x%x)", st);
    return GKS_OK;
}

int gks_step(gks_handle_t c, double dt)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, GKS_ERR_ARG, "dt must be finite and > 0");
    gks::set_dt_kernel<<<1, 1, 0, c->stream>>>(c->dt, dt, c->shadows ? c->updc : nullptr, gks::updc_cw(c->kp, c->dim));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "set dt");
    return two_stages(c);
}

int gks_step_cfl(gks_handle_t c, double cfl, int nsteps)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!(cfl > 0.0) || !std::isfinite(cfl) || nsteps < 0) return fail(c, GKS_ERR_ARG, "cfl > 0 and nsteps >= 0 required");
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = run_wavespeed(c, cfl);
        if (e != cudaSuccess) return cuda_fail(c, e, "time step");
        int r = two_stages(c);
        if (r) return r;
    }
    return GKS_OK;
}

int gks_max_wavespeed(gks_handle_t c, double *out)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!out) return fail(c, GKS_ERR_ARG, "out is NULL");
    cudaError_t e = run_wavespeed(c, 0.0);
    if (e != cudaSuccess) return cuda_fail(c, e, "wavespeed");
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, c->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "wavespeed read");
    double s;
    std::memcpy(&s, &bits, sizeof(s));
    *out = s;
    if (!std::isfinite(s) || s >= 1e299) return fail(c, GKS_ERR_NONPHYSICAL, "non-finite wave speed");
    return GKS_OK;
}

int gks_status(gks_handle_t c)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    return sync_status(c);
}

int gks_profile_enable(gks_handle_t c, int on, int reset)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (on && !c->prof_ev) {
        c->prof_ev = new (std::nothrow) cudaEvent_t[2 * gks::kProfCap];
        c->prof_cls = new (std::nothrow) int[gks::kProfCap];
        if (!c->prof_ev || !c->prof_cls) return fail(c, GKS_ERR_OOM, "profiler allocation");
        for (int i = 0; i < 2 * gks::kProfCap; ++i) {
            cudaError_t e = cudaEventCreate(&c->prof_ev[i]);
            if (e != cudaSuccess) return cuda_fail(c, e, "profiler events");
        }
    }
    if (c->prof_ev) gks::prof_flush(c);
    if (reset) {
        for (int k = 0; k < 8; ++k) {
            c->prof_launches[k] = 0;
            c->prof_ms[k] = 0.0;
        }
    }
    c->prof_on = on ? 1 : 0;
    return GKS_OK;
}

int gks_profile_read(gks_handle_t c, int cls, long *launches, double *ms)
{
    if (!c) return fail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (cls < 0 || cls >= 8) return fail(c, GKS_ERR_ARG, "kernel class out of range");
    if (c->prof_ev) gks::prof_flush(c);
    if (launches) *launches = c->prof_launches[cls];
    if (ms) *ms = c->prof_ms[cls];
    return GKS_OK;
}

int gks_destroy(gks_handle_t c)
{
    if (!c) return GKS_OK;
    cudaStreamSynchronize(c->stream);
    if (c->prof_ev) {
        for (int i = 0; i < 2 * gks::kProfCap; ++i) cudaEventDestroy(c->prof_ev[i]);
        delete[] c->prof_ev;
        delete[] c->prof_cls;
    }
    if (c->stage_out) cudaFree(c->stage_out);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
    return GKS_OK;
}

const char *gks_last_error(gks_handle_t c) { return c ? c->err : g_create_err; }

} // extern "C"
