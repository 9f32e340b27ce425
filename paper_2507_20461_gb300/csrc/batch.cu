/* C ABI of the batched 2D mode (gks_batch_*): many independent grids of
 * uneven sizes, persistent kernels over tile work lists, per-grid time steps
 * on the device, one step captured into a CUDA graph and replayed.  Mixed
 * precision runs each stage as one persistent launch of the fused stage
 * kernel over a list of strips of every grid (persistent blocks take the
 * strips from a work counter); FP64 runs the three kernel
 * classes (reconstruction, flux, update).  The tile size and block size of
 * every kernel class are picked by timing the candidates on the actual grids
 * before the graph is recorded; the choices are cached per (dimension,
 * precision, size class of the batch, SM count), in the process and, if the
 * environment variable GKS_TUNE_CACHE names a file, in that file (one JSON
 * object per line), so a batch of the same size class skips the timing. */
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <algorithm>
#include <string>
#include <vector>

#include "batch.h"

using gks::BatchLaunch;
using gks::GridDesc;
using gks::LaunchShape;
using gks::Tile;

struct gks_batch_ctx {
    int nb, precision;
    double gamma;
    int bc;
    gks_opts_t opts;
    cudaStream_t stream;      /* internal, capturable */
    cudaStream_t user_stream; /* ordering with the caller */
    cudaEvent_t ev_in, ev_out;
    std::vector<GridDesc> hd;
    GridDesc *dd;
    void *ws;
    size_t ws_bytes;
    double *dt;
    unsigned long long *smax;
    int *status; /* per-grid status words status[g] (OR of the ST_* bits) */
    int *queue;  /* work counters of the fused stage kernel (one per stage) */
    Tile *tiles[gks::BK_COUNT];
    int ntiles[gks::BK_COUNT];
    LaunchShape shape[gks::BK_COUNT];
    int tuned;
    /* mixed precision: per grid, gradients held only in the FP32 shadow
     * since the last run (G is filled from it when the state is read) */
    std::vector<char> g_stale;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    double graph_cfl;
    int nsm;
    char tuning[768];
    char err[256];
};

namespace {

thread_local char g_batch_err[256] = "";

int bfail(gks_batch_ctx *b, int code, const char *fmt, ...)
{
    char *buf = b ? b->err : g_batch_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

int bcuda(gks_batch_ctx *b, cudaError_t e, const char *where)
{
    return bfail(b, GKS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

void make_kp(gks::KP &P, int nx, int ny, double h, double gamma, int bc, const gks_opts_t &o)
{
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
    P.foff[0] = 0;
    P.foff[1] = P.nface[0];
    P.nftot = P.nface[0] + P.nface[1];
    gks::set_bcs(P, bc);
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
}

/* item count of kernel class k on grid g (flux: per direction) */
long items(const gks::KP &P, int k, int dir)
{
    switch (k) {
    case gks::BK_SPEED:
    case gks::BK_UPDATE: return P.ncell;
    case gks::BK_POLY: return P.next;
    /* face Gauss points, rounded up to whole 128-item groups (the FP32 flux
     * maps each group to one block; items past the last face write nothing) */
    default: return (P.nface[dir] * 2 + 127) / 128 * 128;
    }
}

/* the strips of the fused stage kernel: per grid, columns in strips of
 * kStageStrip, rows in chunks of `rows` */
void stage_tiles(const gks_batch_ctx *b, long rows, std::vector<Tile> &v)
{
    for (int g = 0; g < b->nb; ++g) {
        const gks::KP &P = b->hd[g].P;
        for (int x0 = 0; x0 < P.n[0]; x0 += gks::kStageStrip)
            for (long y0 = 0; y0 < P.n[1]; y0 += rows) v.push_back(Tile{g, x0, y0, y0 + rows < P.n[1] ? y0 + rows : P.n[1]});
    }
    /* largest strips first (columns x rows), so the work counter ends on small ones */
    auto cost = [b](const Tile &t) {
        const int w = std::min(gks::kStageStrip, b->hd[t.grid].P.n[0] - t.kind);
        return (long)w * (t.end - t.begin);
    };
    std::stable_sort(v.begin(), v.end(), [&](const Tile &a, const Tile &c) { return cost(a) > cost(c); });
}

int build_tiles(gks_batch_ctx *b, int k, long tile)
{
    /* the previous list may still be read by work on the internal stream */
    cudaError_t se = cudaStreamSynchronize(b->stream);
    if (se != cudaSuccess) return bcuda(b, se, "tile list");
    /* flux tiles start on 128-item groups (one group = one 128-thread block
     * of the FP32 face mapping, whose face sums synchronise the block) */
    if (k == gks::BK_FLUX && tile % 128 != 0) return bfail(b, GKS_ERR_ARG, "flux tiles must be whole 128-item groups");
    std::vector<Tile> v;
    if (k == gks::BK_STAGE) stage_tiles(b, tile, v);
    for (int g = 0; g < b->nb && k != gks::BK_STAGE; ++g) {
        const gks::KP &P = b->hd[g].P;
        const int ndir = (k == gks::BK_FLUX) ? 2 : 1;
        for (int d = 0; d < ndir; ++d) {
            const long n = items(P, k, d);
            for (long s = 0; s < n; s += tile) v.push_back(Tile{g, d, s, s + tile < n ? s + tile : n});
        }
    }
    if (b->tiles[k]) cudaFree(b->tiles[k]);
    b->tiles[k] = nullptr;
    cudaError_t e = cudaMalloc(&b->tiles[k], sizeof(Tile) * v.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->tiles[k], v.data(), sizeof(Tile) * v.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "tile list");
    b->ntiles[k] = (int)v.size();
    b->shape[k].tile = tile;
    return GKS_OK;
}

BatchLaunch launch_of(gks_batch_ctx *b, int k)
{
    return BatchLaunch{b->dd, b->tiles[k], b->ntiles[k], b->dt, b->smax, b->status, &b->hd[0].P, b->queue};
}

cudaError_t run_class(gks_batch_ctx *b, int k, int stage)
{
    const BatchLaunch L = launch_of(b, k);
    const LaunchShape &S = b->shape[k];
    const bool f = b->precision == 1;
    switch (k) {
    case gks::BK_SPEED: return f ? gks::batch_speed<float>(L, S, b->stream) : gks::batch_speed<double>(L, S, b->stream);
    /* the three stage kernels run the FP64 batches; mixed precision runs the fused stage kernel */
    case gks::BK_POLY: return f ? cudaErrorInvalidValue : gks::batch_poly<double>(L, S, stage, b->stream);
    case gks::BK_FLUX: return f ? cudaErrorInvalidValue : gks::batch_flux<double>(L, S, stage, b->stream);
    case gks::BK_STAGE: return f ? gks::batch_stage(L, S, stage, b->stream) : cudaErrorInvalidValue;
    default: return f ? cudaErrorInvalidValue : gks::batch_update<double>(L, S, stage, b->stream);
    }
}

/* one full step on the internal stream */
int enqueue_step(gks_batch_ctx *b, double cfl)
{
    cudaError_t e = cudaMemsetAsync(b->smax, 0, sizeof(unsigned long long) * b->nb, b->stream);
    if (e == cudaSuccess) e = run_class(b, gks::BK_SPEED, 1);
    if (e == cudaSuccess) e = gks::batch_dt(b->dd, b->nb, cfl, b->smax, b->dt, b->stream);
    for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage) {
        if (b->precision == 1) {
            e = run_class(b, gks::BK_STAGE, stage);
            continue;
        }
        e = run_class(b, gks::BK_POLY, stage);
        if (e == cudaSuccess) e = run_class(b, gks::BK_FLUX, stage);
        if (e == cudaSuccess) e = run_class(b, gks::BK_UPDATE, stage);
    }
    return e == cudaSuccess ? GKS_OK : bcuda(b, e, "batched step");
}

/* time one launch of class k (after one untimed launch) */
float time_class(gks_batch_ctx *b, int k)
{
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    run_class(b, k, 1);
    cudaEventRecord(a, b->stream);
    run_class(b, k, 1);
    cudaEventRecord(z, b->stream);
    cudaEventSynchronize(z);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, z);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    return ms;
}

/* The kernel classes a batch runs: mixed precision the wave speed and the
 * fused stage kernel, FP64 the wave speed and the three stage kernels. */
std::vector<int> classes_of(const gks_batch_ctx *b)
{
    if (b->precision == 1) return {gks::BK_SPEED, gks::BK_STAGE};
    return {gks::BK_SPEED, gks::BK_POLY, gks::BK_FLUX, gks::BK_UPDATE};
}

const char *class_name(int k)
{
    static const char *names[] = {"speed", "poly", "flux", "update", "stage"};
    return names[k];
}

/* Size class of a batch: powers of two of the grid count, of the total cell
 * count and of the largest side, with the dimension, precision, limiter
 * and the device's SM count. */
std::string size_class(const gks_batch_ctx *b)
{
    long cells = 0;
    int side = 0;
    for (int g = 0; g < b->nb; ++g) {
        cells += b->hd[g].P.ncell;
        side = std::max(side, std::max(b->hd[g].P.n[0], b->hd[g].P.n[1]));
    }
    auto lg = [](double x) { return (int)std::lround(std::log2(x > 1.0 ? x : 1.0)); };
    char k[160];
    snprintf(k, sizeof k, "2d/p%d/l%d/nb%d/cells%d/side%d/sm%d", b->precision, b->opts.limiter, lg(b->nb), lg((double)cells),
             lg(side), b->nsm);
    return k;
}

struct TuneEntry {
    LaunchShape shape[gks::BK_COUNT];
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;
bool g_tune_file_read = false;

/* the cache file named by GKS_TUNE_CACHE: one object per line,
 * {"key": "...", "shapes": [[block, tile, blocks], ... per kernel class]} */
void tune_file_read()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = std::getenv("GKS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        const char *kp = std::strstr(line, "\"key\": \"");
        const char *sp = std::strstr(line, "\"shapes\": [");
        if (!kp || !sp) continue;
        kp += 8;
        const char *ke = std::strchr(kp, '"');
        if (!ke) continue;
        TuneEntry t;
        const char *q = sp + 11;
        bool ok = true;
        for (int k = 0; k < gks::BK_COUNT && ok; ++k) {
            long v[3];
            for (int j = 0; j < 3 && ok; ++j) {
                while (*q && (*q < '0' || *q > '9') && *q != '-') ++q;
                char *end = nullptr;
                v[j] = std::strtol(q, &end, 10);
                ok = end != q;
                q = end;
            }
            if (ok) t.shape[k] = LaunchShape{(int)v[0], v[1], (int)v[2]};
        }
        if (ok) g_tune_cache[std::string(kp, ke)] = t;
    }
    std::fclose(f);
}

void tune_file_append(const std::string &key, const TuneEntry &t)
{
    const char *path = std::getenv("GKS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"shapes\": [", key.c_str());
    for (int k = 0; k < gks::BK_COUNT; ++k)
        std::fprintf(f, "%s[%d, %ld, %d]", k ? ", " : "", t.shape[k].block, t.shape[k].tile, t.shape[k].blocks);
    std::fprintf(f, "]}\n");
    std::fclose(f);
}

/* the shapes of a cached entry: rebuild the tile lists */
int apply_shapes(gks_batch_ctx *b, const TuneEntry &t)
{
    for (int k : classes_of(b)) {
        int r = build_tiles(b, k, t.shape[k].tile);
        if (r) return r;
        b->shape[k] = t.shape[k];
    }
    return GKS_OK;
}

/* Autotuner: for every kernel class the batch runs, tile size x block size
 * candidates (the fused stage kernel: rows per strip), persistent grid = SMs
 * x resident blocks; keep the fastest.  Runs only kernels that write scratch
 * (wave speeds, coefficients, face fluxes, stage-1 outputs), so the state is
 * unchanged.  A batch of a size class tuned before (in this process or in
 * the GKS_TUNE_CACHE file) takes the cached shapes without timing. */
int tune(gks_batch_ctx *b, double cfl)
{
    const std::string key = size_class(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_file_read();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            int r = apply_shapes(b, it->second);
            if (r) return r;
            int pos = snprintf(b->tuning, sizeof(b->tuning), "{\"cached\": true, \"key\": \"%s\"", key.c_str());
            for (int k : classes_of(b))
                pos += snprintf(b->tuning + pos, sizeof(b->tuning) - pos, ", \"%s\": {\"block\": %d, \"tile\": %ld, \"blocks\": %d}",
                                class_name(k), b->shape[k].block, b->shape[k].tile, b->shape[k].blocks);
            snprintf(b->tuning + pos, sizeof(b->tuning) - pos, "}");
            b->tuned = 1;
            return GKS_OK;
        }
    }
    const long tiles[] = {512, 2048, 8192, 32768};
    const long rows_c[] = {16, 32, 64, 128};
    int pos = 0;
    pos += snprintf(b->tuning + pos, sizeof(b->tuning) - pos, "{\"cached\": false, \"key\": \"%s\"", key.c_str());
    for (int k : classes_of(b)) {
        const int blocks_c[2] = {128, 256};
        int nblk = (k == gks::BK_POLY || k == gks::BK_FLUX) ? 1 : 2;
        const bool stg = k == gks::BK_STAGE;
        if (stg) nblk = 1;
        float best = 1e30f;
        LaunchShape bs{stg ? 256 : 128, 2048, b->nsm};
        for (int bi = 0; bi < nblk; ++bi) {
            const int block = stg ? 256 : blocks_c[bi];
            const int occ = gks::batch_occupancy(k, b->precision, block);
            for (int ci = 0; ci < 4; ++ci) {
                const long t = stg ? rows_c[ci] : tiles[ci];
                int r = build_tiles(b, k, t);
                if (r) return r;
                b->shape[k].block = block;
                b->shape[k].blocks = b->nsm * (occ > 0 ? occ : 1);
                if (k == gks::BK_SPEED) cudaMemsetAsync(b->smax, 0, sizeof(unsigned long long) * b->nb, b->stream);
                const float ms = time_class(b, k);
                if (ms < best) {
                    best = ms;
                    bs = b->shape[k];
                    bs.tile = t;
                }
            }
        }
        int r = build_tiles(b, k, bs.tile);
        if (r) return r;
        b->shape[k] = bs;
        if (k == gks::BK_SPEED) {
            cudaMemsetAsync(b->smax, 0, sizeof(unsigned long long) * b->nb, b->stream);
            run_class(b, gks::BK_SPEED, 1);
            gks::batch_dt(b->dd, b->nb, cfl, b->smax, b->dt, b->stream);
        }
        if (k == gks::BK_POLY) run_class(b, gks::BK_POLY, 1);
        pos += snprintf(b->tuning + pos, sizeof(b->tuning) - pos, ", \"%s\": {\"block\": %d, \"tile\": %ld, \"blocks\": %d, \"ms\": %.4f}",
                        class_name(k), bs.block, bs.tile, bs.blocks, best);
    }
    snprintf(b->tuning + pos, sizeof(b->tuning) - pos, "}");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "tuning");
    /* tuning ran stage-1 kernels only; clear the status they may have set */
    cudaMemset(b->status, 0, sizeof(int) * b->nb);
    b->tuned = 1;
    TuneEntry t;
    for (int k = 0; k < gks::BK_COUNT; ++k) t.shape[k] = b->shape[k];
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_tune_cache.emplace(key, t).second) tune_file_append(key, t);
    }
    return GKS_OK;
}

} // namespace

extern "C" {

int gks_batch_create(int nbatch, const int *nx, const int *ny, const double *hs, double gamma, gks_bc_t bc,
                     const gks_opts_t *opts, gks_batch_t *out)
{
    if (!out) return bfail(nullptr, GKS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nbatch < 1 || !nx || !ny || !hs) return bfail(nullptr, GKS_ERR_ARG, "nbatch >= 1 and size arrays required");
    if (!(gamma > 1.0) || (bc != GKS_BC_PERIODIC && bc != GKS_BC_TRANSMISSIVE && bc != GKS_BC_REFLECTIVE &&
                            bc != GKS_BC_NOSLIP))
        return bfail(nullptr, GKS_ERR_ARG, "invalid gamma or boundary condition");
    gks_opts_t o;
    gks_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) return bfail(nullptr, GKS_ERR_ARG, "precision must be 0 or 1");
    if (o.limiter < 0 || o.limiter > 3) return bfail(nullptr, GKS_ERR_ARG, "limiter must be 0..3");
    if (o.limiter >= 2 && (!(o.ao_d0 > 0.0) || !(o.ao_d0 < 1.0) || !(o.teno_ct > 0.0) || !(o.teno_ct < 1.0)))
        return bfail(nullptr, GKS_ERR_ARG, "ao_d0 and teno_ct must lie in (0, 1)");
    if (o.workspace) return bfail(nullptr, GKS_ERR_UNSUPPORTED, "batched mode allocates its own workspace");
    if (o.mu != 0.0) return bfail(nullptr, GKS_ERR_UNSUPPORTED, "batched mode solves the Euler equations only (mu = 0)");
    for (int g = 0; g < nbatch; ++g) {
        if (nx[g] < 1 || ny[g] < 1 || nx[g] > (1 << 20) || ny[g] > (1 << 20) || !(hs[g] > 0.0))
            return bfail(nullptr, GKS_ERR_ARG, "grid %d: invalid size or cell size", g);
        /* the kernels decompose indices in 32-bit arithmetic; the flux's
         * (face, Gauss point) index space is rounded up to 128-item groups */
        const long ext = (long)(nx[g] + 2) * (ny[g] + 2);
        const long gx = ((long)(nx[g] + 1) * ny[g] * 2 + 127) / 128 * 128;
        const long gy = ((long)nx[g] * (ny[g] + 1) * 2 + 127) / 128 * 128;
        if (ext >= (1L << 32) || gx >= (1L << 32) || gy >= (1L << 32))
            return bfail(nullptr, GKS_ERR_UNSUPPORTED, "grid %d too large (an index space reaches 2^32)", g);
    }

    gks_batch_ctx *b = new (std::nothrow) gks_batch_ctx();
    if (!b) return bfail(nullptr, GKS_ERR_OOM, "host allocation");
    b->nb = nbatch;
    b->precision = o.precision;
    b->gamma = gamma;
    b->bc = (int)bc;
    b->opts = o;
    b->user_stream = (cudaStream_t)o.stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int r = bcuda(nullptr, e, "stream/event creation");
        delete b;
        return r;
    }
    const size_t rs = o.precision ? sizeof(float) : sizeof(double);
    b->hd.resize(nbatch);
    b->g_stale.assign(nbatch, 0);
    size_t off = al(sizeof(double) * nbatch) + al(sizeof(unsigned long long) * nbatch) + al(sizeof(int) * 8) +
                 al(sizeof(int) * nbatch);
    std::vector<size_t> base(nbatch);
    for (int g = 0; g < nbatch; ++g) {
        make_kp(b->hd[g].P, nx[g], ny[g], hs[g], gamma, (int)bc, o);
        const gks::KP &P = b->hd[g].P;
        base[g] = off;
        off += al(sizeof(double) * 4 * P.ncell) * 3 + al(sizeof(double) * 8 * P.ncell) * 2 + al(rs * 4 * GENO_NC2 * P.next) +
               al(rs * 3 * 4 * 2 * P.nftot);
        if (o.precision == 1) off += 2 * al(sizeof(float) * 16 * P.ncell); /* shadows: hi, lo, g */
    }
    b->ws_bytes = off;
    e = cudaMalloc(&b->ws, off);
    if (e != cudaSuccess) {
        int r = bfail(nullptr, GKS_ERR_OOM, "cudaMalloc of %zu bytes: %s", off, cudaGetErrorString(e));
        cudaStreamDestroy(b->stream);
        delete b;
        return r;
    }
    char *w = (char *)b->ws;
    b->dt = (double *)w;
    b->smax = (unsigned long long *)(w + al(sizeof(double) * nbatch));
    b->queue = (int *)(w + al(sizeof(double) * nbatch) + al(sizeof(unsigned long long) * nbatch));
    b->status = (int *)((char *)b->queue + al(sizeof(int) * 8));
    for (int g = 0; g < nbatch; ++g) {
        GridDesc &D = b->hd[g];
        const gks::KP &P = D.P;
        size_t o2 = base[g];
        D.W = (double *)(w + o2); o2 += al(sizeof(double) * 4 * P.ncell);
        D.Ws = (double *)(w + o2); o2 += al(sizeof(double) * 4 * P.ncell);
        D.Acc = (double *)(w + o2); o2 += al(sizeof(double) * 4 * P.ncell);
        D.G = (double *)(w + o2); o2 += al(sizeof(double) * 8 * P.ncell);
        D.Gs = (double *)(w + o2); o2 += al(sizeof(double) * 8 * P.ncell);
        D.B = w + o2; o2 += al(rs * 4 * GENO_NC2 * P.next);
        D.ff = w + o2; o2 += al(rs * 3 * 4 * 2 * P.nftot);
        D.s0 = D.s1 = gks::Shadow{nullptr, nullptr, nullptr};
        if (o.precision == 1) {
            float *a = (float *)(w + o2), *c2 = (float *)(w + o2 + al(sizeof(float) * 16 * P.ncell));
            D.s0 = gks::Shadow{a, a + 4 * P.ncell, a + 8 * P.ncell};
            D.s1 = gks::Shadow{c2, c2 + 4 * P.ncell, c2 + 8 * P.ncell};
        }
    }
    e = cudaMalloc(&b->dd, sizeof(GridDesc) * nbatch);
    if (e == cudaSuccess) e = cudaMemcpy(b->dd, b->hd.data(), sizeof(GridDesc) * nbatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->ws, 0, off);
    if (e != cudaSuccess) {
        int r = bcuda(nullptr, e, "batch setup");
        gks_batch_destroy(b);
        return r;
    }
    for (int k : classes_of(b)) {
        const int block = (k == gks::BK_STAGE) ? 256 : 128;
        const int occ = gks::batch_occupancy(k, b->precision, block);
        b->shape[k] = LaunchShape{block, k == gks::BK_STAGE ? 32 : 4096, b->nsm * (occ > 0 ? occ : 1)};
        int r = build_tiles(b, k, b->shape[k].tile);
        if (r) {
            std::memcpy(g_batch_err, b->err, sizeof(g_batch_err));
            gks_batch_destroy(b);
            return r;
        }
    }
    *out = b;
    return GKS_OK;
}

int gks_batch_set_state(gks_batch_t b, int grid, const double *W, const double *G, int on_device)
{
    if (!b) return bfail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (grid < 0 || grid >= b->nb || !W || !G) return bfail(b, GKS_ERR_ARG, "grid index or pointers invalid");
    const GridDesc &D = b->hd[grid];
    const size_t n = (size_t)4 * D.P.ncell;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    /* the caller's buffers may still be written by work on its stream */
    cudaError_t e = cudaEventRecord(b->ev_in, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.W, W, n * sizeof(double), k, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.G, G, 2 * n * sizeof(double), k, b->stream);
    if (e == cudaSuccess && b->precision == 1) e = gks::batch_shadow(D, b->stream);
    b->g_stale[grid] = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status + grid, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? GKS_OK : bcuda(b, e, "batch set_state");
}

int gks_batch_get_state(gks_batch_t b, int grid, double *W, double *G, int on_device)
{
    if (!b) return bfail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (grid < 0 || grid >= b->nb) return bfail(b, GKS_ERR_ARG, "grid index invalid");
    const GridDesc &D = b->hd[grid];
    const size_t n = (size_t)4 * D.P.ncell;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    /* the caller's stream may still use the destination buffers */
    cudaError_t e = cudaEventRecord(b->ev_in, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e == cudaSuccess && G && b->precision && b->g_stale[grid]) {
        e = gks::batch_widen_grad(D, b->stream);
        if (e == cudaSuccess) b->g_stale[grid] = 0;
    }
    if (e == cudaSuccess && W) e = cudaMemcpyAsync(W, D.W, n * sizeof(double), k, b->stream);
    if (e == cudaSuccess && G) e = cudaMemcpyAsync(G, D.G, 2 * n * sizeof(double), k, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch get_state");
    int st = 0;
    e = cudaMemcpy(&st, b->status + grid, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "status read");
    if (st) return bfail(b, GKS_ERR_NONPHYSICAL, "grid %d: non-physical state (status bits 0x%x)", grid, st);
    return GKS_OK;
}

int gks_batch_run(gks_batch_t b, double cfl, int nsteps)
{
    if (!b) return bfail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!(cfl > 0.0) || !std::isfinite(cfl) || nsteps < 0) return bfail(b, GKS_ERR_ARG, "cfl > 0 and nsteps >= 0 required");
    if (b->precision == 1 && nsteps > 0) std::fill(b->g_stale.begin(), b->g_stale.end(), 1);
    cudaError_t e = cudaEventRecord(b->ev_in, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e != cudaSuccess) return bcuda(b, e, "stream ordering");
    if (!b->tuned) {
        int r = tune(b, cfl);
        if (r) return r;
    }
    if (!b->exec || b->graph_cfl != cfl) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcuda(b, e, "begin capture");
        int r = enqueue_step(b, cfl);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->stream, &g);
        if (r) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return bcuda(b, e, "end capture");
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
        b->graph_cfl = cfl;
    }
    for (int s = 0; s < nsteps; ++s) {
        e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "graph launch");
    }
    e = cudaEventRecord(b->ev_out, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user_stream, b->ev_out, 0);
    return e == cudaSuccess ? GKS_OK : bcuda(b, e, "stream ordering");
}

int gks_batch_status(gks_batch_t b)
{
    if (!b) return bfail(nullptr, GKS_ERR_ARG, "NULL handle");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "stream synchronize");
    std::vector<int> st(b->nb);
    e = cudaMemcpy(st.data(), b->status, sizeof(int) * b->nb, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "status read");
    int r = 0;
    for (int v : st) r |= v;
    return r;
}

int gks_batch_grid_status(gks_batch_t b, int *status, int n)
{
    if (!b) return bfail(nullptr, GKS_ERR_ARG, "NULL handle");
    if (!status || n != b->nb) return bfail(b, GKS_ERR_ARG, "status must hold one word per grid (%d)", b->nb);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "stream synchronize");
    e = cudaMemcpy(status, b->status, sizeof(int) * b->nb, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GKS_OK : bcuda(b, e, "status read");
}

const char *gks_batch_tuning(gks_batch_t b) { return b ? b->tuning : ""; }

int gks_batch_destroy(gks_batch_t b)
{
    if (!b) return GKS_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int k = 0; k < gks::BK_COUNT; ++k)
        if (b->tiles[k]) cudaFree(b->tiles[k]);
    if (b->dd) cudaFree(b->dd);
    if (b->ws) cudaFree(b->ws);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return GKS_OK;
}

const char *gks_batch_last_error(gks_batch_t b) { return b ? b->err : g_batch_err; }

} // extern "C"
