/*
 * One stage of the 2D compact GKS with GENO reconstruction as a single
 * kernel (arXiv 2507.20461, Sec. 2: reconstruct, evolve the gas distribution
 * at the interfaces, update the averages by Eq. semifvs and the averaged
 * gradients by Eq. slope), mixed precision: FP32 reconstruction and flux,
 * exact FP32 face sums and double-float / FP64 accumulation.
 *
 * A block owns a strip of TX columns and sweeps it row by row over a chunk
 * of rows, keeping everything between the stage input and the stage output
 * in shared memory:
 *   - a ring of four rows of the stage input (FP32 shadow: hi, lo, grad x,
 *     grad y of the four variables; the strip plus two ghost columns on
 *     each side, mapped and sign-flipped by the boundary conditions),
 *     filled with cp.async one row ahead of its use;
 *   - a ring of two rows of blended GENO cubics (blend_cubic; the strip
 *     plus one column on each side);
 *   - the face values (F, dF/dt, W(dt/2) per Gauss point) of the x faces of
 *     one row and a ring of two rows of y faces.
 * Per row j, two phases separated by block barriers:
 *   A  the cubics of row j + 1 and the stage update of row j - 1
 *      (mixed_update_var), each one item per (cell, variable);
 *   B  the faces of row j: its TX + 1 x faces and the TX y faces between
 *      rows j and j + 1, at both Gauss points; a warp takes 32 faces at one
 *      Gauss point (the evaluation of the cubics does not diverge); with
 *      TX = 62 and 256 threads (or TX = 30 and 128) both phases are one
 *      full round.
 * Only the first cubic rows and y faces of a chunk, and the two columns on
 * each side of a strip, are evaluated twice (by both blocks that touch them,
 * from the same inputs by the same instructions, so both get the same bits
 * and every face's flux still leaves one cell and enters the other exactly:
 * the sums of the averages stay conserved to FP64 rounding).  Neither the
 * cubic coefficients nor the face fluxes go through device memory.
 */
#pragma once
#include "kernels.cuh"

namespace gks {

template <int TX_> struct SweepStrip {
    static constexpr int TX = TX_;
    static constexpr int NV = 4, NC = GENO_NC2;
    /* stage-input rows: the strip plus two ghost columns on each side */
    static constexpr int WX = TX + 4;
    static constexpr int NFIELD = 16; /* hi[v], lo[v], g_x[v], g_y[v] */
    static constexpr int SROW = NFIELD * WX;
    static constexpr int NSLOT = 4;
    /* cubic rows: the strip plus one column on each side */
    static constexpr int CX = TX + 2;
    static constexpr int REC = NV * NC;
    static constexpr int BROW = CX * REC, WROW = CX * NV;
    /* face values: per (face, Gauss point) F, dF/dt, W(dt/2) of the four
     * variables, global variable order */
    static constexpr int FV = 3 * NV;
    static constexpr int NXF = TX + 1, NYF = TX;
    static constexpr int XROW = NXF * 2 * FV, YROW = NYF * 2 * FV;
    /* flux work: 32-face blocks of x faces, then of y faces, each at two
     * Gauss points */
    static constexpr int NXB = (NXF + 31) / 32, NYB = (NYF + 31) / 32, NWI = 2 * (NXB + NYB);
    static constexpr int O_STATE = 0, O_B = O_STATE + NSLOT * SROW, O_W0 = O_B + 2 * BROW, O_XF = O_W0 + 2 * WROW,
                         O_YF = O_XF + XROW, FLOATS = O_YF + 2 * YROW;
    static constexpr size_t SMEM = sizeof(float) * (size_t)FLOATS;
    static_assert(SROW % 4 == 0 && BROW % 4 == 0 && WROW % 4 == 0 && XROW % 4 == 0 && YROW % 4 == 0,
                  "16-byte aligned regions");
};

/* plane of field f of a stage input: f = v (hi), 4 + v (lo), 8 + 4 a + v
 * (gradient along a) */
__device__ __forceinline__ const float *sweep_plane(const Shadow &s, long nc, int f)
{
    return (f < 4) ? s.hi + (long)f * nc : (f < 8) ? s.lo + (long)(f - 4) * nc : s.g + (long)(f - 8) * nc;
}

/* Geometry of one grid: the fields of its parameter block that differ
 * between the grids of a batch (which share every scheme constant). */
struct FusedGeo {
    int nx, ny;
    long nc;
    double ih;
    float fh, fih;
};

__host__ __device__ __forceinline__ FusedGeo fused_geo(const KP &P)
{
    return FusedGeo{P.n[0], P.n[1], P.ncell, P.ih, P.fh, P.fih};
}

/* The stage on the strip of columns x0 .. x0 + TX - 1, rows y0 .. y0 + rows
 * - 1 (clipped to the grid), by the NT threads of the calling block; P holds
 * the scheme constants and boundary types, geo the grid's geometry; smem
 * holds SweepStrip<TX>::FLOATS floats, uc is block-shared.  Every thread of
 * the block calls it. */
template <int STAGE, bool NS, int TX, int NT>
__device__ __forceinline__ void fused2d_strip(const KP &P, const FusedGeo &geo, const Shadow &s0, const Shadow &s1,
                                              double *__restrict__ W, float *__restrict__ acc, double dt,
                                              int *__restrict__ status, int x0, int y0, int rows, float *smem,
                                              UpdC &uc)
{
    using T = SweepStrip<TX>;
    constexpr int NV = T::NV, NC = T::NC, WX = T::WX, CX = T::CX;
    static_assert(NT >= 4 * TX && NT % 32 == 0, "the update of a row takes one thread per (cell, variable)");
    float *const S = smem + T::O_STATE; /* [slot][field][WX] */
    float *const Bc = smem + T::O_B;    /* [slot][cx][v * NC + k] */
    float *const W0 = smem + T::O_W0;   /* [slot][cx][v] signed cell averages (FP32 hi) */
    float *const XF = smem + T::O_XF;   /* [ix][g][12] */
    float *const YF = smem + T::O_YF;   /* [slot][ix][g][12] */

    const Shadow &sin = (STAGE == 1) ? s0 : s1;
    const int nx = geo.nx, ny = geo.ny;
    const long nc = geo.nc;
    const int y1 = min(y0 + rows, ny);
    const int tid = threadIdx.x;
    if (tid == 0) uc = make_updc(dt, geo.ih / 2);
    const bool xin = x0 >= 2 && x0 + TX + 2 <= nx; /* every column of the strip's rows is inside */

    /* stage-input row r into its ring slot; cells that need no sign change
     * are copied with cp.async (completed by cp_wait), mirrored ghost cells
     * whose sign changes are read, negated and stored */
    auto load_row = [&](int r) {
        float *dst = S + (r & 3) * T::SROW;
        const bool rin = r >= 0 && r < ny;
        for (int it = tid; it < T::SROW; it += NT) {
            const int f = it / WX, wx = it - f * WX;
            const int gx = x0 - 2 + wx;
            const float *plane = sweep_plane(sin, nc, f);
            long src;
            bool neg = false;
            if (rin && xin) {
                src = (long)r * nx + gx;
            } else {
                int flip[3] = {0, 0, 0};
                const int ii = map_idx(gx, nx, P.bcs[0][0], P.bcs[0][1], flip[0]);
                const int jj = map_idx(r, ny, P.bcs[1][0], P.bcs[1][1], flip[1]);
                src = (long)jj * nx + ii;
                neg = ghost_sign<2>(P, flip, f & 3) < 0;
                if (f >= 8 && (flip[(f - 8) >> 2] & 1)) neg = !neg;
            }
            if (!neg) {
                const unsigned d = (unsigned)__cvta_generic_to_shared(dst + it);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(plane + src) : "memory");
            } else {
                dst[it] = -plane[src];
            }
        }
    };
    auto cp_wait = [] { asm volatile("cp.async.wait_all;\n" ::: "memory"); };

    /* blended cubic of item it of cubic row r (state rows r - 1 .. r + 1 in the ring) */
    auto recon_item = [&](int r, int it) {
        const int v = it / CX, cx = it - v * CX;
        const float *rm = S + ((r - 1) & 3) * T::SROW, *r0 = S + (r & 3) * T::SROW, *rp = S + ((r + 1) & 3) * T::SROW;
        const int wx = cx + 1;
        const float hr = geo.fh;
        const int fh = v, fl = 4 + v, fgx = 8 + v, fgy = 12 + v;
        const float h0 = r0[fh * WX + wx], l0 = r0[fl * WX + wx];
        float d[GENO_ND2];
        /* q = 2 e + (side > 0): x-, x+, y-, y+ */
        const float *row[4] = {r0, r0, rm, rp};
        const int col[4] = {wx - 1, wx + 1, wx, wx};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            d[q * 3] = (row[q][fh * WX + col[q]] - h0) + (row[q][fl * WX + col[q]] - l0);
            d[q * 3 + 1] = row[q][fgx * WX + col[q]] * hr;
            d[q * 3 + 2] = row[q][fgy * WX + col[q]] * hr;
        }
        d[12] = r0[fgx * WX + wx] * hr;
        d[13] = r0[fgy * WX + wx] * hr;
        float b[NC];
        blend_cubic<float, 2>(P, d, b);
        float *o = Bc + (r & 1) * T::BROW + cx * T::REC + v * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) o[k] = b[k];
        W0[(r & 1) * T::WROW + cx * NV + v] = h0;
    };

    /* flux work item wi (warp-uniform).  y_only: the y faces between rows
     * j - 1 and j; else the x faces of row j (the first NXB face blocks) and
     * the y faces between rows j and j + 1 */
    const float dtf = (float)dt;
    auto flux_item = [&](int j, int wi, bool y_only) {
        const int lane = tid & 31, g = wi & 1, fb = wi >> 1;
        const bool xd = !y_only && fb < T::NXB;
        const int ix = (xd ? fb : fb - (y_only ? 0 : T::NXB)) * 32 + lane;
        if (xd ? ix >= T::NXF : ix >= T::NYF) return;
        const int yr = y_only ? j : j + 1; /* row of the y faces' upper cells */
        const int fi = x0 + ix;
        if (xd ? (fi > nx || j >= ny) : (fi >= nx || yr > ny)) return;
        const float *cL, *cR, *wL, *wR;
        if (xd) {
            cL = Bc + (j & 1) * T::BROW + ix * T::REC;
            cR = cL + T::REC;
            wL = W0 + (j & 1) * T::WROW + ix * NV;
            wR = wL + NV;
        } else {
            cL = Bc + ((yr - 1) & 1) * T::BROW + (ix + 1) * T::REC;
            cR = Bc + (yr & 1) * T::BROW + (ix + 1) * T::REC;
            wL = W0 + ((yr - 1) & 1) * T::WROW + (ix + 1) * NV;
            wR = W0 + (yr & 1) * T::WROW + (ix + 1) * NV;
        }
        const bool wall = xd ? ((fi == 0 && P.bcs[0][0] >= 2) || (fi == nx && P.bcs[0][1] >= 2))
                             : ((yr == 0 && P.bcs[1][0] >= 2) || (yr == ny && P.bcs[1][1] >= 2));
        const float gm1 = P.fgm1, ih = geo.fih, adm = P.fadm;
        float st[2][NV][3], cw[2][NV];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const float4 *cr = reinterpret_cast<const float4 *>(side ? cR : cL);
            const float4 w4 = *reinterpret_cast<const float4 *>(side ? wR : wL);
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
            float rc[T::REC];
#pragma unroll
            for (int k = 0; k < T::REC / 4; ++k) {
                const float4 q = cr[k];
                rc[4 * k] = q.x;
                rc[4 * k + 1] = q.y;
                rc[4 * k + 2] = q.z;
                rc[4 * k + 3] = q.w;
            }
            /* one evaluation code for both directions: a y face of the cubic
             * P(x, y) is the x face of P(y, x), whose coefficients are P's with
             * x and y swapped (monomials y, x, y^2, xy, x^2, y^3, xy^2, x^2y,
             * x^3); its two derivatives swap back */
            constexpr int swp[NC] = {1, 0, 4, 3, 2, 8, 7, 6, 5};
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float c[NC], out[3];
#pragma unroll
                for (int k = 0; k < NC; ++k) c[k] = xd ? rc[v * NC + k] : rc[v * NC + swp[k]];
                if (side == 0) CubicEval<float, 2, 0, 1>::run(g, c, out);
                else CubicEval<float, 2, 0, 0>::run(g, c, out);
                cw[side][v] = wv[v];
                st[side][v][0] = wv[v] + out[0];
                st[side][v][1] = (xd ? out[1] : out[2]) * ih;
                st[side][v][2] = (xd ? out[2] : out[1]) * ih;
            }
            float s[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) s[v] = st[side][v][0];
            if (!admissible<float, 2>(s, cw[side], gm1, adm)) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    st[side][v][0] = cw[side][v];
                    st[side][v][1] = st[side][v][2] = 0.f;
                }
            }
        }
        /* face frame: normal first; for y faces the momenta and the
         * derivative axes swap (selects on the warp-uniform direction, so
         * every array index stays a constant) */
        const bool yd = !xd;
        float Wl[NV], Wr[NV], dWl[2][NV], dWr[2][NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int u = (v == 1 || v == 2) ? 3 - v : v; /* the swapped variable */
            Wl[v] = yd ? st[0][u][0] : st[0][v][0];
            Wr[v] = yd ? st[1][u][0] : st[1][v][0];
            dWl[0][v] = yd ? st[0][u][2] : st[0][v][1];
            dWr[0][v] = yd ? st[1][u][2] : st[1][v][1];
            dWl[1][v] = yd ? st[0][u][1] : st[0][v][2];
            dWr[1][v] = yd ? st[1][u][1] : st[1][v][2];
        }
        float F[NV], Ft[NV], Wh[NV];
        if (!gks_point<float, 2, NS>(P.fp, dtf, Wl, Wr, dWl, dWr, F, Ft, Wh)) {
            atomicOr(status, ST_FLUX);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = Ft[v] = Wh[v] = 0.f;
        }
        if (wall) F[0] = F[NV - 1] = Ft[0] = Ft[NV - 1] = 0.f;
        float q[3][NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int u = (v == 1 || v == 2) ? 3 - v : v;
            q[0][v] = yd ? F[u] : F[v];
            q[1][v] = yd ? Ft[u] : Ft[v];
            q[2][v] = yd ? Wh[u] : Wh[v];
        }
        float *base = xd ? XF : YF + (yr & 1) * T::YROW;
        float4 *o = reinterpret_cast<float4 *>(base + (ix * 2 + g) * T::FV);
#pragma unroll
        for (int r = 0; r < 3; ++r) o[r] = make_float4(q[r][0], q[r][1], q[r][2], q[r][3]);
    };

    /* stage update of row j, one item per (cell, variable): thread t takes
     * variable t % 4 of cell t / 4 (the four variables of a cell in four
     * neighbouring lanes, which then gather the new state for its
     * admissibility flags).  Faces: x faces of row j, y faces below (slot of
     * row j) and above (slot of row j + 1), each face's Gauss points summed
     * in the order (F0 + F1).  Every thread of the block calls it. */
    auto update_row = [&](int j) {
        const int tx = tid >> 2, v = tid & 3;
        const int gx = x0 + tx;
        const bool valid = tid < NV * TX && gx < nx && j < ny;
        float wn = 1.f;
        if (valid) {
            const float *ylo = YF + (j & 1) * T::YROW, *yhi = YF + ((j + 1) & 1) * T::YROW;
            auto fsum = [&](int q, int vv, int d, int plus) -> float {
                const float *p = d == 0 ? XF + (tx + plus) * 2 * T::FV : (plus ? yhi : ylo) + tx * 2 * T::FV;
                return p[q * NV + vv] + p[T::FV + q * NV + vv];
            };
            wn = mixed_update_var<2, STAGE>(nc, geo.fih, fsum, uc, W, acc, s0, s1, (long)j * nx + gx, v);
        }
        const int base = (tid & 31) & ~3;
        float w4[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) w4[k] = __shfl_sync(0xffffffffu, wn, base + k);
        if (valid && v == 0) mixed_state_flags<2>(P, w4, status);
    };

    /* The sweep, one loop for the whole chunk.  Iteration j: phase A, the
     * cubics of row j + 1 and the update of row j - 1; phase B, the load of
     * input row j + 3 and the faces of row j (the x faces of row j and the y
     * faces between rows j and j + 1).  The first two iterations are the
     * prologue (j = y0 - 2: cubic row y0 - 1 only; j = y0 - 1: cubic row y0
     * and the y faces below row y0), the last one the epilogue (j = y1: the
     * update of row y1 - 1 only).  A cubic row or a face on a chunk's edge
     * is also computed by the neighbouring chunk, and conservation needs
     * both results bit-identical: every cubic and every face therefore comes
     * from the one copy of recon_item / flux_item in this loop.  The row
     * index and its phase are opaque values, so the compiler can neither
     * peel the first iterations nor specialise a copy of the code for them. */
    for (int r = y0 - 2; r <= y0; ++r) load_row(r);
    cp_wait();
    __syncthreads();
#pragma unroll 1
    for (int jl = y0 - 2; jl <= y1; ++jl) {
        int j = jl;
        asm volatile("" : "+r"(j));
        /* 0: a full row; 1: cubics and the y faces below row y0; 2: cubics
         * only; 3: the last update only */
        int phase = j >= y1 ? 3 : (j >= y0 ? 0 : (j == y0 - 1 ? 1 : 2));
        asm volatile("" : "+r"(phase));
        /* A: cubics of row j + 1; update of row j - 1 */
        if (phase != 3)
            for (int it = tid; it < NV * CX; it += NT) recon_item(j + 1, it);
        if (j > y0) update_row(j - 1);
        if (phase == 3) break;
        __syncthreads();
        /* B: faces of row j; input row j + 3 in flight meanwhile (the slot
         * of row j - 1, which phase A no longer reads) */
        if (j + 1 < y1) load_row(j + 3);
        if (phase != 2) {
            const bool yo = phase == 1;
            const int nwi = yo ? 2 * T::NYB : T::NWI;
            for (int wi = tid >> 5; wi < nwi; wi += NT / 32) flux_item(yo ? y0 : j, wi, yo);
        }
        cp_wait();
        __syncthreads();
    }
}

/* one grid: block (bx, by) sweeps strip bx over the rows' chunk by */
template <int STAGE, bool NS, int TX, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fused2d_stage_kernel(KP P, Shadow s0, Shadow s1, double *__restrict__ W,
                                                                 float *__restrict__ acc,
                                                                 const double *__restrict__ dtp,
                                                                 int *__restrict__ status, int rows)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ UpdC uc;
    fused2d_strip<STAGE, NS, TX, NT>(P, fused_geo(P), s0, s1, W, acc, dtp[0], status, blockIdx.x * TX,
                                     blockIdx.y * rows, rows, smem, uc);
}

} // namespace gks
