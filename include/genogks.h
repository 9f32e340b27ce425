/*
 * genogks.h - C ABI of the GB300 (sm_103a) compact gas-kinetic scheme with
 * GENO reconstruction (Zhao & Xu, arXiv 2507.20461).
 *
 * The library advances cell averages W and cell-averaged gradients grad W of
 * the Euler equations on uniform 1D/2D/3D Cartesian grids:
 *   - reconstruction (Sec. 3, Sec. 4.2, Sec. 4.3): GENO, R = chi q^H +
 *     (1 - chi) q^L (Eq. HLP) with the path function chi = tanh(C alpha) /
 *     tanh(C) (Eq. HLP-weight) and the ultimate smoothness indicator alpha
 *     (Eq. HLP-sp); q^H is the compact high-order linear polynomial from the
 *     averages and averaged gradients of the face neighbours (p^7 in 1D,
 *     Eq. 8th-compact-HLP; a least-squares cubic on Cartesian cells in 2D/3D,
 *     Eq. 6th-compact-HLP), q^L the ENO-type combination of sub-stencil
 *     polynomials (Eq. HLP-q-loworder);
 *   - flux (Sec. 2): the time-dependent gas-kinetic (BGK) distribution at
 *     every face Gauss point, integrated in time;
 *   - update (Sec. 2, Eq. semifvs, Eq. slope): two-stage fourth-order time
 *     stepping of the averages, and the averaged gradients from the interface
 *     states by the Gauss theorem.
 * The paper defers the flux and the time stepping to earlier work; the
 * formulations used are stated beside each entry point.
 *
 * Conventions for every call:
 *   - Layouts are row-major with x fastest.  W[v][k][j][i] holds the nv =
 *     dim + 2 conservative variables (rho, rho u, [rho v, [rho w]], rho E);
 *     G[d][v][k][j][i] holds dW_v/dx_d in physical units.  No ghost cells.
 *   - Faces of direction d have extent n_d + 1 along d and n_e across; face
 *     arrays list all x faces, then y faces, then z faces (F faces in total,
 *     see gks_face_count).  Face (i,j,k) of direction d lies between cell
 *     (i,j,k) - e_d (its "minus" side) and cell (i,j,k) (its "plus" side).
 *   - Gauss points per face: 1 (1D); 2 (2D) at tangential coordinates
 *     -/+ h/(2 sqrt 3); 4 (3D) as g = a + 2 b, a for the lower tangential axis.
 *   - Pointers are borrowed for the duration of the call.  A pointer flagged
 *     on_device must be device memory of the handle's device; otherwise it is
 *     host memory.  The library owns every buffer it allocates.
 *   - All device work is ordered on the handle's stream (gks_opts_t.stream).
 *     gks_step and gks_step_cfl return before the work finishes; errors of
 *     that work (the status word) are reported by the next synchronising call
 *     (gks_get_state, gks_status, gks_max_wavespeed).
 *   - Return value: GKS_OK (0) or a negative GKS_ERR_* code; gks_last_error
 *     gives a message.  No call aborts the process; no call falls back to the
 *     CPU.
 */
#ifndef GENOGKS_H
#define GENOGKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GKS_OK 0
#define GKS_ERR_ARG (-1)         /* invalid argument                                        */
#define GKS_ERR_CUDA (-2)        /* a CUDA call failed (message in gks_last_error)           */
#define GKS_ERR_OOM (-3)         /* device allocation failed or workspace too small          */
#define GKS_ERR_NONPHYSICAL (-4) /* rho <= 0, p <= 0 or a non-finite value was produced      */
/* (-5) is not used: no kernel of this library waits on another block or
 * on the host, so no device wait can time out */
#define GKS_ERR_UNSUPPORTED (-6) /* combination not provided (e.g. order 8 in 2D)           */

/* Status-word bits (gks_status): which condition was seen by the device. */
#define GKS_ST_RHO 1   /* a cell average with rho <= 0     */
#define GKS_ST_P 2     /* a cell average with p <= 0       */
#define GKS_ST_NAN 4   /* a non-finite cell average        */
#define GKS_ST_FLUX 8  /* a face state the flux could not use (after the fallback) */

typedef struct {
    int dim;         /* 1, 2 or 3                                               */
    int n[3];        /* cells per axis; unused axes must be 1                    */
    double lo[3];    /* domain [lo, hi] per axis; the cell size h must be equal  */
    double hi[3];    /*   on all active axes                                     */
} gks_grid_t;

/* Boundary condition on every side, by ghost cells that are index maps:
 * periodic wraps; transmissive mirrors every variable evenly (the normal
 * derivative changes sign); reflective (a slip wall) mirrors likewise but
 * negates the momentum normal to the wall (used by the paper's blast wave,
 * Sec. 6.6); no-slip (an adiabatic wall at rest, for the Navier-Stokes
 * equations, Sec. 6.9) negates every momentum component. */
typedef enum {
    GKS_BC_PERIODIC = 0,
    GKS_BC_TRANSMISSIVE = 1,
    GKS_BC_REFLECTIVE = 2,
    GKS_BC_NOSLIP = 3
} gks_bc_t;

typedef struct {
    int precision;    /* 0: FP64 throughout; 1: reconstruction and flux in FP32;
                         the averages accumulated exactly (double-float face sums,
                         FP64 state); the averaged gradients, recomputed each
                         stage from the FP32 interface states (Gauss theorem),
                         in FP32 and widened to FP64 when read                   */
    int limiter;      /* 0: GENO; 1: linear scheme (chi = 1); 2: WENO-Z weights
                         (Eq. wgt-WENO-Z); 3: TENO weights (Eq. wgt-TENO-1,
                         Eq. wgt-TENO-2).  2 and 3 use GENO's candidates (the
                         high-order polynomial and the sub-stencil polynomials)
                         in the adaptive-order combination
                         (w0/d0) q^H + sum_k (w_k - (w0/d0) d_k) p_k           */
    double C;         /* path-function steepness, Eq. HLP-weight (20)            */
    double eps;       /* regulariser of the indicators, Eq. HLP-sp (1e-15)       */
    double C0;        /* weight of the central 1D sub-stencil, Sec. 3.3 (8)      */
    double c1_tau;    /* numerical collision time tau_n = c1 dt + c2 |pl - pr| /  */
    double c2_tau;    /*   (pl + pr) dt in the relaxation factor (0.05, 1)        */
    double adm_delta; /* a reconstructed face state whose rho or p is not above
                         adm_delta times its cell's is replaced by the cell
                         average with zero slopes (0.3)                          */
    void *stream;     /* cudaStream_t for all work; NULL = legacy default stream */
    void *workspace;  /* optional caller-owned device memory for all buffers     */
    size_t workspace_bytes; /* its size; see gks_workspace_bytes                 */
    double mu;        /* dynamic viscosity: 0 solves the Euler equations; > 0 the
                         Navier-Stokes equations with Prandtl number 1 (Sec. 2,
                         Sec. 6.9): physical collision time mu / p in the BGK
                         solution, added to tau_n, and the viscous time-step
                         limit in gks_step_cfl (0)                               */
    double ao_d0;     /* limiters 2, 3: linear weight d0 of the high-order
                         candidate; the sub-stencils share 1 - d0 (0.85)         */
    double teno_ct;   /* limiter 3: cut-off C_T (1e-6; the paper uses 1e-3 for
                         the Titarev-Toro problem), Sec. 5.1                     */
    int stage_kernels; /* how a 2D mixed-precision stage runs (gks_step,
                         gks_step_cfl): 0 = three kernels (per-cell
                         reconstruction, per-direction face flux, update) with
                         the blended cubics and face sums in device memory;
                         1 = one fused kernel per stage (reconstruction, flux
                         and update of a strip swept row by row in shared
                         memory).  Both give the same result to FP32 rounding.
                         Other precisions and dimensions always use the
                         three-kernel path (0)                                   */
} gks_opts_t;

typedef struct gks_ctx *gks_handle_t;

/* Fill *o with the defaults above (precision 0, limiter 0, stream NULL,
 * no workspace). */
void gks_default_opts(gks_opts_t *o);

/* Device bytes geno_gks_create needs for this grid and precision (state,
 * stage buffers, reconstruction coefficients, face fluxes).  0 on a bad grid. */
size_t gks_workspace_bytes(const gks_grid_t *grid, int precision);

/* Number of faces F (all directions) of the grid; -1 on a bad grid. */
long gks_face_count(const gks_grid_t *grid);

/* Create a solver for the Euler equations (opts->mu = 0) or the Navier-Stokes
 * equations (opts->mu > 0) with ratio of specific heats gamma (> 1) on `grid`
 * with boundary condition `bc` on every side.
 * order: 8 in 1D (Sec. 4.2, the compact GKS), 4 in 2D/3D (Sec. 4.3); in 1D
 * also 5 or 6: the non-compact GENO finite-volume schemes (Sec. 4.1) with
 * the HLLC flux and classical four-stage RK4 (FP64, inviscid, limiter 0 or 1;
 * otherwise GKS_ERR_UNSUPPORTED).  They use the cell averages only: G is
 * ignored on input and returned unchanged; geno_reconstruct writes zero
 * derivatives, gks_flux the HLLC flux in the F slot and zeros in the dF/dt
 * and W(dt/2) slots, and gks_step takes one RK4 step.  Any other order
 * gives GKS_ERR_UNSUPPORTED.  opts may be NULL (defaults).  If opts->workspace is
 * given it must hold gks_workspace_bytes bytes (else GKS_ERR_OOM) and the
 * library allocates no state memory of its own.  The state starts at zero;
 * set it with gks_set_state.  *out receives the handle. */
int geno_gks_create(const gks_grid_t *grid, double gamma, int order, gks_bc_t bc, const gks_opts_t *opts,
                    gks_handle_t *out);

/* As geno_gks_create with a boundary condition per side: bc[6] =
 * {x low, x high, y low, y high, z low, z high} (entries of inactive axes are
 * ignored).  Periodic must be given on both sides of an axis or on neither
 * (else GKS_ERR_ARG).  Walls on different sides may differ, e.g. the paper's
 * viscous shock tube (Sec. 6.9): no-slip on three sides and a slip
 * (reflective) symmetry line on top. */
int geno_gks_create_sides(const gks_grid_t *grid, double gamma, int order, const gks_bc_t *bc, const gks_opts_t *opts,
                          gks_handle_t *out);

/* Copy the state in: W (nv x cells) and G (dim x nv x cells) doubles in the
 * layouts above (host or device memory per on_device).  Clears the status
 * word.  Synchronous with respect to the caller's buffers. */
int gks_set_state(gks_handle_t h, const double *W, const double *G, int on_device);

/* Copy the state out (same layouts).  Synchronises the stream; returns
 * GKS_ERR_NONPHYSICAL (after copying) if the status word is set. */
int gks_get_state(gks_handle_t h, double *W, double *G, int on_device);

/* GENO interface states of the current state at every face Gauss point
 * (Sec. 3, Eq. HLP; after the admissibility fallback described at
 * adm_delta): face_states[side][v][c][g][face] doubles, side 0 = minus cell,
 * c = 0 value, 1 + e = dW/dx_e (physical, global axes).  2 * nv * (dim + 1) *
 * ng * F doubles.  Synchronises the stream. */
int geno_reconstruct(gks_handle_t h, double *face_states, int on_device);

/* Gas-kinetic interface quantities of the current state for a step dt > 0
 * (Sec. 2): face_flux[q][v][g][face] doubles, q = 0 the flux F recovered at
 * t^n from the time integrals over dt/2 and dt (F = (4 F(dt/2) - F(dt)) / dt),
 * q = 1 its time derivative (4 (F(dt) - 2 F(dt/2)) / dt^2), q = 2 the
 * interface state W(dt/2) used by the gradient update; the normal flux in
 * global variable order.  3 * nv * ng * F doubles.  Synchronises the stream. */
int gks_flux(gks_handle_t h, double dt, double *face_flux, int on_device);

/* One two-stage fourth-order step of size dt > 0 (Sec. 2):
 *   W*  = W^n + dt/2 L(F^n) + dt^2/8 L(dF^n/dt),  G* from W^n_face(dt/2);
 *   W^{n+1} = W^n + dt L(F^n) + dt^2/6 (L(dF^n/dt) + 2 L((dF/dt)^s)),
 *   G^{n+1} from W^s_face(dt/2)   (Eq. slope), superscript s = from (W*, G*),
 * with L(F)_j = -(1/|Omega_j|) sum over the faces and Gauss points
 * (Eq. semifvs).  Asynchronous. */
int gks_step(gks_handle_t h, double dt);

/* nsteps steps, each with dt = cfl h / max_cells max_d(|u_d| + c) computed on
 * the device (no host round trip); with opts->mu > 0 also at most
 * cfl h^2 / (2 (m - 1) nu_max), nu_max = mu / min_cells rho (Sec. 6; the
 * factor 2 (m - 1) is taken as 2 in 1D).  Asynchronous. */
int gks_step_cfl(gks_handle_t h, double cfl, int nsteps);

/* max over cells and axes of |u_d| + c of the current state.  Synchronises. */
int gks_max_wavespeed(gks_handle_t h, double *out);

/* Synchronise the stream and return the status word (>= 0, GKS_ST_* bits),
 * or a negative GKS_ERR_* code if the device work itself failed. */
int gks_status(gks_handle_t h);

/* Kernel profiler.  While enabled, every kernel the handle launches is
 * bracketed by CUDA events on the handle's stream; gks_profile_read
 * synchronises and returns, for one kernel class, the number of launches and
 * their summed device time in milliseconds since the last reset.  Classes:
 * GKS_KC_RECON (per-cell reconstruction), GKS_KC_FACE (per-face
 * reconstruction and gas-kinetic flux), GKS_KC_UPDATE (stage update),
 * GKS_KC_DT (wave-speed reduction and time step), GKS_KC_STAGE (the fused
 * reconstruction + flux + update kernel of one stage). */
#define GKS_KC_RECON 0
#define GKS_KC_FACE 1
#define GKS_KC_UPDATE 2
#define GKS_KC_DT 3
#define GKS_KC_STAGE 4
/* on != 0 starts (0 stops) the bracketing; reset != 0 zeroes the counts.
 * GKS_ERR_ARG for a NULL handle, GKS_ERR_OOM / GKS_ERR_CUDA if the events
 * cannot be created. */
int gks_profile_enable(gks_handle_t h, int on, int reset);
/* launches and ms may be NULL (that output is skipped).  GKS_ERR_ARG for a
 * NULL handle or a class outside 0..7. */
int gks_profile_read(gks_handle_t h, int kernel_class, long *launches, double *ms);

/* Measured throughput of one arithmetic pipe of the current device, the
 * denominator of the stage kernels' rooflines (the paper has no
 * counterpart: measurement infrastructure).  kind 0: FP32 fused multiply-add
 * (2 flops each), 1: FP64 fused multiply-add, 2: the FP32 special-function
 * unit (ex2.approx, 1 op each), 3: FP32 fused multiply-add issued as packed
 * two-lane instructions (fma.rn.f32x2, 4 flops each).  A grid of 8 blocks of 256 threads per SM
 * runs iters x 32 operations per thread on eight independent chains; the
 * second of two launches is timed with CUDA events on `stream` (NULL = the
 * legacy default stream), which the call synchronises.  *ops_per_s receives
 * flops (or ops) per second.  Allocates a small scratch buffer with
 * cudaMallocAsync on `stream` and frees it before returning.
 * GKS_ERR_ARG for a bad kind, iters < 1 or NULL output; GKS_ERR_OOM /
 * GKS_ERR_CUDA if the allocation or a launch fails. */
int gks_pipe_probe(int kind, int iters, double *ops_per_s, void *stream);

/* Free everything the handle owns (not a caller workspace).  NULL is a no-op. */
int gks_destroy(gks_handle_t h);

/* Message of the last error on this handle ("" if none); valid until the next
 * call on the handle.  h == NULL gives the last create error of this thread. */
const char *gks_last_error(gks_handle_t h);

/* ------------------------------------------------------------------ */
/* Flux without allocation                                              */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory (code running where cudaMalloc is not
 * available or not allowed, such as a plugin or callback that must not own
 * memory, a process whose device allocator belongs to another framework, or
 * a latency-critical loop that cannot afford an allocation's implicit
 * synchronisation).
 *
 * Same result as gks_flux on a 2D FP64 grid of nx x ny cells of size h:
 * face_flux[q][v][g][face] (3 * 4 * 2 * F doubles), from the state W
 * (4 x nx x ny) and G (2 x 4 x nx x ny) doubles.  W, G and face_flux are
 * caller-owned DEVICE memory of the current device; the work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call
 * synchronises that stream before it returns.  opts may be NULL (defaults);
 * opts->precision must be 0 and opts->stream / workspace are ignored.
 *
 * It allocates nothing: the only scratch it needs lives in one static device
 * array of 4,147,456 bytes (about 4 MiB) that every GPU which loads the
 * library holds until the process exits, which limits the grid to
 * (nx + 2) * (ny + 2) <= 14400 cells including the one-cell ghost ring (for
 * example 118 x 118); larger grids return
 * GKS_ERR_ARG, as do invalid sizes, h, gamma, bc, dt, NULL pointers and the
 * scheme constants geno_gks_create rejects.
 * GKS_ERR_UNSUPPORTED: precision != 0 or mu != 0 (Euler flux only).
 * GKS_ERR_NONPHYSICAL: a face state the
 * flux could not use.  GKS_ERR_CUDA: a CUDA call failed.
 *
 * The first call on a device looks up the device address of that array
 * (with the device current).  Every call copies the status word to the host
 * and synchronises `stream` before it returns.
 * Every call on a device shares the array and leaves its contents behind;
 * calls that overlap on the GPU (other streams or unordered host threads)
 * race on it and must be serialised by the caller. */
int gks_flux_2d_static(int nx, int ny, double h, double gamma, gks_bc_t bc, const gks_opts_t *opts, const double *W,
                       const double *G, double dt, double *face_flux, void *stream);

/* How much of the high-order linear reconstruction the nonlinear weights keep,
 * evaluated by the reconstruction kernels' own device code (Sec. 3.1 path
 * function, Eq. HLP-weight; Sec. 3.2 ultimate smoothness indicator,
 * Eq. HLP-sp; Sec. 5.1-5.2 WENO-Z / TENO weights and the linearity parameter
 * chi = min_k w_k / d_k, Eq. linearity-paprameter).  For each of n sets i:
 *   IS[i * k .. i * k + k - 1]  the candidates' smoothness indicators
 *                               (k = 2..8), tau[i] the indicator IS^tau;
 *   limiter 0 (GENO): chi[i] = tanh(C alpha) / tanh(C) with IS^H = max,
 *     IS^L = min of the set and exponent r (2 structured, 3 unstructured);
 *   limiter 2 (WENO-Z, tau_Z = tau[i]) or 3 (TENO, cut-off opts->teno_ct):
 *     weights over the k candidates with equal linear weights 1/k,
 *     chi[i] = min_k w_k k;
 *   limiter 1: chi[i] = 1.
 * IS, tau and chi are device pointers.  opts (NULL = defaults) supplies C,
 * eps, teno_ct, and precision (0: FP64 arithmetic, 1: FP32 as in the
 * mixed-precision kernels).  Runs on `stream` and synchronises it.
 * GKS_ERR_ARG on bad arguments, GKS_ERR_CUDA on a launch failure. */
int geno_linearity(const gks_opts_t *opts, int limiter, int r, int k, long n, const double *IS, const double *tau,
                   double *chi, void *stream);

/* ------------------------------------------------------------------ */
/* Batched mode: many independent 2D grids of uneven sizes              */
/* ------------------------------------------------------------------ */
typedef struct gks_batch_ctx *gks_batch_t;

/* nbatch independent 2D grids (all with boundary condition bc), grid b with
 * nx[b] x ny[b] cells of size hs[b]; order 4 (Sec. 4.3 on Cartesian cells).
 * Every grid keeps its own CFL time step.  opts may be NULL; opts->precision
 * and the scheme constants apply to every grid, opts->stream orders the
 * batch's work after the caller's (the batch runs on an internal stream that
 * can be captured); opts->workspace and opts->mu != 0 (the Euler flux only)
 * are not supported (GKS_ERR_UNSUPPORTED).
 * The library allocates one device buffer for all grids. */
int gks_batch_create(int nbatch, const int *nx, const int *ny, const double *hs, double gamma, gks_bc_t bc,
                     const gks_opts_t *opts, gks_batch_t *out);

/* State of grid b (layouts as for a single 2D grid).  Host or device memory.
 * set_state clears that grid's status word; get_state copies the state and
 * then returns GKS_ERR_NONPHYSICAL if that grid's status word is set. */
int gks_batch_set_state(gks_batch_t b, int grid, const double *W, const double *G, int on_device);
int gks_batch_get_state(gks_batch_t b, int grid, double *W, double *G, int on_device);

/* nsteps steps of every grid, grid b with dt_b = cfl h_b / (its max |u_d| + c)
 * computed on the device.  Mixed precision: per stage one persistent launch
 * of the fused stage kernel (reconstruction, flux and update through shared
 * memory), its blocks taking strips of a list spanning every grid from a
 * work counter; FP64: per stage three
 * persistent kernels (per-cell reconstruction, face flux, update) walk tile
 * lists spanning all grids.  The first call picks the tile sizes (rows per
 * strip) and block sizes by timing candidates (an autotuner; only scratch
 * buffers are written), then records one step into a CUDA graph; later calls
 * replay the graph (a new cfl re-records it).  The tuner's choices are cached
 * per (dimension, precision, limiter, size class of the batch, SM count): in
 * the process, and in the file named by the environment variable
 * GKS_TUNE_CACHE if set (one JSON object per line, appended); a batch whose
 * size class is cached skips the timing.  Asynchronous with respect to the
 * host; ordered after the work already on opts->stream, and later work on
 * that stream waits for it. */
int gks_batch_run(gks_batch_t b, double cfl, int nsteps);

/* JSON text of the launch shapes the tuner picked (per kernel class: block
 * size, items per tile or rows per strip, persistent blocks, measured ms;
 * "cached": true and no timings when they came from the cache, with the
 * size-class key); "" before the first gks_batch_run.  Owned by the handle. */
const char *gks_batch_tuning(gks_batch_t b);

/* Synchronise and return the status word (as gks_status): the OR of every
 * grid's status word. */
int gks_batch_status(gks_batch_t b);
/* Synchronise and copy the status word of every grid (as gks_status; 0 for
 * a grid whose states stayed admissible) to status[0 .. n-1], host memory.
 * Each grid's word is cleared by gks_batch_set_state of that grid.
 * GKS_ERR_ARG for a NULL handle or output, or n other than the number of
 * grids; GKS_ERR_CUDA if the copy fails. */
int gks_batch_grid_status(gks_batch_t b, int *status, int n);

/* Wait for the batch's work and free everything it owns.  NULL is a no-op. */
int gks_batch_destroy(gks_batch_t b);
/* Message of the last error on this batch ("" if none); b == NULL gives the
 * last create error of this thread.  Owned by the library. */
const char *gks_batch_last_error(gks_batch_t b);

#ifdef __cplusplus
}
#endif
#endif
