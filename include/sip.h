/*
 * sip.h -- C ABI of the GB300 (sm_103a) Stone SIP solver, libsip.so.
 *
 * The operation: Stone's strongly implicit procedure (SIP), the linear solver
 * of the FASTEST-3D finite-volume code (Scheit, Hager, Treibig, Becker,
 * Wellein, arXiv:1303.4538, Sec. 1; its factorisation lu3d, residual and
 * forward substitution resforward3d and backward substitution backward3d are
 * the routines of Tables 1-4), for the 7-point system A x = b of each
 * hexahedral block:
 *
 *   factorisation  L U = A + N   (Stone's alpha-weighted auxiliary matrix N)
 *   iteration      r = b - A x;  L y = r (ascending);  U d = y (descending);
 *                  x <- x + d;   relres = ||r||_2 / ||b||_2
 *
 * Following the paper's solver redesign (Sec. 4.1: the solver owns its
 * coefficient copies, the factorisation is computed once before the
 * relaxation and reused), sip_factor builds a plan that owns reordered copies
 * of A and the factors; sip_iterate / sip_solve relax with them.
 *
 * Conventions
 *   - Cell (i,j,k), 0-based; natural layout p = i + nx*(j + ny*k) (i fastest).
 *   - Lower neighbours W=(i-1,j,k), S=(i,j-1,k), B=(i,j,k-1); upper E, N, T.
 *   - A holds matrix entries (diagonal AP, off-diagonals AW..AT, normally <= 0;
 *     the paper's Listing 1 stores a_nb = -A_nb).  A coefficient that points
 *     outside its block is ignored (treated as 0), except on a declared
 *     interface (sip_interface), where it couples to the neighbour block.
 *   - All array pointers are DEVICE pointers on the context's device unless
 *     stated otherwise.  Host pointers are marked "host".
 *   - All work is ordered on the context's stream.  Functions that return host
 *     values synchronise that stream before returning.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns SIP_ERR_NO_DEVICE.
 *
 * Return codes: SIP_OK (0), SIP_NOT_CONVERGED (1, outputs valid), or a
 * negative error.  After an error, sip_last_error(ctx) describes it.
 * A context is not thread-safe: one host thread at a time per context.
 */
#ifndef SIP_H
#define SIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIP_OK 0
#define SIP_NOT_CONVERGED 1
#define SIP_ERR_INVALID_ARG (-1)
#define SIP_ERR_NO_DEVICE (-2)
#define SIP_ERR_CUDA (-3)
#define SIP_ERR_OOM (-4)
#define SIP_ERR_BREAKDOWN (-5)      /* zero/non-finite pivot or denominator in the factorisation */
#define SIP_ERR_DEVICE_TIMEOUT (-6) /* a bounded device-side wait gave up (no hang) */
#define SIP_ERR_BUSY (-7)           /* server queue full */
#define SIP_ERR_NOT_FOUND (-8)      /* unknown ticket */

typedef struct sip_ctx sip_ctx;
typedef struct sip_plan sip_plan;

/* Arithmetic of the relaxation sweeps. */
typedef enum {
  SIP_MODE_F64 = 0,         /* FP64 sweeps, FP64 factors */
  SIP_MODE_F32_REFINED = 1, /* FP32 sweeps inside an FP64 residual / refinement loop */
  SIP_MODE_F32 = 2          /* FP32 only (the paper's single-precision relaxation, Sec. 4.1): rhs
                               and solution converted to single, residual, norm and sweeps in
                               FP32, the result converted back; relres is that of the FP32
                               residual and stagnates near the single-precision level */
} sip_mode;

/* One block's system.  Lifetimes: the coefficient arrays are read during
 * sip_factor only (the plan keeps reordered copies).  b and x must stay
 * valid, and b unmodified, during every sip_iterate / sip_solve call on the
 * plan; x is read as the initial guess and overwritten with the result. */
typedef struct {
  int32_t nx, ny, nz;      /* >= 1 each; nx*ny*nz < 2^31 */
  int32_t coef_dtype;      /* 0: coefficient arrays are double, 1: float */
  const void *ap, *aw, *ae, *as, *an, *ab, *at; /* device, natural layout, N entries each.
                              If symmetric != 0, aw/as/ab may be NULL: then
                              AW(P) = AE(W), AS(P) = AN(S), AB(P) = AT(B). */
  const double *b;         /* device, natural layout, N doubles */
  double *x;               /* device, natural layout, N doubles */
  int32_t symmetric;       /* 1: A is symmetric (pressure-correction systems, Sec. 4.1) */
} sip_block_desc;

/* Interface between two blocks of a multi-block mesh (block-structured mesh,
 * Sec. 1; exchange at block boundaries, Sec. 4.2): the +x face of blk_lo touches
 * the -x face of blk_hi on the rectangle j < nj, k < nk (both anchored at
 * j = k = 0).  Across it, blk_lo's AE at i = nx-1 and blk_hi's AW at i = 0
 * (for symmetric blocks: blk_lo's AE on both sides) couple the two blocks;
 * the coupling enters each block's residual with the neighbour's values from
 * the previous iteration (lagged, block Jacobi), so relres and the stop rule
 * refer to the coupled system while each block relaxes with its own factors.
 * In SIP_MODE_F32_REFINED the inner FP32 iterations solve the coupled
 * correction system: after every inner iteration the blocks exchange the
 * interface values of their FP32 correction, whose coupling terms (entries
 * rounded to FP32) enter the next inner residual.
 * Rules: 0 <= blk_lo, blk_hi < nblocks, blk_lo != blk_hi; 1 <= nj <= both
 * blocks' ny, 1 <= nk <= both blocks' nz; each block face carries at most one
 * interface.  Otherwise sip_factor returns SIP_ERR_INVALID_ARG. */
typedef struct {
  int32_t blk_lo, blk_hi;
  int32_t nj, nk;
} sip_interface;

typedef struct {
  double alpha;            /* Stone's cancellation parameter, 0 <= alpha <= 1 (e.g. 0.92) */
  int32_t mode;            /* sip_mode */
  int32_t inner_iters;     /* SIP_MODE_F32_REFINED: FP32 iterations per FP64 correction (>= 1) */
  int64_t max_spin;        /* polls before a device wait gives up (<= 0: default 2^22) */
  int32_t tile_j, tile_k;  /* column-tile shape of the sweeps (0: chosen by the autotuner) */
  int32_t stages;          /* depth of the sweeps' shared-memory prefetch ring: 0 (auto), 3, 4 or 6 */
  int32_t debug_stall;     /* test hook: 1 makes the sweeps wait for a tag no producer
                              writes, so the bounded waits time out (SIP_ERR_DEVICE_TIMEOUT) */
  int32_t graphs;          /* 1: queue iterations by replaying CUDA graphs captured on the
                              context's stream (one replay per 16 iterations; needs a
                              non-NULL stream, ignored while profiling); 0: launch by launch */
  int32_t rows_per_thread; /* rows of a column tile each sweep thread walks (the tile is
                              32 x rows_per_thread * warps): 0 (auto: 1 or 2), 1, 2 or 4 */
  int32_t autotune;        /* 1 (with tile_k, rows_per_thread and stages all 0): sip_factor builds
                              the launch model's best four tile shapes (sip_tile_model), times their forward +
                              backward sweeps on the plan's own work vectors and keeps the
                              fastest plan; with the environment variable SIP_AUTOTUNE_CACHE
                              naming a file, a result for the same signature (GPU SM count,
                              mode, symmetry, coefficient type, block sizes) is read from it
                              and new results are appended.  0: the cost model alone. */
} sip_options;

/* Fills *opt with defaults: alpha 0.92, SIP_MODE_F64, inner_iters 4. Host pointer. */
void sip_default_options(sip_options *opt);

/* Creates a context on CUDA device `device`, ordering all work on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  *ctx (host) receives the
 * handle.  The context's plans take device memory from its own
 * stream-ordered pool (allocated and freed in `stream` order), so creating or
 * destroying a plan does not synchronise the device.  The pool keeps freed
 * memory cached for the next plans: at least 1 GiB, and as much as the
 * largest plan creation on this context used at once (its footprint plus the
 * factorisation's temporary input), so re-creating a plan of the same size
 * maps no new memory; sip_destroy returns it all.
 * Errors: SIP_ERR_NO_DEVICE, SIP_ERR_INVALID_ARG. */
int sip_create(sip_ctx **ctx, int device, void *stream);
/* Synchronises the stream and frees the context, its pool and cached pinned
 * blocks.  Destroy the context's plans first. */
int sip_destroy(sip_ctx *ctx);
/* Synchronises the stream and returns the pool's cached memory (everything
 * not held by a live plan) to the device; the cache limit drops back to
 * 1 GiB until the next plan creation raises it.  Live plans are unaffected.
 * Errors: SIP_ERR_INVALID_ARG (ctx NULL), SIP_ERR_CUDA. */
int sip_trim(sip_ctx *ctx);
/* Description of the last error on ctx (never NULL; valid until the next
 * call on this thread).  ctx == NULL: the last sip_create failure. */
const char *sip_last_error(sip_ctx *ctx);

/* Validates the blocks, copies their coefficients into the plan's plane
 * layout, computes Stone's factorisation (lu3d, Sec. 4.1: once, kept for
 * all later relaxations) and returns the plan in *plan (host).  The plan owns
 * all device memory it allocates.  nifaces > 0 couples blocks (batched mesh).
 * Errors: SIP_ERR_INVALID_ARG, SIP_ERR_OOM, SIP_ERR_CUDA, SIP_ERR_BREAKDOWN,
 * SIP_ERR_DEVICE_TIMEOUT. */
int sip_factor(sip_ctx *ctx, const sip_block_desc *blocks, int nblocks,
               const sip_interface *ifaces, int nifaces, const sip_options *opt,
               sip_plan **plan);

/* Runs exactly `niters` SIP iterations on every block's x (resforward3d then
 * backward3d per iteration, Tables 1-4).  relres_out (host, nullable) receives
 * relres of x before the last update (the norm computed by the last
 * iteration's residual).  In SIP_MODE_F32_REFINED an "iteration" is one FP64
 * correction of inner_iters FP32 iterations.  Errors as above. */
int sip_iterate(sip_plan *plan, int niters, double *relres_out);

/* Iterates until relres(x_n) <= rtol or n == max_iters, where relres(x_n) is
 * computed from the residual of x_n and x_n is returned (the forward result
 * of the deciding iteration is discarded).  iters_out (host, nullable) = n,
 * the number of updates applied (FP64 corrections in the refined mode);
 * relres_out (host, nullable) = relres(x_n).  Returns SIP_OK or
 * SIP_NOT_CONVERGED. */
int sip_solve(sip_plan *plan, double rtol, int max_iters, int *iters_out, double *relres_out);

/* Copies the relres history of the last sip_iterate/sip_solve call into
 * host_out (host, up to cap doubles); *n_out (host) = entries available. */
int sip_get_history(sip_plan *plan, double *host_out, int cap, int *n_out);

/* Writes block `blk`'s FP64 factors in natural layout into seven device
 * arrays of N doubles: LB, LW, LS, 1/LP, UN, UE, UT (test and inspection aid). */
int sip_export_factors(sip_plan *plan, int blk, double *const out[7]);

/* Plane layout used by the sweeps (host-only helper, no device needed):
 * fills rbT (host, nz * (nx+ny+nz-2) int32) so that cell (i,j,k) is stored at
 * rbT[k*(nx+ny+nz-2) + i+j+k] + j of its block's plan arrays.  Cells of one
 * hyperplane i+j+k = s are contiguous, rows k ascend within a plane and j
 * ascends within a row.  Entries of empty rows are INT32_MIN. */
int sip_plane_layout(int nx, int ny, int nz, int32_t *rbT);

/* Launch model of the tile-shape chooser (host-only helper, no device
 * needed): the modelled duration, in SM cycles (*cycles_out, host), of one
 * forward or backward sweep launch over `nblocks` blocks (dims: host,
 * nx ny nz per block) cut into 32 x (rows_per_thread * warps) column tiles
 * that `ctas` resident CTAs on `nsm` SMs claim in the launch's order
 * (anti-diagonal waves, blocks interleaved).  fp64 = 1: FP64 sweeps, 0: FP32.
 * The tile wavefront is the one of the hyperplane ordering of Sec. 2; the
 * per-step cost is fitted on GB300.  SIP_ERR_INVALID_ARG for dims < 1, a
 * rows_per_thread outside {1, 2, 4}, warps outside 1..16, ctas or nsm < 1. */
int sip_tile_model(const int32_t *dims, int nblocks, int rows_per_thread, int warps, int ctas, int nsm, int fp64,
                   double *cycles_out);

/* ||b - A x||_2 (*rnorm_out) and ||b||_2 (*bnorm_out) of one block, computed
 * directly on the descriptor's natural-layout arrays (the residual of
 * resforward3d, Sec. 4.1 / Table 1, without a plan): FP64 arithmetic (FP32
 * coefficients are widened), sums in a fixed order that depends only on N,
 * so results are bitwise reproducible.  Coefficients that point outside the
 * block are ignored; symmetric != 0 reads AW/AS/AB as AE(W)/AN(S)/AT(B).
 * Only blk->ap..at, b, x, dims, coef_dtype and symmetric are read; nothing is
 * written but the outputs.  rnorm_out, bnorm_out: host, nullable.  Allocates
 * and frees 16 bytes of device scratch per 4096 cells for the call and
 * synchronises the context's stream.  Errors: SIP_ERR_INVALID_ARG (bad
 * descriptor), SIP_ERR_OOM, SIP_ERR_CUDA. */
int sip_residual_norm(sip_ctx *ctx, const sip_block_desc *blk, double *rnorm_out, double *bnorm_out);

/* Allocation-free variant of sip_residual_norm (this library's addition; the
 * paper has no counterpart).  Same arithmetic, chunking and summation order,
 * so the same bits, but:
 *   - norms_dev (device, 2 doubles, 8-byte aligned, must not overlap the
 *     block's arrays) receives ||b - A x||_2 and ||b||_2 in stream order; the
 *     call neither synchronises nor copies to the host;
 *   - no device memory is allocated or freed: the partial sums live in one
 *     fixed 256 KiB array of the library per device, so blocks are limited to
 *     SIP_NOALLOC_MAX_CELLS cells (larger: SIP_ERR_INVALID_ARG, nothing
 *     launched).  No part of that array needs to start at zero;
 *   - calls whose work may overlap on one device (other streams, contexts or
 *     threads) race on that array: the caller must order them;
 *   - the first call on each device looks the array's address up (and may
 *     load the library's device code); make it before any stream capture
 *     begins and outside time-critical code.  The address is cached for the
 *     life of the device's primary context: after cudaDeviceReset, calls on
 *     that device are unsafe until the process restarts;
 *   - norms_dev must be device (or managed) memory of the context's device;
 *     host pointers, other devices' memory and unaligned pointers are
 *     rejected (SIP_ERR_INVALID_ARG).
 * Errors: SIP_ERR_INVALID_ARG, SIP_ERR_CUDA. */
#define SIP_NOALLOC_MAX_CELLS 67108864LL
int sip_residual_norm_noalloc(sip_ctx *ctx, const sip_block_desc *blk, double *norms_dev);

/* ---- Pressure-correction coefficient assembly ---------------------------
 * The routine celp2 of Sec. 3.1 (Table 1) builds the symmetric
 * pressure-correction system (Sec. 4.1) that SIP then solves; the paper does
 * not print its discretisation.  This library's stated geometry: one block of
 * nx x ny x nz hexahedral cells on a rectilinear grid, natural layout
 * p = i + nx (j + ny k).  Inputs (device memory of the context's device, FP64):
 *   dx[nx], dy[ny], dz[nz]   cell widths;
 *   rho[n], g[n]             per cell: density and the momentum equation's V / a_P;
 *   ux[(nx+1) ny nz]         x-face normal velocities u*, face i = the west face
 *                            of cell i, index (k ny + j)(nx+1) + i;
 *   uy[nx (ny+1) nz]         y faces, face j = the south face of cell j,
 *                            index (k (ny+1) + j) nx + i;
 *   uz[nx ny (nz+1)]         z faces, face k = the bottom face of cell k,
 *                            index (k ny + j) nx + i;
 *   dirichlet_bottom         1: p' = 0 beyond the k = 0 face (else a wall).
 * Outputs (device, n doubles each): the seven coefficient arrays of
 * sip_block_desc and b, for -div(rho g grad p') = -div(rho u*):
 *   A_N(P) = -rho_f g_f S_f / delta_f on interior faces (rho_f, g_f the mean
 *   of the two cells' values, delta_f the mean of their widths along the
 *   normal, S_f the face area); walls carry no entry; the Dirichlet face adds
 *   rho_P g_P S_z / (dz_0 / 2) to AP; AP = -(sum of the six entries) + that
 *   term; b = -(net outflow of rho u* S) with the cell's own rho on boundary
 *   faces.  Every operation is rounded in a fixed order (no fused
 *   multiply-adds): the matrix is exactly symmetric.  aw, as, ab may be NULL
 *   (symmetric storage, sip_block_desc.symmetric = 1: they are not written).
 * The outputs can be passed to sip_factor directly (no host round trip).
 * Enqueued on the context's stream, asynchronous; allocates nothing.  Outputs
 * must not overlap the inputs.  Errors: SIP_ERR_INVALID_ARG (dimensions < 1,
 * more than 2^31 - 1 cells, a required pointer NULL), SIP_ERR_CUDA. */
typedef struct {
  int32_t nx, ny, nz;
  int32_t dirichlet_bottom;
  const double *dx, *dy, *dz;
  const double *rho, *g;
  const double *ux, *uy, *uz;
} sip_pcorr_desc;
int sip_assemble_pcorr(sip_ctx *ctx, const sip_pcorr_desc *in, double *ap, double *aw, double *ae, double *as,
                       double *an, double *ab, double *at, double *b);

/* ---- Serving (continuous batching of solve requests) ------------------
 * A server runs `max_slots` solver slots, each with its own CUDA stream on the
 * calling thread's current device.  Submitted requests queue in arrival order;
 * a free slot admits the oldest request once its estimated device footprint
 * fits in what is left of `hbm_budget_bytes` (a request larger than the whole
 * budget runs alone), factors it (coefficient copies and factors stay on the
 * device), solves it with sip_solve's stop rule and frees its memory.  Slots
 * run concurrently, so requests arriving while others are on the GPU start as
 * soon as a slot and memory free up, and their kernels overlap.
 * The descriptor's arrays must stay valid (b and the coefficients unmodified)
 * until the request is done; the solution is written into blk->x.  Each slot
 * has its own context, whose memory pool may keep up to 1 GiB cached beyond
 * the admitted footprints. */
typedef struct sip_server sip_server;
/* Starts the slots.  ctx: a context on the device to use (its stream is not
 * used).  Errors: SIP_ERR_INVALID_ARG, SIP_ERR_NO_DEVICE. */
int sip_server_start(sip_ctx *ctx, size_t hbm_budget_bytes, int max_slots, sip_server **srv);
/* Queues one block (opt nullable: defaults); non-blocking.  *ticket (host)
 * identifies the request.  Errors: SIP_ERR_INVALID_ARG, SIP_ERR_BUSY (4096
 * requests waiting). */
int sip_server_submit(sip_server *srv, const sip_block_desc *blk, const sip_options *opt, double rtol,
                      int max_iters, uint64_t *ticket);
/* Non-blocking state of a request (host outputs, nullable): done (0/1); once
 * done, status (the sip_solve / sip_factor return code), iters and relres.  A
 * finished ticket is reported once and then forgotten (SIP_ERR_NOT_FOUND). */
int sip_server_poll(sip_server *srv, uint64_t ticket, int *done, int *status, int *iters, double *relres);
/* Stops accepting requests, runs the queued ones to completion, joins the
 * slots and frees the server. */
int sip_server_stop(sip_server *srv);
/* Counters and state of a server (a snapshot; host struct).  The watchdog
 * field: oldest_running_ms is the age of the longest-running admitted
 * request (0 when none runs), for a caller to act on a stuck or runaway
 * solve (every device wait of a solve is bounded, so a solve always ends;
 * this measures how long it has taken so far). */
typedef struct {
  uint64_t submitted, completed, failed; /* requests; failed: done with a status other than SIP_OK */
  uint32_t queued, running;              /* waiting for admission / on a slot now */
  uint32_t slots;
  size_t budget_bytes, in_use_bytes;     /* HBM budget and the admitted requests' estimated footprint */
  size_t peak_in_use_bytes;
  double oldest_running_ms;
  double busy_ms;                        /* summed wall time of finished requests on their slots */
} sip_server_stats;
int sip_server_get_stats(sip_server *srv, sip_server_stats *out);

/* Measurement aids.  sip_profile_enable(plan, 1) records a CUDA event pair
 * on the plan's stream around every later kernel launch of the plan;
 * sip_profile_read synchronises the stream and writes, for each kernel kind
 * k < nkinds, the summed device time in ms (ms[k], host) and the number of
 * timed launches (counts[k], host) since the last reset (reset != 0 clears).
 * sip_launch_count (host out) = all kernels the plan has launched so far.
 * sip_kernel_name(k) names kind k (NULL past the last kind). */
int sip_profile_enable(sip_plan *plan, int enable);
int sip_profile_read(sip_plan *plan, int nkinds, double *ms, int64_t *counts, int reset);
int sip_launch_count(sip_plan *plan, int64_t *count_out);
const char *sip_kernel_name(int kind);

/* Total device bytes owned by the plan (host out). */
int sip_plan_bytes(sip_plan *plan, size_t *bytes_out);
/* The plan's tile shape: rows per thread, tile height (tile_k) and stage
 * depth of its forward sweep (host pointers, each may be NULL). */
int sip_plan_shape(sip_plan *plan, int *rows_per_thread, int *tile_k, int *stages);
int sip_plan_destroy(sip_plan *plan);

#ifdef __cplusplus
}
#endif
#endif /* SIP_H */
