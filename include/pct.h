/*
 * pct.h -- C ABI of libpct: proton-CT reconstruction of relative stopping
 * power (RSP) on one NVIDIA B300 (sm_103a).
 *
 * The library implements the data-parallel hot path of Karbasi et al.,
 * "A Highly Accelerated Parallel Multi-GPU based Reconstruction Algorithm for
 * Generating Accurate Relative Stopping Powers" (arXiv:1802.01070):
 *   Sec. I   -- the linear system A x = b: A (m x n) holds the path data of the
 *               m protons, b their water-equivalent path lengths (WEPL), x the
 *               RSP of the n voxels; each row follows the proton's most likely
 *               path (MLP), one proton per thread.
 *   Sec. IV-B -- the DROP block-iterative solver; a block is the set of protons
 *               processed in parallel.
 * Rows of A are recomputed on the fly from the proton histories (MLP, then a
 * voxel walk along the MLP polyline) and never stored.
 *
 * Conventions shared by every call:
 *  - Every call returns a pct_status; nothing aborts or throws across the ABI.
 *    On failure pct_last_error(ctx) returns a message, valid until the next
 *    call on that context.
 *  - Device pointers ("device") are owned by the caller and must stay valid
 *    until the work enqueued on the context's stream has finished.  Calls that
 *    take device pointers only enqueue work: they return before the GPU has
 *    finished and do not report errors that happen on the GPU; the next
 *    pct_synchronize() does.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Voxel (ix, iy, iz) covers [o + i*d, o + (i+1)*d) on each axis and has
 *    linear index j = ix + nx*(iy + ny*iz); volumes are float32 arrays of
 *    nx*ny*nz values in that order.
 *  - Proton i of the loaded set is row i of A; protons whose straight tracker
 *    lines miss the hull have an empty row (A x gives 0 there, the solver skips
 *    them).
 */
#ifndef PCT_H_
#define PCT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pct_ctx pct_ctx;

typedef enum pct_status {
    PCT_OK = 0,
    PCT_ERR_ARG = 1,     /* invalid argument: null pointer, size or range */
    PCT_ERR_CUDA = 2,    /* a CUDA runtime call or kernel launch failed */
    PCT_ERR_OOM = 3,     /* device allocation failed or would exceed the memory cap */
    PCT_ERR_STATE = 4,   /* call out of order, e.g. no histories loaded */
    PCT_ERR_TIMEOUT = 5, /* a bounded device-side wait gave up */
    PCT_ERR_DEVICE = 6   /* a device-side check failed (see pct_last_error) */
} pct_status;

/* Reconstruction grid.  Voxel edges in mm; (ox, oy, oz) is the lab position
 * (mm) of the corner of voxel (0, 0, 0). */
typedef struct pct_grid {
    int32_t nx, ny, nz;
    float dx, dy, dz;
    float ox, oy, oz;
} pct_grid;

/* Keys of pct_set_option / pct_get_option. */
enum pct_option {
    /* Threads of one CUDA block of the per-proton kernels (one warp per
     * proton): 32..256, multiple of 32.  Default 256.  Performance only. */
    PCT_OPT_CTA_THREADS = 1,
    /* MLP sample spacing along the beam depth, in micrometres.  Default: the
     * smallest voxel edge.  Changes A (both the solver and any reference that
     * is compared with it must use the same spacing). */
    PCT_OPT_MLP_STEP_UM = 2,
    /* Device-memory cap in bytes for the context's own allocations; 0 = none.
     * An allocation that would pass it fails with PCT_ERR_OOM. */
    PCT_OPT_MEM_CAP_BYTES = 3,
    /* k > 0: record CUDA events around every k-th launch of the DROP block
     * kernel (1 = every launch) so that pct_get_stat(PCT_STAT_FUSED_MS) reports
     * their summed device time and PCT_STAT_TIMED_LAUNCHES their number.  A
     * timed launch costs the stream a few microseconds (the event records), so
     * a long solve of small blocks is best sampled.  Default 0 (off). */
    PCT_OPT_TIMING = 4,
    /* How pct_solve gets the rows of A (one of enum pct_mode).  Default
     * PCT_MODE_FUSED.  Changing it drops stored rows. */
    PCT_OPT_MODE = 5,
    /* pct_solve_batch with this context first: 1 = capture the batch (record
     * preparation, clears, persistent launch) in a CUDA graph on the first call
     * and replay it while the batch arguments stay the same.  Default 0. */
    PCT_OPT_GRAPH = 6,
    /* pct_solve_batch with this context first: 1 = on the first call with a new
     * batch, time one iteration with each of 128- and 256-thread CTAs x 32 and
     * 16 lanes per proton (on scratch copies of x) and keep the fastest.
     * Default 0 (use PCT_OPT_CTA_THREADS and PCT_OPT_BATCH_LANES). */
    PCT_OPT_AUTOTUNE = 7,
    /* Polls a batched-solve barrier wait makes before giving up (each poll
     * sleeps ~64 ns); a wait that gives up ends the launch and
     * pct_synchronize returns PCT_ERR_TIMEOUT.  1..2^30, default 2^27. */
    PCT_OPT_SPIN_LIMIT = 8,
    /* Test only: 1 = the first barrier of the batch's first scan waits for one
     * arrival more than its CTAs make, so the wait runs out (exercises the
     * timeout path without any fault).  Default 0. */
    PCT_OPT_TEST_UNREACHABLE_BARRIER = 9,
    /* Chord code of PCT_MODE_PACKED rows (one of enum pct_chord_code).  Default
     * PCT_CHORD_FIXED16.  Changing it drops packed rows. */
    PCT_OPT_CHORD_CODE = 10,
    /* pct_solve_batch with this context first: lanes per proton, 32 (one
     * proton per warp) or 16 (two per warp), when PCT_OPT_AUTOTUNE is off (the
     * autotuner picks it with the CTA size).  Default 32. */
    PCT_OPT_BATCH_LANES = 11,
    /* How the fused DROP block step (and pct_rows, which reports the rows that
     * step uses) walks a proton's polyline (one of enum pct_walk).  Both give
     * the same rows; performance only.  Default PCT_WALK_LANES (on the torso
     * workload the round walk measured 1.20 ms per 320000-proton block step
     * against 1.03 ms). */
    PCT_OPT_WALK = 12,
    /* pct_solve in PCT_MODE_FUSED with block_size <= this value runs all its
     * block steps and applies in one persistent cooperative launch (the
     * batched solve of pct_solve_batch with this context alone: no launch per
     * block, bounded barrier waits; options of the batched solve apply, and
     * its device errors and barrier timeouts are reported by pct_synchronize).
     * 0 = never.  Default 0: on the head workload (1e7 protons, block 3200)
     * a block step measured 27.2 us this way against 24.8 us with a launch of
     * the block kernel and one of the apply (18.2 us with those launches
     * replayed from a graph, PCT_OPT_SOLVE_GRAPH), so it pays only when
     * several scans share the GPU (pct_solve_batch).  Performance only; PCT_OPT_TIMING does not
     * time the block steps of such a solve. */
    PCT_OPT_PERSISTENT_BLOCK = 13,
    /* pct_solve with at least this many DROP blocks per iteration (and at
     * most 8192, at least 2 iterations, PCT_OPT_TIMING off) records one
     * iteration's block and apply launches as a CUDA graph on an internal
     * stream (ordered after and before the context's stream) and replays it
     * once per iteration;
     * the graph is kept for the next call while x, lambda, the block size and
     * the context's buffers and options stay the same.  Performance only:
     * the same kernels with the same arguments.  0 = never.  Default 64. */
    PCT_OPT_SOLVE_GRAPH = 14
};

/* Walks of one proton's polyline by one warp (PCT_OPT_WALK). */
enum pct_walk {
    PCT_WALK_LANES = 0,  /* each lane walks a range of consecutive segments; runs that cross
                            a lane boundary are joined by shuffles */
    PCT_WALK_ROUNDS = 1  /* rounds of 32 segments, one per lane, walked with a fixed number of
                            predicated steps; runs collected in shared memory, then gathered and
                            scattered lane-strided (protons with more than 4 crossings in one
                            segment, or more than 768 runs, take the lane walk) */
};

/* Row forms of pct_solve.  The stored forms are built by the same walk as the
 * fused form (so they hold the same rows), once per loaded history set, by
 * pct_build_rows or by the first pct_solve that needs them; they are dropped by
 * pct_load_histories and by a change of mode or MLP step. */
enum pct_mode {
    PCT_MODE_FUSED = 0,  /* recompute MLP and walk for every row of every block: no storage */
    PCT_MODE_CSR = 1,    /* int64 row offsets + int32 voxel + FP32 chord per entry (8 B) */
    PCT_MODE_PACKED = 2  /* int64 row offsets + first voxel per row + per entry a 1-byte 3D step
                            code with an in-hull bit and a 16-bit chord (PCT_OPT_CHORD_CODE) (3 B);
                            runs outside the hull are kept (weight 0) so that steps stay between
                            neighbours */
};

/* 16-bit chord codes of packed rows.  A run's chord lies inside one voxel. */
enum pct_chord_code {
    PCT_CHORD_FIXED16 = 0,  /* unsigned fixed point in units of 1.25 x the voxel diagonal / 65535
                               (1 mm voxels: 3.3e-5 mm, rounding error <= 1.7e-5 mm); a chord
                               beyond the range is clamped and flagged (PCT_ERR_DEVICE) */
    PCT_CHORD_FP16 = 1      /* IEEE half precision (relative rounding <= 2^-11) */
};

/* Keys of pct_get_stat.  Counters cover the calls since pct_reset_stats. */
enum pct_stat {
    PCT_STAT_LAUNCHES = 1,        /* kernels launched by the library */
    PCT_STAT_FUSED_LAUNCHES = 2,  /* launches of the fused DROP kernel */
    PCT_STAT_FUSED_MS = 3,        /* summed device time of the timed ones, ms (needs
                                     PCT_OPT_TIMING; synchronizes the stream) */
    PCT_STAT_DEVICE_BYTES = 4,    /* device memory held by the context */
    PCT_STAT_N_PROTONS = 5,       /* protons loaded */
    PCT_STAT_N_HULL_VOXELS = 6,   /* voxels inside the hull mask */
    PCT_STAT_ROW_ENTRIES = 7,     /* entries of the stored rows (0 when none) */
    PCT_STAT_ROW_BYTES = 8,       /* device bytes of the stored rows */
    PCT_STAT_BATCH_CTA = 9,       /* threads per CTA of the last batched solve */
    PCT_STAT_BATCH_CTAS = 10,     /* CTAs of the last batched solve */
    PCT_STAT_GRAPH_REPLAYS = 11,  /* batched solves replayed from a CUDA graph */
    PCT_STAT_TIMED_LAUNCHES = 12, /* launches of the DROP block kernel timed (PCT_OPT_TIMING) */
    PCT_STAT_BATCH_LANES = 13,    /* lanes per proton of the last batched solve */
    PCT_STAT_WALK_FALLBACKS = 14, /* DROP row walks PCT_WALK_ROUNDS passed to the lane walk
                                     (synchronizes the stream) */
    PCT_STAT_SOLVE_GRAPH_REPLAYS = 15  /* pct_solve iterations replayed from a CUDA graph */
};

/* Create a context on CUDA device `device`: the reconstruction volume of
 * Sec. I, x of A x = b, one RSP value per voxel of `grid`.
 *   grid       -- host pointer, copied.
 *   hull_mask  -- host pointer to nx*ny*nz bytes (nonzero = inside the object
 *                 hull), copied; NULL means every voxel is inside.  Rows only
 *                 cover hull voxels (x outside the hull never changes).
 *   cuda_stream-- a cudaStream_t to enqueue all work on (cudaStreamLegacy,
 *                 0x1, selects the legacy default stream), or NULL for a
 *                 non-blocking stream the context creates and owns.
 * The hull is not part of the paper; the reading used is that a proton's path
 * starts where its straight entry tracker line first enters a hull voxel and
 * ends where its straight exit tracker line, followed backwards, first does.
 * The context keeps the mask and, for that search, the chessboard distance of
 * every voxel to the hull (one byte per voxel each), built on the GPU here.
 * Errors: PCT_ERR_ARG (null out/grid, non-positive sizes, grid over 2^31
 * voxels), PCT_ERR_CUDA, PCT_ERR_OOM. */
pct_status pct_create(pct_ctx **out, const pct_grid *grid, const uint8_t *hull_mask, int device,
                      void *cuda_stream);

/* Release every device allocation of the context (after synchronizing its
 * stream) and the context itself.  NULL is ignored. */
void pct_destroy(pct_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed pct_create when
 * ctx is NULL). */
const char *pct_last_error(const pct_ctx *ctx);

pct_status pct_set_option(pct_ctx *ctx, int32_t key, int64_t value);
pct_status pct_get_option(const pct_ctx *ctx, int32_t key, int64_t *value);

/* Load n proton histories (Sec. I: tracker data and WEPL), replacing any
 * previous set.  Every argument points to n float32 values:
 *   in_xyz[0..2]   -- entry tracker point, lab frame, mm
 *   out_xyz[0..2]  -- exit tracker point, lab frame, mm
 *   ang_in[0..1]   -- entry direction angles in rad: theta in the t-u plane,
 *                     psi in the v-u plane of the beam frame
 *   ang_out[0..1]  -- exit direction angles, same convention
 *   gantry_rad     -- gantry angle phi; beam frame u = (cos phi, sin phi, 0),
 *                     t = (-sin phi, cos phi, 0), v = z
 *   wepl_mm        -- measured WEPL (b of A x = b), mm
 * ptrs_on_device = 1: all pointers are device pointers (copied on the stream,
 * asynchronously); 0: host pointers (copied in chunks on an internal stream,
 * the per-proton records of each chunk computed on the context stream as it
 * lands; the call returns when the copies are done, so the host buffers may be
 * reused on return; pinned buffers copy fastest and overlap best).
 * The library keeps its own copy; the caller keeps ownership.  n = 0 is valid.
 * Errors: PCT_ERR_ARG (n < 0 or a null pointer with n > 0), PCT_ERR_OOM,
 * PCT_ERR_CUDA. */
pct_status pct_load_histories(pct_ctx *ctx, int64_t n, const float *const in_xyz[3],
                              const float *const out_xyz[3], const float *const ang_in[2],
                              const float *const ang_out[2], const float *gantry_rad,
                              const float *wepl_mm, int ptrs_on_device);

/* Hull-frame state of protons [first, first+count) (device out, count*12
 * float32, row-major per proton): u_in, u_out (beam-frame depth of the hull
 * entry and exit, mm), t0, theta0, v0, psi0 (entry state), t2, theta2, v2, psi2
 * (exit state), valid (1.0 / 0.0), spare.  Errors: PCT_ERR_ARG, PCT_ERR_STATE. */
pct_status pct_hull_states(pct_ctx *ctx, int64_t first, int64_t count, float *out_states);

/* Copy of the context's hull distance map (device out, nx*ny*nz bytes, x
 * fastest): per voxel the chessboard distance max(|dx|, |dy|, |dz|), in
 * voxels, to the nearest hull voxel, capped at 255; 0 inside the hull, 255
 * everywhere when the hull is empty.  The hull search of every path start
 * skips empty space with it.  Not part of the paper: the hull itself is a
 * reading (see pct_create).  Asynchronous on the context's stream.
 * Errors: PCT_ERR_ARG (null ctx or out), PCT_ERR_CUDA. */
pct_status pct_hull_distance(pct_ctx *ctx, uint8_t *out_dist);

/* MLP polylines of protons [first, first+count) (Sec. I, most likely path):
 * the hull entry point, the MLP at depths u_in + k*du (k >= 1, below u_out by
 * more than du/1000) and the hull exit point, in lab mm.
 *   out_xyz  -- device, count*max_pts*3 float32; proton p's points at
 *               out_xyz[(p*max_pts + k)*3 + {0,1,2}], at most max_pts written
 *   out_npts -- device, count int32: the full point count (0 = empty row); a
 *               count above max_pts means the polyline was cut short
 * Errors: PCT_ERR_ARG (range, max_pts < 2, null), PCT_ERR_STATE. */
pct_status pct_mlp(pct_ctx *ctx, int64_t first, int64_t count, int32_t max_pts, float *out_xyz,
                   int32_t *out_npts);

/* The calls below that walk paths (pct_hull_states, pct_mlp, pct_rows,
 * pct_forward, pct_adjoint, pct_solve, pct_build_rows) first compute the
 * per-proton records of the loaded histories (beam frame, hull entry and exit
 * of the tracker lines, entry and exit states; kernel k_prepare) if they are
 * not yet computed, and keep them until new histories are loaded or the MLP
 * step changes. */

/* Rows of A for protons [first, first+count), in path order: each entry is one
 * visit of the MLP polyline to a hull voxel (a maximal run of the path inside
 * that voxel) with its chord length a_ij in mm.
 *   out_idx  -- device, count*max_nnz int32 voxel indices
 *   out_len  -- device, count*max_nnz float32 chord lengths, mm
 *   out_nnz  -- device, count int32 full row lengths (above max_nnz: cut short)
 * Errors: PCT_ERR_ARG, PCT_ERR_STATE. */
pct_status pct_rows(pct_ctx *ctx, int64_t first, int64_t count, int32_t max_nnz, int32_t *out_idx,
                    float *out_len, int32_t *out_nnz);

/* y = A x, the projection of Sec. I: y_i = sum_j a_ij x_j over the row of
 * proton i (its MLP path data), i.e. the WEPL the volume x predicts for it.
 *   x -- device, n float32 (nx*ny*nz voxels); y -- device, m = protons loaded,
 *        overwritten (0 for rows that miss the hull).
 * Enqueued on the context stream.  Errors: PCT_ERR_ARG (null x or y with
 * protons loaded), PCT_ERR_STATE (no histories), PCT_ERR_CUDA. */
pct_status pct_forward(pct_ctx *ctx, const float *x, float *y);

/* g = A^T y, the back projection along the same rows (Sec. I):
 * g_j = sum_i a_ij y_i; the adjoint of pct_forward (<A x, y> = <x, A^T y>).
 *   y -- device, m float32; g -- device, n float32, overwritten.
 * Enqueued on the context stream.  Errors: PCT_ERR_ARG (null g, or null y
 * with protons loaded), PCT_ERR_STATE, PCT_ERR_CUDA. */
pct_status pct_adjoint(pct_ctx *ctx, const float *y, float *g);

/* DROP reconstruction (Sec. IV-B): `iters` passes over the protons in blocks
 * of `block_size` consecutive rows; for each block, with x frozen,
 *   x_j <- x_j + lambda / s_j * sum_{i in block} a_ij (b_i - a_i.x) / ||a_i||^2
 * where s_j counts the rows of the block that cross voxel j (voxels no row
 * crosses are unchanged; empty rows are skipped).
 *   x -- device, n float32: the initial iterate on entry, the RSP on return.
 * Enqueued on the context stream (a solve of many small blocks may run its
 * launches from a CUDA graph on the context's internal stream, ordered after
 * and before it: PCT_OPT_SOLVE_GRAPH); pct_synchronize reports device errors.
 * Errors: PCT_ERR_ARG (null x, iters < 0, block_size < 1), PCT_ERR_STATE,
 * PCT_ERR_OOM, PCT_ERR_CUDA. */
pct_status pct_solve(pct_ctx *ctx, int32_t iters, float lambda, int64_t block_size, float *x);

/* ---- Gradient-based reconstruction beside DROP -----------------------------
 * The paper solves A x = b with DROP only (Sec. IV-B).  With pct_forward and
 * pct_adjoint as a differentiable projector, a caller can instead minimise
 * ||A x - b||^2 + w TV(x); the two calls below supply the rest.  Neither has a
 * counterpart in the paper. */

/* Isotropic total variation of the volume x (device, n voxels):
 *   value = sum over all voxels v of sqrt(|D+ x|_v^2 + eps^2),
 * D+ the forward differences along x, y, z (zero at each axis' last index).
 * grad (device, n floats, overwritten) = d value / d x; value (device, one
 * double, overwritten).  Enqueued on the context stream.
 * Errors: PCT_ERR_ARG (null pointer, eps < 0), PCT_ERR_CUDA. */
pct_status pct_tv(pct_ctx *ctx, const float *x, float eps, float *grad, double *value);

/* One Adam step (Kingma & Ba) on n parameters, all device arrays:
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   x <- x - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * step counts from 1.  Errors: PCT_ERR_ARG, PCT_ERR_CUDA. */
pct_status pct_adam(pct_ctx *ctx, float *x, const float *grad, float *m, float *v, int64_t n,
                    float lr, float beta1, float beta2, float eps, int32_t step);

/* Build the stored rows of the current mode (PCT_OPT_MODE) for the loaded
 * histories (Sec. I, the path data of A).  No-op in PCT_MODE_FUSED.  Enqueued
 * on the context stream; synchronizes once to size the entry arrays.
 * Errors: PCT_ERR_STATE (no histories), PCT_ERR_OOM, PCT_ERR_CUDA. */
pct_status pct_build_rows(pct_ctx *ctx);

/* As pct_solve, with x in host memory: copies x to the device, solves, copies
 * the result back and synchronizes. */
pct_status pct_solve_host(pct_ctx *ctx, int32_t iters, float lambda, int64_t block_size,
                          float *x_host);

/* Many independent DROP reconstructions (scans) in one persistent launch
 * (Sec. IV-B per scan; the paper runs one scan per solver instance).  Scan k
 * is the histories loaded in ctxs[k] (fused rows), solved in place into x[k]
 * (device, that context's grid) with iters[k], lambda[k], block_size[k].
 * CTAs are split between the scans in proportion to protons x iterations;
 * the CTAs of a scan meet at a barrier after each block step and each apply;
 * scans never wait for each other.  The launch is cooperative (all CTAs
 * resident), its barrier waits are bounded (PCT_OPT_SPIN_LIMIT).  Options of
 * ctxs[0] apply: PCT_OPT_GRAPH, PCT_OPT_AUTOTUNE, PCT_OPT_CTA_THREADS.  The
 * work runs on an internal stream ordered after, and before, ctxs[0]'s
 * stream; other contexts' streams are synchronized first.  Device errors and
 * barrier timeouts are reported by pct_synchronize(ctxs[0]) (PCT_ERR_TIMEOUT).
 * Errors: PCT_ERR_ARG (null, duplicate context, more scans than resident
 * CTAs), PCT_ERR_STATE, PCT_ERR_OOM, PCT_ERR_CUDA. */
pct_status pct_solve_batch(pct_ctx *const *ctxs, int32_t count, const int32_t *iters,
                           const float *lambda, const int64_t *block_size, float *const *x);

/* ---- Data cleaning (Sec. IV-A) ---------------------------------------------
 * The paper reduces each scan before the solve by "identifying and removing
 * statistical outliers" (116 million histories to 21 million) without further
 * detail.  The reading implemented, in FP64:
 *   - each proton falls into a bin (a, k_t, k_v): a = the nearest multiple of
 *     angle_step to its gantry angle, modulo n_angle; t and v = where the
 *     straight chord between its entry and exit tracker points crosses depth
 *     u = 0 of its beam frame, k_t = floor((t - t_min) / dt) in 0..n_t-1,
 *     k_v = floor((v - v_min) / dv) in 0..n_v-1 (protons outside are removed);
 *   - per bin, for q in {WEPL, theta_out - theta_in, psi_out - psi_in}: the
 *     mean mu and the population standard deviation sigma (two passes);
 *   - a proton is kept when |q - mu| <= k_sigma * sigma for all three.
 * Per-bin sums are FP64 atomics, so a proton within rounding of a cut may be
 * decided either way between runs. */
typedef struct pct_clean_params {
    int32_t n_angle, n_t, n_v;  /* bins */
    double angle_step;          /* rad */
    double t_min, dt;           /* mm: lower edge of t bin 0, width */
    double v_min, dv;           /* mm */
    double k_sigma;             /* cut in standard deviations (3 is usual) */
} pct_clean_params;

/* Remove the outliers from the loaded histories: the kept protons replace the
 * loaded set, in their order (proton i of the new set is the i-th kept one);
 * records and stored rows are recomputed when next needed.
 *   keep_out -- device, n bytes (n = protons before the call), or NULL:
 *               1 = kept, 0 = removed, per proton of the set before the call
 *   n_kept   -- host, or NULL: protons kept
 * Needs device scratch of 52 bytes per bin + 5 bytes per proton + a second
 * copy of the histories while it runs.  Synchronizes the context stream.
 * Errors: PCT_ERR_ARG (null params, bin counts < 1 or >= 2^31 bins, widths
 * not finite and > 0, k_sigma < 0), PCT_ERR_STATE (no histories), PCT_ERR_OOM,
 * PCT_ERR_CUDA. */
pct_status pct_clean(pct_ctx *ctx, const pct_clean_params *params, uint8_t *keep_out, int64_t *n_kept);

/* ---- Image regions: the paper's Algorithm 1 on one GPU (Sec. III) ---------
 * The paper splits the volume along z into overlapping regions, solves each
 * region independently with the protons that enter or exit it (one GPU per
 * region, no exchange during the solve), and builds the volume from each
 * region's slices farthest from its overlap.  Here the regions are solved one
 * after the other on this GPU:
 *   1 setupImageRegions: region r's core slices are [r nz / R, (r+1) nz / R)
 *     (integer division), extended by `halo` slices on each side (clamped);
 *   2 identifyProtonsPassingRegions: a proton with a hull path belongs to
 *     region r when the slices of both its hull entry point and its hull exit
 *     point (pct_hull_states; points on the grid's outer z faces count in the
 *     first or last slice) lie in r's extended slices -- it may belong to two
 *     regions, or to none (the paper sizes the overlap for 96 % coverage);
 *   3 allocateMemoryForProtonsPerGPU: each region gets its protons' records
 *     (the full volume's: the same MLP paths) on a grid of its extended slices;
 *   4 iterativelySolvePerGPU: pct_solve on each region (fused rows, which
 *     keep only the voxels of the region's slices), from x's slab;
 *   5 selectSlice: x's core slices of region r come from region r.
 * A region's DROP blocks are block_size consecutive protons of its own list,
 * so with R = 1 this is pct_solve over the protons with a hull path (the plain
 * pct_solve's blocks also hold protons without one, whose rows are empty).
 * The paper's example: nz = 20, two regions,
 * halo 3 (slices 0-12 and 7-19; slices 0-9 and 10-19 kept).
 *   x              -- device, n voxels: initial iterate in, result out
 *   region_protons -- host, n_regions values, or NULL: protons per region
 * Synchronizes the context stream.  Errors: PCT_ERR_ARG (null x, n_regions
 * outside 1..nz, halo < 0, iters < 0, block_size < 1), PCT_ERR_STATE (no
 * histories), PCT_ERR_OOM, PCT_ERR_CUDA, PCT_ERR_DEVICE. */
pct_status pct_solve_regions(pct_ctx *ctx, int32_t n_regions, int32_t halo, int32_t iters, float lambda,
                             int64_t block_size, float *x, int64_t *region_protons);

/* ---- Filtered back-projection: the initial iterate (Sec. I) ---------------
 * The paper starts the solve from "the FBP image as the initial iterate" and
 * gives no detail.  The reading implemented is the textbook parallel-beam FBP,
 * slice by slice, on binned list-mode data:
 *   - sinogram: every loaded proton falls into the bin (a, l, k) of the same
 *     rule as pct_clean (nearest angle step; t, v where the straight tracker
 *     chord crosses depth u = 0; k = floor((t - t_min) / dt), l = floor((v -
 *     v_min) / dv)); p[a][l][k] = the mean WEPL of the bin, 0 when empty;
 *   - filter along t: q[k] = dt * sum_m p[m] h[k - m], h[0] = 1 / (4 dt^2),
 *     h[n] = -1 / (pi^2 n^2 dt^2) for odd n, 0 for even n != 0 (the
 *     band-limited ramp kernel); FP64 sums, q stored as float;
 *   - back-projection: voxel centre (x, y, z), slice l of z:
 *     x_fbp = (pi / n_angle) * sum_a q_a(-x sin(a angle_step) + y cos(a
 *     angle_step)), q_a linear between bin centres t_min + (k + 1/2) dt and 0
 *     beyond the first and last; FP32.  (A full turn sees every line twice.)
 * Voxels outside the hull, or whose z lies outside the v bins, get 0. */
typedef struct pct_fbp_params {
    int32_t n_angle, n_t, n_v;  /* bins: 1..4096 angles, 1..16384 t bins */
    double angle_step;          /* rad */
    double t_min, dt;           /* mm */
    double v_min, dv;           /* mm */
} pct_fbp_params;

/* FBP image of the loaded histories.
 *   x        -- device, n voxels, overwritten (a DROP initial iterate)
 *   sino_out -- device, n_angle * n_v * n_t floats (the filtered sinogram q,
 *               index (a * n_v + l) * n_t + k), or NULL
 * Needs 12 bytes of device scratch per bin (plus 4 without sino_out).
 * Synchronizes the context stream.  Errors: PCT_ERR_ARG (null params or x,
 * bin counts out of range, widths not finite and > 0), PCT_ERR_STATE (no
 * histories), PCT_ERR_OOM, PCT_ERR_CUDA. */
pct_status pct_fbp(pct_ctx *ctx, const pct_fbp_params *params, float *x, float *sino_out);

/* Wait for the context's stream; report asynchronous CUDA errors
 * (PCT_ERR_CUDA) and device-side check failures (PCT_ERR_DEVICE). */
pct_status pct_synchronize(pct_ctx *ctx);

pct_status pct_get_stat(pct_ctx *ctx, int32_t key, double *value);
pct_status pct_reset_stats(pct_ctx *ctx);

/* Diagnostic: out[i] = the FP64 tangent the record kernel applies to tracker
 * angles (Sec. I: straight tracker lines of slope tan(theta) up to the hull),
 * for n angles t (rad).  For |t| <= 0.25 it is the Maclaurin series of tan
 * summed to 11 terms (relative error within 2.3e-16, about one unit in the
 * last place, there); beyond, the CUDA
 * library tan.  t, out: device, n doubles.  stream: a cudaStream_t or NULL
 * (default stream); the call synchronizes it.
 * Errors: PCT_ERR_ARG (n < 0, null pointer with n > 0), PCT_ERR_CUDA. */
pct_status pct_tan_angle(const double *t, double *out, int64_t n, void *cuda_stream);

/* ---- Roofline ceilings measured on the device -------------------------------
 * Not part of the paper: the two limits of the fused DROP block step (its MLP
 * and walk arithmetic, and its scatter), measured so that a reported fraction
 * of peak has a measured denominator.  Each allocates its own scratch, runs on
 * the legacy default stream of `device`, synchronizes, and reports the best of
 * `repeats` timed launches (CUDA events) after one warm-up launch. */

/* FP32 fused multiply-add throughput: every SM filled with threads that each
 * run 8 independent chains of fmaf.  tflops = 2 x FMAs / best time (TFLOP/s);
 * best_ms (may be NULL) = that time.  Errors: PCT_ERR_ARG (bad device, null
 * tflops, repeats < 1), PCT_ERR_CUDA. */
pct_status pct_peak_fp32(int device, int32_t repeats, double *tflops, double *best_ms);

/* Throughput of float2 atomicAdd (one 8-byte vector atomic, as the DROP
 * scatter issues per visit) to addresses spread uniformly by a counter-based
 * hash over an array of n_slots float2 (n_slots * 8 bytes; an array smaller
 * than L2 measures the L2 atomic units).  gatomics = atomics / best time, in
 * 1e9 per second.  Errors: PCT_ERR_ARG (bad device, null gatomics, repeats < 1,
 * n_slots outside 1..2^31), PCT_ERR_CUDA. */
pct_status pct_peak_atomic(int device, int64_t n_slots, int32_t repeats, double *gatomics,
                           double *best_ms);

/* ---- DROP reconstruction without device allocation --------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: for example an application that hands all device
 * memory to its own pool allocator and forbids allocations outside it, or a
 * latency-bound service that cannot accept the device-wide synchronization a
 * cudaMalloc or cudaFree may cause in the middle of a scan.
 *
 * It computes what pct_create + pct_load_histories + pct_solve compute (same
 * kernels, MLP spacing = smallest voxel edge), but takes every input as a
 * device pointer and keeps all scratch (a copy of the histories, the
 * per-proton records, the per-voxel DROP accumulator, the hull distance map
 * of the hull search and its scratch, the per-block lists of protons with a
 * hull path, the MLP table) in fixed device arrays compiled into the library:
 * about 19 MB, held on every GPU that loads the library until the process
 * exits.  Limits: at most
 * PCT_NOALLOC_MAX_PROTONS protons, PCT_NOALLOC_MAX_VOXELS voxels, and a grid
 * diagonal of at most PCT_NOALLOC_MAX_SAMPLES MLP steps; larger inputs are
 * rejected with PCT_ERR_ARG before any GPU work.
 *   grid       -- host pointer, as in pct_create
 *   hull_mask  -- device, nx*ny*nz bytes (nonzero = inside the hull)
 *   n, in_xyz..wepl_mm -- device pointers, as in pct_load_histories
 *   iters, lambda, block_size -- as in pct_solve
 *   x          -- device, n voxels: initial iterate in, RSP out
 *   device     -- CUDA device to run on; cuda_stream -- stream (NULL: the
 *                 default stream)
 * The first call on a device looks up the device addresses of the fixed arrays
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  Every call on a device shares the same arrays and
 * clears the parts that must start at zero itself; calls that overlap on the
 * GPU (from several host threads or streams) race on them.  The call returns
 * after the work has finished: it synchronizes the stream and copies the
 * device status word back to the host.  It allocates and frees no device
 * memory.  Errors (status only; pct_last_error does not cover this call):
 * PCT_ERR_ARG, PCT_ERR_CUDA (every CUDA failure, a launch short of resources
 * included; never PCT_ERR_OOM), PCT_ERR_DEVICE. */
#define PCT_NOALLOC_MAX_PROTONS 65536
#define PCT_NOALLOC_MAX_VOXELS 1048576
#define PCT_NOALLOC_MAX_SAMPLES 4096
pct_status pct_solve_noalloc(const pct_grid *grid, const uint8_t *hull_mask, int64_t n,
                             const float *const in_xyz[3], const float *const out_xyz[3],
                             const float *const ang_in[2], const float *const ang_out[2],
                             const float *gantry_rad, const float *wepl_mm, int32_t iters,
                             float lambda, int64_t block_size, float *x, int device,
                             void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PCT_H_ */
