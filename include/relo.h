/*
 * relo.h — C ABI of the GB300 relocalization scoring library.
 *
 * The library scores positional hypotheses x orientations x LiDAR beams
 * against an occupancy grid for passive 2-D global relocalization (arXiv
 * 2511.01219): the EDT likelihood-field table (Sec. III-A item 3), ray-cast
 * synthesized scans (Eq. 13), SMAD coarse ranking (Eq. 16-20), TAM orientation
 * selection and pose evaluation (Eq. 22-31), and batched multi-stage
 * inference with local top-k and early termination (Sec. III intro,
 * Remarks 2-3).  Every step runs in the library's own CUDA kernels (sm_103a);
 * there is no CPU fallback.
 *
 * Conventions
 *   - Grids are int8, row-major, W columns x H rows; value >= 65 is occupied,
 *     value < 0 is unknown (treated as free by the EDT and by ray casting).
 *     Cell (cx, cy) covers [ox + cx*res, ox + (cx+1)*res) x [oy + cy*res, ...).
 *   - Hypotheses are snapped to cell centres.  Orientations are the shifts m
 *     of Eq. 15, theta_m = m * 2*pi / N_s, reported wrapped to [-pi, pi).
 *   - Beam angles must lie on a uniform panoramic grid of N_s = 2*pi / step
 *     directions (Eq. 14): each within 1e-3 steps of a multiple of 2*pi/N_s,
 *     no two on the same direction, listed in increasing (cyclic) order.
 *   - Pointers named *_dev are device pointers (for example from torch
 *     tensors) valid on the context's stream; all other pointers are host
 *     pointers.  The caller keeps ownership of every buffer it passes; the
 *     library copies what it keeps.  Results are written into caller memory.
 *   - Every call returns RELO_OK (0) or a negative error code; the message is
 *     available from relo_last_error().  A context is not thread-safe.
 */
#ifndef RELO_H
#define RELO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RELO_OK 0
#define RELO_PENDING 1              /* relo_poll only: request still running */
#define RELO_E_INVALID_ARG (-1)
#define RELO_E_BEAM_GRID (-2)       /* angles not on a uniform 2*pi/N_s grid, or n_orient does not divide N_s */
#define RELO_E_NO_HYPOTHESES (-3)
#define RELO_E_OVER_BUDGET (-4)     /* the request or map does not fit the context's HBM budget */
#define RELO_E_CUDA (-5)            /* a CUDA call failed; the context should be destroyed */
#define RELO_E_TIMEOUT (-6)         /* a served request's deadline passed before it was admitted */
#define RELO_E_NO_VALID_BEAMS (-7)  /* no beam with 0 < z < max_range */
#define RELO_E_NOT_FOUND (-8)       /* unknown map id or ticket */

/* Parameters of Eq. 20-31 and of the batched inference.  relo_default_params()
 * fills the values used throughout: z_hit 1, sigma_hit 0.2 m, z_rand 0
 * (Sec. IV-B), eps 1e-6 (Eq. 23), batch 200, local top-20, tau 0.95
 * (Sec. IV-C).  The paper prints neither the Eq. 25 ratio endpoints nor
 * d_max; the defaults (0.9 -> 0.8, 0.8 -> 0.6, 2 m) make the retention fall
 * as the FoV widens, as the text after Eq. 25 describes. */
typedef struct relo_params {
    double z_hit, sigma_hit, z_rand, eps;              /* Eq. 23 */
    double d_max;                                      /* Eq. 29, metres; d_max/res must be an integer <= 90 */
    double a_mid_min, a_mid_max, a_low_min, a_low_max; /* Eq. 25 */
    double tau;                                        /* early-termination threshold (Sec. III) */
    double panoramic_ratio;                            /* Eq. 20: lambda >= this scores m = 0 only */
    int32_t n_orient;                                  /* |Theta| of Eq. 15 (must divide N_s); 0 = N_s */
    int32_t topk;                                      /* SMAD survivors scored by TAM (<= 4096) */
    int32_t batch;                                     /* survivors per batch (<= 1024) */
    int32_t local_topk;                                /* local top-k kept per batch (<= batch) */
    int32_t n_skip_beam;                               /* Eq. 11 beam stride */
    int32_t early_stop;                                /* 1: stop after the first batch whose best >= tau */
    int64_t hbm_budget;                                /* bytes the context may hold; 0 = no limit */
    double max_range;                                  /* metres: the longest scan range maps loaded from now on accept
                                                          (sets the border of the TAM field; default 30) */
    int64_t scan_cache_bytes;                          /* device bytes for resident synthesized scans; 0 = none
                                                          (see relo_scan_cache_stats) */
    int32_t ray_tables;                                /* 1 (default): trace rays tile by tile with per-direction
                                                          tables built once per (N_s, max_range); 0: step cell by
                                                          cell.  Same cells and ranges either way. */
    int32_t coarse_metric;                             /* ranking metric: RELO_COARSE_SMAD (default, Eq. 16-20),
                                                          RELO_COARSE_CAER (Eq. 21, Remark 5: the beam-wise mean
                                                          absolute range error over the same orientations) or
                                                          RELO_COARSE_SMAD_DIRECT (SMAD with every window sum of
                                                          Eq. 18 added up position by position, without the prefix
                                                          sums of Eq. 17: the Table II ablation; same results, more
                                                          work; resident window tables are not used for it) or
                                                          RELO_COARSE_NONE (no coarse ranking, Table II's arm
                                                          without SMAD ordering: no rays are cast, every numerator
                                                          is 0 at m = 0, so the survivors are the first topk
                                                          hypotheses in the order they were set) */
    int32_t fine_metric;                               /* scoring metric: RELO_FINE_TAM (default, Eq. 31),
                                                          RELO_FINE_TAM_MEAN (Eq. 34), RELO_FINE_BASELINE (Eq. 33)
                                                          or RELO_FINE_LF (Eq. 32, a sum of log-likelihoods, so
                                                          negative; tau compares against it as it is) */
    int32_t icp_iters;                                 /* > 0: each batch's local top-k poses are refined by up to
                                                          this many point-to-point ICP iterations against the map's
                                                          occupied cells and scored again at the refined continuous
                                                          pose (Sec. III overview, Remark 2); the batch's best and the
                                                          result are then the best re-evaluated pose.  0 (default):
                                                          no refinement */
} relo_params;

#define RELO_COARSE_SMAD 0
#define RELO_COARSE_CAER 1
#define RELO_COARSE_SMAD_DIRECT 2
#define RELO_COARSE_NONE 3
#define RELO_FINE_TAM 0
#define RELO_FINE_TAM_MEAN 1
#define RELO_FINE_BASELINE 2
#define RELO_FINE_LF 3

/* Result of one relocalization (Eq. 9 restricted to the scored hypotheses). */
typedef struct relo_result {
    double x, y, theta;     /* selected pose: cell centre (metres) and theta_m wrapped to [-pi, pi); with
                               icp_iters > 0 the refined continuous pose */
    double tam;             /* its score by the fine metric: TAM (Eq. 31) unless fine_metric says otherwise */
    double smad;            /* the coarse metric of its position, metres: SMAD (Eq. 20) or CAER (Eq. 21) */
    int64_t smad_num;       /* its numerator in Q16 cell units: |sum R_real - W_m|, or sum |R_i - R^_{i+m}| */
    int64_t n_smad_evals;   /* hypothesis x orientation SMAD evaluations performed */
    int64_t n_tam_evals;    /* hypothesis x orientation TAM evaluations performed */
    int32_t hyp;            /* index of the selected hypothesis in the context's set */
    int32_t m;              /* orientation shift of Eq. 15 */
    int32_t n_batches;      /* batches scored before stopping */
    int32_t status;         /* RELO_OK or an error code */
} relo_result;

typedef struct relo_ctx relo_ctx;

void relo_default_params(relo_params *p);

/* Creates a context on the current CUDA device.  stream: a cudaStream_t to
 * run on (NULL creates a private non-blocking stream of the highest
 * priority).  The context also creates a second stream of the lowest
 * priority, on which a map's EDT computes d2 and the clamped field while the
 * context stream goes on to the next request's ray cast; every reader of
 * those tables waits on an event, so results do not depend on it.  A caller's
 * stream of higher than the default priority lets the ray cast run first.
 * The context owns all device memory it allocates and frees it in
 * relo_destroy. */
int relo_create(const relo_params *p, void *stream, relo_ctx **out);
int relo_destroy(relo_ctx *ctx);
const char *relo_last_error(const relo_ctx *ctx);
/* replaces the parameters (maps keep the field clamp they were built with unless rebuilt) */
int relo_set_params(relo_ctx *ctx, const relo_params *p);

/* Map precompute (Sec. III-A item 3 and the likelihood field of Eq. 23/29):
 * copies the grid to the device and computes, in the library's kernels, the
 * exact squared EDT d2 (cells^2, -1 when the map has no occupied cell), its
 * clamped copy min(d2, (d_max/res)^2) in 8x8-cell tiles, and a 1-bit
 * occupancy bitmap in 8x8 tiles.  W, H in [1, 16384].  Returns a map id. */
int relo_load_map(relo_ctx *ctx, const int8_t *grid, int32_t w, int32_t h, double res, double origin_x,
                  double origin_y, int32_t *map_id);
int relo_load_map_dev(relo_ctx *ctx, const int8_t *grid_dev, int32_t w, int32_t h, double res,
                      double origin_x, double origin_y, int32_t *map_id);
/* Recomputes a loaded map's tables in place from a new grid of the same size
 * (for example after a door opened).  Asynchronous on the context stream. */
int relo_update_map_dev(relo_ctx *ctx, int32_t map_id, const int8_t *grid_dev);
/* Same from a host grid.  The copy is queued on the context stream: a pinned
 * grid must stay unchanged until the stream passes it (any blocking call on
 * the context, such as relo_relocalize, waits for that); a pageable grid may
 * be reused as soon as the call returns. */
int relo_update_map(relo_ctx *ctx, int32_t map_id, const int8_t *grid);
int relo_unload_map(relo_ctx *ctx, int32_t map_id);

/* Copies a map's tables into caller device buffers, row-major W x H:
 * d2_dev (int32, -1 = no obstacle), field_dev (uint16, clamped), occ_dev
 * (uint8, 1 = occupied).  Any pointer may be NULL. */
int relo_map_tables_dev(relo_ctx *ctx, int32_t map_id, int32_t *d2_dev, uint16_t *field_dev, uint8_t *occ_dev);
/* Copies a map's empty boxes of tiles, the table the ray cast of Eq. 13
 * uses to cross empty space, into a caller device buffer of capacity uint16
 * entries.  The map is cut into 8x8-cell tiles, TW = ceil(W / 8) by TH =
 * ceil(H / 8); it is seen in four frames (f = 0 as is, 1 mirrored in x, 2
 * mirrored in y, 3 in both: frame tile (tx, ty) is map tile (TW - 1 - tx)
 * when mirrored in x, (TH - 1 - ty) in y), each with a last column and row
 * of tiles that count as occupied; a tile is empty when none of its cells is
 * occupied (>= 65) or outside the map.  Entry [f][ty][tx], row-major with
 * TW + 1 entries per row and TH + 1 rows per frame, packs three sides, each
 * at most 16 and 0 when the tile is not empty: bits 0-4 the largest s with
 * the tiles [tx, tx + s) x [ty, ty + s) all empty, bits 5-9 the empty run
 * [tx, tx + r) along the row, bits 10-14 the empty run [ty, ty + r) along the
 * column.  *n_out (optional) receives 4 (TW + 1)(TH + 1); RELO_E_INVALID_ARG
 * when capacity is smaller.  Blocking. */
int relo_map_walk_boxes_dev(relo_ctx *ctx, int32_t map_id, uint16_t *boxes_dev, int64_t capacity, int64_t *n_out);

/* Positional hypotheses of Eq. 6 (for example from the RRT of Algorithm 1).
 * xy: n (x, y) pairs in metres (host memory, pinned or not), copied to the
 * device and snapped there to the containing cell, floor((x - origin_x) /
 * res) and likewise in y, in IEEE FP64.  Every one must fall inside the map
 * on a cell that is not occupied; otherwise RELO_E_INVALID_ARG, and the map
 * keeps no hypotheses until the next successful call.  Blocking. */
int relo_set_hypotheses(relo_ctx *ctx, int32_t map_id, const double *xy, int32_t n);
/* Same, from n (cx, cy) int32 cell pairs already on the device. */
int relo_set_hypotheses_cells_dev(relo_ctx *ctx, int32_t map_id, const int32_t *cells_dev, int32_t n);

/* One relocalization (Eq. 3 via Eq. 6-9): plan the scan (Eq. 11-16), ray-cast
 * and SMAD-rank every hypothesis (Eq. 13, 17-20), keep the topk best, score
 * them with TAM in batches over all orientations (Eq. 22-31) with local
 * top-k and early termination, and return the best pose.  ranges: n_beams
 * float32 metres; a beam is valid when finite and 0 < z < max_range.
 * Blocking: returns once the result is in *out. */
int relo_relocalize(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                    float max_range, relo_result *out);
/* Same with the ranges already on the device; the angles (sensor geometry)
 * stay on the host.  The result is written to result_dev (a relo_result in
 * device memory) and the call returns without synchronising. */
int relo_relocalize_dev(relo_ctx *ctx, int32_t map_id, const float *ranges_dev, const float *angles,
                        int32_t n_beams, float max_range, relo_result *result_dev);

/* Served form (continuous batching).  relo_serve_start starts a worker thread
 * that takes submitted requests in arrival order and runs them as batches
 * (relo_relocalize_batch semantics): up to max_batch requests per batch and
 * up to max_inflight batches on the device at once, each on its own stream,
 * so requests arriving while others run are admitted as soon as a batch slot
 * and memory free up and their work overlaps on the device.  A request is
 * admitted only while the scratch of all requests in flight stays within
 * hbm_budget bytes (0 = no limit); one that cannot fit even alone completes
 * with RELO_E_OVER_BUDGET.  While serving, the calling thread may only use
 * relo_submit, relo_poll and relo_serve_stop on this context.
 * relo_submit copies the scan and returns a ticket; relo_poll returns
 * RELO_PENDING until the request is done, then its status with the result and
 * (optional) the latency from submit to completion in seconds, and forgets
 * the ticket.  relo_serve_stop finishes the queued requests and stops. */
int relo_serve_start(relo_ctx *ctx, int32_t max_batch, int32_t max_inflight, int64_t hbm_budget);
int relo_submit(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                float max_range, int64_t *ticket);
/* relo_submit with a deadline: a request still waiting for admission
 * timeout_s seconds after this call (HBM budget or busy slots) is never
 * launched and completes with RELO_E_TIMEOUT; once admitted it runs to the
 * end.  timeout_s = 0: no deadline (relo_submit); negative or NaN:
 * RELO_E_INVALID_ARG.  The deadline is kept by the serving thread on the
 * host; nothing waits on the device. */
int relo_submit_until(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                      float max_range, double timeout_s, int64_t *ticket);
int relo_poll(relo_ctx *ctx, int64_t ticket, relo_result *out, double *latency_s);
int relo_serve_stop(relo_ctx *ctx);

/* A batch of independent relocalizations (workloads with many requests, and
 * the served form): each request names a loaded map (with its hypotheses), a
 * scan and its sensor geometry; maps, beam counts, hypothesis counts and FoVs
 * may all differ.  Every stage runs once for the whole batch: one launch per
 * stage serves all requests from a device work list (Eq. 13-31 per request,
 * exactly as for a single request).  1 <= n <= 256; ceil(topk / batch) <= 64. */
typedef struct relo_request {
    int32_t map_id;
    const float *ranges;   /* n_beams float32 metres: host memory for relo_relocalize_batch, device memory for _dev */
    const float *angles;   /* n_beams float32 radians, host memory */
    int32_t n_beams;
    float max_range;
    int32_t topk;          /* SMAD survivors scored by TAM for this request; 0 = the context's topk */
} relo_request;
/* Blocking; out[i] receives request i's result.  Returns the first error. */
int relo_relocalize_batch(relo_ctx *ctx, const relo_request *reqs, int32_t n, relo_result *out);
/* Asynchronous on the context stream; results_dev[i] (device memory) receives request i's result. */
int relo_relocalize_batch_dev(relo_ctx *ctx, const relo_request *reqs, int32_t n, relo_result *results_dev);

/* Intermediate outputs of the last relocalization (the first request of the
 * last batch), copied to caller device memory (bytes = capacity of dst_dev;
 * the call fails if it is too small):
 *   RELO_STAGE_SMAD_NUM   int64 [N_h]   SMAD numerators (Eq. 20)
 *   RELO_STAGE_SMAD_M     int32 [N_h]   minimising orientation shift m
 *   RELO_STAGE_SURVIVORS  int32 [K]     hypothesis indices in SMAD order
 *   RELO_STAGE_TAM        float [K x n_orient]  TAM of every scored (survivor, orientation); unscored = NaN
 *   RELO_STAGE_BEST_M     int32 [K]     per-survivor argmax shift m of Eq. 22 (-1 if not scored)
 *   RELO_STAGE_LOCAL_TOPK int32 [n_batches x local_topk]  survivor positions of each batch's local top-k
 *   RELO_STAGE_SCAN_INFO  int64 [10]    N_s, n_orient, n_enum, N_valid, k_retained, sum_real, K, batches,
 *                                       cells entered by all rays of the batch (DDA steps), N_h */
#define RELO_STAGE_SMAD_NUM 0
#define RELO_STAGE_SMAD_M 1
#define RELO_STAGE_SURVIVORS 2
#define RELO_STAGE_TAM 3
#define RELO_STAGE_BEST_M 4
#define RELO_STAGE_LOCAL_TOPK 5
#define RELO_STAGE_SCAN_INFO 6
#define RELO_SCAN_INFO_LEN 10
int relo_get_stage(relo_ctx *ctx, int32_t which, void *dst_dev, int64_t bytes);

/* Ray-cast synthesized scans (Eq. 13) for n cells on a loaded map, for the
 * beam grid the angles define: ranges_dev receives n x N_s uint32 Q16 cell
 * ranges (0 = no hit), hit_dev (optional) n x N_s int32 hit cell indices
 * cy*W+cx (-1 = none).  capacity: elements each output buffer holds; the call
 * fails with RELO_E_INVALID_ARG, writing nothing, when n x N_s exceeds it.
 * *ns_out receives N_s. */
int relo_synth_scans_dev(relo_ctx *ctx, int32_t map_id, const int32_t *cells_dev, int32_t n, const float *angles,
                         int32_t n_beams, float max_range, uint32_t *ranges_dev, int32_t *hit_dev, int64_t capacity,
                         int32_t *ns_out);

/* Resident synthesized scans.  The panoramic synthesized scan of a
 * hypothesis (Eq. 13) depends on the map, the hypothesis, the beam grid N_s
 * and the range limit only, never on the real scan, so with
 * scan_cache_bytes > 0 the context keeps, per loaded map, one table of
 * N_h x N_s uint32 Q16 ranges for each (N_s, max_range) it has served: the
 * first request with that sensor geometry casts its rays and stores them,
 * later ones read the table instead of casting (the SMAD, TAM and selection
 * results are identical either way).  Tables count against hbm_budget too;
 * beyond scan_cache_bytes the least recently used ones are freed (after the
 * device finishes its queued work).  Loading a new grid into a map
 * (relo_update_map*), setting its hypotheses, unloading it or changing the
 * parameters frees its tables.
 * For each stored table and sensor plan (FoV intervals, Theta) the context
 * also keeps, within the same budget, the window sums W_m of Eq. 18 of every
 * hypothesis sorted ascending: they do not depend on the real scan either, so
 * the SMAD minimum of Eq. 19-20 becomes a nearest-value search around
 * sum R_real (the same numerator and the same m, ties to the smaller m).
 * relo_scan_cache_stats writes min(n, 7) counters to out: tables held, bytes
 * held (scan and window tables), requests that read a table, requests that
 * cast their rays (and stored them when the budget allowed), tables evicted,
 * window tables held, requests whose SMAD read a window table. */
int relo_scan_cache_stats(relo_ctx *ctx, int64_t *out, int32_t n);

/* Stage timing (tracing).  With profiling on, the context records a CUDA
 * event pair on its stream around every kernel it launches and sums the
 * elapsed device time per stage:
 *   0 EDT map precompute (the occupancy tiles, the walk frames' empty boxes
 *     and the column summaries), 1 scan preparation (a batch that casts no
 *     rays), 2 ray cast (Eq. 13, with the scan preparation), 3 SMAD top-K
 *     (with TAM's work order and endpoint offsets), 4 TAM,
 *   5 batch selection and finalize, 6 SMAD (Eq. 16-20),
 *   7 EDT field pass (d2 and the likelihood field, on the side stream; it
 *     runs beside the next ray cast, so its time includes the shared SMs).
 * relo_stage_times synchronises both streams, writes min(n, RELO_N_STAGES)
 * totals in milliseconds to ms_out and launch counts to launches_out (either
 * may be NULL), and with reset != 0 clears the totals.  Independently of
 * profiling, *kernels_out (optional) receives the number of kernels the
 * context has launched since it was created. */
#define RELO_N_STAGES 8
int relo_set_profiling(relo_ctx *ctx, int32_t enable);
/* Profiles only the stages whose bit is set in stage_mask (bit s = stage s
 * above; 0 = off).  Each event pair costs the launch stream a little time, so
 * a caller timing the whole path can bracket only the kernels it needs. */
int relo_set_profiling_mask(relo_ctx *ctx, uint32_t stage_mask);
int relo_stage_times(relo_ctx *ctx, double *ms_out, int64_t *launches_out, int32_t n, int32_t reset,
                     int64_t *kernels_out);

/* Positional hypotheses by the traversability-constrained RRT (Algorithm 1,
 * Sec. III-A, Remark 4) on the GPU: each round draws ceil(W H res^2 / rho^2)
 * random points from a counter-based generator keyed by (seed, round, index)
 * and extends each from its nearest node (adaptive step eta in [r_robot,
 * eta_max] from the clearance there, segment checked every res / 2 for
 * clearance >= r_robot, inside the map); voxels of side rho keep their first
 * node; rounds stop once one adds at most eps_gain voxels (or after
 * max_rounds, or once the tree holds node_cap nodes).  The nearest-node
 * searches of 256 points run at once and the points are then taken in sample
 * order, so the tree is the one-point-at-a-time tree for those random points,
 * in float32 arithmetic rounded at every step.  clearance_dev: float32
 * [h][w] metres to the nearest occupied or unknown cell centre (device).
 * p0x, p0y: the start, metres from the map corner.  seed: the counter-based
 * sampler's key.  node_cap bounds the tree.
 * Writes up to cap representatives (x, y float32 metres, in order of first
 * insertion) to xy_dev and their count, the rounds run and the tree size to
 * n_out, rounds_out, nodes_out (host).  Blocking; allocates its scratch for
 * the call and frees it.  RELO_E_INVALID_ARG for bad sizes, a start off the
 * map or a rho that gives more than 2^26 points per round; RELO_E_CUDA. */
int relo_rrt_hypotheses_dev(relo_ctx *ctx, const float *clearance_dev, int32_t w, int32_t h, double res, double p0x,
                            double p0y, double rho, double eta_max, double r_robot, int32_t eps_gain, uint64_t seed,
                            int32_t max_rounds, int32_t node_cap, float *xy_dev, int32_t cap, int32_t *n_out,
                            int32_t *rounds_out, int32_t *nodes_out);

/* Launch shapes of the batched stages: the knobs the project's autotuner
 * (paper_2511_01219_gb300/autotune.py) sets from measurements.  The paper has
 * no counterpart.  An entry overrides the built-in choice for the launches it
 * matches; key values of 0 match anything; the first matching entry applies.
 *   RELO_TUNE_TAM   key = {values-per-lane class of the request's TAM kernel
 *                   (relo_tam_class), n_orient, K}; val = {survivors per TAM
 *                   task (a multiple of 8 in [8, 128]; 0 keeps the built-in
 *                   choice), resident CTAs per SM of the TAM launch (0: all
 *                   that fit; a launch takes the smallest of its requests')}.
 *   RELO_TUNE_TAM_ONE  as RELO_TUNE_TAM, for a launch that serves a single
 *                   request (its TAM tasks alone fill the GPU, so the best
 *                   shape differs from a mixed batch's); such a launch falls
 *                   back to RELO_TUNE_TAM entries when none matches.
 *   RELO_TUNE_CAST  key = {N_s of the batch's first ray-casting request, 0,
 *                   0}; val = {CTAs per SM of the ray-cast launch (0: all that
 *                   fit), 0}.
 * relo_set_tuning copies the n entries (n = 0 clears the table).  Results do
 * not depend on the shapes, only the time.  RELO_E_INVALID_ARG for a bad kind
 * or value.  relo_tam_class returns the class for a scan of n_beams beams
 * (after the n_skip_beam stride), or -1 if no TAM kernel holds it. */
#define RELO_TUNE_TAM 1
#define RELO_TUNE_CAST 2
#define RELO_TUNE_TAM_ONE 3
typedef struct relo_tune_entry {
    int32_t kind;
    int32_t key[3];
    int32_t val[2];
} relo_tune_entry;
int relo_set_tuning(relo_ctx *ctx, const relo_tune_entry *entries, int32_t n);
int relo_tam_class(int32_t n_beams);

/* Hypotheses by Algorithm 1 (the traversability-constrained RRT of Sec.
 * III-A with NearestNode, AdaptiveExpandDist, ExtendPoint,
 * TraversabilityCheck and VoxelDownsample, and the gain stop of Remark 4)
 * from the occupancy grid itself.  grid: host int8 [h][w], row-major, the
 * cell values of relo_load_map; the RRT stands only on traversable cells
 * (0 <= v < 65: unknown v < 0 and occupied v >= 65 are blocked, as is the
 * outside of the map).  MinDistToObstacle (Sec. III-A item 3) is a per-cell
 * clearance table built on the device by the library's exact EDT: res times
 * the distance from the cell centre to the nearest blocked cell centre, the
 * cells just outside the map counting as blocked (FP64 square root and
 * product, rounded once to float32).  The tree then grows as in
 * relo_rrt_hypotheses_dev with that table (same arguments).  Writes up to cap
 * representatives (x, y metres from the map corner, in order of first
 * insertion; float32 values widened) to the host array xy_out [cap][2], their
 * count, the rounds run and the tree size to n_out, rounds_out, nodes_out,
 * and, if clearance_out is not NULL, the clearance table (host float [h][w],
 * metres).  Blocking; allocates its device scratch for the call and frees it.
 * RELO_E_INVALID_ARG for bad sizes (w, h in [1, 16382]), a start off the map
 * or a rho that gives more than 2^26 points per round; RELO_E_OVER_BUDGET if
 * the scratch exceeds the context's HBM budget; RELO_E_CUDA. */
int relo_rrt_sample(relo_ctx *ctx, const int8_t *grid, int32_t w, int32_t h, double res, double p0x, double p0y,
                    double rho, double eta_max, double r_robot, int32_t eps_gain, uint64_t seed, int32_t max_rounds,
                    int32_t node_cap, double *xy_out, int32_t cap, int32_t *n_out, int32_t *rounds_out,
                    int32_t *nodes_out, float *clearance_out);

/* Allocation-free EDT.  The paper has no counterpart to this entry point; it
 * serves callers that may not allocate device memory once running, such as a
 * robot's real-time localisation loop that allocates only at start-up, or a
 * framework that owns all device memory through its own pool.
 * Computes the exact squared EDT of grid_dev (int8, row-major, w x h, value
 * >= 65 occupied) into d2_dev (int32, row-major, cells^2, -1 when the grid
 * has no occupied cell), asynchronously on stream (a cudaStream_t; NULL = the
 * default stream), with no context and no allocation: the caller owns the
 * input and the output, and the scratch is a file-scope device array of
 * fixed size (4.5 MiB per device, held until the process exits).
 * Returns RELO_E_INVALID_ARG for null pointers or w, h outside [1, 1024],
 * RELO_E_CUDA if a CUDA call or a launch fails, or if a CUDA error from
 * earlier work is already pending in the calling thread (nothing is then
 * launched and that error is left pending).  The first call on a device looks
 * up the scratch address with that device current: make it before any stream
 * capture.  That address is kept until the process exits, so after
 * cudaDeviceReset, or any other reset of the device's primary context, do not
 * call this entry point on that device again in the same process.  Calls
 * share the scratch, so calls that overlap on the GPU race. */
int relo_edt_noalloc(const int8_t *grid_dev, int32_t w, int32_t h, int32_t *d2_dev, void *stream);

/* L2 bandwidth probes: the denominators of the scoring kernels' L2 roofline
 * (the TAM field and the synthesized ranges are L2-resident, so HBM copy
 * bandwidth does not bound those kernels).  The paper has no counterpart.
 * relo_probe_l2_stream reads the device buffer buf_dev (bytes: a multiple of
 * 16; 16-byte aligned; small enough to stay in L2) once untimed to bring it
 * into L2, then `passes` times with 16-byte loads from every SM, and writes the
 * device time of those passes (ms) to *ms: bytes * passes / time is the
 * streaming L2 read rate.  relo_probe_l2_gather first reads the uint16 array
 * buf_dev of 2^log2_elems elements (log2_elems in [10, 31]) once, then makes
 * at least `gathers` 2-byte loads at uniformly random positions (eight in
 * flight per thread), writing the time to *ms and the loads made to
 * *gathers_done.  Both run on stream (NULL = default), block until done, write
 * no device memory and allocate none.  RELO_E_INVALID_ARG for null pointers
 * and bad sizes, RELO_E_CUDA if a CUDA call fails. */
int relo_probe_l2_stream(const void *buf_dev, int64_t bytes, int32_t passes, void *stream, float *ms);
int relo_probe_l2_gather(const uint16_t *buf_dev, int32_t log2_elems, int64_t gathers, void *stream, float *ms,
                         int64_t *gathers_done);

#ifdef __cplusplus
}
#endif
#endif /* RELO_H */
