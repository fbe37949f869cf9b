// Internal declarations shared by the library's CUDA and host sources.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace relo {

constexpr int kTile = 8;               // the occupancy bitmap is stored in 8x8-cell tiles
// metric codes of relo_params::coarse_metric / fine_metric
constexpr int kCoarseCaer = 1;
constexpr int kFineTamMean = 1, kFineBaseline = 2, kFineLF = 3;

// An unsigned code of a float that orders like the float (negative scores
// too, as the log-likelihood sum of Eq. 32 is): sign bit set for >= 0 floats,
// every bit flipped for negative ones.  0 lies below every finite score.
__host__ __device__ inline unsigned int score_code(float f) {
    unsigned int u;
    memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float score_of(unsigned int c) {
    const unsigned int u = (c & 0x80000000u) ? (c & 0x7fffffffu) : ~c;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

constexpr int kMaxClamp = 8100;        // C = (d_max/res)^2 <= 90^2 so the TAM table fits shared memory
constexpr int kMaxLatticePoints = 25445;   // integer (dy, dx) with dy^2 + dx^2 <= kMaxClamp
constexpr int kMaxValidBeams = 2048;   // register-resident TAM selection holds <= 64 values per lane
constexpr int kMaxNs = 8192;           // panoramic beam count
constexpr int kMaxTopk = 4096;
constexpr int kMaxBatch = 1024;
constexpr int kHypBits = 21;           // SMAD key = numerator << 21 | hypothesis index
constexpr int kD2None = -1;            // exported d2 of a map without occupied cells

// Device-side tables of one loaded map.
struct MapDev {
    int W = 0, H = 0, TW = 0, TH = 0;
    int C = 0;                  // clamp (d_max / res)^2 used by the TAM field
    int32_t *d2 = nullptr;      // [H*W] exact squared EDT, -1 = no obstacle
    uint16_t *field = nullptr;  // [Hp * Wp] min(d2, C) with a border of P cells holding C, in 8-row bands
    int P = 0, Wp = 0, Hp = 0;  // border width; padded width and height (W + 2P, H + 2P rounded up to 8)
    uint64_t *bits = nullptr;   // occupancy, bit (y&7)*8 + (x&7): [TH*TW] the map (cells outside free), then the
                                // four walk frames (walk_frame_words each: native, mirrored in x, y and both)
    uint16_t *reach = nullptr;  // per walk-frame tile, the empty boxes of tiles ahead, then scratch (walk_reach_bytes);
                                // nullptr: no ray is cast on this map
    int32_t *colsq = nullptr;   // [H*W] EDT column-pass scratch
    int2 *summ = nullptr;       // [S*W] EDT column-segment summaries (scratch)
    int8_t *grid = nullptr;     // [H*W] device copy of the grid
};

// The clamped field is stored in bands of 8 rows, each band column by
// column: cell (x, y) of the padded grid (the map cell (x - P, y - P)) sits at
// element 8 ((y / 8) Wp + x) + y % 8.  A 128-byte cache line then holds an
// 8 x 8 block of cells (x a multiple of 8), so the endpoints of neighbouring
// beams, which lie close together in x and in y, share lines; and the index
// stays linear in x, so an endpoint offset (dx, dy) from a cell depends on the
// cell only through y % 8 (its band phase).
__host__ __device__ inline size_t field_index(int x, int y, int Wp) {
    return (((size_t)(y >> 3) * (unsigned)Wp + (unsigned)x) << 3) + (unsigned)(y & 7);
}

// rows per column segment of the EDT column pass: at least 16, at most 64
// segments, a multiple of 8 (the segment pass also builds the 8x8 tiles)
__host__ __device__ inline int edt_segment_rows(int H) {
    int L = (H + 63) / 64;
    L = L < 16 ? 16 : L;
    return (L + 7) & ~7;
}

// A walk frame holds TW+1 x TH+1 tiles: the map's tiles with every cell
// outside the map set, plus a last column and row of tiles with every bit set,
// so a ray that leaves the map (always towards +x, +y in its frame) meets a set
// bit at its first cell outside.
__host__ __device__ inline size_t walk_frame_words(int TW, int TH) { return (size_t)(TW + 1) * (TH + 1); }
__host__ __device__ inline size_t occupancy_words(int TW, int TH) {
    return (size_t)TW * TH + 4 * walk_frame_words(TW, TH);
}

// Empty boxes ahead.  For every tile (tx, ty) of a walk frame, reach packs
// three boxes of empty tiles that start at it, each side at most kReachMax
// (all 0 when the tile itself is not empty): bits 0-4 the side s of the
// largest square [tx, tx + s) x [ty, ty + s), bits 5-9 the run [tx, tx + r) x
// {ty} along the tile's row, bits 10-14 the run {tx} x [ty, ty + r) along its
// column.  A ray in that tile moves towards +x and +y, so every cell it enters
// before it leaves a box lies inside it: the walk may leave the whole box in
// one move.  The walk frames' last column and row are full, so a box never
// leaves the map.
constexpr int kReachMax = 16;
// Hypotheses one ray-cast work item takes, for one chunk of 32 directions
// (the directions' setup is then done once for all of them): at most
// kCastHypsMax, fewer when the batch has too few rays to give every resident
// warp some 16 items after grouping (the last wave's tail would grow).
constexpr int kCastHypsMax = 4;
__host__ __device__ inline long long cast_chunks(int n_hyp, int ns, int per_item) {
    return (long long)((n_hyp + per_item - 1) / per_item) * (((ns + 31) & ~31) >> 5);
}
// words per frame row of the tiles' emptiness bits (one more than the row needs: the 64-tile window of a row's last
// 32 tiles reads it)
__host__ __device__ inline unsigned walk_empty_row_words(int TW) { return ((unsigned)TW + 1u + 31u) / 32u + 1u; }
// MapDev::reach: the packed boxes [4][TH + 1][TW + 1], then the emptiness bits [4 (TH + 1)][walk_empty_row_words]
__host__ __device__ inline size_t walk_reach_bytes(int TW, int TH) {
    const size_t boxes = (4 * walk_frame_words(TW, TH) * sizeof(uint16_t) + 15) & ~(size_t)15;
    return boxes + (size_t)4 * ((size_t)TH + 1) * walk_empty_row_words(TW) * sizeof(uint32_t);
}
__host__ __device__ inline uint32_t *walk_empty_bits(uint16_t *reach, int TW, int TH) {
    return reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(reach) +
                                        ((4 * walk_frame_words(TW, TH) * sizeof(uint16_t) + 15) & ~(size_t)15));
}

__host__ __device__ inline size_t tile_index(int x, int y, int TW) {
    return ((size_t)(y >> 3) * TW + (x >> 3)) * 64 + ((y & 7) << 3) + (x & 7);
}

// Per-scan values produced on the device by the scan-preparation kernel.
struct ScanInfo {
    long long sum_real;             // sum of valid Q16 ranges (Eq. 16 numerator)
    int n_valid;                    // N of Eq. 26 (valid beams)
    int k_ret;                      // median of {k_full, k_mid, k_low} (Eq. 26-27)
    unsigned long long dda_steps;   // cells entered by all rays of the request (work counter)
    unsigned int ray_work;          // next hypothesis for the ray-cast CTAs
    int pad[1];
};

// Running state of the batched selection of one request.
struct SelectState {
    unsigned long long best;   // (T bits << 32) | (0xffffffff - survivor position)
    long long n_tam_evals;
    int n_batches;
    int done;                  // early termination reached
};

// Per-direction traversal tables of one beam grid N_s and range limit lim.
// Every ray starts at a cell centre and follows the integer DDA of its
// direction, so the sequence of x- and y-steps of direction j is the same for
// every hypothesis; the tables describe it once.  Layout [row][j] (row-major,
// N_s entries per row) so the lanes of a warp, which trace neighbouring
// directions, read neighbouring entries.
//   selx[n][j]: index k of the step that makes the n-th x-step (k counts
//               the cells entered, k = |dx| + |dy|); 0xffff when that cell
//               lies beyond the range limit.  sely likewise for y-steps.
//   mask[k][j]: the cells the ray enters after entering cell k (cell k
//               included for k > 0), up to 7 cells further in x and in y
//               and within the range limit, as an 8x8 bit board anchored at
//               cell k: bit 8 |dy| + |dx| for the offsets (dx, dy).
//   kmax[j]:   the last cell index within the range limit.
struct RayTables {
    const uint64_t *mask;
    const uint16_t *selx, *sely;
    const int32_t *kmax;
};
constexpr uint32_t kSelNone = 0xffffu;

// rows of the tables for a range limit lim (cells^2)
__host__ __device__ inline int ray_mask_rows(int lim) {
    // a cell k steps out has |d|^2 >= k^2 / 2, so k <= sqrt(2 lim)
    int k = (int)sqrt(2.0 * (double)lim);
    while ((long long)(k + 1) * (k + 1) <= 2ll * lim) ++k;
    while ((long long)k * k > 2ll * lim) --k;
    return k + 1;
}
__host__ __device__ inline int ray_sel_rows(int lim) {
    int r = (int)sqrt((double)lim);
    while ((long long)(r + 1) * (r + 1) <= (long long)lim) ++r;
    while ((long long)r * r > (long long)lim) --r;
    return r + 8 * kReachMax + 1;   // a cell in range has |dx| <= sqrt(lim); leaving a square adds at most 8 kReachMax
}

// single-request arguments of the synthesized-scan export (relo_synth_scans_dev)
struct RayArgs {
    const uint64_t *bits;   // the map's four occupancy frames (MapDev::bits)
    const uint16_t *reach;  // their empty boxes ahead (MapDev::reach)
    int W, H, TW, TH;
    const int2 *D;          // [ns] Q30 directions
    int ns, ns_pad;         // ns_pad = ns rounded up to 32
    int lim;                // floor(rmax_q16^2 / 2^32): max squared cell distance of an entered cell
    RayTables tab;          // per-direction tables, or tab.mask == nullptr to step cell by cell
    const int2 *hyps;
    int n_hyp;
    const int2 *iv;         // [n_iv] (u, len) FoV intervals
    int n_iv;
    const ScanInfo *scan;
    unsigned long long *dda_steps;   // optional work counter (may be null)
    unsigned int *work;              // hypothesis counter, zero at launch
    int n_enum, n_m;        // orientation stride and count scored by SMAD
    unsigned long long *keys;   // [n_hyp]
    long long *smad_num;        // [n_hyp]
    int32_t *smad_m;            // [n_hyp]
};

// Everything one relocalization request needs on the device: its map's
// tables, its hypotheses, its sensor plan, its scan and its output buffers.
// A batch is an array of these; every stage kernel serves all requests of a
// batch from one launch.
struct ReqDesc {
    // map tables
    const uint64_t *bits;
    const uint16_t *reach;       // empty boxes ahead in the walk frames (MapDev::reach)
    const uint16_t *field;       // padded clamped field (8-row bands, field_index), pointer to padded cell (0, 0)
    int coarse, fine;            // ranking and scoring metrics (RELO_COARSE_*, RELO_FINE_*)
    int icp_iters;               // ICP iterations per local top-k pose (0: no refinement)
    const int32_t *d2map;        // [H*W] exact squared EDT, -1 = no obstacle (ICP pairs)
    const int8_t *grid;          // [H*W] the occupancy grid (ICP pairs)
    const int32_t *sq_off;       // [C+2] start of the offsets with dy^2 + dx^2 = n in sq_rep, for n in [0, C + 1]
    const short2 *sq_rep;        // (dy, dx) offsets by n, each n's ordered by dy, then dx (the ICP pairing order)
    double *ref_pose;            // [K][3] refined pose (x, y, theta) of each refined survivor (map metres)
    float *reev;                 // [K] its re-evaluated score
    const float2 *lut;           // [C+2] (l(b), sqrt(C) - sqrt(b)); entry C+1 = (0, 0) marks "no beam"
    int W, H, TW, TH, C, Wp, P;
    float res, res2, d_max, d_min;
    double resd, ox, oy;
    // hypotheses
    const int2 *hyps;
    int n_hyp;
    // sensor plan
    const int2 *D;               // [ns] Q30 directions
    const int32_t *b;            // [n_beams] panoramic index per beam
    const int2 *iv;              // [n_iv] (u, len) FoV intervals
    int ns, ns_pad, n_iv, n_beams, n_orient, n_enum, n_m;
    int lim;                     // floor(rmax_q16^2 / 2^32)
    RayTables rt;                // per-direction traversal tables, or rt.mask == nullptr
    double a_mid, a_low, fov;
    // scan input
    const float *ranges;
    int skip;
    float max_range;
    // selection
    int K, B, n_batches, L, early_stop;
    double tau;
    long long n_smad_evals;
    // buffers
    int2 *vbR;                   // [n_beams]
    int32_t *Rall;               // [n_beams] every beam's Q16 range in beam order, 0 for an invalid beam (CAER)
    ScanInfo *scan;
    unsigned long long *keys;    // [n_hyp]
    long long *smad_num;         // [n_hyp]
    int32_t *smad_m;             // [n_hyp]
    int32_t *survivors;          // [K]
    // TAM's work order: within each batch the survivor positions grouped by the band phase (y + P) % 8 of
    // their cell, cut into chunks of at most tam_chunk of one phase: (phase, first, end) into surv_perm;
    // the chunks of batches < b are tam_chunks[0, chunk_cnt[b])
    int32_t *surv_perm;          // [K]
    int32_t *tam_offs;           // [8][n_orient][32][tam_stride] TAM endpoint offsets by band phase (tam_offsets.cuh)
    int tam_stride;              // slots per lane in tam_offs
    int4 *tam_chunks;            // [sum over batches of ceil(n_b / tam_chunk) + 8]
    int32_t *chunk_cnt;          // [n_batches + 1]
    int tam_chunk;
    float *T;                    // [K * n_orient]
    unsigned long long *best_key;   // [K]
    int32_t *best_m;             // [K]
    int32_t *local;              // [n_batches * L]
    SelectState *state;
    void *result;                // relo_result in device memory
    // work lists
    int hyp_base;                // first slot of this request in the batch's hypothesis list
    // synthesized scans of (map, hypotheses, N_s, lim): [n_hyp * ns] Q16 ranges, row per hypothesis
    uint32_t *scan_table;
    int scan_mode;               // kScanCast, kScanStore or kScanRead
    int chunk_base;              // first 32-ray chunk of this request in the batch's cast list
    int cast_hyps;               // hypotheses per ray-cast work item (1, 2 or 4; the same for the whole batch)
    // resident window sums of (map, hypotheses, N_s, lim, intervals, Theta): per hypothesis the n_m keys
    // W_m << 13 | q (W_m the window sum of Eq. 18 at m = q n_enum), ascending
    unsigned long long *win;
    int win_mode;                // kWinNone (SMAD from the ranges), kWinBuild or kWinRead
    int wbuild_base, wread_base; // first slot of this request in the window-build / window-read lists
};

// SMAD by window tables.  W_m depends on the map, the hypothesis and the
// sensor plan, never on the real scan, so min over m of |sum R_real - W_m|
// (Eq. 19-20) is a nearest-value search in the sorted W_m.
constexpr int kWinNone = 0;
constexpr int kWinBuild = 1;     // SMAD from the ranges, and the sorted keys stored into win
constexpr int kWinRead = 2;      // SMAD by binary search in win
constexpr int kWinQBits = 13;    // q < 8192 = kMaxNs

// Where a request's synthesized ranges come from.  The cast kernel writes
// them into scan_table (request scratch for kScanCast, a resident table for
// kScanStore); kScanRead requests have no chunks, their table was written by
// an earlier launch.  The SMAD kernel reads scan_table in every mode.
constexpr int kScanCast = 0;
constexpr int kScanStore = 1;
constexpr int kScanRead = 2;

// Counters shared by the whole batch.
struct BatchState {
    unsigned int ray_work;          // next global hypothesis slot for the SMAD CTAs
    unsigned int cast_work;         // next global 32-ray chunk for the cast warps
    unsigned long long dda_steps;   // cells entered by all rays of the batch
};

// TAM work of one request in one launch: the survivors of its batches
// [batch_lo, batch_hi) (none when equal), for each of its orientations.  The
// launch's tasks are (chunk of same-phase survivors, block of orientations);
// the chunks are built on the device (by the top-K launch).
struct TamSeg {
    int batch_lo, batch_hi;
};

constexpr int kMaxBatchRequests = 256;
// survivors of one band phase per TAM task: the most (up to 64, a multiple of
// 8) that still leave about three tasks (blocks of 4 orientations) per
// resident CTA of five per SM, so the launch is not one ragged wave
inline int tam_chunk_for(int K, int n_orient, int n_sm) {
    const long long tasks_per_survivor = (n_orient + 3) / 4;
    long long c = (long long)K * tasks_per_survivor / (3ll * 5 * n_sm);
    c = c / 8 * 8;
    return (int)(c < 8 ? 8 : c > 64 ? 64 : c);
}
// chunks of the TAM work order: per group of survivors (each batch, or all K as one group), its survivors in
// chunks of one phase (at most one part chunk per phase); the per-batch count bounds both
inline int tam_chunk_cap(int K, int B, int n_batches, int chunk) {
    int cap = 0;
    for (int b = 0; b < n_batches; ++b) {
        const int n = (K - b * B < B ? K - b * B : B);
        cap += (n + chunk - 1) / chunk + 8;
    }
    return cap;
}
constexpr int kMaxBatches = 64;      // ceil(K / batch) limit, bounds the TamSeg table

cudaError_t launch_edt(const MapDev &m, cudaStream_t s);          // interior of the field, d2, bitmap
// the same in two parts: the occupancy tiles and column summaries (all the ray cast needs), then, reading the
// summaries and the grid, the column terms, d2 and the interior of the field (TAM and ICP)
cudaError_t launch_edt_tiles(const MapDev &m, cudaStream_t s);
cudaError_t launch_edt_field(const MapDev &m, cudaStream_t s);
cudaError_t launch_field_border(const MapDev &m, cudaStream_t s); // the constant borders of the field and walk frames (once per map)
cudaError_t launch_map_tables(const MapDev &m, int32_t *d2, uint16_t *field, uint8_t *occ, cudaStream_t s);
cudaError_t launch_check_cells(const int2 *cells, int n, const MapDev &m, int *bad, cudaStream_t s);
// metre coordinates (n (x, y) FP64 pairs on the device) to cells; flags[0] off the map, flags[1] on occupied cells
cudaError_t launch_xy_cells(const double *xy, int n, double ox, double oy, double res, const MapDev &m, int2 *cells,
                            int *flags, cudaStream_t s);
cudaError_t launch_synth(const RayArgs &a, uint32_t *ranges, int32_t *hit, cudaStream_t s);
// fills the traversal tables of directions D[0, ns) for range limit lim (buffers sized by ray_*_rows)
cudaError_t launch_ray_tables(const int2 *D, int ns, int lim, uint64_t *mask, uint16_t *selx, uint16_t *sely,
                              int32_t *kmax, cudaStream_t s);

// batched stages; R requests, descriptors in device memory
// scan preparation alone, for a batch that casts no rays (launch_cast does it otherwise)
cudaError_t launch_scan_prep(const ReqDesc *reqs, int R, cudaStream_t s);
// casts the total_chunks 32-ray chunks of the batch into the requests' scan tables
cudaError_t launch_cast(const ReqDesc *reqs, int R, int total_chunks, int cast_hyps, BatchState *bs, int n_sm, int ctas_per_sm,
                        cudaStream_t s);
// SMAD of every hypothesis of the batch from the requests' scan tables
cudaError_t launch_smad(const ReqDesc *reqs, int R, int total_hyp, int max_ns_pad, BatchState *bs, int n_sm,
                        cudaStream_t s);
// the same SMAD by direct window sums, without the prefix sums of Eq. 17 (the Table II ablation)
cudaError_t launch_smad_direct(const ReqDesc *reqs, int R, int total_hyp, int max_ns_pad, BatchState *bs, int n_sm,
                               cudaStream_t s);
// no coarse ranking: numerator 0 and m = 0 for every hypothesis of the batch (Table II's arm without SMAD ordering)
cudaError_t launch_rank_by_index(const ReqDesc *reqs, int R, int total_hyp, int n_sm, cudaStream_t s);
// SMAD of the window-build requests' hypotheses, storing their sorted window keys
cudaError_t launch_win_build(const ReqDesc *reqs, int R, int total, int max_ns_pad, int max_nm, cudaStream_t s);
// SMAD of the window-read requests' hypotheses by search in their window keys
cudaError_t launch_win_read(const ReqDesc *reqs, int R, int total, cudaStream_t s);
// the top-K of every request with its TAM work order, and beside it (extra blocks) every request's TAM endpoint offsets
cudaError_t launch_topk(const ReqDesc *reqs, int R, int max_n_hyp, int max_K, int max_n_orient, int n_sm, cudaStream_t s);
// plans the TAM launch of one batch index: fills segs[R] and returns the task count and grid size
struct TamPlan {
    int total_tasks, grid, vpl;
    size_t smem;
    bool h2;   // selection counts on packed fp16 (table slot of C + 1 at most 6143: C <= 5956)
};
// values per lane the TAM kernel holds for max_beams valid beams (-1 if too many)
int tam_vpl_for(int max_beams);
// the planned launch for the batches [batch_lo[r], batch_hi[r]) of each request r: segs[R], grid and kernel class
TamPlan plan_tam(const int *batch_lo, const int *batch_hi, int R, int max_beams, int max_C, int n_sm,
                 int ctas_per_sm, TamSeg *segs);
// TAM's work order (surv_perm, tam_chunks, chunk_cnt) of every request, after the top-K
// per-lane stride of the TAM endpoint offsets of a values-per-lane class
int tam_offs_stride_for(int vpl);
// every request's TAM endpoint offsets for all band phases and orientations (after the scan preparation)
cudaError_t launch_tam(const ReqDesc *reqs, int R, const TamSeg *segs, const TamPlan &tp, cudaStream_t s);
// selection of batch indexes batch_lo .. batch_hi - 1 in order; with last, also every request's result.
// With icp, only the local top-k (launch_icp and launch_icp_best take the rest).
cudaError_t launch_select_batch(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, bool last, bool icp,
                                cudaStream_t s);
// ICP refinement and re-evaluation of the local top-k of batches batch_lo .. batch_hi - 1, then their best,
// early termination and (with last) the results
cudaError_t launch_icp(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, int max_L, int max_beams,
                       cudaStream_t s);
cudaError_t launch_icp_best(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, bool last, cudaStream_t s);
// Algorithm 1 in batched-expansion form (rrt.cu); blocking on s; *err names a failure
// the RRT's blocked grid with a ring of blocked cells ((W + 2) x (H + 2), occupied = 100) and, from the squared
// EDT of that grid, the clearance table res * sqrt(d2) (metres, W x H)
cudaError_t launch_rrt_blocked(const int8_t *grid, int W, int H, int8_t *out, cudaStream_t s);
cudaError_t launch_rrt_clearance(const int32_t *d2p, int W, int H, double res, float *clr, cudaStream_t s);
int rrt_sample_dev(const float *clr, int W, int H, double res, double p0x, double p0y, double rho, double eta_max,
                   double r_robot, int eps_gain, uint64_t seed, int max_rounds, int node_cap, float *xy_out, int cap,
                   int *n_out, int *rounds_out, int *nodes_out, cudaStream_t s, const char **err);

}  // namespace relo
