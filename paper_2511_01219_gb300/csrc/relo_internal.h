// Internal declarations shared by the library's CUDA and host sources.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace relo {

constexpr int kTile = 8;               // field and bitmap are stored in 8x8-cell tiles
constexpr int kMaxClamp = 8100;        // C = (d_max/res)^2 <= 90^2 so the TAM table fits shared memory
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
    uint16_t *field = nullptr;  // [TH*TW*64] min(d2, C), 8x8 tiles
    uint64_t *bits = nullptr;   // [TH*TW] occupancy, bit (y&7)*8 + (x&7)
    int32_t *colsq = nullptr;   // [H*W] EDT column-pass scratch
    int2 *summ = nullptr;       // [S*W] EDT column-segment summaries (scratch)
    int8_t *grid = nullptr;     // [H*W] device copy of the grid
};

// rows per column segment of the EDT column pass: at least 16, at most 64 segments
__host__ __device__ inline int edt_segment_rows(int H) {
    int L = (H + 63) / 64;
    return L < 16 ? 16 : L;
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

struct RayArgs {
    const uint64_t *bits;
    int W, H, TW;
    const int2 *D;          // [ns] Q30 directions
    int ns, ns_pad;         // ns_pad = ns rounded up to 32
    int lim;                // floor(rmax_q16^2 / 2^32): max squared cell distance of an entered cell
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

struct TamArgs {
    const uint16_t *field;
    int W, H, TW, C;
    const int2 *D;
    int ns;
    const int2 *vbR;            // [n_valid] (b_i, R_i) of the valid beams
    const ScanInfo *scan;
    const int32_t *survivors;   // SMAD order
    int s_begin, s_end;
    const int2 *hyps;
    int n_orient, n_enum;
    const float2 *lut;          // [C+1] (l(b), sqrt(C) - sqrt(b))
    float res, res2, d_max, d_min;
    float *T;                   // [K * n_orient]
    unsigned long long *best_key;   // [K] (T bits << 32) | (0xffffffff - q)
    const SelectState *state;
    int chunk, n_chunks;        // survivors per task and tasks per orientation (set by the launcher)
};

cudaError_t launch_edt(const MapDev &m, cudaStream_t s);
cudaError_t launch_map_tables(const MapDev &m, int32_t *d2, uint16_t *field, uint8_t *occ, cudaStream_t s);
cudaError_t launch_check_cells(const int2 *cells, int n, const MapDev &m, int *bad, cudaStream_t s);
cudaError_t launch_raycast_smad(const RayArgs &a, int n_sm, cudaStream_t s);
cudaError_t launch_synth(const RayArgs &a, uint32_t *ranges, int32_t *hit, cudaStream_t s);
cudaError_t launch_topk(const unsigned long long *keys, int n, int K, int32_t *out, cudaStream_t s);
cudaError_t launch_scan_prep(const float *ranges, int n, int skip, float max_range, double res, const int32_t *b,
                             double a_mid, double a_low, int2 *vbR, ScanInfo *info, cudaStream_t s);
cudaError_t launch_tam(const TamArgs &a, int n_beams_max, int n_sm, cudaStream_t s);
cudaError_t launch_select_batch(const unsigned long long *best_key, int s_begin, int s_end, int n_orient,
                                int n_enum, int local_topk, int batch_idx, double tau, int early_stop,
                                int32_t *best_m, int32_t *local_out, SelectState *st, cudaStream_t s);

struct FinalizeArgs {
    const SelectState *st;
    const int32_t *survivors;
    const int32_t *best_m;
    const int2 *hyps;
    const long long *smad_num;
    const ScanInfo *scan;
    double res, ox, oy, fov_beams;
    int ns;
    long long n_smad_evals;
    void *result;   // relo_result*
};
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);

}  // namespace relo
