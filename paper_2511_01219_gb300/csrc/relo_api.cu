// Host side of the C ABI declared in include/relo.h: contexts, map slots,
// hypothesis sets, the per-sensor plan (Eq. 11-15) and the launch sequence of
// a batch of relocalizations.  All scoring arithmetic runs in the library's
// kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/relo.h"
#include "relo_internal.h"

using namespace relo;

namespace {

struct SensorPlan {
    std::vector<float> angles;   // key: the (downsampled) angles the plan was built from
    int n_skip = 1, n_orient_param = 0;
    int n = 0, ns = 0, n_orient = 0, n_enum = 1, n_m = 1;
    double lam = 0, a_mid = 0, a_low = 0;
    long long fov = 0;
    std::vector<int32_t> b;
    std::vector<int2> D, iv;
    int32_t *b_dev = nullptr;
    int2 *D_dev = nullptr, *iv_dev = nullptr;
    size_t bytes = 0;
    unsigned long long last_use = 0;
};

// Resident synthesized scans of one map and hypothesis set for one beam grid
// N_s and range limit: [n_hyp * ns] uint32 Q16 ranges, row per hypothesis.
// Sorted window sums of one scan table for one sensor plan (intervals, Theta).
struct WinTable {
    int n_enum = 0, n_m = 0;
    std::vector<int2> iv;
    unsigned long long *keys = nullptr;   // [n_hyp][n_m] W_m << 13 | q, ascending per hypothesis
    size_t bytes = 0;
    cudaEvent_t built = nullptr;          // recorded after the kernel that builds it
};

struct ScanTable {
    int ns = 0, lim = 0;
    uint32_t *data = nullptr;
    size_t bytes = 0;
    cudaEvent_t written = nullptr;    // recorded after the ray-cast launch that stores the table
    unsigned long long last_use = 0;
    unsigned long long pin = 0;       // batch sequence number of the last batch that used it
    std::vector<WinTable *> wins;     // derived window tables (freed with the scan table)
};

// Per-direction traversal tables of one (N_s, range limit); see RayTables.
struct RayTab {
    int ns = 0, lim = 0;
    uint64_t *mask = nullptr;
    uint16_t *selx = nullptr, *sely = nullptr;
    int32_t *kmax = nullptr;
    size_t bytes_mask = 0, bytes_sel = 0;
    cudaEvent_t built = nullptr;      // recorded after the build kernel
    unsigned long long last_use = 0;
    unsigned long long pin = 0;       // batch sequence number of the last batch that used it
};

constexpr int kMaxRayTabs = 16;
constexpr size_t kMaxRayTabBytes = size_t(1) << 29;   // larger tables fall back to cell-by-cell stepping

struct MapSlot {
    bool live = false;
    MapDev dev;
    double res = 0, ox = 0, oy = 0;
    int2 *hyps = nullptr;
    int n_hyp = 0, hyp_cap = 0;
    float2 *lut = nullptr;
    int32_t *sq_off = nullptr;   // [kMaxClamp + 2] and [kMaxLatticePoints]: the cells at each squared distance
    short2 *sq_rep = nullptr;
    size_t bytes = 0;
    std::vector<ScanTable *> tables;
    // the map's EDT runs in two parts: the occupancy tiles on the context stream (tiles_ready), then the field and
    // d2 on the context's side stream (field_ready), overlapping the next request's ray cast
    cudaEvent_t tiles_ready = nullptr, field_ready = nullptr;
};

// One request prepared for a batch.
struct Prepared {
    MapSlot *m;
    SensorPlan *P;
    const float *ranges_dev;
    void *result_dev;
    float max_range;
    int lim, K, B, n_batches;
};

constexpr int kMaxPlans = 32;
constexpr size_t kBlobBytes = 30000;   // kernel-parameter upload size

// Device-to-device upload through kernel parameters: the bytes travel with the
// launch, so no host buffer has to outlive the call and nothing is pinned.
struct Blob {
    unsigned int n;
    unsigned char bytes[kBlobBytes];
};

// copies the blob; with bs, also zeroes the batch's work counters
__global__ void k_upload(const __grid_constant__ Blob blob, unsigned char *dst, BatchState *bs) {
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < blob.n; i += gridDim.x * blockDim.x)
        dst[i] = blob.bytes[i];
    if (bs && blockIdx.x == 0 && threadIdx.x == 0) {
        bs->ray_work = 0u;
        bs->cast_work = 0u;
        bs->dda_steps = 0ull;
    }
}

// Device resources of one batch in flight: its stream, descriptors, TAM
// segments, counters, results, scratch arena and uploaded scans.
struct BatchSlot {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ReqDesc *reqs_dev = nullptr;          // descriptors [R], then the TAM segments [batches * R] (one upload)
    BatchState *bs = nullptr;
    relo_result *results_dev = nullptr;   // [kMaxBatchRequests]
    unsigned char *arena = nullptr;       // per-request scratch of the batch
    size_t arena_cap = 0;
    float *ranges_dev = nullptr;          // uploaded scans
    size_t ranges_cap = 0;
    cudaEvent_t done = nullptr;           // recorded after the batch's last kernel (served form)
};

struct Ticket;

}  // namespace

struct relo_ctx {
    relo_params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, n_sm = 0;
    std::vector<MapSlot> maps;
    std::vector<SensorPlan *> plans;
    unsigned long long plan_clock = 0;
    std::string err;
    long long held = 0;
    // batches run by the calling thread use `main` (on the context stream)
    BatchSlot main;
    int *bad = nullptr;                   // hypothesis check flags [2]
    double *xy = nullptr;                 // metre coordinates of relo_set_hypotheses, staged on the device
    size_t xy_cap = 0;
    // served form
    struct Server *server = nullptr;
    Blob *blob = nullptr;                 // host staging of one upload (heap)
    // stage timing
    unsigned profile_mask = 0;   // stages whose launches are bracketed with events
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double stage_ms[RELO_N_STAGES] = {0};
    long long stage_n[RELO_N_STAGES] = {0};
    long long kernels = 0;
    // the first request of the last batch (for relo_get_stage)
    ReqDesc last{};
    BatchState *last_bs = nullptr;
    bool has_last = false;
    // per-direction traversal tables
    std::vector<RayTab *> raytabs;
    // resident synthesized scans
    long long table_bytes = 0, cache_hits = 0, cache_misses = 0, cache_evictions = 0, win_hits = 0;
    unsigned long long table_clock = 0, batch_seq = 0;
    // launch shapes chosen by the autotuner (relo_set_tuning)
    std::vector<relo_tune_entry> tuning;
    // the second stream the EDT's field pass runs on
    cudaStream_t side = nullptr;
};

namespace {

int fail(relo_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(relo_ctx *c, cudaError_t e, const char *what) {
    return fail(c, RELO_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

cudaEvent_t take_event(relo_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Wraps one kernel launch: counts it and, when its stage is profiled, brackets it with events.
template <typename F>
cudaError_t timed_on(relo_ctx *ctx, cudaStream_t st, int stage, int n_kernels, F &&launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    const bool prof = (ctx->profile_mask >> stage) & 1u;
    if (prof) {
        a = take_event(ctx);
        b = take_event(ctx);
        if (a) cudaEventRecord(a, st);
    }
    cudaError_t e = launch();
    ctx->kernels += n_kernels;
    if (prof && a && b) {
        cudaEventRecord(b, st);
        ctx->pending.push_back({stage, a, b});
    }
    return e;
}

template <typename F>
cudaError_t timed(relo_ctx *ctx, int stage, int n_kernels, F &&launch) {
    return timed_on(ctx, ctx->stream, stage, n_kernels, launch);
}

int dev_alloc(relo_ctx *ctx, void **p, size_t bytes, const char *what) {
    if (ctx->p.hbm_budget > 0 && ctx->held + (long long)bytes > ctx->p.hbm_budget)
        return fail(ctx, RELO_E_OVER_BUDGET, std::string(what) + ": over the context's HBM budget");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(ctx, e, what);
    }
    ctx->held += (long long)bytes;
    return RELO_OK;
}

void dev_free(relo_ctx *ctx, void *p, size_t bytes) {
    if (p) {
        cudaFree(p);
        ctx->held -= (long long)bytes;
    }
}

template <typename T>
int ensure(relo_ctx *ctx, T **p, size_t *cap, size_t need, const char *what) {
    if (need <= *cap && *p) return RELO_OK;
    size_t n = std::max(need, *cap * 3 / 2);
    dev_free(ctx, *p, *cap * sizeof(T));
    *p = nullptr;
    *cap = 0;
    int rc = dev_alloc(ctx, (void **)p, n * sizeof(T), what);
    if (rc == RELO_OK) *cap = n;
    return rc;
}

// the first tuning entry of this kind whose nonzero keys equal k0, k1, k2 (nullptr: none)
const relo_tune_entry *tuned(const relo_ctx *ctx, int kind, int k0, int k1, int k2) {
    for (const relo_tune_entry &e : ctx->tuning)
        if (e.kind == kind && (!e.key[0] || e.key[0] == k0) && (!e.key[1] || e.key[1] == k1) &&
            (!e.key[2] || e.key[2] == k2))
            return &e;
    return nullptr;
}

// TAM launch shape of a request: a launch of one request looks for its own entries first
const relo_tune_entry *tuned_tam(const relo_ctx *ctx, int R, int cls, int n_orient, int K) {
    const relo_tune_entry *e = R == 1 ? tuned(ctx, RELO_TUNE_TAM_ONE, cls, n_orient, K) : nullptr;
    return e ? e : tuned(ctx, RELO_TUNE_TAM, cls, n_orient, K);
}

static_assert(kCoarseCaer == RELO_COARSE_CAER && kFineTamMean == RELO_FINE_TAM_MEAN &&
                  kFineBaseline == RELO_FINE_BASELINE && kFineLF == RELO_FINE_LF,
              "metric codes");

int check_params(relo_ctx *ctx, const relo_params &p) {
    if (!(p.z_hit > 0) || !(p.sigma_hit > 0) || !(p.z_rand >= 0) || !(p.eps > 0))
        return fail(ctx, RELO_E_INVALID_ARG, "Eq. 23 needs z_hit > 0, sigma_hit > 0, z_rand >= 0, eps > 0");
    if (!(p.d_max > 0)) return fail(ctx, RELO_E_INVALID_ARG, "d_max must be positive");
    for (double a : {p.a_mid_min, p.a_mid_max, p.a_low_min, p.a_low_max})
        if (!(a > 0 && a <= 1)) return fail(ctx, RELO_E_INVALID_ARG, "retention ratios must lie in (0, 1]");
    if (p.topk < 1 || p.topk > kMaxTopk) return fail(ctx, RELO_E_INVALID_ARG, "topk must be in [1, 4096]");
    if (p.batch < 1 || p.batch > kMaxBatch) return fail(ctx, RELO_E_INVALID_ARG, "batch must be in [1, 1024]");
    if (p.local_topk < 1 || p.local_topk > p.batch)
        return fail(ctx, RELO_E_INVALID_ARG, "local_topk must be in [1, batch]");
    if (p.n_skip_beam < 1) return fail(ctx, RELO_E_INVALID_ARG, "n_skip_beam must be >= 1");
    if (p.n_orient < 0) return fail(ctx, RELO_E_INVALID_ARG, "n_orient must be >= 0");
    if (!(p.max_range > 0)) return fail(ctx, RELO_E_INVALID_ARG, "max_range must be positive");
    if (p.scan_cache_bytes < 0) return fail(ctx, RELO_E_INVALID_ARG, "scan_cache_bytes must be >= 0");
    if (p.coarse_metric < RELO_COARSE_SMAD || p.coarse_metric > RELO_COARSE_NONE)
        return fail(ctx, RELO_E_INVALID_ARG, "coarse_metric must be one of RELO_COARSE_SMAD .. RELO_COARSE_NONE");
    if (p.fine_metric < RELO_FINE_TAM || p.fine_metric > RELO_FINE_LF)
        return fail(ctx, RELO_E_INVALID_ARG, "fine_metric must be one of RELO_FINE_TAM .. RELO_FINE_LF");
    if (p.icp_iters < 0 || p.icp_iters > 1000) return fail(ctx, RELO_E_INVALID_ARG, "icp_iters must be in [0, 1000]");
    return RELO_OK;
}

// border of the padded TAM field: the longest beam in cells, plus one for rounding
int pad_for(double max_range, double res) {
    const double c = ceil(max_range / res) + 1.0;
    return c < 32768.0 ? (int)c : -1;
}

// clamp C = (d_max / res)^2; d_max / res must be an integer
int clamp_for(relo_ctx *ctx, double d_max, double res, int *C) {
    double q = d_max / res;
    long long qi = llround(q);
    if (fabs(q - (double)qi) > 1e-6 || qi < 1 || qi * qi > kMaxClamp)
        return fail(ctx, RELO_E_INVALID_ARG, "d_max / res must be an integer in [1, 90]");
    *C = (int)(qi * qi);
    return RELO_OK;
}

// likelihood table of Eq. 23 and sqrt(C) - sqrt(b), for b in [0, C]
int build_lut(relo_ctx *ctx, MapSlot &m) {
    const relo_params &p = ctx->p;
    const int C = m.dev.C;
    std::vector<float2> h(C + 2);
    const double sc = sqrt((double)C);
    for (int b = 0; b <= C; ++b) {
        double d = m.res * sqrt((double)b);
        double l = log(p.z_hit * exp(-(d * d) / (2.0 * p.sigma_hit * p.sigma_hit)) + p.z_rand + p.eps);
        h[b] = make_float2((float)l, (float)(sc - sqrt((double)b)));
    }
    h[C + 1] = make_float2(0.0f, 0.0f);   // "no beam": contributes nothing
    if (!m.lut) {
        int rc = dev_alloc(ctx, (void **)&m.lut, sizeof(float2) * (kMaxClamp + 2), "likelihood table");
        if (rc) return rc;
        m.bytes += sizeof(float2) * (kMaxClamp + 2);
    }
    CK(cudaMemcpyAsync(m.lut, h.data(), sizeof(float2) * (C + 2), cudaMemcpyHostToDevice, ctx->stream), "lut upload");
    // every (dy, dx) with dy^2 + dx^2 = n <= C, grouped by n and ordered by dy, then dx: the candidates ICP
    // tries, nearest first, when it pairs a beam with an occupied cell
    std::vector<int32_t> off(C + 2, 0);
    std::vector<short2> rep;
    for (int n = 0; n <= C; ++n) {
        off[n] = (int32_t)rep.size();
        const int r = (int)sqrt((double)n) + 1;
        for (int dy = -r; dy <= r; ++dy) {
            const int rest = n - dy * dy;
            if (rest < 0) continue;
            int s = (int)sqrt((double)rest);
            while (s * s > rest) --s;
            while ((s + 1) * (s + 1) <= rest) ++s;
            if (s * s != rest) continue;
            rep.push_back(make_short2((short)dy, (short)-s));
            if (s > 0) rep.push_back(make_short2((short)dy, (short)s));
        }
    }
    off[C + 1] = (int32_t)rep.size();
    if (!m.sq_off) {
        int rc = dev_alloc(ctx, (void **)&m.sq_off, sizeof(int32_t) * (kMaxClamp + 2), "pairing table");
        if (!rc) rc = dev_alloc(ctx, (void **)&m.sq_rep, sizeof(short2) * kMaxLatticePoints, "pairing table");
        if (rc) return rc;
        m.bytes += sizeof(int32_t) * (kMaxClamp + 2) + sizeof(short2) * kMaxLatticePoints;
    }
    CK(cudaMemcpyAsync(m.sq_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, ctx->stream),
       "pairing table upload");
    CK(cudaMemcpyAsync(m.sq_rep, rep.data(), sizeof(short2) * rep.size(), cudaMemcpyHostToDevice, ctx->stream),
       "pairing table upload");
    return RELO_OK;
}

// ---- sensor plan (Eq. 11-15) ----------------------------------------------------------------

void free_plan(relo_ctx *ctx, SensorPlan *P) {
    dev_free(ctx, P->b_dev, sizeof(int32_t) * P->b.size());
    dev_free(ctx, P->D_dev, sizeof(int2) * P->D.size());
    dev_free(ctx, P->iv_dev, sizeof(int2) * P->iv.size());
    delete P;
}

// The plan for these angles, from the cache or newly built (least recently
// used plans are evicted beyond kMaxPlans; a plan in use by queued work is
// never evicted because eviction first waits for the stream).
int plan_for(relo_ctx *ctx, const float *angles_raw, int n_raw, SensorPlan **out) {
    const int skip = ctx->p.n_skip_beam;
    const int n = (n_raw + skip - 1) / skip;   // Eq. 11: beams 0, skip, 2 skip, ...
    std::vector<float> a(n);
    for (int i = 0; i < n; ++i) a[i] = angles_raw[(size_t)i * skip];
    for (SensorPlan *P : ctx->plans) {
        if (P->n_skip == skip && P->n_orient_param == ctx->p.n_orient && P->angles == a) {
            P->last_use = ++ctx->plan_clock;
            *out = P;
            return RELO_OK;
        }
    }
    if (n < 2) return fail(ctx, RELO_E_BEAM_GRID, "need at least two beams");
    const double two_pi = 2.0 * M_PI;
    // Consecutive angles differ by a whole number of grid steps (one inside a
    // contiguous FoV, more across an occluded sector, Eq. 12): count them
    // against the smallest difference and divide the span by the total.
    std::vector<double> dif((size_t)(n - 1));
    double dmin = INFINITY, span = 0.0;
    for (int i = 1; i < n; ++i) {
        double d = (double)a[i] - (double)a[i - 1];
        if (d < 0.0) d += two_pi;
        dif[i - 1] = d;
        span += d;
        if (d < dmin) dmin = d;
    }
    if (!(dmin > 0.0)) return fail(ctx, RELO_E_BEAM_GRID, "two beams share an angle");
    long long steps = 0;
    for (double d : dif) steps += llround(d / dmin);
    const double step = span / (double)steps;
    const long long ns = llround(two_pi / step);   // Eq. 14
    if (ns < n || ns > kMaxNs) return fail(ctx, RELO_E_BEAM_GRID, "N_s out of range");
    const double dphi = two_pi / (double)ns;
    std::vector<int32_t> b(n);
    std::vector<char> seen((size_t)ns, 0);
    for (int i = 0; i < n; ++i) {
        const double q = (double)a[i] / dphi;
        const long long k = llround(q);
        if (fabs(q - (double)k) > 1e-3) return fail(ctx, RELO_E_BEAM_GRID, "beam angle off the panoramic grid");
        const long long bi = ((k % ns) + ns) % ns;
        if (seen[bi]) return fail(ctx, RELO_E_BEAM_GRID, "two beams on one panoramic direction");
        seen[bi] = 1;
        b[i] = (int32_t)bi;
    }
    const int n_orient = ctx->p.n_orient > 0 ? ctx->p.n_orient : (int)ns;
    if (ns % n_orient != 0) return fail(ctx, RELO_E_BEAM_GRID, "n_orient must divide N_s");
    // FoV intervals (Eq. 12): maximal cyclic runs of covered panoramic indices
    std::vector<int2> iv;
    if (n == ns) {
        iv.push_back(make_int2(0, (int)ns));
    } else {
        for (long long j = 0; j < ns; ++j) {
            if (seen[j] && !seen[(j + ns - 1) % ns]) {
                int len = 0;
                while (seen[(j + len) % ns]) ++len;
                iv.push_back(make_int2((int)j, len));
            }
        }
    }
    // directions D_j = llround((cos, sin)(2 pi j / N_s) * 2^30)
    std::vector<int2> D((size_t)ns);
    for (long long j = 0; j < ns; ++j) {
        const double ang = two_pi * (double)j / (double)ns;
        D[j] = make_int2((int)llround(ldexp(cos(ang), 30)), (int)llround(ldexp(sin(ang), 30)));
    }
    long long fov = 0;
    for (auto &v : iv) fov += v.y;
    SensorPlan *P = new (std::nothrow) SensorPlan();
    if (!P) return fail(ctx, RELO_E_INVALID_ARG, "out of host memory");
    const relo_params &p = ctx->p;
    P->lam = (double)fov / (double)ns;
    P->a_mid = p.a_mid_min + P->lam * (p.a_mid_max - p.a_mid_min);   // Eq. 25
    P->a_low = p.a_low_min + P->lam * (p.a_low_max - p.a_low_min);
    P->fov = fov;
    P->n = n;
    P->ns = (int)ns;
    P->n_orient = n_orient;
    P->n_enum = (int)ns / n_orient;
    P->n_m = P->lam >= p.panoramic_ratio ? 1 : n_orient;   // Eq. 20
    P->b = b;
    P->D = D;
    P->iv = iv;
    P->angles = a;
    P->n_skip = skip;
    P->n_orient_param = ctx->p.n_orient;
    int rc;
    if ((rc = dev_alloc(ctx, (void **)&P->b_dev, sizeof(int32_t) * n, "plan beams")) ||
        (rc = dev_alloc(ctx, (void **)&P->D_dev, sizeof(int2) * ns, "plan directions")) ||
        (rc = dev_alloc(ctx, (void **)&P->iv_dev, sizeof(int2) * iv.size(), "plan intervals"))) {
        free_plan(ctx, P);
        return rc;
    }
    CK(cudaMemcpyAsync(P->b_dev, b.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream), "plan upload");
    CK(cudaMemcpyAsync(P->D_dev, D.data(), sizeof(int2) * ns, cudaMemcpyHostToDevice, ctx->stream), "plan upload");
    CK(cudaMemcpyAsync(P->iv_dev, iv.data(), sizeof(int2) * iv.size(), cudaMemcpyHostToDevice, ctx->stream),
       "plan upload");
    // the host vectors of this call must outlive the asynchronous copies
    CK(cudaStreamSynchronize(ctx->stream), "plan upload");
    if ((int)ctx->plans.size() >= kMaxPlans) {
        auto it = std::min_element(ctx->plans.begin(), ctx->plans.end(),
                                   [](SensorPlan *x, SensorPlan *y) { return x->last_use < y->last_use; });
        free_plan(ctx, *it);
        ctx->plans.erase(it);
    }
    P->last_use = ++ctx->plan_clock;
    ctx->plans.push_back(P);
    *out = P;
    return RELO_OK;
}

int edt_segments(int H) {
    const int L = edt_segment_rows(H);
    return (H + L - 1) / L;
}

// The EDT of a map whose grid the context stream is about to hold: the occupancy tiles on the context stream, then
// the field and d2 on the side stream (after the tiles, whose summaries they read).  Every later reader of the field
// or d2 waits on field_ready; the next EDT of the map waits on it before its grid is overwritten.
cudaError_t map_edt(relo_ctx *ctx, MapSlot &m) {
    cudaError_t e = timed(ctx, 0, m.dev.reach ? 3 : 1, [&] { return launch_edt_tiles(m.dev, ctx->stream); });
    if (e == cudaSuccess) e = cudaEventRecord(m.tiles_ready, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, m.tiles_ready, 0);
    if (e == cudaSuccess) e = timed_on(ctx, ctx->side, 7, 2, [&] { return launch_edt_field(m.dev, ctx->side); });
    if (e == cudaSuccess) e = cudaEventRecord(m.field_ready, ctx->side);
    return e;
}

MapSlot *get_map(relo_ctx *ctx, int id) {
    if (id < 0 || id >= (int)ctx->maps.size() || !ctx->maps[id].live) return nullptr;
    return &ctx->maps[id];
}

// ---- resident synthesized scans ------------------------------------------------------------------

void free_win(relo_ctx *ctx, WinTable *w) {
    dev_free(ctx, w->keys, w->bytes);
    ctx->table_bytes -= (long long)w->bytes;
    if (w->built) cudaEventDestroy(w->built);
    delete w;
}

void free_table(relo_ctx *ctx, ScanTable *t) {
    for (WinTable *w : t->wins) free_win(ctx, w);
    t->wins.clear();
    dev_free(ctx, t->data, t->bytes);
    ctx->table_bytes -= (long long)t->bytes;
    if (t->written) cudaEventDestroy(t->written);
    delete t;
}

// Frees every table of the map, once the device has finished the work that may read them.
void drop_tables(relo_ctx *ctx, MapSlot &m) {
    if (m.tables.empty()) return;
    cudaDeviceSynchronize();
    for (ScanTable *t : m.tables) free_table(ctx, t);
    m.tables.clear();
}

WinTable *find_win(ScanTable *t, const SensorPlan &P) {
    for (WinTable *w : t->wins)
        if (w->n_enum == P.n_enum && w->n_m == P.n_m && w->iv.size() == P.iv.size() &&
            std::equal(w->iv.begin(), w->iv.end(), P.iv.begin(),
                       [](const int2 &a, const int2 &b) { return a.x == b.x && a.y == b.y; }))
            return w;
    return nullptr;
}

ScanTable *find_table(MapSlot &m, int ns, int lim) {
    for (ScanTable *t : m.tables)
        if (t->ns == ns && t->lim == lim) return t;
    return nullptr;
}

// Evicts least recently used tables not used by the batch being built until
// `need` more bytes fit the scan-cache budget; false when they cannot.
bool make_room(relo_ctx *ctx, size_t need) {
    const long long cap = ctx->p.scan_cache_bytes;
    if ((long long)need > cap) return false;
    bool synced = false;
    while (ctx->table_bytes + (long long)need > cap) {
        ScanTable *victim = nullptr;
        MapSlot *owner = nullptr;
        for (MapSlot &m : ctx->maps) {
            if (!m.live) continue;
            for (ScanTable *t : m.tables)
                if (t->pin != ctx->batch_seq && (!victim || t->last_use < victim->last_use)) {
                    victim = t;
                    owner = &m;
                }
        }
        if (!victim) return false;
        if (!synced) {
            cudaDeviceSynchronize();   // queued batches may still read it
            synced = true;
        }
        owner->tables.erase(std::find(owner->tables.begin(), owner->tables.end(), victim));
        free_table(ctx, victim);
        ++ctx->cache_evictions;
    }
    return true;
}

// A new, unwritten table for (m, ns, lim), or nullptr when the budget (or
// the context's HBM budget) cannot hold it; failing here is not an error.
ScanTable *new_table(relo_ctx *ctx, MapSlot &m, int ns, int lim) {
    const size_t bytes = sizeof(uint32_t) * (size_t)m.n_hyp * (size_t)ns;
    if (!make_room(ctx, bytes)) return nullptr;
    ScanTable *t = new (std::nothrow) ScanTable();
    if (!t) return nullptr;
    const std::string saved = ctx->err;
    if (dev_alloc(ctx, (void **)&t->data, bytes, "scan table") != RELO_OK) {
        ctx->err = saved;
        delete t;
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&t->written, cudaEventDisableTiming) != cudaSuccess) {
        t->written = nullptr;
        dev_free(ctx, t->data, bytes);
        delete t;
        return nullptr;
    }
    t->ns = ns;
    t->lim = lim;
    t->bytes = bytes;
    ctx->table_bytes += (long long)bytes;
    m.tables.push_back(t);
    return t;
}

// ---- per-direction traversal tables ---------------------------------------------------------------

void free_raytab(relo_ctx *ctx, RayTab *t) {
    dev_free(ctx, t->mask, t->bytes_mask);
    dev_free(ctx, t->selx, t->bytes_sel);
    dev_free(ctx, t->sely, t->bytes_sel);
    dev_free(ctx, t->kmax, sizeof(int32_t) * (size_t)t->ns);
    if (t->built) cudaEventDestroy(t->built);
    delete t;
}

// The traversal tables of (P's directions, lim), from the cache or built on
// stream st (the caller's stream must wait for t->built before using them);
// nullptr when disabled or too large, in which case rays step cell by cell.
RayTab *ray_tables_for(relo_ctx *ctx, const SensorPlan &P, int lim, cudaStream_t st) {
    if (!ctx->p.ray_tables) return nullptr;
    for (RayTab *t : ctx->raytabs)
        if (t->ns == P.ns && t->lim == lim) {
            t->last_use = ++ctx->table_clock;
            t->pin = ctx->batch_seq;
            return t;
        }
    const size_t bm = sizeof(uint64_t) * (size_t)ray_mask_rows(lim) * P.ns;
    const size_t bs = sizeof(uint16_t) * (size_t)ray_sel_rows(lim) * P.ns;
    if (bm + 2 * bs > kMaxRayTabBytes) return nullptr;
    if ((int)ctx->raytabs.size() >= kMaxRayTabs) {
        auto it = ctx->raytabs.end();
        for (auto i = ctx->raytabs.begin(); i != ctx->raytabs.end(); ++i)
            if ((*i)->pin != ctx->batch_seq && (it == ctx->raytabs.end() || (*i)->last_use < (*it)->last_use)) it = i;
        if (it == ctx->raytabs.end()) return nullptr;
        cudaDeviceSynchronize();   // queued work may still read it
        free_raytab(ctx, *it);
        ctx->raytabs.erase(it);
    }
    RayTab *t = new (std::nothrow) RayTab();
    if (!t) return nullptr;
    t->ns = P.ns;
    t->lim = lim;
    t->bytes_mask = bm;   // free_raytab releases whatever was allocated
    t->bytes_sel = bs;
    const std::string saved = ctx->err;
    bool ok = dev_alloc(ctx, (void **)&t->mask, bm, "ray tables") == RELO_OK &&
              dev_alloc(ctx, (void **)&t->selx, bs, "ray tables") == RELO_OK &&
              dev_alloc(ctx, (void **)&t->sely, bs, "ray tables") == RELO_OK &&
              dev_alloc(ctx, (void **)&t->kmax, sizeof(int32_t) * (size_t)P.ns, "ray tables") == RELO_OK &&
              cudaEventCreateWithFlags(&t->built, cudaEventDisableTiming) == cudaSuccess &&
              launch_ray_tables(P.D_dev, P.ns, lim, t->mask, t->selx, t->sely, t->kmax, st) == cudaSuccess &&
              cudaEventRecord(t->built, st) == cudaSuccess;
    if (!ok) {
        ctx->err = saved;
        free_raytab(ctx, t);
        return nullptr;
    }
    ctx->kernels += 1;
    t->last_use = ++ctx->table_clock;
    t->pin = ctx->batch_seq;
    ctx->raytabs.push_back(t);
    return t;
}

RayTables ray_tables_view(const RayTab *t) {
    RayTables v{nullptr, nullptr, nullptr, nullptr};
    if (t) {
        v.mask = t->mask;
        v.selx = t->selx;
        v.sely = t->sely;
        v.kmax = t->kmax;
    }
    return v;
}

// A new, unbuilt window table of scan table t for plan P, or nullptr when the
// budget cannot hold it (not an error: the request then takes SMAD from the ranges).
WinTable *new_win(relo_ctx *ctx, ScanTable *t, const SensorPlan &P, int n_hyp) {
    const size_t bytes = 8 * (size_t)n_hyp * (size_t)P.n_m;
    if (!make_room(ctx, bytes)) return nullptr;
    WinTable *w = new (std::nothrow) WinTable();
    if (!w) return nullptr;
    const std::string saved = ctx->err;
    if (dev_alloc(ctx, (void **)&w->keys, bytes, "window table") != RELO_OK) {
        ctx->err = saved;
        delete w;
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&w->built, cudaEventDisableTiming) != cudaSuccess) {
        w->built = nullptr;
        dev_free(ctx, w->keys, bytes);
        delete w;
        return nullptr;
    }
    w->n_enum = P.n_enum;
    w->n_m = P.n_m;
    w->iv = P.iv;
    w->bytes = bytes;
    ctx->table_bytes += (long long)bytes;
    t->wins.push_back(w);
    return w;
}

void free_map(relo_ctx *ctx, MapSlot &m) {
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (m.tiles_ready) cudaEventDestroy(m.tiles_ready);
    if (m.field_ready) cudaEventDestroy(m.field_ready);
    drop_tables(ctx, m);
    dev_free(ctx, m.dev.d2, sizeof(int32_t) * (size_t)m.dev.W * m.dev.H);
    dev_free(ctx, m.dev.colsq, sizeof(int32_t) * (size_t)m.dev.W * m.dev.H);
    dev_free(ctx, m.dev.summ, sizeof(int2) * (size_t)m.dev.W * edt_segments(m.dev.H));
    dev_free(ctx, m.dev.grid, (size_t)m.dev.W * m.dev.H);
    dev_free(ctx, m.dev.field, sizeof(uint16_t) * (size_t)m.dev.Wp * m.dev.Hp);
    dev_free(ctx, m.dev.bits, sizeof(uint64_t) * occupancy_words(m.dev.TW, m.dev.TH));
    dev_free(ctx, m.dev.reach, walk_reach_bytes(m.dev.TW, m.dev.TH));
    dev_free(ctx, m.hyps, sizeof(int2) * (size_t)m.hyp_cap);
    dev_free(ctx, m.lut, sizeof(float2) * (kMaxClamp + 2));
    dev_free(ctx, m.sq_off, sizeof(int32_t) * (kMaxClamp + 2));
    dev_free(ctx, m.sq_rep, sizeof(short2) * kMaxLatticePoints);
    m = MapSlot();
}

int load_map_impl(relo_ctx *ctx, const int8_t *grid, bool on_device, int32_t w, int32_t h, double res, double ox,
                  double oy, int32_t *map_id) {
    if (!ctx || !grid || !map_id) return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    if (w < 1 || h < 1 || w > 16384 || h > 16384) return fail(ctx, RELO_E_INVALID_ARG, "map size out of range");
    if (!(res > 0) || !isfinite(ox) || !isfinite(oy)) return fail(ctx, RELO_E_INVALID_ARG, "bad resolution or origin");
    MapSlot m;
    m.res = res;
    m.ox = ox;
    m.oy = oy;
    m.dev.W = w;
    m.dev.H = h;
    m.dev.TW = (w + 7) / 8;
    m.dev.TH = (h + 7) / 8;
    int rc = clamp_for(ctx, ctx->p.d_max, res, &m.dev.C);
    if (rc) return rc;
    m.dev.P = pad_for(ctx->p.max_range, res);
    if (m.dev.P < 1) return fail(ctx, RELO_E_INVALID_ARG, "max_range / res must be below 32768 cells");
    m.dev.Wp = (w + 2 * m.dev.P + 7) & ~7;
    m.dev.Hp = (h + 2 * m.dev.P + 7) & ~7;
    if (m.dev.Wp > 65535 || m.dev.Hp > 65535)
        return fail(ctx, RELO_E_INVALID_ARG, "the map with its field border must stay below 65536 cells per side");
    const size_t cells = (size_t)w * h;
    const size_t fcells = (size_t)m.dev.Wp * m.dev.Hp;
    struct { void **p; size_t bytes; } allocs[] = {
        {(void **)&m.dev.d2, cells * 4}, {(void **)&m.dev.colsq, cells * 4}, {(void **)&m.dev.grid, cells},
        {(void **)&m.dev.field, fcells * 2}, {(void **)&m.dev.bits, occupancy_words(m.dev.TW, m.dev.TH) * 8},
        {(void **)&m.dev.reach, walk_reach_bytes(m.dev.TW, m.dev.TH)},
        {(void **)&m.dev.summ, sizeof(int2) * (size_t)w * edt_segments(h)}};
    for (auto &a : allocs) {
        rc = dev_alloc(ctx, a.p, a.bytes, "map tables");
        if (rc) {
            free_map(ctx, m);
            return rc;
        }
        m.bytes += a.bytes;
    }
    cudaError_t e = cudaEventCreateWithFlags(&m.tiles_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m.field_ready, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m.dev.grid, grid, cells, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) e = launch_field_border(m.dev, ctx->stream);
    if (e == cudaSuccess) ctx->kernels += 2;
    if (e == cudaSuccess) e = map_edt(ctx, m);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, m.field_ready, 0);
    if (e != cudaSuccess) {
        free_map(ctx, m);
        return cuda_fail(ctx, e, "map precompute");
    }
    rc = build_lut(ctx, m);
    if (rc) {
        free_map(ctx, m);
        return rc;
    }
    if (!on_device) {
        // the host grid may be released once the call returns
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            free_map(ctx, m);
            return cuda_fail(ctx, e, "map upload");
        }
    } else {
        // the LUT host staging vector was already copied; make that copy complete too
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            free_map(ctx, m);
            return cuda_fail(ctx, e, "map precompute");
        }
    }
    m.live = true;
    int id = -1;
    for (int i = 0; i < (int)ctx->maps.size(); ++i)
        if (!ctx->maps[i].live) { id = i; break; }
    if (id < 0) {
        id = (int)ctx->maps.size();
        ctx->maps.push_back(MapSlot());
    }
    ctx->maps[id] = m;
    *map_id = id;
    return RELO_OK;
}

// room for n hypotheses of map m and the check flags; the map's resident tables (which depend on them) go
int hyp_storage(relo_ctx *ctx, MapSlot &m, int n) {
    int rc = RELO_OK;
    if (n > (1 << kHypBits)) return fail(ctx, RELO_E_INVALID_ARG, "too many hypotheses (max 2^21)");
    drop_tables(ctx, m);
    if (n > m.hyp_cap) {
        dev_free(ctx, m.hyps, sizeof(int2) * (size_t)m.hyp_cap);
        m.hyps = nullptr;
        m.hyp_cap = 0;
        if ((rc = dev_alloc(ctx, (void **)&m.hyps, sizeof(int2) * (size_t)n, "hypotheses"))) return rc;
        m.hyp_cap = n;
    }
    if (!ctx->bad && (rc = dev_alloc(ctx, (void **)&ctx->bad, 2 * sizeof(int), "flags"))) return rc;
    return RELO_OK;
}

int set_hyps_impl(relo_ctx *ctx, MapSlot &m, const int2 *cells, bool on_device, int n) {
    int rc = hyp_storage(ctx, m, n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(m.hyps, cells, sizeof(int2) * (size_t)n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream),
       "hypothesis upload");
    CK(cudaMemsetAsync(ctx->bad, 0, sizeof(int), ctx->stream), "hypothesis check");
    CK(launch_check_cells(m.hyps, n, m.dev, ctx->bad, ctx->stream), "hypothesis check");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, ctx->bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "hypothesis check");
    CK(cudaStreamSynchronize(ctx->stream), "hypothesis check");
    if (bad) {
        m.n_hyp = 0;
        return fail(ctx, RELO_E_INVALID_ARG, std::to_string(bad) + " hypotheses off the map or on occupied cells");
    }
    m.n_hyp = n;
    return RELO_OK;
}


// ---- batches ------------------------------------------------------------------------------------

int upload(relo_ctx *ctx, cudaStream_t st, void *dst, const void *src, size_t bytes, BatchState *bs) {
    const unsigned char *p = static_cast<const unsigned char *>(src);
    unsigned char *d = static_cast<unsigned char *>(dst);
    while (bytes > 0) {
        const size_t n = bytes < kBlobBytes ? bytes : kBlobBytes;
        ctx->blob->n = (unsigned int)n;
        memcpy(ctx->blob->bytes, p, n);
        k_upload<<<(unsigned)((n + 255) / 256 < 16 ? (n + 255) / 256 : 16), 256, 0, st>>>(*ctx->blob, d, bs);
        bs = nullptr;
        CK(cudaGetLastError(), "descriptor upload");
        ctx->kernels += 1;
        p += n;
        d += n;
        bytes -= n;
    }
    return RELO_OK;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Checks one request and resolves its map and sensor plan.
int prepare(relo_ctx *ctx, int32_t map_id, const float *ranges_dev, const float *angles, int32_t n_beams,
            float max_range, void *result_dev, Prepared *out, int topk = 0) {
    if (!ranges_dev || !angles || !result_dev || n_beams < 2)
        return fail(ctx, RELO_E_INVALID_ARG, "bad relocalize arguments");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    if (m->n_hyp <= 0) return fail(ctx, RELO_E_NO_HYPOTHESES, "the map has no hypotheses");
    if (!(max_range > 0) || !isfinite(max_range)) return fail(ctx, RELO_E_INVALID_ARG, "max_range must be positive");
    SensorPlan *P = nullptr;
    int rc = plan_for(ctx, angles, n_beams, &P);
    if (rc) return rc;
    if (P->n > kMaxValidBeams) return fail(ctx, RELO_E_INVALID_ARG, "at most 2048 beams after downsampling");
    const double rq = (double)max_range * 65536.0 / m->res;
    if (!(rq < 2147483647.0)) return fail(ctx, RELO_E_INVALID_ARG, "max_range / res must be below 32768 cells");
    const long long rmax_q16 = llrint(rq);
    if ((double)P->n * (double)rmax_q16 >= 8.0e12)
        return fail(ctx, RELO_E_INVALID_ARG, "beam count x max range too large for the SMAD key");
    if ((double)max_range / m->res + 1.0 > (double)m->dev.P)
        return fail(ctx, RELO_E_INVALID_ARG, "scan max_range exceeds the context's max_range (the map's field border)");
    const relo_params &p = ctx->p;
    out->m = m;
    out->P = P;
    out->ranges_dev = ranges_dev;
    out->result_dev = result_dev;
    out->max_range = max_range;
    out->lim = (int)((rmax_q16 * rmax_q16) >> 32);
    if (topk < 0 || topk > kMaxTopk) return fail(ctx, RELO_E_INVALID_ARG, "topk must be in [0, 4096]");
    out->K = std::min(topk > 0 ? topk : p.topk, m->n_hyp);
    out->B = std::min(p.batch, out->K);
    out->n_batches = (out->K + out->B - 1) / out->B;
    if (out->n_batches > kMaxBatches)
        return fail(ctx, RELO_E_INVALID_ARG, "topk / batch must be at most 64 batches");
    return RELO_OK;
}

// Lays out the batch's scratch, uploads its descriptors and launches every stage once.
int run_batch(relo_ctx *ctx, BatchSlot &sl, const Prepared *pr, int R) {
    if (R < 1 || R > kMaxBatchRequests) return fail(ctx, RELO_E_INVALID_ARG, "1 to 256 requests per batch");
    const relo_params &p = ctx->p;
    ++ctx->batch_seq;
    cudaStream_t st = sl.stream;
    const bool cast = p.coarse_metric != RELO_COARSE_NONE;   // without a coarse ranking no rays are cast
    std::vector<RayTab *> rtab((size_t)R, nullptr);
    for (int r = 0; r < R && cast; ++r) rtab[r] = ray_tables_for(ctx, *pr[r].P, pr[r].lim, st);
    // Resident synthesized scans: read a table stored by an earlier launch, or
    // store a new one (one writer per table; other requests of this batch
    // with the same geometry cast into their scratch).  Tables this batch
    // creates are freed again if the batch fails to launch.
    std::vector<ScanTable *> tab((size_t)R, nullptr);
    std::vector<int> mode((size_t)R, kScanCast);
    struct Created {
        relo_ctx *ctx;
        std::vector<std::pair<MapSlot *, ScanTable *>> list;
        bool keep = false;
        ~Created() {
            if (keep || list.empty()) return;
            cudaDeviceSynchronize();
            for (auto &x : list) {
                auto &v = x.first->tables;
                v.erase(std::find(v.begin(), v.end(), x.second));
                free_table(ctx, x.second);
            }
        }
    } created{ctx, {}, false};
    if (p.scan_cache_bytes > 0 && cast) {
        for (int r = 0; r < R; ++r) {
            MapSlot &m = *pr[r].m;
            ScanTable *t = find_table(m, pr[r].P->ns, pr[r].lim);
            bool fresh = false;
            for (auto &x : created.list) fresh = fresh || x.second == t;
            if (t && !fresh) {
                mode[r] = kScanRead;
                ++ctx->cache_hits;
            } else {
                ++ctx->cache_misses;
                if (!t && (t = new_table(ctx, m, pr[r].P->ns, pr[r].lim))) {
                    mode[r] = kScanStore;
                    created.list.push_back({&m, t});
                } else {
                    t = nullptr;
                }
            }
            if (t) {
                t->last_use = ++ctx->table_clock;
                t->pin = ctx->batch_seq;
                tab[r] = t;
            }
        }
    }
    // Window tables of the requests with a scan table: read one built by an
    // earlier launch, or build it now (one builder per table).
    std::vector<WinTable *> win((size_t)R, nullptr);
    std::vector<int> wmode((size_t)R, kWinNone);
    struct NewWins {   // window tables this batch builds; freed again if the batch fails to launch
        relo_ctx *ctx;
        std::vector<std::pair<ScanTable *, WinTable *>> list;
        bool keep = false;
        bool has(const WinTable *w) const {
            for (auto &x : list)
                if (x.second == w) return true;
            return false;
        }
        ~NewWins() {
            if (keep || list.empty()) return;
            cudaDeviceSynchronize();
            for (auto &x : list) {
                auto &v = x.first->wins;
                v.erase(std::find(v.begin(), v.end(), x.second));
                free_win(ctx, x.second);
            }
        }
    } wnew{ctx, {}, false};
    for (int r = 0; r < R; ++r) {
        if (!tab[r] || p.coarse_metric != RELO_COARSE_SMAD) continue;   // window sums serve SMAD only
        WinTable *w = find_win(tab[r], *pr[r].P);
        if (w && !wnew.has(w)) {
            wmode[r] = kWinRead;
            ++ctx->win_hits;
        } else if (!w && (w = new_win(ctx, tab[r], *pr[r].P, pr[r].m->n_hyp))) {
            wmode[r] = kWinBuild;
            wnew.list.push_back({tab[r], w});
        } else {
            w = nullptr;
        }
        win[r] = w;
    }
    // TAM work of every batch index, one launch per class of requests with the
    // same register-resident values per lane (a 541-beam request does not run
    // at the width of a 1440-beam one); one class if the segment table would
    // not fit the slot
    std::vector<int> vcls((size_t)R);
    for (int r = 0; r < R; ++r) {
        vcls[r] = tam_vpl_for(pr[r].P->n);
        if (vcls[r] < 0) return fail(ctx, RELO_E_INVALID_ARG, "no TAM kernel fits this beam count");
    }
    std::vector<int> classes(vcls);
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    int pre_max_batches = 0;
    for (int r = 0; r < R; ++r) pre_max_batches = std::max(pre_max_batches, pr[r].n_batches);
    if ((size_t)pre_max_batches * classes.size() * R > (size_t)kMaxBatches * kMaxBatchRequests) {
        std::fill(vcls.begin(), vcls.end(), classes.back());
        classes.assign(1, classes.back());
    }
    const int NC = (int)classes.size();
    // survivors per TAM task: the autotuner's choice for the request's shape, else the built-in one
    auto chunk_of = [&](int r) {
        const relo_tune_entry *e = tuned_tam(ctx, R, vcls[r], pr[r].P->n_orient, pr[r].K);
        return e && e->val[0] > 0 ? e->val[0] : tam_chunk_for(pr[r].K, pr[r].P->n_orient, ctx->n_sm);
    };
    std::vector<ReqDesc> desc((size_t)R);
    std::vector<size_t> off((size_t)R);
    size_t total = 0;
    int total_hyp = 0, max_ns_pad = 32, max_n_hyp = 1, max_K = 1, max_beams = 1, max_C = 0, max_batches = 0;
    long long total_chunks = 0;
    for (int r = 0; r < R; ++r) {
        const Prepared &q = pr[r];
        const int n = q.P->n, nh = q.m->n_hyp, K = q.K;
        off[r] = total;
        total += align_up(24ull * K) + align_up(4ull * K);   // refined poses and re-evaluated scores
        total += align_up(sizeof(int2) * n) + align_up(4ull * n) + align_up(sizeof(ScanInfo)) + align_up(8ull * nh) * 2 +
                 align_up(4ull * nh) + align_up(4ull * K) * 3 + align_up(4ull * K * q.P->n_orient) +
                 align_up(16ull * tam_chunk_cap(K, q.B, q.n_batches, chunk_of(r))) + align_up(4ull * (q.n_batches + 1)) +
                 align_up(4ull * 8 * 32 * q.P->n_orient * tam_offs_stride_for(vcls[r])) +
                 align_up(8ull * K) + align_up(4ull * q.n_batches * p.local_topk) + align_up(sizeof(SelectState));
        if (mode[r] == kScanCast) total += align_up(4ull * nh * q.P->ns);   // the request's synthesized ranges
        if (mode[r] != kScanRead && cast) total_chunks += cast_chunks(nh, q.P->ns, 1);
        if ((long long)total_hyp + nh > (1ll << 30) || total_chunks > (1ll << 31) - 1)
            return fail(ctx, RELO_E_INVALID_ARG, "batch too large");
        total_hyp += nh;
        max_ns_pad = std::max(max_ns_pad, (q.P->ns + 31) & ~31);
        max_n_hyp = std::max(max_n_hyp, nh);
        max_K = std::max(max_K, K);
        max_beams = std::max(max_beams, n);
        max_C = std::max(max_C, q.m->dev.C);
        max_batches = std::max(max_batches, q.n_batches);
    }
    // hypotheses per cast work item: group while every resident warp (5 CTAs of 8 warps per SM) keeps 16 or more items
    int cast_hyps = 1;
    while (cast_hyps < kCastHypsMax && total_chunks >= 16ll * 2 * cast_hyps * 40 * ctx->n_sm) cast_hyps *= 2;
    int rc = ensure(ctx, &sl.arena, &sl.arena_cap, total, "request scratch");
    if (rc) return rc;
    for (int r = 0; r < R; ++r) {
        const Prepared &q = pr[r];
        const MapSlot &m = *q.m;
        const SensorPlan &P = *q.P;
        ReqDesc &d = desc[r];
        memset(&d, 0, sizeof d);
        d.bits = m.dev.bits;
        d.reach = m.dev.reach;
        d.field = m.dev.field;
        d.Wp = m.dev.Wp;
        d.P = m.dev.P;
        d.lut = m.lut;
        d.W = m.dev.W;
        d.H = m.dev.H;
        d.TW = m.dev.TW;
        d.TH = m.dev.TH;
        d.C = m.dev.C;
        d.res = (float)m.res;
        d.res2 = (float)(m.res * m.res);
        d.d_max = (float)(m.res * sqrt((double)m.dev.C));
        d.d_min = (float)(m.res / 2.0);
        d.resd = m.res;
        d.ox = m.ox;
        d.oy = m.oy;
        d.hyps = m.hyps;
        d.n_hyp = m.n_hyp;
        d.D = P.D_dev;
        d.b = P.b_dev;
        d.iv = P.iv_dev;
        d.ns = P.ns;
        d.ns_pad = (P.ns + 31) & ~31;
        d.n_iv = (int)P.iv.size();
        d.n_beams = P.n;
        d.n_orient = P.n_orient;
        d.n_enum = P.n_enum;
        d.n_m = P.n_m;
        d.lim = q.lim;
        d.rt = ray_tables_view(rtab[r]);
        d.a_mid = P.a_mid;
        d.a_low = P.a_low;
        d.fov = (double)P.fov;
        d.ranges = q.ranges_dev;
        d.skip = p.n_skip_beam;
        d.max_range = q.max_range;
        d.K = q.K;
        d.B = q.B;
        d.n_batches = q.n_batches;
        d.L = p.local_topk;
        d.early_stop = p.early_stop;
        d.tau = p.tau;
        d.n_smad_evals = cast ? (long long)m.n_hyp * P.n_m : 0;
        unsigned char *a = sl.arena + off[r];
        auto take = [&a](size_t bytes) {
            unsigned char *x = a;
            a += align_up(bytes);
            return x;
        };
        d.vbR = (int2 *)take(sizeof(int2) * P.n);
        d.Rall = (int32_t *)take(4ull * P.n);
        d.coarse = p.coarse_metric;
        d.fine = p.fine_metric;
        d.icp_iters = p.icp_iters;
        d.d2map = m.dev.d2;
        d.grid = m.dev.grid;
        d.sq_off = m.sq_off;
        d.sq_rep = m.sq_rep;
        d.ref_pose = (double *)take(24ull * q.K);
        d.reev = (float *)take(4ull * q.K);
        d.scan = (ScanInfo *)take(sizeof(ScanInfo));
        d.keys = (unsigned long long *)take(8ull * m.n_hyp);
        d.smad_num = (long long *)take(8ull * m.n_hyp);
        d.smad_m = (int32_t *)take(4ull * m.n_hyp);
        d.survivors = (int32_t *)take(4ull * q.K);
        d.tam_chunk = chunk_of(r);
        d.tam_stride = tam_offs_stride_for(vcls[r]);
        d.tam_offs = (int32_t *)take(4ull * 8 * 32 * P.n_orient * d.tam_stride);
        d.surv_perm = (int32_t *)take(4ull * q.K);
        d.tam_chunks = (int4 *)take(16ull * tam_chunk_cap(q.K, q.B, q.n_batches, d.tam_chunk));
        d.chunk_cnt = (int32_t *)take(4ull * (q.n_batches + 1));
        d.best_m = (int32_t *)take(4ull * q.K);
        d.T = (float *)take(4ull * q.K * P.n_orient);
        d.best_key = (unsigned long long *)take(8ull * q.K);
        d.local = (int32_t *)take(4ull * q.n_batches * p.local_topk);
        d.state = (SelectState *)take(sizeof(SelectState));
        d.result = q.result_dev;
        d.scan_table = mode[r] == kScanCast ? (uint32_t *)take(4ull * m.n_hyp * P.ns) : tab[r]->data;
        d.scan_mode = mode[r];
        d.win = win[r] ? win[r]->keys : nullptr;
        d.win_mode = wmode[r];
    }
    // work lists: each kernel sees only its requests (the others take the running base, length 0)
    int base = 0, cbase = 0, bbase = 0, rbase = 0, max_nm = 1;
    for (int r = 0; r < R; ++r) {
        ReqDesc &d = desc[r];
        d.hyp_base = base;
        d.wbuild_base = bbase;
        d.wread_base = rbase;
        d.chunk_base = cbase;
        if (d.win_mode == kWinNone) base += d.n_hyp;
        if (d.win_mode == kWinBuild) bbase += d.n_hyp;
        if (d.win_mode == kWinRead) rbase += d.n_hyp;
        d.cast_hyps = cast_hyps;
        if (d.scan_mode != kScanRead) cbase += (int)cast_chunks(d.n_hyp, d.ns, cast_hyps);
        if (d.win_mode == kWinBuild) max_nm = std::max(max_nm, d.n_m);
    }
    const int total_smad = base, total_build = bbase, total_read = rbase;
    total_chunks = cast ? cbase : 0;   // the cast's work items after grouping hypotheses
    // Without early termination no batch waits on another's outcome: one TAM
    // round scores every batch's survivors and one selection launch takes the
    // batches in order (Remark 2's termination test is then never made).
    bool any_early = false;
    for (int r = 0; r < R; ++r) any_early = any_early || desc[r].early_stop;
    const int tam_rounds = any_early ? max_batches : std::min(max_batches, 1);
    std::vector<TamSeg> segs((size_t)max_batches * NC * R);
    std::vector<TamPlan> plans((size_t)max_batches * NC);
    std::vector<int> blo((size_t)R), bhi((size_t)R);
    for (int bi = 0; bi < tam_rounds; ++bi) {
        for (int c = 0; c < NC; ++c) {
            int beams_c = 1, C_c = 0;
            for (int r = 0; r < R; ++r) {
                const bool in = vcls[r] == classes[c] && bi < desc[r].n_batches;
                blo[r] = any_early ? bi : 0;
                bhi[r] = in ? (any_early ? bi + 1 : desc[r].n_batches) : blo[r];
                if (vcls[r] == classes[c]) {
                    beams_c = std::max(beams_c, pr[r].P->n);
                    C_c = std::max(C_c, pr[r].m->dev.C);
                }
            }
            int cps = 0;   // resident CTAs per SM: the smallest the class's requests are tuned to
            for (int r = 0; r < R; ++r) {
                if (vcls[r] != classes[c]) continue;
                const relo_tune_entry *e = tuned_tam(ctx, R, vcls[r], desc[r].n_orient, desc[r].K);
                if (e && e->val[1] > 0) cps = cps > 0 ? std::min(cps, e->val[1]) : e->val[1];
            }
            TamPlan &tp = plans[(size_t)bi * NC + c];
            tp = plan_tam(blo.data(), bhi.data(), R, beams_c, C_c, ctx->n_sm, cps,
                          &segs[((size_t)bi * NC + c) * R]);
            if (tp.vpl < 0) return fail(ctx, RELO_E_INVALID_ARG, "no TAM kernel fits this beam count");
        }
    }
    // descriptors and TAM segments travel together in one upload
    const size_t seg_off = align_up(sizeof(ReqDesc) * R);
    std::vector<unsigned char> blob(seg_off + sizeof(TamSeg) * segs.size(), 0);
    memcpy(blob.data(), desc.data(), sizeof(ReqDesc) * R);
    memcpy(blob.data() + seg_off, segs.data(), sizeof(TamSeg) * segs.size());
    if ((rc = upload(ctx, st, sl.reqs_dev, blob.data(), blob.size(), sl.bs))) return rc;
    ReqDesc *rq = sl.reqs_dev;
    const TamSeg *segs_dev = reinterpret_cast<const TamSeg *>(reinterpret_cast<unsigned char *>(sl.reqs_dev) + seg_off);
    // the ray-cast launch prepares the scans first; a batch without rays to cast prepares them alone
    if (total_chunks <= 0) CK(timed_on(ctx, st, 1, 1, [&] { return launch_scan_prep(rq, R, st); }), "scan preparation");
    for (int r = 0; r < R; ++r) {
        // the occupancy tiles (the cast) and, before TAM and ICP below, the field and d2 of a map whose EDT may
        // still run on the side stream
        if (st != ctx->stream) CK(cudaStreamWaitEvent(st, pr[r].m->tiles_ready, 0), "map tiles");
        if (mode[r] == kScanRead) CK(cudaStreamWaitEvent(st, tab[r]->written, 0), "scan table");
        if (wmode[r] == kWinRead) CK(cudaStreamWaitEvent(st, win[r]->built, 0), "window table");
        if (rtab[r]) CK(cudaStreamWaitEvent(st, rtab[r]->built, 0), "ray tables");
    }
    if (total_chunks > 0)
        CK(timed_on(ctx, st, 2, 1,
                    [&] {
                        int ns0 = 0;
                        for (int r = 0; r < R && !ns0; ++r)
                            if (mode[r] != kScanRead) ns0 = desc[r].ns;
                        const relo_tune_entry *e = tuned(ctx, RELO_TUNE_CAST, ns0, 0, 0);
                        return launch_cast(rq, R, (int)total_chunks, cast_hyps, sl.bs, ctx->n_sm, e ? e->val[0] : 0, st);
                    }),
           "ray cast");
    if (total_smad > 0)
        CK(timed_on(ctx, st, 6, 1,
                    [&] {
                        if (!cast) return launch_rank_by_index(rq, R, total_smad, ctx->n_sm, st);
                        return p.coarse_metric == RELO_COARSE_SMAD_DIRECT
                                   ? launch_smad_direct(rq, R, total_smad, max_ns_pad, sl.bs, ctx->n_sm, st)
                                   : launch_smad(rq, R, total_smad, max_ns_pad, sl.bs, ctx->n_sm, st);
                    }),
           "SMAD");
    if (total_build > 0) {
        CK(timed_on(ctx, st, 6, 1, [&] { return launch_win_build(rq, R, total_build, max_ns_pad, max_nm, st); }),
           "SMAD window tables");
        for (auto &x : wnew.list) CK(cudaEventRecord(x.second->built, st), "window table");
    }
    if (total_read > 0)
        CK(timed_on(ctx, st, 6, 1, [&] { return launch_win_read(rq, R, total_read, st); }), "SMAD by window tables");
    for (auto &x : created.list) CK(cudaEventRecord(x.second->written, st), "scan table");
    {
        int max_no = 1;
        for (int r = 0; r < R; ++r) max_no = std::max(max_no, desc[r].n_orient);
        // the ranking and TAM's work order, and beside them the endpoint offset table O[m][i] of each request plan,
        // per band phase
        CK(timed_on(ctx, st, 3, 1, [&] { return launch_topk(rq, R, max_n_hyp, max_K, max_no, ctx->n_sm, st); }),
           "SMAD top-K");
    }
    for (int r = 0; r < R; ++r) CK(cudaStreamWaitEvent(st, pr[r].m->field_ready, 0), "map field");
    for (int bi = 0; bi < tam_rounds; ++bi) {
        for (int c = 0; c < NC; ++c) {
            const TamPlan &tp = plans[(size_t)bi * NC + c];
            if (tp.total_tasks <= 0) continue;
            const TamSeg *sg = segs_dev + ((size_t)bi * NC + c) * R;
            CK(timed_on(ctx, st, 4, 1, [&] { return launch_tam(rq, R, sg, tp, st); }), "TAM");
        }
        const int lo = any_early ? bi : 0, hi = any_early ? bi + 1 : max_batches;
        const bool last = bi == tam_rounds - 1;
        if (p.icp_iters > 0) {
            // the local top-k, their ICP refinement and re-evaluation, then the batch's best
            CK(timed_on(ctx, st, 5, 1, [&] { return launch_select_batch(rq, R, lo, hi, false, true, st); }),
               "batch selection");
            CK(timed_on(ctx, st, 5, 1, [&] { return launch_icp(rq, R, lo, hi, p.local_topk, max_beams, st); }),
               "ICP refinement");
            CK(timed_on(ctx, st, 5, 1, [&] { return launch_icp_best(rq, R, lo, hi, last, st); }), "batch selection");
        } else {
            CK(timed_on(ctx, st, 5, 1, [&] { return launch_select_batch(rq, R, lo, hi, last, false, st); }),
               "batch selection");
        }
    }
    created.keep = true;
    wnew.keep = true;
    ctx->last = desc[0];
    ctx->last_bs = sl.bs;
    ctx->has_last = true;
    return RELO_OK;
}

// device bytes of a slot's descriptor region: descriptors, then TAM segments
size_t slot_desc_bytes() {
    return align_up(sizeof(ReqDesc) * kMaxBatchRequests) + sizeof(TamSeg) * kMaxBatches * kMaxBatchRequests;
}

int slot_init(relo_ctx *ctx, BatchSlot &sl, cudaStream_t stream) {
    int rc;
    if (stream) {
        sl.stream = stream;
    } else {
        CK(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "batch stream");
        sl.own_stream = true;
    }
    if ((rc = dev_alloc(ctx, (void **)&sl.reqs_dev, slot_desc_bytes(), "batch state")) ||
        (rc = dev_alloc(ctx, (void **)&sl.bs, sizeof(BatchState), "batch state")) ||
        (rc = dev_alloc(ctx, (void **)&sl.results_dev, sizeof(relo_result) * kMaxBatchRequests, "batch state")))
        return rc;
    return RELO_OK;
}

void slot_free(relo_ctx *ctx, BatchSlot &sl) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    dev_free(ctx, sl.reqs_dev, slot_desc_bytes());
    dev_free(ctx, sl.bs, sizeof(BatchState));
    dev_free(ctx, sl.results_dev, sizeof(relo_result) * kMaxBatchRequests);
    dev_free(ctx, sl.arena, sl.arena_cap);
    dev_free(ctx, sl.ranges_dev, sizeof(float) * sl.ranges_cap);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.own_stream) cudaStreamDestroy(sl.stream);
    sl = BatchSlot();
}



// ---- served form: continuous batching ------------------------------------------------------------

using Clock = std::chrono::steady_clock;

struct Ticket {
    long long id = 0;
    int map_id = -1;
    std::vector<float> ranges, angles;
    float max_range = 0;
    relo_result result{};
    int status = RELO_PENDING;
    Clock::time_point t_submit, t_done;
    bool has_deadline = false;
    Clock::time_point deadline;   // a request still queued at this time completes with RELO_E_TIMEOUT
    size_t bytes = 0;
};

struct InFlight {
    BatchSlot slot;
    std::vector<Ticket *> tickets;
    size_t bytes = 0;
    bool busy = false;
};

}  // namespace

struct Server {
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Ticket *> queue;
    std::unordered_map<long long, Ticket *> tickets;   // submitted and not yet polled
    long long next_id = 1;
    bool running = false;
    int max_batch = 64, max_inflight = 2;
    long long budget = 0;
    size_t inflight_bytes = 0;
    int n_deadlines = 0;   // queued tickets with a deadline
    std::vector<InFlight> slots;
};

namespace {

// device bytes a request occupies while in flight (scratch and its scan)
size_t request_bytes(const relo_ctx *ctx, const Prepared &q) {
    const size_t n = (size_t)q.P->n, nh = (size_t)q.m->n_hyp, K = (size_t)q.K;
    const bool resident = ctx->p.scan_cache_bytes > 0 && find_table(*q.m, q.P->ns, q.lim) != nullptr;
    return align_up(sizeof(int2) * n) + align_up(sizeof(ScanInfo)) + align_up(8 * nh) * 2 + align_up(4 * nh) +
           align_up(4 * K) * 3 + align_up(4 * K * q.P->n_orient) + align_up(8 * K) +
           align_up(16ull * tam_chunk_cap(q.K, q.B, q.n_batches, tam_chunk_for(q.K, q.P->n_orient, ctx->n_sm))) +
           align_up(4ull * (q.n_batches + 1)) +
           align_up(4ull * 8 * 32 * q.P->n_orient * tam_offs_stride_for(tam_vpl_for(q.P->n))) +
           align_up(4ull * q.n_batches * ctx->p.local_topk) + align_up(sizeof(SelectState)) +
           align_up(sizeof(float) * q.P->n * ctx->p.n_skip_beam) + (resident ? 0 : align_up(4 * nh * q.P->ns));
}

void finish(Server *S, Ticket *t, int status, const relo_result *r) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r) t->result = *r;
    t->result.status = status;
    t->status = status;
    t->t_done = Clock::now();
}

// Launches one batch of admitted tickets on a free slot (worker thread only).
void launch_batch(relo_ctx *ctx, InFlight &f, std::vector<Ticket *> &batch, std::vector<Prepared> &pr) {
    Server *S = ctx->server;
    BatchSlot &sl = f.slot;
    size_t total = 0;
    for (Ticket *t : batch) total += t->ranges.size();
    std::vector<float> host(total);
    std::vector<size_t> off(batch.size());
    size_t pos = 0;
    for (size_t i = 0; i < batch.size(); ++i) {
        off[i] = pos;
        memcpy(host.data() + pos, batch[i]->ranges.data(), sizeof(float) * batch[i]->ranges.size());
        pos += batch[i]->ranges.size();
    }
    int rc = ensure(ctx, &sl.ranges_dev, &sl.ranges_cap, total, "scan upload");
    if (rc == RELO_OK && cudaMemcpyAsync(sl.ranges_dev, host.data(), sizeof(float) * total, cudaMemcpyHostToDevice,
                                         sl.stream) != cudaSuccess)
        rc = RELO_E_CUDA;
    if (rc == RELO_OK) {
        for (size_t i = 0; i < batch.size(); ++i) {
            pr[i].ranges_dev = sl.ranges_dev + off[i];
            pr[i].result_dev = sl.results_dev + i;
        }
        rc = run_batch(ctx, sl, pr.data(), (int)batch.size());
    }
    if (rc == RELO_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = RELO_E_CUDA;
    if (rc != RELO_OK) {
        cudaStreamSynchronize(sl.stream);
        for (Ticket *t : batch) finish(S, t, rc, nullptr);
        std::lock_guard<std::mutex> lk(S->mu);
        for (Ticket *t : batch) S->inflight_bytes -= t->bytes;
        return;
    }
    f.tickets = batch;
    f.bytes = 0;
    for (Ticket *t : batch) f.bytes += t->bytes;
    f.busy = true;
}

// Copies the results of a finished slot back and completes its tickets.
void retire(relo_ctx *ctx, InFlight &f, cudaError_t q) {
    Server *S = ctx->server;
    std::vector<relo_result> res(f.tickets.size());
    cudaError_t e = q;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), f.slot.results_dev, sizeof(relo_result) * res.size(), cudaMemcpyDeviceToHost,
                            f.slot.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f.slot.stream);
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t i = 0; i < f.tickets.size(); ++i) {
            Ticket *t = f.tickets[i];
            if (e == cudaSuccess) t->result = res[i];
            t->status = e == cudaSuccess ? res[i].status : RELO_E_CUDA;
            t->result.status = t->status;
            t->t_done = now;
        }
        S->inflight_bytes -= f.bytes;
    }
    f.tickets.clear();
    f.bytes = 0;
    f.busy = false;
}

void serve_loop(relo_ctx *ctx) {
    Server *S = ctx->server;
    for (;;) {
        bool any_busy = false, progressed = false;
        for (InFlight &f : S->slots) {
            if (!f.busy) continue;
            const cudaError_t q = cudaEventQuery(f.slot.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            retire(ctx, f, q);
            progressed = true;
        }
        InFlight *free_slot = nullptr;
        for (InFlight &f : S->slots)
            if (!f.busy) {
                free_slot = &f;
                break;
            }
        std::vector<Ticket *> cand;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // queued requests whose deadline has passed are never admitted
            if (S->n_deadlines > 0) {
                const Clock::time_point now = Clock::now();
                for (auto it = S->queue.begin(); it != S->queue.end();) {
                    Ticket *t = *it;
                    if (t->has_deadline && now >= t->deadline) {
                        t->result.status = RELO_E_TIMEOUT;
                        t->status = RELO_E_TIMEOUT;
                        t->t_done = now;
                        --S->n_deadlines;
                        it = S->queue.erase(it);
                        progressed = true;
                    } else {
                        ++it;
                    }
                }
            }
            if (!S->running && S->queue.empty() && !any_busy) break;
            if (free_slot && !S->queue.empty()) {
                while (!S->queue.empty() && (int)cand.size() < S->max_batch) {
                    Ticket *t = S->queue.front();
                    if (t->has_deadline) --S->n_deadlines;
                    cand.push_back(t);
                    S->queue.pop_front();
                }
            } else if (!progressed) {
                if (!any_busy)
                    S->cv.wait_for(lk, std::chrono::milliseconds(2));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
                continue;
            }
        }
        if (cand.empty()) continue;
        // admission: prepare in FIFO order while the HBM budget allows
        std::vector<Ticket *> batch;
        std::vector<Prepared> pr;
        std::vector<Ticket *> back;
        for (Ticket *t : cand) {
            if (!back.empty()) {
                back.push_back(t);
                continue;
            }
            Prepared q;
            const int rc = prepare(ctx, t->map_id, t->ranges.data(), t->angles.data(), (int)t->ranges.size(),
                                   t->max_range, (void *)1, &q);   // placeholder pointers, replaced at launch
            if (rc != RELO_OK) {
                finish(S, t, rc, nullptr);
                continue;
            }
            t->bytes = request_bytes(ctx, q);
            bool fits;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                fits = S->budget <= 0 || S->inflight_bytes + t->bytes <= (size_t)S->budget;
                if (!fits && S->inflight_bytes == 0 && batch.empty()) {
                    fits = false;
                } else if (fits) {
                    S->inflight_bytes += t->bytes;
                }
            }
            if (fits) {
                batch.push_back(t);
                pr.push_back(q);
            } else if (batch.empty() && !any_busy) {
                finish(S, t, RELO_E_OVER_BUDGET, nullptr);   // can never fit
            } else {
                back.push_back(t);
            }
        }
        if (!back.empty()) {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto it = back.rbegin(); it != back.rend(); ++it) {
                if ((*it)->has_deadline) ++S->n_deadlines;
                S->queue.push_front(*it);
            }
        }
        if (!batch.empty()) launch_batch(ctx, *free_slot, batch, pr);
    }
}

void serve_shutdown(relo_ctx *ctx) {
    Server *S = ctx->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->running = false;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (InFlight &f : S->slots) slot_free(ctx, f.slot);
    for (auto &kv : S->tickets) delete kv.second;
    delete S;
    ctx->server = nullptr;
}

}  // namespace

extern "C" {

void relo_default_params(relo_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->z_hit = 1.0;
    p->sigma_hit = 0.2;
    p->z_rand = 0.0;
    p->eps = 1e-6;
    p->d_max = 2.0;
    p->a_mid_min = 0.9;
    p->a_mid_max = 0.8;
    p->a_low_min = 0.8;
    p->a_low_max = 0.6;
    p->tau = 0.95;
    p->panoramic_ratio = 0.9;
    p->n_orient = 360;
    p->topk = 256;
    p->batch = 200;
    p->local_topk = 20;
    p->n_skip_beam = 1;
    p->early_stop = 1;
    p->hbm_budget = 0;
    p->max_range = 30.0;
    p->ray_tables = 1;
    p->coarse_metric = RELO_COARSE_SMAD;
    p->fine_metric = RELO_FINE_TAM;
    p->icp_iters = 0;
}

int relo_create(const relo_params *p, void *stream, relo_ctx **out) {
    if (!out) return RELO_E_INVALID_ARG;
    *out = nullptr;
    relo_ctx *ctx = new (std::nothrow) relo_ctx();
    if (!ctx) return RELO_E_INVALID_ARG;
    if (p) ctx->p = *p;
    else relo_default_params(&ctx->p);
    int rc = check_params(ctx, ctx->p);
    if (rc) {
        delete ctx;
        return rc;
    }
    ctx->blob = new (std::nothrow) Blob;
    cudaError_t e = ctx->blob ? cudaGetDevice(&ctx->device) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    // The side stream (the EDT's field pass) gets the lowest priority, so the ray cast and SMAD of the context
    // stream go first and the field pass fills what they leave; a stream the context creates itself gets the
    // highest (a caller's stream keeps its own priority).
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) {
        if (stream) {
            ctx->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithPriority(&ctx->stream, cudaStreamNonBlocking, greatest);
            ctx->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, least);
    if (e != cudaSuccess) {
        if (ctx->side) cudaStreamDestroy(ctx->side);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx->blob;
        delete ctx;
        return RELO_E_CUDA;
    }
    if ((rc = slot_init(ctx, ctx->main, ctx->stream)) ||
        (rc = dev_alloc(ctx, (void **)&ctx->bad, 2 * sizeof(int), "hypothesis check flags"))) {
        relo_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return RELO_OK;
}

int relo_destroy(relo_ctx *ctx) {
    if (!ctx) return RELO_E_INVALID_ARG;
    serve_shutdown(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &m : ctx->maps)
        if (m.live) free_map(ctx, m);
    for (SensorPlan *P : ctx->plans) free_plan(ctx, P);
    ctx->plans.clear();
    for (RayTab *t : ctx->raytabs) free_raytab(ctx, t);
    ctx->raytabs.clear();
    slot_free(ctx, ctx->main);
    if (ctx->bad) cudaFree(ctx->bad);
    dev_free(ctx, ctx->xy, ctx->xy_cap * sizeof(double));
    for (auto &pe : ctx->pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx->blob;
    delete ctx;
    return RELO_OK;
}

const char *relo_last_error(const relo_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int relo_set_params(relo_ctx *ctx, const relo_params *p) {
    if (!ctx || !p) return RELO_E_INVALID_ARG;
    int rc = check_params(ctx, *p);
    if (rc) return rc;
    const bool lut_changed = p->z_hit != ctx->p.z_hit || p->sigma_hit != ctx->p.sigma_hit ||
                             p->z_rand != ctx->p.z_rand || p->eps != ctx->p.eps || p->d_max != ctx->p.d_max;
    ctx->p = *p;
    for (auto &m : ctx->maps)
        if (m.live) drop_tables(ctx, m);
    for (SensorPlan *P : ctx->plans) free_plan(ctx, P);   // plans depend on n_orient, n_skip and Eq. 25
    ctx->plans.clear();
    if (lut_changed) {
        for (auto &m : ctx->maps) {
            if (!m.live) continue;
            int C;
            if ((rc = clamp_for(ctx, p->d_max, m.res, &C))) return rc;
            m.dev.C = C;
            CK(cudaStreamWaitEvent(ctx->stream, m.field_ready, 0), "map rebuild");
            CK(launch_field_border(m.dev, ctx->stream), "map rebuild");
            CK(map_edt(ctx, m), "map rebuild");
            CK(cudaStreamWaitEvent(ctx->stream, m.field_ready, 0), "map rebuild");
            if ((rc = build_lut(ctx, m))) return rc;
        }
        CK(cudaStreamSynchronize(ctx->stream), "map rebuild");
    }
    return RELO_OK;
}

int relo_load_map(relo_ctx *ctx, const int8_t *grid, int32_t w, int32_t h, double res, double ox, double oy,
                  int32_t *map_id) {
    return load_map_impl(ctx, grid, false, w, h, res, ox, oy, map_id);
}

int relo_load_map_dev(relo_ctx *ctx, const int8_t *grid_dev, int32_t w, int32_t h, double res, double ox, double oy,
                      int32_t *map_id) {
    return load_map_impl(ctx, grid_dev, true, w, h, res, ox, oy, map_id);
}

int relo_update_map_dev(relo_ctx *ctx, int32_t map_id, const int8_t *grid_dev) {
    if (!ctx || !grid_dev) return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    drop_tables(ctx, *m);
    CK(cudaStreamWaitEvent(ctx->stream, m->field_ready, 0), "map update");   // the last EDT still reads the grid
    CK(cudaMemcpyAsync(m->dev.grid, grid_dev, (size_t)m->dev.W * m->dev.H, cudaMemcpyDeviceToDevice, ctx->stream),
       "map update");
    CK(map_edt(ctx, *m), "map update");
    return RELO_OK;
}

int relo_update_map(relo_ctx *ctx, int32_t map_id, const int8_t *grid) {
    if (!ctx || !grid) return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    drop_tables(ctx, *m);
    CK(cudaStreamWaitEvent(ctx->stream, m->field_ready, 0), "map update");   // the last EDT still reads the grid
    CK(cudaMemcpyAsync(m->dev.grid, grid, (size_t)m->dev.W * m->dev.H, cudaMemcpyHostToDevice, ctx->stream),
       "map update");
    CK(map_edt(ctx, *m), "map update");
    return RELO_OK;
}

int relo_unload_map(relo_ctx *ctx, int32_t map_id) {
    if (!ctx) return RELO_E_INVALID_ARG;
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    CK(cudaStreamSynchronize(ctx->stream), "map unload");
    free_map(ctx, *m);
    return RELO_OK;
}

int relo_map_tables_dev(relo_ctx *ctx, int32_t map_id, int32_t *d2_dev, uint16_t *field_dev, uint8_t *occ_dev) {
    if (!ctx) return RELO_E_INVALID_ARG;
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    CK(cudaStreamWaitEvent(ctx->stream, m->field_ready, 0), "map tables");
    CK(launch_map_tables(m->dev, d2_dev, field_dev, occ_dev, ctx->stream), "map tables");
    CK(cudaStreamSynchronize(ctx->stream), "map tables");
    return RELO_OK;
}

int relo_map_walk_boxes_dev(relo_ctx *ctx, int32_t map_id, uint16_t *boxes_dev, int64_t capacity, int64_t *n_out) {
    if (!ctx) return RELO_E_INVALID_ARG;
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    const int64_t n = (int64_t)(4 * walk_frame_words(m->dev.TW, m->dev.TH));
    if (n_out) *n_out = n;
    if (!boxes_dev || capacity < n) return fail(ctx, RELO_E_INVALID_ARG, "the buffer holds fewer than 4 (TW+1)(TH+1)");
    // the boxes are written on the context stream with the occupancy tiles
    CK(cudaMemcpyAsync(boxes_dev, m->dev.reach, sizeof(uint16_t) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream),
       "walk boxes");
    CK(cudaStreamSynchronize(ctx->stream), "walk boxes");
    return RELO_OK;
}

// The coordinates are copied as given and snapped to cells on the device (k_xy_cells), so the host does no
// per-point work; one blocking read of the two check counts ends the call.
int relo_set_hypotheses(relo_ctx *ctx, int32_t map_id, const double *xy, int32_t n) {
    if (!ctx || (!xy && n > 0) || n < 0) return fail(ctx, RELO_E_INVALID_ARG, "bad hypothesis arguments");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    int rc = hyp_storage(ctx, *m, n);
    if (rc) return rc;
    m->n_hyp = 0;
    if ((rc = ensure(ctx, &ctx->xy, &ctx->xy_cap, 2 * (size_t)(n > 0 ? n : 1), "hypothesis coordinates"))) return rc;
    CK(cudaMemcpyAsync(ctx->xy, xy, 2 * sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream),
       "hypothesis upload");
    CK(cudaMemsetAsync(ctx->bad, 0, 2 * sizeof(int), ctx->stream), "hypothesis check");
    CK(launch_xy_cells(ctx->xy, n, m->ox, m->oy, m->res, m->dev, m->hyps, ctx->bad, ctx->stream), "hypothesis check");
    int flags[2] = {0, 0};
    CK(cudaMemcpyAsync(flags, ctx->bad, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream), "hypothesis check");
    CK(cudaStreamSynchronize(ctx->stream), "hypothesis check");
    if (flags[0]) return fail(ctx, RELO_E_INVALID_ARG, std::to_string(flags[0]) + " hypotheses outside the map");
    if (flags[1]) return fail(ctx, RELO_E_INVALID_ARG, std::to_string(flags[1]) + " hypotheses on occupied cells");
    m->n_hyp = n;
    return RELO_OK;
}

int relo_set_hypotheses_cells_dev(relo_ctx *ctx, int32_t map_id, const int32_t *cells_dev, int32_t n) {
    if (!ctx || (!cells_dev && n > 0) || n < 0) return fail(ctx, RELO_E_INVALID_ARG, "bad hypothesis arguments");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    return set_hyps_impl(ctx, *m, reinterpret_cast<const int2 *>(cells_dev), true, n);
}

int relo_relocalize_dev(relo_ctx *ctx, int32_t map_id, const float *ranges_dev, const float *angles,
                        int32_t n_beams, float max_range, relo_result *result_dev) {
    if (!ctx) return RELO_E_INVALID_ARG;
    Prepared pr;
    int rc = prepare(ctx, map_id, ranges_dev, angles, n_beams, max_range, result_dev, &pr);
    if (rc) return rc;
    return run_batch(ctx, ctx->main, &pr, 1);
}

int relo_relocalize(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                    float max_range, relo_result *out) {
    if (!ctx || !ranges || !angles || !out || n_beams < 2) return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    relo_request rq = {map_id, ranges, angles, n_beams, max_range, 0};
    return relo_relocalize_batch(ctx, &rq, 1, out);
}

int relo_relocalize_batch_dev(relo_ctx *ctx, const relo_request *reqs, int32_t n, relo_result *results_dev) {
    if (!ctx || !reqs || !results_dev || n < 1 || n > kMaxBatchRequests)
        return fail(ctx, RELO_E_INVALID_ARG, "1 to 256 requests per batch");
    std::vector<Prepared> pr((size_t)n);
    for (int i = 0; i < n; ++i) {
        int rc = prepare(ctx, reqs[i].map_id, reqs[i].ranges, reqs[i].angles, reqs[i].n_beams, reqs[i].max_range,
                         results_dev + i, &pr[i], reqs[i].topk);
        if (rc) return rc;
    }
    return run_batch(ctx, ctx->main, pr.data(), n);
}

int relo_relocalize_batch(relo_ctx *ctx, const relo_request *reqs, int32_t n, relo_result *out) {
    if (!ctx || !reqs || !out || n < 1 || n > kMaxBatchRequests)
        return fail(ctx, RELO_E_INVALID_ARG, "1 to 256 requests per batch");
    // The call blocks until the results are back, so the caller's buffers serve
    // directly as copy sources and destinations; nothing is staged or pinned.
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (!reqs[i].ranges || reqs[i].n_beams < 2) return fail(ctx, RELO_E_INVALID_ARG, "bad request");
        total += (size_t)reqs[i].n_beams;
    }
    BatchSlot &sl = ctx->main;
    int rc = ensure(ctx, &sl.ranges_dev, &sl.ranges_cap, total, "scan upload");
    if (rc) return rc;
    std::vector<relo_request> dreq(reqs, reqs + n);
    size_t pos = 0;
    for (int i = 0; i < n; ++i) {
        CK(cudaMemcpyAsync(sl.ranges_dev + pos, reqs[i].ranges, sizeof(float) * reqs[i].n_beams,
                           cudaMemcpyHostToDevice, ctx->stream),
           "scan upload");
        dreq[i].ranges = sl.ranges_dev + pos;
        pos += (size_t)reqs[i].n_beams;
    }
    rc = relo_relocalize_batch_dev(ctx, dreq.data(), n, sl.results_dev);
    if (rc) {
        cudaStreamSynchronize(ctx->stream);
        return rc;
    }
    CK(cudaMemcpyAsync(out, sl.results_dev, sizeof(relo_result) * n, cudaMemcpyDeviceToHost, ctx->stream),
       "result download");
    CK(cudaStreamSynchronize(ctx->stream), "relocalize");
    for (int i = 0; i < n; ++i)
        if (out[i].status != RELO_OK) return fail(ctx, out[i].status, "a scan has no valid beam");
    return RELO_OK;
}

int relo_get_stage(relo_ctx *ctx, int32_t which, void *dst_dev, int64_t bytes) {
    if (!ctx || !dst_dev) return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    if (!ctx->has_last) return fail(ctx, RELO_E_NOT_FOUND, "no relocalization has run");
    const ReqDesc &d = ctx->last;
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
        case RELO_STAGE_SMAD_NUM: src = d.smad_num; need = 8ull * d.n_hyp; break;
        case RELO_STAGE_SMAD_M: src = d.smad_m; need = 4ull * d.n_hyp; break;
        case RELO_STAGE_SURVIVORS: src = d.survivors; need = 4ull * d.K; break;
        case RELO_STAGE_TAM: src = d.T; need = 4ull * d.K * d.n_orient; break;
        case RELO_STAGE_BEST_M: src = d.best_m; need = 4ull * d.K; break;
        case RELO_STAGE_LOCAL_TOPK: src = d.local; need = 4ull * d.n_batches * d.L; break;
        case RELO_STAGE_SCAN_INFO: {
            ScanInfo si;
            SelectState ss;
            BatchState bs;
            CK(cudaMemcpyAsync(&si, d.scan, sizeof si, cudaMemcpyDeviceToHost, ctx->stream), "stage read");
            CK(cudaMemcpyAsync(&ss, d.state, sizeof ss, cudaMemcpyDeviceToHost, ctx->stream), "stage read");
            CK(cudaMemcpyAsync(&bs, ctx->last_bs, sizeof bs, cudaMemcpyDeviceToHost, ctx->stream), "stage read");
            CK(cudaStreamSynchronize(ctx->stream), "stage read");
            long long v[RELO_SCAN_INFO_LEN] = {d.ns, d.n_orient, d.n_enum, si.n_valid, si.k_ret, si.sum_real,
                                               d.K, ss.n_batches, (long long)bs.dda_steps, d.n_hyp};
            need = sizeof v;
            if ((size_t)bytes < need) return fail(ctx, RELO_E_INVALID_ARG, "destination too small");
            CK(cudaMemcpy(dst_dev, v, need, cudaMemcpyHostToDevice), "stage copy");
            return RELO_OK;
        }
        default: return fail(ctx, RELO_E_INVALID_ARG, "unknown stage");
    }
    if ((size_t)bytes < need) return fail(ctx, RELO_E_INVALID_ARG, "destination too small");
    CK(cudaMemcpyAsync(dst_dev, src, need, cudaMemcpyDeviceToDevice, ctx->stream), "stage copy");
    CK(cudaStreamSynchronize(ctx->stream), "stage copy");
    return RELO_OK;
}

int relo_synth_scans_dev(relo_ctx *ctx, int32_t map_id, const int32_t *cells_dev, int32_t n, const float *angles,
                         int32_t n_beams, float max_range, uint32_t *ranges_dev, int32_t *hit_dev, int64_t capacity,
                         int32_t *ns_out) {
    if (!ctx || !cells_dev || !angles || !ranges_dev || n < 0) return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    MapSlot *m = get_map(ctx, map_id);
    if (!m) return fail(ctx, RELO_E_NOT_FOUND, "unknown map id");
    SensorPlan *P = nullptr;
    int rc = plan_for(ctx, angles, n_beams, &P);
    if (rc) return rc;
    if (ns_out) *ns_out = P->ns;
    if ((long long)n * P->ns > capacity) return fail(ctx, RELO_E_INVALID_ARG, "output buffers hold fewer than n x N_s");
    const double rq = (double)max_range * 65536.0 / m->res;
    if (!(max_range > 0) || !(rq < 2147483647.0)) return fail(ctx, RELO_E_INVALID_ARG, "bad max_range");
    const long long rmax_q16 = llrint(rq);
    RayArgs ra;
    memset(&ra, 0, sizeof ra);
    ra.bits = m->dev.bits;
    ra.reach = m->dev.reach;
    ra.W = m->dev.W;
    ra.H = m->dev.H;
    ra.TW = m->dev.TW;
    ra.TH = m->dev.TH;
    ra.D = P->D_dev;
    ra.ns = P->ns;
    ra.ns_pad = (P->ns + 31) & ~31;
    ra.lim = (int)((rmax_q16 * rmax_q16) >> 32);
    ++ctx->batch_seq;
    ra.tab = ray_tables_view(ray_tables_for(ctx, *P, ra.lim, ctx->stream));
    ra.hyps = reinterpret_cast<const int2 *>(cells_dev);
    ra.n_hyp = n;
    CK(launch_synth(ra, ranges_dev, hit_dev, ctx->stream), "synthesized scans");
    CK(cudaStreamSynchronize(ctx->stream), "synthesized scans");
    return RELO_OK;
}

int relo_serve_start(relo_ctx *ctx, int32_t max_batch, int32_t max_inflight, int64_t hbm_budget) {
    if (!ctx) return RELO_E_INVALID_ARG;
    if (ctx->server) return fail(ctx, RELO_E_INVALID_ARG, "already serving");
    if (max_batch < 1 || max_batch > kMaxBatchRequests || max_inflight < 1 || max_inflight > 8 || hbm_budget < 0)
        return fail(ctx, RELO_E_INVALID_ARG, "max_batch in [1, 256], max_inflight in [1, 8], budget >= 0");
    Server *S = new (std::nothrow) Server();
    if (!S) return fail(ctx, RELO_E_INVALID_ARG, "out of host memory");
    S->max_batch = max_batch;
    S->max_inflight = max_inflight;
    S->budget = hbm_budget;
    S->slots.resize((size_t)max_inflight);
    ctx->server = S;
    for (InFlight &f : S->slots) {
        int rc = slot_init(ctx, f.slot, nullptr);
        if (rc == RELO_OK && cudaEventCreateWithFlags(&f.slot.done, cudaEventDisableTiming) != cudaSuccess)
            rc = RELO_E_CUDA;
        if (rc != RELO_OK) {
            serve_shutdown(ctx);
            return rc;
        }
    }
    S->running = true;
    S->worker = std::thread(serve_loop, ctx);
    return RELO_OK;
}

int relo_submit(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                float max_range, int64_t *ticket) {
    return relo_submit_until(ctx, map_id, ranges, angles, n_beams, max_range, 0.0, ticket);
}

int relo_submit_until(relo_ctx *ctx, int32_t map_id, const float *ranges, const float *angles, int32_t n_beams,
                      float max_range, double timeout_s, int64_t *ticket) {
    if (!ctx || !ranges || !angles || !ticket || n_beams < 2 || !(timeout_s >= 0.0))
        return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    Server *S = ctx->server;
    if (!S) return fail(ctx, RELO_E_INVALID_ARG, "not serving: call relo_serve_start first");
    Ticket *t = new (std::nothrow) Ticket();
    if (!t) return fail(ctx, RELO_E_INVALID_ARG, "out of host memory");
    t->map_id = map_id;
    t->ranges.assign(ranges, ranges + n_beams);
    t->angles.assign(angles, angles + n_beams);
    t->max_range = max_range;
    t->t_submit = Clock::now();
    if (timeout_s > 0.0) {
        t->has_deadline = true;
        t->deadline = t->t_submit + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                        std::min(timeout_s, 1e9)));
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->running) {
            delete t;
            return fail(ctx, RELO_E_INVALID_ARG, "server stopping");
        }
        t->id = S->next_id++;
        S->tickets[t->id] = t;
        S->queue.push_back(t);
        if (t->has_deadline) ++S->n_deadlines;
        *ticket = t->id;
    }
    S->cv.notify_one();
    return RELO_OK;
}

int relo_poll(relo_ctx *ctx, int64_t ticket, relo_result *out, double *latency_s) {
    if (!ctx || !out) return RELO_E_INVALID_ARG;
    Server *S = ctx->server;
    if (!S) return RELO_E_NOT_FOUND;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return RELO_E_NOT_FOUND;
    Ticket *t = it->second;
    if (t->status == RELO_PENDING) return RELO_PENDING;
    *out = t->result;
    if (latency_s) latency_s[0] = std::chrono::duration<double>(t->t_done - t->t_submit).count();
    const int st = t->status;
    S->tickets.erase(it);
    delete t;
    return st;
}

int relo_serve_stop(relo_ctx *ctx) {
    if (!ctx) return RELO_E_INVALID_ARG;
    serve_shutdown(ctx);
    return RELO_OK;
}

int relo_rrt_hypotheses_dev(relo_ctx *ctx, const float *clearance_dev, int32_t w, int32_t h, double res, double p0x,
                            double p0y, double rho, double eta_max, double r_robot, int32_t eps_gain, uint64_t seed,
                            int32_t max_rounds, int32_t node_cap, float *xy_dev, int32_t cap, int32_t *n_out,
                            int32_t *rounds_out, int32_t *nodes_out) {
    if (!ctx || !clearance_dev || !xy_dev || !n_out || !rounds_out || !nodes_out)
        return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    if (w < 1 || h < 1 || w > 16384 || h > 16384 || !(res > 0) || !(rho > 0) || !(eta_max > 0) || !(r_robot > 0) ||
        eps_gain < 0 || max_rounds < 1 || node_cap < 1 || cap < 0)
        return fail(ctx, RELO_E_INVALID_ARG, "bad RRT arguments");
    const char *err = "";
    const int rc = rrt_sample_dev(clearance_dev, w, h, res, p0x, p0y, rho, eta_max, r_robot, eps_gain, seed,
                                  max_rounds, node_cap, xy_dev, cap, n_out, rounds_out, nodes_out, ctx->stream, &err);
    if (rc) return fail(ctx, rc, std::string("RRT: ") + err);
    return RELO_OK;
}

int relo_rrt_sample(relo_ctx *ctx, const int8_t *grid, int32_t w, int32_t h, double res, double p0x, double p0y,
                    double rho, double eta_max, double r_robot, int32_t eps_gain, uint64_t seed, int32_t max_rounds,
                    int32_t node_cap, double *xy_out, int32_t cap, int32_t *n_out, int32_t *rounds_out,
                    int32_t *nodes_out, float *clearance_out) {
    if (!ctx || !grid || (!xy_out && cap > 0) || !n_out || !rounds_out || !nodes_out)
        return fail(ctx, RELO_E_INVALID_ARG, "null argument");
    if (w < 1 || h < 1 || w > 16382 || h > 16382 || !(res > 0) || !(rho > 0) || !(eta_max > 0) || !(r_robot > 0) ||
        eps_gain < 0 || max_rounds < 1 || node_cap < 1 || cap < 0)
        return fail(ctx, RELO_E_INVALID_ARG, "bad RRT arguments");
    cudaStream_t st = ctx->stream;
    const size_t cells = (size_t)w * h;
    // the ringed grid's EDT: a temporary map of (w + 2) x (h + 2) cells, no field border
    MapDev t;
    t.W = w + 2;
    t.H = h + 2;
    t.TW = (t.W + 7) / 8;
    t.TH = (t.H + 7) / 8;
    t.C = 65535;
    t.P = 0;
    t.Wp = (t.W + 7) & ~7;
    t.Hp = (t.H + 7) & ~7;
    const size_t pc = (size_t)t.W * t.H, fc = (size_t)t.Wp * t.Hp;
    int8_t *raw = nullptr;
    float *clr = nullptr;
    float2 *xy = nullptr;
    struct { void **p; size_t bytes; } allocs[] = {
        {(void **)&raw, cells}, {(void **)&t.grid, pc}, {(void **)&t.d2, pc * 4}, {(void **)&t.colsq, pc * 4},
        {(void **)&t.summ, sizeof(int2) * (size_t)t.W * edt_segments(t.H)}, {(void **)&t.field, fc * 2},
        {(void **)&t.bits, occupancy_words(t.TW, t.TH) * 8}, {(void **)&clr, cells * 4},
        {(void **)&xy, sizeof(float2) * (size_t)(cap > 0 ? cap : 1)}};
    int rc = RELO_OK;
    for (auto &a : allocs)
        if (rc == RELO_OK) rc = dev_alloc(ctx, a.p, a.bytes, "RRT clearance table");
    cudaError_t e = cudaSuccess;
    if (rc == RELO_OK) {
        e = cudaMemcpyAsync(raw, grid, cells, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_rrt_blocked(raw, w, h, t.grid, st);
        if (e == cudaSuccess) e = launch_edt(t, st);
        if (e == cudaSuccess) e = launch_rrt_clearance(t.d2, w, h, res, clr, st);
        if (e == cudaSuccess) ctx->kernels += 5;
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "RRT clearance table");
    }
    if (rc == RELO_OK) {
        const char *err = "";
        rc = rrt_sample_dev(clr, w, h, res, p0x, p0y, rho, eta_max, r_robot, eps_gain, seed, max_rounds, node_cap,
                            reinterpret_cast<float *>(xy), cap, n_out, rounds_out, nodes_out, st, &err);
        if (rc) rc = fail(ctx, rc, std::string("RRT: ") + err);
    }
    if (rc == RELO_OK) {
        const int n = std::min(*n_out, cap);
        std::vector<float2> host((size_t)(n > 0 ? n : 1));
        if (n > 0) e = cudaMemcpyAsync(host.data(), xy, sizeof(float2) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && clearance_out)
            e = cudaMemcpyAsync(clearance_out, clr, cells * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e, "RRT results");
        } else {
            for (int i = 0; i < n; ++i) {
                xy_out[2 * i] = host[i].x;
                xy_out[2 * i + 1] = host[i].y;
            }
        }
    }
    cudaStreamSynchronize(st);
    for (auto &a : allocs) dev_free(ctx, *a.p, a.bytes);
    return rc;
}

int relo_set_tuning(relo_ctx *ctx, const relo_tune_entry *entries, int32_t n) {
    if (!ctx || n < 0 || (n > 0 && !entries)) return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    for (int i = 0; i < n; ++i) {
        const relo_tune_entry &e = entries[i];
        const bool ok = ((e.kind == RELO_TUNE_TAM || e.kind == RELO_TUNE_TAM_ONE) && e.val[0] >= 0 && e.val[0] <= 128 && e.val[0] % 8 == 0 &&
                         e.val[1] >= 0 && e.val[1] <= 32) ||
                        (e.kind == RELO_TUNE_CAST && e.val[0] >= 0 && e.val[0] <= 32);
        if (!ok) return fail(ctx, RELO_E_INVALID_ARG, "bad tuning entry");
    }
    ctx->tuning.assign(entries, entries + n);
    return RELO_OK;
}

int relo_tam_class(int32_t n_beams) { return n_beams < 1 ? -1 : tam_vpl_for(n_beams); }

int relo_scan_cache_stats(relo_ctx *ctx, int64_t *out, int32_t n) {
    if (!ctx || (!out && n > 0) || n < 0) return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    long long tables = 0;
    for (const MapSlot &m : ctx->maps)
        if (m.live) tables += (long long)m.tables.size();
    long long wins = 0;
    for (const MapSlot &m : ctx->maps)
        if (m.live)
            for (const ScanTable *t : m.tables) wins += (long long)t->wins.size();
    const long long v[7] = {tables, ctx->table_bytes, ctx->cache_hits, ctx->cache_misses, ctx->cache_evictions,
                            wins, ctx->win_hits};
    for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
    return RELO_OK;
}

int relo_set_profiling(relo_ctx *ctx, int32_t enable) {
    if (!ctx) return RELO_E_INVALID_ARG;
    ctx->profile_mask = enable ? (1u << RELO_N_STAGES) - 1u : 0u;
    return RELO_OK;
}

int relo_set_profiling_mask(relo_ctx *ctx, uint32_t stage_mask) {
    if (!ctx) return RELO_E_INVALID_ARG;
    ctx->profile_mask = stage_mask & ((1u << RELO_N_STAGES) - 1u);
    return RELO_OK;
}

int relo_stage_times(relo_ctx *ctx, double *ms_out, int64_t *launches_out, int32_t n, int32_t reset,
                     int64_t *kernels_out) {
    if (!ctx || n < 0) return fail(ctx, RELO_E_INVALID_ARG, "bad arguments");
    CK(cudaStreamSynchronize(ctx->stream), "stage times");
    if (ctx->side) CK(cudaStreamSynchronize(ctx->side), "stage times");
    for (auto &pe : ctx->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, pe.a, pe.b), "stage times");
        ctx->stage_ms[pe.stage] += ms;
        ctx->stage_n[pe.stage] += 1;
        ctx->ev_pool.push_back(pe.a);
        ctx->ev_pool.push_back(pe.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < n && i < RELO_N_STAGES; ++i) {
        if (ms_out) ms_out[i] = ctx->stage_ms[i];
        if (launches_out) launches_out[i] = ctx->stage_n[i];
    }
    if (kernels_out) *kernels_out = ctx->kernels;
    if (reset)
        for (int i = 0; i < RELO_N_STAGES; ++i) {
            ctx->stage_ms[i] = 0;
            ctx->stage_n[i] = 0;
        }
    return RELO_OK;
}

}  // extern "C"
