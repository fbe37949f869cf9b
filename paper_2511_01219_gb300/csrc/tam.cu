// Scan preparation (Eq. 11, 16, 26) and TAM scoring (Eq. 22-31).
//
// k_scan_prep (one CTA): converts the float32 ranges of the (n_skip-strided)
// beams to Q16 cell ranges R_i = llrint(z_i * 65536 / res) for valid beams
// (finite, 0 < z < max_range; invalid beams count 0, Eq. 16 and the
// placeholder rule after Eq. 20), sums them, compacts the valid beams in
// order into (panoramic index b_i, R_i) pairs, and fixes the retained-beam
// count of Eq. 27: the three top-k means of a descending list satisfy
// mean(k_low) >= mean(k_mid) >= mean(k_full) whenever k_low <= k_mid <= k_full
// (a running mean of a descending list never grows), so their median is the
// mean over the median of the three k values.
//
// k_tam: one warp per (survivor, orientation m).  For each valid beam i the
// endpoint cell is hypothesis + round-half-up(R_i * D_{(b_i + m) mod N_s} /
// 2^46); its clamped squared distance b = min(d2, C) is read from the tiled
// field (off-map endpoints take C, i.e. d = d_max).  The likelihood l
// (Eq. 23) falls strictly as b grows, so the descending sort of Eq. 24 is the
// ascending order of b: the warp finds the k-th smallest b by bisection over
// [0, C] with register-resident values, and the top-k sum of l is
// sum_{b < b_k} l(b) + (k - #{b < b_k}) l(b_k).  A shared-memory table holds
// l(b) and sqrt(C) - sqrt(b) for every b in [0, C]; with those and the exact
// integer sum of b, lane 0 evaluates Eq. 27-31:
//     wp = exp(Lbar),  d_max - dbar = res * sum(sqrt(C) - sqrt(b)) / N,
//     s_d = min(d_max - dbar, d_max - d_min) / (d_max - d_min),
//     var = res^2 * sum(b) / N - dbar^2,  c = exp(-var / 2),
//     T = cbrt(wp * s_d * c).
// Summing sqrt(C) - sqrt(b) (never negative) instead of sqrt(b) keeps s_d
// accurate when dbar is close to d_max.  Each score is written out and folded
// into a per-survivor 64-bit key (T bits, then smaller m) with atomicMax:
// that is the orientation argmax of Eq. 22.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTamWarps = 8;
constexpr uint32_t kNoBeam = 0xffffu;

__global__ void __launch_bounds__(1024) k_scan_prep(const float *__restrict__ ranges, int n, int skip,
                                                    float max_range, double res, const int32_t *__restrict__ b,
                                                    double a_mid, double a_low, int2 *__restrict__ vbR,
                                                    ScanInfo *info) {
    __shared__ int warp_cnt[32];
    __shared__ long long warp_sum[32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    long long my_sum = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int R = 0;
        bool ok = false;
        if (i < n) {
            const float z = ranges[(size_t)i * skip];
            ok = isfinite(z) && z > 0.0f && z < max_range;
            if (ok) R = (int)__double2ll_rn(__ddiv_rn(__dmul_rn((double)z, 65536.0), res));
        }
        my_sum += R;
        const unsigned bal = __ballot_sync(kFull, ok);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = lane < (int)(blockDim.x >> 5) ? warp_cnt[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            warp_cnt[lane] = incl - v;   // exclusive
        }
        __syncthreads();
        if (ok) {
            const int pos = s_base + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
            vbR[pos] = make_int2(b[i], R);
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += warp_cnt[warp] + __popc(bal);
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(kFull, my_sum, o);
    if (lane == 0) warp_sum[warp] = my_sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sum[w];
        const int N = s_base;
        int km = (int)floor(__dmul_rn(a_mid, (double)N));
        if (km < 1) km = 1;
        int kl = (int)floor(__dmul_rn(a_low, (double)N));
        if (kl < 1) kl = 1;
        int lo = km < kl ? km : kl, hi = km < kl ? kl : km;
        int k = N < lo ? lo : (N > hi ? hi : N);   // median of {N, km, kl}
        info->sum_real = tot;
        info->n_valid = N;
        info->k_ret = k;
        info->dda_steps = 0ull;
        info->ray_work = 0u;
    }
}

// Work is split into tasks (orientation q, chunk of survivors).  A CTA first
// computes the endpoint offsets of its orientation for every valid beam,
// round-half-up(R_i * D_{(b_i + m) mod N_s} / 2^46) per axis, packed as two
// int16 in shared memory; each warp then scores one survivor at a time with
// those offsets, so the 64-bit offset arithmetic is paid once per
// (orientation, beam) instead of once per (survivor, orientation, beam).
template <int VPL>
__global__ void __launch_bounds__(kTamWarps * 32) k_tam(TamArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = a.state->done;
    const int N = a.scan->n_valid;
    const int k = a.scan->k_ret;
    __syncthreads();
    if (s_stop || N <= 0) return;

    float2 *lut = reinterpret_cast<float2 *>(smem);
    uint32_t *offs = reinterpret_cast<uint32_t *>(smem + (size_t)(a.C + 1) * sizeof(float2));
    for (int i = threadIdx.x; i <= a.C; i += blockDim.x) lut[i] = a.lut[i];

    const int nb = a.s_end - a.s_begin;
    const int n_tasks = a.n_orient * a.n_chunks;
    const float Nf = (float)N;
    for (int task = blockIdx.x; task < n_tasks; task += gridDim.x) {
        const int q = task % a.n_orient;
        const int chunk = task / a.n_orient;
        const int m = q * a.n_enum;
        __syncthreads();   // the previous task's reads of offs are done
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int2 bR = a.vbR[i];
            int j = bR.x + m;
            if (j >= a.ns) j -= a.ns;
            const int2 d = a.D[j];
            const int ox = (int)(((long long)bR.y * d.x + (1ll << 45)) >> 46);
            const int oy = (int)(((long long)bR.y * d.y + (1ll << 45)) >> 46);
            offs[i] = ((uint32_t)ox & 0xffffu) | ((uint32_t)oy << 16);
        }
        __syncthreads();
        const int s_lo = a.s_begin + chunk * a.chunk;
        const int s_hi = min(a.s_end, s_lo + a.chunk);
        for (int s = s_lo + warp; s < s_hi; s += kTamWarps) {
            const int2 hc = a.hyps[a.survivors[s]];
            uint32_t v[VPL];
            int sumb = 0;
#pragma unroll
            for (int t = 0; t < VPL; ++t) {
                const int i = (t << 5) + lane;
                uint32_t bv = kNoBeam;
                if (i < N) {
                    const uint32_t o = offs[i];
                    const int ex = hc.x + (int)(short)(o & 0xffffu);
                    const int ey = hc.y + ((int)o >> 16);
                    bv = ((unsigned)ex < (unsigned)a.W && (unsigned)ey < (unsigned)a.H)
                             ? (uint32_t)__ldg(a.field + tile_index(ex, ey, a.TW))
                             : (uint32_t)a.C;
                    sumb += (int)bv;
                }
                v[t] = bv;
            }
            // smallest b_k with #{b <= b_k} >= k
            int lo = 0, hi = a.C;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                int c = 0;
#pragma unroll
                for (int t = 0; t < VPL; ++t) c += (v[t] <= (uint32_t)mid) ? 1 : 0;
                c = __reduce_add_sync(kFull, c);
                if (c >= k) hi = mid;
                else lo = mid + 1;
            }
            const uint32_t bk = (uint32_t)lo;
            float sg = 0.0f, sl = 0.0f;
            int clt = 0;
#pragma unroll
            for (int t = 0; t < VPL; ++t) {
                if (v[t] != kNoBeam) {
                    const float2 lg = lut[v[t]];
                    sg += lg.y;
                    if (v[t] < bk) {
                        sl += lg.x;
                        ++clt;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sg += __shfl_xor_sync(kFull, sg, o);
                sl += __shfl_xor_sync(kFull, sl, o);
            }
            clt = __reduce_add_sync(kFull, clt);
            sumb = __reduce_add_sync(kFull, sumb);
            if (lane == 0) {
                const float ltop = sl + (float)(k - clt) * lut[bk].x;
                const float lbar = ltop / (float)k;
                const float wp = expf(lbar);
                const float dd = a.res * sg / Nf;   // d_max - dbar
                const float dbar = a.d_max - dd;
                const float span = a.d_max - a.d_min;
                const float sd = fminf(dd, span) / span;
                float var = a.res2 * ((float)sumb / Nf) - dbar * dbar;
                var = fmaxf(var, 0.0f);
                const float c = expf(-0.5f * var);
                const float T = cbrtf(wp * sd * c);
                a.T[(size_t)s * a.n_orient + q] = T;
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(T) << 32) | (unsigned long long)(0xffffffffu - (unsigned)q);
                atomicMax(a.best_key + s, key);
            }
        }
    }
    (void)nb;
}

template <int VPL>
cudaError_t run_tam(TamArgs a, int n_sm, cudaStream_t s, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_tam<VPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tam<VPL>, kTamWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // Pick the number of survivor chunks per orientation so that the tasks
    // fill whole waves of resident CTAs and whole rounds of the CTA's warps.
    const int nb = a.s_end - a.s_begin;
    const int slots = n_sm * occ;
    const int max_chunks = (nb + kTamWarps - 1) / kTamWarps;
    int best_nc = 1;
    double best_eff = -1.0;
    for (int nc = 1; nc <= max_chunks && nc <= 64; ++nc) {
        const int chunk = (nb + nc - 1) / nc;
        const long long tasks = (long long)a.n_orient * ((nb + chunk - 1) / chunk);
        const long long waves = (tasks + slots - 1) / slots;
        const double eff = (double)tasks / (double)(waves * slots) *
                           (double)chunk / (double)(((chunk + kTamWarps - 1) / kTamWarps) * kTamWarps);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_nc = nc;
        }
    }
    a.chunk = (nb + best_nc - 1) / best_nc;
    a.n_chunks = (nb + a.chunk - 1) / a.chunk;
    long long tasks = (long long)a.n_orient * a.n_chunks;
    int grid = (int)(tasks < slots ? tasks : slots);
    if (grid < 1) grid = 1;
    k_tam<VPL><<<grid, kTamWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_prep(const float *ranges, int n, int skip, float max_range, double res, const int32_t *b,
                             double a_mid, double a_low, int2 *vbR, ScanInfo *info, cudaStream_t s) {
    k_scan_prep<<<1, 1024, 0, s>>>(ranges, n, skip, max_range, res, b, a_mid, a_low, vbR, info);
    return cudaGetLastError();
}

cudaError_t launch_tam(const TamArgs &a, int n_beams_max, int n_sm, cudaStream_t s) {
    if (a.s_end <= a.s_begin) return cudaSuccess;
    size_t smem = (size_t)(a.C + 1) * sizeof(float2) + (size_t)n_beams_max * sizeof(uint32_t);
    const int vpl = (n_beams_max + 31) / 32;
#define RELO_TAM_CASE(V) \
    if (vpl <= V) return run_tam<V>(a, n_sm, s, smem);
    RELO_TAM_CASE(8) RELO_TAM_CASE(12) RELO_TAM_CASE(16) RELO_TAM_CASE(20) RELO_TAM_CASE(24) RELO_TAM_CASE(28)
    RELO_TAM_CASE(32) RELO_TAM_CASE(36) RELO_TAM_CASE(40) RELO_TAM_CASE(44) RELO_TAM_CASE(48) RELO_TAM_CASE(52)
    RELO_TAM_CASE(56) RELO_TAM_CASE(60) RELO_TAM_CASE(64)
#undef RELO_TAM_CASE
    return cudaErrorInvalidValue;
}

}  // namespace relo
