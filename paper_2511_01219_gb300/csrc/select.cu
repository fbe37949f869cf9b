// Coarse ranking and batched selection.
//
// k_topk: the K hypotheses with the smallest SMAD (or CAER; Sec. III intro:
// the coarse metric orders all positions, the ordered set is cut into
// batches).  Keys are numerator << 21 | index, so they are unique and
// ascending key order is (numerator, index) order.  One CTA histograms the 11 bits below the keys' highest
// set bit, finds the digit holding the K-th smallest key, and orders the keys
// up to that digit (by rank counting when they are few: keys are unique),
// keeping the first K;
// when too many keys share that digit it falls back to an MSB-first radix
// select over 8-bit digits.
//
// k_select_batch: after TAM has scored one batch, the per-hypothesis
// orientation argmax of Eq. 22 (already reduced by TAM into one 64-bit key per
// survivor), the batch's local top-k by TAM (ties to the earlier survivor) by
// rank counting, the running best over batches, and the early-termination
// flag once a batch's best reaches tau (Remark 2).
//
// With ICP refinement on, k_select_batch stops at the local top-k; k_icp
// (icp.cu) refines and re-scores those poses, and k_icp_best takes the
// running best and the early-termination test on the re-evaluated scores (the
// overview of Sec. III).
//
// The last selection launch also writes the selected pose and counters into
// each request's relo_result.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "../../include/relo.h"
#include "relo_internal.h"
#include "tam_offsets.cuh"

namespace relo {

namespace {

constexpr int kTopkThreads = 1024;
constexpr int kStageMax = 20480;   // keys staged in shared memory (160 KiB)

__device__ void bitonic_sort(unsigned long long *v, int n_pow2) {
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    unsigned long long a = v[i], b = v[p];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        v[i] = b;
                        v[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kRankMax = 512;   // up to this many keys, rank counting (one barrier) beats the sorting network

// The first K of n unique keys v[0 .. n) (v has room for the next power of two)
// in ascending order into the survivor list: by rank counting (each key's
// position is the number of smaller keys) for a few keys, else by sorting.
__device__ void order_out(unsigned long long *v, int n, int K, int32_t *survivors) {
    if (n <= kRankMax) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long me = v[i];
            int rank = 0;
            for (int k = 0; k < n; ++k) rank += v[k] < me ? 1 : 0;   // every thread reads the same v[k]
            if (rank < K) survivors[rank] = (int32_t)(me & ((1ull << kHypBits) - 1));
        }
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + threadIdx.x; i < P; i += blockDim.x) v[i] = ~0ull;
    __syncthreads();
    bitonic_sort(v, P);
    for (int i = threadIdx.x; i < K; i += blockDim.x) survivors[i] = (int32_t)(v[i] & ((1ull << kHypBits) - 1));
}

constexpr int kTopkBins = 2048;   // first pass: the 11 bits below the keys' highest set bit

// The first K keys of request d in ascending order into its survivor list,
// by one CTA (sm: the launch's dynamic shared memory).
__device__ void topk_request(const ReqDesc &d, unsigned long long *sm, int Kp_cap, int stage_cap) {
    const unsigned long long *keys_g = d.keys;
    const int n = d.n_hyp, K = d.K;
    unsigned long long *sortbuf = sm;                                          // [2 * Kp_cap]
    unsigned int *hist = reinterpret_cast<unsigned int *>(sm + 2 * Kp_cap);    // [kTopkBins]
    unsigned long long *keys_s = sm + 2 * Kp_cap + kTopkBins / 2;              // [stage_cap]
    __shared__ unsigned long long s_or;
    __shared__ int s_digit, s_below, s_cnt;
    __shared__ unsigned int s_warp[32];
    const bool staged = n <= stage_cap;
    const unsigned long long *keys = staged ? keys_s : keys_g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_round = (n + blockDim.x - 1) / blockDim.x * blockDim.x;   // whole warps in every round

    if (threadIdx.x == 0) { s_or = 0; s_cnt = 0; }
    for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    unsigned long long orv = 0;
    constexpr int kLoads = 8;   // keys a thread has in flight
    for (int i0 = threadIdx.x; i0 < n; i0 += kLoads * blockDim.x) {
        unsigned long long k[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int i = i0 + u * blockDim.x;
            k[u] = i < n ? keys_g[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int i = i0 + u * blockDim.x;
            if (staged && i < n) keys_s[i] = k[u];
            orv |= k[u];
        }
    }
    for (int o = 16; o > 0; o >>= 1) orv |= __shfl_xor_sync(0xffffffffu, orv, o);
    if (lane == 0) atomicOr(&s_or, orv);
    __syncthreads();
    const int top = s_or ? 63 - __clzll((long long)s_or) : 0;

    // One pass over 11-bit digits finds the digit b* of the K-th smallest key;
    // the keys with digit < b* are all in, those with digit b* are sorted with
    // them and the first K kept.
    const int sh = top >= 10 ? top - 10 : 0;   // every key is < 2^(top + 1), so key >> sh < 2^11
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[keys[i] >> sh], 1u);
    __syncthreads();
    {
        const unsigned a = hist[2 * threadIdx.x], b = hist[2 * threadIdx.x + 1];   // 1024 threads x 2 bins
        unsigned incl = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned v = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            s_warp[lane] = v - s_warp[lane];   // exclusive prefix of the warp totals
        }
        __syncthreads();
        const unsigned excl = s_warp[warp] + incl - (a + b);
        if (excl < (unsigned)K && excl + a + b >= (unsigned)K) {
            if (excl + a >= (unsigned)K) {
                s_digit = 2 * threadIdx.x;
                s_below = (int)excl;
            } else {
                s_digit = 2 * threadIdx.x + 1;
                s_below = (int)(excl + a);
            }
        }
        __syncthreads();
    }
    const unsigned long long dstar = (unsigned long long)s_digit;
    const int n_sel = s_below + (int)hist[s_digit];   // keys with digit <= b*
    if (n_sel <= 2 * Kp_cap) {
        for (int i = threadIdx.x; i < n_round; i += blockDim.x) {   // one slot reservation per warp
            const unsigned long long k = i < n ? keys[i] : ~0ull;
            const bool take = i < n && (k >> sh) <= dstar;
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&s_cnt, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (take) sortbuf[base + __popc(bal & ((1u << lane) - 1u))] = k;
        }
        __syncthreads();
        order_out(sortbuf, n_sel, K, d.survivors);
        return;
    }

    // Many keys share the digit b*: MSB-first radix select over 8-bit digits.
    unsigned long long prefix = 0, mask = 0;
    int remaining = K;
    for (int shift = (top / 8) * 8; shift >= 0; shift -= 8) {
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long k = keys[i];
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned int local = 0;
            for (int dg = 0; dg < 8; ++dg) local += hist[lane * 8 + dg];
            unsigned int incl = local;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            unsigned int excl = incl - local;
            bool here = excl < (unsigned)remaining && incl >= (unsigned)remaining;
            if (here) {
                unsigned int cum = excl;
                for (int dg = 0; dg < 8; ++dg) {
                    unsigned int c = hist[lane * 8 + dg];
                    if (cum + c >= (unsigned)remaining) {
                        s_digit = lane * 8 + dg;
                        s_below = (int)cum;
                        break;
                    }
                    cum += c;
                }
            }
        }
        __syncthreads();
        prefix |= (unsigned long long)s_digit << shift;
        mask |= 255ull << shift;
        remaining -= s_below;
    }
    // prefix is now the K-th smallest key; one slot reservation per warp
    for (int i = threadIdx.x; i < n_round; i += blockDim.x) {
        const unsigned long long k = i < n ? keys[i] : ~0ull;
        const bool take = i < n && k <= prefix;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_cnt, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) sortbuf[base + __popc(bal & ((1u << lane) - 1u))] = k;
    }
    __syncthreads();
    order_out(sortbuf, K, K, d.survivors);
}

// One CTA per request ranks it and then builds its TAM work order from the
// survivors; the CTAs after the first R compute the requests' TAM endpoint
// offsets meanwhile (they need the scan preparation, not the ranking).
__global__ void __launch_bounds__(kTopkThreads) k_topk(const ReqDesc *__restrict__ reqs, int Kp_cap, int stage_cap,
                                                       int R, int max_n_orient) {
    extern __shared__ __align__(16) unsigned long long sm[];
    if ((int)blockIdx.x >= R) {
        for (int t = (int)blockIdx.x - R; t < R * max_n_orient; t += (int)gridDim.x - R) {
            const ReqDesc &o = reqs[t / max_n_orient];
            const int q = t % max_n_orient;
            if (q < o.n_orient && !o.state->done && o.tam_offs) tam_offsets_one(o, q);
        }
        return;
    }
    const ReqDesc &d = reqs[blockIdx.x];
    topk_request(d, sm, Kp_cap, stage_cap);
    __syncthreads();   // every survivor is written
    tam_chunks_one(d);
}

// The request's pose, score and counters into its relo_result (one thread).
__device__ void finalize_request(const ReqDesc &d) {
    relo_result r;
    const SelectState st = *d.state;
    const unsigned tb = (unsigned)(st.best >> 32);
    const int s = (int)(0xffffffffu - (unsigned)(st.best & 0xffffffffu));
    r.n_batches = st.n_batches;
    r.n_tam_evals = st.n_tam_evals;
    r.n_smad_evals = d.n_smad_evals;
    if (d.scan->n_valid <= 0 || st.n_batches == 0) {
        r.status = RELO_E_NO_VALID_BEAMS;
        r.x = r.y = r.theta = r.tam = r.smad = 0.0;
        r.smad_num = 0;
        r.hyp = -1;
        r.m = -1;
        r.n_tam_evals = 0;
    } else {
        const int h = d.survivors[s];
        const int m = d.best_m[s];
        const int2 c = d.hyps[h];
        r.status = RELO_OK;
        r.hyp = h;
        r.m = m;
        r.tam = (double)score_of(tb);
        double th;
        if (d.icp_iters > 0) {   // the refined continuous pose
            const double *ps = d.ref_pose + 3 * (size_t)s;
            r.x = d.ox + ps[0];
            r.y = d.oy + ps[1];
            th = remainder(ps[2], 2.0 * M_PI);
        } else {
            r.x = d.ox + ((double)c.x + 0.5) * d.resd;
            r.y = d.oy + ((double)c.y + 0.5) * d.resd;
            th = (double)m * (2.0 * M_PI) / (double)d.ns;
        }
        if (th >= M_PI) th -= 2.0 * M_PI;
        r.theta = th;
        r.smad_num = d.smad_num[h];
        r.smad = (double)r.smad_num / d.fov / 65536.0 * d.resd;
    }
    *reinterpret_cast<relo_result *>(d.result) = r;
}

// one CTA per request: selection of batches batch_lo .. batch_hi - 1 in
// order (each skipped when the request has fewer batches or already
// terminated early).  Keys (TAM descending, then survivor position) are
// unique, so each survivor's rank is the number of smaller keys; ranks below
// L fill the local top-k directly.  With last, the launch also writes every
// request's result.  With icp the launch stops at the local top-k and the
// counters: k_icp refines and re-scores them, k_icp_best takes their best.
__global__ void __launch_bounds__(1024) k_select_batch(const ReqDesc *__restrict__ reqs, int batch_lo, int batch_hi,
                                                       int last, int icp) {
    __shared__ unsigned long long v[kMaxBatch];
    __shared__ int s_skip;
    const ReqDesc &d = reqs[blockIdx.x];
    const int n_batches = d.n_batches;
    const bool none_valid = d.scan->n_valid <= 0, early = d.early_stop;
    for (int batch_idx = batch_lo; batch_idx < batch_hi; ++batch_idx) {
    __syncthreads();   // the previous batch's ranks and state updates are done
    if (threadIdx.x == 0) s_skip = batch_idx >= n_batches || none_valid || (early && d.state->done);
    __syncthreads();
    if (!s_skip) {
        SelectState *st = d.state;
        const int s_begin = batch_idx * d.B;
        const int s_end = min(d.K, s_begin + d.B);
        const int nb = s_end - s_begin;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const int s = s_begin + i;
            const unsigned long long k = d.best_key[s];
            const unsigned tb = (unsigned)(k >> 32);
            const unsigned q = 0xffffffffu - (unsigned)(k & 0xffffffffu);
            d.best_m[s] = (int)q * d.n_enum;
            v[i] = ((unsigned long long)(~tb) << 32) | (unsigned)s;   // ascending = TAM desc, survivor asc
        }
        __syncthreads();
        const int L = d.L;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const unsigned long long me = v[i];
            int rank = 0;
            for (int k = 0; k < nb; ++k) rank += v[k] < me ? 1 : 0;
            if (rank < L) d.local[(size_t)batch_idx * L + rank] = (int)(me & 0xffffffffu);
            if (rank == 0) {
                const unsigned tb = ~(unsigned)(me >> 32);
                const unsigned s = (unsigned)(me & 0xffffffffu);
                const unsigned long long cand = ((unsigned long long)tb << 32) | (0xffffffffu - s);
                st->n_batches += 1;
                st->n_tam_evals += (long long)nb * d.n_orient;
                if (!icp) {
                    if (cand > st->best) st->best = cand;
                    if (d.early_stop && (double)score_of(tb) >= d.tau) st->done = 1;
                }
            }
        }
        for (int r = nb + threadIdx.x; r < L; r += blockDim.x) d.local[(size_t)batch_idx * L + r] = -1;
    }
    }
    if (last) {
        __syncthreads();   // the selection state of this launch is complete
        if (threadIdx.x == 0) finalize_request(d);
    }
}

// One thread per request, after k_icp: for batches batch_lo .. batch_hi - 1
// in order (each skipped when the request has fewer or already terminated),
// the best re-evaluated local top-k pose (ties to the earlier survivor) joins
// the running best, and early termination follows its score (the overview of
// Sec. III: the test is made on the re-evaluated score).  With last, the
// result.
__global__ void k_icp_best(const ReqDesc *__restrict__ reqs, int R, int batch_lo, int batch_hi, int last) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const ReqDesc &d = reqs[r];
    SelectState *st = d.state;
    if (d.scan->n_valid > 0) {
        for (int b = batch_lo; b < batch_hi && b < d.n_batches; ++b) {
            if (st->done) break;
            unsigned long long top = 0ull;
            for (int i = 0; i < d.L; ++i) {
                const int s = d.local[(size_t)b * d.L + i];
                if (s < 0) continue;
                const unsigned long long key = ((unsigned long long)score_code(d.reev[s]) << 32) |
                                               (0xffffffffu - (unsigned)s);
                top = key > top ? key : top;
            }
            if (top == 0ull) continue;
            if (top > st->best) st->best = top;
            if (d.early_stop && (double)score_of((unsigned)(top >> 32)) >= d.tau) st->done = 1;
        }
    }
    if (last) finalize_request(d);
}

}  // namespace

cudaError_t launch_topk(const ReqDesc *reqs, int R, int max_n_hyp, int max_K, int max_n_orient, int n_sm,
                        cudaStream_t s) {
    int Kp = 1;
    while (Kp < max_K) Kp <<= 1;
    const size_t fixed = (size_t)2 * Kp * 8 + (size_t)kTopkBins * 4;
    const size_t smem_max = 227 * 1024;
    const int stage_cap = (max_n_hyp <= kStageMax && fixed + (size_t)max_n_hyp * 8 <= smem_max) ? max_n_hyp : 0;
    const size_t smem = fixed + (size_t)stage_cap * 8;
    cudaError_t e = cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one CTA per SM for the offsets (the ranking CTAs' shared memory leaves room for no second one)
    const int n_off = std::max(1, std::min(R * std::max(max_n_orient, 1), n_sm));
    k_topk<<<R + n_off, kTopkThreads, smem, s>>>(reqs, Kp, stage_cap, R, std::max(max_n_orient, 1));
    return cudaGetLastError();
}

cudaError_t launch_select_batch(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, bool last, bool icp,
                                cudaStream_t s) {
    k_select_batch<<<R, 1024, 0, s>>>(reqs, batch_lo, batch_hi, last ? 1 : 0, icp ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_icp_best(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, bool last, cudaStream_t s) {
    k_icp_best<<<(R + 63) / 64, 64, 0, s>>>(reqs, R, batch_lo, batch_hi, last ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace relo
