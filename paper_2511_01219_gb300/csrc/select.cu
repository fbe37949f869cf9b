// Coarse ranking and batched selection.
//
// k_topk: the K hypotheses with the smallest SMAD (Sec. III intro: SMAD orders
// all positions, the ordered set is cut into batches).  Keys are
// numerator << 21 | index, so they are unique and ascending key order is
// (SMAD, index) order.  One CTA finds the K-th smallest key by MSB-first radix
// select over 8-bit digits (only the digits below the highest set bit), keeps
// the K keys not above it, and sorts them with a bitonic network.
//
// k_select_batch: after TAM has scored one batch, the per-hypothesis
// orientation argmax of Eq. 22 (already reduced by TAM into one 64-bit key per
// survivor), the batch's local top-k by TAM (ties to the earlier survivor),
// the running best over batches, and the early-termination flag once a
// batch's best reaches tau (Remark 2).
//
// k_finalize: the selected pose and counters into a relo_result.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/relo.h"
#include "relo_internal.h"

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

__global__ void __launch_bounds__(kTopkThreads) k_topk(const unsigned long long *__restrict__ keys_g, int n, int K,
                                                       int Kp, int staged, int32_t *__restrict__ out) {
    extern __shared__ __align__(16) unsigned long long sm[];
    unsigned long long *sortbuf = sm;                                   // [Kp]
    unsigned int *hist = reinterpret_cast<unsigned int *>(sm + Kp);     // [256]
    unsigned long long *keys_s = sm + Kp + 128;                         // [n] when staged
    __shared__ unsigned long long s_or;
    __shared__ int s_digit, s_below, s_cnt;
    const unsigned long long *keys = staged ? keys_s : keys_g;

    if (threadIdx.x == 0) { s_or = 0; s_cnt = 0; }
    __syncthreads();
    unsigned long long orv = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned long long k = keys_g[i];
        if (staged) keys_s[i] = k;
        orv |= k;
    }
    for (int o = 16; o > 0; o >>= 1) orv |= __shfl_xor_sync(0xffffffffu, orv, o);
    if ((threadIdx.x & 31) == 0) atomicOr(&s_or, orv);
    __syncthreads();
    int top = s_or ? 63 - __clzll((long long)s_or) : 0;
    unsigned long long prefix = 0, mask = 0;
    int remaining = K;
    for (int shift = (top / 8) * 8; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            unsigned long long k = keys[i];
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            unsigned int local = 0;
            for (int d = 0; d < 8; ++d) local += hist[lane * 8 + d];
            unsigned int incl = local;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            unsigned int excl = incl - local;
            bool here = excl < (unsigned)remaining && incl >= (unsigned)remaining;
            if (here) {
                unsigned int cum = excl;
                for (int d = 0; d < 8; ++d) {
                    unsigned int c = hist[lane * 8 + d];
                    if (cum + c >= (unsigned)remaining) {
                        s_digit = lane * 8 + d;
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
        __syncthreads();
    }
    // prefix is now the K-th smallest key
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned long long k = keys[i];
        if (k <= prefix) sortbuf[atomicAdd(&s_cnt, 1)] = k;
    }
    for (int i = K + threadIdx.x; i < Kp; i += blockDim.x) sortbuf[i] = ~0ull;
    __syncthreads();
    bitonic_sort(sortbuf, Kp);
    for (int i = threadIdx.x; i < K; i += blockDim.x) out[i] = (int32_t)(sortbuf[i] & ((1ull << kHypBits) - 1));
}

__global__ void __launch_bounds__(1024) k_select_batch(const unsigned long long *__restrict__ best_key, int s_begin,
                                                       int s_end, int n_orient, int n_enum, int local_topk,
                                                       int batch_idx, double tau, int early_stop,
                                                       int32_t *__restrict__ best_m, int32_t *__restrict__ local_out,
                                                       SelectState *st) {
    __shared__ unsigned long long v[kMaxBatch];
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = st->done;
    __syncthreads();
    if (s_skip) return;
    const int nb = s_end - s_begin;
    int np2 = 1;
    while (np2 < nb) np2 <<= 1;
    for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        if (i < nb) {
            const int s = s_begin + i;
            const unsigned long long k = best_key[s];
            const unsigned tb = (unsigned)(k >> 32);
            const unsigned q = 0xffffffffu - (unsigned)(k & 0xffffffffu);
            best_m[s] = (int)q * n_enum;
            v[i] = ((unsigned long long)(~tb) << 32) | (unsigned)s;   // ascending = TAM desc, survivor asc
        } else {
            v[i] = ~0ull;
        }
    }
    __syncthreads();
    bitonic_sort(v, np2);
    const int L = local_topk < nb ? local_topk : nb;
    for (int r = threadIdx.x; r < local_topk; r += blockDim.x)
        local_out[(size_t)batch_idx * local_topk + r] = r < L ? (int)(v[r] & 0xffffffffu) : -1;
    if (threadIdx.x == 0) {
        const unsigned tb = ~(unsigned)(v[0] >> 32);
        const unsigned s = (unsigned)(v[0] & 0xffffffffu);
        const unsigned long long cand = ((unsigned long long)tb << 32) | (0xffffffffu - s);
        if (cand > st->best) st->best = cand;
        st->n_batches += 1;
        st->n_tam_evals += (long long)nb * n_orient;
        if (early_stop && (double)__uint_as_float(tb) >= tau) st->done = 1;
    }
}

__global__ void k_finalize(FinalizeArgs a) {
    relo_result r;
    const SelectState st = *a.st;
    const unsigned tb = (unsigned)(st.best >> 32);
    const int s = (int)(0xffffffffu - (unsigned)(st.best & 0xffffffffu));
    r.n_batches = st.n_batches;
    r.n_tam_evals = st.n_tam_evals;
    r.n_smad_evals = a.n_smad_evals;
    if (a.scan->n_valid <= 0 || st.n_batches == 0) {
        r.status = RELO_E_NO_VALID_BEAMS;
        r.x = r.y = r.theta = r.tam = r.smad = 0.0;
        r.smad_num = 0;
        r.hyp = -1;
        r.m = -1;
    } else {
        const int h = a.survivors[s];
        const int m = a.best_m[s];
        const int2 c = a.hyps[h];
        r.status = RELO_OK;
        r.hyp = h;
        r.m = m;
        r.tam = (double)__uint_as_float(tb);
        r.x = a.ox + ((double)c.x + 0.5) * a.res;
        r.y = a.oy + ((double)c.y + 0.5) * a.res;
        double th = (double)m * (2.0 * M_PI) / (double)a.ns;
        if (th >= M_PI) th -= 2.0 * M_PI;
        r.theta = th;
        r.smad_num = a.smad_num[h];
        r.smad = (double)r.smad_num / a.fov_beams / 65536.0 * a.res;
    }
    *reinterpret_cast<relo_result *>(a.result) = r;
}

}  // namespace

cudaError_t launch_topk(const unsigned long long *keys, int n, int K, int32_t *out, cudaStream_t s) {
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    int staged = n <= kStageMax ? 1 : 0;
    size_t smem = (size_t)Kp * 8 + 256 * 4 + (staged ? (size_t)n * 8 : 0);
    cudaError_t e = cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_topk<<<1, kTopkThreads, smem, s>>>(keys, n, K, Kp, staged, out);
    return cudaGetLastError();
}

cudaError_t launch_select_batch(const unsigned long long *best_key, int s_begin, int s_end, int n_orient, int n_enum,
                                int local_topk, int batch_idx, double tau, int early_stop, int32_t *best_m,
                                int32_t *local_out, SelectState *st, cudaStream_t s) {
    k_select_batch<<<1, 1024, 0, s>>>(best_key, s_begin, s_end, n_orient, n_enum, local_topk, batch_idx, tau,
                                      early_stop, best_m, local_out, st);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s) {
    k_finalize<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace relo
