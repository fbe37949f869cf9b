// Scan preparation (Eq. 11, 16, 26) of one request, as CTA-wide device
// functions: the ray-cast launch runs them first in its first CTAs, and
// k_scan_prep when a batch casts no rays.
//
// scan_prep_request (the whole CTA, any block size that is a multiple of 32)
// converts the float32 ranges of the (n_skip-strided) beams to Q16 cell ranges
// R_i = llrint(z_i * 65536 / res) for valid beams (finite, 0 < z < max_range;
// invalid beams count 0, Eq. 16 and the placeholder rule after Eq. 20), sums
// them, compacts the valid beams in order into (panoramic index b_i, R_i)
// pairs (and keeps every beam's R_i, 0 if invalid, for CAER), and fixes the retained-beam count of Eq. 27: the three top-k means of
// a descending list satisfy mean(k_low) >= mean(k_mid) >= mean(k_full)
// whenever k_low <= k_mid <= k_full (a running mean of a descending list never
// grows), so their median is the mean over the median of the three k values.
// It also resets the request's selection buffers (argmax keys 0, shifts and
// local top-k -1, selection state 0), so a batch needs no separate memsets.
//
// scan_prep_fill writes share `part` of `parts` of the request's TAM scores
// with NaN (unscored).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

static __device__ __forceinline__ void scan_prep_fill(const ReqDesc &d, int part, int parts) {
    const int nT = d.K * d.n_orient;
    for (int i = part * blockDim.x + threadIdx.x; i < nT; i += parts * blockDim.x) d.T[i] = __int_as_float(0x7fffffff);
}

static __device__ __noinline__ void scan_prep_request(const ReqDesc &d) {
    __shared__ int warp_cnt[32];
    __shared__ long long warp_sum[32];
    __shared__ int s_base;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int n = d.n_beams;
    if (threadIdx.x == 0) s_base = 0;
    for (int i = threadIdx.x; i < d.K; i += blockDim.x) {
        d.best_key[i] = 0ull;
        d.best_m[i] = -1;
    }
    for (int i = threadIdx.x; i < d.n_batches * d.L; i += blockDim.x) d.local[i] = -1;
    if (threadIdx.x == 0) {
        d.state->best = 0ull;
        d.state->n_tam_evals = 0;
        d.state->n_batches = 0;
        d.state->done = 0;
    }
    long long my_sum = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int R = 0;
        bool ok = false;
        if (i < n) {
            const float z = d.ranges[(size_t)i * d.skip];
            ok = isfinite(z) && z > 0.0f && z < d.max_range;
            if (ok) R = (int)__double2ll_rn(__ddiv_rn(__dmul_rn((double)z, 65536.0), d.resd));
            d.Rall[i] = R;
        }
        my_sum += R;
        const unsigned bal = __ballot_sync(full, ok);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = lane < nwarps ? warp_cnt[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += t;
            }
            warp_cnt[lane] = incl - v;   // exclusive
        }
        __syncthreads();
        if (ok) {
            const int pos = s_base + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
            d.vbR[pos] = make_int2(d.b[i], R);
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += warp_cnt[warp] + __popc(bal);
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(full, my_sum, o);
    if (lane == 0) warp_sum[warp] = my_sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < nwarps; ++w) tot += warp_sum[w];
        const int N = s_base;
        int km = (int)floor(__dmul_rn(d.a_mid, (double)N));
        if (km < 1) km = 1;
        int kl = (int)floor(__dmul_rn(d.a_low, (double)N));
        if (kl < 1) kl = 1;
        int lo = km < kl ? km : kl, hi = km < kl ? kl : km;
        int k = N < lo ? lo : (N > hi ? hi : N);   // median of {N, km, kl}
        d.scan->sum_real = tot;
        d.scan->n_valid = N;
        d.scan->k_ret = k;
        d.scan->dda_steps = 0ull;
    }
}

}  // namespace relo
