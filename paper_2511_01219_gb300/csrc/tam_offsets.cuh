// TAM's inputs that the top-K launch prepares (select.cu): each request's
// work order (survivors grouped by band phase, in chunks), built by its
// ranking CTA once the survivors are known, and the endpoint offsets of its
// plan (Eq. 13's endpoint cells, as offsets into the banded field), computed
// by the other CTAs of the launch beside the ranking ones.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

// Every request's endpoint offsets, once per batch: for band phase ph,
// orientation q (m = q n_enum) and valid beam i, the field_index offset of the
// endpoint cell round-half-up(R_i * D_{(b_i + m) mod N_s} / 2^46) per axis from
// a cell of band phase ph (linear in the x offset, and in the y offset through
// the bands crossed), laid out [ph][q][lane][slot] with the TAM kernel's
// per-lane stride, so one block's offsets for one phase are one contiguous
// span.  One CTA writes all eight phases of orientation q.
__device__ __forceinline__ void tam_offsets_one(const ReqDesc &d, int q) {
    const int N = d.scan->n_valid;
    const int m = q * d.n_enum;
    const long long Wp8 = 8ll * d.Wp;
    const int kS = d.tam_stride;
    const size_t phase_step = (size_t)d.n_orient * 32 * kS;
    int32_t *oq = d.tam_offs + (size_t)q * 32 * kS;
    // k walks the orientation's table in memory order (lane-major), so every store is coalesced
    for (int k = threadIdx.x; k < 32 * kS; k += blockDim.x) {
        const int i = (k % kS) * 32 + k / kS;   // the beam in slot k % kS of lane k / kS
        if (i >= N) continue;
        const int2 bR = d.vbR[i];
        int j = bR.x + m;
        if (j >= d.ns) j -= d.ns;
        const int2 dir = d.D[j];
        const int ox = (int)(((long long)bR.y * dir.x + (1ll << 45)) >> 46);
        const int oy = (int)(((long long)bR.y * dir.y + (1ll << 45)) >> 46);
        // |ox|, |oy| < P keeps every endpoint inside the field's border
#pragma unroll
        for (int ph = 0; ph < 8; ++ph) {
            const int v = ph + oy;
            oq[ph * phase_step + k] = (int)(8ll * ox + Wp8 * (v >> 3)) + (v & 7);
        }
    }
}

// TAM's work order of request d, by one CTA once its survivors are written:
// within each batch (with early termination; without it TAM scores every
// batch in one launch, so all K positions form one group), the survivor
// positions grouped by the band phase (y + P) % 8 of their cell (the order
// inside a group is immaterial: every position's scores are its own), then
// cut into chunks of at most tam_chunk positions of one phase, so that a TAM
// task uses one phase's endpoint offsets for all its survivors.
__device__ __forceinline__ void tam_chunks_one(const ReqDesc &d) {
    __shared__ int s_cnt[8], s_next[8];
    __shared__ int s_chunks;
    if (threadIdx.x == 0) {
        s_chunks = 0;
        d.chunk_cnt[0] = 0;
    }
    const int groups = d.early_stop ? d.n_batches : 1;
    for (int b = 0; b < groups; ++b) {
        const int lo = b * d.B, hi = d.early_stop ? min(d.K, lo + d.B) : d.K;
        if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&s_cnt[(d.hyps[d.survivors[i]].y + d.P) & 7], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = lo, nc = s_chunks;
            for (int p = 0; p < 8; ++p) {
                s_next[p] = run;
                for (int f = run; f < run + s_cnt[p]; f += d.tam_chunk)
                    d.tam_chunks[nc++] = make_int4(p, f, min(run + s_cnt[p], f + d.tam_chunk), 0);
                run += s_cnt[p];
            }
            s_chunks = nc;
            if (d.early_stop) d.chunk_cnt[b + 1] = nc;
            else
                for (int j = 1; j <= d.n_batches; ++j) d.chunk_cnt[j] = nc;
        }
        __syncthreads();
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
            d.surv_perm[atomicAdd(&s_next[(d.hyps[d.survivors[i]].y + d.P) & 7], 1)] = i;
        __syncthreads();
    }
}

}  // namespace relo
