// The TAM endpoint offsets of a request plan (Eq. 13's endpoint cells, as
// offsets into the banded field), computed by the blocks of the top-K launch
// that do not rank (select.cu), beside the ranking blocks.
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
// span.  CTA (q, request) writes all eight phases of orientation q.
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

}  // namespace relo
