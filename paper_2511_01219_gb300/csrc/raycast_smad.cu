// Ray-cast panoramic synthesized scans (Eq. 13) fused with SMAD (Eq. 16-20).
//
// One warp per hypothesis.  The warp casts the N_s panoramic rays 32 at a
// time (lane = ray within a chunk, so neighbouring lanes trace neighbouring
// directions of similar length), scans each chunk of ranges with warp
// shuffles into per-chunk exclusive prefixes, and keeps a running 64-bit
// chunk prefix: together they give the cyclic prefix sum S of Eq. 17 at any
// index.  The lanes then take the orientations m of Eq. 15 and evaluate each
// window sum of Eq. 18 with two lookups per FoV interval, form the integer
// SMAD numerator |sum R_real - W_m| of Eq. 19 (the shared denominator of the
// two means cancels from every comparison), and reduce the minimum over m
// (Eq. 20; ties keep the smaller m).
//
// Ray traversal.  From the hypothesis cell centre along the Q30 direction D,
// cells are entered in the order of the ray's grid-line crossings: with k x-
// and l y-crossings so far, x is stepped when (2k+1)|Dy| <= (2l+1)|Dx| (a
// corner tie steps x).  The kernel tracks the difference e = (2l+1)|Dx| -
// (2k+1)|Dy| incrementally (e -= 2|Dy| after an x step, e += 2|Dx| after a y
// step); it always lies in [-2^31, 2^31), so a 32-bit integer holds it
// exactly.  The ray stops on leaving the map, on entering a cell whose centre
// lies beyond the maximum range, or on entering an occupied cell; the range of
// a hit is floor(sqrt(|d|^2 * 2^32)) (cells, Q16), else 0 (the placeholder of
// the invalid beam).  Occupancy comes from the 8x8-tile bitmap; the current
// tile's 64-bit word stays in a register until the ray leaves the tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;

__device__ __forceinline__ uint32_t isqrt_q16(int c2) {
    // floor(sqrt(c2 * 2^32)): float estimate, one Newton correction, exact fix-up
    const unsigned long long N = (unsigned long long)(unsigned)c2 << 32;
    unsigned long long r = (unsigned long long)(sqrtf((float)c2) * 65536.0f);
    long long err = (long long)(N - r * r);
    r = (unsigned long long)((long long)r + (long long)((float)err / (2.0f * (float)r + 1.0f)));
    while (r * r > N) --r;
    while ((r + 1) * (r + 1) <= N) ++r;
    return (uint32_t)r;
}

// returns the Q16 range (0 = no hit); *hit receives cy*W+cx or -1, *steps the cells entered
__device__ __forceinline__ uint32_t cast_ray(const uint64_t *__restrict__ bits, int W, int H, int TW, int lim, int hx,
                                             int hy, int2 d, int *hit, int *steps) {
    const int ax = d.x < 0 ? -d.x : d.x, ay = d.y < 0 ? -d.y : d.y;
    const int sx = d.x > 0 ? 1 : -1, sy = d.y > 0 ? 1 : -1;
    const uint32_t two_ax = 2u * (uint32_t)ax, two_ay = 2u * (uint32_t)ay;
    int e = ax - ay;
    int cx = hx, cy = hy, adx = 0, ady = 0, c2 = 0;
    int tile = -1;
    unsigned long long word = 0;
    for (;;) {
        if (e >= 0) {
            cx += sx;
            e = (int)((uint32_t)e - two_ay);
            c2 += 2 * adx + 1;
            ++adx;
        } else {
            cy += sy;
            e = (int)((uint32_t)e + two_ax);
            c2 += 2 * ady + 1;
            ++ady;
        }
        if ((unsigned)cx >= (unsigned)W || (unsigned)cy >= (unsigned)H || c2 > lim) {
            *hit = -1;
            *steps = adx + ady;
            return 0u;
        }
        const int t = (cy >> 3) * TW + (cx >> 3);
        if (t != tile) {
            tile = t;
            word = __ldg(bits + t);
        }
        if ((word >> (((cy & 7) << 3) | (cx & 7))) & 1ull) {
            *hit = cy * W + cx;
            *steps = adx + ady;
            return isqrt_q16(c2);
        }
    }
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(kFull, v, o);
        v = t < v ? t : v;
    }
    return v;
}

__host__ __device__ __forceinline__ size_t warp_smem_bytes(int ns_pad) {
    size_t inner = ((size_t)(ns_pad + 32) * 4 + 7) & ~(size_t)7;
    return inner + (size_t)(ns_pad / 32 + 1) * 8;
}

__global__ void __launch_bounds__(kWarps * 32) k_raycast_smad(RayArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t per_warp = warp_smem_bytes(a.ns_pad);
    const size_t inner_bytes = ((size_t)(a.ns_pad + 32) * 4 + 7) & ~(size_t)7;
    uint32_t *inner = reinterpret_cast<uint32_t *>(smem + warp * per_warp);
    long long *chunkP = reinterpret_cast<long long *>(smem + warp * per_warp + inner_bytes);
    const int nch = a.ns_pad >> 5;
    inner[a.ns_pad + lane] = 0u;   // P(t) for t in [ns_pad, ns_pad + 32) adds nothing
    const long long sum_real = a.scan->sum_real;
    unsigned long long my_steps = 0;

    for (int h = blockIdx.x * kWarps + warp; h < a.n_hyp; h += gridDim.x * kWarps) {
        const int2 hc = a.hyps[h];
        long long carry = 0;
        if (lane == 0) chunkP[0] = 0;
        for (int c = 0; c < nch; ++c) {
            const int j = (c << 5) + lane;
            uint32_t r = 0u;
            int hit, steps = 0;
            if (j < a.ns) r = cast_ray(a.bits, a.W, a.H, a.TW, a.lim, hc.x, hc.y, a.D[j], &hit, &steps);
            my_steps += (unsigned)steps;
            uint32_t s = r;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += t;
            }
            inner[j] = s - r;
            carry += (long long)__shfl_sync(kFull, s, 31);
            if (lane == 0) chunkP[c + 1] = carry;
        }
        __syncwarp();
        unsigned long long best = ~0ull;
        for (int q = lane; q < a.n_m; q += 32) {
            const int m = q * a.n_enum;
            long long Wm = 0;
            for (int k = 0; k < a.n_iv; ++k) {
                const int2 iv = a.iv[k];
                int s0 = iv.x + m;
                if (s0 >= a.ns) s0 -= a.ns;
                const int e = s0 + iv.y;
                const long long p0 = chunkP[s0 >> 5] + inner[s0];
                if (e <= a.ns) {
                    Wm += chunkP[e >> 5] + inner[e] - p0;
                } else {
                    const int e2 = e - a.ns;
                    Wm += (chunkP[a.ns >> 5] + inner[a.ns] - p0) + (chunkP[e2 >> 5] + inner[e2]);
                }
            }
            long long dnum = sum_real - Wm;
            if (dnum < 0) dnum = -dnum;
            const unsigned long long key = ((unsigned long long)dnum << 20) | (unsigned)q;
            best = key < best ? key : best;
        }
        best = warp_min_u64(best);
        if (lane == 0) {
            const unsigned long long num = best >> 20;
            const int q = (int)(best & 0xfffffu);
            a.keys[h] = (num << kHypBits) | (unsigned long long)h;
            a.smad_num[h] = (long long)num;
            a.smad_m[h] = q * a.n_enum;
        }
        __syncwarp();
    }
    if (a.dda_steps) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(kFull, my_steps, o);
        if (lane == 0 && my_steps) atomicAdd(a.dda_steps, my_steps);
    }
}

__global__ void __launch_bounds__(256) k_synth(RayArgs a, uint32_t *__restrict__ ranges, int32_t *__restrict__ hits) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= a.n_hyp) return;
    const int2 hc = a.hyps[warp];
    for (int j = lane; j < a.ns; j += 32) {
        int hit, steps;
        uint32_t r = cast_ray(a.bits, a.W, a.H, a.TW, a.lim, hc.x, hc.y, a.D[j], &hit, &steps);
        ranges[(size_t)warp * a.ns + j] = r;
        if (hits) hits[(size_t)warp * a.ns + j] = hit;
    }
}

}  // namespace

cudaError_t launch_raycast_smad(const RayArgs &a, int n_sm, cudaStream_t s) {
    size_t smem = (size_t)kWarps * warp_smem_bytes(a.ns_pad);
    cudaError_t e = cudaFuncSetAttribute(k_raycast_smad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_raycast_smad, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int want = (a.n_hyp + kWarps - 1) / kWarps;
    int grid = n_sm * occ;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    k_raycast_smad<<<grid, kWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_synth(const RayArgs &a, uint32_t *ranges, int32_t *hit, cudaStream_t s) {
    if (a.n_hyp <= 0) return cudaSuccess;
    int blocks = (a.n_hyp * 32 + 255) / 256;
    k_synth<<<blocks, 256, 0, s>>>(a, ranges, hit);
    return cudaGetLastError();
}

}  // namespace relo
