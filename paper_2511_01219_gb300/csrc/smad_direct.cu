// The ablation arms of Table II: SMAD by direct window sums (without prefix
// sums), and no coarse ranking at all (without SMAD ordering).
//
// SMAD by direct window sums.
// The numerator |sum_real - W_m| and its minimum over Theta (Eq. 18-20) are
// the prefix-sum form's, with W_m summed position by position over the FoV
// intervals for every m instead of read from the cyclic prefix sums of Eq.
// 17: O(|Theta| sum_k |I_k|) additions per hypothesis instead of O(N_s +
// |Theta| n_iv).  The integers are the same, so the keys, numerators and
// minimising m are identical to the prefix-sum kernel's.  One warp per
// hypothesis from the batch's hypothesis counter; the hypothesis's synthesized
// row sits in the warp's slice of shared memory, and for each m the lanes take
// consecutive positions (no bank conflicts) and a warp sum gives W_m.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/relo.h"
#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDirectWarps = 8;   // warps per CTA

__global__ void __launch_bounds__(kDirectWarps * 32) k_smad_direct(const ReqDesc *__restrict__ reqs, int R,
                                                                   int total_hyp, BatchState *bs, int warp_words) {
    extern __shared__ __align__(16) uint32_t s_rows[];
    __shared__ int s_base[kMaxBatchRequests + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].hyp_base;
    if (threadIdx.x == 0) s_base[R] = total_hyp;
    __syncthreads();
    uint32_t *srow = s_rows + (size_t)warp * warp_words;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&bs->ray_work, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= total_hyp) break;
        int lo = 0, hi = R - 1;   // last request whose base <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_base[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const ReqDesc &d = reqs[lo];
        const int h = g - s_base[lo], ns = d.ns;
        const uint32_t *__restrict__ row = d.scan_table + (size_t)h * ns;
        for (int j = lane; j < ns; j += 32) srow[j] = __ldg(row + j);
        __syncwarp();
        const long long sum_real = d.scan->sum_real;
        unsigned long long best = ~0ull;
        for (int q = 0; q < d.n_m; ++q) {
            const int m = q * d.n_enum;
            unsigned long long w = 0;
            for (int k = 0; k < d.n_iv; ++k) {
                const int2 iv = d.iv[k];   // positions [iv.x, iv.x + iv.y), shifted by m, cyclic
                for (int t = lane; t < iv.y; t += 32) {
                    int j = iv.x + m + t;   // < 3 N_s
                    if (j >= ns) j -= ns;
                    if (j >= ns) j -= ns;
                    w += srow[j];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            long long dnum = sum_real - (long long)w;
            if (dnum < 0) dnum = -dnum;
            const unsigned long long key = ((unsigned long long)dnum << 20) | (unsigned)q;
            best = key < best ? key : best;
        }
        if (lane == 0) {
            const unsigned long long num = best >> 20;
            const int q = (int)(best & 0xfffffu);
            d.keys[h] = (num << kHypBits) | (unsigned long long)h;
            d.smad_num[h] = (long long)num;
            d.smad_m[h] = q * d.n_enum;
        }
        __syncwarp();   // the row reads are done before the next hypothesis rewrites it
    }
}

// No coarse ranking: numerator 0 and m = 0 for every hypothesis, so the
// top-K (ordered by numerator, then index) keeps the hypotheses in the order
// they were set.  One thread per hypothesis slot of the batch.
__global__ void __launch_bounds__(256) k_rank_by_index(const ReqDesc *__restrict__ reqs, int R, int total_hyp) {
    __shared__ int s_base[kMaxBatchRequests + 1];
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].hyp_base;
    if (threadIdx.x == 0) s_base[R] = total_hyp;
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_hyp; g += gridDim.x * blockDim.x) {
        int lo = 0, hi = R - 1;   // last request whose base <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_base[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const ReqDesc &d = reqs[lo];
        const int h = g - s_base[lo];
        d.keys[h] = (unsigned long long)h;   // numerator 0 << kHypBits | h
        d.smad_num[h] = 0;
        d.smad_m[h] = 0;
    }
}

}  // namespace

cudaError_t launch_rank_by_index(const ReqDesc *reqs, int R, int total_hyp, int n_sm, cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests || n_sm < 1) return cudaErrorInvalidValue;
    long long grid = ((long long)total_hyp + 255) / 256;
    if (grid > 4ll * n_sm) grid = 4ll * n_sm;
    if (grid < 1) grid = 1;
    k_rank_by_index<<<(int)grid, 256, 0, s>>>(reqs, R, total_hyp);
    return cudaGetLastError();
}

cudaError_t launch_smad_direct(const ReqDesc *reqs, int R, int total_hyp, int max_ns_pad, BatchState *bs, int n_sm,
                               cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests || max_ns_pad < 1) return cudaErrorInvalidValue;
    const int warp_words = (max_ns_pad + 3) & ~3;   // 16-byte aligned slices
    const size_t smem = (size_t)kDirectWarps * warp_words * 4;
    if (smem > (size_t)200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_smad_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_smad_direct, kDirectWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)n_sm * occ;
    const long long need = ((long long)total_hyp + kDirectWarps - 1) / kDirectWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_smad_direct<<<(int)grid, kDirectWarps * 32, smem, s>>>(reqs, R, total_hyp, bs, warp_words);
    return cudaGetLastError();
}

}  // namespace relo
