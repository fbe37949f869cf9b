// TAM scoring (Eq. 22-31), and the stand-alone launch of the scan
// preparation (scan_prep.cuh) for batches that cast no rays.
//
// k_tam: one warp per (survivor, orientation m).  For each valid beam i the
// endpoint cell is hypothesis + round-half-up(R_i * D_{(b_i + m) mod N_s} /
// 2^46); its clamped squared distance b = min(d2, C) is read from the padded
// field, whose border holds C (off-map endpoints take d = d_max), so the read
// needs no bounds test.  The field is stored in bands of 8 rows (field_index):
// a cache line holds an 8 x 8 block of cells, so the endpoints of
// neighbouring beams share lines whichever way the contour runs, and an
// endpoint's offset from its hypothesis depends on the hypothesis only
// through its band phase (y + P) % 8.  The likelihood l
// (Eq. 23) falls strictly as b grows, so the descending sort of Eq. 24 is the
// ascending order of b: the warp finds the k-th smallest b by bisection over
// [0, C] with register-resident values, and the top-k sum of l is
// sum_{b <= b_k} l(b) - (#{b <= b_k} - k) l(b_k), the count being the one the
// search ends on.  The counts run on fp16 patterns 0x6400 + slot(b), two
// beams per instruction, while slot(C + 1) <= 6143 (C <= 5956), and on 32-bit
// slots above.  A shared-memory table holds
// l(b) and sqrt(C) - sqrt(b) for every b in [0, C] (at slot lut_slot(b), and
// the selection runs on slots too, see below); with those and the exact
// integer sum of b, the warp evaluates Eq. 27-30 and, after the block's
// orientations, one lane per orientation takes the exponential and Eq. 31:
//     wp = exp(Lbar),  d_max - dbar = res * sum(sqrt(C) - sqrt(b)) / N,
//     s_d = min(d_max - dbar, d_max - d_min) / (d_max - d_min),
//     var = res^2 * sum(b) / N - dbar^2,  c = exp(-var / 2),
//     T = cbrt(wp * s_d * c).
// Summing sqrt(C) - sqrt(b) (never negative) instead of sqrt(b) keeps s_d
// accurate when dbar is close to d_max.  Each score is written out and folded
// into a per-survivor 64-bit key (the score's order-preserving code, then
// smaller m) with atomicMax: that is the orientation argmax of Eq. 22.
//
// The scoring metric can be switched to those the paper compares TAM with:
// TAM_mean = (wp + s_d + c) / 3 (Eq. 34) from the same components, and the
// likelihood-field sum wp_LF = sum of l over every valid beam (Eq. 32) or its
// normalised form (exp(wp_LF / N) s_d)^(1/2) (Eq. 33), which keep every beam
// (k = N: no retention and no search).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "relo_internal.h"
#include "scan_prep.cuh"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTamWarps = 8;
// Selection values as fp16 bit patterns 0x6400 + s, s the table slot of the
// value (lut_slot, below).  Positive fp16 numbers order like their bit
// patterns, so this is an increasing map of s onto fp16 numbers >= 1024,
// consecutive ones at least 1 apart; it stays finite while 0x6400 + s <=
// 0x7bff, i.e. s <= 6143 (kHalfMaxB).
constexpr uint32_t kHalfBias = 0x6400u;
constexpr int kHalfMaxB = 0x7bff - 0x6400;

// The table slot of value b: b + floor(b / 32), one unused slot after every 32.
// An 8-byte entry's bank pair is its slot mod 16, and the clamped d2 of real
// endpoints crowd onto few residues mod 16 (sums of two squares take 9 of the
// 16; near a wall parallel to an axis they are squares, 0, 1, 4 or 9 mod 16,
// and C itself is often a square), so value-indexed lookups serialise a warp
// on those banks; the gap moves each block of 32 values by one more bank pair.
// The map is strictly increasing, so the kernel holds slots instead of values:
// the k-th smallest slot is the slot of the k-th smallest value, ties stay
// ties, and "b <= b_k" is "slot <= slot(b_k)".  The exact sum of b is taken
// from the values before the map.  The table of C + 2 values spans
// lut_slot(C + 1) + 1 slots.
__host__ __device__ constexpr uint32_t lut_slot(uint32_t b) { return b + (b >> 5); }

// The smallest b in [0, C] with count_le(b) >= k, given count_le(C) = n_C >= k
// (every valid beam is <= C); cnt receives count_le(b).  hint < 0: bisection
// over [0, C].  Otherwise the search starts at hint: two counts confirm an
// unchanged answer; else it gallops away from hint in doubling steps to a
// bracket [lo, hi] with count_le(lo - 1) < k <= count_le(hi) and bisects it.
// The count at hi is carried along, so the answer's count costs nothing.
template <typename F>
__device__ __forceinline__ int kth_smallest(F &&count_le, int k, int C, int n_C, int hint, int &cnt) {
    int lo = 0, hi = C, c_hi = n_C;
    if (hint >= 0) {
        const int ch = count_le(hint);
        if (ch >= k) {
            const int cm = hint == 0 ? 0 : count_le(hint - 1);
            if (cm < k) {
                cnt = ch;
                return hint;
            }
            hi = hint - 1;
            c_hi = cm;
            for (int step = 1;; step <<= 1) {
                const int p = hi - step;
                if (p < 0) {
                    lo = 0;
                    break;
                }
                const int cp = count_le(p);
                if (cp < k) {
                    lo = p + 1;
                    break;
                }
                hi = p;
                c_hi = cp;
            }
        } else {
            lo = hint + 1;   // count_le(lo - 1) < k
            for (int step = 1;; step <<= 1) {
                const int p = lo + step - 1;
                if (p >= C) break;   // hi = C
                const int cp = count_le(p);
                if (cp >= k) {
                    hi = p;
                    c_hi = cp;
                    break;
                }
                lo = p + 1;
            }
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = count_le(mid);
        if (cm >= k) {
            hi = mid;
            c_hi = cm;
        } else {
            lo = mid + 1;
        }
    }
    cnt = c_hi;
    return lo;
}

// Per-lane stride of the endpoint offsets in shared memory: slot s of lane l
// (beam 32 s + l) sits at l * stride + s, so a lane reads four offsets with one
// 16-byte load; stride / 4 odd keeps the eight lanes of each load phase on
// distinct banks.
__host__ __device__ constexpr int tam_offs_stride(int vpl) {
    return ((vpl + 3) & ~3) + ((((vpl + 3) & ~3) / 4) % 2 == 0 ? 4 : 0);
}

// CTA (request, 0) does the scan preparation of scan_prep.cuh and all CTAs
// (request, y) share the fill of its TAM scores with NaN; this launch serves
// batches whose requests all read resident synthesized scans (otherwise the
// ray-cast launch does the same work first).
__global__ void __launch_bounds__(1024) k_scan_prep(const ReqDesc *__restrict__ reqs) {
    const ReqDesc &d = reqs[blockIdx.x];
    scan_prep_fill(d, blockIdx.y, gridDim.y);
    if (blockIdx.y == 0) scan_prep_request(d);
}


// Work is split into tasks (request, chunk of survivors of one band phase,
// block of kTamQ consecutive orientations); the top-K launch builds the chunks
// on the device (tam_offsets.cuh).  A CTA copies the block's endpoint offsets for
// its chunk's phase from the request's table (tam_offsets.cuh: one linear
// offset per phase, orientation and valid beam, computed once per request)
// into shared memory; each warp then scores its survivors of the chunk over
// the block's orientations, every gather one add to the survivor's base.
//
// Selection.  The k-th smallest clamped d2 of a survivor rarely changes from
// one orientation to the next (neighbouring orientations see nearly the same
// contour), so each orientation after the block's first starts from the
// previous answer h: two counts confirm it (#{b <= h} >= k and #{b <= h-1} <
// k); otherwise the search gallops away from h in doubling steps and bisects
// the bracket.  Every step is a warp-wide count, and the result is the same
// smallest b with #{b' <= b} >= k as a bisection over [0, C].  The likelihood
// table is reloaded only when a CTA moves to another request's task.
constexpr int kTamQ = 4;

// resident CTAs per SM the register budget is sized for (measured per values-per-lane class)
__host__ __device__ constexpr int tam_min_blocks(int vpl, bool h2) { return h2 ? (vpl <= 24 ? 6 : vpl <= 40 ? 5 : 4) : (vpl <= 24 ? 3 : 2); }

template <int VPL, bool H2>
__global__ void __launch_bounds__(kTamWarps * 32, tam_min_blocks(VPL, H2)) k_tam(const ReqDesc *__restrict__ reqs,
                                                                             int R, const TamSeg *__restrict__ segs,
                                                                             int total_tasks) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_base[kMaxBatchRequests + 1];
    __shared__ int s_skip, s_lut_r;
    __shared__ float s_ep[5];   // per-task constants of the epilogue
    __shared__ int s_fine;      // the task's scoring metric (read where needed, not held in a register)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // each request's tasks: its chunks in the launch's batches x its orientation blocks (counted on the device)
    if (threadIdx.x == 0) {
        int base = 0;
        for (int r = 0; r < R; ++r) {
            s_base[r] = base;
            const TamSeg sg = segs[r];
            if (sg.batch_hi > sg.batch_lo) {
                const ReqDesc &d = reqs[r];
                base += (d.chunk_cnt[sg.batch_hi] - d.chunk_cnt[sg.batch_lo]) * ((d.n_orient + kTamQ - 1) / kTamQ);
            }
        }
        s_base[R] = base;
        s_lut_r = -1;
    }
    __syncthreads();
    total_tasks = s_base[R];
    float2 *lut = reinterpret_cast<float2 *>(smem);
    for (int task = blockIdx.x; task < total_tasks; task += gridDim.x) {
        int lo = 0, hi = R - 1;   // the request whose tasks hold this one: last r with s_base[r] <= task
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_base[mid] <= task) lo = mid;
            else hi = mid - 1;
        }
        const int r = lo;
        const ReqDesc &d = reqs[r];
        const TamSeg sg = segs[r];
        const int N = d.scan->n_valid;
        // the likelihood-field metrics (Eq. 32-33) keep every beam: no retention, no k-th value to find
        const int k = d.fine < kFineBaseline ? d.scan->k_ret : N;
        __syncthreads();   // the previous task's reads of offs / lut are done
        if (threadIdx.x == 0) {
            s_skip = d.state->done || N <= 0;
            s_fine = d.fine;
            s_ep[0] = 1.0f / (float)k;                // 1 / k
            s_ep[1] = d.res / (float)N;               // res / N
            s_ep[2] = d.d_max - d.d_min;              // span of Eq. 29
            s_ep[3] = 1.0f / (d.d_max - d.d_min);
            s_ep[4] = d.res2 / (float)N;              // res^2 / N
        }
        if (s_lut_r != r) {
            for (int i = threadIdx.x; i <= d.C + 1; i += blockDim.x) lut[lut_slot(i)] = d.lut[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_lut_r = r;
        if (s_skip) continue;
        constexpr int kS = tam_offs_stride(VPL);
        int *offs = reinterpret_cast<int *>(smem + (((size_t)(lut_slot(d.C + 1) + 1) * sizeof(float2) + 15) & ~(size_t)15));
        const int local = task - s_base[r];
        const int nblk = (d.n_orient + kTamQ - 1) / kTamQ;
        const int qb = local % nblk;
        const int4 ck = d.tam_chunks[d.chunk_cnt[sg.batch_lo] + local / nblk];   // (phase, first, end)
        const int ph = ck.x;
        const int q0 = qb * kTamQ;
        const int nq = min(kTamQ, d.n_orient - q0);
        const int C = d.C;
        const uint32_t none = (uint32_t)C + 1u;   // table entry with zero weight
        const float d_max = d.d_max;
        {
            // the block's offsets for phase ph: nq x 32 x kS contiguous ints of the request's table
            const int4 *src = reinterpret_cast<const int4 *>(d.tam_offs + ((size_t)ph * d.n_orient + q0) * 32 * kS);
            int4 *dst = reinterpret_cast<int4 *>(offs);
            const int n4 = nq * 32 * kS / 4;
            for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
        }
        __syncthreads();
        for (int js = ck.y + warp; js < ck.z; js += kTamWarps) {
            const int s = d.surv_perm[js];   // survivor position: its scores go to row s
            const int2 hc = d.hyps[d.survivors[s]];
            // the cell's column at the top of its band; the offsets of its phase lead to each endpoint
            const uint16_t *fh = d.field + 8 * ((size_t)((hc.y + d.P) >> 3) * d.Wp + (hc.x + d.P));
            int hint = -1;   // the previous orientation's k-th smallest value
            float e_arg = 0.0f, e_sd = 0.0f;   // lane qi: orientation qi's exponent and s_d
            for (int qi = 0; qi < nq; ++qi) {
                const int *ol = offs + (qi * 32 + lane) * kS;   // this lane's offsets, slot s = beam 32 s + lane
                int sumb = 0;
                float sgs = 0.0f, sl = 0.0f;
                int bk;
                int cle;   // #{b <= bk} over the valid beams
                if constexpr (H2) {
                    uint32_t hv[VPL / 2];   // fp16 patterns 0x6400 + b of slots 2t (low half) and 2t + 1
#pragma unroll
                    for (int u = 0; u < (VPL + 3) / 4; ++u) {
                        const int4 o4 = *reinterpret_cast<const int4 *>(ol + 4 * u);
                        const int oo[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                        for (int e = 0; e < 4; e += 2) {
                            const int t = 2 * u + e / 2;   // pair of slots 2t, 2t + 1
                            if (t < VPL / 2) {
                                const int i0 = (t << 6) + lane, i1 = i0 + 32;
                                uint32_t b0 = none, b1 = none;
                                if (i0 < N) {
                                    b0 = (uint32_t)__ldg(fh + oo[e]);
                                    sumb += (int)b0;
                                }
                                if (i1 < N) {
                                    b1 = (uint32_t)__ldg(fh + oo[e + 1]);
                                    sumb += (int)b1;
                                }
                                // both slots at once: b + floor(b / 32) per half, plus the bias
                                // (slot(C + 1) <= kHalfMaxB: no carry between the halves)
                                const uint32_t v2 = b0 | (b1 << 16);
                                hv[t] = v2 + ((v2 >> 5) & 0x07ff07ffu) + (kHalfBias | (kHalfBias << 16));
                            }
                        }
                    }
                    // #{b > x} on a lane: f(b) - f(x) saturated to [0, 1] is 1 exactly when b > x (f maps
                    // b to the fp16 number of bits 0x6400 + slot(b); the exact difference is then >= 1,
                    // else <= 0, and rounding keeps both); then #{b <= x} over the warp is the 32 VPL
                    // slots less those (no-beam slots are > C)
                    auto count_le = [&](int x) -> int {
                        const unsigned short fxb = (unsigned short)(kHalfBias + lut_slot((uint32_t)x));
                        const __half2 fx = __halves2half2(__ushort_as_half(fxb), __ushort_as_half(fxb));
                        // two chains (half the add latency); the low half starts at 1024, so the
                        // total 1024 + c (c <= 64) has the fp16 bits 0x6400 + c
                        __half2 acc0 = __halves2half2(__ushort_as_half((unsigned short)kHalfBias), __float2half(0.0f));
                        __half2 acc1 = __float2half2_rn(0.0f);
#pragma unroll
                        for (int t = 0; t < VPL / 2; t += 2) {
                            acc0 = __hadd2(acc0, __hsub2_sat(*reinterpret_cast<const __half2 *>(&hv[t]), fx));
                            if (t + 1 < VPL / 2)
                                acc1 = __hadd2(acc1, __hsub2_sat(*reinterpret_cast<const __half2 *>(&hv[t + 1]), fx));
                        }
                        const __half2 sum = __hadd2(acc0, acc1);
                        const __half2 tot = __hadd2(sum, __lowhigh2highlow(sum));
                        const int gt = __reduce_add_sync(kFull, (int)(__half_as_ushort(__low2half(tot)) & 0x3ffu));
                        return 32 * VPL - gt;
                    };
                    if (s_fine < kFineBaseline) {
                        bk = kth_smallest(count_le, k, C, N, hint, cle);
                    } else {
                        bk = C;   // every valid beam
                        cle = N;
                    }
                    const uint32_t bkb = kHalfBias + lut_slot((uint32_t)bk);
#pragma unroll
                    for (int t = 0; t < VPL / 2; ++t) {
                        const uint32_t p0 = hv[t] & 0xffffu, p1 = hv[t] >> 16;
                        const float2 g0 = lut[p0 - kHalfBias], g1 = lut[p1 - kHalfBias];   // slot(C+1) (no beam) adds zero
                        sgs += g0.y + g1.y;
                        if (p0 <= bkb) sl += g0.x;
                        if (p1 <= bkb) sl += g1.x;
                    }
                } else {
                    uint32_t v[VPL];   // slots of the values
#pragma unroll
                    for (int t = 0; t < VPL; ++t) {
                        const int i = (t << 5) + lane;
                        uint32_t bv = none;
                        if (i < N) {
                            bv = (uint32_t)__ldg(fh + ol[t]);
                            sumb += (int)bv;
                        }
                        v[t] = lut_slot(bv);
                    }
                    auto count_le = [&](int x) -> int {
                        int c = 0;
                        const uint32_t sx = lut_slot((uint32_t)x);
#pragma unroll
                        for (int t = 0; t < VPL; ++t) c += (v[t] <= sx) ? 1 : 0;
                        return __reduce_add_sync(kFull, c);
                    };
                    if (s_fine < kFineBaseline) {
                        bk = kth_smallest(count_le, k, C, N, hint, cle);
                    } else {
                        bk = C;
                        cle = N;
                    }
                    const uint32_t sk = lut_slot((uint32_t)bk);
#pragma unroll
                    for (int t = 0; t < VPL; ++t) {
                        const float2 lg = lut[v[t]];   // the slot of C+1 (no beam) adds zero
                        sgs += lg.y;
                        if (v[t] <= sk) sl += lg.x;
                    }
                }
                hint = bk;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sgs += __shfl_xor_sync(kFull, sgs, o);
                    sl += __shfl_xor_sync(kFull, sl, o);
                }
                sumb = __reduce_add_sync(kFull, sumb);
                {
                    // Eq. 27-30 from the warp totals every lane holds; the top-k sum of l is every
                    // b <= bk less the cle - k ties at bk beyond the k-th; lane qi keeps what its
                    // orientation's score still needs: for TAM the exponent of exp(Lbar) exp(-var / 2)
                    // and s_d
                    const float topsum = sl - (float)(cle - k) * lut[lut_slot(bk)].x;
                    const float lbar = topsum * s_ep[0];
                    const float dd = s_ep[1] * sgs;   // d_max - dbar
                    const float dbar = d_max - dd;
                    const float var = fmaxf(s_ep[4] * (float)sumb - dbar * dbar, 0.0f);
                    const float sd = fminf(dd, s_ep[2]) * s_ep[3];
                    const int fine = s_fine;
                    float a = lbar - 0.5f * var;
                    if (fine == kFineTamMean) a = expf(lbar) + expf(-0.5f * var);   // wp + c (Eq. 34)
                    else if (fine == kFineBaseline) a = lbar;                       // wp_LF / N (Eq. 33)
                    else if (fine == kFineLF) a = topsum;                           // wp_LF (Eq. 32)
                    if (lane == qi) {
                        e_arg = a;
                        e_sd = sd;
                    }
                }
            }
            if (lane < nq) {   // the score of orientation q0 + lane
                const int q = q0 + lane;
                const int fine = s_fine;
                float T = cbrtf(expf(e_arg) * e_sd);                                   // TAM, Eq. 31
                if (fine == kFineTamMean) T = (e_arg + e_sd) * (1.0f / 3.0f);         // Eq. 34
                else if (fine == kFineBaseline) T = sqrtf(expf(e_arg) * e_sd);        // Eq. 33
                else if (fine == kFineLF) T = e_arg;                                  // Eq. 32
                d.T[(size_t)s * d.n_orient + q] = T;
                const unsigned long long key = ((unsigned long long)score_code(T) << 32) |
                                               (unsigned long long)(0xffffffffu - (unsigned)q);
                atomicMax(d.best_key + s, key);
            }
        }
    }
}

template <int VPL, bool H2>
cudaError_t run_tam(const ReqDesc *reqs, int R, const TamSeg *segs, const TamPlan &tp, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_tam<VPL, H2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.smem);
    if (e != cudaSuccess) return e;
    k_tam<VPL, H2><<<tp.grid, kTamWarps * 32, tp.smem, s>>>(reqs, R, segs, tp.total_tasks);
    return cudaGetLastError();
}

template <int VPL, bool H2>
int tam_occupancy(size_t smem) {
    int occ = 0;
    if (cudaFuncSetAttribute(k_tam<VPL, H2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tam<VPL, H2>, kTamWarps * 32, smem) != cudaSuccess)
        return 0;
    return occ;
}

#define RELO_TAM_VPLS(X)                                                                                       \
    X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32) X(34) X(36) X(38) X(40) X(42) X(44) \
        X(46) X(48) X(50) X(52) X(54) X(56) X(58) X(60) X(62) X(64)

int vpl_bucket(int max_beams) {
    const int need = (max_beams + 31) / 32;
#define RELO_TAM_PICK(V) \
    if (need <= V) return V;
    RELO_TAM_VPLS(RELO_TAM_PICK)
#undef RELO_TAM_PICK
    return -1;
}

int occupancy_for(int vpl, bool h2, size_t smem) {
#define RELO_TAM_OCC(V) \
    if (vpl == V) return h2 ? tam_occupancy<V, true>(smem) : tam_occupancy<V, false>(smem);
    RELO_TAM_VPLS(RELO_TAM_OCC)
#undef RELO_TAM_OCC
    return 0;
}

}  // namespace

int tam_vpl_for(int max_beams) { return vpl_bucket(max_beams); }

cudaError_t launch_scan_prep(const ReqDesc *reqs, int R, cudaStream_t s) {
    k_scan_prep<<<dim3(R, 8), 1024, 0, s>>>(reqs);
    return cudaGetLastError();
}

// The launch for the batches [batch_lo[r], batch_hi[r]) of every request:
// its kernel class (values per lane and selection precision for the longest
// scan and the largest clamp), the shared memory (table and one block's
// endpoint offsets) and a grid of every resident CTA (or ctas_per_sm per SM
// when that is fewer); the tasks are counted by the kernel from the
// device-built chunk tables.
TamPlan plan_tam(const int *batch_lo, const int *batch_hi, int R, int max_beams, int max_C, int n_sm,
                 int ctas_per_sm, TamSeg *segs) {
    TamPlan tp{0, 0, vpl_bucket(max_beams), 0, (int)lut_slot(max_C + 1) <= kHalfMaxB};
    if (tp.vpl < 0) return tp;
    tp.smem = (((size_t)(lut_slot(max_C + 1) + 1) * sizeof(float2) + 15) & ~(size_t)15) +
              (size_t)kTamQ * 32 * tam_offs_stride(tp.vpl) * sizeof(int);
    const int occ = occupancy_for(tp.vpl, tp.h2, tp.smem);
    if (occ < 1) {
        tp.vpl = -1;
        return tp;
    }
    bool any = false;
    for (int r = 0; r < R; ++r) {
        segs[r] = TamSeg{batch_lo[r], batch_hi[r]};
        any = any || batch_hi[r] > batch_lo[r];
    }
    tp.total_tasks = any ? 1 : 0;
    tp.grid = n_sm * (ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ);
    return tp;
}

int tam_offs_stride_for(int vpl) { return tam_offs_stride(vpl); }

cudaError_t launch_tam(const ReqDesc *reqs, int R, const TamSeg *segs, const TamPlan &tp, cudaStream_t s) {
    if (tp.total_tasks <= 0) return cudaSuccess;
#define RELO_TAM_RUN(V) \
    if (tp.vpl == V) return tp.h2 ? run_tam<V, true>(reqs, R, segs, tp, s) : run_tam<V, false>(reqs, R, segs, tp, s);
    RELO_TAM_VPLS(RELO_TAM_RUN)
#undef RELO_TAM_RUN
    return cudaErrorInvalidValue;
}

}  // namespace relo
