// Traversability-constrained hypothesis sampling on the GPU (Algorithm 1,
// Sec. III-A, Remark 4).
//
// Algorithm 1 grows the tree one point at a time: every random point extends
// from its nearest node among all nodes so far.  Here a round's points go in
// sub-batches of kRrtSub.  For every point of a sub-batch at once,
// k_rrt_near and k_rrt_extend find the nearest node of the tree as the
// sub-batch began and the extension from it.  k_rrt_resolve (one warp) then
// takes the points in sample order: a point whose nearest node is one accepted
// earlier in the same sub-batch (strictly nearer than its tree node, so ties
// keep the lower index as in the serial search) is extended again from that
// node.  The tree is therefore the serial algorithm's for the same random
// points and the same float32 arithmetic.  A voxel of side rho is represented
// by its lowest-index node; a round's gain is the number of voxels it claimed,
// and sampling stops once a round gains at most eps_gain.  The node count
// lives on the device, so a round waits on the host once, for its gain.
//
// Per sample i of round r: p_rand from a counter-based hash (splitmix64 of
// seed ^ (r << 40 | i << 1 | k), k = 0, 1 for x, y), in [0, W res) x [0, H res);
// NearestNode by brute force (squared distance, ties to the lower index);
// AdaptiveExpandDist eta = eta_max when the clearance d at the nearest node is
// >= 2 r_robot, r_robot when d <= r_robot, linear between; ExtendPoint moves
// min(eta, |p_rand - p_nearest|) towards p_rand; the new point must lie in the
// map rectangle, and every point of the segment at spacing res / 2 (both ends
// included) must have clearance >= r_robot (clearance: a per-cell table in
// metres, 0 off the map).  Positions are float32 metres, and every operation
// is an explicitly rounded float32 one (no contraction), so a host program
// with the same steps gets the same tree.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/relo.h"
#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRrtSub = 256;            // points per sub-batch
constexpr int kSlots = kRrtSub / 32;    // points of a sub-batch per lane of the resolving warp
constexpr int kNearCtas = 304;          // node slices of the nearest-node search (2 CTAs per SM)
constexpr int kNearTile = 1024;         // nodes staged in shared memory at a time

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {   // Steele, Lea and Flood (2014)
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float unit_draw(uint64_t seed, int round, int i, int k) {
    const uint64_t c = seed ^ (((uint64_t)round << 40) | ((uint64_t)i << 1) | (uint64_t)k);
    return (float)((double)(splitmix64(c) >> 11) * (1.0 / 9007199254740992.0));
}

struct RrtArgs {
    const float *clr;   // [H*W] clearance, metres
    int W, H;
    float res, rho, eta_max, r_robot;
    float Wm, Hm;       // map extent, metres: float(W) * res, float(H) * res
    uint64_t seed;
};

// One sample of a sub-batch against the tree as the sub-batch began.
struct RrtCand {
    float rx, ry;   // p_rand
    float d2;       // squared distance to its nearest tree node
    float nx, ny;   // the extension from that node
    float c;        // clearance at (nx, ny)
    int ok;         // the extension is accepted
    int pad;
};

__device__ __forceinline__ float clearance_at(const RrtArgs &a, float x, float y) {
    const int cx = (int)floorf(__fdiv_rn(x, a.res)), cy = (int)floorf(__fdiv_rn(y, a.res));
    if (cx < 0 || cy < 0 || cx >= a.W || cy >= a.H) return 0.0f;
    return a.clr[(size_t)cy * a.W + cx];
}

__device__ __forceinline__ float dist2(float2 p, float rx, float ry) {
    const float ex = __fsub_rn(p.x, rx), ey = __fsub_rn(p.y, ry);
    return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
}

// ExtendPoint from node pn (clearance dn) towards (rx, ry), by the whole warp
// (all lanes pass the same arguments; each checks every 32nd segment point).
// *out receives the new point and *c_out the clearance there; returns whether
// the extension is accepted.
__device__ __forceinline__ int warp_extend(const RrtArgs &a, float2 pn, float dn, float rx, float ry, float2 *out,
                                           float *c_out) {
    const int lane = threadIdx.x & 31;
    float eta;
    if (dn >= 2.0f * a.r_robot) eta = a.eta_max;
    else if (dn <= a.r_robot) eta = a.r_robot;
    else eta = __fadd_rn(a.r_robot, __fdiv_rn(__fmul_rn(__fsub_rn(a.eta_max, a.r_robot), __fsub_rn(dn, a.r_robot)),
                                              a.r_robot));
    const float vx = __fsub_rn(rx, pn.x), vy = __fsub_rn(ry, pn.y);
    const float L = __fsqrt_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)));
    *out = pn;
    *c_out = dn;
    if (!(L > 0.0f)) return 0;
    const float step = fminf(eta, L);
    const float nx = __fadd_rn(pn.x, __fmul_rn(__fdiv_rn(vx, L), step));
    const float ny = __fadd_rn(pn.y, __fmul_rn(__fdiv_rn(vy, L), step));
    *out = make_float2(nx, ny);
    *c_out = 0.0f;
    if (!(nx >= 0.0f && ny >= 0.0f && nx < a.Wm && ny < a.Hm)) return 0;
    const int nseg = (int)ceilf(__fdiv_rn(step, 0.5f * a.res));
    const float sx = __fsub_rn(nx, pn.x), sy = __fsub_rn(ny, pn.y);
    int good = 1;
    for (int t = lane; t <= nseg; t += 32) {
        const float f = nseg ? __fdiv_rn((float)t, (float)nseg) : 0.0f;
        if (clearance_at(a, __fadd_rn(pn.x, __fmul_rn(sx, f)), __fadd_rn(pn.y, __fmul_rn(sy, f))) < a.r_robot)
            good = 0;
    }
    *c_out = clearance_at(a, nx, ny);
    return __all_sync(kFull, good);
}

// Nearest tree node of each point i0 + k of the sub-batch, slice by slice: CTA
// b scans nodes [b per, (b + 1) per) of the tree as the sub-batch began (per =
// ceil(*d_n / gridDim.x)), staged through shared memory, thread k for point k,
// and writes its (squared distance, index) to part[b][k] ((+inf, INT_MAX) for
// an empty slice).
__global__ void __launch_bounds__(kRrtSub) k_rrt_near(RrtArgs a, const float2 *__restrict__ nodes,
                                                      const int *__restrict__ d_n, int i0, int n_sub, int round,
                                                      int2 *__restrict__ part) {
    __shared__ float2 tile[kNearTile];
    const int n0 = *d_n, k = threadIdx.x;
    const int per = (n0 + gridDim.x - 1) / gridDim.x;
    const int lo = min(n0, blockIdx.x * per), hi = min(n0, lo + per);
    float rx = 0.0f, ry = 0.0f;
    if (k < n_sub) {
        rx = __fmul_rn(unit_draw(a.seed, round, i0 + k, 0), a.Wm);
        ry = __fmul_rn(unit_draw(a.seed, round, i0 + k, 1), a.Hm);
    }
    float best2 = INFINITY;
    int best = 0x7fffffff;
    for (int t0 = lo; t0 < hi; t0 += kNearTile) {
        const int tn = min(kNearTile, hi - t0);
        __syncthreads();
        for (int i = k; i < tn; i += blockDim.x) tile[i] = nodes[t0 + i];
        __syncthreads();
        for (int i = 0; i < tn; ++i) {
            const float d2 = dist2(tile[i], rx, ry);
            if (d2 < best2) {   // ascending index
                best2 = d2;
                best = t0 + i;
            }
        }
    }
    if (k < n_sub) part[blockIdx.x * kRrtSub + k] = make_int2(__float_as_int(best2), best);
}

// One warp per point i0 + k: the smallest (squared distance, index) over the
// n_part slices, and the extension from that node.
__global__ void __launch_bounds__(256) k_rrt_extend(RrtArgs a, const float2 *__restrict__ nodes,
                                                    const float *__restrict__ nclr, const int2 *__restrict__ part,
                                                    int n_part, int i0, int n_sub, int round,
                                                    RrtCand *__restrict__ cand) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= n_sub) return;   // the whole warp
    int best = 0x7fffffff;
    float best2 = INFINITY;
    for (int b = lane; b < n_part; b += 32) {
        const int2 v = part[b * kRrtSub + k];
        const float d2 = __int_as_float(v.x);
        if (d2 < best2 || (d2 == best2 && v.y < best)) {
            best2 = d2;
            best = v.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // the warp's smallest (d2, index); every lane ends with it
        const float od = __shfl_xor_sync(kFull, best2, o);
        const int oj = __shfl_xor_sync(kFull, best, o);
        if (od < best2 || (od == best2 && oj < best)) {
            best2 = od;
            best = oj;
        }
    }
    const float rx = __fmul_rn(unit_draw(a.seed, round, i0 + k, 0), a.Wm);
    const float ry = __fmul_rn(unit_draw(a.seed, round, i0 + k, 1), a.Hm);
    float2 nw;
    float cw;
    const int ok = warp_extend(a, nodes[best], nclr[best], rx, ry, &nw, &cw);
    if (lane == 0) cand[k] = RrtCand{rx, ry, best2, nw.x, nw.y, cw, ok, 0};
}

__device__ __forceinline__ int voxel_of(float2 p, float rho, int vw) {
    return (int)floorf(__fdiv_rn(p.y, rho)) * vw + (int)floorf(__fdiv_rn(p.x, rho));
}

// One warp: the sub-batch's points in sample order.  Accepted points join the
// tree as nodes *d_n, *d_n + 1, ... (at most node_cap in all); each claims its
// voxel if no lower node holds it, and the voxels claimed are added to *gain.
__global__ void __launch_bounds__(32) k_rrt_resolve(RrtArgs a, const RrtCand *__restrict__ cand, int n_sub,
                                                    float2 *__restrict__ nodes, float *__restrict__ nclr, int *d_n,
                                                    int node_cap, int vw, int *__restrict__ voxel,
                                                    int *__restrict__ rep, int *gain) {
    __shared__ RrtCand s_c[kRrtSub];
    __shared__ float2 acc[kRrtSub];   // the points accepted so far in this sub-batch
    __shared__ float accc[kRrtSub];   // and the clearance there
    const int lane = threadIdx.x;
    for (int i = lane; i < n_sub; i += 32) s_c[i] = cand[i];
    const int n0 = *d_n;
    __syncwarp();
    int m = 0;
    for (int k = 0; k < n_sub; ++k) {
        const RrtCand ck = s_c[k];
        float bd = INFINITY;
        int bj = 0x7fffffff;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int j = lane + 32 * s;
            if (j < m) {
                const float d2 = dist2(acc[j], ck.rx, ck.ry);
                if (d2 < bd) {
                    bd = d2;
                    bj = j;
                }
            }
        }
        // squared distances are >= +0 (or +inf), so their bit patterns order like the values
        const unsigned mn = __reduce_min_sync(kFull, __float_as_uint(bd));
        float2 nw = make_float2(ck.nx, ck.ny);
        float cw = ck.c;
        int ok = ck.ok;
        if (__uint_as_float(mn) < ck.d2) {   // a point accepted earlier in this sub-batch is nearer
            const int jj = (int)__reduce_min_sync(kFull, __float_as_uint(bd) == mn ? (unsigned)bj : 0xffffffffu);
            ok = warp_extend(a, acc[jj], accc[jj], ck.rx, ck.ry, &nw, &cw);
        }
        if (ok && n0 + m < node_cap) {
            if (lane == 0) {
                acc[m] = nw;
                accc[m] = cw;
            }
            ++m;
            __syncwarp();
        }
    }
    // the new nodes n0 .. n0 + m - 1; each takes its voxel unless a lower node holds it
    int was[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const int j = lane + 32 * s;
        was[s] = -1;
        if (j < m) {
            nodes[n0 + j] = acc[j];
            nclr[n0 + j] = accc[j];
            was[s] = atomicMin(voxel + voxel_of(acc[j], a.rho, vw), n0 + j);
        }
    }
    __syncwarp();   // orders every lane's claim before the reads below
    int c = 0;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const int j = lane + 32 * s;
        if (j < m) {
            // held before this sub-batch: not ours; else ours if no lower node of the sub-batch took it
            const int mine = was[s] > n0 + j && __ldcg(voxel + voxel_of(acc[j], a.rho, vw)) == n0 + j;
            rep[n0 + j] = mine;
            c += mine;
        }
    }
    c = (int)__reduce_add_sync(kFull, (unsigned)c);
    if (lane == 0) {
        *gain += c;
        *d_n = n0 + m;
    }
}

// The first node: p0, its clearance, its voxel and its representative mark; one node, no gain.
__global__ void k_rrt_init(RrtArgs a, float2 p0, float2 *nodes, float *nclr, int vw, int *voxel, int *rep, int *cnt) {
    if (threadIdx.x != 0) return;
    nodes[0] = p0;
    nclr[0] = clearance_at(a, p0.x, p0.y);
    voxel[voxel_of(p0, a.rho, vw)] = 0;
    rep[0] = 1;
    cnt[0] = 1;
    cnt[1] = 0;
}

// One CTA: the flagged entries of src[0 .. n) in order to dst[0 ..), at most
// cap of them; *count receives the number written.
__global__ void __launch_bounds__(1024) k_rrt_compact(const float2 *__restrict__ src, const int *__restrict__ flag,
                                                      int n, float2 *__restrict__ dst, int cap, int *count) {
    __shared__ int warp_cnt[32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const bool take = i < n && flag[i] != 0;
        const unsigned bal = __ballot_sync(kFull, take);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int v = lane < nwarps ? warp_cnt[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            warp_cnt[lane] = incl - v;
        }
        __syncthreads();
        if (take) {
            const int pos = s_base + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) dst[pos] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += warp_cnt[warp] + __popc(bal);
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = min(cap, s_base);
}

__global__ void k_fill_int(int *p, size_t n, int v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

int rrt_sample_dev(const float *clr, int W, int H, double res, double p0x, double p0y, double rho, double eta_max,
                   double r_robot, int eps_gain, uint64_t seed, int max_rounds, int node_cap, float *xy_out, int cap,
                   int *n_out, int *rounds_out, int *nodes_out, cudaStream_t s, const char **err) {
    const double Wm = W * res, Hm = H * res;
    if (!(p0x >= 0 && p0y >= 0 && p0x < Wm && p0y < Hm)) {
        *err = "the start point lies off the map";
        return RELO_E_INVALID_ARG;
    }
    const long long n_s_ll = (long long)ceil((double)W * H * res * res / (rho * rho));
    if (n_s_ll < 1 || n_s_ll > (1ll << 26)) {
        *err = "rho gives too many samples per round";
        return RELO_E_INVALID_ARG;
    }
    const int n_s = (int)n_s_ll;
    const int vw = (int)ceil(Wm / rho) + 1, vh = (int)ceil(Hm / rho) + 1;
    const size_t n_vox = (size_t)vw * vh;
    float2 *nodes = nullptr;
    float *nclr = nullptr;
    RrtCand *cand = nullptr;
    int2 *part = nullptr;
    int *voxel = nullptr, *rep = nullptr, *cnt = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 1);
    };
    alloc((void **)&nodes, sizeof(float2) * (size_t)node_cap);
    alloc((void **)&nclr, sizeof(float) * (size_t)node_cap);
    alloc((void **)&cand, sizeof(RrtCand) * kRrtSub);
    alloc((void **)&part, sizeof(int2) * kNearCtas * kRrtSub);
    alloc((void **)&voxel, sizeof(int) * n_vox);
    alloc((void **)&rep, sizeof(int) * (size_t)node_cap);
    alloc((void **)&cnt, sizeof(int) * 3);   // node count, gain, output count
    int rc = RELO_OK, n = 1, rounds = 0;
    if (e == cudaSuccess) {
        const float fres = (float)res;
        RrtArgs a{clr, W, H, fres, (float)rho, (float)eta_max, (float)r_robot, (float)W * fres, (float)H * fres, seed};
        k_fill_int<<<256, 256, 0, s>>>(voxel, n_vox, 0x7fffffff);
        k_rrt_init<<<1, 32, 0, s>>>(a, make_float2((float)p0x, (float)p0y), nodes, nclr, vw, voxel, rep, cnt);
        while ((e = cudaGetLastError()) == cudaSuccess) {
            k_fill_int<<<1, 32, 0, s>>>(cnt + 1, 1, 0);
            for (int i0 = 0; i0 < n_s; i0 += kRrtSub) {
                const int n_sub = std::min(kRrtSub, n_s - i0);
                k_rrt_near<<<kNearCtas, kRrtSub, 0, s>>>(a, nodes, cnt, i0, n_sub, rounds, part);
                k_rrt_extend<<<(n_sub * 32 + 255) / 256, 256, 0, s>>>(a, nodes, nclr, part, kNearCtas, i0, n_sub,
                                                                      rounds, cand);
                k_rrt_resolve<<<1, 32, 0, s>>>(a, cand, n_sub, nodes, nclr, cnt, node_cap, vw, voxel, rep, cnt + 1);
            }
            int host[2] = {0, 0};
            e = cudaMemcpyAsync(host, cnt, sizeof host, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            n = host[0];
            ++rounds;
            if (host[1] <= eps_gain || rounds >= max_rounds || n >= node_cap) break;
        }
        // the voxel representatives in order of node index
        if (e == cudaSuccess) {
            k_rrt_compact<<<1, 1024, 0, s>>>(nodes, rep, n, reinterpret_cast<float2 *>(xy_out), cap, cnt + 2);
            int reps = 0;
            e = cudaMemcpyAsync(&reps, cnt + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            *n_out = reps;
            *rounds_out = rounds;
            *nodes_out = n;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        rc = RELO_E_CUDA;
    }
    cudaFree(nodes);
    cudaFree(nclr);
    cudaFree(cand);
    cudaFree(part);
    cudaFree(voxel);
    cudaFree(rep);
    cudaFree(cnt);
    return rc;
}

namespace {

// The grid the clearance EDT runs on: the map with a ring of one cell around
// it, every cell occupied (100) that the RRT may not stand on (occupied,
// v >= 65, or unknown, v < 0) and every ring cell occupied (the outside of
// the map is blocked); traversable cells 0.
__global__ void k_rrt_blocked(const int8_t *__restrict__ grid, int W, int H, int8_t *__restrict__ out) {
    const int pw = W + 2, ph = H + 2;
    const long long n = (long long)pw * ph;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / pw) - 1, x = (int)(i % pw) - 1;
        bool blocked = true;
        if (x >= 0 && y >= 0 && x < W && y < H) {
            const int v = grid[(size_t)y * W + x];
            blocked = v < 0 || v >= 65;
        }
        out[i] = blocked ? (int8_t)100 : (int8_t)0;
    }
}

// MinDistToObstacle as a per-cell table (Sec. III-A item 3): res times the
// distance from the cell centre to the nearest blocked cell centre, from the
// exact squared EDT of the ringed grid (never -1: the ring is blocked); the
// square root and the product in FP64, rounded once to float32.
__global__ void k_rrt_clearance(const int32_t *__restrict__ d2p, int W, int H, double res, float *__restrict__ clr) {
    const long long n = (long long)W * H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i % W);
        const int32_t v = d2p[(size_t)(y + 1) * (W + 2) + (x + 1)];
        clr[i] = (float)(res * sqrt((double)v));
    }
}

}  // namespace

cudaError_t launch_rrt_blocked(const int8_t *grid, int W, int H, int8_t *out, cudaStream_t s) {
    k_rrt_blocked<<<1024, 256, 0, s>>>(grid, W, H, out);
    return cudaGetLastError();
}

cudaError_t launch_rrt_clearance(const int32_t *d2p, int W, int H, double res, float *clr, cudaStream_t s) {
    k_rrt_clearance<<<1024, 256, 0, s>>>(d2p, W, H, res, clr);
    return cudaGetLastError();
}

}  // namespace relo
