// Traversability-constrained hypothesis sampling on the GPU (Algorithm 1,
// Sec. III-A, Remark 4), in a batched-expansion form.
//
// Algorithm 1 draws N_sampling random points per round and grows the tree one
// point at a time.  Here every point of a round is drawn and extended at
// once against the tree as it stood when the round began, and the accepted
// points join the tree in sample order at the end of the round; the
// voxel downsampling (side rho, each voxel represented by its lowest-index
// node) and the gain test (stop once a round adds at most eps_gain voxels)
// are Algorithm 1's.  The result covers the reachable free space like the
// serial tree but is not its node set.
//
// Per sample i of round r: p_rand from a counter-based hash (splitmix64 of
// seed ^ (r << 40 | i << 1 | k), k = 0, 1 for x, y); NearestNode by brute
// force over the round's tree (squared distance, ties to the lower index);
// AdaptiveExpandDist eta = eta_max when the clearance d at the nearest node is
// >= 2 r_robot, r_robot when d <= r_robot, linear between; ExtendPoint moves
// min(eta, |p_rand - p_nearest|) towards p_rand; the new point must lie in the
// map rectangle, and every point of the segment at spacing res / 2 (both ends
// included) must have clearance >= r_robot (clearance: a per-cell table in
// metres, 0 off the map).  Positions are float32 metres.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/relo.h"
#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;

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
    uint64_t seed;
};

__device__ __forceinline__ float clearance_at(const RrtArgs &a, float x, float y) {
    const int cx = (int)floorf(x / a.res), cy = (int)floorf(y / a.res);
    if (cx < 0 || cy < 0 || cx >= a.W || cy >= a.H) return 0.0f;
    return a.clr[(size_t)cy * a.W + cx];
}

// one thread per sample: the extended point and whether it is accepted
__global__ void k_rrt_sample(RrtArgs a, const float2 *__restrict__ nodes, int n0, int n_s, int round,
                             float2 *__restrict__ cand, int *__restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_s) return;
    const float Wm = a.W * a.res, Hm = a.H * a.res;
    const float rx = unit_draw(a.seed, round, i, 0) * Wm, ry = unit_draw(a.seed, round, i, 1) * Hm;
    int best = 0;
    float best2 = INFINITY;
    for (int j = 0; j < n0; ++j) {
        const float2 p = nodes[j];
        const float ex = p.x - rx, ey = p.y - ry;
        const float d2 = ex * ex + ey * ey;
        if (d2 < best2) {   // ascending j: ties keep the lower index
            best2 = d2;
            best = j;
        }
    }
    const float2 pn = nodes[best];
    const float d = clearance_at(a, pn.x, pn.y);
    float eta;
    if (d >= 2.0f * a.r_robot) eta = a.eta_max;
    else if (d <= a.r_robot) eta = a.r_robot;
    else eta = a.r_robot + (a.eta_max - a.r_robot) * (d - a.r_robot) / a.r_robot;
    const float vx = rx - pn.x, vy = ry - pn.y;
    const float L = sqrtf(vx * vx + vy * vy);
    int ok = L > 0.0f;
    float nx = pn.x, ny = pn.y;
    if (ok) {
        const float step = fminf(eta, L);
        nx = pn.x + vx / L * step;
        ny = pn.y + vy / L * step;
        ok = nx >= 0.0f && ny >= 0.0f && nx < Wm && ny < Hm;
        const int nseg = (int)ceilf(step / (0.5f * a.res));
        for (int k = 0; k <= nseg && ok; ++k) {
            const float t = nseg ? (float)k / (float)nseg : 0.0f;
            if (clearance_at(a, pn.x + (nx - pn.x) * t, pn.y + (ny - pn.y) * t) < a.r_robot) ok = 0;
        }
    }
    cand[i] = make_float2(nx, ny);
    flag[i] = ok;
}

// One CTA: the flagged entries of src[0 .. n) in order to dst[base ..), at
// most cap - base of them; *count receives how many were flagged (all of
// them, written or not).
__global__ void __launch_bounds__(1024) k_rrt_compact(const float2 *__restrict__ src, const int *__restrict__ flag,
                                                      int n, float2 *__restrict__ dst, int base, int cap,
                                                      int *count) {
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
            const int pos = base + s_base + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) dst[pos] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += warp_cnt[warp] + __popc(bal);
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = s_base;
}

__device__ __forceinline__ int voxel_of(float2 p, float rho, int vw) {
    return (int)floorf(p.y / rho) * vw + (int)floorf(p.x / rho);
}

// nodes [n0, n1): each claims its voxel with the lowest node index
__global__ void k_rrt_claim(const float2 *__restrict__ nodes, int n0, int n1, float rho, int vw, int *voxel) {
    const int j = n0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n1) return;
    atomicMin(voxel + voxel_of(nodes[j], rho, vw), j);
}

// nodes [n0, n1) that hold their voxel: the round's new voxels (the gain); flag marks representatives
__global__ void k_rrt_gain(const float2 *__restrict__ nodes, int n0, int n1, float rho, int vw, const int *voxel,
                           int *rep, int *gain) {
    const int j = n0 + blockIdx.x * blockDim.x + threadIdx.x;
    int mine = 0;
    if (j < n1) {
        mine = voxel[voxel_of(nodes[j], rho, vw)] == j;
        rep[j] = mine;
    }
    const int c = __reduce_add_sync(kFull, mine);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(gain, c);
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
    float2 *nodes = nullptr, *cand = nullptr;
    int *flag = nullptr, *voxel = nullptr, *rep = nullptr, *cnt = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 1);
    };
    alloc((void **)&nodes, sizeof(float2) * (size_t)node_cap);
    alloc((void **)&cand, sizeof(float2) * (size_t)n_s);
    alloc((void **)&flag, sizeof(int) * (size_t)n_s);
    alloc((void **)&voxel, sizeof(int) * n_vox);
    alloc((void **)&rep, sizeof(int) * (size_t)node_cap);
    alloc((void **)&cnt, sizeof(int) * 2);
    int rc = RELO_OK, n = 1, rounds = 0;
    if (e == cudaSuccess) {
        RrtArgs a{clr, W, H, (float)res, (float)rho, (float)eta_max, (float)r_robot, seed};
        const float2 p0 = make_float2((float)p0x, (float)p0y);
        k_fill_int<<<256, 256, 0, s>>>(voxel, n_vox, 0x7fffffff);
        e = cudaMemcpyAsync(nodes, &p0, sizeof p0, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            k_rrt_claim<<<1, 32, 0, s>>>(nodes, 0, 1, a.rho, vw, voxel);
            k_fill_int<<<1, 32, 0, s>>>(rep, 1, 1);
        }
        while (e == cudaSuccess) {
            k_rrt_sample<<<(n_s + 255) / 256, 256, 0, s>>>(a, nodes, n, n_s, rounds, cand, flag);
            k_rrt_compact<<<1, 1024, 0, s>>>(cand, flag, n_s, nodes, n, node_cap, cnt);
            int added = 0;
            e = cudaMemcpyAsync(&added, cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            const int n1 = std::min(node_cap, n + added);
            int gain = 0;
            if (n1 > n) {
                k_fill_int<<<1, 32, 0, s>>>(cnt + 1, 1, 0);
                k_rrt_claim<<<(n1 - n + 255) / 256, 256, 0, s>>>(nodes, n, n1, a.rho, vw, voxel);
                k_rrt_gain<<<(n1 - n + 255) / 256, 256, 0, s>>>(nodes, n, n1, a.rho, vw, voxel, rep, cnt + 1);
                e = cudaMemcpyAsync(&gain, cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
            n = n1;
            ++rounds;
            if (gain <= eps_gain || rounds >= max_rounds || n >= node_cap) break;
        }
        // the voxel representatives in order of node index
        if (e == cudaSuccess) {
            k_rrt_compact<<<1, 1024, 0, s>>>(nodes, rep, n, reinterpret_cast<float2 *>(xy_out), 0, cap, cnt);
            int reps = 0;
            e = cudaMemcpyAsync(&reps, cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
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
    cudaFree(cand);
    cudaFree(flag);
    cudaFree(voxel);
    cudaFree(rep);
    cudaFree(cnt);
    return rc;
}

}  // namespace relo
