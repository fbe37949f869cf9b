// ICP refinement of the local top-k poses and their re-evaluation (the last
// step of the framework overview, Sec. III: the local top-k poses are aligned
// to the whole map and scored again; Remark 2 names the refinement operator).
//
// k_icp: one warp per local top-k pose.  The pose starts at its hypothesis
// cell centre and orientation theta_m.  Beam i is the sensor-frame point
// (z_i, a_i), z_i = R_i res / 2^16 (its Q16 range) and a_i = 2 pi b_i / N_s (its
// panoramic grid angle).  An iteration maps every valid beam to its world
// point, pairs it with the centre of the nearest occupied cell to the cell it
// falls in (the radius is the exact EDT value there; ties go to the smaller
// dy, then the smaller dx; pairs farther than the TAM clamp C = (d_max /
// res)^2 are dropped), and applies the rigid motion that minimises the
// squared pair distances: with the centroids mw, mc and the centred cross and
// dot sums, phi = atan2(cross, dot) and t = mc - R(phi) mw.  It stops after
// icp_iters iterations, when fewer than 2 pairs remain, or when the motion is
// below 1e-9 rad and 1e-9 m.  All pose arithmetic is FP64.
//
// The refined pose is then scored like TAM: each beam ends in the cell
// floor(world / res), takes min(d2, C) (C off the map), and the k-th smallest
// value, the likelihood table and the epilogue of Eq. 23-31 (or the metric
// fine_metric selects) give the score, in the same FP32 arithmetic as k_tam.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int isqrt_floor(int v) {   // v >= 0
    int r = (int)sqrtf((float)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// The nearest occupied cell to cell (x, y) when its squared distance is at
// most cap: the cells at exactly the EDT distance, by increasing dy, then dx.
__device__ bool nearest_occupied(const ReqDesc &d, int x, int y, int cap, int &ox, int &oy) {
    if (x < 0 || y < 0 || x >= d.W || y >= d.H) return false;
    const int d2 = d.d2map[(size_t)y * d.W + x];
    if (d2 < 0 || d2 > cap) return false;
    const int r = isqrt_floor(d2);
    for (int dy = -r; dy <= r; ++dy) {
        const int rest = d2 - dy * dy;
        const int s = isqrt_floor(rest);
        if (s * s != rest) continue;
        for (int k = 0; k < (s == 0 ? 1 : 2); ++k) {
            const int cx = x + (k == 0 ? -s : s), cy = y + dy;
            if (cx < 0 || cy < 0 || cx >= d.W || cy >= d.H) continue;
            if (d.grid[(size_t)cy * d.W + cx] >= 65) {
                ox = cx;
                oy = cy;
                return true;
            }
        }
    }
    return false;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int clamped_d2(const ReqDesc &d, int x, int y) {
    if (x < 0 || y < 0 || x >= d.W || y >= d.H) return d.C;
    const int v = d.d2map[(size_t)y * d.W + x];
    return (v < 0 || v > d.C) ? d.C : v;
}

__global__ void __launch_bounds__(32) k_icp(const ReqDesc *__restrict__ reqs, int batch_lo, int batch_hi) {
    extern __shared__ int qv[];   // [valid beams] clamped d2 at the refined endpoints
    const ReqDesc &d = reqs[blockIdx.x];
    const int lane = threadIdx.x;
    const int slot = blockIdx.y;
    if (slot >= (batch_hi - batch_lo) * d.L) return;
    const int b = batch_lo + slot / d.L;
    if (b >= d.n_batches) return;
    const int s = d.local[(size_t)b * d.L + slot % d.L];
    const int N = d.scan->n_valid;
    if (s < 0 || N <= 0) return;
    const int2 hc = d.hyps[d.survivors[s]];
    const double res = d.resd, q16 = res / 65536.0, ang = 2.0 * M_PI / (double)d.ns;
    double px = ((double)hc.x + 0.5) * res, py = ((double)hc.y + 0.5) * res;
    double th = (double)d.best_m[s] * ang;
    for (int it = 0; it < d.icp_iters; ++it) {
        double n = 0, swx = 0, swy = 0, scx = 0, scy = 0, sdot = 0, scr = 0;
        for (int i = lane; i < N; i += 32) {
            const int2 bR = d.vbR[i];
            const double z = (double)bR.y * q16;
            double sn, cs;
            sincos(th + (double)bR.x * ang, &sn, &cs);
            const double wx = px + z * cs, wy = py + z * sn;
            int ox, oy;
            if (!nearest_occupied(d, (int)floor(wx / res), (int)floor(wy / res), d.C, ox, oy)) continue;
            const double cx = ((double)ox + 0.5) * res, cy = ((double)oy + 0.5) * res;
            n += 1.0;
            swx += wx;
            swy += wy;
            scx += cx;
            scy += cy;
            sdot += wx * cx + wy * cy;
            scr += wx * cy - wy * cx;
        }
        n = warp_sum_d(n);
        if (n < 2.0) break;
        swx = warp_sum_d(swx);
        swy = warp_sum_d(swy);
        scx = warp_sum_d(scx);
        scy = warp_sum_d(scy);
        sdot = warp_sum_d(sdot);
        scr = warp_sum_d(scr);
        const double mwx = swx / n, mwy = swy / n, mcx = scx / n, mcy = scy / n;
        const double f = atan2(scr - n * (mwx * mcy - mwy * mcx), sdot - n * (mwx * mcx + mwy * mcy));
        double sf, cf;
        sincos(f, &sf, &cf);
        const double tx = mcx - (cf * mwx - sf * mwy), ty = mcy - (sf * mwx + cf * mwy);
        const double nx = cf * px - sf * py + tx, ny = sf * px + cf * py + ty;
        const double moved = fabs(nx - px) + fabs(ny - py);
        px = nx;
        py = ny;
        th += f;
        if (fabs(f) < 1e-9 && moved < 1e-9) break;
    }
    // the refined pose scored again
    int sumb = 0;
    for (int i = lane; i < N; i += 32) {
        const int2 bR = d.vbR[i];
        const double z = (double)bR.y * q16;
        double sn, cs;
        sincos(th + (double)bR.x * ang, &sn, &cs);
        const int q = clamped_d2(d, (int)floor((px + z * cs) / res), (int)floor((py + z * sn) / res));
        qv[i] = q;
        sumb += q;
    }
    __syncwarp();
    sumb = __reduce_add_sync(kFull, sumb);
    const int C = d.C;
    const int k = d.fine < kFineBaseline ? d.scan->k_ret : N;
    auto count_le = [&](int x) {
        int c = 0;
        for (int i = lane; i < N; i += 32) c += qv[i] <= x ? 1 : 0;
        return __reduce_add_sync(kFull, c);
    };
    int bk = C, cle = N;
    if (k < N) {   // the smallest b with #{q <= b} >= k, by bisection over [0, C]
        int lo = 0, hi = C, c_hi = N;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int c = count_le(mid);
            if (c >= k) {
                hi = mid;
                c_hi = c;
            } else {
                lo = mid + 1;
            }
        }
        bk = lo;
        cle = c_hi;
    }
    float sl = 0.0f, sgs = 0.0f;
    for (int i = lane; i < N; i += 32) {
        const float2 g = d.lut[qv[i]];
        sgs += g.y;
        if (qv[i] <= bk) sl += g.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sl += __shfl_xor_sync(kFull, sl, o);
        sgs += __shfl_xor_sync(kFull, sgs, o);
    }
    if (lane == 0) {
        // Eq. 27-31 as k_tam evaluates them
        const float topsum = sl - (float)(cle - k) * d.lut[bk].x;
        const float lbar = topsum * (1.0f / (float)k);
        const float dd = d.res / (float)N * sgs;   // d_max - dbar
        const float dbar = d.d_max - dd;
        const float var = fmaxf(d.res2 / (float)N * (float)sumb - dbar * dbar, 0.0f);
        const float sd = fminf(dd, d.d_max - d.d_min) * (1.0f / (d.d_max - d.d_min));
        float T = cbrtf(expf(lbar - 0.5f * var) * sd);
        if (d.fine == kFineTamMean) T = (expf(lbar) + sd + expf(-0.5f * var)) * (1.0f / 3.0f);
        else if (d.fine == kFineBaseline) T = sqrtf(expf(lbar) * sd);
        else if (d.fine == kFineLF) T = topsum;
        double *ps = d.ref_pose + 3 * (size_t)s;
        ps[0] = px;
        ps[1] = py;
        ps[2] = th;
        d.reev[s] = T;
    }
}

}  // namespace

cudaError_t launch_icp(const ReqDesc *reqs, int R, int batch_lo, int batch_hi, int max_L, int max_beams,
                       cudaStream_t s) {
    const int slots = (batch_hi - batch_lo) * max_L;
    if (R < 1 || slots < 1) return cudaSuccess;
    const size_t smem = sizeof(int) * (size_t)(max_beams > 0 ? max_beams : 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_icp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_icp<<<dim3(R, slots), 32, smem, s>>>(reqs, batch_lo, batch_hi);
    return cudaGetLastError();
}

}  // namespace relo
