// ICP refinement of the local top-k poses and their re-evaluation (the last
// step of the framework overview, Sec. III: the local top-k poses are aligned
// to the whole map and scored again; Remark 2 names the refinement operator).
//
// k_icp: one CTA of kIcpThreads per local top-k pose.  The pose starts at its hypothesis
// cell centre and orientation theta_m.  Beam i is the sensor-frame point
// (z_i, a_i), z_i = R_i res / 2^16 (its Q16 range) and a_i = 2 pi b_i / N_s (its
// panoramic grid angle); its sensor-frame point s_i = (z_i cos a_i, z_i sin
// a_i) is computed once.  An iteration maps every valid beam to its world
// point w = p + R(theta) s (each product and sum rounded on its own, as the
// oracle does; its cell is floor(w * (1 / res))), pairs it with the centre of
// the nearest occupied cell to the cell it
// falls in (the radius is the exact EDT value there; ties go to the smaller
// dy, then the smaller dx; pairs farther than the TAM clamp C = (d_max /
// res)^2 are dropped), and applies the rigid motion that minimises the
// squared pair distances: with the centroids mw, mc and the centred cross and
// dot sums, phi = atan2(cross, dot) and t = mc - R(phi) mw.  It stops after
// icp_iters iterations, when fewer than 2 pairs remain, or when the motion is
// below 1e-9 rad and 1e-9 m.  All pose arithmetic is FP64.
//
// The refined pose is then scored like TAM: each beam ends in the cell of its
// world point, takes min(d2, C) (C off the map), and the k-th smallest
// value, the likelihood table and the epilogue of Eq. 23-31 (or the metric
// fine_metric selects) give the score, in the same FP32 arithmetic as k_tam.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kIcpThreads = 256;
constexpr int kIcpWarps = kIcpThreads / 32;

// The nearest occupied cell to cell (x, y) when its squared distance is at
// most cap (<= C): the cells at exactly the EDT distance, by increasing dy,
// then dx, from the map's table of the offsets at each squared distance.
__device__ bool nearest_occupied(const ReqDesc &d, int x, int y, int cap, int &ox, int &oy) {
    if (x < 0 || y < 0 || x >= d.W || y >= d.H) return false;
    const int d2 = d.d2map[(size_t)y * d.W + x];
    if (d2 < 0 || d2 > cap) return false;
    const int e1 = d.sq_off[d2 + 1];
    for (int e = d.sq_off[d2]; e < e1; ++e) {
        const short2 o = d.sq_rep[e];
        const int cx = x + o.y, cy = y + o.x;
        if (cx < 0 || cy < 0 || cx >= d.W || cy >= d.H) continue;
        if (d.grid[(size_t)cy * d.W + cx] >= 65) {
            ox = cx;
            oy = cy;
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sums of V values over the CTA: every thread gets the same totals (the warp
// partials are added in warp order by every thread).  red: [V][kIcpWarps].
template <int V>
__device__ __forceinline__ void block_sums(double (&v)[V], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const double w = warp_sum_d(v[j]);
        if (lane == 0) red[j * kIcpWarps + warp] = w;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < V; ++j) {
        double t = 0.0;
        for (int w = 0; w < kIcpWarps; ++w) t += red[j * kIcpWarps + w];
        v[j] = t;
    }
    __syncthreads();   // red is free again
}

// world point and cell of a sensor-frame point at pose (x, y) with ct, st = cos, sin of theta
__device__ __forceinline__ void world_point(double x, double y, double ct, double st, double sx, double sy,
                                            double inv_res, double &wx, double &wy, int &cx, int &cy) {
    wx = __dadd_rn(x, __dsub_rn(__dmul_rn(ct, sx), __dmul_rn(st, sy)));
    wy = __dadd_rn(y, __dadd_rn(__dmul_rn(st, sx), __dmul_rn(ct, sy)));
    cx = (int)floor(__dmul_rn(wx, inv_res));
    cy = (int)floor(__dmul_rn(wy, inv_res));
}

__device__ __forceinline__ int clamped_d2(const ReqDesc &d, int x, int y) {
    if (x < 0 || y < 0 || x >= d.W || y >= d.H) return d.C;
    const int v = d.d2map[(size_t)y * d.W + x];
    return (v < 0 || v > d.C) ? d.C : v;
}

__global__ void __launch_bounds__(kIcpThreads) k_icp(const ReqDesc *__restrict__ reqs, int batch_lo, int batch_hi) {
    extern __shared__ double spt[];   // [2 N] sensor-frame points, then [N] int clamped d2 of the refined endpoints
    __shared__ double red[7 * kIcpWarps];
    const ReqDesc &d = reqs[blockIdx.x];
    const int tid = threadIdx.x;
    const int slot = blockIdx.y;
    if (slot >= (batch_hi - batch_lo) * d.L) return;
    const int b = batch_lo + slot / d.L;
    if (b >= d.n_batches) return;
    const int s = d.local[(size_t)b * d.L + slot % d.L];
    const int N = d.scan->n_valid;
    if (s < 0 || N <= 0) return;
    int *qv = reinterpret_cast<int *>(spt + 2 * (size_t)N);
    const int2 hc = d.hyps[d.survivors[s]];
    const double res = d.resd, q16 = res / 65536.0, ang = 2.0 * M_PI / (double)d.ns, inv_res = 1.0 / res;
    for (int i = tid; i < N; i += kIcpThreads) {
        const int2 bR = d.vbR[i];
        const double z = __dmul_rn((double)bR.y, q16), a = __dmul_rn((double)bR.x, ang);
        spt[2 * i] = __dmul_rn(z, cos(a));
        spt[2 * i + 1] = __dmul_rn(z, sin(a));
    }
    __syncthreads();
    double px = __dmul_rn((double)hc.x + 0.5, res), py = __dmul_rn((double)hc.y + 0.5, res);
    double th = __ddiv_rn(__dmul_rn((double)d.best_m[s], 2.0 * M_PI), (double)d.ns);
    for (int it = 0; it < d.icp_iters; ++it) {
        double v[7] = {0, 0, 0, 0, 0, 0, 0};   // pairs, sums of w, of c, of w.c and of w x c
        const double ct = cos(th), st = sin(th);
        for (int i = tid; i < N; i += kIcpThreads) {
            double wx, wy;
            int ex, ey, ox, oy;
            world_point(px, py, ct, st, spt[2 * i], spt[2 * i + 1], inv_res, wx, wy, ex, ey);
            if (!nearest_occupied(d, ex, ey, d.C, ox, oy)) continue;
            const double cx = ((double)ox + 0.5) * res, cy = ((double)oy + 0.5) * res;
            v[0] += 1.0;
            v[1] += wx;
            v[2] += wy;
            v[3] += cx;
            v[4] += cy;
            v[5] += wx * cx + wy * cy;
            v[6] += wx * cy - wy * cx;
        }
        block_sums(v, red);
        const double n = v[0], swx = v[1], swy = v[2], scx = v[3], scy = v[4], sdot = v[5], scr = v[6];
        if (n < 2.0) break;
        const double mwx = swx / n, mwy = swy / n, mcx = scx / n, mcy = scy / n;
        const double f = atan2(scr - n * (mwx * mcy - mwy * mcx), sdot - n * (mwx * mcx + mwy * mcy));
        const double cf = cos(f), sf = sin(f);
        const double tx = __dsub_rn(mcx, __dsub_rn(__dmul_rn(cf, mwx), __dmul_rn(sf, mwy)));
        const double ty = __dsub_rn(mcy, __dadd_rn(__dmul_rn(sf, mwx), __dmul_rn(cf, mwy)));
        const double nx = __dadd_rn(__dsub_rn(__dmul_rn(cf, px), __dmul_rn(sf, py)), tx);
        const double ny = __dadd_rn(__dadd_rn(__dmul_rn(sf, px), __dmul_rn(cf, py)), ty);
        const double moved = fabs(nx - px) + fabs(ny - py);
        px = nx;
        py = ny;
        th = __dadd_rn(th, f);
        if (fabs(f) < 1e-9 && moved < 1e-9) break;
    }
    // the refined pose scored again
    int sumb = 0;
    {
        const double ct = cos(th), st = sin(th);
        for (int i = tid; i < N; i += kIcpThreads) {
            double wx, wy;
            int ex, ey;
            world_point(px, py, ct, st, spt[2 * i], spt[2 * i + 1], inv_res, wx, wy, ex, ey);
            const int q = clamped_d2(d, ex, ey);
            qv[i] = q;
            sumb += q;
        }
    }
    {
        double t[1] = {(double)sumb};
        block_sums(t, red);   // also makes qv visible to the whole CTA
        sumb = (int)t[0];
    }
    const int C = d.C;
    const int k = d.fine < kFineBaseline ? d.scan->k_ret : N;
    auto count_le = [&](int x) {
        double c[1] = {0.0};
        for (int i = tid; i < N; i += kIcpThreads) c[0] += qv[i] <= x ? 1.0 : 0.0;
        block_sums(c, red);
        return (int)c[0];
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
    for (int i = tid; i < N; i += kIcpThreads) {
        const float2 g = d.lut[qv[i]];
        sgs += g.y;
        if (qv[i] <= bk) sl += g.x;
    }
    {
        double t[2] = {(double)sl, (double)sgs};
        block_sums(t, red);
        sl = (float)t[0];
        sgs = (float)t[1];
    }
    if (tid == 0) {
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
    const size_t smem = (2 * sizeof(double) + sizeof(int)) * (size_t)(max_beams > 0 ? max_beams : 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_icp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_icp<<<dim3(R, slots), kIcpThreads, smem, s>>>(reqs, batch_lo, batch_hi);
    return cudaGetLastError();
}

}  // namespace relo
