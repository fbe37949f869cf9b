// Ray-cast panoramic synthesized scans (Eq. 13) and SMAD (Eq. 16-20).
//
// Two kernels per batch.  k_cast casts every ray of every hypothesis, 32
// neighbouring directions per warp (lane = ray, so the lanes of a warp trace
// rays of similar length), into a per-request table of Q16 ranges.  Work
// items run over the hypotheses for one 32-direction chunk after another, so
// the warps in flight share a few directions' tables (they stay in L1).  k_smad
// then reads a hypothesis's row, forms chunk prefixes that
// give the cyclic prefix sum S of Eq. 17 at any index, evaluates the window
// sums of Eq. 18 for the orientations m of Eq. 15 with two lookups per FoV
// interval, and minimises the integer SMAD numerator |sum R_real - W_m| of
// Eq. 19 over m (Eq. 20; ties keep the smaller m; the shared denominator of
// the two means cancels from every comparison).
//
// Ray traversal.  From the hypothesis cell centre along the Q30 direction D,
// cells are entered in the order of the ray's grid-line crossings: with k x-
// and l y-crossings so far, x is stepped when (2k+1)|Dy| <= (2l+1)|Dx| (a
// corner tie steps x).  The recurrence tracks the difference e = (2l+1)|Dx| -
// (2k+1)|Dy| incrementally (e -= 2|Dy| after an x step, e += 2|Dx| after a y
// step); it always lies in [-2^31, 2^31), so a 32-bit integer holds it
// exactly.  The ray stops on leaving the map, on entering a cell whose centre
// lies beyond the maximum range, or on entering an occupied cell; the range of
// a hit is floor(sqrt(|d|^2 * 2^32)) (cells, Q16), else 0 (the placeholder of
// the invalid beam).  Occupancy comes from the 8x8-tile bitmap.  The default
// traversal (walk_ray) moves tile by tile with per-direction tables built
// once per (N_s, range limit); cast_ray steps cell by cell with the same
// recurrence.
//
// A panoramic synthesized scan depends only on the map, the hypothesis, the
// beam grid N_s and the range limit, not on the real scan.  The table a
// request casts into is either its scratch (kScanCast) or a resident table
// (kScanStore) that later requests with the same map, hypotheses, N_s and
// limit read without casting (kScanRead).
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "relo_internal.h"
#include "scan_prep.cuh"

namespace relo {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t isqrt_q16(int c2) {
    // floor(sqrt(c2 * 2^32)): float estimate, one Newton correction, exact fix-up
    const unsigned long long N = (unsigned long long)(unsigned)c2 << 32;
    unsigned long long r = (unsigned long long)(sqrtf((float)c2) * 65536.0f);
    long long err = (long long)(N - r * r);
    r = (unsigned long long)((long long)r + (long long)__fdividef((float)err, 2.0f * (float)r + 1.0f));
    while (r * r > N) --r;
    while ((r + 1) * (r + 1) <= N) ++r;
    return (uint32_t)r;
}

// State of one ray's traversal.  advance() enters the next cell, or crosses a
// whole empty tile at once, and reports whether the ray has stopped.
//
// Empty tiles are crossed in one move.  Inside a tile whose 64-bit word is 0
// no cell can stop the ray except by leaving the map or the range, and both
// of those only grow along the ray, so jumping straight to the first cell
// past the tile gives the same answer as stepping through it.  With nx
// x-steps and ny y-steps left to the tile's x and y boundaries, the ray
// leaves through the x boundary iff its nx-th x crossing comes no later than
// its ny-th y crossing: e + 2(ny-1)|Dx| - 2(nx-1)|Dy| >= 0.  It then also
// makes the j y-steps whose crossings come strictly earlier, j = the smallest
// integer with 2 j |Dx| >= 2(nx-1)|Dy| - e; leaving through y, it makes the i
// x-steps whose crossings come no later (ties step x first), i = 0 if
// B = e + 2(ny-1)|Dx| < 0, else floor(B / (2|Dy|)) + 1.  Both counts are at
// most 7.
struct Ray {
    int ax, ay, sx, sy, e, cx, cy, adx, ady, c2, n, tile;
    unsigned long long word;

    __device__ __forceinline__ void init(int2 d, int hx, int hy, int tile0, unsigned long long word0) {
        ax = d.x < 0 ? -d.x : d.x;
        ay = d.y < 0 ? -d.y : d.y;
        sx = d.x > 0 ? 1 : -1;
        sy = d.y > 0 ? 1 : -1;
        e = ax - ay;
        cx = hx;
        cy = hy;
        adx = ady = c2 = n = 0;
        tile = tile0;
        word = word0;
    }

    // true once the ray stopped; *range = Q16 range of a hit, else 0
    __device__ __forceinline__ bool advance(const uint64_t *__restrict__ bits, int W, int H, int TW, int lim,
                                            uint32_t *range) {
        if (word == 0ull) {
            const int nx = sx > 0 ? 8 - (cx & 7) : (cx & 7) + 1;
            const int ny = sy > 0 ? 8 - (cy & 7) : (cy & 7) + 1;
            bool xexit;
            if (ay == 0) xexit = true;
            else if (ax == 0) xexit = false;
            else xexit = (long long)e + 2ll * (ny - 1) * ax - 2ll * (nx - 1) * ay >= 0;
            if (xexit) {
                // j = smallest integer with j * 2|Dx| >= A (0 when A <= 0), A = 2(nx-1)|Dy| - e
                const long long A = 2ll * (nx - 1) * ay - e;
                const long long dd = 2ll * ax;
                int j = 0;
                if (A > 0) {
                    j = (int)ceilf((float)A / (float)dd);
                    if ((long long)(j - 1) * dd >= A) --j;
                    if ((long long)j * dd < A) ++j;
                }
                e = (int)((long long)e - 2ll * nx * ay + 2ll * j * ax);
                cx += sx * nx;
                cy += sy * j;
                adx += nx;
                ady += j;
                n += nx + j;
            } else {
                // i = 0 if B < 0, else floor(B / (2|Dy|)) + 1, B = e + 2(ny-1)|Dx|
                const long long B = (long long)e + 2ll * (ny - 1) * ax;
                const long long dd = 2ll * ay;
                int i = 0;
                if (B >= 0) {
                    i = (int)floorf((float)B / (float)dd) + 1;
                    if ((long long)(i - 1) * dd > B) --i;
                    if ((long long)i * dd <= B) ++i;
                }
                e = (int)((long long)e + 2ll * ny * ax - 2ll * i * ay);
                cx += sx * i;
                cy += sy * ny;
                adx += i;
                ady += ny;
                n += ny + i;
            }
            c2 = adx * adx + ady * ady;
        } else if (e >= 0) {
            cx += sx;
            e = (int)((uint32_t)e - 2u * (uint32_t)ay);
            c2 += 2 * adx + 1;
            ++adx;
            ++n;
        } else {
            cy += sy;
            e = (int)((uint32_t)e + 2u * (uint32_t)ax);
            c2 += 2 * ady + 1;
            ++ady;
            ++n;
        }
        if ((unsigned)cx >= (unsigned)W || (unsigned)cy >= (unsigned)H || c2 > lim) {
            *range = 0u;
            return true;
        }
        const int t = (cy >> 3) * TW + (cx >> 3);
        if (t != tile) {
            tile = t;
            word = __ldg(bits + t);
        }
        if ((word >> (((cy & 7) << 3) | (cx & 7))) & 1ull) {
            *range = isqrt_q16(c2);
            return true;
        }
        return false;
    }
};

// whole ray: Q16 range (0 = no hit); *hit receives cy*W+cx or -1, *steps the cells entered
__device__ __forceinline__ uint32_t cast_ray(const uint64_t *__restrict__ bits, int W, int H, int TW, int lim, int hx,
                                             int hy, int2 d, int *hit, int *steps) {
    Ray ray;
    const int tile0 = (hy >> 3) * TW + (hx >> 3);
    ray.init(d, hx, hy, tile0, __ldg(bits + tile0));
    uint32_t r = 0u;
    while (!ray.advance(bits, W, H, TW, lim, &r)) {
    }
    *hit = r ? ray.cy * W + ray.cx : -1;
    *steps = ray.n;
    return r;
}

// Tile walk with the per-direction tables (RayTables).  The ray moves from
// tile to tile in its own frame, the map mirrored in x when D_x <= 0 (x' =
// 8 TW - 1 - x) and in y when D_y <= 0, so that it always travels towards +x
// and +y.  Each of the four frames is stored as a walk frame: cells outside
// the map are set and a last column and row of full tiles follow the map, so
// the first cell outside the map stops the ray like an occupied one and is
// recognised after the loop, which needs no bounds test per tile.  In a tile
// whose word is not zero, the word moved to the current cell
// is ANDed with the table's bit board of the cells still ahead; on a
// staircase that only moves +x and +y the cell order along the ray is the
// row-major bit order, so the lowest common bit is the hit.  Otherwise the
// ray leaves the tile at the cell of step min(selx[|dx| + nx], sely[|dy| +
// ny]), nx and ny being the x- and y-steps to the tile's far edges.  An empty
// tile is left as a whole box of empty tiles ahead (MapDev::reach) when that
// box is larger: the run along the tile's row for a ray within about 14
// degrees of the x axis, the run along its column within 14 degrees of the y
// axis, the empty square otherwise; the same lookups then take the box's far
// edges, since no cell inside it can stop the ray.  Same cells, same hit, same
// range as cast_ray.
__device__ __forceinline__ uint32_t walk_ray(const uint64_t *__restrict__ bits, const uint16_t *__restrict__ reach,
                                             int W, int H, int TW, int TH, const RayTables &t, int ns, int j, int hx,
                                             int hy, int2 d, int *hit, int *steps) {
    const bool xneg = d.x <= 0, yneg = d.y <= 0;
    const unsigned WB = (unsigned)TW + 1u;   // walk frame row, with the border column
    const size_t frame = (size_t)((xneg ? 1 : 0) + (yneg ? 2 : 0)) * walk_frame_words(TW, TH);
    const uint64_t *__restrict__ bq = bits + (size_t)TW * TH + frame;
    const uint16_t *__restrict__ rq = reach + frame;
    // which box of the packed reach the ray leaves: width (reach >> wsh) & 31, height (reach >> hsh) & 31, each
    // at least 1 (bit 15 and up are 0, so a shift of 15 reads a side of 1 tile)
    const long long adir = d.x < 0 ? -(long long)d.x : d.x, bdir = d.y < 0 ? -(long long)d.y : d.y;
    const bool shallow = 4 * bdir <= adir, steep = 4 * adir <= bdir;
    const unsigned wsh = shallow ? 5u : steep ? 15u : 0u;
    const unsigned hsh = steep ? 10u : shallow ? 15u : 0u;
    const int xlo = xneg ? 8 * TW - W : 0, ylo = yneg ? 8 * TH - H : 0;   // the map in the ray's frame
    const int fx = xneg ? 8 * TW - 1 - hx : hx, fy = yneg ? 8 * TH - 1 - hy : hy;
    const uint16_t *__restrict__ selx = t.selx + j;
    const uint16_t *__restrict__ sely = t.sely + j;
    const uint64_t *__restrict__ mk = t.mask + j;
    const unsigned uns = (unsigned)ns;
    // The loop only finds where the ray stops; the range is computed after it,
    // once for the whole warp, rather than in a divergent branch per lane.
    // Cells outside the map are set in the walk frames, so leaving the map
    // ends the loop as a hit and is told apart afterwards.  Indexes are
    // unsigned 32-bit (every table and map index fits).
    int adx = 0, ady = 0, cx = fx, cy = fy;
    int stop;   // 1 hit (or left the map), 2 range limit
    for (;;) {
        const int lx = cx & 7, ly = cy & 7;
        // the tile's word, its boxes and the tile's exit steps are loaded together: one memory round trip
        // per tile (a second one when the ray leaves a larger box)
        const unsigned ti = (unsigned)(cy >> 3) * WB + (unsigned)(cx >> 3);
        const uint64_t word = __ldg(bq + ti);
        const unsigned rv = __ldg(rq + ti);
        uint32_t kx = __ldg(selx + (unsigned)(adx + 8 - lx) * uns);
        uint32_t ky = __ldg(sely + (unsigned)(ady + 8 - ly) * uns);
        const unsigned bw = max(1u, (rv >> wsh) & 31u), bh = max(1u, (rv >> hsh) & 31u);   // the box, in tiles
        const int ex = 8 * (int)bw - lx, ey = 8 * (int)bh - ly;   // x- and y-steps to its far edges
        if ((bw | bh) > 1u) {
            kx = __ldg(selx + (unsigned)(adx + ex) * uns);
            ky = __ldg(sely + (unsigned)(ady + ey) * uns);
        }
        if (word) {
            // move the current cell to bit 0; bits that wrap into the row below
            // sit in columns the board's column mask removes
            const uint64_t w = word >> (lx + 8 * ly);
            const uint32_t cm = 0x01010101u * (0xffu >> lx);   // board columns dx <= 7 - lx, every row
            const uint64_t R = __ldg(mk + (unsigned)(adx + ady) * uns) & (((uint64_t)cm << 32) | cm);
            const uint64_t hm = R & w;
            if (hm) {
                const int b = __ffsll((long long)hm) - 1;
                adx += b & 7;
                ady += b >> 3;
                stop = 1;
                break;
            }
        }
        if (min(kx, ky) == kSelNone) {   // the next cell lies beyond the range limit
            stop = 2;
            break;
        }
        if (kx < ky) {
            adx += ex;
            ady = (int)kx - adx;
        } else {
            ady += ey;
            adx = (int)ky - ady;
        }
        cx = fx + adx;
        cy = fy + ady;
    }
    if (stop == 1 && ((unsigned)(fx + adx - xlo) >= (unsigned)W || (unsigned)(fy + ady - ylo) >= (unsigned)H))
        stop = 3;   // the first cell outside the map
    const int sx = xneg ? -1 : 1, sy = yneg ? -1 : 1;
    cx = hx + sx * adx;
    cy = hy + sy * ady;
    *hit = stop == 1 ? cy * W + cx : -1;
    *steps = stop == 2 ? __ldg(t.kmax + j) + 1 : adx + ady;
    const uint32_t r = isqrt_q16(stop == 1 ? adx * adx + ady * ady : 0);   // a hit lies within the range limit
    return stop == 1 ? r : 0u;
}

// One thread per direction: the DDA of cast_ray from (0, 0), recorded.  The
// forward pass writes the step indexes into selx / sely and, as scratch, the
// kind of step k + 1 into mask row k; the backward pass turns those into the
// bit boards, mask(k) = cell k plus mask(k + 1) moved one cell back along
// step k + 1 (cells that fall off the 8x8 board are dropped).  mask rows must
// start at 0 and selx / sely at kSelNone.
__global__ void k_ray_tables(const int2 *__restrict__ D, int ns, int lim, uint64_t *mask, uint16_t *selx,
                             uint16_t *sely, int32_t *kmax) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const int2 d = D[j];
    const int ax = d.x < 0 ? -d.x : d.x, ay = d.y < 0 ? -d.y : d.y;
    int e = ax - ay, adx = 0, ady = 0, k = 0;
    for (;;) {
        const bool xs = e >= 0;
        const long long nx = adx + (xs ? 1 : 0), ny = ady + (xs ? 0 : 1);
        if (nx * nx + ny * ny > (long long)lim) break;
        mask[(size_t)k * ns + j] = xs ? 1ull : 0ull;
        e = xs ? (int)((uint32_t)e - 2u * (uint32_t)ay) : (int)((uint32_t)e + 2u * (uint32_t)ax);
        adx = (int)nx;
        ady = (int)ny;
        ++k;
        if (xs) selx[(size_t)adx * ns + j] = (uint16_t)k;
        else sely[(size_t)ady * ns + j] = (uint16_t)k;
    }
    kmax[j] = k;
    uint64_t R = 1ull;
    for (int kk = k; kk >= 0; --kk) {
        if (kk < k) {
            const bool xs = mask[(size_t)kk * ns + j] != 0ull;
            R = 1ull | (xs ? ((R & ~0x8080808080808080ull) << 1) : (R << 8));
        }
        mask[(size_t)kk * ns + j] = kk == 0 ? (R & ~1ull) : R;   // the start cell itself is never tested
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

// CAER (Eq. 21) of hypothesis h, by one warp: its synthesized row in the
// warp's shared memory, then for each orientation of the SMAD set the lanes
// sum |R_i - row[(b_i + m) mod N_s]| over every beam (invalid beams carry R
// = 0, as in SMAD) and the warp adds the lane sums; the minimum over m (ties
// to the smaller m) is written like a SMAD numerator, so the ranking that
// follows is unchanged.  O(beams) per orientation, where SMAD's window sums
// are O(intervals): the cost Remark 5 describes.
__device__ __forceinline__ void caer_hypothesis(const ReqDesc &d, int h, uint32_t *srow, int lane) {
    const int ns = d.ns, n = d.n_beams;
    const uint32_t *__restrict__ row = d.scan_table + (size_t)h * ns;
    for (int j = lane; j < ns; j += 32) srow[j] = __ldg(row + j);
    __syncwarp();
    const int32_t *__restrict__ b = d.b;
    const int32_t *__restrict__ Rq = d.Rall;
    unsigned long long best = ~0ull;
    for (int q = 0; q < d.n_m; ++q) {
        const int m = q * d.n_enum;
        unsigned long long e = 0;
        for (int i = lane; i < n; i += 32) {
            int j = __ldg(b + i) + m;
            if (j >= ns) j -= ns;
            const int diff = __ldg(Rq + i) - (int)srow[j];   // both in [0, 2^31)
            e += (unsigned)(diff < 0 ? -diff : diff);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
        const unsigned long long key = (e << 20) | (unsigned)q;
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

// shared memory of one SMAD warp: in-chunk prefixes [ns_pad + 32] and chunk prefixes [ns_pad / 32 + 1]
__host__ __device__ __forceinline__ size_t smad_warp_bytes(int ns_pad) {
    return (((size_t)(ns_pad + 32) * 4 + 7) & ~(size_t)7) + (size_t)(ns_pad / 32 + 1) * 8;
}

// Casting.  The batch's rays form one list of work items (request r owns
// items [chunk_base_r, chunk_base_r + ceil(n_hyp_r / G) * N_s_pad / 32), G =
// cast_hyps hypotheses for one chunk of 32 directions each, hypothesis group
// by hypothesis group); every warp takes items from a device counter until
// none is left, casts its 32 neighbouring directions (lane = ray) from each
// of the item's hypotheses in turn (the directions' setup is shared) and
// writes their ranges into the request's scan table, 128 contiguous bytes per
// hypothesis.  No
// warp waits for another, so long and short rays, hypotheses and requests
// mix freely across the GPU.
constexpr int kCastThreads = 256;

template <int G>
__global__ void __launch_bounds__(kCastThreads, 5) k_cast(const ReqDesc *__restrict__ reqs, int R, int total_chunks,
                                                       BatchState *bs) {
    __shared__ int s_base[kMaxBatchRequests + 1];
    const int lane = threadIdx.x & 31;
    // first the scan preparation, which the later stages need and the cast does
    // not: every CTA fills its share of the TAM scores, CTA r prepares request r
    for (int r = 0; r < R; ++r) scan_prep_fill(reqs[r], blockIdx.x, gridDim.x);
    if ((int)blockIdx.x < R) scan_prep_request(reqs[blockIdx.x]);
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].chunk_base;
    if (threadIdx.x == 0) s_base[R] = total_chunks;
    __syncthreads();
    unsigned long long my_steps = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&bs->cast_work, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= total_chunks) break;
        int lo = 0, hi = R - 1;   // last request whose chunk_base <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_base[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const ReqDesc &d = reqs[lo];
        const int local = g - s_base[lo];
        const int nhc = (d.n_hyp + G - 1) / G;   // items per direction chunk (G = d.cast_hyps)
        const int jc = local / nhc;   // hypothesis-minor: concurrent warps share 32 directions' tables
        const int h0 = (local - jc * nhc) * G, h1 = min(h0 + G, d.n_hyp);
        const int j = (jc << 5) + lane;
        if (j < d.ns) {
            const int2 dir = d.D[j];
            for (int h = h0; h < h1; ++h) {
                const int2 hc = d.hyps[h];
                int hit, steps = 0;
                const uint32_t r = d.rt.mask ? walk_ray(d.bits, d.reach, d.W, d.H, d.TW, d.TH, d.rt, d.ns, j, hc.x, hc.y,
                                                        dir, &hit, &steps)
                                             : cast_ray(d.bits, d.W, d.H, d.TW, d.lim, hc.x, hc.y, dir, &hit, &steps);
                d.scan_table[(size_t)h * d.ns + j] = r;
                my_steps += (unsigned)steps;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(kFull, my_steps, o);
    if (lane == 0 && my_steps) atomicAdd(&bs->dda_steps, my_steps);
}

constexpr int kSmadLoads = 16;   // 32-range chunks a SMAD warp has in flight

// SMAD.  One warp per hypothesis, taken from a device counter over the
// batch's hypothesis list (request r owns slots [hyp_base_r, hyp_base_r +
// n_hyp_r)).  The warp reads the hypothesis's N_s ranges 32 at a time,
// scans each chunk with shuffles into exclusive in-chunk prefixes and carries
// the 64-bit chunk prefix; P(t) = chunkP[t / 32] + inner[t] is then the cyclic
// prefix sum of Eq. 17 for t in [0, N_s].  The lanes split the orientations,
// evaluate Eq. 18-19 per m and reduce the minimum (Eq. 20).  With a single
// orientation (m = 0) the warp sums the row over the FoV intervals directly.
// No CTA barrier: each warp owns its slice of shared memory.
__global__ void __launch_bounds__(256) k_smad(const ReqDesc *__restrict__ reqs, int R, int total_hyp,
                                              BatchState *bs, int warp_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_base[kMaxBatchRequests + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].hyp_base;
    if (threadIdx.x == 0) s_base[R] = total_hyp;
    __syncthreads();
    unsigned char *mine = smem + (size_t)warp * warp_bytes;
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
        const int h = g - s_base[lo];
        const int ns = d.ns, ns_pad = d.ns_pad, nch = ns_pad >> 5;
        if (d.coarse == kCoarseCaer) {
            caer_hypothesis(d, h, reinterpret_cast<uint32_t *>(mine), lane);
            continue;
        }
        const uint32_t *__restrict__ row = d.scan_table + (size_t)h * ns;
        if (d.n_m == 1) {
            // a single orientation, m = 0 (Eq. 20 when lambda >= 0.9): W_0 is the row summed over the FoV
            // intervals, read once and coalesced; no prefixes are needed
            long long w = 0;
            for (int k = 0; k < d.n_iv; ++k) {
                const int2 iv = d.iv[k];
                for (int t = lane; t < iv.y; t += 32) {
                    int j = iv.x + t;
                    if (j >= ns) j -= ns;
                    w += __ldg(row + j);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            if (lane == 0) {
                long long dnum = d.scan->sum_real - w;
                if (dnum < 0) dnum = -dnum;
                d.keys[h] = ((unsigned long long)dnum << kHypBits) | (unsigned long long)h;
                d.smad_num[h] = dnum;
                d.smad_m[h] = 0;
            }
            continue;
        }
        uint32_t *inner = reinterpret_cast<uint32_t *>(mine);
        long long *chunkP = reinterpret_cast<long long *>(mine + (((size_t)(ns_pad + 32) * 4 + 7) & ~(size_t)7));
        long long carry = 0;
        for (int c0 = 0; c0 < nch; c0 += kSmadLoads) {
            uint32_t r[kSmadLoads];
#pragma unroll
            for (int u = 0; u < kSmadLoads; ++u) {   // kSmadLoads loads in flight
                const int jj = ((c0 + u) << 5) + lane;
                r[u] = (c0 + u < nch && jj < ns) ? __ldg(row + jj) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kSmadLoads; ++u) {
                if (c0 + u >= nch) break;
                uint32_t sc = r[u];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, sc, o);
                    if (lane >= o) sc += t;
                }
                inner[((c0 + u) << 5) + lane] = sc - r[u];
                if (lane == 0) chunkP[c0 + u] = carry;
                carry += __shfl_sync(kFull, sc, 31);
            }
        }
        inner[ns_pad + lane] = 0u;   // P(t) for t in [ns_pad, ns_pad + 32) adds nothing
        if (lane == 0) chunkP[nch] = carry;
        __syncwarp();
        const long long sum_real = d.scan->sum_real;
        unsigned long long best = ~0ull;
        for (int q = lane; q < d.n_m; q += 32) {
            const int m = q * d.n_enum;
            long long Wm = 0;
            for (int k = 0; k < d.n_iv; ++k) {
                const int2 iv = d.iv[k];
                int s0 = iv.x + m;
                if (s0 >= ns) s0 -= ns;
                const int e = s0 + iv.y;
                const long long p0 = chunkP[s0 >> 5] + inner[s0];
                if (e <= ns) {
                    Wm += chunkP[e >> 5] + inner[e] - p0;
                } else {
                    const int e2 = e - ns;
                    Wm += (chunkP[ns >> 5] + inner[ns] - p0) + (chunkP[e2 >> 5] + inner[e2]);
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
            d.keys[h] = (num << kHypBits) | (unsigned long long)h;
            d.smad_num[h] = (long long)num;
            d.smad_m[h] = q * d.n_enum;
        }
        __syncwarp();   // the orientation reads are done before the next hypothesis rewrites the prefixes
    }
}

// Window tables.  k_win_build: one CTA per hypothesis of the build list.
// It scans the hypothesis's row into prefixes (as k_smad), evaluates W_m of
// Eq. 18 for every m of Theta, takes the SMAD minimum as k_smad does, and
// sorts the keys W_m << 13 | q ascending (bitonic, in shared memory) into the
// request's window table.
__device__ __forceinline__ int list_request(const int *s_base, int R, int g) {   // last request whose base <= g
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_win_build(const ReqDesc *__restrict__ reqs, int R, int total, int nm_pad_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_base[kMaxBatchRequests + 1];
    __shared__ unsigned long long s_best[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].wbuild_base;
    if (threadIdx.x == 0) s_base[R] = total;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem);   // [nm_pad_max]
    unsigned char *rest = smem + (size_t)nm_pad_max * 8;
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        __syncthreads();   // s_base ready; the previous hypothesis is done with shared memory
        const int r = list_request(s_base, R, g);
        const ReqDesc &d = reqs[r];
        const int h = g - s_base[r];
        const int ns = d.ns, ns_pad = d.ns_pad, nch = ns_pad >> 5, n_m = d.n_m;
        uint32_t *inner = reinterpret_cast<uint32_t *>(rest);
        long long *chunkP = reinterpret_cast<long long *>(rest + (((size_t)(ns_pad + 32) * 4 + 7) & ~(size_t)7));
        if (threadIdx.x < 32) inner[ns_pad + lane] = 0u;
        const uint32_t *__restrict__ row = d.scan_table + (size_t)h * ns;
        for (int c = warp; c < nch; c += nwarps) {
            const int jj = (c << 5) + lane;
            const uint32_t rv = jj < ns ? __ldg(row + jj) : 0u;
            uint32_t sc = rv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, sc, o);
                if (lane >= o) sc += t;
            }
            inner[jj] = sc - rv;
            if (lane == 31) chunkP[c + 1] = (long long)sc;
        }
        __syncthreads();
        if (warp == 0) {
            long long carry = 0;
            for (int c0 = 0; c0 < nch; c0 += 32) {
                const int c = c0 + lane;
                long long v = c < nch ? chunkP[c + 1] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long t = __shfl_up_sync(kFull, v, o);
                    if (lane >= o) v += t;
                }
                if (c < nch) chunkP[c + 1] = carry + v;
                carry += __shfl_sync(kFull, v, 31);
            }
            if (lane == 0) chunkP[0] = 0;
        }
        __syncthreads();
        int nm_pad = 1;
        while (nm_pad < n_m) nm_pad <<= 1;
        const long long sum_real = d.scan->sum_real;
        unsigned long long best = ~0ull;
        for (int q = threadIdx.x; q < nm_pad; q += blockDim.x) {
            if (q >= n_m) {
                keys[q] = ~0ull;
                continue;
            }
            const int m = q * d.n_enum;
            long long Wm = 0;
            for (int k = 0; k < d.n_iv; ++k) {
                const int2 iv = d.iv[k];
                int s0 = iv.x + m;
                if (s0 >= ns) s0 -= ns;
                const int e = s0 + iv.y;
                const long long p0 = chunkP[s0 >> 5] + inner[s0];
                if (e <= ns) {
                    Wm += chunkP[e >> 5] + inner[e] - p0;
                } else {
                    const int e2 = e - ns;
                    Wm += (chunkP[ns >> 5] + inner[ns] - p0) + (chunkP[e2 >> 5] + inner[e2]);
                }
            }
            keys[q] = ((unsigned long long)Wm << kWinQBits) | (unsigned)q;
            long long dnum = sum_real - Wm;
            if (dnum < 0) dnum = -dnum;
            const unsigned long long key = ((unsigned long long)dnum << 20) | (unsigned)q;
            best = key < best ? key : best;
        }
        best = warp_min_u64(best);
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = s_best[0];
            for (int w = 1; w < nwarps; ++w) b = s_best[w] < b ? s_best[w] : b;
            const unsigned long long num = b >> 20;
            const int q = (int)(b & 0xfffffu);
            d.keys[h] = (num << kHypBits) | (unsigned long long)h;
            d.smad_num[h] = (long long)num;
            d.smad_m[h] = q * d.n_enum;
        }
        // bitonic sort of the keys, ascending
        for (int k = 2; k <= nm_pad; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < nm_pad; i += blockDim.x) {
                    const int p = i ^ j;
                    if (p > i) {
                        const unsigned long long a = keys[i], b = keys[p];
                        if ((a > b) == ((i & k) == 0)) {
                            keys[i] = b;
                            keys[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        unsigned long long *out = d.win + (size_t)h * n_m;
        for (int i = threadIdx.x; i < n_m; i += blockDim.x) out[i] = keys[i];
    }
}

// k_win_read: one thread per hypothesis of the read list.  With S = sum
// R_real, the nearest W_m at or above S is the first key >= S << 13, and the
// nearest below is the key before it; each run of equal W_m starts with its
// smallest q, so the run start found by a second search is the smaller m of
// that value.  The closer of the two wins and a tie goes to the smaller m:
// exactly the minimum k_smad takes (Eq. 20).
__device__ __forceinline__ int lower_bound_u64(const unsigned long long *__restrict__ a, int n, unsigned long long x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_win_read(const ReqDesc *__restrict__ reqs, int R, int total) {
    __shared__ int s_base[kMaxBatchRequests + 1];
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_base[r] = reqs[r].wread_base;
    if (threadIdx.x == 0) s_base[R] = total;
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int r = list_request(s_base, R, g);
        const ReqDesc &d = reqs[r];
        const int h = g - s_base[r];
        const int n_m = d.n_m;
        const unsigned long long *keys = d.win + (size_t)h * n_m;
        const long long S = d.scan->sum_real;
        const unsigned long long qmask = (1ull << kWinQBits) - 1ull;
        const int pa = lower_bound_u64(keys, n_m, (unsigned long long)S << kWinQBits);
        long long dist = -1;
        unsigned q = 0;
        if (pa < n_m) {
            const unsigned long long ka = __ldg(keys + pa);
            dist = (long long)(ka >> kWinQBits) - S;
            q = (unsigned)(ka & qmask);
        }
        if (pa > 0) {
            const unsigned long long wb = __ldg(keys + pa - 1) >> kWinQBits;
            const long long db = S - (long long)wb;
            if (dist < 0 || db <= dist) {
                const int pb = lower_bound_u64(keys, pa - 1, wb << kWinQBits);   // start of the run of wb
                const unsigned qb = (unsigned)(__ldg(keys + pb) & qmask);
                if (dist < 0 || db < dist || qb < q) q = qb;
                dist = db;
            }
        }
        d.keys[h] = ((unsigned long long)dist << kHypBits) | (unsigned long long)h;
        d.smad_num[h] = dist;
        d.smad_m[h] = (int)q * d.n_enum;
    }
}

__global__ void __launch_bounds__(256) k_synth(RayArgs a, uint32_t *__restrict__ ranges, int32_t *__restrict__ hits) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= a.n_hyp) return;
    const int2 hc = a.hyps[warp];
    for (int j = lane; j < a.ns; j += 32) {
        int hit, steps;
        uint32_t r = a.tab.mask ? walk_ray(a.bits, a.reach, a.W, a.H, a.TW, a.TH, a.tab, a.ns, j, hc.x, hc.y, a.D[j],
                                           &hit, &steps)
                                : cast_ray(a.bits, a.W, a.H, a.TW, a.lim, hc.x, hc.y, a.D[j], &hit, &steps);
        ranges[(size_t)warp * a.ns + j] = r;
        if (hits) hits[(size_t)warp * a.ns + j] = hit;
    }
}

}  // namespace

cudaError_t launch_cast(const ReqDesc *reqs, int R, int total_chunks, int cast_hyps, BatchState *bs, int n_sm,
                        int ctas_per_sm, cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests) return cudaErrorInvalidValue;
    if (total_chunks <= 0) return cudaSuccess;
    // one instance per group size: a single hypothesis keeps the loop-free body
    void (*kern)(const ReqDesc *, int, int, BatchState *) =
        cast_hyps == 4 ? k_cast<4> : cast_hyps == 2 ? k_cast<2> : cast_hyps == 1 ? k_cast<1> : nullptr;
    if (!kern) return cudaErrorInvalidValue;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCastThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;   // a tuned launch shape
    const long long warps = (long long)total_chunks;
    long long grid = (long long)n_sm * occ;
    if (grid * (kCastThreads / 32) > warps) grid = (warps + kCastThreads / 32 - 1) / (kCastThreads / 32);
    if (grid < R) grid = R;   // one CTA per request for the scan preparation
    kern<<<(int)grid, kCastThreads, 0, s>>>(reqs, R, total_chunks, bs);
    return cudaGetLastError();
}

cudaError_t launch_smad(const ReqDesc *reqs, int R, int total_hyp, int max_ns_pad, BatchState *bs, int n_sm,
                        cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests) return cudaErrorInvalidValue;
    const size_t wb = smad_warp_bytes(max_ns_pad);
    // warps per CTA: the most resident warps per SM that shared memory allows
    // (a long row's scratch fills an SM before its thread limit; smaller CTAs
    // waste less of it), the larger CTA on ties
    cudaError_t e = cudaFuncSetAttribute(k_smad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::min((size_t)8 * wb, (size_t)200 * 1024));
    if (e != cudaSuccess) return e;
    int wpc = 0, occ = 0;
    for (int w = 8; w >= 1; --w) {
        if ((size_t)w * wb > (size_t)200 * 1024) continue;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_smad, w * 32, (size_t)w * wb);
        if (e != cudaSuccess) return e;
        if (o * w > occ * wpc) {
            wpc = w;
            occ = o;
        }
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)wpc * wb;
    long long grid = (long long)n_sm * occ;
    const long long need = ((long long)total_hyp + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_smad<<<(int)grid, wpc * 32, smem, s>>>(reqs, R, total_hyp, bs, (int)wb);
    return cudaGetLastError();
}

cudaError_t launch_win_build(const ReqDesc *reqs, int R, int total, int max_ns_pad, int max_nm, cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests) return cudaErrorInvalidValue;
    if (total <= 0) return cudaSuccess;
    int nm_pad = 1;
    while (nm_pad < max_nm) nm_pad <<= 1;
    const size_t smem = (size_t)nm_pad * 8 + (((size_t)(max_ns_pad + 32) * 4 + 7) & ~(size_t)7) +
                        (size_t)(max_ns_pad / 32 + 1) * 8;
    cudaError_t e = cudaFuncSetAttribute(k_win_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, n_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_win_build, 256, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = total < n_sm * occ ? total : n_sm * occ;
    k_win_build<<<grid, 256, smem, s>>>(reqs, R, total, nm_pad);
    return cudaGetLastError();
}

cudaError_t launch_win_read(const ReqDesc *reqs, int R, int total, cudaStream_t s) {
    if (R < 1 || R > kMaxBatchRequests) return cudaErrorInvalidValue;
    if (total <= 0) return cudaSuccess;
    k_win_read<<<(total + 255) / 256, 256, 0, s>>>(reqs, R, total);
    return cudaGetLastError();
}

cudaError_t launch_ray_tables(const int2 *D, int ns, int lim, uint64_t *mask, uint16_t *selx, uint16_t *sely,
                              int32_t *kmax, cudaStream_t s) {
    const size_t rows_m = (size_t)ray_mask_rows(lim), rows_s = (size_t)ray_sel_rows(lim);
    cudaError_t e = cudaMemsetAsync(mask, 0, sizeof(uint64_t) * rows_m * ns, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(selx, 0xff, sizeof(uint16_t) * rows_s * ns, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sely, 0xff, sizeof(uint16_t) * rows_s * ns, s);
    if (e != cudaSuccess) return e;
    k_ray_tables<<<(ns + 127) / 128, 128, 0, s>>>(D, ns, lim, mask, selx, sely, kmax);
    return cudaGetLastError();
}

cudaError_t launch_synth(const RayArgs &a, uint32_t *ranges, int32_t *hit, cudaStream_t s) {
    if (a.n_hyp <= 0) return cudaSuccess;
    int blocks = (a.n_hyp * 32 + 255) / 256;
    k_synth<<<blocks, 256, 0, s>>>(a, ranges, hit);
    return cudaGetLastError();
}

}  // namespace relo
