// Map precompute: exact squared Euclidean distance transform (the EDT lookup
// table of Sec. III-A item 3, used by the likelihood field of Eq. 23 and the
// distance statistics of Eq. 29-30), its clamped padded copy for TAM, and the
// tiled occupancy bitmap for ray casting (Eq. 13) with, per walk frame, the
// empty squares of tiles ahead of every tile.
//
// The clamped field is stored in bands of 8 rows (field_index) with a border
// of P cells holding C on every side, P at least the longest beam in cells, so
// every beam endpoint of TAM falls inside the array and needs no bounds test.
//
// d2(x, y) = min over occupied (x', y') of (x - x')^2 + (y - y')^2 separates
// into a column term g2(x', y) = min over occupied y' in column x' of
// (y - y')^2 and a row minimisation d2(x, y) = min over x' of (x - x')^2 +
// g2(x', y).  The column term comes from two sweeps per column (coalesced
// across columns); the row minimisation stages one row in shared memory and
// each thread scans outward from its cell, stopping once (x - x')^2 alone
// reaches the best value found, which no further column can beat.
#include <cuda_runtime.h>
#include <stdint.h>

#include "relo_internal.h"

namespace relo {

namespace {

constexpr int kInf = 0x7fffffff;

// Column term, step 1: for every (column, segment of L rows) the first and the
// last occupied row inside the segment (-1 if none).  The same pass builds the
// occupancy bitmaps: a warp covers 32 consecutive columns (four 8x8 tiles) and
// L is a multiple of 8, so the ballot of each row gives four tile rows, which
// lanes 0-3 collect into their tile's word (cells outside the map are free).
// The word is stored as is, and, with the cells outside the map set, into the
// four walk frames: as is, and mirrored in x (x' = 8 TW - 1 - x: tile TW - 1 -
// tx, bits reversed within each row), in y (rows reversed) and in both (all 64
// bits reversed), which the ray cast uses so that every ray travels towards +x
// and +y.
__global__ void k_edt_col_summary(const int8_t *__restrict__ grid, int W, int H, int L, int TW, int TH,
                                  int2 *__restrict__ summ, uint64_t *__restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int x0 = x - lane;
    const int sgm = blockIdx.y;
    if (x0 >= W) return;   // the whole warp lies right of the map
    const int y0 = sgm * L;
    int first = -1, last = -1;
    // a tile row (8 grid rows; L and y0 are multiples of 8) at a time, its 8 loads issued together
    for (int yb = y0; yb < y0 + L; yb += 8) {
        bool occ8[8], in8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            in8[u] = x < W && yb + u < H;
            occ8[u] = in8[u] && grid[(size_t)(yb + u) * W + x] >= 65;
        }
        uint64_t word = 0ull, wword = 0ull;   // the map's word; the walk frames' word (outside cells set)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (occ8[u]) {
                if (first < 0) first = yb + u;
                last = yb + u;
            }
            const unsigned b = __ballot_sync(0xffffffffu, occ8[u]);
            const unsigned bw = __ballot_sync(0xffffffffu, occ8[u] || !in8[u]);
            word |= (uint64_t)((b >> (8 * (lane & 3))) & 0xffu) << (8 * u);
            wword |= (uint64_t)((bw >> (8 * (lane & 3))) & 0xffu) << (8 * u);
        }
        const int tx = (x0 >> 3) + lane, ty = yb >> 3;
        if (lane < 4 && tx < TW && ty < TH) {
            const size_t WB = (size_t)TW + 1, n = walk_frame_words(TW, TH);
            uint64_t *wf = bits + (size_t)TW * TH;
            const uint64_t rev = __brevll(wword);   // both mirrors
            const uint64_t ymir = ((uint64_t)__byte_perm((uint32_t)wword, 0u, 0x0123u) << 32) |
                                  (uint64_t)__byte_perm((uint32_t)(wword >> 32), 0u, 0x0123u);
            const uint64_t xmir = ((uint64_t)__byte_perm((uint32_t)rev, 0u, 0x0123u) << 32) |
                                  (uint64_t)__byte_perm((uint32_t)(rev >> 32), 0u, 0x0123u);
            bits[(size_t)ty * TW + tx] = word;
            wf[(size_t)ty * WB + tx] = wword;
            wf[n + (size_t)ty * WB + (TW - 1 - tx)] = xmir;
            wf[2 * n + (size_t)(TH - 1 - ty) * WB + tx] = ymir;
            wf[3 * n + (size_t)(TH - 1 - ty) * WB + (TW - 1 - tx)] = rev;
        }
    }
    if (x < W) summ[(size_t)sgm * W + x] = make_int2(first, last);
}

// Column term, step 2: the nearest occupied rows above and below the segment
// come from the other segments' summaries; one downward and one upward sweep
// inside the segment then give g(x, y) = distance to the nearest occupied
// cell of the column, stored squared (kInf when the column has none).
__global__ void k_edt_col_final(const int8_t *__restrict__ grid, int W, int H, int L, int S,
                                const int2 *__restrict__ summ, int32_t *__restrict__ colsq) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int sgm = blockIdx.y;
    if (x >= W) return;
    int last = -1;    // nearest occupied row above the segment
    for (int t = 0; t < sgm; ++t) {
        const int v = summ[(size_t)t * W + x].y;
        if (v >= 0) last = v;
    }
    int next = -1;    // nearest occupied row below the segment
    for (int t = S - 1; t > sgm; --t) {
        const int v = summ[(size_t)t * W + x].x;
        if (v >= 0) next = v;
    }
    const int y0 = sgm * L, y1 = min(H, y0 + L);
    for (int y = y0; y < y1; ++y) {
        const size_t i = (size_t)y * W + x;
        if (grid[i] >= 65) last = y;
        colsq[i] = last < 0 ? kInf : y - last;
    }
    for (int y = y1 - 1; y >= y0; --y) {
        const size_t i = (size_t)y * W + x;
        if (grid[i] >= 65) next = y;
        const int up = colsq[i];
        const int dn = next < 0 ? kInf : next - y;
        const int g = up < dn ? up : dn;
        colsq[i] = g == kInf ? kInf : g * g;
    }
}

// The row is staged with W + 4 cells of sentinel on each side and "no
// obstacle in this column" as the same sentinel, a value larger than any
// squared distance that still leaves room for dx^2, so the outward scan needs
// no bounds or sentinel tests: a sentinel never improves the minimum.  The
// scan takes four distances per step (their loads independent of each other),
// so a cell waits on a shared-memory round trip once per four columns; the up
// to three columns it looks at beyond the stopping distance are ordinary
// candidates and leave the minimum exact.
constexpr int kRowSentinel = 0x3fffffff;
constexpr int kRowPad = 4;   // the scan's step, and the extra sentinels it may read past the row's reach

__global__ void k_edt_rows(const int32_t *__restrict__ colsq, int W, int C, int P, int Wp, int32_t *__restrict__ d2,
                           uint16_t *__restrict__ field) {
    extern __shared__ int32_t rowbuf[];   // [3W + 2 kRowPad]: sentinels, the row, sentinels
    int32_t *row = rowbuf + W + kRowPad;
    const int y = blockIdx.x;
    const int32_t *src = colsq + (size_t)y * W;
    for (int x = threadIdx.x; x < W + kRowPad; x += blockDim.x) {
        rowbuf[x] = kRowSentinel;
        row[W + x] = kRowSentinel;
    }
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int v = src[x];
        row[x] = v == kInf ? kRowSentinel : v;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        int best = row[x];
        const int reach = x > W - 1 - x ? x : W - 1 - x;   // past this both sides are sentinels
        for (int dx = 1; dx <= reach && dx * dx < best; dx += kRowPad) {
            const int a = min(row[x - dx], row[x + dx]) + dx * dx;
            const int b = min(row[x - dx - 1], row[x + dx + 1]) + (dx + 1) * (dx + 1);
            const int c = min(row[x - dx - 2], row[x + dx + 2]) + (dx + 2) * (dx + 2);
            const int e4 = min(row[x - dx - 3], row[x + dx + 3]) + (dx + 3) * (dx + 3);
            best = min(best, min(min(a, b), min(c, e4)));
        }
        d2[(size_t)y * W + x] = best >= kRowSentinel ? kD2None : best;
        field[field_index(x + P, y + P, Wp)] = (uint16_t)(best > C ? C : best);
    }
}

// the border of the padded field: every cell outside the map reads C (d = d_max)
__global__ void k_field_border(uint16_t *__restrict__ fieldp, int W, int H, int P, int Wp, int Hp, int C) {
    const size_t n = (size_t)Hp * Wp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t c = i >> 3;   // column of a band, then the row inside the band (field_index)
        const int y = (int)(c / Wp) * 8 + (int)(i & 7) - P, x = (int)(c % Wp) - P;
        if (x < 0 || y < 0 || x >= W || y >= H) fieldp[i] = (uint16_t)C;
    }
}

// Which walk-frame tiles are empty, one bit per tile: word [row][k] of a
// frame row holds tiles 32 k .. 32 k + 31 (tiles past the row count as not
// empty, and one more word of zeros ends every row).
__global__ void k_walk_empty(const uint64_t *__restrict__ wf, int TW, uint32_t *__restrict__ emp) {
    const unsigned WB = (unsigned)TW + 1u, SW = walk_empty_row_words(TW);
    const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t row = blockIdx.y;   // frame * (TH + 1) + ty
    const unsigned bal = __ballot_sync(0xffffffffu, x < WB && wf[row * WB + x] == 0ull);
    if ((threadIdx.x & 31) == 0 && (x >> 5) < SW) emp[row * SW + (x >> 5)] = bal;
}

// The empty boxes ahead of every walk-frame tile (MapDev::reach).  A warp
// takes 32 tiles of a row: lanes k < kReachMax load the emptiness word of row
// ty + k covering its tiles and lanes kReachMax + k the next word.  For each
// of the kReachMax rows from theirs, a lane shifts the 64 bits of that pair
// down by its own position, so bit i says whether the tile i to its right is
// empty (i + 31 < 64: a window of kReachMax + 1 bits always fits).  Its row
// run is the block of set bits from bit 0 of the first row, its column run
// the rows that keep bit 0, and its square the largest s whose s rows' AND
// keeps bits 0 .. s - 1.
__global__ void k_walk_reach(const uint32_t *__restrict__ emp, int TW, int TH, uint16_t *__restrict__ reach) {
    static_assert(2 * kReachMax <= 32, "one emptiness word per lane");
    const int lane = threadIdx.x & 31;
    const unsigned WB = (unsigned)TW + 1u, HB = (unsigned)TH + 1u, SW = walk_empty_row_words(TW);
    const unsigned strip = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (strip * 32u >= WB) return;   // the whole warp lies past the row
    const unsigned fy = blockIdx.y, ty = fy % HB;   // frame * HB + ty
    const unsigned k = (unsigned)lane % kReachMax, y = ty + k;
    const uint32_t wv = y < HB ? emp[(size_t)(fy + k) * SW + strip + lane / kReachMax] : 0u;
    uint32_t e0 = 0u, a = ~0u;
    int s = 0, yr = 0;
    bool sq = true, col = true;
#pragma unroll
    for (int r = 0; r < kReachMax; ++r) {
        const uint32_t e = __funnelshift_r(__shfl_sync(0xffffffffu, wv, r),
                                           __shfl_sync(0xffffffffu, wv, r + kReachMax), (unsigned)lane);
        if (r == 0) e0 = e;
        col = col && (e & 1u);
        if (col) yr = r + 1;
        a &= e;
        const uint32_t mr = (2u << r) - 1u;   // bits 0 .. r
        sq = sq && (a & mr) == mr;
        if (sq) s = r + 1;
        if (!__any_sync(0xffffffffu, sq || col)) break;   // no lane's boxes grow further
    }
    // the sentinel bit caps the row run at kReachMax
    const int xr = __ffs((int)(~e0 | (1u << kReachMax))) - 1;
    const unsigned xa = strip * 32u + lane;
    if (xa < WB) reach[(size_t)fy * WB + xa] = (uint16_t)(s | (xr << 5) | (yr << 10));
}

// the last column and row of tiles of each walk frame: every bit set
__global__ void k_walk_border(uint64_t *__restrict__ wf, int TW, int TH) {
    uint64_t *f = wf + (size_t)blockIdx.x * walk_frame_words(TW, TH);
    const int WB = TW + 1;
    for (int i = threadIdx.x; i <= TH; i += blockDim.x) f[(size_t)i * WB + TW] = ~0ull;
    for (int i = threadIdx.x; i < TW; i += blockDim.x) f[(size_t)TH * WB + i] = ~0ull;
}

__global__ void k_map_tables(const int32_t *__restrict__ d2s, const uint16_t *__restrict__ fs,
                             const uint64_t *__restrict__ bs, int W, int H, int TW, int P, int Wp, int32_t *d2,
                             uint16_t *field,
                             uint8_t *occ) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)W * H) return;
    int x = (int)(i % W), y = (int)(i / W);
    if (d2) d2[i] = d2s[i];
    if (field) field[i] = fs[field_index(x + P, y + P, Wp)];
    if (occ) occ[i] = (uint8_t)((bs[(size_t)(y >> 3) * TW + (x >> 3)] >> (((y & 7) << 3) | (x & 7))) & 1ull);
}

__global__ void k_check_cells(const int2 *__restrict__ cells, int n, const uint64_t *__restrict__ bits, int W,
                              int H, int TW, int *bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 c = cells[i];
    bool ok = (unsigned)c.x < (unsigned)W && (unsigned)c.y < (unsigned)H;
    if (ok) ok = !((bits[(size_t)(c.y >> 3) * TW + (c.x >> 3)] >> (((c.y & 7) << 3) | (c.x & 7))) & 1ull);
    if (!ok) atomicAdd(bad, 1);
}

// Hypotheses given in metres (Eq. 6): the containing cell (floor((x - ox) /
// res), floor((y - oy) / res)) in FP64, each operation rounded as IEEE
// prescribes, so the cells equal those of the same expression on the host.
// flags[0] counts points off the map (or not finite), flags[1] points on
// occupied cells; an off-map point's cell is written as (0, 0).
__global__ void k_xy_cells(const double2 *__restrict__ xy, int n, double ox, double oy, double res,
                           const uint64_t *__restrict__ bits, int W, int H, int TW, int2 *__restrict__ cells,
                           int *flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 p = xy[i];
    const double fx = floor((p.x - ox) / res), fy = floor((p.y - oy) / res);
    if (!(fx >= 0.0 && fy >= 0.0 && fx < (double)W && fy < (double)H)) {
        cells[i] = make_int2(0, 0);
        atomicAdd(flags, 1);
        return;
    }
    const int cx = (int)fx, cy = (int)fy;
    cells[i] = make_int2(cx, cy);
    if ((bits[(size_t)(cy >> 3) * TW + (cx >> 3)] >> (((cy & 7) << 3) | (cx & 7))) & 1ull) atomicAdd(flags + 1, 1);
}

}  // namespace

cudaError_t launch_xy_cells(const double *xy, int n, double ox, double oy, double res, const MapDev &m, int2 *cells,
                            int *flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_xy_cells<<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const double2 *>(xy), n, ox, oy, res, m.bits, m.W,
                                               m.H, m.TW, cells, flags);
    return cudaGetLastError();
}

cudaError_t launch_edt_tiles(const MapDev &m, cudaStream_t s) {
    const int L = edt_segment_rows(m.H), S = (m.H + L - 1) / L;
    const dim3 cgrid((m.W + 127) / 128, S);
    k_edt_col_summary<<<cgrid, 128, 0, s>>>(m.grid, m.W, m.H, L, m.TW, m.TH, m.summ, m.bits);
    if (m.reach) {
        // the walk frames' empty boxes (their border tiles, full, were written when the map was loaded)
        const unsigned WB = (unsigned)m.TW + 1u, SW = walk_empty_row_words(m.TW), rows = 4u * ((unsigned)m.TH + 1u);
        uint32_t *emp = walk_empty_bits(m.reach, m.TW, m.TH);
        k_walk_empty<<<dim3((32u * SW + 255u) / 256u, rows), 256, 0, s>>>(m.bits + (size_t)m.TW * m.TH, m.TW, emp);
        k_walk_reach<<<dim3((WB + 255u) / 256u, rows), 256, 0, s>>>(emp, m.TW, m.TH, m.reach);
    }
    return cudaGetLastError();
}

cudaError_t launch_edt_field(const MapDev &m, cudaStream_t s) {
    const int L = edt_segment_rows(m.H), S = (m.H + L - 1) / L;
    const dim3 cgrid((m.W + 127) / 128, S);
    k_edt_col_final<<<cgrid, 128, 0, s>>>(m.grid, m.W, m.H, L, S, m.summ, m.colsq);
    size_t smem = ((size_t)3 * m.W + 2 * kRowPad) * sizeof(int32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // 512 threads: shared memory admits 4 rows of 49 KB per SM at W = 4096, and 16 warps each fill all 64 warp
    // slots (256 threads left half of them empty: 171 -> 148 us per warehouse launch)
    k_edt_rows<<<m.H, 512, smem, s>>>(m.colsq, m.W, m.C, m.P, m.Wp, m.d2, m.field);
    return cudaGetLastError();
}

cudaError_t launch_edt(const MapDev &m, cudaStream_t s) {
    cudaError_t e = launch_edt_tiles(m, s);
    return e == cudaSuccess ? launch_edt_field(m, s) : e;
}

cudaError_t launch_field_border(const MapDev &m, cudaStream_t s) {
    k_field_border<<<1024, 256, 0, s>>>(m.field, m.W, m.H, m.P, m.Wp, m.Hp, m.C);
    k_walk_border<<<4, 256, 0, s>>>(m.bits + (size_t)m.TW * m.TH, m.TW, m.TH);
    return cudaGetLastError();
}

cudaError_t launch_map_tables(const MapDev &m, int32_t *d2, uint16_t *field, uint8_t *occ, cudaStream_t s) {
    size_t n = (size_t)m.W * m.H;
    k_map_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m.d2, m.field, m.bits, m.W, m.H, m.TW, m.P, m.Wp, d2, field,
                                                             occ);
    return cudaGetLastError();
}

cudaError_t launch_check_cells(const int2 *cells, int n, const MapDev &m, int *bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_check_cells<<<(n + 255) / 256, 256, 0, s>>>(cells, n, m.bits, m.W, m.H, m.TW, bad);
    return cudaGetLastError();
}

}  // namespace relo
