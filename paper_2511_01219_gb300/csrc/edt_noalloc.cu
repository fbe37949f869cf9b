// relo_edt_noalloc: the exact squared EDT of a grid, for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all once they are running: a
// robot's real-time localisation loop that only allocates at start-up
// (a device allocation can block inside the driver for an unbounded time),
// or a host framework that owns every byte of device memory through its own
// pool and forbids raw allocations by the libraries it loads.  This entry
// point lets them compute the EDT lookup table with memory they already own:
// the caller passes the grid and the output, and the only scratch, the column
// distances and the column-segment summaries, lives in file-scope __device__
// arrays of a fixed maximum size.
//
// Consequences, stated for the user:
//   - Maps up to kNoAllocMaxSide x kNoAllocMaxSide cells (1024 x 1024) are
//     accepted; larger ones are rejected with RELO_E_INVALID_ARG.
//   - Every GPU that loads the library holds the scratch (4.5 MiB) until the
//     process exits.
//   - The first call on a device looks up the scratch's device address with
//     that device current; make that first call before any stream capture.
//     The address is kept for the life of the process: after cudaDeviceReset
//     (or any reset of the device's primary context) the module, and with it
//     the scratch, is gone, so do not call this entry point on that device
//     again in the same process.
//   - A CUDA error already pending in the calling thread (left by earlier
//     work) is reported as RELO_E_CUDA before anything is launched, and is
//     left in place for its owner; each of the three launches is checked on
//     its own, and a failed launch stops the call.
//   - All calls on one device share the scratch: calls whose work overlaps on
//     the GPU (for example on two streams at once) race and give wrong
//     results.  Each call overwrites every scratch element it reads, so
//     nothing has to start at zero and no clearing is needed.
//   - No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/relo.h"

namespace {

constexpr int kNoAllocMaxSide = 1024;
constexpr int kNoAllocSegRows = 16;                        // rows per column segment
constexpr int kNoAllocMaxSegs = kNoAllocMaxSide / kNoAllocSegRows;
constexpr int kInf = 0x7fffffff;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t g_colsq[kNoAllocMaxSide * kNoAllocMaxSide];
static __device__ __align__(256) int2 g_summ[kNoAllocMaxSegs * kNoAllocMaxSide];

std::mutex g_mu;
int32_t *g_colsq_addr[kMaxDevices] = {nullptr};
int2 *g_summ_addr[kMaxDevices] = {nullptr};

// first and last occupied row of every (column, segment)
__global__ void k_na_summary(const int8_t *__restrict__ grid, int W, int H, int2 *__restrict__ summ) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int sgm = blockIdx.y;
    if (x >= W) return;
    const int y0 = sgm * kNoAllocSegRows, y1 = min(H, y0 + kNoAllocSegRows);
    int first = -1, last = -1;
    for (int y = y0; y < y1; ++y)
        if (grid[(size_t)y * W + x] >= 65) {
            if (first < 0) first = y;
            last = y;
        }
    summ[(size_t)sgm * W + x] = make_int2(first, last);
}

// squared distance to the nearest occupied cell of the same column
__global__ void k_na_columns(const int8_t *__restrict__ grid, int W, int H, int S, const int2 *__restrict__ summ,
                             int32_t *__restrict__ colsq) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int sgm = blockIdx.y;
    if (x >= W) return;
    int last = -1, next = -1;
    for (int t = 0; t < sgm; ++t) {
        const int v = summ[(size_t)t * W + x].y;
        if (v >= 0) last = v;
    }
    for (int t = S - 1; t > sgm; --t) {
        const int v = summ[(size_t)t * W + x].x;
        if (v >= 0) next = v;
    }
    const int y0 = sgm * kNoAllocSegRows, y1 = min(H, y0 + kNoAllocSegRows);
    for (int y = y0; y < y1; ++y) {
        const size_t i = (size_t)y * W + x;
        if (grid[i] >= 65) last = y;
        colsq[i] = last < 0 ? kInf : y - last;
    }
    for (int y = y1 - 1; y >= y0; --y) {
        const size_t i = (size_t)y * W + x;
        if (grid[i] >= 65) next = y;
        const int up = colsq[i], dn = next < 0 ? kInf : next - y;
        const int g = up < dn ? up : dn;
        colsq[i] = g == kInf ? kInf : g * g;
    }
}

// d2(x, y) = min over x' of (x - x')^2 + colsq(x', y), scanning outward from x
__global__ void k_na_rows(const int32_t *__restrict__ colsq, int W, int32_t *__restrict__ d2) {
    extern __shared__ int32_t row[];
    const int y = blockIdx.x;
    for (int x = threadIdx.x; x < W; x += blockDim.x) row[x] = colsq[(size_t)y * W + x];
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        int best = row[x];
        for (int dx = 1; (long long)dx * dx < best; ++dx) {
            const int xl = x - dx, xr = x + dx;
            if (xl < 0 && xr >= W) break;
            if (xl >= 0 && row[xl] != kInf && row[xl] + dx * dx < best) best = row[xl] + dx * dx;
            if (xr < W && row[xr] != kInf && row[xr] + dx * dx < best) best = row[xr] + dx * dx;
        }
        d2[(size_t)y * W + x] = best == kInf ? -1 : best;
    }
}

// device addresses of the scratch arrays for the current device (looked up once per device)
cudaError_t scratch_for_current_device(int32_t **colsq, int2 **summ) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_colsq_addr[dev]) {
        void *p = nullptr, *q = nullptr;
        e = cudaGetSymbolAddress(&p, g_colsq);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&q, g_summ);
        if (e != cudaSuccess) return e;
        g_colsq_addr[dev] = static_cast<int32_t *>(p);
        g_summ_addr[dev] = static_cast<int2 *>(q);
    }
    *colsq = g_colsq_addr[dev];
    *summ = g_summ_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int relo_edt_noalloc(const int8_t *grid_dev, int32_t w, int32_t h, int32_t *d2_dev, void *stream) {
    if (!grid_dev || !d2_dev || w < 1 || h < 1) return RELO_E_INVALID_ARG;
    if (w > kNoAllocMaxSide || h > kNoAllocMaxSide) return RELO_E_INVALID_ARG;
    int32_t *colsq = nullptr;
    int2 *summ = nullptr;
    if (scratch_for_current_device(&colsq, &summ) != cudaSuccess) return RELO_E_CUDA;
    // an error left by the caller's own earlier work: report it, launch nothing, leave it pending
    if (cudaPeekAtLastError() != cudaSuccess) return RELO_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int S = (h + kNoAllocSegRows - 1) / kNoAllocSegRows;
    const dim3 grid((w + 127) / 128, S);
    k_na_summary<<<grid, 128, 0, s>>>(grid_dev, w, h, summ);
    if (cudaGetLastError() != cudaSuccess) return RELO_E_CUDA;
    k_na_columns<<<grid, 128, 0, s>>>(grid_dev, w, h, S, summ, colsq);
    if (cudaGetLastError() != cudaSuccess) return RELO_E_CUDA;
    k_na_rows<<<h, 256, (size_t)w * sizeof(int32_t), s>>>(colsq, w, d2_dev);
    if (cudaGetLastError() != cudaSuccess) return RELO_E_CUDA;
    return RELO_OK;
}
