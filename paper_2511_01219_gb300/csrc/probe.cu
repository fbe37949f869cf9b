// L2 bandwidth probes: the denominators of the scoring kernels' L2 roofline.
//
// The field TAM gathers from (a few to 56 MB of uint16) and the synthesized
// ranges SMAD streams (4 B per hypothesis and direction, written just before
// by the ray cast) live in the 126 MB L2, so HBM copy bandwidth does not bound
// either kernel.  These two kernels measure what does, on this GPU:
//   k_probe_stream  every SM reads an L2-resident buffer with 16-byte loads,
//                   four in flight per thread (the streaming L2 read rate);
//   k_probe_gather  every thread makes independent 2-byte loads at uniformly
//                   random positions of an L2-resident uint16 array, eight in
//                   flight (the random gather rate, one 32-byte sector per
//                   load: the rate a gather with no locality can reach).
// Each thread folds what it read into a value that is stored only when it
// equals a constant no input produces, so no load can be dropped and nothing
// is written.  The paper has no counterpart; the bench reports the two rates
// beside the kernels' achieved rates.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/relo.h"

namespace {

__device__ unsigned int g_probe_sink;
constexpr unsigned int kNever = 0x9e3779b9u;

__global__ void __launch_bounds__(256) k_probe_stream(const int4 *__restrict__ buf, long long n16, int passes) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int acc = 0;
    for (int p = 0; p < passes; ++p) {
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const int4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                       d = __ldcg(buf + i + 3 * stride);
            acc ^= (unsigned)(a.x ^ a.y ^ a.z ^ a.w) + (unsigned)(b.x ^ b.y ^ b.z ^ b.w) +
                   (unsigned)(c.x ^ c.y ^ c.z ^ c.w) + (unsigned)(d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n16; i += stride) {
            const int4 a = __ldcg(buf + i);
            acc ^= (unsigned)(a.x ^ a.y ^ a.z ^ a.w);
        }
    }
    if (acc == kNever) g_probe_sink = acc;
}

// positions from eight independent 32-bit linear congruential streams per
// thread (Numerical Recipes constants); the top bits index the array
__global__ void __launch_bounds__(256) k_probe_gather(const uint16_t *__restrict__ buf, int log2_n, int rounds) {
    const unsigned int tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (tid * 8u + (unsigned)j) * 2654435761u + 12345u;
    const int sh = 32 - log2_n;
    unsigned int acc = 0;
    for (int r = 0; r < rounds; ++r) {
        unsigned int v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x[j] = x[j] * 1664525u + 1013904223u;
            v[j] = __ldg(buf + (x[j] >> sh));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) acc += v[j];
    }
    if (acc == kNever) g_probe_sink = acc;
}

int probe_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

template <typename F>
int timed(cudaStream_t s, F &&launch, float *ms) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return RELO_E_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return RELO_E_CUDA;
    }
    cudaError_t e = cudaEventRecord(a, s);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e == cudaSuccess ? RELO_OK : RELO_E_CUDA;
}

}  // namespace

extern "C" int relo_probe_l2_stream(const void *buf_dev, int64_t bytes, int32_t passes, void *stream, float *ms) {
    if (!buf_dev || !ms || bytes < 16 || (bytes & 15) || ((uintptr_t)buf_dev & 15) || passes < 1)
        return RELO_E_INVALID_ARG;
    const int n_sm = probe_sms();
    if (n_sm < 1) return RELO_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int4 *buf = static_cast<const int4 *>(buf_dev);
    const long long n16 = bytes / 16;
    const int grid = n_sm * 8;
    k_probe_stream<<<grid, 256, 0, s>>>(buf, n16, 1);   // brings the buffer into L2
    if (cudaGetLastError() != cudaSuccess) return RELO_E_CUDA;
    return timed(s, [&] { k_probe_stream<<<grid, 256, 0, s>>>(buf, n16, passes); }, ms);
}

extern "C" int relo_probe_l2_gather(const uint16_t *buf_dev, int32_t log2_elems, int64_t gathers, void *stream,
                                    float *ms, int64_t *gathers_done) {
    if (!buf_dev || !ms || !gathers_done || log2_elems < 10 || log2_elems > 31 || gathers < 1)
        return RELO_E_INVALID_ARG;
    const int n_sm = probe_sms();
    if (n_sm < 1) return RELO_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = n_sm * 8;
    const long long per_round = (long long)grid * 256 * 8;
    const long long rounds = (gathers + per_round - 1) / per_round;
    if (rounds > (1ll << 30)) return RELO_E_INVALID_ARG;
    k_probe_stream<<<grid, 256, 0, s>>>(reinterpret_cast<const int4 *>(buf_dev), (1ll << log2_elems) / 8, 1);
    if (cudaGetLastError() != cudaSuccess) return RELO_E_CUDA;
    *gathers_done = rounds * per_round;
    return timed(s, [&] { k_probe_gather<<<grid, 256, 0, s>>>(buf_dev, log2_elems, (int)rounds); }, ms);
}
