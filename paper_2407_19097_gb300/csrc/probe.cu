// Microbenchmarks for the rooflines that the measured-peaks file does not hold: the
// FP32 FMA throughput of the CUDA cores (the FP32 form of the network runs there) and
// the rate of random 64-bit atomicMin on an L2-resident buffer (the render pass's
// depth test, Sec. 3.2).  Timed by the caller with events around the launch.
#include "internal.h"

namespace nrv {
namespace {

// Eight independent FMA chains per thread, `iters` steps each: 16 * iters FLOPs per thread.
__global__ void __launch_bounds__(256) ffma_kernel(float* out, int iters, float b, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 finaliser (Steele, Lea and Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Operation i: atomicMin(buf[h(i) mod n], h'(i)) with h, h' from one 64-bit hash.
__global__ void atomic_min_kernel(unsigned long long* buf, int64_t n_words, int64_t n_ops,
                                  uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_ops;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));
        atomicMin(buf + (h >> 20) % (uint64_t)n_words, (unsigned long long)(h & 0xFFFFFFFFFFull));
    }
}

}  // namespace
}  // namespace nrv

using namespace nrv;

extern "C" nrv_status nrv_probe_ffma(float* out, int blocks, int iters, nrv_stream stream) {
    clear_error();
    if (!out || blocks < 1 || iters < 1) return fail(NRV_ERR_ARG, "bad argument");
    ffma_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-3f);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

extern "C" nrv_status nrv_probe_atomic_min(unsigned long long* buf, int64_t n_words, int64_t n_ops,
                                           uint64_t seed, nrv_stream stream) {
    clear_error();
    if (!buf || n_words < 1 || n_ops < 1) return fail(NRV_ERR_ARG, "bad argument");
    atomic_min_kernel<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(buf, n_words, n_ops, seed);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}
