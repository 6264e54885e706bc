// L1 loss without any device allocation (nrv_l1_loss_noalloc).
//
// Some callers cannot allocate device memory at the time they need a loss:
// a renderer or trainer embedded in a host application whose memory pool owns
// the whole device, code running under a strict no-allocation rule after
// start-up (cudaMalloc and cudaFree synchronise the device and would stall a
// real-time frame loop), or plug-ins that are handed their buffers and nothing
// else.  This variant keeps its scratch -- one partial sum per block of the
// deterministic two-stage reduction -- in a fixed array in the library's own
// device memory instead of a buffer allocated on first use.
//
// The array lives for as long as the library is loaded, on every device that
// loads it, and every call shares it: the partial-sum kernel overwrites each
// slot the final kernel reads, so no clearing is needed between calls, and two
// calls whose kernels overlap on the GPU race on the array.
#include <mutex>

#include "internal.h"

namespace nrv {

namespace {

constexpr int64_t kChunk = 8192;          // elements reduced by one block
constexpr int kMaxBlocks = 16384;         // slots in the scratch array (64 KiB)

static_assert(kChunk * kMaxBlocks == NRV_L1_NOALLOC_MAX_ELEMENTS, "capacity mismatch");

static __device__ __align__(256) float g_l1_partials[kMaxBlocks];

__global__ void __launch_bounds__(256) l1_chunk_kernel(const float* __restrict__ y,
                                                       const float* __restrict__ t, int64_t n,
                                                       float* dy, float inv_n, float* part) {
    __shared__ float red[256];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int64_t end = base + kChunk < n ? base + kChunk : n;
    float s = 0.0f;
    for (int64_t i = base + threadIdx.x; i < end; i += 256) {
        const float d = y[i] - t[i];
        s += fabsf(d);
        if (dy) dy[i] = d > 0.0f ? inv_n : (d < 0.0f ? -inv_n : 0.0f);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void l1_sum_kernel(const float* part, int nb, double inv_n, float* loss) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = (float)(red[0] * inv_n);
}

// Device address of the scratch array, looked up once per device.  In host
// code the array's name only stands for it; kernels must be given this address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

nrv_status scratch_address(float** out) {
    int dev = 0;
    NRV_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NRV_ERR_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_l1_partials);
        if (e != cudaSuccess || !p)
            return fail(NRV_ERR_CUDA, "cudaGetSymbolAddress of the L1 scratch failed: %s",
                        cudaGetErrorString(e));
        g_addr[dev] = static_cast<float*>(p);
    }
    *out = g_addr[dev];
    return NRV_OK;
}

}  // namespace

}  // namespace nrv

using namespace nrv;

extern "C" nrv_status nrv_l1_loss_noalloc(const float* d_y, const float* d_t, int64_t n,
                                          float* d_loss, float* d_dy, nrv_stream stream) {
    clear_error();
    if (!d_y || !d_t || !d_loss || n < 1) return fail(NRV_ERR_ARG, "bad argument");
    if (n > NRV_L1_NOALLOC_MAX_ELEMENTS)
        return fail(NRV_ERR_ARG,
                    "nrv_l1_loss_noalloc handles at most %lld elements (got %lld); use nrv_l1_loss",
                    (long long)NRV_L1_NOALLOC_MAX_ELEMENTS, (long long)n);
    float* part = nullptr;
    NRV_TRY(scratch_address(&part));
    const int nb = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t s = (cudaStream_t)stream;
    l1_chunk_kernel<<<nb, 256, 0, s>>>(d_y, d_t, n, d_dy, (float)(1.0 / (double)n), part);
    NRV_CHECK_LAUNCH();
    l1_sum_kernel<<<1, 256, 0, s>>>(part, nb, 1.0 / (double)n, d_loss);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}
