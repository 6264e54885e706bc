// Network parameters in and out of a handle: seeded Xavier-uniform initialisation
// (the paper trains from scratch, Sec. 3.3; the draw is this library's convention),
// a device copy of the master weights, and a small binary file format.
//
// Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014).  The i-th output of the
// sequence whose state starts at s is mix(s + (i + 1) * gamma); a stream's
// state is the stream-th output of the sequence seeded with `seed`.  Element i
// of layer t's weight (PyTorch layout order) draws u = top 53 bits of output i
// of stream 1000 + t as a double in [0, 1) and becomes the float nearest to
// -b + 2b u, b = sqrt(6 / (fan_in + fan_out)), fan = channels x kernel area
// (Glorot and Bengio 2010).  Biases are zero.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "net.h"

namespace nrv {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// w[i] = float(-b + 2b u_i), the double operations rounded one by one (no contraction)
__global__ void xavier_kernel(float* __restrict__ w, int64_t n, uint64_t seed, uint64_t stream,
                              double b) {
    const uint64_t key = splitmix_mix(seed + (stream + 1) * kGamma);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t bits = splitmix_mix(key + ((uint64_t)i + 1) * kGamma);
        const double u = __dmul_rn((double)(bits >> 11), 0x1.0p-53);
        w[i] = __double2float_rn(__dadd_rn(-b, __dmul_rn(__dadd_rn(b, b), u)));
    }
}

constexpr char kMagic[8] = {'N', 'R', 'V', 'N', 'E', 'T', '0', '1'};

}  // namespace

nrv_status net_init_params(const Net* net, uint64_t seed, float* d_params, cudaStream_t s) {
    NRV_CHECK_CUDA(cudaMemsetAsync(d_params, 0, net->n_params * sizeof(float), s));
    for (int t = 0; t < NUM_LAYERS; ++t) {
        const Layer& L = net->layers[t];
        const int k2 = L.kind == CONV3 ? 9 : (L.kind == UPCONV2 ? 4 : 1);
        const int64_t n = (int64_t)L.cin * L.cout * k2;
        const double b = sqrt(6.0 / ((double)L.cin * k2 + (double)L.cout * k2));
        int64_t blocks = (n + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        xavier_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_params + L.woff, n, seed,
                                                       1000u + (uint64_t)t, b);
        NRV_CHECK_LAUNCH();
    }
    return NRV_OK;
}

// File: magic "NRVNET01", int32 c_in, int32 flags (bit 0: FP8 scales present),
// int64 parameter count, the FP32 parameters, then NUM_ACTS + 1 FP32 scales.
nrv_status net_save(const Net* net, const char* path, cudaStream_t s) {
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    std::vector<float> p((size_t)net->n_params);
    NRV_CHECK_CUDA(cudaMemcpyAsync(p.data(), net->params.p, p.size() * sizeof(float),
                                   cudaMemcpyDeviceToHost, s));
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(NRV_ERR_ARG, "cannot open %s for writing", path);
    const int32_t hdr[2] = {net->c_in, net->fp8_ready ? 1 : 0};
    const int64_t count = net->n_params;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, 4, 2, f) == 2 &&
              fwrite(&count, 8, 1, f) == 1 && fwrite(p.data(), 4, p.size(), f) == p.size() &&
              fwrite(net->act_scale, 4, NUM_ACTS + 1, f) == (size_t)(NUM_ACTS + 1);
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(NRV_ERR_ARG, "writing %s failed", path);
    return NRV_OK;
}

nrv_status net_load(Net* net, const char* path, cudaStream_t s) {
    FILE* f = fopen(path, "rb");
    if (!f) return fail(NRV_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t hdr[2] = {0, 0};
    int64_t count = 0;
    std::vector<float> p;
    float scales[NUM_ACTS + 1];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(hdr, 4, 2, f) == 2 && fread(&count, 8, 1, f) == 1;
    if (ok && (hdr[0] != net->c_in || count != net->n_params)) {
        fclose(f);
        return fail(NRV_ERR_ARG, "%s holds a network for %d input channels (%lld parameters), "
                    "this one has %d", path, hdr[0], (long long)count, net->c_in);
    }
    if (ok) {
        p.resize((size_t)count);
        ok = fread(p.data(), 4, p.size(), f) == p.size() &&
             fread(scales, 4, NUM_ACTS + 1, f) == (size_t)(NUM_ACTS + 1);
    }
    fclose(f);
    if (!ok) return fail(NRV_ERR_ARG, "%s is not a network file", path);
    if (hdr[1] & 1)
        for (int a = 0; a <= NUM_ACTS; ++a)
            if (!(scales[a] > 0.0f) || !isfinite(scales[a]))
                return fail(NRV_ERR_ARG, "%s: FP8 scale %d is not positive", path, a);
    NRV_TRY(net->params.ensure(net->n_params * sizeof(float)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(net->params.p, p.data(), p.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, s));
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));   // the host copy goes out of scope
    net->fp8_ready = (hdr[1] & 1) != 0;         // net_repack then packs the FP8 weights too
    if (net->fp8_ready)
        for (int a = 0; a <= NUM_ACTS; ++a) net->act_scale[a] = scales[a];
    NRV_TRY(net_repack(net, s));
    net->has_params = true;
    return NRV_OK;
}

}  // namespace nrv
