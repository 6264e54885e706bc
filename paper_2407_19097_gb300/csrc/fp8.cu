// FP8 (E4M3) form of the U-Net forward (the paper's App. B quantises the
// network to fp16; this goes to 8-bit floats).  Every stored tensor t holds
// E4M3 codes q with value q * s_t (one scale per tensor); weights hold E4M3
// codes per output column with their own scale.  Scales come from calibration:
// s_t = max|t| / 448 over a BF16 forward on sample inputs.  Pooling keeps its
// input's scale, so pooled codes are the E4M3 rounding of the mean of the four
// decoded codes.
#include "net.h"

namespace nrv {

__device__ __forceinline__ float dec8(uint8_t b) {
    __nv_fp8_e4m3 v;
    v.__x = b;
    return float(v);
}

__device__ __forceinline__ uint8_t enc8(float f) {
    return __nv_cvt_float_to_fp8(f, __NV_SATFINITE, __NV_E4M3);
}

// y = E4M3(mean of the 2x2 window), input and output share one scale.  Tensors
// are row-planar (planes of 16 channels x w pixels per image row); one thread
// makes one 16-byte output chunk, pixels fastest.
__global__ void pool2_fp8_kernel(const uint8_t* __restrict__ x, uint8_t* __restrict__ y, int c,
                                 int n, int ho, int wo) {
    const int nch = c / 16;
    const size_t total = (size_t)n * ho * wo * nch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int xo = (int)(i % wo);
        const int ch = (int)((i / wo) % nch);
        const size_t row = i / ((size_t)wo * nch);   // img * ho + yo
        const int yo = (int)(row % ho);
        const size_t img = row / ho;
        const int wi = 2 * wo;
        const size_t r0 = img * 2 * ho + 2 * yo;
        const uint8_t* p0 = x + ((r0 * nch + ch) * wi + 2 * xo) * 16;
        const uint8_t* p1 = x + (((r0 + 1) * nch + ch) * wi + 2 * xo) * 16;
        const uint4 a = *reinterpret_cast<const uint4*>(p0);
        const uint4 b = *reinterpret_cast<const uint4*>(p0 + 16);
        const uint4 d = *reinterpret_cast<const uint4*>(p1);
        const uint4 e = *reinterpret_cast<const uint4*>(p1 + 16);
        const uint8_t* pa = reinterpret_cast<const uint8_t*>(&a);
        const uint8_t* pb = reinterpret_cast<const uint8_t*>(&b);
        const uint8_t* pd = reinterpret_cast<const uint8_t*>(&d);
        const uint8_t* pe = reinterpret_cast<const uint8_t*>(&e);
        uint4 o;
        uint8_t* po = reinterpret_cast<uint8_t*>(&o);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            po[k] = enc8(0.25f * ((dec8(pa[k]) + dec8(pb[k])) + (dec8(pd[k]) + dec8(pe[k]))));
        *reinterpret_cast<uint4*>(y + i * 16) = o;
    }
}

// Level 0 -> level 1 of the mixed network: y = E4M3((mean of the 2x2 window of the BF16
// tensor x) * inv_scale), the mean with the pool kernel's arithmetic.  x row-planar BF16
// [n][2ho][c/8][2wo][8], y row-planar E4M3 [n][ho][c/16][wo][16]; one thread per 16 output
// channels of one pixel, pixels fastest.
__global__ void pool2_bf16_to_fp8_kernel(const __nv_bfloat16* __restrict__ x, uint8_t* __restrict__ y,
                                         int c, int n, int ho, int wo, float inv_scale) {
    const int nch = c / 16, nb = c / 8;
    const size_t total = (size_t)n * ho * wo * nch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int xo = (int)(i % wo);
        const int ch = (int)((i / wo) % nch);
        const size_t row = i / ((size_t)wo * nch);   // img * ho + yo
        const int yo = (int)(row % ho);
        const size_t img = row / ho;
        const int wi = 2 * wo;
        const size_t r0 = img * 2 * ho + 2 * yo;
        uint32_t wd[4] = {0u, 0u, 0u, 0u};
        for (int hp = 0; hp < 2; ++hp) {   // the two BF16 planes of this 16-channel group
            const int pl = 2 * ch + hp;
            const __nv_bfloat16* p0 = x + ((r0 * nb + pl) * (size_t)wi + 2 * xo) * 8;
            const __nv_bfloat16* p1 = x + (((r0 + 1) * nb + pl) * (size_t)wi + 2 * xo) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float a = __bfloat162float(p0[k]), b = __bfloat162float(p0[8 + k]);
                const float d = __bfloat162float(p1[k]), e = __bfloat162float(p1[8 + k]);
                const float m = 0.25f * ((a + b) + (d + e));
                const int j = 8 * hp + k;
                wd[j >> 2] |= (uint32_t)enc8(m * inv_scale) << (8 * (j & 3));
            }
        }
        *reinterpret_cast<uint4*>(y + ((row * nch + ch) * (size_t)wo + xo) * 16) =
            make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
}

// Level 1 -> level 0 of the mixed network: y = BF16(decoded E4M3 code * scale); x row-planar
// E4M3 [rows][c/16][w][16], y row-planar BF16 [rows][c/8][w][8]; one thread per 8 values.
__global__ void fp8_to_bf16_kernel(const uint8_t* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                   int c, size_t rows, int w, float scale) {
    const int nb = c / 8, nch = c / 16;
    const size_t total = rows * (size_t)w * nb;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % w);
        const int pl = (int)((i / w) % nb);
        const size_t row = i / ((size_t)w * nb);
        const uint8_t* src = x + ((row * nch + pl / 2) * (size_t)w + xx) * 16 + 8 * (pl & 1);
        const uint2 raw = *reinterpret_cast<const uint2*>(src);
        const uint8_t* b = reinterpret_cast<const uint8_t*>(&raw);
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 h2 = __floats2bfloat162_rn(dec8(b[2 * j]) * scale, dec8(b[2 * j + 1]) * scale);
            pk[j] = *reinterpret_cast<uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(y + ((row * nb + pl) * (size_t)w + xx) * 8) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// rgb[o] = bias[o] + sum_c W[o][c] * (x_c * s), cropped to h x wd (16 channels:
// one plane, so the row-planar tensor is also plain NHWC).
__global__ void head_fp8_kernel(const uint8_t* __restrict__ x, float s, const float* w,
                                const float* bias, float* rgb, int n, int hn, int wn, int h,
                                int wd, RgbTab tab) {
    const size_t total = (size_t)n * h * wd;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % wd), Y = (int)((i / wd) % h);
        const size_t img = i / ((size_t)wd * h);
        const size_t q = (img * hn + Y) * wn + X;
        const uint4 raw = *reinterpret_cast<const uint4*>(x + q * 16);
        const uint8_t* p = reinterpret_cast<const uint8_t*>(&raw);
        float v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = dec8(p[c]) * s;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float acc = bias[o];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc = fmaf(w[o * 16 + c], v[c], acc);
            rgb_image(rgb, tab, img, (size_t)h * wd)[3 * ((size_t)Y * wd + X) + o] = acc;
        }
    }
}

// out[0] = max(out[0], max |x|) as float bits (non-negative floats order like their bits).
__global__ void amax_bf16_kernel(const __nv_bfloat16* __restrict__ x, size_t n, unsigned* out) {
    float m = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__bfloat162float(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

static int blocks_for(size_t work, int per = 256) {
    size_t b = (work + per - 1) / per;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b > 0 ? b : 1);
}

nrv_status net_calibrate(Net* net, const void* netin, int n, int H, int W, cudaStream_t s) {
    // a BF16 forward, then the largest magnitude of the input and of every activation
    NRV_TRY(net->partial.ensure(((size_t)n * H * W * 3 + 64) * sizeof(float)));
    float* rgb = (float*)net->partial.p;
    unsigned* amax = (unsigned*)(rgb + (size_t)n * H * W * 3);
    NRV_TRY(net_forward(net, netin, n, H, W, NRV_PREC_BF16, rgb, s));
    NRV_CHECK_CUDA(cudaMemsetAsync(amax, 0, (NUM_ACTS + 1) * sizeof(unsigned), s));
    const Geo& g = net->geo;
    const size_t nin = g.px(0) * net->c0p;
    amax_bf16_kernel<<<blocks_for(nin), 256, 0, s>>>((const __nv_bfloat16*)netin, nin, amax);
    NRV_CHECK_LAUNCH();
    for (int a = 0; a < NUM_ACTS; ++a) {
        const size_t cnt = g.px(net->act_level[a]) * net->act_c[a];
        amax_bf16_kernel<<<blocks_for(cnt), 256, 0, s>>>(
            (const __nv_bfloat16*)((char*)net->acts.p + net->act_off[a]), cnt, amax + 1 + a);
        NRV_CHECK_LAUNCH();
    }
    unsigned host[NUM_ACTS + 1];
    NRV_CHECK_CUDA(cudaMemcpyAsync(host, amax, sizeof(host), cudaMemcpyDeviceToHost, s));
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a <= NUM_ACTS; ++a) {
        float m;
        memcpy(&m, &host[a], 4);
        net->act_scale[a] = m > 0.0f ? m / 448.0f : 1.0f;
    }
    // a pooled tensor keeps the scale of the tensor it pools
    net->act_scale[1 + A_P0] = net->act_scale[1 + A_E0B];
    net->act_scale[1 + A_P1] = net->act_scale[1 + A_E1B];
    net->act_scale[1 + A_P2] = net->act_scale[1 + A_E2B];
    return NRV_OK;
}

nrv_status forward_fp8(Net* net, const uint8_t* netin, float* rgb, cudaStream_t s, bool keep_acts) {
    if (!net->fp8_ready) return fail(NRV_ERR_STATE, "FP8 needs activation scales (calibrate first)");
    const Geo& g = net->geo;
    auto A = [&](int a) { return (uint8_t*)net->acts.p + net->act_off[a]; };
    auto inv = [&](int a) { return 1.0f / net->act_scale[1 + a]; };
    auto conv = [&](int l, const void* x1, int c1, const void* x2, int c2, int out,
                    int level) -> nrv_status {
        net->backend[l] = 1;
        return tc_conv3(net, l, x1, c1, x2, c2, A(out), g, level, NRV_PREC_FP8_E4M3, s, inv(out));
    };
    auto pool = [&](int in, int out, int level_out) -> nrv_status {
        const int c = net->act_c[in];
        pool2_fp8_kernel<<<blocks_for(g.px(level_out) * c / 16), 256, 0, s>>>(
            A(in), A(out), c, g.n, g.h[level_out], g.w[level_out]);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    };
    auto up = [&](int l, int in, int out, int level_in) -> nrv_status {
        net->backend[l] = 1;
        return tc_upconv(net, l, A(in), A(out), g, level_in, NRV_PREC_FP8_E4M3, s, inv(out));
    };
    // a 3x3 conv and the pool of its output to the next level (separate kernels: at level 0
    // the FP8 epilogue is the bottleneck and a fused pool measured slower)
    auto conv_pool = [&](int l, int in, int c1, int out, int level, int pooled) -> nrv_status {
        NRV_TRY(conv(l, A(in), c1, nullptr, 0, out, level));
        return pool(out, pooled, level + 1);
    };
    NRV_TRY(conv(L_E0A, netin, 16, nullptr, 0, A_E0A, 0));
    NRV_TRY(conv_pool(L_E0B, A_E0A, 16, A_E0B, 0, A_P0));
    NRV_TRY(conv(L_E1A, A(A_P0), 16, nullptr, 0, A_E1A, 1));
    NRV_TRY(conv_pool(L_E1B, A_E1A, 32, A_E1B, 1, A_P1));
    NRV_TRY(conv(L_E2A, A(A_P1), 32, nullptr, 0, A_E2A, 2));
    NRV_TRY(conv_pool(L_E2B, A_E2A, 64, A_E2B, 2, A_P2));
    NRV_TRY(conv(L_E3A, A(A_P2), 64, nullptr, 0, A_E3A, 3));
    NRV_TRY(conv(L_E3B, A(A_E3A), 128, nullptr, 0, A_E3B, 3));
    NRV_TRY(up(L_UP3, A_E3B, A_UP3, 3));
    NRV_TRY(conv(L_D2A, A(A_UP3), 64, A(A_E2B), 64, A_D2A, 2));
    NRV_TRY(conv(L_D2B, A(A_D2A), 64, nullptr, 0, A_D2B, 2));
    NRV_TRY(up(L_UP2, A_D2B, A_UP2, 2));
    NRV_TRY(conv(L_D1A, A(A_UP2), 32, A(A_E1B), 32, A_D1A, 1));
    NRV_TRY(conv(L_D1B, A(A_D1A), 32, nullptr, 0, A_D1B, 1));
    NRV_TRY(up(L_UP1, A_D1B, A_UP1, 1));
    NRV_TRY(conv(L_D0A, A(A_UP1), 16, A(A_E0B), 16, A_D0A, 0));
    const Layer& Lh = net->layers[L_HEAD];
    {
        // the head in the last conv's epilogue
        const float* P = (const float*)net->params.p;
        const TcHead head{P + Lh.woff, P + Lh.boff, rgb, net->geo_H, net->geo_W,
                          net->act_scale[1 + A_D0B], keep_acts, net->rgb_tab};
        const nrv_status st = tc_conv3(net, L_D0B, A(A_D0A), 16, nullptr, 0, A(A_D0B), g, 0,
                                       NRV_PREC_FP8_E4M3, s, inv(A_D0B), &head);
        net->backend[L_D0B] = 1;
        if (st != NRV_ERR_UNSUPPORTED) return st;
        clear_error();
    }
    NRV_TRY(conv(L_D0B, A(A_D0A), 16, nullptr, 0, A_D0B, 0));
    head_fp8_kernel<<<blocks_for((size_t)g.n * net->geo_H * net->geo_W), 256, 0, s>>>(
        A(A_D0B), net->act_scale[1 + A_D0B], (const float*)net->params.p + Lh.woff,
        (const float*)net->params.p + Lh.boff, rgb, g.n, g.h[0], g.w[0], net->geo_H, net->geo_W,
        net->rgb_tab);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

nrv_status forward_fp8_mixed(Net* net, const void* netin, float* rgb, cudaStream_t s) {
    if (!net->fp8_ready) return fail(NRV_ERR_STATE, "FP8 needs activation scales (calibrate first)");
    const Geo& g = net->geo;
    auto A = [&](int a) { return (uint8_t*)net->acts.p + net->act_off[a]; };
    auto inv = [&](int a) { return 1.0f / net->act_scale[1 + a]; };
    for (int l = 0; l < NUM_LAYERS; ++l) net->backend[l] = net->layers[l].kind == HEAD1 ? 0 : 1;
    auto conv8 = [&](int l, const void* x1, int c1, const void* x2, int c2, int out,
                     int level) -> nrv_status {
        return tc_conv3(net, l, x1, c1, x2, c2, A(out), g, level, NRV_PREC_FP8_E4M3, s, inv(out));
    };
    auto pool8 = [&](int in, int out, int level_out) -> nrv_status {
        const int c = net->act_c[in];
        pool2_fp8_kernel<<<blocks_for(g.px(level_out) * c / 16), 256, 0, s>>>(
            A(in), A(out), c, g.n, g.h[level_out], g.w[level_out]);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    };
    auto up8 = [&](int l, int in, int out, int level_in) -> nrv_status {
        return tc_upconv(net, l, A(in), A(out), g, level_in, NRV_PREC_FP8_E4M3, s, inv(out));
    };
    // level 0 encoder in BF16 from the BF16 input
    NRV_TRY(tc_conv3(net, L_E0A, netin, net->c0p, nullptr, 0, A(A_E0A), g, 0, NRV_PREC_BF16, s));
    NRV_TRY(tc_conv3(net, L_E0B, A(A_E0A), 16, nullptr, 0, A(A_E0B), g, 0, NRV_PREC_BF16, s));
    // pooled to level 1 and quantised with the scale of e0b's output
    pool2_bf16_to_fp8_kernel<<<blocks_for(g.px(1)), 256, 0, s>>>(
        (const __nv_bfloat16*)A(A_E0B), A(A_P0), 16, g.n, g.h[1], g.w[1], inv(A_P0));
    NRV_CHECK_LAUNCH();
    // levels 1-3 in E4M3
    NRV_TRY(conv8(L_E1A, A(A_P0), 16, nullptr, 0, A_E1A, 1));
    NRV_TRY(conv8(L_E1B, A(A_E1A), 32, nullptr, 0, A_E1B, 1));
    NRV_TRY(pool8(A_E1B, A_P1, 2));
    NRV_TRY(conv8(L_E2A, A(A_P1), 32, nullptr, 0, A_E2A, 2));
    NRV_TRY(conv8(L_E2B, A(A_E2A), 64, nullptr, 0, A_E2B, 2));
    NRV_TRY(pool8(A_E2B, A_P2, 3));
    NRV_TRY(conv8(L_E3A, A(A_P2), 64, nullptr, 0, A_E3A, 3));
    NRV_TRY(conv8(L_E3B, A(A_E3A), 128, nullptr, 0, A_E3B, 3));
    NRV_TRY(up8(L_UP3, A_E3B, A_UP3, 3));
    NRV_TRY(conv8(L_D2A, A(A_UP3), 64, A(A_E2B), 64, A_D2A, 2));
    NRV_TRY(conv8(L_D2B, A(A_D2A), 64, nullptr, 0, A_D2B, 2));
    NRV_TRY(up8(L_UP2, A_D2B, A_UP2, 2));
    NRV_TRY(conv8(L_D1A, A(A_UP2), 32, A(A_E1B), 32, A_D1A, 1));
    NRV_TRY(conv8(L_D1B, A(A_D1A), 32, nullptr, 0, A_D1B, 1));
    // back to BF16 for level 0: d1b's output decoded into d1a's slot (no longer read)
    const size_t rows1 = (size_t)g.n * g.h[1];
    fp8_to_bf16_kernel<<<blocks_for(rows1 * g.w[1] * 4), 256, 0, s>>>(
        A(A_D1B), (__nv_bfloat16*)A(A_D1A), 32, rows1, g.w[1], net->act_scale[1 + A_D1B]);
    NRV_CHECK_LAUNCH();
    NRV_TRY(tc_upconv(net, L_UP1, A(A_D1A), A(A_UP1), g, 1, NRV_PREC_BF16, s));
    NRV_TRY(tc_conv3(net, L_D0A, A(A_UP1), 16, A(A_E0B), 16, A(A_D0A), g, 0, NRV_PREC_BF16, s));
    const Layer& Lh = net->layers[L_HEAD];
    const float* P = (const float*)net->params.p;
    const TcHead head{P + Lh.woff, P + Lh.boff, rgb, net->geo_H, net->geo_W, 1.0f, false,
                      net->rgb_tab};
    return tc_conv3(net, L_D0B, A(A_D0A), 16, nullptr, 0, A(A_D0B), g, 0, NRV_PREC_BF16, s, 1.0f,
                    &head);
}

}  // namespace nrv
