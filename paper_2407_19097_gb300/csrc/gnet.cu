// The gated post-processing network (Sec. 3.3's form): gated convolutions with ELU,
// a 1x1 convolution of the G-buffers injected at every encoder level, average pooling in the
// encoder, transposed convolutions and skip concatenations in the decoder, a 1x1 head to RGB.
// Four levels of 16/32/64/128 channels (the paper's progression starts at 64 over five
// levels); BF16 activations, every 3x3 and transposed convolution on the tensor-core kernel
// (gated: the feature and gate convolutions as one GEMM whose epilogue computes
// ELU(feature) * sigmoid(gate)), the pools fused into the encoder convs and the head into the
// last conv.
//
//   g0 = 1x1(x)        g_l = avgpool(g_{l-1})
//   e0 = gated(g0)     e_l = gated([avgpool(e_{l-1}), g_l])   l = 1..3
//   u_l = convT(d_{l+1}),  d_l = gated([u_l, e_l])   l = 2, 1, 0   (d_3 = e_3)
//   rgb = 1x1(d0)
#include <string.h>

#include "net.h"
#include "net_simt.cuh"

namespace nrv {

namespace {

constexpr int GN_LAYERS = 12;
enum { G_INJ, G_E0, G_E1, G_E2, G_E3, G_UP2, G_D2, G_UP1, G_D1, G_UP0, G_D0, G_HEAD };
enum { GK_CONV1 = 2, GK_GATED = 3 };   // kinds beyond CONV3 / UPCONV2 (nrv_layer_info.kind)
constexpr int GW[4] = {16, 32, 64, 128};

struct GLayer {
    char name[8];
    int kind, cin, cout;
    int64_t woff, boff, woff2, boff2;
};

// Layer table and flat parameter layout: per layer the weight then the bias; a gated layer
// holds W_f (C_out, C_in, 3, 3), b_f, W_g (C_out, C_in, 3, 3), b_g.
int64_t gnet_layers(int c0, GLayer* L) {
    const struct { const char* n; int k, ci, co; } t[GN_LAYERS] = {
        {"inj", GK_CONV1, c0, c0},          {"e0", GK_GATED, c0, GW[0]},
        {"e1", GK_GATED, GW[0] + c0, GW[1]}, {"e2", GK_GATED, GW[1] + c0, GW[2]},
        {"e3", GK_GATED, GW[2] + c0, GW[3]}, {"up2", UPCONV2, GW[3], GW[2]},
        {"d2", GK_GATED, 2 * GW[2], GW[2]},  {"up1", UPCONV2, GW[2], GW[1]},
        {"d1", GK_GATED, 2 * GW[1], GW[1]},  {"up0", UPCONV2, GW[1], GW[0]},
        {"d0", GK_GATED, 2 * GW[0], GW[0]},  {"head", GK_CONV1, GW[0], 3}};
    int64_t off = 0;
    for (int i = 0; i < GN_LAYERS; ++i) {
        memset(L[i].name, 0, sizeof(L[i].name));
        strncpy(L[i].name, t[i].n, sizeof(L[i].name) - 1);
        L[i].kind = t[i].k;
        L[i].cin = t[i].ci;
        L[i].cout = t[i].co;
        const int64_t wsz = (int64_t)t[i].ci * t[i].co *
                            (t[i].k == GK_GATED ? 9 : t[i].k == UPCONV2 ? 4 : 1);
        L[i].woff = off;
        L[i].boff = off + wsz;
        off += wsz + t[i].co;
        L[i].woff2 = L[i].boff2 = -1;
        if (t[i].k == GK_GATED) {
            L[i].woff2 = off;
            L[i].boff2 = off + wsz;
            off += wsz + t[i].co;
        }
    }
    return off;
}

// g[o] = b[o] + sum_c W[o][c] x[c] for o < c0, zero for c0 <= o < 8: the 1x1 projection of the
// packed G-buffers (8 BF16 channels per pixel in and out), FP32 accumulation.
__global__ void inj_kernel(const uint4* __restrict__ x, uint4* __restrict__ g, size_t npx, int c0,
                           const float* __restrict__ w, const float* __restrict__ b) {
    // the weights in registers (channels from c0 on are neither read nor written but as zero)
    float wr[8][8], br[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        br[k] = k < c0 ? b[k] : 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) wr[k][c] = (k < c0 && c < c0) ? w[k * c0 + c] : 0.0f;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npx;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint4 raw = x[i];
        const uint32_t rw[4] = {raw.x, raw.y, raw.z, raw.w};
        float in[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&rw[j]);
            in[2 * j] = __low2float(h2);
            in[2 * j + 1] = __high2float(h2);
        }
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float acc = br[k];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < c0) acc = fmaf(wr[k][c], in[c], acc);
            o[k] = acc;
        }
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 h2 = __floats2bfloat162_rn(o[2 * j], o[2 * j + 1]);
            pk[j] = *reinterpret_cast<uint32_t*>(&h2);
        }
        g[i] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

int blocks(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b > 0 ? b : 1);
}

}  // namespace

struct GNet {
    int c_in = 0;
    GLayer L[GN_LAYERS];
    int64_t n_params = 0;
    bool has_params = false;
    DevBuf params;
    DevBuf acts;
    DevBuf layer_ws;   // row-planar copies for nrv_gnet_run_layer
    TcPacked* tc = nullptr;
    ~GNet() { tc_generic_free(tc); }
};

}  // namespace nrv

using namespace nrv;

struct nrv_gnet : GNet {};

extern "C" int nrv_gnet_num_layers(void) { return GN_LAYERS; }

extern "C" nrv_status nrv_gnet_param_count(int c_in, int64_t* count) {
    clear_error();
    if (c_in < 1 || c_in > 8 || !count) return fail(NRV_ERR_ARG, "c_in must be 1..8");
    GLayer L[GN_LAYERS];
    *count = gnet_layers(c_in, L);
    return NRV_OK;
}

extern "C" nrv_status nrv_gnet_layer(int c_in, int layer, nrv_layer_info* out) {
    clear_error();
    if (c_in < 1 || c_in > 8 || layer < 0 || layer >= GN_LAYERS || !out)
        return fail(NRV_ERR_ARG, "bad layer query");
    GLayer L[GN_LAYERS];
    gnet_layers(c_in, L);
    memset(out, 0, sizeof(*out));
    memcpy(out->name, L[layer].name, sizeof(out->name));
    out->kind = L[layer].kind;
    out->c_in = L[layer].cin;
    out->c_out = L[layer].cout;
    out->weight_offset = L[layer].woff;
    out->bias_offset = L[layer].boff;
    return NRV_OK;
}

extern "C" nrv_status nrv_gnet_create(int c_in, nrv_gnet** out) {
    clear_error();
    if (!out) return fail(NRV_ERR_ARG, "null argument");
    *out = nullptr;
    if (c_in < 1 || c_in > 8) return fail(NRV_ERR_ARG, "c_in must be 1..8");
    nrv_gnet* g = new nrv_gnet;
    g->c_in = c_in;
    g->n_params = gnet_layers(c_in, g->L);
    *out = g;
    return NRV_OK;
}

extern "C" nrv_status nrv_gnet_destroy(nrv_gnet* g) {
    clear_error();
    delete g;
    return NRV_OK;
}

extern "C" nrv_status nrv_gnet_set_params(nrv_gnet* g, const float* d_params, nrv_stream stream) {
    clear_error();
    if (!g || !d_params) return fail(NRV_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    NRV_TRY(g->params.ensure(g->n_params * sizeof(float)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(g->params.p, d_params, g->n_params * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s));
    // the tensor-core layers: gated 3x3 convs and transposed convs, BF16 row-planar; the
    // encoder convs take [pooled features, injected G-buffers (8 stored channels)]
    TcGeneric T[10];
    int n = 0;
    auto add = [&](int l, int c1, int c2) {
        const GLayer& L = g->L[l];
        T[n++] = TcGeneric{L.kind == GK_GATED ? CONV3 : UPCONV2, L.kind == GK_GATED ? 1 : 0, c1,
                           c2, L.cin, L.cout, L.woff, L.boff, L.woff2, L.boff2};
    };
    add(G_E0, 8, 0);
    add(G_E1, GW[0], 8);
    add(G_E2, GW[1], 8);
    add(G_E3, GW[2], 8);
    add(G_UP2, GW[3], 0);
    add(G_D2, GW[2], GW[2]);
    add(G_UP1, GW[2], 0);
    add(G_D1, GW[1], GW[1]);
    add(G_UP0, GW[1], 0);
    add(G_D0, GW[0], GW[0]);
    NRV_TRY(tc_generic_prepare(T, n, (const float*)g->params.p, &g->tc, s));
    g->has_params = true;
    return NRV_OK;
}

// indices into the tensor-core layer list built by nrv_gnet_set_params
enum { T_E0, T_E1, T_E2, T_E3, T_UP2, T_D2, T_UP1, T_D1, T_UP0, T_D0 };

extern "C" nrv_status nrv_gnet_shade(nrv_gnet* g, const void* netin, int n, int h, int w,
                                     float* rgb, nrv_stream stream) {
    clear_error();
    if (!g || !netin || !rgb) return fail(NRV_ERR_ARG, "null argument");
    if (!g->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (((uintptr_t)netin & 31) != 0) return fail(NRV_ERR_ARG, "d_netin must be 32-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int H[4], W[4];
    H[0] = nrv_pad8(h);
    W[0] = nrv_pad8(w);
    for (int l = 1; l < 4; ++l) { H[l] = H[l - 1] / 2; W[l] = W[l - 1] / 2; }
    auto px = [&](int l) { return (size_t)n * H[l] * W[l]; };
    // activations (BF16, row-planar): g0..g3 (8 ch), e0..e3, p0..p2 (pooled e0..e2), u2, d2,
    // u1, d1, u0
    size_t off = 0, o_g[4], o_e[4], o_p[3], o_u[3], o_d[3];
    auto take = [&](size_t bytes) { const size_t r = off; off += (bytes + 1023) / 1024 * 1024; return r; };
    for (int l = 0; l < 4; ++l) o_g[l] = take(px(l) * 8 * 2);
    for (int l = 0; l < 4; ++l) o_e[l] = take(px(l) * GW[l] * 2);
    for (int l = 0; l < 3; ++l) o_p[l] = take(px(l + 1) * GW[l] * 2);
    for (int l = 0; l < 3; ++l) o_u[l] = take(px(l) * GW[l] * 2);
    for (int l = 1; l < 3; ++l) o_d[l] = take(px(l) * GW[l] * 2);
    o_d[0] = 0;
    NRV_TRY(g->acts.ensure(off));
    char* A = (char*)g->acts.p;
    const float* P = (const float*)g->params.p;
    // injection: the 1x1 projection and its pyramid
    inj_kernel<<<blocks(px(0)), 256, 0, s>>>((const uint4*)netin, (uint4*)(A + o_g[0]), px(0),
                                             g->c_in, P + g->L[G_INJ].woff, P + g->L[G_INJ].boff);
    NRV_CHECK_LAUNCH();
    using T = __nv_bfloat16;
    for (int l = 1; l < 4; ++l) {
        pool2_kernel<T><<<blocks(px(l)), 256, 0, s>>>(TView<const T>{(const T*)(A + o_g[l - 1]), 8, 1},
                                                      TView<T>{(T*)(A + o_g[l]), 8, 1}, 8, n, H[l], W[l]);
        NRV_CHECK_LAUNCH();
    }
    const TcPacked* tc = g->tc;
    // encoder (pools fused into e0..e2)
    NRV_TRY(tc_generic_run(tc, T_E0, P, A + o_g[0], nullptr, A + o_e[0], n, H[0], W[0], s, nullptr,
                           A + o_p[0]));
    NRV_TRY(tc_generic_run(tc, T_E1, P, A + o_p[0], A + o_g[1], A + o_e[1], n, H[1], W[1], s,
                           nullptr, A + o_p[1]));
    NRV_TRY(tc_generic_run(tc, T_E2, P, A + o_p[1], A + o_g[2], A + o_e[2], n, H[2], W[2], s,
                           nullptr, A + o_p[2]));
    NRV_TRY(tc_generic_run(tc, T_E3, P, A + o_p[2], A + o_g[3], A + o_e[3], n, H[3], W[3], s));
    // decoder
    NRV_TRY(tc_generic_run(tc, T_UP2, P, A + o_e[3], nullptr, A + o_u[2], n, H[3], W[3], s));
    NRV_TRY(tc_generic_run(tc, T_D2, P, A + o_u[2], A + o_e[2], A + o_d[2], n, H[2], W[2], s));
    NRV_TRY(tc_generic_run(tc, T_UP1, P, A + o_d[2], nullptr, A + o_u[1], n, H[2], W[2], s));
    NRV_TRY(tc_generic_run(tc, T_D1, P, A + o_u[1], A + o_e[1], A + o_d[1], n, H[1], W[1], s));
    NRV_TRY(tc_generic_run(tc, T_UP0, P, A + o_d[1], nullptr, A + o_u[0], n, H[1], W[1], s));
    // the last gated conv with the 1x1 head in its epilogue (its own output is not stored)
    const GLayer& Lh = g->L[G_HEAD];
    const TcHead head{P + Lh.woff, P + Lh.boff, rgb, h, w, 1.0f, false, RgbTab{}};
    return tc_generic_run(tc, T_D0, P, A + o_u[0], A + o_e[0], A + o_e[0], n, H[0], W[0], s, &head);
}

// One layer alone (NHWC BF16 in and out), through the same kernels as nrv_gnet_shade.
extern "C" nrv_status nrv_gnet_run_layer(nrv_gnet* g, int layer, const void* x1, const void* x2,
                                         int n, int h, int w, void* y, nrv_stream stream) {
    clear_error();
    if (!g || !x1 || !y) return fail(NRV_ERR_ARG, "null argument");
    if (!g->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (layer < 0 || layer >= G_HEAD) return fail(NRV_ERR_ARG, "layer %d has no single-layer form", layer);
    if (n < 1 || h < 1 || w < 1 || (h & 1) || (w & 1) || h > 16384 || w > 16384)
        return fail(NRV_ERR_ARG, "bad size (even h, w)");
    cudaStream_t s = (cudaStream_t)stream;
    const GLayer& L = g->L[layer];
    if (layer == G_INJ) {
        inj_kernel<<<blocks((size_t)n * h * w), 256, 0, s>>>((const uint4*)x1, (uint4*)y,
                                                             (size_t)n * h * w, g->c_in,
                                                             (const float*)g->params.p + L.woff,
                                                             (const float*)g->params.p + L.boff);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    }
    // the tensor-core layer list index and the stored channels of its sources
    static const int tix[G_HEAD] = {-1, T_E0, T_E1, T_E2, T_E3, T_UP2, T_D2, T_UP1, T_D1, T_UP0, T_D0};
    const int t = tix[layer];
    const bool concat = layer == G_E1 || layer == G_E2 || layer == G_E3 || layer == G_D2 ||
                        layer == G_D1 || layer == G_D0;
    if (concat != (x2 != nullptr)) return fail(NRV_ERR_ARG, "x2 must be %s", concat ? "given" : "NULL");
    int c1 = L.cin, c2 = 0;
    if (layer == G_E0) c1 = 8;
    if (layer == G_E1 || layer == G_E2 || layer == G_E3) { c1 = L.cin - g->c_in; c2 = 8; }
    if (layer == G_D2 || layer == G_D1 || layer == G_D0) { c1 = L.cin / 2; c2 = L.cin / 2; }
    const bool up = L.kind == UPCONV2;
    const size_t rows = (size_t)n * h, rows_out = up ? 2 * rows : rows;
    const int w_out = up ? 2 * w : w;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b1 = al(rows * w * c1 * 2), b2 = al(rows * w * c2 * 2), by = al(rows_out * w_out * L.cout * 2);
    NRV_TRY(g->layer_ws.ensure(b1 + b2 + by));
    char* ws = (char*)g->layer_ws.p;
    NRV_TRY(relayout(x1, ws, rows, w, c1, 2, true, s));
    if (c2) NRV_TRY(relayout(x2, ws + b1, rows, w, c2, 2, true, s));
    NRV_TRY(tc_generic_run(g->tc, t, (const float*)g->params.p, ws, c2 ? ws + b1 : nullptr,
                           ws + b1 + b2, n, h, w, s));
    return relayout(ws + b1 + b2, y, rows_out, w_out, L.cout, 2, false, s);
}
