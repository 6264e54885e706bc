// U-Net of the neural deferred renderer (Sec. 3.3): layer table, weight
// re-packing, activation workspace and the forward pass.
#include <string.h>

#include "net.h"
#include "net_simt.cuh"

namespace nrv {

nrv_status DevBuf::ensure(size_t b) {
    if (b <= bytes) return NRV_OK;
    release();
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(NRV_ERR_OOM, "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    }
    bytes = b;
    return NRV_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

int net_layers(int c_in, Layer* L) {
    struct { const char* n; int k, ci, co; } t[NUM_LAYERS] = {
        {"e0a", CONV3, c_in, 16}, {"e0b", CONV3, 16, 16}, {"e1a", CONV3, 16, 32},
        {"e1b", CONV3, 32, 32},   {"e2a", CONV3, 32, 64}, {"e2b", CONV3, 64, 64},
        {"e3a", CONV3, 64, 128},  {"e3b", CONV3, 128, 128}, {"up3", UPCONV2, 128, 64},
        {"d2a", CONV3, 128, 64},  {"d2b", CONV3, 64, 64}, {"up2", UPCONV2, 64, 32},
        {"d1a", CONV3, 64, 32},   {"d1b", CONV3, 32, 32}, {"up1", UPCONV2, 32, 16},
        {"d0a", CONV3, 32, 16},   {"d0b", CONV3, 16, 16}, {"head", HEAD1, 16, 3}};
    int64_t off = 0;
    for (int i = 0; i < NUM_LAYERS; ++i) {
        memset(L[i].name, 0, sizeof(L[i].name));
        strncpy(L[i].name, t[i].n, sizeof(L[i].name) - 1);
        L[i].kind = t[i].k;
        L[i].cin = t[i].ci;
        L[i].cout = t[i].co;
        const int k2 = t[i].k == CONV3 ? 9 : t[i].k == UPCONV2 ? 4 : 1;
        L[i].woff = off;
        off += (int64_t)k2 * t[i].ci * t[i].co;
        L[i].boff = off;
        off += t[i].co;
    }
    return (int)off;
}

// bytes per stored activation value (the mixed FP8 network keeps level 0 in BF16)
size_t elem_size(nrv_prec p) { return p == NRV_PREC_F32 ? 4 : (p == NRV_PREC_FP8_E4M3 ? 1 : 2); }

static inline int padded_cin(const Net* net, int l) {
    return l == L_E0A ? net->c0p : net->layers[l].cin;
}

// ------------------------------------------------------------------ weight re-packing
// conv forward   wf[tap][c][o]  = W[o][c][tap]      (c < padded cin, zero beyond cin)
// conv backward  wt[tap][o][c]  = W[o][c][8 - tap]  (180-degree rotation, transposed)
// upconv         wf[a][b][c][o] = W[c][o][a][b]
// All layers in one launch: element i belongs to the layer whose range holds it.
struct RepackJobs {
    int n;
    size_t start[NUM_LAYERS + 1];
    Layer L[NUM_LAYERS];
    int cinp[NUM_LAYERS];
    size_t off[NUM_LAYERS];   // offset (floats) in wf and wt
};

__global__ void repack_f32_kernel(const float* __restrict__ P, const __grid_constant__ RepackJobs J,
                                  float* wf_all, float* wt_all) {
    const size_t all = J.start[J.n];
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < all;
         g += (size_t)gridDim.x * blockDim.x) {
        int j = 0;
        while (g >= J.start[j + 1]) ++j;
        const Layer& L = J.L[j];
        const int cinp = J.cinp[j];
        float* wf = wf_all + J.off[j];
        float* wt = wt_all + J.off[j];
        const size_t i = g - J.start[j];
        const int o = (int)(i % L.cout);
        const int c = (int)((i / L.cout) % cinp);
        const int tap = (int)(i / ((size_t)L.cout * cinp));
        if (L.kind == CONV3) {
            wf[i] = c < L.cin ? P[L.woff + ((size_t)o * L.cin + c) * 9 + tap] : 0.0f;
            // wt index: [tap][o][c] holds W[o][c][8 - tap]
            const size_t it = ((size_t)tap * L.cout + o) * cinp + c;
            wt[it] = c < L.cin ? P[L.woff + ((size_t)o * L.cin + c) * 9 + (8 - tap)] : 0.0f;
        } else {
            wf[i] = P[L.woff + ((size_t)c * L.cout + o) * 4 + tap];
        }
    }
}

nrv_status tc_repack(Net* net, cudaStream_t s);  // tc.cu

nrv_status net_repack(Net* net, cudaStream_t s) {
    size_t off = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const Layer& L = net->layers[l];
        net->wf_off[l] = off;
        const int kk = L.kind == CONV3 ? 9 : L.kind == UPCONV2 ? 4 : 0;
        off += ((size_t)kk * padded_cin(net, l) * L.cout + 63) / 64 * 64;
    }
    NRV_TRY(net->wf32.ensure(off * 4));
    NRV_TRY(net->wtf32.ensure(off * 4));
    const float* P = (const float*)net->params.p;
    RepackJobs J;
    memset(&J, 0, sizeof(J));
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const Layer& L = net->layers[l];
        if (L.kind == HEAD1) continue;
        const int kk = L.kind == CONV3 ? 9 : 4;
        J.L[J.n] = L;
        J.cinp[J.n] = padded_cin(net, l);
        J.off[J.n] = net->wf_off[l];
        J.start[J.n + 1] = J.start[J.n] + (size_t)kk * J.cinp[J.n] * L.cout;
        ++J.n;
    }
    size_t blocks = (J.start[J.n] + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    repack_f32_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, s>>>(P, J, (float*)net->wf32.p,
                                                                    (float*)net->wtf32.p);
    NRV_CHECK_LAUNCH();
    return tc_repack(net, s);
}

// ------------------------------------------------------------------ workspace
static const int kActC[NUM_ACTS] = {16, 16, 16, 32, 32, 32, 64, 64, 64, 128, 128,
                                    64, 64, 64, 32, 32, 32, 16, 16, 16};
static const int kActL[NUM_ACTS] = {0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};

nrv_status net_prepare(Net* net, int n, int H, int W, nrv_prec prec) {
    Geo g;
    g.n = n;
    g.h[0] = nrv_pad8(H);
    g.w[0] = nrv_pad8(W);
    for (int l = 1; l < 4; ++l) { g.h[l] = g.h[l - 1] / 2; g.w[l] = g.w[l - 1] / 2; }
    size_t off = 0;
    const size_t es = elem_size(prec);
    for (int a = 0; a < NUM_ACTS; ++a) {
        net->act_c[a] = kActC[a];
        net->act_level[a] = kActL[a];
        net->act_off[a] = off;
        off += (g.px(kActL[a]) * kActC[a] * es + 1023) / 1024 * 1024;
    }
    NRV_TRY(net->acts.ensure(off));
    net->geo = g;
    net->geo_H = H;
    net->geo_W = W;
    net->act_prec = prec;
    return NRV_OK;
}

template <typename T>
static T* act(Net* net, int a) {
    return reinterpret_cast<T*>((char*)net->acts.p + net->act_off[a]);
}

static int blocks_for(size_t work, int per = 256) {
    size_t b = (work + per - 1) / per;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b > 0 ? b : 1);
}

template <typename T>
static nrv_status simt_conv3(const Net* net, int l, TView<const T> x1, int c1, TView<const T> x2,
                             int c2, TView<T> y, const Geo& g, int level, bool relu,
                             cudaStream_t s) {
    const Layer& L = net->layers[l];
    Conv3Args<T> a;
    a.x1 = x1; a.x2 = x2; a.c1 = c1; a.c2 = c2;
    a.w = (const float*)net->wf32.p + net->wf_off[l];
    a.bias = (const float*)net->params.p + L.boff;
    a.y = y;
    a.cout = L.cout;
    a.n = g.n; a.h = g.h[level]; a.w_ = g.w[level];
    a.relu = relu ? 1 : 0;
    a.mask = TView<const T>{nullptr, 0};
    const size_t npx = g.px(level);
    dim3 grid((unsigned)((npx + 127) / 128), L.cout / 16);
    const size_t smem = (size_t)9 * (c1 + c2) * 16 * 4;
    conv3_simt_kernel<T><<<grid, 128, smem, s>>>(a);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

template <typename T>
static nrv_status simt_upconv(const Net* net, int l, TView<const T> x, TView<T> y, int n, int hi,
                              int wi, cudaStream_t s) {
    const Layer& L = net->layers[l];
    const size_t npx = (size_t)n * hi * wi * 4;
    dim3 grid((unsigned)((npx + 127) / 128), L.cout / 16);
    upconv2_kernel<T><<<grid, 128, (size_t)4 * L.cin * 16 * 4, s>>>(
        x, L.cin, (const float*)net->wf32.p + net->wf_off[l], (const float*)net->params.p + L.boff,
        y, L.cout, n, hi, wi);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

template <typename T>
static nrv_status forward_t(Net* net, const T* netin, float* rgb, cudaStream_t s, bool use_tc,
                            nrv_prec prec, bool keep_acts) {
    const Geo& g = net->geo;
    // BF16 activations are row-planar (the tensor-core layout), FP32 ones NHWC
    const int planar = sizeof(T) == 2 ? 1 : 0;
    auto V = [&](int a) { return TView<T>{act<T>(net, a), net->act_c[a], planar}; };
    auto CV = [&](int a) { return TView<const T>{act<T>(net, a), net->act_c[a], planar}; };
    auto conv = [&](int l, TView<const T> x1, int c1, TView<const T> x2, int c2, int out,
                    int level) -> nrv_status {
        if (use_tc) {
            nrv_status st = tc_conv3(net, l, x1.p, c1, x2.p, c2, act<T>(net, out), g, level, prec, s);
            net->backend[l] = 1;
            if (st != NRV_ERR_UNSUPPORTED) return st;
            clear_error();
        }
        net->backend[l] = 0;
        return simt_conv3<T>(net, l, x1, c1, x2, c2, V(out), g, level, true, s);
    };
    auto pool = [&](int in, int out, int level_out) -> nrv_status {
        const int c = net->act_c[in];
        pool2_kernel<T><<<blocks_for(g.px(level_out) * c / 8), 256, 0, s>>>(
            CV(in), V(out), c, g.n, g.h[level_out], g.w[level_out]);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    };
    auto upconv = [&](int l, int in, int out, int level_in) -> nrv_status {
        const Layer& L = net->layers[l];
        if (use_tc) {
            nrv_status st = tc_upconv(net, l, act<T>(net, in), act<T>(net, out), g, level_in, prec, s);
            net->backend[l] = 1;
            if (st != NRV_ERR_UNSUPPORTED) return st;
            clear_error();
        }
        net->backend[l] = 0;
        (void)L;
        return simt_upconv<T>(net, l, CV(in), V(out), g.n, g.h[level_in], g.w[level_in], s);
    };
    // a 3x3 conv whose output is also pooled to the next level (fused on the tensor cores)
    auto conv_pool = [&](int l, int in, int c1, int out, int level, int pooled) -> nrv_status {
        if (use_tc) {
            nrv_status st = tc_conv3(net, l, act<T>(net, in), c1, nullptr, 0, act<T>(net, out), g,
                                     level, prec, s, 1.0f, nullptr, act<T>(net, pooled));
            net->backend[l] = 1;
            if (st != NRV_ERR_UNSUPPORTED) return st;
            clear_error();
        }
        NRV_TRY(conv(l, CV(in), c1, TView<const T>{nullptr, 0}, 0, out, level));
        return pool(out, pooled, level + 1);
    };
    const TView<const T> x{netin, net->c0p, planar};   // one plane: also plain NHWC
    const TView<const T> none{nullptr, 0};
    NRV_TRY(conv(L_E0A, x, net->c0p, none, 0, A_E0A, 0));
    NRV_TRY(conv_pool(L_E0B, A_E0A, 16, A_E0B, 0, A_P0));
    NRV_TRY(conv(L_E1A, CV(A_P0), 16, none, 0, A_E1A, 1));
    NRV_TRY(conv_pool(L_E1B, A_E1A, 32, A_E1B, 1, A_P1));
    NRV_TRY(conv(L_E2A, CV(A_P1), 32, none, 0, A_E2A, 2));
    NRV_TRY(conv_pool(L_E2B, A_E2A, 64, A_E2B, 2, A_P2));
    NRV_TRY(conv(L_E3A, CV(A_P2), 64, none, 0, A_E3A, 3));
    NRV_TRY(conv(L_E3B, CV(A_E3A), 128, none, 0, A_E3B, 3));
    NRV_TRY(upconv(L_UP3, A_E3B, A_UP3, 3));
    NRV_TRY(conv(L_D2A, CV(A_UP3), 64, CV(A_E2B), 64, A_D2A, 2));
    NRV_TRY(conv(L_D2B, CV(A_D2A), 64, none, 0, A_D2B, 2));
    NRV_TRY(upconv(L_UP2, A_D2B, A_UP2, 2));
    NRV_TRY(conv(L_D1A, CV(A_UP2), 32, CV(A_E1B), 32, A_D1A, 1));
    NRV_TRY(conv(L_D1B, CV(A_D1A), 32, none, 0, A_D1B, 1));
    NRV_TRY(upconv(L_UP1, A_D1B, A_UP1, 1));
    NRV_TRY(conv(L_D0A, CV(A_UP1), 16, CV(A_E0B), 16, A_D0A, 0));
    const Layer& Lh = net->layers[L_HEAD];
    if (use_tc) {
        // the head in the last conv's epilogue
        const float* P = (const float*)net->params.p;
        const TcHead head{P + Lh.woff, P + Lh.boff, rgb, net->geo_H, net->geo_W, 1.0f, keep_acts,
                          net->rgb_tab};
        const nrv_status st = tc_conv3(net, L_D0B, act<T>(net, A_D0A), 16, nullptr, 0,
                                       act<T>(net, A_D0B), g, 0, prec, s, 1.0f, &head);
        net->backend[L_D0B] = 1;
        if (st != NRV_ERR_UNSUPPORTED) return st;
        clear_error();
    }
    NRV_TRY(conv(L_D0B, CV(A_D0A), 16, none, 0, A_D0B, 0));
    head_kernel<T><<<blocks_for((size_t)g.n * net->geo_H * net->geo_W), 256, 0, s>>>(
        CV(A_D0B), (const float*)net->params.p + Lh.woff, (const float*)net->params.p + Lh.boff,
        rgb, g.n, g.h[0], g.w[0], net->geo_H, net->geo_W, net->rgb_tab);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

static bool g_attr_set = false;

static nrv_status set_kernel_attrs() {
    if (g_attr_set) return NRV_OK;
    NRV_CHECK_CUDA(cudaFuncSetAttribute(conv3_simt_kernel<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 9 * 128 * 16 * 4));
    NRV_CHECK_CUDA(cudaFuncSetAttribute(conv3_simt_kernel<__nv_bfloat16>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 9 * 128 * 16 * 4));
    g_attr_set = true;
    return NRV_OK;
}

nrv_status net_forward(Net* net, const void* netin, int n, int H, int W, nrv_prec prec, float* rgb,
                       cudaStream_t s, bool keep_acts) {
    NRV_TRY(set_kernel_attrs());
    NRV_TRY(net_prepare(net, n, H, W, prec));
    net->saved = false;
    for (int l = 0; l < NUM_LAYERS; ++l) net->backend[l] = net->layers[l].kind == CONV3 ? -1 : 0;
    if (prec == NRV_PREC_F32)
        return forward_t<float>(net, (const float*)netin, rgb, s, false, prec, keep_acts);
    if (prec == NRV_PREC_BF16)
        return forward_t<__nv_bfloat16>(net, (const __nv_bfloat16*)netin, rgb, s, true, prec,
                                        keep_acts);
    if (prec == NRV_PREC_FP8) return forward_fp8_mixed(net, netin, rgb, s);
    return forward_fp8(net, (const uint8_t*)netin, rgb, s, keep_acts);
}

}  // namespace nrv

namespace nrv {

// 16-byte chunks between NHWC and row-planar order: `rows` image rows of w
// pixels with nch chunks each (planar index (row * nch + ch) * w + x).
__global__ void relayout_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t rows,
                                int w, int nch, int to_planar) {
    const size_t total = rows * (size_t)w * nch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % w);
        const size_t t = i / w;
        const int ch = (int)(t % nch);
        const size_t row = t / nch;
        const size_t nhwc = (row * w + x) * nch + ch;
        if (to_planar) dst[i] = src[nhwc];
        else dst[nhwc] = src[i];
    }
}

nrv_status relayout(const void* src, void* dst, size_t rows, int w, int c, size_t es,
                           bool to_planar, cudaStream_t s) {
    const int nch = (int)(c * es / 16);
    relayout_kernel<<<blocks_for(rows * w * nch), 256, 0, s>>>((const uint4*)src, (uint4*)dst, rows,
                                                               w, nch, to_planar ? 1 : 0);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

// One layer alone (nrv_net_run_layer): same kernels and dispatch as the forward
// pass.  The caller's tensors are NHWC; BF16 and FP8 layers run on row-planar
// copies in the handle's scratch, as inside the network.
nrv_status net_run_layer(Net* net, int l, const void* x1, const void* x2, int n, int h, int w,
                         nrv_prec prec, void* y, cudaStream_t s) {
    NRV_TRY(set_kernel_attrs());
    const Layer& L = net->layers[l];
    const bool up = L.kind == UPCONV2;
    int c1 = L.cin, c2 = 0;
    if (!up) {
        c1 = l == L_E0A ? (prec == NRV_PREC_FP8_E4M3 ? 16 : net->c0p) : L.cin;
        if (l == L_D2A || l == L_D1A || l == L_D0A) {
            c1 = L.cin / 2;
            c2 = L.cin / 2;
        }
    }
    if ((c2 > 0) != (x2 != nullptr))
        return fail(NRV_ERR_ARG, "layer %s: x2 must be %s", L.name, c2 ? "given" : "NULL");
    Geo g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.h[0] = h;
    g.w[0] = w;
    if (prec == NRV_PREC_F32) {
        net->backend[l] = 0;
        if (up)
            return simt_upconv<float>(net, l, TView<const float>{(const float*)x1, L.cin},
                                      TView<float>{(float*)y, L.cout}, n, h, w, s);
        return simt_conv3<float>(net, l, TView<const float>{(const float*)x1, c1}, c1,
                                 TView<const float>{(const float*)x2, c2}, c2,
                                 TView<float>{(float*)y, L.cout}, g, 0, true, s);
    }
    if (prec != NRV_PREC_BF16 && prec != NRV_PREC_FP8_E4M3)
        return fail(NRV_ERR_UNSUPPORTED, "nrv_net_run_layer: unknown precision");
    const size_t es = elem_size(prec);
    const size_t rows_in = (size_t)n * h, rows_out = up ? 2 * rows_in : rows_in;
    const int w_out = up ? 2 * w : w;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b1 = al(rows_in * w * c1 * es), b2 = al(rows_in * w * c2 * es);
    const size_t by = al(rows_out * w_out * L.cout * es);
    NRV_TRY(net->layer_ws.ensure(b1 + b2 + by));
    char* ws = (char*)net->layer_ws.p;
    void *p1 = ws, *p2 = c2 ? ws + b1 : nullptr, *py = ws + b1 + b2;
    NRV_TRY(relayout(x1, p1, rows_in, w, c1, es, true, s));
    if (c2) NRV_TRY(relayout(x2, p2, rows_in, w, c2, es, true, s));
    float inv_out = 1.0f;
    if (prec == NRV_PREC_FP8_E4M3) {
        int in1, in2, out;
        layer_scale_index(l, &in1, &in2, &out);
        inv_out = 1.0f / net->act_scale[out];
    }
    nrv_status st = up ? tc_upconv(net, l, p1, py, g, 0, prec, s, inv_out)
                       : tc_conv3(net, l, p1, c1, p2, c2, py, g, 0, prec, s, inv_out);
    net->backend[l] = 1;
    if (st == NRV_ERR_UNSUPPORTED && prec == NRV_PREC_BF16) {
        clear_error();
        net->backend[l] = 0;
        using T = __nv_bfloat16;
        st = up ? simt_upconv<T>(net, l, TView<const T>{(const T*)p1, L.cin, 1},
                                 TView<T>{(T*)py, L.cout, 1}, n, h, w, s)
                : simt_conv3<T>(net, l, TView<const T>{(const T*)p1, c1, 1}, c1,
                                TView<const T>{(const T*)p2, c2, 1}, c2,
                                TView<T>{(T*)py, L.cout, 1}, g, 0, true, s);
    }
    NRV_TRY(st);
    return relayout(py, y, rows_out, w_out, L.cout, es, false, s);
}

}  // namespace nrv
