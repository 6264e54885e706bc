// The U-Net handle: layer table, packed weights, activation workspace.
#pragma once
#include <cuda.h>

#include "internal.h"

namespace nrv {

// Device buffer owned by a handle; grows, never shrinks.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    nrv_status ensure(size_t b);
    void release();
    ~DevBuf() { release(); }
};

// Per-level geometry of one network invocation.
struct Geo {
    int n, h[4], w[4];
    size_t px(int l) const { return (size_t)n * h[l] * w[l]; }
};

// Activations of one forward pass (element type given by the precision).
enum Act {
    A_E0A, A_E0B, A_P0, A_E1A, A_E1B, A_P1, A_E2A, A_E2B, A_P2, A_E3A, A_E3B, A_UP3, A_D2A,
    A_D2B, A_UP2, A_D1A, A_D1B, A_UP1, A_D0A, A_D0B, NUM_ACTS
};

struct Net {
    int c_in = 0, c0p = 8;
    Layer layers[NUM_LAYERS];
    int64_t n_params = 0;
    bool has_params = false;
    float act_scale[NUM_ACTS + 1];   // FP8 scales: [0] input, [1 + a] activation a
    bool fp8_ready = false;          // FP8 weights packed for the current scales
    DevBuf params;     // FP32 master copy (flat layout)
    DevBuf wf32;       // FP32 packed forward weights, per layer at wf_off
    DevBuf wtf32;      // FP32 packed backward-data weights, per layer at wf_off
    DevBuf wbf16;      // BF16 tcgen05 operand layout, per layer at wb_off
    DevBuf wtbf16;     // BF16 backward-data operand layout
    DevBuf wfp8;       // FP8 tcgen05 operand layout
    DevBuf wscale8;    // FP8 per-output-channel weight scales (floats)
    size_t wf_off[NUM_LAYERS];
    size_t wb_off[NUM_LAYERS];
    size_t ws8_off[NUM_LAYERS];
    // workspace of the last forward
    DevBuf acts;
    size_t act_off[NUM_ACTS];
    int act_c[NUM_ACTS];
    int act_level[NUM_ACTS];
    Geo geo{};
    int geo_H = 0, geo_W = 0;
    nrv_prec act_prec = NRV_PREC_F32;
    int backend[NUM_LAYERS];   // 0 SIMT, 1 tcgen05, -1 not run (last forward)
    nrv_loss_weights loss_w{1.0f, 0.0f, 0.0f};   // training loss of nrv_train_step (L1)
    RgbTab rgb_tab{};        // per-image RGB destinations of the next forward (render batches)
    bool saved = false;      // a training forward's activations are in place
    const void* saved_in = nullptr;   // that forward's input (the first layer's weight gradient reads it)
    // backward scratch
    DevBuf grads;            // gradient tensors
    DevBuf partial;          // wgrad partial sums
    DevBuf tmaps;            // device copies of TMA descriptors (unused when passed by value)
    // render-batch resources
    DevBuf batch_ws;
    DevBuf layer_ws;         // row-planar copies for nrv_net_run_layer
};

size_t elem_size(nrv_prec p);
nrv_status net_prepare(Net* net, int n, int H, int W, nrv_prec prec);
// keep_acts false: the last conv's output, which only a backward reads, need not be stored
nrv_status net_forward(Net* net, const void* netin, int n, int H, int W, nrv_prec prec, float* rgb,
                       cudaStream_t s, bool keep_acts = true);
nrv_status net_backward(Net* net, const float* drgb, float* dparams, cudaStream_t s);
// weight and bias gradient of one 3x3 conv layer from NHWC tensors (train.cu)
nrv_status net_layer_wgrad(Net* net, int l, const void* dy, const void* x1, const void* x2, int n,
                           int h, int w, nrv_prec prec, float* dgrad, cudaStream_t s);
// data gradient of one 3x3 conv layer from NHWC tensors (train.cu)
nrv_status net_layer_dgrad(Net* net, int l, const void* dy, const void* mask, int n, int h, int w,
                           nrv_prec prec, void* dx, cudaStream_t s);
// 16-byte chunks between NHWC and row-planar order (net.cu): `rows` rows of w pixels, c
// channels of es bytes
nrv_status relayout(const void* src, void* dst, size_t rows, int w, int c, size_t es,
                    bool to_planar, cudaStream_t s);
nrv_status net_repack(Net* net, cudaStream_t s);
// parameters in and out (netio.cu): Xavier-uniform draw into d_params, file save / load
nrv_status net_init_params(const Net* net, uint64_t seed, float* d_params, cudaStream_t s);
nrv_status net_save(const Net* net, const char* path, cudaStream_t s);
nrv_status net_load(Net* net, const char* path, cudaStream_t s);

// The 1x1 head fused into the last conv's epilogue: weights w[3][16], bias b[3], output
// rgb[n][h][w_px][3] FP32 cropped to h x w_px; scale: E4M3 scale of the stored conv output
// (1 for BF16); store_y false skips storing the conv output itself.
struct TcHead {
    const float* w;
    const float* b;
    float* rgb;
    int h, w_px;
    float scale;
    bool store_y;
    RgbTab tab;      // per-image destinations (tab.on), else rgb + img * h * w_px * 3
};

// tensor-core convolution (tc.cu); returns NRV_ERR_UNSUPPORTED when a shape is not covered
nrv_status tc_conv3(const Net* net, int layer, const void* x1, int c1, const void* x2, int c2,
                    void* y, const Geo& g, int level, nrv_prec prec, cudaStream_t s,
                    float inv_out = 1.0f, const TcHead* head = nullptr,
                    void* pool_y = nullptr);   // pool_y: also the 2x2 average pool of y
nrv_status tc_upconv(const Net* net, int layer, const void* x, void* y, const Geo& g, int level_in,
                     nrv_prec prec, cudaStream_t s, float inv_out = 1.0f);
nrv_status tc_repack_fp8(Net* net, cudaStream_t s);
// TMA map of a row-planar tensor [n][h][nch][w][16 bytes] (tc.cu): boxes of 128 pixels x
// box_planes planes of one row
nrv_status tc_planar_map(CUtensorMap* map, const void* base, int n, int h, int w, int nch,
                         int box_planes);
// TMA map of the pixels of one parity b of a row-planar tensor with `rows` rows (all images)
// of w pixels (w even) and nch planes: 8-byte elements (half, parity, pixel pair, plane, row);
// a box is 128 pixel pairs x box_planes planes of one row at one parity (tc.cu)
nrv_status tc_parity_map(CUtensorMap* map, const void* base, int rows, int w, int nch,
                         int box_planes);
// Weight gradient of a 2x2 stride-2 transposed conv on the tensor cores (wgrad_tc.cu):
// part[split][c][ab * C_out + o] over the input level (n, H, W); x at (H, W), g at (2H, 2W),
// both BF16 row-planar; g holds g_ld channels of which C_out from channel g_off on (the
// upsampled half of a concatenation's gradient).
nrv_status tc_wgrad_up(const Net* net, int l, const void* g, int g_ld, int g_off, const void* x,
                       int n, int H, int W, float* part, size_t part_floats, float* partb,
                       int* nsplit, cudaStream_t s);
// Weight gradient of 3x3 conv layer l on the tensor cores (wgrad_tc.cu), BF16 row-planar:
// part[split][o][tap][c] (FP32 partial sums over each split's pixels, c over all input channels)
// for the output gradient g (C_out channels) and the layer input (x1: c1 channels, x2: c2 or
// none), and partb[split][o] (bias; the transposed conv: partb[split][ab * C_out + o]);
// *nsplit receives the number of splits.  NRV_ERR_UNSUPPORTED when the shape is not covered
// (input channels not a multiple of 16, except one group of 8).
nrv_status tc_wgrad(const Net* net, int l, const void* g, const void* x1, int c1, const void* x2,
                    int c2, int n, int H, int W, float* part, size_t part_floats, float* partb,
                    int* nsplit, cudaStream_t s);
// data gradient of 3x3 conv layer l on the tensor cores (BF16, row-planar): out = conv3x3 of
// the output gradient gin with the flipped, transposed kernel, zeroed where mask <= 0 (mask
// may be null); NRV_ERR_UNSUPPORTED when the layer has no such path
nrv_status tc_dgrad(const Net* net, int l, const void* gin, void* out, const void* mask, int n, int H,
                    int W, cudaStream_t s);
// data gradient of transposed conv l on the tensor cores (BF16, row-planar): out (C_in at the
// input level (n, H, W)) from the output gradient g at (2H, 2W), which holds g_ld channels of
// which C_out from g_off on, zeroed where mask (shaped like out) is not positive
nrv_status tc_updgrad(const Net* net, int l, const void* g, int g_ld, int g_off, const void* mask,
                      void* out, int n, int H, int W, cudaStream_t s);
// A layer of another network on the tensor-core conv kernel (tc.cu): a 3x3 conv (plain or
// gated) or a 2x2 stride-2 transposed conv, BF16 row-planar in and out.  c1, c2: the stored
// channels of the sources (multiples of 8; c2 = 0 without a second source), cin_real: the
// weights' input channels (<= c1 + c2; the real channels come first in each source);
// woff / boff: the weights and bias in the flat parameter vector, woff2 / boff2 the gate's.
struct TcGeneric {
    int kind, gated;
    int c1, c2, cin_real, cout;
    int64_t woff, boff, woff2, boff2;
};
struct TcPacked;
nrv_status tc_generic_prepare(const TcGeneric* L, int n, const float* params, TcPacked** state,
                              cudaStream_t s);
nrv_status tc_generic_run(const TcPacked* st, int l, const float* params, const void* x1,
                          const void* x2, void* y, int n, int H, int W, cudaStream_t s,
                          const TcHead* head = nullptr, void* pool_y = nullptr);
void tc_generic_free(TcPacked* st);
nrv_status forward_fp8(Net* net, const uint8_t* netin, float* rgb, cudaStream_t s, bool keep_acts);
// levels 1-3 in E4M3, level 0 in BF16 (fp8.cu); netin is the BF16 packed input
nrv_status forward_fp8_mixed(Net* net, const void* netin, float* rgb, cudaStream_t s);
// FP8 scale indices (0 input, 1 + Act) of a layer's first input, second input (-1 if none)
// and output (-1 for the head)
void layer_scale_index(int l, int* in1, int* in2, int* out);
nrv_status net_calibrate(Net* net, const void* netin, int n, int H, int W, cudaStream_t s);

// training kernels (train.cu)
nrv_status launch_l1(const float* y, const float* t, int64_t n, float* loss, float* dy,
                     cudaStream_t s);
nrv_status launch_recon(const float* y, const float* t, int n_img, int h, int w,
                        const nrv_loss_weights& wt, float* loss, float* dy, cudaStream_t s);
nrv_status launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step,
                       float lr, float b1, float b2, float eps, cudaStream_t s);

}  // namespace nrv

namespace nrv {
nrv_status net_run_layer(Net* net, int l, const void* x1, const void* x2, int n, int h, int w,
                     nrv_prec prec, void* y, cudaStream_t s);
}
