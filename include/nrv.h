/*
 * nrv.h -- C ABI of libnrv, a GB300 (sm_103a) implementation of the hot path of
 * NARVis, the neural accelerated renderer for scientific point clouds
 * (arXiv 2407.19097):
 *
 *   1. the multi-attribute compute rasterizer (Sec. 3.2): a render pass that
 *      projects every point and keeps, per pixel, the closest one via a 64-bit
 *      atomic minimum of (depth bits << 32 | point index), then a resolve pass
 *      that copies the winner's attributes, depth and coverage into G-buffers;
 *   2. the neural deferred renderer (Sec. 3.3): a U-Net that turns the packed
 *      G-buffer into the final RGB image, with its forward and backward passes,
 *      an L1 loss and Adam for training (Sec. 3.3, training details).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an nrv_status.  NRV_OK is 0.  On failure the
 *    message of the calling thread's last error is available from
 *    nrv_last_error().  No C++ exception crosses this boundary.
 *  - Pointers named d_* are CUDA device pointers owned by the caller.  The
 *    library borrows them for the duration of the call (or, for a scene, for
 *    the scene's lifetime) and never frees them.  Handles own only their
 *    internal scratch (packed weights, activation workspaces, graphs).
 *  - All device work is enqueued on the given stream (NULL = the legacy
 *    default stream) and is asynchronous: an error inside a kernel shows up at
 *    a later synchronisation, or as a status word read by nrv_sync_status().
 *  - Images are row-major with row 0 at the top.  Network tensors are NHWC.
 *  - The library runs on the current CUDA device of the calling thread.  It
 *    has no CPU fallback: without a CUDA device every call that launches work
 *    returns NRV_ERR_CUDA.
 *  - Calls that launch work share process-wide tables (the packed-weight
 *    layouts of the tensor-core kernels, the tuned render-pass variant, kernel
 *    attributes): make them from one host thread at a time.  A scene or net
 *    handle and its workspaces serve one call at a time.
 */
#ifndef NRV_H
#define NRV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared opaquely so this header needs no CUDA headers. */
typedef struct CUstream_st* nrv_stream;

typedef enum {
    NRV_OK = 0,
    NRV_ERR_ARG = 1,          /* invalid argument: null, misaligned, out of range */
    NRV_ERR_CUDA = 2,         /* a CUDA runtime/driver call failed */
    NRV_ERR_OOM = 3,          /* device allocation failed */
    NRV_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    NRV_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement */
    NRV_ERR_STATE = 6         /* call out of order (e.g. backward before forward) */
} nrv_status;

/* Attribute word formats (Sec. 3.2: "formats uint8 and fp32"), and the derived
 * channels the resolve can compute from the winning point (Sec. 3.2 and Sec. 4.5):
 *  NRV_VEL2D_X, NRV_VEL2D_Y, NRV_VEL2D_ANGLE, NRV_VEL2D_MAG -- "Vel2D" (Sec. 4.5,
 *    Tab. 7): the point's velocity v = (word w, w+1, w+2 as FP32) projected by the
 *    camera.  With s(p) = ((c.x/c.w + 1) W/2, (1 - c.y/c.w) H/2), c = viewproj (p, 1),
 *    v' = (ds/dp) v in pixels per unit time (x right, y down), the channels are
 *    v'.x, v'.y, atan2(v'.y, v'.x) in (-pi, pi] and |v'|;
 *  NRV_SPLAT_RADIUS -- the projected splat radius (Sec. 3.2, terrain): a world
 *    radius r (word w as FP32) in pixels, r (H/2) |viewproj row 1 (x, y, z)| / c.w,
 *    the pixel radius of a camera-facing disc for a perspective camera.
 * Derived channels are computed in FP32 (not bit-exact: within about 1e-5 of an FP64
 * evaluation) and need the point's position and the camera, so only the passes that
 * resolve from the key image take them (nrv_resolve_pack, nrv_render_batch). */
typedef enum {
    NRV_F32 = 0, NRV_U32 = 1, NRV_U8X4 = 2,
    NRV_VEL2D_X = 3, NRV_VEL2D_Y = 4, NRV_VEL2D_ANGLE = 5, NRV_VEL2D_MAG = 6,
    NRV_SPLAT_RADIUS = 7
} nrv_fmt;

/* Network precision.  Accumulation is FP32 in every mode (the paper's App. B quantises to
 * fp16; the reduced-precision modes here go to BF16 and 8 bits).
 *  NRV_PREC_F32       FP32 on the CUDA cores.
 *  NRV_PREC_BF16      BF16 operands and activations on the tensor cores.
 *  NRV_PREC_FP8       the FP8 network: E4M3 operands and activations for levels 1-3, BF16
 *                     for the full-resolution level 0 (its input is the BF16 G-buffer).  With
 *                     Xavier-initialised weights it stays within 2e-2 max abs (and 45 dB) of
 *                     an FP64 forward on full frames; with trained weights its PSNR stays
 *                     above 45 dB but single pixels reach several percent of the output
 *                     range (E4M3 keeps 3 mantissa bits).
 *  NRV_PREC_FP8_E4M3  every stored tensor E4M3 (a 16-channel E4M3 input): faster, but its
 *                     3-bit mantissas compound over the full-resolution layers to max-abs
 *                     errors of about 0.1 on full frames, above that bound. */
typedef enum {
    NRV_PREC_F32 = 0,
    NRV_PREC_BF16 = 1,
    NRV_PREC_FP8_E4M3 = 2,
    NRV_PREC_FP8 = 3
} nrv_prec;

/* --------------------------------------------------------------------------
 * Library
 * ------------------------------------------------------------------------ */

/* Message of the calling thread's most recent failure ("" if none).  The
 * pointer stays valid until the thread's next nrv_* call. */
const char* nrv_last_error(void);

/* ABI version, currently 1. */
int nrv_version(void);

/* Number of kernels the library has launched in this process so far (all
 * devices, all threads).  Replays of captured frames count the kernels they
 * contain.  For benchmarking. */
uint64_t nrv_launch_count(void);

/* Number of compiled variants of the render pass (visibility) kernel for one
 * view (multi_view = 0) or a batch of views (multi_view != 0).  All variants
 * compute the same keys; the library times them on the first large launch and
 * keeps the fastest.  Setting the environment variable NRV_VIS_VARIANT to an
 * index below this count pins that variant (used to check each one).  The
 * kernels of the chunk-culling variants and the tensor-core network layers are
 * launched as programmatic dependents of their predecessors (each waits for the
 * previous kernel before reading its results); NRV_PDL=0 launches them plainly. */
int nrv_render_variants(int multi_view);

/* --------------------------------------------------------------------------
 * Scene (the point cloud of Sec. 3.2; memory N * sum(B_i) bytes, Sec. 4.5)
 * ------------------------------------------------------------------------ */

typedef struct {
    uint64_t n_points;       /* N, 0 <= N < 2^32 (the index is the key's low word) */
    const float* d_xyz;      /* device, N*3 floats (x, y, z), base 16-byte aligned */
    const uint32_t* d_attr;  /* device, N*stride_words words: one record per point */
    int stride_words;        /* record stride in 32-bit words: 1, 2, 4 or 8 */
    int n_words;             /* K: record words copied to the G-buffer, 1..stride_words
                                (Sec. 3.2 tests up to 8 attributes) */
    int point_stride;        /* 0 or 1: every point.  S > 1: the scene's point j is point j*S of
                                the arrays (position d_xyz[3 j S], record d_attr at j S
                                stride_words) and keys carry j*S -- a masked render pass over a
                                sparse subset, e.g. the glyph points (every 50th, Sec. 4.3) for
                                "VisGlyph" (Tab. 2: the frontmost glyph point, ignoring the
                                non-glyph points in front of it).  N counts the subset */
    uint64_t index_base;     /* global index of the first point (0 for a whole scene): key
                                low words are index_base + i, index_base + N < 2^32.  A
                                shard of a larger scene takes its first point's index, so
                                keys rendered from several shards can be combined by a
                                minimum, and the resolve of a shard treats winners outside
                                its own index range as empty pixels */
} nrv_scene_desc;

typedef struct nrv_scene nrv_scene;

/* Describe a scene.  Borrows d_xyz and d_attr, which must outlive the scene.
 * The first render derives from d_xyz a bounding box for every chunk of 32
 * consecutive points and for each of its four sub-chunks of 8 points
 * (ceil(N/32) * 120 bytes of device memory, owned by the scene) for occlusion
 * culling in the render pass.
 * Errors: NRV_ERR_ARG for a null pointer with N > 0, a d_xyz base that is not
 * 16-byte aligned, a d_attr base not aligned to min(16, 4*stride_words) bytes,
 * N >= 2^32, a stride not in {1,2,4,8} or K out of range. */
nrv_status nrv_create_scene(const nrv_scene_desc* desc, nrv_scene** out);
nrv_status nrv_destroy_scene(nrv_scene* scene);

/* Tell the scene that the positions behind d_xyz changed: the next render
 * recomputes the chunk bounds (on its stream) before it uses them.  Rendering
 * after a change without this call may drop points that are now visible.
 * No counterpart in the paper (its rasterizer relies on early depth tests
 * alone).  Errors: NRV_ERR_ARG for a null scene. */
nrv_status nrv_scene_refresh(nrv_scene* scene);

/* One camera.  clip = viewproj * (x, y, z, 1)^T with viewproj row-major FP32;
 * clip.w is the eye-space depth.  A point is kept when znear <= w <= zfar and
 * its pixel ((ndc.x + 1) W/2, (1 - ndc.y) H/2), truncated, is on screen. */
typedef struct {
    float viewproj[16];
    int width, height;       /* 1..16384 each */
    float znear, zfar;       /* 0 < znear <= zfar */
} nrv_view;

/* Raw G-buffer planes of one view, caller-owned device memory of H*W pixels.
 * d_key is required.  d_depth (FP32 bits of the winner's w), d_mask (1 where
 * covered) and d_attr (K planar u32 planes, plane c at d_attr + c*H*W) may be
 * NULL to skip them.  Empty pixels get key ~0 and zeros in every other plane. */
typedef struct {
    uint64_t* d_key;
    uint32_t* d_depth;
    uint8_t* d_mask;
    uint32_t* d_attr;
} nrv_gbuffer;

/* Render + resolve passes of the multi-attribute compute rasterizer (Sec. 3.2)
 * for n_views views of one scene: clear every key image, project each point
 * once per view and keep the minimum key (bits(w) << 32 | index; ties to the
 * lowest index), then resolve every pixel.  The render pass may skip chunks of
 * points that provably cannot set a key (outside every view, or behind the
 * depths already written over all the pixels they can reach); the keys are the
 * same as when every point is projected.
 * Keys and planes are bit-exact: the projection is the fixed FP32 sequence
 *   c = ((m0*x + m1*y) + m2*z) + m3 per row (no fused multiply-add),
 *   ndc = c.xy / c.w (IEEE division).
 * n_views in 1..8; gbufs has n_views entries.  Errors: NRV_ERR_ARG. */
nrv_status nrv_rasterize(nrv_scene* scene, const nrv_view* views, int n_views,
                         const nrv_gbuffer* gbufs, nrv_stream stream);

/* Resolve pass alone (Sec. 3.2) from a key image d_key ([H][W], e.g. combined from
 * several shards): gbuf's d_depth, d_mask and d_attr planes (any may be NULL) get the
 * winner's depth bits, coverage and record words where the winner belongs to this
 * scene (index_base <= index < index_base + N) and zeros elsewhere, so the planes of
 * all shards add up to those of the whole scene.  gbuf->d_key is ignored.
 * Errors: NRV_ERR_ARG. */
nrv_status nrv_resolve(nrv_scene* scene, const nrv_view* view, const uint64_t* d_key,
                       const nrv_gbuffer* gbuf, nrv_stream stream);

/* Flip bit 63 of n keys in place (an involution).  It maps the unsigned order of keys
 * onto the signed order of int64 -- the empty key ~0 becomes INT64_MAX -- so that a
 * signed 64-bit minimum (a collective's MIN on int64) combines key images of shards.
 * No counterpart in the paper.  Errors: NRV_ERR_ARG. */
nrv_status nrv_keys_flip_sign(uint64_t* d_key, int64_t n, nrv_stream stream);

/* How to turn one view's G-buffer into the network input ("channel-wise
 * processing" of the rasterizer output, Sec. 4.5 / Tab. 3).  Channel j < n_channels
 * reads G-buffer word word[j] as f32, u32 or byte comp[j] of a u8x4 word (or, for a
 * derived format, computes its value from the winning point, see nrv_fmt) and
 * becomes f = float(v) * scale[j] + offset[j] (separate FP32 multiply and add).
 * Then comes depth (float of the depth plane, same affine map with depth_scale
 * and depth_offset), then coverage (1.0), then zero padding.  Empty pixels are
 * all zero.  C_in of the network = n_channels + 2 (at most 8). */
typedef struct {
    int n_channels;          /* 1..6 */
    int word[6];
    int fmt[6];              /* nrv_fmt */
    int comp[6];             /* byte 0..3 for NRV_U8X4 */
    float scale[6];
    float offset[6];
    float depth_scale, depth_offset;
} nrv_pack_desc;

/* Network-input geometry for an H x W view: the canvas is Hn x Wn with
 * Hn, Wn = H, W rounded up to multiples of 8 (zero margin, cropped again at
 * the output) and C channels per pixel: 8 for F32, BF16 and FP8 (a BF16 input),
 * 16 for FP8_E4M3. */
int nrv_pad8(int v);
int nrv_netin_channels(nrv_prec prec);

/* Pack one view's G-buffer (d_depth, d_mask and d_attr required) into the
 * network input d_netin: NHWC [Hn][Wn][C] of float, bf16 (round to nearest
 * even) or e4m3 (of f * in_scale_inv, saturating, round to nearest even).
 * Errors: NRV_ERR_ARG (also for derived channel formats: use nrv_resolve_pack). */
nrv_status nrv_pack(const nrv_gbuffer* gbuf, int height, int width, const nrv_pack_desc* desc,
                    nrv_prec prec, float in_scale_inv, void* d_netin, nrv_stream stream);

/* Resolve pass fused with the packing (Sec. 3.2 resolve + Sec. 4.5 channel
 * processing): from one view's key image d_key ([H][W], as written by
 * nrv_rasterize for that view) straight to the network input d_netin (layout of
 * nrv_pack), gathering the winner's record -- and, for derived channels, its
 * position -- from the scene.  The same pass nrv_render_batch runs.
 * Errors: NRV_ERR_ARG (null, misaligned, a channel reading past the record). */
nrv_status nrv_resolve_pack(nrv_scene* scene, const nrv_view* view, const uint64_t* d_key,
                            const nrv_pack_desc* desc, nrv_prec prec, float in_scale_inv,
                            void* d_netin, nrv_stream stream);

/* --------------------------------------------------------------------------
 * Network (post-processing U-Net, Sec. 3.3)
 *
 * Fixed architecture: levels l = 0..3 at H/2^l with 16/32/64/128 channels;
 * encoder: two 3x3 same convolutions + bias + ReLU per level and 2x2 average
 * pooling between levels; decoder: 2x2 stride-2 transposed convolution (bias,
 * no activation), concatenation [upsampled, skip], two 3x3 conv + ReLU; head:
 * 1x1 convolution to RGB, linear.  Layer order: e0a e0b e1a e1b e2a e2b e3a
 * e3b up3 d2a d2b up2 d1a d1b up1 d0a d0b head.
 *
 * Parameters are exchanged as one flat FP32 vector: per layer in that order,
 * the weight in PyTorch's layout -- conv (C_out, C_in, 3, 3), transposed conv
 * (C_in, C_out, 2, 2), head (C_out, C_in) -- followed by the bias (C_out).
 * ------------------------------------------------------------------------ */

typedef struct nrv_net nrv_net;

typedef struct {
    char name[8];
    int kind;                /* 0 = 3x3 conv, 1 = 2x2 stride-2 transposed conv, 2 = 1x1 head */
    int c_in, c_out;
    int64_t weight_offset;   /* offset of the weight in the flat vector (floats) */
    int64_t bias_offset;
} nrv_layer_info;

/* Number of layers (18), per-layer layout and the total parameter count for a
 * network with c_in input channels (1..8).  Errors: NRV_ERR_ARG. */
int nrv_net_num_layers(void);
nrv_status nrv_net_layer(int c_in, int layer, nrv_layer_info* out);
nrv_status nrv_net_param_count(int c_in, int64_t* count);

/* Create a network for c_in input channels.  The library allocates only its
 * packed low-precision weight copies and workspaces.  Errors: NRV_ERR_ARG,
 * NRV_ERR_OOM. */
nrv_status nrv_create_net(int c_in, nrv_net** out);
nrv_status nrv_destroy_net(nrv_net* net);

/* Load weights from a flat FP32 device vector (layout above) and re-derive the
 * packed BF16 and FP8 copies (FP8: per-output-channel scale amax/448).  Call
 * again after the parameters change.  Errors: NRV_ERR_ARG. */
nrv_status nrv_net_set_params(nrv_net* net, const float* d_params, nrv_stream stream);

/* Fill the caller's d_params (parameter count floats, device) with a seeded
 * Xavier-uniform draw and load it: biases 0; element i of layer t's weight (in
 * the layout above) = the FP32 value nearest to -b + 2b*u, b = sqrt(6 / (fan_in
 * + fan_out)), fan = channels x kernel area, u = the top 53 bits of output i of
 * SplitMix64 stream 1000 + t as a double in [0, 1).  The stream's state is the
 * (stream)-th output of the SplitMix64 sequence seeded with `seed`; the i-th
 * output of a sequence with state s is mix(s + (i+1) * 0x9E3779B97F4A7C15).  The
 * paper trains its network from scratch (Sec. 3.3) and gives no initialisation;
 * this is the library's.  Errors: NRV_ERR_ARG. */
nrv_status nrv_net_init_params(nrv_net* net, uint64_t seed, float* d_params, nrv_stream stream);

/* Copy the net's FP32 parameters (layout above) to the caller's device buffer.
 * Errors: NRV_ERR_ARG, NRV_ERR_STATE (no parameters loaded). */
nrv_status nrv_net_get_params(const nrv_net* net, float* d_out, nrv_stream stream);

/* Save the parameters and, when set, the FP8 activation scales to a file, or
 * load them (replacing both, repacking every low-precision copy).  Format:
 * "NRVNET01", int32 c_in, int32 flags (bit 0: scales present), int64 parameter
 * count, the FP32 parameters, 21 FP32 scales; little-endian.  Both synchronise
 * the stream.  No counterpart in the paper.  Errors: NRV_ERR_ARG (I/O, a file
 * for another input width, a malformed file), NRV_ERR_STATE (save without
 * parameters). */
nrv_status nrv_net_save(const nrv_net* net, const char* path, nrv_stream stream);
nrv_status nrv_net_load(nrv_net* net, const char* path, nrv_stream stream);

/* E4M3 tensors of the FP8 modes: every E4M3 tensor the network stores holds codes q with
 * value q * scale, one scale per tensor; weights hold E4M3 codes per output
 * column with scale max|column| / 448 (App. B quantises to fp16; this goes to
 * 8 bits).  The 21 tensor scales, in this order: the network input, then
 * e0a e0b p0 e1a e1b p1 e2a e2b p2 e3a e3b up3 d2a d2b up2 d1a d1b up1 d0a d0b
 * (the outputs of those layers; p0..p2 the pooled tensors, which must carry the
 * scale of the tensor they pool).  For NRV_PREC_FP8_E4M3 the input is packed by
 * nrv_pack / passed to nrv_render_batch with in_scale_inv = 1 / scale[0].
 *
 * nrv_net_calibrate runs a BF16 forward on n sample inputs (BF16 NHWC, as for
 * nrv_shade), sets every scale to max|tensor| / 448 and packs the E4M3 weights.
 * It synchronises the stream.  nrv_net_set_act_scales sets the scales directly
 * (positive, finite) and packs the weights; nrv_net_get_act_scales reads them.
 * Both packers need parameters loaded (NRV_ERR_STATE otherwise) and are rerun
 * by nrv_net_set_params once scales exist.
 *
 * NRV_PREC_FP8 uses the scales of levels 1-3 only: level 0 (the input, e0a, e0b,
 * up1, d0a, d0b) stays BF16 and the input is the BF16 packed input.
 * NRV_PREC_FP8_E4M3 uses all of them.  Both need the scales (NRV_ERR_STATE). */
nrv_status nrv_net_calibrate(nrv_net* net, const void* d_netin_bf16, int n, int height, int width,
                             nrv_stream stream);
nrv_status nrv_net_set_act_scales(nrv_net* net, const float* scale, int n, nrv_stream stream);
nrv_status nrv_net_get_act_scales(const nrv_net* net, float* scale, int n);

/* Forward pass (inference) on n images: d_netin is n packed inputs
 * [n][Hn][Wn][C] in the dtype of prec (nrv_netin_channels), d_rgb receives
 * [n][height][width][3] FP32, cropped to height x width.
 * Errors: NRV_ERR_ARG, NRV_ERR_STATE (no parameters loaded), NRV_ERR_OOM. */
nrv_status nrv_shade(nrv_net* net, const void* d_netin, int n, int height, int width,
                     nrv_prec prec, float* d_rgb, nrv_stream stream);

/* One layer of the net on its own, NHWC, input [n][h][w][.]:
 *  - a 3x3 convolution (kind 0): y = ReLU(conv3x3(concat(x1, x2)) + bias), zero
 *    "same" padding, y [n][h][w][C_out].  x1 has the layer's first-source
 *    channels (8 for e0a, C_in/2 for the concatenating layers d2a/d1a/d0a, C_in
 *    otherwise); x2 holds the skip half for d2a/d1a/d0a, NULL for the others;
 *  - a 2x2 stride-2 transposed convolution (kind 1): y[2i+a][2j+b][o] =
 *    bias[o] + sum_c x1[i][j][c] W[c][o][a][b], y [n][2h][2w][C_out]; x2 NULL.
 * Element type from prec: F32 (SIMT kernels) or BF16 (tensor-core kernels).  The
 * building blocks of nrv_shade, exposed so a layer can be checked or reused alone.
 * Errors: NRV_ERR_ARG, NRV_ERR_STATE (no parameters), NRV_ERR_UNSUPPORTED. */
nrv_status nrv_net_run_layer(nrv_net* net, int layer, const void* d_x1, const void* d_x2, int n,
                             int h, int w, nrv_prec prec, void* d_y, nrv_stream stream);

/* Weight and bias gradient of one 3x3 or 2x2 stride-2 transposed convolution layer
 * (Sec. 3.3's network; the backward of nrv_net_backward, exposed so that it can be
 * checked or reused alone):
 *   3x3:        dW[o][c][u][v] = sum_p dy[p][o] * x[p + (u - 1, v - 1)][c]  (zero outside),
 *   transposed: dW[c][o][a][b] = sum_(i,j) x[i][j][c] * dy[2i + a][2j + b][o],
 *   db[o] = sum of dy[.][o] over all output pixels.
 * d_x1: [n][h][w][c1] and d_x2: [n][h][w][c2] for the concatenating decoder layers
 * (else NULL); d_dy: [n][h][w][C_out] (3x3: the gradient at the layer's pre-activation
 * output) or [n][2h][2w][C_out] (transposed); all NHWC in `prec` (F32 or BF16; the
 * first layer's input has the padded width of nrv_pack).  Writes dW (PyTorch
 * layout) and db into their places in d_grad (the flat parameter layout); other
 * entries are untouched.  BF16 runs on the tensor cores (FP32 accumulation, then a
 * fixed-order sum of partials: deterministic); F32 on the CUDA cores.  Uses the
 * net's workspaces (one call at a time per net).
 * Errors: NRV_ERR_ARG (null, misaligned, the head, x2 given or missing),
 * NRV_ERR_UNSUPPORTED (FP8). */
nrv_status nrv_net_layer_wgrad(nrv_net* net, int layer, const void* d_dy, const void* d_x1,
                               const void* d_x2, int n, int h, int w, nrv_prec prec,
                               float* d_grad, nrv_stream stream);

/* Data gradient of one 3x3 or 2x2 stride-2 transposed convolution layer (the backward of
 * Sec. 3.3's network, exposed like nrv_net_layer_wgrad):
 *   3x3:        dx[p][c] = sum_{o,u,v} W[o][c][u][v] * dy[p - (u - 1, v - 1)][o]  (zero outside),
 *   transposed: dx[i][j][c] = sum_{o,a,b} W[c][o][a][b] * dy[2i + a][2j + b][o],
 * then dx[p][c] = 0 where d_mask[p][c] <= 0 when d_mask is not NULL (the ReLU of the layer
 * below: pass its output; required for a transposed conv).  d_dy: [n][h][w][C_out] (3x3) or
 * [n][2h][2w][C_out] (transposed); d_mask and d_dx: [n][h][w][C_in] (both halves of a
 * concatenation); NHWC in `prec` (F32 or BF16).  BF16 runs on the tensor cores (the 3x3
 * kernel flipped and transposed; the transposed conv's four kernel positions as one K),
 * FP32 accumulation, BF16 output; F32 on the CUDA cores.  Not for the first layer (its input
 * needs no gradient).
 * Errors: NRV_ERR_ARG (null, misaligned, the head, the first layer, a transposed conv without
 * mask), NRV_ERR_STATE (no parameters), NRV_ERR_UNSUPPORTED (FP8). */
nrv_status nrv_net_layer_dgrad(nrv_net* net, int layer, const void* d_dy, const void* d_mask,
                               int n, int h, int w, nrv_prec prec, void* d_dx, nrv_stream stream);

/* --------------------------------------------------------------------------
 * Gated post-processing network (Sec. 3.3's form of the network)
 *
 * Gated convolutions (feature and gate 3x3 convolutions, out = ELU(feature) *
 * sigmoid(gate)), a 1x1 convolution of the G-buffers (keeping their C_in channels)
 * injected, average-pooled by 0.5 per level, into the first block of every encoder
 * level; 2x2 average pooling in the encoder, 2x2 stride-2 transposed convolutions and
 * skip concatenations in the decoder, a linear 1x1 head to RGB.  Four levels of
 * 16/32/64/128 channels (the paper's progression starts at 64 over five levels; at
 * this width every layer keeps its weights resident on the tensor-core kernel):
 *   g0 = 1x1(x), g_l = avgpool(g_{l-1});  e0 = gated(g0), e_l = gated([avgpool(e_{l-1}), g_l]);
 *   u_l = convT(d_{l+1}), d_l = gated([u_l, e_l]) for l = 2, 1, 0 (d_3 = e_3);  rgb = 1x1(d0).
 * Layer order: inj e0 e1 e2 e3 up2 d2 up1 d1 up0 d0 head; nrv_gnet_layer reports kind
 * 2 (1x1), 1 (transposed) or 3 (gated, with weight_offset the feature weight W_f
 * (C_out, C_in, 3, 3) and bias_offset its bias; the gate's W_g and b_g follow).  The
 * flat FP32 parameters: per layer its weight(s) and bias(es) in that order, PyTorch
 * layouts.  Inference only, BF16 activations with FP32 accumulation: nrv_gnet_shade
 * takes n BF16 packed inputs [n][Hn][Wn][8] (nrv_pack) and writes [n][height][width][3]
 * FP32.  Errors: NRV_ERR_ARG, NRV_ERR_STATE (no parameters), NRV_ERR_OOM. */
typedef struct nrv_gnet nrv_gnet;
int nrv_gnet_num_layers(void);
nrv_status nrv_gnet_layer(int c_in, int layer, nrv_layer_info* out);
nrv_status nrv_gnet_param_count(int c_in, int64_t* count);
nrv_status nrv_gnet_create(int c_in, nrv_gnet** out);
nrv_status nrv_gnet_destroy(nrv_gnet* net);
nrv_status nrv_gnet_set_params(nrv_gnet* net, const float* d_params, nrv_stream stream);
nrv_status nrv_gnet_shade(nrv_gnet* net, const void* d_netin_bf16, int n, int height, int width,
                          float* d_rgb, nrv_stream stream);
/* One layer (inj .. d0) alone, NHWC BF16 [n][h][w][.] in and out (h, w even), on the kernels
 * nrv_gnet_shade runs: inj reads the 8-channel packed input and writes 8 channels (C_in real);
 * the encoder layers e1..e3 take x1 = the pooled features and x2 = the injected 8-channel
 * tensor, the decoder layers d2..d0 x1 = upsampled and x2 = skip; e0 and the transposed convs
 * take x1 only (x2 NULL); a transposed conv writes [n][2h][2w][C_out].
 * Errors: NRV_ERR_ARG, NRV_ERR_STATE. */
nrv_status nrv_gnet_run_layer(nrv_gnet* net, int layer, const void* d_x1, const void* d_x2, int n,
                              int h, int w, void* d_y, nrv_stream stream);

/* Microbenchmarks behind rooflines that need a measured peak (asynchronous on `stream`;
 * the caller times them).  nrv_probe_ffma: `blocks` blocks of 256 threads, each thread
 * 8 independent FP32 FMA chains of `iters` steps (16 * iters FLOPs per thread), one result
 * per thread into d_out (blocks * 256 floats).  nrv_probe_atomic_min: n_ops 64-bit
 * atomicMin at pseudo-random words of d_buf[n_words] (SplitMix64 of seed and the operation
 * index).  Errors: NRV_ERR_ARG. */
nrv_status nrv_probe_ffma(float* d_out, int blocks, int iters, nrv_stream stream);
nrv_status nrv_probe_atomic_min(unsigned long long* d_buf, int64_t n_words, int64_t n_ops,
                                uint64_t seed, nrv_stream stream);

/* Which kernel family ran layer `layer` in the net's most recent forward pass:
 * 0 = SIMT (CUDA cores), 1 = tensor cores (tcgen05), -1 = not run yet or a
 * bad argument.  Lets callers check that a precision ran where they expect. */
int nrv_net_layer_backend(const nrv_net* net, int layer);

/* Training forward: like nrv_shade, but keeps the activations the backward
 * pass needs in the net's workspace (F32 or BF16 only). */
nrv_status nrv_net_forward_train(nrv_net* net, const void* d_netin, int n, int height, int width,
                                 nrv_prec prec, float* d_rgb, nrv_stream stream);

/* Backward pass of the last nrv_net_forward_train: d_drgb = dL/d(rgb)
 * [n][height][width][3] FP32; writes dL/d(params) into d_grad (flat FP32,
 * parameter layout, overwritten, deterministic).  Errors: NRV_ERR_STATE when no
 * training forward preceded it. */
nrv_status nrv_net_backward(nrv_net* net, const float* d_drgb, float* d_grad, nrv_stream stream);

/* L1 loss of Sec. 3.3's reconstruction term, in the L1 form:
 * loss = mean |y - t| over n floats, written to d_loss[0]; if d_dy is not NULL,
 * d_dy = sign(y - t) / n with sign(0) = 0.  Deterministic. */
nrv_status nrv_l1_loss(const float* d_y, const float* d_t, int64_t n, float* d_loss, float* d_dy,
                       nrv_stream stream);

/* Same loss as nrv_l1_loss for callers that cannot allocate device memory: an
 * application whose memory pool owns the whole device, a real-time frame loop
 * that must not stall on the implicit device synchronisation of cudaMalloc and
 * cudaFree, or a plug-in that is handed its buffers and nothing else.  It
 * allocates nothing; its scratch (one partial sum per 8192 elements) is a fixed
 * 64 KiB array in the library's device memory, kept on every device that loads
 * the library until the process exits.  The paper has no counterpart of this
 * entry point.
 *  - n may be at most NRV_L1_NOALLOC_MAX_ELEMENTS; larger n returns NRV_ERR_ARG
 *    with a message and launches nothing (use nrv_l1_loss then).
 *  - The first call on a device looks up the array's device address (kept for the
 *    process; a cudaDeviceReset of that device invalidates it, so do not call this
 *    entry point after one).  Under CUDA's lazy module loading that first call also
 *    loads the library's device code and this array onto the device, which is
 *    device memory and work at first use: make one warm-up call at start-up, before
 *    the frame loop and before any stream capture on that device.  Later calls
 *    allocate nothing.
 *  - All calls share the array.  Each call overwrites every slot it reads, so
 *    nothing has to be cleared between calls, but calls whose kernels overlap on
 *    the GPU (different streams without ordering) race on it.
 * Results agree with nrv_l1_loss to FP32 rounding (the partial sums differ in
 * grouping); d_dy is identical. */
#define NRV_L1_NOALLOC_MAX_ELEMENTS 134217728LL
nrv_status nrv_l1_loss_noalloc(const float* d_y, const float* d_t, int64_t n, float* d_loss,
                               float* d_dy, nrv_stream stream);

/* Reconstruction and total-variation loss (Eq. 1 without its perceptual term, which
 * needs pretrained VGG weights) on RGB images y, t [n][height][width][3] FP32:
 *   loss = l1 mean|y - t| + l2 mean (y - t)^2
 *        + tv (mean over horizontal neighbour pairs |y(x+1) - y(x)|
 *              + mean over vertical neighbour pairs |y(y+1) - y(y)|),
 * every mean over its own count (all images and channels); the TV term is the
 * anisotropic L1 total variation of the output alone.  d_loss[0] receives the loss,
 * d_dy (if not NULL) its gradient with sign(0) = 0.  Deterministic.
 * nrv_net_set_loss picks the weights nrv_train_step uses (default l1 = 1, l2 = tv = 0,
 * the L1 loss).  Errors: NRV_ERR_ARG (null, bad size, negative or non-finite weight). */
typedef struct {
    float l1, l2, tv;
} nrv_loss_weights;
nrv_status nrv_recon_loss(const float* d_y, const float* d_t, int n, int height, int width,
                          const nrv_loss_weights* weights, float* d_loss, float* d_dy,
                          nrv_stream stream);
nrv_status nrv_net_set_loss(nrv_net* net, const nrv_loss_weights* weights);

/* Adam (Kingma & Ba; Sec. 3.3 uses it with lr 1e-3), no weight decay, step >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps), all FP32. */
nrv_status nrv_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t n,
                         int step, float lr, float beta1, float beta2, float eps, nrv_stream stream);

/* One training step on a batch: forward (saving activations), the loss chosen by
 * nrv_net_set_loss (L1 unless set) against d_target [n][height][width][3], backward, Adam update of d_params with
 * moments d_m, d_v (all flat FP32, parameter layout), then the packed weights
 * are re-derived.  d_loss[0] receives the loss.  prec: F32 or BF16. */
nrv_status nrv_train_step(nrv_net* net, float* d_params, float* d_grad, float* d_m, float* d_v,
                          int step, float lr, const void* d_netin, const float* d_target, int n,
                          int height, int width, nrv_prec prec, float* d_loss, nrv_stream stream);

/* --------------------------------------------------------------------------
 * Whole frames
 * ------------------------------------------------------------------------ */

/* Render n_views views end to end: rasterize, pack and shade every view, each
 * into d_rgb[i] ([H_i][W_i][3] FP32, caller-owned).  Views may have different
 * sizes.  The device work is captured once per (scene, net, sizes, prec) into a
 * CUDA graph and replayed on later calls; a replay copies one 712-byte table of
 * the views from host memory (stream-ordered, before the graph launch).  The
 * G-buffers and network inputs live in the net's workspace.  in_scale_inv is the
 * E4M3 input scale inverse for NRV_PREC_FP8_E4M3 (ignored otherwise,
 * NRV_PREC_FP8 included).  Errors: NRV_ERR_ARG, NRV_ERR_OOM, NRV_ERR_CUDA. */
nrv_status nrv_render_batch(nrv_scene* scene, nrv_net* net, const nrv_pack_desc* desc,
                            const nrv_view* views, int n_views, float* const* d_rgb,
                            nrv_prec prec, float in_scale_inv, nrv_stream stream);

/* Stage timing of nrv_render_batch.  While profiling is on (nrv_set_profiling(1)),
 * every call records CUDA events around its stages on the caller's stream
 * without synchronising.  nrv_get_timings waits for them and writes the mean
 * device milliseconds per call of: [0] clearing the key images, [1] the render
 * (visibility) pass, [2] resolve + pack, [3] the network; then it forgets the
 * recorded calls.  Returns the number of values written (<= cap, at most 4). */
nrv_status nrv_set_profiling(int on);
int nrv_get_timings(float* ms, int cap);

/* Tuned launch choices.  The render pass picks one of its variants (per view-count
 * class and point-count class) by timing them on the real data at the first uncaptured
 * launch that needs the choice; the tensor-core convolution does the same for its
 * launch shape (image rows per tile, accumulator buffers, ring slots, CTAs per SM; per
 * layer, shape and precision) when the environment variable NRV_TC_TUNE is 1, and
 * otherwise uses a choice found in the table or its default shape.  Every candidate
 * computes the same result.  nrv_tune_save writes the choices made or loaded so far to a text
 * file, nrv_tune_load reads one back (a later process then skips the timing); when the
 * environment variable NRV_TUNE_CACHE names an existing file, the library loads it at
 * its first lookup.  Format: '#' comment lines and one choice per line,
 * "<key> = <value>", the key free text ("render multi=1 log2n=27", "conv ...") and
 * the value a non-negative integer.  nrv_tune_count gives the number of choices held,
 * nrv_tune_timings the number of tuning runs this process made.  No counterpart in
 * the paper.  Errors: NRV_ERR_ARG (null path, I/O, a malformed line). */
nrv_status nrv_tune_load(const char* path);
nrv_status nrv_tune_save(const char* path);
int nrv_tune_count(void);
uint64_t nrv_tune_timings(void);

/* Reads and clears the library's device status word (bounded waits that gave
 * up, bad indices caught by device checks).  Synchronises the stream. */
nrv_status nrv_sync_status(nrv_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* NRV_H */
