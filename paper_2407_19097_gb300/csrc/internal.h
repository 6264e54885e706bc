// Internal declarations shared by the library's own translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nrv.h"

namespace nrv {

nrv_status fail(nrv_status s, const char* fmt, ...);
void clear_error();

#define NRV_CHECK_CUDA(call)                                                             \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::nrv::fail(NRV_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Kernels launched by the library so far (nrv_launch_count).
void count_launch();

// Tuned launch choices (tune.cu): look up / record a choice by key; count a tuning run.
bool tune_get(const std::string& key, int* value);
void tune_put(const std::string& key, int value);
void tune_count_timing();

#define NRV_CHECK_LAUNCH()                                                               \
    do {                                                                                 \
        ::nrv::count_launch();                                                           \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess)                                                           \
            return ::nrv::fail(NRV_ERR_CUDA, "kernel launch at %s:%d failed: %s", __FILE__, \
                               __LINE__, cudaGetErrorString(e_));                        \
    } while (0)

#define NRV_TRY(expr)                          \
    do {                                       \
        nrv_status s_ = (expr);                \
        if (s_ != NRV_OK) return s_;           \
    } while (0)

// Device status word: kernels OR error bits into it instead of trapping.
enum : unsigned { STATUS_TIMEOUT = 1u, STATUS_BAD_INDEX = 2u };
unsigned* status_word();  // device pointer, allocated on first use

// --------------------------------------------------------------------- rasterizer
struct RView {
    float m[12];          // rows 0, 1 and 3 of the view-projection, row-major
    float hw, hh;         // 0.5*W, 0.5*H
    float fw, fh;         // W, H as floats
    float znear, zfar;
    int width, height;
    unsigned long long* key;
};

struct RViews {
    RView v[8];
    int n;
    uint32_t base;        // global index of the scene's first point (the key's low word is base + i)
};

struct ResolveArgs {
    const unsigned long long* key;
    uint32_t base;          // the scene's points have global indices base .. base + n_local - 1;
    uint32_t n_local;       // a winner outside that range belongs to another shard: empty here
    const uint32_t* attr;   // records
    int stride_words, n_words;
    int width, height;      // view
    int wn, hn;             // canvas (>= view), used when packing
    uint32_t* depth;        // planes, may be null
    uint8_t* mask;
    uint32_t* gattr;
    void* netin;            // packed network input, may be null
    int out_fmt;            // 0 f32, 1 bf16, 2 e4m3
    float in_scale_inv;
    int n_ch;
    int ch_word[6], ch_fmt[6], ch_comp[6];
    float ch_scale[6], ch_offset[6];
    float d_scale, d_offset;
    // derived channels (formats NRV_VEL2D_* and NRV_SPLAT_RADIUS): the winner's position
    // and the camera
    int derived;            // some channel is derived
    const float* xyz;
    float vm[12];           // rows 0, 1 and 3 of the view-projection, row-major
    float vhw, vhh;         // W/2, H/2
    const RView* view_dev;  // if set, the camera is read from here instead (graph replays)
};

nrv_status launch_clear_keys(const RViews& views, cudaStream_t s);
// Render pass.  `tiles` is scratch for the per-tile depth bounds of the culling
// variants: visibility_scratch_bytes(views) bytes of device memory (may be null,
// which disables culling).  `chunks` holds the bounding boxes of the scene's
// 32-point chunks (6 floats each, chunk_count(n) of them) followed by those of
// their 8-point sub-chunks (RENDER_SUBS per chunk, 6 floats each), from
// launch_chunk_bounds (chunk_box_bytes(n) bytes); may be null, which disables
// chunk culling.
size_t visibility_scratch_bytes(const RViews& views);
constexpr int RENDER_CHUNK = 32;
constexpr int RENDER_SUB = 8;                               // points per sub-chunk
constexpr int RENDER_SUBS = RENDER_CHUNK / RENDER_SUB;      // sub-chunks per chunk
__host__ __device__ inline uint64_t chunk_count(uint64_t n) { return (n + RENDER_CHUNK - 1) / RENDER_CHUNK; }
inline size_t chunk_box_bytes(uint64_t n) { return chunk_count(n) * (1 + RENDER_SUBS) * 6 * sizeof(float); }
nrv_status launch_chunk_bounds(const float* xyz, uint64_t n, void* chunks, cudaStream_t s);
// Render-pass variants (raster.cu): how many there are for one view / a batch, and their names.
int visibility_variant_count(int multi);
const char* visibility_variant_name(int multi, int i);
nrv_status launch_visibility(const float* xyz, uint64_t n, const RViews& views, cudaStream_t s,
                             const RViews* views_dev = nullptr, uint32_t* tiles = nullptr,
                             const void* chunks = nullptr);
// Render pass over every S-th point (scene point j is array point j * S; keys carry j * S):
// one point per thread, no culling.
nrv_status launch_visibility_strided(const float* xyz, uint64_t n, int stride, const RViews& views,
                                     cudaStream_t s, const RViews* views_dev = nullptr);
nrv_status launch_resolve(const ResolveArgs& a, cudaStream_t s);
nrv_status launch_flip_sign(uint64_t* keys, int64_t n, cudaStream_t s);
nrv_status launch_pack_planes(const uint32_t* depth, const uint8_t* mask, const uint32_t* gattr,
                              const ResolveArgs& a, cudaStream_t s);

// --------------------------------------------------------------------- network
// Per-image RGB destinations of one network call (views of one size shaded together, each into
// its caller's buffer); off: image i goes to base + i * H * W * 3.
struct RgbTab {
    float* p[8];
    int on;
};

// Where image img's RGB row-major pixel array starts.
__host__ __device__ inline float* rgb_image(float* base, const RgbTab& t, size_t img, size_t hw) {
    return t.on ? t.p[img] : base + img * hw * 3;
}

enum LayerKind { CONV3 = 0, UPCONV2 = 1, HEAD1 = 2 };

struct Layer {
    char name[8];
    int kind, cin, cout;
    int64_t woff, boff;
};

constexpr int NUM_LAYERS = 18;
int net_layers(int c_in, Layer* out);      // returns the parameter count

// Layer indices
enum {
    L_E0A, L_E0B, L_E1A, L_E1B, L_E2A, L_E2B, L_E3A, L_E3B, L_UP3, L_D2A, L_D2B, L_UP2, L_D1A,
    L_D1B, L_UP1, L_D0A, L_D0B, L_HEAD
};

struct Net;  // defined in net.cu

}  // namespace nrv
