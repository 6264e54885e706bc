// C ABI entry points (include/nrv.h): argument checks, handles and the
// orchestration of the rasterizer and network stages.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <vector>

#include "net.h"

namespace nrv {

static thread_local char g_err[512];

nrv_status fail(nrv_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

void clear_error() { g_err[0] = 0; }

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static unsigned* g_status = nullptr;

unsigned* status_word() {
    if (!g_status) {
        if (cudaMalloc(&g_status, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            g_status = nullptr;
            return nullptr;
        }
        cudaMemset(g_status, 0, sizeof(unsigned));
    }
    return g_status;
}


}  // namespace nrv

using namespace nrv;

struct nrv_scene {
    nrv_scene_desc d;
    DevBuf tiles;    // per-tile depth bounds of the render pass (nrv_rasterize)
    DevBuf chunks;   // bounding boxes of every 32-point chunk and its 8-point sub-chunks (culling)
    bool chunks_ok = false;
};

// The chunk bounds are derived from the positions on first use and after nrv_scene_refresh.
static nrv_status ensure_chunks(nrv_scene* s, cudaStream_t st) {
    if (s->chunks_ok || s->d.n_points == 0 || s->d.point_stride > 1) return NRV_OK;
    NRV_TRY(s->chunks.ensure(chunk_box_bytes(s->d.n_points)));
    NRV_TRY(launch_chunk_bounds(s->d.d_xyz, s->d.n_points, s->chunks.p, st));
    s->chunks_ok = true;
    return NRV_OK;
}

// A captured whole frame (nrv_render_batch) and the device copy of the cameras it reads.
struct BatchGraph {
    std::vector<uint64_t> sig;
    cudaGraphExec_t exec = nullptr;
    RViews* views_dev = nullptr;
    uint64_t kernels = 0;   // kernel nodes in the graph
};

struct nrv_net : Net {
    std::vector<BatchGraph> graphs;
    void drop_graphs() {
        for (BatchGraph& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.views_dev) cudaFree(g.views_dev);
        }
        graphs.clear();
    }
    ~nrv_net() { drop_graphs(); }
};

// --------------------------------------------------------------------- library
extern "C" const char* nrv_last_error(void) { return g_err; }
extern "C" int nrv_version(void) { return 1; }
extern "C" uint64_t nrv_launch_count(void) { return g_launches.load(); }
extern "C" int nrv_render_variants(int multi_view) {
    return nrv::visibility_variant_count(multi_view != 0);
}
extern "C" int nrv_pad8(int v) { return (v + 7) / 8 * 8; }
extern "C" int nrv_netin_channels(nrv_prec p) { return p == NRV_PREC_FP8_E4M3 ? 16 : 8; }
// precision of the packed network input (the mixed FP8 network reads a BF16 input)
static nrv_prec netin_prec(nrv_prec p) { return p == NRV_PREC_FP8 ? NRV_PREC_BF16 : p; }

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// --------------------------------------------------------------------- scene
extern "C" nrv_status nrv_create_scene(const nrv_scene_desc* d, nrv_scene** out) {
    clear_error();
    if (!d || !out) return fail(NRV_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->point_stride < 0) return fail(NRV_ERR_ARG, "point_stride must be >= 0");
    const uint64_t ps = d->point_stride > 1 ? (uint64_t)d->point_stride : 1;
    if (d->n_points >= (1ull << 32) || d->index_base + d->n_points * ps > 0xFFFFFFFFull)
        return fail(NRV_ERR_ARG, "index_base + n_points * point_stride must be < 2^32");
    const int sw = d->stride_words;
    if (!(sw == 1 || sw == 2 || sw == 4 || sw == 8))
        return fail(NRV_ERR_ARG, "stride_words must be 1, 2, 4 or 8 (got %d)", sw);
    if (d->n_words < 1 || d->n_words > sw)
        return fail(NRV_ERR_ARG, "n_words must be in 1..stride_words (got %d)", d->n_words);
    if (d->n_points > 0) {
        if (!d->d_xyz || !d->d_attr) return fail(NRV_ERR_ARG, "null point or attribute pointer");
        if (!aligned(d->d_xyz, 16)) return fail(NRV_ERR_ARG, "d_xyz must be 16-byte aligned");
        const size_t ra = sw * 4 < 16 ? (size_t)sw * 4 : 16;
        if (!aligned(d->d_attr, ra)) return fail(NRV_ERR_ARG, "d_attr must be %zu-byte aligned", ra);
    }
    nrv_scene* s = new nrv_scene;
    s->d = *d;
    s->d.point_stride = (int)ps;
    *out = s;
    return NRV_OK;
}

extern "C" nrv_status nrv_destroy_scene(nrv_scene* s) {
    clear_error();
    delete s;
    return NRV_OK;
}

extern "C" nrv_status nrv_scene_refresh(nrv_scene* s) {
    clear_error();
    if (!s) return fail(NRV_ERR_ARG, "null scene");
    s->chunks_ok = false;
    return NRV_OK;
}

static nrv_status check_view(const nrv_view& v) {
    if (v.width < 1 || v.height < 1 || v.width > 16384 || v.height > 16384)
        return fail(NRV_ERR_ARG, "view size %dx%d out of range", v.width, v.height);
    if (!(v.znear > 0.0f) || !(v.zfar >= v.znear)) return fail(NRV_ERR_ARG, "need 0 < znear <= zfar");
    for (int i = 0; i < 16; ++i)
        if (!isfinite(v.viewproj[i])) return fail(NRV_ERR_ARG, "view matrix must be finite");
    return NRV_OK;
}

static RView make_rview(const nrv_view& v, uint64_t* key) {
    RView r;
    const int rows[3] = {0, 1, 3};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) r.m[4 * i + j] = v.viewproj[4 * rows[i] + j];
    r.hw = 0.5f * (float)v.width;
    r.hh = 0.5f * (float)v.height;
    r.fw = (float)v.width;
    r.fh = (float)v.height;
    r.znear = v.znear;
    r.zfar = v.zfar;
    r.width = v.width;
    r.height = v.height;
    r.key = reinterpret_cast<unsigned long long*>(key);
    return r;
}

static bool is_derived(int fmt) { return fmt >= NRV_VEL2D_X && fmt <= NRV_SPLAT_RADIUS; }

static nrv_status check_pack(const nrv_pack_desc* d, int n_words, bool allow_derived = true) {
    if (!d) return fail(NRV_ERR_ARG, "null pack descriptor");
    if (d->n_channels < 1 || d->n_channels > 6) return fail(NRV_ERR_ARG, "n_channels must be 1..6");
    for (int j = 0; j < d->n_channels; ++j) {
        const int last = d->word[j] + (d->fmt[j] >= NRV_VEL2D_X && d->fmt[j] <= NRV_VEL2D_MAG ? 2 : 0);
        if (d->word[j] < 0 || last >= n_words)
            return fail(NRV_ERR_ARG, "channel %d reads words %d..%d of %d", j, d->word[j], last,
                        n_words);
        if (d->fmt[j] < 0 || d->fmt[j] > NRV_SPLAT_RADIUS)
            return fail(NRV_ERR_ARG, "channel %d: bad format", j);
        if (is_derived(d->fmt[j]) && !allow_derived)
            return fail(NRV_ERR_ARG, "channel %d: derived channels need the scene (nrv_resolve_pack)", j);
        if (d->fmt[j] == NRV_U8X4 && (d->comp[j] < 0 || d->comp[j] > 3))
            return fail(NRV_ERR_ARG, "channel %d: byte index must be 0..3", j);
    }
    return NRV_OK;
}

static void fill_pack(ResolveArgs& a, const nrv_pack_desc* d, nrv_prec prec, float inv) {
    prec = netin_prec(prec);
    a.out_fmt = prec == NRV_PREC_F32 ? 0 : prec == NRV_PREC_BF16 ? 1 : 2;
    a.in_scale_inv = inv;
    a.n_ch = d->n_channels;
    for (int j = 0; j < 6; ++j) {
        a.ch_word[j] = j < d->n_channels ? d->word[j] : 0;
        a.ch_fmt[j] = j < d->n_channels ? d->fmt[j] : 0;
        a.ch_comp[j] = j < d->n_channels ? d->comp[j] : 0;
        a.ch_scale[j] = j < d->n_channels ? d->scale[j] : 0.0f;
        a.ch_offset[j] = j < d->n_channels ? d->offset[j] : 0.0f;
    }
    a.d_scale = d->depth_scale;
    a.d_offset = d->depth_offset;
}

// What the derived channels read: the scene's positions and the view's camera.
static void fill_derived(ResolveArgs& a, const nrv_pack_desc* d, const nrv_view& v, const float* xyz) {
    a.derived = 0;
    for (int j = 0; j < d->n_channels; ++j)
        if (is_derived(d->fmt[j])) a.derived = 1;
    a.xyz = xyz;
    const int rows[3] = {0, 1, 3};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) a.vm[4 * i + j] = v.viewproj[4 * rows[i] + j];
    a.vhw = 0.5f * (float)v.width;
    a.vhh = 0.5f * (float)v.height;
    a.view_dev = nullptr;
}

static nrv_status raster_views(nrv_scene* s, const nrv_view* views, int n, uint64_t* const* keys,
                               cudaStream_t st) {
    RViews rv;
    memset(&rv, 0, sizeof(rv));
    rv.n = n;
    rv.base = (uint32_t)s->d.index_base;
    for (int i = 0; i < n; ++i) rv.v[i] = make_rview(views[i], keys[i]);
    NRV_TRY(launch_clear_keys(rv, st));
    if (s->d.point_stride > 1)
        return launch_visibility_strided(s->d.d_xyz, s->d.n_points, s->d.point_stride, rv, st, nullptr);
    NRV_TRY(s->tiles.ensure(visibility_scratch_bytes(rv)));
    NRV_TRY(ensure_chunks(s, st));
    return launch_visibility(s->d.d_xyz, s->d.n_points, rv, st, nullptr, (uint32_t*)s->tiles.p,
                             s->chunks.p);
}

extern "C" nrv_status nrv_rasterize(nrv_scene* s, const nrv_view* views, int n,
                                    const nrv_gbuffer* gb, nrv_stream stream) {
    clear_error();
    if (!s || !views || !gb) return fail(NRV_ERR_ARG, "null argument");
    if (n < 1 || n > 8) return fail(NRV_ERR_ARG, "n_views must be 1..8");
    uint64_t* keys[8];
    for (int i = 0; i < n; ++i) {
        NRV_TRY(check_view(views[i]));
        if (!gb[i].d_key || !aligned(gb[i].d_key, 16))
            return fail(NRV_ERR_ARG, "view %d: d_key must be non-null and 16-byte aligned", i);
        keys[i] = gb[i].d_key;
    }
    cudaStream_t st = (cudaStream_t)stream;
    NRV_TRY(raster_views(s, views, n, keys, st));
    for (int i = 0; i < n; ++i) {
        if (!gb[i].d_depth && !gb[i].d_mask && !gb[i].d_attr) continue;
        ResolveArgs a;
        memset(&a, 0, sizeof(a));
        a.key = reinterpret_cast<const unsigned long long*>(gb[i].d_key);
        a.attr = s->d.d_attr;
        a.base = (uint32_t)s->d.index_base;
        a.n_local = (uint32_t)(s->d.n_points * s->d.point_stride);
        a.stride_words = s->d.stride_words;
        a.n_words = s->d.n_words;
        a.width = views[i].width;
        a.height = views[i].height;
        a.depth = gb[i].d_depth;
        a.mask = gb[i].d_mask;
        a.gattr = gb[i].d_attr;
        NRV_TRY(launch_resolve(a, st));
    }
    return NRV_OK;
}

extern "C" nrv_status nrv_pack(const nrv_gbuffer* gb, int h, int w, const nrv_pack_desc* d,
                               nrv_prec prec, float inv, void* netin, nrv_stream stream) {
    clear_error();
    if (!gb || !netin || !gb->d_depth || !gb->d_mask || !gb->d_attr)
        return fail(NRV_ERR_ARG, "pack needs depth, mask and attribute planes and an output");
    if (h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (prec < NRV_PREC_F32 || prec > NRV_PREC_FP8) return fail(NRV_ERR_ARG, "bad precision");
    if (!aligned(netin, 32)) return fail(NRV_ERR_ARG, "d_netin must be 32-byte aligned");
    NRV_TRY(check_pack(d, 8, false));
    ResolveArgs a;
    memset(&a, 0, sizeof(a));
    a.width = w;
    a.height = h;
    a.wn = nrv_pad8(w);
    a.hn = nrv_pad8(h);
    a.netin = netin;
    fill_pack(a, d, prec, inv);
    return launch_pack_planes(gb->d_depth, gb->d_mask, gb->d_attr, a, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_resolve(nrv_scene* s, const nrv_view* view, const uint64_t* key,
                                  const nrv_gbuffer* gb, nrv_stream stream) {
    clear_error();
    if (!s || !view || !key || !gb) return fail(NRV_ERR_ARG, "null argument");
    NRV_TRY(check_view(*view));
    if (!aligned(key, 16)) return fail(NRV_ERR_ARG, "d_key must be 16-byte aligned");
    if (!gb->d_depth && !gb->d_mask && !gb->d_attr) return NRV_OK;
    ResolveArgs a;
    memset(&a, 0, sizeof(a));
    a.key = reinterpret_cast<const unsigned long long*>(key);
    a.attr = s->d.d_attr;
    a.base = (uint32_t)s->d.index_base;
    a.n_local = (uint32_t)(s->d.n_points * s->d.point_stride);
    a.stride_words = s->d.stride_words;
    a.n_words = s->d.n_words;
    a.width = view->width;
    a.height = view->height;
    a.depth = gb->d_depth;
    a.mask = gb->d_mask;
    a.gattr = gb->d_attr;
    return launch_resolve(a, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_keys_flip_sign(uint64_t* key, int64_t n, nrv_stream stream) {
    clear_error();
    if (!key || n < 0) return fail(NRV_ERR_ARG, "bad argument");
    if (n == 0) return NRV_OK;
    return launch_flip_sign(key, n, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_resolve_pack(nrv_scene* s, const nrv_view* view, const uint64_t* key,
                                       const nrv_pack_desc* d, nrv_prec prec, float inv,
                                       void* netin, nrv_stream stream) {
    clear_error();
    if (!s || !view || !key || !netin) return fail(NRV_ERR_ARG, "null argument");
    NRV_TRY(check_view(*view));
    if (prec < NRV_PREC_F32 || prec > NRV_PREC_FP8) return fail(NRV_ERR_ARG, "bad precision");
    if (!aligned(netin, 32) || !aligned(key, 16))
        return fail(NRV_ERR_ARG, "d_netin must be 32-byte and d_key 16-byte aligned");
    NRV_TRY(check_pack(d, s->d.n_words));
    ResolveArgs a;
    memset(&a, 0, sizeof(a));
    a.key = reinterpret_cast<const unsigned long long*>(key);
    a.attr = s->d.d_attr;
    a.base = (uint32_t)s->d.index_base;
    a.n_local = (uint32_t)(s->d.n_points * s->d.point_stride);
    a.stride_words = s->d.stride_words;
    a.n_words = s->d.n_words;
    a.width = view->width;
    a.height = view->height;
    a.wn = nrv_pad8(a.width);
    a.hn = nrv_pad8(a.height);
    a.netin = netin;
    fill_pack(a, d, prec, inv);
    fill_derived(a, d, *view, s->d.d_xyz);
    return launch_resolve(a, (cudaStream_t)stream);
}

// --------------------------------------------------------------------- network
extern "C" int nrv_net_num_layers(void) { return NUM_LAYERS; }

extern "C" nrv_status nrv_net_layer(int c_in, int layer, nrv_layer_info* out) {
    clear_error();
    if (c_in < 1 || c_in > 8 || layer < 0 || layer >= NUM_LAYERS || !out)
        return fail(NRV_ERR_ARG, "bad layer query");
    Layer L[NUM_LAYERS];
    net_layers(c_in, L);
    memset(out, 0, sizeof(*out));
    memcpy(out->name, L[layer].name, sizeof(out->name));
    out->kind = L[layer].kind;
    out->c_in = L[layer].cin;
    out->c_out = L[layer].cout;
    out->weight_offset = L[layer].woff;
    out->bias_offset = L[layer].boff;
    return NRV_OK;
}

extern "C" nrv_status nrv_net_param_count(int c_in, int64_t* count) {
    clear_error();
    if (c_in < 1 || c_in > 8 || !count) return fail(NRV_ERR_ARG, "c_in must be 1..8");
    Layer L[NUM_LAYERS];
    *count = net_layers(c_in, L);
    return NRV_OK;
}

extern "C" nrv_status nrv_create_net(int c_in, nrv_net** out) {
    clear_error();
    if (!out) return fail(NRV_ERR_ARG, "null argument");
    *out = nullptr;
    if (c_in < 1 || c_in > 8) return fail(NRV_ERR_ARG, "c_in must be 1..8");
    nrv_net* net = new nrv_net;
    net->c_in = c_in;
    net->c0p = 8;
    net->n_params = net_layers(c_in, net->layers);
    for (int l = 0; l < NUM_LAYERS; ++l) net->backend[l] = -1;
    for (int a = 0; a <= NUM_ACTS; ++a) net->act_scale[a] = 1.0f;
    *out = net;
    return NRV_OK;
}

extern "C" nrv_status nrv_destroy_net(nrv_net* net) {
    clear_error();
    delete net;
    return NRV_OK;
}

extern "C" nrv_status nrv_net_set_params(nrv_net* net, const float* d_params, nrv_stream stream) {
    clear_error();
    if (!net || !d_params) return fail(NRV_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    NRV_TRY(net->params.ensure(net->n_params * sizeof(float)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(net->params.p, d_params, net->n_params * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st));
    NRV_TRY(net_repack(net, st));
    net->has_params = true;
    return NRV_OK;
}

extern "C" nrv_status nrv_net_init_params(nrv_net* net, uint64_t seed, float* d_params,
                                          nrv_stream stream) {
    clear_error();
    if (!net || !d_params) return fail(NRV_ERR_ARG, "null argument");
    NRV_TRY(net_init_params(net, seed, d_params, (cudaStream_t)stream));
    return nrv_net_set_params(net, d_params, stream);
}

extern "C" nrv_status nrv_net_get_params(const nrv_net* net, float* d_out, nrv_stream stream) {
    clear_error();
    if (!net || !d_out) return fail(NRV_ERR_ARG, "null argument");
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    NRV_CHECK_CUDA(cudaMemcpyAsync(d_out, net->params.p, net->n_params * sizeof(float),
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return NRV_OK;
}

extern "C" nrv_status nrv_net_save(const nrv_net* net, const char* path, nrv_stream stream) {
    clear_error();
    if (!net || !path) return fail(NRV_ERR_ARG, "null argument");
    return net_save(net, path, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_net_load(nrv_net* net, const char* path, nrv_stream stream) {
    clear_error();
    if (!net || !path) return fail(NRV_ERR_ARG, "null argument");
    net->drop_graphs();   // captured frames hold the old packed weights' addresses
    return net_load(net, path, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_net_set_act_scales(nrv_net* net, const float* s, int n,
                                             nrv_stream stream) {
    clear_error();
    if (!net || !s || n != NUM_ACTS + 1) return fail(NRV_ERR_ARG, "need %d scales", NUM_ACTS + 1);
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    for (int a = 0; a <= NUM_ACTS; ++a)
        if (!(s[a] > 0.0f) || !isfinite(s[a])) return fail(NRV_ERR_ARG, "scale %d must be > 0", a);
    for (int a = 0; a <= NUM_ACTS; ++a) net->act_scale[a] = s[a];
    net->fp8_ready = false;
    NRV_TRY(tc_repack_fp8(net, (cudaStream_t)stream));
    net->fp8_ready = true;
    return NRV_OK;
}

extern "C" nrv_status nrv_net_get_act_scales(const nrv_net* net, float* s, int n) {
    clear_error();
    if (!net || !s || n != NUM_ACTS + 1) return fail(NRV_ERR_ARG, "need %d scales", NUM_ACTS + 1);
    for (int a = 0; a <= NUM_ACTS; ++a) s[a] = net->act_scale[a];
    return NRV_OK;
}

extern "C" nrv_status nrv_net_calibrate(nrv_net* net, const void* d_netin, int n, int h, int w,
                                        nrv_stream stream) {
    clear_error();
    if (!net || !d_netin) return fail(NRV_ERR_ARG, "null argument");
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (!aligned(d_netin, 32)) return fail(NRV_ERR_ARG, "d_netin must be 32-byte aligned");
    NRV_TRY(net_calibrate(net, d_netin, n, h, w, (cudaStream_t)stream));
    net->fp8_ready = false;
    NRV_TRY(tc_repack_fp8(net, (cudaStream_t)stream));
    net->fp8_ready = true;
    return NRV_OK;
}

static nrv_status check_shade(nrv_net* net, const void* in, int n, int h, int w, nrv_prec prec,
                              const float* rgb) {
    if (!net || !in || !rgb) return fail(NRV_ERR_ARG, "null argument");
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (prec < NRV_PREC_F32 || prec > NRV_PREC_FP8) return fail(NRV_ERR_ARG, "bad precision");
    if (!aligned(in, 32)) return fail(NRV_ERR_ARG, "d_netin must be 32-byte aligned");
    return NRV_OK;
}

extern "C" nrv_status nrv_shade(nrv_net* net, const void* netin, int n, int h, int w,
                                nrv_prec prec, float* rgb, nrv_stream stream) {
    clear_error();
    NRV_TRY(check_shade(net, netin, n, h, w, prec, rgb));
    return net_forward(net, netin, n, h, w, prec, rgb, (cudaStream_t)stream, false);
}

extern "C" nrv_status nrv_net_run_layer(nrv_net* net, int layer, const void* x1, const void* x2,
                                        int n, int h, int w, nrv_prec prec, void* y,
                                        nrv_stream stream) {
    clear_error();
    if (!net || !x1 || !y) return fail(NRV_ERR_ARG, "null argument");
    if (layer < 0 || layer >= NUM_LAYERS || net->layers[layer].kind == HEAD1)
        return fail(NRV_ERR_ARG, "layer %d is not a 3x3 or transposed convolution", layer);
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (!aligned(x1, 32) || (x2 && !aligned(x2, 32)) || !aligned(y, 32))
        return fail(NRV_ERR_ARG, "tensors must be 32-byte aligned");
    return net_run_layer(net, layer, x1, x2, n, h, w, prec, y, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_net_layer_wgrad(nrv_net* net, int layer, const void* dy, const void* x1,
                                          const void* x2, int n, int h, int w, nrv_prec prec,
                                          float* grad, nrv_stream stream) {
    clear_error();
    if (!net || !dy || !x1 || !grad) return fail(NRV_ERR_ARG, "null argument");
    if (layer < 0 || layer >= NUM_LAYERS) return fail(NRV_ERR_ARG, "bad layer %d", layer);
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (!aligned(dy, 32) || !aligned(x1, 32) || (x2 && !aligned(x2, 32)) || !aligned(grad, 16))
        return fail(NRV_ERR_ARG, "tensors must be 32-byte aligned (grad 16-byte)");
    return net_layer_wgrad(net, layer, dy, x1, x2, n, h, w, prec, grad, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_net_layer_dgrad(nrv_net* net, int layer, const void* dy, const void* mask,
                                          int n, int h, int w, nrv_prec prec, void* dx,
                                          nrv_stream stream) {
    clear_error();
    if (!net || !dy || !dx) return fail(NRV_ERR_ARG, "null argument");
    if (layer < 0 || layer >= NUM_LAYERS) return fail(NRV_ERR_ARG, "bad layer %d", layer);
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    if (!aligned(dy, 32) || !aligned(dx, 32) || (mask && !aligned(mask, 32)))
        return fail(NRV_ERR_ARG, "tensors must be 32-byte aligned");
    return net_layer_dgrad(net, layer, dy, mask, n, h, w, prec, dx, (cudaStream_t)stream);
}

extern "C" int nrv_net_layer_backend(const nrv_net* net, int layer) {
    if (!net || layer < 0 || layer >= NUM_LAYERS) return -1;
    return net->backend[layer];
}

extern "C" nrv_status nrv_net_forward_train(nrv_net* net, const void* netin, int n, int h, int w,
                                            nrv_prec prec, float* rgb, nrv_stream stream) {
    clear_error();
    NRV_TRY(check_shade(net, netin, n, h, w, prec, rgb));
    if (prec >= NRV_PREC_FP8_E4M3) return fail(NRV_ERR_UNSUPPORTED, "training runs in F32 or BF16");
    NRV_TRY(net_forward(net, netin, n, h, w, prec, rgb, (cudaStream_t)stream));
    net->saved_in = netin;
    net->saved = true;
    return NRV_OK;
}

extern "C" nrv_status nrv_net_backward(nrv_net* net, const float* drgb, float* dparams,
                                       nrv_stream stream) {
    clear_error();
    if (!net || !drgb || !dparams) return fail(NRV_ERR_ARG, "null argument");
    return net_backward(net, drgb, dparams, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_l1_loss(const float* y, const float* t, int64_t n, float* loss,
                                  float* dy, nrv_stream stream) {
    clear_error();
    if (!y || !t || !loss || n < 1) return fail(NRV_ERR_ARG, "bad argument");
    return launch_l1(y, t, n, loss, dy, (cudaStream_t)stream);
}

static nrv_status check_weights(const nrv_loss_weights* w) {
    if (!w) return fail(NRV_ERR_ARG, "null weights");
    for (float v : {w->l1, w->l2, w->tv})
        if (!(v >= 0.0f) || !isfinite(v)) return fail(NRV_ERR_ARG, "loss weights must be finite and >= 0");
    return NRV_OK;
}

extern "C" nrv_status nrv_recon_loss(const float* y, const float* t, int n, int h, int w,
                                     const nrv_loss_weights* wt, float* loss, float* dy,
                                     nrv_stream stream) {
    clear_error();
    if (!y || !t || !loss) return fail(NRV_ERR_ARG, "null argument");
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384) return fail(NRV_ERR_ARG, "bad size");
    NRV_TRY(check_weights(wt));
    return launch_recon(y, t, n, h, w, *wt, loss, dy, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_net_set_loss(nrv_net* net, const nrv_loss_weights* wt) {
    clear_error();
    if (!net) return fail(NRV_ERR_ARG, "null net");
    NRV_TRY(check_weights(wt));
    net->loss_w = *wt;
    return NRV_OK;
}

extern "C" nrv_status nrv_adam_step(float* p, const float* g, float* m, float* v, int64_t n,
                                    int step, float lr, float b1, float b2, float eps,
                                    nrv_stream stream) {
    clear_error();
    if (!p || !g || !m || !v || n < 1 || step < 1) return fail(NRV_ERR_ARG, "bad argument");
    return launch_adam(p, g, m, v, n, step, lr, b1, b2, eps, (cudaStream_t)stream);
}

extern "C" nrv_status nrv_train_step(nrv_net* net, float* params, float* grad, float* m, float* v,
                                     int step, float lr, const void* netin, const float* target,
                                     int n, int h, int w, nrv_prec prec, float* loss,
                                     nrv_stream stream) {
    clear_error();
    if (!params || !grad || !m || !v || !target || !loss || step < 1)
        return fail(NRV_ERR_ARG, "bad argument");
    NRV_TRY(check_shade(net, netin, n, h, w, prec, target));
    if (prec >= NRV_PREC_FP8_E4M3) return fail(NRV_ERR_UNSUPPORTED, "training runs in F32 or BF16");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nout = (size_t)n * h * w * 3;
    NRV_TRY(net->batch_ws.ensure(2 * nout * sizeof(float)));
    float* y = (float*)net->batch_ws.p;
    float* dy = y + nout;
    NRV_TRY(net_forward(net, netin, n, h, w, prec, y, st));
    net->saved_in = netin;
    net->saved = true;
    const nrv_loss_weights& lw = net->loss_w;
    if (lw.l1 == 1.0f && lw.l2 == 0.0f && lw.tv == 0.0f)
        NRV_TRY(launch_l1(y, target, (int64_t)nout, loss, dy, st));
    else
        NRV_TRY(launch_recon(y, target, n, h, w, lw, loss, dy, st));
    NRV_TRY(net_backward(net, dy, grad, st));
    NRV_TRY(launch_adam(params, grad, m, v, net->n_params, step, lr, 0.9f, 0.999f, 1e-8f, st));
    NRV_CHECK_CUDA(cudaMemcpyAsync(net->params.p, params, net->n_params * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st));
    return net_repack(net, st);
}

// --------------------------------------------------------------------- whole frames
// Profiling: each nrv_render_batch call records events around its stages on the
// caller's stream (no synchronisation); nrv_get_timings waits for the last one
// and returns per-call averages, then forgets them.
static bool g_profile = false;
static std::vector<std::vector<cudaEvent_t>> g_prof_events;
enum { ST_CLEAR, ST_VIS, ST_RESOLVE, ST_NET, NUM_STAGES };

extern "C" nrv_status nrv_set_profiling(int on) {
    clear_error();
    g_profile = on != 0;
    return NRV_OK;
}

extern "C" int nrv_get_timings(float* ms, int cap) {
    double acc[NUM_STAGES] = {0, 0, 0, 0};
    int calls = 0;
    for (auto& ev : g_prof_events) {
        if (cudaEventSynchronize(ev.back()) != cudaSuccess) continue;
        for (int k = 0; k < NUM_STAGES; ++k) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
        ++calls;
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    g_prof_events.clear();
    int k = 0;
    for (; k < NUM_STAGES && k < cap; ++k) ms[k] = calls ? (float)(acc[k] / calls) : 0.0f;
    return k;
}

static void prof_mark(std::vector<cudaEvent_t>& ev, cudaStream_t st) {
    if (!g_profile) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back(e);
}

extern "C" nrv_status nrv_render_batch(nrv_scene* s, nrv_net* net, const nrv_pack_desc* d,
                                       const nrv_view* views, int n, float* const* rgb,
                                       nrv_prec prec, float inv, nrv_stream stream) {
    clear_error();
    if (!s || !net || !views || !rgb) return fail(NRV_ERR_ARG, "null argument");
    if (n < 1 || n > 8) return fail(NRV_ERR_ARG, "n_views must be 1..8");
    if (!net->has_params) return fail(NRV_ERR_STATE, "no parameters loaded");
    NRV_TRY(check_pack(d, s->d.n_words));
    if (d->n_channels + 2 != net->c_in)
        return fail(NRV_ERR_ARG, "pack gives %d channels, network expects %d", d->n_channels + 2,
                    net->c_in);
    cudaStream_t st = (cudaStream_t)stream;
    size_t key_off[8], in_off[8], tot = 0;
    const size_t es = elem_size(netin_prec(prec)) * nrv_netin_channels(netin_prec(prec));
    for (int i = 0; i < n; ++i) {
        NRV_TRY(check_view(views[i]));
        if (!rgb[i]) return fail(NRV_ERR_ARG, "null output %d", i);
        key_off[i] = tot;
        tot += ((size_t)views[i].width * views[i].height * 8 + 1023) / 1024 * 1024;
    }
    // views of one size are shaded by one network call: their inputs sit back to back
    int group_of[8], ngroups = 0, group_first[8], group_n[8];
    for (int i = 0; i < n; ++i) {
        group_of[i] = -1;
        for (int g = 0; g < ngroups; ++g)
            if (views[group_first[g]].width == views[i].width &&
                views[group_first[g]].height == views[i].height)
                group_of[i] = g;
        if (group_of[i] < 0) {
            group_of[i] = ngroups;
            group_first[ngroups] = i;
            group_n[ngroups++] = 0;
        }
        ++group_n[group_of[i]];
    }
    for (int g = 0; g < ngroups; ++g) {
        const size_t per = (size_t)nrv_pad8(views[group_first[g]].width) *
                           nrv_pad8(views[group_first[g]].height) * es;
        int j = 0;
        for (int i = 0; i < n; ++i)
            if (group_of[i] == g) in_off[i] = tot + per * j++;
        tot += (per * group_n[g] + 1023) / 1024 * 1024;
    }
    const size_t tiles_off = tot;
    {
        RViews tmp;
        memset(&tmp, 0, sizeof(tmp));
        tmp.n = n;
        for (int i = 0; i < n; ++i) tmp.v[i] = make_rview(views[i], nullptr);
        tot += (visibility_scratch_bytes(tmp) + 1023) / 1024 * 1024;
    }
    NRV_TRY(net->batch_ws.ensure(tot));
    char* base = (char*)net->batch_ws.p;
    RViews rv;
    memset(&rv, 0, sizeof(rv));
    rv.n = n;
    rv.base = (uint32_t)s->d.index_base;
    for (int i = 0; i < n; ++i) rv.v[i] = make_rview(views[i], (uint64_t*)(base + key_off[i]));

    // everything but the cameras is fixed by this signature; a captured frame is replayed
    auto make_sig = [&]() {
        std::vector<uint64_t> sig = {(uint64_t)(uintptr_t)s->d.d_xyz, s->d.n_points,
                                     (uint64_t)(uintptr_t)s->chunks.p,
                                     (uint64_t)(uintptr_t)s->d.d_attr, (uint64_t)s->d.stride_words,
                                     (uint64_t)s->d.n_words, (uint64_t)prec, (uint64_t)n};
        for (int i = 0; i < n; ++i) {
            sig.push_back(((uint64_t)views[i].width << 32) | (uint32_t)views[i].height);
            sig.push_back((uint64_t)(uintptr_t)rgb[i]);
        }
        uint64_t dw[(sizeof(nrv_pack_desc) + 7) / 8] = {};
        memcpy(dw, d, sizeof(nrv_pack_desc));
        for (uint64_t w : dw) sig.push_back(w);
        uint32_t inv_bits;
        memcpy(&inv_bits, &inv, 4);
        sig.push_back(inv_bits);
        // the captured kernels hold these buffers' addresses
        for (const DevBuf* b : {&net->batch_ws, &net->acts, &net->params, &net->wf32, &net->wbf16}) {
            sig.push_back((uint64_t)(uintptr_t)b->p);
            sig.push_back(b->bytes);
        }
        return sig;
    };
    NRV_TRY(ensure_chunks(s, st));
    std::vector<uint64_t> sig = make_sig();

    auto frame = [&](const RViews* views_dev, std::vector<cudaEvent_t>* ev,
                     cudaStream_t q) -> nrv_status {
        if (ev) prof_mark(*ev, q);
        NRV_TRY(launch_clear_keys(rv, q));
        if (ev) prof_mark(*ev, q);
        if (s->d.point_stride > 1)
            NRV_TRY(launch_visibility_strided(s->d.d_xyz, s->d.n_points, s->d.point_stride, rv, q,
                                              views_dev));
        else
            NRV_TRY(launch_visibility(s->d.d_xyz, s->d.n_points, rv, q, views_dev,
                                      (uint32_t*)(base + tiles_off), s->chunks.p));
        if (ev) prof_mark(*ev, q);
        for (int i = 0; i < n; ++i) {
            ResolveArgs a;
            memset(&a, 0, sizeof(a));
            a.key = reinterpret_cast<const unsigned long long*>(base + key_off[i]);
            a.attr = s->d.d_attr;
            a.base = (uint32_t)s->d.index_base;
            a.n_local = (uint32_t)(s->d.n_points * s->d.point_stride);
            a.stride_words = s->d.stride_words;
            a.n_words = s->d.n_words;
            a.width = views[i].width;
            a.height = views[i].height;
            a.wn = nrv_pad8(a.width);
            a.hn = nrv_pad8(a.height);
            a.netin = base + in_off[i];
            fill_pack(a, d, prec, inv);
            fill_derived(a, d, views[i], s->d.d_xyz);
            // replays take the cameras of the call from the device copy of the views
            if (views_dev) a.view_dev = &views_dev->v[i];
            NRV_TRY(launch_resolve(a, q));
        }
        if (ev) prof_mark(*ev, q);
        for (int g = 0; g < ngroups; ++g) {
            const int i0 = group_first[g];
            RgbTab tab{};
            tab.on = 1;
            for (int i = 0, j = 0; i < n; ++i)
                if (group_of[i] == g) tab.p[j++] = rgb[i];
            net->rgb_tab = tab;
            const nrv_status st = net_forward(net, base + in_off[i0], group_n[g], views[i0].height,
                                              views[i0].width, prec, rgb[i0], q, false);
            net->rgb_tab = RgbTab{};
            NRV_TRY(st);
        }
        if (ev) prof_mark(*ev, q);
        return NRV_OK;
    };

    if (g_profile) {  // eager, with stage events
        std::vector<cudaEvent_t> ev;
        NRV_TRY(frame(nullptr, &ev, st));
        g_prof_events.push_back(ev);
        return NRV_OK;
    }
    for (BatchGraph& g : net->graphs)
        if (g.sig == sig) {
            NRV_CHECK_CUDA(cudaMemcpyAsync(g.views_dev, &rv, sizeof(RViews), cudaMemcpyHostToDevice, st));
            NRV_CHECK_CUDA(cudaGraphLaunch(g.exec, st));
            g_launches.fetch_add(g.kernels);
            return NRV_OK;
        }
    // first frame of this signature: run it, then capture the same work for replay
    NRV_TRY(frame(nullptr, nullptr, st));
    if (net->graphs.size() >= 8) net->drop_graphs();
    BatchGraph g;
    g.sig = make_sig();   // the eager frame may have grown the workspaces
    NRV_CHECK_CUDA(cudaMalloc(&g.views_dev, sizeof(RViews)));
    cudaStream_t cap;
    NRV_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    // the capture stream starts after the eager frame
    cudaEvent_t ready;
    NRV_CHECK_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    NRV_CHECK_CUDA(cudaEventRecord(ready, st));
    NRV_CHECK_CUDA(cudaStreamWaitEvent(cap, ready, 0));
    cudaGraph_t graph = nullptr;
    nrv_status fs = NRV_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const uint64_t before = g_launches.load();
        fs = frame(g.views_dev, nullptr, cap);
        e = cudaStreamEndCapture(cap, &graph);
        // captured launches run only when the graph is replayed
        g.kernels = g_launches.load() - before;
        g_launches.fetch_sub(g.kernels);
    }
    if (e == cudaSuccess && fs == NRV_OK) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(cap);
    cudaStreamDestroy(cap);
    cudaEventDestroy(ready);
    if (e != cudaSuccess || fs != NRV_OK) {
        cudaGetLastError();
        cudaFree(g.views_dev);
        // the eager frame already produced the output; replay is only an optimisation
        clear_error();
        return NRV_OK;
    }
    net->graphs.push_back(g);
    return NRV_OK;
}

extern "C" nrv_status nrv_sync_status(nrv_stream stream) {
    clear_error();
    NRV_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned* w = status_word();
    if (!w) return fail(NRV_ERR_CUDA, "status word unavailable");
    unsigned h = 0;
    NRV_CHECK_CUDA(cudaMemcpy(&h, w, sizeof(h), cudaMemcpyDeviceToHost));
    NRV_CHECK_CUDA(cudaMemset(w, 0, sizeof(unsigned)));
    if (h & STATUS_TIMEOUT) return fail(NRV_ERR_TIMEOUT, "a device-side wait gave up (status %u)", h);
    if (h) return fail(NRV_ERR_CUDA, "device status %u", h);
    return NRV_OK;
}
