/*
 * CPU ORACLE -- test infrastructure only.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may call this code; the rendering library never
 * does, and this file shares nothing with it.
 *
 * Plain, slow, obviously-correct statements of what the method computes:
 *   - the render (visibility) pass of the multi-attribute compute rasterizer:
 *     per pixel, the closest point with the lowest depth (Sec. 3.2), as a
 *     sequential min over all points of a 64-bit key (depth bits, point index);
 *   - the resolve pass: copy the winning point's attributes, depth and
 *     coverage into G-buffer planes, no colour averaging (Sec. 3.2);
 *   - packing of the G-buffer into the network's input tensor (the paper's
 *     "channel-wise processing" of the rasterizer output, Sec. 4.5, Tab. 3);
 *   - a front-to-back alpha-compositing Gaussian splat renderer that stands in
 *     for the Gaussian Renderer that makes training targets (Sec. 4.2).
 *
 * Compiled with -ffp-contract=off -fno-fast-math: every float multiply, add
 * and divide below is a separately rounded IEEE operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

static inline uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float bitsf(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/*
 * Render pass (Sec. 3.2): world -> screen, then keep per pixel the point with the
 * smallest depth, ties to the lowest index.  The key is (bits(w) << 32) | i where
 * w is the clip-space w (eye-space depth, positive in front of the camera); for
 * positive floats the bit pattern orders like the value.  Pixel row 0 is the top.
 * M is row-major, clip = M * (x, y, z, 1).  key[H*W] is overwritten; empty = ~0.
 */
void oracle_visibility(const float* xyz, uint64_t n, const float* M, int W, int H, float znear,
                       float zfar, uint64_t* key) {
    for (int64_t p = 0; p < (int64_t)W * H; ++p) key[p] = ~0ull;
    const float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    for (uint64_t i = 0; i < n; ++i) {
        float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        float cx = ((M[0] * x + M[1] * y) + M[2] * z) + M[3];
        float cy = ((M[4] * x + M[5] * y) + M[6] * z) + M[7];
        float cw = ((M[12] * x + M[13] * y) + M[14] * z) + M[15];
        if (!(cw >= znear && cw <= zfar)) continue;
        float nx = cx / cw, ny = cy / cw;
        float sx = (nx + 1.0f) * hw, sy = (1.0f - ny) * hh;
        if (!(sx >= 0.0f && sx < (float)W && sy >= 0.0f && sy < (float)H)) continue;
        int px = (int)sx, py = (int)sy;
        uint64_t k = ((uint64_t)fbits(cw) << 32) | (uint64_t)i;
        int64_t p = (int64_t)py * W + px;
        if (k < key[p]) key[p] = k;
    }
}

/*
 * The same render pass on all cores: each thread keeps its own key image over a
 * contiguous range of points (the per-pixel minimum of its points), then the
 * images are combined by an element-wise minimum.  A minimum does not depend on
 * the order its operands are taken in, so the keys equal oracle_visibility's.
 */
void oracle_visibility_mt(const float* xyz, uint64_t n, const float* M, int W, int H,
                          float znear, float zfar, uint64_t* key) {
    const int nth = omp_get_max_threads();
    const int64_t npx = (int64_t)W * H;
    uint64_t* part = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)npx * (size_t)nth);
#pragma omp parallel num_threads(nth)
    {
        const int t = omp_get_thread_num();
        const uint64_t lo = n * (uint64_t)t / (uint64_t)nth, hi = n * (uint64_t)(t + 1) / (uint64_t)nth;
        uint64_t* k = part + (size_t)npx * (size_t)t;
        oracle_visibility(xyz + 3 * lo, hi - lo, M, W, H, znear, zfar, k);
        /* the sub-range's indices start at lo */
        for (int64_t p = 0; p < npx; ++p)
            if (k[p] != ~0ull) k[p] += lo;
    }
#pragma omp parallel for
    for (int64_t p = 0; p < npx; ++p) {
        uint64_t m = ~0ull;
        for (int t = 0; t < nth; ++t) {
            const uint64_t v = part[(size_t)npx * (size_t)t + (size_t)p];
            if (v < m) m = v;
        }
        key[p] = m;
    }
    free(part);
}

/*
 * Resolve pass (Sec. 3.2): for each pixel with a winner, depth = high key word,
 * mask = 1, attribute word c = word c of the winner's record (bit copy).  Empty
 * pixels get zeros everywhere.  gattr is planar: gattr[c * npx + p].
 */
void oracle_resolve(const uint64_t* key, int64_t npx, const uint32_t* attr, int64_t stride_words,
                    int K, uint32_t* depth, uint8_t* mask, uint32_t* gattr) {
    for (int64_t p = 0; p < npx; ++p) {
        uint64_t k = key[p];
        if (k == ~0ull) {
            depth[p] = 0u; mask[p] = 0u;
            for (int c = 0; c < K; ++c) gattr[(int64_t)c * npx + p] = 0u;
        } else {
            uint64_t i = k & 0xFFFFFFFFull;
            depth[p] = (uint32_t)(k >> 32); mask[p] = 1u;
            for (int c = 0; c < K; ++c) gattr[(int64_t)c * npx + p] = attr[i * stride_words + c];
        }
    }
}

/* float32 -> bfloat16, round to nearest even (the format's definition). */
uint16_t oracle_bf16(float f) {
    uint32_t u = fbits(f);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

/*
 * float32 -> FP8 E4M3 (OCP "fn" variant: bias 7, no infinities, max 448,
 * subnormal step 2^-9), round to nearest even, saturating to +-448, NaN -> 0x7F.
 */
uint8_t oracle_e4m3(float f) {
    if (isnan(f)) return 0x7F;
    uint8_t s = signbit(f) ? 0x80 : 0x00;
    double a = fabs((double)f);
    if (a >= 448.0) return s | 0x7E;
    int e;
    double q;                        /* grid spacing around a */
    if (a < 0x1.0p-6) { e = -6; q = 0x1.0p-9; }
    else { frexp(a, &e); e -= 1; q = ldexp(1.0, e - 3); }
    double r = nearbyint(a / q) * q; /* ties to even under the default rounding mode */
    if (r >= 448.0) return s | 0x7E;
    if (r < 0x1.0p-6) return s | (uint8_t)(r / 0x1.0p-9);          /* subnormal or zero */
    int er;
    double mr = frexp(r, &er);       /* r = mr * 2^er, mr in [0.5, 1) */
    int exp_field = er - 1 + 7;
    int man = (int)((mr * 2.0 - 1.0) * 8.0);
    return s | (uint8_t)(exp_field << 3) | (uint8_t)man;
}

/*
 * Pack the G-buffer into the network input, NHWC with cpad channels over an
 * Hn x Wn canvas (Hn >= H, Wn >= W; the margin is zero).  Channel order: the
 * nch attribute channels, then depth, then coverage, then zeros.  Attribute
 * channel j reads G-buffer word ch_word[j] as f32 (fmt 0), u32 (fmt 1) or byte
 * ch_comp[j] of a u8x4 word (fmt 2), converts it to float and applies
 * f = v * scale + offset (separate multiply and add).  Depth is the float whose
 * bits are the depth plane, scaled the same way; coverage is 1.  Empty pixels
 * are all zero.  out_fmt 0 = f32, 1 = bf16 (RNE), 2 = e4m3 of f * in_scale_inv.
 */
void oracle_pack(const uint32_t* depth, const uint8_t* mask, const uint32_t* gattr, int H, int W,
                 int Hn, int Wn, int nch, const int* ch_word, const int* ch_fmt, const int* ch_comp,
                 const float* ch_scale, const float* ch_offset, float d_scale, float d_offset,
                 int cpad, int out_fmt, float in_scale_inv, void* out) {
    int64_t npx = (int64_t)H * W;
    float* vals = (float*)malloc(sizeof(float) * (size_t)cpad);
    for (int y = 0; y < Hn; ++y)
        for (int x = 0; x < Wn; ++x) {
            for (int c = 0; c < cpad; ++c) vals[c] = 0.0f;
            if (y < H && x < W && mask[(int64_t)y * W + x]) {
                int64_t p = (int64_t)y * W + x;
                for (int j = 0; j < nch; ++j) {
                    uint32_t w = gattr[(int64_t)ch_word[j] * npx + p];
                    float v;
                    if (ch_fmt[j] == 0) v = bitsf(w);
                    else if (ch_fmt[j] == 1) v = (float)w;
                    else v = (float)((w >> (8 * ch_comp[j])) & 255u);
                    float t = v * ch_scale[j];
                    vals[j] = t + ch_offset[j];
                }
                float t = bitsf(depth[p]) * d_scale;
                vals[nch] = t + d_offset;
                vals[nch + 1] = 1.0f;
            }
            int64_t o = ((int64_t)y * Wn + x) * cpad;
            for (int c = 0; c < cpad; ++c) {
                if (out_fmt == 0) ((float*)out)[o + c] = vals[c];
                else if (out_fmt == 1) ((uint16_t*)out)[o + c] = oracle_bf16(vals[c]);
                else ((uint8_t*)out)[o + c] = oracle_e4m3(vals[c] * in_scale_inv);
            }
        }
    free(vals);
}

/* ---------------------------------------------------------------------------
 * Gaussian splat renderer (stands in for the Gaussian Renderer of Sec. 4.2).
 * Every point whose centre projects (same FP32 sequence as above, up to sx, sy)
 * within 3 sigma of the image is an isotropic 2-D Gaussian at the continuous
 * centre (sx, sy).  Points are ordered by (w, index) ascending.  For each pixel
 * centre p = (px + 0.5, py + 0.5), walking that order over the Gaussians with
 * |p - mu|^2 <= (3 sigma)^2:  a = alpha * exp(-|p - mu|^2 / (2 sigma^2)),
 * C += T * a * c, T *= (1 - a), stopping once T < 1e-4.  Black background.
 * Double precision.
 *
 * The steps run on all cores (OpenMP) without changing the result:
 *  1. project and keep the points near the image, in index order (each thread
 *     counts its contiguous block, then writes it at its prefix offset);
 *  2. sort by (w, index): w > 0, so the key (bits(w) << 32) | j, j the kept
 *     point's position in index order, orders like (w, index); an LSD radix
 *     sort, eight passes of eight bits, stable in every pass;
 *  3. bin the sorted Gaussians into every 16 x 16 tile their 3-sigma disc may
 *     touch, each tile's list in sorted order (threads take contiguous runs
 *     of the sorted order and write them at per-(tile, thread) prefix offsets);
 *  4. composite each tile's pixels from its list (tiles are independent).
 * ------------------------------------------------------------------------- */

typedef struct { uint32_t i; double sx, sy; } splat_t;

void oracle_splat(const float* xyz, uint64_t n, const float* M, int W, int H, float znear,
                  float zfar, const float* colour, double sigma, double alpha, double* out) {
    const double rad = 3.0 * sigma, rad2 = rad * rad;
    const float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    const int nth = omp_get_max_threads();
    /* 1. project and filter, keeping index order */
    uint64_t* cnt_th = (uint64_t*)calloc((size_t)nth + 1, sizeof(uint64_t));
    splat_t* s = (splat_t*)malloc(sizeof(splat_t) * (size_t)(n > 0 ? n : 1));
    float* wv = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel num_threads(nth)
        {
            const int t = omp_get_thread_num();
            const uint64_t lo = n * (uint64_t)t / (uint64_t)nth, hi = n * (uint64_t)(t + 1) / (uint64_t)nth;
            uint64_t m = pass ? cnt_th[t] : 0;
            for (uint64_t i = lo; i < hi; ++i) {
                float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
                float cx = ((M[0] * x + M[1] * y) + M[2] * z) + M[3];
                float cy = ((M[4] * x + M[5] * y) + M[6] * z) + M[7];
                float cw = ((M[12] * x + M[13] * y) + M[14] * z) + M[15];
                if (!(cw >= znear && cw <= zfar)) continue;
                float nx = cx / cw, ny = cy / cw;
                float sx = (nx + 1.0f) * hw, sy = (1.0f - ny) * hh;
                if (!((double)sx >= -rad && (double)sx < W + rad && (double)sy >= -rad &&
                      (double)sy < H + rad))
                    continue;
                if (pass) {
                    s[m].i = (uint32_t)i; s[m].sx = sx; s[m].sy = sy; wv[m] = cw;
                }
                ++m;
            }
            if (!pass) cnt_th[t + 1] = m;
        }
        if (!pass)
            for (int t = 0; t < nth; ++t) cnt_th[t + 1] += cnt_th[t];
    }
    const uint64_t m = cnt_th[nth];
    /* 2. sort by (w, index) */
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for num_threads(nth)
    for (int64_t j = 0; j < (int64_t)m; ++j) key[j] = ((uint64_t)fbits(wv[j]) << 32) | (uint64_t)j;
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * 256 * (size_t)nth);
    for (int shift = 0; shift < 64; shift += 8) {
#pragma omp parallel num_threads(nth)
        {
            const int t = omp_get_thread_num();
            const uint64_t lo = m * (uint64_t)t / (uint64_t)nth, hi = m * (uint64_t)(t + 1) / (uint64_t)nth;
            uint64_t* h = hist + 256 * (size_t)t;
            memset(h, 0, 256 * sizeof(uint64_t));
            for (uint64_t j = lo; j < hi; ++j) ++h[(key[j] >> shift) & 255];
#pragma omp barrier
#pragma omp single
            {
                uint64_t acc = 0;   /* offsets: digit-major, then thread order (stable) */
                for (int d = 0; d < 256; ++d)
                    for (int u = 0; u < nth; ++u) {
                        const uint64_t c = hist[256 * (size_t)u + d];
                        hist[256 * (size_t)u + d] = acc;
                        acc += c;
                    }
            }
            for (uint64_t j = lo; j < hi; ++j) tmp[h[(key[j] >> shift) & 255]++] = key[j];
        }
        uint64_t* sw = key; key = tmp; tmp = sw;
    }
    free(hist);
    free(tmp);
    free(wv);
    /* 3. bin the sorted splats into every tile their 3-sigma disc may touch, keeping order */
    const int T = 16;
    const int tx = (W + T - 1) / T, ty = (H + T - 1) / T, nt = tx * ty;
    int64_t* cnt = (int64_t*)calloc((size_t)nt * (size_t)nth + 1, sizeof(int64_t));   /* [tile][thread] */
    int64_t* tile_start = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
    uint32_t* list = NULL;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            int64_t acc = 0;
            for (int t = 0; t < nt; ++t) {
                tile_start[t] = acc;
                for (int u = 0; u < nth; ++u) {
                    const int64_t c = cnt[(size_t)t * nth + u];
                    cnt[(size_t)t * nth + u] = acc;
                    acc += c;
                }
            }
            tile_start[nt] = acc;
            list = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(acc > 0 ? acc : 1));
        }
#pragma omp parallel num_threads(nth)
        {
            const int u = omp_get_thread_num();
            const uint64_t lo = m * (uint64_t)u / (uint64_t)nth, hi = m * (uint64_t)(u + 1) / (uint64_t)nth;
            for (uint64_t k = lo; k < hi; ++k) {
                const splat_t* g = &s[key[k] & 0xFFFFFFFFull];
                int x0 = (int)floor((g->sx - rad) / T), x1 = (int)floor((g->sx + rad) / T);
                int y0 = (int)floor((g->sy - rad) / T), y1 = (int)floor((g->sy + rad) / T);
                if (x0 < 0) x0 = 0;
                if (y0 < 0) y0 = 0;
                if (x1 > tx - 1) x1 = tx - 1;
                if (y1 > ty - 1) y1 = ty - 1;
                for (int b = y0; b <= y1; ++b)
                    for (int a = x0; a <= x1; ++a) {
                        int64_t* c = &cnt[(size_t)(b * tx + a) * nth + u];
                        if (pass == 0) ++*c;
                        else list[(*c)++] = (uint32_t)(key[k] & 0xFFFFFFFFull);
                    }
            }
        }
    }
    /* 4. composite */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
    for (int t = 0; t < nt; ++t) {
        int bx = (t % tx) * T, by = (t / tx) * T;
        for (int py = by; py < by + T && py < H; ++py)
            for (int px = bx; px < bx + T && px < W; ++px) {
                double cx = px + 0.5, cy = py + 0.5, Tr = 1.0;
                double acc[3] = {0.0, 0.0, 0.0};
                for (int64_t q = tile_start[t]; q < tile_start[t + 1]; ++q) {
                    const splat_t* g = &s[list[q]];
                    double dx = cx - g->sx, dy = cy - g->sy, d2 = dx * dx + dy * dy;
                    if (d2 > rad2) continue;
                    double a = alpha * exp(-d2 / (2.0 * sigma * sigma));
                    const float* c = colour + 3 * (uint64_t)g->i;
                    for (int j = 0; j < 3; ++j) acc[j] += Tr * a * (double)c[j];
                    Tr *= 1.0 - a;
                    if (Tr < 1e-4) break;
                }
                double* o = out + 3 * ((int64_t)py * W + px);
                o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
            }
    }
    free(list);
    free(tile_start);
    free(cnt);
    free(key);
    free(cnt_th);
    free(s);
}

/* ---------------------------------------------------------------------------
 * Anisotropic Gaussian splat renderer (the Gaussian Renderer's elongated
 * Gaussians, Sec. 4.2): every point is a 3-D Gaussian N(p, Sigma) with
 * Sigma = r0^2 R diag(s^2, 1, 1) R^T, R a rotation whose first axis is the
 * point's velocity v (Sigma = r0^2 (I + (s^2 - 1) u u^T), u = v / |v|; an
 * isotropic r0^2 I where v = 0).  It is projected to the screen with the
 * Jacobian J of the screen map at p (first-order, EWA-style):
 *   J_x = (W/2) (M_0 c_w - c_x M_3) / c_w^2,  J_y = -(H/2) (M_1 c_w - c_y M_3) / c_w^2,
 *   Sigma' = J Sigma J^T = [[a, b], [b, c]],
 * centred at the same (sx, sy) as the isotropic renderer.  For a pixel centre p
 * the Mahalanobis distance q = d^T Sigma'^-1 d, d = p - (sx, sy); a Gaussian
 * counts where q <= 9 (3 sigma) with alpha * exp(-q / 2), composited front to
 * back in (w, index) order exactly as the isotropic renderer (T < 1e-4 stops).
 * Points whose 3-sigma box misses the image, or whose Sigma' is singular, are
 * dropped.  Serial and plain: it pins and makes small stylised targets.
 * ------------------------------------------------------------------------- */
typedef struct { float w; uint32_t i; double sx, sy, a, b, c, rx, ry; } asplat_t;

static int asplat_cmp(const void* x, const void* y) {
    const asplat_t* p = (const asplat_t*)x;
    const asplat_t* q = (const asplat_t*)y;
    if (p->w < q->w) return -1;
    if (p->w > q->w) return 1;
    return (p->i > q->i) - (p->i < q->i);
}

void oracle_splat_aniso(const float* xyz, uint64_t n, const float* M, int W, int H, float znear,
                        float zfar, const float* colour, const float* vel, double r0, double s,
                        double alpha, double* out) {
    const float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    asplat_t* g = (asplat_t*)malloc(sizeof(asplat_t) * (size_t)(n > 0 ? n : 1));
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        float cx = ((M[0] * x + M[1] * y) + M[2] * z) + M[3];
        float cy = ((M[4] * x + M[5] * y) + M[6] * z) + M[7];
        float cw = ((M[12] * x + M[13] * y) + M[14] * z) + M[15];
        if (!(cw >= znear && cw <= zfar)) continue;
        float nx = cx / cw, ny = cy / cw;
        float sx = (nx + 1.0f) * hw, sy = (1.0f - ny) * hh;
        /* the 3-D covariance */
        double v[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double S3[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double u_rk = vn > 0.0 ? (v[r] / vn) * (v[k] / vn) : 0.0;
                S3[r][k] = r0 * r0 * ((r == k ? 1.0 : 0.0) + (s * s - 1.0) * u_rk);
            }
        /* the screen-map Jacobian at p, in double from the FP32 clip coordinates */
        double dcw = cw, dcx = cx, dcy = cy, J[2][3];
        for (int k = 0; k < 3; ++k) {
            J[0][k] = 0.5 * W * ((double)M[k] * dcw - dcx * (double)M[12 + k]) / (dcw * dcw);
            J[1][k] = -0.5 * H * ((double)M[4 + k] * dcw - dcy * (double)M[12 + k]) / (dcw * dcw);
        }
        double JS[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                JS[r][k] = J[r][0] * S3[0][k] + J[r][1] * S3[1][k] + J[r][2] * S3[2][k];
        double a = JS[0][0] * J[0][0] + JS[0][1] * J[0][1] + JS[0][2] * J[0][2];
        double b = JS[0][0] * J[1][0] + JS[0][1] * J[1][1] + JS[0][2] * J[1][2];
        double c = JS[1][0] * J[1][0] + JS[1][1] * J[1][1] + JS[1][2] * J[1][2];
        if (!(a > 0.0 && c > 0.0 && a * c - b * b > 0.0)) continue;
        double rx = 3.0 * sqrt(a), ry = 3.0 * sqrt(c);
        if (!((double)sx + rx >= 0.0 && (double)sx - rx < W && (double)sy + ry >= 0.0 &&
              (double)sy - ry < H))
            continue;
        asplat_t* o = &g[m++];
        o->w = cw; o->i = (uint32_t)i; o->sx = sx; o->sy = sy;
        o->a = a; o->b = b; o->c = c; o->rx = rx; o->ry = ry;
    }
    qsort(g, (size_t)m, sizeof(asplat_t), asplat_cmp);
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            double cxp = px + 0.5, cyp = py + 0.5, Tr = 1.0;
            double acc[3] = {0.0, 0.0, 0.0};
            for (uint64_t k = 0; k < m; ++k) {
                const asplat_t* e = &g[k];
                double dx = cxp - e->sx, dy = cyp - e->sy;
                if (fabs(dx) > e->rx || fabs(dy) > e->ry) continue;
                double det = e->a * e->c - e->b * e->b;
                double q = (e->c * dx * dx - 2.0 * e->b * dx * dy + e->a * dy * dy) / det;
                if (q > 9.0) continue;
                double al = alpha * exp(-0.5 * q);
                const float* col = colour + 3 * (uint64_t)e->i;
                for (int j = 0; j < 3; ++j) acc[j] += Tr * al * (double)col[j];
                Tr *= 1.0 - al;
                if (Tr < 1e-4) break;
            }
            double* o = out + 3 * ((int64_t)py * W + px);
            o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
        }
    free(g);
}

void oracle_bf16_array(const float* in, int64_t n, uint16_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_bf16(in[i]);
}

void oracle_e4m3_array(const float* in, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_e4m3(in[i]);
}
