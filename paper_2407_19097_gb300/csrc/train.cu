// Training of the post-processing network (Sec. 3.3, training details): the
// backward pass of every layer, the L1 reconstruction loss and Adam.
//
// Gradients of the weights are reductions over all pixels.  They are computed
// in fixed pixel chunks whose partial sums are added in a fixed order by a
// second kernel, so a step is bit-for-bit reproducible.
#include "net.h"
#include "net_simt.cuh"

namespace nrv {

// ------------------------------------------------------------------ weight gradients, 3x3 conv
// part[blk][o][tap*cin + c] = sum over the pixels of block blk's tiles of g[q][o] * x[q + tap][c];
// partb[blk][o] = sum of g.  A tile is 256 pixels: R rows x TW pixels, TW = 128, 64 or 32
// (the widest that the image width fills), R = 256 / TW.  The block stages the tile's
// gradients (16 output channels) and its input rows with a one-pixel halo (CG input
// channels) in shared memory as FP32, then each thread accumulates a 4 (output) x 4 (input)
// block of one tap -- 16 FMAs per pair of 16-byte shared loads.  Grid: (blocks over tiles,
// output groups of 16, input groups of CG); 144 threads = 9 taps x 4 x 4 blocks (CG = 16) or
// 72 (CG = 8).  Each block takes a contiguous run of tiles, so partials are summed in a
// fixed order: the result is deterministic.
constexpr int WG_TILE = 256;          // pixels per tile
constexpr int WG_THREADS = 144;
constexpr int WG_XS = 520;            // staged input pixels: max over TW of (R + 2) x (TW + 2)

inline int wgrad_tile_width(int w) { return w >= 128 ? 128 : (w >= 64 ? 64 : 32); }

template <typename T>
__global__ void __launch_bounds__(WG_THREADS) wgrad3_kernel(TView<const T> g, int cout,
                                                            TView<const T> x1, int c1,
                                                            TView<const T> x2, int c2, int n,
                                                            int h, int w, int TW,
                                                            int tiles_per_block, float* part,
                                                            float* partb) {
    constexpr int CGMAX = 16;
    __shared__ __align__(16) float gs[WG_TILE][16];
    __shared__ __align__(16) float xs[WG_XS][CGMAX];
    const int R = WG_TILE / TW;
    const int cin = c1 + c2;
    const int CG = cin < 16 ? cin : 16;   // 8 (the packed first-layer input) or 16
    const int og = blockIdx.y * 16, cg = blockIdx.z * CG;
    const int t = threadIdx.x;
    const int ncb = CG / 4;               // 4-channel blocks of the input group
    const bool active = t < 9 * 4 * ncb;
    const int tap = t / (4 * ncb), ob = (t / ncb) % 4, cb = t % ncb;
    const int dy = tap / 3, dx = tap % 3;
    // which source holds this input group
    const TView<const T> xv = cg < c1 ? x1 : x2;
    const int cx = cg < c1 ? cg : cg - c1;
    const int tiles_x = (w + TW - 1) / TW, pairs = (h + R - 1) / R;
    const long long ntiles = (long long)n * pairs * tiles_x;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    float bsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const long long t0 = (long long)blockIdx.x * tiles_per_block;
    const long long t1 = t0 + tiles_per_block < ntiles ? t0 + tiles_per_block : ntiles;
    for (long long tile = t0; tile < t1; ++tile) {
        const int xt = (int)(tile % tiles_x);
        const long long rest = tile / tiles_x;
        const int pr = (int)(rest % pairs);
        const int img = (int)(rest / pairs);
        const int x0 = xt * TW, y0 = R * pr;
        __syncthreads();
        // gradients of the tile's R x TW pixels, 16 output channels (zero outside the image)
        for (int i = t; i < WG_TILE * 2; i += WG_THREADS) {
            const int half = i & 1, px = (i >> 1) % TW, py = (i >> 1) / TW;
            const int y = y0 + py, x = x0 + px;
            float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (y < h && x < w) ld8<T>(g.at((size_t)img * h + y, x, og + 8 * half, w), v);
#pragma unroll
            for (int k = 0; k < 8; ++k) gs[py * TW + px][8 * half + k] = v[k];
        }
        // input rows y0-1 .. y0+R, pixels x0-1 .. x0+TW, CG channels (zero padding)
        const int nxh = CG / 8;
        for (int i = t; i < (R + 2) * (TW + 2) * nxh; i += WG_THREADS) {
            const int part8 = i % nxh, px = (i / nxh) % (TW + 2), ry = (i / nxh) / (TW + 2);
            const int y = y0 - 1 + ry, x = x0 - 1 + px;
            float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (y >= 0 && y < h && x >= 0 && x < w)
                ld8<T>(xv.at((size_t)img * h + y, x, cx + 8 * part8, w), v);
#pragma unroll
            for (int k = 0; k < 8; ++k) xs[ry * (TW + 2) + px][8 * part8 + k] = v[k];
        }
        __syncthreads();
        if (active) {
            for (int py = 0; py < R; ++py) {
                const float* grow = &gs[py * TW][4 * ob];
                const float* xrow = &xs[(py + dy) * (TW + 2) + dx][4 * cb];
#pragma unroll 4
                for (int px = 0; px < TW; ++px) {
                    const float4 gv = *reinterpret_cast<const float4*>(grow + px * 16);
                    const float4 xv4 = *reinterpret_cast<const float4*>(xrow + px * CGMAX);
                    const float ga[4] = {gv.x, gv.y, gv.z, gv.w};
                    const float xa[4] = {xv4.x, xv4.y, xv4.z, xv4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ga[i], xa[j], acc[i][j]);
                    if (tap == 0 && cb == 0) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) bsum[i] += ga[i];
                    }
                }
            }
        }
    }
    if (!active) return;
    const int K = 9 * cin;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            part[((size_t)blockIdx.x * cout + og + 4 * ob + i) * K + tap * cin + cg + 4 * cb + j] =
                acc[i][j];
    if (blockIdx.z == 0 && tap == 0 && cb == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) partb[(size_t)blockIdx.x * cout + og + 4 * ob + i] = bsum[i];
}

// Sums of per-chunk partials: sum i = part[0*stride + i] + part[1*stride + i] + ..., eight
// threads per sum each taking every eighth chunk, their results added in a fixed order (the
// result does not depend on timing).  `mode` says where sum i goes (PyTorch layouts):
//  0  3x3 conv weight: i = o*9*cin + tap*cin + c -> dw[(o*cin_real + c)*9 + tap] (c < cin_real)
//  1  transposed conv weight: i = c*4*cout + ab*cout + o -> dw[(c*cout + o)*4 + ab]
//  2  copy: dw[i]
//  3  transposed conv bias: i = o, each chunk contributing part[ab*cout + o] for ab = 0..3
struct ReduceSeg {
    const float* part;
    int nchunks;
    size_t stride;
    int count, mode, cout, cin, cin_real;
    float* dw;
};

__device__ __forceinline__ void reduce_item(const ReduceSeg& R, int i, int tx, int ty,
                                            float (*red)[33]) {
    float s = 0.0f;
    if (i < R.count)
        for (int ch = ty; ch < R.nchunks; ch += 8) {
            const float* pc = R.part + (size_t)ch * R.stride;
            if (R.mode == 3) s += ((pc[i] + pc[R.cout + i]) + pc[2 * R.cout + i]) + pc[3 * R.cout + i];
            else s += pc[i];
        }
    red[ty][tx] = s;
    __syncthreads();
    if (ty != 0 || i >= R.count) return;
    float t = red[0][tx];
    for (int k = 1; k < 8; ++k) t += red[k][tx];
    if (R.mode == 0) {
        const int K = 9 * R.cin, o = i / K, k = i % K, tap = k / R.cin, c = k % R.cin;
        if (c < R.cin_real) R.dw[((size_t)o * R.cin_real + c) * 9 + tap] = t;
    } else if (R.mode == 1) {
        const int K = 4 * R.cout, c = i / K, k = i % K, ab = k / R.cout, o = k % R.cout;
        R.dw[((size_t)c * R.cout + o) * 4 + ab] = t;
    } else {
        R.dw[i] = t;
    }
}

// Two reductions (a layer's weights and its bias) in one launch: the first segment's
// blocks, then the second's.
__global__ void reduce_partials_kernel(const __grid_constant__ ReduceSeg A,
                                       const __grid_constant__ ReduceSeg B) {
    __shared__ float red[8][33];
    const int nba = (A.count + 31) / 32;
    const bool first = (int)blockIdx.x < nba;
    const int blk = first ? (int)blockIdx.x : (int)blockIdx.x - nba;
    reduce_item(first ? A : B, blk * 32 + threadIdx.x, threadIdx.x, threadIdx.y, red);
}

static nrv_status reduce_partials(const float* part, int nchunks, size_t stride, int count, int mode,
                                  int cout, int cin, int cin_real, float* dw, cudaStream_t s,
                                  const ReduceSeg* second = nullptr) {
    const ReduceSeg A{part, nchunks, stride, count, mode, cout, cin, cin_real, dw};
    ReduceSeg B;
    memset(&B, 0, sizeof(B));
    if (second) B = *second;
    const int blocks = (A.count + 31) / 32 + (B.count + 31) / 32;
    reduce_partials_kernel<<<blocks, dim3(32, 8), 0, s>>>(A, B);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

// ------------------------------------------------------------------ weight gradients, 2x2 transposed conv
// part[chunk][c][ab*cout + o] = sum_{input px in chunk} x[q][c] * g[out(q, ab)][o]
// partb[chunk][ab*cout + o]   = sum g   (only written by the c-group 0 blocks)
template <typename T>
__global__ void __launch_bounds__(256) wgrad_up_kernel(TView<const T> x, int cin, TView<const T> g,
                                                       int cout, int n, int hi, int wi,
                                                       size_t chunk_px, float* part, float* partb) {
    __shared__ float xs[32][16];
    const int cg = blockIdx.y * 16;
    const int K = 4 * cout;
    const size_t npx = (size_t)n * hi * wi;
    const size_t q0 = blockIdx.x * chunk_px;
    const size_t q1 = q0 + chunk_px < npx ? q0 + chunk_px : npx;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
    float bsum = 0.0f;
    const int k = threadIdx.x;
    const int ab = k / cout, o = k % cout;
    for (size_t qb = q0; qb < q1; qb += 32) {
        __syncthreads();
        for (int i = threadIdx.x; i < 512; i += 256) {
            const size_t q = qb + (i >> 4);
            xs[i >> 4][i & 15] =
                q < q1 ? ld1<T>(x.at(q / wi, (int)(q % wi), cg + (i & 15), wi)) : 0.0f;
        }
        __syncthreads();
        const int nb = (int)(q1 - qb < 32 ? q1 - qb : 32);
        if (k < K)
            for (int r = 0; r < nb; ++r) {
                const size_t q = qb + r;
                const int X = (int)(q % wi), Y = (int)((q / wi) % hi);
                const size_t img = q / ((size_t)wi * hi);
                const float gv = ld1<T>(
                    g.at(img * 2 * hi + 2 * Y + (ab >> 1), 2 * X + (ab & 1), o, 2 * wi));
                bsum += gv;
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = fmaf(xs[r][j], gv, acc[j]);
            }
    }
    if (k < K) {
#pragma unroll
        for (int j = 0; j < 16; ++j) part[((size_t)blockIdx.x * cin + cg + j) * K + k] = acc[j];
        if (blockIdx.y == 0) partb[(size_t)blockIdx.x * K + k] = bsum;
    }
}

// ------------------------------------------------------------------ head
// gd[q][c] = (sum_o drgb[o] W[o][c]) * (x[q][c] > 0) over the canvas (zero outside the view)
template <typename T>
__global__ void head_dgrad_kernel(const float* drgb, const float* w, TView<const T> x, TView<T> gd,
                                  int n, int hn, int wn, int h, int wd) {
    const size_t total = (size_t)n * hn * wn;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(q % wn), Y = (int)((q / wn) % hn);
        const size_t img = q / ((size_t)wn * hn);
        float out[16];
        if (X < wd && Y < h) {
            const float* gr = drgb + 3 * ((img * h + Y) * wd + X);
            float xv[16];
            ld8<T>(x.at(img * hn + Y, X, 0, wn), xv);
            ld8<T>(x.at(img * hn + Y, X, 8, wn), xv + 8);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float s = fmaf(gr[2], w[32 + c], fmaf(gr[1], w[16 + c], gr[0] * w[c]));
                out[c] = xv[c] > 0.0f ? s : 0.0f;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) out[c] = 0.0f;
        }
        st8<T>(gd.at(img * hn + Y, X, 0, wn), out);
        st8<T>(gd.at(img * hn + Y, X, 8, wn), out + 8);
    }
}

// part[blk][o*16 + c] = sum drgb[o] * x[c]; part[blk][48 + o] = sum drgb[o], over the block's
// chunk of cropped pixels: every thread keeps all 51 sums, then the block adds them (warp
// shuffles, then the 8 warps in order).
template <typename T>
__global__ void __launch_bounds__(256) head_wgrad_kernel(const float* drgb, TView<const T> x, int n,
                                                         int hn, int wn, int h, int wd,
                                                         size_t chunk, float* part) {
    __shared__ float red[8][51];
    float acc[51];
#pragma unroll
    for (int k = 0; k < 51; ++k) acc[k] = 0.0f;
    const size_t total = (size_t)n * h * wd;
    const size_t i0 = blockIdx.x * chunk, i1 = i0 + chunk < total ? i0 + chunk : total;
    for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int X = (int)(i % wd), Y = (int)((i / wd) % h);
        const size_t img = i / ((size_t)wd * h);
        float v[16];
        ld8<T>(x.at(img * hn + Y, X, 0, wn), v);
        ld8<T>(x.at(img * hn + Y, X, 8, wn), v + 8);
        const float d[3] = {drgb[3 * i], drgb[3 * i + 1], drgb[3 * i + 2]};
#pragma unroll
        for (int o = 0; o < 3; ++o) {
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[o * 16 + c] = fmaf(d[o], v[c], acc[o * 16 + c]);
            acc[48 + o] += d[o];
        }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 51; ++k) {
        float a = acc[k];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) red[wp][k] = a;
    }
    __syncthreads();
    if (threadIdx.x < 51) {
        float a = red[0][threadIdx.x];
        for (int k = 1; k < (int)(blockDim.x / 32); ++k) a += red[k][threadIdx.x];
        part[blockIdx.x * 51 + threadIdx.x] = a;
    }
}

// ------------------------------------------------------------------ pooling backward
// ge[q][c] = (0.25 * gp[q/2][c] + gs[q][c]) * (e[q][c] > 0)
template <typename T>
__global__ void pool_bwd_kernel(TView<const T> gp, TView<const T> gs, TView<const T> e, TView<T> ge,
                                int c, int n, int h, int w) {
    const size_t total = (size_t)n * h * w * (c / 8);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int cg = (int)(i % (c / 8)) * 8;
        const size_t q = i / (c / 8);
        const int X = (int)(q % w), Y = (int)((q / w) % h);
        const size_t img = q / ((size_t)w * h);
        const size_t row = img * h + Y;
        float a[8], b[8], m[8], r[8];
        ld8<T>(gp.at(img * (h / 2) + Y / 2, X / 2, cg, w / 2), a);
        ld8<T>(gs.at(row, X, cg, w), b);
        ld8<T>(e.at(row, X, cg, w), m);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = m[k] > 0.0f ? fmaf(0.25f, a[k], b[k]) : 0.0f;
        st8<T>(ge.at(row, X, cg, w), r);
    }
}

// ------------------------------------------------------------------ loss and optimizer
__global__ void l1_partial_kernel(const float* y, const float* t, int64_t n, float* dy,
                                  float inv_n, float* part) {
    __shared__ float red[256];
    float s = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
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

__global__ void l1_final_kernel(const float* part, int nb, double inv_n, float* loss) {
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

static DevBuf g_l1_part;

nrv_status launch_l1(const float* y, const float* t, int64_t n, float* loss, float* dy,
                     cudaStream_t s) {
    const int nb = 512;
    NRV_TRY(g_l1_part.ensure(nb * sizeof(float)));
    l1_partial_kernel<<<nb, 256, 0, s>>>(y, t, n, dy, (float)(1.0 / (double)n), (float*)g_l1_part.p);
    NRV_CHECK_LAUNCH();
    l1_final_kernel<<<1, 256, 0, s>>>((const float*)g_l1_part.p, nb, 1.0 / (double)n, loss);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

// Reconstruction + total-variation loss (Eq. 1 without its perceptual term) on RGB images
// y, t [n][h][w][3]: l1 mean|y - t| + l2 mean (y - t)^2 + tv (mean over horizontal neighbour
// pairs of |y_right - y| + mean over vertical pairs of |y_below - y|), each mean over its
// own count.  dy (if not null) is the gradient, sign(0) = 0.  Partial sums per block, summed
// in a fixed order (deterministic).
__global__ void recon_partial_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                     int64_t n, int h, int w, float* dy, float l1, float l2,
                                     float tv, float inv_n, float inv_nh, float inv_nv,
                                     float* part) {
    __shared__ float red[256];
    auto sgn = [](float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); };
    const int64_t row = 3 * (int64_t)w;
    float s = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float yi = y[i], d = yi - t[i];
        const int x = (int)((i / 3) % w), yy = (int)((i / row) % h);
        float l = l1 * fabsf(d) * inv_n + l2 * d * d * inv_n;
        float g = l1 * sgn(d) * inv_n + 2.0f * l2 * d * inv_n;
        if (tv != 0.0f) {
            if (x + 1 < w) {
                const float e = y[i + 3] - yi;
                l += tv * fabsf(e) * inv_nh;
                g -= tv * sgn(e) * inv_nh;
            }
            if (x > 0) g += tv * sgn(yi - y[i - 3]) * inv_nh;
            if (yy + 1 < h) {
                const float e = y[i + row] - yi;
                l += tv * fabsf(e) * inv_nv;
                g -= tv * sgn(e) * inv_nv;
            }
            if (yy > 0) g += tv * sgn(yi - y[i - row]) * inv_nv;
        }
        s += l;
        if (dy) dy[i] = g;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

nrv_status launch_recon(const float* y, const float* t, int n_img, int h, int w,
                        const nrv_loss_weights& wt, float* loss, float* dy, cudaStream_t s) {
    const int nb = 512;
    NRV_TRY(g_l1_part.ensure(nb * sizeof(float)));
    const int64_t n = (int64_t)n_img * h * w * 3;
    const double nh = (double)n_img * h * (w - 1) * 3, nv = (double)n_img * (h - 1) * w * 3;
    recon_partial_kernel<<<nb, 256, 0, s>>>(y, t, n, h, w, dy, wt.l1, wt.l2, wt.tv,
                                            (float)(1.0 / (double)n), nh > 0 ? (float)(1.0 / nh) : 0.0f,
                                            nv > 0 ? (float)(1.0 / nv) : 0.0f, (float*)g_l1_part.p);
    NRV_CHECK_LAUNCH();
    l1_final_kernel<<<1, 256, 0, s>>>((const float*)g_l1_part.p, nb, 1.0, loss);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

nrv_status launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                       float b1, float b2, float eps, cudaStream_t s) {
    const float bc1 = (float)(1.0 - pow((double)b1, step));
    const float bc2 = (float)(1.0 - pow((double)b2, step));
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    adam_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

// ------------------------------------------------------------------ backward orchestration
static int blocks_for(size_t work, int per = 256) {
    size_t b = (work + per - 1) / per;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b > 0 ? b : 1);
}

template <typename T>
struct Bwd {
    Net* net;
    cudaStream_t s;
    const Geo& g;
    float* dparams;
    T* W1[4];
    T* W2[4];

    T* A(int a) const { return reinterpret_cast<T*>((char*)net->acts.p + net->act_off[a]); }
    // saved activations: row-planar in BF16 (the tensor-core layout), NHWC in FP32
    TView<const T> CA(int a) const {
        return TView<const T>{A(a), net->act_c[a], sizeof(T) == 2 ? 1 : 0};
    }

    nrv_status wgrad_conv(int l, TView<const T> gpre, TView<const T> x1, int c1, TView<const T> x2,
                          int c2, int level) {
        const Layer& L = net->layers[l];
        const int cin = c1 + c2;
        if (sizeof(T) == 2) {
            // BF16: the weight gradient on the tensor cores, the bias gradient beside it
            const bool fits = gpre.planar && !gpre.coff && gpre.ld == L.cout && x1.planar &&
                              !x1.coff && x1.ld == c1 &&
                              (!c2 || (x2.planar && !x2.coff && x2.ld == c2));
            if (fits) {
                const int groups = cin / 16 > 0 ? cin / 16 : 1;
                const size_t per_split = (size_t)L.cout * 9 * cin;
                const size_t max_split = (size_t)(304 + groups - 1) / groups;
                NRV_TRY(net->partial.ensure((max_split * (per_split + L.cout)) * sizeof(float)));
                float* part = (float*)net->partial.p;
                float* partb = part + max_split * per_split;
                int nsplit = 0;
                const nrv_status st = tc_wgrad(net, l, gpre.p, x1.p, c1, c2 ? x2.p : nullptr, c2, g.n,
                                               g.h[level], g.w[level], part, max_split * per_split,
                                               partb, &nsplit, s);
                if (st == NRV_OK) {
                    const ReduceSeg bias{partb, nsplit, (size_t)L.cout, L.cout, 2, L.cout, cin, L.cin,
                                         dparams + L.boff};
                    return reduce_partials(part, nsplit, per_split, (int)per_split, 0, L.cout, cin,
                                           L.cin, dparams + L.woff, s, &bias);
                }
                if (st != NRV_ERR_UNSUPPORTED) return st;
                clear_error();
            }
        }
        const int CG = cin < 16 ? cin : 16;
        if (cin % CG || (c2 && c1 % CG) || L.cout % 16)
            return fail(NRV_ERR_UNSUPPORTED, "weight gradient: channel groups");
        const int h = g.h[level], w = g.w[level];
        const int TW = wgrad_tile_width(w), R = WG_TILE / TW;
        const long long ntiles = (long long)g.n * ((h + R - 1) / R) * ((w + TW - 1) / TW);
        const int groups = (L.cout / 16) * (cin / CG);
        // about 4 blocks per SM in all, each a contiguous run of tiles
        long long nblk = (152LL * 4 + groups - 1) / groups;
        if (nblk > ntiles) nblk = ntiles;
        if (nblk < 1) nblk = 1;
        const int tpb = (int)((ntiles + nblk - 1) / nblk);
        nblk = (ntiles + tpb - 1) / tpb;
        const size_t need = ((size_t)nblk * L.cout * 9 * cin + (size_t)nblk * L.cout) * sizeof(float);
        NRV_TRY(net->partial.ensure(need));
        float* part = (float*)net->partial.p;
        float* partb = part + (size_t)nblk * L.cout * 9 * cin;
        wgrad3_kernel<T><<<dim3((unsigned)nblk, L.cout / 16, cin / CG), WG_THREADS, 0, s>>>(
            gpre, L.cout, x1, c1, x2, c2, g.n, h, w, TW, tpb, part, partb);
        NRV_CHECK_LAUNCH();
        NRV_TRY(reduce_partials(part, (int)nblk, (size_t)L.cout * 9 * cin, L.cout * 9 * cin, 0, L.cout,
                                cin, L.cin, dparams + L.woff, s));
        return reduce_partials(partb, (int)nblk, L.cout, L.cout, 2, L.cout, cin, L.cin,
                               dparams + L.boff, s);
    }

    nrv_status dgrad_conv(int l, TView<const T> gpre, TView<T> out, TView<const T> mask,
                          int level) {
        // BF16: on the tensor cores (a 3x3 conv with the flipped, transposed kernel)
        if (sizeof(T) == 2) {
            const Layer& L = net->layers[l];
            const bool fits = gpre.planar && out.planar && !gpre.coff && !out.coff &&
                              gpre.ld == L.cout && out.ld == L.cin &&
                              (!mask.p || (mask.planar && !mask.coff && mask.ld == L.cin));
            if (fits) {
                const nrv_status st = tc_dgrad(net, l, gpre.p, out.p, mask.p, g.n, g.h[level],
                                               g.w[level], s);
                if (st != NRV_ERR_UNSUPPORTED) return st;
                clear_error();
            }
        }
        // this translation unit has its own instance of the kernel template
        static bool attr = false;
        if (!attr) {
            NRV_CHECK_CUDA(cudaFuncSetAttribute(conv3_simt_kernel<T>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                9 * 128 * 16 * 4));
            attr = true;
        }
        const Layer& L = net->layers[l];
        Conv3Args<T> a;
        a.x1 = gpre;
        a.c1 = L.cout;
        a.x2 = TView<const T>{nullptr, 0};
        a.c2 = 0;
        a.w = (const float*)net->wtf32.p + net->wf_off[l];
        a.bias = nullptr;
        a.y = out;
        a.cout = L.cin;
        a.n = g.n; a.h = g.h[level]; a.w_ = g.w[level];
        a.relu = 0;
        a.mask = mask;
        const size_t npx = g.px(level);
        dim3 grid((unsigned)((npx + 127) / 128), L.cin / 16);
        conv3_simt_kernel<T><<<grid, 128, (size_t)9 * L.cout * 16 * 4, s>>>(a);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    }

    // weight and bias gradient of transposed conv l: x at level_in, gout one level up
    nrv_status wgrad_up(int l, TView<const T> x, TView<const T> gout, int level_in) {
        const Layer& L = net->layers[l];
        if (sizeof(T) == 2 && x.planar && !x.coff && x.ld == L.cin && gout.planar &&
            gout.ld % 8 == 0 && gout.coff % 8 == 0 && gout.coff + L.cout <= gout.ld) {
            // BF16: on the tensor cores, the bias gradient beside it
            const int groups = 4 * L.cout <= 128 ? 1 : 2;
            const size_t per_split = (size_t)L.cin * 4 * L.cout;
            const size_t max_split = (size_t)(304 + groups - 1) / groups;
            NRV_TRY(net->partial.ensure((max_split * (per_split + 4 * L.cout)) * sizeof(float)));
            float* part = (float*)net->partial.p;
            float* partb = part + max_split * per_split;
            int nsplit = 0;
            const nrv_status st = tc_wgrad_up(net, l, gout.p, gout.ld, gout.coff, x.p, g.n,
                                              g.h[level_in], g.w[level_in], part,
                                              max_split * per_split, partb, &nsplit, s);
            if (st == NRV_OK) {
                // bias, per split: the four kernel positions' sums of each channel
                const ReduceSeg bias{partb, nsplit, (size_t)4 * L.cout, L.cout, 3, L.cout, L.cin,
                                     L.cin, dparams + L.boff};
                return reduce_partials(part, nsplit, per_split, (int)per_split, 1, L.cout, L.cin,
                                       L.cin, dparams + L.woff, s, &bias);
            }
            if (st != NRV_ERR_UNSUPPORTED) return st;
            clear_error();
        }
        const size_t npx = g.px(level_in);
        const int groups = L.cin / 16;
        size_t nch = (608 + groups - 1) / groups;
        const size_t maxch = (npx + 127) / 128;
        if (nch > maxch) nch = maxch;
        if (nch < 1) nch = 1;
        const size_t chunk = (npx + nch - 1) / nch;
        nch = (npx + chunk - 1) / chunk;
        const int K = 4 * L.cout;
        NRV_TRY(net->partial.ensure((nch * L.cin * K + nch * K) * sizeof(float)));
        float* part = (float*)net->partial.p;
        float* partb = part + nch * L.cin * K;
        wgrad_up_kernel<T><<<dim3((unsigned)nch, groups), 256, 0, s>>>(
            x, L.cin, gout, L.cout, g.n, g.h[level_in], g.w[level_in], chunk, part, partb);
        NRV_CHECK_LAUNCH();
        NRV_TRY(reduce_partials(part, (int)nch, (size_t)L.cin * K, L.cin * K, 1, L.cout, L.cin, L.cin,
                                dparams + L.woff, s));
        return reduce_partials(partb, (int)nch, K, L.cout, 3, L.cout, L.cin, L.cin,
                               dparams + L.boff, s);
    }

    // data gradient of transposed conv l at level_in, zeroed where the layer's input xm (a
    // ReLU output) is not positive
    nrv_status dgrad_up(int l, TView<const T> gout, TView<const T> xm, TView<T> gx, int level_in) {
        const Layer& L = net->layers[l];
        const size_t npx = g.px(level_in);
        if (sizeof(T) == 2 && gout.planar && gx.planar && !gx.coff && gx.ld == L.cin && xm.planar &&
            !xm.coff && xm.ld == L.cin) {
            // BF16: on the tensor cores
            const nrv_status st = tc_updgrad(net, l, gout.p, gout.ld, gout.coff, xm.p, gx.p, g.n,
                                             g.h[level_in], g.w[level_in], s);
            if (st != NRV_ERR_UNSUPPORTED) return st;
            clear_error();
        }
        dim3 grid((unsigned)((npx + 127) / 128), L.cin / 16);
        upconv2_dgrad_kernel<T><<<grid, 128, (size_t)4 * 16 * L.cout * 4, s>>>(
            gout, L.cout, (const float*)net->wf32.p + net->wf_off[l], L.cin, xm, gx, g.n,
            g.h[level_in], g.w[level_in]);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    }

    nrv_status upconv_bwd(int l, int xin, TView<const T> gout, TView<T> gx, int level_in) {
        NRV_TRY(wgrad_up(l, CA(xin), gout, level_in));
        return dgrad_up(l, gout, CA(xin), gx, level_in);
    }

    nrv_status pool_bwd(TView<const T> gp, TView<const T> gs, int e, TView<T> ge, int level) {
        const int c = net->act_c[e];
        pool_bwd_kernel<T><<<blocks_for(g.px(level) * c / 8), 256, 0, s>>>(
            gp, gs, CA(e), ge, c, g.n, g.h[level], g.w[level]);
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    }

    // gradients: row-planar in BF16 (the tensor-core layout), NHWC in FP32; coff selects a
    // channel range (the skip half of a concatenation's gradient)
    static constexpr int kPlanar = sizeof(T) == 2 ? 1 : 0;
    static TView<T> V(T* p, int ld) { return TView<T>{p, ld, kPlanar}; }
    static TView<const T> C(T* p, int ld, int coff = 0) {
        return TView<const T>{p, ld, kPlanar, coff};
    }

    nrv_status run(const float* drgb, const T* netin) {
        const TView<const T> none{nullptr, 0};
        const int H = net->geo_H, Wd = net->geo_W;
        // head
        const Layer& Lh = net->layers[L_HEAD];
        head_dgrad_kernel<T><<<blocks_for(g.px(0)), 256, 0, s>>>(
            drgb, (const float*)net->params.p + Lh.woff, CA(A_D0B), V(W1[0], 16), g.n, g.h[0],
            g.w[0], H, Wd);
        NRV_CHECK_LAUNCH();
        {
            const size_t tot = (size_t)g.n * H * Wd;
            size_t nch = 608;
            size_t chunk = (tot + nch - 1) / nch;
            if (chunk < 64) chunk = 64;
            nch = (tot + chunk - 1) / chunk;
            NRV_TRY(net->partial.ensure(nch * 51 * sizeof(float)));
            head_wgrad_kernel<T><<<(unsigned)nch, 256, 0, s>>>(drgb, CA(A_D0B), g.n, g.h[0], g.w[0],
                                                               H, Wd, chunk, (float*)net->partial.p);
            NRV_CHECK_LAUNCH();
            // weight (48) and bias (3) are consecutive in the parameter vector
            if (Lh.boff != Lh.woff + 48) return fail(NRV_ERR_STATE, "head parameter layout");
            NRV_TRY(reduce_partials((const float*)net->partial.p, (int)nch, 51, 51, 2, 3, 16, 16,
                                    dparams + Lh.woff, s));
        }
        // level 0 decoder
        NRV_TRY(wgrad_conv(L_D0B, C(W1[0], 16), CA(A_D0A), 16, none, 0, 0));
        NRV_TRY(dgrad_conv(L_D0B, C(W1[0], 16), V(W2[0], 16), CA(A_D0A), 0));
        NRV_TRY(wgrad_conv(L_D0A, C(W2[0], 16), CA(A_UP1), 16, CA(A_E0B), 16, 0));
        NRV_TRY(dgrad_conv(L_D0A, C(W2[0], 16), V(W1[0], 32), none, 0));
        NRV_TRY(upconv_bwd(L_UP1, A_D1B, C(W1[0], 32), V(W1[1], 32), 1));
        // level 1 decoder
        NRV_TRY(wgrad_conv(L_D1B, C(W1[1], 32), CA(A_D1A), 32, none, 0, 1));
        NRV_TRY(dgrad_conv(L_D1B, C(W1[1], 32), V(W2[1], 32), CA(A_D1A), 1));
        NRV_TRY(wgrad_conv(L_D1A, C(W2[1], 32), CA(A_UP2), 32, CA(A_E1B), 32, 1));
        NRV_TRY(dgrad_conv(L_D1A, C(W2[1], 32), V(W1[1], 64), none, 1));
        NRV_TRY(upconv_bwd(L_UP2, A_D2B, C(W1[1], 64), V(W1[2], 64), 2));
        // level 2 decoder
        NRV_TRY(wgrad_conv(L_D2B, C(W1[2], 64), CA(A_D2A), 64, none, 0, 2));
        NRV_TRY(dgrad_conv(L_D2B, C(W1[2], 64), V(W2[2], 64), CA(A_D2A), 2));
        NRV_TRY(wgrad_conv(L_D2A, C(W2[2], 64), CA(A_UP3), 64, CA(A_E2B), 64, 2));
        NRV_TRY(dgrad_conv(L_D2A, C(W2[2], 64), V(W1[2], 128), none, 2));
        NRV_TRY(upconv_bwd(L_UP3, A_E3B, C(W1[2], 128), V(W1[3], 128), 3));
        // bottom level
        NRV_TRY(wgrad_conv(L_E3B, C(W1[3], 128), CA(A_E3A), 128, none, 0, 3));
        NRV_TRY(dgrad_conv(L_E3B, C(W1[3], 128), V(W2[3], 128), CA(A_E3A), 3));
        NRV_TRY(wgrad_conv(L_E3A, C(W2[3], 128), CA(A_P2), 64, none, 0, 3));
        NRV_TRY(dgrad_conv(L_E3A, C(W2[3], 128), V(W1[3], 64), none, 3));
        // level 2 encoder: skip gradient sits in channels 64..127 of W1[2]
        NRV_TRY(pool_bwd(C(W1[3], 64), C(W1[2], 128, 64), A_E2B, V(W2[2], 64), 2));
        NRV_TRY(wgrad_conv(L_E2B, C(W2[2], 64), CA(A_E2A), 64, none, 0, 2));
        NRV_TRY(dgrad_conv(L_E2B, C(W2[2], 64), V(W1[2], 64), CA(A_E2A), 2));
        NRV_TRY(wgrad_conv(L_E2A, C(W1[2], 64), CA(A_P1), 32, none, 0, 2));
        NRV_TRY(dgrad_conv(L_E2A, C(W1[2], 64), V(W2[2], 32), none, 2));
        // level 1 encoder: skip gradient in channels 32..63 of W1[1]
        NRV_TRY(pool_bwd(C(W2[2], 32), C(W1[1], 64, 32), A_E1B, V(W2[1], 32), 1));
        NRV_TRY(wgrad_conv(L_E1B, C(W2[1], 32), CA(A_E1A), 32, none, 0, 1));
        NRV_TRY(dgrad_conv(L_E1B, C(W2[1], 32), V(W1[1], 32), CA(A_E1A), 1));
        NRV_TRY(wgrad_conv(L_E1A, C(W1[1], 32), CA(A_P0), 16, none, 0, 1));
        NRV_TRY(dgrad_conv(L_E1A, C(W1[1], 32), V(W2[1], 16), none, 1));
        // level 0 encoder: skip gradient in channels 16..31 of W1[0]
        NRV_TRY(pool_bwd(C(W2[1], 16), C(W1[0], 32, 16), A_E0B, V(W2[0], 16), 0));
        NRV_TRY(wgrad_conv(L_E0B, C(W2[0], 16), CA(A_E0A), 16, none, 0, 0));
        NRV_TRY(dgrad_conv(L_E0B, C(W2[0], 16), V(W1[0], 16), CA(A_E0A), 0));
        NRV_TRY(wgrad_conv(L_E0A, C(W1[0], 16), C(const_cast<T*>(netin), net->c0p), net->c0p, none,
                           0, 0));
        return NRV_OK;
    }
};

// The training forward keeps its input pointer for the first layer's weight gradient.

nrv_status net_layer_wgrad(Net* net, int l, const void* dy, const void* x1, const void* x2, int n,
                           int h, int w, nrv_prec prec, float* dgrad, cudaStream_t s) {
    const Layer& L = net->layers[l];
    if (L.kind == UPCONV2) {
        // transposed conv: x1 at (n, h, w), dy at (n, 2h, 2w)
        if (x2) return fail(NRV_ERR_ARG, "layer %s: x2 must be NULL", L.name);
        Geo g;
        memset(&g, 0, sizeof(g));
        g.n = n;
        g.h[0] = h;
        g.w[0] = w;
        if (prec == NRV_PREC_F32) {
            using T = float;
            Bwd<T> b{net, s, g, dgrad, {}, {}};
            return b.wgrad_up(l, TView<const T>{(const T*)x1, L.cin},
                              TView<const T>{(const T*)dy, L.cout}, 0);
        }
        if (prec != NRV_PREC_BF16) return fail(NRV_ERR_UNSUPPORTED, "weight gradients in F32 or BF16");
        using T = __nv_bfloat16;
        const size_t rows = (size_t)n * h;
        auto al = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
        const size_t bg = al(4 * rows * w * L.cout * 2), bx = al(rows * w * L.cin * 2);
        NRV_TRY(net->layer_ws.ensure(bg + bx));
        char* ws = (char*)net->layer_ws.p;
        T *pg = (T*)ws, *px = (T*)(ws + bg);
        NRV_TRY(relayout(dy, pg, 2 * rows, 2 * w, L.cout, 2, true, s));
        NRV_TRY(relayout(x1, px, rows, w, L.cin, 2, true, s));
        Bwd<T> b{net, s, g, dgrad, {}, {}};
        return b.wgrad_up(l, TView<const T>{px, L.cin, 1}, TView<const T>{pg, L.cout, 1}, 0);
    }
    if (L.kind != CONV3) return fail(NRV_ERR_ARG, "layer %s has no weight gradient here", L.name);
    int c1 = l == L_E0A ? net->c0p : L.cin, c2 = 0;
    if (l == L_D2A || l == L_D1A || l == L_D0A) c1 = c2 = L.cin / 2;
    if ((c2 > 0) != (x2 != nullptr))
        return fail(NRV_ERR_ARG, "layer %s: x2 must be %s", L.name, c2 ? "given" : "NULL");
    Geo g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.h[0] = h;
    g.w[0] = w;
    if (prec == NRV_PREC_F32) {
        using T = float;
        Bwd<T> b{net, s, g, dgrad, {}, {}};
        return b.wgrad_conv(l, TView<const T>{(const T*)dy, L.cout}, TView<const T>{(const T*)x1, c1},
                            c1, TView<const T>{(const T*)x2, c2}, c2, 0);
    }
    if (prec != NRV_PREC_BF16) return fail(NRV_ERR_UNSUPPORTED, "weight gradients in F32 or BF16");
    // BF16: row-planar copies, as the backward pass keeps its tensors
    using T = __nv_bfloat16;
    const size_t rows = (size_t)n * h;
    auto al = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
    const size_t bg = al(rows * w * L.cout * 2), b1 = al(rows * w * c1 * 2), b2 = al(rows * w * c2 * 2);
    NRV_TRY(net->layer_ws.ensure(bg + b1 + b2));
    char* ws = (char*)net->layer_ws.p;
    T *pg = (T*)ws, *p1 = (T*)(ws + bg), *p2 = c2 ? (T*)(ws + bg + b1) : nullptr;
    NRV_TRY(relayout(dy, pg, rows, w, L.cout, 2, true, s));
    NRV_TRY(relayout(x1, p1, rows, w, c1, 2, true, s));
    if (c2) NRV_TRY(relayout(x2, p2, rows, w, c2, 2, true, s));
    Bwd<T> b{net, s, g, dgrad, {}, {}};
    return b.wgrad_conv(l, TView<const T>{pg, L.cout, 1}, TView<const T>{p1, c1, 1}, c1,
                        TView<const T>{p2, c2, 1}, c2, 0);
}

nrv_status net_layer_dgrad(Net* net, int l, const void* dy, const void* mask, int n, int h, int w,
                           nrv_prec prec, void* dx, cudaStream_t s) {
    const Layer& L = net->layers[l];
    if (L.kind == UPCONV2) {
        // transposed conv: dy at (n, 2h, 2w), mask and dx at (n, h, w)
        if (!mask) return fail(NRV_ERR_ARG, "layer %s: the mask (the layer's input) is required", L.name);
        Geo g;
        memset(&g, 0, sizeof(g));
        g.n = n;
        g.h[0] = h;
        g.w[0] = w;
        if (prec == NRV_PREC_F32) {
            using T = float;
            Bwd<T> b{net, s, g, nullptr, {}, {}};
            return b.dgrad_up(l, TView<const T>{(const T*)dy, L.cout}, TView<const T>{(const T*)mask, L.cin},
                              TView<T>{(T*)dx, L.cin}, 0);
        }
        if (prec != NRV_PREC_BF16) return fail(NRV_ERR_UNSUPPORTED, "data gradients in F32 or BF16");
        using T = __nv_bfloat16;
        const size_t rows = (size_t)n * h;
        auto al = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
        const size_t bg = al(4 * rows * w * L.cout * 2), bm = al(rows * w * L.cin * 2),
                     bo = al(rows * w * L.cin * 2);
        NRV_TRY(net->layer_ws.ensure(bg + bm + bo));
        char* ws = (char*)net->layer_ws.p;
        T *pg = (T*)ws, *pm = (T*)(ws + bg), *po = (T*)(ws + bg + bm);
        NRV_TRY(relayout(dy, pg, 2 * rows, 2 * w, L.cout, 2, true, s));
        NRV_TRY(relayout(mask, pm, rows, w, L.cin, 2, true, s));
        Bwd<T> b{net, s, g, nullptr, {}, {}};
        NRV_TRY(b.dgrad_up(l, TView<const T>{pg, L.cout, 1}, TView<const T>{pm, L.cin, 1},
                           TView<T>{po, L.cin, 1}, 0));
        return relayout(po, dx, rows, w, L.cin, 2, false, s);
    }
    if (L.kind != CONV3 || l == L_E0A)
        return fail(NRV_ERR_ARG, "layer %s has no data gradient here", L.name);
    Geo g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.h[0] = h;
    g.w[0] = w;
    if (prec == NRV_PREC_F32) {
        using T = float;
        Bwd<T> b{net, s, g, nullptr, {}, {}};
        return b.dgrad_conv(l, TView<const T>{(const T*)dy, L.cout}, TView<T>{(T*)dx, L.cin},
                            TView<const T>{(const T*)mask, mask ? L.cin : 0}, 0);
    }
    if (prec != NRV_PREC_BF16) return fail(NRV_ERR_UNSUPPORTED, "data gradients in F32 or BF16");
    using T = __nv_bfloat16;
    const size_t rows = (size_t)n * h;
    auto al = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
    const size_t bg = al(rows * w * L.cout * 2), bm = mask ? al(rows * w * L.cin * 2) : 0,
                 bo = al(rows * w * L.cin * 2);
    NRV_TRY(net->layer_ws.ensure(bg + bm + bo));
    char* ws = (char*)net->layer_ws.p;
    T *pg = (T*)ws, *pm = mask ? (T*)(ws + bg) : nullptr, *po = (T*)(ws + bg + bm);
    NRV_TRY(relayout(dy, pg, rows, w, L.cout, 2, true, s));
    if (mask) NRV_TRY(relayout(mask, pm, rows, w, L.cin, 2, true, s));
    Bwd<T> b{net, s, g, nullptr, {}, {}};
    NRV_TRY(b.dgrad_conv(l, TView<const T>{pg, L.cout, 1}, TView<T>{po, L.cin, 1},
                         TView<const T>{pm, mask ? L.cin : 0, mask ? 1 : 0}, 0));
    return relayout(po, dx, rows, w, L.cin, 2, false, s);
}

nrv_status net_backward(Net* net, const float* drgb, float* dparams, cudaStream_t s) {
    if (!net->saved) return fail(NRV_ERR_STATE, "backward without a preceding training forward");
    const Geo& g = net->geo;
    const size_t es = elem_size(net->act_prec);
    size_t off[9], tot = 0;
    const int chans[4] = {32, 64, 128, 128};
    for (int l = 0; l < 4; ++l) {
        off[2 * l] = tot;
        tot += (g.px(l) * chans[l] * es + 1023) / 1024 * 1024;
        off[2 * l + 1] = tot;
        tot += (g.px(l) * chans[l] * es + 1023) / 1024 * 1024;
    }
    NRV_TRY(net->grads.ensure(tot));
    if (net->act_prec == NRV_PREC_F32) {
        Bwd<float> b{net, s, g, dparams, {}, {}};
        for (int l = 0; l < 4; ++l) {
            b.W1[l] = (float*)((char*)net->grads.p + off[2 * l]);
            b.W2[l] = (float*)((char*)net->grads.p + off[2 * l + 1]);
        }
        return b.run(drgb, (const float*)net->saved_in);
    }
    if (net->act_prec == NRV_PREC_BF16) {
        Bwd<__nv_bfloat16> b{net, s, g, dparams, {}, {}};
        for (int l = 0; l < 4; ++l) {
            b.W1[l] = (__nv_bfloat16*)((char*)net->grads.p + off[2 * l]);
            b.W2[l] = (__nv_bfloat16*)((char*)net->grads.p + off[2 * l + 1]);
        }
        return b.run(drgb, (const __nv_bfloat16*)net->saved_in);
    }
    return fail(NRV_ERR_UNSUPPORTED, "backward is available for FP32 and BF16 only");
}

}  // namespace nrv
