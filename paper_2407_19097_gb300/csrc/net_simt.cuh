// SIMT kernels of the post-processing U-Net (Sec. 3.3): the FP32 form of the
// network, and the small memory-bound layers (pooling, transposed conv, head)
// of every precision.  Tensors are views {ptr, channels, layout} in NHWC or in
// the row-planar layout of the tensor-core path (see TView); storage is float
// or bfloat16, arithmetic always FP32 with FMA.
#pragma once
#include "internal.h"

namespace nrv {

template <typename T> __device__ __forceinline__ float ld1(const T* p);
template <> __device__ __forceinline__ float ld1<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld1<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <typename T> __device__ __forceinline__ T cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// 8 consecutive channels (16-byte aligned for bf16, 32-byte for float).
template <typename T> __device__ __forceinline__ void ld8(const T* p, float* v);
template <> __device__ __forceinline__ void ld8<float>(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <> __device__ __forceinline__ void ld8<__nv_bfloat16>(const __nv_bfloat16* p, float* v) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
    }
}
template <typename T> __device__ __forceinline__ void st8(T* p, const float* v);
template <> __device__ __forceinline__ void st8<float>(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}
template <> __device__ __forceinline__ void st8<__nv_bfloat16>(__nv_bfloat16* p, const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// A tensor of `ld` channels per pixel, rows of w pixels (w passed per access).
//  planar == 0: NHWC, element (row, x, c) at (row * w + x) * ld + c;
//  planar == 1: row-planar, the layout of the BF16 / FP8 activations of the
//     tensor-core path: each image row holds its channels as ld / ce planes of
//     w pixels x 16 bytes (ce = 16 / sizeof(T) channels per plane), so element
//     (row, x, c) sits at ((row * (ld / ce) + c / ce) * w + x) * ce + c % ce.
// Accesses of 8 channels start at a multiple of 8, inside one plane.
// coff: the view starts at channel coff of the tensor (a channel range of a wider tensor,
// e.g. the skip half of a concatenation's gradient).
template <typename T>
struct TView {
    T* p;
    int ld;          // channels per pixel of the underlying tensor
    int planar = 0;
    int coff = 0;
    __device__ __forceinline__ T* at(size_t row, int x, int c, int w) const {
        c += coff;
        if (!planar) return p + (row * (size_t)w + x) * ld + c;
        constexpr int ce = 16 / (int)sizeof(T);
        return p + ((row * (size_t)(ld / ce) + c / ce) * w + x) * ce + c % ce;
    }
};

// ---------------------------------------------------------------- 3x3 conv
// y[q][o] = bias[o] + sum_{tap,c} w[tap][c][o] * x[q + tap][c]  (zero padding),
// x = concat(x1[:c1], x2[:c2]); then ReLU (relu != 0), then multiplied by
// (mask[q][o] > 0) when mask is given (used by the backward data pass).
// One thread = one pixel x 16 output channels; the block's weights sit in
// shared memory as [9][cin][16].
template <typename T>
struct Conv3Args {
    TView<const T> x1, x2;
    int c1, c2;
    const float* w;       // [9][cin][cout]
    const float* bias;    // may be null
    TView<T> y;
    int cout;
    int n, h, w_;
    int relu;
    TView<const T> mask;  // p may be null
};

template <typename T>
__global__ void __launch_bounds__(128) conv3_simt_kernel(Conv3Args<T> a) {
    extern __shared__ float ws[];
    const int cin = a.c1 + a.c2;
    const int og = blockIdx.y * 16;
    for (int i = threadIdx.x; i < 9 * cin * 16; i += blockDim.x) {
        const int j = i & 15, tc = i >> 4;
        ws[i] = a.w[(size_t)tc * a.cout + og + j];
    }
    __syncthreads();
    const size_t npx = (size_t)a.n * a.h * a.w_;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npx) return;
    const int x = (int)(q % a.w_);
    const int y = (int)((q / a.w_) % a.h);
    const size_t img = q / ((size_t)a.w_ * a.h);
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = a.bias ? a.bias[og + j] : 0.0f;
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        if (yy < 0 || yy >= a.h || xx < 0 || xx >= a.w_) continue;
        const size_t rr = img * a.h + yy;
        const float* wt = ws + (size_t)tap * cin * 16;
        for (int c = 0; c < cin; c += 8) {
            float v[8];
            if (c < a.c1) ld8<T>(a.x1.at(rr, xx, c, a.w_), v);
            else ld8<T>(a.x2.at(rr, xx, c - a.c1, a.w_), v);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4* w4 = reinterpret_cast<const float4*>(wt + (c + k) * 16);
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) {
                    const float4 wv = w4[j4];
                    acc[4 * j4 + 0] = fmaf(v[k], wv.x, acc[4 * j4 + 0]);
                    acc[4 * j4 + 1] = fmaf(v[k], wv.y, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(v[k], wv.z, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(v[k], wv.w, acc[4 * j4 + 3]);
                }
            }
        }
    }
    if (a.relu) {
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = fmaxf(acc[j], 0.0f);
    }
    const size_t row = img * a.h + y;
    if (a.mask.p) {
        float m[16];
        ld8<T>(a.mask.at(row, x, og, a.w_), m);
        ld8<T>(a.mask.at(row, x, og + 8, a.w_), m + 8);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = m[j] > 0.0f ? acc[j] : 0.0f;
    }
    st8<T>(a.y.at(row, x, og, a.w_), acc);
    st8<T>(a.y.at(row, x, og + 8, a.w_), acc + 8);
}

// ---------------------------------------------------------------- 2x2 average pool
// Threads walk the channel groups fastest for NHWC and the pixels fastest for
// row-planar tensors, so neighbouring threads touch neighbouring bytes.
template <typename T>
__global__ void pool2_kernel(TView<const T> x, TView<T> y, int c, int n, int ho, int wo) {
    const int ng = c / 8;
    const size_t total = (size_t)n * ho * wo * ng;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int cg, xo;
        size_t row;   // output row img * ho + yo
        if (y.planar) {
            xo = (int)(i % wo);
            cg = (int)((i / wo) % ng) * 8;
            row = i / ((size_t)wo * ng);
        } else {
            cg = (int)(i % ng) * 8;
            xo = (int)((i / ng) % wo);
            row = i / ((size_t)ng * wo);
        }
        const int yo = (int)(row % ho);
        const size_t img = row / ho;
        const int wi = 2 * wo;
        const size_t r0 = img * 2 * ho + 2 * yo;
        float a[8], b[8], cc[8], d[8], r[8];
        ld8<T>(x.at(r0, 2 * xo, cg, wi), a);
        ld8<T>(x.at(r0, 2 * xo + 1, cg, wi), b);
        ld8<T>(x.at(r0 + 1, 2 * xo, cg, wi), cc);
        ld8<T>(x.at(r0 + 1, 2 * xo + 1, cg, wi), d);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = 0.25f * ((a[k] + b[k]) + (cc[k] + d[k]));
        st8<T>(y.at(row, xo, cg, wo), r);
    }
}

// ---------------------------------------------------------------- 2x2 stride-2 transposed conv
// y[2i+a][2j+b][o] = bias[o] + sum_c x[i][j][c] * w[a][b][c][o]; weights [2][2][cin][cout].
// One thread = one output pixel x 16 channels; used forward (with bias) and,
// with weights [2][2][cout][cin] and a mask, never -- the backward data pass
// of this layer has its own kernel below.
template <typename T>
__global__ void __launch_bounds__(128) upconv2_kernel(TView<const T> x, int cin, const float* w,
                                                      const float* bias, TView<T> y, int cout,
                                                      int n, int hi, int wi) {
    extern __shared__ float ws[];
    const int og = blockIdx.y * 16;
    for (int i = threadIdx.x; i < 4 * cin * 16; i += blockDim.x) {
        const int j = i & 15, tc = i >> 4;
        ws[i] = w[(size_t)tc * cout + og + j];
    }
    __syncthreads();
    const int ho = 2 * hi, wo = 2 * wi;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)n * ho * wo) return;
    const int X = (int)(q % wo), Y = (int)((q / wo) % ho);
    const size_t img = q / ((size_t)wo * ho);
    const size_t ri = img * hi + Y / 2;
    const float* wt = ws + (size_t)((Y & 1) * 2 + (X & 1)) * cin * 16;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = bias[og + j];
    for (int c = 0; c < cin; c += 8) {
        float v[8];
        ld8<T>(x.at(ri, X / 2, c, wi), v);
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(v[k], wt[(c + k) * 16 + j], acc[j]);
    }
    const size_t ro = img * ho + Y;
    st8<T>(y.at(ro, X, og, wo), acc);
    st8<T>(y.at(ro, X, og + 8, wo), acc + 8);
}

// Backward data pass of the transposed conv, masked by (xin > 0) (the input was
// a ReLU output): gx[i][j][c] = (sum_{a,b,o} g[2i+a][2j+b][o] w[a][b][c][o]) * (xin>0).
// Weights in shared memory as [2][2][16 c][cout] for the block's c group.
template <typename T>
__global__ void __launch_bounds__(128) upconv2_dgrad_kernel(TView<const T> g, int cout,
                                                            const float* w, int cin,
                                                            TView<const T> xin, TView<T> gx,
                                                            int n, int hi, int wi) {
    extern __shared__ float ws[];
    const int cg = blockIdx.y * 16;
    for (int i = threadIdx.x; i < 4 * 16 * cout; i += blockDim.x) {
        const int o = i % cout, k = (i / cout) % 16, ab = i / (16 * cout);
        ws[i] = w[((size_t)ab * cin + cg + k) * cout + o];
    }
    __syncthreads();
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)n * hi * wi) return;
    const int X = (int)(q % wi), Y = (int)((q / wi) % hi);
    const size_t img = q / ((size_t)wi * hi);
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
    for (int ab = 0; ab < 4; ++ab) {
        const size_t ro = img * 2 * hi + 2 * Y + (ab >> 1);
        const int xo = 2 * X + (ab & 1);
        const float* wt = ws + (size_t)ab * 16 * cout;
        for (int o = 0; o < cout; o += 8) {
            float v[8];
            ld8<T>(g.at(ro, xo, o, 2 * wi), v);
#pragma unroll
            for (int m = 0; m < 8; ++m)
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] = fmaf(v[m], wt[k * cout + o + m], acc[k]);
        }
    }
    const size_t ri = img * hi + Y;
    float mk[16];
    ld8<T>(xin.at(ri, X, cg, wi), mk);
    ld8<T>(xin.at(ri, X, cg + 8, wi), mk + 8);
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = mk[k] > 0.0f ? acc[k] : 0.0f;
    st8<T>(gx.at(ri, X, cg, wi), acc);
    st8<T>(gx.at(ri, X, cg + 8, wi), acc + 8);
}

// ---------------------------------------------------------------- 1x1 head -> RGB (cropped)
template <typename T>
__global__ void head_kernel(TView<const T> x, const float* w, const float* bias, float* rgb,
                            int n, int hn, int wn, int h, int wd, RgbTab tab) {
    const size_t total = (size_t)n * h * wd;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % wd), Y = (int)((i / wd) % h);
        const size_t img = i / ((size_t)wd * h);
        const size_t r = img * hn + Y;
        float v[16];
        ld8<T>(x.at(r, X, 0, wn), v);
        ld8<T>(x.at(r, X, 8, wn), v + 8);
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float s = bias[o];
#pragma unroll
            for (int c = 0; c < 16; ++c) s = fmaf(w[o * 16 + c], v[c], s);
            rgb_image(rgb, tab, img, (size_t)h * wd)[3 * ((size_t)Y * wd + X) + o] = s;
        }
    }
}

}  // namespace nrv
