// Tensor-core 3x3 convolution of the U-Net (Sec. 3.3) as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05 + TMEM), BF16 operands, FP32 accumulation.
//
//   D[m][n] = sum_k A[m][k] * B[n][k],   m = 128 consecutive pixels of one row,
//   n = output channel, k = (tap, input channel) -- K = 9 * C_in.
//
// A tile of 128 output pixels needs the input rows y-1..y+1 and pixels
// x0-1..x0+128 ("halo").  One 5-D TMA load brings them into shared memory as
// planes of [pixel][8 channels] (16 bytes per pixel): plane (row, chunk) holds
// 130 pixels.  Each tap's A operand is then just a shared-memory descriptor
// pointing dx pixels into the plane of row dy -- the nine taps share one copy
// of the data, zero padding comes from TMA's out-of-bounds fill.  Operands use
// the no-swizzle K-major layout: core matrices of 8 rows x 16 bytes, rows 16
// bytes apart (SBO = 128 bytes between 8-row groups), the two 8-element K
// halves of one MMA (K = 16) LBO bytes apart.
//
// The weights of the CTA's output-channel slice stay resident in shared memory
// ([k-step][half][n][8] BF16).  Warp roles: warp 0 issues TMA loads, warp 1
// owns TMEM and issues the MMAs, warps 2-5 drain the FP32 accumulator
// (tcgen05.ld), add the bias, apply ReLU and store BF16 NHWC.  Halo buffers and
// accumulators are double-buffered so loads, MMAs and the epilogue overlap
// across the CTA's pixel tiles.  Every wait is bounded: on timeout the kernel
// records STATUS_TIMEOUT in the status word, drains what it started, frees TMEM
// and returns.
#include <cuda.h>
#include <string.h>

#include "net.h"

namespace nrv {

namespace {

constexpr int HALO_W = 130;
constexpr int PLANE = HALO_W * 16;  // bytes of one (row, 8-channel chunk) plane
constexpr int MAX_KS = 80;
constexpr int TILE_M = 128;
constexpr int NTHREADS = 192;

struct TcParams {
    int n, h, w;             // level geometry
    int tiles_x, num_ptiles; // pixel tiles
    int nslices, n_slice;    // output-channel slices and their width
    int nks;                 // K-steps of 16 channels
    int nbuf;                // halo buffers (1..4)
    int cout;                // output channels (pixel stride of the output)
    int mode;                // 0: 3x3 conv + bias + ReLU; 1: 2x2 stride-2 transposed conv + bias
    int row0;                // first halo row relative to the tile's row (-1 conv, 0 transposed)
    int has_src2;
    uint32_t halo_bytes;     // bytes of one halo buffer (both sources)
    uint32_t src2_off;       // offset of source 2 planes inside a buffer
    uint32_t tx1, tx2;       // bytes delivered by each TMA load
    uint32_t w_bytes;        // bytes of one weight slice
    uint32_t w_region;       // bytes reserved for the weights (aligned)
    uint32_t idesc;
    uint32_t tmem_cols;
    const uint8_t* wpk;      // packed weights [slice][ks][half][n][16 bytes] (BF16 or E4M3)
    const float* bias;
    void* y;                 // BF16 or E4M3 NHWC output
    unsigned* status;
    int fp8;                 // E4M3 operands (kind::f8f6f4) and an E4M3 output
    float inv_out;           // FP8: 1 / scale of the output tensor
    const float* colscale;   // FP8: per GEMM column, input scale x weight scale
    uint32_t a_off[MAX_KS];  // A start offset in the halo buffer, per K-step
    uint32_t a_lbo[MAX_KS];  // A K-direction byte offset (second half), per K-step
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (about 2 s): false on timeout or when another role aborted.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                          unsigned* status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > 2000000000ull) {
            *abort_flag = 1;
            atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// UMMA shared-memory descriptor, no swizzle (sm_100 format, version 1).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_fp8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1)
    conv3_tc_kernel(const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
                    const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bars[16];
    __shared__ float bias_s[256];
    __shared__ float colscale_s[256];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t s_w = smem_u32(smem);
    const uint32_t s_halo = s_w + P.w_region;
    const uint32_t b_w = smem_u32(&bars[0]);
    auto b_hfull = [&](int i) { return smem_u32(&bars[1 + i]); };
    auto b_hempty = [&](int i) { return smem_u32(&bars[5 + i]); };
    auto b_afull = [&](int i) { return smem_u32(&bars[9 + i]); };
    auto b_aempty = [&](int i) { return smem_u32(&bars[11 + i]); };
    const uint32_t b_done = smem_u32(&bars[13]);

    // this CTA's output-channel slice and its pixel tiles
    const int slice = blockIdx.x % P.nslices;
    const int cta_in_slice = blockIdx.x / P.nslices;
    const int ctas_per_slice = gridDim.x / P.nslices;
    const int my_tiles = cta_in_slice < P.num_ptiles
                             ? (P.num_ptiles - 1 - cta_in_slice) / ctas_per_slice + 1
                             : 0;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(b_w, 1);
        for (int i = 0; i < 4; ++i) {
            mbar_init(b_hfull(i), 1);
            mbar_init(b_hempty(i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_afull(i), 1);
            mbar_init(b_aempty(i), 4);
        }
        mbar_init(b_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // per output column of this slice: its bias (column n maps to channel n mod cout)
    for (int i = threadIdx.x; i < P.n_slice; i += NTHREADS) {
        bias_s[i] = P.bias[(slice * P.n_slice + i) % P.cout];
        colscale_s[i] = P.fp8 ? P.colscale[slice * P.n_slice + i] : 1.0f;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // weights once, then the halo of every tile
            mbar_expect_tx(b_w, P.w_bytes);
            const uint8_t* src = P.wpk + (size_t)slice * P.w_bytes;
            for (uint32_t o = 0; o < P.w_bytes; o += 16384) {
                const uint32_t len = P.w_bytes - o < 16384 ? P.w_bytes - o : 16384;
                bulk_load(s_w + o, src + o, len, b_w);
            }
            int issued = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int buf = i % P.nbuf, u = i / P.nbuf;
                if (!mbar_wait(b_hempty(buf), (u & 1) ^ 1, &abort_flag, P.status)) break;
                const int pt = cta_in_slice + i * ctas_per_slice;
                const int xt = pt % P.tiles_x, rest = pt / P.tiles_x;
                const int yr = rest % P.h, img = rest / P.h;
                const uint32_t dst = s_halo + (uint32_t)buf * P.halo_bytes;
                mbar_expect_tx(b_hfull(buf), P.tx1 + P.tx2);
                tma_load_5d(dst, &tm1, 0, xt * TILE_M - 1, 0, yr + P.row0, img, b_hfull(buf));
                if (P.has_src2)
                    tma_load_5d(dst + P.src2_off, &tm2, 0, xt * TILE_M - 1, 0, yr + P.row0, img,
                                b_hfull(buf));
                issued = i + 1;
            }
            // every load issued must have landed before the CTA may exit
            for (int i = issued - P.nbuf > 0 ? issued - P.nbuf : 0; i < issued; ++i)
                mbar_wait(b_hfull(i % P.nbuf), (i / P.nbuf) & 1, &abort_flag, P.status);
            mbar_wait(b_w, 0, &abort_flag, P.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(b_w, 0, &abort_flag, P.status);
            const uint32_t b_lbo = (uint32_t)P.n_slice * 16;
            for (int i = 0; ok && i < my_tiles; ++i) {
                const int buf = i % P.nbuf, u = i / P.nbuf;
                const int ab = i & 1, ua = i >> 1;
                if (!mbar_wait(b_hfull(buf), u & 1, &abort_flag, P.status)) break;
                if (!mbar_wait(b_aempty(ab), (ua & 1) ^ 1, &abort_flag, P.status)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * P.n_slice);
                const uint32_t hb = s_halo + (uint32_t)buf * P.halo_bytes;
                for (int ks = 0; ks < P.nks; ++ks) {
                    const uint64_t a = sdesc(hb + P.a_off[ks], P.a_lbo[ks], 128);
                    const uint64_t b = sdesc(s_w + (uint32_t)ks * 2 * b_lbo, b_lbo, 128);
                    if (P.fp8) mma_fp8(d, a, b, P.idesc, ks > 0 ? 1u : 0u);
                    else mma_bf16(d, a, b, P.idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(b_hempty(buf));
                mma_commit(b_afull(ab));
            }
            // wait until every MMA issued above has completed
            mma_commit(b_done);
            mbar_wait(b_done, 0, &abort_flag, P.status);
        }
    } else {
        // epilogue: warps 2..5 own TMEM lanes 32*(warp%4) ..; one lane per warp polls
        const int q = warp & 3;
        const int m = 32 * q + lane;
        for (int i = 0; i < my_tiles; ++i) {
            const int ab = i & 1, ua = i >> 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(b_afull(ab), ua & 1, &abort_flag, P.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int pt = cta_in_slice + i * ctas_per_slice;
            const int xt = pt % P.tiles_x, rest = pt / P.tiles_x;
            const int yr = rest % P.h, img = rest / P.h;
            const int x = xt * TILE_M + m;
            for (int c0 = 0; c0 < P.n_slice; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * P.n_slice + c0), r);
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = fmaf(__uint_as_float(r[j]), colscale_s[c0 + j], bias_s[c0 + j]);
                    if (P.mode == 0) v[j] = fmaxf(v[j], 0.0f);
                }
                if (x < P.w) {
                    const int ng = slice * P.n_slice + c0;
                    size_t e;   // element offset of the 16 outputs
                    if (P.mode == 0) {
                        e = (((size_t)img * P.h + yr) * P.w + x) * P.cout + ng;
                    } else {
                        // transposed conv: column ng = (2a + b) * cout + o  ->  pixel (2y+a, 2x+b)
                        const int abi = ng / P.cout, o = ng % P.cout;
                        e = (((size_t)img * 2 * P.h + 2 * yr + (abi >> 1)) * 2 * P.w + 2 * x +
                             (abi & 1)) * P.cout + o;
                    }
                    if (P.fp8) {
                        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(
                                v[j] * P.inv_out, __NV_SATFINITE, __NV_E4M3);
                            w[j >> 2] |= (uint32_t)q << (8 * (j & 3));
                        }
                        *reinterpret_cast<uint4*>((uint8_t*)P.y + e) = make_uint4(w[0], w[1], w[2], w[3]);
                    } else {
                        uint32_t packed[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            packed[j] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        uint4* o4 = reinterpret_cast<uint4*>((__nv_bfloat16*)P.y + e);
                        o4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                        o4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_aempty(ab));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(P.tmem_cols)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// NHWC tensor [n][h][w][c] of `es`-byte elements viewed as (ce, w, c/ce, h, n),
// ce = 16 / es elements per 16-byte chunk, so that one box of
// (ce, 130, c/ce, rows, 1) lands in shared memory as [row][chunk][pixel][16 bytes].
nrv_status make_halo_map(CUtensorMap* map, const void* base, int n, int h, int w, int c, int rows,
                         int es) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(NRV_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)base & 15) != 0) return fail(NRV_ERR_ARG, "tensor base not 16-byte aligned");
    const int ce = 16 / es;
    const cuuint64_t dims[5] = {(cuuint64_t)ce, (cuuint64_t)w, (cuuint64_t)(c / ce), (cuuint64_t)h,
                                (cuuint64_t)n};
    const cuuint64_t strides[4] = {(cuuint64_t)c * es, 16, (cuuint64_t)w * c * es,
                                   (cuuint64_t)h * w * c * es};
    const cuuint32_t box[5] = {(cuuint32_t)ce, HALO_W, (cuuint32_t)(c / ce), (cuuint32_t)rows, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                     5, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NRV_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NRV_OK;
}

// One half of a K-step: one 16-byte chunk of channels (8 BF16 or 16 E4M3) of one
// tap from one source.
struct Half {
    int tap, src, chunk;  // src 0 or 1; tap < 0 marks the zero phantom
};

// Per-layer tensor-core configuration.  A 3x3 conv reads a 3-row halo and has
// K = 9 * C_in; a 2x2 stride-2 transposed conv is a plain GEMM of one input row
// (K = C_in) against all four kernel positions at once (N = 4 * C_out), and its
// epilogue scatters column (2a + b) * C_out + o to output pixel (2y + a, 2x + b).
struct TcLayerCfg {
    bool ok = false;
    int kind = CONV3;
    int c1 = 0, c2 = 0;      // channels per source (padded input width for the first layer)
    int rows = 3, row0 = -1;
    int ncols = 0;           // GEMM N (C_out, or 4 C_out)
    int n_slice = 0, nslices = 0, nks = 0;
    std::vector<Half> halves;
    size_t w_off = 0;        // byte offset of the packed weights
    uint32_t w_bytes = 0;    // per slice
    size_t cs_off = 0;       // FP8: offset (floats) of the per-column scales
};

TcLayerCfg g_cfg[2][NUM_LAYERS];   // [BF16, FP8]

// out[slice][ks][half][n][ce], ce = 8 (BF16) or 16 (E4M3).  FP8 weights are
// W * fold / s_w[n] in E4M3, fold = scale(skip) / scale(upsampled) for the second
// source of a concatenating layer, 1 otherwise.
__global__ void pack_tc_weights_kernel(const float* __restrict__ P, int64_t woff, int kind,
                                       int cin_real, int cout, int n_slice, int nslices, int nks,
                                       const int4* __restrict__ halves, int c1, int fp8,
                                       float fold, const float* __restrict__ s_w, uint8_t* out) {
    const int ce = fp8 ? 16 : 8;
    const size_t total = (size_t)nslices * nks * 2 * n_slice * ce;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % ce);
        const int nl = (int)((i / ce) % n_slice);
        const int hf = (int)((i / (ce * (size_t)n_slice)) % 2);
        const int ks = (int)((i / (2 * ce * (size_t)n_slice)) % nks);
        const int sl = (int)(i / (2 * ce * (size_t)n_slice * nks));
        const int4 h = halves[2 * ks + hf];
        const int n = sl * n_slice + nl;
        float v = 0.0f;
        if (h.x >= 0) {
            const int c = (h.y == 0 ? 0 : c1) + ce * h.z + e;
            if (c < cin_real) {
                if (kind == CONV3) v = P[woff + ((size_t)n * cin_real + c) * 9 + h.x];
                else v = P[woff + ((size_t)c * cout + n % cout) * 4 + n / cout];
                if (h.y == 1) v *= fold;
            }
        }
        if (fp8) {
            out[i] = __nv_cvt_float_to_fp8(v / s_w[n], __NV_SATFINITE, __NV_E4M3);
        } else {
            __nv_bfloat16 b = __float2bfloat16_rn(v);
            reinterpret_cast<uint16_t*>(out)[i] = *reinterpret_cast<uint16_t*>(&b);
        }
    }
}

// FP8 column scales: s_w[n] = (largest |W * fold| of column n) / 448 (1 if the column
// is zero) and colscale[n] = s_in * s_w[n], s_in the scale of the layer's input.
__global__ void fp8_column_scales_kernel(const float* __restrict__ P, int64_t woff, int kind,
                                         int cin_real, int c1_real, int cout, int ncols,
                                         float fold, float s_in, float* s_w, float* colscale) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= ncols) return;
    float amax = 0.0f;
    for (int c = 0; c < cin_real; ++c) {
        const float f = c >= c1_real ? fold : 1.0f;
        if (kind == CONV3) {
            for (int t = 0; t < 9; ++t)
                amax = fmaxf(amax, fabsf(P[woff + ((size_t)n * cin_real + c) * 9 + t] * f));
        } else {
            amax = fmaxf(amax, fabsf(P[woff + ((size_t)c * cout + n % cout) * 4 + n / cout] * f));
        }
    }
    const float sw = amax > 0.0f ? amax / 448.0f : 1.0f;
    s_w[n] = sw;
    colscale[n] = s_in * sw;
}

DevBuf g_halves[2];

}  // namespace

static int src_split(int l, int cin_padded, int* c2) {
    if (l == L_D2A || l == L_D1A || l == L_D0A) {
        *c2 = cin_padded / 2;
        return cin_padded / 2;
    }
    *c2 = 0;
    return cin_padded;
}

// Layer configurations and packed weights for one operand precision (0 BF16, 1 FP8).
static nrv_status build_cfg(Net* net, int pi, std::vector<int4>& all_halves,
                            std::vector<size_t>& hoff, size_t& wbytes_total) {
    const int ce = pi ? 16 : 8;
    size_t off = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        TcLayerCfg& c = g_cfg[pi][l];
        c = TcLayerCfg();
        const Layer& L = net->layers[l];
        if (L.kind == HEAD1) continue;
        c.kind = L.kind;
        if (L.kind == CONV3) {
            const int cinp = l == L_E0A ? (pi ? 16 : net->c0p) : L.cin;
            c.c1 = src_split(l, cinp, &c.c2);
            c.rows = 3;
            c.row0 = -1;
            c.ncols = L.cout;
            for (int tap = 0; tap < 9; ++tap)
                for (int src = 0; src < 2; ++src) {
                    const int cs = src == 0 ? c.c1 : c.c2;
                    for (int ch = 0; ch < cs / ce; ++ch) c.halves.push_back(Half{tap, src, ch});
                }
        } else {
            c.c1 = L.cin;
            c.c2 = 0;
            c.rows = 1;
            c.row0 = 0;
            c.ncols = 4 * L.cout;
            // the one "tap" reads row 0 of the halo at pixel offset +1 (tap index 1)
            for (int ch = 0; ch < L.cin / ce; ++ch) c.halves.push_back(Half{1, 0, ch});
        }
        if (c.halves.size() % 2) c.halves.push_back(Half{-1, 0, 0});
        c.nks = (int)c.halves.size() / 2;
        if (c.nks > MAX_KS) continue;
        // widest output slice whose weights fit in 80 KB
        int ns = c.ncols;
        while (ns > 16 && (size_t)c.nks * 2 * ns * 16 > 80 * 1024) ns /= 2;
        c.n_slice = ns;
        c.nslices = c.ncols / ns;
        c.w_bytes = (uint32_t)c.nks * 2 * ns * 16;
        c.w_off = off;
        off += ((size_t)c.w_bytes * c.nslices + 1023) / 1024 * 1024;
        hoff[l] = all_halves.size();
        for (const Half& h : c.halves) all_halves.push_back(make_int4(h.tap, h.src, h.chunk, 0));
        c.ok = true;
    }
    wbytes_total = off;
    return NRV_OK;
}

nrv_status tc_repack(Net* net, cudaStream_t s) {
    std::vector<int4> all_halves;
    std::vector<size_t> hoff(NUM_LAYERS, 0);
    size_t off = 0;
    NRV_TRY(build_cfg(net, 0, all_halves, hoff, off));
    if (off == 0) return NRV_OK;
    NRV_TRY(net->wbf16.ensure(off));
    NRV_TRY(g_halves[0].ensure(all_halves.size() * sizeof(int4)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(g_halves[0].p, all_halves.data(), all_halves.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const TcLayerCfg& c = g_cfg[0][l];
        if (!c.ok) continue;
        const Layer& L = net->layers[l];
        pack_tc_weights_kernel<<<64, 256, 0, s>>>(
            (const float*)net->params.p, L.woff, c.kind, L.cin, L.cout, c.n_slice, c.nslices, c.nks,
            (const int4*)g_halves[0].p + hoff[l], c.c1, 0, 1.0f, nullptr,
            (uint8_t*)net->wbf16.p + c.w_off);
        NRV_CHECK_LAUNCH();
    }
    // the host copy of the halves must stay valid until the copy ran
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));
    if (net->fp8_ready) return tc_repack_fp8(net, s);
    return NRV_OK;
}

// Activation-scale index (0 input, 1 + Act) of each layer's input (first source),
// second source and output.
void layer_scale_index(int l, int* in1, int* in2, int* out) {
    static const int t[NUM_LAYERS][3] = {
        {0, -1, 1 + A_E0A},         {1 + A_E0A, -1, 1 + A_E0B}, {1 + A_P0, -1, 1 + A_E1A},
        {1 + A_E1A, -1, 1 + A_E1B}, {1 + A_P1, -1, 1 + A_E2A},  {1 + A_E2A, -1, 1 + A_E2B},
        {1 + A_P2, -1, 1 + A_E3A},  {1 + A_E3A, -1, 1 + A_E3B}, {1 + A_E3B, -1, 1 + A_UP3},
        {1 + A_UP3, 1 + A_E2B, 1 + A_D2A}, {1 + A_D2A, -1, 1 + A_D2B}, {1 + A_D2B, -1, 1 + A_UP2},
        {1 + A_UP2, 1 + A_E1B, 1 + A_D1A}, {1 + A_D1A, -1, 1 + A_D1B}, {1 + A_D1B, -1, 1 + A_UP1},
        {1 + A_UP1, 1 + A_E0B, 1 + A_D0A}, {1 + A_D0A, -1, 1 + A_D0B}, {1 + A_D0B, -1, -1}};
    *in1 = t[l][0];
    *in2 = t[l][1];
    *out = t[l][2];
}

nrv_status tc_repack_fp8(Net* net, cudaStream_t s) {
    std::vector<int4> all_halves;
    std::vector<size_t> hoff(NUM_LAYERS, 0);
    size_t off = 0;
    NRV_TRY(build_cfg(net, 1, all_halves, hoff, off));
    size_t cs = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        TcLayerCfg& c = g_cfg[1][l];
        if (!c.ok) continue;
        c.cs_off = cs;
        cs += (size_t)c.ncols;
    }
    NRV_TRY(net->wfp8.ensure(off));
    NRV_TRY(net->wscale8.ensure(2 * cs * sizeof(float)));
    NRV_TRY(g_halves[1].ensure(all_halves.size() * sizeof(int4)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(g_halves[1].p, all_halves.data(), all_halves.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
    float* s_w = (float*)net->wscale8.p;
    float* colscale = s_w + cs;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const TcLayerCfg& c = g_cfg[1][l];
        if (!c.ok) continue;
        const Layer& L = net->layers[l];
        int in1, in2, out;
        layer_scale_index(l, &in1, &in2, &out);
        const float s_in = net->act_scale[in1];
        const float fold = in2 >= 0 ? net->act_scale[in2] / s_in : 1.0f;
        const int c1_real = c.c2 > 0 ? c.c1 : L.cin;
        fp8_column_scales_kernel<<<(c.ncols + 127) / 128, 128, 0, s>>>(
            (const float*)net->params.p, L.woff, c.kind, L.cin, c1_real, L.cout, c.ncols, fold,
            s_in, s_w + c.cs_off, colscale + c.cs_off);
        NRV_CHECK_LAUNCH();
        pack_tc_weights_kernel<<<64, 256, 0, s>>>(
            (const float*)net->params.p, L.woff, c.kind, L.cin, L.cout, c.n_slice, c.nslices, c.nks,
            (const int4*)g_halves[1].p + hoff[l], c.c1, 1, fold, s_w + c.cs_off,
            (uint8_t*)net->wfp8.p + c.w_off);
        NRV_CHECK_LAUNCH();
    }
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));
    return NRV_OK;
}

static int g_num_sms = 0;

// Launch one tensor-core layer on a level of geometry (n, H, W): a 3x3 conv
// writes [n][H][W][C_out]; a transposed conv reads level (H, W) and writes
// [n][2H][2W][C_out].  FP8: operands and output E4M3, inv_out = 1 / output scale.
static nrv_status tc_launch(const Net* net, int l, const void* x1, int c1, const void* x2, int c2,
                            void* y, int n, int H, int W, cudaStream_t s, int fp8, float inv_out) {
    const TcLayerCfg& c = g_cfg[fp8][l];
    if (!c.ok || c.c1 != c1 || c.c2 != c2) return fail(NRV_ERR_UNSUPPORTED, "layer not configured");
    if (fp8 && !net->fp8_ready) return fail(NRV_ERR_STATE, "FP8 needs activation scales");
    const Layer& L = net->layers[l];
    const int es = fp8 ? 1 : 2, ce = 16 / es;
    TcParams P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.h = H;
    P.w = W;
    P.tiles_x = (W + TILE_M - 1) / TILE_M;
    P.num_ptiles = P.tiles_x * H * n;
    P.nslices = c.nslices;
    P.n_slice = c.n_slice;
    P.nks = c.nks;
    P.cout = L.cout;
    P.mode = c.kind == CONV3 ? 0 : 1;
    P.row0 = c.row0;
    P.has_src2 = c.c2 > 0;
    const uint32_t nch1 = c.c1 / ce, nch2 = c.c2 / ce;
    P.tx1 = c.rows * nch1 * PLANE;
    P.tx2 = c.rows * nch2 * PLANE;
    P.src2_off = (P.tx1 + 127) / 128 * 128;   // TMA destinations are 128-byte aligned
    P.halo_bytes = (P.src2_off + P.tx2 + 127) / 128 * 128;
    P.w_bytes = c.w_bytes;
    P.w_region = (c.w_bytes + 1023) / 1024 * 1024;
    // halo stages: as many as fit (up to 4) while the CTA stays under ~110 KB, at least 1
    int nbuf = 4;
    while (nbuf > 1 && P.w_region + nbuf * P.halo_bytes > 110 * 1024) --nbuf;
    P.nbuf = nbuf;
    const uint32_t smem = P.w_region + P.nbuf * P.halo_bytes;
    if (smem > 220 * 1024) return fail(NRV_ERR_UNSUPPORTED, "tile does not fit in shared memory");
    // instruction descriptor: FP32 accumulator; A/B BF16 (kind::f16) or E4M3 (kind::f8f6f4)
    const uint32_t ab_fmt = fp8 ? 0u : 1u;
    P.idesc = (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(c.n_slice >> 3) << 17) |
              ((uint32_t)(TILE_M >> 4) << 24);
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * c.n_slice)) cols *= 2;
    P.tmem_cols = cols;
    P.wpk = (const uint8_t*)(fp8 ? net->wfp8.p : net->wbf16.p) + c.w_off;
    P.bias = (const float*)net->params.p + L.boff;
    P.y = y;
    P.fp8 = fp8;
    P.inv_out = inv_out;
    if (fp8) {
        size_t cs_total = net->wscale8.bytes / (2 * sizeof(float));
        P.colscale = (const float*)net->wscale8.p + cs_total + c.cs_off;
    }
    P.status = status_word();
    if (!P.status) return fail(NRV_ERR_CUDA, "status word unavailable");
    for (int ks = 0; ks < c.nks; ++ks) {
        const Half& h0 = c.halves[2 * ks];
        const Half& h1 = c.halves[2 * ks + 1];
        auto off = [&](const Half& h) -> uint32_t {
            const uint32_t base = h.src == 0 ? 0u : P.src2_off;
            const uint32_t nch = h.src == 0 ? nch1 : nch2;
            const uint32_t row = c.kind == CONV3 ? (uint32_t)(h.tap / 3) : 0u;
            return base + (row * nch + (uint32_t)h.chunk) * PLANE + (uint32_t)(h.tap % 3) * 16;
        };
        P.a_off[ks] = off(h0);
        const uint32_t o1 = h1.tap < 0 ? P.a_off[ks] : off(h1);
        if (o1 < P.a_off[ks]) return fail(NRV_ERR_UNSUPPORTED, "descending K layout");
        P.a_lbo[ks] = o1 - P.a_off[ks];
        // both K halves read 128 rows of 16 bytes inside the buffer
        if (o1 + TILE_M * 16 > P.halo_bytes || P.a_lbo[ks] >= (1u << 18))
            return fail(NRV_ERR_UNSUPPORTED, "A operand outside the halo buffer");
    }
    CUtensorMap m1, m2;
    NRV_TRY(make_halo_map(&m1, x1, n, H, W, c.c1, c.rows, es));
    if (P.has_src2) NRV_TRY(make_halo_map(&m2, x2, n, H, W, c.c2, c.rows, es));
    else m2 = m1;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    static bool attr_set = false;
    if (!attr_set) {
        NRV_CHECK_CUDA(cudaFuncSetAttribute(conv3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            220 * 1024));
        attr_set = true;
    }
    // resident CTAs per SM from registers, threads, shared memory and TMEM columns
    static cudaFuncAttributes fa;
    static cudaDeviceProp prop;
    static bool have_fa = false;
    if (!have_fa) {
        NRV_CHECK_CUDA(cudaFuncGetAttributes(&fa, conv3_tc_kernel));
        int dev = 0;
        NRV_CHECK_CUDA(cudaGetDevice(&dev));
        NRV_CHECK_CUDA(cudaGetDeviceProperties(&prop, dev));
        have_fa = true;
    }
    const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int occ = prop.regsPerMultiprocessor / (regs_per_warp * (NTHREADS / 32));
    occ = occ < prop.maxThreadsPerMultiProcessor / NTHREADS ? occ : prop.maxThreadsPerMultiProcessor / NTHREADS;
    const size_t smem_cta = smem + fa.sharedSizeBytes + prop.reservedSharedMemPerBlock;
    const int by_smem = (int)(prop.sharedMemPerMultiprocessor / smem_cta);
    occ = occ < by_smem ? occ : by_smem;
    occ = occ < prop.maxBlocksPerMultiProcessor ? occ : prop.maxBlocksPerMultiProcessor;
    if (occ * (int)cols > 512) occ = 512 / (int)cols;
    if (occ < 1) occ = 1;
    int per_slice = (g_num_sms * occ) / c.nslices;
    if (per_slice < 1) per_slice = 1;
    if (per_slice > P.num_ptiles) per_slice = P.num_ptiles;
    conv3_tc_kernel<<<per_slice * c.nslices, NTHREADS, smem, s>>>(m1, m2, P);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

nrv_status tc_conv3(const Net* net, int l, const void* x1, int c1, const void* x2, int c2, void* y,
                    const Geo& g, int level, nrv_prec prec, cudaStream_t s, float inv_out) {
    if (prec != NRV_PREC_BF16 && prec != NRV_PREC_FP8)
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core path is BF16 or FP8");
    if (net->layers[l].kind != CONV3) return fail(NRV_ERR_UNSUPPORTED, "not a 3x3 conv");
    return tc_launch(net, l, x1, c1, x2, c2, y, g.n, g.h[level], g.w[level], s,
                     prec == NRV_PREC_FP8, inv_out);
}

nrv_status tc_upconv(const Net* net, int l, const void* x, void* y, const Geo& g, int level_in,
                     nrv_prec prec, cudaStream_t s, float inv_out) {
    if (prec != NRV_PREC_BF16 && prec != NRV_PREC_FP8)
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core path is BF16 or FP8");
    if (net->layers[l].kind != UPCONV2) return fail(NRV_ERR_UNSUPPORTED, "not a transposed conv");
    return tc_launch(net, l, x, net->layers[l].cin, nullptr, 0, y, g.n, g.h[level_in],
                     g.w[level_in], s, prec == NRV_PREC_FP8, inv_out);
}

}  // namespace nrv
