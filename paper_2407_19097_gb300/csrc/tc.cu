// Tensor-core 3x3 convolution of the U-Net (Sec. 3.3) as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05 + TMEM), BF16 or E4M3 operands, FP32
// accumulation.
//
//   D[m][n] = sum_k A[m][k] * B[n][k],   m = output pixel of a row tile,
//   n = output channel, k = (tap, input channel) -- K = 9 * C_in.
//
// Activations are stored row-planar: each image row holds its channels as
// planes of W pixels x 16 bytes (8 BF16 or 16 E4M3 channels per plane).  One
// 4-D TMA load (box: 128 pixels x all planes of one row) brings an input row
// into a shared-memory slot as planes of 128 pixels; every plane is one
// contiguous 2 KB run in global memory.  A tile makes 126 output pixels
// x0..x0+125 from the 128 loaded pixels x0-1..x0+126 of the rows y-1, y, y+1;
// each tap's A operand is a shared-memory descriptor pointing dx pixels into
// the plane of its row, so the nine taps share one copy of the data and zero
// padding comes from TMA's out-of-bounds fill.  The MMA still computes 128
// rows; rows 126 and 127 read past their plane (into slack) and are dropped.
//
// Each CTA walks a contiguous run of tiles down the image rows of one tile
// column, so input rows sit in a ring of slots: a tile loads only the one row
// it adds, and a slot is released (by tcgen05.commit) once the following tile
// no longer reads it.  Operands use the no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes, rows 16 bytes apart (SBO = 128 bytes between
// 8-row groups), the two 16-byte K halves of one MMA LBO bytes apart -- both
// halves always come from the same row slot.
//
// The weights of the CTA's output-channel slice stay resident in shared memory
// ([k-step][half][n][16 bytes]).  Warp roles: warp 0 issues TMA loads, warps 1
// and 6 issue the MMAs (alternate K-steps into two partial accumulators where
// TMEM allows; warp 1 owns the allocation), warps 2-5 drain the FP32
// accumulators (tcgen05.ld), add the partials, scale, add the bias, apply ReLU
// (or a data gradient's ReLU mask) and store row-planar output -- and, where
// asked, the 2x2 average pool of that output or the 1x1 head on it.
// Accumulators are double-buffered.  The loader reads activations only after
// griddepcontrol.wait (programmatic dependent launch: the setup and the weight
// load overlap the previous kernel).  The MMA issue loop is kept free of
// branches and of dependent parameter loads (the operand kind is a template
// parameter, the per-K-step descriptor words sit in shared memory and are read
// one step ahead): with narrow N the issuing thread, not the tensor pipe, sets
// the pace.  Every wait is bounded: on timeout the
// kernel records STATUS_TIMEOUT in the status word, waits (bounded) for its
// own copies in flight, frees TMEM and returns.
//
// The data gradient of the 2x2 stride-2 transposed conv (mode 2) is a GEMM of one input
// row's pixels (M) against K = (a, b, C_out): each "row load" is four 5-D TMA boxes of the
// output gradient at output row 2y + a and pixel parity b (dense [plane][pixel][16 bytes]
// tiles, K-major like any input row), the weights W[c][o][a][b] resident as B, and the
// epilogue of mode 0 (mask, no bias, no ReLU).
//
// The 2x2 stride-2 transposed conv runs through the same kernel as a GEMM of
// one input row (K = C_in, tiles of 128 pixels, no halo) against all four
// kernel positions at once (N = 4 C_out); its epilogue scatters column
// (2a + b) * C_out + o to output pixel (2y + a, 2x + b), both pixel parities of an
// 8-channel chunk together.
//
// Row streaming (the STREAM instantiations; every forward 3x3 conv): the tile walk above
// becomes a stream of input rows.  The weights of the slice's three kernel rows sit side by
// side as B (N = 3 * n_slice, columns [row 2 | row 1 | row 0]), each input row is multiplied
// once (K = 3 taps * C_in) into three consecutive blocks of a ring of TMEM blocks (output row
// q in block q mod nb; an MMA whose blocks straddle the ring's end is split in two), the
// epilogue zeroes each block after draining it, and input rows are committed in groups (one
// commit per group releases the group's slots to the loader and hands its final output rows
// to the epilogue).  One MMA issuer; two groups of four epilogue warps (warps 2-5 and 6-9)
// take alternate groups and drain two output rows at a time, 8 channels per step, with the
// fused 2x2 pool computed from the even/odd pair in registers.
#include <cuda.h>
#include <string.h>

#include <algorithm>

#include "net.h"
#include "tcgen05.cuh"

namespace nrv {

namespace {

constexpr int PLANE = 2048;   // bytes of one (row, 16-byte channel chunk) plane: 128 pixels
constexpr int MAX_KS = 80;
constexpr int MAX_SLOTS = 16;
constexpr int MAX_ACC = 4;      // accumulator buffers in TMEM (a power of two)
constexpr int TILE_M = 128;
constexpr int NTHREADS = 224;   // producer, MMA issuer, 4 epilogue warps, second MMA issuer
constexpr int NTHREADS_S = 320; // row streaming: producer, MMA issuer, two groups of 4 epilogue warps

struct TcParams {
    int n, h, w;             // input level geometry
    int tile_w;              // output pixels per tile row (126 conv, 128 transposed conv)
    int rpt;                 // image rows per tile (1 or 2): a tile is rpt rows of tile_w pixels
    int hr;                  // tile rows per tile column: ceil(h / rpt)
    int xoff;                // first loaded pixel relative to the tile's first pixel
    int tiles_x, ntiles;     // tile columns per image row, tiles per slice (n * tiles_x * hr)
    int ctas_per_slice;
    int nslices, n_slice;    // output-channel slices and their width
    int nks;                 // K-steps (two 16-byte halves each)
    int rows, row0;          // input rows per tile, first one relative to the tile's row
    int nslot;               // row slots in the ring
    int nissue;              // MMA issuers (1 or 2): issuer i takes the K-steps ks = i (mod nissue)
                             // into its own partial accumulator, the epilogue adds them
    int nacc, acc_shift;     // accumulator buffers in TMEM (2 or 4) and log2 of that: tile i uses
                             // buffer i mod nacc, so the issuers run up to nacc tiles ahead
    int cout;                // output channels
    int out_nch;             // 16-byte planes per output row
    int mode;                // 0: 3x3 conv (+ bias, ReLU); 1: 2x2 stride-2 transposed conv + bias;
                             // 2: data gradient of the transposed conv (stored like mode 0)
    int parity_plane0;       // mode 2: first plane of the output gradient's channels
    uint32_t ab_bytes;       // mode 2: bytes of one (a, b) block of a row slot
    int relu;                // mode 0: apply ReLU (forward); 0 for the data gradient
    int has_src2;
    uint32_t slot_bytes;     // bytes of one row slot (both sources, plus read slack)
    uint32_t src2_off;       // offset of source 2 planes inside a slot
    uint32_t tx_bytes;       // bytes one row load delivers (both sources)
    uint32_t w_bytes;        // bytes of one weight slice
    uint32_t w_region;       // bytes reserved for the weights (aligned)
    uint32_t idesc;
    uint32_t tmem_cols;
    const uint8_t* wpk;      // packed weights [slice][ks][half][n][16 bytes] (BF16 or E4M3)
    const float* bias;       // null: no bias (the data gradient)
    int gated;               // gated conv: columns in groups of 32 -- 16 feature columns, then
                             // the 16 gate columns of the same output channels; the output is
                             // ELU(feature + bias) * sigmoid(gate + bias2), C_out = N / 2
    const float* bias2;      // gated: the gate convolution's bias
    const uint8_t* mask;     // null, or a row-planar BF16 tensor shaped like the output: outputs
                             // where it is not positive are zeroed (ReLU of the layer below)
    void* y;                 // BF16 or E4M3 row-planar output
    unsigned* status;
    int fp8;                 // E4M3 operands (kind::f8f6f4) and an E4M3 output
    float inv_out;           // FP8: 1 / scale of the output tensor
    const float* colscale;   // FP8: per GEMM column, input scale x weight scale
    // optional 1x1 head on the stored outputs of a 16-channel conv (one slice):
    // rgb[img][y][x][o] = head_b[o] + sum_c head_w[o][c] * stored_c (as read back,
    // E4M3 codes times head_s), for y < rgb_h, x < rgb_w; store_y 0 skips the store
    const float* head_w;
    const float* head_b;
    float* rgb;
    RgbTab rgb_tab;
    int rgb_h, rgb_w;
    float head_s;
    int store_y;
    // optional 2x2 average pool of the stored output (mode 0, even h and w, two rows per
    // tile): row-planar [n][h/2][out_nch][w/2][16 bytes]
    void* pool_y;            // (BF16 only)
    uint32_t stash_off;      // pool: shared-memory copy of the tile's even row as stored,
                             // [16-byte word][128 lanes][16 bytes], after the ring
    // Row streaming (mode 0): the weights of the three kernel rows side by side as B,
    // N = 3 n_slice, columns [kernel row 2 | row 1 | row 0]; each input row is multiplied
    // once and its products land in the TMEM blocks of the output rows above, at and below
    // it.  The blocks form a ring of nb blocks of n_slice columns (output row slot q uses
    // block q mod nb), zeroed by the epilogue after it drains them, so every MMA
    // accumulates.  Input rows are committed in groups of grp; the issuer stays at most
    // gm groups ahead of the epilogue.
    int stream;
    int nb, grp, gm;
    uint32_t idesc2, idesc1;   // instruction descriptors for N = 2 n_slice and n_slice
    // per K-step of one input row (every row of a tile has the same pattern):
    // low word of the A descriptor relative to the row's slot,
    // (offset >> 4) | (LBO >> 4) << 16; K-step ks reads row ks / (nks / rows)
    uint32_t a_lo[MAX_KS];
};

// Tile t of a slice covers pixels [xt * tile_w, +tile_w) of rows y .. y + rpt - 1 of image
// img, t = (img * tiles_x + xt) * hr + y / rpt: consecutive tiles walk down one column.
// The walker steps through a run of tiles without divisions.
struct TileWalk {
    int col, yr, y, img, xt;
    __device__ __forceinline__ void init(const TcParams& P, int t) {
        col = t / P.hr;
        yr = t - col * P.hr;
        y = yr * P.rpt;
        img = col / P.tiles_x;
        xt = col - img * P.tiles_x;
    }
    __device__ __forceinline__ void next(const TcParams& P) {
        y += P.rpt;
        if (++yr == P.hr) {
            yr = 0;
            y = 0;
            ++col;
            if (++xt == P.tiles_x) {
                xt = 0;
                ++img;
            }
        }
    }
};

// Row streaming: the output row held by each ring slot in turn.  A CTA's run of tiles splits
// into segments (one tile column each); a segment of R output rows streams R + 2 input rows,
// and its slots hold output rows y0 - 2 .. y0 + R - 1, the first two belonging to no one.
struct SlotCursor {
    int t, seg_left, y0, r, img, x;
    bool vx;
    __device__ __forceinline__ void init(int t_begin) {
        t = t_begin;
        seg_left = 0;
        y0 = r = img = x = 0;
        vx = false;
    }
    __device__ __forceinline__ void next(const TcParams& P, int t_end, int m, bool& real, int& si,
                                         int& sx, bool& sv, int& sy) {
        if (seg_left == 0) {
            const int col = t / P.hr;
            const int te = t_end < (col + 1) * P.hr ? t_end : (col + 1) * P.hr;
            y0 = (t - col * P.hr) * P.rpt;
            seg_left = (te - t) * P.rpt + 2;
            r = 0;
            img = col / P.tiles_x;
            x = (col - img * P.tiles_x) * P.tile_w + m;
            vx = m < P.tile_w && x < P.w;
            t = te;
        }
        real = r >= 2;
        si = img;
        sx = x;
        sy = y0 + r - 2;
        sv = vx && sy < P.h;
        ++r;
        --seg_left;
    }
};

// Two floats as a BF16 pair (lo in the low half), rounded to nearest; with relu, negative
// values (and -0) become +0 in the same conversion.
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t bf16x2_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Ring position (slot, phase parity of its use) advanced without divisions.
__device__ __forceinline__ void ring_next(int& slot, uint32_t& phase, int nslot) {
    if (++slot == nslot) {
        slot = 0;
        phase ^= 1u;
    }
}

// rgb of one pixel from its 16 stored channels (the 1x1 head, bias first, then
// one fused multiply-add per channel in channel order)
__device__ __forceinline__ void head_store(const TcParams& P, const float* hw, int img, int y,
                                           int x, const float* v) {
    if (y >= P.rgb_h || x >= P.rgb_w) return;
    float* out = rgb_image(P.rgb, P.rgb_tab, (size_t)img, (size_t)P.rgb_h * P.rgb_w) +
                 ((size_t)y * P.rgb_w + x) * 3;
    const float4* h4 = reinterpret_cast<const float4*>(hw);   // 16-byte aligned
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        float acc = hw[48 + o];
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            const float4 w4 = h4[o * 4 + c4];
            acc = fmaf(w4.x, v[4 * c4], acc);
            acc = fmaf(w4.y, v[4 * c4 + 1], acc);
            acc = fmaf(w4.z, v[4 * c4 + 2], acc);
            acc = fmaf(w4.w, v[4 * c4 + 3], acc);
        }
        out[o] = acc;
    }
}

template <bool FP8, bool STREAM, bool GATED>
__global__ void __launch_bounds__(STREAM ? NTHREADS_S : NTHREADS, STREAM ? 2 : 4)
    conv3_tc_kernel(const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
                    const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bars[2 * MAX_SLOTS + 2 * MAX_ACC + 2];
    // row streaming: "group k's MMAs are done" (ring of 16, k mod 16): the epilogue's signal to
    // drain the group and the loader's to reuse the slots of its rows
    __shared__ __align__(8) uint64_t bars_g[16];
    __shared__ __align__(16) float bias_s[256];
    __shared__ __align__(16) float colscale_s[256];
    __shared__ __align__(16) float head_ws[52];
    __shared__ uint32_t alo_s[MAX_KS + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t s_w = smem_u32(smem);
    const uint32_t s_ring = s_w + P.w_region;
    const uint32_t b_w = smem_u32(&bars[0]);
    auto b_hfull = [&](int i) { return smem_u32(&bars[1 + i]); };
    auto b_hempty = [&](int i) { return smem_u32(&bars[1 + MAX_SLOTS + i]); };
    auto b_afull = [&](int i) { return smem_u32(&bars[1 + 2 * MAX_SLOTS + i]); };
    auto b_aempty = [&](int i) { return smem_u32(&bars[1 + 2 * MAX_SLOTS + MAX_ACC + i]); };
    const uint32_t b_done = smem_u32(&bars[1 + 2 * MAX_SLOTS + 2 * MAX_ACC]);

    // this CTA's output-channel slice and its run of tiles
    const int slice = blockIdx.x % P.nslices;
    const int cta = blockIdx.x / P.nslices;
    const int t_begin = (int)(((long long)cta * P.ntiles) / P.ctas_per_slice);
    const int t_end = (int)(((long long)(cta + 1) * P.ntiles) / P.ctas_per_slice);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(b_w, 1);
        for (int i = 0; i < MAX_SLOTS; ++i) {
            mbar_init(b_hfull(i), 1);
            mbar_init(b_hempty(i), P.nissue);
        }
        for (int i = 0; i < MAX_ACC; ++i) {
            mbar_init(b_afull(i), P.nissue);
            mbar_init(b_aempty(i), 4);
        }
        mbar_init(b_done, P.nissue);
        if (STREAM)
            for (int i = 0; i < 16; ++i) mbar_init(smem_u32(&bars_g[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the weights (packed long before this launch; see the dependency wait below)
        mbar_expect_tx(b_w, P.w_bytes);
        const uint8_t* src = P.wpk + (size_t)slice * P.w_bytes;
        for (uint32_t o = 0; o < P.w_bytes; o += 16384) {
            const uint32_t len = P.w_bytes - o < 16384 ? P.w_bytes - o : 16384;
            bulk_load(s_w + o, src + o, len, b_w);
        }
    }
    // per output column of this slice: its bias (column n maps to channel n mod cout)
    constexpr int NT = STREAM ? NTHREADS_S : NTHREADS;
    for (int i = threadIdx.x; i < P.n_slice; i += NT) {
        const int gcol = slice * P.n_slice + i;
        if (GATED) {
            const int ch = 16 * (gcol / 32) + (gcol & 15);
            bias_s[i] = (gcol & 16) ? P.bias2[ch] : P.bias[ch];
        } else {
            bias_s[i] = P.bias ? P.bias[gcol % P.cout] : 0.0f;
        }
        colscale_s[i] = FP8 ? P.colscale[slice * P.n_slice + i] : 1.0f;
    }
    for (int i = threadIdx.x; i <= MAX_KS; i += NT) alo_s[i] = i < P.nks ? P.a_lo[i] : 0u;
    if (P.head_w && threadIdx.x < 51)
        head_ws[threadIdx.x] = threadIdx.x < 48 ? P.head_w[threadIdx.x] : P.head_b[threadIdx.x - 48];
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
    if (STREAM) {
        // row streaming accumulates into every block: start from zeros
        if (warp >= 2 && warp <= 5) {
            const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
            for (int c = 0; c < P.nb * P.n_slice; c += 16) tmem_zero16(tmem + lanes + (uint32_t)c);
            tmem_st_wait();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // Programmatic dependent launch: everything above may overlap the previous kernel
    // (it reads only weights, biases and scales, written at least two launches earlier);
    // activations are read, and outputs written, only after the previous kernel has
    // completed.  Dependents may start once every CTA has issued its last row load (after
    // this wait), so anything they read before their own wait was written at least two
    // launches back.  Both instructions do nothing for a plain launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            // each input row once per run of tiles (the weights are already on their way)
            TileWalk w;
            w.init(P, t_begin);
            int cur_col = -1, next_row = 0, nloads = 0, slot = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = t_begin; ok && t < t_end; ++t, w.next(P)) {
                if (w.col != cur_col) {
                    cur_col = w.col;
                    next_row = w.y + P.row0;
                }
                const int last = w.y + P.row0 + P.rows + P.rpt - 2;
                // 8-byte elements: pixel x starts at element 2x (16-byte aligned)
                const int xe = 2 * (w.xt * P.tile_w + P.xoff);
                for (; next_row <= last; ++next_row) {
                    if (STREAM) {
                        // load number nloads reuses the slot of input row nloads - nslot: wait
                        // until that row's group has committed
                        if (nloads >= P.nslot) {
                            const int g = (nloads - P.nslot) / P.grp;
                            if (!mbar_wait(smem_u32(&bars_g[g & 15]), (uint32_t)(g >> 4) & 1u,
                                           &abort_flag, P.status)) {
                                ok = false;
                                break;
                            }
                        }
                    } else if (!mbar_wait(b_hempty(slot), phase ^ 1u, &abort_flag, P.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = s_ring + (uint32_t)slot * P.slot_bytes;
                    mbar_expect_tx(b_hfull(slot), P.tx_bytes);
                    if (P.mode == 2) {
                        // output rows 2y + a, pixels 2x + b of the gradient: four blocks
                        for (int k = 0; k < 4; ++k)
                            tma_load_5d(dst + (uint32_t)k * P.ab_bytes, &tm1, 0, k & 1, xe >> 1,
                                        P.parity_plane0, (w.img * P.h + next_row) * 2 + (k >> 1),
                                        b_hfull(slot));
                    } else {
                        tma_load_4d(dst, &tm1, xe, 0, next_row, w.img, b_hfull(slot));
                        if (P.has_src2)
                            tma_load_4d(dst + P.src2_off, &tm2, xe, 0, next_row, w.img,
                                        b_hfull(slot));
                    }
                    ++nloads;
                    ring_next(slot, phase, P.nslot);
                }
            }
            // this CTA's inputs are all requested: the next layer may start launching
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            // every load issued must have landed before the CTA may exit: the last
            // min(nloads, nslot) loads, walking the ring backwards
            for (int q = nloads < P.nslot ? nloads : P.nslot; q > 0; --q) {
                if (slot == 0) {
                    slot = P.nslot - 1;
                    phase ^= 1u;
                } else {
                    --slot;
                }
                mbar_wait(b_hfull(slot), phase, &abort_flag, P.status, false);
            }
            mbar_wait(b_w, 0, &abort_flag, P.status, false);
        }
    } else if (warp == 1 || (!STREAM && warp == 6)) {
        const int iss = warp == 1 ? 0 : 1;   // this warp's issuer number
        if (lane == 0 && iss < P.nissue) {
            bool ok = mbar_wait(b_w, 0, &abort_flag, P.status);
            // descriptor high words: SBO = 128 bytes, version 1; B: K halves n_slice * 16 bytes apart
            const uint64_t hi = (uint64_t)((128u >> 4) | (1u << 14)) << 32;
            const uint32_t b_lbo = (uint32_t)P.n_slice * 16;
            const uint32_t b_lo0 = ((s_w >> 4) & 0x3FFFu) | ((b_lbo >> 4) << 16);
            const uint32_t b_step = (2 * b_lbo) >> 4;
            const uint32_t ring16 = s_ring >> 4, slot16 = P.slot_bytes >> 4;
            const int ks_row = P.nks / P.rows;   // K-steps per input row
            const int nis = P.nissue;
            if (STREAM) {
                // B of one row K-step: 3 n_slice rows, halves 3 n_slice * 16 bytes apart
                const uint32_t b_lbo3 = (uint32_t)P.n_slice * 48;
                const uint32_t b_lo0s = ((s_w >> 4) & 0x3FFFu) | ((b_lbo3 >> 4) << 16);
                const uint32_t b_jstep = (2 * b_lbo3) >> 4;
                const uint32_t b_n1 = (uint32_t)P.n_slice;   // n_slice rows of B, in 16 bytes
                const uint32_t ns = (uint32_t)P.n_slice;
                int slot = 0, blk = 0, gin = 0, k = 0;
                uint32_t ph = 0;
                uint32_t alo_r[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) alo_r[j] = j < ks_row ? alo_s[j] : 0u;
                // segments: runs of tiles in one tile column; a segment of R output rows
                // streams its R + 2 input rows, whose slots hold output rows y0 - 2 .. y0 + R - 1
                for (int t = t_begin; ok && t < t_end;) {
                    const int col = t / P.hr;
                    const int te = t_end < (col + 1) * P.hr ? t_end : (col + 1) * P.hr;
                    const int nrows = (te - t) * P.rpt + 2;
                    t = te;
                    for (int r = 0; r < nrows; ++r) {
                        if (gin == 0 && k >= P.gm) {
                            // the blocks this group writes were last drained in group k - gm
                            const int kk = k - P.gm;
                            if (!mbar_wait(b_aempty(kk & 3), (kk >> 2) & 1, &abort_flag, P.status)) {
                                ok = false;
                                break;
                            }
                        }
                        if (!mbar_wait(b_hfull(slot), ph, &abort_flag, P.status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = ring16 + (uint32_t)slot * slot16;
                        const uint32_t d = tmem + (uint32_t)blk * ns;
                        uint32_t b_lo = b_lo0s;
                        if (blk <= P.nb - 3 && ks_row <= 6) {
                            // short rows (the narrow layers): descriptor words from registers
#pragma unroll
                            for (int j = 0; j < 6; ++j)
                                if (j < ks_row) {
                                    const uint64_t a = hi | (uint64_t)(base + alo_r[j]);
                                    const uint64_t b = hi | (uint64_t)(b_lo0s + (uint32_t)j * b_jstep);
                                    if (FP8) mma_fp8(d, a, b, P.idesc, 1u);
                                    else mma_bf16(d, a, b, P.idesc, 1u);
                                }
                        } else if (blk <= P.nb - 3) {
                            for (int j = 0; j < ks_row; ++j, b_lo += b_jstep) {
                                const uint64_t a = hi | (uint64_t)(base + alo_s[j]);
                                if (FP8) mma_fp8(d, a, hi | (uint64_t)b_lo, P.idesc, 1u);
                                else mma_bf16(d, a, hi | (uint64_t)b_lo, P.idesc, 1u);
                            }
                        } else {
                            // the three blocks wrap around the ring: two MMAs per K-step
                            const uint32_t id_a = blk == P.nb - 2 ? P.idesc2 : P.idesc1;
                            const uint32_t id_b = blk == P.nb - 2 ? P.idesc1 : P.idesc2;
                            const uint32_t b_off = blk == P.nb - 2 ? 2 * b_n1 : b_n1;
                            for (int j = 0; j < ks_row; ++j, b_lo += b_jstep) {
                                const uint64_t a = hi | (uint64_t)(base + alo_s[j]);
                                if (FP8) {
                                    mma_fp8(d, a, hi | (uint64_t)b_lo, id_a, 1u);
                                    mma_fp8(tmem, a, hi | (uint64_t)(b_lo + b_off), id_b, 1u);
                                } else {
                                    mma_bf16(d, a, hi | (uint64_t)b_lo, id_a, 1u);
                                    mma_bf16(tmem, a, hi | (uint64_t)(b_lo + b_off), id_b, 1u);
                                }
                            }
                        }
                        ring_next(slot, ph, P.nslot);
                        if (++blk == P.nb) blk = 0;
                        if (++gin == P.grp) {
                            // the group's rows are consumed and its output rows final
                            mma_commit(smem_u32(&bars_g[k & 15]));
                            gin = 0;
                            ++k;
                        }
                    }
                }
                if (ok && gin > 0) mma_commit(smem_u32(&bars_g[k & 15]));   // the last, partial group
            } else {
            TileWalk w;
            w.init(P, t_begin);
            int cur_col = -1, next_row = 0;
            int loaded = 0, waited = 0, released = 0;   // row-load counts
            int end_slot = 0;                         // slot of load number `loaded`
            int wslot = 0, rslot = 0;
            uint32_t wphase = 0;
            for (int t = t_begin, i = 0; ok && t < t_end; ++t, ++i) {
                // the same row schedule as the loader
                if (w.col != cur_col) {
                    cur_col = w.col;
                    next_row = w.y + P.row0;
                }
                const int last = w.y + P.row0 + P.rows + P.rpt - 2;
                for (; next_row <= last; ++next_row) {
                    ++loaded;
                    if (++end_slot == P.nslot) end_slot = 0;
                }
                for (; waited < loaded; ++waited) {
                    if (!mbar_wait(b_hfull(wslot), wphase, &abort_flag, P.status)) {
                        ok = false;
                        break;
                    }
                    ring_next(wslot, wphase, P.nslot);
                }
                if (!ok) break;
                const int ab = i & (P.nacc - 1);
                if (!mbar_wait(b_aempty(ab), ((i >> P.acc_shift) & 1) ^ 1, &abort_flag, P.status))
                    break;
                tc_fence_after();
                // the tile's rows y+row0 .. y+row0+rows+rpt-2 are the last rows+rpt-1 loads;
                // image row y + r reads rows+... from slot s0 + r on
                int s0 = end_slot - (P.rows + P.rpt - 1);
                if (s0 < 0) s0 += P.nslot;
                const uint32_t b_adv = (uint32_t)nis * b_step;
                for (int r = 0; r < P.rpt; ++r) {
                    const uint32_t d =
                        tmem + (uint32_t)(((ab * P.rpt + r) * nis + iss) * P.n_slice);
                    int sr = s0 + r;
                    if (sr >= P.nslot) sr -= P.nslot;
                    // K-steps iss, iss + nis, ...: row k = ks / ks_row, position j = ks % ks_row
                    uint32_t b_lo = b_lo0 + (uint32_t)iss * b_step;
                    uint32_t base = ring16 + (uint32_t)sr * slot16;
                    int j = iss;
                    uint32_t e = alo_s[j];
                    for (int ks = iss; ks < P.nks; ks += nis) {
                        int jn = j + nis;                              // next position, read ahead
                        const bool wrap = jn >= ks_row;
                        if (wrap) jn -= ks_row;
                        const uint32_t e_next = alo_s[jn];
                        const uint64_t a = hi | (uint64_t)(base + e);
                        const uint64_t b = hi | (uint64_t)b_lo;
                        if (FP8) mma_fp8(d, a, b, P.idesc, ks >= nis ? 1u : 0u);
                        else mma_bf16(d, a, b, P.idesc, ks >= nis ? 1u : 0u);
                        if (wrap) {
                            if (++sr == P.nslot) sr = 0;
                            base = ring16 + (uint32_t)sr * slot16;
                        }
                        j = jn;
                        e = e_next;
                        b_lo += b_adv;
                    }
                }
                // release the rows the next tile of this run no longer reads
                int keep = loaded;
                TileWalk w2 = w;
                w2.next(P);
                if (t + 1 < t_end && w2.col == cur_col) {
                    const int last2 = w2.y + P.row0 + P.rows + P.rpt - 2;
                    keep = loaded + (last2 >= next_row ? last2 - next_row + 1 : 0) -
                           (P.rows + P.rpt - 1);
                }
                for (; released < keep; ++released) {
                    mma_commit(b_hempty(rslot));
                    if (++rslot == P.nslot) rslot = 0;
                }
                mma_commit(b_afull(ab));
                w = w2;
            }
            }
            // wait until every MMA issued above (by both issuers) has completed
            mma_commit(b_done);
            mbar_wait(b_done, 0, &abort_flag, P.status, false);
        }
    } else if ((warp >= 2 && warp <= 5) || (STREAM && warp >= 6 && warp <= 9)) {
        // epilogue: warps 2..5 own TMEM lanes 32*(warp%4) ..; one lane per warp polls
        const int q = warp & 3;
        const int m = 32 * q + lane;
        constexpr int ce = FP8 ? 16 : 8;   // channels per 16-byte plane
        // one output row of this thread's pixel x from the accumulator columns at tbase (and,
        // with two issuers, their partials n_slice columns on): scale, bias, activation,
        // mask, store, and the fused pool (even rows kept, odd rows pooled) and head
        auto emit_row = [&](uint32_t tbase, int img, int x, bool valid, int yy) {
            for (int c0 = 0; c0 < P.n_slice; c0 += (GATED ? 32 : 16)) {
                uint32_t v32[16];
                tmem_ld16(tbase + (uint32_t)c0, v32);
                float acc[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = __uint_as_float(v32[j]);
                if (P.nissue == 2) {
                    tmem_ld16(tbase + (uint32_t)(P.n_slice + c0), v32);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(v32[j]);
                }
                // scale (FP8: input x weight scale per column) and bias, four columns per
                // shared-memory load
                float v[16];
                const float4* b4 = reinterpret_cast<const float4*>(bias_s + c0);
                const float4* s4 = reinterpret_cast<const float4*>(colscale_s + c0);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const float4 bb = b4[q4];
                    const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
                    float sq[4] = {1.0f, 1.0f, 1.0f, 1.0f};
                    if (FP8) {
                        const float4 ss = s4[q4];
                        sq[0] = ss.x;
                        sq[1] = ss.y;
                        sq[2] = ss.z;
                        sq[3] = ss.w;
                    }
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const int j = 4 * q4 + i4;
                        v[j] = FP8 ? fmaf(acc[j], sq[i4], bq[i4]) : acc[j] + bq[i4];
                        if (P.relu) v[j] = fmaxf(v[j], 0.0f);
                    }
                }
                if (!FP8 && GATED) {
                    // ELU(feature) * sigmoid(gate): the gate columns follow the features
                    tmem_ld16(tbase + (uint32_t)(c0 + 16), v32);
                    float gte[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) gte[j] = __uint_as_float(v32[j]);
                    if (P.nissue == 2) {
                        tmem_ld16(tbase + (uint32_t)(P.n_slice + c0 + 16), v32);
#pragma unroll
                        for (int j = 0; j < 16; ++j) gte[j] += __uint_as_float(v32[j]);
                    }
                    // ELU(f) = f for f > 0, e^f - 1 otherwise; sigmoid(g) = 1 / (1 + e^-g) --
                    // with the fast exponential and quotient (relative error ~1e-6, far below
                    // the BF16 rounding of the stored result), free of branches so that the 16
                    // columns overlap
                    const float4* g4 = reinterpret_cast<const float4*>(bias_s + c0 + 16);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 gb = g4[q4];
                        const float gq[4] = {gb.x, gb.y, gb.z, gb.w};
#pragma unroll
                        for (int i4 = 0; i4 < 4; ++i4) {
                            const int j = 4 * q4 + i4;
                            const float gv = gte[j] + gq[i4];
                            const float ef = __expf(fminf(v[j], 0.0f));
                            const float f = v[j] > 0.0f ? v[j] : ef - 1.0f;
                            v[j] = __fdividef(f, 1.0f + __expf(-gv));
                        }
                    }
                }
                if (valid) {
                    const int ng = (slice * P.n_slice + c0) >> (GATED ? 1 : 0);
                    size_t row;   // output image row
                    int xo, wo, o;
                    if (P.mode != 1) {
                        row = (size_t)img * P.h + yy;
                        xo = x;
                        wo = P.w;
                        o = ng;
                    } else {
                        // transposed conv: column ng = (2a + b) * cout + o  ->  pixel (2y+a, 2x+b)
                        const int abi = ng / P.cout;
                        o = ng - abi * P.cout;
                        row = (size_t)img * 2 * P.h + 2 * yy + (abi >> 1);
                        xo = 2 * x + (abi & 1);
                        wo = 2 * P.w;
                    }
                    uint8_t* dst = (uint8_t*)P.y +
                                   ((row * P.out_nch + (size_t)(o / ce)) * wo + xo) * 16;
                    if (FP8) {
                        uint32_t wd[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const __nv_fp8_storage_t c8 = __nv_cvt_float_to_fp8(
                                v[j] * P.inv_out, __NV_SATFINITE, __NV_E4M3);
                            wd[j >> 2] |= (uint32_t)c8 << (8 * (j & 3));
                        }
                        if (P.store_y)
                            *reinterpret_cast<uint4*>(dst) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                        if (P.head_w) {
                            // the decoded codes, as a separate head kernel would read them
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                __nv_fp8_e4m3 qv;
                                qv.__x = (uint8_t)(wd[j >> 2] >> (8 * (j & 3)));
                                v[j] = float(qv) * P.head_s;
                            }
                            head_store(P, head_ws, img, yy, x, v);
                        }
                    } else {
                        if (P.mask) {
                            // the same two planes of the mask tensor
                            const size_t off = (size_t)(dst - (uint8_t*)P.y);
                            const uint4 m0 = *reinterpret_cast<const uint4*>(P.mask + off);
                            const uint4 m1 =
                                *reinterpret_cast<const uint4*>(P.mask + off + (size_t)wo * 16);
                            const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const uint32_t bits = (mw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                                // BF16 bits of a positive number: sign clear, not +0, not NaN
                                const bool pos = bits != 0u && bits < 0x7F81u;
                                if (!pos) v[j] = 0.0f;
                            }
                        }
                        uint32_t packed[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            packed[j] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        // channels o..o+7 and o+8..o+15 sit in consecutive planes
                        if (P.store_y) {
                            *reinterpret_cast<uint4*>(dst) =
                                make_uint4(packed[0], packed[1], packed[2], packed[3]);
                            *reinterpret_cast<uint4*>(dst + (size_t)wo * 16) =
                                make_uint4(packed[4], packed[5], packed[6], packed[7]);
                        }
                        if (P.pool_y && !(yy & 1)) {
                            // the even row as stored, for the pool after the odd row
                            uint4* st = reinterpret_cast<uint4*>(smem + P.stash_off) +
                                        ((c0 >> (GATED ? 1 : 0)) / 8) * TILE_M + m;
                            st[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                            st[TILE_M] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                        }
                        if (P.head_w) {
                            // the rounded BF16 values, as a separate head kernel would read them
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const __nv_bfloat162 h2 =
                                    *reinterpret_cast<const __nv_bfloat162*>(&packed[j]);
                                v[2 * j] = __low2float(h2);
                                v[2 * j + 1] = __high2float(h2);
                            }
                            head_store(P, head_ws, img, yy, x, v);
                        }
                    }
                }
                if (!FP8 && P.pool_y && (yy & 1)) {
                    // 2x2 average pool (BF16) of the tile's two rows: the even row (kept in
                    // shared memory by this thread) and this one, pixels x (this lane) and
                    // x + 1 (the next lane), as stored; the mean is rounded to BF16
                    const size_t prow = (size_t)img * (P.h >> 1) + (yy >> 1);
                    const int wp = P.w >> 1;
                    const int o = (slice * P.n_slice + c0) >> (GATED ? 1 : 0);
#pragma unroll
                    for (int h8 = 0; h8 < 16; h8 += 8) {
                        float a[8], c[8];
                        if (valid) {
                            const uint4 raw = *reinterpret_cast<const uint4*>(
                                smem + P.stash_off +
                                ((((c0 >> (GATED ? 1 : 0)) + h8) / 8) * TILE_M + m) * 16);
                            const uint32_t rw[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const __nv_bfloat162 h2 =
                                    *reinterpret_cast<const __nv_bfloat162*>(&rw[j]);
                                a[2 * j] = __low2float(h2);
                                a[2 * j + 1] = __high2float(h2);
                            }
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                c[j] = __bfloat162float(__float2bfloat16_rn(v[h8 + j]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) a[j] = c[j] = 0.0f;
                        }
                        float rr[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float b = __shfl_down_sync(0xffffffffu, a[j], 1);
                            const float d = __shfl_down_sync(0xffffffffu, c[j], 1);
                            rr[j] = 0.25f * ((a[j] + b) + (c[j] + d));
                        }
                        if (valid && !(m & 1)) {
                            uint32_t pk[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                __nv_bfloat162 h2 = __floats2bfloat162_rn(rr[2 * j], rr[2 * j + 1]);
                                pk[j] = *reinterpret_cast<uint32_t*>(&h2);
                            }
                            uint8_t* dst = (uint8_t*)P.pool_y +
                                ((prow * P.out_nch + (size_t)((o + h8) / 8)) * wp + (x >> 1)) * 16;
                            *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                    }
                }
            }
        };
        // Two consecutive output rows of this thread's pixel from two TMEM blocks (BF16, not
        // gated, row streaming): row a and row b, either absent (ra / rb false: a slot that
        // holds no output row of this CTA) -- processed together, 8 output channels (one
        // plane) at a time, so that the two rows' loads and arithmetic overlap.  With the
        // fused pool the pair is an even and the following odd row, pooled from registers.
        auto emit_pair = [&](uint32_t ta, bool ra, int imga, int xa, bool va, int ya, uint32_t tb,
                             bool rb, int imgb, int xb, bool vb, int yb) {
            // 8-output-channel chunks (one plane each); gated: features and gates of 8 channels
            const int nchunk = GATED ? P.n_slice / 16 : P.n_slice / 8;
            const int oc0 = (slice * P.n_slice) >> (GATED ? 1 : 0);   // first output channel
            const int plane0 = oc0 / 8;                                    // (BF16 planes)
            const size_t pstride = (size_t)P.w * 16;   // bytes between planes of a row
            // this pixel's 16-byte word in plane 0 of rows a and b
            uint8_t* const pya = (uint8_t*)P.y + (((size_t)imga * P.h + ya) * P.out_nch * P.w + xa) * 16;
            uint8_t* const pyb = (uint8_t*)P.y + (((size_t)imgb * P.h + yb) * P.out_nch * P.w + xb) * 16;
            const bool sa = P.store_y && ra && va, sb = P.store_y && rb && vb;
            const bool relu = P.relu != 0;
            const bool pool = P.pool_y && ra && rb;
            const bool vp = va && vb;
            float ha[3] = {0.0f, 0.0f, 0.0f}, hb[3] = {0.0f, 0.0f, 0.0f};
            if (P.head_w) {
#pragma unroll
                for (int o = 0; o < 3; ++o) ha[o] = hb[o] = head_ws[48 + o];
            }
#pragma unroll 1
            for (int ch = 0; ch < nchunk; ++ch) {
                const int cf = GATED ? (ch >> 1) * 32 + (ch & 1) * 8 : ch * 8;
                uint32_t fa[8], fb[8], ga[8], gb[8];
                if (ra) tmem_ld8_nowait(ta + (uint32_t)cf, fa);
                if (rb) tmem_ld8_nowait(tb + (uint32_t)cf, fb);
                if (GATED) {
                    if (ra) tmem_ld8_nowait(ta + (uint32_t)(cf + 16), ga);
                    if (rb) tmem_ld8_nowait(tb + (uint32_t)(cf + 16), gb);
                }
                tmem_ld_wait();
                tmem_tie8(fa);
                tmem_tie8(fb);
                if (GATED) {
                    tmem_tie8(ga);
                    tmem_tie8(gb);
                }
                const float4* b4 = reinterpret_cast<const float4*>(bias_s + cf);
                const float4 bb0 = b4[0], bb1 = b4[1];
                const float bq[8] = {bb0.x, bb0.y, bb0.z, bb0.w, bb1.x, bb1.y, bb1.z, bb1.w};
                float gq[8];
                if (GATED) {
                    const float4 g0 = b4[4], g1 = b4[5];   // the gate columns' biases, 16 on
                    gq[0] = g0.x; gq[1] = g0.y; gq[2] = g0.z; gq[3] = g0.w;
                    gq[4] = g1.x; gq[5] = g1.y; gq[6] = g1.z; gq[7] = g1.w;
                }
                // scale, bias, activation and the stored form: BF16 pairs, or E4M3 codes of
                // v / s_out (8 channels = 8 bytes, half of a 16-channel plane)
                uint32_t pa[4], pb[4];
                uint32_t qa[2] = {0u, 0u}, qb[2] = {0u, 0u};
                if (FP8) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float sc = colscale_s[cf + j];
                        float u = fmaf(__uint_as_float(fa[j]), sc, bq[j]);
                        float w = fmaf(__uint_as_float(fb[j]), sc, bq[j]);
                        if (relu) {
                            u = fmaxf(u, 0.0f);
                            w = fmaxf(w, 0.0f);
                        }
                        const uint32_t ca = __nv_cvt_float_to_fp8(u * P.inv_out, __NV_SATFINITE, __NV_E4M3);
                        const uint32_t cb = __nv_cvt_float_to_fp8(w * P.inv_out, __NV_SATFINITE, __NV_E4M3);
                        qa[j >> 2] |= ca << (8 * (j & 3));
                        qb[j >> 2] |= cb << (8 * (j & 3));
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float u0 = __uint_as_float(fa[2 * j]) + bq[2 * j];
                        float u1 = __uint_as_float(fa[2 * j + 1]) + bq[2 * j + 1];
                        float w0 = __uint_as_float(fb[2 * j]) + bq[2 * j];
                        float w1 = __uint_as_float(fb[2 * j + 1]) + bq[2 * j + 1];
                        if (GATED) {
                            // ELU(f) * sigmoid(g), as in the per-row epilogue
                            auto gate = [](float f, float g) {
                                const float e = __expf(fminf(f, 0.0f));
                                return __fdividef(f > 0.0f ? f : e - 1.0f, 1.0f + __expf(-g));
                            };
                            u0 = gate(u0, __uint_as_float(ga[2 * j]) + gq[2 * j]);
                            u1 = gate(u1, __uint_as_float(ga[2 * j + 1]) + gq[2 * j + 1]);
                            w0 = gate(w0, __uint_as_float(gb[2 * j]) + gq[2 * j]);
                            w1 = gate(w1, __uint_as_float(gb[2 * j + 1]) + gq[2 * j + 1]);
                        }
                        if (!GATED && relu) {
                            pa[j] = bf16x2_relu(u0, u1);
                            pb[j] = bf16x2_relu(w0, w1);
                        } else {
                            pa[j] = bf16x2(u0, u1);
                            pb[j] = bf16x2(w0, w1);
                        }
                    }
                }
                if (FP8) {
                    const int oc = oc0 + 8 * ch;
                    const size_t poff = (size_t)(oc / 16) * pstride + (size_t)(oc & 15);
                    if (sa) *reinterpret_cast<uint2*>(pya + poff) = make_uint2(qa[0], qa[1]);
                    if (sb) *reinterpret_cast<uint2*>(pyb + poff) = make_uint2(qb[0], qb[1]);
                } else {
                    const size_t poff = (size_t)(plane0 + ch) * pstride;
                    if (sa) *reinterpret_cast<uint4*>(pya + poff) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
                    if (sb) *reinterpret_cast<uint4*>(pyb + poff) = make_uint4(pb[0], pb[1], pb[2], pb[3]);
                }
                if (P.head_w || pool) {
                    // the values as stored (BF16-rounded, or E4M3 decoded), for the head and pool
                    float a8[8], b8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (FP8) {
                            __nv_fp8_e4m3 x8, y8;
                            x8.__x = (uint8_t)(qa[j >> 2] >> (8 * (j & 3)));
                            y8.__x = (uint8_t)(qb[j >> 2] >> (8 * (j & 3)));
                            a8[j] = float(x8) * P.head_s;
                            b8[j] = float(y8) * P.head_s;
                        } else {
                            const __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162*>(&pa[j >> 1]);
                            const __nv_bfloat162 y2 = *reinterpret_cast<const __nv_bfloat162*>(&pb[j >> 1]);
                            a8[j] = (j & 1) ? __high2float(x2) : __low2float(x2);
                            b8[j] = (j & 1) ? __high2float(y2) : __low2float(y2);
                        }
                    }
                    if (P.head_w) {
                        // the 1x1 head: channels in order, one fused multiply-add each
#pragma unroll
                        for (int o = 0; o < 3; ++o) {
                            const float4* h4 =
                                reinterpret_cast<const float4*>(head_ws + o * 16 + 8 * ch);
                            const float4 w0 = h4[0], w1 = h4[1];
                            const float wq[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                ha[o] = fmaf(wq[j], a8[j], ha[o]);
                                hb[o] = fmaf(wq[j], b8[j], hb[o]);
                            }
                        }
                    }
                    if (pool) {
                        // 2x2 average of rows a (even) and b (odd), pixels x and x + 1 (next lane)
                        float rr[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float av = vp ? a8[j] : 0.0f, cv = vp ? b8[j] : 0.0f;
                            const float bv = __shfl_down_sync(0xffffffffu, av, 1);
                            const float dv = __shfl_down_sync(0xffffffffu, cv, 1);
                            rr[j] = 0.25f * ((av + bv) + (cv + dv));
                        }
                        if (vp && !(m & 1)) {
                            uint32_t pk[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                __nv_bfloat162 h2 = __floats2bfloat162_rn(rr[2 * j], rr[2 * j + 1]);
                                pk[j] = *reinterpret_cast<uint32_t*>(&h2);
                            }
                            const int wp = P.w >> 1;
                            *reinterpret_cast<uint4*>((uint8_t*)P.pool_y +
                                ((((size_t)imga * (P.h >> 1) + (ya >> 1)) * P.out_nch + plane0 + ch) *
                                     wp + (xa >> 1)) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                    }
                }
            }
            if (P.head_w) {
                if (ra && va && ya < P.rgb_h && xa < P.rgb_w) {
                    float* out = rgb_image(P.rgb, P.rgb_tab, (size_t)imga, (size_t)P.rgb_h * P.rgb_w) +
                                 ((size_t)ya * P.rgb_w + xa) * 3;
                    out[0] = ha[0];
                    out[1] = ha[1];
                    out[2] = ha[2];
                }
                if (rb && vb && yb < P.rgb_h && xb < P.rgb_w) {
                    float* out = rgb_image(P.rgb, P.rgb_tab, (size_t)imgb, (size_t)P.rgb_h * P.rgb_w) +
                                 ((size_t)yb * P.rgb_w + xb) * 3;
                    out[0] = hb[0];
                    out[1] = hb[1];
                    out[2] = hb[2];
                }
            }
        };
        if (STREAM) {
            // the issuer's slot sequence: slot q is final once group q / grp has committed;
            // slots 0 and 1 of a segment hold the two rows above it (not its own rows)
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            int S = 0;
            for (int tt = t_begin; tt < t_end;) {
                const int col = tt / P.hr;
                const int te = t_end < (col + 1) * P.hr ? t_end : (col + 1) * P.hr;
                S += (te - tt) * P.rpt + 2;
                tt = te;
            }
            SlotCursor cur;
            cur.init(t_begin);
            // two groups of epilogue warps (2-5 and 6-9) take alternate slot groups
            const int wg = warp >= 6 ? 1 : 0;
            int blk = 0, k = 0;
            for (int q0 = 0; q0 < S; q0 += P.grp, ++k) {
                if ((k & 1) != wg) {
                    // the other warp group's slots: step the cursor and the ring past them
                    const int qe = q0 + P.grp < S ? q0 + P.grp : S;
                    for (int qq = q0; qq < qe; ++qq) {
                        bool rr = false, vv = false;
                        int ii = 0, xx = 0, yy = 0;
                        cur.next(P, t_end, m, rr, ii, xx, vv, yy);
                        if (++blk == P.nb) blk = 0;
                    }
                    continue;
                }
                int okw = 1;
                if (lane == 0)
                    okw = mbar_wait(smem_u32(&bars_g[k & 15]), (k >> 4) & 1, &abort_flag, P.status) ? 1 : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) break;
                tc_fence_after();
                const int qe = q0 + P.grp < S ? q0 + P.grp : S;
                for (int qq = q0; qq < qe; qq += 2) {
                    bool ra = false, rb = false, va = false, vb = false;
                    int ia = 0, xa = 0, ya = 0, ib = 0, xb = 0, yb = 0;
                    cur.next(P, t_end, m, ra, ia, xa, va, ya);
                    const uint32_t ta = tmem + lanes + (uint32_t)(blk * P.n_slice);
                    if (++blk == P.nb) blk = 0;
                    const bool hasb = qq + 1 < qe;
                    uint32_t tb = ta;
                    if (hasb) {
                        cur.next(P, t_end, m, rb, ib, xb, vb, yb);
                        tb = tmem + lanes + (uint32_t)(blk * P.n_slice);
                        if (++blk == P.nb) blk = 0;
                    }
                    emit_pair(ta, ra, ia, xa, va, ya, tb, rb, ib, xb, vb, yb);
                    // zero the blocks for their next output rows
                    for (int c = 0; c < P.n_slice; c += 16) tmem_zero16(ta + (uint32_t)c);
                    if (hasb)
                        for (int c = 0; c < P.n_slice; c += 16) tmem_zero16(tb + (uint32_t)c);
                }
                if (qe - q0 == P.grp) {
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_aempty(k & 3));
                }
            }
            tmem_st_wait();
        } else {
        // The 2x2 stride-2 transposed conv (BF16, one slice of all 4 C_out columns): column
        // (2a + b) C_out + o of input row y, pixel x goes to output row 2y + a, pixel 2x + b.
        // Both pixel parities of one 8-channel chunk are loaded together and stored as 32
        // contiguous bytes.
        auto emit_up = [&](uint32_t tbase, int img, int x, bool valid, int yy) {
            const size_t wo = 2 * (size_t)P.w;
#pragma unroll 1
            for (int a = 0; a < 2; ++a) {
                uint8_t* const prow =
                    (uint8_t*)P.y + ((((size_t)img * 2 * P.h + 2 * yy + a) * P.out_nch) * wo + 2 * x) * 16;
#pragma unroll 1
                for (int o8 = 0; o8 < P.cout; o8 += 8) {
                    const int c0 = 2 * a * P.cout + o8, c1 = c0 + P.cout;   // b = 0 and b = 1
                    uint32_t f0[8], f1[8];
                    tmem_ld8_nowait(tbase + (uint32_t)c0, f0);
                    tmem_ld8_nowait(tbase + (uint32_t)c1, f1);
                    tmem_ld_wait();
                    tmem_tie8(f0);
                    tmem_tie8(f1);
                    const float4* b4 = reinterpret_cast<const float4*>(bias_s + c0);
                    const float4 bb0 = b4[0], bb1 = b4[1];
                    const float bq[8] = {bb0.x, bb0.y, bb0.z, bb0.w, bb1.x, bb1.y, bb1.z, bb1.w};
                    uint32_t p0[4], p1[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float u[2], v[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int q = 2 * j + e;
                            u[e] = __uint_as_float(f0[q]);
                            v[e] = __uint_as_float(f1[q]);
                            u[e] += bq[q];
                            v[e] += bq[q];
                        }
                        p0[j] = P.relu ? bf16x2_relu(u[0], u[1]) : bf16x2(u[0], u[1]);
                        p1[j] = P.relu ? bf16x2_relu(v[0], v[1]) : bf16x2(v[0], v[1]);
                    }
                    if (valid) {
                        uint4* dst = reinterpret_cast<uint4*>(prow + (size_t)(o8 / 8) * wo * 16);
                        dst[0] = make_uint4(p0[0], p0[1], p0[2], p0[3]);
                        dst[1] = make_uint4(p1[0], p1[1], p1[2], p1[3]);
                    }
                }
            }
        };
        const bool up_fast = !FP8 && !GATED && P.mode == 1 && P.nslices == 1 && P.nissue == 1 &&
                             !P.mask &&
                             P.store_y && !P.head_w && !P.pool_y && (P.cout % 8) == 0;
        TileWalk w;
        w.init(P, t_begin);
        for (int t = t_begin, i = 0; t < t_end; ++t, ++i, w.next(P)) {
            const int ab = i & (P.nacc - 1);
            int ok = 1;
            if (lane == 0)
                ok = mbar_wait(b_afull(ab), (i >> P.acc_shift) & 1, &abort_flag, P.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int x = w.xt * P.tile_w + m;
            const bool valid_x = m < P.tile_w && x < P.w;
#pragma unroll 1
            for (int r = 0; r < P.rpt; ++r) {
                const int yy = w.y + r;
                const bool valid = valid_x && yy < P.h;
                const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) +
                                       (uint32_t)((ab * P.rpt + r) * P.nissue * P.n_slice);
                if (up_fast) emit_up(tbase, w.img, x, valid, yy);
                else emit_row(tbase, w.img, x, valid, yy);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_aempty(ab));
        }
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

// Row-planar tensor [n][h][nch][w][16 bytes] viewed as 8-byte elements
// (2w, nch, h, n): one box of (256, nch, 1, 1) is 128 pixels of every plane of
// one row and lands in shared memory as [plane][128 pixels][16 bytes].  Each
// plane is a contiguous 2 KB run in global memory.  Pixels outside [0, w) and
// rows outside [0, h) read as zero.
nrv_status make_planar_map(CUtensorMap* map, const void* base, int n, int h, int w, int nch,
                           int box_planes = 0) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(NRV_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)base & 15) != 0) return fail(NRV_ERR_ARG, "tensor base not 16-byte aligned");
    if (nch < 1 || nch > 256) return fail(NRV_ERR_UNSUPPORTED, "planes per row out of range");
    if (box_planes <= 0) box_planes = nch;
    if (box_planes > nch) return fail(NRV_ERR_UNSUPPORTED, "box wider than the tensor");
    const cuuint64_t dims[4] = {(cuuint64_t)2 * w, (cuuint64_t)nch, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t row = (cuuint64_t)w * 16;
    const cuuint64_t strides[3] = {row, row * nch, row * nch * h};
    const cuuint32_t box[4] = {2 * TILE_M, (cuuint32_t)box_planes, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
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
    int gated = 0;           // gated 3x3 conv: N = 2 C_out in groups of 16 feature + 16 gate columns
    int c1 = 0, c2 = 0;      // channels per source (padded input width for the first layer)
    int rows = 3, row0 = -1;
    int ncols = 0;           // GEMM N (C_out, or 4 C_out)
    int n_slice = 0, nslices = 0, nks = 0;
    std::vector<Half> halves;
    size_t w_off = 0;        // byte offset of the packed weights
    uint32_t w_bytes = 0;    // per slice
    size_t cs_off = 0;       // FP8: offset (floats) of the per-column scales
    int stream = 0;          // 3x3 conv run by row streaming (weights packed for it)
};

TcLayerCfg g_cfg[2][NUM_LAYERS];   // [BF16, FP8]
TcLayerCfg g_cfg_dg[NUM_LAYERS];   // BF16 data gradients of the 3x3 convs

constexpr int KIND_DGRAD = 3;    // packing of the 3x3 data-gradient weights (BF16)
constexpr int KIND_UPDGRAD = 4;  // packing of the transposed conv's data-gradient weights

// out[slice][ks][half][n][ce], ce = 8 (BF16) or 16 (E4M3).  FP8 weights are
// W * fold / s_w[n] in E4M3, fold = scale(skip) / scale(upsampled) for the second
// source of a concatenating layer, 1 otherwise.
// One packing job: a layer's weights in one operand layout.
struct PackJob {
    int64_t woff;
    int64_t woff2;           // gated: the gate weights (the feature weights at woff)
    int gated;
    int kind, cin_real, cout, n_slice, nslices, nks, c1, fp8;
    float fold;
    const float* s_w;
    const int4* halves;
    uint8_t* out;
    int stream;              // row-streaming layout: [slice][row K-step][half][3 n_slice][ce]
};

// Element i of job J (i < nslices * nks * 2 * n_slice * ce).
__device__ __forceinline__ void pack_element(const float* __restrict__ P, const PackJob& J,
                                             size_t i) {
    const int ce = J.fp8 ? 16 : 8;
    const int e = (int)(i % ce);
    int nl, hf, ks, sl;
    if (J.stream) {
        // the weights of kernel rows 2, 1, 0 side by side: column n3 = (2 - dy) * n_slice + nl
        // of row K-step j, which is K-step dy * (nks / 3) + j of the tile layout
        const int n3w = 3 * J.n_slice, ksr = J.nks / 3;
        const int n3 = (int)((i / ce) % n3w);
        hf = (int)((i / (ce * (size_t)n3w)) % 2);
        const int j = (int)((i / (2 * ce * (size_t)n3w)) % ksr);
        sl = (int)(i / (2 * ce * (size_t)n3w * ksr));
        nl = n3 % J.n_slice;
        ks = (2 - n3 / J.n_slice) * ksr + j;
    } else {
        nl = (int)((i / ce) % J.n_slice);
        hf = (int)((i / (ce * (size_t)J.n_slice)) % 2);
        ks = (int)((i / (2 * ce * (size_t)J.n_slice)) % J.nks);
        sl = (int)(i / (2 * ce * (size_t)J.n_slice * J.nks));
    }
    const int4 h = J.halves[2 * ks + hf];
    const int n = sl * J.n_slice + nl;
    float v = 0.0f;
    if (h.x >= 0) {
        const int c = (h.y == 0 ? 0 : J.c1) + ce * h.z + e;
        if (J.kind == KIND_UPDGRAD) {
            // column n = the transposed conv's input channel, K = (a b, output channel c):
            // W[n][c][a][b]
            if (c < J.cout && n < J.cin_real) v = P[J.woff + ((size_t)n * J.cout + c) * 4 + h.x];
        } else if (J.kind == KIND_DGRAD) {
            // data gradient: column n = forward input channel, K = (tap, forward output
            // channel c); the kernel flipped: W[c][n][8 - tap]
            if (c < J.cout && n < J.cin_real)
                v = P[J.woff + ((size_t)c * J.cin_real + n) * 9 + (8 - h.x)];
        } else if (c < J.cin_real) {
            if (J.kind == CONV3 && J.gated) {
                // column n: group n / 32 of 16 output channels, feature (n % 32 < 16) or gate
                const int o = 16 * (n / 32) + (n & 15);
                v = P[((n & 16) ? J.woff2 : J.woff) + ((size_t)o * J.cin_real + c) * 9 + h.x];
            } else if (J.kind == CONV3) v = P[J.woff + ((size_t)n * J.cin_real + c) * 9 + h.x];
            else v = P[J.woff + ((size_t)c * J.cout + n % J.cout) * 4 + n / J.cout];
            if (h.y == 1) v *= J.fold;
        }
    }
    if (J.fp8) {
        J.out[i] = __nv_cvt_float_to_fp8(v / J.s_w[n], __NV_SATFINITE, __NV_E4M3);
    } else {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        reinterpret_cast<uint16_t*>(J.out)[i] = *reinterpret_cast<uint16_t*>(&b);
    }
}

__device__ __forceinline__ size_t pack_count(const PackJob& J) {
    return (size_t)J.nslices * J.nks * 2 * J.n_slice * (J.fp8 ? 16 : 8);
}

__global__ void pack_tc_weights_kernel(const float* __restrict__ P, const __grid_constant__ PackJob J) {
    const size_t total = pack_count(J);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        pack_element(P, J, i);
}

// Every layer of one layout in one launch: element i belongs to the job whose range holds it.
struct PackJobs {
    int n;
    size_t start[NUM_LAYERS + 1];
    PackJob job[NUM_LAYERS];
};

__global__ void pack_tc_weights_all_kernel(const float* __restrict__ P,
                                           const __grid_constant__ PackJobs J) {
    const size_t total = J.start[J.n];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int j = 0;
        while (i >= J.start[j + 1]) ++j;
        pack_element(P, J.job[j], i - J.start[j]);
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

DevBuf g_halves[3];   // K orders of the BF16, FP8 and data-gradient weights
std::vector<int4> g_halves_host[3];   // what g_halves holds (the copy's source stays valid)

// Upload a K-order table when it differs from the device copy.  Only then does the host
// wait for the copy (the table depends on layer shapes, not on weight values).
nrv_status upload_halves(int k, const std::vector<int4>& h, cudaStream_t s) {
    if (h.size() == g_halves_host[k].size() &&
        memcmp(h.data(), g_halves_host[k].data(), h.size() * sizeof(int4)) == 0 && g_halves[k].p)
        return NRV_OK;
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));   // an earlier copy may still read the old table
    g_halves_host[k] = h;
    NRV_TRY(g_halves[k].ensure(h.size() * sizeof(int4)));
    NRV_CHECK_CUDA(cudaMemcpyAsync(g_halves[k].p, g_halves_host[k].data(), h.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
    return NRV_OK;
}

// One launch for a table of packing jobs.
nrv_status pack_all(const float* P, PackJobs& J, cudaStream_t s) {
    J.start[0] = 0;
    for (int j = 0; j < J.n; ++j)
        J.start[j + 1] = J.start[j] + (size_t)J.job[j].nslices * J.job[j].nks * 2 * J.job[j].n_slice *
                                          (J.job[j].fp8 ? 16 : 8);
    if (J.n == 0) return NRV_OK;
    size_t blocks = (J.start[J.n] + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    pack_tc_weights_all_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, J);
    NRV_CHECK_LAUNCH();
    return NRV_OK;
}

}  // namespace

// Row streaming for the 3x3 convs (on unless NRV_TC_STREAM=0, read once per process): the
// weight layout and the launch both follow it.
static bool stream_enabled() {
    static const bool on = [] {
        const char* e = getenv("NRV_TC_STREAM");
        return !(e && e[0] == '0');
    }();
    return on;
}

// A 3x3 conv slice is streamed when its three kernel rows fit in one MMA (N = 3 n_slice <= 256).
static int stream_ok(const TcLayerCfg& c) {
    return stream_enabled() && c.kind == CONV3 && c.rows == 3 && c.nks % 3 == 0 &&
           3 * c.n_slice <= 256 && c.n_slice % 16 == 0;
}

// Streamed slices are at most 32 columns wide: a ring of 8 blocks then fits in 256 TMEM
// columns and the epilogue drains two rows per group.
static int stream_slice(const TcLayerCfg& c, int ns) {
    if (stream_enabled() && c.kind == CONV3 && c.rows == 3 && c.nks % 3 == 0 && ns > 32 &&
        c.ncols % 32 == 0)
        return 32;
    return ns;
}

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
            // K order: kernel row dy, then dx, source, channel chunk; the two halves
            // of a K-step come from one input row (a zero phantom pads an odd row)
            for (int dy = 0; dy < 3; ++dy) {
                const size_t start = c.halves.size();
                for (int dx = 0; dx < 3; ++dx)
                    for (int src = 0; src < 2; ++src) {
                        const int cs = src == 0 ? c.c1 : c.c2;
                        for (int ch = 0; ch < cs / ce; ++ch)
                            c.halves.push_back(Half{3 * dy + dx, src, ch});
                    }
                if ((c.halves.size() - start) % 2) c.halves.push_back(Half{-1, 0, 0});
            }
        } else {
            c.c1 = L.cin;
            c.c2 = 0;
            c.rows = 1;
            c.row0 = 0;
            c.ncols = 4 * L.cout;
            // one input row, no halo: every chunk at tap 0
            for (int ch = 0; ch < L.cin / ce; ++ch) c.halves.push_back(Half{0, 0, ch});
            if (c.halves.size() % 2) c.halves.push_back(Half{-1, 0, 0});
        }
        c.nks = (int)c.halves.size() / 2;
        if (c.nks > MAX_KS) continue;
        // widest output slice whose weights fit in 80 KB
        int ns = c.ncols;
        while (ns > 16 && (size_t)c.nks * 2 * ns * 16 > 80 * 1024) ns /= 2;
        ns = stream_slice(c, ns);
        c.n_slice = ns;
        c.nslices = c.ncols / ns;
        c.stream = stream_ok(c);
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

// Data gradients of the 3x3 convs as 3x3 convs of the output gradient (C_out channels in)
// with the kernel flipped and transposed (C_in channels out); BF16 only.  Not for the first
// layer: the network input needs no gradient.
static nrv_status build_cfg_dgrad(Net* net, std::vector<int4>& all_halves, std::vector<size_t>& hoff,
                                  size_t& wbytes_total) {
    const int ce = 8;
    size_t off = 0;
    for (int l = 0; l < NUM_LAYERS; ++l) {
        TcLayerCfg& c = g_cfg_dg[l];
        c = TcLayerCfg();
        const Layer& L = net->layers[l];
        if (L.kind == UPCONV2 && L.cout % 16 == 0 && L.cin % 16 == 0) {
            // transposed conv: K = (a b, C_out) from the four parity blocks of a row slot
            c.kind = KIND_UPDGRAD;
            c.c1 = L.cout;
            c.c2 = 0;
            c.rows = 1;
            c.row0 = 0;
            c.ncols = L.cin;
            for (int ab = 0; ab < 4; ++ab)
                for (int ch = 0; ch < L.cout / ce; ++ch) c.halves.push_back(Half{ab, 0, ch});
            c.nks = (int)c.halves.size() / 2;
            if (c.nks > MAX_KS) continue;
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
            continue;
        }
        if (L.kind != CONV3 || l == L_E0A || L.cout % ce || L.cin % 16) continue;
        c.kind = CONV3;
        c.c1 = L.cout;
        c.c2 = 0;
        c.rows = 3;
        c.row0 = -1;
        c.ncols = L.cin;
        for (int dy = 0; dy < 3; ++dy) {
            const size_t start = c.halves.size();
            for (int dx = 0; dx < 3; ++dx)
                for (int ch = 0; ch < L.cout / ce; ++ch) c.halves.push_back(Half{3 * dy + dx, 0, ch});
            if ((c.halves.size() - start) % 2) c.halves.push_back(Half{-1, 0, 0});
        }
        c.nks = (int)c.halves.size() / 2;
        if (c.nks > MAX_KS) continue;
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

static nrv_status tc_repack_dgrad(Net* net, cudaStream_t s) {
    std::vector<int4> all_halves;
    std::vector<size_t> hoff(NUM_LAYERS, 0);
    size_t off = 0;
    NRV_TRY(build_cfg_dgrad(net, all_halves, hoff, off));
    if (off == 0) return NRV_OK;
    NRV_TRY(net->wtbf16.ensure(off));
    NRV_TRY(upload_halves(2, all_halves, s));
    PackJobs J;
    memset(&J, 0, sizeof(J));
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const TcLayerCfg& c = g_cfg_dg[l];
        if (!c.ok) continue;
        const Layer& L = net->layers[l];
        const int kind = c.kind == KIND_UPDGRAD ? KIND_UPDGRAD : KIND_DGRAD;
        J.job[J.n++] = PackJob{L.woff, 0, 0, kind, L.cin, L.cout, c.n_slice, c.nslices, c.nks, c.c1, 0,
                               1.0f, nullptr, (const int4*)g_halves[2].p + hoff[l],
                               (uint8_t*)net->wtbf16.p + c.w_off};
    }
    return pack_all((const float*)net->params.p, J, s);
}

nrv_status tc_repack(Net* net, cudaStream_t s) {
    std::vector<int4> all_halves;
    std::vector<size_t> hoff(NUM_LAYERS, 0);
    size_t off = 0;
    NRV_TRY(build_cfg(net, 0, all_halves, hoff, off));
    if (off == 0) return NRV_OK;
    NRV_TRY(net->wbf16.ensure(off));
    NRV_TRY(upload_halves(0, all_halves, s));
    PackJobs J;
    memset(&J, 0, sizeof(J));
    for (int l = 0; l < NUM_LAYERS; ++l) {
        const TcLayerCfg& c = g_cfg[0][l];
        if (!c.ok) continue;
        const Layer& L = net->layers[l];
        J.job[J.n++] = PackJob{L.woff, 0, 0, c.kind, L.cin, L.cout, c.n_slice, c.nslices, c.nks, c.c1, 0,
                               1.0f, nullptr, (const int4*)g_halves[0].p + hoff[l],
                               (uint8_t*)net->wbf16.p + c.w_off, c.stream};
    }
    NRV_TRY(pack_all((const float*)net->params.p, J, s));
    NRV_TRY(tc_repack_dgrad(net, s));
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
    NRV_TRY(upload_halves(1, all_halves, s));
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
        const PackJob job{L.woff, 0, 0, c.kind, L.cin, L.cout, c.n_slice, c.nslices, c.nks, c.c1, 1,
                          fold, s_w + c.cs_off, (const int4*)g_halves[1].p + hoff[l],
                          (uint8_t*)net->wfp8.p + c.w_off, c.stream};
        pack_tc_weights_kernel<<<64, 256, 0, s>>>((const float*)net->params.p, job);
        NRV_CHECK_LAUNCH();
    }
    return NRV_OK;
}

static int g_num_sms = 0;

// Programmatic dependent launch of the tensor-core layers, unless NRV_PDL=0.
static bool pdl_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("NRV_PDL");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

// Launch one tensor-core layer on a level of geometry (n, H, W): a 3x3 conv
// writes [n][H][W][C_out]; a transposed conv reads level (H, W) and writes
// [n][2H][2W][C_out]; all tensors row-planar.  FP8: operands and output E4M3,
// inv_out = 1 / output scale.
// c: the layer configuration; wpk: its packed weights; bias (null: none); relu; mask (null:
// none); cout: the output channels (C_out of the conv, or C_in of a data gradient).
static nrv_status tc_launch(const Net* net, const TcLayerCfg& c, const uint8_t* wpk,
                            const float* bias, int relu, const void* mask, int cout, const void* x1,
                            int c1, const void* x2, int c2, void* y, int n, int H, int W,
                            cudaStream_t s, int fp8, float inv_out, const TcHead* head = nullptr,
                            void* pool_y = nullptr, int g_ld = 0, int g_off = 0,
                            const float* bias2 = nullptr) {
    if (!c.ok || c.c1 != c1 || c.c2 != c2) return fail(NRV_ERR_UNSUPPORTED, "layer not configured");
    if (fp8 && !net->fp8_ready) return fail(NRV_ERR_STATE, "FP8 needs activation scales");
    if (n <= 0 || H <= 0 || W <= 0) return fail(NRV_ERR_ARG, "empty tensor");
    const int es = fp8 ? 1 : 2, ce = 16 / es;
    const bool conv = c.kind == CONV3;
    const bool updg = c.kind == KIND_UPDGRAD;   // mode 2
    TcParams P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.h = H;
    P.w = W;
    P.tile_w = conv ? TILE_M - 2 : TILE_M;
    P.xoff = conv ? -1 : 0;
    P.tiles_x = (W + P.tile_w - 1) / P.tile_w;
    if ((long long)P.tiles_x * H * n > 0x3FFFFFFFll) return fail(NRV_ERR_UNSUPPORTED, "too many tiles");
    P.nslices = c.nslices;
    P.n_slice = c.n_slice;
    P.nks = c.nks;
    P.rows = c.rows;
    P.row0 = c.row0;
    P.cout = cout;
    P.out_nch = cout / ce;
    P.mode = conv ? 0 : (updg ? 2 : 1);
    P.relu = relu;
    P.gated = c.gated;
    P.bias2 = bias2;
    if (c.gated && (fp8 || !bias || !bias2 || relu || mask || c.n_slice % 32))
        return fail(NRV_ERR_UNSUPPORTED, "gated conv: BF16, both biases, slices of 32 columns");
    P.mask = (const uint8_t*)mask;
    P.has_src2 = c.c2 > 0;
    const uint32_t nch1 = c.c1 / ce, nch2 = c.c2 / ce;
    P.src2_off = (nch1 * PLANE + 127) / 128 * 128;   // TMA destinations are 128-byte aligned
    P.ab_bytes = nch1 * PLANE;
    const uint32_t used = updg ? 4 * nch1 * PLANE : (nch2 ? P.src2_off + nch2 * PLANE : nch1 * PLANE);
    // slack: rows 126 and 127 of a conv tile read up to 32 bytes past their plane
    P.slot_bytes = (used + 32 + 127) / 128 * 128;
    P.tx_bytes = updg ? 4 * nch1 * PLANE : (nch1 + nch2) * PLANE;
    P.w_bytes = c.w_bytes;
    P.w_region = (c.w_bytes + 1023) / 1024 * 1024;
    // two MMA issuers where both partial accumulators of both tile buffers fit in 256
    // TMEM columns and every input row has at least two K-steps (the issue loop's read-ahead)
    // (transposed convs: one, their N is 4 C_out wide and their epilogue reads no partials)
    P.nissue = (4 * c.n_slice <= 256 && c.nks / c.rows >= 2 && c.kind != UPCONV2) ? 2 : 1;
    P.stream = c.stream && conv && !mask ? 1 : 0;
    if (P.stream) {
        // one issuer; a ring of nb blocks in 128 TMEM columns for 16-column slices (four CTAs
        // per SM), 256 otherwise; groups of grp rows, gm groups in flight, gm * grp + 2 <= nb
        P.nissue = 1;
        P.nb = 256 / c.n_slice;
        P.grp = (P.nb - 2) / 3;
        P.gm = 3;
        if (P.grp < 1) {
            P.grp = 1;
            P.gm = P.nb - 2;
        }
        if (P.nb < 4 || P.gm * P.grp + 2 > P.nb || P.gm > 3 || (P.grp & 1))
            return fail(NRV_ERR_UNSUPPORTED, "row streaming: TMEM ring");
    }
    // TMEM columns for rpt rows per tile and nacc accumulator buffers (a power of two >= 32)
    auto cols_for = [&](int rpt, int nacc) {
        uint32_t cols = 32;
        const uint32_t need =
            P.stream ? (uint32_t)(P.nb * c.n_slice) : (uint32_t)(nacc * rpt * P.nissue * c.n_slice);
        while (cols < need) cols *= 2;
        return cols;
    };
    // kernel variant: operand type, row streaming, gated epilogue (BF16 only)
    const int kv = fp8 ? 4 + P.stream : 2 * P.stream + (P.gated ? 1 : 0);
    auto kern = fp8 ? (P.stream ? conv3_tc_kernel<true, true, false>
                                : conv3_tc_kernel<true, false, false>)
                    : (P.stream ? (P.gated ? conv3_tc_kernel<false, true, true>
                                           : conv3_tc_kernel<false, true, false>)
                                : (P.gated ? conv3_tc_kernel<false, false, true>
                                           : conv3_tc_kernel<false, false, false>));
    static bool attr_set[6] = {false, false, false, false, false, false};
    if (!attr_set[kv]) {
        NRV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            220 * 1024));
        attr_set[kv] = true;
    }
    // resident CTAs per SM from registers, threads, shared memory and TMEM columns
    static cudaFuncAttributes fa_k[6];
    static cudaDeviceProp prop;
    static bool have_fa[6] = {false, false, false, false, false, false}, have_prop = false;
    if (!have_prop) {
        int dev = 0;
        NRV_CHECK_CUDA(cudaGetDevice(&dev));
        NRV_CHECK_CUDA(cudaGetDeviceProperties(&prop, dev));
        have_prop = true;
    }
    if (!have_fa[kv]) {
        NRV_CHECK_CUDA(cudaFuncGetAttributes(&fa_k[kv], kern));
        have_fa[kv] = true;
    }
    const cudaFuncAttributes& fa = fa_k[kv];
    auto occupancy = [&](uint32_t smem_dyn, uint32_t cols, bool count_tmem = true) {
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int nt = P.stream ? NTHREADS_S : NTHREADS;
        int o = prop.regsPerMultiprocessor / (regs_per_warp * (nt / 32));
        o = o < prop.maxThreadsPerMultiProcessor / nt ? o : prop.maxThreadsPerMultiProcessor / nt;
        const size_t smem_cta = smem_dyn + fa.sharedSizeBytes + prop.reservedSharedMemPerBlock;
        const int by_smem = (int)(prop.sharedMemPerMultiprocessor / smem_cta);
        o = o < by_smem ? o : by_smem;
        o = o < prop.maxBlocksPerMultiProcessor ? o : prop.maxBlocksPerMultiProcessor;
        if (count_tmem && o * (int)cols > 512) o = 512 / (int)cols;
        return o;
    };
    // Default launch shape (the tuner below may pick another): one image row per tile (two
    // when the 2x2 pool is fused, whose row pairs a tile then holds), two accumulator buffers,
    // two ring rows of read-ahead -- one where that admits more CTAs per SM (BF16) -- and then
    // as many more as keep that occupancy, within 215 KB.
    // pool: one 16-byte word per 16 stored bytes of a lane, 128 lanes
    const uint32_t stash_bytes = pool_y ? (uint32_t)(c.n_slice * es / 16) * TILE_M * 16 : 0u;
    auto smem_for = [&](int ns) { return P.w_region + (uint32_t)ns * P.slot_bytes + stash_bytes; };
    const int rpt0 = pool_y ? 2 : 1, nacc0 = 2;
    const uint32_t cols0 = cols_for(rpt0, nacc0);
    // row streaming reads each row once: two slots suffice, the rest is read-ahead
    const int min_slots = P.stream ? 2 : c.rows + rpt0;
    int nslot = min_slots + 1;
    while (nslot > min_slots - 1 && smem_for(nslot) > 215 * 1024) --nslot;
    if (nslot < min_slots || smem_for(nslot) > 215 * 1024)
        return fail(NRV_ERR_UNSUPPORTED, "tile does not fit in shared memory");
    if (!fp8 && nslot > min_slots &&
        occupancy(smem_for(min_slots), cols0) > occupancy(smem_for(nslot), cols0))
        nslot = min_slots;
    const int occ0 = occupancy(smem_for(nslot), cols0);
    while (nslot < MAX_SLOTS && smem_for(nslot + 1) <= 215 * 1024 &&
           occupancy(smem_for(nslot + 1), cols0) >= occ0)
        ++nslot;
    // instruction descriptor: FP32 accumulator; A/B BF16 (kind::f16) or E4M3 (kind::f8f6f4)
    const uint32_t ab_fmt = fp8 ? 0u : 1u;
    auto idesc_n = [&](int nn) {
        return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(nn >> 3) << 17) |
               ((uint32_t)(TILE_M >> 4) << 24);
    };
    P.idesc = idesc_n(P.stream ? 3 * c.n_slice : c.n_slice);
    P.idesc2 = idesc_n(2 * c.n_slice);
    P.idesc1 = idesc_n(c.n_slice);
    P.wpk = wpk;
    P.bias = bias;
    P.y = y;
    P.fp8 = fp8;
    P.inv_out = inv_out;
    P.store_y = 1;
    if (pool_y) {
        if (!conv || fp8 || (H & 1) || (W & 1) || mask || head)
            return fail(NRV_ERR_UNSUPPORTED, "the fused pool needs a 3x3 conv on an even grid");
        P.pool_y = pool_y;
    }
    if (head) {
        if (!conv || c.nslices != 1 || c.n_slice != (c.gated ? 32 : 16) || cout != 16 ||
            !(relu || c.gated))
            return fail(NRV_ERR_UNSUPPORTED, "the fused head needs a 16-channel conv");
        P.head_w = head->w;
        P.head_b = head->b;
        P.rgb = head->rgb;
        P.rgb_tab = head->tab;
        if (head->tab.on && n > 8) return fail(NRV_ERR_ARG, "per-image outputs for at most 8 images");
        P.rgb_h = head->h;
        P.rgb_w = head->w_px;
        P.head_s = head->scale;
        P.store_y = head->store_y ? 1 : 0;
    }
    if (fp8) {
        size_t cs_total = net->wscale8.bytes / (2 * sizeof(float));
        P.colscale = (const float*)net->wscale8.p + cs_total + c.cs_off;
    }
    P.status = status_word();
    if (!P.status) return fail(NRV_ERR_CUDA, "status word unavailable");
    if (c.nks % c.rows) return fail(NRV_ERR_UNSUPPORTED, "K-steps not a whole number per row");
    const int ks_row = c.nks / c.rows;
    for (int ks = 0; ks < c.nks; ++ks) {
        const Half& h0 = c.halves[2 * ks];
        const Half& h1 = c.halves[2 * ks + 1];
        auto rel = [&](const Half& h) -> uint32_t {
            if (updg) return (uint32_t)h.tap * P.ab_bytes + (uint32_t)h.chunk * PLANE;
            return (h.src == 0 ? 0u : P.src2_off) + (uint32_t)h.chunk * PLANE +
                   (uint32_t)(conv ? h.tap % 3 : 0) * 16;
        };
        const int dy = conv ? h0.tap / 3 : 0;
        if (h0.tap < 0 || dy != ks / ks_row || (h1.tap >= 0 && conv && h1.tap / 3 != dy))
            return fail(NRV_ERR_UNSUPPORTED, "K-step halves out of row order");
        const uint32_t o0 = rel(h0), o1 = h1.tap < 0 ? o0 : rel(h1);
        if (o1 < o0) return fail(NRV_ERR_UNSUPPORTED, "descending K layout");
        // both halves read 128 rows of 16 bytes inside the slot (with its slack)
        if (o1 + TILE_M * 16 > P.slot_bytes || (o1 - o0) >= (1u << 18))
            return fail(NRV_ERR_UNSUPPORTED, "A operand outside the row slot");
        const uint32_t word = (o0 >> 4) | (((o1 - o0) >> 4) << 16);
        if (ks < ks_row) P.a_lo[ks] = word;
        else if (P.a_lo[ks % ks_row] != word)
            return fail(NRV_ERR_UNSUPPORTED, "rows of a tile with different K patterns");
    }
    CUtensorMap m1, m2;
    if (updg) {
        // the output gradient at (2H, 2W), g_ld channels of which C_out from g_off on
        if (g_ld < (int)c.c1 || g_off < 0 || g_off % ce || g_off + c.c1 > g_ld || g_ld % ce)
            return fail(NRV_ERR_ARG, "gradient view");
        P.parity_plane0 = g_off / ce;
        NRV_TRY(tc_parity_map(&m1, x1, n * 2 * H, 2 * W, g_ld / ce, (int)nch1));
    } else {
        NRV_TRY(make_planar_map(&m1, x1, n, H, W, (int)nch1));
    }
    if (P.has_src2) NRV_TRY(make_planar_map(&m2, x2, n, H, W, (int)nch2));
    else m2 = m1;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    // One launch with rpt image rows per tile, nacc accumulator buffers, `ns` ring slots and
    // at most `cap` CTAs per SM (0: as many as fit).
    auto launch_with = [&](int rpt, int nacc, int ns, int cap) -> nrv_status {
        P.rpt = rpt;
        P.hr = (H + rpt - 1) / rpt;
        P.ntiles = P.tiles_x * P.hr * n;
        P.nacc = nacc;
        P.acc_shift = nacc == 4 ? 2 : 1;
        const uint32_t cols = cols_for(rpt, nacc);
        P.tmem_cols = cols;
        P.nslot = ns;
        uint32_t smem = smem_for(ns);
        P.stash_off = P.w_region + (uint32_t)ns * P.slot_bytes;
        int occ = occupancy(smem, cols);
        if (occ < 1) occ = 1;
        if (cap > 0 && cap < occ) occ = cap;
        // The block scheduler does not see TMEM: where registers and shared memory would admit
        // more CTAs per SM than the TMEM columns (or the cap), pad the shared memory so that it
        // does not place them (a CTA beyond the TMEM budget would stall in its allocation while
        // other SMs idle, e.g. when CTAs are placed while the previous kernel drains).
        if (occupancy(smem, cols, false) > occ) {
            const size_t per_cta = prop.sharedMemPerMultiprocessor / (size_t)(occ + 1) + 1;
            const size_t fixed = fa.sharedSizeBytes + prop.reservedSharedMemPerBlock;
            if (per_cta > fixed) {
                const uint32_t pad = (uint32_t)((per_cta - fixed + 127) / 128 * 128);
                if (pad > smem && pad <= 215 * 1024) smem = pad;
            }
        }
        int per_slice = (g_num_sms * occ) / c.nslices;
        if (per_slice < 1) per_slice = 1;
        if (per_slice > P.ntiles) per_slice = P.ntiles;
        P.ctas_per_slice = per_slice;
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(per_slice * c.nslices));
        cfg.blockDim = dim3(P.stream ? NTHREADS_S : NTHREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        NRV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, m1, m2, P));
        NRV_CHECK_LAUNCH();
        return NRV_OK;
    };
    // Tuned launch shape for this layer shape: a choice in the tuned-choice table (loaded from a
    // cache file) is used; with NRV_TC_TUNE=1 a missing one is timed on the real data at this
    // first launch unless the stream is capturing (every candidate computes the same output; the
    // chosen one runs last).  Otherwise the default shape above.  Tuning is opt-in: its timings
    // are only as good as the quiet of the GPU it runs on (a profiler's serialisation, for one,
    // misleads it), and it gains about 1% on the 1080p network.
    static const int tune_on = [] {
        const char* e = getenv("NRV_TC_TUNE");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    char key[200];
    snprintf(key, sizeof(key),
             "conv fp8=%d mode=%d c1=%d c2=%d cout=%d nks=%d slice=%dx%d pool=%d head=%d mask=%d "
             "n=%d h=%d w=%d",
             fp8, P.mode, c.c1, c.c2, cout, c.nks, c.n_slice, c.nslices, pool_y ? 1 : 0,
             head ? 1 : 0, mask ? 1 : 0, n, H, W);
    // a choice: (rpt << 20) | (nacc << 16) | (slots << 8) | cap
    auto valid_choice = [&](int v) {
        const int rpt = (v >> 20) & 15, nacc = (v >> 16) & 15, ns = (v >> 8) & 255;
        return (rpt == 1 || rpt == 2) && (!pool_y || rpt == 2) && (nacc == 2 || nacc == 4) &&
               ns >= c.rows + rpt && ns <= MAX_SLOTS && smem_for(ns) <= 215 * 1024 &&
               cols_for(rpt, nacc) <= 512;
    };
    auto launch_choice = [&](int v) {
        return launch_with((v >> 20) & 15, (v >> 16) & 15, (v >> 8) & 255, v & 255);
    };
    if (P.stream) return launch_with(rpt0, nacc0, nslot, 0);
    int choice = 0;
    if (tune_get(key, &choice) && valid_choice(choice)) return launch_choice(choice);
    if (!tune_on) return launch_with(rpt0, nacc0, nslot, 0);
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    NRV_CHECK_CUDA(cudaStreamIsCapturing(s, &capst));
    if (capst != cudaStreamCaptureStatusNone) return launch_with(rpt0, nacc0, nslot, 0);
    std::vector<int> cands;
    for (int rpt = pool_y ? 2 : 1; rpt <= 2; ++rpt)
        for (int nacc : {2, 4}) {
            const uint32_t cols = cols_for(rpt, nacc);
            if (cols > 512) continue;
            for (int ns : {c.rows + rpt, c.rows + rpt + 2, c.rows + rpt + 6, nslot, MAX_SLOTS}) {
                if (ns < c.rows + rpt || ns > MAX_SLOTS || smem_for(ns) > 215 * 1024) continue;
                const int o = occupancy(smem_for(ns), cols);
                for (int cap : {o, o - 1}) {
                    if (cap < 1 || (cap == o - 1 && o <= 1)) continue;
                    const int v = (rpt << 20) | (nacc << 16) | (ns << 8) | cap;
                    if (std::find(cands.begin(), cands.end(), v) == cands.end()) cands.push_back(v);
                }
            }
        }
    cudaEvent_t e0, e1;
    NRV_CHECK_CUDA(cudaEventCreate(&e0));
    NRV_CHECK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int arg = cands.empty() ? ((rpt0 << 20) | (nacc0 << 16) | (nslot << 8)) : cands[0];
    for (int v : cands) {
        // the fastest of three runs (the first also warms the caches)
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            float t = 0.0f;
            NRV_CHECK_CUDA(cudaEventRecord(e0, s));
            NRV_TRY(launch_choice(v));
            NRV_CHECK_CUDA(cudaEventRecord(e1, s));
            NRV_CHECK_CUDA(cudaEventSynchronize(e1));
            NRV_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (t < ms) ms = t;
        }
        if (ms < best) {
            best = ms;
            arg = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_put(key, arg);
    tune_count_timing();
    return launch_choice(arg);
}

// ------------------------------------------------------------------ layers of other networks
// The same kernel for a list of layers described by TcGeneric (the gated network): their
// configurations, their K-order tables and their BF16 weights, packed from a flat parameter
// vector in one launch.
struct TcPacked {
    std::vector<TcGeneric> spec;
    std::vector<TcLayerCfg> cfg;
    DevBuf w;        // packed BF16 weights of every layer
    DevBuf halves;   // K-order tables of every layer
};

nrv_status tc_generic_prepare(const TcGeneric* L, int n, const float* params, TcPacked** state,
                              cudaStream_t s) {
    if (n < 1 || n > NUM_LAYERS) return fail(NRV_ERR_ARG, "1..%d layers", NUM_LAYERS);
    TcPacked* st = *state;
    if (!st) *state = st = new TcPacked();
    st->spec.assign(L, L + n);
    st->cfg.assign(n, TcLayerCfg());
    std::vector<int4> all;
    std::vector<size_t> hoff(n, 0);
    size_t off = 0;
    const int ce = 8;
    for (int l = 0; l < n; ++l) {
        TcLayerCfg& c = st->cfg[l];
        c.kind = L[l].kind;
        c.gated = L[l].gated;
        c.c1 = L[l].c1;
        c.c2 = L[l].c2;
        if (c.c1 % ce || c.c2 % ce || L[l].cout % 16) return fail(NRV_ERR_UNSUPPORTED, "channel counts");
        if (c.kind == CONV3) {
            c.rows = 3;
            c.row0 = -1;
            c.ncols = (c.gated ? 2 : 1) * L[l].cout;
            // K order within a kernel row: source, channel chunk, dx -- ascending slot offsets,
            // so the two halves of every K-step are in order whatever the chunk counts
            for (int dy = 0; dy < 3; ++dy) {
                const size_t start = c.halves.size();
                for (int src = 0; src < 2; ++src)
                    for (int ch = 0; ch < (src == 0 ? c.c1 : c.c2) / ce; ++ch)
                        for (int dx = 0; dx < 3; ++dx)
                            c.halves.push_back(Half{3 * dy + dx, src, ch});
                if ((c.halves.size() - start) % 2) c.halves.push_back(Half{-1, 0, 0});
            }
        } else if (c.kind == UPCONV2 && !c.gated && c.c2 == 0) {
            c.rows = 1;
            c.row0 = 0;
            c.ncols = 4 * L[l].cout;
            for (int ch = 0; ch < c.c1 / ce; ++ch) c.halves.push_back(Half{0, 0, ch});
            if (c.halves.size() % 2) c.halves.push_back(Half{-1, 0, 0});
        } else {
            return fail(NRV_ERR_UNSUPPORTED, "layer kind");
        }
        c.nks = (int)c.halves.size() / 2;
        if (c.nks > MAX_KS) return fail(NRV_ERR_UNSUPPORTED, "K too long for resident weights");
        // widest output slice whose weights fit in 80 KB (gated: whole 32-column groups)
        const int minw = c.gated ? 32 : 16;
        int ns = c.ncols;
        while (ns > minw && (size_t)c.nks * 2 * ns * 16 > 80 * 1024) ns /= 2;
        ns = stream_slice(c, ns);
        if (c.ncols % ns || ns % minw) return fail(NRV_ERR_UNSUPPORTED, "slice width");
        c.n_slice = ns;
        c.nslices = c.ncols / ns;
        c.stream = stream_ok(c);
        c.w_bytes = (uint32_t)c.nks * 2 * ns * 16;
        c.w_off = off;
        off += ((size_t)c.w_bytes * c.nslices + 1023) / 1024 * 1024;
        hoff[l] = all.size();
        for (const Half& h : c.halves) all.push_back(make_int4(h.tap, h.src, h.chunk, 0));
        c.ok = true;
    }
    NRV_TRY(st->w.ensure(off));
    NRV_TRY(st->halves.ensure(all.size() * sizeof(int4)));
    // the tables depend on shapes only; the copy is stream-ordered before the packing
    NRV_CHECK_CUDA(cudaMemcpyAsync(st->halves.p, all.data(), all.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
    NRV_CHECK_CUDA(cudaStreamSynchronize(s));   // `all` goes out of scope
    PackJobs J;
    memset(&J, 0, sizeof(J));
    for (int l = 0; l < n; ++l) {
        const TcLayerCfg& c = st->cfg[l];
        J.job[J.n++] = PackJob{L[l].woff, L[l].woff2, L[l].gated, c.kind, L[l].cin_real, L[l].cout,
                               c.n_slice, c.nslices, c.nks, c.c1, 0, 1.0f, nullptr,
                               (const int4*)st->halves.p + hoff[l], (uint8_t*)st->w.p + c.w_off,
                               c.stream};
    }
    return pack_all(params, J, s);
}

void tc_generic_free(TcPacked* st) { delete st; }

nrv_status tc_generic_run(const TcPacked* st, int l, const float* params, const void* x1,
                          const void* x2, void* y, int n, int H, int W, cudaStream_t s,
                          const TcHead* head, void* pool_y) {
    if (!st || l < 0 || l >= (int)st->cfg.size()) return fail(NRV_ERR_ARG, "bad layer");
    const TcLayerCfg& c = st->cfg[l];
    const TcGeneric& L = st->spec[l];
    return tc_launch(nullptr, c, (const uint8_t*)st->w.p + c.w_off, params + L.boff,
                     (c.kind == CONV3 && !c.gated) ? 1 : 0, nullptr, L.cout, x1, c.c1, x2, c.c2, y,
                     n, H, W, s, 0, 1.0f, head, pool_y, 0, 0, c.gated ? params + L.boff2 : nullptr);
}

nrv_status tc_conv3(const Net* net, int l, const void* x1, int c1, const void* x2, int c2, void* y,
                    const Geo& g, int level, nrv_prec prec, cudaStream_t s, float inv_out,
                    const TcHead* head, void* pool_y) {
    if (prec != NRV_PREC_BF16 && prec != NRV_PREC_FP8_E4M3)
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core path is BF16 or FP8");
    const Layer& L = net->layers[l];
    if (L.kind != CONV3) return fail(NRV_ERR_UNSUPPORTED, "not a 3x3 conv");
    const int fp8 = prec == NRV_PREC_FP8_E4M3;
    const TcLayerCfg& c = g_cfg[fp8][l];
    const uint8_t* w = (const uint8_t*)(fp8 ? net->wfp8.p : net->wbf16.p) + c.w_off;
    return tc_launch(net, c, w, (const float*)net->params.p + L.boff, 1, nullptr, L.cout, x1, c1,
                     x2, c2, y, g.n, g.h[level], g.w[level], s, fp8, inv_out, head, pool_y);
}

nrv_status tc_dgrad(const Net* net, int l, const void* gin, void* out, const void* mask, int n, int H,
                    int W, cudaStream_t s) {
    const Layer& L = net->layers[l];
    const TcLayerCfg& c = g_cfg_dg[l];
    if (L.kind != CONV3 || !c.ok) return fail(NRV_ERR_UNSUPPORTED, "no tensor-core data gradient");
    const uint8_t* w = (const uint8_t*)net->wtbf16.p + c.w_off;
    return tc_launch(net, c, w, nullptr, 0, mask, L.cin, gin, L.cout, nullptr, 0, out, n, H, W, s, 0,
                     1.0f);
}

nrv_status tc_planar_map(CUtensorMap* map, const void* base, int n, int h, int w, int nch,
                         int box_planes) {
    return make_planar_map(map, base, n, h, w, nch, box_planes);
}

nrv_status tc_parity_map(CUtensorMap* map, const void* base, int rows, int w, int nch,
                         int box_planes) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(NRV_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)base & 15) != 0) return fail(NRV_ERR_ARG, "tensor base not 16-byte aligned");
    if ((w & 1) || nch < 1 || nch > 256 || box_planes < 1 || box_planes > nch)
        return fail(NRV_ERR_UNSUPPORTED, "parity view shape");
    // 8-byte elements: (half, parity, pixel pair, plane, row)
    const cuuint64_t dims[5] = {2, 2, (cuuint64_t)w / 2, (cuuint64_t)nch, (cuuint64_t)rows};
    const cuuint64_t row = (cuuint64_t)w * 16;
    const cuuint64_t strides[4] = {16, 32, row, row * nch};
    const cuuint32_t box[5] = {2, 1, TILE_M, (cuuint32_t)box_planes, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NRV_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NRV_OK;
}

nrv_status tc_updgrad(const Net* net, int l, const void* g, int g_ld, int g_off, const void* mask,
                      void* out, int n, int H, int W, cudaStream_t s) {
    const Layer& L = net->layers[l];
    const TcLayerCfg& c = g_cfg_dg[l];
    if (L.kind != UPCONV2 || !c.ok || c.kind != KIND_UPDGRAD)
        return fail(NRV_ERR_UNSUPPORTED, "no tensor-core data gradient");
    const uint8_t* w = (const uint8_t*)net->wtbf16.p + c.w_off;
    return tc_launch(net, c, w, nullptr, 0, mask, L.cin, g, L.cout, nullptr, 0, out, n, H, W, s, 0,
                     1.0f, nullptr, nullptr, g_ld, g_off);
}

nrv_status tc_upconv(const Net* net, int l, const void* x, void* y, const Geo& g, int level_in,
                     nrv_prec prec, cudaStream_t s, float inv_out) {
    if (prec != NRV_PREC_BF16 && prec != NRV_PREC_FP8_E4M3)
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core path is BF16 or FP8");
    const Layer& L = net->layers[l];
    if (L.kind != UPCONV2) return fail(NRV_ERR_UNSUPPORTED, "not a transposed conv");
    const int fp8 = prec == NRV_PREC_FP8_E4M3;
    const TcLayerCfg& c = g_cfg[fp8][l];
    const uint8_t* w = (const uint8_t*)(fp8 ? net->wfp8.p : net->wbf16.p) + c.w_off;
    return tc_launch(net, c, w, (const float*)net->params.p + L.boff, 0, nullptr, L.cout, x, L.cin,
                     nullptr, 0, y, g.n, g.h[level_in], g.w[level_in], s, fp8, inv_out);
}

}  // namespace nrv
