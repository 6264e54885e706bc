// Weight gradient of a 3x3 convolution on the tensor cores (the backward pass of
// Sec. 3.3's network, trained with Adam as in Sec. 4.1):
//
//   dW[o][c][tap] = sum over pixels p of  g[p][o] * x[p + shift(tap)][c]
//
// as a GEMM with M = output channel o (padded to the 128 lanes of TMEM), K = pixels and
// N = (tap, c) for a group of 16 input channels: N = 9 x 16 = 144, so one MMA of K = 16
// pixels serves all nine taps.  Both operands come straight from the row-planar BF16
// layout ([row][plane][pixel][8 channels]), which is the MN-major no-swizzle operand
// layout: a core matrix is 8 consecutive pixels (K) x 16 bytes (8 channels of M or N),
// K-adjacent core matrices 128 bytes apart (LBO), MN-adjacent ones one 2 KB plane apart
// (SBO).  A tile is 128 pixels x0..x0+127 of one row: its A block is the output gradient
// (all C_out planes), its B block nine shifted copies of the group's two input planes --
// rows y-1, y, y+1 at pixel offsets -1, 0, +1 -- loaded by TMA, so the nine taps are
// nine consecutive N blocks and zero padding is TMA's out-of-bounds fill.
//
// The 2x2 stride-2 transposed conv's weight gradient,
//
//   dW[c][o][a][b] = sum over input pixels (i, j) of  x[i][j][c] * g[2i + a][2j + b][o],
//
// runs through the same kernel with the roles turned: M = (a, b, o) -- four kernel
// positions of C_out channels, split over CTAs by a where 4 C_out > 128 -- K = input
// pixels j of one row and N = C_in.  A 5-D TMA view of the output gradient (8-byte half,
// pixel parity b, j, plane, row) loads the pixels of one parity as a dense tile, so each
// (a, b) block is again an MN-major operand; the input row is the B block.
//
// The bias gradient comes out of the same MMAs: two constant planes of BF16 ones follow
// each B block, so 16 more accumulator columns hold sum_p g[p][row].
//
// Each CTA takes a channel group and a contiguous range of tiles (a split of K), sums
// its MMAs in one TMEM accumulator and writes its partial dW; partials are added in a
// fixed order afterwards (deterministic).  Warp 0 issues TMA into two stages, warp 1
// owns TMEM and issues the MMAs, warps 2-5 read the accumulator at the end.  Waits are
// bounded: on timeout the kernel sets STATUS_TIMEOUT, drains its copies, frees TMEM and
// returns.
#include "net.h"
#include "tcgen05.cuh"

namespace nrv {

namespace {

constexpr int WG_NT = 192;           // producer, MMA issuer, 4 epilogue warps
constexpr int WG_PLANE = 2048;       // one plane of a 128-pixel tile
constexpr int WG_N = 144;            // 9 taps x 16 channels
constexpr uint32_t WG_B_BYTES = 9 * 2 * WG_PLANE;
constexpr uint32_t WG_ONES = 2 * WG_PLANE;   // two planes of ones after each B block
constexpr int WG_COLS = 256;         // TMEM columns allocated (>= WG_N)

struct WgParams {
    int mode;              // 0: 3x3 conv; 1: 2x2 stride-2 transposed conv
    int n, h, w;           // input level geometry
    int tiles_x, ntiles;   // tiles of 128 pixels: t = (img * h + y) * tiles_x + xt
    int nsplit;            // CTAs per channel group (blockIdx.x)
    int cout, cin;         // channels of the output gradient and of the whole input
    int groups1;           // channel groups that read source 1 (the rest read source 2)
    int n_ab;              // mode 1: kernel positions (a, b) per CTA (4, or 2 when split by a)
    int g_plane0;          // mode 1: first plane of the output gradient's channels
    int m_real;            // mode 1: A rows that hold data (n_ab * C_out)
    int ncols;             // weight columns of the accumulator (144, or C_in); the bias
                           // column follows
    int b_planes;          // mode 0: planes per tap loaded (2, or 1 for an 8-channel input)
    uint32_t b_bytes;      // bytes TMA brings into the B block per stage
    uint32_t b_bytes_span; // B block size in shared memory (the ones planes follow it)
    uint32_t a_bytes;      // output-gradient block of a stage (C_out / 8 planes)
    uint32_t stage_bytes;  // a_bytes + the nine input blocks
    uint32_t idesc;
    float* part;           // [split][o][tap][c] (mode 0) or [split][c][ab * C_out + o]
    float* partb;          // bias: [split][o] (mode 0) or [split][ab * C_out + o]
    unsigned* status;
};

__device__ __forceinline__ uint64_t wg_desc(uint32_t saddr) {
    // start address, LBO = 128 bytes (K), SBO = one plane (M / N), version 1, no swizzle
    const uint64_t lo = ((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16);
    const uint64_t hi = (uint64_t)((WG_PLANE >> 4) | (1u << 14));
    return lo | (hi << 32);
}

__global__ void __launch_bounds__(WG_NT, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tg, const __grid_constant__ CUtensorMap t1,
                    const __grid_constant__ CUtensorMap t2, const __grid_constant__ WgParams P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bars[5];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t s0 = smem_u32(smem);
    auto b_full = [&](int i) { return smem_u32(&bars[i]); };
    auto b_empty = [&](int i) { return smem_u32(&bars[2 + i]); };
    const uint32_t b_done = smem_u32(&bars[4]);

    const int split = blockIdx.x, grp = blockIdx.y;
    const int t_begin = (int)(((long long)split * P.ntiles) / P.nsplit);
    const int t_end = (int)(((long long)(split + 1) * P.ntiles) / P.nsplit);
    const CUtensorMap* tx = grp < P.groups1 ? &t1 : &t2;
    const int plane0 = P.b_planes * (grp < P.groups1 ? grp : grp - P.groups1);   // in its source
    const int ab0 = grp * P.n_ab;   // mode 1: first kernel position of this CTA

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_full(i), 1);
            mbar_init(b_empty(i), 1);
        }
        mbar_init(b_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    {
        // constant parts of both stages: the ones planes (BF16 1.0), and for a one-plane
        // input the unused second plane of every tap (zero)
        const uint4 one = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        for (int st = 0; st < 2; ++st) {
            uint8_t* b = smem + (size_t)st * P.stage_bytes + P.a_bytes;
            uint4* ones = reinterpret_cast<uint4*>(b + P.b_bytes_span);
            for (int i = threadIdx.x; i < (int)(WG_ONES / 16); i += WG_NT) ones[i] = one;
            if (P.mode == 0 && P.b_planes == 1)
                for (int i = threadIdx.x; i < 9 * WG_PLANE / 16; i += WG_NT) {
                    const int tap = i / (WG_PLANE / 16), r = i % (WG_PLANE / 16);
                    reinterpret_cast<uint4*>(b + (size_t)tap * 2 * WG_PLANE + WG_PLANE)[r] =
                        make_uint4(0u, 0u, 0u, 0u);
                }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(WG_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int nloads = 0;
            for (int t = t_begin, i = 0; t < t_end; ++t, ++i) {
                const int st = i & 1;
                if (!mbar_wait(b_empty(st), ((i >> 1) & 1) ^ 1u, &abort_flag, P.status)) break;
                const int xt = t % P.tiles_x;
                const int row = t / P.tiles_x;
                const int y = row % P.h, img = row / P.h;
                const int x0 = xt * 128;
                const uint32_t sa = s0 + (uint32_t)st * P.stage_bytes;
                const uint32_t sb = sa + P.a_bytes;
                mbar_expect_tx(b_full(st), P.a_bytes + P.b_bytes);
                if (P.mode == 0) {
                    tma_load_4d(sa, &tg, 2 * x0, 0, y, img, b_full(st));
                    for (int dy = 0; dy < 3; ++dy)
                        for (int dx = 0; dx < 3; ++dx)
                            tma_load_4d(sb + (uint32_t)(3 * dy + dx) * 2 * WG_PLANE, tx,
                                        2 * (x0 - 1 + dx), plane0, y + dy - 1, img, b_full(st));
                } else {
                    // kernel position (a, b): output row 2y + a, output pixels 2j + b
                    const uint32_t ab_bytes = P.a_bytes / (uint32_t)P.n_ab;
                    for (int k = 0; k < P.n_ab; ++k) {
                        const int ab = ab0 + k;
                        tma_load_5d(sa + (uint32_t)k * ab_bytes, &tg, 0, ab & 1, x0, P.g_plane0,
                                    (img * P.h + y) * 2 + (ab >> 1), b_full(st));
                    }
                    tma_load_4d(sb, &t1, 2 * x0, 0, y, img, b_full(st));
                }
                ++nloads;
            }
            // the last loads issued must land before the CTA may exit
            const int last = nloads;
            for (int i = last - 2 < 0 ? 0 : last - 2; i < last; ++i)
                mbar_wait(b_full(i & 1), (i >> 1) & 1, &abort_flag, P.status, false);
        }
    } else if (warp == 1) {
        if (lane == 0 && t_end > t_begin) {
            bool ok = true;
            for (int t = t_begin, i = 0; ok && t < t_end; ++t, ++i) {
                const int st = i & 1;
                if (!mbar_wait(b_full(st), (i >> 1) & 1, &abort_flag, P.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = s0 + (uint32_t)st * P.stage_bytes;
                const uint32_t sb = sa + P.a_bytes;
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)   // 16 pixels per K-step
                    mma_bf16(tmem, wg_desc(sa + 256u * ks), wg_desc(sb + 256u * ks), P.idesc,
                             (i > 0 || ks > 0) ? 1u : 0u);
                mma_commit(b_empty(st));
            }
            mma_commit(b_done);
            mbar_wait(b_done, 0, &abort_flag, P.status, false);
        }
    } else {
        // epilogue: TMEM lane o (warp quadrant q = warp % 4) holds dW[o][tap][16 channels]
        const int q = warp & 3;
        const int o = 32 * q + lane;
        bool ok = true;
        if (t_end > t_begin) {
            int r = 1;
            if (lane == 0) r = mbar_wait(b_done, 0, &abort_flag, P.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, r, 0) != 0;
            tc_fence_after();
        }
        if (ok && P.mode == 1 && 32 * q < P.m_real) {
            // row m = (ab - ab0) * C_out + o; column c -> part[split][c][ab * C_out + o]
            const int k4 = 4 * P.cout;
            float* dst = P.part + (size_t)split * P.cin * k4 + ab0 * P.cout + o;
            for (int c0 = 0; c0 < P.ncols; c0 += 16) {
                uint32_t v[16];
                if (t_end > t_begin) {
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0u;
                }
                if (o < P.m_real) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) dst[(size_t)(c0 + j) * k4] = __uint_as_float(v[j]);
                }
            }
            // bias column: sum of the output gradient at this row's kernel position
            uint32_t v[16];
            if (t_end > t_begin) {
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)P.ncols, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
            if (o < P.m_real) P.partb[(size_t)split * k4 + ab0 * P.cout + o] = __uint_as_float(v[0]);
        }
        if (ok && P.mode == 0 && 32 * q < P.cout) {
            float* dst = P.part + ((size_t)split * P.cout + o) * 9 * P.cin + 8 * P.b_planes * grp;
            for (int tap = 0; tap < 9; ++tap) {
                uint32_t v[16];
                if (t_end > t_begin) {
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * tap), v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0u;   // an empty split adds nothing
                }
                if (o < P.cout) {
                    // 16 channels of the group (8 with a one-plane input)
                    float4* d = reinterpret_cast<float4*>(dst + (size_t)tap * P.cin);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (j < 2 * P.b_planes) d[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                           __uint_as_float(v[4 * j + 2]),
                                           __uint_as_float(v[4 * j + 3]));
                }
            }
            if (grp == 0) {
                // bias column (every channel group computes it; the first one writes it)
                uint32_t v[16];
                if (t_end > t_begin) {
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)P.ncols, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0u;
                }
                if (o < P.cout) P.partb[(size_t)split * P.cout + o] = __uint_as_float(v[0]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(WG_COLS)
                     : "memory");
    }
}

}  // namespace

// Launch: grid (splits, groups), two stages of (A block, B block), partials in `part`.
static nrv_status wg_launch(WgParams& P, int groups, const CUtensorMap& mg, const CUtensorMap& m1,
                            const CUtensorMap& m2, size_t per_split, float* part,
                            size_t part_floats, float* partb, int* nsplit, cudaStream_t s) {
    P.status = status_word();
    if (!P.status) return fail(NRV_ERR_CUDA, "status word unavailable");
    // the A descriptor spans 16 planes (M = 128) from its block: keep that inside the stage
    P.stage_bytes = P.a_bytes + P.b_bytes_span + WG_ONES;
    if (P.stage_bytes < 16u * WG_PLANE) P.stage_bytes = 16u * WG_PLANE;
    const uint32_t smem = 2 * P.stage_bytes;
    if (smem > 215 * 1024) return fail(NRV_ERR_UNSUPPORTED, "stages do not fit");
    static bool attr = false;
    if (!attr) {
        NRV_CHECK_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 215 * 1024));
        attr = true;
    }
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        NRV_CHECK_CUDA(cudaGetDevice(&dev));
        NRV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (sms <= 0) sms = 148;
    }
    const int per_sm = smem <= 110 * 1024 ? 2 : 1;   // TMEM: 256 columns each
    long long ns = (long long)sms * per_sm / groups;
    if (ns < 1) ns = 1;
    if (ns > P.ntiles) ns = P.ntiles;
    if ((size_t)ns * per_split > part_floats) ns = (long long)(part_floats / per_split);
    if (ns < 1) return fail(NRV_ERR_ARG, "partial buffer too small");
    P.nsplit = (int)ns;
    P.part = part;
    P.partb = partb;
    wgrad_tc_kernel<<<dim3((unsigned)ns, (unsigned)groups), WG_NT, smem, s>>>(mg, m1, m2, P);
    NRV_CHECK_LAUNCH();
    *nsplit = (int)ns;
    return NRV_OK;
}

static nrv_status wg_geometry(WgParams& P, int n, int H, int W) {
    if (n <= 0 || H <= 0 || W <= 0) return fail(NRV_ERR_ARG, "empty tensor");
    P.n = n;
    P.h = H;
    P.w = W;
    P.tiles_x = (W + 127) / 128;
    const long long ntiles = (long long)P.tiles_x * H * n;
    if (ntiles > 0x3FFFFFFFll) return fail(NRV_ERR_UNSUPPORTED, "too many tiles");
    P.ntiles = (int)ntiles;
    return NRV_OK;
}

// instruction descriptor: FP32 accumulator, A and B BF16 MN-major, M = 128
static uint32_t wg_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

nrv_status tc_wgrad(const Net* net, int l, const void* g, const void* x1, int c1, const void* x2,
                    int c2, int n, int H, int W, float* part, size_t part_floats, float* partb,
                    int* nsplit, cudaStream_t s) {
    const Layer& L = net->layers[l];
    const int cin = c1 + c2;
    // channel groups of 16 (two planes per tap), or one group of 8 (the packed input)
    const int bp = (c1 % 16 == 0 && c2 % 16 == 0) ? 2 : (c1 == 8 && c2 == 0 ? 1 : 0);
    if (L.kind != CONV3 || !bp || L.cout % 8 || L.cout > 128 || (bp == 2 && cin != L.cin))
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core weight gradient: channel counts");
    WgParams P;
    memset(&P, 0, sizeof(P));
    P.mode = 0;
    NRV_TRY(wg_geometry(P, n, H, W));
    P.cout = L.cout;
    P.cin = cin;
    P.groups1 = c1 / (8 * bp);
    P.n_ab = 1;
    P.m_real = L.cout;
    P.ncols = WG_N;
    P.b_planes = bp;
    P.a_bytes = (uint32_t)(L.cout / 8) * WG_PLANE;
    P.b_bytes = 9u * bp * WG_PLANE;
    P.b_bytes_span = WG_B_BYTES;
    P.idesc = wg_idesc(WG_N + 16);
    CUtensorMap mg, m1, m2;
    NRV_TRY(tc_planar_map(&mg, g, n, H, W, L.cout / 8, L.cout / 8));
    NRV_TRY(tc_planar_map(&m1, x1, n, H, W, c1 / 8, bp));
    if (c2) NRV_TRY(tc_planar_map(&m2, x2, n, H, W, c2 / 8, bp));
    else m2 = m1;
    return wg_launch(P, cin / (8 * bp), mg, m1, m2, (size_t)L.cout * 9 * cin, part, part_floats,
                     partb, nsplit, s);
}

nrv_status tc_wgrad_up(const Net* net, int l, const void* g, int g_ld, int g_off, const void* x,
                       int n, int H, int W, float* part, size_t part_floats, float* partb,
                       int* nsplit, cudaStream_t s) {
    const Layer& L = net->layers[l];
    if (L.kind != UPCONV2 || L.cin % 16 || L.cin > 128 || L.cout % 8 || L.cout > 64 || g_ld % 8 ||
        g_off % 8 || g_off + L.cout > g_ld)
        return fail(NRV_ERR_UNSUPPORTED, "tensor-core weight gradient: channel counts");
    WgParams P;
    memset(&P, 0, sizeof(P));
    P.mode = 1;
    NRV_TRY(wg_geometry(P, n, H, W));
    P.cout = L.cout;
    P.cin = L.cin;
    P.groups1 = 0;
    // kernel positions per CTA: all four while 4 C_out rows fit in M = 128, else split by a
    const int groups = 4 * L.cout <= 128 ? 1 : 2;
    P.n_ab = 4 / groups;
    P.m_real = P.n_ab * L.cout;
    P.ncols = L.cin;
    P.b_planes = 2;
    P.a_bytes = (uint32_t)P.n_ab * (L.cout / 8) * WG_PLANE;
    P.b_bytes = (uint32_t)(L.cin / 8) * WG_PLANE;
    P.b_bytes_span = P.b_bytes;
    P.idesc = wg_idesc(L.cin + 16);
    CUtensorMap mg, m1;
    P.g_plane0 = g_off / 8;
    NRV_TRY(tc_parity_map(&mg, g, n * 2 * H, 2 * W, g_ld / 8, L.cout / 8));
    NRV_TRY(tc_planar_map(&m1, x, n, H, W, L.cin / 8, L.cin / 8));
    return wg_launch(P, groups, mg, m1, m1, (size_t)L.cin * 4 * L.cout, part, part_floats, partb,
                     nsplit, s);
}

}  // namespace nrv
