// Same-grid 3x3 convolution (the ResNet, concatenation, input and output
// layers of the encoder-solver network, Fig. 1 caption) as an implicit GEMM on
// the tensor cores, with the input staged once per tile by TMA.
//
// A CTA owns `rows` output rows x `tw` output columns of one image.  For every
// group of 16 input channels, TMA copies the (rows + 2) x (tw + 2) halo tile of
// the NHWC input into shared memory as two 8-channel planes, each stored
// pixel-major with 16 bytes per pixel: exactly the K-major, no-swizzle
// core-matrix layout (8 pixels x 16 bytes per core matrix) that tcgen05.mma
// reads.  The A operand of tap (dy, dx) for a block of 128 output pixels is then
// the same planes seen from a start address shifted by (dy * pitch + dx) pixels
// -- the nine taps need no gather at all.  Out-of-image halo pixels are
// zero-filled by TMA.  The weights of the group (9 taps x 16 channels x N) are
// copied by TMA into the same layout.
//
// When the image is narrower than 128 pixels the tile holds whole rows and an
// M block runs across row ends: the two halo columns between rows produce
// accumulator rows that the epilogue discards (each accumulator row depends
// only on its own A row).
//
// Warp 4 lane 0 issues the TMA copies and the MMAs (FP32 accumulators in TMEM,
// one 128 x N block per 128 output pixels); warps 0-3 run the epilogue (bias,
// residual, ReLU, BF16 or FP32 store).  Stages are released through mbarriers
// that tcgen05.commit arrives on.  Every wait is bounded; on expiry the kernel
// raises the error flag, waits (bounded) for the copies it issued, frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "helm_internal.cuh"
#include "conv.cuh"
#include "tc_ptx.cuh"

namespace helm {

namespace {

constexpr int EPI = 128;                        // epilogue threads = TMEM lanes = rows of an M block
constexpr int NT = EPI + 64;                    // + a TMA-producer warp and an MMA-issuer warp
constexpr int MAX_NS = 4;                       // stages (one 16-channel group of one tile each)
constexpr long long WAIT_LIMIT = 1ll << 22;     // polls of try_wait before a wait gives up
constexpr int SLACK_PX = 144;                   // plane padding read by the last M block of a narrow tile
constexpr size_t STAGE_BUDGET = 56 * 1024;      // bytes of one stage at most (fewer rows otherwise)
constexpr size_t RING_BUDGET = 112 * 1024;      // bytes of the stage ring: two CTAs per SM

struct Geometry {
    int tw, rows, pw;        // output tile width/height; staged row pitch = tw + 2
    int mb;                  // 128-pixel M blocks per tile
    int rowaligned;          // 1: M block m is output row m (tw >= 127)
    int tiles_x, tiles_y, tiles;
    int plane;               // bytes of one staged 8-channel plane (with slack)
    int wbytes;              // bytes of one group's weights (9 taps x 2 planes x npad rows x 16 B)
    int stage;               // bytes of one stage
    int groups, groups0;     // 16-channel groups in total / taken from x0
    int ns;                  // stages in the ring
    uint32_t tx;             // bytes TMA delivers per stage
    uint32_t acc_cols;       // TMEM columns of one accumulator buffer (mb * npad)
    uint32_t tmem_cols;      // allocated: two accumulator buffers, power of two
};

// Bounded wait that also gives up once another role has raised the abort flag.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_v) {
    long long it = 0;
    while (!tc::mbar_try_wait(bar, parity)) {
        ++it;
        if (it > WAIT_LIMIT) return false;
        if ((it & 255) == 0 && *abort_v) return false;
    }
    return true;
}

// Persistent: CTA k processes tiles k, k + gridDim.x, ...  Warp 4 (lane 0)
// streams the 16-channel groups of its tiles through a ring of `ns` stages;
// warp 5 (lane 0) issues the MMAs of a tile into one of two TMEM accumulator
// buffers; warps 0-3 drain the other buffer (the previous tile) meanwhile.
__global__ void __launch_bounds__(NT) conv3x3_tma_kernel(const __grid_constant__ CUtensorMap tm_x0,
                                                         const __grid_constant__ CUtensorMap tm_x1,
                                                         const __grid_constant__ CUtensorMap tm_w, ConvArgs a,
                                                         Geometry g) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[MAX_NS], empty[MAX_NS], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, g.tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < MAX_NS; ++s) {
            tc::mbar_init(&full[s], 1);     // the producer's expect_tx arrival + the TMA bytes
            tc::mbar_init(&empty[s], 1);    // one tcgen05.commit per use
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);    // tcgen05.commit after the last MMA of a tile
            tc::mbar_init(&tempty[i], EPI); // every epilogue thread, after its TMEM loads
        }
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    volatile int* abort_v = &abort_flag;
    const int cin = a.c0 + a.c1;
    const int G = g.groups;
    const int ntiles = g.tiles > (int)blockIdx.x ? (g.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    auto tile_coords = [&](int k, int& b, int& xs, int& ys) {
        int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int tx = t % g.tiles_x;
        t /= g.tiles_x;
        const int ty = t % g.tiles_y;
        b = t / g.tiles_y;
        xs = tx * g.tw;
        ys = ty * g.rows;
    };

    if (tid == EPI) {
        // ---------------- TMA producer ----------------
        const uint32_t wplane = (uint32_t)a.npad * 16;
        long long j = 0;
        bool ok = true;
        for (int k = 0; k < ntiles && ok; ++k) {
            int b, xs, ys;
            tile_coords(k, b, xs, ys);
            const int b1 = a.c1 ? (a.x1_map ? __ldg(a.x1_map + b) : (a.x1_bcast ? 0 : b)) : 0;
            for (int gi = 0; gi < G; ++gi, ++j) {
                const int s = (int)(j % g.ns);
                const long long use = j / g.ns;
                if (use > 0 && !wait_bar(&empty[s], (uint32_t)((use - 1) & 1), abort_v)) { ok = false; break; }
                unsigned char* st = smem + (size_t)s * g.stage;
                tc::mbar_arrive_expect_tx(&full[s], g.tx);
                for (int h = 0; h < 2; ++h) {
                    const int c = gi * 16 + h * 8;
                    if (gi < g.groups0)
                        tc::tma_load_4d(st + h * g.plane, &tm_x0, c, xs - 1, ys - 1, b, &full[s]);
                    else
                        tc::tma_load_4d(st + h * g.plane, &tm_x1, c - a.c0, xs - 1, ys - 1, b1, &full[s]);
                }
                unsigned char* ws = st + 2 * g.plane;
                for (int tap = 0; tap < 9; ++tap)
                    for (int h = 0; h < 2; ++h)
                        tc::tma_load_2d(ws + (tap * 2 + h) * wplane, &tm_w, tap * cin + gi * 16 + h * 8, 0, &full[s]);
            }
        }
        if (!ok) {
            *abort_v = 1;
            // the copies of the last issued stages land before the CTA exits (bounded)
            for (long long jj = j - 1; jj >= 0 && jj >= j - g.ns; --jj) {
                long long it = 0;
                while (!tc::mbar_try_wait(&full[jj % g.ns], (uint32_t)((jj / g.ns) & 1)) && ++it < WAIT_LIMIT) {
                }
            }
        }
    } else if (tid == EPI + 32) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = tc::idesc_bf16_f32(128, a.npad);
        const uint32_t wplane = (uint32_t)a.npad * 16;
        long long j = 0;
        bool ok = true;
        for (int k = 0; k < ntiles && ok; ++k) {
            const int acc = k & 1;
            const int ause = k >> 1;
            if (ause > 0 && !wait_bar(&tempty[acc], (uint32_t)((ause - 1) & 1), abort_v)) { ok = false; break; }
            tc::tc_fence_after_sync();
            const uint32_t dbase = tmem + (uint32_t)acc * g.acc_cols;
            for (int gi = 0; gi < G; ++gi, ++j) {
                const int s = (int)(j % g.ns);
                if (!wait_bar(&full[s], (uint32_t)((j / g.ns) & 1), abort_v)) { ok = false; break; }
                tc::tc_fence_after_sync();
                const uint32_t a0 = tc::smem_u32(smem + (size_t)s * g.stage);
                const uint32_t w0 = a0 + 2 * g.plane;
                for (int m = 0; m < g.mb; ++m) {
                    const int q0 = g.rowaligned ? m * g.pw : m * 128;
                    const uint32_t d = dbase + (uint32_t)(m * a.npad);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap % 3;   // tap offset + 1
                        const uint64_t ad =
                            tc::smem_desc(a0 + (uint32_t)(q0 + dy * g.pw + dx) * 16u, (uint32_t)g.plane, 128);
                        const uint64_t bd = tc::smem_desc(w0 + (uint32_t)tap * 2u * wplane, wplane, 128);
                        tc::mma_bf16(d, ad, bd, idesc, (gi > 0 || tap > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            if (ok) tc::mma_commit(&tfull[acc]);
        }
        if (!ok) *abort_v = 1;
        tc::mma_commit(&done);   // every MMA issued so far completes before `done`
        long long it = 0;
        while (!tc::mbar_try_wait(&done, 0u) && ++it < WAIT_LIMIT) {
        }
    } else if (warp < 4) {
        // ---------------- epilogue ----------------
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int k = 0; k < ntiles; ++k) {
            const int acc = k & 1;
            if (!wait_bar(&tfull[acc], (uint32_t)((k >> 1) & 1), abort_v)) { *abort_v = 1; break; }
            tc::tc_fence_after_sync();
            int b, xs, ys;
            tile_coords(k, b, xs, ys);
            const uint32_t dbase = lane_base + (uint32_t)acc * g.acc_cols;
            for (int m = 0; m < g.mb; ++m) {
                const int q = (g.rowaligned ? m * g.pw : m * 128) + tid;
                const int yy = q / g.pw, xx = q - yy * g.pw;
                const int oy = ys + yy, ox = xs + xx;
                const bool valid = xx < g.tw && yy < g.rows && oy < a.hout && ox < a.wout;
                const long long p = ((long long)b * a.hout + oy) * a.wout + ox;
                for (int col0 = 0; col0 < a.npad; col0 += 16) {
                    float v[16];
                    tc::tmem_ld16(dbase + (uint32_t)(m * a.npad + col0), v);
                    if (!valid) continue;
                    if (!a.accum) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += __ldg(a.bias + col0 + i);
                    }
                    if (a.res) {
                        const uint4* rp = reinterpret_cast<const uint4*>(a.res + (size_t)p * a.npad + col0);
                        uint4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
                        const __nv_bfloat16* rb0 = reinterpret_cast<const __nv_bfloat16*>(&r0);
                        const __nv_bfloat16* rb1 = reinterpret_cast<const __nv_bfloat16*>(&r1);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            v[i] += __bfloat162float(rb0[i]);
                            v[8 + i] += __bfloat162float(rb1[i]);
                        }
                    }
                    if (a.relu) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
                    }
                    if (a.out_fp32) {
                        float* yo = reinterpret_cast<float*>(a.y) + (size_t)p * a.cstore;
                        if (a.accum) {
                            for (int i = 0; i < 16; ++i)
                                if (col0 + i < a.cstore) yo[col0 + i] += v[i];
                        } else {
                            for (int i = 0; i < 16; ++i)
                                if (col0 + i < a.cstore) yo[col0 + i] = v[i];
                        }
                    } else {
                        uint4 o0, o1;
                        __nv_bfloat16* ob0 = reinterpret_cast<__nv_bfloat16*>(&o0);
                        __nv_bfloat16* ob1 = reinterpret_cast<__nv_bfloat16*>(&o1);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            ob0[i] = __float2bfloat16_rn(v[i]);
                            ob1[i] = __float2bfloat16_rn(v[8 + i]);
                        }
                        uint4* yp = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.y) +
                                                             (size_t)p * a.npad + col0);
                        yp[0] = o0;
                        yp[1] = o1;
                    }
                }
            }
            // this thread's TMEM reads of the buffer are complete (tcgen05.ld waited)
            tc::tc_fence_before_sync();
            tc::mbar_arrive(&tempty[acc]);
        }
    }

    tc::tc_fence_before_sync();
    __syncthreads();
    if (*abort_v && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, g.tmem_cols);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// NHWC BF16 activation [n][h][w][c] viewed as a 4-D tensor (c, w, h, n); box =
// 8 channels x (tw + 2) x (rows + 2) x 1 image.
bool encode_act(CUtensorMap* m, const void* base, int c, int w, int h, int n, int box_w, int box_h) {
    const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)c * 2 * w, (cuuint64_t)c * 2 * w * h};
    const cuuint32_t box[4] = {8u, (cuuint32_t)box_w, (cuuint32_t)box_h, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// weights [npad][9 * cin] viewed as 2-D; box = 8 input channels x npad rows.
bool encode_w(CUtensorMap* m, const void* base, int cin, int npad) {
    const cuuint64_t dims[2] = {(cuuint64_t)9 * cin, (cuuint64_t)npad};
    const cuuint64_t strides[1] = {(cuuint64_t)9 * cin * 2};
    const cuuint32_t box[2] = {8u, (cuuint32_t)npad};
    const cuuint32_t estr[2] = {1u, 1u};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::atomic<int> g_rows_cap{0};   // tile-height limit set by cnn_set_conv_tiling (0 = automatic)

Geometry plan(const ConvArgs& a) {
    Geometry g{};
    const int H = a.hout, W = a.wout;
    g.groups = (a.c0 + a.c1) / 16;
    g.groups0 = a.c0 / 16;
    g.tw = W >= 128 ? 128 : W;
    g.pw = g.tw + 2;
    g.rowaligned = g.tw >= 127;          // a row (plus its halo) no longer fits one M block
    const int maxmb = 128 / a.npad;      // two accumulator buffers of at most 128 TMEM columns
    g.wbytes = 9 * 2 * a.npad * 16;
    auto fill = [&](int rows) {
        g.rows = rows;
        g.mb = g.rowaligned ? rows : (rows * g.pw + 127) / 128;
        g.plane = (((rows + 2) * g.pw + SLACK_PX) * 16 + 127) / 128 * 128;
        g.stage = 2 * g.plane + g.wbytes;
    };
    int rmax = g.rowaligned ? maxmb : (maxmb * 128) / g.pw;
    const int cap = g_rows_cap.load();
    if (cap > 0 && rmax > cap) rmax = cap;
    if (rmax < 1) rmax = 1;
    if (rmax > H) rmax = H;
    if (rmax > 254) rmax = 254;
    int rows = rmax;
    fill(rows);
    while (rows > 1 && (size_t)g.stage > STAGE_BUDGET) fill(--rows);
    g.ns = (int)(RING_BUDGET / (size_t)g.stage);
    if (g.ns > MAX_NS) g.ns = MAX_NS;
    if (g.ns < 2) g.ns = 2;
    g.tiles_x = (W + g.tw - 1) / g.tw;
    g.tiles_y = (H + g.rows - 1) / g.rows;
    g.tx = (uint32_t)(2 * (g.rows + 2) * g.pw * 16 + g.wbytes);
    g.acc_cols = (uint32_t)(g.mb * a.npad);
    uint32_t cols = 32;
    while (cols < 2 * g.acc_cols) cols <<= 1;
    g.tmem_cols = cols;
    return g;
}

int sm_count() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
        (void)cudaGetLastError();
    });
    return n > 0 ? n : 148;
}

}  // namespace

// Same-grid layers through TMA-staged halo tiles; returns HELM_EINVAL (nothing
// launched) when the layer does not fit this path, so that the caller can use
// the gather kernel instead.
int launch_conv3x3_tma(const ConvArgs& a, cudaStream_t st) {
    if (a.mode != 0 || a.hin != a.hout || a.win != a.wout || !encode_fn()) return HELM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.x0) & 15) || (a.c1 && (reinterpret_cast<uintptr_t>(a.x1) & 15)) ||
        (reinterpret_cast<uintptr_t>(a.w) & 15))
        return HELM_EINVAL;
    const Geometry g = plan(a);
    if (g.pw > 256 || g.rows + 2 > 256) return HELM_EINVAL;
    const size_t smem = (size_t)g.ns * g.stage;
    if (smem > 200 * 1024 || g.tmem_cols > 256) return HELM_EINVAL;
    alignas(64) CUtensorMap tm0, tm1, tmw;
    if (!encode_act(&tm0, a.x0, a.c0, a.win, a.hin, a.nb, g.pw, g.rows + 2)) return HELM_EINVAL;
    if (a.c1) {
        const int n1 = a.nb1 > 0 ? a.nb1 : (a.x1_bcast ? 1 : a.nb);
        if (!encode_act(&tm1, a.x1, a.c1, a.win, a.hin, n1, g.pw, g.rows + 2)) return HELM_EINVAL;
    } else {
        tm1 = tm0;
    }
    if (!encode_w(&tmw, a.w, a.c0 + a.c1, a.npad)) return HELM_EINVAL;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(conv3x3_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    const long long tiles = (long long)g.tiles_x * g.tiles_y * a.nb;
    if (tiles > 0x7fffffffLL) return HELM_EINVAL;
    Geometry gg = g;
    gg.tiles = (int)tiles;
    // two CTAs per SM (ring and TMEM budgets), persistent over the tiles
    const long long grid = std::min<long long>(tiles, 2LL * sm_count());
    // at least 80 KB of shared memory per CTA keeps a third CTA (and its TMEM) off an SM
    const size_t smem_req = std::max<size_t>(smem, 80 * 1024);
    conv3x3_tma_kernel<<<(unsigned)grid, NT, smem_req, st>>>(tm0, tm1, tmw, a, gg);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

}  // namespace helm

extern "C" int cnn_set_conv_tiling(int max_rows) {
    if (max_rows < 0 || max_rows > 254) {
        helm::set_error("cnn_set_conv_tiling: max_rows must be in [0, 254]");
        return HELM_EINVAL;
    }
    helm::g_rows_cap.store(max_rows);
    return HELM_OK;
}
