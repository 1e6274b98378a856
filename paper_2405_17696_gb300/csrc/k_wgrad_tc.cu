// Weight gradient of the network's 3x3 convolutions on the tensor cores
// (training by Adam, Sec. 4.1; the backward pass of the layers of the Fig. 1
// caption), with a deterministic reduction.
//
//   dW[co][t][ci] = sum over output pixels p of g[p][co] * x(src_t(p))[ci]
//
// is a GEMM whose reduction dimension K is the output pixels:
//   D[(t, ci)][co] = sum_k X9[k][(t, ci)] g[k][co],   M = (tap, input channel), N = co.
// For a K tile of P output pixels (a rows x tw rectangle) TMA stages, per tap t,
// the input pixels under the tile shifted by the tap ("X9": nine planes per
// 8-channel chunk, [tap][chunk][pixel][8 channels]) and the output gradient g
// ([chunk][pixel][8 channels]).  Both are channel-contiguous: 16 bytes per pixel,
// eight consecutive pixels per 128-byte core matrix, i.e. the MN-major
// no-swizzle operand layout with the 8-channel chunks SBO = P * 16 bytes apart
// and the 8-pixel K groups LBO = 128 bytes apart.  An M block of 128 rows is 16
// consecutive (tap, chunk) planes, so one descriptor covers it.
//
// Sampling (tile grid, tap source, g):
//   mode 0 same grid:  tile on the output grid; tap source (y + dy, x + dx).
//   mode 1 stride-2:   tile on the output grid; tap source (2Y + 1 + dy, 2X + 1 + dx),
//                      a box traversed with element stride 2.
//   mode 2 nearest x2: tile on the coarse input grid, one pass per output parity
//                      (py, px): g is the parity sub-plane (element stride 2) and the
//                      tap source the coarse node (Y + floor((py + dy) / 2), X + floor((px + dx) / 2)).
// Pixels outside an image are zero-filled by TMA (g is zero there, so they add nothing).
//
// Work split: blockIdx.y picks a group of taps (as many as the 512 TMEM columns
// allow: M blocks x N columns); blockIdx.x a set of K tiles (k = blockIdx.x,
// blockIdx.x + gridDim.x, ...), accumulated in TMEM in that order.  Each CTA
// writes its FP32 partial sums once; a second kernel adds the partials of all
// CTAs in a fixed order.  No floating-point atomics: the result is the same on
// every run.
//
// Warp roles (192 threads): warps 0-3 read TMEM at the end (lane = M row),
// warp 4 lane 0 issues TMA, warp 5 walks the MMA loop (lane 0 issues
// tcgen05.mma).  Every wait is bounded and gives up when another role aborts;
// on expiry the kernel raises the error flag, waits (bounded) for its copies
// and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "helm_internal.cuh"
#include "conv.cuh"
#include "tc_ptx.cuh"
#include "wgrad.cuh"

namespace helm {
namespace {

constexpr int WG_NT = 192;
constexpr int WG_MAX_NS = 4;
constexpr long long WG_WAIT_LIMIT = 1ll << 22;
constexpr size_t WG_SMEM_MAX = 200 * 1024;

__device__ __forceinline__ bool wg_wait(uint64_t* bar, uint32_t parity, volatile int* abort_v, unsigned sleep_ns) {
    long long it = 0;
    while (!tc::mbar_try_wait(bar, parity)) {
        ++it;
        if (it > WG_WAIT_LIMIT) return false;
        if ((it & 255) == 0 && *abort_v) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return true;
}

// floor(v / 2) for v in [-1, 2]
__device__ __forceinline__ int fdiv2(int v) { return (v + 2) / 2 - 1; }

template <int MODE>
__global__ void __launch_bounds__(WG_NT) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tm_x0,
                                                        const __grid_constant__ CUtensorMap tm_x1,
                                                        const __grid_constant__ CUtensorMap tm_g, WgradArgs a,
                                                        WgradGeom g) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[WG_MAX_NS], empty[WG_MAX_NS], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int grp = blockIdx.y;
    const int t0 = grp * g.taps_per_group;
    const int ntap = min(9, t0 + g.taps_per_group) - t0;
    const int chunks = ntap * g.cx;                      // real (tap, chunk) planes of this group
    const int mblocks = (chunks + 15) / 16;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, g.tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < WG_MAX_NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
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
    const long long ntiles = g.ktiles > (long long)blockIdx.x ? (g.ktiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int gofs = g.max_chunks * g.plane;             // the g planes within a stage

    // K tile k -> image b, tile origin on the tile grid, output parity
    auto tile_of = [&](long long k, int& b, int& xs, int& ys, int& ph) {
        long long t = (long long)blockIdx.x + k * gridDim.x;
        ph = (int)(t % g.phases);
        t /= g.phases;
        const int tx = (int)(t % g.tiles_x);
        t /= g.tiles_x;
        const int ty = (int)(t % g.tiles_y);
        b = (int)(t / g.tiles_y);
        xs = tx * g.tw;
        ys = ty * g.rows;
    };

    if (warp == 4) {
        // ---------------- TMA producer ----------------
        if ((tid & 31) == 0) {
            const uint32_t tx = (uint32_t)((chunks + g.gchunks) * g.plane);
            bool ok = true;
            long long k = 0;
            for (; k < ntiles && ok; ++k) {
                const int s = (int)(k % g.ns);
                const long long use = k / g.ns;
                if (use > 0 && !wg_wait(&empty[s], (uint32_t)((use - 1) & 1), abort_v, 32)) { ok = false; break; }
                int b, xs, ys, ph;
                tile_of(k, b, xs, ys, ph);
                const int b1 = a.c1 ? (a.x1_map ? __ldg(a.x1_map + b) : (a.x1_bcast ? 0 : b)) : 0;
                unsigned char* st = smem + (size_t)s * g.stage;
                tc::mbar_arrive_expect_tx(&full[s], tx);
                const int py = ph >> 1, px = ph & 1;
                for (int i = 0; i < ntap; ++i) {
                    const int t = t0 + i, dy = t / 3 - 1, dx = t % 3 - 1;
                    unsigned char* d0 = st + (size_t)(i * g.cx) * g.plane;
                    unsigned char* d1 = d0 + (size_t)g.cx0 * g.plane;
                    if (MODE == 0) {
                        tc::tma_load_4d(d0, &tm_x0, 2 * (xs + dx), ys + dy, 0, b, &full[s]);
                        if (a.c1) tc::tma_load_4d(d1, &tm_x1, 2 * (xs + dx), ys + dy, 0, b1, &full[s]);
                    } else if (MODE == 1) {
                        tc::tma_load_5d(d0, &tm_x0, 0, 2 * xs + 1 + dx, 2 * ys + 1 + dy, 0, b, &full[s]);
                        if (a.c1) tc::tma_load_5d(d1, &tm_x1, 0, 2 * xs + 1 + dx, 2 * ys + 1 + dy, 0, b1, &full[s]);
                    } else {
                        const int fx = fdiv2(px + dx), fy = fdiv2(py + dy);
                        tc::tma_load_4d(d0, &tm_x0, 2 * (xs + fx), ys + fy, 0, b, &full[s]);
                        if (a.c1) tc::tma_load_4d(d1, &tm_x1, 2 * (xs + fx), ys + fy, 0, b1, &full[s]);
                    }
                }
                if (MODE == 2)
                    tc::tma_load_5d(st + gofs, &tm_g, 0, 2 * xs + px, 2 * ys + py, 0, b, &full[s]);
                else
                    tc::tma_load_4d(st + gofs, &tm_g, 2 * xs, ys, 0, b, &full[s]);
            }
            if (!ok) {
                *abort_v = 1;
                // the copies of the stages issued last land before the CTA exits (bounded)
                for (long long kk = k - 1; kk >= 0 && kk >= k - g.ns; --kk) {
                    long long it = 0;
                    while (!tc::mbar_try_wait(&full[kk % g.ns], (uint32_t)((kk / g.ns) & 1)) && ++it < WG_WAIT_LIMIT) {
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        const bool leader = (tid & 31) == 0;
        // both operands MN-major (transpose bits 15 and 16): chunks SBO = plane apart, K groups LBO = 128 B
        const uint32_t idesc = tc::idesc_bf16_f32(128, a.npad) | (1u << 15) | (1u << 16);
        const uint64_t desc0 = tc::smem_desc(0u, 128u, (uint32_t)g.plane);
        const uint32_t d_lo = (uint32_t)desc0, d_hi = (uint32_t)(desc0 >> 32);
        const uint32_t plane16 = (uint32_t)g.plane >> 4;
        const int ksteps = g.P / 16;
        bool ok = true;
        for (long long k = 0; k < ntiles && ok; ++k) {
            const int s = (int)(k % g.ns);
            const bool f_ok = wg_wait(&full[s], (uint32_t)((k / g.ns) & 1), abort_v, 32);
            if (!__all_sync(0xffffffffu, f_ok)) { ok = false; break; }
            tc::tc_fence_after_sync();
            const uint32_t s16 = (tc::smem_u32(smem + (size_t)s * g.stage) & 0x3FFFFu) >> 4;
            const uint32_t b_lo = d_lo + s16 + ((uint32_t)gofs >> 4);
            for (int mb = 0; mb < mblocks; ++mb) {
                const uint32_t a_lo = d_lo + s16 + (uint32_t)(16 * mb) * plane16;
                const uint32_t d = tmem + (uint32_t)(mb * a.npad);
                for (int kk = 0; kk < ksteps; ++kk) {
                    if (leader) {
                        const uint64_t ad = ((uint64_t)d_hi << 32) | (a_lo + (uint32_t)(kk * 16));   // 256 B per K step
                        const uint64_t bd = ((uint64_t)d_hi << 32) | (b_lo + (uint32_t)(kk * 16));
                        tc::mma_bf16(d, ad, bd, idesc, (k > 0 || kk > 0) ? 1u : 0u);
                    }
                }
            }
            __syncwarp();
            if (leader) tc::mma_commit(&empty[s]);
        }
        if (!ok) *abort_v = 1;
        __syncwarp();
        if (leader) {
            tc::mma_commit(&done);   // every MMA issued so far completes before `done`
            if (!ok) {
                // aborting: the MMAs in flight finish before the TMEM is freed (bounded)
                long long it = 0;
                while (!tc::mbar_try_wait(&done, 0u) && ++it < WG_WAIT_LIMIT) {
                }
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- epilogue: TMEM -> FP32 partial sums of this CTA ----------------
        // (one wait for the CTA's whole K range: its poll limit grows with the tiles)
        bool got = false;
        {
            const long long limit = WG_WAIT_LIMIT * (1 + ntiles / 256);
            long long it = 0;
            while (!(got = tc::mbar_try_wait(&done, 0u))) {
                if (++it > limit || ((it & 255) == 0 && *abort_v)) break;
                __nanosleep(256);
            }
        }
        if (!got) *abort_v = 1;
        tc::tc_fence_after_sync();
        const int row = warp * 32 + (tid & 31);
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const int Cpad = g.cx * 8;
        float* part = a.partials + (size_t)blockIdx.x * (size_t)9 * Cpad * a.npad;
        for (int mb = 0; mb < mblocks; ++mb) {
            const int rel = 16 * mb + (row >> 3);            // (tap, chunk) plane of this row
            const bool real = got && ntiles > 0 && rel < chunks;
            const int gc = t0 * g.cx + rel;
            const int t = gc / g.cx, ci = (gc % g.cx) * 8 + (row & 7);
            float* dst = part + ((size_t)t * Cpad + ci) * a.npad;
            for (int c0 = 0; c0 < a.npad; c0 += 16) {
                float v[16];
                tc::tmem_ld16(lane_base + (uint32_t)(mb * a.npad + c0), v);
                if (rel < chunks) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4*>(dst + c0 + i) =
                            real ? make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (*abort_v && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, g.tmem_cols);
}

// dW[co][t][ci] += sum over CTAs s (in order) of partial[s][t * Cpad + ci][co]
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int splits, int Cpad, int npad, int cin, int cout,
                                    float* __restrict__ dW) {
    const long long rows = 9ll * Cpad;
    const long long n = rows * npad;
    const long long per = n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % npad);
        const long long r = i / npad;
        const int t = (int)(r / Cpad), ci = (int)(r % Cpad);
        if (co >= cout || ci >= cin) continue;
        float acc = 0.0f;
#pragma unroll 8
        for (int s = 0; s < splits; ++s) acc += part[(size_t)s * per + i];   // loads in flight, sum in order
        dW[((size_t)co * 9 + t) * cin + ci] += acc;
    }
}

// Per-segment sums of g over its pixels: bpart[seg][c] = sum of g[p][c] for the pixels of
// segment seg (grid (segments, npad / 8); fixed order: per thread, then a shared-memory tree)
__global__ void __launch_bounds__(256) bias_partial_kernel(const __nv_bfloat16* __restrict__ gr, int npad,
                                                            long long hw, long long npix, long long seg_len,
                                                            float* __restrict__ bpart) {
    const int c8 = blockIdx.y, seg = blockIdx.x;
    const long long p0 = (long long)seg * seg_len, p1 = min(npix, p0 + seg_len);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const long long b = p / hw, pix = p - b * hw;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(gr + nc8(b, 8 * c8, pix, npad, hw)));
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(h[j]);
    }
    __shared__ float red[256][9];
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = acc[j];
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int j = 0; j < 8; ++j) red[threadIdx.x][j] += red[threadIdx.x + w][j];
        __syncthreads();
    }
    if (threadIdx.x < 8) bpart[(size_t)seg * npad + 8 * c8 + threadIdx.x] = red[0][threadIdx.x];
}

// db[co] += sum over segments of bpart[seg][co], one warp per channel (grid = cout): lane l
// adds segments l, l + 32, ... in order, then a fixed shuffle tree adds the lanes (FP64)
__global__ void bias_reduce_kernel(const float* __restrict__ bpart, int nseg, int npad, int cout, float* __restrict__ db) {
    const int co = blockIdx.x, lane = threadIdx.x;
    if (co >= cout) return;
    double acc = 0.0;
#pragma unroll 4
    for (int s = lane; s < nseg; s += 32) acc += (double)bpart[(size_t)s * npad + co];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) db[co] += (float)acc;
}

int sm_count_wg() {
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

template <int MODE>
int launch_wg_mode(const CUtensorMap& tx0, const CUtensorMap& tx1, const CUtensorMap& tg, const WgradArgs& a,
                   const WgradGeom& g, cudaStream_t st) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(wgrad_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM_MAX);
        cudaFuncSetAttribute(wgrad_tc_kernel<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    // at least 116 KB, so that one CTA per SM holds the TMEM (up to all 512 columns)
    const size_t smem = std::max<size_t>((size_t)g.ns * g.stage + g.slack, 116 * 1024);
    { wgrad_tc_kernel<MODE><<<dim3((unsigned)g.splits, (unsigned)g.ngroups), WG_NT, smem, st>>>(tx0, tx1, tg, a, g); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

}  // namespace

// Tile plan of the weight-gradient kernel (host only); .ktiles = 0 when the layer
// does not fit it.
WgradGeom wgrad_plan(int mode, int c0, int c1, int npad, int hin, int win, int hout, int wout, int nb, int sms) {
    WgradGeom g{};
    if (mode < 0 || mode > 2 || c0 < 8 || c0 % 8 || c1 < 0 || c1 % 8 || npad < 16 || npad % 16 || npad > 128 ||
        nb < 1)
        return WgradGeom{};
    if (mode == 0 && (hin != hout || win != wout)) return WgradGeom{};
    if (mode == 1 && (hin != 2 * hout || win != 2 * wout)) return WgradGeom{};
    if (mode == 2 && (hout != 2 * hin || wout != 2 * win)) return WgradGeom{};
    g.mode = mode;
    g.cx0 = c0 / 8;
    g.cx = (c0 + c1) / 8;
    if (g.cx0 > 256 || g.cx - g.cx0 > 256) return WgradGeom{};
    g.gchunks = npad / 8;
    g.phases = mode == 2 ? 4 : 1;
    // taps per group: as many as the 512 TMEM columns hold (M blocks x npad columns)
    g.taps_per_group = 0;
    for (int tpg = 9; tpg >= 1; --tpg)
        if (((tpg * g.cx + 15) / 16) * npad <= 512) { g.taps_per_group = tpg; break; }
    if (g.taps_per_group < 1) return WgradGeom{};
    g.ngroups = (9 + g.taps_per_group - 1) / g.taps_per_group;
    g.max_chunks = g.taps_per_group * g.cx;
    const int mb_max = (g.max_chunks + 15) / 16;
    uint32_t cols = 32;
    while (cols < (uint32_t)(mb_max * npad)) cols <<= 1;
    if (cols > 512) return WgradGeom{};
    g.tmem_cols = cols;
    const int Ht = mode == 2 ? hin : hout, Wt = mode == 2 ? win : wout;
    // K tile: tw pixels (a multiple of 16, at most 128: a box row is 2 tw 8-byte elements)
    // by rows, P = rows tw <= 128 pixels, shrunk until two stages and the slack fit
    int tw = std::min(128, (Wt + 15) / 16 * 16);
    int rows = std::max(1, std::min(128 / tw, Ht));
    for (;;) {
        g.P = rows * tw;
        g.plane = g.P * 16;
        g.stage = (g.max_chunks + g.gchunks) * g.plane;
        g.slack = 16 * g.plane + 2048;   // reads of the last M block's unused rows stay inside
        if (2 * (size_t)g.stage + g.slack <= WG_SMEM_MAX) break;
        if (rows > 1) rows = (rows + 1) / 2;
        else if (tw > 16) tw = std::max(16, tw / 2 / 16 * 16);
        else return WgradGeom{};
    }
    g.tw = tw;
    g.rows = rows;
    g.ns = (int)std::min<size_t>(WG_MAX_NS, (WG_SMEM_MAX - g.slack) / g.stage);
    g.tiles_x = (Wt + tw - 1) / tw;
    g.tiles_y = (Ht + rows - 1) / rows;
    g.ktiles = (long long)nb * g.tiles_x * g.tiles_y * g.phases;
    const int per_group = std::max(1, (sms + g.ngroups - 1) / g.ngroups);
    g.splits = (int)std::max<long long>(1, std::min<long long>(g.ktiles, per_group));
    return g;
}

int launch_wgrad_tc(const WgradArgs& a, cudaStream_t st) {
    const WgradGeom g = wgrad_plan(a.mode, a.c0, a.c1, a.npad, a.hin, a.win, a.hout, a.wout, a.nb, sm_count_wg());
    if (g.ktiles <= 0 || g.splits > a.max_splits) return HELM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.x0) & 15) || (a.c1 && (reinterpret_cast<uintptr_t>(a.x1) & 15)) ||
        (reinterpret_cast<uintptr_t>(a.g) & 15))
        return HELM_EINVAL;
    alignas(64) CUtensorMap tx0, tx1, tg;
    const int es_x = a.mode == 1 ? 2 : 1, es_g = a.mode == 2 ? 2 : 1;
    const int bw_x = es_x == 2 ? 2 * g.tw : g.tw, bh_x = es_x == 2 ? 2 * g.rows : g.rows;
    const int bw_g = es_g == 2 ? 2 * g.tw : g.tw, bh_g = es_g == 2 ? 2 * g.rows : g.rows;
    if (!tma_map_act(&tx0, a.x0, a.c0, a.win, a.hin, a.nb, bw_x, bh_x, g.cx0, es_x)) return HELM_EINVAL;
    if (a.c1) {
        const int n1 = a.nb1 > 0 ? a.nb1 : (a.x1_bcast ? 1 : a.nb);
        if (!tma_map_act(&tx1, a.x1, a.c1, a.win, a.hin, n1, bw_x, bh_x, g.cx - g.cx0, es_x)) return HELM_EINVAL;
    } else {
        tx1 = tx0;
    }
    if (!tma_map_act(&tg, a.g, a.npad, a.wout, a.hout, a.nb, bw_g, bh_g, g.gchunks, es_g)) return HELM_EINVAL;
    int s;
    switch (a.mode) {
        case 0: s = launch_wg_mode<0>(tx0, tx1, tg, a, g, st); break;
        case 1: s = launch_wg_mode<1>(tx0, tx1, tg, a, g, st); break;
        default: s = launch_wg_mode<2>(tx0, tx1, tg, a, g, st); break;
    }
    if (s != HELM_OK) return s;
    const long long n = 9ll * g.cx * 8 * a.npad;
    { wgrad_reduce_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(
        a.partials, g.splits, g.cx * 8, a.npad, a.cin, a.cout, a.dW); count_launch(); }
    if (cudaGetLastError() != cudaSuccess) return HELM_ECUDA;
    // bias: per-segment sums of g, then their sum in a fixed order
    const long long hw = (long long)a.hout * a.wout, npix = (long long)a.nb * hw;
    const int nseg = (int)std::min<long long>(a.max_bias_segments, std::max<long long>(1, (npix + 4095) / 4096));
    const long long seg_len = (npix + nseg - 1) / nseg;
    { bias_partial_kernel<<<dim3((unsigned)nseg, (unsigned)(a.npad / 8)), 256, 0, st>>>(a.g, a.npad, hw, npix, seg_len,
                                                                                     a.bias_partials); count_launch(); }
    { bias_reduce_kernel<<<(unsigned)a.cout, 32, 0, st>>>(a.bias_partials, nseg, a.npad, a.cout, a.db); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

}  // namespace helm

// Tile plan of the weight-gradient kernel for a layer shape (host only, no GPU
// needed), for checking its bounds on the CPU: out20 = {K tiles, tw, rows, P,
// tiles_x, tiles_y, phases, cx, cx0, gchunks, taps per group, groups, max chunks,
// plane bytes, stage bytes, stages, slack bytes, TMEM columns, splits, dynamic
// shared memory bytes}.  HELM_EINVAL when the kernel does not take the layer.
extern "C" int cnn_wgrad_plan(int mode, int c0, int c1, int npad, int hin, int win, int nb, int sms, long long* out20) {
    if (!out20) return HELM_EINVAL;
    const int hout = mode == 1 ? hin / 2 : (mode == 2 ? 2 * hin : hin);
    const int wout = mode == 1 ? win / 2 : (mode == 2 ? 2 * win : win);
    const helm::WgradGeom g = helm::wgrad_plan(mode, c0, c1, npad, hin, win, hout, wout, nb, sms > 0 ? sms : 148);
    const long long smem = std::max<long long>((long long)g.ns * g.stage + g.slack, 116 * 1024);
    const long long v[20] = {g.ktiles, g.tw, g.rows, g.P, g.tiles_x, g.tiles_y, g.phases, g.cx, g.cx0, g.gchunks,
                             g.taps_per_group, g.ngroups, g.max_chunks, g.plane, g.stage, g.ns, g.slack,
                             (long long)g.tmem_cols, g.splits, smem};
    for (int i = 0; i < 20; ++i) out20[i] = v[i];
    if (g.ktiles <= 0) {
        helm::set_error("cnn_wgrad_plan: the layer does not fit the tensor-core weight-gradient kernel");
        return HELM_EINVAL;
    }
    return HELM_OK;
}
