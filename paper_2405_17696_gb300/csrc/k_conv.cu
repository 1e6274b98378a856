// 3x3 convolution layers of the encoder-solver network (Fig. 1 caption,
// Sec. 3.4) as implicit GEMMs on the sm_100-family tensor cores.
//
//   y[p, n] = act( bias[n] + res[p, n] + sum_{tap, c} W[n, tap, c] x(src(p, tap), c) )
//
// M = output pixels (128 per CTA), N = output channels (all of them per CTA,
// 16..128), K = 9 taps x input channels.  The input may be the channel
// concatenation of two tensors (the second one optionally shared by the
// whole batch: the encoder's context features), and is sampled in one of
// three modes: same grid, stride-2 'down' (output node (Y, X) centred on input
// node (2Y+1, 2X+1)) or nearest-neighbour 'up' (output on the doubled grid).
//
// Per K stage (one tap x CK channels) the 128 threads gather their pixel's
// channels and the weights into shared memory in the K-major core-matrix
// layout (8 rows x 16 bytes per core matrix, no swizzle); one thread issues
// tcgen05.mma (M=128, N, K=16, BF16 in, FP32 accumulate in TMEM) and commits
// to the stage's mbarrier, so gathering stage k+1 overlaps the MMAs of stage
// k.  The epilogue reads the accumulator rows with tcgen05.ld, adds bias and
// residual, applies ReLU and stores BF16 (or FP32 for the output layer).
// Every mbarrier wait is bounded; on expiry the kernel raises an error flag,
// drains what it issued (again bounded), frees its TMEM and returns.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "helm_internal.cuh"
#include "conv.cuh"
#include "tc_ptx.cuh"

namespace helm {

namespace {

constexpr int CT = 128;                 // threads per CTA = rows of the M tile
constexpr long long WAIT_LIMIT = 1ll << 20;   // about a second of try_wait polls

__device__ __forceinline__ bool src_coord(int mode, int o, int d, int n_in, int* i) {
    int v;
    if (mode == 0) v = o + d;
    else if (mode == 1) v = 2 * o + 1 + d;
    else if (mode == 3) {
        const int u = o - 1 - d;
        if (u < 0 || (u & 1)) return false;
        v = u >> 1;
    } else {
        int u = o + d;
        if (u < 0 || u >= 2 * n_in) return false;
        *i = u >> 1;
        return true;
    }
    if (v < 0 || v >= n_in) return false;
    *i = v;
    return true;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity) {
    long long it = 0;
    while (!tc::mbar_try_wait(bar, parity))
        if (++it > WAIT_LIMIT) return false;
    return true;
}

// Warp-specialised pipeline: warps 0-3 gather stages into a ring of NS
// shared-memory buffers and arrive on full[s]; warp 4 (one elected lane)
// waits for full[s], issues the MMAs of the stage and commits them to
// empty[s], which frees the buffer for the producers; the last commit also
// arrives on `done`, after which warps 0-3 run the epilogue from TMEM.
// pipeline stages: 64 KB of ring at most, so that three CTAs fit on an SM
constexpr int ns_of(int ck) { return ck == 64 ? 2 : 4; }
constexpr int NT = CT + 32;             // 4 producer/epilogue warps + 1 MMA warp

template <int CK>
__global__ void __launch_bounds__(NT) conv3x3_tc_kernel(ConvArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NS = ns_of(CK);
    constexpr int TILE_BYTES = CT * CK * 2;       // one operand tile (A, or B with up to 128 rows)
    constexpr int STAGE_BYTES = 2 * TILE_BYTES;
    constexpr int KG = CK / 8;                    // core matrices along K per row group
    __shared__ uint64_t full[NS], empty[NS], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t ncols = a.npad < 32 ? 32u : (uint32_t)a.npad;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], CT);     // every producer thread arrives once per stage
            tc::mbar_init(&empty[s], 1);     // one tcgen05.commit per stage
        }
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    const long long mtot = (long long)a.nb * a.hout * a.wout;
    const int cin = a.c0 + a.c1;
    const int cper = cin / CK;                    // stages per tap
    const int nchunks = 9 * cper;
    volatile int* abort_v = &abort_flag;

    if (warp < 4) {
        // ---------------- producers: one output pixel (A row) per thread ----------------
        const long long p = (long long)blockIdx.x * CT + tid;
        const bool valid = p < mtot;
        int b = 0, oy = 0, ox = 0;
        if (valid) {
            b = (int)(p / ((long long)a.hout * a.wout));
            const int r = (int)(p - (long long)b * a.hout * a.wout);
            oy = r / a.wout;
            ox = r - oy * a.wout;
        }
        const int b1 = (a.c1 && valid) ? (a.x1_map ? __ldg(a.x1_map + b) : (a.x1_bcast ? 0 : b)) : 0;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % NS;
            if (c >= NS) {
                // the MMAs that read this buffer NS chunks ago must be done
                if (!bounded_wait(&empty[s], (uint32_t)(((c / NS) - 1) & 1))) { *abort_v = 1; }
            }
            if (*abort_v) break;
            const int tap = c / cper;
            const int cc = (c - tap * cper) * CK;
            unsigned char* As = smem + s * STAGE_BYTES;
            unsigned char* Bs = As + TILE_BYTES;
            const __nv_bfloat16* src = nullptr;
            const size_t hw_in = (size_t)a.hin * a.win;
            if (valid) {
                int iy, ix;
                if (src_coord(a.mode, oy, tap / 3 - 1, a.hin, &iy) && src_coord(a.mode, ox, tap % 3 - 1, a.win, &ix)) {
                    const long long pix = (long long)iy * a.win + ix;
                    if (cc < a.c0)
                        src = a.x0 + nc8(b, cc, pix, a.c0, (long long)hw_in);
                    else
                        src = a.x1 + nc8(b1, cc - a.c0, pix, a.c1, (long long)hw_in);
                }
            }
            unsigned char* arow = As + (tid >> 3) * (KG * 128) + (tid & 7) * 16;
            uint4 va[KG];
#pragma unroll
            for (int kg = 0; kg < KG; ++kg)   // consecutive 8-channel chunks are planes hw_in pixels apart
                va[kg] = src ? __ldg(reinterpret_cast<const uint4*>(src + (size_t)kg * hw_in * 8))
                             : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int kg = 0; kg < KG; ++kg) *reinterpret_cast<uint4*>(arow + kg * 128) = va[kg];
            if (tid < a.npad) {
                const __nv_bfloat16* wr = a.w + ((size_t)tid * 9 + tap) * cin + cc;
                unsigned char* brow = Bs + (tid >> 3) * (KG * 128) + (tid & 7) * 16;
#pragma unroll
                for (int kg = 0; kg < KG; ++kg)
                    *reinterpret_cast<uint4*>(brow + kg * 128) = __ldg(reinterpret_cast<const uint4*>(wr) + kg);
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[s]);
        }
    } else if (tid == CT) {
        // ---------------- MMA issuer: one thread of warp 4 ----------------
        const uint32_t idesc = tc::idesc_bf16_f32(CT, a.npad);
        const uint32_t sbo = KG * 128;
        int c = 0;
        for (; c < nchunks; ++c) {
            const int s = c % NS;
            if (!bounded_wait(&full[s], (uint32_t)((c / NS) & 1)) || *abort_v) { *abort_v = 1; break; }
            tc::tc_fence_after_sync();
            const uint32_t a0 = tc::smem_u32(smem + s * STAGE_BYTES), b0 = a0 + TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < CK / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, sbo);
                const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, sbo);
                tc::mma_bf16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[s]);
        }
        // every MMA issued so far completes before `done` (also on the abort path)
        tc::mma_commit(&done);
    }
    // ---------------- epilogue (warps 0-3) ----------------
    bool ok = true;
    if (warp < 4) ok = bounded_wait(&done, 0u);
    if (!ok) *abort_v = 1;
    tc::tc_fence_after_sync();
    __syncthreads();
    if (*abort_v) {
        if (tid == 0) atomicExch(a.err, 1);
        tc::tc_fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tmem, ncols);
        return;
    }
    if (warp < 4) {
        const long long p = (long long)blockIdx.x * CT + tid;
        const bool valid = p < mtot;
        const long long hw_out = (long long)a.hout * a.wout;
        const long long pb = valid ? p / hw_out : 0, ppix = valid ? p - pb * hw_out : 0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int col0 = 0; col0 < a.npad; col0 += 16) {
            float v[16];
            tc::tmem_ld16(trow + col0, v);
            if (!valid) continue;
            if (!a.accum) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += __ldg(a.bias + col0 + i);
            }
            if (a.res) {
                const __nv_bfloat16* rq = a.res + nc8(pb, col0, ppix, a.npad, hw_out);
                uint4 r0 = __ldg(reinterpret_cast<const uint4*>(rq));
                uint4 r1 = __ldg(reinterpret_cast<const uint4*>(rq + (size_t)hw_out * 8));
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
                __nv_bfloat16* yq = reinterpret_cast<__nv_bfloat16*>(a.y) + nc8(pb, col0, ppix, a.npad, hw_out);
                *reinterpret_cast<uint4*>(yq) = o0;
                *reinterpret_cast<uint4*>(yq + (size_t)hw_out * 8) = o1;
            }
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

template <int CK>
int launch_ck(const ConvArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)ns_of(CK) * 2 * CT * CK * 2;
    static bool configured = false;   // attribute is per function; setting it twice is harmless
    if (!configured) {
        cudaFuncSetAttribute(conv3x3_tc_kernel<CK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    const long long mtot = (long long)a.nb * a.hout * a.wout;
    const unsigned grid = (unsigned)((mtot + CT - 1) / CT);
    { conv3x3_tc_kernel<CK><<<grid, NT, smem, st>>>(a); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

}  // namespace

namespace {
std::atomic<int> g_conv_path{0};
std::atomic<long long> g_launch_tma{0}, g_launch_gather{0};
}  // namespace

// Validates the shapes and launches; returns HELM_EINVAL for unsupported ones.
// Layers go through the TMA halo-tile kernel unless the gather kernel is
// forced (cnn_set_conv_path) or the layer does not fit it.
int launch_conv3x3(const ConvArgs& a, cudaStream_t st) {
    const int cin = a.c0 + a.c1;
    if (a.npad != 16 && a.npad != 32 && a.npad != 64 && a.npad != 128) {
        set_error("conv3x3: output channels must be padded to 16, 32, 64 or 128");
        return HELM_EINVAL;
    }
    if (a.c0 % 16 || a.c1 % 16 || cin < 16 || !a.x0 || (a.c1 && !a.x1) || !a.w || !a.y || !a.err) {
        set_error("conv3x3: input channels must be multiples of 16 and pointers non-null");
        return HELM_EINVAL;
    }
    if (a.nb < 1 || a.hin < 1 || a.win < 1 || a.mode < 0 || a.mode > 3 || (a.accum && !a.out_fp32) ||
        (!a.accum && !a.bias)) {
        set_error("conv3x3: bad shape or mode");
        return HELM_EINVAL;
    }
    const int path = g_conv_path.load();
    if (path != 1) {
        const int t = launch_conv3x3_tma(a, st, path == 2 ? 1 : (path == 3 ? 2 : 0));
        if (t == HELM_OK) {
            ++g_launch_tma;
            return HELM_OK;
        }
        if (t != HELM_EINVAL) {
            set_error(std::string("conv3x3 (TMA) launch: ") + cudaGetErrorString(cudaGetLastError()));
            return t;
        }
    }
    ++g_launch_gather;
    int ck = 64;
    if (a.c0 % 64 || (a.c1 && a.c1 % 64)) ck = 32;
    if (a.c0 % 32 || (a.c1 && a.c1 % 32)) ck = 16;
    int s;
    if (ck == 64) s = launch_ck<64>(a, st);
    else if (ck == 32) s = launch_ck<32>(a, st);
    else s = launch_ck<16>(a, st);
    if (s != HELM_OK) set_error(std::string("conv3x3 launch: ") + cudaGetErrorString(cudaGetLastError()));
    return s;
}

}  // namespace helm

extern "C" int cnn_set_conv_path(int path) {
    if (path < 0 || path > 3) {
        helm::set_error("cnn_set_conv_path: path must be 0 (automatic), 1 (gather kernel only), 2 (TMA "
                        "kernel with the column-taps-in-N variant) or 3 (TMA kernel with the row-taps-in-N variant)");
        return HELM_EINVAL;
    }
    helm::g_conv_path.store(path);
    return HELM_OK;
}

extern "C" void cnn_conv_launch_counts(long long* tma, long long* gather) {
    if (tma) *tma = helm::g_launch_tma.load();
    if (gather) *gather = helm::g_launch_gather.load();
}
