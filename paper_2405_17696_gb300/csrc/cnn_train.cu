// Training of the encoder-solver network (Sec. 4.1, Eq. 4.2; Alg. 2):
// the MSE loss between the network's error estimate and the true error, the
// backward pass through the recorded forward tape, and Adam (Kingma & Ba).
//
// Backward of one convolution y = act(W * x + b [+ res]) with upstream
// gradient G_y (FP32):
//   g      = G_y . [y > 0]  (BF16 operand; FP32 copy added to G_res for a ResNet skip)
//   dW, db += sum over pixels of g (x) x_tap    (tensor cores, K = pixels, deterministic
//            reduction over CTAs: k_wgrad_tc.cu; the FP32 CUDA-core kernel below is
//            the second path, cnn_set_wgrad_path(1), and the fallback)
//   G_x   += W^T * g   on the tensor cores with the same kernel as the forward:
//            'same'  -> same-grid convolution with transposed, tap-flipped weights,
//            'down'  -> the transpose-of-down gather mode with transposed weights,
//            'up'    -> same-grid convolution on the fine grid, then a 2x2 sum.
// The context features of the solver's concatenations (one image per
// frequency, shared by every sample of that frequency) collect their
// gradient summed over the samples that use them, and flow into the encoder.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <atomic>

#include "cnn_internal.cuh"
#include "reduce.cuh"
#include "wgrad.cuh"

namespace helm {
namespace {

// out = bf16(G . [y > 0]) over cg gradient channels into cpad channels (out and
// the activation y, cy channels, in the chunked layout; G is FP32 [n][cg]); when
// res_grad is given, res_grad += the FP32 masked gradient (same layout as G).
__global__ void mask_to_bf16_kernel(const float* __restrict__ G, int cg, const __nv_bfloat16* __restrict__ y,
                                    int cy, int cpad, long long n, long long hw, __nv_bfloat16* __restrict__ out,
                                    float* __restrict__ res_grad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * cpad;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / cpad;
        const int c = (int)(i - p * cpad);
        const long long b = p / hw, pix = p - b * hw;
        float v = 0.0f;
        if (c < cg) {
            v = G[p * cg + c];
            if (y && !(__bfloat162float(y[nc8(b, c, pix, cy, hw)]) > 0.0f)) v = 0.0f;
            if (res_grad) res_grad[p * cg + c] += v;
        }
        out[nc8(b, c, pix, cpad, hw)] = __float2bfloat16_rn(v);
    }
}

// The same for cg == cpad, a multiple of 8: one thread per (pixel, 8-channel chunk) with
// 16-byte loads and stores (grid.y = chunk, grid.z = image: no division per element).
__global__ void mask_to_bf16_vec_kernel(const float* __restrict__ G, const __nv_bfloat16* __restrict__ y, int cy,
                                        int cpad, long long hw, __nv_bfloat16* __restrict__ out,
                                        float* __restrict__ res_grad) {
    const int c8 = blockIdx.y;
    const long long b = blockIdx.z;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < hw;
         pix += (long long)gridDim.x * blockDim.x) {
        const long long p = b * hw + pix;
        const float4* g4 = reinterpret_cast<const float4*>(G + p * cpad + 8 * c8);
        float4 a = g4[0], c = g4[1];
        float v[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
        if (y) {
            const uint4 yv = *reinterpret_cast<const uint4*>(y + nc8(b, 8 * c8, pix, cy, hw));
            const __nv_bfloat16* yh = reinterpret_cast<const __nv_bfloat16*>(&yv);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (!(__bfloat162float(yh[j]) > 0.0f)) v[j] = 0.0f;
        }
        if (res_grad) {
            float4* r4 = reinterpret_cast<float4*>(res_grad + p * cpad + 8 * c8);
            float4 r0 = r4[0], r1 = r4[1];
            r0.x += v[0]; r0.y += v[1]; r0.z += v[2]; r0.w += v[3];
            r1.x += v[4]; r1.y += v[5]; r1.z += v[6]; r1.w += v[7];
            r4[0] = r0;
            r4[1] = r1;
        }
        uint4 o;
        __nv_bfloat16* oh = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
        for (int j = 0; j < 8; ++j) oh[j] = __float2bfloat16_rn(v[j]);
        *reinterpret_cast<uint4*>(out + nc8(b, 8 * c8, pix, cpad, hw)) = o;
    }
}

// Wt[ci][t][co] = W[co][flip ? 8 - t : t][off + ci]   (dgrad weights of one input part)
__global__ void transpose_weights_kernel(const __nv_bfloat16* __restrict__ W, int npad, int cin_pad, int off,
                                         int cpart, int flip, __nv_bfloat16* __restrict__ Wt) {
    const int total = cpart * 9 * npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int co = i % npad, t = (i / npad) % 9, ci = i / (9 * npad);
        Wt[i] = W[((size_t)co * 9 + (flip ? 8 - t : t)) * cin_pad + off + ci];
    }
}

// coarse[b][i][j][c] += sum of the 2x2 block of fine[b][2i..2i+1][2j..2j+1][c]
__global__ void sumpool_accum_kernel(const float* __restrict__ fine, int nb, int h, int w, int c,
                                     float* __restrict__ coarse) {
    const long long total = (long long)nb * h * w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const int b = (int)(r / h);
        const size_t W2 = 2 * (size_t)w;
        const size_t base = (((size_t)b * 2 * h + 2 * y) * W2 + 2 * x) * c + ch;
        coarse[i] += fine[base] + fine[base + c] + fine[base + W2 * c] + fine[base + W2 * c + c];
    }
}

// G_ctx[f] += sum over the samples b that use context image f (map(b) == f, or f = 0
// when bcast == 1) of tmp[b], summed in the order of b: one thread per context element,
// no atomics, so that the gradient is the same on every run
__global__ void reduce_to_context_kernel(const float* __restrict__ tmp, long long per_image, int nb,
                                         const int* __restrict__ map, int bcast, int nctx, float* __restrict__ gctx) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_image * nctx;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / per_image);
        const long long q = i - (long long)f * per_image;
        float acc = 0.0f;
        for (int b = 0; b < nb; ++b)
            if ((bcast == 1 ? 0 : __ldg(map + b)) == f) acc += tmp[(long long)b * per_image + q];
        gctx[i] += acc;
    }
}

struct WgArgs {
    const __nv_bfloat16* x0;
    int c0;
    const __nv_bfloat16* x1;
    int c1;
    int x1_bcast;
    const int* x1_map;
    int nb, hin, win, hout, wout, mode;
    const __nv_bfloat16* g;   // [nb][npad/8][hout][wout][8] (chunked layout)
    int npad, cout, cin;      // cin: logical input channels (weights layout [cout][9][cin])
    float* dW;
    float* db;
};

__device__ __forceinline__ bool fwd_src(int mode, int o, int d, int n_in, int* i) {
    int v;
    if (mode == 0) v = o + d;
    else if (mode == 1) v = 2 * o + 1 + d;
    else {
        const int u = o + d;
        if (u < 0 || u >= 2 * n_in) return false;
        *i = u >> 1;
        return true;
    }
    if (v < 0 || v >= n_in) return false;
    *i = v;
    return true;
}

// Weight gradient on the CUDA cores (FP32):
//   dW[co][t][ci] += sum_p g[p][co] x(src(p, t))[ci],   db[co] += sum_p g[p][co].
// A CTA owns a block of 16 output x 16 input channels and loops over tiles of
// th x tw output pixels.  Per tile it stages g (16 channels), the input
// rectangle the tile's taps read (16 channels, zero outside the image) and a
// table pixel x tap -> staged input pixel (a zero row for taps outside), all
// in shared memory.  Thread (lane l, warp w): output channels 4 (l / 8) .. +3,
// input channels 2 (l % 8) .. +1, all nine taps (72 FP32 accumulators), over
// the pixels p = w, w + 8, ...; the eight warps' sums are combined in shared
// memory and added to dW once per CTA.
struct Wg2 {
    int th, tw;                 // output pixel tile
    int tiles_x, tiles_y;       // tiles per image
    int sh, sw;                 // staged input rectangle (rows x columns)
};

__device__ __forceinline__ void wg_rect(int mode, int oy0, int ox0, int* r0, int* s0) {
    if (mode == 0) { *r0 = oy0 - 1; *s0 = ox0 - 1; }
    else if (mode == 1) { *r0 = 2 * oy0; *s0 = 2 * ox0; }
    else { *r0 = (oy0 >> 1) - 1; *s0 = (ox0 >> 1) - 1; }
}

__global__ void __launch_bounds__(256) wgrad_kernel(WgArgs a, Wg2 w) {
    extern __shared__ float wsm[];
    const int np = w.th * w.tw;
    const int nst = w.sh * w.sw;                     // staged pixels; row nst is all zero
    float* xs = wsm;                                 // [nst + 1][16]
    float* gs = xs + (size_t)(nst + 1) * 16;         // [np][16]
    int* tab = reinterpret_cast<int*>(gs + (size_t)np * 16);   // [np][9]
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int n_l = (lane >> 3) * 4, c_l = (lane & 7) * 2;
    const int cb = blockIdx.y * 16, nbk = blockIdx.z * 16;
    const int ctot = a.c0 + a.c1;
    const long long tiles = (long long)a.nb * w.tiles_y * w.tiles_x;
    float acc[9][4][2];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[t][i][0] = acc[t][i][1] = 0.0f;
    float accb[4] = {0.f, 0.f, 0.f, 0.f};
    if (tid < 16) xs[(size_t)nst * 16 + tid] = 0.0f;

    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int tx = (int)(tile % w.tiles_x);
        const long long r = tile / w.tiles_x;
        const int ty = (int)(r % w.tiles_y);
        const int b = (int)(r / w.tiles_y);
        const int oy0 = ty * w.th, ox0 = tx * w.tw;
        int r0, s0;
        wg_rect(a.mode, oy0, ox0, &r0, &s0);
        __syncthreads();   // the previous tile's reads are done
        // g: 16 channels of the output gradient
        for (int i = tid; i < np * 16; i += 256) {
            const int pp = i >> 4, k = i & 15;
            const int oy = oy0 + pp / w.tw, ox = ox0 + pp % w.tw;
            float v = 0.0f;
            if (oy < a.hout && ox < a.wout)
                v = __bfloat162float(a.g[nc8(b, nbk + k, (long long)oy * a.wout + ox, a.npad,
                                             (long long)a.hout * a.wout)]);
            gs[i] = v;
        }
        // input rectangle: 16 channels of x0 or x1
        const bool second = cb >= a.c0;
        const __nv_bfloat16* xsrc = second ? a.x1 : a.x0;
        const int cstride = second ? a.c1 : a.c0;
        const int coff = second ? cb - a.c0 : cb;
        const int bx = second ? (a.x1_map ? __ldg(a.x1_map + b) : (a.x1_bcast ? 0 : b)) : b;
        for (int i = tid; i < nst * 16; i += 256) {
            const int q = i >> 4, k = i & 15;
            const int iy = r0 + q / w.sw, ix = s0 + q % w.sw;
            float v = 0.0f;
            if (iy >= 0 && iy < a.hin && ix >= 0 && ix < a.win && cb + k < ctot)
                v = __bfloat162float(xsrc[nc8(bx, coff + k, (long long)iy * a.win + ix, cstride,
                                              (long long)a.hin * a.win)]);
            xs[i] = v;
        }
        // pixel x tap -> staged input pixel (nst: outside the input)
        for (int i = tid; i < np * 9; i += 256) {
            const int pp = i / 9, t = i - pp * 9;
            const int oy = oy0 + pp / w.tw, ox = ox0 + pp % w.tw;
            int iy, ix, idx = nst;
            if (fwd_src(a.mode, oy, t / 3 - 1, a.hin, &iy) && fwd_src(a.mode, ox, t % 3 - 1, a.win, &ix))
                idx = (iy - r0) * w.sw + (ix - s0);
            tab[i] = idx;
        }
        __syncthreads();
        for (int pp = grp; pp < np; pp += 8) {
            const float4 g4 = *reinterpret_cast<const float4*>(gs + pp * 16 + n_l);
            const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) accb[i] += gv[i];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float2 x2 = *reinterpret_cast<const float2*>(xs + (size_t)tab[pp * 9 + t] * 16 + c_l);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[t][i][0] = fmaf(gv[i], x2.x, acc[t][i][0]);
                    acc[t][i][1] = fmaf(gv[i], x2.y, acc[t][i][1]);
                }
            }
        }
    }
    // combine the eight pixel groups (warps) through shared memory, then one atomic per weight
    __syncthreads();
    float* red = wsm;   // [32 lanes][76]
    for (int src = 1; src < 8; ++src) {
        if (grp == src) {
            float* o = red + lane * 76;
#pragma unroll
            for (int t = 0; t < 9; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) { o[t * 8 + i * 2] = acc[t][i][0]; o[t * 8 + i * 2 + 1] = acc[t][i][1]; }
#pragma unroll
            for (int i = 0; i < 4; ++i) o[72 + i] = accb[i];
        }
        __syncthreads();
        if (grp == 0) {
            const float* o = red + lane * 76;
#pragma unroll
            for (int t = 0; t < 9; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) { acc[t][i][0] += o[t * 8 + i * 2]; acc[t][i][1] += o[t * 8 + i * 2 + 1]; }
#pragma unroll
            for (int i = 0; i < 4; ++i) accb[i] += o[72 + i];
        }
        __syncthreads();
    }
    if (grp == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int co = nbk + n_l + i;
            if (co >= a.cout) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int ci = cb + c_l + j;
                if (ci >= a.cin) continue;
#pragma unroll
                for (int t = 0; t < 9; ++t) atomicAdd(a.dW + ((size_t)co * 9 + t) * a.cin + ci, acc[t][i][j]);
            }
            if (blockIdx.y == 0 && c_l == 0) atomicAdd(a.db + co, accb[i]);
        }
    }
}

}  // namespace

std::atomic<int> g_wgrad_path{0};   // 0: tensor cores (k_wgrad_tc.cu), 1: CUDA cores

// Scratch of the tensor-core weight gradient (partial sums per CTA, bias partials),
// grown on demand; *buf / *cap owned by the caller.
int wgrad_scratch(float** buf, size_t* cap, size_t need) {
    if (*cap >= need) return HELM_OK;
    if (*buf) {
        cudaFree(*buf);   // (synchronises the device: no kernel of ours is reading it)
        *buf = nullptr;
        *cap = 0;
    }
    if (cudaMalloc(buf, need * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        *buf = nullptr;
        set_error("out of device memory for the weight-gradient scratch");
        return HELM_ENOMEM;
    }
    *cap = need;
    return HELM_OK;
}

constexpr int WG_BIAS_SEGMENTS = 1184;

// dW, db += the weight and bias gradient of one layer: g is the BF16 masked output
// gradient (chunked layout, npad channels), x0 / x1 the layer's inputs.
int layer_wgrad(const __nv_bfloat16* x0, int c0, const __nv_bfloat16* x1, int c1, int x1_bcast, const int* x1_map,
                int nb1, int nb, int hin, int win, int hout, int wout, int mode, const __nv_bfloat16* g, int npad,
                int cout, int cin, float* dW, float* db, float** scratch, size_t* scratch_cap, int* err,
                cudaStream_t st, const helm_ctx* prof_ctx) {
    if (g_wgrad_path.load() == 0) {
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            sms = 148;
        }
        const WgradGeom geo = wgrad_plan(mode, c0, c1, npad, hin, win, hout, wout, nb, sms);
        if (geo.ktiles > 0) {
            const size_t part = (size_t)geo.splits * 9 * (size_t)(c0 + c1) * npad;
            HELM_TRY(wgrad_scratch(scratch, scratch_cap, part + (size_t)WG_BIAS_SEGMENTS * npad));
            WgradArgs wa;
            wa.x0 = x0; wa.c0 = c0; wa.x1 = x1; wa.c1 = c1; wa.x1_bcast = x1_bcast; wa.x1_map = x1_map; wa.nb1 = nb1;
            wa.nb = nb; wa.hin = hin; wa.win = win; wa.hout = hout; wa.wout = wout; wa.mode = mode;
            wa.g = g; wa.npad = npad; wa.cout = cout; wa.cin = cin; wa.dW = dW; wa.db = db;
            wa.partials = *scratch; wa.max_splits = geo.splits;
            wa.bias_partials = *scratch + part; wa.max_bias_segments = WG_BIAS_SEGMENTS;
            wa.err = err;
            int s;
            {
                LaunchScope scope(prof_ctx, K_WGRAD);
                s = launch_wgrad_tc(wa, st);
            }
            if (s == HELM_OK && prof_ctx && prof_ctx->prof.on) {
                // algorithmic traffic: the layer's inputs and output gradient once, the weight and bias
                // gradients once; flops: 2 x 9 x C_in x C_out per output pixel (logical channels)
                const int nx1 = x1_bcast == 1 ? 1 : nb1;
                const double pin = (double)hin * win, pout = (double)nb * hout * wout;
                const double bytes = 2.0 * pin * ((double)nb * c0 + (double)nx1 * c1) + 2.0 * pout * npad +
                                     4.0 * ((double)cout * 9 * cin + cout);
                prof_add(prof_ctx, K_WGRAD, bytes, 2.0 * 9.0 * cin * cout * pout);
            }
            if (s != HELM_EINVAL) return s;
        }
    }
    // CUDA-core path (and the fallback for a layer the tensor-core kernel does not take)
    WgArgs a;
    a.x0 = x0; a.c0 = c0; a.x1 = x1; a.c1 = c1; a.x1_bcast = x1_bcast; a.x1_map = x1_map;
    a.nb = nb; a.hin = hin; a.win = win; a.hout = hout; a.wout = wout; a.mode = mode;
    a.g = g; a.npad = npad; a.cout = cout; a.cin = cin; a.dW = dW; a.db = db;
    Wg2 w;
    if (mode == 1) { w.th = 4; w.tw = 32; } else { w.th = 8; w.tw = 32; }
    w.tiles_x = (wout + w.tw - 1) / w.tw;
    w.tiles_y = (hout + w.th - 1) / w.th;
    if (mode == 0) { w.sh = w.th + 2; w.sw = w.tw + 2; }
    else if (mode == 1) { w.sh = 2 * w.th + 1; w.sw = 2 * w.tw + 1; }
    else { w.sh = w.th / 2 + 2; w.sw = w.tw / 2 + 2; }
    const size_t np = (size_t)w.th * w.tw;
    const size_t smem = std::max<size_t>(((size_t)(w.sh * w.sw + 1) * 16 + np * 16) * sizeof(float) +
                                             np * 9 * sizeof(int), 32 * 76 * sizeof(float));
    const unsigned gy = (unsigned)((c0 + c1 + 15) / 16), gz = (unsigned)(npad / 16);
    const long long tiles = (long long)nb * w.tiles_x * w.tiles_y;
    const long long gx = std::max<long long>(1, std::min<long long>(tiles, 1216 / (gy * gz)));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    LaunchScope scope(prof_ctx, K_WGRAD);
    { wgrad_kernel<<<dim3((unsigned)gx, gy, gz), 256, smem, st>>>(a, w); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

// target += the input gradient W^T g of one input part (channels off .. off + cp - 1 of the
// layer's padded input) on the tensor cores: 'same' -> same-grid convolution with
// transposed, tap-flipped weights; 'down' -> the transpose-of-down mode; 'up' -> a
// same-grid convolution on the fine grid, then a 2 x 2 sum.  target FP32 [nb][hin][win][cp];
// Wt: scratch of cp x 9 x npad BF16; fine: scratch of nb x hout x wout x cp FP32 (mode 2).
int layer_dgrad(const __nv_bfloat16* g, int npad, const __nv_bfloat16* W, int cin_pad, int off, int cp, int mode,
                int nb, int hin, int win, int hout, int wout, float* target, __nv_bfloat16* Wt, float* fine, int* err,
                cudaStream_t st, const helm_ctx* prof_ctx) {
    {
        LaunchScope scope(prof_ctx, K_CNN_IO);
        { transpose_weights_kernel<<<256, 256, 0, st>>>(W, npad, cin_pad, off, cp, mode == 1 ? 0 : 1, Wt); count_launch(); }
    }
    ConvArgs ca;
    ca.x0 = g; ca.c0 = npad; ca.x1 = nullptr; ca.c1 = 0; ca.x1_bcast = 0; ca.x1_map = nullptr;
    ca.nb = nb; ca.w = Wt; ca.bias = nullptr; ca.res = nullptr; ca.npad = cp; ca.cstore = cp;
    ca.relu = 0; ca.out_fp32 = 1; ca.accum = 1; ca.err = err;
    ca.hin = hout; ca.win = wout;
    if (mode == 0 || mode == 1) {
        ca.hout = hin; ca.wout = win; ca.mode = mode == 0 ? 0 : 3; ca.y = target;
        LaunchScope scope(prof_ctx, K_CONV);
        return launch_conv3x3(ca, st);
    }
    const long long nout = (long long)nb * hout * wout;
    if (cudaMemsetAsync(fine, 0, (size_t)nout * cp * sizeof(float), st) != cudaSuccess) return HELM_ECUDA;
    ca.hout = hout; ca.wout = wout; ca.mode = 0; ca.y = fine;
    int s;
    {
        LaunchScope scope(prof_ctx, K_CONV);
        s = launch_conv3x3(ca, st);
    }
    if (s) return s;
    LaunchScope scope(prof_ctx, K_CNN_IO);
    { sumpool_accum_kernel<<<1184, 256, 0, st>>>(fine, nb, hin, win, cp, target); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

namespace {

// wt[b] = 1 / ||e_b||^2 (one block per sample; FP32 partial sums per thread, FP64
// from the warp sums on); 0 for a zero sample
__global__ void inv_energy_kernel(const float2* __restrict__ e, long long n, float* __restrict__ wt) {
    const int b = blockIdx.x;
    float af = 0.0f;
    for (long long p = threadIdx.x; p < n; p += blockDim.x) {
        const float2 v = e[(long long)b * n + p];
        af = fmaf(v.x, v.x, fmaf(v.y, v.y, af));
    }
    __shared__ double sm[32];
    double acc = warp_sum((double)af);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        wt[b] = t > 0.0 ? (float)(1.0 / t) : 0.0f;
    }
}

// loss = (1/m) sum_b wt_b ||e_net - e_true||^2 with e_net = h^2 rms (o_0 + i o_1)
// (wt = 1: Eq. 4.2; wt_b = 1 / ||e_b||^2: relative error); gout = dloss/do.
// grid (slices, nb): sample b = blockIdx.y; FP32 partial sums per thread, FP64 from
// the warp sums on.
__global__ void mse_grad_kernel(const float* __restrict__ out, const float2* __restrict__ et,
                                const float* __restrict__ rms, const float* __restrict__ wt, float h2, long long n,
                                int nb, float inv_m, float* __restrict__ gout, double* __restrict__ loss) {
    const int b = blockIdx.y;
    const float s = h2 * rms[b];
    const float w = wt ? wt[b] : 1.0f;
    float af = 0.0f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const long long i = (long long)b * n + p;
        const float2 o = reinterpret_cast<const float2*>(out)[i];
        const float2 t = et[i];
        const float dr = s * o.x - t.x, di = s * o.y - t.y;
        af = fmaf(dr, dr, fmaf(di, di, af));
        reinterpret_cast<float2*>(gout)[i] = make_float2(2.0f * inv_m * w * dr * s, 2.0f * inv_m * w * di * s);
    }
    __shared__ double sm[32];
    double acc = (double)w * warp_sum((double)af);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        atomicAdd(loss, t * (double)inv_m);
    }
}

// Adam (Kingma & Ba, Alg. 1) on the flat FP32 parameters; clears the gradient
__global__ void adam_kernel(float* __restrict__ th, float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        g[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// the backward pass over a tape
// ---------------------------------------------------------------------------
class Backward {
   public:
    Backward(cnn_model* m, const helm_ctx* c, cudaStream_t st) : m_(m), c_(c), st_(st) {}

    // gradient buffer of an activation (allocated and zeroed on first use)
    float* grad_of(const void* act, size_t n) {
        auto it = G_.find(act);
        if (it != G_.end()) return it->second;
        float* p = (float*)alloc(n * sizeof(float));
        if (!p) return nullptr;
        if (cudaMemsetAsync(p, 0, n * sizeof(float), st_) != cudaSuccess) ok_ = false;
        G_[act] = p;
        return p;
    }
    void seed(const void* act, float* g) { G_[act] = g; }

    int run(const std::vector<TapeOp>& tape, int nctx) {
        std::unordered_set<const void*> produced;
        for (const TapeOp& op : tape) produced.insert(op.y);
        for (int k = (int)tape.size() - 1; k >= 0 && ok_; --k) {
            const TapeOp& op = tape[k];
            auto it = G_.find(op.y);
            if (it == G_.end()) continue;
            const float* Gy = it->second;
            const Layer& L = m_->layers[op.layer];
            const bool is_out = L.cout < 16;   // the 2-channel output layer (FP32 output, no activation)
            const long long nout = (long long)op.nb * op.hout * op.wout;
            const int cg = is_out ? L.cout : L.npad;
            __nv_bfloat16* g = (__nv_bfloat16*)alloc((size_t)nout * L.npad * sizeof(__nv_bfloat16));
            float* rg = op.res ? grad_of(op.res, (size_t)nout * L.npad) : nullptr;
            if (!ok_) break;
            {
                LaunchScope scope(c_, K_CNN_IO);
                const __nv_bfloat16* ymask = L.relu ? (const __nv_bfloat16*)op.y : nullptr;
                if (cg == L.npad && cg % 8 == 0)
                {
                    const long long hw = (long long)op.hout * op.wout;
                    const long long bx = std::max<long long>(1, std::min<long long>((hw + 255) / 256, 1184 / op.nb));
                    mask_to_bf16_vec_kernel<<<dim3((unsigned)bx, (unsigned)(cg / 8), (unsigned)op.nb), 256, 0, st_>>>(
                        Gy, ymask, L.npad, L.npad, hw, g, rg);
                    count_launch();
                }
                else
                    { mask_to_bf16_kernel<<<1184, 256, 0, st_>>>(Gy, cg, ymask, L.npad, L.npad, nout,
                                                              (long long)op.hout * op.wout, g, rg); count_launch(); }
            }
            // weight and bias gradient
            {
                const int nb1 = op.x1_bcast == 1 ? 1 : (op.x1_bcast == 2 ? nctx : op.nb);
                const int s = layer_wgrad(op.x0, op.c0, op.x1, op.c1, op.x1_bcast, op.zmap, nb1, op.nb, op.hin,
                                          op.win, op.hout, op.wout, L.mode, g, L.npad, L.cout, L.cin,
                                          m_->grad + L.off, m_->grad + L.off + (long long)L.cout * 9 * L.cin,
                                          &m_->wg_scratch, &m_->wg_scratch_n, m_->err, st_, c_);
                if (s != HELM_OK) { ok_ = false; break; }
            }
            if (cudaGetLastError() != cudaSuccess) { ok_ = false; break; }
            // input gradients
            for (int part = 0; part < 2 && ok_; ++part) {
                const __nv_bfloat16* x = part ? op.x1 : op.x0;
                const int cp = part ? op.c1 : op.c0;
                if (!x || cp == 0 || !produced.count(x)) continue;
                const int shared = part == 1 && op.x1_bcast != 0;
                const long long nin = (long long)op.nb * op.hin * op.win;
                __nv_bfloat16* Wt = (__nv_bfloat16*)alloc((size_t)cp * 9 * L.npad * sizeof(__nv_bfloat16));
                if (!ok_) break;
                float* target;
                if (shared) {
                    target = (float*)alloc((size_t)nin * cp * sizeof(float));
                    if (target) cudaMemsetAsync(target, 0, (size_t)nin * cp * sizeof(float), st_);
                } else {
                    target = grad_of(x, (size_t)nin * cp);
                }
                float* fine = L.mode == 2 ? (float*)alloc((size_t)nout * cp * sizeof(float)) : nullptr;
                if (!ok_ || !target) { ok_ = false; break; }
                const int s = layer_dgrad(g, L.npad, L.w, L.cin_pad, part ? op.c0 : 0, cp, L.mode, op.nb, op.hin,
                                          op.win, op.hout, op.wout, target, Wt, fine, m_->err, st_, c_);
                if (s != HELM_OK) { ok_ = false; break; }
                if (shared) {
                    const long long per = (long long)op.hin * op.win * cp;
                    float* gctx = grad_of(x, (size_t)(op.x1_bcast == 1 ? 1 : nctx) * per);
                    if (!gctx) { ok_ = false; break; }
                    LaunchScope scope(c_, K_CNN_IO);
                    { reduce_to_context_kernel<<<1184, 256, 0, st_>>>(target, per, op.nb, op.zmap, op.x1_bcast,
                                                                    op.x1_bcast == 1 ? 1 : nctx, gctx); count_launch(); }
                }
            }
        }
        if (cudaGetLastError() != cudaSuccess) ok_ = false;
        return ok_ ? HELM_OK : HELM_ECUDA;
    }

   private:
    // scratch of the backward pass from the model's arena (the k-th request of a pass reuses
    // the k-th buffer of the previous step: one training step's pass has the same sequence)
    void* alloc(size_t bytes) {
        void* p = arena_buffer(m_->bw_arena, m_->bw_arena_bytes, next_++, bytes);
        if (!p) {
            ok_ = false;
            set_error("out of device memory in the backward pass");
        }
        return p;
    }
    size_t next_ = 0;
    cnn_model* m_;
    const helm_ctx* c_;
    cudaStream_t st_;
    std::unordered_map<const void*, float*> G_;
    bool ok_ = true;
};

int ensure_train_state(cnn_model* m) {
    if (m->grad) return HELM_OK;
    const size_t n = (size_t)m->nparams;
    HELM_CK(cudaMalloc(&m->grad, n * sizeof(float)));
    HELM_CK(cudaMalloc(&m->adam_m, n * sizeof(float)));
    HELM_CK(cudaMalloc(&m->adam_v, n * sizeof(float)));
    m->allocations.push_back(m->grad);
    m->allocations.push_back(m->adam_m);
    m->allocations.push_back(m->adam_v);
    HELM_CK(cudaMemset(m->grad, 0, n * sizeof(float)));
    HELM_CK(cudaMemset(m->adam_m, 0, n * sizeof(float)));
    HELM_CK(cudaMemset(m->adam_v, 0, n * sizeof(float)));
    m->adam_t = 0;
    return HELM_OK;
}

}  // namespace

int cnn_refresh_weights(cnn_model* m, cudaStream_t st);   // cnn.cu
int cnn_encoder_input(const helm_ctx* c, void* out);       // cnn.cu
int cnn_solver_input(const helm_ctx* c, const float2* r, int nb, void* out, float* rms);   // cnn.cu

// Loss (Eq. 4.2) and gradient (accumulated into net->grad) for a batch of
// (residual, error) pairs of the context's medium.
int cnn_loss_grad_impl(cnn_model* m, helm_ctx* c, const float2* r, const float2* e, int nb, double* loss) {
    HELM_TRY(ensure_train_state(m));
    cudaStream_t st = c->stream;
    const long long n = (long long)c->nx * c->nz;
    const int nfreq = c->nfreq;
    int s = HELM_OK;
    auto ck = [&](cudaError_t e2) { if (e2 != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(e2)); s = HELM_ECUDA; } };
    // loss inputs and outputs from the model's arena (slots 2.. ; 0 and 1 hold the batch)
    size_t slot = 2;
    auto io = [&](size_t bytes) -> void* {
        void* p = arena_buffer(m->io_arena, m->io_arena_bytes, slot++, bytes);
        if (!p && s == HELM_OK) { set_error("out of device memory for the training step"); s = HELM_ENOMEM; }
        return p;
    };
    auto* xe = (__nv_bfloat16*)io((size_t)nfreq * n * 16 * sizeof(__nv_bfloat16));
    auto* xs = (__nv_bfloat16*)io((size_t)nb * n * 16 * sizeof(__nv_bfloat16));
    auto* out = (float*)io((size_t)nb * n * 2 * sizeof(float));
    auto* gout = (float*)io((size_t)nb * n * 2 * sizeof(float));
    auto* rms = (float*)io((size_t)nb * sizeof(float));
    auto* wt = m->loss_kind == 1 ? (float*)io((size_t)nb * sizeof(float)) : nullptr;
    auto* dloss = (double*)io(sizeof(double));
    if (!s) ck(cudaMemsetAsync(dloss, 0, sizeof(double), st));
    if (!s) s = cnn_encoder_input(c, xe);
    if (!s) s = cnn_solver_input(c, r, nb, xs, rms);
    std::vector<TapeOp> tape;
    if (!s) {
        Runner run(m, c, st, &m->fw_arena, &m->fw_arena_bytes);   // activations live until the backward pass is done
        run.set_tape(&tape);
        run.set_zmap(c->rhs_freq, c->nfreq);
        std::vector<__nv_bfloat16*> z;
        if (!run.encoder(xe, nfreq, c->nz, c->nx, z)) s = HELM_ECUDA;
        if (!s && !run.solver(xs, nb, c->nz, c->nx, z, 2, out)) s = HELM_ECUDA;
        if (!s) {
            LaunchScope scope(c, K_CNN_IO);
            if (wt) { inv_energy_kernel<<<nb, 256, 0, st>>>(e, n, wt); count_launch(); }
            { mse_grad_kernel<<<dim3((unsigned)std::min<long long>((n + 255) / 256, 128), nb), 256, 0, st>>>(
                out, e, rms, wt, c->hx * c->hz, n, nb, 1.0f / (float)nb, gout,
                                                  dloss); count_launch(); }
            ck(cudaGetLastError());
        }
        if (!s) {
            Backward bw(m, c, st);
            bw.seed(out, gout);
            s = bw.run(tape, nfreq);
            ck(cudaStreamSynchronize(st));
        }
        // (the encoder's context features are arena buffers of the model: nothing to free)
    }
    if (!s) s = check_conv_error(m, st);
    if (!s && loss) ck(cudaMemcpy(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost));
    return s;
}

int cnn_adam_impl(cnn_model* m, float lr, cudaStream_t st) {
    HELM_TRY(ensure_train_state(m));
    m->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - std::pow(b1, (double)m->adam_t));
    const float bc2 = (float)(1.0 - std::pow(b2, (double)m->adam_t));
    { adam_kernel<<<1184, 256, 0, st>>>(m->master, m->grad, m->adam_m, m->adam_v, m->nparams, lr, (float)b1, (float)b2,
                                      1e-8f, bc1, bc2); count_launch(); }
    HELM_CK(cudaGetLastError());
    return cnn_refresh_weights(m, st);
}

}  // namespace helm

using namespace helm;

namespace {

int upload_freqs(helm_ctx* c, const int* freq_idx, int nb) {
    if (nb > c->cap) { set_error("batch larger than the context's max_rhs"); return HELM_EINVAL; }
    std::vector<int> f(nb, 0);
    if (freq_idx)
        for (int i = 0; i < nb; ++i) {
            if (freq_idx[i] < 0 || freq_idx[i] >= c->nfreq) { set_error("freq_idx outside [0, nfreq)"); return HELM_EINVAL; }
            f[i] = freq_idx[i];
        }
    HELM_CK(cudaMemcpyAsync(c->rhs_freq, f.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    HELM_CK(cudaStreamSynchronize(c->stream));
    return HELM_OK;
}

}  // namespace

extern "C" {

int cnn_loss_grad(cnn_model* net, helm_ctx* c, const helm_c64* r, const helm_c64* e, const int* freq_idx, int nb,
                  double* loss, float* grad_out) {
    set_error("");
    if (!net || !c || !r || !e || nb < 1) { set_error("cnn_loss_grad: invalid argument"); return HELM_EINVAL; }
    HELM_TRY(upload_freqs(c, freq_idx, nb));
    HELM_TRY(ensure_train_state(net));
    const size_t n = (size_t)c->nx * c->nz;
    auto* dr = (float2*)arena_buffer(net->io_arena, net->io_arena_bytes, 0, nb * n * sizeof(float2));
    auto* de = (float2*)arena_buffer(net->io_arena, net->io_arena_bytes, 1, nb * n * sizeof(float2));
    if (!dr || !de) { set_error("cnn_loss_grad: out of device memory"); return HELM_ENOMEM; }
    int s = HELM_OK;
    if (cudaMemcpy(dr, r, nb * n * sizeof(float2), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(de, e, nb * n * sizeof(float2), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemsetAsync(net->grad, 0, net->nparams * sizeof(float), c->stream) != cudaSuccess) {
        set_error("cnn_loss_grad: copy failed");
        s = HELM_ECUDA;
    }
    if (!s) s = cnn_loss_grad_impl(net, c, dr, de, nb, loss);
    if (!s && grad_out && cudaMemcpy(grad_out, net->grad, net->nparams * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
        set_error("cnn_loss_grad: gradient copy failed");
        s = HELM_ECUDA;
    }
    return s;
}

int cnn_train_step(cnn_model* net, helm_ctx* c, const helm_c64* r, const helm_c64* e, const int* freq_idx, int nb,
                   float lr, double* loss) {
    int s = cnn_loss_grad(net, c, r, e, freq_idx, nb, loss, nullptr);
    if (s) return s;
    HELM_TRY(cnn_adam_impl(net, lr, c->stream));
    HELM_CK(cudaStreamSynchronize(c->stream));
    // the context's preconditioner sees the updated network: its context features are
    // recomputed before the next use (the loss pass runs its own encoder)
    if (c->net == net) c->cnn_stale = true;
    return HELM_OK;
}

int cnn_adam_reset(cnn_model* net) {
    set_error("");
    if (!net) { set_error("cnn_adam_reset: null network"); return HELM_EINVAL; }
    HELM_TRY(ensure_train_state(net));
    HELM_CK(cudaMemset(net->adam_m, 0, net->nparams * sizeof(float)));
    HELM_CK(cudaMemset(net->adam_v, 0, net->nparams * sizeof(float)));
    HELM_CK(cudaMemset(net->grad, 0, net->nparams * sizeof(float)));
    net->adam_t = 0;
    return HELM_OK;
}

}  // extern "C"

extern "C" int cnn_set_loss(cnn_model* net, int kind) {
    if (!net || (kind != 0 && kind != 1)) {
        helm::set_error("cnn_set_loss: kind must be 0 (Eq. 4.2) or 1 (relative)");
        return HELM_EINVAL;
    }
    net->loss_kind = kind;
    return HELM_OK;
}

extern "C" int cnn_set_wgrad_path(int path) {
    if (path != 0 && path != 1) {
        helm::set_error("cnn_set_wgrad_path: path must be 0 (tensor cores) or 1 (CUDA cores)");
        return HELM_EINVAL;
    }
    helm::g_wgrad_path.store(path);
    return HELM_OK;
}
