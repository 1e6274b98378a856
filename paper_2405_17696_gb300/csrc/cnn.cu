// The encoder-solver network (Fig. 1 caption, Sec. 3.4, Eq. 3.13-3.14, 4.1)
// on the GPU: parameters, forward passes built from the tensor-core 3x3
// convolution, the packing of the network inputs and the unpacking of its
// output, and the network preconditioner M_VU used by helm_solve.
//
// Architecture (L levels, widths c_0..c_{L-1}; the figure is not available,
// the caption is read as follows):
//   ResNet layer R(x) = relu(x + conv_b(relu(conv_a(x))))
//   encoder: in 3->c0, R, R; per level down c_{l-1}->c_l, R, R;
//            up path: up c_{l+1}->c_l, concat with e_l, conv 2c_l->c_l, R  => z_l
//   solver:  in 3->c0, concat z_0, conv 2c0->c0, R; per level down, concat z_l,
//            conv, R; up path: up, concat s_l, conv, R; out conv c0->2.
// Every conv except the second of a ResNet layer (whose ReLU follows the skip
// addition) and the output conv is followed by ReLU.  Parameters are a flat
// FP32 vector, per layer weights [cout][9][cin] then bias [cout], in the
// order encoder then solver as listed above.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "helm_internal.cuh"
#include "cnn_internal.cuh"
#include "conv.cuh"
#include "reduce.cuh"

namespace helm {

int pad16(int c) { return (c + 15) / 16 * 16; }
int npad_of(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : (c <= 64 ? 64 : 128)); }

namespace {

void add_layer(cnn_model* m, const std::string& name, int cin, int cout, int mode, int relu) {
    Layer L;
    L.name = name;
    L.cin = cin;
    L.cout = cout;
    L.mode = mode;
    L.relu = relu;
    L.cin_pad = pad16(cin);
    L.npad = npad_of(cout);
    L.off = m->nparams;
    m->nparams += (long long)cout * 9 * cin + cout;
    m->layers.push_back(L);
}

void build_specs(cnn_model* m) {
    const int L = m->levels;
    const std::vector<int>& c = m->widths;
    auto res = [&](const std::string& p, int ch) {
        add_layer(m, p + ".a", ch, ch, 0, 1);
        add_layer(m, p + ".b", ch, ch, 0, 1);   // ReLU after the skip addition
    };
    add_layer(m, "enc.in", 3, c[0], 0, 1);
    res("enc.r0.0", c[0]);
    res("enc.r0.1", c[0]);
    for (int l = 1; l < L; ++l) {
        add_layer(m, "enc.down" + std::to_string(l), c[l - 1], c[l], 1, 1);
        res("enc.r" + std::to_string(l) + ".0", c[l]);
        res("enc.r" + std::to_string(l) + ".1", c[l]);
    }
    for (int l = L - 2; l >= 0; --l) {
        add_layer(m, "enc.up" + std::to_string(l), c[l + 1], c[l], 2, 1);
        add_layer(m, "enc.cat" + std::to_string(l), 2 * c[l], c[l], 0, 1);
        res("enc.ru" + std::to_string(l), c[l]);
    }
    add_layer(m, "sol.in", 3, c[0], 0, 1);
    add_layer(m, "sol.cat0", 2 * c[0], c[0], 0, 1);
    res("sol.r0", c[0]);
    for (int l = 1; l < L; ++l) {
        add_layer(m, "sol.down" + std::to_string(l), c[l - 1], c[l], 1, 1);
        add_layer(m, "sol.cat" + std::to_string(l), 2 * c[l], c[l], 0, 1);
        res("sol.r" + std::to_string(l), c[l]);
    }
    for (int l = L - 2; l >= 0; --l) {
        add_layer(m, "sol.up" + std::to_string(l), c[l + 1], c[l], 2, 1);
        add_layer(m, "sol.ucat" + std::to_string(l), 2 * c[l], c[l], 0, 1);
        res("sol.ru" + std::to_string(l), c[l]);
    }
    add_layer(m, "sol.out", c[0], 2, 0, 0);
}

template <class T>
int malloc_m(cnn_model* m, T** p, size_t n) {
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("cudaMalloc failed for network storage");
        return HELM_ENOMEM;
    }
    m->allocations.push_back(*p);
    return HELM_OK;
}

// master FP32 [cout][9][cin] + bias -> padded BF16 [npad][9][cin_pad] + FP32 bias [npad]
__global__ void pack_weights_kernel(const float* __restrict__ master, long long off, int cin, int cout, int cin_pad,
                                    int npad, __nv_bfloat16* __restrict__ w, float* __restrict__ b) {
    const int total = npad * 9 * cin_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int ci = i % cin_pad, t = (i / cin_pad) % 9, co = i / (9 * cin_pad);
        float v = (co < cout && ci < cin) ? master[off + ((long long)co * 9 + t) * cin + ci] : 0.0f;
        w[i] = __float2bfloat16_rn(v);
        if (i < npad) b[i] = i < cout ? master[off + (long long)cout * 9 * cin + i] : 0.0f;
    }
}

// master FP32 [cout][9][cin] -> the phase-merged BF16 weights [npad][16][cin_pad] of an up
// layer: row up_merged_index(py, px, dy, dx) holds the sum, in FP32, of the taps (dy, dx) of
// output parity (py, px) that read the same coarse node, rounded once
__global__ void pack_up_weights_kernel(const float* __restrict__ master, long long off, int cin, int cout,
                                       int cin_pad, int npad, __nv_bfloat16* __restrict__ wup) {
    const int total = npad * 16 * cin_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int ci = i % cin_pad, r = (i / cin_pad) % 16, co = i / (16 * cin_pad);
        const int ph = r >> 2;
        float v = 0.0f;
        if (co < cout && ci < cin)
            for (int t = 0; t < 9; ++t)
                if (up_merged_index(ph >> 1, ph & 1, t / 3 - 1, t % 3 - 1) == r)
                    v += master[off + ((long long)co * 9 + t) * cin + ci];
        wup[i] = __float2bfloat16_rn(v);
    }
}

// FP32 [n][ny][nx][3] -> BF16 chunked [n][2][ny][nx][8] (channels 3..15 zero); hw = ny nx
__global__ void pack_input3_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long npix,
                                   long long hw) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        __nv_bfloat16 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16_rn(c < 3 ? in[p * 3 + c] : 0.0f);
        const long long b = p / hw, pix = p - b * hw;
        *reinterpret_cast<uint4*>(out + nc8(b, 0, pix, 16, hw)) = *reinterpret_cast<uint4*>(&v[0]);
        *reinterpret_cast<uint4*>(out + nc8(b, 8, pix, 16, hw)) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// FP32 [n][c] (n pixels, hw per image) -> BF16 chunked [n/hw][cpad/8][hw][8] (channels c..cpad-1 zero)
__global__ void pack_channels_kernel(const float* __restrict__ in, int c, int cpad, __nv_bfloat16* __restrict__ out,
                                     long long n, long long hw) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * cpad;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / cpad;
        const int k = (int)(i - p * cpad);
        const long long b = p / hw, pix = p - b * hw;
        out[nc8(b, k, pix, cpad, hw)] = __float2bfloat16_rn(k < c ? in[p * c + k] : 0.0f);
    }
}

// BF16 chunked (cpad channels) -> FP32 [n][c]
__global__ void unpack_channels_kernel(const __nv_bfloat16* __restrict__ in, int cpad, int c, float* __restrict__ out,
                                       long long n, long long hw) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * c;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / c;
        const int k = (int)(i - p * c);
        const long long b = p / hw, pix = p - b * hw;
        out[i] = __bfloat162float(in[nc8(b, k, pix, cpad, hw)]);
    }
}

}  // namespace

namespace {

// encoder input of every frequency: BF16 chunked [nfreq][2][nz][nx][8] = [c_ref kappa, gamma, w h kappa, 0...]
__global__ void encoder_input_kernel(const float2* __restrict__ mg, const float* __restrict__ omega, float h,
                                     int nfreq, long long n, __nv_bfloat16* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nfreq;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / n);
        const long long p = i - (long long)f * n;
        const float2 kg = mg[p];
        __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.0f);
        v[0] = __float2bfloat16_rn(1500.0f * kg.x);
        v[1] = __float2bfloat16_rn(kg.y);
        v[2] = __float2bfloat16_rn(omega[f] * h * kg.x);
        *reinterpret_cast<uint4*>(out + nc8(f, 0, p, 16, n)) = *reinterpret_cast<uint4*>(&v[0]);
        *reinterpret_cast<uint4*>(out + nc8(f, 8, p, 16, n)) = *reinterpret_cast<uint4*>(&v[8]);
    }
}

// acc[b] += sum over a slice of RHS b of |r|^2 (grid (slices, nb); FP64; acc zeroed before)
__global__ void sumsq_kernel(const float2* __restrict__ r, long long n, const int* mask, double* __restrict__ acc) {
    const int b = blockIdx.y;
    if (mask && !mask[b]) return;
    const float4* rb = reinterpret_cast<const float4*>(r + (long long)b * n);   // n even: two nodes per load
    // FP32 partial sums per thread (a few hundred terms), FP64 from the warp sums on
    float af = 0.0f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n / 2; q += (long long)gridDim.x * blockDim.x) {
        const float4 v = rb[q];
        af = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, af))));
    }
    __shared__ double sm[32];
    double a = warp_sum((double)af);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        atomicAdd(acc + b, t);
    }
}

__global__ void rms_finalize_kernel(const double* __restrict__ acc, long long n, int nb, const int* mask,
                                    float* __restrict__ rms) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) rms[b] = (mask && !mask[b]) ? 0.0f : (float)sqrt(acc[b] / (double)n);
}

// rms(r) per RHS (one block per RHS)
__global__ void rms_kernel(const float2* __restrict__ r, long long n, float* __restrict__ rms, const int* mask) {
    const int b = blockIdx.x;
    if (mask && !mask[b]) { if (threadIdx.x == 0) rms[b] = 0.0f; return; }
    float af = 0.0f;   // FP32 partial sum per thread, FP64 from the warp sums on
    for (long long p = threadIdx.x; p < n; p += blockDim.x) {
        float2 v = r[(long long)b * n + p];
        af = fmaf(v.x, v.x, fmaf(v.y, v.y, af));
    }
    __shared__ double sm[32];
    double acc = warp_sum((double)af);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        rms[b] = (float)sqrt(t / (double)n);
    }
}

// solver input BF16 chunked [nb][2][n][8] = [Re r / rms, Im r / rms, gamma, 0...]; grid
// (slices, nb).  The second plane (channels 8-15) is zero and written only when
// zero_plane1 is set (a buffer that already holds zeros there keeps them).
// Image b of the solver input from RHS idx[b] (idx == nullptr: RHS b).
__global__ void solver_input_kernel(const float2* __restrict__ r, const float* __restrict__ rms,
                                    const float2* __restrict__ mg, long long n, int zero_plane1,
                                    __nv_bfloat16* __restrict__ out, const int* __restrict__ idx) {
    const int b = blockIdx.y;
    const int src = idx ? idx[b] : b;
    const float s = rms[src] > 0.0f ? 1.0f / rms[src] : 0.0f;
    const float2* rb = r + (long long)src * n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const float2 v = rb[p];
        __nv_bfloat16 q[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) q[c] = __float2bfloat16_rn(0.0f);
        q[0] = __float2bfloat16_rn(v.x * s);
        q[1] = __float2bfloat16_rn(v.y * s);
        q[2] = __float2bfloat16_rn(mg[p].y);
        *reinterpret_cast<uint4*>(out + nc8(b, 0, p, 16, n)) = *reinterpret_cast<uint4*>(&q[0]);
        if (zero_plane1) *reinterpret_cast<uint4*>(out + nc8(b, 8, p, 16, n)) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// r' = r - H e0 (FP32, complex64): the residual the network leaves
__global__ void net_residual_kernel(OpFine5 op, const float2* __restrict__ r, const float2* __restrict__ e0,
                                    float2* __restrict__ out, int nb) {
    const long long n = (long long)op.nx * op.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nb;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / n);
        const int p = (int)(i - (long long)b * n);
        const int iz = p / op.nx, ix = p - iz * op.nx;
        const float2 he = op.apply(e0 + (long long)b * n, b, ix, iz);
        out[i] = make_float2(r[i].x - he.x, r[i].y - he.y);
    }
}

// z += e0
// Guarded composition: per RHS, t = H e0 and acc[b] = {Re <t, r>, Im <t, r>, <t, t>}
// (FP32 partial sums per thread, FP64 from the warp sums on; blocks of a RHS add
// their sums atomically; acc zeroed before).  Block x takes grid rows x, x + gridDim.x, ...
// A RHS that is not guarded (guard non-null and guard[b] = 0) takes a = 1 and
// needs no sums.
__global__ void net_scale_dots_kernel(OpFine5 op, const float2* __restrict__ r, const float2* __restrict__ e0,
                                      const int* mask, const int* guard, double* __restrict__ acc) {
    const int b = blockIdx.y;
    if ((mask && !mask[b]) || (guard && !guard[b])) return;
    const long long n = (long long)op.nx * op.nz;
    const float2* eb = e0 + (long long)b * n;
    const float2* rb = r + (long long)b * n;
    float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
    for (int iz = blockIdx.x; iz < op.nz; iz += gridDim.x)
        for (int ix = threadIdx.x; ix < op.nx; ix += blockDim.x) {
            const float2 t = op.apply(eb, b, ix, iz);
            const float2 v = rb[(long long)iz * op.nx + ix];
            f0 += t.x * v.x + t.y * v.y;
            f1 += t.x * v.y - t.y * v.x;
            f2 += t.x * t.x + t.y * t.y;
        }
    __shared__ double sm[3][32];
    double a0 = warp_sum((double)f0);
    double a1 = warp_sum((double)f1);
    double a2 = warp_sum((double)f2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sm[0][w] = a0; sm[1][w] = a1; sm[2][w] = a2; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[threadIdx.x][k];
        atomicAdd(acc + 3 * b + threadIdx.x, t);
    }
}

// a = 1 unless the RHS is guarded (guard == nullptr: always) and the network's step
// raises the residual (||r - t|| > ||r||, i.e. <t, t> > 2 Re <t, r>); then the
// a = <t, r> / <t, t> that minimises ||r - a t||
__device__ __forceinline__ float2 net_alpha(const double* acc, const int* guard, int b) {
    if (guard && !guard[b]) return make_float2(1.f, 0.f);
    const double tr = acc[3 * b], tt = acc[3 * b + 2];
    if (tt <= 2.0 * tr) return make_float2(1.f, 0.f);
    return tt > 0.0 ? make_float2((float)(tr / tt), (float)(acc[3 * b + 1] / tt)) : make_float2(0.f, 0.f);
}

// out = r - a_b H e0 on node pairs (ix, ix + 1), ix even (16-byte access; nx even);
// RHS with a zero mask entry are skipped.  grid (x tiles of 32 pairs, z rows / 8, nb), block (32, 8)
__global__ void net_scaled_residual2_kernel(OpFine5 op, const float2* __restrict__ r, const float2* __restrict__ e0,
                                            float2* __restrict__ out, const double* __restrict__ acc,
                                            const int* guard, const int* mask) {
    const int b = blockIdx.z;
    if (mask && !mask[b]) return;
    const int ix = 2 * (blockIdx.x * blockDim.x + threadIdx.x), iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= op.nx || iz >= op.nz) return;
    const long long n = (long long)op.nx * op.nz;
    const long long i = (long long)b * n + (long long)iz * op.nx + ix;
    float2 h0, h1;
    op.apply2(e0 + (long long)b * n, b, ix, iz, h0, h1);
    const float2 al = net_alpha(acc, guard, b);
    const float4 rv = *reinterpret_cast<const float4*>(r + i);
    *reinterpret_cast<float4*>(out + i) =
        make_float4(rv.x - (al.x * h0.x - al.y * h0.y), rv.y - (al.x * h0.y + al.y * h0.x),
                    rv.z - (al.x * h1.x - al.y * h1.y), rv.w - (al.x * h1.y + al.y * h1.x));
}

// out = r - a_b H e0 (any nx); grid (x tiles of 32, z rows / 8, nb), block (32, 8)
__global__ void net_scaled_residual_kernel(OpFine5 op, const float2* __restrict__ r, const float2* __restrict__ e0,
                                           float2* __restrict__ out, const double* __restrict__ acc,
                                           const int* guard, const int* mask) {
    const int b = blockIdx.z;
    if (mask && !mask[b]) return;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= op.nx || iz >= op.nz) return;
    const long long n = (long long)op.nx * op.nz;
    const long long i = (long long)b * n + (long long)iz * op.nx + ix;
    const float2 he = op.apply(e0 + (long long)b * n, b, ix, iz);
    const float2 al = net_alpha(acc, guard, b);
    out[i] = make_float2(r[i].x - (al.x * he.x - al.y * he.y), r[i].y - (al.x * he.y + al.y * he.x));
}

// z += a_b e0 on node pairs (n even); RHS with a zero mask entry are skipped; grid (slices, nb)
__global__ void add_scaled_kernel(float2* __restrict__ z, const float2* __restrict__ e0, long long n,
                                  const double* __restrict__ acc, const int* guard, const int* mask) {
    const int b = blockIdx.y;
    if (mask && !mask[b]) return;
    const float2 al = net_alpha(acc, guard, b);
    float4* zb = reinterpret_cast<float4*>(z + (long long)b * n);
    const float4* eb = reinterpret_cast<const float4*>(e0 + (long long)b * n);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n / 2;
         p += (long long)gridDim.x * blockDim.x) {
        const float4 e = eb[p];
        const float4 v = zb[p];
        zb[p] = make_float4(v.x + al.x * e.x - al.y * e.y, v.y + al.x * e.y + al.y * e.x,
                            v.z + al.x * e.z - al.y * e.w, v.w + al.x * e.w + al.y * e.z);
    }
}

__global__ void add_kernel(float2* __restrict__ z, const float2* __restrict__ e0, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = make_float2(z[i].x + e0[i].x, z[i].y + e0[i].y);
}

// e0 = h^2 rms (out_0 + i out_1)
// e0 = h^2 rms (o_0 + i o_1); grid (slices, nb)
// Image b of the solver output to RHS idx[b] (idx == nullptr: RHS b).
__global__ void solver_output_kernel(const float* __restrict__ out, const float* __restrict__ rms, float h2,
                                     long long n, float2* __restrict__ e0, const int* __restrict__ idx) {
    const int b = blockIdx.y;
    const int dst = idx ? idx[b] : b;
    const float s = h2 * rms[dst];
    const float2* ob = reinterpret_cast<const float2*>(out) + (long long)b * n;
    float2* eb = e0 + (long long)dst * n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const float2 o = ob[p];
        eb[p] = make_float2(s * o.x, s * o.y);
    }
}

}  // namespace

// Rebuild the padded BF16 weights from the FP32 master parameters.
int cnn_refresh_weights(cnn_model* m, cudaStream_t st) {
    for (const Layer& l : m->layers) {
        { pack_weights_kernel<<<64, 256, 0, st>>>(m->master, l.off, l.cin, l.cout, l.cin_pad, l.npad, l.w, l.b); count_launch(); }
        if (l.wup) { pack_up_weights_kernel<<<64, 256, 0, st>>>(m->master, l.off, l.cin, l.cout, l.cin_pad, l.npad, l.wup); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    return HELM_OK;
}

// Encoder input of every frequency of the context, BF16 [nfreq][nz][nx][16].
int cnn_encoder_input(const helm_ctx* c, void* out) {
    const long long n = (long long)c->nx * c->nz;
    LaunchScope scope(c, K_CNN_IO);
    { encoder_input_kernel<<<1184, 256, 0, c->stream>>>(c->mg, c->omega_d, std::sqrt(c->hx * c->hz), c->nfreq, n, (__nv_bfloat16*)out); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

// Solver input of nb residuals, BF16 [nb][nz][nx][16], and rms(r) per residual.
int cnn_solver_input(const helm_ctx* c, const float2* r, int nb, void* out, float* rms) {
    const long long n = (long long)c->nx * c->nz;
    {
        LaunchScope scope(c, K_CNN_IO);
        { rms_kernel<<<nb, 1024, 0, c->stream>>>(r, n, rms, nullptr); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    LaunchScope scope(c, K_CNN_IO);
    { solver_input_kernel<<<dim3((unsigned)std::min<long long>((n + 255) / 256, 512), nb), 256, 0, c->stream>>>(
        r, rms, c->mg, n, 1, (__nv_bfloat16*)out, nullptr); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

void cnn_ctx_free(helm_ctx* c) {
    for (void* p : c->cnn_z) cudaFree(p);
    c->cnn_z.clear();
    for (void* p : c->cnn_arena) cudaFree(p);
    c->cnn_arena.clear();
    c->cnn_arena_bytes.clear();
    cudaFree(c->cnn_in);
    cudaFree(c->cnn_out);
    cudaFree(c->cnn_e0);
    cudaFree(c->cnn_rres);
    cudaFree(c->cnn_rms);
    cudaFree(c->cnn_alpha);
    cudaFree(c->cnn_idx);
    cudaFree(c->cnn_zmapc);
    cudaFreeHost(c->cnn_idx_host);
    cudaFreeHost(c->cnn_act_host);
    c->cnn_idx = c->cnn_zmapc = c->cnn_idx_host = c->cnn_act_host = nullptr;
    c->cnn_nact = -1;
    c->cnn_alpha = nullptr;
    c->cnn_rres = nullptr;
    c->cnn_in = nullptr;
    c->cnn_out = nullptr;
    c->cnn_e0 = nullptr;
    c->cnn_rms = nullptr;
}

int cnn_ctx_setup(helm_ctx* c) {
    cnn_model* m = c->net;
    const int div = 1 << (m->levels - 1);
    if (c->nx % div || c->nz % div) {
        set_error("grid not divisible by 2^(network levels - 1)");
        return HELM_EINVAL;
    }
    const long long n = (long long)c->nx * c->nz;
    if (!c->cnn_in) {
        HELM_CK(cudaMalloc(&c->cnn_in, (size_t)std::max<long long>(c->cap, c->nfreq) * n * 16 * sizeof(__nv_bfloat16)));
        // the solver input writes only its first 8-channel plane; the second stays zero
        HELM_CK(cudaMemset(c->cnn_in, 0, (size_t)std::max<long long>(c->cap, c->nfreq) * n * 16 * sizeof(__nv_bfloat16)));
        HELM_CK(cudaMalloc(&c->cnn_out, (size_t)c->cap * n * 2 * sizeof(float)));
        HELM_CK(cudaMalloc(&c->cnn_e0, (size_t)c->cap * n * sizeof(float2)));
        HELM_CK(cudaMalloc(&c->cnn_rres, (size_t)c->cap * n * sizeof(float2)));
        HELM_CK(cudaMalloc(&c->cnn_rms, (size_t)c->cap * sizeof(float)));
        HELM_CK(cudaMalloc(&c->cnn_alpha, (size_t)c->cap * 3 * sizeof(double)));
        HELM_CK(cudaMalloc(&c->cnn_idx, (size_t)c->cap * sizeof(int)));
        HELM_CK(cudaMalloc(&c->cnn_zmapc, (size_t)c->cap * sizeof(int)));
        HELM_CK(cudaMallocHost(&c->cnn_idx_host, (size_t)c->cap * sizeof(int)));
        HELM_CK(cudaMallocHost(&c->cnn_act_host, (size_t)c->cap * sizeof(int)));
    }
    for (void* p : c->cnn_z) cudaFree(p);
    c->cnn_z.clear();
    {
        LaunchScope scope(c, K_CNN_IO);
        { encoder_input_kernel<<<1184, 256, 0, c->stream>>>(c->mg, c->omega_d, std::sqrt(c->hx * c->hz), c->nfreq, n,
                                                          (__nv_bfloat16*)c->cnn_in); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    Runner r(m, c, c->stream);
    std::vector<__nv_bfloat16*> z;
    if (!r.encoder((const __nv_bfloat16*)c->cnn_in, c->nfreq, c->nz, c->nx, z)) {
        if (std::string(helm_last_error()).empty()) set_error("encoder pass failed");
        return HELM_ECUDA;
    }
    for (__nv_bfloat16* p : z) c->cnn_z.push_back(p);
    HELM_CK(cudaStreamSynchronize(c->stream));
    return check_conv_error(m, c->stream);
}

__global__ void gather_int_kernel(const int* __restrict__ src, const int* __restrict__ idx, int n,
                                  int* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// After a restart check: list the RHS whose outer iteration is still running
// (flags already copied to cnn_act_host and the stream synchronised) so that the
// next cycle's network passes take only those.
int cnn_ctx_compact(helm_ctx* c, int nb) {
    c->cnn_nact = -1;
    if (!c->net || !c->cnn_idx_host || !c->cnn_act_host) return HELM_OK;
    int n = 0;
    for (int b = 0; b < nb; ++b)
        if (c->cnn_act_host[b]) c->cnn_idx_host[n++] = b;
    if (n == 0 || n == nb) return HELM_OK;
    HELM_CK(cudaMemcpyAsync(c->cnn_idx, c->cnn_idx_host, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    { gather_int_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(c->rhs_freq, c->cnn_idx, n, c->cnn_zmapc); count_launch(); }
    HELM_CK(cudaGetLastError());
    c->cnn_nact = n;
    return HELM_OK;
}

int cnn_ctx_precondition(helm_ctx* c, float2* z, const float2* v, int nb, const int* mask, int with_vcycle) {
    // context features computed with the network's current weights (stale after training steps)
    if (c->cnn_stale) {
        HELM_TRY(cnn_ctx_setup(c));
        c->cnn_stale = false;
    }
    cnn_model* m = c->net;
    const long long n = (long long)c->nx * c->nz;
    {
        LaunchScope scope(c, K_CNN_IO);
        // sum of |r|^2 per RHS into the scaled composition's sums (reset before they are used)
        HELM_CK(cudaMemsetAsync(c->cnn_alpha, 0, (size_t)nb * sizeof(double), c->stream));
        { sumsq_kernel<<<dim3(32, nb), 256, 0, c->stream>>>(v, n, mask, c->cnn_alpha); count_launch(); }
        { rms_finalize_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(c->cnn_alpha, n, nb, mask, c->cnn_rms); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    const dim3 g2((unsigned)std::min<long long>((n + 255) / 256, 512), nb);
    // inside FGMRES (mask = the cycle's active flags) only the RHS still iterating at
    // the last restart go through the network; the others keep a stale e0 that the
    // masked kernels below never read
    const bool compact = mask == c->fine.active && c->cnn_nact > 0 && c->cnn_nact < nb;
    const int nnet = compact ? c->cnn_nact : nb;
    const int* idx = compact ? c->cnn_idx : nullptr;
    const dim3 gn(g2.x, (unsigned)nnet);
    {
        LaunchScope scope(c, K_CNN_IO);
        { solver_input_kernel<<<gn, 256, 0, c->stream>>>(v, c->cnn_rms, c->mg, n, 0, (__nv_bfloat16*)c->cnn_in, idx); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    Runner r(m, c, c->stream, &c->cnn_arena, &c->cnn_arena_bytes);
    r.set_zmap(compact ? c->cnn_zmapc : c->rhs_freq, c->nfreq);
    std::vector<__nv_bfloat16*> zz;
    for (void* p : c->cnn_z) zz.push_back((__nv_bfloat16*)p);
    if (!r.solver((const __nv_bfloat16*)c->cnn_in, nnet, c->nz, c->nx, zz, 2, c->cnn_out)) {
        if (std::string(helm_last_error()).empty()) set_error("solver pass failed");
        return HELM_ECUDA;
    }
    {
        LaunchScope scope(c, K_CNN_IO);
        float2* e0 = with_vcycle ? c->cnn_e0 : z;
        { solver_output_kernel<<<gn, 256, 0, c->stream>>>(c->cnn_out, c->cnn_rms, c->hx * c->hz, n, e0, idx); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    if (!with_vcycle) return HELM_OK;
    if (c->opt.cnn_vcycle == 1)
        return vcycle_apply(c, z, c->cnn_e0, v, nb, mask);   // V-cycle on P u = r from u0 = e_0
    float2* rr = c->cnn_rres;
    const bool scaled = c->opt.cnn_vcycle >= 2;
    // composition 2: guarded only for RHS whose restart cycles stall; 3: always guarded
    const int* guard = c->opt.cnn_vcycle == 2 ? c->outer.guard : nullptr;
    if (scaled) {
        // a e_0 + V(r - a H e_0): a = 1 unless the network's step would raise the
        // residual the V-cycle sees, then the a that minimises it (per RHS)
        double* acc = c->cnn_alpha;
        LaunchScope scope(c, K_CNN_IO);
        HELM_CK(cudaMemsetAsync(acc, 0, (size_t)3 * nb * sizeof(double), c->stream));
        { net_scale_dots_kernel<<<dim3(64, nb), 256, 0, c->stream>>>(fine_op(c, 0), v, c->cnn_e0, mask, guard, acc); count_launch(); }
        if (c->nx % 2 == 0)
            { net_scaled_residual2_kernel<<<dim3((c->nx / 2 + 31) / 32, (c->nz + 7) / 8, nb), dim3(32, 8), 0,
                                          c->stream>>>(fine_op(c, 0), v, c->cnn_e0, rr, acc, guard, mask); count_launch(); }
        else
            { net_scaled_residual_kernel<<<dim3((c->nx + 31) / 32, (c->nz + 7) / 8, nb), dim3(32, 8), 0, c->stream>>>(
                fine_op(c, 0), v, c->cnn_e0, rr, acc, guard, mask); count_launch(); }
        HELM_CK(cudaGetLastError());
    } else {
        // e_0 + V(r - H e_0): the V-cycle corrects what the network leaves of H e = r
        LaunchScope scope(c, K_CNN_IO);
        { net_residual_kernel<<<1184, 256, 0, c->stream>>>(fine_op(c, 0), v, c->cnn_e0, rr, nb); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    HELM_TRY(vcycle_apply(c, z, nullptr, rr, nb, mask));
    LaunchScope scope(c, K_CNN_IO);
    if (scaled)
        { add_scaled_kernel<<<g2, 256, 0, c->stream>>>(z, c->cnn_e0, n, c->cnn_alpha, guard, mask); count_launch(); }
    else
        { add_kernel<<<1184, 256, 0, c->stream>>>(z, c->cnn_e0, n * nb); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

}  // namespace helm

namespace helm {
namespace {

// Timing input of the autotuner: unit-scale values from a hash of the index.
__global__ void synth_residual_kernel(float2* __restrict__ r, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float a = (float)(z & 0xFFFFFFu) * (1.0f / 16777216.0f) - 0.5f;
        const float b = (float)((z >> 24) & 0xFFFFFFu) * (1.0f / 16777216.0f) - 0.5f;
        r[i] = make_float2(a, b);
    }
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

int cnn_precond_apply(helm_ctx* c, const helm_c64* r, helm_c64* e, int nrhs, const int* freq_idx, int with_vcycle) {
    set_error("");
    if (!c || !r || !e || nrhs < 0 || !c->net) {
        set_error("cnn_precond_apply: invalid argument or no network in the context");
        return HELM_EINVAL;
    }
    const size_t N = (size_t)c->nx * c->nz;
    for (int b0 = 0; b0 < nrhs; b0 += c->cap) {
        const int nb = nrhs - b0 < c->cap ? nrhs - b0 : c->cap;
        std::vector<int> f(nb, 0);
        if (freq_idx)
            for (int i = 0; i < nb; ++i) {
                if (freq_idx[b0 + i] < 0 || freq_idx[b0 + i] >= c->nfreq) { set_error("freq_idx outside [0, nfreq)"); return HELM_EINVAL; }
                f[i] = freq_idx[b0 + i];
            }
        HELM_CK(cudaMemcpyAsync(c->rhs_freq, f.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        float2 *dr = nullptr, *de = nullptr;
        HELM_CK(cudaMalloc(&dr, nb * N * sizeof(float2)));
        HELM_CK(cudaMalloc(&de, nb * N * sizeof(float2)));
        HELM_CK(cudaMemcpyAsync(dr, r + b0 * N, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
        // outside a solve no restart cycle has stalled: composition 2 is the plain one
        HELM_CK(cudaMemsetAsync(c->outer.guard, 0, nb * sizeof(int), c->stream));
        int s = cnn_ctx_precondition(c, de, dr, nb, c->ones, with_vcycle);
        if (!s) {
            cudaError_t ce = cudaMemcpyAsync(e + b0 * N, de, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream);
            if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); s = HELM_ECUDA; }
        }
        cudaError_t ce = cudaStreamSynchronize(c->stream);
        cudaFree(dr);
        cudaFree(de);
        if (s) return s;
        if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return HELM_ECUDA; }
        HELM_TRY(check_conv_error(c->net, c->stream));
    }
    return HELM_OK;
}


int cnn_autotune(helm_ctx* c, int nrhs, int* n_shapes) {
    set_error("");
    if (!c || !c->net || nrhs < 1 || nrhs > c->cap) {
        set_error("cnn_autotune: needs a context with a network and 1 <= nrhs <= max_rhs");
        return HELM_EINVAL;
    }
    const long long n = (long long)npts(c) * nrhs;
    float2 *r = nullptr, *e = nullptr;
    HELM_CK(cudaMalloc(&r, n * sizeof(float2)));
    if (cudaMalloc(&e, n * sizeof(float2)) != cudaSuccess) {
        cudaFree(r);
        set_error("cnn_autotune: out of device memory");
        return HELM_ENOMEM;
    }
    { synth_residual_kernel<<<1184, 256, 0, c->stream>>>(r, n); count_launch(); }
    int s = cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_ECUDA;
    if (!s) {
        conv_tuning(true);
        s = cnn_ctx_precondition(c, e, r, nrhs, c->ones, 0);
        conv_tuning(false);
    }
    const cudaError_t ce = cudaStreamSynchronize(c->stream);
    cudaFree(r);
    cudaFree(e);
    if (s) return s;
    if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return HELM_ECUDA; }
    HELM_TRY(check_conv_error(c->net, c->stream));
    if (n_shapes) *n_shapes = conv_tuned_count();
    return HELM_OK;
}

void cnn_autotune_reset(void) { conv_tune_reset(); }

namespace {
// the network without initial weights (all zero)
int create_zero(cnn_model** out, int levels, const int* widths) {
    if (!out || levels < 2 || levels > 6 || !widths) { set_error("cnn_create: invalid argument"); return HELM_EINVAL; }
    for (int l = 0; l < levels; ++l)
        if (widths[l] < 16 || widths[l] > 128 || widths[l] % 16) {
            set_error("cnn_create: widths must be multiples of 16 in [16, 128]");
            return HELM_EINVAL;
        }
    cnn_model* m = new cnn_model();
    m->levels = levels;
    m->widths.assign(widths, widths + levels);
    build_specs(m);
    int s = malloc_m(m, &m->master, (size_t)m->nparams);
    if (!s) s = malloc_m(m, &m->err, 1);
    for (Layer& l : m->layers) {
        if (s) break;
        s = malloc_m(m, &l.w, (size_t)l.npad * 9 * l.cin_pad);
        if (!s && l.mode == 2) s = malloc_m(m, &l.wup, (size_t)l.npad * 16 * l.cin_pad);
        if (!s) s = malloc_m(m, &l.b, (size_t)l.npad);
    }
    if (s) { cnn_destroy(m); return s; }
    cudaMemset(m->master, 0, m->nparams * sizeof(float));
    cudaMemset(m->err, 0, sizeof(int));
    for (Layer& l : m->layers) {
        cudaMemset(l.w, 0, (size_t)l.npad * 9 * l.cin_pad * sizeof(__nv_bfloat16));
        if (l.wup) cudaMemset(l.wup, 0, (size_t)l.npad * 16 * l.cin_pad * sizeof(__nv_bfloat16));
        cudaMemset(l.b, 0, (size_t)l.npad * sizeof(float));
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { set_error("cnn_create: device error"); cnn_destroy(m); return HELM_ECUDA; }
    *out = m;
    return HELM_OK;
}
}  // namespace

int cnn_create(cnn_model** out, int levels, const int* widths, unsigned long long seed) {
    set_error("");
    cnn_model* m = nullptr;
    HELM_TRY(create_zero(&m, levels, widths));
    const int s = cnn_init_params(m, seed, 0.5f);
    if (s) {
        cnn_destroy(m);
        return s;
    }
    *out = m;
    return HELM_OK;
}

void cnn_destroy(cnn_model* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    if (m->wg_scratch) cudaFree(m->wg_scratch);
    for (auto* a : {&m->fw_arena, &m->bw_arena, &m->io_arena})
        for (void* p : *a)
            if (p) cudaFree(p);
    for (void* p : m->allocations) cudaFree(p);
    delete m;
}

long long cnn_num_params(const cnn_model* m) { return m ? m->nparams : -1; }

int cnn_set_params(cnn_model* m, const float* params, long long n) {
    set_error("");
    if (!m || !params || n != m->nparams) { set_error("cnn_set_params: size differs from cnn_num_params"); return HELM_EINVAL; }
    HELM_CK(cudaMemcpy(m->master, params, n * sizeof(float), cudaMemcpyDefault));
    HELM_TRY(cnn_refresh_weights(m, nullptr));
    HELM_CK(cudaDeviceSynchronize());
    return HELM_OK;
}

// He-normal initial weights (std = gain * sqrt(2 / (9 C_in))), zero biases.
// Normal draws: Box-Muller on two uniforms from splitmix64 (Steele, Lea and
// Flood 2014) started at `seed`; the same values on every platform.
int cnn_init_params(cnn_model* m, unsigned long long seed, float gain) {
    set_error("");
    if (!m || !(gain > 0.0f)) { set_error("cnn_init_params: null model or gain <= 0"); return HELM_EINVAL; }
    unsigned long long state = seed;
    auto next = [&state]() {
        unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uniform = [&]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };   // (0, 1)
    std::vector<float> h((size_t)m->nparams, 0.0f);
    for (const Layer& l : m->layers) {
        const double sd = gain * std::sqrt(2.0 / (9.0 * l.cin));
        const long long nw = (long long)l.cout * 9 * l.cin;
        for (long long i = 0; i < nw; i += 2) {
            const double u1 = uniform(), u2 = uniform();
            const double r = std::sqrt(-2.0 * std::log(u1)), t = 6.283185307179586 * u2;
            h[(size_t)(l.off + i)] = (float)(sd * r * std::cos(t));
            if (i + 1 < nw) h[(size_t)(l.off + i + 1)] = (float)(sd * r * std::sin(t));
        }
    }
    HELM_CK(cudaMemcpy(m->master, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    HELM_TRY(cnn_refresh_weights(m, nullptr));
    HELM_CK(cudaDeviceSynchronize());
    return HELM_OK;
}

int cnn_get_params(const cnn_model* m, float* params, long long n) {
    set_error("");
    if (!m || !params || n != m->nparams) { set_error("cnn_get_params: size differs from cnn_num_params"); return HELM_EINVAL; }
    HELM_CK(cudaMemcpy(params, m->master, n * sizeof(float), cudaMemcpyDefault));
    return HELM_OK;
}

// Raw network forward for parity tests and offline use: FP32 inputs are
// rounded to BF16, the network runs on the tensor cores, output FP32.
//   enc_in : [nenc][ny][nx][3]   sol_in : [nsol][ny][nx][3]   out : [nsol][ny][nx][2]
//   the solver images share encoder image 0 when nenc == 1, else image i uses encoder image i.
int cnn_forward(cnn_model* m, const float* enc_in, int nenc, const float* sol_in, int nsol, int ny, int nx,
                float* out) {
    set_error("");
    if (!m || !enc_in || !sol_in || !out || nenc < 1 || nsol < 1 || (nenc != 1 && nenc != nsol)) {
        set_error("cnn_forward: invalid argument");
        return HELM_EINVAL;
    }
    const int div = 1 << (m->levels - 1);
    if (ny % div || nx % div) { set_error("cnn_forward: ny, nx must be divisible by 2^(levels-1)"); return HELM_EINVAL; }
    cudaStream_t st = nullptr;
    const size_t npix = (size_t)ny * nx;
    float *ein = nullptr, *sin_ = nullptr, *o = nullptr;
    __nv_bfloat16 *xe = nullptr, *xs = nullptr;
    int s = HELM_OK;
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; } };
    ck(cudaMalloc(&ein, nenc * npix * 3 * sizeof(float)));
    ck(cudaMalloc(&sin_, nsol * npix * 3 * sizeof(float)));
    ck(cudaMalloc(&o, nsol * npix * 2 * sizeof(float)));
    ck(cudaMalloc(&xe, nenc * npix * 16 * sizeof(__nv_bfloat16)));
    ck(cudaMalloc(&xs, nsol * npix * 16 * sizeof(__nv_bfloat16)));
    if (!s) {
        ck(cudaMemcpy(ein, enc_in, nenc * npix * 3 * sizeof(float), cudaMemcpyDefault));
        ck(cudaMemcpy(sin_, sol_in, nsol * npix * 3 * sizeof(float), cudaMemcpyDefault));
        { pack_input3_kernel<<<256, 256>>>(ein, xe, (long long)nenc * npix, (long long)npix); count_launch(); }
        { pack_input3_kernel<<<256, 256>>>(sin_, xs, (long long)nsol * npix, (long long)npix); count_launch(); }
        ck(cudaGetLastError());
    }
    if (!s) {
        Runner r(m, nullptr, st);
        std::vector<__nv_bfloat16*> z;
        if (!r.encoder(xe, nenc, ny, nx, z)) s = HELM_ECUDA;
        if (!s && !r.solver(xs, nsol, ny, nx, z, nenc == 1 ? 1 : 0, o)) s = HELM_ECUDA;
        ck(cudaDeviceSynchronize());
        for (__nv_bfloat16* p : z) cudaFree(p);
        if (!s) s = check_conv_error(m, st);
    }
    if (!s) ck(cudaMemcpy(out, o, nsol * npix * 2 * sizeof(float), cudaMemcpyDefault));
    cudaFree(ein); cudaFree(sin_); cudaFree(o); cudaFree(xe); cudaFree(xs);
    return s;
}

// One 3x3 convolution layer as the network uses it: FP32 in/out (host or device),
// BF16 operands and FP32 accumulation on the tensor cores.
int cnn_conv3x3(const float* x0, int c0, const float* x1, int c1, int x1_bcast, int nb, int hin, int win,
                const float* w, const float* bias, int cout, const float* res, int mode, int relu, float* y) {
    set_error("");
    if (!x0 || !w || !bias || !y || c0 < 1 || c1 < 0 || (c1 > 0 && !x1) || nb < 1 || hin < 1 || win < 1 ||
        cout < 1 || cout > 128 || mode < 0 || mode > 2) {
        set_error("cnn_conv3x3: invalid argument");
        return HELM_EINVAL;
    }
    const int cp0 = pad16(c0), cp1 = c1 ? pad16(c1) : 0, cin = c0 + c1, cinp = cp0 + cp1, npad = npad_of(cout);
    const int hout = mode == 1 ? hin / 2 : (mode == 2 ? 2 * hin : hin);
    const int wout = mode == 1 ? win / 2 : (mode == 2 ? 2 * win : win);
    const long long nin = (long long)nb * hin * win, nin1 = (long long)(x1_bcast ? 1 : nb) * hin * win;
    const long long nout = (long long)nb * hout * wout;
    float *fx0 = nullptr, *fx1 = nullptr, *fw = nullptr, *fb = nullptr, *fr = nullptr, *fy = nullptr, *bp = nullptr;
    __nv_bfloat16 *bx0 = nullptr, *bx1 = nullptr, *bw = nullptr, *bwup = nullptr, *br = nullptr, *by = nullptr;
    int* err = nullptr;
    int s = HELM_OK;
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; } };
    ck(cudaMalloc(&fx0, nin * c0 * sizeof(float)));
    ck(cudaMalloc(&bx0, nin * cp0 * sizeof(__nv_bfloat16)));
    if (c1) { ck(cudaMalloc(&fx1, nin1 * c1 * sizeof(float))); ck(cudaMalloc(&bx1, nin1 * cp1 * sizeof(__nv_bfloat16))); }
    ck(cudaMalloc(&fw, (size_t)cout * 9 * cin * sizeof(float) + cout * sizeof(float)));
    ck(cudaMalloc(&bw, (size_t)npad * 9 * cinp * sizeof(__nv_bfloat16)));
    if (mode == 2) ck(cudaMalloc(&bwup, (size_t)npad * 16 * cinp * sizeof(__nv_bfloat16)));
    ck(cudaMalloc(&bp, npad * sizeof(float)));
    ck(cudaMalloc(&fy, nout * cout * sizeof(float)));
    ck(cudaMalloc(&by, nout * npad * sizeof(__nv_bfloat16)));
    ck(cudaMalloc(&err, sizeof(int)));
    if (res) { ck(cudaMalloc(&fr, nout * cout * sizeof(float))); ck(cudaMalloc(&br, nout * npad * sizeof(__nv_bfloat16))); }
    if (!s) {
        ck(cudaMemset(err, 0, sizeof(int)));
        ck(cudaMemcpy(fx0, x0, nin * c0 * sizeof(float), cudaMemcpyDefault));
        if (c1) ck(cudaMemcpy(fx1, x1, nin1 * c1 * sizeof(float), cudaMemcpyDefault));
        ck(cudaMemcpy(fw, w, (size_t)cout * 9 * cin * sizeof(float), cudaMemcpyDefault));
        ck(cudaMemcpy(fw + (size_t)cout * 9 * cin, bias, cout * sizeof(float), cudaMemcpyDefault));
        if (res) ck(cudaMemcpy(fr, res, nout * cout * sizeof(float), cudaMemcpyDefault));
    }
    if (!s) {
        const long long hwi = (long long)hin * win, hwo = (long long)hout * wout;
        { pack_channels_kernel<<<256, 256>>>(fx0, c0, cp0, bx0, nin, hwi); count_launch(); }
        if (c1) { pack_channels_kernel<<<256, 256>>>(fx1, c1, cp1, bx1, nin1, hwi); count_launch(); }
        if (res) { pack_channels_kernel<<<256, 256>>>(fr, cout, npad, br, nout, hwo); count_launch(); }
        // weights: logical [cout][9][c0 + c1] -> padded [npad][9][cp0 + cp1] (concat parts padded separately)
        std::vector<float> hw((size_t)cout * 9 * cin + cout);
        ck(cudaMemcpy(hw.data(), fw, hw.size() * sizeof(float), cudaMemcpyDeviceToHost));
        std::vector<__nv_bfloat16> hbw((size_t)npad * 9 * cinp, __float2bfloat16_rn(0.0f));
        std::vector<float> hb(npad, 0.0f);
        for (int co = 0; co < cout; ++co) {
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < cin; ++ci) {
                    int cpi = ci < c0 ? ci : cp0 + (ci - c0);
                    hbw[((size_t)co * 9 + t) * cinp + cpi] = __float2bfloat16_rn(hw[((size_t)co * 9 + t) * cin + ci]);
                }
            hb[co] = hw[(size_t)cout * 9 * cin + co];
        }
        ck(cudaMemcpy(bw, hbw.data(), hbw.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        if (mode == 2) {
            // the phase-merged weights of the up layer (summed in FP32 in tap order, rounded once)
            std::vector<float> acc((size_t)npad * 16 * cinp, 0.0f);
            for (int co = 0; co < cout; ++co)
                for (int t = 0; t < 9; ++t)
                    for (int ph = 0; ph < 4; ++ph) {
                        const int r = up_merged_index(ph >> 1, ph & 1, t / 3 - 1, t % 3 - 1);
                        if (r >> 2 != ph) continue;
                        for (int ci = 0; ci < cin; ++ci) {
                            const int cpi = ci < c0 ? ci : cp0 + (ci - c0);
                            acc[((size_t)co * 16 + r) * cinp + cpi] += hw[((size_t)co * 9 + t) * cin + ci];
                        }
                    }
            std::vector<__nv_bfloat16> hup(acc.size());
            for (size_t i = 0; i < acc.size(); ++i) hup[i] = __float2bfloat16_rn(acc[i]);
            ck(cudaMemcpy(bwup, hup.data(), hup.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        }
        ck(cudaMemcpy(bp, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice));
        ck(cudaGetLastError());
    }
    if (!s) {
        ConvArgs a;
        a.x0 = bx0; a.c0 = cp0; a.x1 = bx1; a.c1 = cp1; a.x1_bcast = x1_bcast; a.x1_map = nullptr;
        a.nb = nb; a.hin = hin; a.win = win; a.hout = hout; a.wout = wout; a.mode = mode;
        a.w = bw; a.wup = bwup; a.bias = bp; a.res = br; a.y = by; a.npad = npad; a.cstore = cout; a.relu = relu;
        a.out_fp32 = 0;
        a.accum = 0;
        a.err = err;
        {
            LaunchScope scope(nullptr, K_CONV);
            s = launch_conv3x3(a, nullptr);
        }
        if (!s) {
            { unpack_channels_kernel<<<256, 256>>>(by, npad, cout, fy, nout, (long long)hout * wout); count_launch(); }
            ck(cudaGetLastError());
            ck(cudaDeviceSynchronize());
            int herr = 0;
            ck(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
            if (!s && herr) { set_error("cnn_conv3x3: a tensor-core wait expired"); s = HELM_ETIMEOUT; }
        }
        if (!s) ck(cudaMemcpy(y, fy, nout * cout * sizeof(float), cudaMemcpyDefault));
    }
    cudaFree(fx0); cudaFree(fx1); cudaFree(fw); cudaFree(fb); cudaFree(fr); cudaFree(fy); cudaFree(bp);
    cudaFree(bx0); cudaFree(bx1); cudaFree(bw); cudaFree(bwup); cudaFree(br); cudaFree(by); cudaFree(err);
    return s;
}

// One layer's backward pass for parity tests: FP32 in and out (inputs, weights and
// the upstream gradient rounded to BF16 inside), the same kernels as the network's
// backward pass (tensor-core input gradient; weight gradient on the path chosen by
// cnn_set_wgrad_path).  Outputs are overwritten; any may be NULL.
int cnn_conv3x3_backward(const float* x0, int c0, const float* x1, int c1, int x1_bcast, int nb, int hin, int win,
                         const float* w, int cout, int mode, const float* gy, float* gx0, float* gx1, float* dw,
                         float* db) {
    set_error("");
    if (!x0 || !w || !gy || c0 < 1 || c1 < 0 || (c1 > 0 && (!x1 || c0 % 16)) || nb < 1 || hin < 1 || win < 1 ||
        cout < 1 || cout > 128 || mode < 0 || mode > 2 || x1_bcast < 0 || x1_bcast > 1) {
        set_error("cnn_conv3x3_backward: invalid argument");
        return HELM_EINVAL;
    }
    const int cp0 = pad16(c0), cp1 = c1 ? pad16(c1) : 0, cin = c0 + c1, cinp = cp0 + cp1, npad = npad_of(cout);
    const int hout = mode == 1 ? hin / 2 : (mode == 2 ? 2 * hin : hin);
    const int wout = mode == 1 ? win / 2 : (mode == 2 ? 2 * win : win);
    const int nb1 = c1 ? (x1_bcast ? 1 : nb) : 0;
    const long long hwi = (long long)hin * win, hwo = (long long)hout * wout;
    const long long nin = (long long)nb * hwi, nin1 = (long long)nb1 * hwi, nout = (long long)nb * hwo;
    std::vector<void*> tmp;
    int s = HELM_OK;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (s == HELM_OK && cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cnn_conv3x3_backward: out of device memory");
            s = HELM_ENOMEM;
            return nullptr;
        }
        tmp.push_back(p);
        return p;
    };
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; } };
    float* fx0 = (float*)alloc(nin * c0 * sizeof(float));
    float* fx1 = c1 ? (float*)alloc(nin1 * c1 * sizeof(float)) : nullptr;
    float* fgy = (float*)alloc(nout * cout * sizeof(float));
    auto* bx0 = (__nv_bfloat16*)alloc(nin * cp0 * sizeof(__nv_bfloat16));
    auto* bx1 = c1 ? (__nv_bfloat16*)alloc(nin1 * cp1 * sizeof(__nv_bfloat16)) : nullptr;
    auto* bg = (__nv_bfloat16*)alloc(nout * npad * sizeof(__nv_bfloat16));
    auto* bw = (__nv_bfloat16*)alloc((size_t)npad * 9 * cinp * sizeof(__nv_bfloat16));
    float* dW = (float*)alloc((size_t)cout * 9 * cin * sizeof(float));
    float* dB = (float*)alloc((size_t)cout * sizeof(float));
    int* err = (int*)alloc(sizeof(int));
    if (s) { for (void* p : tmp) cudaFree(p); return s; }
    ck(cudaMemset(err, 0, sizeof(int)));
    ck(cudaMemset(dW, 0, (size_t)cout * 9 * cin * sizeof(float)));
    ck(cudaMemset(dB, 0, (size_t)cout * sizeof(float)));
    ck(cudaMemcpy(fx0, x0, nin * c0 * sizeof(float), cudaMemcpyDefault));
    if (c1) ck(cudaMemcpy(fx1, x1, nin1 * c1 * sizeof(float), cudaMemcpyDefault));
    ck(cudaMemcpy(fgy, gy, nout * cout * sizeof(float), cudaMemcpyDefault));
    {
        // weights: logical [cout][9][c0 + c1] -> padded BF16 [npad][9][cp0 + cp1]
        std::vector<float> hw((size_t)cout * 9 * cin);
        ck(cudaMemcpy(hw.data(), w, hw.size() * sizeof(float), cudaMemcpyDefault));
        std::vector<__nv_bfloat16> hbw((size_t)npad * 9 * cinp, __float2bfloat16_rn(0.0f));
        for (int co = 0; co < cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < cin; ++ci) {
                    const int cpi = ci < c0 ? ci : cp0 + (ci - c0);
                    hbw[((size_t)co * 9 + t) * cinp + cpi] = __float2bfloat16_rn(hw[((size_t)co * 9 + t) * cin + ci]);
                }
        ck(cudaMemcpy(bw, hbw.data(), hbw.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
    }
    if (!s) {
        { pack_channels_kernel<<<256, 256>>>(fx0, c0, cp0, bx0, nin, hwi); count_launch(); }
        if (c1) { pack_channels_kernel<<<256, 256>>>(fx1, c1, cp1, bx1, nin1, hwi); count_launch(); }
        { pack_channels_kernel<<<256, 256>>>(fgy, cout, npad, bg, nout, hwo); count_launch(); }
        ck(cudaGetLastError());
    }
    float* scratch = nullptr;
    size_t scap = 0;
    if (!s && (dw || db))
        s = layer_wgrad(bx0, cp0, bx1, cp1, x1_bcast, nullptr, nb1, nb, hin, win, hout, wout, mode, bg, npad, cout,
                        cin, dW, dB, &scratch, &scap, err, nullptr, nullptr);
    // input gradients of the two parts, FP32 [n][cp] accumulated, then narrowed to [n][c]
    for (int part = 0; part < 2 && !s; ++part) {
        float* out = part ? gx1 : gx0;
        const int c = part ? c1 : c0, cp = part ? cp1 : cp0;
        if (!out || c == 0) continue;
        float* target = (float*)alloc(nin * cp * sizeof(float));
        auto* Wt = (__nv_bfloat16*)alloc((size_t)cp * 9 * npad * sizeof(__nv_bfloat16));
        float* fine = mode == 2 ? (float*)alloc(nout * cp * sizeof(float)) : nullptr;
        if (s) break;
        ck(cudaMemset(target, 0, nin * cp * sizeof(float)));
        if (!s) s = layer_dgrad(bg, npad, bw, cinp, part ? cp0 : 0, cp, mode, nb, hin, win, hout, wout, target, Wt,
                                fine, err, nullptr, nullptr);
        ck(cudaDeviceSynchronize());
        if (s) break;
        // narrow (and, for a broadcast x1, sum over the images) on the host
        std::vector<float> h((size_t)nin * cp);
        ck(cudaMemcpy(h.data(), target, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
        const long long nimg = part && x1_bcast ? 1 : nb;
        std::vector<float> o((size_t)nimg * hwi * c, 0.0f);
        for (long long b = 0; b < nb; ++b)
            for (long long q = 0; q < hwi; ++q)
                for (int k = 0; k < c; ++k)
                    o[((size_t)(nimg == 1 ? 0 : b) * hwi + q) * c + k] += h[((size_t)b * hwi + q) * cp + k];
        ck(cudaMemcpy(out, o.data(), o.size() * sizeof(float), cudaMemcpyDefault));
    }
    ck(cudaDeviceSynchronize());
    if (!s) {
        int herr = 0;
        ck(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (!s && herr) { set_error("cnn_conv3x3_backward: a tensor-core wait expired"); s = HELM_ETIMEOUT; }
    }
    if (!s && dw) ck(cudaMemcpy(dw, dW, (size_t)cout * 9 * cin * sizeof(float), cudaMemcpyDefault));
    if (!s && db) ck(cudaMemcpy(db, dB, (size_t)cout * sizeof(float), cudaMemcpyDefault));
    if (scratch) cudaFree(scratch);
    for (void* p : tmp) cudaFree(p);
    return s;
}

// ---- checkpoints ------------------------------------------------------------
namespace {

constexpr char CKPT_MAGIC[8] = {'H', 'E', 'L', 'M', 'C', 'N', 'N', '1'};

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t levels;
    uint32_t widths[8];
    int64_t nparams;
    int64_t adam_t;
    uint32_t flags;
    uint32_t loss_kind;
    uint64_t checksum;
};

// FNV-1a, 64-bit (Fowler, Noll, Vo)
uint64_t fnv1a(const void* data, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace

int cnn_save(const cnn_model* m, const char* path) {
    set_error("");
    if (!m || !path) { set_error("cnn_save: null argument"); return HELM_EINVAL; }
    const size_t n = (size_t)m->nparams;
    const bool adam = m->adam_m && m->adam_v;
    std::vector<float> buf(n * (adam ? 3 : 1));
    HELM_CK(cudaMemcpy(buf.data(), m->master, n * sizeof(float), cudaMemcpyDeviceToHost));
    if (adam) {
        HELM_CK(cudaMemcpy(buf.data() + n, m->adam_m, n * sizeof(float), cudaMemcpyDeviceToHost));
        HELM_CK(cudaMemcpy(buf.data() + 2 * n, m->adam_v, n * sizeof(float), cudaMemcpyDeviceToHost));
    }
    CkptHeader h{};
    std::memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 1;
    h.levels = (uint32_t)m->levels;
    for (int l = 0; l < m->levels && l < 8; ++l) h.widths[l] = (uint32_t)m->widths[l];
    h.nparams = m->nparams;
    h.adam_t = adam ? m->adam_t : 0;
    h.flags = adam ? 1u : 0u;
    h.loss_kind = (uint32_t)m->loss_kind;
    h.checksum = fnv1a(buf.data(), buf.size() * sizeof(float));
    FILE* f = std::fopen(path, "wb");
    if (!f) { set_error(std::string("cnn_save: cannot open ") + path); return HELM_EINVAL; }
    const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
                    std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) { set_error(std::string("cnn_save: write failed: ") + path); return HELM_EINVAL; }
    return HELM_OK;
}

int cnn_load(cnn_model** out, const char* path) {
    set_error("");
    if (!out || !path) { set_error("cnn_load: null argument"); return HELM_EINVAL; }
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) { set_error(std::string("cnn_load: cannot open ") + path); return HELM_EINVAL; }
    CkptHeader h{};
    if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != 1 ||
        h.levels < 2 || h.levels > 6 || (h.flags & ~1u) || h.loss_kind > 1) {
        std::fclose(f);
        set_error(std::string("cnn_load: not a network checkpoint of this library: ") + path);
        return HELM_EINVAL;
    }
    // the whole file is checked on the host before anything touches the device
    int widths[8];
    cnn_model spec;
    spec.levels = (int)h.levels;
    for (int l = 0; l < 8; ++l) widths[l] = (int)h.widths[l];
    bool widths_ok = true;
    for (int l = 0; l < spec.levels; ++l)
        widths_ok = widths_ok && widths[l] >= 16 && widths[l] <= 128 && widths[l] % 16 == 0;
    if (widths_ok) {
        spec.widths.assign(widths, widths + spec.levels);
        build_specs(&spec);
    }
    if (!widths_ok || h.nparams != spec.nparams) {
        std::fclose(f);
        set_error("cnn_load: the header's architecture and parameter count do not match");
        return HELM_EINVAL;
    }
    const size_t n = (size_t)spec.nparams;
    const bool adam = h.flags & 1u;
    std::vector<float> buf(n * (adam ? 3 : 1));
    const bool ok = std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    unsigned char extra;
    const bool at_end = std::fread(&extra, 1, 1, f) == 0;
    std::fclose(f);
    if (!ok || !at_end || fnv1a(buf.data(), buf.size() * sizeof(float)) != h.checksum) {
        set_error(std::string("cnn_load: truncated or corrupted checkpoint: ") + path);
        return HELM_EINVAL;
    }
    cnn_model* m = nullptr;
    int s = create_zero(&m, (int)h.levels, widths);
    if (s) return s;
    s = cnn_set_params(m, buf.data(), m->nparams);
    if (!s) s = cnn_set_loss(m, (int)h.loss_kind);
    if (!s && adam) {
        s = cnn_adam_reset(m);
        if (!s && (cudaMemcpy(m->adam_m, buf.data() + n, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                   cudaMemcpy(m->adam_v, buf.data() + 2 * n, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)) {
            set_error("cnn_load: Adam state upload failed");
            s = HELM_ECUDA;
        }
        if (!s) m->adam_t = h.adam_t;
    }
    if (s) {
        cnn_destroy(m);
        return s;
    }
    *out = m;
    return HELM_OK;
}

}  // extern "C"
