// Coarsest-level solve of the V-cycle: a fixed number of plain GMRES steps on
// the Galerkin shifted Laplacian from a zero initial guess (Sec. 3.4; the
// paper leaves the coarsest solve open).  One thread block owns one
// right-hand side and runs every Arnoldi step, the Givens rotations and the
// final combination in a single launch: the coarse vectors (8192 nodes x 8 B
// per vector on a 512x256 grid with three levels) stay in L2, the inner
// products are block reductions (FP32 per thread, FP64 across the block) and
// no global scratch is needed for them.
#include <type_traits>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {
namespace {

// Threads per block (one block per RHS): 512 when every RHS has an SM of its
// own, 256 (two blocks per SM) when the batch is larger than the SM count, so
// that the whole batch runs in one wave.

// Sum nv complex values held per thread over the block (FP64), result in out[0..nv).
template <int CB, int NV>
__device__ void block_sum(const float2 (&v)[NV], int nv, double2* red /*[CW][NV]*/, double2* out) {
    constexpr int CW = CB / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            double a = warp_sum((double)v[i].x);
            double b = warp_sum((double)v[i].y);
            if (lane == 0) red[warp * NV + i] = make_double2(a, b);
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double2 acc = make_double2(0.0, 0.0);
        for (int w = 0; w < CW; ++w) acc = dadd(acc, red[w * NV + threadIdx.x]);
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

template <int CB>
__global__ void __launch_bounds__(CB, 512 / CB)
coarse_gmres_kernel(OpC9 op, float2* __restrict__ V, size_t vstride, float2* __restrict__ W, float2* __restrict__ u,
                    int kmax, const int* mask, Tally tl) {
    const int b = blockIdx.x;
    if (!mask[b]) return;
    tally_once(tl, true);
    const int nx = op.nx, nz = op.nz;
    const int n = nx * nz;
    float2* Vb = V + (size_t)b * n;       // vector i at Vb + i * vstride
    float2* Wb = W + (size_t)b * n;
    constexpr int CW = CB / 32;
    __shared__ double2 red[CW * (KMAX + 1)];
    __shared__ double2 sums[KMAX + 1];
    __shared__ double2 H[KMAX][KMAX + 1];  // H[j][i] = h_{i,j}
    __shared__ double sc[KMAX + 1];        // 1 / ||stored v_i||
    __shared__ double cs[KMAX];
    __shared__ double2 sn[KMAX];
    __shared__ double2 g[KMAX + 1];
    __shared__ double2 yv[KMAX];
    __shared__ float2 cfs[KMAX + 1];       // update / combination coefficients
    __shared__ int steps;

    // beta = ||f||, f stored as v_0
    {
        float2 a[1] = {make_float2(0.f, 0.f)};
        for (int p = 2 * threadIdx.x; p < n; p += 2 * CB) {
            const float4 f = *reinterpret_cast<const float4*>(Vb + p);
            a[0].x += f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
        }
        block_sum<CB, 1>(a, 1, red, sums);
    }
    const double beta = sqrt(sums[0].x);
    if (!(beta > 0.0) || !isfinite(beta)) {
        for (int p = threadIdx.x; p < n; p += CB) u[(size_t)b * n + p] = make_float2(0.f, 0.f);
        return;
    }
    if (threadIdx.x == 0) {
        sc[0] = 1.0 / beta;
        g[0] = make_double2(beta, 0.0);
        steps = 0;
    }
    __syncthreads();

    for (int j = 0; j < kmax; ++j) {
        // pass A: w = A (s_j v_j) and <s_i v_i, w>, i <= j
        const float sj = (float)sc[j];
        float2 acc[KMAX + 1];
#pragma unroll
        for (int i = 0; i <= KMAX; ++i) acc[i] = make_float2(0.f, 0.f);
        const float2* vj = Vb + (size_t)j * vstride;
        // two nodes per thread (n even, vectors 16-byte aligned): 16-byte loads
        for (int p = 2 * threadIdx.x; p < n; p += 2 * CB) {
            const int iz = p / nx, ix = p - iz * nx;
            float2 y0 = op.apply(vj, b, ix, iz), y1 = op.apply(vj, b, ix + 1, iz);
            y0.x *= sj;
            y0.y *= sj;
            y1.x *= sj;
            y1.y *= sj;
            *reinterpret_cast<float4*>(Wb + p) = make_float4(y0.x, y0.y, y1.x, y1.y);
#pragma unroll
            for (int i = 0; i <= KMAX; ++i) {
                if (i <= j) {
                    const float4 v = *reinterpret_cast<const float4*>(Vb + (size_t)i * vstride + p);
                    acc[i].x += v.x * y0.x + v.y * y0.y + v.z * y1.x + v.w * y1.y;
                    acc[i].y += v.x * y0.y - v.y * y0.x + v.z * y1.y - v.w * y1.x;
                }
            }
        }
        block_sum<CB, KMAX + 1>(acc, j + 1, red, sums);
        if (threadIdx.x <= j) {
            double s = sc[threadIdx.x];
            double2 h = make_double2(sums[threadIdx.x].x * s, sums[threadIdx.x].y * s);
            H[j][threadIdx.x] = h;
            cfs[threadIdx.x] = make_float2((float)(h.x * s), (float)(h.y * s));
        }
        __syncthreads();
        // pass B: w' = w - sum_i h_ij s_i v_i stored as v_{j+1}; ||w'||
        float2 nacc[1] = {make_float2(0.f, 0.f)};
        float2* vn = Vb + (size_t)(j + 1) * vstride;
        for (int p = 2 * threadIdx.x; p < n; p += 2 * CB) {
            float4 y = *reinterpret_cast<const float4*>(Wb + p);
#pragma unroll
            for (int i = 0; i <= KMAX; ++i) {
                if (i <= j) {
                    const float4 v = *reinterpret_cast<const float4*>(Vb + (size_t)i * vstride + p);
                    const float2 cf = cfs[i];
                    y.x -= cf.x * v.x - cf.y * v.y;
                    y.y -= cf.x * v.y + cf.y * v.x;
                    y.z -= cf.x * v.z - cf.y * v.w;
                    y.w -= cf.x * v.w + cf.y * v.z;
                }
            }
            *reinterpret_cast<float4*>(vn + p) = y;
            nacc[0].x += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
        }
        block_sum<CB, 1>(nacc, 1, red, sums);
        if (threadIdx.x == 0) {
            const double hb = sqrt(sums[0].x);
            double2* hc = H[j];
            for (int i = 0; i < j; ++i) {
                double2 a = hc[i], bb = hc[i + 1];
                double c = cs[i];
                double2 s = sn[i];
                hc[i] = dadd(make_double2(c * a.x, c * a.y), dmul(s, bb));
                hc[i + 1] = dadd(make_double2(-(s.x * a.x + s.y * a.y), -(s.x * a.y - s.y * a.x)),
                                 make_double2(c * bb.x, c * bb.y));
            }
            double2 a = hc[j];
            double na = sqrt(dabs2(a));
            double nu = sqrt(na * na + hb * hb);
            double c;
            double2 s;
            if (na == 0.0) {
                c = 0.0;
                s = make_double2(1.0, 0.0);
                hc[j] = make_double2(hb, 0.0);
            } else {
                c = na / nu;
                s = make_double2(a.x / na * hb / nu, a.y / na * hb / nu);
                hc[j] = make_double2(a.x / na * nu, a.y / na * nu);
            }
            cs[j] = c;
            sn[j] = s;
            double2 gj = g[j];
            g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
            g[j] = make_double2(c * gj.x, c * gj.y);
            sc[j + 1] = hb > 0.0 ? 1.0 / hb : 0.0;
            steps = j + 1;
        }
        __syncthreads();
        if (!(sc[j + 1] > 0.0) || !isfinite(sc[j + 1]) || sc[j + 1] > 1e300) break;   // exact or broken-down step
    }
    // back substitution R y = g, then u = sum_i y_i s_i v_i
    if (threadIdx.x == 0) {
        const int m = steps;
        for (int i = m - 1; i >= 0; --i) {
            double2 acc = g[i];
            for (int cc = i + 1; cc < m; ++cc) acc = dsub(acc, dmul(H[cc][i], yv[cc]));
            double2 d = H[i][i];
            double dd = dabs2(d);
            yv[i] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                             : make_double2(0.0, 0.0);
        }
    }
    __syncthreads();
    const int m = steps;
    if (threadIdx.x < m) {
        double2 v = yv[threadIdx.x];
        double s = sc[threadIdx.x];
        cfs[threadIdx.x] = make_float2((float)(v.x * s), (float)(v.y * s));
    }
    __syncthreads();
    for (int p = 2 * threadIdx.x; p < n; p += 2 * CB) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
            if (i < m) {
                const float4 v = *reinterpret_cast<const float4*>(Vb + (size_t)i * vstride + p);
                const float2 yc = cfs[i];
                acc.x += yc.x * v.x - yc.y * v.y;
                acc.y += yc.x * v.y + yc.y * v.x;
                acc.z += yc.x * v.z - yc.y * v.w;
                acc.w += yc.x * v.w + yc.y * v.z;
            }
        }
        *reinterpret_cast<float4*>(u + (size_t)b * n + p) = acc;
    }
}

}  // namespace

int launch_coarse_gmres(const helm_ctx* c, int level, float2* u_out, int nb, const int* mask) {
    const Level& L = c->lev[level];
    const size_t Nc = (size_t)L.nx * L.nz;
    const int k = c->opt.coarse_iters;
    if (Nc % 2) {
        set_error("coarsest multigrid level needs an even number of nodes (two per thread)");
        return HELM_EINVAL;
    }
    // per RHS: ||f|| (1 vector), step j: 2(j + 1) basis reads + v_j + w write/read + v_{j+1} write,
    // final combination k reads + 1 write: 8 Nc (k^2 + 5k + 2) bytes
    LaunchScope scope(c, K_COARSE_GMRES);
    const unsigned long long kk = (unsigned long long)k;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = 0;
    }
    const Tally tl = tally(c, K_COARSE_GMRES, 8ull * Nc * (kk * kk + 5 * kk + 2));
    if (sms > 0 && nb > sms)
        { coarse_gmres_kernel<256><<<nb, 256, 0, c->stream>>>(coarse_op(c, level), c->Vc, (size_t)c->cap * Nc, c->Wc,
                                                            u_out, k, mask, tl); count_launch(); }
    else
        { coarse_gmres_kernel<512><<<nb, 512, 0, c->stream>>>(coarse_op(c, level), c->Vc, (size_t)c->cap * Nc, c->Wc,
                                                            u_out, k, mask, tl); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

}  // namespace helm
