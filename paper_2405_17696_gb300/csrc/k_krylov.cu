// Batched (flexible) GMRES building blocks: fused operator application with
// the classical Gram-Schmidt inner products, the orthogonalising update with
// its norm, the FP64 Givens/Hessenberg step, the least-squares solve and the
// solution update.  Every right-hand side of the batch runs its own Arnoldi
// process; finished right-hand sides are masked out.
//
// No pass is spent on normalisation.  The fused operator kernel also reduces
// ||w||^2, so the update kernel can write v~_{j+1} = w' / est with the
// Pythagorean estimate est^2 = ||w||^2 - sum |h_ij|^2; the exact norm of the
// stored vector is reduced in the same pass and kept as s_{j+1} = 1/||v~_{j+1}||,
// so v_{j+1} = s_{j+1} v~_{j+1} exactly and h_{j+1,j} = est ||v~_{j+1}||.  The
// stored vectors therefore stay near unit norm (no drift of scale from one
// step to the next, which would underflow FP32 products), inner products and
// update coefficients absorb s_i, and the preconditioned direction z_j = M(v~_j)
// is a valid flexible-GMRES direction whatever its scale.
#include <type_traits>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {

namespace {

constexpr int NTHREADS = TILE_X * TILE_Y;
constexpr int NWARPS = NTHREADS / 32;

__device__ __forceinline__ double2* kcol(const KState& st, int b, int j) {
    return st.H + ((size_t)b * st.k + j) * (st.k + 1);
}

// One Givens step on column j of RHS b after h_{j+1,j} is known (Saad 2003,
// Sec. 6.5.3, complex form: rotation [c s; -conj(s) c] with real c).
__device__ void givens_step(const KState& st, int b, int j, double hnext, double s_next, const int* iters_base,
                            int max_iter, int* status) {
    double2* hc = kcol(st, b, j);
    hc[j + 1] = make_double2(hnext, 0.0);
    double* cs = st.cs + (size_t)b * st.k;
    double2* sn = st.sn + (size_t)b * st.k;
    for (int i = 0; i < j; ++i) {
        double2 a = hc[i], bb = hc[i + 1];
        double c = cs[i];
        double2 s = sn[i];
        hc[i] = dadd(make_double2(c * a.x, c * a.y), dmul(s, bb));
        hc[i + 1] = dadd(make_double2(-(s.x * a.x + s.y * a.y), -(s.x * a.y - s.y * a.x)),
                         make_double2(c * bb.x, c * bb.y));
    }
    double2 a = hc[j];
    double hb = hc[j + 1].x;
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
    hc[j + 1] = make_double2(0.0, 0.0);
    cs[j] = c;
    sn[j] = s;
    double2* g = st.g + (size_t)b * (st.k + 1);
    double2 gj = g[j];
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
    g[j] = make_double2(c * gj.x, c * gj.y);
    double est = sqrt(dabs2(g[j + 1]));
    st.steps[b] = j + 1;
    st.s[(size_t)b * (st.k + 1) + j + 1] = s_next;
    bool finite = isfinite(est) && isfinite(hb) && isfinite(nu);
    bool tiny = !(hb > 1e-300);
    bool cap = iters_base && (iters_base[b] + j + 1 >= max_iter);
    if (!finite && status) status[b] = HELM_EBREAKDOWN;
    if (!finite || tiny || est <= st.tol_abs[b] || cap || j + 1 >= st.k) st.active[b] = 0;
}

// w = A z for RHS b and the inner products h_{i,j} = s_i <v~_i, w>, i <= j,
// plus ||w||^2 for the scaled store of the next basis vector.  J = j is a
// template parameter so that only the j+2 accumulators that are live occupy
// registers.
template <class Op, int J>
__global__ void __launch_bounds__(NTHREADS, 3) arnoldi_dots_kernel(Op op, KState st, const float2* __restrict__ z,
                                                                   float2* __restrict__ w,
                                                                   const float2* __restrict__ V, size_t vstride,
                                                                   int nx, int nz, Tally tl) {
    const int b = blockIdx.z;
    if (!st.active[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const size_t N = (size_t)nx * nz;
    const float2* zb = z + (size_t)b * N;
    float2* wb = w + (size_t)b * N;
    const float2* Vb = V + (size_t)b * N;
    const int ix = blockIdx.x * TILE_X + threadIdx.x;
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    float2 acc[J + 2];   // acc[i] = <v~_i, w> for i <= J, acc[J+1] = ||w||^2
#pragma unroll
    for (int i = 0; i < J + 2; ++i) acc[i] = make_float2(0.f, 0.f);
    if (ix < nx) {
#pragma unroll 2
        for (int r = 0; r < ROWS; ++r) {
            int iz = iz0 + r;
            if (iz >= nz) break;
            size_t p = (size_t)iz * nx + ix;
            float2 v[J + 1];
#pragma unroll
            for (int i = 0; i <= J; ++i) v[i] = Vb[(size_t)i * vstride + p];
            float2 y = op.apply(zb, b, ix, iz);
            wb[p] = y;
#pragma unroll
            for (int i = 0; i <= J; ++i) {
                acc[i].x += v[i].x * y.x + v[i].y * y.y;   // conj(v) y
                acc[i].y += v[i].x * y.y - v[i].y * y.x;
            }
            acc[J + 1].x += y.x * y.x + y.y * y.y;
        }
    }
    __shared__ double2 sm[NWARPS * (J + 2)];
    __shared__ double hsq[J + 2];
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = st.partials + ((size_t)b * st.max_tiles) * (KMAX + 2);
    bool last = reduce_block_last<J + 2>(acc, J + 2, part + (size_t)tile * (KMAX + 2), st.counters + b, ntiles, sm);
    if (last) {
        const int tid = threadIdx.x + threadIdx.y * blockDim.x;
        if (tid <= J + 1) {
            double2 h = sum_partials(part, ntiles, KMAX + 2, tid);
            if (tid <= J) {
                double sc = st.s[(size_t)b * (st.k + 1) + tid];
                h = make_double2(h.x * sc, h.y * sc);
                kcol(st, b, J)[tid] = h;
                hsq[tid] = dabs2(h);
            } else {
                hsq[tid] = h.x;   // ||w||^2
            }
        }
        __syncthreads();
        if (tid == 0) {
            double w2 = hsq[J + 1], proj = 0.0;
            for (int i = 0; i <= J; ++i) proj += hsq[i];
            double est2 = w2 - proj;
            // a cancelled estimate only changes the scale the vector is stored at
            if (!(est2 > 1e-12 * w2)) est2 = 1e-12 * w2;
            double est = sqrt(est2);
            st.inv_est[b] = (est > 0.0 && isfinite(est)) ? 1.0 / est : 1.0;
        }
    }
}

// v~_{j+1} = (w - sum_i h_{i,j} s_i v~_i) / est, its norm, then the Givens step.
template <int J>
__global__ void __launch_bounds__(NTHREADS, 3) arnoldi_update_kernel(KState st, const float2* __restrict__ w,
                                                                     float2* __restrict__ V, size_t vstride,
                                                                     int nx, int nz, const int* iters_base,
                                                                     int max_iter, int* status, Tally tl) {
    const int b = blockIdx.z;
    if (!st.active[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const size_t N = (size_t)nx * nz;
    __shared__ float2 coef[J + 1];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const double inv = st.inv_est[b];
    if (tid <= J) {
        double2 h = kcol(st, b, J)[tid];
        double sc = st.s[(size_t)b * (st.k + 1) + tid] * inv;
        coef[tid] = make_float2((float)(h.x * sc), (float)(h.y * sc));
    }
    __syncthreads();
    const float finv = (float)inv;
    const float2* wb = w + (size_t)b * N;
    float2* Vb = V + (size_t)b * N;
    float2* vout = Vb + (size_t)(J + 1) * vstride;
    const int ix = blockIdx.x * TILE_X + threadIdx.x;
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    float acc = 0.f;
    if (ix < nx) {
#pragma unroll 2
        for (int r = 0; r < ROWS; ++r) {
            int iz = iz0 + r;
            if (iz >= nz) break;
            size_t p = (size_t)iz * nx + ix;
            float2 v[J + 1];
#pragma unroll
            for (int i = 0; i <= J; ++i) v[i] = Vb[(size_t)i * vstride + p];
            float2 y = wb[p];
            y.x *= finv;
            y.y *= finv;
#pragma unroll
            for (int i = 0; i <= J; ++i) {
                const float2 c = coef[i];
                y.x -= c.x * v[i].x - c.y * v[i].y;
                y.y -= c.x * v[i].y + c.y * v[i].x;
            }
            vout[p] = y;
            acc += y.x * y.x + y.y * y.y;
        }
    }
    __shared__ double2 sm[NWARPS];
    double2 vals[1] = {make_double2((double)acc, 0.0)};
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = st.partials + ((size_t)b * st.max_tiles) * (KMAX + 2);
    bool last = reduce_block_last<1>(vals, 1, part + (size_t)tile * (KMAX + 2), st.counters + b, ntiles, sm);
    if (last && tid == 0) {
        double nrm = sqrt(sum_partials(part, ntiles, KMAX + 2, 0).x);   // ||v~_{j+1}||
        double hnext = nrm / inv;                                       // ||w'|| = est ||v~_{j+1}||
        givens_step(st, b, J, hnext, nrm > 0.0 ? 1.0 / nrm : 0.0, iters_base, max_iter, status);
    }
}

// ||v0||^2 per RHS, then g_0 = ||v0||, s_0 = 1/||v0||, steps = 0, active = mask && ||v0|| > 0.
__global__ void __launch_bounds__(NTHREADS) kstate_init_kernel(KState st, const float2* __restrict__ v0, int nx,
                                                               int nz, const int* mask, Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
            st.active[b] = 0;
            st.steps[b] = 0;
        }
        return;
    }
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const size_t N = (size_t)nx * nz;
    const float2* vb = v0 + (size_t)b * N;
    const int ix = blockIdx.x * TILE_X + threadIdx.x;
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    float acc = 0.f;
    if (ix < nx) {
        for (int r = 0; r < ROWS; ++r) {
            int iz = iz0 + r;
            if (iz >= nz) break;
            float2 v = vb[(size_t)iz * nx + ix];
            acc += v.x * v.x + v.y * v.y;
        }
    }
    __shared__ double2 sm[NWARPS];
    double2 vals[1] = {make_double2((double)acc, 0.0)};
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = st.partials + ((size_t)b * st.max_tiles) * (KMAX + 2);
    bool last = reduce_block_last<1>(vals, 1, part + (size_t)tile * (KMAX + 2), st.counters + b, ntiles, sm);
    if (last && threadIdx.x == 0 && threadIdx.y == 0) {
        double n = sqrt(sum_partials(part, ntiles, KMAX + 2, 0).x);
        st.g[(size_t)b * (st.k + 1)] = make_double2(n, 0.0);
        st.s[(size_t)b * (st.k + 1)] = n > 0.0 ? 1.0 / n : 0.0;
        st.inv_est[b] = n > 0.0 ? 1.0 / n : 0.0;
        st.steps[b] = 0;
        st.tol_abs[b] = 0.0;
        st.active[b] = (n > 0.0 && isfinite(n)) ? 1 : 0;
    }
}

// v~_0 <- v~_0 / ||v~_0|| (the scale left in inv_est by the kernel that
// reduced the norm), s_0 <- 1: the first basis vector is stored at unit norm
// like the others.
__global__ void normalize_v0_kernel(KState st, float2* __restrict__ v0, size_t n) {
    const int b = blockIdx.y;
    if (!st.active[b]) return;
    const float sc = (float)st.inv_est[b];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        float2 v = v0[(size_t)b * n + p];
        v0[(size_t)b * n + p] = make_float2(v.x * sc, v.y * sc);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st.s[(size_t)b * (st.k + 1)] = 1.0;
}

// Back substitution R y = g for every RHS (FP64, one thread per RHS).
__global__ void lsq_kernel(KState st, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int n = st.steps[b];
    double2* y = st.y + (size_t)b * st.k;
    const double2* g = st.g + (size_t)b * (st.k + 1);
    for (int i = n - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int c = i + 1; c < n; ++c) acc = dsub(acc, dmul(kcol(st, b, c)[i], y[c]));
        double2 d = kcol(st, b, i)[i];
        double dd = dabs2(d);
        y[i] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                        : make_double2(0.0, 0.0);
    }
}

// out = sum_{i < steps} y_i Z_i (float)
__global__ void combine_kernel(KState st, float2* __restrict__ out, const float2* __restrict__ Zb, size_t zstride,
                               size_t n, const int* mask, Tally tl) {
    const int b = blockIdx.y;
    if (!mask[b]) return;
    int ns = st.steps[b];
    tally_once(tl, blockIdx.x == 0, ns);
    __shared__ float2 yc[KMAX];
    if (threadIdx.x < KMAX) {
        double2 v = threadIdx.x < ns ? st.y[(size_t)b * st.k + threadIdx.x] : make_double2(0.0, 0.0);
        yc[threadIdx.x] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < ns; ++i) {
            float2 zv = Zb[(size_t)i * zstride + (size_t)b * n + p];
            acc.x += yc[i].x * zv.x - yc[i].y * zv.y;
            acc.y += yc[i].x * zv.y + yc[i].y * zv.x;
        }
        out[(size_t)b * n + p] = acc;
    }
}

// x += sum_{i < steps} y_i Z_i with x in complex128.  The correction is a
// combination of complex64 directions and is summed in FP32; only the
// accumulation into the iterate is FP64 (its rounding is removed by the FP64
// restart residual).
__global__ void update_x64_kernel(KState st, double2* __restrict__ x, const float2* __restrict__ Zb, size_t zstride,
                                  size_t n, Tally tl) {
    const int b = blockIdx.y;
    int ns = st.steps[b];
    if (ns == 0) return;
    tally_once(tl, blockIdx.x == 0, ns);
    __shared__ float2 yc[KMAX];
    if (threadIdx.x < KMAX) {
        double2 v = threadIdx.x < ns ? st.y[(size_t)b * st.k + threadIdx.x] : make_double2(0.0, 0.0);
        yc[threadIdx.x] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        float ax = 0.f, ay = 0.f;
        for (int i = 0; i < ns; ++i) {
            float2 zv = Zb[(size_t)i * zstride + (size_t)b * n + p];
            ax += yc[i].x * zv.x - yc[i].y * zv.y;
            ay += yc[i].x * zv.y + yc[i].y * zv.x;
        }
        double2 xv = x[(size_t)b * n + p];
        x[(size_t)b * n + p] = make_double2(xv.x + (double)ax, xv.y + (double)ay);
    }
}

}  // namespace

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

// The fine-grid Arnoldi dots with two nodes per thread (16-byte loads of every
// basis vector and of z), otherwise as arnoldi_dots_kernel: w = H z and the
// inner products <v~_i, w>, ||w||^2 with the last-block reduction.
template <int J>
__global__ void __launch_bounds__(NTHREADS, 3) arnoldi_dots_fine2_kernel(OpFine5 op, KState st,
                                                                        const float2* __restrict__ z,
                                                                        float2* __restrict__ w,
                                                                        const float2* __restrict__ V,
                                                                        size_t vstride, int nx, int nz, Tally tl) {
    const int b = blockIdx.z;
    if (!st.active[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const size_t N = (size_t)nx * nz;
    const float2* zb = z + (size_t)b * N;
    float2* wb = w + (size_t)b * N;
    const float2* Vb = V + (size_t)b * N;
    const int ix = 2 * (blockIdx.x * TILE_X + threadIdx.x);
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    float2 acc[J + 2];
#pragma unroll
    for (int i = 0; i < J + 2; ++i) acc[i] = make_float2(0.f, 0.f);
    if (ix < nx) {
#pragma unroll 2
        for (int r = 0; r < ROWS; ++r) {
            const int iz = iz0 + r;
            if (iz >= nz) break;
            const size_t p = (size_t)iz * nx + ix;
            float4 v[J + 1];
#pragma unroll
            for (int i = 0; i <= J; ++i) v[i] = *reinterpret_cast<const float4*>(Vb + (size_t)i * vstride + p);
            float2 y0, y1;
            op.apply2(zb, b, ix, iz, y0, y1);
            *reinterpret_cast<float4*>(wb + p) = make_float4(y0.x, y0.y, y1.x, y1.y);
#pragma unroll
            for (int i = 0; i <= J; ++i) {
                acc[i].x += v[i].x * y0.x + v[i].y * y0.y + v[i].z * y1.x + v[i].w * y1.y;
                acc[i].y += v[i].x * y0.y - v[i].y * y0.x + v[i].z * y1.y - v[i].w * y1.x;
            }
            acc[J + 1].x += y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
        }
    }
    __shared__ double2 sm[NWARPS * (J + 2)];
    __shared__ double hsq[J + 2];
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = st.partials + ((size_t)b * st.max_tiles) * (KMAX + 2);
    bool last = reduce_block_last<J + 2>(acc, J + 2, part + (size_t)tile * (KMAX + 2), st.counters + b, ntiles, sm);
    if (last) {
        const int tid = threadIdx.x + threadIdx.y * blockDim.x;
        if (tid <= J + 1) {
            double2 h = sum_partials(part, ntiles, KMAX + 2, tid);
            if (tid <= J) {
                double sc = st.s[(size_t)b * (st.k + 1) + tid];
                h = make_double2(h.x * sc, h.y * sc);
                kcol(st, b, J)[tid] = h;
                hsq[tid] = dabs2(h);
            } else {
                hsq[tid] = h.x;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double w2 = hsq[J + 1], proj = 0.0;
            for (int i = 0; i <= J; ++i) proj += hsq[i];
            double est2 = w2 - proj;
            if (!(est2 > 1e-12 * w2)) est2 = 1e-12 * w2;
            double est = sqrt(est2);
            st.inv_est[b] = (est > 0.0 && isfinite(est)) ? 1.0 / est : 1.0;
        }
    }
}

static dim3 tiled_grid(int nx, int nz, int nb) {
    return dim3((nx + TILE_X - 1) / TILE_X, (nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS), nb);
}

#define HELM_J_CASES(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15)

template <class Op>
int launch_arnoldi_dots(const helm_ctx* c, const Op& op, KState& st, const float2* z, float2* w,
                        const float2* V, size_t vstride, int j, int nx, int nz, int nb) {
    static_assert(KMAX == 16, "dispatch covers j < 16");
    LaunchScope scope(c, std::is_same<Op, OpFine5>::value ? K_DOTS_FINE : K_DOTS_COARSE);
    const Tally tl = tally(c, std::is_same<Op, OpFine5>::value ? K_DOTS_FINE : K_DOTS_COARSE,
                           8ull * nx * nz * (j + 3));
    if constexpr (std::is_same<Op, OpFine5>::value) {
        if (nx % 2 == 0) {
            const dim3 grid2((nx / 2 + TILE_X - 1) / TILE_X, (nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS), nb),
                block2(TILE_X, TILE_Y);
            switch (j) {
#define HELM_DOTS2_CASE(J)                                                                                  \
    case J:                                                                                                 \
        { arnoldi_dots_fine2_kernel<J><<<grid2, block2, 0, c->stream>>>(op, st, z, w, V, vstride, nx, nz, tl); count_launch(); } \
        break;
                HELM_J_CASES(HELM_DOTS2_CASE)
#undef HELM_DOTS2_CASE
                default:
                    set_error("Arnoldi step beyond KMAX");
                    return HELM_EINVAL;
            }
            HELM_CK(cudaGetLastError());
            return HELM_OK;
        }
    }
    const dim3 grid = tiled_grid(nx, nz, nb), block(TILE_X, TILE_Y);
    switch (j) {
#define HELM_DOTS_CASE(J)                                                                                     \
    case J:                                                                                                   \
        { arnoldi_dots_kernel<Op, J><<<grid, block, 0, c->stream>>>(op, st, z, w, V, vstride, nx, nz, tl); count_launch(); }   \
        break;
        HELM_J_CASES(HELM_DOTS_CASE)
#undef HELM_DOTS_CASE
        default:
            set_error("Arnoldi step beyond KMAX");
            return HELM_EINVAL;
    }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}
template int launch_arnoldi_dots<OpFine5>(const helm_ctx*, const OpFine5&, KState&, const float2*, float2*,
                                          const float2*, size_t, int, int, int, int);
template int launch_arnoldi_dots<OpC9>(const helm_ctx*, const OpC9&, KState&, const float2*, float2*,
                                       const float2*, size_t, int, int, int, int);

int launch_arnoldi_update_ex(const helm_ctx* c, KState& st, const float2* w, float2* V, size_t vstride, int j,
                             int nx, int nz, int nb, const int* iters_base, int max_iter, int* status) {
    const int kid = st.H == c->fine.H ? K_UPDATE_FINE : K_UPDATE_COARSE;
    LaunchScope scope(c, kid);
    const Tally tl = tally(c, kid, 8ull * nx * nz * (j + 3));
    const dim3 grid = tiled_grid(nx, nz, nb), block(TILE_X, TILE_Y);
    switch (j) {
#define HELM_UPD_CASE(J)                                                                                        \
    case J:                                                                                                     \
        { arnoldi_update_kernel<J><<<grid, block, 0, c->stream>>>(st, w, V, vstride, nx, nz, iters_base, max_iter, \
                                                                 status, tl); count_launch(); }                                  \
        break;
        HELM_J_CASES(HELM_UPD_CASE)
#undef HELM_UPD_CASE
        default:
            set_error("Arnoldi step beyond KMAX");
            return HELM_EINVAL;
    }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_arnoldi_update(const helm_ctx* c, KState& st, const float2* w, float2* V, size_t vstride, int j,
                          int nx, int nz, int nb) {
    return launch_arnoldi_update_ex(c, st, w, V, vstride, j, nx, nz, nb, nullptr, 0, nullptr);
}

int launch_kstate_init(const helm_ctx* c, KState& st, const float2* v0, int nx, int nz, int nb,
                       const int* mask) {
    LaunchScope scope(c, K_KINIT);
    { kstate_init_kernel<<<tiled_grid(nx, nz, nb), dim3(TILE_X, TILE_Y), 0, c->stream>>>(st, v0, nx, nz, mask,
                                                                                    tally(c, K_KINIT, 8ull * nx * nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_normalize_v0(const helm_ctx* c, KState& st, float2* v0, size_t n, int nb) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 64) blocks = 64;
    LaunchScope scope(c, K_MISC);
    { normalize_v0_kernel<<<dim3((unsigned)blocks, nb), 256, 0, c->stream>>>(st, v0, n); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_lsq(const helm_ctx* c, KState& st, int nb) {
    LaunchScope scope(c, K_LSQ);
    { lsq_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(st, nb); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

static int grid_for(size_t n) {
    size_t blocks = (n + 255) / 256;
    return (int)(blocks > 1184 ? 1184 : (blocks == 0 ? 1 : blocks));
}

int launch_combine(const helm_ctx* c, const KState& st, float2* out, const float2* Zb, size_t zstride, size_t n,
                   int nb, const int* mask) {
    LaunchScope scope(c, K_COMBINE);
    { combine_kernel<<<dim3(grid_for(n) / 8 + 1, nb), 256, 0, c->stream>>>(st, out, Zb, zstride, n, mask,
                                                                                  tally(c, K_COMBINE, 8ull * n, 8ull * n)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_update_x64(const helm_ctx* c, const KState& st, double2* x, const float2* Zb, size_t zstride,
                      size_t n, int nb) {
    LaunchScope scope(c, K_UPDATE_X);
    { update_x64_kernel<<<dim3(grid_for(n) / 8 + 1, nb), 256, 0, c->stream>>>(st, x, Zb, zstride, n,
                                                                                     tally(c, K_UPDATE_X, 32ull * n, 8ull * n)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

}  // namespace helm
