// Shifted-Laplacian multigrid kernels (Sec. 3.4, Eq. 3.12): damped Jacobi,
// full-weighting restriction of the residual, bilinear prolongation with
// correction, and the Galerkin coarse operators R P 4R^T.  Coarse node (J, I)
// of a level sits on node (2J+1, 2I+1) of the level above; values outside a
// grid are zero.  All kernels are batched over right-hand sides (blockIdx.z)
// and skip right-hand sides whose mask entry is zero.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "helm_internal.cuh"

namespace helm {

namespace {

// u_out = u_in + w D^-1 (f - A u_in)    (u_in == nullptr: u_in = 0)
// One damped Jacobi sweep on the fine grid with two nodes per thread (16-byte
// loads); nx even.
__global__ void jacobi_fine2_kernel(OpFine5 op, float2* __restrict__ u_out, const float2* __restrict__ u_in,
                                    const float2* __restrict__ f, float w, int nx, int nz, const int* mask,
                                    Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int ix = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const size_t N = (size_t)nx * nz;
    const size_t p = (size_t)iz * nx + ix;
    const float2* ub = u_in + (size_t)b * N;
    const float4 fv = *reinterpret_cast<const float4*>(f + (size_t)b * N + p);
    const float4 uv = *reinterpret_cast<const float4*>(ub + p);
    float2 y0, y1;
    op.apply2(ub, b, ix, iz, y0, y1);
    const float2 q0 = cdiv(make_float2(fv.x - y0.x, fv.y - y0.y), op.diag(b, (int)p));
    const float2 q1 = cdiv(make_float2(fv.z - y1.x, fv.w - y1.y), op.diag(b, (int)p + 1));
    *reinterpret_cast<float4*>(u_out + (size_t)b * N + p) =
        make_float4(uv.x + w * q0.x, uv.y + w * q0.y, uv.z + w * q1.x, uv.w + w * q1.y);
}

// One damped Jacobi sweep of a coarse level for the RHS pair (2z, 2z + 1): the nine
// Galerkin coefficients of a node are loaded once for both when the two RHS share a
// frequency (they are read from L2 for every RHS otherwise).
__global__ void jacobi_c9_pair_kernel(OpC9 op, float2* __restrict__ u_out, const float2* __restrict__ u_in,
                                      const float2* __restrict__ f, float w, int nx, int nz, int nb,
                                      const int* mask, Tally tl) {
    const int b0 = 2 * blockIdx.z, b1 = b0 + 1;
    const bool a0 = mask[b0] != 0, a1 = b1 < nb && mask[b1] != 0;
    if (!a0 && !a1) return;
    if (a0) tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    if (a1) tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const size_t N = (size_t)nx * nz;
    const int idx = iz * nx + ix;
    const int f0 = __ldg(op.rhs_freq + b0), f1 = a1 ? __ldg(op.rhs_freq + b1) : f0;
    const float2* c0 = op.base(f0);
    const float2* c1 = op.base(f1);
    const bool same = f0 == f1;
    const float2* u0b = u_in ? u_in + (size_t)b0 * N : nullptr;
    const float2* u1b = u_in ? u_in + (size_t)b1 * N : nullptr;
    float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
    if (u_in) {
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int jz = iz + dz, jx = ix + dx;
                if (jz < 0 || jz >= nz || jx < 0 || jx >= nx) continue;
                const size_t off = (size_t)((dz + 1) * 3 + (dx + 1)) * N + idx;
                const float2 k0 = __ldg(c0 + off);
                const float2 k1 = same ? k0 : __ldg(c1 + off);
                const int q = jz * nx + jx;
                if (a0) {
                    const float2 v = u0b[q];
                    y0.x += k0.x * v.x - k0.y * v.y;
                    y0.y += k0.x * v.y + k0.y * v.x;
                }
                if (a1) {
                    const float2 v = u1b[q];
                    y1.x += k1.x * v.x - k1.y * v.y;
                    y1.y += k1.x * v.y + k1.y * v.x;
                }
            }
        }
    }
    const float2 d0 = __ldg(c0 + 4 * N + idx);
    const float2 d1 = same ? d0 : __ldg(c1 + 4 * N + idx);
    if (a0) {
        const size_t i = (size_t)b0 * N + idx;
        const float2 u0 = u_in ? u_in[i] : make_float2(0.f, 0.f);
        const float2 q = cdiv(csub(f[i], y0), d0);
        u_out[i] = make_float2(u0.x + w * q.x, u0.y + w * q.y);
    }
    if (a1) {
        const size_t i = (size_t)b1 * N + idx;
        const float2 u0 = u_in ? u_in[i] : make_float2(0.f, 0.f);
        const float2 q = cdiv(csub(f[i], y1), d1);
        u_out[i] = make_float2(u0.x + w * q.x, u0.y + w * q.y);
    }
}

template <class Op>
__global__ void jacobi_kernel(Op op, float2* __restrict__ u_out, const float2* __restrict__ u_in,
                              const float2* __restrict__ f, float w, int nx, int nz, const int* mask, Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const size_t N = (size_t)nx * nz;
    const size_t p = (size_t)iz * nx + ix;
    float2 r = f[(size_t)b * N + p];
    float2 u0 = make_float2(0.f, 0.f);
    if (u_in) {
        const float2* ub = u_in + (size_t)b * N;
        u0 = ub[p];
        r = csub(r, op.apply(ub, b, ix, iz));
    }
    float2 d = op.diag(b, (int)p);
    float2 q = cdiv(r, d);
    u_out[(size_t)b * N + p] = make_float2(u0.x + w * q.x, u0.y + w * q.y);
}

// rc(J, I) = sum_{a,b} w_a w_b / 16 (f - A u)(2J+1+a, 2I+1+b)   (u == nullptr: u = 0),
// full weighting with each fine residual computed once: a block of 32 x 8 coarse
// nodes first writes f - A u on its 65 x 17 fine window (the nodes 2J .. 2J+2,
// 2I .. 2I+2 of its coarse nodes; zero outside the grid) to shared memory, then
// weights it.
template <class Op>
__global__ void __launch_bounds__(256) restrict_residual_tiled_kernel(Op op, float2* __restrict__ rc,
                                                                      const float2* __restrict__ u,
                                                                      const float2* __restrict__ f, int nx, int nz,
                                                                      const int* mask, Tally tl) {
    constexpr int TX = 32, TY = 8, WX = 2 * TX + 1, WY = 2 * TY + 1;
    __shared__ float2 rs[WY][WX + 1];
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int nxc = nx / 2, nzc = nz / 2;
    const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY;
    const size_t N = (size_t)nx * nz;
    const float2* fb = f + (size_t)b * N;
    const float2* ub = u ? u + (size_t)b * N : nullptr;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int t = tid; t < WX * WY; t += TX * TY) {
        const int lz = t / WX, lx = t - lz * WX;
        const int iz = 2 * J0 + lz, ix = 2 * I0 + lx;
        float2 r = make_float2(0.f, 0.f);
        if (iz < nz && ix < nx) {
            r = fb[(size_t)iz * nx + ix];
            if (ub) r = csub(r, op.apply(ub, b, ix, iz));
        }
        rs[lz][lx] = r;
    }
    __syncthreads();
    const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
    if (I >= nxc || J >= nzc) return;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float wa = a == 1 ? 2.f : 1.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float wt = wa * (c == 1 ? 2.f : 1.f) * (1.0f / 16.0f);
            const float2 r = rs[2 * threadIdx.y + a][2 * threadIdx.x + c];
            acc.x += wt * r.x;
            acc.y += wt * r.y;
        }
    }
    rc[(size_t)b * nxc * nzc + (size_t)J * nxc + I] = acc;
}

// u += bilinear interpolation of ec for the fine node pair (iz, 2k), (iz, 2k+1) of each
// thread (16-byte access to u; nx even): the odd node takes coarse column k, the even
// node the mean of columns k-1 and k; an odd row takes coarse row (iz-1)/2, an even
// row the mean of rows iz/2 - 1 and iz/2.
__global__ void prolong_add2_kernel(float2* __restrict__ u, const float2* __restrict__ ec, int nx, int nz,
                                    const int* mask, Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    const int nxc = nx / 2, nzc = nz / 2;
    if (2 * k >= nx || iz >= nz) return;
    const float2* eb = ec + (size_t)b * nxc * nzc;
    int jz0, jz1;
    float wz0, wz1;
    if (iz & 1) { jz0 = (iz - 1) >> 1; wz0 = 1.f; jz1 = -1; wz1 = 0.f; }
    else { jz0 = (iz >> 1) - 1; wz0 = 0.5f; jz1 = iz >> 1; wz1 = 0.5f; }
    float2 em = make_float2(0.f, 0.f), e0 = make_float2(0.f, 0.f);   // columns k-1 and k, rows weighted
    auto row = [&](int jz, float wz) {
        if (jz < 0 || jz >= nzc || wz == 0.f) return;
        const float2* er = eb + (size_t)jz * nxc;
        if (k < nxc) { const float2 v = er[k]; e0.x += wz * v.x; e0.y += wz * v.y; }
        if (k >= 1) { const float2 v = er[k - 1]; em.x += wz * v.x; em.y += wz * v.y; }
    };
    row(jz0, wz0);
    row(jz1, wz1);
    float4* up = reinterpret_cast<float4*>(u + (size_t)b * nx * nz + (size_t)iz * nx + 2 * k);
    float4 v = *up;
    v.x += 0.5f * (em.x + e0.x);
    v.y += 0.5f * (em.y + e0.y);
    v.z += e0.x;
    v.w += e0.y;
    *up = v;
}

// u += bilinear interpolation of ec (coarse node (J, I) on fine node (2J+1, 2I+1)).
__global__ void prolong_add_kernel(float2* __restrict__ u, const float2* __restrict__ ec, int nx, int nz,
                                   const int* mask, Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const int nxc = nx / 2, nzc = nz / 2;
    const float2* eb = ec + (size_t)b * nxc * nzc;
    // 1D: odd fine index 2J+1 <- J (weight 1); even 2J <- J-1 and J (1/2 each)
    int jz[2], jx[2];
    float wz[2], wx[2];
    int nzt, nxt;
    if (iz & 1) { jz[0] = (iz - 1) >> 1; wz[0] = 1.f; nzt = 1; }
    else { jz[0] = (iz >> 1) - 1; wz[0] = 0.5f; jz[1] = iz >> 1; wz[1] = 0.5f; nzt = 2; }
    if (ix & 1) { jx[0] = (ix - 1) >> 1; wx[0] = 1.f; nxt = 1; }
    else { jx[0] = (ix >> 1) - 1; wx[0] = 0.5f; jx[1] = ix >> 1; wx[1] = 0.5f; nxt = 2; }
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < nzt; ++s) {
        if (jz[s] < 0 || jz[s] >= nzc) continue;
        for (int t = 0; t < nxt; ++t) {
            if (jx[t] < 0 || jx[t] >= nxc) continue;
            float wt = wz[s] * wx[t];
            float2 e = eb[(size_t)jz[s] * nxc + jx[t]];
            acc.x += wt * e.x;
            acc.y += wt * e.y;
        }
    }
    const size_t p = (size_t)b * nx * nz + (size_t)iz * nx + ix;
    float2 v = u[p];
    u[p] = make_float2(v.x + acc.x, v.y + acc.y);
}

__global__ void copy_masked_kernel(float2* __restrict__ dst, const float2* __restrict__ src, size_t n,
                                   const int* mask, Tally tl) {
    const int b = blockIdx.y;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0);
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        dst[(size_t)b * n + p] = src[(size_t)b * n + p];
}

// 1D interpolation weight of fine index k from coarse index J: 1 if k = 2J+1,
// 1/2 if |k - (2J+1)| = 1, else 0.
__device__ __forceinline__ double pw(int k, int J) {
    int d = k - (2 * J + 1);
    return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);
}

// Galerkin coarse operator A_c = R A_f (4 R^T) for frequency f, one thread per coarse node.
template <class OpF>
__global__ void galerkin_kernel(OpF fine, int f, float2* __restrict__ out, int nxf, int nzf) {
    const int nxc = nxf / 2, nzc = nzf / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= nxc || J >= nzc) return;
    double2 acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int a = -1; a <= 1; ++a) {
        int iz = 2 * J + 1 + a;
        if (iz < 0 || iz >= nzf) continue;
        for (int c = -1; c <= 1; ++c) {
            int ix = 2 * I + 1 + c;
            if (ix < 0 || ix >= nxf) continue;
            double wr = (a == 0 ? 2.0 : 1.0) * (c == 0 ? 2.0 : 1.0) / 16.0;
            for (int k = 0; k < 9; ++k) {
                int kz = iz + k / 3 - 1, kx = ix + k % 3 - 1;
                if (kz < 0 || kz >= nzf || kx < 0 || kx >= nxf) continue;
                double2 A = fine.entry(f, iz, ix, k);
                if (A.x == 0.0 && A.y == 0.0) continue;
                for (int dJ = -1; dJ <= 1; ++dJ) {
                    int Jp = J + dJ;
                    if (Jp < 0 || Jp >= nzc) continue;
                    double pz = pw(kz, Jp);
                    if (pz == 0.0) continue;
                    for (int dI = -1; dI <= 1; ++dI) {
                        int Ip = I + dI;
                        if (Ip < 0 || Ip >= nxc) continue;
                        double px = pw(kx, Ip);
                        if (px == 0.0) continue;
                        double wgt = wr * pz * px;
                        int t = (dJ + 1) * 3 + (dI + 1);
                        acc[t].x += wgt * A.x;
                        acc[t].y += wgt * A.y;
                    }
                }
            }
        }
    }
    const size_t plane = (size_t)nxc * nzc;
    float2* o = out + (size_t)f * 9 * plane;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[(size_t)k * plane + (size_t)J * nxc + I] = make_float2((float)acc[k].x, (float)acc[k].y);
}

dim3 grid2(int nx, int nz, int nb) { return dim3((nx + 31) / 32, (nz + 7) / 8, nb); }

// ---------------------------------------------------------------------------
// Block shapes of the Jacobi sweeps, chosen by timing.  While tuning is on (see
// stencil_tuning), the first launch of a sweep on a (kernel, grid) pair runs each
// candidate shape twice, times the second run with CUDA events on the context's
// stream, and records the fastest in a process-wide table that every later launch
// on that grid uses (any batch size).  Re-running a sweep is harmless: its output
// never aliases its input.
// ---------------------------------------------------------------------------
constexpr int N_SHAPES = 6;
constexpr int SHAPES[N_SHAPES][2] = {{32, 8}, {64, 4}, {32, 4}, {128, 2}, {32, 16}, {16, 16}};
std::mutex g_shape_mu;
std::map<std::tuple<int, int, int>, int> g_shape;   // (kernel, nx, nz) -> index into SHAPES
std::atomic<int> g_stencil_tuning{0};

int shape_of(int kernel, int nx, int nz, bool* tune) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shape.find(std::make_tuple(kernel, nx, nz));
    if (it != g_shape.end()) {
        *tune = false;
        return it->second;
    }
    *tune = g_stencil_tuning.load() != 0;
    return 0;
}

// launch(shape index) for every candidate, timed; records and returns the fastest index
template <class F>
int tune_shape(const helm_ctx* c, int kernel, int nx, int nz, F launch) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return 0;
    }
    int best = 0;
    float best_ms = 1e30f;
    for (int i = 0; i < N_SHAPES; ++i) {
        launch(i);
        cudaEventRecord(e0, c->stream);
        launch(i);
        cudaEventRecord(e1, c->stream);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape[std::make_tuple(kernel, nx, nz)] = best;
    return best;
}

}  // namespace

void stencil_tuning(bool on) { g_stencil_tuning.store(on ? 1 : 0); }
int stencil_tuned_count() {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    return (int)g_shape.size();
}
void stencil_tune_reset() {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape.clear();
}

template <class Op>
int launch_jacobi(const helm_ctx* c, const Op& op, float2* u_out, const float2* u_in, const float2* f, int nx,
                  int nz, int nb, const int* mask) {
    LaunchScope scope(c, (std::is_same<Op, OpFine5>::value ? K_JACOBI_FINE : K_JACOBI_COARSE));
    if constexpr (std::is_same<Op, OpFine5>::value) {
        if (u_in && nx % 2 == 0) {
            const Tally tl = tally(c, K_JACOBI_FINE, 24ull * nx * nz);
            auto launch = [&](int i) {
                const int bx = SHAPES[i][0], by = SHAPES[i][1];
                const dim3 g((nx / 2 + bx - 1) / bx, (nz + by - 1) / by, nb);
                { jacobi_fine2_kernel<<<g, dim3(bx, by), 0, c->stream>>>(op, u_out, u_in, f, c->opt.jacobi_w, nx, nz,
                                                                        mask, tl); count_launch(); }
            };
            bool tune = false;
            int i = shape_of(0, nx, nz, &tune);
            if (tune && u_out != u_in) i = tune_shape(c, 0, nx, nz, launch);
            launch(i);
            HELM_CK(cudaGetLastError());
            return HELM_OK;
        }
    }
    if constexpr (std::is_same<Op, OpC9>::value) {
        const Tally tl = tally(c, K_JACOBI_COARSE, (u_in ? 24ull : 16ull) * nx * nz);
        auto launch = [&](int i) {
            const int bx = SHAPES[i][0], by = SHAPES[i][1];
            const dim3 g((nx + bx - 1) / bx, (nz + by - 1) / by, (nb + 1) / 2);
            { jacobi_c9_pair_kernel<<<g, dim3(bx, by), 0, c->stream>>>(op, u_out, u_in, f, c->opt.jacobi_w, nx, nz, nb,
                                                                      mask, tl); count_launch(); }
        };
        bool tune = false;
        int i = shape_of(1, nx, nz, &tune);
        if (tune && u_out != u_in) i = tune_shape(c, 1, nx, nz, launch);
        launch(i);
        HELM_CK(cudaGetLastError());
        return HELM_OK;
    }
    { jacobi_kernel<Op><<<grid2(nx, nz, nb), dim3(32, 8), 0, c->stream>>>(
        op, u_out, u_in, f, c->opt.jacobi_w, nx, nz, mask,
        tally(c, std::is_same<Op, OpFine5>::value ? K_JACOBI_FINE : K_JACOBI_COARSE,
              (u_in ? 24ull : 16ull) * nx * nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}
template int launch_jacobi<OpFine5>(const helm_ctx*, const OpFine5&, float2*, const float2*, const float2*, int,
                                    int, int, const int*);
template int launch_jacobi<OpC9>(const helm_ctx*, const OpC9&, float2*, const float2*, const float2*, int, int,
                                 int, const int*);

template <class Op>
int launch_restrict_residual(const helm_ctx* c, const Op& op, float2* rc, const float2* u, const float2* f,
                             int nx, int nz, int nb, const int* mask) {
    LaunchScope scope(c, (std::is_same<Op, OpFine5>::value ? K_RESTRICT_FINE : K_RESTRICT_COARSE));
    { restrict_residual_tiled_kernel<Op><<<grid2(nx / 2, nz / 2, nb), dim3(32, 8), 0, c->stream>>>(
        op, rc, u, f, nx, nz, mask,
        tally(c, std::is_same<Op, OpFine5>::value ? K_RESTRICT_FINE : K_RESTRICT_COARSE,
              (u ? 16ull : 8ull) * nx * nz + 2ull * nx * nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}
template int launch_restrict_residual<OpFine5>(const helm_ctx*, const OpFine5&, float2*, const float2*,
                                               const float2*, int, int, int, const int*);
template int launch_restrict_residual<OpC9>(const helm_ctx*, const OpC9&, float2*, const float2*, const float2*,
                                            int, int, int, const int*);

int launch_prolong_add(const helm_ctx* c, float2* u, const float2* ec, int nx, int nz, int nb, const int* mask) {
    LaunchScope scope(c, K_PROLONG);
    if (nx % 2 == 0) {
        { prolong_add2_kernel<<<grid2(nx / 2, nz, nb), dim3(32, 8), 0, c->stream>>>(
            u, ec, nx, nz, mask, tally(c, K_PROLONG, 18ull * nx * nz)); count_launch(); }
        HELM_CK(cudaGetLastError());
        return HELM_OK;
    }
    { prolong_add_kernel<<<grid2(nx, nz, nb), dim3(32, 8), 0, c->stream>>>(u, ec, nx, nz, mask,
                                                                          tally(c, K_PROLONG, 18ull * nx * nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_copy_masked(const helm_ctx* c, float2* dst, const float2* src, size_t n, int nb, const int* mask) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 148) blocks = 148;
    LaunchScope scope(c, K_COPY);
    { copy_masked_kernel<<<dim3((unsigned)blocks, nb), 256, 0, c->stream>>>(dst, src, n, mask, tally(c, K_COPY, 16ull * n)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_galerkin(helm_ctx* c, int level) {
    // builds lev[level].coef9 from lev[level-1] for every frequency
    const Level& F = c->lev[level - 1];
    for (int f = 0; f < c->nfreq; ++f) {
        dim3 grid((F.nx / 2 + 31) / 32, (F.nz / 2 + 7) / 8);
        if (level == 1) {
            LaunchScope scope(c, K_GALERKIN);
            { galerkin_kernel<OpFine5><<<grid, dim3(32, 8), 0, c->stream>>>(fine_op(c, 1), f, c->lev[level].coef9,
                                                                         F.nx, F.nz); count_launch(); }
        } else {
            LaunchScope scope(c, K_GALERKIN);
            { galerkin_kernel<OpC9><<<grid, dim3(32, 8), 0, c->stream>>>(coarse_op(c, level - 1), f,
                                                                      c->lev[level].coef9, F.nx, F.nz); count_launch(); }
        }
        HELM_CK(cudaGetLastError());
    }
    return HELM_OK;
}

}  // namespace helm
