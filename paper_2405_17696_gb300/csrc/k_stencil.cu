// Fine-grid Helmholtz kernels: the matrix-free five-point operator H(m, w)
// of Eq. 3.1-3.2 (and the shifted Laplacian of Eq. 3.12), the FP64 true
// residual used at every FGMRES restart, and the per-RHS restart logic.
#include <type_traits>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {

namespace {

constexpr int NTHREADS = TILE_X * TILE_Y;
constexpr int NWARPS = NTHREADS / 32;

__global__ void apply_fine_kernel(OpFine5 op, const float2* __restrict__ x, float2* __restrict__ y,
                                  const int* mask, Tally tl) {
    const int b = blockIdx.z;
    if (!mask[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= op.nx || iz >= op.nz) return;
    const size_t N = (size_t)op.nx * op.nz;
    y[(size_t)b * N + (size_t)iz * op.nx + ix] = op.apply(x + (size_t)b * N, b, ix, iz);
}

// r = b - H x evaluated in FP64 from the complex128 iterate x (b conjugated
// when solving the adjoint system); r is stored in complex64 as the first
// (unscaled) Krylov vector.  ||r||^2 and, on the first call, ||b||^2 are
// reduced per RHS in FP64.
__global__ void __launch_bounds__(NTHREADS) residual64_kernel(OpFine5 op, const double2* __restrict__ x,
                                                              const float2* __restrict__ bvec,
                                                              float2* __restrict__ r, int conj_b, int first,
                                                              double ax, double az, OuterState os, Tally tl) {
    const int b = blockIdx.z;
    if (!os.outer_active[b]) return;
    tally_once(tl, blockIdx.x == 0 && blockIdx.y == 0);
    const int nx = op.nx, nz = op.nz;
    const size_t N = (size_t)nx * nz;
    const double2* xb = x + (size_t)b * N;
    const float2* bb = bvec + (size_t)b * N;
    float2* rb = r + (size_t)b * N;
    const int ix = blockIdx.x * TILE_X + threadIdx.x;
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    const double wf = op.omega[op.rhs_freq[b]];
    const double w2 = wf * wf;
    double acc_r = 0.0, acc_b = 0.0;
    if (ix < nx) {
        for (int rr = 0; rr < ROWS; ++rr) {
            int iz = iz0 + rr;
            if (iz >= nz) break;
            size_t p = (size_t)iz * nx + ix;
            double2 z0 = make_double2(0.0, 0.0);
            double2 xc = xb[p];
            double2 xw = ix > 0 ? xb[p - 1] : z0;
            double2 xe = ix < nx - 1 ? xb[p + 1] : z0;
            double2 xn = iz > 0 ? xb[p - nx] : z0;
            double2 xs = iz < nz - 1 ? xb[p + nx] : z0;
            float2 mg = op.mg[p];
            double s = w2 * ((double)mg.x * (double)mg.x);
            double ci = -s * (double)mg.y;                 // c = s (1 - i gamma)
            double hx_ = ax * (2.0 * xc.x - xw.x - xe.x) + az * (2.0 * xc.x - xn.x - xs.x) - (s * xc.x - ci * xc.y);
            double hy_ = ax * (2.0 * xc.y - xw.y - xe.y) + az * (2.0 * xc.y - xn.y - xs.y) - (s * xc.y + ci * xc.x);
            float2 bv = bb[p];
            double bx = bv.x, by = conj_b ? -(double)bv.y : (double)bv.y;
            double rx = bx - hx_, ry = by - hy_;
            rb[p] = make_float2((float)rx, (float)ry);
            acc_r += rx * rx + ry * ry;
            acc_b += bx * bx + by * by;
        }
    }
    __shared__ double2 sm[NWARPS];
    double2 vals[1] = {make_double2(acc_r, acc_b)};
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = os.partials + (size_t)b * os.max_tiles;
    bool last = reduce_block_last<1>(vals, 1, part + tile, os.counters + b, ntiles, sm);
    if (last && threadIdx.x == 0 && threadIdx.y == 0) {
        double2 t = sum_partials(part, ntiles, 1, 0);
        os.rnorm2[b] = t.x;
        if (first) os.bnorm2[b] = t.y;
    }
}

__global__ void conj64_kernel(double2* x, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        x[p].y = -x[p].y;
}

// Decide per RHS after the restart residual: converged, out of steps,
// broken down, or start another cycle (g_0 = ||r||, s_0 = 1/||r||).
__global__ void restart_check_kernel(OuterState os, KState st, int nb, double tol, int max_iter, double inner,
                                     int* n_active) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int act = os.outer_active[b];
    if (act) {
        os.iters[b] += st.steps[b];
        double rn = sqrt(os.rnorm2[b]);
        double bn = sqrt(os.bnorm2[b]);
        if (!isfinite(rn) || os.status[b] == HELM_EBREAKDOWN) {
            os.status[b] = HELM_EBREAKDOWN;
            act = 0;
        } else if (bn == 0.0 || rn <= tol * bn) {
            os.status[b] = HELM_OK;
            act = 0;
        } else if (os.iters[b] >= max_iter) {
            os.status[b] = HELM_ENOCONV;
            act = 0;
        } else {
            // a restart cycle that lowered the residual by less than 10 % marks the RHS:
            // its network composition is guarded from now on
            if (os.rprev[b] > 0.0 && rn > 0.9 * os.rprev[b]) os.guard[b] = 1;
            os.rprev[b] = rn;
            st.g[(size_t)b * (st.k + 1)] = make_double2(rn, 0.0);
            st.s[(size_t)b * (st.k + 1)] = 1.0 / rn;
            st.inv_est[b] = 1.0 / rn;
            st.tol_abs[b] = inner * tol * bn;
            atomicAdd(n_active, 1);
        }
        os.outer_active[b] = act;
    }
    st.steps[b] = 0;
    st.active[b] = act;
}

__global__ void outer_init_kernel(OuterState os, KState st, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    os.iters[b] = 0;
    os.status[b] = HELM_OK;
    os.outer_active[b] = 1;
    os.rnorm2[b] = 0.0;
    os.bnorm2[b] = 0.0;
    os.rprev[b] = 0.0;
    os.guard[b] = 0;
    st.steps[b] = 0;
    st.active[b] = 0;
}

// x = 0 for right-hand sides that are identically zero
__global__ void zero_x_kernel(OuterState os, double2* x, size_t n) {
    const int b = blockIdx.y;
    if (os.bnorm2[b] != 0.0) return;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        x[(size_t)b * n + p] = make_double2(0.0, 0.0);
}

}  // namespace

int launch_apply_fine(const helm_ctx* c, const OpFine5& op, const float2* x, float2* y, int nb, const int* mask) {
    LaunchScope scope(c, K_APPLY);
    { apply_fine_kernel<<<dim3((op.nx + 31) / 32, (op.nz + 7) / 8, nb), dim3(32, 8), 0, c->stream>>>(op, x, y, mask,
                                                                                               tally(c, K_APPLY, 16ull * op.nx * op.nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_residual64(helm_ctx* c, const double2* x, const float2* b, float2* r, int nb, int conj_b, int first) {
    OpFine5 op = fine_op(c, 0);
    dim3 grid((c->nx + TILE_X - 1) / TILE_X, (c->nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS), nb);
    LaunchScope scope(c, K_RESIDUAL64);
    { residual64_kernel<<<grid, dim3(TILE_X, TILE_Y), 0, c->stream>>>(op, x, b, r, conj_b, first,
                                                                    1.0 / ((double)c->hx * c->hx),
                                                                    1.0 / ((double)c->hz * c->hz), c->outer,
                                                                    tally(c, K_RESIDUAL64, 32ull * c->nx * c->nz)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_conj64(helm_ctx* c, double2* x, int nb) {
    size_t n = (size_t)nb * npts(c);
    LaunchScope scope(c, K_MISC);
    { conj64_kernel<<<1184, 256, 0, c->stream>>>(x, n); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_outer_init(helm_ctx* c, int nb) {
    LaunchScope scope(c, K_MISC);
    { outer_init_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(c->outer, c->fine, nb); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_zero_x(helm_ctx* c, double2* x, int nb) {
    LaunchScope scope(c, K_MISC);
    { zero_x_kernel<<<dim3(64, nb), 256, 0, c->stream>>>(c->outer, x, npts(c)); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

int launch_restart_check_dev(helm_ctx* c, int nb, double tol, int* n_active_dev) {
    LaunchScope scope(c, K_RESTART);
    { restart_check_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(c->outer, c->fine, nb, tol, c->opt.max_iter, 0.7,
                                                                  n_active_dev); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

}  // namespace helm
