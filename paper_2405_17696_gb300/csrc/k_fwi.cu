// FWI data misfit and adjoint-state gradient (Eq. 3.5 with Sigma = I and no
// regulariser, Sec. 4.3).  For every (frequency j, source s):
//   u_sj  = H(m, w_j)^{-1} g_s               forward solve
//   r_sj  = P_s^T u_sj - d_sj                 residual at the receivers
//   Phi  += ||r_sj||^2
//   mu_sj = H(m, w_j)^{-1} P_s conj(r_sj)     adjoint solve through conjugation (Eq. 4.8)
//   grad += 2 w_j^2 Re((1 - i gamma) u_sj mu_sj)
// The last line is the derivative of Eq. 3.5 for the operator of Eq. 3.1:
// dH/dm_k = -w^2 (1 - i gamma_k) e_k e_k^T gives du = w^2 H^{-1} diag((1 - i gamma) u) dm,
// and H^* = conj(H) (complex symmetry) turns the adjoint solve into a forward
// solve of the conjugated receiver residual.
#include <type_traits>
#include <vector>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {
namespace {

// g_s = e_{src} / (hx hz) for every RHS slot b of a chunk that starts at global slot b0,
// global slot b0 + b = j * nsrc + s
__global__ void point_sources_kernel(float2* __restrict__ g, const int* __restrict__ src, int nsrc, int b0,
                                     size_t n, float amp) {
    const int b = blockIdx.y;
    const int s = (b0 + b) % nsrc;
    const int k = src[s];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        g[(size_t)b * n + p] = make_float2(p == (size_t)k ? amp : 0.f, 0.f);
}

// r = P^T u - d at the receivers of every RHS; misfit partial per RHS (FP64)
__global__ void receiver_residual_kernel(const double2* __restrict__ u, const float2* __restrict__ d,
                                         const int* __restrict__ rcv, int nrcv, size_t n, double2* __restrict__ r,
                                         double* __restrict__ phi_rhs) {
    const int b = blockIdx.x;
    __shared__ double sm[32];
    double acc = 0.0;
    for (int q = threadIdx.x; q < nrcv; q += blockDim.x) {
        double2 uv = u[(size_t)b * n + rcv[q]];
        float2 dv = d[(size_t)b * nrcv + q];
        double2 rv = make_double2(uv.x - dv.x, uv.y - dv.y);
        r[(size_t)b * nrcv + q] = rv;
        acc += rv.x * rv.x + rv.y * rv.y;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        phi_rhs[b] = t;
    }
}

// q = P conj(r): the conjugated receiver residual scattered onto the grid
// (receivers at distinct nodes; a repeated node accumulates)
__global__ void scatter_adjoint_kernel(const double2* __restrict__ r, const int* __restrict__ rcv, int nrcv,
                                       size_t n, float2* __restrict__ q) {
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < nrcv; i += blockDim.x) {
        double2 rv = r[(size_t)b * nrcv + i];
        atomicAdd(&q[(size_t)b * n + rcv[i]].x, (float)rv.x);
        atomicAdd(&q[(size_t)b * n + rcv[i]].y, (float)-rv.y);
    }
}

// grad[p] = sum_b 2 w_{f(b)}^2 Re((1 - i gamma_p) u_b[p] mu_b[p])   (FP64 accumulation)
__global__ void gradient_kernel(const double2* __restrict__ u, const double2* __restrict__ mu,
                                const float2* __restrict__ mg, const float* __restrict__ omega,
                                const int* __restrict__ rhs_freq, int nb, size_t n, float* __restrict__ grad,
                                int accumulate) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        double gam = mg[p].y;
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) {
            double2 a = u[(size_t)b * n + p], m = mu[(size_t)b * n + p];
            double2 um = make_double2(a.x * m.x - a.y * m.y, a.x * m.y + a.y * m.x);
            // Re((1 - i gam) um) = um.x + gam um.y
            double w = omega[rhs_freq[b]];
            acc += 2.0 * w * w * (um.x + gam * um.y);
        }
        grad[p] = (float)(accumulate ? (double)grad[p] + acc : acc);
    }
}

__global__ void zero_c64_kernel(float2* q, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        q[p] = make_float2(0.f, 0.f);
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" int fwi_misfit_grad(helm_ctx* c, const int* src_idx, int nsrc, const int* rcv_idx, int nrcv,
                               const helm_c64* d_obs, double tol, double* misfit_out, float* grad_m_out) {
    set_error("");
    if (!c || !src_idx || !rcv_idx || !d_obs || !misfit_out || !grad_m_out || nsrc < 1 || nrcv < 1 || !(tol > 0)) {
        set_error("fwi_misfit_grad: invalid argument");
        return HELM_EINVAL;
    }
    const size_t N = npts(c);
    for (int i = 0; i < nsrc; ++i)
        if (src_idx[i] < 0 || (size_t)src_idx[i] >= N) { set_error("fwi_misfit_grad: source index outside the grid"); return HELM_EINVAL; }
    for (int i = 0; i < nrcv; ++i)
        if (rcv_idx[i] < 0 || (size_t)rcv_idx[i] >= N) { set_error("fwi_misfit_grad: receiver index outside the grid"); return HELM_EINVAL; }
    const int nfreq = c->nfreq;
    const int nb_tot = nfreq * nsrc;
    // chunks of up to max_rhs (frequency, source) slots, a frequency's sources possibly split
    const int nbc = c->cap < nb_tot ? c->cap : nb_tot;
    if (nbc < 1) { set_error("fwi_misfit_grad: context without RHS capacity"); return HELM_EINVAL; }

    float2 *g = nullptr, *q = nullptr, *d_dev = nullptr;
    float* grad_dev = nullptr;
    double2 *u = nullptr, *mu = nullptr, *r = nullptr;
    double* phi = nullptr;
    int *src = nullptr, *rcv = nullptr;
    int status = HELM_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && status == HELM_OK) { set_error(cudaGetErrorString(e)); status = HELM_ECUDA; }
        return status == HELM_OK;
    };
    bool grad_is_dev = false;
    {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, grad_m_out) == cudaSuccess)
            grad_is_dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        (void)cudaGetLastError();
    }
    bool d_is_dev = false;
    {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, d_obs) == cudaSuccess)
            d_is_dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        (void)cudaGetLastError();
    }
    ck(cudaMalloc(&g, (size_t)nbc * N * sizeof(float2)));
    ck(cudaMalloc(&q, (size_t)nbc * N * sizeof(float2)));
    ck(cudaMalloc(&u, (size_t)nbc * N * sizeof(double2)));
    ck(cudaMalloc(&mu, (size_t)nbc * N * sizeof(double2)));
    ck(cudaMalloc(&r, (size_t)nbc * nrcv * sizeof(double2)));
    ck(cudaMalloc(&phi, (size_t)nb_tot * sizeof(double)));
    ck(cudaMalloc(&src, nsrc * sizeof(int)));
    ck(cudaMalloc(&rcv, nrcv * sizeof(int)));
    if (!d_is_dev) ck(cudaMalloc(&d_dev, (size_t)nb_tot * nrcv * sizeof(float2)));
    if (!grad_is_dev) ck(cudaMalloc(&grad_dev, N * sizeof(float)));
    if (status == HELM_OK) {
        ck(cudaMemcpyAsync(src, src_idx, nsrc * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        ck(cudaMemcpyAsync(rcv, rcv_idx, nrcv * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        if (!d_is_dev)
            ck(cudaMemcpyAsync(d_dev, d_obs, (size_t)nb_tot * nrcv * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
        ck(cudaStreamSynchronize(c->stream));
    }
    const float2* dptr = d_is_dev ? (const float2*)d_obs : d_dev;
    float* gptr = grad_is_dev ? grad_m_out : grad_dev;
    std::vector<int> fidx(nbc);
    for (int b0 = 0; b0 < nb_tot && status == HELM_OK; b0 += nbc) {
        const int nb = nb_tot - b0 < nbc ? nb_tot - b0 : nbc;
        for (int i = 0; i < nb; ++i) fidx[i] = (b0 + i) / nsrc;
        {
            LaunchScope scope(c, K_MISC);
            { point_sources_kernel<<<dim3(64, nb), 256, 0, c->stream>>>(g, src, nsrc, b0, N, 1.0f / (c->hx * c->hz)); count_launch(); }
            ck(cudaGetLastError());
        }
        if (status) break;
        int s = helm_solve(c, (const helm_c64*)g, (helm_c128*)u, nb, fidx.data(), tol, HELM_SOLVE_ZERO_X0, nullptr);
        if (s != HELM_OK) { status = s; break; }
        {
            LaunchScope scope(c, K_MISC);
            { receiver_residual_kernel<<<nb, 256, 0, c->stream>>>(u, dptr + (size_t)b0 * nrcv, rcv, nrcv, N, r,
                                                                  phi + b0); count_launch(); }
            ck(cudaGetLastError());
        }
        {
            LaunchScope scope(c, K_MISC);
            { zero_c64_kernel<<<1184, 256, 0, c->stream>>>(q, (size_t)nb * N); count_launch(); }
            ck(cudaGetLastError());
        }
        {
            LaunchScope scope(c, K_MISC);
            { scatter_adjoint_kernel<<<nb, 256, 0, c->stream>>>(r, rcv, nrcv, N, q); count_launch(); }
            ck(cudaGetLastError());
        }
        if (status) break;
        s = helm_solve(c, (const helm_c64*)q, (helm_c128*)mu, nb, fidx.data(), tol, HELM_SOLVE_ZERO_X0, nullptr);
        if (s != HELM_OK) { status = s; break; }
        // helm_solve left the frequency of every slot in rhs_freq
        {
            LaunchScope scope(c, K_MISC);
            { gradient_kernel<<<1184, 256, 0, c->stream>>>(u, mu, c->mg, c->omega_d, c->rhs_freq, nb, N, gptr,
                                                         b0 > 0 ? 1 : 0); count_launch(); }
            ck(cudaGetLastError());
        }
    }
    std::vector<double> hphi(nb_tot, 0.0);
    if (status == HELM_OK) {
        ck(cudaMemcpyAsync(hphi.data(), phi, nb_tot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (!grad_is_dev) ck(cudaMemcpyAsync(grad_m_out, grad_dev, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        ck(cudaStreamSynchronize(c->stream));
    }
    if (status == HELM_OK) {
        double t = 0.0;
        for (double v : hphi) t += v;
        *misfit_out = t;
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(g); cudaFree(q); cudaFree(u); cudaFree(mu); cudaFree(r); cudaFree(phi); cudaFree(src); cudaFree(rcv);
    if (d_dev) cudaFree(d_dev);
    if (grad_dev) cudaFree(grad_dev);
    return status;
}
