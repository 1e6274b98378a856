// Sensitivity products and the Gauss-Newton iteration of frequency-domain FWI
// (Sec. 3.2-3.3, Alg. 1; the sensitivity of Eq. 3.10 written out from the
// operator of Eq. 3.1).  For a survey of encoded sources (simultaneous sources,
// Sec. 3.2: source k is sum_s w_ks e_{src_s} / (hx hz), or the point sources
// themselves) and shared receivers, per frequency j and source k:
//   u   = H(m, w_j)^{-1} q_k                                        forward field
//   J v : du = w_j^2 H^{-1} ((1 - i gamma) u v),  (J v)_jk = P^T du    (tol_sens)
//   J^T d: mu = H^{-1} P conj(d_jk),  (J^T d) += w_j^2 Re((1 - i gamma) u mu)
//          (the conjugation identity of Sec. 4.3 turns H^* into a forward solve;
//           J^T is Re(J^H), the adjoint for real model perturbations)
//   Gauss-Newton on Phi(m) + a R(m) (Eq. 3.5 and a regulariser of Sec. 5.1 on
//   v = m - m_ref, R = v^T K v with K = L or L^2, L = -Lap_h): dm by cg_iters
//   conjugate gradient steps on (J^T J + a K + reg I) dm = -(J^T r + a K v) from
//   dm = 0, r = P^T u - d_obs, then a backtracking step m <- clip(m + alpha dm),
//   alpha = 1, 1/2, ... while the objective does not drop.
// Every solve is helm_solve with the context's preconditioner (multigrid or the
// encoder-solver network), and the Helmholtz iterations of every solve are
// counted.  Model-space vectors are FP64 on the device; their inner products
// are per-block partial sums added in a fixed order.
#include <cmath>
#include <string>
#include <vector>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {
namespace {

constexpr int DOT_BLOCKS = 512;

// q[b] = sum_s w[k(b)][s] e_{src[s]} amp for the RHS b of a chunk (k(b) = (b0 + b) % nsim);
// w == nullptr: source k is the point source k.  One thread per RHS, sources in order.
__global__ void encoded_sources_kernel(float2* __restrict__ q, const int* __restrict__ src, const float* __restrict__ w,
                                       int nsrc, int nsim, int b0, int nb, size_t n, float amp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int k = (b0 + b) % nsim;
    float2* qb = q + (size_t)b * n;
    if (!w) {
        qb[src[k]].x += amp;
        return;
    }
    for (int s = 0; s < nsrc; ++s) qb[src[s]].x += amp * w[(size_t)k * nsrc + s];
}

// d[b][q] = u[b][rcv[q]]  (complex128 field -> complex64 data)
__global__ void sample_kernel(const double2* __restrict__ u, const int* __restrict__ rcv, int nrcv, size_t n, int nb,
                              float2* __restrict__ d) {
    const long long total = (long long)nb * nrcv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / nrcv), q = (int)(i % nrcv);
        const double2 v = u[(size_t)b * n + rcv[q]];
        d[i] = make_float2((float)v.x, (float)v.y);
    }
}

// r[b][q] = P^T u - d_obs in FP64 and the misfit of every RHS (one block per RHS)
__global__ void data_residual_kernel(const double2* __restrict__ u, const float2* __restrict__ d_obs,
                                     const int* __restrict__ rcv, int nrcv, size_t n, float2* __restrict__ r,
                                     double* __restrict__ phi) {
    const int b = blockIdx.x;
    double acc = 0.0;
    for (int q = threadIdx.x; q < nrcv; q += blockDim.x) {
        const double2 uv = u[(size_t)b * n + rcv[q]];
        const float2 dv = d_obs[(size_t)b * nrcv + q];
        const double rx = uv.x - dv.x, ry = uv.y - dv.y;
        r[(size_t)b * nrcv + q] = make_float2((float)rx, (float)ry);
        acc += rx * rx + ry * ry;
    }
    __shared__ double sm[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        phi[b] = t;
    }
}

// q[b] = P conj(d[b]) (q zeroed before; one thread per RHS adds its receivers in order)
__global__ void scatter_conj_kernel(const float2* __restrict__ d, const int* __restrict__ rcv, int nrcv, size_t n, int nb,
                                    float2* __restrict__ q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int i = 0; i < nrcv; ++i) {
        const float2 v = d[(size_t)b * nrcv + i];
        float2* t = q + (size_t)b * n + rcv[i];
        t->x += v.x;
        t->y -= v.y;
    }
}

// f[b] = w_b^2 (1 - i gamma) u_b v   (the right-hand side of the sensitivity solve)
__global__ void born_rhs_kernel(const double2* __restrict__ u, const double* __restrict__ v,
                                const float2* __restrict__ mg, const float* __restrict__ omega,
                                const int* __restrict__ rhs_freq, int nb, size_t n, float2* __restrict__ f) {
    const long long total = (long long)nb * (long long)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / (long long)n);
        const size_t p = (size_t)(i - (long long)b * (long long)n);
        const double w = omega[rhs_freq[b]];
        const double s = w * w * v[p], g = mg[p].y;
        const double2 a = u[i];
        // (1 - i g)(a.x + i a.y) = (a.x + g a.y) + i (a.y - g a.x)
        f[i] = make_float2((float)(s * (a.x + g * a.y)), (float)(s * (a.y - g * a.x)));
    }
}

// acc[p] += scale sum_b w_b^2 Re((1 - i gamma_p) u_b[p] mu_b[p])   (FP64, RHS in order)
__global__ void adjoint_accum_kernel(const double2* __restrict__ u, const double2* __restrict__ mu,
                                     const float2* __restrict__ mg, const float* __restrict__ omega,
                                     const int* __restrict__ rhs_freq, int nb, size_t n, double scale,
                                     double* __restrict__ acc) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const double g = mg[p].y;
        double t = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double2 a = u[(size_t)b * n + p], m = mu[(size_t)b * n + p];
            const double re = a.x * m.x - a.y * m.y, im = a.x * m.y + a.y * m.x;
            const double w = omega[rhs_freq[b]];
            t += w * w * (re + g * im);
        }
        acc[p] += scale * t;
    }
}

// per-block partial sums of a . b (fixed grid, fixed order)
__global__ void dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                                   double* __restrict__ part) {
    double t = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        t += a[p] * b[p];
    __shared__ double sm[32];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
        part[blockIdx.x] = s;
    }
}

// y = a x + b y
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        y[p] = a * x[p] + b * y[p];
}

// y = a L v + b y (b = 0: y is not read), L = G^T G the negative five-point Laplacian of the
// regularisers of Sec. 5.1: G takes forward differences on the interior edges (scaled by 1/hx,
// 1/hz), so (L v)_p = sum over the neighbours q of p of (v_p - v_q) / h^2 and the boundary is
// natural (no edge leaves the grid).  ax = 1/hx^2, az = 1/hz^2.
__global__ void neg_lap_kernel(const double* __restrict__ v, double* __restrict__ y, int nx, int nz, double ax,
                               double az, double a, double b) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    if (ix >= nx || iz >= nz) return;
    const size_t p = (size_t)iz * nx + ix;
    const double vc = v[p];
    double s = 0.0;
    if (ix > 0) s += ax * (vc - v[p - 1]);
    if (ix < nx - 1) s += ax * (vc - v[p + 1]);
    if (iz > 0) s += az * (vc - v[p - nx]);
    if (iz < nz - 1) s += az * (vc - v[p + nx]);
    y[p] = b == 0.0 ? a * s : a * s + b * y[p];
}

// v = m - m_ref in FP64 (m_ref null: zero)
__global__ void model_diff_kernel(const float* __restrict__ m, const float* __restrict__ m_ref, double* __restrict__ v,
                                  size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        v[p] = (double)m[p] - (m_ref ? (double)m_ref[p] : 0.0);
}

__global__ void f64_of_f32_kernel(const float* __restrict__ x, double* __restrict__ y, double s, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        y[p] = s * (double)x[p];
}
__global__ void f32_of_f64_kernel(const double* __restrict__ x, float* __restrict__ y, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        y[p] = (float)x[p];
}

// m_out = clip(m + alpha dm, lo, hi); kappa = sqrt(m_out); gamma copied from the packed medium
__global__ void model_step_kernel(const float* __restrict__ m, const double* __restrict__ dm, double alpha, float lo,
                                  float hi, const float2* __restrict__ mg, float* __restrict__ m_out,
                                  float* __restrict__ kappa, float* __restrict__ gamma, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        float v = dm ? (float)((double)m[p] + alpha * dm[p]) : m[p];
        v = fminf(fmaxf(v, lo), hi);
        m_out[p] = v;
        kappa[p] = sqrtf(v);
        gamma[p] = mg[p].y;
    }
}

// d_enc[j][k][q] = sum_s w[k][s] d[j][s][q]   (the data of the encoded sources)
__global__ void encode_data_kernel(const float2* __restrict__ d, const float* __restrict__ w, int nfreq, int nsrc,
                                   int nsim, int nrcv, float2* __restrict__ d_enc) {
    const long long total = (long long)nfreq * nsim * nrcv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i % nrcv);
        const int k = (int)((i / nrcv) % nsim);
        const int j = (int)(i / ((long long)nrcv * nsim));
        double re = 0.0, im = 0.0;
        for (int s = 0; s < nsrc; ++s) {
            const float2 v = d[((size_t)j * nsrc + s) * nrcv + q];
            const double ws = w[(size_t)k * nsrc + s];
            re += ws * v.x;
            im += ws * v.y;
        }
        d_enc[i] = make_float2((float)re, (float)im);
    }
}

__global__ void sqrt_kernel(const float* __restrict__ m, float* __restrict__ kappa, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        kappa[p] = sqrtf(fmaxf(m[p], 0.0f));
}

__global__ void zero_f2_kernel(float2* q, size_t n) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        q[p] = make_float2(0.f, 0.f);
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// One call's survey on the device, its scratch, and the solves.
class Fwi {
   public:
    Fwi(helm_ctx* c, const fwi_survey* sv) : c_(c), sv_(sv) {}
    ~Fwi() {
        cudaStreamSynchronize(c_->stream);
        for (void* p : owned_) cudaFree(p);
    }
    int init() {
        const fwi_survey* s = sv_;
        if (!s || !s->src_idx || !s->rcv_idx || s->nsrc < 1 || s->nrcv < 1 || (s->src_w && s->nsim < 1)) {
            set_error("fwi: invalid survey");
            return HELM_EINVAL;
        }
        N_ = npts(c_);
        for (int i = 0; i < s->nsrc; ++i)
            if (s->src_idx[i] < 0 || (size_t)s->src_idx[i] >= N_) { set_error("fwi: source index outside the grid"); return HELM_EINVAL; }
        for (int i = 0; i < s->nrcv; ++i)
            if (s->rcv_idx[i] < 0 || (size_t)s->rcv_idx[i] >= N_) { set_error("fwi: receiver index outside the grid"); return HELM_EINVAL; }
        nsim_ = s->src_w ? s->nsim : s->nsrc;
        nb_tot_ = c_->nfreq * nsim_;
        nbc_ = c_->cap < nb_tot_ ? c_->cap : nb_tot_;
        HELM_TRY(alloc(&src_, s->nsrc));
        HELM_TRY(alloc(&rcv_, s->nrcv));
        HELM_CK(cudaMemcpyAsync(src_, s->src_idx, s->nsrc * sizeof(int), cudaMemcpyHostToDevice, c_->stream));
        HELM_CK(cudaMemcpyAsync(rcv_, s->rcv_idx, s->nrcv * sizeof(int), cudaMemcpyHostToDevice, c_->stream));
        if (s->src_w) {
            HELM_TRY(alloc(&w_, (size_t)nsim_ * s->nsrc));
            HELM_CK(cudaMemcpyAsync(w_, s->src_w, (size_t)nsim_ * s->nsrc * sizeof(float), cudaMemcpyHostToDevice,
                                    c_->stream));
        }
        HELM_TRY(alloc(&q_, (size_t)nbc_ * N_));
        HELM_TRY(alloc(&x_, (size_t)nbc_ * N_));
        HELM_TRY(alloc(&part_, DOT_BLOCKS));
        return HELM_OK;
    }
    int nb_tot() const { return nb_tot_; }
    const int* rcv() const { return rcv_; }
    int nbc() const { return nbc_; }
    int nrcv() const { return sv_->nrcv; }
    size_t N() const { return N_; }
    long long iterations() const { return iters_; }

    template <class T>
    int alloc(T** p, size_t n) {
        if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("fwi: out of device memory");
            return HELM_ENOMEM;
        }
        owned_.push_back(*p);
        return HELM_OK;
    }
    // frequency index of the RHS b0 .. b0 + nb - 1 (frequency-major: b = j nsim + k)
    void freqs(int b0, int nb, std::vector<int>& f) const {
        f.resize(nb);
        for (int i = 0; i < nb; ++i) f[i] = (b0 + i) / nsim_;
    }
    // x = H^{-1} f for nb RHS (frequencies of b0 ..), counting Helmholtz iterations
    int solve(const float2* f, double2* x, int b0, int nb, double tol) {
        std::vector<int> fi, it(nb), st(nb);
        std::vector<double> rel(nb);
        freqs(b0, nb, fi);
        helm_stats stats{it.data(), rel.data(), st.data()};
        const int s = helm_solve(c_, (const helm_c64*)f, (helm_c128*)x, nb, fi.data(), tol, HELM_SOLVE_ZERO_X0, &stats);
        for (int i = 0; i < nb; ++i) iters_ += it[i];
        return s;
    }
    // the encoded sources of RHS b0 .. b0 + nb - 1 into q_
    int sources(int b0, int nb) {
        {
            LaunchScope scope(c_, K_MISC);
            { zero_f2_kernel<<<1184, 256, 0, c_->stream>>>(q_, (size_t)nb * N_); count_launch(); }
        }
        LaunchScope scope(c_, K_MISC);
        { encoded_sources_kernel<<<(nb + 127) / 128, 128, 0, c_->stream>>>(q_, src_, w_, sv_->nsrc, nsim_, b0, nb, N_,
                                                                         1.0f / (c_->hx * c_->hz)); count_launch(); }
        HELM_CK(cudaGetLastError());
        return HELM_OK;
    }
    // forward fields of RHS b0 .. + nb into u (complex128 [nb][N])
    int forward(int b0, int nb, double2* u, double tol) {
        HELM_TRY(sources(b0, nb));
        return solve(q_, u, b0, nb, tol);
    }
    // dd (complex64 [nb][nrcv]) = J v for RHS b0 .. + nb with forward fields u
    int jv(const double2* u, const double* v, int b0, int nb, double tol, float2* dd) {
        {
            LaunchScope scope(c_, K_MISC);
            std::vector<int> fi;
            freqs(b0, nb, fi);
            HELM_CK(cudaMemcpyAsync(c_->rhs_freq, fi.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c_->stream));
            { born_rhs_kernel<<<1184, 256, 0, c_->stream>>>(u, v, c_->mg, c_->omega_d, c_->rhs_freq, nb, N_, q_); count_launch(); }
            HELM_CK(cudaGetLastError());
            HELM_CK(cudaStreamSynchronize(c_->stream));   // fi leaves scope
        }
        HELM_TRY(solve(q_, x_, b0, nb, tol));
        LaunchScope scope(c_, K_MISC);
        { sample_kernel<<<256, 256, 0, c_->stream>>>(x_, rcv_, sv_->nrcv, N_, nb, dd); count_launch(); }
        HELM_CK(cudaGetLastError());
        return HELM_OK;
    }
    // acc += scale J^T dd for RHS b0 .. + nb with forward fields u
    int jtd(const double2* u, const float2* dd, int b0, int nb, double tol, double scale, double* acc) {
        {
            LaunchScope scope(c_, K_MISC);
            { zero_f2_kernel<<<1184, 256, 0, c_->stream>>>(q_, (size_t)nb * N_); count_launch(); }
            { scatter_conj_kernel<<<(nb + 127) / 128, 128, 0, c_->stream>>>(dd, rcv_, sv_->nrcv, N_, nb, q_); count_launch(); }
            HELM_CK(cudaGetLastError());
        }
        HELM_TRY(solve(q_, x_, b0, nb, tol));
        // helm_solve left the frequency of every slot in rhs_freq
        LaunchScope scope(c_, K_MISC);
        { adjoint_accum_kernel<<<1184, 256, 0, c_->stream>>>(u, x_, c_->mg, c_->omega_d, c_->rhs_freq, nb, N_, scale, acc); count_launch(); }
        HELM_CK(cudaGetLastError());
        return HELM_OK;
    }
    int dot(const double* a, const double* b, double* out) {
        {
            LaunchScope scope(c_, K_MISC);
            { dot_partial_kernel<<<DOT_BLOCKS, 256, 0, c_->stream>>>(a, b, N_, part_); count_launch(); }
            HELM_CK(cudaGetLastError());
        }
        std::vector<double> h(DOT_BLOCKS);
        HELM_CK(cudaMemcpyAsync(h.data(), part_, DOT_BLOCKS * sizeof(double), cudaMemcpyDeviceToHost, c_->stream));
        HELM_CK(cudaStreamSynchronize(c_->stream));
        double t = 0.0;
        for (double v : h) t += v;
        *out = t;
        return HELM_OK;
    }

    // misfit of Eq. 3.5 for the context's current medium; the forward fields go to U
    // (complex128 [nb_tot][N]) and the data residual to R ([nb_tot][nrcv]) when given
    int misfit(const float2* d_obs, double tol, double2* U, float2* R, double* phi) {
        double2* tmp = nullptr;
        float2* rtmp = nullptr;
        if (!U) HELM_TRY(alloc(&tmp, (size_t)nbc_ * N_));
        if (!R) HELM_TRY(alloc(&rtmp, (size_t)nbc_ * sv_->nrcv));
        if (!phi_dev_) HELM_TRY(alloc(&phi_dev_, (size_t)nb_tot_));
        for (int b0 = 0; b0 < nb_tot_; b0 += nbc_) {
            const int nb = std::min(nbc_, nb_tot_ - b0);
            double2* ub = U ? U + (size_t)b0 * N_ : tmp;
            float2* rb = R ? R + (size_t)b0 * sv_->nrcv : rtmp;
            HELM_TRY(forward(b0, nb, ub, tol));
            LaunchScope scope(c_, K_MISC);
            { data_residual_kernel<<<nb, 256, 0, c_->stream>>>(ub, d_obs + (size_t)b0 * sv_->nrcv, rcv_, sv_->nrcv, N_,
                                                             rb, phi_dev_ + b0); count_launch(); }
            HELM_CK(cudaGetLastError());
        }
        std::vector<double> h(nb_tot_);
        HELM_CK(cudaMemcpyAsync(h.data(), phi_dev_, nb_tot_ * sizeof(double), cudaMemcpyDeviceToHost, c_->stream));
        HELM_CK(cudaStreamSynchronize(c_->stream));
        double t = 0.0;
        for (double v : h) t += v;
        *phi = t;
        if (tmp) free_last(tmp);
        if (rtmp) free_last(rtmp);
        return HELM_OK;
    }
    void free_last(void* p) {
        cudaStreamSynchronize(c_->stream);
        for (size_t i = 0; i < owned_.size(); ++i)
            if (owned_[i] == p) {
                cudaFree(p);
                owned_.erase(owned_.begin() + (long)i);
                return;
            }
    }

   private:
    helm_ctx* c_;
    const fwi_survey* sv_;
    double* phi_dev_ = nullptr;
    size_t N_ = 0;
    int nsim_ = 0, nb_tot_ = 0, nbc_ = 0;
    int *src_ = nullptr, *rcv_ = nullptr;
    float* w_ = nullptr;
    float2* q_ = nullptr;
    double2* x_ = nullptr;
    double* part_ = nullptr;
    long long iters_ = 0;
    std::vector<void*> owned_;
};

// device copy of a host or device array of n elements (nullptr on failure)
template <class T>
const T* device_view(Fwi& F, const T* p, size_t n, cudaStream_t st, int* status) {
    if (is_device_ptr(p)) return p;
    T* d = nullptr;
    if ((*status = F.alloc(&d, n)) != HELM_OK) return nullptr;
    if (cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("fwi: upload failed");
        *status = HELM_ECUDA;
        return nullptr;
    }
    return d;
}

// copy n elements to a host or device destination
template <class T>
int copy_out(T* dst, const T* src, size_t n, cudaStream_t st) {
    HELM_CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDefault, st));
    HELM_CK(cudaStreamSynchronize(st));
    return HELM_OK;
}

// set the context's medium to m = kappa^2 (gamma kept): m_out = clip(m0 + alpha dm)
int set_model(helm_ctx* c, Fwi& F, const float* m0, const double* dm, double alpha, float lo, float hi, float* m_out) {
    const size_t N = F.N();
    float *kap = nullptr, *gam = nullptr;
    HELM_TRY(F.alloc(&kap, N));
    HELM_TRY(F.alloc(&gam, N));
    {
        LaunchScope scope(c, K_MISC);
        { model_step_kernel<<<1184, 256, 0, c->stream>>>(m0, dm, alpha, lo, hi, c->mg, m_out, kap, gam, N); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    const int s = helm_set_medium(c, kap, gam, c->omega_d, c->nfreq);
    F.free_last(gam);
    F.free_last(kap);
    return s;
}

// y = a L v + b y on the context's grid
int apply_neg_lap(helm_ctx* c, const double* v, double* y, double a, double b) {
    LaunchScope scope(c, K_MISC);
    { neg_lap_kernel<<<dim3((c->nx + 31) / 32, (c->nz + 7) / 8), dim3(32, 8), 0, c->stream>>>(
          v, y, c->nx, c->nz, 1.0 / ((double)c->hx * c->hx), 1.0 / ((double)c->hz * c->hz), a, b); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}

// The regulariser of Sec. 5.1 at the model m: R = v^T K v and K v for v = m - m_ref, with
// K = L (R_diff = ||G v||^2) or K = L^2 (R_high = ||L v||^2, L = -Lap_h).  Scratch v, t of N.
int regulariser(helm_ctx* c, Fwi& F, int kind, const float* m, const float* m_ref, double* v, double* t, double* kv,
                double* R) {
    {
        LaunchScope scope(c, K_MISC);
        { model_diff_kernel<<<1184, 256, 0, c->stream>>>(m, m_ref, v, F.N()); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    if (kind == 1) {
        HELM_TRY(apply_neg_lap(c, v, kv, 1.0, 0.0));
        return F.dot(v, kv, R);
    }
    HELM_TRY(apply_neg_lap(c, v, t, 1.0, 0.0));
    HELM_TRY(apply_neg_lap(c, t, kv, 1.0, 0.0));
    return F.dot(t, t, R);
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

void fwi_default_gn_opts(fwi_gn_opts* o) {
    if (!o) return;
    o->tol = 1e-6;
    o->tol_sens = 1e-4;
    o->cg_iters = 5;
    o->reg = 0.0f;
    o->m_min = 0.0f;
    o->m_max = 1e30f;
    o->max_backtracks = 4;
    o->reg_kind = 0;
    o->alpha = 0.0f;
    o->m_ref = nullptr;
}

int fwi_model_to_kappa(const float* m, float* kappa, long long n) {
    set_error("");
    if (!m || !kappa || n < 1 || !is_device_ptr(m) || !is_device_ptr(kappa)) {
        set_error("fwi_model_to_kappa: device arrays of n >= 1 elements expected");
        return HELM_EINVAL;
    }
    { sqrt_kernel<<<1184, 256>>>(m, kappa, (size_t)n); count_launch(); }
    HELM_CK(cudaGetLastError());
    HELM_CK(cudaDeviceSynchronize());
    return HELM_OK;
}

int fwi_forward_data(helm_ctx* c, const fwi_survey* sv, double tol, helm_c64* d_out, long long* iters_out) {
    set_error("");
    if (!c || !d_out || !(tol > 0)) { set_error("fwi_forward_data: invalid argument"); return HELM_EINVAL; }
    Fwi F(c, sv);
    HELM_TRY(F.init());
    double2* u = nullptr;
    float2* d = nullptr;
    HELM_TRY(F.alloc(&u, (size_t)F.nbc() * F.N()));
    HELM_TRY(F.alloc(&d, (size_t)F.nb_tot() * F.nrcv()));
    for (int b0 = 0; b0 < F.nb_tot(); b0 += F.nbc()) {
        const int nb = std::min(F.nbc(), F.nb_tot() - b0);
        HELM_TRY(F.forward(b0, nb, u, tol));
        LaunchScope scope(c, K_MISC);
        { sample_kernel<<<256, 256, 0, c->stream>>>(u, F.rcv(), F.nrcv(), F.N(), nb, d + (size_t)b0 * F.nrcv()); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    if (iters_out) *iters_out = F.iterations();
    return copy_out((float2*)d_out, (const float2*)d, (size_t)F.nb_tot() * F.nrcv(), c->stream);
}

int fwi_jacobian(helm_ctx* c, const fwi_survey* sv, const float* dm, double tol, helm_c64* dd_out) {
    set_error("");
    if (!c || !dm || !dd_out || !(tol > 0)) { set_error("fwi_jacobian: invalid argument"); return HELM_EINVAL; }
    Fwi F(c, sv);
    HELM_TRY(F.init());
    int st = HELM_OK;
    const float* dmd = device_view(F, dm, F.N(), c->stream, &st);
    if (st) return st;
    double* v = nullptr;
    double2* u = nullptr;
    float2* dd = nullptr;
    HELM_TRY(F.alloc(&v, F.N()));
    HELM_TRY(F.alloc(&u, (size_t)F.nbc() * F.N()));
    HELM_TRY(F.alloc(&dd, (size_t)F.nb_tot() * F.nrcv()));
    {
        LaunchScope scope(c, K_MISC);
        { f64_of_f32_kernel<<<1184, 256, 0, c->stream>>>(dmd, v, 1.0, F.N()); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    for (int b0 = 0; b0 < F.nb_tot(); b0 += F.nbc()) {
        const int nb = std::min(F.nbc(), F.nb_tot() - b0);
        HELM_TRY(F.forward(b0, nb, u, tol));
        HELM_TRY(F.jv(u, v, b0, nb, tol, dd + (size_t)b0 * F.nrcv()));
    }
    return copy_out((float2*)dd_out, (const float2*)dd, (size_t)F.nb_tot() * F.nrcv(), c->stream);
}

int fwi_jacobian_adjoint(helm_ctx* c, const fwi_survey* sv, const helm_c64* dd, double tol, float* dm_out) {
    set_error("");
    if (!c || !dd || !dm_out || !(tol > 0)) { set_error("fwi_jacobian_adjoint: invalid argument"); return HELM_EINVAL; }
    Fwi F(c, sv);
    HELM_TRY(F.init());
    int st = HELM_OK;
    const float2* ddd = device_view(F, (const float2*)dd, (size_t)F.nb_tot() * F.nrcv(), c->stream, &st);
    if (st) return st;
    double* acc = nullptr;
    double2* u = nullptr;
    float* out = nullptr;
    HELM_TRY(F.alloc(&acc, F.N()));
    HELM_TRY(F.alloc(&u, (size_t)F.nbc() * F.N()));
    HELM_TRY(F.alloc(&out, F.N()));
    HELM_CK(cudaMemsetAsync(acc, 0, F.N() * sizeof(double), c->stream));
    for (int b0 = 0; b0 < F.nb_tot(); b0 += F.nbc()) {
        const int nb = std::min(F.nbc(), F.nb_tot() - b0);
        HELM_TRY(F.forward(b0, nb, u, tol));
        HELM_TRY(F.jtd(u, ddd + (size_t)b0 * F.nrcv(), b0, nb, tol, 1.0, acc));
    }
    {
        LaunchScope scope(c, K_MISC);
        { f32_of_f64_kernel<<<1184, 256, 0, c->stream>>>(acc, out, F.N()); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    return copy_out(dm_out, (const float*)out, F.N(), c->stream);
}

int fwi_gn_iteration(helm_ctx* c, const fwi_survey* sv, const helm_c64* d_obs, const fwi_gn_opts* opts, float* m,
                     fwi_gn_info* info) {
    set_error("");
    if (!c || !d_obs || !m) { set_error("fwi_gn_iteration: invalid argument"); return HELM_EINVAL; }
    fwi_gn_opts o;
    fwi_default_gn_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0) || !(o.tol_sens > 0) || o.cg_iters < 0 || !(o.reg >= 0) || !(o.m_max > o.m_min) ||
        o.max_backtracks < 0 || o.reg_kind < 0 || o.reg_kind > 2 || !(o.alpha >= 0) || !std::isfinite(o.alpha)) {
        set_error("fwi_gn_iteration: invalid options");
        return HELM_EINVAL;
    }
    // the regulariser's term (none when its weight is zero)
    const int rk = o.alpha > 0 ? o.reg_kind : 0;
    const double ra = rk ? (double)o.alpha : 0.0;
    Fwi F(c, sv);
    HELM_TRY(F.init());
    const size_t N = F.N();
    int st = HELM_OK;
    // observed data per point source; encoded here for simultaneous sources
    const size_t nd_pt = (size_t)c->nfreq * sv->nsrc * sv->nrcv;
    const float2* dobs = device_view(F, (const float2*)d_obs, nd_pt, c->stream, &st);
    if (st) return st;
    if (sv->src_w) {
        float2* denc = nullptr;
        float* wd = nullptr;
        HELM_TRY(F.alloc(&denc, (size_t)F.nb_tot() * F.nrcv()));
        HELM_TRY(F.alloc(&wd, (size_t)sv->nsim * sv->nsrc));
        HELM_CK(cudaMemcpyAsync(wd, sv->src_w, (size_t)sv->nsim * sv->nsrc * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream));
        LaunchScope scope(c, K_MISC);
        { encode_data_kernel<<<256, 256, 0, c->stream>>>(dobs, wd, c->nfreq, sv->nsrc, sv->nsim, sv->nrcv, denc); count_launch(); }
        HELM_CK(cudaGetLastError());
        dobs = denc;
    }
    const float* mref = nullptr;
    if (rk && o.m_ref) {
        mref = device_view(F, o.m_ref, N, c->stream, &st);
        if (st) return st;
    }
    float *m0 = nullptr, *mt = nullptr;
    double *g = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *ap = nullptr;
    double *rv = nullptr, *rt = nullptr, *rkv = nullptr;
    if (rk) {
        HELM_TRY(F.alloc(&rv, N));
        HELM_TRY(F.alloc(&rt, N));
        HELM_TRY(F.alloc(&rkv, N));
    }
    double2* U = nullptr;
    float2 *R = nullptr, *dd = nullptr;
    HELM_TRY(F.alloc(&m0, N));
    HELM_TRY(F.alloc(&mt, N));
    HELM_TRY(F.alloc(&g, N));
    HELM_TRY(F.alloc(&x, N));
    HELM_TRY(F.alloc(&r, N));
    HELM_TRY(F.alloc(&p, N));
    HELM_TRY(F.alloc(&ap, N));
    HELM_TRY(F.alloc(&U, (size_t)F.nb_tot() * N));
    HELM_TRY(F.alloc(&R, (size_t)F.nb_tot() * F.nrcv()));
    HELM_TRY(F.alloc(&dd, (size_t)F.nbc() * F.nrcv()));
    HELM_CK(cudaMemcpyAsync(m0, m, N * sizeof(float), cudaMemcpyDefault, c->stream));
    // the medium of the current model (clipped to the bounds)
    HELM_TRY(set_model(c, F, m0, nullptr, 0.0, o.m_min, o.m_max, m0));
    long long it0 = F.iterations();
    double phi0 = 0.0;
    HELM_TRY(F.misfit(dobs, o.tol, U, R, &phi0));
    const long long it_fwd = F.iterations() - it0;
    // gradient of Eq. 3.5: 2 J^T r with the tolerance of the forward problem
    HELM_CK(cudaMemsetAsync(g, 0, N * sizeof(double), c->stream));
    it0 = F.iterations();
    for (int b0 = 0; b0 < F.nb_tot(); b0 += F.nbc()) {
        const int nb = std::min(F.nbc(), F.nb_tot() - b0);
        HELM_TRY(F.jtd(U + (size_t)b0 * N, R + (size_t)b0 * F.nrcv(), b0, nb, o.tol, 2.0, g));
    }
    const long long it_adj = F.iterations() - it0;
    // the regulariser at the current model: objective Phi + alpha R, gradient += 2 alpha K v
    double R0 = 0.0;
    if (rk) {
        HELM_TRY(regulariser(c, F, rk, m0, mref, rv, rt, rkv, &R0));
        LaunchScope scope(c, K_MISC);
        { axpby_kernel<<<1184, 256, 0, c->stream>>>(2.0 * ra, rkv, 1.0, g, N); count_launch(); }
        HELM_CK(cudaGetLastError());
    }
    const double obj0 = phi0 + ra * R0;
    // conjugate gradients on (J^T J + alpha K + reg I) x = -g / 2 from x = 0
    HELM_CK(cudaMemsetAsync(x, 0, N * sizeof(double), c->stream));
    {
        LaunchScope scope(c, K_MISC);
        { axpby_kernel<<<1184, 256, 0, c->stream>>>(-0.5, g, 0.0, r, N); count_launch(); }   // r = -g / 2
        { axpby_kernel<<<1184, 256, 0, c->stream>>>(1.0, r, 0.0, p, N); count_launch(); }    // p = r
        HELM_CK(cudaGetLastError());
    }
    double rr = 0.0;
    HELM_TRY(F.dot(r, r, &rr));
    it0 = F.iterations();
    int cg_done = 0;
    for (int k = 0; k < o.cg_iters && rr > 0.0; ++k, ++cg_done) {
        HELM_CK(cudaMemsetAsync(ap, 0, N * sizeof(double), c->stream));
        for (int b0 = 0; b0 < F.nb_tot(); b0 += F.nbc()) {
            const int nb = std::min(F.nbc(), F.nb_tot() - b0);
            HELM_TRY(F.jv(U + (size_t)b0 * N, p, b0, nb, o.tol_sens, dd));
            HELM_TRY(F.jtd(U + (size_t)b0 * N, dd, b0, nb, o.tol_sens, 1.0, ap));
        }
        if (o.reg > 0) {
            LaunchScope scope(c, K_MISC);
            { axpby_kernel<<<1184, 256, 0, c->stream>>>((double)o.reg, p, 1.0, ap, N); count_launch(); }
            HELM_CK(cudaGetLastError());
        }
        if (rk == 1) {
            HELM_TRY(apply_neg_lap(c, p, ap, ra, 1.0));   // ap += alpha L p
        } else if (rk == 2) {
            HELM_TRY(apply_neg_lap(c, p, rt, 1.0, 0.0));
            HELM_TRY(apply_neg_lap(c, rt, ap, ra, 1.0));  // ap += alpha L^2 p
        }
        double pap = 0.0;
        HELM_TRY(F.dot(p, ap, &pap));
        if (!(pap > 0.0)) break;
        const double alpha = rr / pap;
        {
            LaunchScope scope(c, K_MISC);
            { axpby_kernel<<<1184, 256, 0, c->stream>>>(alpha, p, 1.0, x, N); count_launch(); }     // x += alpha p
            { axpby_kernel<<<1184, 256, 0, c->stream>>>(-alpha, ap, 1.0, r, N); count_launch(); }   // r -= alpha A p
            HELM_CK(cudaGetLastError());
        }
        double rr_new = 0.0;
        HELM_TRY(F.dot(r, r, &rr_new));
        {
            LaunchScope scope(c, K_MISC);
            { axpby_kernel<<<1184, 256, 0, c->stream>>>(1.0, r, rr_new / rr, p, N); count_launch(); }   // p = r + beta p
            HELM_CK(cudaGetLastError());
        }
        rr = rr_new;
    }
    const long long it_sens = F.iterations() - it0;
    // backtracking: m <- clip(m0 + alpha x) for alpha = 1, 1/2, ... while the objective does not drop
    it0 = F.iterations();
    double step = 1.0, phi1 = phi0, obj1 = obj0;
    bool accepted = false;
    for (int t = 0; t <= o.max_backtracks; ++t, step *= 0.5) {
        HELM_TRY(set_model(c, F, m0, x, step, o.m_min, o.m_max, mt));
        HELM_TRY(F.misfit(dobs, o.tol, nullptr, nullptr, &phi1));
        double R1 = 0.0;
        if (rk) HELM_TRY(regulariser(c, F, rk, mt, mref, rv, rt, rkv, &R1));
        obj1 = phi1 + ra * R1;
        if (obj1 < obj0) { accepted = true; break; }
    }
    const long long it_ls = F.iterations() - it0;
    if (accepted) {
        HELM_TRY(copy_out(m, (const float*)mt, N, c->stream));
    } else {
        // no step lowered the misfit: keep the model (and its medium)
        HELM_TRY(set_model(c, F, m0, nullptr, 0.0, o.m_min, o.m_max, mt));
        step = 0.0;
        phi1 = phi0;
        obj1 = obj0;
    }
    if (info) {
        info->misfit_before = phi0;
        info->misfit_after = phi1;
        info->objective_before = obj0;
        info->objective_after = obj1;
        info->step = step;
        info->cg_iters = cg_done;
        info->iters_forward = it_fwd;
        info->iters_adjoint = it_adj;
        info->iters_sensitivity = it_sens;
        info->iters_line_search = it_ls;
    }
    return HELM_OK;
}

}  // extern "C"
