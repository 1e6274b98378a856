// C ABI of libhelm: context set-up (medium, frequencies, Galerkin multigrid
// hierarchy, workspace), the batched FGMRES driver, the V-cycle driver and
// the operator application.  See include/helm.h for the contract.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <type_traits>

#include "helm_internal.cuh"

namespace helm {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // this thread's launches (graph capture accounting)

void set_error(const std::string& msg) { g_last_error = msg; }

const char* kernel_name(int id) {
    static const char* names[K_COUNT] = {
        "stencil_apply", "residual64", "arnoldi_dots_fine", "arnoldi_dots_coarse", "arnoldi_update_fine",
        "arnoldi_update_coarse", "krylov_init", "lsq", "combine", "update_x64", "jacobi_fine", "jacobi_coarse",
        "restrict_fine", "restrict_coarse", "prolong_add", "galerkin", "copy", "restart_check", "coarse_gmres",
        "conv3x3_tc", "cnn_io", "wgrad", "misc"};
    return (id >= 0 && id < K_COUNT) ? names[id] : "?";
}

void count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}

LaunchScope::LaunchScope(const helm_ctx* ctx, int kid) : c(const_cast<helm_ctx*>(ctx)), id(kid), slot(0) {
    if (!c) return;
    c->prof.launches[id] += 1;
    if (!c->prof.on) return;
    Profiler& p = c->prof;
    if (p.used + 2 > 1 << 16) prof_flush(c);
    while (p.pool.size() < p.used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { p.on = false; return; }
        p.pool.push_back(e);
    }
    slot = p.used;
    p.used += 2;
    p.ids.push_back(id);
    cudaEventRecord(p.pool[slot], c->stream);
}

LaunchScope::~LaunchScope() {
    if (c && c->prof.on && slot + 1 < c->prof.pool.size()) cudaEventRecord(c->prof.pool[slot + 1], c->stream);
}

void prof_add(const helm_ctx* c, int id, double bytes, double flops) {
    if (!c || !c->prof.on || id < 0 || id >= K_COUNT) return;
    helm_ctx* m = const_cast<helm_ctx*>(c);
    m->prof.host_bytes[id] += bytes;
    m->prof.flops[id] += flops;
}

void prof_flush(helm_ctx* c) {
    Profiler& p = c->prof;
    if (p.used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (size_t i = 0; i < p.ids.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.pool[2 * i], p.pool[2 * i + 1]) == cudaSuccess) p.ms[p.ids[i]] += ms;
    }
    (void)cudaGetLastError();
    p.ids.clear();
    p.used = 0;
}

int launch_outer_init(helm_ctx* c, int nb);
int launch_zero_x(helm_ctx* c, double2* x, int nb);
int launch_restart_check_dev(helm_ctx* c, int nb, double tol, int* n_active_dev);

OpFine5 fine_op(const helm_ctx* c, int sl) {
    OpFine5 op;
    op.mg = c->mg;
    op.omega = c->omega_d;
    op.rhs_freq = c->rhs_freq;
    op.nx = c->nx;
    op.nz = c->nz;
    op.ax = 1.0f / (c->hx * c->hx);
    op.az = 1.0f / (c->hz * c->hz);
    op.beta = c->opt.sl_beta;
    op.sl = sl;
    op.incg = c->opt.sl_include_gamma;
    return op;
}

OpC9 coarse_op(const helm_ctx* c, int level) {
    OpC9 op;
    op.coef = c->lev[level].coef9;
    op.rhs_freq = c->rhs_freq;
    op.nx = c->lev[level].nx;
    op.nz = c->lev[level].nz;
    return op;
}

namespace {

// {kappa, gamma} interleaved so that one 8-byte load serves a grid point;
// the frequencies are copied next to them.
__global__ void pack_medium_kernel(const float* __restrict__ kappa, const float* __restrict__ gamma,
                                   float2* __restrict__ mg, size_t n, const float* __restrict__ omega,
                                   float* __restrict__ omega_d, int nfreq) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < (size_t)nfreq) omega_d[i] = omega[i];
    for (; i < n; i += (size_t)gridDim.x * blockDim.x) mg[i] = make_float2(kappa[i], gamma[i]);
}

__global__ void fill_int_kernel(int* p, int v, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

template <class T>
int dalloc(helm_ctx* c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error(std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed: " +
                  cudaGetErrorString(e));
        return HELM_ENOMEM;
    }
    c->allocations.push_back((void*)*p);
    return HELM_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A device view of a caller array: the array itself when it is device
// memory, else a staging buffer of the context filled from the host.
struct Staged {
    void* dev = nullptr;
    bool owned = false;
};

int stage_in(helm_ctx* c, const void* p, size_t bytes, Staged* s, bool copy) {
    if (is_device_ptr(p)) {
        s->dev = const_cast<void*>(p);
        s->owned = false;
        return HELM_OK;
    }
    HELM_CK(cudaMalloc(&s->dev, bytes));
    s->owned = true;
    if (copy) HELM_CK(cudaMemcpyAsync(s->dev, p, bytes, cudaMemcpyHostToDevice, c->stream));
    return HELM_OK;
}

int stage_out(helm_ctx* c, void* host, Staged* s, size_t bytes) {
    if (!s->owned) return HELM_OK;
    HELM_CK(cudaMemcpyAsync(host, s->dev, bytes, cudaMemcpyDeviceToHost, c->stream));
    return HELM_OK;
}

void stage_free(helm_ctx* c, Staged* s) {
    if (s->owned && s->dev) {
        cudaStreamSynchronize(c->stream);
        cudaFree(s->dev);
    }
    s->dev = nullptr;
    s->owned = false;
}

int alloc_kstate(helm_ctx* c, KState& st, int k, int max_tiles) {
    st.k = k;
    st.max_tiles = max_tiles;
    size_t cap = c->cap;
    HELM_TRY(dalloc(c, &st.H, cap * k * (k + 1)));
    HELM_TRY(dalloc(c, &st.s, cap * (k + 1)));
    HELM_TRY(dalloc(c, &st.cs, cap * k));
    HELM_TRY(dalloc(c, &st.sn, cap * k));
    HELM_TRY(dalloc(c, &st.g, cap * (k + 1)));
    HELM_TRY(dalloc(c, &st.y, cap * k));
    HELM_TRY(dalloc(c, &st.active, cap));
    HELM_TRY(dalloc(c, &st.steps, cap));
    HELM_TRY(dalloc(c, &st.tol_abs, cap));
    HELM_TRY(dalloc(c, &st.inv_est, cap));
    HELM_TRY(dalloc(c, &st.partials, cap * (size_t)max_tiles * (KMAX + 2)));
    HELM_TRY(dalloc(c, &st.counters, cap));
    HELM_CK(cudaMemsetAsync(st.counters, 0, cap * sizeof(unsigned), c->stream));
    HELM_CK(cudaMemsetAsync(st.active, 0, cap * sizeof(int), c->stream));
    HELM_CK(cudaMemsetAsync(st.steps, 0, cap * sizeof(int), c->stream));
    HELM_CK(cudaMemsetAsync(st.tol_abs, 0, cap * sizeof(double), c->stream));
    return HELM_OK;
}

int tiles_of(int nx, int nz) {
    return ((nx + TILE_X - 1) / TILE_X) * ((nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS));
}

int upload_freq(helm_ctx* c, const int* freq_idx, int nb) {
    std::vector<int> f(nb, 0);
    if (freq_idx) {
        for (int i = 0; i < nb; ++i) {
            if (freq_idx[i] < 0 || freq_idx[i] >= c->nfreq) {
                set_error("freq_idx[" + std::to_string(i) + "] = " + std::to_string(freq_idx[i]) +
                          " outside [0, nfreq)");
                return HELM_EINVAL;
            }
            f[i] = freq_idx[i];
        }
    }
    HELM_CK(cudaMemcpyAsync(c->rhs_freq, f.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    // the host vector dies at return: make the copy complete first
    HELM_CK(cudaStreamSynchronize(c->stream));
    return HELM_OK;
}

// ---------------------------------------------------------------------------
// V-cycle (Sec. 3.4): u_out = V-cycle on level l for P_l u = f from u0.
// ---------------------------------------------------------------------------
int coarsest_solve(helm_ctx* c, int l, float2* u_out, const float2* f, int nb, const int* mask) {
    Level& L = c->lev[l];
    size_t Nc = (size_t)L.nx * L.nz;
    if (c->opt.coarse_kind == HELM_COARSE_GMRES) {
        // f is stored in Vc[0]; plain GMRES(k) from zero, one thread block per RHS
        if (f != c->Vc) HELM_TRY(launch_copy_masked(c, c->Vc, f, Nc, nb, mask));
        return launch_coarse_gmres(c, l, u_out, nb, mask);
    }
    // fixed number of damped-Jacobi sweeps from zero, last one into u_out
    int n = c->opt.coarse_iters;
    float2* bufs[2] = {u_out, L.t};
    const float2* cur = nullptr;
    OpC9 op = coarse_op(c, l);
    for (int i = 0; i < n; ++i) {
        float2* dst = bufs[((n - 1 - i) % 2 == 0) ? 0 : 1];
        HELM_TRY(launch_jacobi(c, op, dst, cur, f, L.nx, L.nz, nb, mask));
        cur = dst;
    }
    return HELM_OK;
}

template <class Op>
int smooth_and_recurse(helm_ctx* c, const Op& op, int l, float2* u_out, const float2* u0, const float2* f, int nb,
                       const int* mask);

int vcycle_level(helm_ctx* c, int l, float2* u_out, const float2* u0, const float2* f, int nb, const int* mask) {
    if (l == (int)c->lev.size() - 1) return coarsest_solve(c, l, u_out, f, nb, mask);
    if (l == 0) return smooth_and_recurse(c, fine_op(c, 1), l, u_out, u0, f, nb, mask);
    return smooth_and_recurse(c, coarse_op(c, l), l, u_out, u0, f, nb, mask);
}

template <class Op>
int smooth_and_recurse(helm_ctx* c, const Op& op, int l, float2* u_out, const float2* u0, const float2* f, int nb,
                       const int* mask) {
    Level& L = c->lev[l];
    Level& C = c->lev[l + 1];
    const int pre = c->opt.pre, post = c->opt.post, n = pre + post;
    float2* bufs[2] = {u_out, L.t};
    const float2* cur = u0;
    int done = 0;
    for (int i = 0; i < pre; ++i, ++done) {
        float2* dst = bufs[((n - 1 - done) % 2 == 0) ? 0 : 1];
        HELM_TRY(launch_jacobi(c, op, dst, cur, f, L.nx, L.nz, nb, mask));
        cur = dst;
    }
    HELM_TRY(launch_restrict_residual(c, op, C.f, cur, f, L.nx, L.nz, nb, mask));
    HELM_TRY(vcycle_level(c, l + 1, C.u, nullptr, C.f, nb, mask));
    HELM_TRY(launch_prolong_add(c, const_cast<float2*>(cur), C.u, L.nx, L.nz, nb, mask));
    for (int i = 0; i < post; ++i, ++done) {
        float2* dst = bufs[((n - 1 - done) % 2 == 0) ? 0 : 1];
        HELM_TRY(launch_jacobi(c, op, dst, cur, f, L.nx, L.nz, nb, mask));
        cur = dst;
    }
    return HELM_OK;
}

int precondition(helm_ctx* c, float2* z, const float2* v, int nb, const int* mask) {
    if (c->opt.precond == HELM_PC_MG) return vcycle_level(c, 0, z, nullptr, v, nb, mask);
    if (c->opt.precond == HELM_PC_CNN) return cnn_ctx_precondition(c, z, v, nb, mask, 1);
    set_error("preconditioner kind not available in this context");
    return HELM_EUNSUPPORTED;
}

// owns the instantiated restart-cycle graph of one solve
struct GraphGuard {
    cudaGraphExec_t exec = nullptr;
    ~GraphGuard() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// ---------------------------------------------------------------------------
// restarted FGMRES for one batch of nb <= cap right-hand sides (device data)
// ---------------------------------------------------------------------------
int fgmres_batch(helm_ctx* c, const float2* rhs, double2* x, int nb, double tol, int adjoint, helm_stats* stats,
                 int* n_active_dev, int* n_active_host, const int* steps_cap = nullptr) {
    const size_t N = npts(c);
    const size_t vs = (size_t)c->cap * N;
    const int k = c->fine.k;
    const bool pc = c->opt.precond != HELM_PC_NONE;
    // the network pass of each cycle takes only the RHS still running at its restart
    const bool compact = c->opt.precond == HELM_PC_CNN && c->cnn_act_host;
    c->cnn_nact = -1;
    HELM_TRY(launch_outer_init(c, nb));
    if (steps_cap) {
        // fixed number of steps per RHS (no convergence test): start the step
        // counter at max_iter - cap so that the cap ends the RHS
        std::vector<int> it0(nb);
        for (int i = 0; i < nb; ++i) it0[i] = c->opt.max_iter - steps_cap[i];
        HELM_CK(cudaMemcpyAsync(c->outer.iters, it0.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        HELM_CK(cudaStreamSynchronize(c->stream));
    }
    if (adjoint) HELM_TRY(launch_conj64(c, x, nb));
    HELM_TRY(launch_residual64(c, x, rhs, c->V, nb, adjoint, 1));
    HELM_CK(cudaMemsetAsync(n_active_dev, 0, sizeof(int), c->stream));
    HELM_TRY(launch_restart_check_dev(c, nb, tol, n_active_dev));
    HELM_TRY(launch_zero_x(c, x, nb));
    HELM_CK(cudaMemcpyAsync(n_active_host, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HELM_CK(cudaStreamSynchronize(c->stream));
    OpFine5 H = fine_op(c, 0);
    // One restart cycle: k Arnoldi steps, the update of x, the true residual and the
    // restart check, whose count lands in n_active_host once the stream is synchronised.
    auto cycle = [&]() -> int {
        HELM_TRY(launch_normalize_v0(c, c->fine, c->V, N, nb));
        for (int j = 0; j < k; ++j) {
            float2* vj = c->V + (size_t)j * vs;
            float2* zj = pc ? c->Z + (size_t)j * vs : vj;
            if (pc) HELM_TRY(precondition(c, zj, vj, nb, c->fine.active));
            HELM_TRY(launch_arnoldi_dots(c, H, c->fine, zj, c->W, c->V, vs, j, c->nx, c->nz, nb));
            HELM_TRY(launch_arnoldi_update_ex(c, c->fine, c->W, c->V, vs, j, c->nx, c->nz, nb, c->outer.iters,
                                              c->opt.max_iter, c->outer.status));
        }
        HELM_TRY(launch_lsq(c, c->fine, nb));
        HELM_TRY(launch_update_x64(c, c->fine, x, pc ? c->Z : c->V, vs, N, nb));
        HELM_TRY(launch_residual64(c, x, rhs, c->V, nb, adjoint, 0));
        HELM_CK(cudaMemsetAsync(n_active_dev, 0, sizeof(int), c->stream));
        HELM_TRY(launch_restart_check_dev(c, nb, tol, n_active_dev));
        HELM_CK(cudaMemcpyAsync(n_active_host, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        if (compact)
            HELM_CK(cudaMemcpyAsync(c->cnn_act_host, c->outer.outer_active, nb * sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream));
        return HELM_OK;
    };
    // MG or no preconditioner: the second cycle is captured as a CUDA graph (on a
    // private stream, so that the caller's stream may be the legacy default stream)
    // and every later cycle replays it; the network's cycles vary with the RHS still
    // running and the profiler brackets single launches, so those run eagerly.
    GraphGuard gg;
    bool use_graph = c->graphs && c->opt.precond != HELM_PC_CNN && !c->prof.on;
    long long g_delta = 0, k_delta[K_COUNT] = {};
    for (int ncycle = 0; *n_active_host > 0; ++ncycle) {
        if (use_graph && ncycle == 1 && !gg.exec) {
            if (!c->capture_stream &&
                cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
                (void)cudaGetLastError();
                c->capture_stream = nullptr;
            }
            const long long g0 = t_launches;   // this thread's count: other threads may launch meanwhile
            long long k0[K_COUNT];
            for (int i = 0; i < K_COUNT; ++i) k0[i] = c->prof.launches[i];
            bool ok = false;
            if (c->capture_stream) {
                // the capture stream starts after everything queued so far on the caller's stream
                cudaStream_t user = c->stream;
                ok = cudaStreamSynchronize(user) == cudaSuccess &&
                     cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    c->stream = c->capture_stream;
                    const int st = cycle();
                    c->stream = user;
                    cudaGraph_t graph = nullptr;
                    ok = cudaStreamEndCapture(c->capture_stream, &graph) == cudaSuccess && graph && st == HELM_OK;
                    if (ok) ok = cudaGraphInstantiate(&gg.exec, graph, 0) == cudaSuccess;
                    if (graph) cudaGraphDestroy(graph);
                }
            }
            // the captured launches did not run: count them per replay instead
            g_delta = t_launches - g0;
            g_launches.fetch_sub(g_delta);
            t_launches -= g_delta;
            for (int i = 0; i < K_COUNT; ++i) {
                k_delta[i] = c->prof.launches[i] - k0[i];
                c->prof.launches[i] = k0[i];
            }
            if (!ok) {
                (void)cudaGetLastError();
                if (gg.exec) cudaGraphExecDestroy(gg.exec);
                gg.exec = nullptr;
                use_graph = false;
                set_error("");
            }
        }
        if (gg.exec) {
            HELM_CK(cudaGraphLaunch(gg.exec, c->stream));
            g_launches.fetch_add(g_delta);
            t_launches += g_delta;
            for (int i = 0; i < K_COUNT; ++i) c->prof.launches[i] += k_delta[i];
        } else {
            HELM_TRY(cycle());
        }
        HELM_CK(cudaStreamSynchronize(c->stream));
        if (compact && *n_active_host > 0) HELM_TRY(cnn_ctx_compact(c, nb));
    }
    c->cnn_nact = -1;
    if (adjoint) HELM_TRY(launch_conj64(c, x, nb));
    return HELM_OK;
}

__global__ void widen_kernel(const float2* __restrict__ a, double2* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = make_double2(a[i].x, a[i].y);
}

// out = a - b (complex64 minus complex128, computed in FP64, stored complex64)
__global__ void diff_kernel(const float2* __restrict__ a, const double2* __restrict__ b, float2* __restrict__ out,
                            size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = b[i];
        out[i] = make_float2((float)((double)a[i].x - v.x), (float)((double)a[i].y - v.y));
    }
}

// d = a - b in FP64 (complex64 minus complex128): b <- d, out <- complex64(d)
__global__ void diff64_kernel(const float2* __restrict__ a, double2* __restrict__ b, float2* __restrict__ out,
                              size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = b[i];
        double2 d = make_double2((double)a[i].x - v.x, (double)a[i].y - v.y);
        b[i] = d;
        out[i] = make_float2((float)d.x, (float)d.y);
    }
}

__global__ void negate_kernel(const float2* a, float2* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(-a[i].x, -a[i].y);
}

// Fixed-step FGMRES(H, M = V-cycle, b, x0) for the data of Eq. 4.3 and Alg. 2:
// x (complex128, device) holds x0 on entry and the iterate after steps[i] steps.
int fixed_step_solve(helm_ctx* c, const float2* b, double2* x, int nb, const int* steps) {
    int* n_active_dev = nullptr;
    int* n_active_host = nullptr;
    HELM_CK(cudaMalloc(&n_active_dev, sizeof(int)));
    if (cudaMallocHost(&n_active_host, sizeof(int)) != cudaSuccess) { cudaFree(n_active_dev); return HELM_ENOMEM; }
    const int pc = c->opt.precond;
    c->opt.precond = HELM_PC_MG;      // the data of Eq. 4.3 comes from the plain V-cycle
    int s = fgmres_batch(c, b, x, nb, 1e-300, 0, nullptr, n_active_dev, n_active_host, steps);
    c->opt.precond = pc;
    cudaFree(n_active_dev);
    cudaFreeHost(n_active_host);
    return s;
}

}  // namespace

int vcycle_apply(helm_ctx* c, float2* u_out, const float2* u0, const float2* f, int nb, const int* mask) {
    return vcycle_level(c, 0, u_out, u0, f, nb, mask);
}

}  // namespace helm

using namespace helm;

extern "C" {

const char* helm_last_error(void) { return g_last_error.c_str(); }

void helm_default_opts(helm_opts* o) {
    if (!o) return;
    o->restart = 10;
    o->max_iter = 300;
    o->mg_levels = 3;
    o->pre = 2;
    o->post = 2;
    o->jacobi_w = 0.8f;
    o->sl_beta = 0.5f;
    o->sl_include_gamma = 1;
    o->coarse_kind = HELM_COARSE_GMRES;
    o->coarse_iters = 10;
    o->precond = HELM_PC_MG;
    o->max_rhs = 256;
    o->cnn_vcycle = 2;
    o->autotune = 0;
    o->stream = nullptr;
}

void helm_destroy(helm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    cnn_ctx_free(c);
    cnn_retrain_free(c);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (void* p : c->allocations) cudaFree(p);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    delete c;
}

int helm_setup(helm_ctx** out, const float* kappa, const float* gamma, int nx, int nz, float hx, float hz,
               const float* omegas, int nfreq, const cnn_model* net, const helm_opts* opts) {
    g_last_error.clear();
    if (!out || !kappa || !gamma || !omegas) { set_error("null pointer argument"); return HELM_EINVAL; }
    *out = nullptr;
    helm_opts o;
    helm_default_opts(&o);
    if (opts) o = *opts;
    if (nx < 2 || nz < 2 || nfreq < 1 || !(hx > 0) || !(hz > 0)) {
        set_error("invalid grid: need nx, nz >= 2, nfreq >= 1, hx, hz > 0");
        return HELM_EINVAL;
    }
    if (o.restart < 1 || o.restart > KMAX || o.coarse_iters < 1 || o.coarse_iters > KMAX) {
        set_error("restart and coarse_iters must be in [1, " + std::to_string(KMAX) + "]");
        return HELM_EINVAL;
    }
    if (o.mg_levels < 2 || o.pre < 1 || o.post < 1 || o.max_rhs < 1 || o.max_iter < 1) {
        set_error("need mg_levels >= 2, pre >= 1, post >= 1, max_rhs >= 1, max_iter >= 1");
        return HELM_EINVAL;
    }
    int div = 1 << (o.mg_levels - 1);
    if (nx % div || nz % div) {
        set_error("nx and nz must be divisible by 2^(mg_levels-1) = " + std::to_string(div));
        return HELM_EINVAL;
    }
    if (o.precond == HELM_PC_CNN && !net) { set_error("HELM_PC_CNN needs a network"); return HELM_EINVAL; }
    if (o.cnn_vcycle < 0 || o.cnn_vcycle > 3) { set_error("cnn_vcycle must be 0, 1, 2 or 3"); return HELM_EINVAL; }

    helm_ctx* c = new helm_ctx();
    c->nx = nx; c->nz = nz; c->nfreq = nfreq; c->hx = hx; c->hz = hz; c->opt = o;
    c->net = const_cast<cnn_model*>(net);
    c->stream = (cudaStream_t)o.stream;
    c->cap = o.max_rhs;
    const size_t N = (size_t)nx * nz;
    int st = HELM_OK;
    auto fail = [&](int s) { helm_destroy(c); return s; };

    if ((st = dalloc(c, &c->mg, N))) return fail(st);
    if ((st = dalloc(c, &c->omega_d, nfreq))) return fail(st);
    if ((st = dalloc(c, &c->rhs_freq, c->cap))) return fail(st);
    if ((st = dalloc(c, &c->ones, c->cap))) return fail(st);
    {
        Staged sk, sg, so;
        if ((st = stage_in(c, kappa, N * sizeof(float), &sk, true))) return fail(st);
        if ((st = stage_in(c, gamma, N * sizeof(float), &sg, true))) { stage_free(c, &sk); return fail(st); }
        if ((st = stage_in(c, omegas, nfreq * sizeof(float), &so, true))) { stage_free(c, &sk); stage_free(c, &sg); return fail(st); }
        LaunchScope scope(c, K_MISC);
        { pack_medium_kernel<<<1184, 256, 0, c->stream>>>((const float*)sk.dev, (const float*)sg.dev, c->mg, N,
                                                         (const float*)so.dev, c->omega_d, nfreq); count_launch(); }
        cudaError_t e = cudaGetLastError();
        std::vector<float> om(nfreq);
        cudaError_t e2 = cudaMemcpyAsync(om.data(), so.dev, nfreq * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        stage_free(c, &sk); stage_free(c, &sg); stage_free(c, &so);
        if (e != cudaSuccess || e2 != cudaSuccess) { set_error("medium upload failed"); return fail(HELM_ECUDA); }
        c->omega = om;
    }
    {
        LaunchScope scope(c, K_MISC);
        { fill_int_kernel<<<(c->cap + 127) / 128, 128, 0, c->stream>>>(c->ones, 1, c->cap); count_launch(); }
    }
    {
        LaunchScope scope(c, K_MISC);
        { fill_int_kernel<<<(c->cap + 127) / 128, 128, 0, c->stream>>>(c->rhs_freq, 0, c->cap); count_launch(); }
    }

    // multigrid levels
    c->lev.resize(o.mg_levels);
    for (int l = 0; l < o.mg_levels; ++l) {
        c->lev[l].nx = nx >> l;
        c->lev[l].nz = nz >> l;
    }
    const size_t cap = c->cap;
    const int L = o.mg_levels;
    for (int l = 0; l < L; ++l) {
        Level& V = c->lev[l];
        size_t n = (size_t)V.nx * V.nz;
        if (l >= 1 && (st = dalloc(c, &V.coef9, (size_t)nfreq * 9 * n))) return fail(st);
        if ((st = dalloc(c, &V.t, cap * n))) return fail(st);
        if (l >= 1) {
            if ((st = dalloc(c, &V.u, cap * n))) return fail(st);
            if (!(l == L - 1 && o.coarse_kind == HELM_COARSE_GMRES))
                if ((st = dalloc(c, &V.f, cap * n))) return fail(st);
        }
    }
    // fine Krylov workspace
    const int k = o.restart;
    if ((st = dalloc(c, &c->V, (size_t)(k + 1) * cap * N))) return fail(st);
    if (o.precond != HELM_PC_NONE && (st = dalloc(c, &c->Z, (size_t)k * cap * N))) return fail(st);
    if ((st = dalloc(c, &c->W, cap * N))) return fail(st);
    if ((st = alloc_kstate(c, c->fine, k, tiles_of(nx, nz)))) return fail(st);
    // outer state
    {
        OuterState& os = c->outer;
        os.max_tiles = tiles_of(nx, nz);
        if ((st = dalloc(c, &os.bnorm2, cap)) || (st = dalloc(c, &os.rnorm2, cap)) ||
            (st = dalloc(c, &os.iters, cap)) || (st = dalloc(c, &os.status, cap)) ||
            (st = dalloc(c, &os.outer_active, cap)) || (st = dalloc(c, &os.partials, cap * os.max_tiles)) ||
            (st = dalloc(c, &os.counters, cap)) || (st = dalloc(c, &os.rprev, cap)) ||
            (st = dalloc(c, &os.guard, cap)))
            return fail(st);
        if (cudaMemsetAsync(os.counters, 0, cap * sizeof(unsigned), c->stream) != cudaSuccess ||
            cudaMemsetAsync(os.guard, 0, cap * sizeof(int), c->stream) != cudaSuccess)
            return fail(HELM_ECUDA);
    }
    // coarsest GMRES workspace
    {
        Level& C = c->lev[L - 1];
        size_t Nc = (size_t)C.nx * C.nz;
        if (o.coarse_kind == HELM_COARSE_GMRES) {
            int kc = o.coarse_iters;
            if ((st = dalloc(c, &c->Vc, (size_t)(kc + 1) * cap * Nc))) return fail(st);
            if ((st = dalloc(c, &c->Wc, cap * Nc))) return fail(st);
            if ((st = alloc_kstate(c, c->coarse, kc, tiles_of(C.nx, C.nz)))) return fail(st);
            C.f = c->Vc;   // the restricted residual lands in the first coarse Krylov vector
        }
    }
    // Galerkin hierarchy for every frequency
    for (int l = 1; l < L; ++l)
        if ((st = launch_galerkin(c, l))) return fail(st);
    // network context features for every frequency (Eq. 3.13, once per medium)
    if (c->net && (st = cnn_ctx_setup(c))) return fail(st);
    // block shapes of the sweeps and tiling of every convolution shape, timed on this device
    if (o.autotune && (st = helm_autotune(c, c->cap, nullptr))) return fail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_error(std::string("setup failed: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(HELM_ECUDA);
    }
    *out = c;
    return HELM_OK;
}

int helm_set_medium(helm_ctx* c, const float* kappa, const float* gamma, const float* omegas, int nfreq) {
    g_last_error.clear();
    if (!c || !kappa || !gamma || !omegas) { set_error("helm_set_medium: null argument"); return HELM_EINVAL; }
    if (nfreq != c->nfreq) { set_error("helm_set_medium: nfreq differs from the context's"); return HELM_EINVAL; }
    const size_t N = npts(c);
    Staged sk, sg, so;
    int s = stage_in(c, kappa, N * sizeof(float), &sk, true);
    if (!s) s = stage_in(c, gamma, N * sizeof(float), &sg, true);
    if (!s) s = stage_in(c, omegas, nfreq * sizeof(float), &so, true);
    if (!s) {
        LaunchScope scope(c, K_MISC);
        { pack_medium_kernel<<<1184, 256, 0, c->stream>>>((const float*)sk.dev, (const float*)sg.dev, c->mg, N,
                                                         (const float*)so.dev, c->omega_d, nfreq); count_launch(); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; }
    }
    for (int l = 1; !s && l < (int)c->lev.size(); ++l) s = launch_galerkin(c, l);
    if (!s && c->net) s = cnn_ctx_setup(c);
    if (!s) c->cnn_stale = false;
    if (!s) {
        c->omega.resize(nfreq);
        cudaError_t e = cudaMemcpyAsync(c->omega.data(), so.dev, nfreq * sizeof(float), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    stage_free(c, &sk);
    stage_free(c, &sg);
    stage_free(c, &so);
    if (!s && e != cudaSuccess) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; }
    return s;
}

int helm_residual(helm_ctx* c, const helm_c64* rhs, const helm_c128* x, helm_c64* r, int nrhs,
                  const int* freq_idx, double* rel_res) {
    g_last_error.clear();
    if (!c || !rhs || !x || !r || nrhs < 0) { set_error("helm_residual: invalid argument"); return HELM_EINVAL; }
    const size_t N = npts(c);
    std::vector<double> rn2, bn2;
    for (int b0 = 0; b0 < nrhs; b0 += c->cap) {
        int nb = nrhs - b0 < c->cap ? nrhs - b0 : c->cap;
        HELM_TRY(upload_freq(c, freq_idx ? freq_idx + b0 : nullptr, nb));
        Staged sb, sx, sr;
        int s = stage_in(c, rhs + (size_t)b0 * N, nb * N * sizeof(float2), &sb, true);
        if (!s) s = stage_in(c, x + (size_t)b0 * N, nb * N * sizeof(double2), &sx, true);
        if (!s) s = stage_in(c, r + (size_t)b0 * N, nb * N * sizeof(float2), &sr, false);
        if (!s) s = launch_outer_init(c, nb);
        if (!s) s = launch_residual64(c, (const double2*)sx.dev, (const float2*)sb.dev, (float2*)sr.dev, nb, 0, 1);
        if (!s) s = stage_out(c, r + (size_t)b0 * N, &sr, nb * N * sizeof(float2));
        rn2.resize(nb);
        bn2.resize(nb);
        if (!s && rel_res) {
            cudaMemcpyAsync(rn2.data(), c->outer.rnorm2, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(bn2.data(), c->outer.bnorm2, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        }
        cudaError_t e = cudaStreamSynchronize(c->stream);
        stage_free(c, &sb);
        stage_free(c, &sx);
        stage_free(c, &sr);
        if (s) return s;
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return HELM_ECUDA; }
        if (rel_res)
            for (int i = 0; i < nb; ++i)
                rel_res[b0 + i] = bn2[i] > 0 ? std::sqrt(rn2[i] / bn2[i]) : std::sqrt(rn2[i]);
    }
    return HELM_OK;
}

int helm_apply(helm_ctx* c, const helm_c64* x, helm_c64* y, int nrhs, const int* freq_idx, int op) {
    g_last_error.clear();
    if (!c || !x || !y || nrhs < 0 || (op != HELM_OP_H && op != HELM_OP_SL)) {
        set_error("helm_apply: invalid argument");
        return HELM_EINVAL;
    }
    const size_t N = npts(c);
    for (int b0 = 0; b0 < nrhs; b0 += c->cap) {
        int nb = nrhs - b0 < c->cap ? nrhs - b0 : c->cap;
        Staged sx, sy;
        HELM_TRY(upload_freq(c, freq_idx ? freq_idx + b0 : nullptr, nb));
        HELM_TRY(stage_in(c, x + (size_t)b0 * N, nb * N * sizeof(float2), &sx, true));
        int s = stage_in(c, y + (size_t)b0 * N, nb * N * sizeof(float2), &sy, false);
        if (s) { stage_free(c, &sx); return s; }
        s = launch_apply_fine(c, fine_op(c, op == HELM_OP_SL), (const float2*)sx.dev, (float2*)sy.dev, nb, c->ones);
        if (!s) s = stage_out(c, y + (size_t)b0 * N, &sy, nb * N * sizeof(float2));
        cudaError_t e = cudaStreamSynchronize(c->stream);
        stage_free(c, &sx);
        stage_free(c, &sy);
        if (s) return s;
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return HELM_ECUDA; }
    }
    return HELM_OK;
}

int helm_vcycle(helm_ctx* c, const helm_c64* f, const helm_c64* u0, helm_c64* u, int nrhs, const int* freq_idx) {
    g_last_error.clear();
    if (!c || !f || !u || nrhs < 0) { set_error("helm_vcycle: invalid argument"); return HELM_EINVAL; }
    const size_t N = npts(c);
    for (int b0 = 0; b0 < nrhs; b0 += c->cap) {
        int nb = nrhs - b0 < c->cap ? nrhs - b0 : c->cap;
        HELM_TRY(upload_freq(c, freq_idx ? freq_idx + b0 : nullptr, nb));
        Staged sf, su0, su;
        HELM_TRY(stage_in(c, f + (size_t)b0 * N, nb * N * sizeof(float2), &sf, true));
        int s = HELM_OK;
        if (u0) {
            // always copy u0 so that it can never alias the output
            s = stage_in(c, u0 + (size_t)b0 * N, nb * N * sizeof(float2), &su0, true);
            if (!s && !su0.owned) {
                void* tmp = nullptr;
                if (cudaMalloc(&tmp, nb * N * sizeof(float2)) != cudaSuccess) s = HELM_ENOMEM;
                else {
                    cudaMemcpyAsync(tmp, su0.dev, nb * N * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
                    su0.dev = tmp;
                    su0.owned = true;
                }
            }
        }
        if (!s) s = stage_in(c, u + (size_t)b0 * N, nb * N * sizeof(float2), &su, false);
        if (!s) s = vcycle_level(c, 0, (float2*)su.dev, u0 ? (const float2*)su0.dev : nullptr,
                                 (const float2*)sf.dev, nb, c->ones);
        if (!s) s = stage_out(c, u + (size_t)b0 * N, &su, nb * N * sizeof(float2));
        cudaError_t e = cudaStreamSynchronize(c->stream);
        stage_free(c, &sf);
        stage_free(c, &su0);
        stage_free(c, &su);
        if (s) return s;
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return HELM_ECUDA; }
    }
    return HELM_OK;
}

int helm_solve(helm_ctx* c, const helm_c64* rhs, helm_c128* x, int nrhs, const int* freq_idx, double tol,
               int flags, helm_stats* stats) {
    const int adjoint = (flags & HELM_SOLVE_ADJOINT) ? 1 : 0;
    const bool zero_x0 = (flags & HELM_SOLVE_ZERO_X0) != 0;
    g_last_error.clear();
    if (!c || !rhs || !x || nrhs < 0 || !(tol > 0)) { set_error("helm_solve: invalid argument"); return HELM_EINVAL; }
    const size_t N = npts(c);
    int* n_active_dev = nullptr;
    int* n_active_host = nullptr;
    HELM_CK(cudaMalloc(&n_active_dev, sizeof(int)));
    if (cudaMallocHost(&n_active_host, sizeof(int)) != cudaSuccess) {
        cudaFree(n_active_dev);
        set_error("cudaMallocHost failed");
        return HELM_ENOMEM;
    }
    int result = HELM_OK;   // HELM_OK, or the soft status HELM_ENOCONV / HELM_EBREAKDOWN
    int hard = HELM_OK;     // an error that stops the call
    std::vector<int> iters, status;
    std::vector<double> rn2, bn2;
    for (int b0 = 0; b0 < nrhs && hard == HELM_OK; b0 += c->cap) {
        int nb = nrhs - b0 < c->cap ? nrhs - b0 : c->cap;
        Staged sb, sx;
        int s = upload_freq(c, freq_idx ? freq_idx + b0 : nullptr, nb);
        if (!s) s = stage_in(c, rhs + (size_t)b0 * N, nb * N * sizeof(float2), &sb, true);
        if (!s) s = stage_in(c, x + (size_t)b0 * N, nb * N * sizeof(double2), &sx, !zero_x0);
        if (!s && zero_x0) {
            cudaError_t ez = cudaMemsetAsync(sx.dev, 0, nb * N * sizeof(double2), c->stream);
            if (ez != cudaSuccess) { set_error(cudaGetErrorString(ez)); s = HELM_ECUDA; }
        }
        if (!s) s = fgmres_batch(c, (const float2*)sb.dev, (double2*)sx.dev, nb, tol, adjoint, stats, n_active_dev,
                                 n_active_host);
        if (!s) s = stage_out(c, x + (size_t)b0 * N, &sx, nb * N * sizeof(double2));
        iters.resize(nb); status.resize(nb); rn2.resize(nb); bn2.resize(nb);
        if (!s) {
            cudaMemcpyAsync(iters.data(), c->outer.iters, nb * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(status.data(), c->outer.status, nb * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(rn2.data(), c->outer.rnorm2, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(bn2.data(), c->outer.bnorm2, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        }
        cudaError_t e = cudaStreamSynchronize(c->stream);
        stage_free(c, &sb);
        stage_free(c, &sx);
        if (s) { hard = s; break; }
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); hard = HELM_ECUDA; break; }
        for (int i = 0; i < nb; ++i) {
            if (stats && stats->iters) stats->iters[b0 + i] = iters[i];
            if (stats && stats->status) stats->status[b0 + i] = status[i];
            if (stats && stats->rel_res)
                stats->rel_res[b0 + i] = bn2[i] > 0 ? std::sqrt(rn2[i] / bn2[i]) : std::sqrt(rn2[i]);
            if (status[i] == HELM_EBREAKDOWN) result = HELM_EBREAKDOWN;
            if (status[i] == HELM_ENOCONV && result == HELM_OK) result = HELM_ENOCONV;
        }
    }
    cudaFree(n_active_dev);
    cudaFreeHost(n_active_host);
    if (c->prof.on) prof_flush(c);
    if (hard != HELM_OK) return hard;
    if (result == HELM_ENOCONV) set_error("some right-hand sides did not reach tol within max_iter");
    if (result == HELM_EBREAKDOWN) set_error("breakdown (NaN/Inf) in some right-hand sides");
    return result;
}

int helm_set_graphs(helm_ctx* c, int on) {
    if (!c) { set_error("null context"); return HELM_EINVAL; }
    c->graphs = on != 0;
    return HELM_OK;
}

int helm_profile_enable(helm_ctx* c, int on) {
    if (!c) { set_error("null context"); return HELM_EINVAL; }
    prof_flush(c);
    for (int i = 0; i < K_COUNT; ++i) {
        c->prof.ms[i] = 0.0;
        c->prof.launches[i] = 0;
        c->prof.host_bytes[i] = 0.0;
        c->prof.flops[i] = 0.0;
    }
    if (on && !c->prof.d_bytes) HELM_TRY(dalloc(c, &c->prof.d_bytes, K_COUNT));
    if (c->prof.d_bytes)
        HELM_CK(cudaMemsetAsync(c->prof.d_bytes, 0, K_COUNT * sizeof(unsigned long long), c->stream));
    c->prof.on = on != 0;
    return HELM_OK;
}

int helm_profile_read(helm_ctx* c, int max, const char** names, double* ms, long long* launches,
                      double* bytes, int* count) {
    if (!c) { set_error("null context"); return HELM_EINVAL; }
    prof_flush(c);
    unsigned long long hb[K_COUNT] = {0};
    if (c->prof.d_bytes) {
        HELM_CK(cudaMemcpyAsync(hb, c->prof.d_bytes, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
        HELM_CK(cudaStreamSynchronize(c->stream));
    }
    int n = 0;
    for (int i = 0; i < K_COUNT && n < max; ++i, ++n) {
        if (names) names[n] = kernel_name(i);
        if (ms) ms[n] = c->prof.ms[i];
        if (launches) launches[n] = c->prof.launches[i];
        if (bytes) bytes[n] = (double)hb[i] + c->prof.host_bytes[i];
    }
    if (count) *count = n;
    return HELM_OK;
}

int helm_profile_flops(helm_ctx* c, int max, double* flops, int* count) {
    if (!c) { set_error("null context"); return HELM_EINVAL; }
    int n = 0;
    for (int i = 0; i < K_COUNT && n < max; ++i, ++n)
        if (flops) flops[n] = c->prof.flops[i];
    if (count) *count = n;
    return HELM_OK;
}

long long helm_launch_count(void) { return g_launches.load(); }

int helm_autotune(helm_ctx* c, int nrhs, int* n_shapes) {
    g_last_error.clear();
    if (!c || nrhs < 1 || nrhs > c->cap) { set_error("helm_autotune: need 1 <= nrhs <= max_rhs"); return HELM_EINVAL; }
    const size_t N = npts(c);
    float2 *f = nullptr, *u = nullptr;
    HELM_CK(cudaMalloc(&f, (size_t)nrhs * N * sizeof(float2)));
    if (cudaMalloc(&u, (size_t)nrhs * N * sizeof(float2)) != cudaSuccess) {
        cudaFree(f);
        set_error("helm_autotune: out of device memory");
        return HELM_ENOMEM;
    }
    int s = HELM_OK;
    // a V-cycle on a synthetic right-hand side (frequency 0) with the sweeps' shapes tuned
    if (cudaMemsetAsync(f, 0, (size_t)nrhs * N * sizeof(float2), c->stream) != cudaSuccess) s = HELM_ECUDA;
    if (!s) {
        LaunchScope scope(c, K_MISC);
        { fill_int_kernel<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(c->rhs_freq, 0, nrhs); count_launch(); }
        if (cudaGetLastError() != cudaSuccess) s = HELM_ECUDA;
    }
    if (!s) {
        stencil_tuning(true);
        s = vcycle_apply(c, u, nullptr, f, nrhs, c->ones);
        stencil_tuning(false);
    }
    if (!s && cudaStreamSynchronize(c->stream) != cudaSuccess) s = HELM_ECUDA;
    cudaFree(f);
    cudaFree(u);
    if (!s && c->net) s = cnn_autotune(c, nrhs, nullptr);
    if (n_shapes) *n_shapes = stencil_tuned_count();
    return s;
}

void helm_autotune_reset(void) { stencil_tune_reset(); }

int cnn_make_samples(helm_ctx* c, const helm_c64* x, const int* freq_idx, const int* iters, int nb, helm_c64* r_out,
                     helm_c64* e_out) {
    g_last_error.clear();
    if (!c || !x || !iters || !r_out || !e_out || nb < 1 || nb > c->cap) {
        set_error("cnn_make_samples: invalid argument (nb must be in [1, max_rhs])");
        return HELM_EINVAL;
    }
    for (int i = 0; i < nb; ++i)
        if (iters[i] < 1 || iters[i] > c->opt.restart) { set_error("cnn_make_samples: iters must be in [1, restart]"); return HELM_EINVAL; }
    const size_t N = npts(c);
    HELM_TRY(upload_freq(c, freq_idx, nb));
    float2 *dx = nullptr, *db = nullptr, *dr = nullptr, *de = nullptr;
    double2* xt = nullptr;
    int s = HELM_OK;
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(e)); s = HELM_ECUDA; } };
    ck(cudaMalloc(&dx, nb * N * sizeof(float2)));
    ck(cudaMalloc(&db, nb * N * sizeof(float2)));
    ck(cudaMalloc(&dr, nb * N * sizeof(float2)));
    ck(cudaMalloc(&de, nb * N * sizeof(float2)));
    ck(cudaMalloc(&xt, nb * N * sizeof(double2)));
    if (!s) ck(cudaMemcpyAsync(dx, x, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (!s) ck(cudaMemsetAsync(xt, 0, nb * N * sizeof(double2), c->stream));
    if (!s) s = launch_apply_fine(c, fine_op(c, 0), dx, db, nb, c->ones);          // b = H x
    if (!s) s = fixed_step_solve(c, db, xt, nb, iters);                            // x~ (Eq. 4.3)
    // r = b - H x~ = H e: formed as H e in FP64 from e = x - x~, so that the stored
    // pair satisfies H e = r up to its own complex64 rounding (b in complex64
    // carries a rounding of |H| |x| u, far above r once GMRES has converged)
    if (!s) {
        LaunchScope scope(c, K_MISC);
        { diff64_kernel<<<1184, 256, 0, c->stream>>>(dx, xt, de, nb * N); count_launch(); }            // e = x - x~
        ck(cudaGetLastError());
    }
    if (!s) ck(cudaMemsetAsync(db, 0, nb * N * sizeof(float2), c->stream));
    if (!s) s = launch_outer_init(c, nb);
    if (!s) s = launch_residual64(c, xt, db, dr, nb, 0, 1);                        // -H e
    if (!s) {
        LaunchScope scope(c, K_MISC);
        { negate_kernel<<<1184, 256, 0, c->stream>>>(dr, dr, nb * N); count_launch(); }                // r = H e
        ck(cudaGetLastError());
    }
    if (!s) ck(cudaMemcpyAsync(r_out, dr, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (!s) ck(cudaMemcpyAsync(e_out, de, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    cudaFree(dx); cudaFree(db); cudaFree(dr); cudaFree(de); cudaFree(xt);
    return s;
}

int cnn_refine_samples(helm_ctx* c, const helm_c64* r, const helm_c64* e, const int* freq_idx, int nb, int literal,
                       helm_c64* r_out, helm_c64* e_out) {
    g_last_error.clear();
    if (!c || !c->net || !r || !e || !r_out || !e_out || nb < 1 || nb > c->cap) {
        set_error("cnn_refine_samples: invalid argument or no network in the context");
        return HELM_EINVAL;
    }
    const size_t N = npts(c);
    HELM_TRY(upload_freq(c, freq_idx, nb));
    float2 *dr = nullptr, *de = nullptr, *en = nullptr, *ro = nullptr, *eo = nullptr;
    double2* xt = nullptr;
    int s = HELM_OK;
    auto ck = [&](cudaError_t er) { if (er != cudaSuccess && s == HELM_OK) { set_error(cudaGetErrorString(er)); s = HELM_ECUDA; } };
    ck(cudaMalloc(&dr, nb * N * sizeof(float2)));
    ck(cudaMalloc(&de, nb * N * sizeof(float2)));
    ck(cudaMalloc(&en, nb * N * sizeof(float2)));
    ck(cudaMalloc(&ro, nb * N * sizeof(float2)));
    ck(cudaMalloc(&eo, nb * N * sizeof(float2)));
    ck(cudaMalloc(&xt, nb * N * sizeof(double2)));
    if (!s) ck(cudaMemcpyAsync(dr, r, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (!s) ck(cudaMemcpyAsync(de, e, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (!s) s = cnn_ctx_precondition(c, en, dr, nb, c->ones, 0);                   // e_net = network(r)
    if (!s) {
        LaunchScope scope(c, K_MISC);
        { widen_kernel<<<1184, 256, 0, c->stream>>>(en, xt, nb * N); count_launch(); }
        ck(cudaGetLastError());
    }
    std::vector<int> one(nb, 1);
    if (!s) s = fixed_step_solve(c, dr, xt, nb, one.data());                       // e~ = GMRES(H, V, r, e_net, 1)
    if (!s && literal) {
        // the pair (H e~, e~) of Alg. 2 as printed
        ck(cudaMemsetAsync(en, 0, nb * N * sizeof(float2), c->stream));
        if (!s) s = launch_outer_init(c, nb);
        if (!s) s = launch_residual64(c, xt, en, eo, nb, 0, 1);                    // eo = 0 - H e~
        if (!s) {
            LaunchScope scope(c, K_MISC);
            { negate_kernel<<<1184, 256, 0, c->stream>>>(eo, ro, nb * N); count_launch(); }           // r' = H e~
            ck(cudaGetLastError());
        }
        if (!s) {
            LaunchScope scope(c, K_MISC);
            { diff_kernel<<<1184, 256, 0, c->stream>>>(en, xt, eo, nb * N); count_launch(); }          // 0 - e~
            ck(cudaGetLastError());
        }
        if (!s) {
            LaunchScope scope(c, K_MISC);
            { negate_kernel<<<1184, 256, 0, c->stream>>>(eo, eo, nb * N); count_launch(); }           // e' = e~
            ck(cudaGetLastError());
        }
    }
    if (!s && !literal) {
        if (!s) s = launch_outer_init(c, nb);
        if (!s) s = launch_residual64(c, xt, dr, ro, nb, 0, 1);                    // r' = r - H e~
        if (!s) {
            LaunchScope scope(c, K_MISC);
            { diff_kernel<<<1184, 256, 0, c->stream>>>(de, xt, eo, nb * N); count_launch(); }          // e' = e - e~
            ck(cudaGetLastError());
        }
    }
    if (!s) ck(cudaMemcpyAsync(r_out, ro, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (!s) ck(cudaMemcpyAsync(e_out, eo, nb * N * sizeof(float2), cudaMemcpyDefault, c->stream));
    ck(cudaStreamSynchronize(c->stream));
    cudaFree(dr); cudaFree(de); cudaFree(en); cudaFree(ro); cudaFree(eo); cudaFree(xt);
    return s;
}

}  // extern "C"
