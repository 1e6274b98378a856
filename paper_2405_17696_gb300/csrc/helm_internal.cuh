// Internal declarations of libhelm: context layout, stencil functors, the
// per-RHS Krylov state and the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "helm.h"

namespace helm {

constexpr int KMAX = 16;          // largest restart / coarse-GMRES length supported
constexpr int TILE_X = 32;        // threads per block along x
constexpr int TILE_Y = 8;         // threads per block along z
constexpr int ROWS = 8;           // rows of z handled per thread in tiled kernels

void set_error(const std::string& msg);

#define HELM_CK(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::helm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return HELM_ECUDA;                                                     \
        }                                                                          \
    } while (0)

#define HELM_TRY(expr)               \
    do {                             \
        int s_ = (expr);             \
        if (s_ != HELM_OK) return s_; \
    } while (0)

// ----------------------------------------------------------------------------
// complex helpers (float2 / double2 as complex numbers)
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// a / b for complex b != 0
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
    float d = 1.0f / (b.x * b.x + b.y * b.y);
    return make_float2((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}
__host__ __device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// ----------------------------------------------------------------------------
// Stencil functors.  apply() returns (A u) at one node with zero ghost values;
// diag() the diagonal entry; entry(k) the 3x3 stencil entry k = (dz+1)*3+(dx+1).
// ----------------------------------------------------------------------------

// Fine level: -Lap_h - w^2 m (1 - i sigma), sigma = gamma (H) or beta + incg*gamma (P).
struct OpFine5 {
    const float2* mg;        // [nz][nx] {kappa, gamma}; m = kappa^2
    const float* omega;      // [nfreq] w (rad/s)
    const int* rhs_freq;     // [cap] frequency index per RHS slot
    int nx, nz;
    float ax, az;            // 1/hx^2, 1/hz^2
    float beta;
    int sl;                  // 0: Helmholtz H, 1: shifted Laplacian P
    int incg;                // P keeps gamma in its shift

    __device__ __forceinline__ float2 coef(int b, int idx) const {
        float2 p = __ldg(mg + idx);
        float w = __ldg(omega + __ldg(rhs_freq + b));
        float s = (w * w) * (p.x * p.x);
        float sig = sl ? (beta + (incg ? p.y : 0.0f)) : p.y;
        return make_float2(s, -s * sig);          // s (1 - i sig)
    }
    __device__ __forceinline__ float2 diag(int b, int idx) const {
        float2 c = coef(b, idx);
        return make_float2(2.0f * (ax + az) - c.x, -c.y);
    }
    __device__ __forceinline__ float2 apply(const float2* __restrict__ u, int b, int ix, int iz) const {
        int idx = iz * nx + ix;
        float2 uc = u[idx];
        float2 z0 = make_float2(0.f, 0.f);
        float2 uw = ix > 0 ? u[idx - 1] : z0;
        float2 ue = ix < nx - 1 ? u[idx + 1] : z0;
        float2 un = iz > 0 ? u[idx - nx] : z0;
        float2 us = iz < nz - 1 ? u[idx + nx] : z0;
        float2 c = coef(b, idx);
        float2 y;
        y.x = ax * (2.f * uc.x - uw.x - ue.x) + az * (2.f * uc.x - un.x - us.x) - (c.x * uc.x - c.y * uc.y);
        y.y = ax * (2.f * uc.y - uw.y - ue.y) + az * (2.f * uc.y - un.y - us.y) - (c.x * uc.y + c.y * uc.x);
        return y;
    }
    // (H u) at the node pair (ix, ix + 1), ix even and nx even: 16-byte loads
    __device__ __forceinline__ void apply2(const float2* __restrict__ u, int b, int ix, int iz, float2& y0,
                                           float2& y1) const {
        const int idx = iz * nx + ix;
        const float4 c = *reinterpret_cast<const float4*>(u + idx);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 n = iz > 0 ? *reinterpret_cast<const float4*>(u + idx - nx) : zero;
        const float4 s = iz < nz - 1 ? *reinterpret_cast<const float4*>(u + idx + nx) : zero;
        const float2 w0 = ix > 0 ? u[idx - 1] : make_float2(0.f, 0.f);
        const float2 e1 = ix + 2 < nx ? u[idx + 2] : make_float2(0.f, 0.f);
        const float4 mm = __ldg(reinterpret_cast<const float4*>(mg + idx));
        const float wf = __ldg(omega + __ldg(rhs_freq + b));
        const float w2 = wf * wf;
        const float s0 = w2 * (mm.x * mm.x), s1 = w2 * (mm.z * mm.z);
        const float g0 = sl ? (beta + (incg ? mm.y : 0.0f)) : mm.y;
        const float g1 = sl ? (beta + (incg ? mm.w : 0.0f)) : mm.w;
        const float2 k0 = make_float2(s0, -s0 * g0), k1 = make_float2(s1, -s1 * g1);
        // node 0: west w0, east = node 1
        y0.x = ax * (2.f * c.x - w0.x - c.z) + az * (2.f * c.x - n.x - s.x) - (k0.x * c.x - k0.y * c.y);
        y0.y = ax * (2.f * c.y - w0.y - c.w) + az * (2.f * c.y - n.y - s.y) - (k0.x * c.y + k0.y * c.x);
        // node 1: west = node 0, east e1
        y1.x = ax * (2.f * c.z - c.x - e1.x) + az * (2.f * c.z - n.z - s.z) - (k1.x * c.z - k1.y * c.w);
        y1.y = ax * (2.f * c.w - c.y - e1.y) + az * (2.f * c.w - n.w - s.w) - (k1.x * c.w + k1.y * c.z);
    }
    __device__ __forceinline__ double2 entry(int f, int iz, int ix, int k) const {
        // fine stencil entries in double for the Galerkin product (frequency f)
        int dz = k / 3 - 1, dx = k % 3 - 1;
        if (dz == 0 && dx == 0) {
            float2 p = mg[iz * nx + ix];
            double w = omega[f], k = p.x;
            double s = (w * w) * (k * k);
            double sig = sl ? ((double)beta + (incg ? (double)p.y : 0.0)) : (double)p.y;
            return make_double2(2.0 * ((double)ax + (double)az) - s, s * sig);
        }
        if (dz == 0) return make_double2(-(double)ax, 0.0);
        if (dx == 0) return make_double2(-(double)az, 0.0);
        return make_double2(0.0, 0.0);
    }
};

// Coarse levels: Galerkin 9-point stencils, coefficients [nfreq][9][nz][nx].
struct OpC9 {
    const float2* coef;
    const int* rhs_freq;
    int nx, nz;

    __device__ __forceinline__ const float2* base(int f) const {
        return coef + (size_t)f * 9 * (size_t)nx * nz;
    }
    __device__ __forceinline__ float2 diag(int b, int idx) const {
        return __ldg(base(__ldg(rhs_freq + b)) + 4 * (size_t)nx * nz + idx);
    }
    __device__ __forceinline__ float2 apply(const float2* __restrict__ u, int b, int ix, int iz) const {
        const float2* c = base(__ldg(rhs_freq + b));
        size_t plane = (size_t)nx * nz;
        int idx = iz * nx + ix;
        float2 y = make_float2(0.f, 0.f);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                int jz = iz + dz, jx = ix + dx;
                if (jz < 0 || jz >= nz || jx < 0 || jx >= nx) continue;
                float2 a = __ldg(c + (size_t)((dz + 1) * 3 + (dx + 1)) * plane + idx);
                float2 v = u[jz * nx + jx];
                y.x += a.x * v.x - a.y * v.y;
                y.y += a.x * v.y + a.y * v.x;
            }
        }
        return y;
    }
    __device__ __forceinline__ double2 entry(int f, int iz, int ix, int k) const {
        float2 a = coef[(size_t)f * 9 * (size_t)nx * nz + (size_t)k * nx * nz + iz * nx + ix];
        return make_double2(a.x, a.y);
    }
};

// ----------------------------------------------------------------------------
// Per-RHS state of one batched (F)GMRES instance.  All arrays are device
// arrays indexed by the RHS slot b in [0, cap).
// ----------------------------------------------------------------------------
struct KState {
    int k;                 // steps per cycle
    double2* H;            // [cap][k][k+1]: column j holds h_{0..j+1, j}
    double* s;             // [cap][k+1]: 1/||v~_i|| (stored basis vectors are only near unit norm)
    double* cs;            // [cap][k]   Givens cosines
    double2* sn;           // [cap][k]   Givens sines
    double2* g;            // [cap][k+1] rotated right-hand side beta e_1
    double2* y;            // [cap][k]   least-squares solution
    int* active;           // [cap] 1 while iterating in this cycle
    int* steps;            // [cap] steps taken in this cycle
    double* tol_abs;       // [cap] stop when |g_{j+1}| <= tol_abs
    double* inv_est;       // [cap] 1 / (estimate of ||w'||) applied when v~_{j+1} is written
    double2* partials;     // [cap][max_tiles][KMAX + 2]
    unsigned* counters;    // [cap] arrival counters of the last-block reductions
    int max_tiles;
};

// Per-RHS bookkeeping of the outer solve (device arrays [cap]).
struct OuterState {
    double* bnorm2;        // ||b||^2
    double* rnorm2;        // ||b - A x||^2 at the last restart
    int* iters;            // total FGMRES steps
    int* status;           // HELM_OK / HELM_ENOCONV / HELM_EBREAKDOWN / -1 (running)
    int* outer_active;     // 1 while not finished
    double* rprev;         // ||b - A x|| at the previous restart (0 before the first)
    int* guard;            // 1 once a restart cycle barely lowered the residual (network composition guarded)
    double2* partials;     // [cap][max_tiles][2]
    unsigned* counters;
    int max_tiles;
};

// Kernel classes for launch counting and optional per-class CUDA-event timing.
enum KernelId {
    K_APPLY = 0, K_RESIDUAL64, K_DOTS_FINE, K_DOTS_COARSE, K_UPDATE_FINE, K_UPDATE_COARSE, K_KINIT, K_LSQ,
    K_COMBINE, K_UPDATE_X, K_JACOBI_FINE, K_JACOBI_COARSE, K_RESTRICT_FINE, K_RESTRICT_COARSE, K_PROLONG,
    K_GALERKIN, K_COPY, K_RESTART, K_COARSE_GMRES, K_CONV, K_CNN_IO, K_WGRAD, K_MISC, K_COUNT
};
const char* kernel_name(int id);

// Algorithmic bytes a kernel moves for one right-hand side (base + per_step *
// steps); when profiling, the first block of every processed RHS adds them to
// a device counter of the kernel's class.
struct Tally {
    unsigned long long* ctr = nullptr;
    unsigned long long base = 0;
    unsigned long long per_step = 0;
};
// `first` marks the first block of the RHS being processed.
__device__ __forceinline__ void tally_once(const Tally& t, bool first, int steps = 0) {
    if (t.ctr && first && threadIdx.x == 0 && threadIdx.y == 0)
        atomicAdd(t.ctr, t.base + t.per_step * (unsigned long long)steps);
}

struct Profiler {
    bool on = false;
    unsigned long long* d_bytes = nullptr;   // [K_COUNT] device counters
    std::vector<cudaEvent_t> pool;       // reusable events
    std::vector<int> ids;                // kernel class of each recorded pair
    size_t used = 0;                     // events used in the current window
    double ms[K_COUNT] = {0};
    long long launches[K_COUNT] = {0};
    double host_bytes[K_COUNT] = {0};   // algorithmic bytes of launches whose size the host knows
    double flops[K_COUNT] = {0};        // algorithmic flops (tensor-core kernels)
};

struct Level {
    int nx, nz;
    float2* coef9 = nullptr;    // levels >= 1: [nfreq][9][nz][nx]
    float2* f = nullptr;        // right-hand side   [cap][nz][nx]
    float2* u = nullptr;        // solution          [cap][nz][nx]
    float2* t = nullptr;        // Jacobi partner    [cap][nz][nx]
};

struct RetrainState;   // cnn_retrain.cu: the dataset and schedule of cnn_retrain_step

}  // namespace helm

struct helm_ctx {
    int nx = 0, nz = 0, nfreq = 0;
    float hx = 0, hz = 0;
    helm_opts opt{};
    cudaStream_t stream = nullptr;
    // restart cycles of MG-preconditioned (or plain) FGMRES are captured once per solve
    // as a CUDA graph on capture_stream and replayed on stream (helm_set_graphs)
    int graphs = 1;
    cudaStream_t capture_stream = nullptr;
    std::vector<float> omega;       // host copy (rad/s)
    float2* mg = nullptr;           // [nz][nx] {kappa, gamma}
    float* omega_d = nullptr;       // [nfreq] angular frequencies
    int cap = 0;                    // RHS slots in the workspace
    int* rhs_freq = nullptr;        // [cap]
    int* ones = nullptr;            // [cap] all ones (mask for unmasked launches)
    std::vector<helm::Level> lev;   // multigrid levels (lev[0] is the fine grid)
    // fine-grid Krylov workspace
    float2* V = nullptr;            // [k+1][cap][N]
    float2* Z = nullptr;            // [k][cap][N]
    float2* W = nullptr;            // [cap][N]
    helm::KState fine{};
    helm::OuterState outer{};
    // coarsest-level GMRES workspace
    float2* Vc = nullptr;           // [kc+1][cap][Nc]
    float2* Wc = nullptr;           // [cap][Nc]
    helm::KState coarse{};
    // staging for host pointers
    void* stage = nullptr;
    size_t stage_bytes = 0;
    std::vector<void*> allocations;
    helm::Profiler prof;
    // encoder-solver network preconditioner (HELM_PC_CNN)
    cnn_model* net = nullptr;
    std::vector<void*> cnn_z;        // context features per level, [nfreq][nz_l][nx_l][c_l] (BF16)
    void* cnn_in = nullptr;          // solver input, BF16 [cap][nz][nx][16]
    float* cnn_out = nullptr;        // solver output, FP32 [cap][nz][nx][2]
    float2* cnn_e0 = nullptr;        // network error estimate, [cap][nz][nx]
    float2* cnn_rres = nullptr;      // residual left by the network, [cap][nz][nx]
    double* cnn_alpha = nullptr;     // [cap][3] sums of the scaled composition (<t, r>, <t, t>)
    float* cnn_rms = nullptr;        // [cap]
    // Active-RHS compaction of the network pass inside FGMRES: at each restart the
    // RHS still iterating are listed (cnn_idx, their context indices in cnn_zmapc)
    // and only those cnn_nact images go through the network (-1: off, all RHS).
    int* cnn_idx = nullptr;          // [cap] device
    int* cnn_zmapc = nullptr;        // [cap] device
    int* cnn_idx_host = nullptr;     // [cap] pinned
    int* cnn_act_host = nullptr;     // [cap] pinned copy of the outer active flags
    int cnn_nact = -1;
    std::vector<void*> cnn_arena;    // one activation buffer per convolution of the solver pass
    std::vector<size_t> cnn_arena_bytes;
    helm::RetrainState* retrain = nullptr;   // Alg. 2 dataset and schedule (cnn_retrain_step)
    bool cnn_stale = false;          // the weights changed since the context features were computed
};

namespace helm {

inline size_t npts(const helm_ctx* c) { return (size_t)c->nx * c->nz; }

// Counts one kernel launch of the library (helm_launch_count); every launch site
// calls it right after its launch.
void count_launch();

// Counts the launches of a kernel class per context; when profiling is on,
// brackets them with a pair of CUDA events on the context's stream.
struct LaunchScope {
    helm_ctx* c;
    int id;
    size_t slot;
    LaunchScope(const helm_ctx* ctx, int kid);
    ~LaunchScope();
};
void prof_flush(helm_ctx* c);       // accumulate recorded pairs (synchronises the stream)
// add algorithmic bytes / flops of one launch to its class (no-op unless profiling)
void prof_add(const helm_ctx* c, int id, double bytes, double flops);
inline Tally tally(const helm_ctx* c, int id, unsigned long long base, unsigned long long per_step = 0) {
    Tally t;
    t.ctr = c->prof.on && c->prof.d_bytes ? c->prof.d_bytes + id : nullptr;
    t.base = base;
    t.per_step = per_step;
    return t;
}

OpFine5 fine_op(const helm_ctx* c, int sl);
OpC9 coarse_op(const helm_ctx* c, int level);

// ---- launchers (all on ctx->stream; masks are [cap] device arrays) ----
int launch_apply_fine(const helm_ctx* c, const OpFine5& op, const float2* x, float2* y, int nb, const int* mask);
int launch_residual64(helm_ctx* c, const double2* x, const float2* b, float2* r, int nb, int conj_b,
                      int first);
int launch_conj64(helm_ctx* c, double2* x, int nb);
int launch_galerkin(helm_ctx* c, int level);

template <class Op>
int launch_jacobi(const helm_ctx* c, const Op& op, float2* u_out, const float2* u_in, const float2* f,
                  int nx, int nz, int nb, const int* mask);
template <class Op>
int launch_restrict_residual(const helm_ctx* c, const Op& op, float2* rc, const float2* u, const float2* f,
                             int nx, int nz, int nb, const int* mask);
int launch_prolong_add(const helm_ctx* c, float2* u, const float2* ec, int nx, int nz, int nb, const int* mask);
int launch_copy_masked(const helm_ctx* c, float2* dst, const float2* src, size_t n_per_rhs, int nb, const int* mask);

// Krylov pieces
int launch_kstate_init(const helm_ctx* c, KState& st, const float2* v0, int nx, int nz, int nb,
                       const int* mask);
template <class Op>
int launch_arnoldi_dots(const helm_ctx* c, const Op& op, KState& st, const float2* z, float2* w,
                        const float2* V, size_t vstride, int j, int nx, int nz, int nb);
int launch_arnoldi_update(const helm_ctx* c, KState& st, const float2* w, float2* V, size_t vstride, int j,
                          int nx, int nz, int nb);
int launch_arnoldi_update_ex(const helm_ctx* c, KState& st, const float2* w, float2* V, size_t vstride, int j,
                             int nx, int nz, int nb, const int* iters_base, int max_iter, int* status);
int launch_lsq(const helm_ctx* c, KState& st, int nb);
int launch_normalize_v0(const helm_ctx* c, KState& st, float2* v0, size_t n, int nb);
int launch_coarse_gmres(const helm_ctx* c, int level, float2* u_out, int nb, const int* mask);
int launch_combine(const helm_ctx* c, const KState& st, float2* out, const float2* Zb, size_t zstride,
                   size_t n, int nb, const int* mask);
int launch_update_x64(const helm_ctx* c, const KState& st, double2* x, const float2* Zb, size_t zstride,
                      size_t n, int nb);
int launch_restart_check(helm_ctx* c, int nb, double tol, int* n_active_host);

// V-cycle on P u = f from u0 (nullptr: zero) into u_out, for the RHS with mask != 0.
int vcycle_apply(helm_ctx* c, float2* u_out, const float2* u0, const float2* f, int nb, const int* mask);
// network preconditioner hooks (cnn.cu)
int cnn_ctx_setup(helm_ctx* c);      // allocate buffers and run the encoder for every frequency
void cnn_ctx_free(helm_ctx* c);
int cnn_ctx_precondition(helm_ctx* c, float2* z, const float2* v, int nb, const int* mask, int with_vcycle);
int cnn_ctx_compact(helm_ctx* c, int nb);   // list the RHS still running (flags in cnn_act_host)
void cnn_retrain_free(helm_ctx* c);         // cnn_retrain.cu
// Block-shape autotuning of the Jacobi sweeps (k_multigrid.cu): while on, the first launch
// on a grid times the candidate shapes and records the fastest (process-wide table).
void stencil_tuning(bool on);
int stencil_tuned_count();
void stencil_tune_reset();

}  // namespace helm
