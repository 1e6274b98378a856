// Light-weight retraining of the encoder-solver network inside the library
// (Sec. 4.2, Alg. 2), one unit per call of cnn_retrain_step:
//
//   * the first call builds the initial dataset of Eq. 4.3 for the context's
//     medium: x ~ CN(0, 1), b = H x, x~ after k V-cycle-preconditioned FGMRES
//     steps (k uniform on 1..max_gmres_steps), pair (r, e) = (b - H x~, x - x~);
//   * every call takes the next batch of the current epoch (a fresh permutation of
//     the dataset per epoch) through one Adam step on the loss of Eq. 4.2;
//   * at the end of each of the first data_epochs epochs every pair is refined by
//     the network's estimate and one preconditioned GMRES step (Alg. 2), which
//     doubles the dataset (initial_size 2^data_epochs pairs at the end).
//
// Random draws.  They cannot be passed in per call, so they come from one
// counter-based generator written from its published definition: the output
// function of splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014) applied to key + n * 0x9E3779B97F4A7C15, with
// the keys K_s = mix(seed + s * 0x9E3779B97F4A7C15) of the streams s = 1 (the
// draws x), s = 2 (the GMRES step counts) and s = 16 + epoch (the permutation of
// that epoch).  A uniform u = ((z >> 11) + 1/2) 2^-53 is in (0, 1).
//   x of pair i, node p (q = i N + p): u1, u2 from counters 2q + 1, 2q + 2;
//       x = sqrt(-ln u1) (cos 2 pi u2 + i sin 2 pi u2)   (Box-Muller; Re, Im ~ N(0, 1/2))
//   step count of pair i: 1 + floor(u k_max) with u from counter i + 1
//   permutation of epoch e: Fisher-Yates from the last position down, position j
//       swapped with floor(u (j + 1)), u from counters 1, 2, ...
// Pair i has the frequency index i mod nfreq of the context.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <string>
#include <vector>

#include "cnn_internal.cuh"

namespace helm {

constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double sm_uniform(uint64_t key, uint64_t n) {
    return ((double)(sm_mix(key + n * SM_GAMMA) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
inline uint64_t sm_key(uint64_t seed, uint64_t stream) { return sm_mix(seed + stream * SM_GAMMA); }

namespace {

// x[j] for the pairs first .. first + nb - 1 (j over nb N nodes)
__global__ void draw_cn01_kernel(float2* __restrict__ x, long long n, long long q0, uint64_t key) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const uint64_t q = (uint64_t)(q0 + j);
        const double u1 = sm_uniform(key, 2 * q + 1), u2 = sm_uniform(key, 2 * q + 2);
        const double rho = sqrt(-log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        x[j] = make_float2((float)(rho * cs), (float)(rho * sn));
    }
}

}  // namespace

struct RetrainState {
    cnn_retrain_opts opt{};
    int cap = 0;                 // pairs the dataset holds (initial_size 2^data_epochs)
    int size = 0;                // pairs generated so far (0: the next step builds the initial set)
    int epoch = 0;               // epochs completed
    int pos = 0;                 // pairs of the current epoch already trained on
    long long steps = 0;         // Adam steps taken
    std::vector<int> perm;       // order of the current epoch
    std::vector<int> freq;       // frequency index per pair
    float2* R = nullptr;         // [cap][N]
    float2* E = nullptr;         // [cap][N]
    float2* rb = nullptr;        // batch [bcap][N]
    float2* eb = nullptr;
    int bcap = 0;
    double last_loss = 0.0;
    std::vector<void*> owned;
    ~RetrainState() {
        for (void* p : owned) cudaFree(p);
    }
};

void cnn_retrain_free(helm_ctx* c) {
    delete c->retrain;
    c->retrain = nullptr;
}

namespace {

int ralloc(RetrainState* s, float2** p, size_t n) {
    if (cudaMalloc(p, n * sizeof(float2)) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        set_error("cnn_retrain: out of device memory for the dataset");
        return HELM_ENOMEM;
    }
    s->owned.push_back(*p);
    return HELM_OK;
}

void permute(RetrainState* s) {
    const int n = s->size;
    s->perm.resize(n);
    for (int i = 0; i < n; ++i) s->perm[i] = i;
    const uint64_t key = sm_key(s->opt.seed, 16 + (uint64_t)s->epoch);
    uint64_t ctr = 1;
    for (int j = n - 1; j >= 1; --j) {
        int k = (int)(sm_uniform(key, ctr++) * (double)(j + 1));
        if (k > j) k = j;
        std::swap(s->perm[j], s->perm[k]);
    }
}

// The initial dataset of Eq. 4.3, in chunks of the context's max_rhs.
int build_initial(helm_ctx* c, RetrainState* s) {
    const size_t N = npts(c);
    const int n0 = s->opt.initial_size;
    const int chunk = c->cap;
    float2* x = nullptr;   // the draws of one chunk
    if (cudaMalloc(&x, (size_t)chunk * N * sizeof(float2)) != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("cnn_retrain: out of device memory for the draws");
        return HELM_ENOMEM;
    }
    const uint64_t kx = sm_key(s->opt.seed, 1), ki = sm_key(s->opt.seed, 2);
    int st = HELM_OK;
    for (int i0 = 0; i0 < n0 && !st; i0 += chunk) {
        const int nb = std::min(chunk, n0 - i0);
        std::vector<int> iters(nb), fi(nb);
        for (int i = 0; i < nb; ++i) {
            int k = 1 + (int)(sm_uniform(ki, (uint64_t)(i0 + i) + 1) * (double)s->opt.max_gmres_steps);
            iters[i] = std::min(k, s->opt.max_gmres_steps);
            fi[i] = s->freq[i0 + i];
        }
        { draw_cn01_kernel<<<1184, 256, 0, c->stream>>>(x, (long long)nb * (long long)N, (long long)i0 * (long long)N, kx); count_launch(); }
        if (cudaGetLastError() != cudaSuccess) {
            set_error("cnn_retrain: draw kernel launch failed");
            st = HELM_ECUDA;
            break;
        }
        st = cnn_make_samples(c, (const helm_c64*)x, fi.data(), iters.data(), nb, (helm_c64*)(s->R + (size_t)i0 * N),
                              (helm_c64*)(s->E + (size_t)i0 * N));
    }
    cudaFree(x);
    if (st) return st;
    s->size = n0;
    return HELM_OK;
}

// Alg. 2 data step: one refined pair per existing pair, appended after them.
int refine_all(helm_ctx* c, RetrainState* s) {
    const size_t N = npts(c);
    const int n = s->size, chunk = c->cap;
    for (int i0 = 0; i0 < n; i0 += chunk) {
        const int nb = std::min(chunk, n - i0);
        std::vector<int> fi(s->freq.begin() + i0, s->freq.begin() + i0 + nb);
        HELM_TRY(cnn_refine_samples(c, (const helm_c64*)(s->R + (size_t)i0 * N), (const helm_c64*)(s->E + (size_t)i0 * N),
                                    fi.data(), nb, s->opt.literal, (helm_c64*)(s->R + (size_t)(n + i0) * N),
                                    (helm_c64*)(s->E + (size_t)(n + i0) * N)));
    }
    s->size = 2 * n;
    return HELM_OK;
}

int begin(helm_ctx* c, const cnn_retrain_opts* o) {
    cnn_retrain_opts opt;
    cnn_retrain_default_opts(&opt);
    if (o) opt = *o;
    if (opt.initial_size < 1 || opt.data_epochs < 0 || opt.data_epochs > 10 || opt.epochs < 1 ||
        opt.max_gmres_steps < 1 || opt.max_gmres_steps > c->opt.restart || (opt.literal != 0 && opt.literal != 1)) {
        set_error("cnn_retrain_begin: need initial_size >= 1, data_epochs in [0, 10], epochs >= 1, "
                  "max_gmres_steps in [1, restart], literal 0 or 1");
        return HELM_EINVAL;
    }
    const long long cap = (long long)opt.initial_size << opt.data_epochs;
    if (cap > (1ll << 24)) { set_error("cnn_retrain_begin: dataset too large"); return HELM_EINVAL; }
    cnn_retrain_free(c);
    RetrainState* s = new RetrainState();
    s->opt = opt;
    s->cap = (int)cap;
    s->freq.resize(s->cap);
    for (int i = 0; i < s->cap; ++i) s->freq[i] = i % c->nfreq;
    const size_t N = npts(c);
    int st = ralloc(s, &s->R, (size_t)s->cap * N);
    if (!st) st = ralloc(s, &s->E, (size_t)s->cap * N);
    if (st) { delete s; return st; }
    c->retrain = s;
    return HELM_OK;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

void cnn_retrain_default_opts(cnn_retrain_opts* o) {
    if (!o) return;
    o->initial_size = 128;
    o->data_epochs = 3;
    o->epochs = 30;
    o->max_gmres_steps = 10;
    o->literal = 0;
    o->seed = 3;
}

int cnn_retrain_begin(helm_ctx* c, const cnn_retrain_opts* opts) {
    set_error("");
    if (!c || !c->net) { set_error("cnn_retrain_begin: needs a context created with a network"); return HELM_EINVAL; }
    return begin(c, opts);
}

int cnn_retrain_step(cnn_model* net, helm_ctx* c, int batch, float lr, float* loss_out) {
    set_error("");
    if (!net || !c || c->net != net) {
        set_error("cnn_retrain_step: the context must have been created with this network");
        return HELM_EINVAL;
    }
    if (batch < 1 || batch > c->cap || !(lr >= 0.0f)) {
        set_error("cnn_retrain_step: batch must be in [1, max_rhs] and lr >= 0");
        return HELM_EINVAL;
    }
    if (!c->retrain) HELM_TRY(begin(c, nullptr));
    RetrainState* s = c->retrain;
    const size_t N = npts(c);
    if (s->bcap < batch) {
        HELM_TRY(ralloc(s, &s->rb, (size_t)batch * N));
        HELM_TRY(ralloc(s, &s->eb, (size_t)batch * N));
        s->bcap = batch;
    }
    if (s->size == 0) HELM_TRY(build_initial(c, s));
    if (s->pos == 0) permute(s);
    const int nb = std::min(batch, s->size - s->pos);
    std::vector<int> fi(nb);
    for (int i = 0; i < nb; ++i) {
        const int p = s->perm[s->pos + i];
        fi[i] = s->freq[p];
        HELM_CK(cudaMemcpyAsync(s->rb + (size_t)i * N, s->R + (size_t)p * N, N * sizeof(float2),
                                cudaMemcpyDeviceToDevice, c->stream));
        HELM_CK(cudaMemcpyAsync(s->eb + (size_t)i * N, s->E + (size_t)p * N, N * sizeof(float2),
                                cudaMemcpyDeviceToDevice, c->stream));
    }
    double loss = 0.0;
    HELM_TRY(cnn_train_step(net, c, (const helm_c64*)s->rb, (const helm_c64*)s->eb, fi.data(), nb, lr, &loss));
    s->last_loss = loss;
    if (loss_out) *loss_out = (float)loss;
    ++s->steps;
    s->pos += nb;
    if (s->pos >= s->size) {
        // end of an epoch: the data epochs double the dataset (Alg. 2)
        s->pos = 0;
        ++s->epoch;
        if (s->epoch <= s->opt.data_epochs && 2 * s->size <= s->cap) HELM_TRY(refine_all(c, s));
    }
    return HELM_OK;
}

int cnn_retrain_state(const helm_ctx* c, long long* out6) {
    set_error("");
    if (!c || !out6) { set_error("cnn_retrain_state: null argument"); return HELM_EINVAL; }
    const RetrainState* s = c->retrain;
    if (!s) {
        for (int i = 0; i < 6; ++i) out6[i] = 0;
        return HELM_OK;
    }
    out6[0] = s->epoch;
    out6[1] = s->pos;
    out6[2] = s->size;
    out6[3] = s->steps;
    out6[4] = s->epoch >= s->opt.epochs ? 1 : 0;
    out6[5] = s->cap;
    return HELM_OK;
}

int cnn_retrain_pairs(helm_ctx* c, int first, int n, helm_c64* r_out, helm_c64* e_out, int* freq_out) {
    set_error("");
    if (!c || !c->retrain || n < 0 || first < 0 || first + n > c->retrain->size || (n && (!r_out || !e_out))) {
        set_error("cnn_retrain_pairs: pairs outside the dataset built so far");
        return HELM_EINVAL;
    }
    const RetrainState* s = c->retrain;
    const size_t N = npts(c);
    if (n) {
        HELM_CK(cudaMemcpyAsync(r_out, s->R + (size_t)first * N, (size_t)n * N * sizeof(float2), cudaMemcpyDefault,
                                c->stream));
        HELM_CK(cudaMemcpyAsync(e_out, s->E + (size_t)first * N, (size_t)n * N * sizeof(float2), cudaMemcpyDefault,
                                c->stream));
    }
    if (freq_out)
        for (int i = 0; i < n; ++i) freq_out[i] = s->freq[first + i];
    HELM_CK(cudaStreamSynchronize(c->stream));
    return HELM_OK;
}

}  // extern "C"
