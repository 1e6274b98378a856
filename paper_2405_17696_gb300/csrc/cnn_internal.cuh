// Network internals shared by the forward (cnn.cu) and training
// (cnn_train.cu) translation units: layer table, model state, and the runner
// that issues the convolutions of one pass (optionally recording a tape of
// them for the backward pass).
#pragma once

#include <cuda_bf16.h>

#include <string>
#include <vector>

#include "conv.cuh"
#include "helm_internal.cuh"

namespace helm {

struct Layer {
    std::string name;
    int cin, cout, mode;     // logical channels; mode 0 same, 1 down, 2 up
    int cin_pad, npad;       // padded to multiples of 16 (npad: 16, 32, 64 or 128)
    int relu;
    long long off;           // offset of this layer's weights in the flat vector
    __nv_bfloat16* w = nullptr;   // [npad][9][cin_pad]
    __nv_bfloat16* wup = nullptr; // mode 2: phase-merged [npad][16][cin_pad] (up_merged_index)
    float* b = nullptr;           // [npad]
};

}  // namespace helm

struct cnn_model {
    int levels = 0;
    // training state (FP32, flat like the parameters): gradient and Adam moments
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    int loss_kind = 0;            // 0: Eq. 4.2 (mean squared error); 1: each sample's error relative to ||e||^2
    std::vector<int> widths;
    std::vector<helm::Layer> layers;
    long long nparams = 0;
    float* master = nullptr;      // flat FP32 parameters (device)
    int* err = nullptr;           // device error flag of the conv kernels
    std::vector<void*> allocations;
    float* wg_scratch = nullptr;  // weight-gradient partial sums (grown on demand, freed with the model)
    size_t wg_scratch_n = 0;
    // Buffers of a training step, reused by call order from step to step (the k-th buffer
    // of a pass serves the k-th request of every later pass; grown when a request is larger):
    // the forward pass's activations, the backward pass's scratch, the loss inputs/outputs.
    std::vector<void*> fw_arena, bw_arena, io_arena;
    std::vector<size_t> fw_arena_bytes, bw_arena_bytes, io_arena_bytes;
};

namespace helm {

// The k-th buffer of an arena, at least `bytes` long (reallocated when smaller); nullptr
// when the device is out of memory.
inline void* arena_buffer(std::vector<void*>& bufs, std::vector<size_t>& sizes, size_t k, size_t bytes) {
    if (k >= bufs.size()) {
        bufs.resize(k + 1, nullptr);
        sizes.resize(k + 1, 0);
    }
    if (sizes[k] < bytes) {
        if (bufs[k]) cudaFree(bufs[k]);
        bufs[k] = nullptr;
        sizes[k] = 0;
        if (cudaMalloc(&bufs[k], bytes ? bytes : 16) != cudaSuccess) {
            (void)cudaGetLastError();
            bufs[k] = nullptr;
            return nullptr;
        }
        sizes[k] = bytes;
    }
    return bufs[k];
}

int pad16(int c);
int npad_of(int c);

// One convolution of a pass, as recorded for the backward pass.
struct TapeOp {
    int layer;                       // index into cnn_model::layers
    const __nv_bfloat16* x0;
    int c0;
    const __nv_bfloat16* x1;
    int c1;
    int x1_bcast;                    // 0 batch-matched, 1 shared image 0, 2 mapped by zmap
    const int* zmap;
    int nb, hin, win, hout, wout;
    const __nv_bfloat16* res;        // residual input (ResNet second conv) or nullptr
    const void* y;                   // output (BF16, or FP32 for the output layer)
};

struct NetBuffers {
    // encoder outputs z_l: [nenc][ny_l][nx_l][c_l]
    std::vector<__nv_bfloat16*> z;
    int nenc = 0;
};

class Runner {
   public:
    Runner(cnn_model* m, const helm_ctx* ctx, cudaStream_t st, std::vector<void*>* arena = nullptr,
           std::vector<size_t>* arena_bytes = nullptr)
        : m_(m), ctx_(ctx), st_(st), arena_(arena), arena_bytes_(arena_bytes) {}
    ~Runner() {
        for (void* p : tmp_) cudaFree(p);
    }
    __nv_bfloat16* alloc(size_t n) {
        if (arena_) {
            // the k-th buffer of a pass is reused by the k-th call of every later pass
            const size_t k = next_++;
            const size_t bytes = n * sizeof(__nv_bfloat16);
            if (k >= arena_->size()) {
                arena_->push_back(nullptr);
                arena_bytes_->push_back(0);
            }
            if ((*arena_bytes_)[k] < bytes) {
                if ((*arena_)[k]) cudaFree((*arena_)[k]);
                (*arena_)[k] = nullptr;
                (*arena_bytes_)[k] = 0;
                if (cudaMalloc(&(*arena_)[k], bytes) != cudaSuccess) {
                    (void)cudaGetLastError();
                    (*arena_)[k] = nullptr;
                    ok_ = false;
                    return nullptr;
                }
                (*arena_bytes_)[k] = bytes;
            }
            return (__nv_bfloat16*)(*arena_)[k];
        }
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(__nv_bfloat16)) != cudaSuccess) {
            (void)cudaGetLastError();
            ok_ = false;
            return nullptr;
        }
        tmp_.push_back(p);
        return (__nv_bfloat16*)p;
    }
    bool ok() const { return ok_; }
    const Layer& L(const std::string& name) const {
        for (const Layer& l : m_->layers)
            if (l.name == name) return l;
        return m_->layers[0];
    }
    // y = act(conv(cat(x0, x1)) [+ res]) ; returns y (allocated here) and its spatial size
    __nv_bfloat16* conv(const std::string& name, const __nv_bfloat16* x0, int c0, const __nv_bfloat16* x1, int c1,
                        int x1_bcast, int nb, int hin, int win, const __nv_bfloat16* res, int* hout, int* wout,
                        void* y_fp32 = nullptr) {
        if (!ok_) return nullptr;
        const Layer& l = L(name);
        int ho = hin, wo = win;
        if (l.mode == 1) { ho = hin / 2; wo = win / 2; }
        if (l.mode == 2) { ho = hin * 2; wo = win * 2; }
        __nv_bfloat16* y = nullptr;
        if (!y_fp32) {
            y = alloc((size_t)nb * ho * wo * l.npad);
            if (!y) return nullptr;
        }
        ConvArgs a;
        a.x0 = x0; a.c0 = c0; a.x1 = x1; a.c1 = c1; a.x1_bcast = x1_bcast; a.x1_map = x1_bcast == 2 ? zmap_ : nullptr;
        a.nb1 = x1_bcast == 1 ? 1 : (x1_bcast == 2 ? nctx_ : nb);
        a.nb = nb; a.hin = hin; a.win = win; a.hout = ho; a.wout = wo; a.mode = l.mode;
        a.w = l.w; a.wup = l.wup; a.bias = l.b; a.res = res; a.y = y_fp32 ? y_fp32 : (void*)y;
        a.npad = l.npad; a.cstore = l.cout; a.relu = l.relu; a.out_fp32 = y_fp32 ? 1 : 0; a.accum = 0;
        a.err = m_->err;
        int s;
        {
            LaunchScope scope(ctx_, K_CONV);
            s = launch_conv3x3(a, st_);
        }
        if (ctx_ && ctx_->prof.on) {
            // algorithmic traffic: every input, residual and output element once, the weights once
            const double pin = (double)hin * win, pout = (double)nb * ho * wo;
            const int n1 = x1 ? (x1_bcast == 1 ? 1 : (x1_bcast == 2 ? nctx_ : nb)) : 0;
            double bytes = 2.0 * pin * ((double)nb * c0 + (double)n1 * c1) + 2.0 * 9.0 * l.npad * (c0 + c1);
            if (res) bytes += 2.0 * pout * l.npad;
            bytes += y_fp32 ? 4.0 * pout * l.cout : 2.0 * pout * l.npad;
            prof_add(ctx_, K_CONV, bytes, 2.0 * 9.0 * l.cin * l.cout * pout);
        }
        if (s != HELM_OK) { ok_ = false; return nullptr; }
        if (tape_) {
            TapeOp op;
            op.layer = (int)(&l - &m_->layers[0]);
            op.x0 = x0; op.c0 = c0; op.x1 = x1; op.c1 = c1; op.x1_bcast = x1_bcast;
            op.zmap = x1_bcast == 2 ? zmap_ : nullptr;
            op.nb = nb; op.hin = hin; op.win = win; op.hout = ho; op.wout = wo; op.res = res;
            op.y = y_fp32 ? (const void*)y_fp32 : (const void*)y;
            tape_->push_back(op);
        }
        if (hout) *hout = ho;
        if (wout) *wout = wo;
        return y;
    }
    __nv_bfloat16* res(const std::string& p, const __nv_bfloat16* x, int ch, int nb, int h, int w) {
        __nv_bfloat16* t = conv(p + ".a", x, ch, nullptr, 0, 0, nb, h, w, nullptr, nullptr, nullptr);
        return conv(p + ".b", t, ch, nullptr, 0, 0, nb, h, w, x, nullptr, nullptr);
    }

    // z_l for nenc encoder images (input BF16 [nenc][ny][nx][16]); the z buffers are
    // owned by the caller-provided vector of pointers (allocated here, not freed by ~Runner)
    bool encoder(const __nv_bfloat16* xin, int nenc, int ny, int nx, std::vector<__nv_bfloat16*>& z) {
        const int Lv = m_->levels;
        const std::vector<int>& c = m_->widths;
        std::vector<__nv_bfloat16*> e(Lv);
        std::vector<int> hy(Lv), wx(Lv);
        int h = ny, w = nx;
        __nv_bfloat16* t = conv("enc.in", xin, 16, nullptr, 0, 0, nenc, h, w, nullptr, nullptr, nullptr);
        t = res("enc.r0.0", t, c[0], nenc, h, w);
        t = res("enc.r0.1", t, c[0], nenc, h, w);
        e[0] = t; hy[0] = h; wx[0] = w;
        for (int l = 1; l < Lv; ++l) {
            t = conv("enc.down" + std::to_string(l), t, c[l - 1], nullptr, 0, 0, nenc, h, w, nullptr, &h, &w);
            t = res("enc.r" + std::to_string(l) + ".0", t, c[l], nenc, h, w);
            t = res("enc.r" + std::to_string(l) + ".1", t, c[l], nenc, h, w);
            e[l] = t; hy[l] = h; wx[l] = w;
        }
        std::vector<__nv_bfloat16*> zz(Lv);
        zz[Lv - 1] = e[Lv - 1];
        for (int l = Lv - 2; l >= 0; --l) {
            __nv_bfloat16* u = conv("enc.up" + std::to_string(l), t, c[l + 1], nullptr, 0, 0, nenc, h, w, nullptr, &h, &w);
            t = conv("enc.cat" + std::to_string(l), u, c[l], e[l], c[l], 0, nenc, h, w, nullptr, nullptr, nullptr);
            t = res("enc.ru" + std::to_string(l), t, c[l], nenc, h, w);
            zz[l] = t;
        }
        if (!ok_) return false;
        z = zz;
        if (arena_) return true;   // arena buffers belong to the arena owner
        // hand the context features over to the caller (they outlive this runner)
        for (__nv_bfloat16* p : zz) {
            for (size_t i = 0; i < tmp_.size(); ++i)
                if (tmp_[i] == p) { tmp_.erase(tmp_.begin() + i); break; }
        }
        return true;
    }

    // out (FP32 [nb][ny][nx][2]) for solver inputs xin BF16 [nb][ny][nx][16]; the
    // context image of solver image b is z[.][zmap ? zmap[b] : 0] -- handled by the
    // caller passing per-image contexts through `zsel` (one z pointer set per call)
    bool solver(const __nv_bfloat16* xin, int nb, int ny, int nx, const std::vector<__nv_bfloat16*>& z, int z_bcast,
                float* out) {
        const int Lv = m_->levels;
        const std::vector<int>& c = m_->widths;
        std::vector<__nv_bfloat16*> s(Lv);
        int h = ny, w = nx;
        __nv_bfloat16* t = conv("sol.in", xin, 16, nullptr, 0, 0, nb, h, w, nullptr, nullptr, nullptr);
        t = conv("sol.cat0", t, c[0], z[0], c[0], z_bcast, nb, h, w, nullptr, nullptr, nullptr);
        t = res("sol.r0", t, c[0], nb, h, w);
        s[0] = t;
        for (int l = 1; l < Lv; ++l) {
            t = conv("sol.down" + std::to_string(l), t, c[l - 1], nullptr, 0, 0, nb, h, w, nullptr, &h, &w);
            t = conv("sol.cat" + std::to_string(l), t, c[l], z[l], c[l], z_bcast, nb, h, w, nullptr, nullptr, nullptr);
            t = res("sol.r" + std::to_string(l), t, c[l], nb, h, w);
            s[l] = t;
        }
        for (int l = Lv - 2; l >= 0; --l) {
            __nv_bfloat16* u = conv("sol.up" + std::to_string(l), t, c[l + 1], nullptr, 0, 0, nb, h, w, nullptr, &h, &w);
            t = conv("sol.ucat" + std::to_string(l), u, c[l], s[l], c[l], 0, nb, h, w, nullptr, nullptr, nullptr);
            t = res("sol.ru" + std::to_string(l), t, c[l], nb, h, w);
        }
        conv("sol.out", t, c[0], nullptr, 0, 0, nb, h, w, nullptr, nullptr, nullptr, out);
        return ok_;
    }

    // per-image context index (device array) into nctx context images
    void set_zmap(const int* zmap, int nctx) { zmap_ = zmap; nctx_ = nctx; }
    void set_tape(std::vector<TapeOp>* t) { tape_ = t; }

   private:
    const int* zmap_ = nullptr;   // per-image context index used when x1_bcast == 2
    int nctx_ = 1;                // context images zmap_ indexes
    std::vector<TapeOp>* tape_ = nullptr;
    std::vector<void*>* arena_;
    std::vector<size_t>* arena_bytes_;
    size_t next_ = 0;
    cnn_model* m_;
    const helm_ctx* ctx_;
    cudaStream_t st_;
    std::vector<void*> tmp_;
    bool ok_ = true;
};

// Backward pieces of one convolution layer (cnn_train.cu).
// dW, db += weight and bias gradient (tensor cores, deterministic; CUDA-core path 1 or fallback)
int layer_wgrad(const __nv_bfloat16* x0, int c0, const __nv_bfloat16* x1, int c1, int x1_bcast, const int* x1_map,
                int nb1, int nb, int hin, int win, int hout, int wout, int mode, const __nv_bfloat16* g, int npad,
                int cout, int cin, float* dW, float* db, float** scratch, size_t* scratch_cap, int* err,
                cudaStream_t st, const helm_ctx* prof_ctx);
// target += W^T g for input channels off .. off + cp - 1 (tensor cores)
int layer_dgrad(const __nv_bfloat16* g, int npad, const __nv_bfloat16* W, int cin_pad, int off, int cp, int mode,
                int nb, int hin, int win, int hout, int wout, float* target, __nv_bfloat16* Wt, float* fine, int* err,
                cudaStream_t st, const helm_ctx* prof_ctx);

inline int check_conv_error(cnn_model* m, cudaStream_t st) {
    int h = 0;
    HELM_CK(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaStreamSynchronize(st));
    if (h) {
        set_error("a tensor-core convolution wait expired");
        cudaMemsetAsync(m->err, 0, sizeof(int), st);
        return HELM_ETIMEOUT;
    }
    return HELM_OK;
}


}  // namespace helm
