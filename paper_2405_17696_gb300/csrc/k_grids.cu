// Several grids at once (per-frequency grids of the FWI windows: each frequency
// window solved on a grid of about ten points per wavelength over the same
// rectangle, so that the low frequencies cost far less than the high ones):
//   * helm_resample: a field moved between two node grids that cover the same
//     rectangle (bilinear interpolation), to carry the model m from the fine grid
//     to a window's grid and the window's model update back;
//   * helm_solve_multi: the batches of several contexts (grids of different
//     sizes) solved in one call, each context on its own stream from its own host
//     thread, so that their kernels share the GPU.
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "helm_internal.cuh"

namespace helm {
namespace {

// node (i, j) of an n_x x n_z grid covering [0, Lx] x [0, Lz] sits at the cell centre
// ((i + 1/2) Lx / n_x, (j + 1/2) Lz / n_z); dst = alpha * bilinear(src) + beta * dst,
// with the source coordinates clamped to its outermost nodes
__global__ void resample_kernel(const float* __restrict__ src, int nx0, int nz0, float* __restrict__ dst, int nx1,
                                int nz1, float alpha, float beta) {
    const long long n = (long long)nx1 * nz1;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx1), j = (int)(p / nx1);
        // position in source node units, (i + 1/2) nx0 / nx1 - 1/2 = ((2i + 1) nx0 - nx1) / (2 nx1),
        // split exactly into its integer part and fraction (clamped to the outermost nodes)
        int i0, j0;
        float fx, fz;
        {
            const long long num = (2ll * i + 1) * nx0 - nx1, den = 2ll * nx1;
            if (num <= 0) { i0 = 0; fx = 0.0f; }
            else if (num >= (long long)(nx0 - 1) * den) { i0 = nx0 - 1; fx = 0.0f; }
            else { i0 = (int)(num / den); fx = (float)(num - (long long)i0 * den) / (float)den; }
        }
        {
            const long long num = (2ll * j + 1) * nz0 - nz1, den = 2ll * nz1;
            if (num <= 0) { j0 = 0; fz = 0.0f; }
            else if (num >= (long long)(nz0 - 1) * den) { j0 = nz0 - 1; fz = 0.0f; }
            else { j0 = (int)(num / den); fz = (float)(num - (long long)j0 * den) / (float)den; }
        }
        const int i1 = min(i0 + 1, nx0 - 1), j1 = min(j0 + 1, nz0 - 1);
        const float a = src[(size_t)j0 * nx0 + i0], b = src[(size_t)j0 * nx0 + i1];
        const float c = src[(size_t)j1 * nx0 + i0], d = src[(size_t)j1 * nx0 + i1];
        const float v = (1.0f - fz) * ((1.0f - fx) * a + fx * b) + fz * ((1.0f - fx) * c + fx * d);
        dst[p] = alpha * v + (beta != 0.0f ? beta * dst[p] : 0.0f);
    }
}

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

int helm_resample(const float* src, int nx0, int nz0, float* dst, int nx1, int nz1, float alpha, float beta,
                  void* stream) {
    set_error("");
    if (!src || !dst || nx0 < 1 || nz0 < 1 || nx1 < 1 || nz1 < 1 || !device_ptr(src) || !device_ptr(dst)) {
        set_error("helm_resample: device arrays and positive sizes expected");
        return HELM_EINVAL;
    }
    if (src == dst) { set_error("helm_resample: src and dst must not alias"); return HELM_EINVAL; }
    const cudaStream_t st = (cudaStream_t)stream;
    { resample_kernel<<<1184, 256, 0, st>>>(src, nx0, nz0, dst, nx1, nz1, alpha, beta); count_launch(); }
    HELM_CK(cudaGetLastError());
    HELM_CK(cudaStreamSynchronize(st));
    return HELM_OK;
}

int helm_solve_multi(helm_ctx* const* ctxs, int nctx, const helm_c64* const* rhs, helm_c128* const* x,
                     const int* nrhs, const int* const* freq_idx, double tol, int flags, helm_stats* stats) {
    set_error("");
    if (!ctxs || nctx < 1 || !rhs || !x || !nrhs) { set_error("helm_solve_multi: invalid argument"); return HELM_EINVAL; }
    for (int i = 0; i < nctx; ++i) {
        if (!ctxs[i] || nrhs[i] < 0) { set_error("helm_solve_multi: invalid context or batch size"); return HELM_EINVAL; }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) { set_error("helm_solve_multi: a context appears twice"); return HELM_EINVAL; }
    }
    std::vector<int> status(nctx, HELM_OK);
    std::vector<std::string> errors(nctx);
    std::vector<std::thread> threads;
    threads.reserve(nctx);
    int dev = 0;
    HELM_CK(cudaGetDevice(&dev));
    for (int i = 0; i < nctx; ++i)
        threads.emplace_back([&, i] {
            cudaSetDevice(dev);   // the caller's device, in this thread too
            status[i] = helm_solve(ctxs[i], rhs[i], x[i], nrhs[i], freq_idx ? freq_idx[i] : nullptr, tol, flags,
                                   stats ? &stats[i] : nullptr);
            errors[i] = helm_last_error();
        });
    for (std::thread& t : threads) t.join();
    // the first hard error wins, else the first soft status (ENOCONV / EBREAKDOWN)
    int soft = HELM_OK;
    for (int i = 0; i < nctx; ++i) {
        if (status[i] == HELM_OK) continue;
        if (status[i] == HELM_ENOCONV || status[i] == HELM_EBREAKDOWN) {
            if (soft == HELM_OK) {
                soft = status[i];
                set_error("context " + std::to_string(i) + ": " + errors[i]);
            }
            continue;
        }
        set_error("context " + std::to_string(i) + ": " + errors[i]);
        return status[i];
    }
    return soft;
}

}  // extern "C"
