// helm_residual_noalloc: the FP64 residual r = b - H x and its per-RHS
// relative norm ||r|| / ||b|| (the computation behind helm_residual), for
// callers that cannot allocate device memory.  Some callers cannot call
// cudaMalloc: a process whose device memory is already reserved by another
// allocator (a framework's caching pool that owns the whole budget), or a
// latency-critical loop where an allocation and the synchronisation it can
// imply are not acceptable.  This entry point allocates nothing: it takes no
// context, every input and output is a caller-provided device pointer, and
// the only scratch it needs (per-block partial sums and per-RHS arrival
// counters) lives in a file-scope device array of fixed size that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "helm_internal.cuh"
#include "reduce.cuh"

namespace helm {
namespace {

// Scratch capacity: partial sums for at most NOALLOC_MAX_PARTIALS (RHS, tile)
// pairs and arrival counters for at most NOALLOC_MAX_RHS right-hand sides.
// A tile is 32 x 64 grid nodes, so a 512 x 256 grid has 64 tiles and up to
// 1024 such right-hand sides fit in one call.
constexpr int NOALLOC_MAX_RHS = 4096;
constexpr int NOALLOC_MAX_PARTIALS = 65536;
constexpr size_t NOALLOC_PARTIAL_BYTES = (size_t)NOALLOC_MAX_PARTIALS * sizeof(double2);   // 1 MiB
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_PARTIAL_BYTES + (size_t)NOALLOC_MAX_RHS * sizeof(unsigned);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NT = TILE_X * TILE_Y;

__global__ void __launch_bounds__(NT) residual_noalloc_kernel(const float* __restrict__ kappa,
                                                              const float* __restrict__ gamma, int nx, int nz,
                                                              double ax, double az, const float* __restrict__ omega,
                                                              const float2* __restrict__ bvec,
                                                              const double2* __restrict__ x,
                                                              float2* __restrict__ r, double* __restrict__ rel,
                                                              double2* __restrict__ partials,
                                                              unsigned* __restrict__ counters) {
    const int b = blockIdx.z;
    const size_t N = (size_t)nx * nz;
    const double2* xb = x + (size_t)b * N;
    const float2* bb = bvec + (size_t)b * N;
    float2* rb = r + (size_t)b * N;
    const int ix = blockIdx.x * TILE_X + threadIdx.x;
    const int iz0 = (blockIdx.y * TILE_Y + threadIdx.y) * ROWS;
    const double w = omega[b];
    double acc_r = 0.0, acc_b = 0.0;
    if (ix < nx) {
        for (int rr = 0; rr < ROWS; ++rr) {
            const int iz = iz0 + rr;
            if (iz >= nz) break;
            const size_t p = (size_t)iz * nx + ix;
            const double2 z0 = make_double2(0.0, 0.0);
            const double2 xc = xb[p];
            const double2 xw = ix > 0 ? xb[p - 1] : z0;
            const double2 xe = ix < nx - 1 ? xb[p + 1] : z0;
            const double2 xn = iz > 0 ? xb[p - nx] : z0;
            const double2 xs = iz < nz - 1 ? xb[p + nx] : z0;
            const double k = kappa[p];
            const double s = w * w * (k * k);
            const double ci = -s * (double)gamma[p];        // w^2 m (1 - i gamma) = s + i ci
            const double hre = ax * (2.0 * xc.x - xw.x - xe.x) + az * (2.0 * xc.x - xn.x - xs.x) - (s * xc.x - ci * xc.y);
            const double him = ax * (2.0 * xc.y - xw.y - xe.y) + az * (2.0 * xc.y - xn.y - xs.y) - (s * xc.y + ci * xc.x);
            const float2 bv = bb[p];
            const double rx = (double)bv.x - hre, ry = (double)bv.y - him;
            rb[p] = make_float2((float)rx, (float)ry);
            acc_r += rx * rx + ry * ry;
            acc_b += (double)bv.x * bv.x + (double)bv.y * bv.y;
        }
    }
    __shared__ double2 sm[NT / 32];
    double2 vals[1] = {make_double2(acc_r, acc_b)};
    const int ntiles = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    double2* part = partials + (size_t)b * ntiles;
    const bool last = reduce_block_last<1>(vals, 1, part + tile, counters + b, ntiles, sm);
    if (last && threadIdx.x == 0 && threadIdx.y == 0) {
        const double2 t = sum_partials(part, ntiles, 1, 0);
        rel[b] = t.y > 0.0 ? sqrt(t.x / t.y) : sqrt(t.x);
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the symbol is not a device address).
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {nullptr};

int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return HELM_ECUDA; }
    if (dev < 0 || dev >= 64) { set_error("helm_residual_noalloc: device ordinal above 63"); return HELM_EUNSUPPORTED; }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return HELM_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HELM_OK;
}

// Device memory of the current device `dev` (managed memory is reachable from
// every device); memory of another GPU is rejected, since the kernel would read
// it through the peer path, which faults where peer access is not enabled.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" int helm_residual_noalloc(const float* kappa, const float* gamma, int nx, int nz, float hx, float hz,
                                     const float* omega_rhs, const helm_c64* rhs, const helm_c128* x, helm_c64* r,
                                     double* rel_res, int nrhs, void* stream) {
    set_error("");
    if (nrhs == 0) return HELM_OK;
    if (!kappa || !gamma || !omega_rhs || !rhs || !x || !r || !rel_res || nrhs < 0 || nx < 1 || nz < 1 ||
        !(hx > 0) || !(hz > 0)) {
        set_error("helm_residual_noalloc: invalid argument");
        return HELM_EINVAL;
    }
    const int tiles = ((nx + TILE_X - 1) / TILE_X) * ((nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS));
    if (nrhs > NOALLOC_MAX_RHS || (long long)nrhs * tiles > NOALLOC_MAX_PARTIALS) {
        set_error("helm_residual_noalloc: " + std::to_string(nrhs) + " right-hand sides of " + std::to_string(nx) +
                  "x" + std::to_string(nz) + " need " + std::to_string((long long)nrhs * tiles) +
                  " partial sums; the fixed scratch holds " + std::to_string(NOALLOC_MAX_PARTIALS) + " and " +
                  std::to_string(NOALLOC_MAX_RHS) + " right-hand sides");
        return HELM_EINVAL;
    }
    int dev = 0;
    HELM_CK(cudaGetDevice(&dev));
    const void* ptrs[] = {kappa, gamma, omega_rhs, rhs, x, r, rel_res};
    for (const void* p : ptrs)
        if (!on_device(p, dev)) {
            set_error("helm_residual_noalloc: every array must be device memory of the current device "
                      "(nothing is staged)");
            return HELM_EINVAL;
        }
    void* base = nullptr;
    HELM_TRY(noalloc_scratch(&base));
    double2* partials = (double2*)base;
    unsigned* counters = (unsigned*)((unsigned char*)base + NOALLOC_PARTIAL_BYTES);
    cudaStream_t st = (cudaStream_t)stream;
    // the counters must start at zero; the array keeps whatever the last call left
    HELM_CK(cudaMemsetAsync(counters, 0, (size_t)nrhs * sizeof(unsigned), st));
    dim3 grid((nx + TILE_X - 1) / TILE_X, (nz + TILE_Y * ROWS - 1) / (TILE_Y * ROWS), nrhs);
    { residual_noalloc_kernel<<<grid, dim3(TILE_X, TILE_Y), 0, st>>>(
        kappa, gamma, nx, nz, 1.0 / ((double)hx * hx), 1.0 / ((double)hz * hz), omega_rhs, (const float2*)rhs,
        (const double2*)x, (float2*)r, rel_res, partials, counters); count_launch(); }
    HELM_CK(cudaGetLastError());
    return HELM_OK;
}
