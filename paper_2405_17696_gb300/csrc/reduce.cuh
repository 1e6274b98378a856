// Block reductions with a per-RHS "last block finishes" step: every block of
// one right-hand side writes its partial sums, the last block to arrive sums
// them in tile order (deterministic) and runs a finishing step.
#pragma once

#include "helm_internal.cuh"

namespace helm {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Reduce `nv` double2 values (vals[i] valid for i < nv) over the block, store
// the block's partials to `dst[0..nv)`, and report whether this block is the
// last of `ntiles` blocks of its RHS to finish (the counter is reset then).
// `smem` must hold (blockDim/32) * NV double2.  All threads must call it.
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

template <int NV, class T>
__device__ bool reduce_block_last(const T (&vals)[NV], int nv, double2* dst, unsigned* counter,
                                  int ntiles, double2* smem) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            double2 v = to_d2(vals[i]);
            double a = warp_sum(v.x);
            double b = warp_sum(v.y);
            if (lane == 0) smem[warp * NV + i] = make_double2(a, b);
        }
    }
    __syncthreads();
    if (tid < nv) {
        double2 acc = make_double2(0.0, 0.0);
        for (int w = 0; w < nwarps; ++w) acc = dadd(acc, smem[w * NV + tid]);
        dst[tid] = acc;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned s_last;
    if (tid == 0) {
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == (unsigned)ntiles - 1u) ? 1u : 0u;
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0u;
}

// Sum partials[t][i] over tiles t in order (t fastest stride `stride`).
__device__ __forceinline__ double2 sum_partials(const double2* p, int ntiles, int stride, int i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < ntiles; ++t) {
        double2 v = __ldcg(p + (size_t)t * stride + i);
        acc = dadd(acc, v);
    }
    return acc;
}

}  // namespace helm
