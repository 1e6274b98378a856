// Weight gradient of the 3x3 convolutions on the tensor cores (k_wgrad_tc.cu),
// used by the backward pass (cnn_train.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace helm {

struct WgradArgs {
    const __nv_bfloat16* x0;     // layer input [nb][c0/8][hin][win][8] (chunked layout)
    int c0;
    const __nv_bfloat16* x1;     // concatenated second input or nullptr
    int c1;
    int x1_bcast;                // 1: x1 has one image
    const int* x1_map;           // or the image of x1 per output image (device), else b
    int nb1;                     // images in x1 (0: 1 when x1_bcast, else nb)
    int nb, hin, win, hout, wout;
    int mode;                    // 0 same, 1 stride-2 down, 2 nearest-x2 up
    const __nv_bfloat16* g;      // output gradient [nb][npad/8][hout][wout][8]
    int npad, cout, cin;         // N of the GEMM; logical output / input channels (weights [cout][9][cin])
    float* dW;                   // += weight gradient
    float* db;                   // += bias gradient
    float* partials;             // scratch: max_splits x 9 x (c0 + c1) x npad floats
    int max_splits;
    float* bias_partials;        // scratch: max_bias_segments x npad floats
    int max_bias_segments;
    int* err;                    // set to 1 when a bounded wait expires
};

struct WgradGeom {
    int mode;
    int tw, rows, P;             // K tile: rows x tw pixels of the tile grid, P = rows tw (a multiple of 16)
    int tiles_x, tiles_y, phases;
    long long ktiles;            // nb x tiles x phases
    int cx, cx0;                 // 8-channel chunks of the input per tap (all / from x0)
    int gchunks;                 // 8-channel chunks of g (npad / 8)
    int taps_per_group, ngroups, max_chunks;
    int plane;                   // bytes of one staged plane (P x 16)
    int stage, ns, slack;        // bytes per stage, stages, bytes after the ring
    uint32_t tmem_cols;
    int splits;                  // CTAs along K (gridDim.x)
};

WgradGeom wgrad_plan(int mode, int c0, int c1, int npad, int hin, int win, int hout, int wout, int nb, int sms);
// HELM_EINVAL when the layer does not fit the kernel (nothing launched)
int launch_wgrad_tc(const WgradArgs& a, cudaStream_t st);

}  // namespace helm
