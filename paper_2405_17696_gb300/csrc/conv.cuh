// Arguments of the tensor-core 3x3 convolution (k_conv.cu), shared with the
// network driver (cnn.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace helm {

// Activations of the network are BF16 in the chunked layout [n][C/8][H][W][8]:
// per image, one plane per 8 channels with 16 bytes per pixel (C a multiple of
// 8).  A plane row is contiguous, so a TMA box of one plane is long rows, and
// the plane is exactly the K-major core-matrix layout of the tensor cores.
__host__ __device__ __forceinline__ size_t nc8(long long b, int c, long long pix, int C, long long hw) {
    return (((size_t)b * (size_t)(C >> 3) + (size_t)(c >> 3)) * (size_t)hw + (size_t)pix) * 8 + (size_t)(c & 7);
}

// Nearest x2 upsampling followed by a 3x3 convolution (mode 2) is, per output
// parity p in {0, 1} along an axis, a 2-tap convolution on the coarse grid: the
// fine node 2Y + p with tap d in {-1, 0, 1} reads the coarse node
// floor((2Y + p + d) / 2) = Y + floor((p + d) / 2), which is Y + p - 1 + e for
// e = up_phase_tap(p, d) in {0, 1}.  The weights of the taps that share e add up.
__host__ __device__ __forceinline__ int up_phase_tap(int p, int d) { return (p + d + 2) / 2 - 1 - p + 1; }
// merged tap of output parity ph = 2 py + px and coarse offset (ey, ex): row ph * 4 + 2 ey + ex
__host__ __device__ __forceinline__ int up_merged_index(int py, int px, int dy, int dx) {
    return (2 * py + px) * 4 + 2 * up_phase_tap(py, dy) + up_phase_tap(px, dx);
}

struct ConvArgs {
    const __nv_bfloat16* x0;   // [nb][c0/8][hin][win][8] (chunked layout, see nc8)
    int c0;
    const __nv_bfloat16* x1;   // second input concatenated after x0's channels, or nullptr
    int c1;
    int x1_bcast;              // 1: x1 has one image shared by the whole batch
    const int* x1_map;         // or: image of x1 used by output image b (device array), else b
    int nb1 = 0;               // images in x1 (0: 1 when x1_bcast, else nb)
    int nb, hin, win, hout, wout;
    int mode;                  // 0 same, 1 down (output node (Y,X) on input node (2Y+1,2X+1)), 2 up (nearest x2),
                               // 3 transpose of down: output on the fine grid, tap d of output node f reads
                               //   input node (f - 1 - d) / 2 when that is an integer inside the input
    const __nv_bfloat16* w;    // [npad][9][c0 + c1]
    const __nv_bfloat16* wup = nullptr;   // mode 2: the phase-merged weights [npad][16][c0 + c1]
                                          // (up_merged_index), which the tensor-map kernel needs
    const float* bias;         // [npad]
    const __nv_bfloat16* res;  // [nb][npad/8][hout][wout][8] added before the activation, or nullptr
    void* y;                   // bf16 [nb][npad/8][hout][wout][8], or fp32 [nb][hout][wout][cstore]
    int npad;                  // N of the MMA: 16, 32, 64 or 128
    int cstore;                // channels stored when out_fp32
    int relu;
    int out_fp32;
    int accum;                 // with out_fp32: y += result (no bias, no activation)
    int* err;                  // set to 1 when a bounded wait expires
};

int launch_conv3x3(const ConvArgs& a, cudaStream_t st);
// layers through TMA-staged halo tiles (k_conv_tma.cu); HELM_EINVAL = not launched.
// narrow: 0 plain; 1, 16-channel same-grid layers take the column-taps-in-N variant;
// 2, 16- and 32-channel same-grid layers take the row-taps-in-N variant (three tap rows
// of a staged row in one MMA's N).
int launch_conv3x3_tma(const ConvArgs& a, cudaStream_t st, int narrow);
// Autotuning of the TMA kernel's tiling: while on, the first launch of each layer
// shape times the candidate tilings and records the fastest, which every later
// launch of that shape uses (process-wide table).
void conv_tuning(bool on);
// TMA tensor map of a chunked activation (k_conv_tma.cu): es 1 plain, es 2 with
// element stride 2 along w and h; a box lands as [chunk][row][pixel][8].
bool tma_map_act(CUtensorMap* m, const void* base, int c, int w, int h, int n, int box_w, int box_h, int box_chunks,
                 int es);
int conv_tuned_count();
void conv_tune_reset();

}  // namespace helm
