// Tensor-core 3x3 convolution (implicit GEMM on tcgen05) used by the fusion
// network: internal interface between conv_tc.cu and fuse.cu.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "common.cuh"

namespace mrs {

// Epilogue modes of the tensor-core convolution
enum TcMode : int {
    TC_RELU_BF16 = 0,   // out_bf16[p][64] = relu(acc + b)
    TC_RESID_BF16 = 1,  // out_bf16[p][64] = res[p] + (acc + b)   (res may alias out)
    TC_FINAL_F32 = 2,   // out_f32[p][3]  = (acc + b) + bilinear_up(lrhs)[p]
    TC_PLAIN_F32 = 3,   // out_f32[p][cout] = acc + b, optional relu
    TC_LIN_BF16 = 4,    // out_bf16[p][64] = acc + b
    TC_MASK_BF16 = 5,   // out_bf16[p][64] = mask[p] > 0 ? acc + b : 0   (mask via tmap_res)
    TC_RESRELU_BF16 = 6,// out_bf16[p][64] = res[p] + relu(acc + b)
};

enum TcOperand : int { TC_BF16 = 0, TC_FP8 = 1 };

struct TcConvArgs {
    const CUtensorMap* tmap_x;   // A operand [N][H][W][64] (bf16 or fp8, kABox-pixel boxes)
    const CUtensorMap* tmap_res; // TC_RESID_BF16 residual (bf16, kOutBox-pixel boxes)
    const CUtensorMap* tmap_out; // TC_RELU_BF16 / TC_RESID_BF16 output (bf16, kOutBox-pixel boxes)
    const CUtensorMap* tmap_w;   // packed weights [9 * nout][64]
    const float* bias;           // [nout] (padded)
    const float* wscale;         // fp8 only: per-output-channel dequant scale (may be NULL)
    float xscale;                // fp8 only: activation dequant scale
    const void* res;             // TC_RESID_BF16 residual (bf16 [p][64])
    void* out;                   // output
    const float* lrhs;           // TC_FINAL_F32: [N][h][w][3]
    int N, H, W, scale;
    int nout;                    // 64 or 16 (MMA N)
    int cout;                    // valid output channels (TC_PLAIN_F32 / TC_FINAL_F32)
    int relu;                    // TC_PLAIN_F32
    int mode;
    int operand;                 // TC_BF16 / TC_FP8
    int* err;                    // device error word (timeouts)
    // TC_RELU_BF16 / TC_RESID_BF16 with fp8 operands: also emit the fp8 copy
    void* out_fp8;
    float out_fp8_inv_scale;
    // with out_fp8: write only the fp8 copy (the bf16 result has no reader)
    int fp8_only;
    // A convolution over kc > 1 input tensors of 64 channels each (the
    // concatenation of their channels) in ONE launch: amaps = DEVICE array of
    // kc A-operand maps (64-byte aligned, alive until the kernel completes),
    // weights of chunk j at rows w_row0 + (9 j + t) nout of tmap_w.  kc <= 1:
    // tmap_x, weights at rows w_row0 + t nout.
    const CUtensorMap* amaps;
    int kc;
    int w_row0;
};

// Box widths (pixels): the conv reads one 130-pixel A box per input row (a
// tile's 128 outputs plus a halo pixel on each side) and moves 128-pixel
// residual / output boxes.  Maps passed to tc_conv3x3 use these widths (the
// same for both operand types).
constexpr int kABox = 130;
constexpr int kOutBox = 128;
inline int tc_a_box(int /*operand*/) { return kABox; }
inline int tc_out_box(int /*operand*/) { return kOutBox; }
// Encode a tiled tensor map for a [N][H][W][64] activation tensor (rows of 128
// bytes in bf16, 64 in fp8): box = box_px pixels of one image row.
mrs_status tc_make_act_map(CUtensorMap* m, const void* ptr, int N, int H, int W, int operand,
                           int box_px = 128);
// Tensor map for a strided view of a bf16 activation tensor: element (x, y, n)
// of the view is the 64-channel row at ptr + x * px_stride + y * row_stride +
// n * img_stride (bytes, multiples of 16).  Views select a sub-pixel grid of
// a larger image (a deshuffle chunk as an A operand, or a shuffle target as
// an output) without moving data.
mrs_status tc_make_view_map(CUtensorMap* m, const void* ptr, int N, int H, int W,
                            long long px_stride, long long row_stride, long long img_stride,
                            int box_px);
// Tensor map for packed weights [rows][64 (bf16) | 64 (fp8)].
mrs_status tc_make_w_map(CUtensorMap* m, const void* ptr, int rows, int nout, int operand);

mrs_status tc_conv3x3(const TcConvArgs& a, cudaStream_t st);
// input-row ring depth of every later conv launch (0: the most that fits)
void tc_set_ring(int stages);

// Weight and bias gradients of a 3x3 conv (zero padding 1) on the tensor
// cores, as per-CTA partial sums:
//   part[g][t][o][c] (t = ky * 3 + kx) = sum over CTA g's pixels p of
//       dy[p][o] * x[p + (ky - 1, kx - 1)][c],   dbpart[g][o] = sum dy[p][o]
// for o < cout, c < cin.  x and dy are bf16 [N][H][W][64] tensors described
// by tc_make_act_map with box widths kWgKB + 2 (x) and kWgKB (dy).  *nparts
// receives the number of partials written (at most tc_wgrad_max_parts()).
constexpr int kWgKB = 64;
struct TcWgradArgs {
    const CUtensorMap* tmap_x;
    const CUtensorMap* tmap_dy;
    float* part;
    float* dbpart;
    int N, H, W, cin, cout;
    int* err;
    // at most this many CTAs (= partials), 0: one per SM.  Several small
    // gradients launched side by side on different streams, each on a share
    // of the SMs, write that many fewer partials each.
    int max_ctas = 0;
};
int tc_wgrad_max_parts();
mrs_status tc_conv3x3_wgrad(const TcWgradArgs& a, int* nparts, cudaStream_t st);

// Launches a kernel whose bounded mbarrier wait can never complete; *gave_up
// = 1 if the wait gave up after limit_cycles and raised the error word.
mrs_status tc_wait_selftest(long long limit_cycles, int* gave_up, cudaStream_t st);

}  // namespace mrs
