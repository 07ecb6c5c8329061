// Internal interface shared by the fusion-network translation units (fuse.cu:
// the all-high-resolution network, metrics and gate; rdn.cu: the method's own
// two-encoder network of Sec. 4).
#pragma once

#include "common.cuh"

namespace mrs {

// Epilogues of the FP32 SIMT 3x3 convolution
enum SimtMode {
    SIMT_PLAIN = 0,    // out = acc + b (optional ReLU)
    SIMT_RESID = 1,    // out = res + (acc + b)
    SIMT_FINAL = 2,    // out[p][c < 3] = (acc + b) + bilinear_up(lrhs)[p]
    SIMT_MASK = 3,     // out = res > 0 ? acc + b : 0
    SIMT_RESRELU = 4,  // out = res + relu(acc + b)
};

// FP32 3x3 convolution with zero padding 1 on [N][H][W][.] tensors:
// out[p][o] (o < cout, pixel stride os) from x[p][c] (c < cin, pixel stride
// xs); res has pixel stride rs.  Asynchronous on st.
mrs_status simt_conv3x3(const float* x, int cin, int xs, const float* w, const float* b, int cout,
                        int mode, int relu, const float* res, int rs, float* out, int os,
                        const float* lrhs, int N, int H, int W, int s, cudaStream_t st);

// ---- FP32 training launches (fuse.cu), asynchronous on st ------------------
constexpr int kDwParts = 64;       // pixel-split partial sums of dw_tiles_f32
constexpr int kLossParts = 1024;   // float64 partial sums of loss_grad_f32

// Weight / bias gradient partial sums of a convolution with zero padding 1:
// x [P][xs] (first cin channels), dy [P][ys] (first cout), any cin / cout, in
// 64 x 64 channel tiles z = ot * ceil(cin / 64) + ct.  part holds
// [z][kDwParts][ntaps][64 * 64] floats (ntaps = 9, or 1 when centre_only: the
// centre tap alone, a 1x1 conv), tile z's tap j at part[z][g][j] as
// [cout_t][cin_t];
// dbpart holds [ot][kDwParts * 64] floats, [g][cout_t] packed.  The sums over
// g are left to the caller.
mrs_status dw_tiles_f32(const float* x, int cin, int xs, const float* dy, int cout, int ys, int N,
                        int H, int W, int centre_only, float* part, float* dbpart, cudaStream_t st);
// transposed-conv weights wt[c][t][o] = w[o][8 - t][c] (w [cout][9][cin])
void wtrans_f32(const float* w, int cin, int cout, float* wt, cudaStream_t st);
// training loss (MRS_LOSS_*) of y against min(target, clip) over n values:
// dy = dL/dy, *sum (device double) = the sum of the per-value losses,
// parts = kLossParts doubles of scratch
mrs_status loss_grad_f32(const float* y, const float* tgt, size_t n, float clip, int kind,
                         float beta, float* dy, double* parts, double* sum, cudaStream_t st);
// one bias-corrected Adam update (beta1 0.9, beta2 0.999, eps 1e-8) at step `step` (>= 1)
mrs_status adam_f32(float* p, const float* g, float* m, float* v, size_t n, float lr, int64_t step,
                    cudaStream_t st);

}  // namespace mrs
