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

}  // namespace mrs
