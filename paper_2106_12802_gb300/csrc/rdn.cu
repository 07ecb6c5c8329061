// The method's own fusion network (Sec. 4, "two-encoder-one-decoder"): two
// shallow encoders (H_lrhs on the LRHS at low resolution, H_hrls on the HRLS
// and its layers at high resolution), D = log2(s) deshuffle layers that bring
// the HRLS features down to the LRHS grid, a 1x1 fuse conv, G = 3 residual
// dense groups of B = 5 blocks (Eqs. RDG, F_DF), shuffle upscaling and H_Rec.
// Readings: each block has three dense 3x3 convs and a 3x3 local-fusion conv
// over the 256-channel concatenation, then the local residual; every conv but
// H_Rec is followed by a ReLU; Eq. F_DF adds F_0; the deshuffle / shuffle
// channel order is that of pixel_unshuffle / pixel_shuffle (stride 2).
//
// FP32 path (reference precision): SIMT convolutions over concatenation
// buffers ([P][256] per block: F_in, F_1, F_2, F_3 side by side), the fuse conv
// over an explicitly deshuffled [P][64 + 64 s^2] buffer.
//
// BF16 path (tensor cores, conv_tc.cu): a conv over 64 c input channels is
// ONE launch that accumulates its c 64-channel chunks in TMEM (chunk-major
// over sub-pieces of at most six output rows; the chunk maps are passed in
// device memory).  Nothing is concatenated or rearranged in memory: a dense
// block's inputs stay separate [P][64] tensors, a deshuffle chunk is a
// strided tensor-map view of the HR feature map (sub-pixel (oy, ox) of every
// s x s block), the 1x1 fuse conv is the centre tap of 3x3 chunks, and a
// shuffle is four launches whose outputs are strided views of the 2x larger
// feature map.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <array>
#include <vector>

#include "conv_tc.cuh"
#include "fuse.cuh"

namespace mrs {
namespace {

constexpr int kF = 64;       // feature channels
constexpr int kRDG = 3;      // G
constexpr int kRDB = 5;      // B
constexpr int kConv = 4;     // convs per block

int depth_of(int s) { return s == 2 ? 1 : s == 4 ? 2 : s == 8 ? 3 : -1; }

struct RLayer {
    int k, cin, cout;
    size_t woff, boff;
};

// layers in forward (= parameter) order: H_lrhs, H_hrls, fuse, 60 block
// convs, D upsampling convs, H_Rec
std::vector<RLayer> rdn_layers(int s, int c_hr)
{
    std::vector<RLayer> L;
    size_t o = 0;
    auto add = [&](int k, int ci, int co) {
        L.push_back({k, ci, co, o, o + (size_t)co * k * k * ci});
        o += (size_t)co * k * k * ci + co;
    };
    add(3, 3, kF);
    add(3, c_hr, kF);
    add(1, kF + kF * s * s, kF);
    for (int g = 0; g < kRDG; ++g)
        for (int b = 0; b < kRDB; ++b)
            for (int c = 1; c <= kConv; ++c) add(3, kF * c, kF);
    for (int d = 0; d < depth_of(s); ++d) add(3, kF, 4 * kF);
    add(3, kF, 3);
    return L;
}

size_t rdn_nparams(int s, int c_hr)
{
    const auto L = rdn_layers(s, c_hr);
    return L.back().boff + L.back().cout;
}

// channel of the D-times deshuffled map that holds channel c of HR sub-pixel
// (oy, ox) of each s x s block: c s^2 + sum over steps d = 1..D of
// (2 dy_d + dx_d) 4^(D - d), dy_d / dx_d bit d - 1 of oy / ox
__host__ __device__ __forceinline__ int dsf_channel(int c, int oy, int ox, int D)
{
    int k = c;
    for (int d = 1; d <= D; ++d) k = 4 * k + 2 * ((oy >> (d - 1)) & 1) + ((ox >> (d - 1)) & 1);
    return k;
}

// ---- elementwise kernels ----------------------------------------------------
// I_HRLS of one pixel: RGB, albedo, normal (+ diffuse, specular, log(1 + var))
__device__ __forceinline__ int hr_pixel(const float* hrls, const float* alb, const float* nrm,
                                        const float* extra, size_t p, float* v)
{
    for (int k = 0; k < 3; ++k) {
        v[k] = __ldg(hrls + 3 * p + k);
        v[3 + k] = __ldg(alb + 3 * p + k);
        v[6 + k] = __ldg(nrm + 3 * p + k);
    }
    if (!extra) return 9;
    for (int k = 0; k < 6; ++k) v[9 + k] = __ldg(extra + 9 * p + k);
    for (int k = 0; k < 3; ++k) v[15 + k] = log1pf(fmaxf(__ldg(extra + 9 * p + 6 + k), 0.0f));
    return 18;
}

__global__ void k_hr_input_f32(const float* hrls, const float* alb, const float* nrm,
                               const float* extra, size_t P, float* out)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        float v[18];
        int c = hr_pixel(hrls, alb, nrm, extra, p, v);
        for (int k = 0; k < c; ++k) out[p * c + k] = v[k];
    }
}

// bf16 [P][64] rows, channels past the input's zero
__global__ void k_hr_input_bf16(const float* hrls, const float* alb, const float* nrm,
                                const float* extra, size_t P, __nv_bfloat16* out)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        float v[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0.0f;
        hr_pixel(hrls, alb, nrm, extra, p, v);
        uint4* o = (uint4*)(out + p * 64);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 u;
            __nv_bfloat162* h2 = (__nv_bfloat162*)&u;
#pragma unroll
            for (int e = 0; e < 4; ++e) h2[e] = __floats2bfloat162_rn(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
            o[j] = u;
        }
        const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 3; j < 8; ++j) o[j] = z;
    }
}

__global__ void k_lr_input_bf16(const float* lrhs, size_t P, __nv_bfloat16* out)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        uint4* o = (uint4*)(out + p * 64);
        uint4 u;
        __nv_bfloat162* h2 = (__nv_bfloat162*)&u;
        h2[0] = __floats2bfloat162_rn(__ldg(lrhs + 3 * p), __ldg(lrhs + 3 * p + 1));
        h2[1] = __floats2bfloat162_rn(__ldg(lrhs + 3 * p + 2), 0.0f);
        h2[2] = h2[3] = __floats2bfloat162_rn(0.0f, 0.0f);
        o[0] = u;
        const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 1; j < 8; ++j) o[j] = z;
    }
}

// D-times deshuffle of F [N][H][W][64] into channels [64, 64 + 64 s^2) of
// cat [N][H/s][W/s][os]: one thread per (HR pixel, channel)
__global__ void k_deshuffle_f32(const float* __restrict__ F, int N, int H, int W, int s, int D,
                                float* __restrict__ cat, int os)
{
    const size_t total = (size_t)N * H * W * 64;
    const int h = H / s, w = W / s;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(i % 64);
        size_t px = i / 64;
        int X = (int)(px % W);
        size_t r = px / W;
        int Y = (int)(r % H), n = (int)(r / H);
        int k = dsf_channel(c, Y % s, X % s, D);
        cat[(((size_t)n * h + Y / s) * w + X / s) * os + 64 + k] = F[i];
    }
}

// x2 shuffle: T [N][h][w][ts] (256 channels used) -> U [N][2h][2w][64],
// U[2y + dy][2x + dx][c] = T[y][x][4c + 2dy + dx]
__global__ void k_shuffle_f32(const float* __restrict__ T, int ts, int N, int h, int w,
                              float* __restrict__ U)
{
    const size_t total = (size_t)N * 4 * h * w * 64;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(i % 64);
        size_t px = i / 64;
        int X = (int)(px % (2 * w));
        size_t r = px / (2 * w);
        int Y = (int)(r % (2 * h)), n = (int)(r / (2 * h));
        U[i] = T[(((size_t)n * h + Y / 2) * w + X / 2) * ts + 4 * c + 2 * (Y & 1) + (X & 1)];
    }
}

// dst[p][c] (+)= src[p][c] for c < 64 (pixel strides ds, ss)
__global__ void k_ch64_f32(float* __restrict__ dst, int ds, const float* __restrict__ src, int ss,
                           size_t P, int add)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 64;
        int c = (int)(i % 64);
        float v = src[p * ss + c];
        dst[p * ds + c] = add ? dst[p * ds + c] + v : v;
    }
}

// dst += src over bf16 [n] (8 values per thread)
__global__ void k_add_bf16(__nv_bfloat16* __restrict__ dst, const __nv_bfloat16* __restrict__ src,
                           size_t n8)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8;
         i += (size_t)gridDim.x * blockDim.x) {
        uint4 a = ((const uint4*)dst)[i], b = ((const uint4*)src)[i];
        __nv_bfloat162* pa = (__nv_bfloat162*)&a;
        const __nv_bfloat162* pb = (const __nv_bfloat162*)&b;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 x = __bfloat1622float2(pa[e]), y = __bfloat1622float2(pb[e]);
            pa[e] = __floats2bfloat162_rn(x.x + y.x, x.y + y.y);
        }
        ((uint4*)dst)[i] = a;
    }
}

// the 1x1 fuse weights [64][cin] as 3x3 weights with only the centre tap
__global__ void k_centre_tap(const float* __restrict__ w1, int cin, float* __restrict__ w3)
{
    size_t n = (size_t)64 * 9 * cin;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(i % cin);
        int t = (int)((i / cin) % 9);
        size_t o = i / ((size_t)cin * 9);
        w3[i] = t == 4 ? w1[o * cin + c] : 0.0f;
    }
}

// ---- training (FP32): elementwise steps of the backward pass --------------
// dst[p][c] = ((a + b) + c2) + d2 for c < 64, the sources added in that order
// (c2 / d2 may be NULL); pixel strides ds, as, bs, cs, es
__global__ void k_sum64(float* __restrict__ dst, int ds, const float* a, int as, const float* b,
                        int bs, const float* c2, int cs, const float* d2, int es, size_t P)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 64;
        int c = (int)(i % 64);
        float v = a[p * as + c] + b[p * bs + c];
        if (c2) v = v + c2[p * cs + c];
        if (d2) v = v + d2[p * es + c];
        dst[p * ds + c] = v;
    }
}

// out[p][c] = act[p][c] > 0 ? d[p][c] : 0 for c < 64 (a ReLU's gradient mask
// from its output; out may be d)
__global__ void k_mask64(const float* d, int dstr, const float* __restrict__ act, int astr,
                         float* out, int ostr, size_t P)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 64;
        int c = (int)(i % 64);
        out[p * ostr + c] = act[p * astr + c] > 0.0f ? d[p * dstr + c] : 0.0f;
    }
}

// start of a dense block's backward: dCat [P][256] holds dF_out in channels
// 0..63 (the block's residual skip passes it to F_in unchanged); dz4 = dF_out
// masked by the local-fusion ReLU (R = its output), channels 64..255 cleared
__global__ void k_block_bwd_init(float* __restrict__ dcat, const float* __restrict__ R,
                                 float* __restrict__ dz4, size_t P)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 256;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 256;
        int c = (int)(i % 256);
        if (c < 64) dz4[p * 64 + c] = R[p * 64 + c] > 0.0f ? dcat[i] : 0.0f;
        else dcat[i] = 0.0f;
    }
}

// gradient of the x2 shuffle, masked by the upsampling conv's ReLU:
// dz[y][x][4c + 2dy + dx] = dU[2y + dy][2x + dx][c] if T[y][x][4c + 2dy + dx] > 0
// (T = that conv's ReLU output [N][h][w][256], dU [N][2h][2w][64])
__global__ void k_unshuffle_mask(const float* __restrict__ dU, const float* __restrict__ T, int N,
                                 int h, int w, float* __restrict__ dz)
{
    const size_t total = (size_t)N * h * w * 256;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(i % 256);
        size_t px = i / 256;
        int x = (int)(px % w);
        size_t r = px / w;
        int y = (int)(r % h), n = (int)(r / h);
        int c = k >> 2, dy = (k >> 1) & 1, dx = k & 1;
        float g = dU[(((size_t)n * 2 * h + 2 * y + dy) * 2 * w + 2 * x + dx) * 64 + c];
        dz[i] = T[i] > 0.0f ? g : 0.0f;
    }
}

// gradient of the D deshuffles, masked by H_hrls's ReLU: dz [N][H][W][64] from
// channels [64, 64 + 64 s^2) of dcat [N][H/s][W/s][cs] (the inverse of
// k_deshuffle_f32's permutation); F = H_hrls's ReLU output
__global__ void k_dsf_grad_mask(const float* __restrict__ dcat, int cs, const float* __restrict__ F,
                                int N, int H, int W, int s, int D, float* __restrict__ dz)
{
    const size_t total = (size_t)N * H * W * 64;
    const int h = H / s, w = W / s;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(i % 64);
        size_t px = i / 64;
        int X = (int)(px % W);
        size_t r = px / W;
        int Y = (int)(r % H), n = (int)(r / H);
        int k = dsf_channel(c, Y % s, X % s, D);
        float g = dcat[(((size_t)n * h + Y / s) * w + X / s) * cs + 64 + k];
        dz[i] = F[i] > 0.0f ? g : 0.0f;
    }
}

// gw[o][t][c] (a layer's [cout][ntaps][cin] gradient) and gb[o] = sums over
// the kDwParts pixel splits of dw_tiles_f32's 64 x 64 tiles, in split order
__global__ void k_dw_reduce_tiles(const float* __restrict__ part, const float* __restrict__ dbpart,
                                  int ntaps, int cin, int cout, float* __restrict__ gw,
                                  float* __restrict__ gb)
{
    const size_t nw = (size_t)cout * ntaps * cin;
    const int ctiles = (cin + 63) / 64;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nw + cout;
         i += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        if (i < nw) {
            int c = (int)(i % cin), t = (int)((i / cin) % ntaps), o = (int)(i / ((size_t)cin * ntaps));
            int ct = c / 64, ot = o / 64;
            int cin_t = min(64, cin - 64 * ct), cout_t = min(64, cout - 64 * ot);
            const float* q = part + (size_t)(ot * ctiles + ct) * kDwParts * ntaps * 4096 +
                             (size_t)t * cout_t * cin_t + (size_t)(o % 64) * cin_t + c % 64;
            for (int g = 0; g < kDwParts; ++g) acc += q[(size_t)g * ntaps * cout_t * cin_t];
            gw[i] = acc;
        } else {
            int o = (int)(i - nw), ot = o / 64, cout_t = min(64, cout - 64 * ot);
            const float* q = dbpart + (size_t)ot * kDwParts * 64 + o % 64;
            for (int g = 0; g < kDwParts; ++g) acc += q[(size_t)g * cout_t];
            gb[o] = acc;
        }
    }
}

// packed[i] = bf16(src[idx[i]]) (0 where idx[i] < 0): weights re-packed from
// the FP32 parameters through a layout's index table
__global__ void k_gather_bf16(const float* __restrict__ src, const int* __restrict__ idx, size_t n,
                              __nv_bfloat16* __restrict__ packed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = idx[i];
        packed[i] = __float2bfloat16_rn(k >= 0 ? src[k] : 0.0f);
    }
}
__global__ void k_gather_f32(const float* __restrict__ src, const int* __restrict__ idx, size_t n,
                             float* __restrict__ out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = idx[i];
        out[i] = k >= 0 ? src[k] : 0.0f;
    }
}

// ---- training (BF16): elementwise steps ------------------------------------
// out[i] = act[i] > 0 ? d[i] : 0 (out may be d)
__global__ void k_mask_copy_bf16(const __nv_bfloat16* d, const __nv_bfloat16* __restrict__ act,
                                 size_t n, __nv_bfloat16* out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(act[i]) > 0.0f ? d[i] : __float2bfloat16_rn(0.0f);
}

// out = a + b (+ c) (+ e), summed in FP32 and rounded once; when act is given,
// out = act > 0 ? that : 0
__global__ void k_sum_bf16(__nv_bfloat16* out, const __nv_bfloat16* a, const __nv_bfloat16* b,
                           const __nv_bfloat16* c, const __nv_bfloat16* e,
                           const __nv_bfloat16* __restrict__ act, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float v = __bfloat162float(a[i]) + __bfloat162float(b[i]);
        if (c) v += __bfloat162float(c[i]);
        if (e) v += __bfloat162float(e[i]);
        if (act && !(__bfloat162float(act[i]) > 0.0f)) v = 0.0f;
        out[i] = __float2bfloat16_rn(v);
    }
}

// bf16 [P][64] rows from FP32 [P][cin] (channels past cin zero)
__global__ void k_f32_to_bf16_rows(const float* __restrict__ x, size_t P, int cin,
                                   __nv_bfloat16* __restrict__ o)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / 64;
        const int c = (int)(i % 64);
        o[i] = __float2bfloat16_rn(c < cin ? x[p * cin + c] : 0.0f);
    }
}

// One tensor-core weight-gradient tile (part [G][9][cout_t][cin_t], dbpart
// [G][cout_t]) summed over its G partials into a layer's gradient
// [cout][KK][cin] (KK = 9, or 1 for a 1x1 layer: tap 4 of the tile):
// tile output o' is layer output o_mul o' + o_add, tile input c' is layer input
// c0 + c', or, for chunk q >= 1 of the fuse conv, 64 + dsf_channel(c', oy, ox, D)
// with q - 1 = oy s + ox.  The bias is written when with_bias.  A block takes
// 32 consecutive values; warp w sums partials w, w + 8, ... (one coalesced
// 128-byte row per partial), the eight sums are added in warp order: a fixed
// order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_wg_reduce(const float* __restrict__ part,
                                                   const float* __restrict__ dbpart, int G, int cin_t,
                                                   int cout_t, int KK, int CIN, int o_mul, int o_add,
                                                   int c0, int q, int s, int D, int with_bias,
                                                   float* __restrict__ gw, float* __restrict__ gb)
{
    __shared__ float red[8][32];
    const size_t nw = (size_t)cout_t * KK * cin_t, ntot = nw + (with_bias ? cout_t : 0);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const size_t gstride = (size_t)9 * cout_t * cin_t;
    for (size_t e0 = (size_t)blockIdx.x * 32; e0 < ntot; e0 += (size_t)gridDim.x * 32) {
        const size_t e = e0 + lane;
        float acc = 0.0f;
        if (e < nw) {
            const int c = (int)(e % cin_t), tl = (int)((e / cin_t) % KK), o = (int)(e / ((size_t)cin_t * KK));
            const float* src = part + ((size_t)(KK == 9 ? tl : 4) * cout_t + o) * cin_t + c;
            for (int g = wp; g < G; g += 8) acc += src[(size_t)g * gstride];
        } else if (e < ntot) {
            const int o = (int)(e - nw);
            for (int g = wp; g < G; g += 8) acc += dbpart[(size_t)g * cout_t + o];
        }
        red[wp][lane] = acc;
        __syncthreads();
        if (wp == 0 && e < ntot) {
            float v = red[0][lane];
            for (int k = 1; k < 8; ++k) v += red[k][lane];
            if (e < nw) {
                const int c = (int)(e % cin_t), tl = (int)((e / cin_t) % KK), o = (int)(e / ((size_t)cin_t * KK));
                const int ci = q > 0 ? 64 + dsf_channel(c, (q - 1) / s, (q - 1) % s, D) : c0 + c;
                gw[((size_t)(o_mul * o + o_add) * KK + tl) * CIN + ci] = v;
            } else {
                gb[o_mul * (int)(e - nw) + o_add] = v;
            }
        }
        __syncthreads();
    }
}

inline int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    return (int)(g < 8192 ? (g ? g : 1) : 8192);
}

struct WChunk {
    size_t off;          // bf16 elements into wbf ([9][nout][64])
    int nout;            // 64 or 16
    CUtensorMap map;
};

// what a recorded BF16 training step depends on besides the handle's weights
struct TrainKey {
    int N = -1, H = -1, W = -1, kind = -1;
    float beta = 0.0f;
    void* buf = nullptr;
    bool operator==(const TrainKey& o) const
    {
        return N == o.N && H == o.H && W == o.W && kind == o.kind && beta == o.beta && buf == o.buf;
    }
};

}  // namespace
}  // namespace mrs

using namespace mrs;

struct mrs_rdn_s {
    int s = 0, D = 0, c_hr = 0;
    size_t np = 0;
    std::vector<RLayer> L;
    float* master = nullptr;       // FP32 parameters (oracle layout)
    float* w_fuse3 = nullptr;      // fuse weights as 3x3 centre taps (FP32 path)
    __nv_bfloat16* wbf = nullptr;  // packed BF16 chunks
    float* bch = nullptr;          // chunk biases [nchunks][64]
    std::vector<WChunk> ch;
    std::vector<int> first;        // first chunk of each layer
    std::vector<int> widx, bidx;   // packing index tables (parameter of each packed value, -1: 0)
    int* d_widx = nullptr;         // ... on the device (uploaded by the first BF16 training step)
    int* d_bidx = nullptr;
    // transposed chunks of the BF16 training step's input gradients: layer li's
    // chunk j at rows tfirst[li] + 9 * 64 * j of wmapT_all (-1: none)
    std::vector<int> tidx, tfirst;
    int* d_tidx = nullptr;
    __nv_bfloat16* wbfT = nullptr;
    CUtensorMap wmapT_all;
    Buf trb;                       // BF16 training workspace
    cudaGraphExec_t tgraph = nullptr;   // its launches for one shape (see rdn_train_bf16)
    mrs::TrainKey tkey;
    uint64_t tgraph_kernels = 0;
    cudaStream_t tcap = nullptr;        // stream they are recorded on
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // weight-gradient tiles side by side
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    Buf tdmaps;                    // its multi-chunk A-operand maps on the device
    CUtensorMap wmap_all;          // every chunk's weights as one [rows][64] tensor
    std::vector<CUtensorMap> hmaps;  // A-operand maps of the multi-chunk convs of a call
    Buf dmaps;                     // their device copy
    Buf f32, bf;                   // activation workspaces
    int* err = nullptr;
    // training state (allocated by the first training step)
    float* grad = nullptr;         // gradient of the last step (parameter layout)
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t step = 0;              // Adam steps taken
    bool bf_stale = false;         // BF16 chunks older than the FP32 weights
    Buf tr;                        // training workspace (tape + backward)
};

namespace mrs {
namespace {

// BF16 chunks of every layer, [tap][o][c] (o < nout, c < 64) for conv_tc,
// with per-chunk biases (the layer bias on the chunk that starts a chain, zero
// elsewhere).  The layout is an index table built once on the host: for each
// packed weight and bias, the parameter it holds (or -1: zero).  mrs_rdn_create
// packs through it on the host; a training step re-packs the updated FP32
// weights through the same table on the device (k_gather_bf16), into the same
// buffers, so the tensor maps stay valid.
void build_pack_index(mrs_rdn_s* r)
{
    std::vector<int>& wi = r->widx;
    std::vector<int>& bi = r->bidx;
    wi.clear();
    bi.clear();
    r->ch.clear();
    r->first.clear();
    auto chunk = [&](int nout, auto wfun, auto bfun) {
        WChunk c;
        c.off = wi.size();
        c.nout = nout;
        for (int t = 0; t < 9; ++t)
            for (int o = 0; o < nout; ++o)
                for (int k = 0; k < 64; ++k) wi.push_back(wfun(t, o, k));
        for (int o = 0; o < 64; ++o) bi.push_back(o < nout ? bfun(o) : -1);
        r->ch.push_back(c);
    };
    const int D = r->D, s = r->s;
    for (size_t li = 0; li < r->L.size(); ++li) {
        const RLayer& l = r->L[li];
        r->first.push_back((int)r->ch.size());
        const int w = (int)l.woff, b = (int)l.boff;
        const bool is_up = li + 1 < r->L.size() && l.cout == 4 * kF;
        if (li == 2) {
            // fuse: chunk 0 = F_LRHS channels, chunk 1 + oy s + ox = HR sub-pixel (oy, ox)
            for (int q = 0; q <= s * s; ++q) {
                int oy = q ? (q - 1) / s : 0, ox = q ? (q - 1) % s : 0;
                chunk(64, [&](int t, int o, int k) -> int {
                    if (t != 4) return -1;
                    int ci = q == 0 ? k : 64 + dsf_channel(k, oy, ox, D);
                    return w + o * l.cin + ci;
                }, [&](int o) -> int { return q == 0 ? b + o : -1; });
            }
        } else if (is_up) {
            // upsampling conv: chunk q = 2 dy + dx computes output channels 4c + q
            for (int q = 0; q < 4; ++q)
                chunk(64, [&](int t, int o, int k) -> int {
                    return w + ((4 * o + q) * 9 + t) * l.cin + k;
                }, [&](int o) -> int { return b + 4 * o + q; });
        } else {
            const int nout = l.cout > 16 ? 64 : 16;
            const int nch = (l.cin + 63) / 64;
            for (int j = 0; j < nch; ++j)
                chunk(nout, [&](int t, int o, int k) -> int {
                    int ci = 64 * j + k;
                    return (o < l.cout && ci < l.cin) ? w + (o * 9 + t) * l.cin + ci : -1;
                }, [&](int o) -> int { return (j == 0 && o < l.cout) ? b + o : -1; });
        }
    }
}

mrs_status pack_chunks(mrs_rdn_s* r, const float* P)
{
    build_pack_index(r);
    std::vector<__nv_bfloat16> wb(r->widx.size());
    std::vector<float> bb(r->bidx.size());
    for (size_t i = 0; i < wb.size(); ++i)
        wb[i] = __float2bfloat16_rn(r->widx[i] >= 0 ? P[r->widx[i]] : 0.0f);
    for (size_t i = 0; i < bb.size(); ++i) bb[i] = r->bidx[i] >= 0 ? P[r->bidx[i]] : 0.0f;
    if (r->wbf) cudaFree(r->wbf);
    if (r->bch) cudaFree(r->bch);
    r->wbf = nullptr;
    r->bch = nullptr;
    MRS_CHECK(cudaMalloc(&r->wbf, wb.size() * sizeof(__nv_bfloat16)));
    MRS_CHECK(cudaMalloc(&r->bch, bb.size() * sizeof(float)));
    MRS_CHECK(cudaMemcpy(r->wbf, wb.data(), wb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
    MRS_CHECK(cudaMemcpy(r->bch, bb.data(), bb.size() * sizeof(float), cudaMemcpyHostToDevice));
    for (auto& c : r->ch) {
        mrs_status st = tc_make_w_map(&c.map, r->wbf + c.off, 9 * c.nout, c.nout, TC_BF16);
        if (st != MRS_OK) return st;
    }
    // chunk c of a 64-output layer starts at row c.off / 64 of this map
    return tc_make_w_map(&r->wmap_all, r->wbf, (int)(wb.size() / 64), 64, TC_BF16);
}

mrs_status rdn_f32(mrs_rdn_s* r, const float* lrhs, const float* hrls, const float* alb,
                   const float* nrm, const float* extra, int N, int H, int W, float* out,
                   cudaStream_t st)
{
    const int s = r->s, D = r->D, h = H / s, w = W / s;
    const size_t Pl = (size_t)N * h * w, Ph = (size_t)N * H * W;
    const int Ccat = kF + kF * s * s;
    // workspace: inH | cat | Fh0 | A | B | F0 | Pg | T | U  (floats)
    const size_t nT = Ph / 4 * 256, nU = Ph * 64;
    const size_t need = (Ph * r->c_hr + Pl * Ccat + Ph * 64 + 2 * Pl * 256 + 2 * Pl * 64 + nT + nU) * 4;
    mrs_status rc = r->f32.ensure(need);
    if (rc != MRS_OK) return rc;
    float* inH = r->f32.as<float>();
    float* cat = inH + Ph * r->c_hr;
    float* Fh0 = cat + Pl * Ccat;
    float* A = Fh0 + Ph * 64;
    float* B = A + Pl * 256;
    float* F0 = B + Pl * 256;
    float* Pg = F0 + Pl * 64;
    float* T = Pg + Pl * 64;
    float* U = T + nT;
    const float* M = r->master;
    const auto& L = r->L;

    k_hr_input_f32<<<grid_for(Ph), 256, 0, st>>>(hrls, alb, nrm, extra, Ph, inH);
    MRS_LAUNCHED(1);
    // F_LRHS into cat[:, 0:64]; F0_HRLS; deshuffle into cat[:, 64:]
    rc = simt_conv3x3(lrhs, 3, 3, M + L[0].woff, M + L[0].boff, kF, SIMT_PLAIN, 1, nullptr, 0, cat,
                      Ccat, nullptr, N, h, w, 1, st);
    if (rc == MRS_OK)
        rc = simt_conv3x3(inH, r->c_hr, r->c_hr, M + L[1].woff, M + L[1].boff, kF, SIMT_PLAIN, 1,
                          nullptr, 0, Fh0, kF, nullptr, N, H, W, 1, st);
    if (rc != MRS_OK) return rc;
    k_deshuffle_f32<<<grid_for(Ph * 64), 256, 0, st>>>(Fh0, N, H, W, s, D, cat, Ccat);
    MRS_LAUNCHED(1);
    k_centre_tap<<<grid_for((size_t)64 * 9 * Ccat), 256, 0, st>>>(M + L[2].woff, Ccat, r->w_fuse3);
    MRS_LAUNCHED(1);
    // F_0 = relu(fuse(cat)) into A[:, 0:64] and F0
    rc = simt_conv3x3(cat, Ccat, Ccat, r->w_fuse3, M + L[2].boff, kF, SIMT_PLAIN, 1, nullptr, 0, A,
                      256, nullptr, N, h, w, 1, st);
    if (rc != MRS_OK) return rc;
    k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(F0, 64, A, 256, Pl, 0);
    MRS_LAUNCHED(1);
    int li = 3;
    for (int g = 0; g < kRDG && rc == MRS_OK; ++g) {
        k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(Pg, 64, A, 256, Pl, 0);
        MRS_LAUNCHED(1);
        for (int b = 0; b < kRDB && rc == MRS_OK; ++b) {
            for (int c = 1; c < kConv && rc == MRS_OK; ++c, ++li)
                rc = simt_conv3x3(A, kF * c, 256, M + L[li].woff, M + L[li].boff, kF, SIMT_PLAIN, 1,
                                  nullptr, 0, A + kF * c, 256, nullptr, N, h, w, 1, st);
            if (rc != MRS_OK) break;
            rc = simt_conv3x3(A, 256, 256, M + L[li].woff, M + L[li].boff, kF, SIMT_RESRELU, 0, A,
                              256, B, 256, nullptr, N, h, w, 1, st);
            ++li;
            float* t = A;
            A = B;
            B = t;
        }
        k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(A, 256, Pg, 64, Pl, 1);
        MRS_LAUNCHED(1);
    }
    if (rc != MRS_OK) return rc;
    k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(A, 256, F0, 64, Pl, 1);
    MRS_LAUNCHED(1);
    // UP: D x (conv 64 -> 256 + ReLU, shuffle); U alternates between U and Fh0
    const float* cur = A;
    int cs = 256, ch = h, cw = w;
    float* dst = U;
    for (int d = 0; d < D && rc == MRS_OK; ++d, ++li) {
        rc = simt_conv3x3(cur, kF, cs, M + L[li].woff, M + L[li].boff, 4 * kF, SIMT_PLAIN, 1,
                          nullptr, 0, T, 256, nullptr, N, ch, cw, 1, st);
        if (rc != MRS_OK) break;
        k_shuffle_f32<<<grid_for((size_t)N * 4 * ch * cw * 64), 256, 0, st>>>(T, 256, N, ch, cw, dst);
        MRS_LAUNCHED(1);
        cur = dst;
        cs = kF;
        ch *= 2;
        cw *= 2;
        dst = dst == U ? Fh0 : U;
    }
    if (rc != MRS_OK) return rc;
    rc = simt_conv3x3(cur, kF, kF, M + L[li].woff, M + L[li].boff, 3, SIMT_PLAIN, 0, nullptr, 0, out,
                      3, nullptr, N, H, W, 1, st);
    if (rc != MRS_OK) return rc;
    return cuda_status(cudaGetLastError(), "rdn fp32");
}

mrs_status rdn_bf16(mrs_rdn_s* r, const float* lrhs, const float* hrls, const float* alb,
                    const float* nrm, const float* extra, int N, int H, int W, float* out,
                    cudaStream_t st)
{
    const int s = r->s, D = r->D, h = H / s, w = W / s;
    const size_t Pl = (size_t)N * h * w, Ph = (size_t)N * H * W;
    // bf16 workspace: inL | inH | Flr | Fh0 | F0 | X[0..5] | U (sum of 4^d Pl, d = 1..D)
    size_t nU = 0;
    for (int d = 1; d <= D; ++d) nU += Pl << (2 * d);
    const int kX = 6;
    const size_t elems = (Pl + Ph + Pl + Ph + Pl + kX * Pl + nU) * 64;
    const size_t need = elems * 2 + 4096;
    mrs_status rc = r->bf.ensure(need);
    if (rc != MRS_OK) return rc;
    __nv_bfloat16* inL = r->bf.as<__nv_bfloat16>();
    __nv_bfloat16* inH = inL + Pl * 64;
    __nv_bfloat16* Flr = inH + Ph * 64;
    __nv_bfloat16* Fh0 = Flr + Pl * 64;
    __nv_bfloat16* F0 = Fh0 + Ph * 64;
    __nv_bfloat16* X[kX];
    X[0] = F0 + Pl * 64;
    for (int i = 1; i < kX; ++i) X[i] = X[i - 1] + Pl * 64;
    __nv_bfloat16* Ud[4];
    Ud[0] = nullptr;
    __nv_bfloat16* u = X[kX - 1] + Pl * 64;
    for (int d = 1; d <= D; ++d) { Ud[d] = u; u += (Pl << (2 * d)) * 64; }

    k_lr_input_bf16<<<grid_for(Pl), 256, 0, st>>>(lrhs, Pl, inL);
    MRS_LAUNCHED(1);
    k_hr_input_bf16<<<grid_for(Ph), 256, 0, st>>>(hrls, alb, nrm, extra, Ph, inH);
    MRS_LAUNCHED(1);
    if ((rc = cuda_status(cudaGetLastError(), "rdn input")) != MRS_OK) return rc;

    // tensor maps: A operands and outputs / residuals, with the box widths of
    // the BF16 tensor-core conv
    auto amap = [&](CUtensorMap* m, const void* p, int n, int hh, int ww) {
        return tc_make_act_map(m, p, n, hh, ww, TC_BF16, tc_a_box(TC_BF16));
    };
    auto omap = [&](CUtensorMap* m, const void* p, int n, int hh, int ww) {
        return tc_make_act_map(m, p, n, hh, ww, TC_BF16, tc_out_box(TC_BF16));
    };
    CUtensorMap inLA, inHA, FlrA, FlrO, Fh0O, F0A, F0O, XA[kX], XO[kX];
    if ((rc = amap(&inLA, inL, N, h, w)) != MRS_OK) return rc;
    if ((rc = amap(&inHA, inH, N, H, W)) != MRS_OK) return rc;
    if ((rc = amap(&FlrA, Flr, N, h, w)) != MRS_OK) return rc;
    if ((rc = omap(&FlrO, Flr, N, h, w)) != MRS_OK) return rc;
    if ((rc = omap(&Fh0O, Fh0, N, H, W)) != MRS_OK) return rc;
    if ((rc = amap(&F0A, F0, N, h, w)) != MRS_OK) return rc;
    if ((rc = omap(&F0O, F0, N, h, w)) != MRS_OK) return rc;
    for (int i = 0; i < kX; ++i) {
        if ((rc = amap(&XA[i], X[i], N, h, w)) != MRS_OK) return rc;
        if ((rc = omap(&XO[i], X[i], N, h, w)) != MRS_OK) return rc;
    }
    // deshuffle chunks: sub-pixel (oy, ox) of every s x s block of Fh0
    std::vector<CUtensorMap> dsf(s * s);
    for (int q = 0; q < s * s && rc == MRS_OK; ++q) {
        int oy = q / s, ox = q % s;
        rc = tc_make_view_map(&dsf[q], Fh0 + ((size_t)oy * W + ox) * 64, N, h, w, (long long)s * 128,
                              (long long)s * W * 128, (long long)H * W * 128, tc_a_box(TC_BF16));
    }
    if (rc != MRS_OK) return rc;

    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.scale = 1; a.operand = TC_BF16; a.err = r->err; a.nout = 64; a.cout = 64;
    // The launch sequence runs twice: a dry pass collects the A-operand maps
    // of the multi-chunk convs (a conv over 64 c input channels is ONE launch
    // accumulating its c chunks in TMEM; the kernel reads the chunk maps from
    // device memory), they are copied to the device, then the real pass
    // launches.
    bool dry = true;
    size_t mc = 0;                 // next multi-chunk conv's first map
    auto layer = [&](int li, const CUtensorMap* const* A, int n, int hh, int ww, int mode,
                     const CUtensorMap* o, const CUtensorMap* res) -> mrs_status {
        if (n > 1) {
            if (dry) {
                for (int j = 0; j < n; ++j) r->hmaps.push_back(*A[j]);
                return MRS_OK;
            }
            const WChunk& c0 = r->ch[r->first[li]];
            a.H = hh; a.W = ww;
            a.tmap_x = A[0];
            a.amaps = r->dmaps.as<CUtensorMap>() + mc;
            a.kc = n;
            a.w_row0 = (int)(c0.off / 64);
            a.tmap_w = &r->wmap_all;
            a.bias = r->bch + (size_t)r->first[li] * 64;
            a.nout = 64; a.relu = 0;
            a.mode = mode; a.tmap_out = o; a.tmap_res = res;
            mc += n;
            mrs_status e = tc_conv3x3(a, st);
            a.amaps = nullptr; a.kc = 0; a.w_row0 = 0;
            return e;
        }
        if (dry) return MRS_OK;
        const WChunk& c = r->ch[r->first[li]];
        a.H = hh; a.W = ww;
        a.tmap_x = A[0];
        a.tmap_w = &c.map;
        a.bias = r->bch + (size_t)r->first[li] * 64;
        a.nout = c.nout;
        a.relu = 0;
        a.mode = mode; a.tmap_out = o; a.tmap_res = res;
        return tc_conv3x3(a, st);
    };

    auto run = [&]() -> mrs_status {
    mrs_status rc = MRS_OK;
    // encoders
    const CUtensorMap* one[1];
    one[0] = &inLA;
    if ((rc = layer(0, one, 1, h, w, TC_RELU_BF16, &FlrO, nullptr)) != MRS_OK) return rc;
    one[0] = &inHA;
    if ((rc = layer(1, one, 1, H, W, TC_RELU_BF16, &Fh0O, nullptr)) != MRS_OK) return rc;
    // fuse: F_LRHS chunk + s^2 deshuffle views, one launch
    std::vector<const CUtensorMap*> fin(1 + s * s);
    fin[0] = &FlrA;
    for (int q = 0; q < s * s; ++q) fin[1 + q] = &dsf[q];
    if ((rc = layer(2, fin.data(), 1 + s * s, h, w, TC_RELU_BF16, &F0O, nullptr)) != MRS_OK) return rc;

    // residual dense groups.  Buffers: F0 stays; X[0..2] rotate as block
    // inputs / outputs, X[3..5] hold the dense features F_1..F_3
    int li = 3;
    int pg = -1;          // index into X of the group input (-1 = F0)
    int cur = -1;         // block input
    for (int g = 0; g < kRDG; ++g) {
        pg = cur;
        for (int b = 0; b < kRDB; ++b) {
            const CUtensorMap* inA = cur < 0 ? &F0A : &XA[cur];
            const CUtensorMap* inO = cur < 0 ? &F0O : &XO[cur];
            int outi = 0;
            while (outi == cur || outi == pg) ++outi;
            const CUtensorMap* ins[4] = {inA, &XA[3], &XA[4], &XA[5]};
            for (int c = 1; c < kConv; ++c, ++li)
                if ((rc = layer(li, ins, c, h, w, TC_RELU_BF16, &XO[2 + c], nullptr)) != MRS_OK) return rc;
            if ((rc = layer(li, ins, kConv, h, w, TC_RESRELU_BF16, &XO[outi], inO)) != MRS_OK) return rc;
            ++li;
            cur = outi;
        }
        // group skip: F_g = blocks + F_{g-1}
        if (!dry) {
            k_add_bf16<<<grid_for(Pl * 8), 256, 0, st>>>(X[cur], pg < 0 ? F0 : X[pg], Pl * 8);
            MRS_LAUNCHED(1);
        }
    }
    if (dry) return MRS_OK;
    // Eq. F_DF: + F_0
    k_add_bf16<<<grid_for(Pl * 8), 256, 0, st>>>(X[cur], F0, Pl * 8);
    MRS_LAUNCHED(1);
    if ((rc = cuda_status(cudaGetLastError(), "rdn add")) != MRS_OK) return rc;
    // UP: stage d reads U_d (U_0 = F_DF) and writes the four sub-pixel views of U_{d+1}
    CUtensorMap UA;
    const CUtensorMap* src = &XA[cur];
    int ch = h, cw = w;
    for (int d = 0; d < D; ++d, ++li) {
        __nv_bfloat16* nx = Ud[d + 1];
        for (int q = 0; q < 4; ++q) {
            int dy = q >> 1, dx = q & 1;
            CUtensorMap vo;
            rc = tc_make_view_map(&vo, nx + ((size_t)dy * 2 * cw + dx) * 64, N, ch, cw, 256,
                                  (long long)4 * cw * 128, (long long)4 * ch * cw * 128,
                                  tc_out_box(TC_BF16));
            if (rc != MRS_OK) return rc;
            a.H = ch; a.W = cw;
            const WChunk& c = r->ch[r->first[li] + q];
            a.tmap_x = src; a.tmap_w = &c.map; a.bias = r->bch + (size_t)(r->first[li] + q) * 64;
            a.nout = 64; a.tmap_res = nullptr; a.tmap_out = &vo;
            a.mode = TC_RELU_BF16; a.relu = 0;
            if ((rc = tc_conv3x3(a, st)) != MRS_OK) return rc;
        }
        ch *= 2;
        cw *= 2;
        if ((rc = amap(&UA, nx, N, ch, cw)) != MRS_OK) return rc;
        src = &UA;
    }
    // H_Rec: 64 -> 3, no ReLU, FP32 out
    const WChunk& c = r->ch[r->first[li]];
    a.H = H; a.W = W; a.tmap_x = src; a.tmap_w = &c.map; a.bias = r->bch + (size_t)r->first[li] * 64;
    a.nout = c.nout; a.tmap_out = nullptr; a.tmap_res = nullptr;
    a.mode = TC_PLAIN_F32; a.out = out; a.cout = 3; a.relu = 0;
    return tc_conv3x3(a, st);
    };

    r->hmaps.clear();
    if ((rc = run()) != MRS_OK) return rc;
    if ((rc = r->dmaps.ensure(r->hmaps.size() * sizeof(CUtensorMap) + 64)) != MRS_OK) return rc;
    MRS_CHECK(cudaMemcpyAsync(r->dmaps.p, r->hmaps.data(), r->hmaps.size() * sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice, st));
    dry = false;
    return run();
}


// ---- training step (FP32) ----------------------------------------------------
constexpr float kTrainClip = 100.0f;   // firefly clipping of the training target (Sec. 3.2)

// gradient of one layer: partial sums over 64 x 64 channel tiles, then the
// fixed-order reduction into grad (parameter layout)
mrs_status layer_grad(mrs_rdn_s* r, int li, const float* x, int xs, const float* dz, int zs, int N,
                      int H, int W, float* part, float* dbpart, cudaStream_t st)
{
    const RLayer& l = r->L[li];
    mrs_status rc = dw_tiles_f32(x, l.cin, xs, dz, l.cout, zs, N, H, W, l.k == 1, part, dbpart, st);
    if (rc != MRS_OK) return rc;
    const size_t n = (size_t)l.cout * l.k * l.k * l.cin + l.cout;
    k_dw_reduce_tiles<<<grid_for(n), 256, 0, st>>>(part, dbpart, l.k * l.k, l.cin, l.cout,
                                                   r->grad + l.woff, r->grad + l.boff);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "rdn layer grad");
}

// forward keeping the activations the backward reads (the same arithmetic, in
// the same order, as rdn_f32), the loss, the backward of every step in
// reverse, one Adam update
mrs_status rdn_train_f32(mrs_rdn_s* r, const float* lrhs, const float* hrls, const float* alb,
                         const float* nrm, const float* extra, const float* tgt, int N, int H, int W,
                         int kind, float beta, float lr, float* yout, double* loss_out,
                         cudaStream_t st)
{
    const int s = r->s, D = r->D, h = H / s, w = W / s, c_hr = r->c_hr;
    const int Ccat = kF + kF * s * s, nblk = kRDG * kRDB;
    const size_t Pl = (size_t)N * h * w, Ph = (size_t)N * H * W;
    size_t Pd[4];
    Pd[0] = Pl;
    for (int d = 0; d < D; ++d) Pd[d + 1] = Pd[d] * 4;
    size_t nT = 0, nU = 0;
    for (int d = 0; d < D; ++d) nT += Pd[d] * 256;
    for (int d = 0; d <= D; ++d) nU += Pd[d] * 64;
    const size_t nwt = (size_t)(Ccat > 256 ? Ccat : 256) * 9 * 64;
    const size_t npart = (size_t)kDwParts * 4096 * (Ccat / 64 > 36 ? Ccat / 64 : 36);
    // floats: inH cat Fh0 F0 blk R T U y | dy dA dB dCat dz dSkip dxf wt zero part dbpart
    const size_t nf = Ph * c_hr + Pl * Ccat + Ph * 64 + Pl * 64 + nblk * Pl * 256 + nblk * Pl * 64 +
                      nT + nU + Ph * 3 + Ph * 3 + 2 * Ph * 64 + Pl * 256 + 2 * Pl * 64 + Pl * Ccat +
                      nwt + Ccat + npart + 4 * kDwParts * 64;
    mrs_status rc = r->tr.ensure(nf * 4 + (kLossParts + 2) * 8 + 256);
    if (rc != MRS_OK) return rc;
    double* lparts = r->tr.as<double>();
    double* lsum = lparts + kLossParts;
    float* inH = (float*)(lsum + 2);
    float* cat = inH + Ph * c_hr;
    float* Fh0 = cat + Pl * Ccat;
    float* F0 = Fh0 + Ph * 64;
    float* blk = F0 + Pl * 64;
    float* R = blk + nblk * Pl * 256;
    float* Tb = R + nblk * Pl * 64;
    float* Ub = Tb + nT;
    float* y = Ub + nU;
    float* dy = y + Ph * 3;
    float* dA = dy + Ph * 3;
    float* dB = dA + Ph * 64;
    float* dCat = dB + Ph * 64;
    float* dz = dCat + Pl * 256;
    float* dSkip = dz + Pl * 64;
    float* dxf = dSkip + Pl * 64;
    float* wt = dxf + Pl * Ccat;
    float* zero = wt + nwt;
    float* part = zero + Ccat;
    float* dbpart = part + npart;
    float* T[3];
    float* U[4];
    {
        float* t = Tb;
        for (int d = 0; d < D; ++d) { T[d] = t; t += Pd[d] * 256; }
        float* u = Ub;
        for (int d = 0; d <= D; ++d) { U[d] = u; u += Pd[d] * 64; }
    }
    auto X = [&](int k) { return blk + (size_t)k * Pl * 256; };
    auto Rk = [&](int k) { return R + (size_t)k * Pl * 64; };
    const float* M = r->master;
    const auto& L = r->L;
    MRS_CHECK(cudaMemsetAsync(zero, 0, (size_t)Ccat * 4, st));

    // ---- forward with the tape
    k_hr_input_f32<<<grid_for(Ph), 256, 0, st>>>(hrls, alb, nrm, extra, Ph, inH);
    MRS_LAUNCHED(1);
    rc = simt_conv3x3(lrhs, 3, 3, M + L[0].woff, M + L[0].boff, kF, SIMT_PLAIN, 1, nullptr, 0, cat,
                      Ccat, nullptr, N, h, w, 1, st);
    if (rc == MRS_OK)
        rc = simt_conv3x3(inH, c_hr, c_hr, M + L[1].woff, M + L[1].boff, kF, SIMT_PLAIN, 1, nullptr,
                          0, Fh0, kF, nullptr, N, H, W, 1, st);
    if (rc != MRS_OK) return rc;
    k_deshuffle_f32<<<grid_for(Ph * 64), 256, 0, st>>>(Fh0, N, H, W, s, D, cat, Ccat);
    MRS_LAUNCHED(1);
    k_centre_tap<<<grid_for((size_t)64 * 9 * Ccat), 256, 0, st>>>(M + L[2].woff, Ccat, r->w_fuse3);
    MRS_LAUNCHED(1);
    rc = simt_conv3x3(cat, Ccat, Ccat, r->w_fuse3, M + L[2].boff, kF, SIMT_PLAIN, 1, nullptr, 0, F0,
                      kF, nullptr, N, h, w, 1, st);
    if (rc != MRS_OK) return rc;
    k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(X(0), 256, F0, 64, Pl, 0);
    MRS_LAUNCHED(1);
    int li = 3;
    for (int g = 0; g < kRDG; ++g) {
        const float* Fprev = X(kRDB * g);
        for (int b = 0; b < kRDB; ++b) {
            const int k = kRDB * g + b;
            float* x = X(k);
            for (int c = 1; c < kConv && rc == MRS_OK; ++c, ++li)
                rc = simt_conv3x3(x, kF * c, 256, M + L[li].woff, M + L[li].boff, kF, SIMT_PLAIN, 1,
                                  nullptr, 0, x + kF * c, 256, nullptr, N, h, w, 1, st);
            if (rc == MRS_OK)
                rc = simt_conv3x3(x, 256, 256, M + L[li].woff, M + L[li].boff, kF, SIMT_PLAIN, 1,
                                  nullptr, 0, Rk(k), 64, nullptr, N, h, w, 1, st);
            if (rc != MRS_OK) return rc;
            ++li;
            // block output F_in + relu(z4); after a group's last block + F_{g-1};
            // after the last group + F_0 (Eq. F_DF)
            const bool last = b == kRDB - 1;
            float* dst = k + 1 < nblk ? X(k + 1) : U[0];
            k_sum64<<<grid_for(Pl * 64), 256, 0, st>>>(dst, k + 1 < nblk ? 256 : 64, x, 256, Rk(k), 64,
                                                      last ? Fprev : nullptr, 256,
                                                      k + 1 == nblk ? F0 : nullptr, 64, Pl);
            MRS_LAUNCHED(1);
        }
    }
    int ch = h, cw = w;
    for (int d = 0; d < D; ++d, ++li) {
        rc = simt_conv3x3(U[d], kF, kF, M + L[li].woff, M + L[li].boff, 4 * kF, SIMT_PLAIN, 1, nullptr,
                          0, T[d], 256, nullptr, N, ch, cw, 1, st);
        if (rc != MRS_OK) return rc;
        k_shuffle_f32<<<grid_for(Pd[d + 1] * 64), 256, 0, st>>>(T[d], 256, N, ch, cw, U[d + 1]);
        MRS_LAUNCHED(1);
        ch *= 2;
        cw *= 2;
    }
    rc = simt_conv3x3(U[D], kF, kF, M + L[li].woff, M + L[li].boff, 3, SIMT_PLAIN, 0, nullptr, 0, y, 3,
                      nullptr, N, H, W, 1, st);
    if (rc != MRS_OK) return rc;
    if (yout) MRS_CHECK(cudaMemcpyAsync(yout, y, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));

    // ---- loss and dL/dI_SR
    if ((rc = loss_grad_f32(y, tgt, Ph * 3, kTrainClip, kind, beta, dy, lparts, lsum, st)) != MRS_OK)
        return rc;

    // ---- backward: H_Rec, then the upsampling convs through the shuffles
    if ((rc = layer_grad(r, li, U[D], kF, dy, 3, N, H, W, part, dbpart, st)) != MRS_OK) return rc;
    wtrans_f32(M + L[li].woff, kF, 3, wt, st);
    rc = simt_conv3x3(dy, 3, 3, wt, zero, kF, SIMT_PLAIN, 0, nullptr, 0, dA, kF, nullptr, N, H, W, 1, st);
    if (rc != MRS_OK) return rc;
    for (int d = D - 1; d >= 0; --d) {
        --li;
        ch /= 2;
        cw /= 2;
        k_unshuffle_mask<<<grid_for(Pd[d] * 256), 256, 0, st>>>(dA, T[d], N, ch, cw, dB);
        MRS_LAUNCHED(1);
        if ((rc = layer_grad(r, li, U[d], kF, dB, 256, N, ch, cw, part, dbpart, st)) != MRS_OK) return rc;
        wtrans_f32(M + L[li].woff, kF, 4 * kF, wt, st);
        rc = simt_conv3x3(dB, 4 * kF, 4 * kF, wt, zero, kF, SIMT_PLAIN, 0, nullptr, 0, dA, kF, nullptr,
                          N, ch, cw, 1, st);
        if (rc != MRS_OK) return rc;
    }
    // dA = dF_DF: to F_G (the chain) and to F_0 (kept in dA)
    k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(dCat, 256, dA, 64, Pl, 0);
    MRS_LAUNCHED(1);
    // ---- residual dense groups in reverse; dCat [Pl][256] holds the current
    // block's concatenation gradient, channels 0..63 the gradient of its F_in
    for (int g = kRDG - 1; g >= 0; --g) {
        k_ch64_f32<<<grid_for(Pl * 64), 256, 0, st>>>(dSkip, 64, dCat, 256, Pl, 0);
        MRS_LAUNCHED(1);
        for (int b = kRDB - 1; b >= 0; --b) {
            const int k = kRDB * g + b, lb = 3 + kConv * k;
            const float* x = X(k);
            k_block_bwd_init<<<grid_for(Pl * 256), 256, 0, st>>>(dCat, Rk(k), dz, Pl);
            MRS_LAUNCHED(1);
            // local fusion: dCat[:, 0:256] += conv^T(dz)
            if ((rc = layer_grad(r, lb + 3, x, 256, dz, kF, N, h, w, part, dbpart, st)) != MRS_OK) return rc;
            wtrans_f32(M + L[lb + 3].woff, 256, kF, wt, st);
            rc = simt_conv3x3(dz, kF, kF, wt, zero, 256, SIMT_RESID, 0, dCat, 256, dCat, 256, nullptr, N,
                              h, w, 1, st);
            // dense conv c: its output's gradient (channels 64 (c + 1) ..) is
            // complete once the later convs have added theirs
            for (int c = kConv - 2; c >= 0 && rc == MRS_OK; --c) {
                float* dzc = dCat + kF * (c + 1);
                k_mask64<<<grid_for(Pl * 64), 256, 0, st>>>(dzc, 256, x + kF * (c + 1), 256, dzc, 256, Pl);
                MRS_LAUNCHED(1);
                const int ci = kF * (c + 1);
                if ((rc = layer_grad(r, lb + c, x, 256, dzc, 256, N, h, w, part, dbpart, st)) != MRS_OK)
                    return rc;
                wtrans_f32(M + L[lb + c].woff, ci, kF, wt, st);
                rc = simt_conv3x3(dzc, kF, 256, wt, zero, ci, SIMT_RESID, 0, dCat, 256, dCat, 256,
                                  nullptr, N, h, w, 1, st);
            }
            if (rc != MRS_OK) return rc;
        }
        // F_g = chain(F_{g-1}) + F_{g-1}
        k_sum64<<<grid_for(Pl * 64), 256, 0, st>>>(dCat, 256, dCat, 256, dSkip, 64, nullptr, 0, nullptr,
                                                  0, Pl);
        MRS_LAUNCHED(1);
    }
    // ---- fuse: dz = (dF_DF + chain gradient) masked by relu(F_0)
    k_sum64<<<grid_for(Pl * 64), 256, 0, st>>>(dz, 64, dA, 64, dCat, 256, nullptr, 0, nullptr, 0, Pl);
    MRS_LAUNCHED(1);
    k_mask64<<<grid_for(Pl * 64), 256, 0, st>>>(dz, 64, F0, 64, dz, 64, Pl);
    MRS_LAUNCHED(1);
    if ((rc = layer_grad(r, 2, cat, Ccat, dz, kF, N, h, w, part, dbpart, st)) != MRS_OK) return rc;
    wtrans_f32(r->w_fuse3, Ccat, kF, wt, st);
    rc = simt_conv3x3(dz, kF, kF, wt, zero, Ccat, SIMT_PLAIN, 0, nullptr, 0, dxf, Ccat, nullptr, N, h, w,
                      1, st);
    if (rc != MRS_OK) return rc;
    // ---- encoders: H_lrhs from channels 0..63, H_hrls through the deshuffles
    k_mask64<<<grid_for(Pl * 64), 256, 0, st>>>(dxf, Ccat, cat, Ccat, dz, 64, Pl);
    MRS_LAUNCHED(1);
    if ((rc = layer_grad(r, 0, lrhs, 3, dz, kF, N, h, w, part, dbpart, st)) != MRS_OK) return rc;
    k_dsf_grad_mask<<<grid_for(Ph * 64), 256, 0, st>>>(dxf, Ccat, Fh0, N, H, W, s, D, dB);
    MRS_LAUNCHED(1);
    if ((rc = layer_grad(r, 1, inH, c_hr, dB, kF, N, H, W, part, dbpart, st)) != MRS_OK) return rc;

    // ---- Adam on the FP32 weights
    r->step += 1;
    if ((rc = adam_f32(r->master, r->grad, r->adam_m, r->adam_v, r->np, lr, r->step, st)) != MRS_OK)
        return rc;
    r->bf_stale = true;
    if (loss_out) {
        double hsum = 0;
        MRS_CHECK(cudaMemcpyAsync(&hsum, lsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        *loss_out = hsum / (double)(Ph * 3);
    }
    return cuda_status(cudaGetLastError(), "rdn train step");
}

mrs_status ensure_train_state(mrs_rdn_s* r)
{
    if (r->grad) return MRS_OK;
    float* p[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i) {
        if (cudaMalloc(&p[i], r->np * 4) != cudaSuccess || cudaMemset(p[i], 0, r->np * 4) != cudaSuccess) {
            for (int j = 0; j <= i; ++j)
                if (p[j]) cudaFree(p[j]);
            cudaGetLastError();
            set_error("cudaMalloc(rdn training state) failed");
            return MRS_ERR_OOM;
        }
    }
    r->grad = p[0];
    r->adam_m = p[1];
    r->adam_v = p[2];
    r->step = 0;
    return MRS_OK;
}

// Transposed, tap-flipped chunks for the input gradients (dx = conv(dz, w^T)):
// [tap][c][o] = w[o][8 - tap][c] for a dgrad output channel c (a forward input
// channel) and a dgrad input channel o (a forward output channel), in 64 x 64
// chunks: one per 64 forward input channels (a dense conv's concatenation
// parts, the fuse conv's F_LRHS part and deshuffle views, centre tap only),
// one per sub-pixel view q for an upsampling conv (its dgrad sums the four
// views in one multi-chunk launch), one for H_Rec (forward outputs 3, the rest
// zero).  The encoders need none (their inputs are images).
void build_tpack_index(mrs_rdn_s* r)
{
    std::vector<int>& ti = r->tidx;
    ti.clear();
    r->tfirst.assign(r->L.size(), -1);
    auto tchunk = [&](auto f) {
        for (int t = 0; t < 9; ++t)
            for (int c = 0; c < 64; ++c)
                for (int o = 0; o < 64; ++o) ti.push_back(f(t, c, o));
    };
    const int D = r->D, s = r->s, nl = (int)r->L.size();
    for (int li = 2; li < nl; ++li) {
        const RLayer& l = r->L[li];
        const int w = (int)l.woff;
        r->tfirst[li] = (int)(ti.size() / 64);
        if (li == 2) {
            for (int q = 0; q <= s * s; ++q) {
                const int oy = q ? (q - 1) / s : 0, ox = q ? (q - 1) % s : 0;
                tchunk([&](int t, int c, int o) -> int {
                    if (t != 4) return -1;
                    const int ci = q == 0 ? c : 64 + dsf_channel(c, oy, ox, D);
                    return w + o * l.cin + ci;
                });
            }
        } else if (li == nl - 1) {
            tchunk([&](int t, int c, int o) -> int { return o < l.cout ? w + (o * 9 + (8 - t)) * l.cin + c : -1; });
        } else if (l.cout == 4 * kF) {
            for (int q = 0; q < 4; ++q)
                tchunk([&](int t, int c, int o) -> int { return w + ((4 * o + q) * 9 + (8 - t)) * l.cin + c; });
        } else {
            for (int j = 0; j < l.cin / 64; ++j)
                tchunk([&](int t, int c, int o) -> int { return w + (o * 9 + (8 - t)) * l.cin + 64 * j + c; });
        }
    }
}

// the BF16 chunks from the current FP32 weights (after training steps), on
// the device through the packing index tables (uploaded on first use)
mrs_status upload_index(const std::vector<int>& h, int** d)
{
    if (*d) return MRS_OK;
    MRS_CHECK(cudaMalloc(d, h.size() * sizeof(int) + 4));
    MRS_CHECK(cudaMemcpy(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice));
    return MRS_OK;
}

mrs_status repack_bf16(mrs_rdn_s* r, cudaStream_t st)
{
    mrs_status rc = upload_index(r->widx, &r->d_widx);
    if (rc == MRS_OK) rc = upload_index(r->bidx, &r->d_bidx);
    if (rc != MRS_OK) return rc;
    k_gather_bf16<<<grid_for(r->widx.size()), 256, 0, st>>>(r->master, r->d_widx, r->widx.size(), r->wbf);
    k_gather_f32<<<grid_for(r->bidx.size()), 256, 0, st>>>(r->master, r->d_bidx, r->bidx.size(), r->bch);
    MRS_LAUNCHED(2);
    r->bf_stale = false;
    return cuda_status(cudaGetLastError(), "rdn repack");
}

mrs_status repack_if_stale(mrs_rdn_s* r, cudaStream_t st)
{
    return r->bf_stale ? repack_bf16(r, st) : MRS_OK;
}

// ---- training step (BF16 tensor cores) ---------------------------------------
// The forward of rdn_bf16 with every tensor the backward reads kept apart
// (each block's input, F_1..F_3 and ReLU(local fusion); a block's output is
// its input + that ReLU output, summed in FP32 and rounded once, plus the
// group and Eq. F_DF skips), the loss on the FP32 I_SR, then the backward:
// input gradients as tensor-core convs with the transposed, tap-flipped chunk
// weights (ReLU masks as epilogues or elementwise passes, the dense parts'
// gradients accumulated in place by residual epilogues, the shuffle and
// deshuffle exchanged through strided views), weight gradients on k_wgrad_tc
// per 64 x 64 tile with a fixed-order reduction into the FP32 gradient, Adam
// on the FP32 weights.  Activations and their gradients are BF16.
mrs_status rdn_train_bf16(mrs_rdn_s* r, const float* lrhs, const float* hrls, const float* alb,
                          const float* nrm, const float* extra, const float* tgt, int N, int H, int W,
                          int kind, float beta, float lr, float* yout, double* loss_out,
                          cudaStream_t st)
{
    const int s = r->s, D = r->D, h = H / s, w = W / s, SS = s * s;
    const int nblk = kRDG * kRDB, nl = (int)r->L.size();
    const size_t Pl = (size_t)N * h * w, Ph = (size_t)N * H * W;
    size_t Pd[4];
    int hd[4], wd[4];
    Pd[0] = Pl; hd[0] = h; wd[0] = w;
    size_t nUrows = 0;
    for (int d = 0; d < D; ++d) {
        Pd[d + 1] = 4 * Pd[d]; hd[d + 1] = 2 * hd[d]; wd[d + 1] = 2 * wd[d];
        nUrows += Pd[d + 1];
    }
    mrs_status rc = MRS_OK;
    // weights: forward chunks and transposed chunks from the FP32 parameters
    if (r->tidx.empty()) {
        build_tpack_index(r);
        if ((rc = upload_index(r->tidx, &r->d_tidx)) != MRS_OK) return rc;
        MRS_CHECK(cudaMalloc(&r->wbfT, r->tidx.size() * sizeof(__nv_bfloat16)));
        if ((rc = tc_make_w_map(&r->wmapT_all, r->wbfT, (int)(r->tidx.size() / 64), 64, TC_BF16)) != MRS_OK)
            return rc;
    }
    // workspace: BF16 [P][64] tensors, then FP32
    const size_t rows = Pl * (3 + 15 + 4 * nblk + 10) + Ph * 6 + nUrows;
    const int maxp = tc_wgrad_max_parts();
    const size_t nf = Ph * 6 + (size_t)maxp * 9 * 4096 + (size_t)maxp * 64 + 64 + Pl * 3 + Ph * 21;
    if ((rc = r->trb.ensure(rows * 128 + nf * 4 + (kLossParts + 2) * 8 + 4096)) != MRS_OK) return rc;
    __nv_bfloat16* bp = r->trb.as<__nv_bfloat16>();
    auto take = [&](size_t P) { __nv_bfloat16* q = bp; bp += P * 64; return q; };
    __nv_bfloat16* inL = take(Pl);
    __nv_bfloat16* inH = take(Ph);
    __nv_bfloat16* Flr = take(Pl);
    __nv_bfloat16* Fh0 = take(Ph);
    __nv_bfloat16* F0 = take(Pl);
    __nv_bfloat16* X[kRDG * kRDB + 1];       // block inputs; X[nblk] = F_DF
    X[0] = F0;
    for (int k = 1; k <= nblk; ++k) X[k] = take(Pl);
    __nv_bfloat16* Fk[kRDG * kRDB][4];       // F_1, F_2, F_3, ReLU(local fusion) of each block
    for (int k = 0; k < nblk; ++k)
        for (int j = 0; j < 4; ++j) Fk[k][j] = take(Pl);
    __nv_bfloat16* U[4];                      // U[0] = F_DF, U[d + 1] the output of upsampling stage d
    U[0] = X[nblk];
    for (int d = 1; d <= D; ++d) U[d] = take(Pd[d]);
    __nv_bfloat16* dyb = take(Ph);
    __nv_bfloat16* dU[2] = {take(Ph), take(Ph)};
    __nv_bfloat16* G = take(Pl);              // gradient of the current block's output / input
    __nv_bfloat16* dp[4];                     // dp[0] = G; dp[1..3]: the block's F_1..F_3 gradients
    dp[0] = G;
    for (int j = 1; j < 4; ++j) dp[j] = take(Pl);
    __nv_bfloat16* dz4 = take(Pl);
    __nv_bfloat16* dSkip = take(Pl);
    __nv_bfloat16* dzf = take(Pl);
    __nv_bfloat16* dzlr = take(Pl);
    __nv_bfloat16* dz1 = take(Ph);
    float* y = (float*)bp;
    float* dy = y + Ph * 3;
    float* part = dy + Ph * 3;
    float* dbpart = part + (size_t)maxp * 9 * 4096;
    float* zero = dbpart + (size_t)maxp * 64;   // zero biases of the input-gradient convs
    // staging: the caller's batch, copied here every step (the recorded launches read these)
    float* sLr = zero + 64;
    float* sHr = sLr + Pl * 3;
    float* sAlb = sHr + Ph * 3;
    float* sNrm = sAlb + Ph * 3;
    float* sEx = sNrm + Ph * 3;
    float* sTgt = sEx + Ph * 9;
    double* lparts = (double*)(((uintptr_t)(sTgt + Ph * 3) + 7) & ~(uintptr_t)7);
    double* lsum = lparts + kLossParts;
    MRS_CHECK(cudaMemcpyAsync(sLr, lrhs, Pl * 3 * 4, cudaMemcpyDeviceToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(sHr, hrls, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(sAlb, alb, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(sNrm, nrm, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));
    if (extra) MRS_CHECK(cudaMemcpyAsync(sEx, extra, Ph * 9 * 4, cudaMemcpyDeviceToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(sTgt, tgt, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));

    // The launches of a step depend only on the shapes, the loss and the
    // workspace: the first step of a shape runs them directly and records
    // them as a CUDA graph (on a private stream), later steps replay it.
    // (with per-launch event timing on, steps run directly and nothing is
    // recorded: the timing events must be real ones)
    const TrainKey key{N, H, W, kind, beta, r->trb.p};
    const bool timing = prof_on();
    if (r->tgraph && key == r->tkey && !timing) {
        MRS_CHECK(cudaGraphLaunch(r->tgraph, st));
        launch_counter() += r->tgraph_kernels;
    } else {
    if (r->tgraph) { cudaGraphExecDestroy(r->tgraph); r->tgraph = nullptr; }

    // tensor maps
    auto amap = [&](CUtensorMap* m, const void* q, int hh, int ww) { return tc_make_act_map(m, q, N, hh, ww, TC_BF16, kABox); };
    auto omap = [&](CUtensorMap* m, const void* q, int hh, int ww) { return tc_make_act_map(m, q, N, hh, ww, TC_BF16, kOutBox); };
    auto xmap = [&](CUtensorMap* m, const void* q, int hh, int ww) { return tc_make_act_map(m, q, N, hh, ww, TC_BF16, kWgKB + 2); };
    auto ymap = [&](CUtensorMap* m, const void* q, int hh, int ww) { return tc_make_act_map(m, q, N, hh, ww, TC_BF16, kWgKB); };
    // sub-pixel (oy, ox) of every sub x sub block of a [N][HH][WW][64] tensor
    auto view = [&](CUtensorMap* m, const __nv_bfloat16* base, int sub, int oy, int ox, int HH, int WW, int box) {
        return tc_make_view_map(m, base + ((size_t)oy * WW + ox) * 64, N, HH / sub, WW / sub,
                                (long long)sub * 128, (long long)sub * WW * 128, (long long)HH * WW * 128, box);
    };
    struct M4 { CUtensorMap a, o, x, y; };   // the four box kinds of one tensor
    auto all4 = [&](M4& m, const void* q, int hh, int ww) {
        mrs_status e = amap(&m.a, q, hh, ww);
        if (e == MRS_OK) e = omap(&m.o, q, hh, ww);
        if (e == MRS_OK) e = xmap(&m.x, q, hh, ww);
        if (e == MRS_OK) e = ymap(&m.y, q, hh, ww);
        return e;
    };
    M4 mInL, mInH, mFlr, mFh0, mX[kRDG * kRDB + 1], mF[kRDG * kRDB][4], mU[4], mDyb, mDU[2], mDp[4], mDz4,
        mDzf, mDzlr, mDz1;
    if (rc == MRS_OK) rc = all4(mInL, inL, h, w);
    if (rc == MRS_OK) rc = all4(mInH, inH, H, W);
    if (rc == MRS_OK) rc = all4(mFlr, Flr, h, w);
    if (rc == MRS_OK) rc = all4(mFh0, Fh0, H, W);
    for (int k = 0; k <= nblk && rc == MRS_OK; ++k) rc = all4(mX[k], X[k], h, w);
    for (int k = 0; k < nblk; ++k)
        for (int j = 0; j < 4 && rc == MRS_OK; ++j) rc = all4(mF[k][j], Fk[k][j], h, w);
    for (int d = 0; d <= D && rc == MRS_OK; ++d) rc = all4(mU[d], U[d], hd[d], wd[d]);
    if (rc == MRS_OK) rc = all4(mDyb, dyb, H, W);
    for (int j = 0; j < 4 && rc == MRS_OK; ++j) rc = all4(mDp[j], dp[j], h, w);
    if (rc == MRS_OK) rc = all4(mDz4, dz4, h, w);
    if (rc == MRS_OK) rc = all4(mDzf, dzf, h, w);
    if (rc == MRS_OK) rc = all4(mDzlr, dzlr, h, w);
    if (rc == MRS_OK) rc = all4(mDz1, dz1, H, W);
    if (rc != MRS_OK) return rc;
    // the level-(d + 1) gradient of the upsampling path sits in dU[(D - 1 - d) & 1]
    // ([P_{d+1}][64]); its plain maps per level, and the deshuffle views
    std::vector<M4> mDUl(D + 1);
    for (int d = 0; d <= D && rc == MRS_OK; ++d) rc = all4(mDUl[d], dU[(D - d) & 1], hd[d], wd[d]);
    std::vector<CUtensorMap> dsfA(SS), dsfO(SS), dsfX(SS), dz1O(SS);
    for (int q = 0; q < SS && rc == MRS_OK; ++q) {
        const int oy = q / s, ox = q % s;
        rc = view(&dsfA[q], Fh0, s, oy, ox, H, W, kABox);
        if (rc == MRS_OK) rc = view(&dsfO[q], Fh0, s, oy, ox, H, W, kOutBox);
        if (rc == MRS_OK) rc = view(&dsfX[q], Fh0, s, oy, ox, H, W, kWgKB + 2);
        if (rc == MRS_OK) rc = view(&dz1O[q], dz1, s, oy, ox, H, W, kOutBox);
    }
    // upsampling stage d: output views of U[d + 1] (forward) and views of the
    // level-(d + 1) gradient (A operands and weight-gradient dy)
    std::vector<std::array<CUtensorMap, 4>> upO(D), dupA(D), dupY(D);
    for (int d = 0; d < D && rc == MRS_OK; ++d)
        for (int q = 0; q < 4 && rc == MRS_OK; ++q) {
            const int dy_ = q >> 1, dx_ = q & 1;
            const __nv_bfloat16* g = dU[(D - 1 - d) & 1];
            rc = view(&upO[d][q], U[d + 1], 2, dy_, dx_, hd[d + 1], wd[d + 1], kOutBox);
            if (rc == MRS_OK) rc = view(&dupA[d][q], g, 2, dy_, dx_, hd[d + 1], wd[d + 1], kABox);
            if (rc == MRS_OK) rc = view(&dupY[d][q], g, 2, dy_, dx_, hd[d + 1], wd[d + 1], kWgKB);
        }
    if (rc != MRS_OK) return rc;
    // multi-chunk A-operand arrays: the fuse conv's 17 inputs, each block's 4
    // concatenation parts, each upsampling stage's 4 gradient views
    std::vector<CUtensorMap> mc;
    const size_t mc_fuse = mc.size();
    mc.push_back(mFlr.a);
    for (int q = 0; q < SS; ++q) mc.push_back(dsfA[q]);
    std::vector<size_t> mc_blk(nblk), mc_up(D);
    for (int k = 0; k < nblk; ++k) {
        mc_blk[k] = mc.size();
        mc.push_back(mX[k].a);
        for (int j = 0; j < 3; ++j) mc.push_back(mF[k][j].a);
    }
    for (int d = 0; d < D; ++d) {
        mc_up[d] = mc.size();
        for (int q = 0; q < 4; ++q) mc.push_back(dupA[d][q]);
    }
    if ((rc = r->tdmaps.ensure(mc.size() * sizeof(CUtensorMap) + 64)) != MRS_OK) return rc;
    const CUtensorMap* dmc = r->tdmaps.as<CUtensorMap>();
    MRS_CHECK(cudaMemcpyAsync(r->tdmaps.p, mc.data(), mc.size() * sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice, st));

    auto body = [&](cudaStream_t st) -> mrs_status {
    mrs_status rc = repack_bf16(r, st);
    if (rc != MRS_OK) return rc;
    k_gather_bf16<<<grid_for(r->tidx.size()), 256, 0, st>>>(r->master, r->d_tidx, r->tidx.size(), r->wbfT);
    MRS_LAUNCHED(1);
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.scale = 1; a.operand = TC_BF16; a.err = r->err;
    // one tensor-core conv: mc_off >= 0 = a kc-chunk launch over dmc[mc_off ..]
    auto conv = [&](int hh, int ww, const CUtensorMap* A, long mc_off, int kc, const CUtensorMap* wm,
                    int w_row0, const float* bias, int nout, int mode, const CUtensorMap* res,
                    const CUtensorMap* out, float* outf = nullptr, int cout = 64) -> mrs_status {
        a.H = hh; a.W = ww; a.tmap_x = A;
        a.amaps = mc_off >= 0 ? dmc + mc_off : nullptr;
        a.kc = mc_off >= 0 ? kc : 0;
        a.tmap_w = wm; a.w_row0 = w_row0; a.bias = bias; a.nout = nout; a.mode = mode;
        a.tmap_res = res; a.tmap_out = out; a.out = outf; a.cout = cout; a.relu = 0;
        return tc_conv3x3(a, st);
    };
    const WChunk* CH = r->ch.data();
    auto fmap = [&](int li, int j) { return &CH[r->first[li] + j].map; };       // single forward chunk
    auto frow = [&](int li) { return (int)(CH[r->first[li]].off / 64); };       // a layer's chunks in wmap_all
    auto fbias = [&](int li, int j) { return r->bch + (size_t)(r->first[li] + j) * 64; };
    auto trow = [&](int li, int j) { return r->tfirst[li] + 9 * 64 * j; };      // transposed chunk j
    MRS_CHECK(cudaMemsetAsync(zero, 0, 64 * sizeof(float), st));

    // ---- forward
    k_lr_input_bf16<<<grid_for(Pl), 256, 0, st>>>(sLr, Pl, inL);
    k_hr_input_bf16<<<grid_for(Ph), 256, 0, st>>>(sHr, sAlb, sNrm, extra ? sEx : nullptr, Ph, inH);
    MRS_LAUNCHED(2);
    if ((rc = conv(h, w, &mInL.a, -1, 1, fmap(0, 0), 0, fbias(0, 0), 64, TC_RELU_BF16, nullptr, &mFlr.o)) != MRS_OK) return rc;
    if ((rc = conv(H, W, &mInH.a, -1, 1, fmap(1, 0), 0, fbias(1, 0), 64, TC_RELU_BF16, nullptr, &mFh0.o)) != MRS_OK) return rc;
    if ((rc = conv(h, w, &mFlr.a, (long)mc_fuse, 1 + SS, &r->wmap_all, frow(2), fbias(2, 0), 64, TC_RELU_BF16,
                   nullptr, &mX[0].o)) != MRS_OK) return rc;
    int li = 3;
    for (int g = 0; g < kRDG; ++g) {
        for (int b = 0; b < kRDB; ++b) {
            const int k = kRDB * g + b;
            for (int c = 1; c <= kConv; ++c, ++li) {
                const CUtensorMap* out = &mF[k][c - 1].o;        // F_1, F_2, F_3, ReLU(local fusion)
                rc = c == 1 ? conv(h, w, &mX[k].a, -1, 1, fmap(li, 0), 0, fbias(li, 0), 64, TC_RELU_BF16, nullptr, out)
                            : conv(h, w, &mX[k].a, (long)mc_blk[k], c, &r->wmap_all, frow(li), fbias(li, 0), 64,
                                   TC_RELU_BF16, nullptr, out);
                if (rc != MRS_OK) return rc;
            }
            // block output; + F_{g-1} after a group's last block; + F_0 at the end (Eq. F_DF)
            const bool last = b == kRDB - 1;
            k_sum_bf16<<<grid_for(Pl * 64), 256, 0, st>>>(X[k + 1], X[k], Fk[k][3], last ? X[kRDB * g] : nullptr,
                                                          k + 1 == nblk ? F0 : nullptr, nullptr, Pl * 64);
            MRS_LAUNCHED(1);
        }
    }
    for (int d = 0; d < D; ++d, ++li)
        for (int q = 0; q < 4; ++q)
            if ((rc = conv(hd[d], wd[d], &mU[d].a, -1, 1, fmap(li, q), 0, fbias(li, q), 64, TC_RELU_BF16,
                           nullptr, &upO[d][q])) != MRS_OK) return rc;
    const int li_rec = li;
    if ((rc = conv(H, W, &mU[D].a, -1, 1, fmap(li_rec, 0), 0, fbias(li_rec, 0), CH[r->first[li_rec]].nout,
                   TC_PLAIN_F32, nullptr, nullptr, y, 3)) != MRS_OK) return rc;

    // ---- loss and dL/dI_SR
    if ((rc = loss_grad_f32(y, sTgt, Ph * 3, kTrainClip, kind, beta, dy, lparts, lsum, st)) != MRS_OK) return rc;
    k_f32_to_bf16_rows<<<grid_for(Ph * 64), 256, 0, st>>>(dy, Ph, 3, dyb);
    MRS_LAUNCHED(1);

    // ---- backward
    // Weight gradients, one 64 x 64 tile per launch (see k_wg_reduce for the
    // mappings into the layer gradient).  A group of tiles (a conv's input
    // parts, an upsampling conv's four views, the fuse conv's 17 chunks) runs
    // side by side on up to kWgStreams streams, each tile on its stream's
    // share of the SMs: at the LR grid a tile is little work, and a tile on
    // fewer CTAs writes (and its reduction reads) that many fewer partials.
    struct WgTile {
        const CUtensorMap* xm;
        const CUtensorMap* ym;
        int hh, ww, cin_t, cout_t, lidx, o_mul, o_add, c0, q;
        bool with_bias;
    };
    constexpr int kWgStreams = 4;
    auto wgrad_group = [&](int ntile, auto tile) -> mrs_status {
        const int S = ntile < kWgStreams ? ntile : kWgStreams;
        const int cap = maxp / S;
        cudaStream_t ss[kWgStreams] = {st, nullptr, nullptr, nullptr};
        for (int i = 1; i < S; ++i) {
            if (!r->side[i - 1]) MRS_CHECK(cudaStreamCreateWithFlags(&r->side[i - 1], cudaStreamNonBlocking));
            if (!r->ev_join[i - 1]) MRS_CHECK(cudaEventCreateWithFlags(&r->ev_join[i - 1], cudaEventDisableTiming));
            ss[i] = r->side[i - 1];
        }
        if (S > 1) {
            if (!r->ev_fork) MRS_CHECK(cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming));
            MRS_CHECK(cudaEventRecord(r->ev_fork, st));
            for (int i = 1; i < S; ++i) MRS_CHECK(cudaStreamWaitEvent(ss[i], r->ev_fork, 0));
        }
        for (int i = 0; i < ntile; ++i) {
            const WgTile t = tile(i);
            cudaStream_t sq = ss[i % S];
            float* pt = part + (size_t)(i % S) * cap * 9 * 4096;
            float* pb = dbpart + (size_t)(i % S) * cap * 64;
            TcWgradArgs wa;
            wa.tmap_x = t.xm; wa.tmap_dy = t.ym; wa.part = pt; wa.dbpart = pb;
            wa.N = N; wa.H = t.hh; wa.W = t.ww; wa.cin = t.cin_t; wa.cout = t.cout_t; wa.err = r->err;
            wa.max_ctas = cap;
            int np = 0;
            mrs_status e = tc_conv3x3_wgrad(wa, &np, sq);
            if (e != MRS_OK) return e;
            const RLayer& l = r->L[t.lidx];
            const int KK = l.k * l.k;
            const size_t n = (size_t)t.cout_t * KK * t.cin_t + t.cout_t;
            k_wg_reduce<<<(int)((n + 31) / 32), 256, 0, sq>>>(pt, pb, np, t.cin_t, t.cout_t, KK, l.cin, t.o_mul,
                                                              t.o_add, t.c0, t.q, s, D, t.with_bias ? 1 : 0,
                                                              r->grad + l.woff, r->grad + l.boff);
            MRS_LAUNCHED(1);
        }
        for (int i = 1; i < S; ++i) {
            MRS_CHECK(cudaEventRecord(r->ev_join[i - 1], ss[i]));
            MRS_CHECK(cudaStreamWaitEvent(st, r->ev_join[i - 1], 0));
        }
        return cuda_status(cudaGetLastError(), "rdn wgrad");
    };
    auto mask = [&](const __nv_bfloat16* d, const __nv_bfloat16* act, size_t P, __nv_bfloat16* out) {
        k_mask_copy_bf16<<<grid_for(P * 64), 256, 0, st>>>(d, act, P * 64, out);
        MRS_LAUNCHED(1);
    };
    const CUtensorMap* WT = &r->wmapT_all;
    // H_Rec
    if ((rc = wgrad_group(1, [&](int) { return WgTile{&mU[D].x, &mDyb.y, H, W, 64, 3, li_rec, 1, 0, 0, 0, true}; }))
        != MRS_OK) return rc;
    if ((rc = conv(H, W, &mDyb.a, -1, 1, WT, trow(li_rec, 0), zero, 64, TC_LIN_BF16, nullptr, &mDUl[D].o)) != MRS_OK)
        return rc;
    // upsampling stages in reverse: the level-(d + 1) gradient masked by U[d + 1] > 0
    for (int d = D - 1; d >= 0; --d) {
        const int lu = 3 + kConv * nblk + d;
        __nv_bfloat16* gd = dU[(D - 1 - d) & 1];
        mask(gd, U[d + 1], Pd[d + 1], gd);
        if ((rc = wgrad_group(4, [&](int q) {
                 return WgTile{&mU[d].x, &dupY[d][q], hd[d], wd[d], 64, 64, lu, 4, q, 0, 0, true}; })) != MRS_OK)
            return rc;
        if ((rc = conv(hd[d], wd[d], &dupA[d][0], (long)mc_up[d], 4, WT, trow(lu, 0), zero, 64, TC_LIN_BF16,
                       nullptr, &mDUl[d].o)) != MRS_OK) return rc;
    }
    __nv_bfloat16* gdf = dU[D & 1];               // dL/dF_DF: to F_G (the chain) and to F_0
    MRS_CHECK(cudaMemcpyAsync(G, gdf, Pl * 128, cudaMemcpyDeviceToDevice, st));
    for (int g = kRDG - 1; g >= 0; --g) {
        MRS_CHECK(cudaMemcpyAsync(dSkip, G, Pl * 128, cudaMemcpyDeviceToDevice, st));
        for (int b = kRDB - 1; b >= 0; --b) {
            const int k = kRDB * g + b, lb = 3 + kConv * k;
            // local fusion: dz4 = G masked by its ReLU output; one weight tile per
            // concatenation part; part 0's gradient = G + conv^T, parts 1..3 start here
            mask(G, Fk[k][3], Pl, dz4);
            if ((rc = wgrad_group(4, [&](int j) {
                     return WgTile{j ? &mF[k][j - 1].x : &mX[k].x, &mDz4.y, h, w, 64, 64, lb + 3, 1, 0, 64 * j, 0,
                                   j == 0}; })) != MRS_OK) return rc;
            if ((rc = conv(h, w, &mDz4.a, -1, 1, WT, trow(lb + 3, 0), zero, 64, TC_RESID_BF16, &mDp[0].o,
                           &mDp[0].o)) != MRS_OK) return rc;
            for (int j = 1; j < 4; ++j)
                if ((rc = conv(h, w, &mDz4.a, -1, 1, WT, trow(lb + 3, j), zero, 64, TC_LIN_BF16, nullptr,
                               &mDp[j].o)) != MRS_OK) return rc;
            // dense convs 3, 2, 1: the gradient of F_c is complete once the later
            // convs have added theirs; masked by F_c, then its weight tiles and
            // its input gradients added into parts 0 .. c - 1
            for (int c = kConv - 1; c >= 1; --c) {
                const int lc = lb + c - 1;
                mask(dp[c], Fk[k][c - 1], Pl, dp[c]);
                if ((rc = wgrad_group(c, [&](int j) {
                         return WgTile{j ? &mF[k][j - 1].x : &mX[k].x, &mDp[c].y, h, w, 64, 64, lc, 1, 0, 64 * j, 0,
                                       j == 0}; })) != MRS_OK) return rc;
                for (int j = 0; j < c; ++j)
                    if ((rc = conv(h, w, &mDp[c].a, -1, 1, WT, trow(lc, j), zero, 64, TC_RESID_BF16, &mDp[j].o,
                                   &mDp[j].o)) != MRS_OK) return rc;
            }
        }
        // F_g = chain(F_{g-1}) + F_{g-1}
        k_sum_bf16<<<grid_for(Pl * 64), 256, 0, st>>>(G, G, dSkip, nullptr, nullptr, nullptr, Pl * 64);
        MRS_LAUNCHED(1);
    }
    // fuse: dz = (dL/dF_DF + the chain's gradient) masked by F_0
    k_sum_bf16<<<grid_for(Pl * 64), 256, 0, st>>>(dzf, gdf, G, nullptr, nullptr, F0, Pl * 64);
    MRS_LAUNCHED(1);
    if ((rc = wgrad_group(SS + 1, [&](int q) {
             return WgTile{q ? &dsfX[q - 1] : &mFlr.x, &mDzf.y, h, w, 64, 64, 2, 1, 0, 0, q, q == 0}; })) != MRS_OK)
        return rc;
    // its input gradients, masked by the encoders' ReLU outputs: chunk 0 into
    // F_LRHS's gradient, chunk q into deshuffle view q of F0_HRLS's
    if ((rc = conv(h, w, &mDzf.a, -1, 1, WT, trow(2, 0), zero, 64, TC_MASK_BF16, &mFlr.o, &mDzlr.o)) != MRS_OK)
        return rc;
    for (int q = 1; q <= SS; ++q)
        if ((rc = conv(h, w, &mDzf.a, -1, 1, WT, trow(2, q), zero, 64, TC_MASK_BF16, &dsfO[q - 1],
                       &dz1O[q - 1])) != MRS_OK) return rc;
    // encoders
    if ((rc = wgrad_group(2, [&](int e) {
             return e == 0 ? WgTile{&mInL.x, &mDzlr.y, h, w, 3, 64, 0, 1, 0, 0, 0, true}
                           : WgTile{&mInH.x, &mDz1.y, H, W, r->c_hr, 64, 1, 1, 0, 0, 0, true}; })) != MRS_OK)
        return rc;

    return MRS_OK;
    };
    // this step, directly
    if ((rc = body(st)) != MRS_OK) return rc;
    // recorded for the next steps of this shape
    if (!timing) {
    if (!r->tcap) MRS_CHECK(cudaStreamCreateWithFlags(&r->tcap, cudaStreamNonBlocking));
    const uint64_t before = launch_counter().load();
    MRS_CHECK(cudaStreamBeginCapture(r->tcap, cudaStreamCaptureModeThreadLocal));
    mrs_status cr = body(r->tcap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(r->tcap, &g);
    const uint64_t recorded = launch_counter().load() - before;
    launch_counter() -= recorded;              // recorded, not run
    if (cr == MRS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&r->tgraph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cr != MRS_OK || e != cudaSuccess) {
        r->tgraph = nullptr;
        cudaGetLastError();
    } else {
        r->tkey = key;
        r->tgraph_kernels = recorded;
    }
    }
    }
    if (yout) MRS_CHECK(cudaMemcpyAsync(yout, y, Ph * 3 * 4, cudaMemcpyDeviceToDevice, st));

    // ---- Adam on the FP32 weights
    r->step += 1;
    if ((rc = adam_f32(r->master, r->grad, r->adam_m, r->adam_v, r->np, lr, r->step, st)) != MRS_OK) return rc;
    r->bf_stale = true;
    if (loss_out) {
        double hsum = 0;
        int herr = 0;
        MRS_CHECK(cudaMemcpyAsync(&hsum, lsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaMemcpyAsync(&herr, r->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        if (herr) {
            cudaMemset(r->err, 0, 4);
            set_error("tensor-core wait timed out in the training step");
            return MRS_ERR_TIMEOUT;
        }
        *loss_out = hsum / (double)(Ph * 3);
    }
    return cuda_status(cudaGetLastError(), "rdn train step bf16");
}

}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_rdn_nparams(int32_t scale, int32_t hr_channels, int64_t* n)
{
    MRS_ARG(n != nullptr, "n is NULL");
    MRS_ARG(depth_of(scale) > 0, "scale must be 2, 4 or 8");
    MRS_ARG(hr_channels == 9 || hr_channels == 18, "hr_channels must be 9 or 18");
    *n = (int64_t)rdn_nparams(scale, hr_channels);
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_free(mrs_rdn r)
{
    if (!r) return MRS_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {r->master, r->w_fuse3, r->wbf, r->bch, r->err, r->grad, r->adam_m, r->adam_v,
                    r->d_widx, r->d_bidx, r->d_tidx, r->wbfT};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (r->tgraph) cudaGraphExecDestroy(r->tgraph);
    if (r->tcap) cudaStreamDestroy(r->tcap);
    for (int i = 0; i < 3; ++i) {
        if (r->side[i]) cudaStreamDestroy(r->side[i]);
        if (r->ev_join[i]) cudaEventDestroy(r->ev_join[i]);
    }
    if (r->ev_fork) cudaEventDestroy(r->ev_fork);
    r->f32.release();
    r->bf.release();
    r->tr.release();
    r->trb.release();
    r->dmaps.release();
    delete r;
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_create(int32_t scale, int32_t hr_channels, const float* params,
                                     int64_t n_params, mrs_rdn* out)
{
    MRS_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MRS_ARG(params != nullptr, "params is NULL");
    MRS_ARG(depth_of(scale) > 0, "scale must be 2, 4 or 8");
    MRS_ARG(hr_channels == 9 || hr_channels == 18, "hr_channels must be 9 or 18");
    MRS_ARG(n_params == (int64_t)rdn_nparams(scale, hr_channels), "n_params must equal mrs_rdn_nparams");
    mrs_rdn_s* r = new mrs_rdn_s();
    r->s = scale;
    r->D = depth_of(scale);
    r->c_hr = hr_channels;
    r->np = (size_t)n_params;
    r->L = rdn_layers(scale, hr_channels);
    const int Ccat = kF + kF * scale * scale;
    mrs_status s = cuda_status(cudaMalloc(&r->master, r->np * 4), "cudaMalloc(rdn)");
    if (s == MRS_OK) s = cuda_status(cudaMalloc(&r->w_fuse3, (size_t)64 * 9 * Ccat * 4), "cudaMalloc(rdn)");
    if (s == MRS_OK) s = cuda_status(cudaMalloc(&r->err, 4), "cudaMalloc(rdn)");
    if (s == MRS_OK) s = cuda_status(cudaMemset(r->err, 0, 4), "memset");
    if (s == MRS_OK)
        s = cuda_status(cudaMemcpy(r->master, params, r->np * 4, cudaMemcpyHostToDevice), "params");
    if (s == MRS_OK) s = pack_chunks(r, params);
    if (s != MRS_OK) { mrs_rdn_free(r); return s; }
    *out = r;
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_fuse(mrs_rdn r, const float* lrhs, const float* hrls,
                                   const float* albedo, const float* normal, const float* extra,
                                   int32_t N, int32_t H, int32_t W, int32_t precision, float* out,
                                   void* stream)
{
    MRS_ARG(r != nullptr, "rdn is NULL");
    MRS_ARG(lrhs && hrls && albedo && normal && out, "NULL image pointer");
    MRS_ARG((extra != nullptr) == (r->c_hr == 18), "extra must be given exactly for hr_channels 18");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1, "N, H, W must be >= 1");
    MRS_ARG(H % r->s == 0 && W % r->s == 0, "H and W must be multiples of the scale");
    MRS_ARG((int64_t)N * H * W <= (int64_t(1) << 26), "N*H*W exceeds 2^26 pixels");
    MRS_ARG(precision == MRS_PREC_FP32 || precision == MRS_PREC_BF16,
            "precision must be MRS_PREC_FP32 or MRS_PREC_BF16");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MRS_PREC_BF16) {
        mrs_status rc = repack_if_stale(r, st);
        if (rc != MRS_OK) return rc;
    }
    mrs_status rc = precision == MRS_PREC_FP32
                        ? rdn_f32(r, lrhs, hrls, albedo, normal, extra, N, H, W, out, st)
                        : rdn_bf16(r, lrhs, hrls, albedo, normal, extra, N, H, W, out, st);
    return rc;
}

extern "C" mrs_status mrs_rdn_train_step(mrs_rdn r, const float* lrhs, const float* hrls,
                                         const float* albedo, const float* normal, const float* extra,
                                         const float* target, int32_t N, int32_t H, int32_t W,
                                         int32_t loss, float beta, float lr, int32_t precision,
                                         float* out, double* loss_out, void* stream)
{
    MRS_ARG(r != nullptr, "rdn is NULL");
    MRS_ARG(lrhs && hrls && albedo && normal && target, "NULL image pointer");
    MRS_ARG((extra != nullptr) == (r->c_hr == 18), "extra must be given exactly for hr_channels 18");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1, "N, H, W must be >= 1");
    MRS_ARG(H % r->s == 0 && W % r->s == 0, "H and W must be multiples of the scale");
    MRS_ARG((int64_t)N * H * W <= (int64_t(1) << 24), "N*H*W exceeds 2^24 pixels");
    MRS_ARG(loss == MRS_LOSS_L1LOG || loss == MRS_LOSS_ROBUST, "loss must be MRS_LOSS_L1LOG or MRS_LOSS_ROBUST");
    MRS_ARG(loss != MRS_LOSS_ROBUST || beta > 0.0f, "beta must be > 0");
    MRS_ARG(lr >= 0.0f, "lr must be >= 0");
    MRS_ARG(precision == MRS_PREC_FP32 || precision == MRS_PREC_BF16,
            "precision must be MRS_PREC_FP32 or MRS_PREC_BF16");
    mrs_status rc = ensure_train_state(r);
    if (rc != MRS_OK) return rc;
    if (precision == MRS_PREC_BF16)
        return rdn_train_bf16(r, lrhs, hrls, albedo, normal, extra, target, N, H, W, loss, beta, lr, out,
                              loss_out, (cudaStream_t)stream);
    return rdn_train_f32(r, lrhs, hrls, albedo, normal, extra, target, N, H, W, loss, beta, lr, out,
                         loss_out, (cudaStream_t)stream);
}

extern "C" mrs_status mrs_rdn_get_grads(mrs_rdn r, float* grads, int64_t n_params)
{
    MRS_ARG(r != nullptr && grads != nullptr, "NULL argument");
    MRS_ARG(n_params == (int64_t)r->np, "n_params must equal mrs_rdn_nparams");
    MRS_ARG(r->grad != nullptr, "no training step taken");
    MRS_CHECK(cudaDeviceSynchronize());
    MRS_CHECK(cudaMemcpy(grads, r->grad, r->np * 4, cudaMemcpyDeviceToHost));
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_get_state(mrs_rdn r, float* params, float* adam_m, float* adam_v,
                                        int64_t n_params, int64_t* step)
{
    MRS_ARG(r != nullptr && params != nullptr, "NULL argument");
    MRS_ARG(n_params == (int64_t)r->np, "n_params must equal mrs_rdn_nparams");
    MRS_CHECK(cudaDeviceSynchronize());
    MRS_CHECK(cudaMemcpy(params, r->master, r->np * 4, cudaMemcpyDeviceToHost));
    float* mv[2] = {adam_m, adam_v};
    float* dv[2] = {r->adam_m, r->adam_v};
    for (int i = 0; i < 2; ++i) {
        if (!mv[i]) continue;
        if (dv[i]) MRS_CHECK(cudaMemcpy(mv[i], dv[i], r->np * 4, cudaMemcpyDeviceToHost));
        else memset(mv[i], 0, r->np * 4);
    }
    if (step) *step = r->step;
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_set_state(mrs_rdn r, const float* params, const float* adam_m,
                                        const float* adam_v, int64_t n_params, int64_t step)
{
    MRS_ARG(r != nullptr && params != nullptr, "NULL argument");
    MRS_ARG(n_params == (int64_t)r->np, "n_params must equal mrs_rdn_nparams");
    MRS_ARG(step >= 0, "step must be >= 0");
    mrs_status rc = ensure_train_state(r);
    if (rc != MRS_OK) return rc;
    MRS_CHECK(cudaDeviceSynchronize());
    MRS_CHECK(cudaMemcpy(r->master, params, r->np * 4, cudaMemcpyHostToDevice));
    const float* mv[2] = {adam_m, adam_v};
    float* dv[2] = {r->adam_m, r->adam_v};
    for (int i = 0; i < 2; ++i) {
        if (mv[i]) MRS_CHECK(cudaMemcpy(dv[i], mv[i], r->np * 4, cudaMemcpyHostToDevice));
        else MRS_CHECK(cudaMemset(dv[i], 0, r->np * 4));
    }
    r->step = step;
    r->bf_stale = true;
    return MRS_OK;
}

extern "C" mrs_status mrs_rdn_check(mrs_rdn r)
{
    MRS_ARG(r != nullptr, "rdn is NULL");
    int h = 0;
    MRS_CHECK(cudaMemcpy(&h, r->err, 4, cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(r->err, 0, 4);
        set_error("tensor-core conv wait timed out");
        return MRS_ERR_TIMEOUT;
    }
    return MRS_OK;
}
