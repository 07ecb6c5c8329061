// Fusion network of the multi-resolution sampling method (Sec. 4): I_SR from
// the LRHS render and the HRLS render + albedo / normal layers, plus the image
// metrics of Sec. 5 (sRGB PSNR via Eq. cvt_color, RelMSE) and the fallback gate
// of the hybrid renderer.
//
// Precisions: FP32 (SIMT direct convolution; reference precision), BF16
// (tcgen05 implicit GEMM, conv_tc.cu) and FP8-E4M3 (tcgen05 kind::f8f6f4 with
// per-output-channel weight scales and calibrated per-layer activation scales).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <mutex>
#include <vector>

#include "conv_tc.cuh"
#include "fuse.cuh"

namespace mrs {
namespace {

constexpr int kLayers = 18;
constexpr int kFeat = 64;

struct LayerShape { int cin, cout; size_t woff, boff; };

// Layer shapes for a network whose first conv reads cin0 = 12 channels (the
// base input) or 21 (with the extra HRLS layers: diffuse, specular, variance)
const std::vector<LayerShape>& shapes(int cin0)
{
    static std::vector<LayerShape> v12, v21;
    std::vector<LayerShape>& v = cin0 == 21 ? v21 : v12;
    if (v.empty()) {
        size_t o = 0;
        for (int l = 0; l < kLayers; ++l) {
            int cin = l == 0 ? cin0 : kFeat, cout = l == kLayers - 1 ? 3 : kFeat;
            v.push_back({cin, cout, o, o + (size_t)cout * 9 * cin});
            o += (size_t)cout * 9 * cin + cout;
        }
    }
    return v;
}
constexpr size_t kParams12 = 599555;
constexpr size_t kParams21 = 604739;
constexpr int kCinMax = 21;

inline int nout_of(int l) { return l == kLayers - 1 ? 16 : 64; }

// ---- input assembly ---------------------------------------------------------
__device__ __forceinline__ void up_pixel(const float* __restrict__ lr, int h, int w, int s, int x,
                                         int y, float o[3])
{
    float inv = 1.0f / (float)s;
    float sy = fmaxf(((float)y + 0.5f) * inv - 0.5f, 0.0f);
    float sx = fmaxf(((float)x + 0.5f) * inv - 0.5f, 0.0f);
    int y0 = min((int)sy, h - 1), x0 = min((int)sx, w - 1);
    int y1 = min(y0 + 1, h - 1), x1 = min(x0 + 1, w - 1);
    float ly = sy - (float)y0, lx = sx - (float)x0;
    const float* a = lr + ((size_t)y0 * w + x0) * 3;
    const float* b = lr + ((size_t)y0 * w + x1) * 3;
    const float* c = lr + ((size_t)y1 * w + x0) * 3;
    const float* d = lr + ((size_t)y1 * w + x1) * 3;
    for (int k = 0; k < 3; ++k) {
        float top = __ldg(a + k) * (1.0f - lx) + __ldg(b + k) * lx;
        float bot = __ldg(c + k) * (1.0f - lx) + __ldg(d + k) * lx;
        o[k] = top * (1.0f - ly) + bot * ly;
    }
}

// Fusion-input channels of pixel p: up(LRHS), HRLS, albedo, normal (12) and,
// when extra != NULL (extra [P][9] = diffuse, specular, variance of the HRLS,
// Sec. 4), diffuse, specular and log(1 + max(variance, 0)) (21).  clip > 0:
// the radiance channels (up(LRHS), HRLS, diffuse, specular) are clipped at
// `clip` (the training data's firefly clipping, Sec. 3.2).  Returns the count.
__device__ __forceinline__ int input_px(const float* lrhs, const float* hrls, const float* alb,
                                        const float* nrm, const float* extra, int H, int W, int s,
                                        size_t p, float clip, float* v)
{
    int x = (int)(p % W);
    size_t r = p / W;
    int y = (int)(r % H), n = (int)(r / H);
    int h = H / s, w = W / s;
    up_pixel(lrhs + (size_t)n * h * w * 3, h, w, s, x, y, v);
    for (int k = 0; k < 3; ++k) {
        v[3 + k] = __ldg(hrls + 3 * p + k);
        v[6 + k] = __ldg(alb + 3 * p + k);
        v[9 + k] = __ldg(nrm + 3 * p + k);
    }
    if (clip > 0.0f)
        for (int k = 0; k < 6; ++k) v[k] = fminf(v[k], clip);
    if (!extra) return 12;
    for (int k = 0; k < 6; ++k) {
        float e = __ldg(extra + 9 * p + k);
        v[12 + k] = clip > 0.0f ? fminf(e, clip) : e;
    }
    for (int k = 0; k < 3; ++k) v[18 + k] = log1pf(fmaxf(__ldg(extra + 9 * p + 6 + k), 0.0f));
    return 21;
}

__global__ void k_input_f32(const float* lrhs, const float* hrls, const float* alb,
                            const float* nrm, const float* extra, int H, int W, int s, size_t P,
                            float* x0, float clip = 0.0f)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        float v[kCinMax];
        int c = input_px(lrhs, hrls, alb, nrm, extra, H, W, s, p, clip, v);
        for (int k = 0; k < c; ++k) x0[c * p + k] = v[k];
    }
}

// bf16 [P][64] or fp8 [P][64] scaled by inv_scale; channels past the input's
// 12 or 21 are zero (the first 24 bf16 / 32 fp8 channels are written from v,
// the rest as zero 16-byte words)
__global__ void k_input_q(const float* lrhs, const float* hrls, const float* alb,
                          const float* nrm, const float* extra, int H, int W, int s, size_t P,
                          void* x0, int fp8, float inv_scale, float clip = 0.0f)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P;
         p += (size_t)gridDim.x * blockDim.x) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.0f;
        input_px(lrhs, hrls, alb, nrm, extra, H, W, s, p, clip, v);
        const uint4 z = make_uint4(0, 0, 0, 0);
        if (!fp8) {
            uint4* o = (uint4*)((__nv_bfloat16*)x0 + p * 64);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                uint4 u;
                __nv_bfloat162* h2 = (__nv_bfloat162*)&u;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    h2[e] = __floats2bfloat162_rn(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
                o[j] = u;
            }
#pragma unroll
            for (int j = 3; j < 8; ++j) o[j] = z;
        } else {
            uint4* o = (uint4*)((uint8_t*)x0 + p * 64);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint4 u;
                uint8_t* b8 = (uint8_t*)&u;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    b8[e] = (uint8_t)__nv_cvt_float_to_fp8(v[16 * j + e] * inv_scale, __NV_SATFINITE, __NV_E4M3);
                o[j] = u;
            }
            o[2] = z;
            o[3] = z;
        }
    }
}

// ---- FP32 SIMT direct convolution -------------------------------------------
// block = (8 SP) x 16 output pixels and 16 output channels (grid.z over images
// x channel groups), 128 threads; a thread computes SP consecutive pixels of
// one row x 16 channels (16 SP accumulators).  Input channels go through
// shared memory in stages (8 channels for SP = 2, 4 for SP = 4, whose 64
// accumulators leave registers for 4 blocks per SM), with a 1-pixel halo, in
// two buffers: the asynchronous copies (cp.async, zero-filled outside the
// image and past cin) of the next stage are in flight while the current one
// is used.  Per (channel, kernel row) a thread reads SP + 2 inputs and, per
// column tap, 16 weights (broadcast) for 16 SP FMAs.  The input rows are
// padded so that a warp's reads (8 threads along x, 4 rows) fall in distinct
// banks (SP = 4) or at most two to a bank (SP = 2).
constexpr int kSY = 16, kSO = 16;
constexpr int simt_pitch(int sp) { return sp == 4 ? 37 : 19; }
constexpr int simt_stage(int sp) { return sp == 4 ? 4 : 8; }
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}
// x [P][xs] (first cin channels read), out / res [P][os] / [P][rs] (first
// cout written / read): strides let a layer read a prefix of a concatenation
// buffer and write into a channel slice of another
template <int kSP>
__global__ void __launch_bounds__(128, kSP == 4 ? 4 : 5)
    k_conv_simt(const float* __restrict__ x, int cin, int xs, const float* __restrict__ w,
                const float* __restrict__ b, int cout, int mode, int relu,
                const float* __restrict__ res, int rs, float* __restrict__ out, int os,
                const float* __restrict__ lrhs, int H, int W, int s)
{
    constexpr int kSX = 8 * kSP, kSPitch = simt_pitch(kSP), kSC = simt_stage(kSP);
    __shared__ float sin_[2][kSC][kSY + 2][kSPitch];
    __shared__ __align__(16) float sw[2][9][kSC][kSO];
    const int tx = threadIdx.x % (kSX / kSP), ty = threadIdx.x / (kSX / kSP);
    const int x0 = blockIdx.x * kSX, y0 = blockIdx.y * kSY;
    const int ngrp = (cout + kSO - 1) / kSO;
    const int n = blockIdx.z / ngrp;
    const int o0 = (blockIdx.z % ngrp) * kSO;
    const float* xin = x + (size_t)n * H * W * xs;
    // channels c0 .. c0 + 7 of the input tile and of the weights into buffer q
    auto stage = [&](int c0, int q) {
        for (int i = threadIdx.x; i < (kSY + 2) * (kSX + 2) * kSC; i += 128) {
            const int c = i % kSC, px = (i / kSC) % (kSX + 2), py = i / (kSC * (kSX + 2));
            const int gx = x0 + px - 1, gy = y0 + py - 1;
            const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H && c0 + c < cin;
            cp_async4(&sin_[q][c][py][px], ok ? xin + ((size_t)gy * W + gx) * xs + c0 + c : x, ok);
        }
        for (int i = threadIdx.x; i < 9 * kSC * kSO; i += 128) {
            const int c = i % kSC, t = (i / kSC) % 9, o = i / (kSC * 9);
            const bool ok = o0 + o < cout && c0 + c < cin;
            cp_async4(&sw[q][t][c][o], ok ? w + ((size_t)(o0 + o) * 9 + t) * cin + c0 + c : w, ok);
        }
        cp_async_commit();
    };
    float acc[kSP][kSO];
#pragma unroll
    for (int p = 0; p < kSP; ++p)
#pragma unroll
        for (int o = 0; o < kSO; ++o) acc[p][o] = 0.0f;
    const int nk = (cin + kSC - 1) / kSC;
    stage(0, 0);
    for (int k = 0; k < nk; ++k) {
        if (k + 1 < nk) {
            stage((k + 1) * kSC, (k + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int q = k & 1;
#pragma unroll 2
        for (int c = 0; c < kSC; ++c) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const float* row = &sin_[q][c][ty + dy][tx * kSP];
                float in[kSP + 2];
#pragma unroll
                for (int k2 = 0; k2 < kSP + 2; ++k2) in[k2] = row[k2];
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float4* w4 = (const float4*)sw[q][dy * 3 + dx][c];
                    float wv[kSO];
#pragma unroll
                    for (int j = 0; j < kSO / 4; ++j) {
                        const float4 t4 = w4[j];
                        wv[4 * j] = t4.x; wv[4 * j + 1] = t4.y; wv[4 * j + 2] = t4.z; wv[4 * j + 3] = t4.w;
                    }
#pragma unroll
                    for (int p = 0; p < kSP; ++p)
#pragma unroll
                        for (int o = 0; o < kSO; ++o) acc[p][o] += in[p + dx] * wv[o];
                }
            }
        }
        // the next iteration's copies overwrite the buffer read here
        __syncthreads();
    }
    const int gy = y0 + ty;
    if (gy >= H) return;
#pragma unroll
    for (int p = 0; p < kSP; ++p) {
        const int gx = x0 + tx * kSP + p;
        if (gx >= W) break;
        const size_t pp = ((size_t)n * H + gy) * W + gx;
        if (mode == SIMT_FINAL) {
            float up[3];
            const int h = H / s, wl = W / s;
            up_pixel(lrhs + (size_t)n * h * wl * 3, h, wl, s, gx, gy, up);
            for (int o = 0; o < kSO; ++o)
                if (o0 + o < 3) out[pp * 3 + o0 + o] = (acc[p][o] + __ldg(b + o0 + o)) + up[o0 + o];
            continue;
        }
#pragma unroll
        for (int o = 0; o < kSO; ++o) {
            if (o0 + o >= cout) break;
            float v = acc[p][o] + __ldg(b + o0 + o);
            if (mode == SIMT_RESID) v = res[pp * rs + o0 + o] + v;
            else if (mode == SIMT_MASK) v = res[pp * rs + o0 + o] > 0.0f ? v : 0.0f;
            else if (mode == SIMT_RESRELU) v = res[pp * rs + o0 + o] + fmaxf(v, 0.0f);
            else if (relu) v = fmaxf(v, 0.0f);
            out[pp * os + o0 + o] = v;
        }
    }
}

// Four pixels per thread (4 blocks per SM) pays on large grids, two (5 blocks
// per SM, more warps to hide latency) below about four waves of the former
int simt_sp(int N, int H, int W, int cout)
{
    const long long blocks4 = (long long)((W + 31) / 32) * ((H + kSY - 1) / kSY) * N *
                              ((cout + kSO - 1) / kSO);
    return blocks4 >= 16LL * sm_count() ? 4 : 2;
}

}  // namespace

mrs_status simt_conv3x3(const float* x, int cin, int xs, const float* w, const float* b, int cout,
                        int mode, int relu, const float* res, int rs, float* out, int os,
                        const float* lrhs, int N, int H, int W, int s, cudaStream_t st)
{
    const int sp = simt_sp(N, H, W, cout);
    dim3 grid((W + 8 * sp - 1) / (8 * sp), (H + kSY - 1) / kSY, N * ((cout + kSO - 1) / kSO));
    if (sp == 4)
        MRS_TIMED(PK_CONV_SIMT, st, k_conv_simt<4><<<grid, 128, 0, st>>>(x, cin, xs, w, b, cout, mode, relu, res, rs, out, os, lrhs, H, W, s));
    else
        MRS_TIMED(PK_CONV_SIMT, st, k_conv_simt<2><<<grid, 128, 0, st>>>(x, cin, xs, w, b, cout, mode, relu, res, rs, out, os, lrhs, H, W, s));
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "conv_simt launch");
}

namespace {

mrs_status conv_simt(const float* x, int cin, const float* w, const float* b, int cout, int mode,
                     int relu, const float* res, float* out, const float* lrhs, int N, int H,
                     int W, int s, cudaStream_t st)
{
    return simt_conv3x3(x, cin, cin, w, b, cout, mode, relu, res, cout, out, cout, lrhs, N, H, W,
                        s, st);
}

// ---- weight packing ---------------------------------------------------------
// packed[tap][o][c] (o < nout, c < 64), zero padded; layer l at l * 9*64*64
__global__ void k_pack_bf16(const float* __restrict__ master, size_t woff, size_t boff, int cin,
                            int cout, int nout, __nv_bfloat16* __restrict__ wp, float* __restrict__ bp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 64) bp[i] = i < cout ? master[boff + i] : 0.0f;
    if (i >= 9 * nout * 64) return;
    int c = i % 64, o = (i / 64) % nout, t = i / (64 * nout);
    float v = (o < cout && c < cin) ? master[woff + ((size_t)o * 9 + t) * cin + c] : 0.0f;
    wp[i] = __float2bfloat16_rn(v);
}

// fp8: per-output-channel scale = amax / 448 over that channel's weights
__global__ void k_pack_fp8(const float* __restrict__ master, size_t woff, size_t boff, int cin,
                           int cout, int nout, uint8_t* __restrict__ wp, float* __restrict__ bp,
                           float* __restrict__ wscale)
{
    __shared__ float amax[64];
    int tid = threadIdx.x;
    if (tid < 64) {
        float m = 0.0f;
        if (tid < cout)
            for (int k = 0; k < 9 * cin; ++k) m = fmaxf(m, fabsf(master[woff + (size_t)tid * 9 * cin + k]));
        amax[tid] = m > 0.0f ? m / 448.0f : 1.0f;
        wscale[tid] = amax[tid];
        bp[tid] = tid < cout ? master[boff + tid] : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < 9 * nout * 64; i += blockDim.x) {
        int c = i % 64, o = (i / 64) % nout, t = i / (64 * nout);
        float v = (o < cout && c < cin) ? master[woff + ((size_t)o * 9 + t) * cin + c] / amax[o] : 0.0f;
        wp[i] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

// amax of a bf16 [P][64] tensor (for fp8 activation calibration)
__global__ void k_amax_bf16(const __nv_bfloat16* __restrict__ x, size_t n, float* out)
{
    float m = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__bfloat162float(x[i])));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int*)out, __float_as_int(m));
}

// ---- metrics ----------------------------------------------------------------
__device__ __forceinline__ double srgb(double l)
{
    if (l <= 0.0) return 0.0;
    if (l <= 0.0031308) return 12.92 * l;
    if (l < 1.0) return 1.055 * pow(l, 1.0 / 2.4) - 0.055;
    return 1.0;
}

constexpr int kRedBlocks = 1024;
static_assert(kRedBlocks == kLossParts, "loss partial sums");

__global__ void k_metrics_partial(const float* __restrict__ x, const float* __restrict__ ref,
                                  int64_t n, double l1, double l2, double* part)
{
    __shared__ double s[3][256];
    double a = 0, b = 0, c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xv = x[i], rv = ref[i];
        double d = srgb(xv) - srgb(rv);
        a += d * d;
        double e = xv - rv;
        b += l1 * e * e / (rv * rv + l2);
        c += e * e;
    }
    s[0][threadIdx.x] = a; s[1][threadIdx.x] = b; s[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = s[threadIdx.x][0];
}

// out[c] = sum over i of part[i k + c] (c < k <= 4), one block of 256
// threads: strided per-thread sums, then a fixed-order tree (deterministic)
__global__ void k_reduce_parts(const double* part, int nparts, int k, double* out)
{
    __shared__ double sh[4][256];
    for (int c = 0; c < k; ++c) {
        double acc = 0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i * k + c];
        sh[c][threadIdx.x] = acc;
    }
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < k; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < k) out[threadIdx.x] = sh[threadIdx.x][0];
}

// per LR pixel: RelMSE terms of box_s(fused) vs LRHS
__global__ void k_gate_partial(const float* __restrict__ fused, const float* __restrict__ lrhs,
                               int N, int H, int W, int s, double* part)
{
    __shared__ double sh[256];
    int h = H / s, w = W / s;
    int64_t nlr = (int64_t)N * h * w;
    double acc = 0;
    double inv = 1.0 / ((double)s * s);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlr;
         i += (int64_t)gridDim.x * blockDim.x) {
        int xl = (int)(i % w);
        int64_t r = i / w;
        int yl = (int)(r % h), n = (int)(r / h);
        for (int c = 0; c < 3; ++c) {
            double m = 0;
            for (int dy = 0; dy < s; ++dy)
                for (int dx = 0; dx < s; ++dx)
                    m += fused[(((int64_t)n * H + yl * s + dy) * W + xl * s + dx) * 3 + c];
            m *= inv;
            double ref = lrhs[i * 3 + c];
            double e = m - ref;
            acc += 0.5 * e * e / (ref * ref + 0.01);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// bf16 [P][64] rows of input channels c0 .. c0 + 63 of x [P][cin] (zero past cin)
__global__ void k_to_operand_chunk(const float* x, size_t P, int cin, int c0, __nv_bfloat16* o)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 64;
        int c = c0 + (int)(i % 64);
        o[i] = __float2bfloat16_rn(c < cin ? x[p * cin + c] : 0.0f);
    }
}

// packed[tap][o][c] of input channels c0 .. c0 + 63 of w [cout][3][3][cin]
__global__ void k_pack_bf16_chunk(const float* __restrict__ w, int cin, int c0, int cout, int nout,
                                  __nv_bfloat16* __restrict__ wp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * nout * 64) return;
    int c = i % 64, o = (i / 64) % nout, t = i / (64 * nout);
    float v = (o < cout && c0 + c < cin) ? w[((size_t)o * 9 + t) * cin + c0 + c] : 0.0f;
    wp[i] = __float2bfloat16_rn(v);
}

__global__ void k_to_operand(const float* x, size_t P, int cin, void* o, int fp8, float inv)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 64;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / 64;
        int c = (int)(i % 64);
        float v = c < cin ? x[p * cin + c] : 0.0f;
        if (fp8) ((uint8_t*)o)[i] = (uint8_t)__nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
        else ((__nv_bfloat16*)o)[i] = __float2bfloat16_rn(v);
    }
}

__global__ void k_amax_f32(const float* __restrict__ x, size_t n, float* out)
{
    float m = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int*)out, __float_as_int(m));
}

// ---- training kernels (FP32) -----------------------------------------------
// transposed-conv weights: wt[c][t][o] = w[o][8 - t][c]  (flipped taps)
__global__ void k_wtrans(const float* __restrict__ w, int cin, int cout, float* __restrict__ wt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cin * 9 * cout) return;
    int o = i % cout, t = (i / cout) % 9, c = i / (cout * 9);
    wt[i] = w[((size_t)o * 9 + (8 - t)) * cin + c];
}

// dW[o][t][c] = sum_p dy[p][o] * x[p shifted by tap t][c] (zero padded), db[o] = sum_p dy[p][o]
// grid (G, ntaps, otiles * ctiles): block (g, j, z) reduces pixel tiles g, g+G, ... for tap
// t = t0 + j of the 64 x 64 channel tile z = (output tile ot, input tile ct) into
// part[z][g][j][o][c] (each z a [G][ntaps][64 * 64] slab holding the tile's cout_t x cin_t
// values packed) and, for ct = 0 and j = 0, db into dbpart[ot][g][o] (a [G * 64] slab per
// ot, cout_t values per g packed)
constexpr int kDwTile = 64;
__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// x [P][xs] (first cin channels used), dy [P][ys] (first cout used); fp32 or bf16
template <typename TX, typename TY>
__global__ void __launch_bounds__(256)
    k_dw_partial(const TX* __restrict__ x, int cin, int xs, const TY* __restrict__ dy, int cout,
                 int ys, int N, int H, int W, float* __restrict__ part, float* __restrict__ dbpart,
                 int t0, int ctiles)
{
    __shared__ __align__(16) float sdy[kDwTile][64];
    __shared__ __align__(16) float sx[kDwTile][64];
    const int j = blockIdx.y, t = t0 + j, g = blockIdx.x, G = gridDim.x;
    const int ot = blockIdx.z / ctiles, ct = blockIdx.z % ctiles;
    x += 64 * ct;
    dy += 64 * ot;
    cin = min(64, cin - 64 * ct);
    cout = min(64, cout - 64 * ot);
    const bool do_db = j == 0 && ct == 0;
    const int dyo = t / 3 - 1, dxo = t % 3 - 1;
    const int og = threadIdx.x / 16, cg = threadIdx.x % 16;
    const size_t P = (size_t)N * H * W;
    const size_t ntiles = (P + kDwTile - 1) / kDwTile;
    float acc[4][4] = {{0}};
    float dbacc[4] = {0, 0, 0, 0};
    for (size_t tile = g; tile < ntiles; tile += G) {
        size_t p0 = tile * kDwTile;
        for (int i = threadIdx.x; i < kDwTile * 64; i += 256) {
            int px = i / 64, ch = i % 64;
            size_t p = p0 + px;
            float vd = 0.0f, vx = 0.0f;
            if (p < P) {
                if (ch < cout) vd = ldf(dy + p * ys + ch);
                int xx = (int)(p % W), yy = (int)((p / W) % H);
                size_t n = p / ((size_t)W * H);
                int sx_ = xx + dxo, sy_ = yy + dyo;
                if (ch < cin && sx_ >= 0 && sx_ < W && sy_ >= 0 && sy_ < H)
                    vx = ldf(x + ((n * H + sy_) * W + sx_) * xs + ch);
            }
            sdy[px][ch] = vd;
            sx[px][ch] = vx;
        }
        __syncthreads();
#pragma unroll 4
        for (int px = 0; px < kDwTile; ++px) {
            float4 a = *(const float4*)&sdy[px][og * 4];
            float4 b = *(const float4*)&sx[px][cg * 4];
            float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] += av[i] * bv[k];
            if (do_db && cg == 0)
                for (int i = 0; i < 4; ++i) dbacc[i] += av[i];
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.z * G * gridDim.y * 4096 + ((size_t)g * gridDim.y + j) * cout * cin;
    for (int i = 0; i < 4; ++i) {
        int o = og * 4 + i;
        if (o >= cout) continue;
        for (int k = 0; k < 4; ++k) {
            int c = cg * 4 + k;
            if (c < cin) out[(size_t)o * cin + c] = acc[i][k];
        }
        if (do_db && cg == 0) dbpart[(size_t)ot * G * 64 + (size_t)g * cout + o] = dbacc[i];
    }
}

// grad[o][t][c] (params layout) = sum_g part[g][t][o][c]; grad_b[o] = sum_g dbpart[g][o]
// A block takes 32 consecutive values; warp w sums partials w, w + 8, ... (one
// coalesced 128-byte row per partial) and the eight sums are added in warp
// order: a fixed order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_dw_reduce(const float* __restrict__ part,
                                                   const float* __restrict__ dbpart, int G, int cin,
                                                   int cout, float* __restrict__ gw,
                                                   float* __restrict__ gb)
{
    __shared__ float red[8][32];
    const int nw = cout * 9 * cin, ntot = nw + cout;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const size_t gstride = (size_t)9 * cout * cin;
    for (int e0 = blockIdx.x * 32; e0 < ntot; e0 += gridDim.x * 32) {
        const int e = e0 + lane;
        float acc = 0.0f;
        if (e < nw) {
            const int c = e % cin, t = (e / cin) % 9, o = e / (cin * 9);
            const float* src = part + ((size_t)t * cout + o) * cin + c;
            for (int g = wp; g < G; g += 8) acc += src[(size_t)g * gstride];
        } else if (e < ntot) {
            const int o = e - nw;
            for (int g = wp; g < G; g += 8) acc += dbpart[(size_t)g * cout + o];
        }
        red[wp][lane] = acc;
        __syncthreads();
        if (wp == 0 && e < ntot) {
            float v = red[0][lane];
            for (int k = 1; k < 8; ++k) v += red[k][lane];
            if (e < nw) gw[e] = v;
            else gb[e - nw] = v;
        }
        __syncthreads();
    }
}

// Training losses, reduced in float64 per block; dy receives dL/dy.
//   MRS_LOSS_L1LOG: L1 on slog(x) = sign(x) log1p(|x|) (= log(1 + x) for
//     x >= 0): d = slog(y) - slog(min(t, clip)); dy = sign(d) / (1 + |y|) / n
//   MRS_LOSS_ROBUST: the robust loss l_r of Sec. 3, e = y - min(t, clip),
//     |e| / (beta + |e|) per value; dy = sign(e) beta / (beta + |e|)^2 / n
__device__ __forceinline__ double slog(double x) { return x < 0.0 ? -log1p(-x) : log1p(x); }

__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ tgt, size_t n,
                       float clip, int kind, float beta, float* __restrict__ dy,
                       double* __restrict__ part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    const float inv_n = 1.0f / (float)n;
    const double b = (double)beta, dinv_n = 1.0 / (double)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float yp = y[i];
        float tv = clip > 0.0f ? fminf(tgt[i], clip) : tgt[i];
        float g = 0.0f;
        if (kind == MRS_LOSS_ROBUST) {
            double e = (double)yp - (double)tv, a = fabs(e);
            acc += a / (b + a);
            if (e != 0.0) g = (float)((e > 0.0 ? b : -b) / ((b + a) * (b + a)) * dinv_n);
        } else {
            double d = slog((double)yp) - slog((double)tv);
            acc += fabs(d);
            if (d != 0.0) g = (d > 0.0 ? 1.0f : -1.0f) / (1.0f + fabsf(yp)) * inv_n;
        }
        dy[i] = g;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mask_inplace(float* __restrict__ d, const float* __restrict__ act, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        if (!(act[i] > 0.0f)) d[i] = 0.0f;
}

// bias-corrected Adam (Kingma & Ba): bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi;
        float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float mh = mi / bc1, vh = vi / bc2;
        p[i] = p[i] - lr * mh / (sqrtf(vh) + eps);
    }
}

}  // namespace

// ---- training launches shared with the method's own network (rdn.cu) -------
mrs_status dw_tiles_f32(const float* x, int cin, int xs, const float* dy, int cout, int ys, int N,
                        int H, int W, int centre_only, float* part, float* dbpart, cudaStream_t st)
{
    const int ctiles = (cin + 63) / 64, otiles = (cout + 63) / 64;
    dim3 grid(kDwParts, centre_only ? 1 : 9, otiles * ctiles);
    k_dw_partial<float, float><<<grid, 256, 0, st>>>(x, cin, xs, dy, cout, ys, N, H, W, part, dbpart,
                                                     centre_only ? 4 : 0, ctiles);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "dw tiles");
}

void wtrans_f32(const float* w, int cin, int cout, float* wt, cudaStream_t st)
{
    int n = cin * 9 * cout;
    k_wtrans<<<(n + 255) / 256, 256, 0, st>>>(w, cin, cout, wt);
    MRS_LAUNCHED(1);
}

mrs_status loss_grad_f32(const float* y, const float* tgt, size_t n, float clip, int kind,
                         float beta, float* dy, double* parts, double* sum, cudaStream_t st)
{
    k_loss<<<kRedBlocks, 256, 0, st>>>(y, tgt, n, clip, kind, beta, dy, parts);
    MRS_LAUNCHED(1);
    k_reduce_parts<<<1, 256, 0, st>>>(parts, kRedBlocks, 1, sum);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "loss");
}

mrs_status adam_f32(float* p, const float* g, float* m, float* v, size_t n, float lr, int64_t step,
                    cudaStream_t st)
{
    const double b1 = 0.9, b2 = 0.999;
    float bc1 = (float)(1.0 - pow(b1, (double)step));
    float bc2 = (float)(1.0 - pow(b2, (double)step));
    size_t gsz = (n + 255) / 256;
    k_adam<<<(int)(gsz < 4096 ? (gsz ? gsz : 1) : 4096), 256, 0, st>>>(p, g, m, v, n, lr, (float)b1,
                                                                     (float)b2, 1e-8f, bc1, bc2);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "adam");
}

namespace {

// gate decision on the device: D = sum / count; use_plain = D > tau
__global__ void k_gate_decide(const double* part, int nparts, double count, double tau,
                              int use_plain_avail, int* used_plain, double* D)
{
    // the same fixed-order reduction as k_reduce_parts
    __shared__ double sh[256];
    double a = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double acc = sh[0];
        double d = acc / count;
        if (D) *D = d;
        int u = d > tau ? 1 : 0;
        used_plain[0] = u;
        used_plain[1] = u && use_plain_avail;     // whether `out` takes the plain render
    }
}

// out = plain if the gate chose it (and a plain render was given), else fused
__global__ void k_gate_select(const float* __restrict__ fused, const float* __restrict__ plain,
                              size_t n, const int* __restrict__ choice, float* __restrict__ out)
{
    const float* src = choice[1] != 0 ? plain : fused;
    if (src == out) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = src[i];
}

// transposed, tap-flipped weights of layer (cin, cout) packed as the
// tensor-core operand of dX = conv(dY): wp[t][c][o] = w[o][8 - t][c]
// (rows c < cin of nout, columns o < cout of 64, zero padded)
__global__ void k_pack_bf16_T(const float* __restrict__ master, size_t woff, int cin, int cout,
                              int nout, __nv_bfloat16* __restrict__ wp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * nout * 64) return;
    int o = i % 64, c = (i / 64) % nout, t = i / (64 * nout);
    float v = (c < cin && o < cout) ? master[woff + ((size_t)o * 9 + (8 - t)) * cin + c] : 0.0f;
    wp[i] = __float2bfloat16_rn(v);
}

// d[i] = act[i] > 0 ? d[i] : 0 over bf16 tensors
__global__ void k_mask_bf16(__nv_bfloat16* __restrict__ d, const __nv_bfloat16* __restrict__ act, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[i]) > 0.0f)) d[i] = __float2bfloat16_rn(0.0f);
}

// out[p][c] = float(o[p][c]) for c < cin from bf16 [P][64] rows
__global__ void k_from_operand(const __nv_bfloat16* __restrict__ o, size_t P, int cin,
                               float* __restrict__ out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * cin;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / cin;
        int c = (int)(i % cin);
        out[i] = __bfloat162float(o[p * 64 + c]);
    }
}

struct Scratch {
    std::mutex mu;
    Buf b;
};
Scratch& scratch()
{
    static Scratch s;
    return s;
}

}  // namespace
}  // namespace mrs

using namespace mrs;

struct mrs_net_s {
    int cin0 = 12;                 // input channels of the first conv (12 or 21)
    size_t np = kParams12;         // parameter count
    float* master = nullptr;       // [np]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    int64_t step = 0;
    __nv_bfloat16* wbf = nullptr;  // [18][9][64][64]
    uint8_t* wf8 = nullptr;        // [18][9][64][64]
    float* bias = nullptr;         // [18][64]
    float* bias8 = nullptr;        // [18][64]
    float* wscale = nullptr;       // [18][64]
    bool bf_valid = false, f8_valid = false;
    float xscale[kLayers];         // fp8 activation scales (calibrated)
    bool xscale_valid = false;
    CUtensorMap wmap_bf[kLayers], wmap_f8[kLayers], wmap_bfT[kLayers];
    __nv_bfloat16* wbfT = nullptr; // [18][9][64][64] transposed, tap-flipped (backward)
    bool bfT_valid = false;
    Buf act;                       // activation workspace
    Buf aux;                       // small device scratch
    Buf tact;                      // training activations
    Buf ttmp;                      // training scratch (transposed weights, dW partials, loss)
    int* err = nullptr;            // device error word
    int loss_kind = MRS_LOSS_L1LOG;
    float loss_beta = 0.1f;
};

namespace mrs {
namespace {

mrs_status pack_bf16(mrs_net_s* net, cudaStream_t st)
{
    if (net->bf_valid) return MRS_OK;
    const auto& L = shapes(net->cin0);
    for (int l = 0; l < kLayers; ++l) {
        int nout = nout_of(l);
        k_pack_bf16<<<(9 * nout * 64 + 255) / 256, 256, 0, st>>>(
            net->master, L[l].woff, L[l].boff, L[l].cin, L[l].cout, nout,
            net->wbf + (size_t)l * 9 * 64 * 64, net->bias + l * 64);
        MRS_LAUNCHED(1);
        mrs_status s = tc_make_w_map(&net->wmap_bf[l], net->wbf + (size_t)l * 9 * 64 * 64, 9 * nout, nout, TC_BF16);
        if (s != MRS_OK) return s;
    }
    net->bf_valid = true;
    return cuda_status(cudaGetLastError(), "pack bf16");
}

mrs_status pack_fp8(mrs_net_s* net, cudaStream_t st)
{
    if (net->f8_valid) return MRS_OK;
    const auto& L = shapes(net->cin0);
    for (int l = 0; l < kLayers; ++l) {
        int nout = nout_of(l);
        k_pack_fp8<<<1, 256, 0, st>>>(net->master, L[l].woff, L[l].boff, L[l].cin, L[l].cout, nout,
                                      net->wf8 + (size_t)l * 9 * 64 * 64, net->bias8 + l * 64,
                                      net->wscale + l * 64);
        MRS_LAUNCHED(1);
        mrs_status s = tc_make_w_map(&net->wmap_f8[l], net->wf8 + (size_t)l * 9 * 64 * 64, 9 * nout, nout, TC_FP8);
        if (s != MRS_OK) return s;
    }
    net->f8_valid = true;
    return cuda_status(cudaGetLastError(), "pack fp8");
}

mrs_status fuse_f32(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                    const float* nrm, const float* extra, int N, int H, int W, int s, float* out,
                    cudaStream_t st)
{
    size_t P = (size_t)N * H * W;
    const int c0 = net->cin0;
    mrs_status rc = net->act.ensure(P * (c0 + 64 + 64) * 4);
    if (rc != MRS_OK) return rc;
    float* x0 = net->act.as<float>();
    float* h = x0 + P * c0;
    float* r = h + P * 64;
    const auto& L = shapes(net->cin0);
    k_input_f32<<<(int)((P + 255) / 256 < 65535 ? (P + 255) / 256 : 65535), 256, 0, st>>>(
        lrhs, hrls, alb, nrm, extra, H, W, s, P, x0);
    MRS_LAUNCHED(1);
    rc = conv_simt(x0, c0, net->master + L[0].woff, net->master + L[0].boff, 64, SIMT_PLAIN, 1,
                   nullptr, h, nullptr, N, H, W, s, st);
    for (int k = 0; k < 8 && rc == MRS_OK; ++k) {
        const LayerShape& a = L[1 + 2 * k];
        const LayerShape& b = L[2 + 2 * k];
        rc = conv_simt(h, 64, net->master + a.woff, net->master + a.boff, 64, SIMT_PLAIN, 1,
                       nullptr, r, nullptr, N, H, W, s, st);
        if (rc == MRS_OK)
            rc = conv_simt(r, 64, net->master + b.woff, net->master + b.boff, 64, SIMT_RESID, 0, h,
                           h, nullptr, N, H, W, s, st);
    }
    if (rc == MRS_OK)
        rc = conv_simt(h, 64, net->master + L[17].woff, net->master + L[17].boff, 3, SIMT_FINAL, 0,
                       nullptr, out, lrhs, N, H, W, s, st);
    return rc;
}

mrs_status calibrate_fp8(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                         const float* nrm, const float* extra, int N, int H, int W, int s,
                         cudaStream_t st);

mrs_status fuse_tc(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                   const float* nrm, const float* extra, int N, int H, int W, int s, int prec, float* out,
                   cudaStream_t st, bool calib = false)
{
    size_t P = (size_t)N * H * W;
    const bool f8 = prec == MRS_PREC_FP8 && !calib;
    mrs_status rc = pack_bf16(net, st);
    if (rc != MRS_OK) return rc;
    if (f8) {
        if ((rc = pack_fp8(net, st)) != MRS_OK) return rc;
        if (!net->xscale_valid &&
            (rc = calibrate_fp8(net, lrhs, hrls, alb, nrm, extra, N, H, W, s, st)) != MRS_OK)
            return rc;
    }
    // workspace: x0, h, r in bf16 (128 B/px each); fp8 adds x0, h, r copies (64 B/px)
    size_t need = P * 128 * 3 + (f8 ? P * 64 * 3 : 0) + 1024;
    if ((rc = net->act.ensure(need)) != MRS_OK) return rc;
    uint8_t* base = net->act.as<uint8_t>();
    void* x0 = base;
    void* h = base + P * 128;
    void* r = base + P * 256;
    uint8_t* x08 = base + P * 384;
    uint8_t* h8 = x08 + P * 64;
    uint8_t* r8 = h8 + P * 64;
    int g = (int)((P + 255) / 256 < 65535 ? (P + 255) / 256 : 65535);
    k_input_q<<<g, 256, 0, st>>>(lrhs, hrls, alb, nrm, extra, H, W, s, P, f8 ? (void*)x08 : x0, f8 ? 1 : 0,
                                 f8 ? 1.0f / net->xscale[0] : 1.0f);
    MRS_LAUNCHED(1);
    if ((rc = cuda_status(cudaGetLastError(), "input")) != MRS_OK) return rc;
    // A-operand maps (bf16: 130-pixel halo boxes; fp8: 128) and the bf16
    // residual / output maps (128-pixel boxes)
    CUtensorMap mx, mh, mr, oh, orr;
    int oper = f8 ? TC_FP8 : TC_BF16;
    const int abox = tc_a_box(oper), obox = tc_out_box(oper);
    if ((rc = tc_make_act_map(&mx, f8 ? (void*)x08 : x0, N, H, W, oper, abox)) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&mh, f8 ? (void*)h8 : h, N, H, W, oper, abox)) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&mr, f8 ? (void*)r8 : r, N, H, W, oper, abox)) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&oh, h, N, H, W, TC_BF16, obox)) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&orr, r, N, H, W, TC_BF16, obox)) != MRS_OK) return rc;
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.H = H; a.W = W; a.scale = s;
    a.operand = oper;
    a.err = net->err;
    const int nl = calib ? kLayers - 1 : kLayers;
    for (int l = 0; l < nl && rc == MRS_OK; ++l) {
        a.tmap_w = f8 ? &net->wmap_f8[l] : &net->wmap_bf[l];
        a.bias = (f8 ? net->bias8 : net->bias) + l * 64;
        a.wscale = f8 ? net->wscale + l * 64 : nullptr;
        a.xscale = f8 ? net->xscale[l] : 1.0f;
        a.nout = nout_of(l);
        a.out_fp8 = nullptr;
        a.fp8_only = 0;
        a.tmap_res = nullptr;
        a.tmap_out = nullptr;
        if (l == 0) {
            a.tmap_x = &mx; a.mode = TC_RELU_BF16; a.out = h; a.res = nullptr; a.tmap_out = &oh;
            if (f8) { a.out_fp8 = h8; a.out_fp8_inv_scale = 1.0f / net->xscale[1]; }
        } else if (l == kLayers - 1) {
            a.tmap_x = &mh; a.mode = TC_FINAL_F32; a.out = out; a.lrhs = lrhs; a.cout = 3;
        } else if (l % 2 == 1) {
            a.tmap_x = &mh; a.mode = TC_RELU_BF16; a.out = r; a.res = nullptr; a.tmap_out = &orr;
            // r is read only as the next conv's operand: with fp8 operands
            // only its fp8 copy is written (not during calibration, which
            // measures the bf16 r)
            if (f8) { a.out_fp8 = r8; a.out_fp8_inv_scale = 1.0f / net->xscale[l + 1]; a.fp8_only = 1; }
        } else {
            a.tmap_x = &mr; a.mode = TC_RESID_BF16; a.out = h; a.res = h;
            a.tmap_res = &oh; a.tmap_out = &oh;
            if (f8) { a.out_fp8 = h8; a.out_fp8_inv_scale = 1.0f / net->xscale[l + 1]; }
        }
        rc = tc_conv3x3(a, st);
        if (calib && rc == MRS_OK && l < kLayers - 1) {
            // amax of the input of layer l + 1 (h after conv_in / blocks, r after conv1)
            const void* nxt = (l % 2 == 1) ? r : h;
            float* am = net->aux.as<float>() + l + 1;
            k_amax_bf16<<<512, 256, 0, st>>>((const __nv_bfloat16*)nxt, P * 64, am);
            MRS_LAUNCHED(1);
            rc = cuda_status(cudaGetLastError(), "amax");
        }
    }
    return rc;
}

// per-layer activation scales from one BF16 pass over the first input:
// xscale[l] = amax(input of layer l) / 448
mrs_status calibrate_fp8(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                         const float* nrm, const float* extra, int N, int H, int W, int s,
                         cudaStream_t st)
{
    mrs_status rc = net->aux.ensure(4096);
    if (rc != MRS_OK) return rc;
    MRS_CHECK(cudaMemsetAsync(net->aux.p, 0, 4096, st));
    size_t P = (size_t)N * H * W;
    rc = fuse_tc(net, lrhs, hrls, alb, nrm, extra, N, H, W, s, MRS_PREC_BF16, nullptr, st, true);
    (void)P;
    if (rc != MRS_OK) return rc;
    // layer 0 input: amax of the bf16 fusion input x0
    k_amax_bf16<<<512, 256, 0, st>>>(net->act.as<__nv_bfloat16>(), P * 64, net->aux.as<float>());
    MRS_LAUNCHED(1);
    float am[kLayers];
    MRS_CHECK(cudaMemcpyAsync(am, net->aux.p, sizeof(am), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    for (int l = 0; l < kLayers; ++l) net->xscale[l] = am[l] > 0.0f ? am[l] / 448.0f : 1.0f;
    net->xscale_valid = true;
    return MRS_OK;
}

}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_net_create(const float* params, int32_t n_params, mrs_net* out)
{
    MRS_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MRS_ARG(params != nullptr, "params is NULL");
    MRS_ARG(n_params == (int32_t)kParams12 || n_params == (int32_t)kParams21,
            "n_params must equal MRS_NET_NPARAMS or MRS_NET_NPARAMS_EXTRA");
    mrs_net_s* net = new mrs_net_s();
    net->np = (size_t)n_params;
    net->cin0 = n_params == (int32_t)kParams21 ? 21 : 12;
    mrs_status s = MRS_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (s == MRS_OK) s = cuda_status(cudaMalloc(p, bytes), "cudaMalloc(net)");
    };
    alloc((void**)&net->master, net->np * 4);
    alloc((void**)&net->adam_m, net->np * 4);
    alloc((void**)&net->adam_v, net->np * 4);
    alloc((void**)&net->grad, net->np * 4);
    alloc((void**)&net->wbf, (size_t)kLayers * 9 * 64 * 64 * 2);
    alloc((void**)&net->wbfT, (size_t)kLayers * 9 * 64 * 64 * 2);
    alloc((void**)&net->wf8, (size_t)kLayers * 9 * 64 * 64);
    alloc((void**)&net->bias, kLayers * 64 * 4);
    alloc((void**)&net->bias8, kLayers * 64 * 4);
    alloc((void**)&net->wscale, kLayers * 64 * 4);
    alloc((void**)&net->err, 4);
    if (s == MRS_OK) s = mrs_net_set_params(net, params);
    if (s != MRS_OK) { mrs_net_free(net); return s; }
    *out = net;
    return MRS_OK;
}

extern "C" mrs_status mrs_net_free(mrs_net net)
{
    if (!net) return MRS_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {net->master, net->adam_m, net->adam_v, net->grad, net->wbf, net->wbfT, net->wf8,
                    net->bias, net->bias8, net->wscale, net->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    net->act.release();
    net->aux.release();
    delete net;
    return MRS_OK;
}

extern "C" mrs_status mrs_net_set_params(mrs_net net, const float* params)
{
    MRS_ARG(net && params, "NULL argument");
    MRS_CHECK(cudaMemcpy(net->master, params, net->np * 4, cudaMemcpyHostToDevice));
    MRS_CHECK(cudaMemset(net->adam_m, 0, net->np * 4));
    MRS_CHECK(cudaMemset(net->adam_v, 0, net->np * 4));
    MRS_CHECK(cudaMemset(net->err, 0, 4));
    net->step = 0;
    net->bf_valid = net->f8_valid = net->xscale_valid = net->bfT_valid = false;
    return MRS_OK;
}

extern "C" mrs_status mrs_net_get_params(mrs_net net, float* params)
{
    MRS_ARG(net && params, "NULL argument");
    MRS_CHECK(cudaMemcpy(params, net->master, net->np * 4, cudaMemcpyDeviceToHost));
    return MRS_OK;
}

extern "C" mrs_status mrs_net_input_channels(mrs_net net, int32_t* channels)
{
    MRS_ARG(net && channels, "NULL argument");
    *channels = net->cin0;
    return MRS_OK;
}

extern "C" mrs_status mrs_fuse(mrs_net net, const float* lrhs, const float* hrls,
                               const float* albedo, const float* normal, int32_t N, int32_t H,
                               int32_t W, int32_t scale, int32_t precision, float* out, void* stream)
{
    return mrs_fuse_extra(net, lrhs, hrls, albedo, normal, nullptr, N, H, W, scale, precision, out,
                          stream);
}

extern "C" mrs_status mrs_fuse_extra(mrs_net net, const float* lrhs, const float* hrls,
                                     const float* albedo, const float* normal, const float* extra,
                                     int32_t N, int32_t H, int32_t W, int32_t scale,
                                     int32_t precision, float* out, void* stream)
{
    MRS_ARG(net != nullptr, "net is NULL");
    MRS_ARG(lrhs && hrls && albedo && normal && out, "NULL image pointer");
    MRS_ARG((extra != nullptr) == (net->cin0 == 21),
            "extra layers must be given exactly for a net with MRS_NET_NPARAMS_EXTRA parameters");
    MRS_ARG(scale == 1 || scale == 2 || scale == 4 || scale == 8, "scale must be 1, 2, 4 or 8");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1, "N, H, W must be >= 1");
    MRS_ARG(H % scale == 0 && W % scale == 0, "H and W must be multiples of scale");
    MRS_ARG((int64_t)N * H * W <= (int64_t(1) << 27), "N*H*W exceeds 2^27 pixels");
    MRS_ARG(precision >= MRS_PREC_FP32 && precision <= MRS_PREC_FP8, "precision");
    cudaStream_t st = (cudaStream_t)stream;
    mrs_status rc;
    if (precision == MRS_PREC_FP32)
        rc = fuse_f32(net, lrhs, hrls, albedo, normal, extra, N, H, W, scale, out, st);
    else
        rc = fuse_tc(net, lrhs, hrls, albedo, normal, extra, N, H, W, scale, precision, out, st);
    return rc;
}

extern "C" mrs_status mrs_image_metrics(const float* x, const float* ref, int64_t n, double l1,
                                        double l2, double* out, void* stream)
{
    MRS_ARG(x && ref && out, "NULL pointer");
    MRS_ARG(n >= 1, "n must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch& S = scratch();
    std::lock_guard<std::mutex> g(S.mu);
    mrs_status rc = S.b.ensure(sizeof(double) * (kRedBlocks * 3 + 8));
    if (rc != MRS_OK) return rc;
    double* part = S.b.as<double>();
    double* res = part + kRedBlocks * 3;
    k_metrics_partial<<<kRedBlocks, 256, 0, st>>>(x, ref, n, l1, l2, part);
    MRS_LAUNCHED(1);
    k_reduce_parts<<<1, 256, 0, st>>>(part, kRedBlocks, 3, res);
    MRS_LAUNCHED(1);
    double h[3];
    MRS_CHECK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    double mse_s = h[0] / (double)n;
    out[0] = mse_s == 0.0 ? INFINITY : 10.0 * log10(1.0 / mse_s);
    out[1] = h[1] / (double)n;
    out[2] = h[2] / (double)n;
    return MRS_OK;
}

extern "C" mrs_status mrs_gate(const float* fused, const float* lrhs, const float* plain,
                               int32_t N, int32_t H, int32_t W, int32_t scale, double tau,
                               float* out, int32_t* used_plain, double* D, void* stream)
{
    MRS_ARG(fused && lrhs, "NULL pointer");
    MRS_ARG(scale >= 1 && N >= 1 && H >= scale && W >= scale && H % scale == 0 && W % scale == 0,
            "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch& S = scratch();
    std::lock_guard<std::mutex> g(S.mu);
    mrs_status rc = S.b.ensure(sizeof(double) * (kRedBlocks + 8));
    if (rc != MRS_OK) return rc;
    double* part = S.b.as<double>();
    double* res = part + kRedBlocks;
    k_gate_partial<<<kRedBlocks, 256, 0, st>>>(fused, lrhs, N, H, W, scale, part);
    MRS_LAUNCHED(1);
    k_reduce_parts<<<1, 256, 0, st>>>(part, kRedBlocks, 1, res);
    MRS_LAUNCHED(1);
    double d;
    MRS_CHECK(cudaMemcpyAsync(&d, res, sizeof(d), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    d /= (double)N * (H / scale) * (W / scale) * 3;
    bool use_plain = d > tau;
    if (D) *D = d;
    if (used_plain) *used_plain = use_plain ? 1 : 0;
    size_t bytes = (size_t)N * H * W * 3 * 4;
    if (out) {
        const float* src = (use_plain && plain) ? plain : fused;
        if (src != out) MRS_CHECK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, st));
    }
    return MRS_OK;
}

namespace mrs {
namespace {
// BF16 3x3 conv over more than 64 input channels: the input is split into
// 64-channel operand tensors and ONE tensor-core launch accumulates all of
// them (multi-chunk conv, chunk maps passed in device memory)
mrs_status conv3x3_chunked(Scratch& S, const float* x, int N, int H, int W, int cin, int cout,
                           const float* w, const float* b, int relu, float* out, cudaStream_t st)
{
    const size_t P = (size_t)N * H * W;
    const int nch = (cin + 63) / 64;
    const int nout = cout > 16 ? 64 : 16;
    const size_t wbytes = (size_t)cout * 9 * cin * 4;
    const size_t chunk_el = (size_t)9 * nout * 64;               // packed bf16 weights per chunk
    const size_t wpk_bytes = ((nch * chunk_el * 2 + 1023) / 1024) * 1024;
    const size_t xq_bytes = ((P * 128 + 1023) / 1024) * 1024;    // one [P][64] bf16 operand
    size_t need = wbytes + 64 * 4 + 1024 + wpk_bytes + nch * xq_bytes + nch * sizeof(CUtensorMap) + 1024;
    mrs_status rc = S.b.ensure(need);
    if (rc != MRS_OK) return rc;
    uint8_t* base = S.b.as<uint8_t>();
    float* dw = (float*)base;
    float* db = dw + (size_t)cout * 9 * cin;
    uint8_t* wpk = (uint8_t*)(((uintptr_t)(db + 64) + 1023) & ~(uintptr_t)1023);
    uint8_t* xq = wpk + wpk_bytes;
    CUtensorMap* dmaps = (CUtensorMap*)(xq + nch * xq_bytes);
    MRS_CHECK(cudaMemsetAsync(db, 0, 64 * 4, st));
    MRS_CHECK(cudaMemcpyAsync(dw, w, wbytes, cudaMemcpyHostToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(db, b, cout * 4, cudaMemcpyHostToDevice, st));
    static int* err = nullptr;
    if (!err) { MRS_CHECK(cudaMalloc(&err, 4)); MRS_CHECK(cudaMemset(err, 0, 4)); }
    std::vector<CUtensorMap> hm(nch);
    for (int j = 0; j < nch; ++j) {
        k_pack_bf16_chunk<<<(9 * nout * 64 + 255) / 256, 256, 0, st>>>(
            dw, cin, 64 * j, cout, nout, (__nv_bfloat16*)wpk + j * chunk_el);
        MRS_LAUNCHED(1);
        __nv_bfloat16* xj = (__nv_bfloat16*)(xq + j * xq_bytes);
        k_to_operand_chunk<<<1024, 256, 0, st>>>(x, P, cin, 64 * j, xj);
        MRS_LAUNCHED(1);
        if ((rc = tc_make_act_map(&hm[j], xj, N, H, W, TC_BF16, tc_a_box(TC_BF16))) != MRS_OK) return rc;
    }
    CUtensorMap wm;
    if ((rc = tc_make_w_map(&wm, wpk, nch * 9 * nout, nout, TC_BF16)) != MRS_OK) return rc;
    MRS_CHECK(cudaMemcpyAsync(dmaps, hm.data(), nch * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.tmap_x = &hm[0]; a.tmap_w = &wm; a.amaps = dmaps; a.kc = nch; a.w_row0 = 0;
    a.bias = db; a.out = out; a.N = N; a.H = H; a.W = W; a.scale = 1; a.nout = nout;
    a.cout = cout; a.relu = relu; a.mode = TC_PLAIN_F32; a.operand = TC_BF16; a.err = err;
    rc = tc_conv3x3(a, st);
    // the host map array and the scratch stay valid until the stream is synchronised
    if (rc == MRS_OK) rc = cuda_status(cudaStreamSynchronize(st), "conv3x3 sync");
    int herr = 0;
    if (rc == MRS_OK) {
        MRS_CHECK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
        if (herr) { cudaMemset(err, 0, 4); set_error("tensor-core conv wait timed out"); return MRS_ERR_TIMEOUT; }
    }
    return rc;
}
}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_conv3x3(const float* x, int32_t N, int32_t H, int32_t W, int32_t cin,
                                  int32_t cout, const float* w, const float* b, int32_t relu,
                                  int32_t precision, float* out, void* stream)
{
    MRS_ARG(x && w && b && out, "NULL pointer");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1 && cin >= 1 && cout >= 1, "sizes must be >= 1");
    MRS_ARG(precision == MRS_PREC_FP32 || cout <= 64, "tensor-core conv needs cout <= 64");
    MRS_ARG(precision == MRS_PREC_FP32 || cin <= 64 || (precision == MRS_PREC_BF16 && cin <= 1024),
            "tensor-core conv needs cin <= 64 (FP8) or cin <= 1024 (BF16)");
    cudaStream_t st = (cudaStream_t)stream;
    size_t P = (size_t)N * H * W;
    Scratch& S = scratch();
    std::lock_guard<std::mutex> g(S.mu);
    if (precision == MRS_PREC_BF16 && cin > 64)
        return conv3x3_chunked(S, x, N, H, W, cin, cout, w, b, relu, out, st);
    size_t wbytes = (size_t)cout * 9 * cin * 4;
    size_t need = wbytes + cout * 4 + 9 * 64 * 64 * 2 + 64 * 4 * 2 + 1024 +
                  (precision == MRS_PREC_FP32 ? 0 : P * 128) + 16;
    mrs_status rc = S.b.ensure(need);
    if (rc != MRS_OK) return rc;
    uint8_t* base = S.b.as<uint8_t>();
    float* dw = (float*)base;
    float* db = dw + (size_t)cout * 9 * cin;
    uint8_t* q = (uint8_t*)(((uintptr_t)(db + cout) + 255) & ~(uintptr_t)255);
    MRS_CHECK(cudaMemcpyAsync(dw, w, wbytes, cudaMemcpyHostToDevice, st));
    MRS_CHECK(cudaMemcpyAsync(db, b, cout * 4, cudaMemcpyHostToDevice, st));
    if (precision == MRS_PREC_FP32) {
        rc = conv_simt(x, cin, dw, db, cout, SIMT_PLAIN, relu, nullptr, out, nullptr, N, H, W, 1, st);
        if (rc == MRS_OK) rc = cuda_status(cudaStreamSynchronize(st), "conv3x3 sync");
        return rc;
    }
    // tensor cores: pack weights and input into the operand format
    int nout = cout > 16 ? 64 : 16;
    int oper = precision == MRS_PREC_BF16 ? TC_BF16 : TC_FP8;
    void* wp = q;
    float* bp = (float*)(q + 9 * 64 * 64 * 2);
    float* ws = bp + 64;
    float* amax_slot = ws + 64;   // one float, then the operand buffer (1024-aligned)
    void* xq = (void*)(((uintptr_t)(amax_slot + 4) + 1023) & ~(uintptr_t)1023);
    static int* err = nullptr;
    if (!err) { MRS_CHECK(cudaMalloc(&err, 4)); MRS_CHECK(cudaMemset(err, 0, 4)); }
    float xscale = 1.0f;
    if (oper == TC_BF16) {
        k_pack_bf16<<<(9 * nout * 64 + 255) / 256, 256, 0, st>>>(dw, 0, (size_t)cout * 9 * cin, cin, cout, nout,
                                                                 (__nv_bfloat16*)wp, bp);
        MRS_LAUNCHED(1);
    } else {
        k_pack_fp8<<<1, 256, 0, st>>>(dw, 0, (size_t)cout * 9 * cin, cin, cout, nout, (uint8_t*)wp, bp, ws);
        MRS_LAUNCHED(1);
    }
    // input conversion: x fp32 [P][cin] -> [P][64] operand rows (fp8: per-tensor
    // scale amax / 448, computed on the device)
    if (oper == TC_FP8) {
        float* amax = amax_slot;
        MRS_CHECK(cudaMemsetAsync(amax, 0, 4, st));
        k_amax_f32<<<512, 256, 0, st>>>(x, P * cin, amax);
        MRS_LAUNCHED(1);
        float hm = 0;
        MRS_CHECK(cudaMemcpyAsync(&hm, amax, 4, cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        xscale = hm > 0 ? hm / 448.0f : 1.0f;
    }
    k_to_operand<<<1024, 256, 0, st>>>(x, P, cin, xq, oper == TC_FP8, 1.0f / xscale);
    MRS_LAUNCHED(1);
    CUtensorMap mx, mw;
    if ((rc = tc_make_act_map(&mx, xq, N, H, W, oper, tc_a_box(oper))) != MRS_OK) return rc;
    if ((rc = tc_make_w_map(&mw, wp, 9 * nout, nout, oper)) != MRS_OK) return rc;
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.tmap_x = &mx; a.tmap_w = &mw; a.bias = bp; a.wscale = ws; a.xscale = xscale;
    a.out = out; a.N = N; a.H = H; a.W = W; a.scale = 1; a.nout = nout; a.cout = cout;
    a.relu = relu; a.mode = TC_PLAIN_F32; a.operand = oper; a.err = err;
    rc = tc_conv3x3(a, st);
    if (rc == MRS_OK) rc = cuda_status(cudaStreamSynchronize(st), "conv3x3 sync");
    int herr = 0;
    if (rc == MRS_OK) {
        MRS_CHECK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
        if (herr) { cudaMemset(err, 0, 4); set_error("tensor-core conv wait timed out"); return MRS_ERR_TIMEOUT; }
    }
    return rc;
}


namespace mrs {
namespace {

constexpr int kDwSplits = 64;
constexpr float kClip = 100.0f;

__global__ void k_clip_copy(const float* __restrict__ x, size_t n, float clip, float* __restrict__ y)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        y[i] = fminf(x[i], clip);
}

inline int grid1d(size_t n) { size_t g = (n + 255) / 256; return (int)(g < 4096 ? (g ? g : 1) : 4096); }

// dW / db of layer l from its input x [P][cin] and output gradient dy [P][cout]
mrs_status layer_dw(mrs_net_s* net, int l, const float* x, const float* dy, int N, int H, int W,
                    float* part, float* dbpart, cudaStream_t st)
{
    const LayerShape& L = shapes(net->cin0)[l];
    dim3 grid(kDwSplits, 9);
    MRS_TIMED(PK_TRAIN, st, (k_dw_partial<float, float><<<grid, 256, 0, st>>>(x, L.cin, L.cin, dy, L.cout, L.cout, N, H, W, part, dbpart, 0, 1)));
    MRS_LAUNCHED(1);
    int nw = L.cout * 9 * L.cin + L.cout;
    MRS_TIMED(PK_TRAIN, st, k_dw_reduce<<<(nw + 31) / 32, 256, 0, st>>>(part, dbpart, kDwSplits, L.cin, L.cout,
                                                         net->grad + L.woff, net->grad + L.boff));
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "dw");
}

// transposed conv of layer l: dx [P][cin] = conv(dy [P][cout], flipped w^T), epilogue `mode`
mrs_status layer_dx(mrs_net_s* net, int l, const float* dy, float* wt, const float* zero,
                    int mode, const float* res, float* dx, int N, int H, int W, cudaStream_t st)
{
    const LayerShape& L = shapes(net->cin0)[l];
    int n = L.cin * 9 * L.cout;
    k_wtrans<<<(n + 255) / 256, 256, 0, st>>>(net->master + L.woff, L.cin, L.cout, wt);
    MRS_LAUNCHED(1);
    return conv_simt(dy, L.cout, wt, zero, L.cin, mode, 0, res, dx, nullptr, N, H, W, 1, st);
}

mrs_status train_step_f32(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                          const float* nrm, const float* extra, const float* target, int N, int H,
                          int W, int s, float lr, double* loss_out, cudaStream_t st)
{
    const int c0 = net->cin0;
    const size_t P = (size_t)N * H * W;
    const size_t F = P * 64;
    const size_t nlr = (size_t)N * (H / s) * (W / s) * 3;
    // activations: x0 | h0..h8 | r0..r7 | y | dy | dh | da | lrhs_clipped
    size_t need = (P * c0 + 9 * F + 8 * F + 2 * P * 3 + 2 * F + nlr) * 4;
    mrs_status rc = net->tact.ensure(need);
    if (rc != MRS_OK) return rc;
    size_t tneed = (64 * 9 * 64 + 64) * 4 + ((size_t)kDwSplits * 9 * 64 * 64 + kDwSplits * 64) * 4 +
                   (kRedBlocks + 8) * 8;
    if ((rc = net->ttmp.ensure(tneed)) != MRS_OK) return rc;
    float* x0 = net->tact.as<float>();
    float* hs = x0 + P * c0;
    float* rs = hs + 9 * F;
    float* y = rs + 8 * F;
    float* dy = y + P * 3;
    float* dh = dy + P * 3;
    float* da = dh + F;
    float* lrc = da + F;
    float* wt = net->ttmp.as<float>();
    float* zero = wt + 64 * 9 * 64;
    float* part = zero + 64;
    float* dbpart = part + (size_t)kDwSplits * 9 * 64 * 64;
    double* lparts = (double*)(dbpart + kDwSplits * 64);
    double* lres = lparts + kRedBlocks;
    MRS_CHECK(cudaMemsetAsync(zero, 0, 64 * 4, st));
    const auto& L = shapes(net->cin0);
    const float* M = net->master;

    // forward, keeping every activation the backward needs
    k_clip_copy<<<grid1d(nlr), 256, 0, st>>>(lrhs, nlr, kClip, lrc);
    MRS_LAUNCHED(1);
    k_input_f32<<<grid1d(P), 256, 0, st>>>(lrc, hrls, alb, nrm, extra, H, W, s, P, x0, kClip);
    MRS_LAUNCHED(1);
    rc = conv_simt(x0, c0, M + L[0].woff, M + L[0].boff, 64, SIMT_PLAIN, 1, nullptr, hs, nullptr, N, H, W, s, st);
    for (int k = 0; k < 8 && rc == MRS_OK; ++k) {
        const LayerShape& a = L[1 + 2 * k];
        const LayerShape& b = L[2 + 2 * k];
        rc = conv_simt(hs + k * F, 64, M + a.woff, M + a.boff, 64, SIMT_PLAIN, 1, nullptr, rs + k * F,
                       nullptr, N, H, W, s, st);
        if (rc == MRS_OK)
            rc = conv_simt(rs + k * F, 64, M + b.woff, M + b.boff, 64, SIMT_RESID, 0, hs + k * F,
                           hs + (k + 1) * F, nullptr, N, H, W, s, st);
    }
    if (rc == MRS_OK)
        rc = conv_simt(hs + 8 * F, 64, M + L[17].woff, M + L[17].boff, 3, SIMT_FINAL, 0, nullptr, y, lrc,
                       N, H, W, s, st);
    if (rc != MRS_OK) return rc;

    // loss (float64 reduction) and dL/dy
    MRS_TIMED(PK_TRAIN, st, k_loss<<<kRedBlocks, 256, 0, st>>>(y, target, P * 3, kClip, net->loss_kind,
                                                               net->loss_beta, dy, lparts));
    MRS_LAUNCHED(1);
    k_reduce_parts<<<1, 256, 0, st>>>(lparts, kRedBlocks, 1, lres);
    MRS_LAUNCHED(1);

    // backward
    if ((rc = layer_dw(net, 17, hs + 8 * F, dy, N, H, W, part, dbpart, st)) != MRS_OK) return rc;
    if ((rc = layer_dx(net, 17, dy, wt, zero, SIMT_PLAIN, nullptr, dh, N, H, W, st)) != MRS_OK) return rc;
    for (int k = 7; k >= 0; --k) {
        int l2 = 2 + 2 * k, l1 = 1 + 2 * k;
        if ((rc = layer_dw(net, l2, rs + k * F, dh, N, H, W, part, dbpart, st)) != MRS_OK) return rc;
        if ((rc = layer_dx(net, l2, dh, wt, zero, SIMT_MASK, rs + k * F, da, N, H, W, st)) != MRS_OK) return rc;
        if ((rc = layer_dw(net, l1, hs + k * F, da, N, H, W, part, dbpart, st)) != MRS_OK) return rc;
        if ((rc = layer_dx(net, l1, da, wt, zero, SIMT_RESID, dh, dh, N, H, W, st)) != MRS_OK) return rc;
    }
    k_mask_inplace<<<grid1d(F), 256, 0, st>>>(dh, hs, F);
    MRS_LAUNCHED(1);
    if ((rc = layer_dw(net, 0, x0, dh, N, H, W, part, dbpart, st)) != MRS_OK) return rc;

    // Adam on the FP32 master weights
    net->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    float bc1 = (float)(1.0 - pow(b1, (double)net->step));
    float bc2 = (float)(1.0 - pow(b2, (double)net->step));
    MRS_TIMED(PK_TRAIN, st, k_adam<<<grid1d(net->np), 256, 0, st>>>(net->master, net->grad, net->adam_m, net->adam_v,
                                                        net->np, lr, (float)b1, (float)b2, 1e-8f, bc1, bc2));
    MRS_LAUNCHED(1);
    net->bf_valid = net->f8_valid = net->xscale_valid = net->bfT_valid = false;
    if (loss_out) {
        double h = 0;
        MRS_CHECK(cudaMemcpyAsync(&h, lres, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        *loss_out = h / (double)(P * 3);
    }
    return cuda_status(cudaGetLastError(), "train step");
}

mrs_status pack_bf16_T(mrs_net_s* net, cudaStream_t st)
{
    if (net->bfT_valid) return MRS_OK;
    const auto& L = shapes(net->cin0);
    for (int l = 1; l < kLayers; ++l) {
        __nv_bfloat16* wp = net->wbfT + (size_t)l * 9 * 64 * 64;
        k_pack_bf16_T<<<(9 * 64 * 64 + 255) / 256, 256, 0, st>>>(net->master, L[l].woff, L[l].cin,
                                                                 L[l].cout, 64, wp);
        MRS_LAUNCHED(1);
        mrs_status rc = tc_make_w_map(&net->wmap_bfT[l], wp, 9 * 64, 64, TC_BF16);
        if (rc != MRS_OK) return rc;
    }
    net->bfT_valid = true;
    return cuda_status(cudaGetLastError(), "pack bf16 T");
}

// BF16 training step: forward and transposed convolutions on the tensor-core
// kernel with BF16 activations / activation gradients, FP32 accumulation,
// FP32 dW / db reductions and FP32 master weights + Adam
mrs_status train_step_bf16(mrs_net_s* net, const float* lrhs, const float* hrls, const float* alb,
                           const float* nrm, const float* extra, const float* target, int N, int H,
                           int W, int s, float lr, double* loss_out, cudaStream_t st)
{
    const size_t P = (size_t)N * H * W;
    const size_t F = P * 64;                       // bf16 elements of one [P][64] tensor
    const size_t nlr = (size_t)N * (H / s) * (W / s) * 3;
    size_t need = (size_t)(1 + 9 + 8 + 3) * F * 2 + (2 * P * 3 + nlr + P * 3) * 4 + 4096;
    mrs_status rc = net->tact.ensure(need);
    if (rc != MRS_OK) return rc;
    const size_t maxp = (size_t)std::max(kDwSplits, tc_wgrad_max_parts());
    size_t tneed = (64 * 9 * 64 + 64) * 4 + (maxp * 9 * 64 * 64 + maxp * 64) * 4 + (kRedBlocks + 8) * 8;
    if ((rc = net->ttmp.ensure(tneed)) != MRS_OK) return rc;
    if ((rc = pack_bf16(net, st)) != MRS_OK) return rc;
    if ((rc = pack_bf16_T(net, st)) != MRS_OK) return rc;
    __nv_bfloat16* x0 = net->tact.as<__nv_bfloat16>();
    __nv_bfloat16* hs = x0 + F;
    __nv_bfloat16* rs = hs + 9 * F;
    __nv_bfloat16* dyb = rs + 8 * F;
    __nv_bfloat16* dh = dyb + F;
    __nv_bfloat16* da = dh + F;
    float* y = (float*)(da + F);
    float* dy = y + P * 3;
    float* lrc = dy + P * 3;
    float* hrc = lrc + nlr;
    float* zero = net->ttmp.as<float>() + 64 * 9 * 64;
    float* part = zero + 64;
    float* dbpart = part + maxp * 9 * 64 * 64;
    double* lparts = (double*)(dbpart + maxp * 64);
    double* lres = lparts + kRedBlocks;
    MRS_CHECK(cudaMemsetAsync(zero, 0, 64 * 4, st));
    const auto& L = shapes(net->cin0);

    // tensor maps: A operands (130-pixel boxes) and residual / output (128-pixel)
    auto amap = [&](CUtensorMap* m, const void* ptr) { return tc_make_act_map(m, ptr, N, H, W, TC_BF16, tc_a_box(TC_BF16)); };
    auto omap = [&](CUtensorMap* m, const void* ptr) { return tc_make_act_map(m, ptr, N, H, W, TC_BF16, tc_out_box(TC_BF16)); };
    std::vector<CUtensorMap> hA(9), hO(9), rA(8), rO(8);
    CUtensorMap x0A, dybA, dhA, dhO, daA, daO;
    for (int k = 0; k < 9 && rc == MRS_OK; ++k) {
        if ((rc = amap(&hA[k], hs + k * F)) == MRS_OK) rc = omap(&hO[k], hs + k * F);
        if (k < 8 && rc == MRS_OK) { if ((rc = amap(&rA[k], rs + k * F)) == MRS_OK) rc = omap(&rO[k], rs + k * F); }
    }
    if (rc == MRS_OK) rc = amap(&x0A, x0);
    if (rc == MRS_OK) rc = amap(&dybA, dyb);
    if (rc == MRS_OK) rc = amap(&dhA, dh);
    if (rc == MRS_OK) rc = omap(&dhO, dh);
    if (rc == MRS_OK) rc = amap(&daA, da);
    if (rc == MRS_OK) rc = omap(&daO, da);
    // weight-gradient operands: x rows with a one-pixel halo, dy rows
    auto xwmap = [&](CUtensorMap* m, const void* ptr) { return tc_make_act_map(m, ptr, N, H, W, TC_BF16, kWgKB + 2); };
    auto dwmap = [&](CUtensorMap* m, const void* ptr) { return tc_make_act_map(m, ptr, N, H, W, TC_BF16, kWgKB); };
    std::vector<CUtensorMap> hX(9), rX(8);
    CUtensorMap x0X, dybD, dhD, daD;
    for (int k = 0; k < 9 && rc == MRS_OK; ++k) {
        rc = xwmap(&hX[k], hs + k * F);
        if (k < 8 && rc == MRS_OK) rc = xwmap(&rX[k], rs + k * F);
    }
    if (rc == MRS_OK) rc = xwmap(&x0X, x0);
    if (rc == MRS_OK) rc = dwmap(&dybD, dyb);
    if (rc == MRS_OK) rc = dwmap(&dhD, dh);
    if (rc == MRS_OK) rc = dwmap(&daD, da);
    if (rc != MRS_OK) return rc;
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.H = H; a.W = W; a.scale = s; a.operand = TC_BF16; a.err = net->err; a.nout = 64;
    auto conv = [&](const CUtensorMap* A, const CUtensorMap* Wm, const float* bias, int mode,
                    const CUtensorMap* res, const CUtensorMap* out, int nout) {
        a.tmap_x = A; a.tmap_w = Wm; a.bias = bias; a.mode = mode; a.tmap_res = res;
        a.tmap_out = out; a.nout = nout;
        return tc_conv3x3(a, st);
    };

    // forward
    k_clip_copy<<<grid1d(nlr), 256, 0, st>>>(lrhs, nlr, kClip, lrc);
    MRS_LAUNCHED(1);
    k_clip_copy<<<grid1d(P * 3), 256, 0, st>>>(hrls, P * 3, kClip, hrc);
    MRS_LAUNCHED(1);
    k_input_q<<<grid1d(P), 256, 0, st>>>(lrc, hrc, alb, nrm, extra, H, W, s, P, x0, 0, 1.0f, kClip);
    MRS_LAUNCHED(1);
    rc = conv(&x0A, &net->wmap_bf[0], net->bias, TC_RELU_BF16, nullptr, &hO[0], 64);
    for (int k = 0; k < 8 && rc == MRS_OK; ++k) {
        rc = conv(&hA[k], &net->wmap_bf[1 + 2 * k], net->bias + (1 + 2 * k) * 64, TC_RELU_BF16,
                  nullptr, &rO[k], 64);
        if (rc == MRS_OK)
            rc = conv(&rA[k], &net->wmap_bf[2 + 2 * k], net->bias + (2 + 2 * k) * 64, TC_RESID_BF16,
                      &hO[k], &hO[k + 1], 64);
    }
    if (rc == MRS_OK) {
        a.out = y; a.lrhs = lrc; a.cout = 3;
        rc = conv(&hA[8], &net->wmap_bf[17], net->bias + 17 * 64, TC_FINAL_F32, nullptr, nullptr, 16);
    }
    if (rc != MRS_OK) return rc;

    // loss
    MRS_TIMED(PK_TRAIN, st, k_loss<<<kRedBlocks, 256, 0, st>>>(y, target, P * 3, kClip, net->loss_kind,
                                                               net->loss_beta, dy, lparts));
    MRS_LAUNCHED(1);
    k_reduce_parts<<<1, 256, 0, st>>>(lparts, kRedBlocks, 1, lres);
    MRS_LAUNCHED(1);

    // backward: weight gradients on the tensor cores (per-CTA partials, then a
    // deterministic reduction), data gradients as convs with the flipped,
    // transposed weights
    auto dw = [&](int l, const CUtensorMap* xm, const CUtensorMap* dym) {
        const LayerShape& S_ = L[l];
        TcWgradArgs wa;
        wa.tmap_x = xm; wa.tmap_dy = dym; wa.part = part; wa.dbpart = dbpart;
        wa.N = N; wa.H = H; wa.W = W; wa.cin = S_.cin; wa.cout = S_.cout; wa.err = net->err;
        int np = 0;
        mrs_status r = tc_conv3x3_wgrad(wa, &np, st);
        if (r != MRS_OK) return r;
        int nw = S_.cout * 9 * S_.cin + S_.cout;
        MRS_TIMED(PK_TRAIN, st, k_dw_reduce<<<(nw + 31) / 32, 256, 0, st>>>(part, dbpart, np, S_.cin, S_.cout,
                                                       net->grad + S_.woff, net->grad + S_.boff));
        MRS_LAUNCHED(1);
        return cuda_status(cudaGetLastError(), "dw");
    };
    k_to_operand<<<1024, 256, 0, st>>>(dy, P, 3, dyb, 0, 1.0f);
    MRS_LAUNCHED(1);
    if ((rc = dw(17, &hX[8], &dybD)) != MRS_OK) return rc;
    if ((rc = conv(&dybA, &net->wmap_bfT[17], zero, TC_LIN_BF16, nullptr, &dhO, 64)) != MRS_OK) return rc;
    for (int k = 7; k >= 0; --k) {
        int l2 = 2 + 2 * k, l1 = 1 + 2 * k;
        if ((rc = dw(l2, &rX[k], &dhD)) != MRS_OK) return rc;
        if ((rc = conv(&dhA, &net->wmap_bfT[l2], zero, TC_MASK_BF16, &rO[k], &daO, 64)) != MRS_OK) return rc;
        if ((rc = dw(l1, &hX[k], &daD)) != MRS_OK) return rc;
        if ((rc = conv(&daA, &net->wmap_bfT[l1], zero, TC_RESID_BF16, &dhO, &dhO, 64)) != MRS_OK) return rc;
    }
    k_mask_bf16<<<grid1d(F), 256, 0, st>>>(dh, hs, F);
    MRS_LAUNCHED(1);
    if ((rc = dw(0, &x0X, &dhD)) != MRS_OK) return rc;

    // Adam on the FP32 master weights
    net->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    float bc1 = (float)(1.0 - pow(b1, (double)net->step));
    float bc2 = (float)(1.0 - pow(b2, (double)net->step));
    MRS_TIMED(PK_TRAIN, st, k_adam<<<grid1d(net->np), 256, 0, st>>>(net->master, net->grad, net->adam_m, net->adam_v,
                                                        net->np, lr, (float)b1, (float)b2, 1e-8f, bc1, bc2));
    MRS_LAUNCHED(1);
    net->bf_valid = net->f8_valid = net->xscale_valid = net->bfT_valid = false;
    if (loss_out) {
        double h = 0;
        MRS_CHECK(cudaMemcpyAsync(&h, lres, sizeof(double), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        *loss_out = h / (double)(P * 3);
    }
    return cuda_status(cudaGetLastError(), "train step bf16");
}

}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_train_step(mrs_net net, const float* lrhs, const float* hrls,
                                     const float* albedo, const float* normal, const float* target,
                                     int32_t N, int32_t H, int32_t W, int32_t scale, float lr,
                                     int32_t precision, double* loss_out, void* stream)
{
    return mrs_train_step_extra(net, lrhs, hrls, albedo, normal, nullptr, target, N, H, W, scale,
                                lr, precision, loss_out, stream);
}

extern "C" mrs_status mrs_train_step_extra(mrs_net net, const float* lrhs, const float* hrls,
                                           const float* albedo, const float* normal,
                                           const float* extra, const float* target, int32_t N,
                                           int32_t H, int32_t W, int32_t scale, float lr,
                                           int32_t precision, double* loss_out, void* stream)
{
    MRS_ARG(net != nullptr, "net is NULL");
    MRS_ARG(lrhs && hrls && albedo && normal && target, "NULL image pointer");
    MRS_ARG((extra != nullptr) == (net->cin0 == 21),
            "extra layers must be given exactly for a net with MRS_NET_NPARAMS_EXTRA parameters");
    MRS_ARG(scale == 1 || scale == 2 || scale == 4 || scale == 8, "scale must be 1, 2, 4 or 8");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1 && H % scale == 0 && W % scale == 0, "bad sizes");
    MRS_ARG((int64_t)N * H * W <= (int64_t(1) << 22), "training batch exceeds 2^22 pixels");
    MRS_ARG(lr >= 0.0f, "lr < 0");
    MRS_ARG(precision == MRS_PREC_FP32 || precision == MRS_PREC_BF16,
            "training precision must be MRS_PREC_FP32 or MRS_PREC_BF16");
    if (precision == MRS_PREC_BF16)
        return train_step_bf16(net, lrhs, hrls, albedo, normal, extra, target, N, H, W, scale, lr,
                               loss_out, (cudaStream_t)stream);
    return train_step_f32(net, lrhs, hrls, albedo, normal, extra, target, N, H, W, scale, lr,
                          loss_out, (cudaStream_t)stream);
}

extern "C" mrs_status mrs_net_get_grads(mrs_net net, float* grads)
{
    MRS_ARG(net && grads, "NULL argument");
    MRS_CHECK(cudaMemcpy(grads, net->grad, net->np * 4, cudaMemcpyDeviceToHost));
    return MRS_OK;
}

extern "C" mrs_status mrs_net_get_state(mrs_net net, float* params, float* adam_m, float* adam_v,
                                        int64_t* step)
{
    MRS_ARG(net && params && adam_m && adam_v && step, "NULL argument");
    MRS_CHECK(cudaMemcpy(params, net->master, net->np * 4, cudaMemcpyDeviceToHost));
    MRS_CHECK(cudaMemcpy(adam_m, net->adam_m, net->np * 4, cudaMemcpyDeviceToHost));
    MRS_CHECK(cudaMemcpy(adam_v, net->adam_v, net->np * 4, cudaMemcpyDeviceToHost));
    *step = net->step;
    return MRS_OK;
}

extern "C" mrs_status mrs_net_set_state(mrs_net net, const float* params, const float* adam_m,
                                        const float* adam_v, int64_t step)
{
    MRS_ARG(net && params && adam_m && adam_v, "NULL argument");
    MRS_ARG(step >= 0, "step < 0");
    MRS_CHECK(cudaMemcpy(net->master, params, net->np * 4, cudaMemcpyHostToDevice));
    MRS_CHECK(cudaMemcpy(net->adam_m, adam_m, net->np * 4, cudaMemcpyHostToDevice));
    MRS_CHECK(cudaMemcpy(net->adam_v, adam_v, net->np * 4, cudaMemcpyHostToDevice));
    net->step = step;
    net->bf_valid = net->f8_valid = net->xscale_valid = net->bfT_valid = false;
    return MRS_OK;
}

// ---- checkpoints and seeded initialisation ----------------------------------
namespace mrs {
namespace {

static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "checkpoint I/O assumes a little-endian host");

constexpr char kCkptMagic[8] = {'M', 'R', 'S', 'N', 'E', 'T', 'v', '2'};
constexpr uint32_t kCkptVersion = 2;

// header of a checkpoint file (64 bytes, little-endian, no padding)
struct CkptHeader {
    char magic[8];
    uint32_t header_bytes;   // 64
    uint32_t version;        // 2
    int64_t n_params;
    int64_t step;
    uint64_t seed;           // the caller's data / RNG seed, stored for resume
    int32_t input_channels;  // 12 or 21
    int32_t loss;            // MRS_LOSS_*
    float beta;
    uint32_t reserved;
    uint64_t checksum;       // FNV-1a 64 over the three float arrays' bytes
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header layout");

uint64_t fnv1a(uint64_t h, const void* data, size_t n)
{
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 0x100000001B3ull; }
    return h;
}

// splitmix64 (Steele, Lea, Flood 2014): the initialiser's uniform stream
uint64_t splitmix64(uint64_t& x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// zero-mean, unit-variance approximately normal draw: the sum of 12
// uniforms minus 6 (Irwin-Hall), integer and IEEE arithmetic only, so that
// the same seed gives the same weights on every host
double normal12(uint64_t& x)
{
    double s = 0.0;
    for (int i = 0; i < 12; ++i) s += (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
    return s - 6.0;
}

}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_net_save(mrs_net net, const char* path, uint64_t seed)
{
    using namespace mrs;
    MRS_ARG(net != nullptr && path != nullptr, "NULL argument");
    std::vector<float> host(3 * net->np);
    int64_t step = 0;
    mrs_status rc = mrs_net_get_state(net, host.data(), host.data() + net->np,
                                      host.data() + 2 * net->np, &step);
    if (rc != MRS_OK) return rc;
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.header_bytes = sizeof(CkptHeader);
    h.version = kCkptVersion;
    h.n_params = (int64_t)net->np;
    h.step = step;
    h.seed = seed;
    h.input_channels = net->cin0;
    h.loss = net->loss_kind;
    h.beta = net->loss_beta;
    h.checksum = fnv1a(0xCBF29CE484222325ull, host.data(), host.size() * 4);
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) { set_error("cannot open %s for writing", tmp.c_str()); return MRS_ERR_IO; }
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(host.data(), 4, host.size(), f) == host.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        set_error("writing checkpoint %s failed", path);
        return MRS_ERR_IO;
    }
    return MRS_OK;
}

extern "C" mrs_status mrs_net_load(mrs_net net, const char* path, uint64_t* seed)
{
    using namespace mrs;
    MRS_ARG(net != nullptr && path != nullptr, "NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return MRS_ERR_IO; }
    CkptHeader h;
    std::vector<float> host;
    mrs_status rc = MRS_OK;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kCkptMagic, 8) != 0 ||
        h.header_bytes != sizeof(CkptHeader) || h.version != kCkptVersion) {
        set_error("%s is not a version-%u fusion-network checkpoint", path, kCkptVersion);
        rc = MRS_ERR_FORMAT;
    } else if (h.n_params != (int64_t)net->np || h.input_channels != net->cin0) {
        set_error("checkpoint holds %lld parameters (%d input channels), the net %zu (%d)",
                  (long long)h.n_params, h.input_channels, net->np, net->cin0);
        rc = MRS_ERR_FORMAT;
    } else if ((h.loss != MRS_LOSS_L1LOG && h.loss != MRS_LOSS_ROBUST) || !(h.beta > 0.0f) ||
               h.step < 0) {
        set_error("checkpoint %s has an invalid loss, beta or step", path);
        rc = MRS_ERR_FORMAT;
    } else {
        host.resize(3 * net->np);
        if (fread(host.data(), 4, host.size(), f) != host.size() || fgetc(f) != EOF) {
            set_error("checkpoint %s is truncated or has trailing bytes", path);
            rc = MRS_ERR_FORMAT;
        } else if (fnv1a(0xCBF29CE484222325ull, host.data(), host.size() * 4) != h.checksum) {
            set_error("checkpoint %s fails its checksum", path);
            rc = MRS_ERR_FORMAT;
        }
    }
    fclose(f);
    if (rc != MRS_OK) return rc;
    rc = mrs_net_set_state(net, host.data(), host.data() + net->np, host.data() + 2 * net->np, h.step);
    if (rc != MRS_OK) return rc;
    net->loss_kind = h.loss;
    net->loss_beta = h.beta;
    if (seed) *seed = h.seed;
    return MRS_OK;
}

extern "C" mrs_status mrs_net_create_seeded(int32_t input_channels, uint64_t init_seed,
                                            float resid_gain, mrs_net* out)
{
    using namespace mrs;
    MRS_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MRS_ARG(input_channels == 12 || input_channels == 21, "input_channels must be 12 or 21");
    MRS_ARG(resid_gain >= 0.0f && resid_gain <= 1.0f, "resid_gain must be in [0, 1]");
    const auto& L = shapes(input_channels);
    size_t np = input_channels == 21 ? kParams21 : kParams12;
    std::vector<float> p(np, 0.0f);
    uint64_t x = init_seed ^ 0x6D72732D6E657430ull;
    for (int l = 0; l < kLayers; ++l) {
        if (l == kLayers - 1) break;   // the 3-channel head starts at zero
        double sd = sqrt(2.0 / (9.0 * L[l].cin));
        if (l >= 1 && l % 2 == 0) sd *= resid_gain;   // second conv of a residual block
        for (size_t i = 0; i < (size_t)L[l].cout * 9 * L[l].cin; ++i)
            p[L[l].woff + i] = (float)(sd * normal12(x));
    }
    return mrs_net_create(p.data(), (int32_t)np, out);
}

extern "C" mrs_status mrs_selftest_wait_timeout(int32_t limit_us, void* stream)
{
    MRS_ARG(limit_us >= 1 && limit_us <= 100000, "limit_us must be in [1, 100000]");
    int clk_khz = 0, dev = 0;
    MRS_CHECK(cudaGetDevice(&dev));
    MRS_CHECK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    long long cycles = (long long)limit_us * (clk_khz > 0 ? clk_khz : 2000000) / 1000;
    int gave_up = 0;
    mrs_status rc = tc_wait_selftest(cycles, &gave_up, (cudaStream_t)stream);
    if (rc != MRS_OK) return rc;
    if (gave_up) {
        set_error("device wait gave up after %d us (self-test)", limit_us);
        return MRS_ERR_TIMEOUT;
    }
    return MRS_OK;
}

extern "C" mrs_status mrs_gate_async(const float* fused, const float* lrhs, const float* plain,
                                     int32_t N, int32_t H, int32_t W, int32_t scale, double tau,
                                     float* out, int32_t* used_plain, double* D, void* stream)
{
    MRS_ARG(fused && lrhs && out && used_plain, "NULL pointer");
    MRS_ARG(scale >= 1 && N >= 1 && H >= scale && W >= scale && H % scale == 0 && W % scale == 0,
            "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    static std::mutex mu;
    static Buf parts;
    std::lock_guard<std::mutex> g(mu);
    mrs_status rc = parts.ensure(sizeof(double) * kRedBlocks);
    if (rc != MRS_OK) return rc;
    k_gate_partial<<<kRedBlocks, 256, 0, st>>>(fused, lrhs, N, H, W, scale, parts.as<double>());
    MRS_LAUNCHED(1);
    k_gate_decide<<<1, 256, 0, st>>>(parts.as<double>(), kRedBlocks,
                                    (double)N * (H / scale) * (W / scale) * 3, tau,
                                    plain ? 1 : 0, used_plain, D);
    MRS_LAUNCHED(1);
    size_t n = (size_t)N * H * W * 3;
    k_gate_select<<<1024, 256, 0, st>>>(fused, plain ? plain : fused, n, used_plain, out);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "gate_async launch");
}

extern "C" mrs_status mrs_conv3x3_wgrad(const float* x, const float* dy, int32_t N, int32_t H,
                                        int32_t W, int32_t cin, int32_t cout, int32_t precision,
                                        float* dw, float* db, void* stream)
{
    using namespace mrs;
    MRS_ARG(x && dy && dw && db, "NULL pointer");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1, "sizes must be >= 1");
    MRS_ARG(cin >= 1 && cin <= 64 && cout >= 1 && cout <= 64, "cin, cout must be in [1, 64]");
    MRS_ARG(precision == MRS_PREC_FP32 || precision == MRS_PREC_BF16, "precision must be FP32 or BF16");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)N * H * W;
    const size_t nw = (size_t)cout * 9 * cin;
    const size_t maxp = (size_t)std::max(kDwSplits, tc_wgrad_max_parts());
    Scratch& S = scratch();
    std::lock_guard<std::mutex> g(S.mu);
    size_t need = (nw + cout) * 4 + maxp * (9 * 64 * 64 + 64) * 4 + 4096 +
                  (precision == MRS_PREC_BF16 ? 2 * P * 128 : 0);
    mrs_status rc = S.b.ensure(need);
    if (rc != MRS_OK) return rc;
    float* gw = S.b.as<float>();
    float* gb = gw + nw;
    float* part = (float*)(((uintptr_t)(gb + cout) + 255) & ~(uintptr_t)255);
    float* dbpart = part + maxp * 9 * 64 * 64;
    static int* err = nullptr;
    if (!err) { MRS_CHECK(cudaMalloc(&err, 4)); MRS_CHECK(cudaMemset(err, 0, 4)); }
    int np = 0;
    if (precision == MRS_PREC_FP32) {
        k_dw_partial<float, float><<<dim3(kDwSplits, 9), 256, 0, st>>>(x, cin, cin, dy, cout, cout, N, H, W,
                                                                      part, dbpart, 0, 1);
        MRS_LAUNCHED(1);
        np = kDwSplits;
    } else {
        uint8_t* xq = (uint8_t*)(((uintptr_t)(dbpart + maxp * 64) + 1023) & ~(uintptr_t)1023);
        uint8_t* dq = xq + P * 128;
        k_to_operand<<<1024, 256, 0, st>>>(x, P, cin, xq, 0, 1.0f);
        MRS_LAUNCHED(1);
        k_to_operand<<<1024, 256, 0, st>>>(dy, P, cout, dq, 0, 1.0f);
        MRS_LAUNCHED(1);
        CUtensorMap mx, md;
        if ((rc = tc_make_act_map(&mx, xq, N, H, W, TC_BF16, kWgKB + 2)) != MRS_OK) return rc;
        if ((rc = tc_make_act_map(&md, dq, N, H, W, TC_BF16, kWgKB)) != MRS_OK) return rc;
        TcWgradArgs wa;
        wa.tmap_x = &mx; wa.tmap_dy = &md; wa.part = part; wa.dbpart = dbpart;
        wa.N = N; wa.H = H; wa.W = W; wa.cin = cin; wa.cout = cout; wa.err = err;
        if ((rc = tc_conv3x3_wgrad(wa, &np, st)) != MRS_OK) return rc;
    }
    k_dw_reduce<<<(int)((nw + cout + 31) / 32), 256, 0, st>>>(part, dbpart, np, cin, cout, gw, gb);
    MRS_LAUNCHED(1);
    MRS_CHECK(cudaMemcpyAsync(dw, gw, nw * 4, cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaMemcpyAsync(db, gb, cout * 4, cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    int herr = 0;
    MRS_CHECK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
    if (herr) { cudaMemset(err, 0, 4); set_error("tensor-core weight-gradient wait timed out"); return MRS_ERR_TIMEOUT; }
    return MRS_OK;
}

extern "C" mrs_status mrs_conv3x3_dgrad(const float* dy, int32_t N, int32_t H, int32_t W,
                                        int32_t cin, int32_t cout, const float* w, int32_t mode,
                                        const float* aux, int32_t precision, float* out,
                                        void* stream)
{
    using namespace mrs;
    MRS_ARG(dy && w && out, "NULL pointer");
    MRS_ARG(N >= 1 && H >= 1 && W >= 1, "sizes must be >= 1");
    MRS_ARG(cin >= 1 && cin <= 64 && cout >= 1 && cout <= 64, "cin, cout must be in [1, 64]");
    MRS_ARG(mode == MRS_DGRAD_LINEAR || mode == MRS_DGRAD_RELU_MASK || mode == MRS_DGRAD_RESIDUAL,
            "unknown mode");
    MRS_ARG(mode == MRS_DGRAD_LINEAR || aux != nullptr, "aux is required by this mode");
    MRS_ARG(precision == MRS_PREC_FP32 || precision == MRS_PREC_BF16, "precision must be FP32 or BF16");
    MRS_ARG((int64_t)N * H * W <= (int64_t(1) << 26), "more than 2^26 pixels");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)N * H * W;
    const size_t nw = (size_t)cout * 9 * cin;
    Scratch& S = scratch();
    std::lock_guard<std::mutex> g(S.mu);
    const size_t opb = ((P * 128 + 1023) / 1024) * 1024;   // one bf16 [P][64] operand
    size_t need = nw * 4 + 64 * 4 + 2048 + 9 * 64 * 64 * 4 + 1024 +
                  (precision == MRS_PREC_BF16 ? 3 * opb : 0);
    mrs_status rc = S.b.ensure(need);
    if (rc != MRS_OK) return rc;
    float* dw = S.b.as<float>();
    float* zero = dw + nw;
    uint8_t* q = (uint8_t*)(((uintptr_t)(zero + 64) + 1023) & ~(uintptr_t)1023);
    MRS_CHECK(cudaMemcpyAsync(dw, w, nw * 4, cudaMemcpyHostToDevice, st));
    MRS_CHECK(cudaMemsetAsync(zero, 0, 64 * 4, st));
    if (precision == MRS_PREC_FP32) {
        // the FP32 training step's transposed conv: flipped, transposed
        // weights through the SIMT convolution with the step's epilogues
        float* wt = (float*)q;
        k_wtrans<<<(int)((nw + 255) / 256), 256, 0, st>>>(dw, cin, cout, wt);
        MRS_LAUNCHED(1);
        int sm = mode == MRS_DGRAD_LINEAR ? SIMT_PLAIN : mode == MRS_DGRAD_RELU_MASK ? SIMT_MASK : SIMT_RESID;
        rc = conv_simt(dy, cout, wt, zero, cin, sm, 0, aux, out, nullptr, N, H, W, 1, st);
        if (rc == MRS_OK) rc = cuda_status(cudaStreamSynchronize(st), "conv3x3 dgrad sync");
        return rc;
    }
    // BF16: the tensor-core conv with the training step's transposed-weight
    // packing and epilogue modes (linear; ReLU mask by the layer's output;
    // residual added in place into the incoming gradient)
    __nv_bfloat16* wp = (__nv_bfloat16*)q;
    uint8_t* dyq = q + ((9 * 64 * 64 * 2 + 1023) / 1024) * 1024;
    uint8_t* auxq = dyq + opb;
    uint8_t* outq = auxq + opb;
    static int* err = nullptr;
    if (!err) { MRS_CHECK(cudaMalloc(&err, 4)); MRS_CHECK(cudaMemset(err, 0, 4)); }
    k_pack_bf16_T<<<(9 * 64 * 64 + 255) / 256, 256, 0, st>>>(dw, 0, cin, cout, 64, wp);
    MRS_LAUNCHED(1);
    k_to_operand<<<1024, 256, 0, st>>>(dy, P, cout, dyq, 0, 1.0f);
    MRS_LAUNCHED(1);
    if (mode == MRS_DGRAD_RELU_MASK) {
        k_to_operand<<<1024, 256, 0, st>>>(aux, P, cin, auxq, 0, 1.0f);
        MRS_LAUNCHED(1);
    } else if (mode == MRS_DGRAD_RESIDUAL) {
        k_to_operand<<<1024, 256, 0, st>>>(aux, P, cin, outq, 0, 1.0f);
        MRS_LAUNCHED(1);
    }
    CUtensorMap ma, mo, mr, mw;
    if ((rc = tc_make_w_map(&mw, wp, 9 * 64, 64, TC_BF16)) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&ma, dyq, N, H, W, TC_BF16, tc_a_box(TC_BF16))) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&mo, outq, N, H, W, TC_BF16, tc_out_box(TC_BF16))) != MRS_OK) return rc;
    if ((rc = tc_make_act_map(&mr, auxq, N, H, W, TC_BF16, tc_out_box(TC_BF16))) != MRS_OK) return rc;
    TcConvArgs a;
    memset(&a, 0, sizeof(a));
    a.tmap_x = &ma; a.tmap_w = &mw; a.bias = zero; a.tmap_out = &mo;
    a.N = N; a.H = H; a.W = W; a.scale = 1; a.nout = 64; a.operand = TC_BF16; a.err = err;
    if (mode == MRS_DGRAD_LINEAR) { a.mode = TC_LIN_BF16; }
    else if (mode == MRS_DGRAD_RELU_MASK) { a.mode = TC_MASK_BF16; a.tmap_res = &mr; }
    else { a.mode = TC_RESID_BF16; a.tmap_res = &mo; }
    if ((rc = tc_conv3x3(a, st)) != MRS_OK) return rc;
    k_from_operand<<<1024, 256, 0, st>>>((const __nv_bfloat16*)outq, P, cin, out);
    MRS_LAUNCHED(1);
    rc = cuda_status(cudaStreamSynchronize(st), "conv3x3 dgrad sync");
    int herr = 0;
    if (rc == MRS_OK) {
        MRS_CHECK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
        if (herr) { cudaMemset(err, 0, 4); set_error("tensor-core conv wait timed out"); return MRS_ERR_TIMEOUT; }
    }
    return rc;
}

extern "C" mrs_status mrs_conv_set_ring(int32_t stages)
{
    MRS_ARG(stages == 0 || (stages >= 3 && stages <= 12), "stages must be 0 or in [3, 12]");
    mrs::tc_set_ring(stages);
    return MRS_OK;
}

extern "C" mrs_status mrs_net_set_loss(mrs_net net, int32_t loss, float beta)
{
    MRS_ARG(net != nullptr, "net is NULL");
    MRS_ARG(loss == MRS_LOSS_L1LOG || loss == MRS_LOSS_ROBUST, "unknown loss");
    MRS_ARG(beta > 0.0f && beta < 1e30f, "beta must be positive and finite");
    net->loss_kind = loss;
    net->loss_beta = beta;
    return MRS_OK;
}
