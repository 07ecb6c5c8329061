// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA), BF16 or
// FP8-E4M3 operands with FP32 accumulation, and the weight gradient of the
// same convolution (k_wgrad_tc, below).
//
// The convolution (k_conv_fold) folds the three kernel ROWS into the MMA N
// dimension; see the comment above the kernel for the schedule.  Each
// activation row (64 channels) is 128 bytes (bf16) or 64 bytes (fp8), stored
// with the matching TMA swizzle (128B / 64B) so that the shared-memory
// descriptors address it directly; out-of-range parts of a TMA box are
// zero-filled, which is the convolution's zero padding.  All 9 taps of the
// layer's weights stay resident in shared memory for the whole persistent CTA.
//
// Warp roles (640 threads, one CTA per SM):
//   warp 0: TMA producer (weights once, then one A box per input row through
//           an S-stage ring)
//   warp 1: TMEM allocator and MMA issuer (one thread)
//   warps 2-17: epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and 16 of
//           the 64 output channels: dequantisation (fp8), bias, ReLU /
//           residual / mask / FP32 partial sum / bilinear skip, BF16 results
//           written into the staging slot (swizzled) and sent out by one TMA
//           store per tile, or FP32 results stored directly
//   warp 18: residual prefetch into one of three staging slots
//   warp 19: output TMA stores from the staging slots
// Every wait is bounded (no hardware barrier inside the role loops): on
// timeout the kernel sets *err, all roles unwind, TMEM is freed, and the host
// reports MRS_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <string.h>

#include <atomic>

#include "conv_tc.cuh"

namespace mrs {
namespace {

constexpr int kEpiWarps = 16;                  // 4 per TMEM lane quarter
constexpr int kResWarp = 2 + kEpiWarps;        // residual-prefetch warp
constexpr int kStoreWarp = kResWarp + 1;       // output-store warp
constexpr int kThreads = 32 * (kStoreWarp + 1);  // A-TMA, MMA, epilogue, residual, store warps
constexpr int kSlots = 3;                      // residual / output staging slots
constexpr long long kTimeoutCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// as above, but the thread may be suspended (up to `ns` nanoseconds) until the
// phase completes instead of spinning in a loop that takes issue slots from
// the working warps
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// bounded wait; false if this or another role gave up.  Each poll lets the
// hardware suspend the thread (1 ms limit) until the phase completes; the
// error word and the clock are consulted between polls
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, int* err,
                                                long long limit_cycles, uint32_t sleep_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, sleep_ns)) return true;
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > limit_cycles) {
            atomicExch(err, 1);
            return false;
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err)
{
    return mbar_wait_limit(bar, parity, err, kTimeoutCycles, 1000000u);
}

// warp-wide wait: lane 0 polls, then every lane observes the completed phase
// once (acquiring the data the phase guards)
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, int* err)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, err);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) (void)mbar_try_wait(bar, parity);
    return ok;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// tcgen05 shared-memory matrix descriptor, K-major, swizzled rows of
// `row_bytes` (128 -> SWIZZLE_128B, 64 -> SWIZZLE_64B), 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int row_bytes)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                                  // LBO (unused when swizzled)
    d |= (uint64_t)((8 * row_bytes) >> 4) << 32;              // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                                  // descriptor version
    d |= (uint64_t)(row_bytes == 128 ? 2 : 4) << 61;         // swizzle mode
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_f8(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// bilinear x s upsampling of LRHS at HR pixel (x, y): half-pixel centres,
// clamped at the borders
__device__ __forceinline__ void bilinear(const float* __restrict__ lr, int h, int w, int s, int x,
                                         int y, float out[3])
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
        out[k] = top * (1.0f - ly) + bot * ly;
    }
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0,
                                             int c1, int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
            (uint64_t)map),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Work split: the layer is T = N * XB * H tiles (one tile = one output row of
// one 128-pixel column strip), flattened as f = (n * XB + xb) * H + y.  CTA c
// takes the contiguous run [T c / G, T (c + 1) / G), cut at strip boundaries
// into pieces; a piece is a run of rows of one strip, streamed through the
// input-row ring with its own halo rows.  piece_rows returns the piece that
// starts at f (< f1) and advances f past it.
__device__ __forceinline__ void piece_rows(long long& f, long long f1, int XB, int H, int& xb,
                                           int& n, int& y0, int& y1)
{
    const long long k = f / H;
    y0 = (int)(f - k * H);
    const long long left = f1 - f;
    y1 = (int)((long long)y0 + left < (long long)H ? (long long)y0 + left : (long long)H);
    xb = (int)(k % XB);
    n = (int)(k / XB);
    f += y1 - y0;
}

// byte offset of 16-byte chunk j of row m in a SWIZZLE_128B tile
__device__ __forceinline__ uint32_t sw128(int m, int j) { return m * 128 + ((j ^ (m & 7)) << 4); }

// ---------------------------------------------------------------------------
// 3x3 convolution with the kernel ROWS folded into the MMA N dimension.
//
// Input row r of a column strip meets the weights of all three kernel rows in
// one MMA: B = [w(dy 0, dx); w(dy 1, dx); w(dy 2, dx)] (3 NOUT rows) gives
// column block j = the contribution of row r to output row r + 1 - j.  The
// accumulators of consecutive output rows sit in consecutive NOUT-column
// slots of TMEM in DEcreasing order (slot(t) = (-t) mod NS for the CTA's t-th
// output row), so one MMA with D at slot(r + 1) adds to output rows r + 1, r,
// r - 1 at once; where the three slots wrap around the end of TMEM the MMA is
// split in two.  The column taps dx are row-shifted A descriptors into one
// 130-pixel box per input row (x0 - 1 .. x0 + 128), so an output pixel's sum
// is complete in its own TMEM lane: the epilogue reads one NOUT-column slot
// per output row, without cross-lane shuffles, and zeroes it for reuse (every
// MMA accumulates onto zeroed TMEM).  Each input row is consumed by the 12
// MMAs (3 dx x 4 K steps) issued right after it lands and then released, so
// the whole ring is prefetch depth.  An output tile is 128 pixels of one row.
// FP8 operands (kind::f8f6f4, K = 32 per MMA, 64-byte rows with the 64B
// swizzle) follow the same schedule with one-row (64-byte) descriptor shifts,
// per-output-channel weight scales and a per-layer activation scale; their
// BF16 outputs also leave an FP8 copy for the next layer's operand.
// Consecutive MMAs into different D regions do not pipeline, so the wrap
// rows issue all MMAs of one region before the other.
constexpr int kFoldTile = 128;               // output pixels per tile (= MMA M)
constexpr int kFoldABox = kFoldTile + 2;     // input pixels per row box (one halo each side)
constexpr int kFoldMaxRows = 6;              // output rows per sub-piece of a multi-chunk conv
// bytes per activation row of the operand type, ring slot (1024-aligned)
constexpr int fold_rowb(int oper) { return oper == TC_BF16 ? 128 : 64; }
constexpr int fold_aslot(int oper) { return ((kFoldABox * fold_rowb(oper) + 1023) / 1024) * 1024; }

template <int NOUT, int OPER> size_t fold_smem_bytes(int stages)
{
    return 1024 + ((9 * NOUT * fold_rowb(OPER) + 1023) & ~1023) + (size_t)stages * fold_aslot(OPER) +
           (size_t)kSlots * kFoldTile * 128 + 64 * 4 + 8 * (2 * stages + 2 + 2 * (512 / NOUT) + 3 * kSlots) + 16;
}

template <int NOUT, int OPER>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv_fold(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_w,
                const __grid_constant__ CUtensorMap tmap_res,
                const __grid_constant__ CUtensorMap tmap_out, TcConvArgs a, int stages)
{
    constexpr int NS = 512 / NOUT;                            // TMEM accumulator slots
    constexpr int ROWB = fold_rowb(OPER);                     // bytes per operand row
    constexpr int ASLOT = fold_aslot(OPER);
    constexpr int KSTEPS = OPER == TC_BF16 ? 4 : 2;           // MMAs per 64 input channels (K 16 / 32)
    constexpr int WBYTES = 9 * NOUT * ROWB;
    constexpr int SBYTES = kFoldTile * 128;
    constexpr int BROWS = 3 * NOUT;                           // B rows per dx: dy 0, 1, 2
    constexpr uint32_t kTmemCols = 512;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sW = smem;
    uint8_t* sA = smem + ((WBYTES + 1023) & ~1023);
    uint8_t* sS = sA + stages * ASLOT;
    float* sBias = (float*)(sS + kSlots * SBYTES);
    uint64_t* bars = (uint64_t*)(sBias + 64);
    uint64_t* full = bars;
    uint64_t* empty = bars + stages;
    uint64_t* wbar = bars + 2 * stages;                       // weights landed
    uint64_t* wempty = wbar + 1;                              // weight buffer free
    uint64_t* tfull = wempty + 1;                             // [NS] output row complete
    uint64_t* sfree = tfull + NS;                             // [NS] slot read and zeroed
    uint64_t* rfull = sfree + NS;
    uint64_t* rempty = rfull + kSlots;
    uint64_t* edone = rempty + kSlots;
    uint32_t* tslot = (uint32_t*)(edone + kSlots);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int XB = (a.W + kFoldTile - 1) / kFoldTile;
    const long long T = (long long)a.N * XB * a.H;
    const long long f0 = T * blockIdx.x / gridDim.x, f1 = T * (blockIdx.x + 1) / gridDim.x;
    const bool bf_out = a.mode == TC_RELU_BF16 || a.mode == TC_RESID_BF16 ||
                        a.mode == TC_LIN_BF16 || a.mode == TC_MASK_BF16 ||
                        a.mode == TC_RESRELU_BF16;
    const bool loads_res = a.mode == TC_RESID_BF16 || a.mode == TC_MASK_BF16 ||
                           a.mode == TC_RESRELU_BF16;
    // a bf16 result that nobody reads (fp8 operands: only the fp8 copy) is
    // neither staged nor stored
    const bool stores_bf = bf_out && !(a.fp8_only && a.out_fp8);

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(wbar, 1);
        mbar_init(wempty, 1);
        for (int i = 0; i < NS; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&sfree[i], kEpiWarps);
        }
        for (int i = 0; i < kSlots; ++i) {
            mbar_init(&rfull[i], 1);
            mbar_init(&rempty[i], 1);
            mbar_init(&edone[i], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x < 64) sBias[threadIdx.x] = threadIdx.x < NOUT ? a.bias[threadIdx.x] : 0.0f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *(volatile uint32_t*)tslot;
    // every accumulator slot starts at zero (the MMAs always accumulate)
    if (warp >= 2 && warp < 2 + kEpiWarps) {
        const int q = warp & 3, grp = (warp - 2) >> 2;
        uint32_t z[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) z[e] = 0u;
        for (int c = grp * 16; c < (int)kTmemCols; c += 64) tmem_st16(tmem + ((uint32_t)(q * 32) << 16) + c, z);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // programmatic dependent launch: the next conv may be scheduled now; every
    // access to data of the previous kernel in the stream waits for its
    // completion (griddepcontrol.wait).  The weights and biases come from
    // before the previous kernel (packed at set-up or by a non-overlapping
    // kernel), so the weight load is issued before that wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (!(warp == 0 && lane == 0)) asm volatile("griddepcontrol.wait;" ::: "memory");

    // A convolution over kc > 1 inputs (64-channel chunks, each its own tensor
    // map in a.amaps, weights chunk after chunk in tmap_w) accumulates all
    // chunks in TMEM: a piece is cut into sub-pieces of at most kMaxRows
    // output rows, whose accumulators all stay live while the chunks pass
    // (chunk-major order; the weight buffer is reloaded per chunk).
    const int kc = a.kc > 1 ? a.kc : 1;
    const int maxr = kc > 1 ? kFoldMaxRows : (1 << 30);
    if (warp == 0) {
        if (lane == 0) {
            // A producer: per (sub-piece, chunk), input rows ys-1 .. ye, 130
            // pixels from x0-1; the first weights are loaded here, before the
            // wait for the previous kernel
            mbar_expect_tx(wbar, WBYTES);
            // tap (dy, dx) at B row (3 dx + dy) NOUT: per dx the three kernel rows are contiguous
            for (int t = 0; t < 9; ++t)
                tma_load_2d(sW + ((t % 3) * 3 + t / 3) * NOUT * ROWB, &tmap_w, 0, a.w_row0 + t * NOUT, wbar);
            asm volatile("griddepcontrol.wait;" ::: "memory");
            uint32_t it = 0;
            bool ok = true;
            for (long long f = f0; ok && f < f1;) {
                int xb, n, y0, y1;
                piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
                for (int ys = y0; ok && ys < y1; ys += maxr) {
                    const int ye = min(y1, ys + maxr);
                    for (int j = 0; ok && j < kc; ++j) {
                        const CUtensorMap* am = kc > 1 ? a.amaps + j : &tmap_x;
                        // a map in global memory, written by the host before
                        // the launch: acquire it for the tensor-map proxy
                        if (kc > 1)
                            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                             (uint64_t)am)
                                         : "memory");
                        for (int r = ys - 1; r <= ye; ++r, ++it) {
                            int s = it % stages;
                            if (!mbar_wait(&empty[s], ((it / stages) & 1) ^ 1, a.err)) { ok = false; break; }
                            mbar_expect_tx(&full[s], kFoldABox * ROWB);
                            tma_load_4d(sA + s * ASLOT, am, 0, xb * kFoldTile - 1, r, n, &full[s]);
                        }
                    }
                }
            }
        } else if (lane == 16 && kc > 1) {
            // weight loader for every (sub-piece, chunk) pass after the first:
            // waits for the MMAs of the previous pass to finish with the buffer
            uint32_t k = 0;
            bool ok = true;
            for (long long f = f0; ok && f < f1;) {
                int xb, n, y0, y1;
                piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
                for (int ys = y0; ok && ys < y1; ys += maxr)
                    for (int j = 0; ok && j < kc; ++j, ++k) {
                        if (k == 0) continue;
                        if (!mbar_wait(wempty, (k - 1) & 1, a.err)) { ok = false; break; }
                        mbar_expect_tx(wbar, WBYTES);
                        for (int t = 0; t < 9; ++t)
                            tma_load_2d(sW + ((t % 3) * 3 + t / 3) * NOUT * ROWB, &tmap_w, 0,
                                        a.w_row0 + (j * 9 + t) * NOUT, wbar);
                    }
            }
        }
    } else if (warp == kResWarp) {
        if (lane == 0) {
            uint32_t j = 0;
            bool ok = true;
            for (long long f = f0; ok && f < f1;) {
                int xb, n, y0, y1;
                piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
                for (int y = y0; y < y1; ++y, ++j) {
                    uint32_t slot = j % kSlots, use = j / kSlots;
                    if (!mbar_wait(&rempty[slot], (use & 1) ^ 1, a.err)) { ok = false; break; }
                    if (loads_res) {
                        mbar_expect_tx(&rfull[slot], SBYTES);
                        tma_load_4d(sS + slot * SBYTES, &tmap_res, 0, xb * kFoldTile, y, n, &rfull[slot]);
                    } else {
                        mbar_arrive(&rfull[slot]);
                    }
                }
            }
        }
    } else if (warp == kStoreWarp) {
        if (lane == 0) {
            uint32_t j = 0;
            bool ok = true;
            for (long long f = f0; ok && f < f1;) {
                int xb, n, y0, y1;
                piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
                for (int y = y0; y < y1; ++y, ++j) {
                    uint32_t slot = j % kSlots, use = j / kSlots;
                    if (!mbar_wait(&edone[slot], use & 1, a.err)) { ok = false; break; }
                    if (stores_bf) {
                        tma_store_4d(&tmap_out, sS + slot * SBYTES, 0, xb * kFoldTile, y, n);
                        bulk_commit();
                        bulk_wait_read0();
                    }
                    mbar_arrive(&rempty[slot]);
                }
            }
            bulk_wait_all();
        }
    } else if (warp == 1) {
        // MMA issuer: for each input row r of a piece, the blocks j whose output
        // row r + 1 - j lies in the piece, in one MMA per (dx, K step) (two
        // where the slots wrap)
        if (lane == 0) {
            bool ok = true;
            uint32_t it = 0, k = 0;
            int s = 0;                                          // ring slot of row `it`
            uint32_t ph = 0;                                    // its fill phase parity
            long long t0 = 0;                                   // CTA output-row counter at sub-piece start
            const uint32_t wbase = smem_u32(sW), abase = smem_u32(sA);
            // descriptors differ only in their start-address field (address / 16,
            // bits 0-13): each MMA's pair is a base pair plus a constant offset
            const uint64_t adesc0 = sdesc(abase, ROWB), bdesc0 = sdesc(wbase, ROWB);
            for (long long f = f0; ok && f < f1;) {
                int xb, n, y0, y1;
                piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
                for (int ys = y0; ok && ys < y1; ys += maxr) {
                  const int ye = min(y1, ys + maxr);
                  for (int j = 0; ok && j < kc; ++j, ++k) {
                    // weights of this pass (loaded once when kc == 1)
                    if ((kc > 1 || k == 0) && !mbar_wait(wbar, k & 1, a.err)) { ok = false; break; }
                    for (int r = ys - 1; ok && r <= ye; ++r, ++it, s = (s + 1 == stages ? 0 : s + 1),
                                                        ph ^= (s == 0 ? 1u : 0u)) {
                        const int jlo = max(0, r + 2 - ye), jhi = min(2, r + 1 - ys);
                        // output row of block jb: CTA counter t0 + (r + 1 - jb - ys)
                        const long long tlo = t0 + (r + 1 - jlo - ys);   // newest row (highest t)
                        if (jlo == 0 && j == 0) {
                            // block 0 of the first chunk starts output row tlo: its slot must
                            // have been read and zeroed by the epilogue of row tlo - NS
                            const int sl = (int)(tlo % NS);
                            const uint32_t use = (uint32_t)(tlo / NS);
                            if (!mbar_wait(&sfree[(NS - sl) % NS], (use & 1) ^ 1, a.err)) { ok = false; break; }
                        }
                        if (!mbar_wait(&full[s], ph, a.err)) { ok = false; break; }
                        tc_fence_after();
                        const int nb = jhi - jlo + 1;
                        const int c0 = (int)((NS - (int)(tlo % NS)) % NS);   // slot of block jlo
                        const int n1 = min(nb, NS - c0);                    // blocks before the wrap
                        // all MMAs of one D region back to back: the region before
                        // the wrap, then (rarely) the one after it; consecutive
                        // MMAs into different regions do not pipeline
                        for (int part = 0; part < (n1 < nb ? 2 : 1); ++part) {
                            const uint32_t dcol = part ? 0u : (uint32_t)(c0 * NOUT);
                            const int b0 = part ? n1 : 0, nbp = part ? nb - n1 : n1;
                            const uint32_t idesc = (1u << 4) | ((OPER == TC_BF16 ? 1u : 0u) << 7) |
                                                   ((OPER == TC_BF16 ? 1u : 0u) << 10) |
                                                   ((uint32_t)((nbp * NOUT) >> 3) << 17) |
                                                   ((uint32_t)(kFoldTile >> 4) << 24);
                            const uint64_t arow = adesc0 + (uint64_t)((s * ASLOT) >> 4);
                            const uint64_t brow0 = bdesc0 + (uint64_t)(((jlo + b0) * NOUT * ROWB) >> 4);
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                                for (int kk = 0; kk < KSTEPS; ++kk) {
                                    const uint64_t ad = arow + (uint64_t)((dx * ROWB + kk * 32) >> 4);
                                    const uint64_t bd = brow0 + (uint64_t)((dx * BROWS * ROWB + kk * 32) >> 4);
                                    if (OPER == TC_BF16) mma_f16(tmem + dcol, ad, bd, idesc, 1u);
                                    else mma_f8(tmem + dcol, ad, bd, idesc, 1u);
                                }
                            }
                        }
                        mma_commit(&empty[s]);
                        if (jhi == 2 && j == kc - 1) {
                            // output row r - 1 (block 2 of the last chunk) is complete
                            const long long td = tlo - (2 - jlo);
                            mma_commit(&tfull[(NS - (int)(td % NS)) % NS]);
                        }
                    }
                    // the weight buffer is free once this pass's MMAs complete
                    if (kc > 1) mma_commit(wempty);
                  }
                  t0 += ye - ys;
                }
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 q .. 32 q + 31 (output pixels
        // x0 + 32 q + lane) and channels [16 grp, 16 grp + 16) of the finished
        // output row's slot, then zeroes them
        const int q = warp & 3, grp = (warp - 2) >> 2;
        const int j = q * 32 + lane;
        const bool active = grp * 16 < NOUT;
        uint32_t lt = 0;
        bool stop = false;
        for (long long f = f0; !stop && f < f1;) {
          int xb, n, y0, y1;
          piece_rows(f, f1, XB, a.H, xb, n, y0, y1);
          for (int y = y0; y < y1; ++y, ++lt) {
            const int sl = (int)((NS - (int)(lt % NS)) % NS);
            const uint32_t use = lt / NS;
            const uint32_t slot = lt % kSlots, suse = lt / kSlots;
            const int x = xb * kFoldTile + j;
            const bool valid = x < a.W;
            const size_t p = ((size_t)n * a.H + y) * a.W + (valid ? x : 0);
            if (!mbar_wait_warp(&tfull[sl], use & 1, a.err)) { stop = true; break; }
            tc_fence_after();
            if (!mbar_wait_warp(&rfull[slot], suse & 1, a.err)) { stop = true; break; }
            uint8_t* srow = sS + slot * SBYTES;
            if (active) {
                const int c0 = grp * 16;
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(sl * NOUT + c0);
                uint32_t r0[16];
                tmem_ld16(taddr, r0);
                tmem_wait_ld();
                uint32_t z[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) z[e] = 0u;
                tmem_st16(taddr, z);
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r0[e]);
                if (OPER == TC_FP8) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        v[e] = v[e] * (__ldg(a.wscale + (c0 + e < NOUT ? c0 + e : 0)) * a.xscale);
                }
                if (bf_out) {
                    float o[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) o[e] = v[e] + sBias[c0 + e];
                    if (a.mode == TC_RELU_BF16) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) o[e] = fmaxf(o[e], 0.0f);
                    } else if (a.mode == TC_MASK_BF16) {
#pragma unroll
                        for (int jj = 0; jj < 2; ++jj) {
                            uint4 u = *(const uint4*)(srow + sw128(j, c0 / 8 + jj));
                            const __nv_bfloat162* h2 = (const __nv_bfloat162*)&u;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 fv = __bfloat1622float2(h2[e]);
                                if (!(fv.x > 0.0f)) o[8 * jj + 2 * e] = 0.0f;
                                if (!(fv.y > 0.0f)) o[8 * jj + 2 * e + 1] = 0.0f;
                            }
                        }
                    } else if (a.mode == TC_RESID_BF16 || a.mode == TC_RESRELU_BF16) {
                        const bool rl = a.mode == TC_RESRELU_BF16;
#pragma unroll
                        for (int jj = 0; jj < 2; ++jj) {
                            uint4 u = *(const uint4*)(srow + sw128(j, c0 / 8 + jj));
                            const __nv_bfloat162* h2 = (const __nv_bfloat162*)&u;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 fv = __bfloat1622float2(h2[e]);
                                float o0 = o[8 * jj + 2 * e], o1 = o[8 * jj + 2 * e + 1];
                                if (rl) { o0 = fmaxf(o0, 0.0f); o1 = fmaxf(o1, 0.0f); }
                                o[8 * jj + 2 * e] = fv.x + o0;
                                o[8 * jj + 2 * e + 1] = fv.y + o1;
                            }
                        }
                    }
                    if (stores_bf) {
#pragma unroll
                        for (int jj = 0; jj < 2; ++jj) {
                            uint4 u;
                            __nv_bfloat162* h2 = (__nv_bfloat162*)&u;
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                h2[e] = __floats2bfloat162_rn(o[8 * jj + 2 * e], o[8 * jj + 2 * e + 1]);
                            *(uint4*)(srow + sw128(j, c0 / 8 + jj)) = u;
                        }
                    }
                    if (a.out_fp8 && valid) {
                        // the next layer's FP8 operand row
                        uint4 u;
                        uint8_t* b8 = (uint8_t*)&u;
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            b8[e] = (uint8_t)__nv_cvt_float_to_fp8(o[e] * a.out_fp8_inv_scale,
                                                                   __NV_SATFINITE, __NV_E4M3);
                        *(uint4*)((uint8_t*)a.out_fp8 + p * 64 + c0) = u;
                    }
                } else if (valid) {
                    if (a.mode == TC_FINAL_F32) {
                        if (c0 == 0) {
                            float up[3];
                            bilinear(a.lrhs + (size_t)n * (a.H / a.scale) * (a.W / a.scale) * 3,
                                     a.H / a.scale, a.W / a.scale, a.scale, x, y, up);
                            float* op = (float*)a.out + p * 3;
                            for (int c = 0; c < 3; ++c) op[c] = (v[c] + sBias[c]) + up[c];
                        }
                    } else if (a.cout == 64 && ((uintptr_t)a.out & 15) == 0) {
                        float4* op = (float4*)((float*)a.out + p * 64 + c0);
#pragma unroll
                        for (int i4 = 0; i4 < 4; ++i4) {
                            float4 t = make_float4(v[4 * i4] + sBias[c0 + 4 * i4],
                                                   v[4 * i4 + 1] + sBias[c0 + 4 * i4 + 1],
                                                   v[4 * i4 + 2] + sBias[c0 + 4 * i4 + 2],
                                                   v[4 * i4 + 3] + sBias[c0 + 4 * i4 + 3]);
                            if (a.relu) {
                                t.x = fmaxf(t.x, 0.0f); t.y = fmaxf(t.y, 0.0f);
                                t.z = fmaxf(t.z, 0.0f); t.w = fmaxf(t.w, 0.0f);
                            }
                            op[i4] = t;
                        }
                    } else {
                        float* op = (float*)a.out + p * a.cout;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            if (c0 + e < a.cout) {
                                float o = v[e] + sBias[c0 + e];
                                op[c0 + e] = a.relu ? fmaxf(o, 0.0f) : o;
                            }
                        }
                    }
                }
                tmem_wait_st();
            }
            // the slot is read and zeroed; the staging slot goes to the store warp
            tc_fence_before();
            if (stores_bf) fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sfree[sl]);
                mbar_arrive(&edone[slot]);
            }
          }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// input-row ring depth of the conv (0: the most that fits shared memory)
std::atomic<int> g_fold_ring{0};

template <int NOUT, int OPER>
mrs_status launch_fold(const TcConvArgs& a, cudaStream_t st)
{
    int smax = 4;
    while (fold_smem_bytes<NOUT, OPER>(smax + 1) <= 227 * 1024 && smax < 12) ++smax;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_fold<NOUT, OPER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fold_smem_bytes<NOUT, OPER>(smax));
        if (e != cudaSuccess) return cuda_status(e, "conv smem attribute");
        attr = true;
    }
    const int want = g_fold_ring.load(std::memory_order_relaxed);
    const int stages = want >= 3 ? (want < smax ? want : smax) : smax;
    size_t smem = fold_smem_bytes<NOUT, OPER>(stages);
    TcConvArgs b = a;
    const long long T = (long long)a.N * ((a.W + kFoldTile - 1) / kFoldTile) * a.H;
    int grid = T < sm_count() ? (int)T : sm_count();
    if (grid < 1) return MRS_OK;
    const CUtensorMap* res = a.tmap_res ? a.tmap_res : a.tmap_x;
    const CUtensorMap* out = a.tmap_out ? a.tmap_out : a.tmap_x;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    cudaError_t le = cudaSuccess;
    MRS_TIMED(PK_CONV_TC, st, (le = cudaLaunchKernelEx(&cfg, k_conv_fold<NOUT, OPER>, *a.tmap_x, *a.tmap_w, *res, *out, b, stages)));
    MRS_LAUNCHED(1);
    if (le != cudaSuccess) return cuda_status(le, "conv launch");
    return cuda_status(cudaGetLastError(), "conv launch");
}

}  // namespace

mrs_status tc_make_act_map(CUtensorMap* m, const void* ptr, int N, int H, int W, int operand,
                           int box_px)
{
    auto fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled unavailable"); return MRS_ERR_CUDA; }
    int rowb = operand == TC_BF16 ? 128 : 64;
    cuuint64_t dims[4] = {64, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    cuuint64_t strides[3] = {(cuuint64_t)rowb, (cuuint64_t)rowb * W, (cuuint64_t)rowb * W * H};
    cuuint32_t box[4] = {64, (cuuint32_t)box_px, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, operand == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                    4, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    operand == TC_BF16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled(act) failed: %d", (int)r); return MRS_ERR_CUDA; }
    return MRS_OK;
}

mrs_status tc_make_view_map(CUtensorMap* m, const void* ptr, int N, int H, int W,
                            long long px_stride, long long row_stride, long long img_stride,
                            int box_px)
{
    auto fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled unavailable"); return MRS_ERR_CUDA; }
    if (((uintptr_t)ptr & 15) || (px_stride & 15) || (row_stride & 15) || (img_stride & 15)) {
        set_error("tc_make_view_map: base and strides must be multiples of 16 bytes");
        return MRS_ERR_ARG;
    }
    cuuint64_t dims[4] = {64, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    cuuint64_t strides[3] = {(cuuint64_t)px_stride, (cuuint64_t)row_stride, (cuuint64_t)img_stride};
    cuuint32_t box[4] = {64, (cuuint32_t)box_px, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled(view) failed: %d", (int)r); return MRS_ERR_CUDA; }
    return MRS_OK;
}

mrs_status tc_make_w_map(CUtensorMap* m, const void* ptr, int rows, int nout, int operand)
{
    auto fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled unavailable"); return MRS_ERR_CUDA; }
    int rowb = operand == TC_BF16 ? 128 : 64;
    cuuint64_t dims[2] = {64, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)rowb};
    cuuint32_t box[2] = {64, (cuuint32_t)nout};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, operand == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                    2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    operand == TC_BF16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled(w) failed: %d", (int)r); return MRS_ERR_CUDA; }
    return MRS_OK;
}

namespace {
// waits on an mbarrier that nothing completes; the bounded wait must give up,
// raise the error word and return (exercises the kernels' timeout path)
__global__ void k_wait_selftest(int* err, long long limit_cycles, int* gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = mbar_wait_limit(&bar, 0, err, limit_cycles, 1000u);
        *gave_up = ok ? 0 : 1;
    }
}
}  // namespace

mrs_status tc_wait_selftest(long long limit_cycles, int* gave_up, cudaStream_t st)
{
    int* d = nullptr;
    MRS_CHECK(cudaMalloc(&d, 2 * sizeof(int)));
    MRS_CHECK(cudaMemsetAsync(d, 0, 2 * sizeof(int), st));
    k_wait_selftest<<<1, 32, 0, st>>>(d, limit_cycles, d + 1);
    MRS_LAUNCHED(1);
    int h[2] = {0, 0};
    mrs_status rc = cuda_status(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st), "selftest copy");
    if (rc == MRS_OK) rc = cuda_status(cudaStreamSynchronize(st), "selftest sync");
    cudaFree(d);
    if (rc != MRS_OK) return rc;
    *gave_up = h[1] && h[0];
    return MRS_OK;
}

void tc_set_ring(int stages) { g_fold_ring.store(stages, std::memory_order_relaxed); }

mrs_status tc_conv3x3(const TcConvArgs& a, cudaStream_t st)
{
    if (a.kc > 1 && (!a.amaps || ((uintptr_t)a.amaps & 63))) {
        set_error("tc_conv3x3: kc > 1 needs a 64-byte aligned device array of kc maps");
        return MRS_ERR_ARG;
    }
    if (a.nout == 64) return a.operand == TC_BF16 ? launch_fold<64, TC_BF16>(a, st) : launch_fold<64, TC_FP8>(a, st);
    if (a.nout == 16) return a.operand == TC_BF16 ? launch_fold<16, TC_BF16>(a, st) : launch_fold<16, TC_FP8>(a, st);
    set_error("tc_conv3x3: nout must be 64 or 16");
    return MRS_ERR_ARG;
}


// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: the GEMM
//     D[(t, c)][o] = sum_p x[p + shift_t][c] * dy[p][o]
// with K = pixels.  Both tensors keep their [pixel][64-channel] layout, which
// for this GEMM is MN-major (the M or N index is the contiguous one): a TMA
// box of pixels with 128-byte swizzled rows is the canonical MN-major
// SWIZZLE_128B operand, one 128-byte row per K index, 8-row groups 1024 bytes
// apart.  M = 128 is made of two 64-channel MN atoms LBO bytes apart, so one
// MMA covers two taps:
//   MMA dx     (dx = 0..2): rows 0-63 tap (ky 0, dx), rows 64-127 tap (ky 1, dx)
//                           (input rows y-1 and y sit in slots RB bytes apart)
//   MMA 3 + dx            : rows 0-63 tap (ky 2, dx), rows 64-127 read a
//                           region of ones, which makes those rows db[o]
// A job is kWgKB output pixels of one image row.  Per job the producer loads
// input rows y-1, y, y+1 (kWgKB + 2 pixels from x0 - 1, zero-filled outside
// the image: the zero padding) and dy row y (kWgKB pixels); the kx shift is a
// descriptor start offset of kx 128-byte rows.  Each CTA takes a contiguous
// run of jobs, accumulates all 9 taps in TMEM (6 x 64 fp32 columns) and writes
// one partial; the partials are summed by a separate reduction.
// Warp 0 lane 0: TMA producer; warp 1: TMEM allocator, lane 0 MMA issuer;
// warps 0-3: epilogue (warp w reads TMEM lanes 32w .. 32w + 31).
namespace {

constexpr int kWgThreads = 128;
constexpr int kWgRB = ((kWgKB + 2) * 128 + 1023) & ~1023;   // one input-row slot
constexpr int kWgBB = kWgKB * 128;                           // dy slot
constexpr int kWgStage = 3 * kWgRB + kWgBB;
constexpr uint32_t kWgTx = 3 * (kWgKB + 2) * 128 + kWgKB * 128;   // bytes landed per job

// MN-major SWIZZLE_128B descriptor: `lbo` = bytes to the next 64-element MN
// atom, SBO = 1024 bytes to the next group of 8 K rows
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// waits for a phase regardless of the error word (used to drain copies in
// flight before the CTA exits); gives up after `limit_cycles`
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, long long limit_cycles)
{
    long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, 100000u))
        if (clock64() - t0 > limit_cycles) return;
}

__global__ void __launch_bounds__(kWgThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_dy,
               TcWgradArgs a, int stages)
{
    // kind::f16, D f32, A and B bf16, both MN-major, N = 64, M = 128
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t kTmemCols = 512;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sOnes = smem + (size_t)stages * kWgStage;
    uint64_t* full = (uint64_t*)(sOnes + kWgRB);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tslot = (uint32_t*)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int XS = (a.W + kWgKB - 1) / kWgKB;
    const long long njobs = (long long)a.N * a.H * XS;
    const long long j0 = njobs * blockIdx.x / gridDim.x;
    const long long j1 = njobs * (blockIdx.x + 1) / gridDim.x;

    for (int i = threadIdx.x; i < kWgRB / 4; i += kWgThreads) ((uint32_t*)sOnes)[i] = 0x3F803F80u;  // bf16 1.0
    fence_async_smem();
    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *(volatile uint32_t*)tslot;

    if (warp == 0 && lane == 0) {
        uint32_t it = 0, ph = 0;
        int s = 0;
        for (long long j = j0; j < j1; ++j, ++it, s = (s + 1 == stages ? 0 : s + 1),
                       ph ^= (s == 0 ? 1u : 0u)) {
            int xs = (int)(j % XS);
            long long rest = j / XS;
            int y = (int)(rest % a.H), n = (int)(rest / a.H);
            if (!mbar_wait(&empty[s], ph ^ 1, a.err)) break;
            mbar_expect_tx(&full[s], kWgTx);
            uint8_t* sb = smem + (size_t)s * kWgStage;
            for (int r = 0; r < 3; ++r)
                tma_load_4d(sb + r * kWgRB, &tmap_x, 0, xs * kWgKB - 1, y - 1 + r, n, &full[s]);
            tma_load_4d(sb + 3 * kWgRB, &tmap_dy, 0, xs * kWgKB, y, n, &full[s]);
        }
        // no copy may still be landing when the CTA exits
        for (uint32_t i = it > (uint32_t)stages ? it - stages : 0; i < it; ++i)
            mbar_drain(&full[i % stages], (i / stages) & 1, kTimeoutCycles);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer.  A job's 24 MMAs use 6 A descriptors (tap pairs q) and
        // one B descriptor, all built once per job; each K step of 16 pixels
        // (2048 bytes further into every operand) only adds 2048 / 16 = 128
        // to their start-address field (bits 0-13; shared-memory addresses
        // stay far below the field's 256 KB).  The ring slot and its phase
        // advance incrementally (no division per job).
        const uint32_t ones = smem_u32(sOnes);
        const uint32_t sbase = smem_u32(smem);
        uint32_t it = 0, ph = 0;
        int s = 0;
        for (long long j = j0; j < j1; ++j, ++it) {
            if (!mbar_wait(&full[s], ph, a.err)) break;
            tc_fence_after();
            const uint32_t base = sbase + (uint32_t)s * kWgStage;
            const uint32_t top2 = base + 2 * kWgRB;
            uint64_t ad[6];
#pragma unroll
            for (int q = 0; q < 6; ++q)
                ad[q] = sdesc_mn((q < 3 ? base : top2) + (q % 3) * 128,
                                 q < 3 ? (uint32_t)kWgRB : ones - top2);
            const uint64_t bd0 = sdesc_mn(base + 3 * kWgRB, kWgBB);
#pragma unroll
            for (int kk = 0; kk < kWgKB / 16; ++kk) {
                const uint64_t step = (uint64_t)(kk * 128);
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    mma_f16(tmem + q * 64, ad[q] + step, bd0 + step, IDESC,
                            (it > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            if (++s == stages) { s = 0; ph ^= 1u; }
        }
        mma_commit(done);   // arrives once every MMA issued above has completed
    }
    __syncwarp();

    const bool ok = mbar_wait_warp(done, 0, a.err);
    tc_fence_after();
    if (ok) {
        const bool have = j1 > j0;
        const int m = 32 * warp + lane, c = m & 63;
        float* P = a.part + (size_t)blockIdx.x * 9 * a.cout * a.cin;
        for (int q = 0; q < 6; ++q) {
            // TMEM lane m of MMA q: tap t (or the bias row when t < 0)
            const int t = q < 3 ? (m < 64 ? q : 3 + q) : (m < 64 ? 3 + q : -1);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + q * 64 + h * 16, r);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int o = h * 16 + i;
                    const float v = have ? __uint_as_float(r[i]) : 0.0f;
                    if (o >= a.cout) continue;
                    if (t >= 0) {
                        if (c < a.cin) P[((size_t)t * a.cout + o) * a.cin + c] = v;
                    } else if (q == 3 && m == 64) {
                        a.dbpart[(size_t)blockIdx.x * a.cout + o] = v;
                    }
                }
            }
        }
    }
    // on the error path the MMAs may still run: TMEM is freed only after them
    if (!ok && warp == 1 && lane == 0) mbar_drain(done, 0, kTimeoutCycles);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

size_t wgrad_smem(int stages)
{
    return 1024 + (size_t)stages * kWgStage + kWgRB + 8 * (2 * stages + 1) + 16;
}

}  // namespace

int tc_wgrad_max_parts() { return sm_count(); }

mrs_status tc_conv3x3_wgrad(const TcWgradArgs& a, int* nparts, cudaStream_t st)
{
    if (a.cin < 1 || a.cin > 64 || a.cout < 1 || a.cout > 64) {
        set_error("tc_conv3x3_wgrad: cin, cout must be in [1, 64]");
        return MRS_ERR_ARG;
    }
    int stages = 2;
    while (wgrad_smem(stages + 1) <= 227 * 1024 && stages < 8) ++stages;
    size_t smem = wgrad_smem(stages);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e, "wgrad smem attribute");
        attr = true;
    }
    long long njobs = (long long)a.N * a.H * ((a.W + kWgKB - 1) / kWgKB);
    const int cap = a.max_ctas > 0 && a.max_ctas < sm_count() ? a.max_ctas : sm_count();
    int grid = njobs < cap ? (int)njobs : cap;
    *nparts = grid;
    if (grid < 1) return MRS_OK;
    MRS_TIMED(PK_WGRAD_TC, st, (k_wgrad_tc<<<grid, kWgThreads, smem, st>>>(*a.tmap_x, *a.tmap_dy, a, stages)));
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "wgrad launch");
}

}  // namespace mrs
