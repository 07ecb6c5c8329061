// Render-tree construction on the GPU: centroid bounds, 30-bit Morton codes,
// a stable LSD radix sort of (code, triangle index), then the binary radix
// tree of Karras (HPG 2012) with a bottom-up box refit, or locally-ordered
// clustering over the sorted leaves (in grid-wide rounds, or inside the radix
// tree's subtrees in one launch); every tree is written in the same traversal
// node layout (both child boxes + child ids in one 64-byte node).
//
// Compiled with --fmad=false: the Morton quantisation must round exactly like
// the oracle's ((v0 + v1) + v2) * (1/3), (c - lo) * (1024 / extent).
#include <float.h>
#include <stdarg.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "../../synth/scenegen.h"

namespace mrs {

static thread_local char g_err[512];
void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* last_error() { return g_err; }

std::atomic<unsigned long long>& launch_counter()
{
    static std::atomic<unsigned long long> c{0};
    return c;
}

namespace {
struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PK_COUNT];
};
Prof& prof()
{
    static Prof p;
    return p;
}
}  // namespace

bool prof_on() { return prof().on; }
cudaEvent_t prof_record(cudaStream_t st)
{
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, st);
    return e;
}
void prof_push(int k, cudaEvent_t a, cudaEvent_t b)
{
    if (!b) { cudaEventDestroy(a); return; }
    std::lock_guard<std::mutex> g(prof().mu);
    prof().ev[k].push_back({a, b});
}

namespace {

constexpr int kBlock = 256;
constexpr int kSortItems = 8;                 // keys per thread per sort tile
constexpr int kTile = kBlock * kSortItems;    // 2048 keys per tile

__device__ __forceinline__ float centroid(const float* V, int i, int a)
{
    const float* p = V + (size_t)i * 9;
    return ((p[a] + p[3 + a]) + p[6 + a]) * 0.333333343267f;
}

// per-block min/max of centroids -> part[block][6]; over triangles idx[0..n)
// (or 0..n-1 when idx is NULL)
__global__ void k_bounds_partial(const float* __restrict__ V, int n, float* __restrict__ part,
                                 const int* __restrict__ idx = nullptr)
{
    __shared__ float s[6][kBlock];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = blockIdx.x * kBlock + threadIdx.x; k < n; k += gridDim.x * kBlock)
        for (int a = 0; a < 3; ++a) {
            float c = centroid(V, idx ? idx[k] : k, a);
            lo[a] = fminf(lo[a], c);
            hi[a] = fmaxf(hi[a], c);
        }
    for (int a = 0; a < 3; ++a) { s[a][threadIdx.x] = lo[a]; s[3 + a][threadIdx.x] = hi[a]; }
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fminf(s[a][threadIdx.x], s[a][threadIdx.x + w]);
                s[3 + a][threadIdx.x] = fmaxf(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// reduce the partials (one block) and emit Morton codes (grid-stride) of
// triangles idx[0..n) (or 0..n-1): keys[k], vals[k] = triangle; codes[triangle]
// too when codes is not NULL
__global__ void k_morton(const float* __restrict__ V, int n, const float* __restrict__ part,
                         int nparts, uint32_t* __restrict__ codes, uint32_t* __restrict__ keys,
                         int* __restrict__ vals, const int* __restrict__ idx = nullptr)
{
    __shared__ float lo[3], sc[3];
    if (threadIdx.x < 32) {
        // the first warp: partials strided over its lanes, then a butterfly
        // (min and max are exact, so the order does not matter)
        float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b = threadIdx.x; b < nparts; b += 32)
            for (int a = 0; a < 3; ++a) {
                l[a] = fminf(l[a], part[b * 6 + a]);
                h[a] = fmaxf(h[a], part[b * 6 + 3 + a]);
            }
        for (int off = 16; off > 0; off >>= 1)
            for (int a = 0; a < 3; ++a) {
                l[a] = fminf(l[a], __shfl_xor_sync(0xffffffffu, l[a], off));
                h[a] = fmaxf(h[a], __shfl_xor_sync(0xffffffffu, h[a], off));
            }
        if (threadIdx.x == 0)
            for (int a = 0; a < 3; ++a) {
                const float ext = h[a] - l[a];
                lo[a] = l[a];
                sc[a] = ext > 0.0f ? 1024.0f / ext : 0.0f;
            }
    }
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = idx ? idx[k] : k;
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            float f = (centroid(V, i, a) - lo[a]) * sc[a];
            if (!(f > 0.0f)) f = 0.0f;
            uint32_t u = (uint32_t)f;
            q[a] = u > 1023u ? 1023u : u;
        }
        uint32_t code = 0;
        for (int b = 0; b < 10; ++b)
            code |= (((q[0] >> b) & 1u) << (3 * b + 2)) | (((q[1] >> b) & 1u) << (3 * b + 1)) |
                    (((q[2] >> b) & 1u) << (3 * b));
        if (codes) codes[i] = code;
        keys[k] = code;
        vals[k] = i;
    }
}

// ---- stable LSD radix sort, 8-bit digits ---------------------------------
__global__ void k_sort_hist(const uint32_t* __restrict__ keys, int n, int shift,
                            uint32_t* __restrict__ counts, int ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kTile;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kBlock + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of counts[0..m) in place, one block of 1024 threads: warp w
// owns a contiguous chunk, which it reads 32 consecutive counts at a time
// (coalesced); a first pass sums each chunk, one warp scans the 32 chunk
// totals, and a second pass scans each chunk group by group by shuffles,
// carrying the running offset (integer sums: the order does not change the
// result)
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ counts, int m)
{
    __shared__ uint32_t s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = ((m + 31) / 32 + 31) & ~31;
    const int b0 = warp * chunk;
    uint32_t sum = 0;
#pragma unroll 8
    for (int k = lane; k < chunk; k += 32) {
        const int i = b0 + k;
        if (i < m) sum += counts[i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) s[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += t;
        }
        s[lane] = w;
    }
    __syncthreads();
    uint32_t carry = warp > 0 ? s[warp - 1] : 0u;
#pragma unroll 4
    for (int k = lane; k < chunk; k += 32) {
        const int i = b0 + k;
        const uint32_t v = i < m ? counts[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += t;
        }
        if (i < m) counts[i] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
}

// scatter: rank of each key among equal digits = tile offset + keys before it
// in the tile (round-major, then warp, then lane order == index order)
__global__ void k_sort_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                               uint32_t* __restrict__ kout, int* __restrict__ vout, int n,
                               int shift, const uint32_t* __restrict__ offs, int ntiles)
{
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[kBlock / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = offs[threadIdx.x * ntiles + blockIdx.x];
    int base = blockIdx.x * kTile;
    for (int k = 0; k < kSortItems; ++k) {
        for (int w = 0; w < kBlock / 32; ++w) wc[w][threadIdx.x] = 0;
        __syncthreads();
        int i = base + k * kBlock + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        unsigned lt = (1u << lane) - 1u;
        uint32_t lrank = __popc(peers & lt);
        if (valid && lrank == 0) wc[warp][digit] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps; advance the running offset
        {
            uint32_t acc = 0;
            for (int w = 0; w < kBlock / 32; ++w) {
                uint32_t c = wc[w][threadIdx.x];
                wc[w][threadIdx.x] = acc;
                acc += c;
            }
            wc[0][threadIdx.x] += 0;   // keep layout; prefix stored in wc
            __syncthreads();
            if (valid) {
                uint32_t pos = run[digit] + wc[warp][digit] + lrank;
                kout[pos] = key;
                vout[pos] = vin[i];
            }
            __syncthreads();
            run[threadIdx.x] += acc;
        }
        __syncthreads();
    }
}

// ---- Karras radix tree ------------------------------------------------------
__device__ __forceinline__ int delta(const uint32_t* code, const int* order, int n, int i, int j)
{
    if (j < 0 || j > n - 1) return -1;
    uint64_t a = ((uint64_t)code[i] << 32) | (uint32_t)order[i];
    uint64_t b = ((uint64_t)code[j] << 32) | (uint32_t)order[j];
    return __clzll(a ^ b);
}

__global__ void k_karras(const uint32_t* __restrict__ code, const int* __restrict__ order, int n,
                         int* __restrict__ left, int* __restrict__ right, int* __restrict__ parent)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(code, order, n, i, i + 1) - delta(code, order, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = delta(code, order, n, i, i - d);
    int lmax = 2;
    while (delta(code, order, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(code, order, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(code, order, n, i, j);
    int s = 0, div = 2, t;
    do {
        t = (l + div - 1) / div;
        if (delta(code, order, n, i, i + (s + t) * d) > dnode) s += t;
        div <<= 1;
    } while (t > 1);
    int gamma = i + s * d + (d < 0 ? -1 : 0);
    int L = (min(i, j) == gamma) ? (n - 1) + gamma : gamma;
    int R = (max(i, j) == gamma + 1) ? (n - 1) + gamma + 1 : gamma + 1;
    left[i] = L;
    right[i] = R;
    parent[L] = i;
    parent[R] = i;
    if (i == 0) parent[0] = -1;
}

// leaves: sorted triangle records, material/light, leaf boxes
__global__ void k_leaves(const float* __restrict__ V, const int* __restrict__ tri_mat,
                         const int* __restrict__ tri_light, const int* __restrict__ order, int n,
                         float4* __restrict__ tris, int2* __restrict__ tri_ml,
                         float* __restrict__ box, int* __restrict__ visit)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n - 1) visit[k] = 0;
    if (k >= n) return;
    int prim = order[k];
    const float* p = V + (size_t)prim * 9;
    float v0x = p[0], v0y = p[1], v0z = p[2];
    tris[3 * k + 0] = make_float4(v0x, v0y, v0z, __int_as_float(prim));
    tris[3 * k + 1] = make_float4(p[3] - v0x, p[4] - v0y, p[5] - v0z, 0.0f);
    tris[3 * k + 2] = make_float4(p[6] - v0x, p[7] - v0y, p[8] - v0z, 0.0f);
    tri_ml[k] = make_int2(tri_mat[prim], tri_light[prim]);
    float* b = box + (size_t)(n - 1 + k) * 6;
    for (int a = 0; a < 3; ++a) {
        b[a] = fminf(fminf(p[a], p[3 + a]), p[6 + a]);
        b[3 + a] = fmaxf(fmaxf(p[a], p[3 + a]), p[6 + a]);
    }
}

// records of the exhaustively tested (large) triangles at positions ns..n-1
__global__ void k_big_leaves(const float* __restrict__ V, const int* __restrict__ tri_mat,
                             const int* __restrict__ tri_light, const int* __restrict__ big_idx,
                             int ns, int nb, int* __restrict__ order, float4* __restrict__ tris,
                             int2* __restrict__ tri_ml)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int prim = big_idx[b], k = ns + b;
    const float* p = V + (size_t)prim * 9;
    float v0x = p[0], v0y = p[1], v0z = p[2];
    order[k] = prim;
    tris[3 * k + 0] = make_float4(v0x, v0y, v0z, __int_as_float(prim));
    tris[3 * k + 1] = make_float4(p[3] - v0x, p[4] - v0y, p[5] - v0z, 0.0f);
    tris[3 * k + 2] = make_float4(p[6] - v0x, p[7] - v0y, p[8] - v0z, 0.0f);
    tri_ml[k] = make_int2(tri_mat[prim], tri_light[prim]);
}

// atomic add at GPU scope: acquire-release (publishes the box this thread
// wrote before it), or acquire only (a leaf's box comes from an earlier kernel)
__device__ __forceinline__ int add_acq_rel(int* p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int add_acquire(int* p, int v)
{
    int old;
    asm volatile("atom.acquire.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// bottom-up refit: the second child to arrive at a parent computes its box
// and writes the 64-byte traversal node (both child boxes + child ids)
__global__ void k_refit(int n, const int* __restrict__ left, const int* __restrict__ right,
                        const int* __restrict__ parent, float* box, int* visit,
                        float4* __restrict__ nodes)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int node = parent[(n - 1) + k];
    bool wrote = false;
    while (node >= 0) {
        // first arrival: the sibling finishes (the exchange releases the box
        // written below, and acquires the sibling's)
        if ((wrote ? add_acq_rel(&visit[node], 1) : add_acquire(&visit[node], 1)) == 0) return;
        wrote = true;
        int l = left[node], r = right[node];
        const volatile float* bl = box + (size_t)l * 6;
        const volatile float* br = box + (size_t)r * 6;
        float L[6], R[6];
        for (int a = 0; a < 6; ++a) { L[a] = bl[a]; R[a] = br[a]; }
        float* b = box + (size_t)node * 6;
        for (int a = 0; a < 3; ++a) {
            b[a] = fminf(L[a], R[a]);
            b[3 + a] = fmaxf(L[3 + a], R[3 + a]);
        }
        nodes[4 * node + 0] = make_float4(L[0], L[1], L[2], L[3]);
        nodes[4 * node + 1] = make_float4(L[4], L[5], R[0], R[1]);
        nodes[4 * node + 2] = make_float4(R[2], R[3], R[4], R[5]);
        nodes[4 * node + 3] = make_float4(__int_as_float(l), __int_as_float(r), 0.0f, 0.0f);
        node = parent[node];
    }
}

inline int blocks_for(int64_t n, int per) { return (int)((n + per - 1) / per); }

// ---- locally-ordered clustering (the render tree) ---------------------------
// The tree the renders traverse is built bottom-up by agglomerative
// clustering over the Morton-sorted leaves (Meister & Bittner, "Parallel
// Locally-Ordered Clustering for Bounding Volume Hierarchy Construction"):
// every cluster finds the neighbour within kPlocR positions of the sorted
// cluster list whose merged box has the smallest surface area (ties broken by
// a hash of the position pair, then by the smaller position: a strict order
// on pairs, so at least one pair is mutual; ordering ties by position alone
// would chain equal boxes and merge one pair per round), every mutual pair
// merges into a new node at the
// lower position, and the list is compacted; repeated until one cluster is
// left.  Internal node ids are handed out downwards from ns - 2 in merge
// order, so the root (the last merge) is node 0; leaves keep the LBVH's ids
// (ns - 1 + sorted position).  Nodes are written at merge time in the same
// 64-byte layout as k_refit's.  Its surface-area cost is about 20% below the
// LBVH's on the procedural scenes and renders take 6-8% less time, but its
// build takes about 3x the LBVH's (some 20 short rounds at 200k triangles), so
// it is the choice for a scene built once and rendered many times, and the
// LBVH stays the default.  The closest hit does not depend on the tree.
constexpr int kPlocR = 16;          // search radius (positions)
constexpr int kPlocCap = 2048;      // clusters the single-block finish takes
constexpr int kPlocIters = 64;      // bound on the grid-wide iterations
constexpr int kPlocBatch = 24;      // grid-wide rounds per graph / per count read-back (200k
                                    // triangles need 20 before the finish takes over)

// half the surface area of the union of two boxes (lo.xyz, hi.x | hi.yz)
__device__ __forceinline__ float union_half_area(float4 a0, float4 a1, float4 b0, float4 b1)
{
    float ex = fmaxf(a0.w, b0.w) - fminf(a0.x, b0.x);
    float ey = fmaxf(a1.x, b1.x) - fminf(a0.y, b0.y);
    float ez = fmaxf(a1.y, b1.y) - fminf(a0.z, b0.z);
    return ex * ey + ey * ez + ez * ex;
}

// tie-break key of the unordered position pair (i, j): the finaliser of
// MurmurHash3 (Appleby) over min * 2^16 + max mixed with the golden-ratio word
__device__ __forceinline__ uint32_t pair_key(int i, int j)
{
    uint32_t x = (uint32_t)min(i, j) * 0x9E3779B1u ^ (uint32_t)max(i, j);
    x ^= x >> 16; x *= 0x85EBCA6Bu;
    x ^= x >> 13; x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}
// candidate (a, h, j) ahead of the best so far (ba, bh, bj)
__device__ __forceinline__ bool nn_ahead(float a, uint32_t h, int j, float ba, uint32_t bh, int bj)
{
    return a < ba || (a == ba && (h < bh || (h == bh && j < bj)));
}

// the node record of a merge (children a, b with their boxes) and the merged box
__device__ __forceinline__ void ploc_write_node(int id, int ca, float4 a0, float4 a1, int cb,
                                                float4 b0, float4 b1, float4* __restrict__ nodes,
                                                float* __restrict__ box, float4& u0, float4& u1)
{
    nodes[4 * id + 0] = make_float4(a0.x, a0.y, a0.z, a0.w);
    nodes[4 * id + 1] = make_float4(a1.x, a1.y, b0.x, b0.y);
    nodes[4 * id + 2] = make_float4(b0.z, b0.w, b1.x, b1.y);
    nodes[4 * id + 3] = make_float4(__int_as_float(ca), __int_as_float(cb), 0.0f, 0.0f);
    u0 = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), fmaxf(a0.w, b0.w));
    u1 = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), 0.0f, 0.0f);
    float* bx = box + (size_t)id * 6;
    bx[0] = u0.x; bx[1] = u0.y; bx[2] = u0.z; bx[3] = u0.w; bx[4] = u1.x; bx[5] = u1.y;
}

// clusters = the sorted leaves; counts of iteration 0
__global__ void k_ploc_init(int ns, const float* __restrict__ box, int* __restrict__ ids,
                            float4* __restrict__ cb, int* cnt, int* nxt, int* err)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) { cnt[0] = ns; nxt[0] = ns - 2; *err = 0; }
    if (k >= ns) return;
    const float* b = box + (size_t)(ns - 1 + k) * 6;
    ids[k] = ns - 1 + k;
    cb[2 * k] = make_float4(b[0], b[1], b[2], b[3]);
    cb[2 * k + 1] = make_float4(b[4], b[5], 0.0f, 0.0f);
}

// nearest neighbour of every cluster (positions i - R .. i + R), through a
// shared-memory window of the block's clusters and their halo
__global__ void __launch_bounds__(256) k_ploc_nn(const float4* __restrict__ cb, const int* cnt,
                                                 int it, int* __restrict__ nn)
{
    __shared__ float4 s[256 + 2 * kPlocR][2];
    const int N = cnt[it];
    const int b0 = blockIdx.x * 256;
    if (N <= kPlocCap || b0 >= N) return;
    for (int t = threadIdx.x; t < 256 + 2 * kPlocR; t += 256) {
        int g = b0 - kPlocR + t;
        if (g >= 0 && g < N) { s[t][0] = cb[2 * g]; s[t][1] = cb[2 * g + 1]; }
    }
    __syncthreads();
    const int i = b0 + threadIdx.x;
    if (i >= N) return;
    const float4 a0 = s[threadIdx.x + kPlocR][0], a1 = s[threadIdx.x + kPlocR][1];
    float best = INFINITY;
    uint32_t bh = 0xFFFFFFFFu;
    int bj = -1;
    for (int d = -kPlocR; d <= kPlocR; ++d) {
        const int j = i + d;
        if (d == 0 || j < 0 || j >= N) continue;
        const float a = union_half_area(a0, a1, s[threadIdx.x + kPlocR + d][0], s[threadIdx.x + kPlocR + d][1]);
        const uint32_t h = pair_key(i, j);
        if (nn_ahead(a, h, j, best, bh, bj)) { best = a; bh = h; bj = j; }
    }
    nn[i] = bj;
}

// keep (not the upper member of a mutual pair) and lead (the lower member)
__device__ __forceinline__ void ploc_flags(const int* __restrict__ nn, int i, int N, int& keep,
                                           int& lead)
{
    keep = 0;
    lead = 0;
    if (i >= N) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    keep = !(mutual && j < i);
    lead = mutual && i < j;
}

// exclusive block-wide ranks of two flags (256 threads) and the block's totals
__device__ __forceinline__ void block_rank2(int a, int b, int& ra, int& rb, int& ta, int& tb)
{
    __shared__ int sa[8], sb[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ma = __ballot_sync(0xffffffffu, a), mb = __ballot_sync(0xffffffffu, b);
    const unsigned below = (1u << lane) - 1u;
    if (lane == 0) { sa[w] = __popc(ma); sb[w] = __popc(mb); }
    __syncthreads();
    int oa = 0, ob = 0;
    ta = 0;
    tb = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) { oa += sa[k]; ob += sb[k]; }
        ta += sa[k];
        tb += sb[k];
    }
    ra = oa + __popc(ma & below);
    rb = ob + __popc(mb & below);
    __syncthreads();
}

// per block: clusters kept and merges led
__global__ void __launch_bounds__(256) k_ploc_count(const int* __restrict__ nn, const int* cnt, int it,
                                                    int2* __restrict__ blk)
{
    const int N = cnt[it];
    const int b0 = blockIdx.x * 256;
    if (N <= kPlocCap || b0 >= N) return;
    int keep, lead, rk, rl, tk, tl;
    ploc_flags(nn, b0 + threadIdx.x, N, keep, lead);
    block_rank2(keep, lead, rk, rl, tk, tl);
    if (threadIdx.x == 0) blk[blockIdx.x] = make_int2(tk, tl);
}

// exclusive scan of the block totals (one block of 1024); counts of the next iteration
__global__ void __launch_bounds__(1024) k_ploc_scan(int2* __restrict__ blk, int* cnt, int* nxt, int it)
{
    __shared__ int2 s[1024];
    __shared__ int2 carry;
    const int N = cnt[it];
    if (N <= kPlocCap) {
        if (threadIdx.x == 0) { cnt[it + 1] = N; nxt[it + 1] = nxt[it]; }
        return;
    }
    const int nb = (N + 255) / 256;
    if (threadIdx.x == 0) carry = make_int2(0, 0);
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        int2 v = i < nb ? blk[i] : make_int2(0, 0);
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {     // inclusive Hillis-Steele scan
            int2 t = threadIdx.x >= off ? s[threadIdx.x - off] : make_int2(0, 0);
            __syncthreads();
            s[threadIdx.x].x += t.x;
            s[threadIdx.x].y += t.y;
            __syncthreads();
        }
        const int2 c = carry;
        if (i < nb) blk[i] = make_int2(c.x + s[threadIdx.x].x - v.x, c.y + s[threadIdx.x].y - v.y);
        __syncthreads();
        if (threadIdx.x == 1023) carry = make_int2(c.x + s[1023].x, c.y + s[1023].y);
        __syncthreads();
    }
    if (threadIdx.x == 0) { cnt[it + 1] = carry.x; nxt[it + 1] = nxt[it] - carry.y; }
}

// compaction into the other cluster buffer; every lead writes its merge's node
__global__ void __launch_bounds__(256) k_ploc_compact(const int* __restrict__ ids,
                                                      const float4* __restrict__ cb,
                                                      const int* __restrict__ nn,
                                                      const int2* __restrict__ blk, const int* cnt,
                                                      const int* nxt, int it, int* __restrict__ ids_o,
                                                      float4* __restrict__ cb_o,
                                                      float4* __restrict__ nodes,
                                                      float* __restrict__ box)
{
    const int N = cnt[it];
    if (N <= kPlocCap) {    // the finish takes over: carry the clusters across unchanged
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
            ids_o[i] = ids[i];
            cb_o[2 * i] = cb[2 * i];
            cb_o[2 * i + 1] = cb[2 * i + 1];
        }
        return;
    }
    const int b0 = blockIdx.x * 256;
    if (b0 >= N) return;
    const int i = b0 + threadIdx.x;
    int keep, lead, rk, rl, tk, tl;
    ploc_flags(nn, i, N, keep, lead);
    block_rank2(keep, lead, rk, rl, tk, tl);
    if (!keep) return;
    const int2 off = blk[blockIdx.x];
    const int pos = off.x + rk;
    if (lead) {
        const int j = nn[i];
        const int id = nxt[it] - (off.y + rl);
        float4 u0, u1;
        ploc_write_node(id, ids[i], cb[2 * i], cb[2 * i + 1], ids[j], cb[2 * j], cb[2 * j + 1], nodes,
                        box, u0, u1);
        ids_o[pos] = id;
        cb_o[2 * pos] = u0;
        cb_o[2 * pos + 1] = u1;
    } else {
        ids_o[pos] = ids[i];
        cb_o[2 * pos] = cb[2 * i];
        cb_o[2 * pos + 1] = cb[2 * i + 1];
    }
}

// the last iterations (N <= kPlocCap clusters) in one block of 1024 threads,
// the clusters in shared memory; *err = 1 unless it ends with the root as node 0
constexpr size_t kPlocFinishSmem = (size_t)kPlocCap * (4 * sizeof(float4) + 3 * sizeof(int));
__global__ void __launch_bounds__(1024) k_ploc_finish(const int* __restrict__ ids_g,
                                                      const float4* __restrict__ cb_g, const int* cnt,
                                                      const int* nxt, int it,
                                                      float4* __restrict__ nodes,
                                                      float* __restrict__ box, int* err)
{
    extern __shared__ float4 sm[];
    __shared__ int wk[32], wl[32];
    float4* cbA = sm;
    float4* cbB = cbA + 2 * kPlocCap;
    int* idA = (int*)(cbB + 2 * kPlocCap);
    int* idB = idA + kPlocCap;
    int* snn = idB + kPlocCap;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int N = cnt[it], next = nxt[it];
    if (N > kPlocCap) {
        if (tid == 0) *err = 1;
        return;
    }
    for (int i = tid; i < N; i += 1024) {
        idA[i] = ids_g[i];
        cbA[2 * i] = cb_g[2 * i];
        cbA[2 * i + 1] = cb_g[2 * i + 1];
    }
    __syncthreads();
    for (int round = 0; round < kPlocCap && N > 1; ++round) {
        for (int i = tid; i < N; i += 1024) {
            const float4 a0 = cbA[2 * i], a1 = cbA[2 * i + 1];
            float best = INFINITY;
            uint32_t bh = 0xFFFFFFFFu;
            int bj = -1;
            for (int d = -kPlocR; d <= kPlocR; ++d) {
                const int j = i + d;
                if (d == 0 || j < 0 || j >= N) continue;
                const float a = union_half_area(a0, a1, cbA[2 * j], cbA[2 * j + 1]);
                const uint32_t h = pair_key(i, j);
                if (nn_ahead(a, h, j, best, bh, bj)) { best = a; bh = h; bj = j; }
            }
            snn[i] = bj;
        }
        __syncthreads();
        const int i0 = 2 * tid, i1 = 2 * tid + 1;
        int k0, l0, k1, l1;
        ploc_flags(snn, i0, N, k0, l0);
        ploc_flags(snn, i1, N, k1, l1);
        const int tk = k0 + k1, tl = l0 + l1;
        int xk = tk, xl = tl;
        for (int off = 1; off < 32; off <<= 1) {
            const int yk = __shfl_up_sync(0xffffffffu, xk, off), yl = __shfl_up_sync(0xffffffffu, xl, off);
            if (lane >= off) { xk += yk; xl += yl; }
        }
        if (lane == 31) { wk[w] = xk; wl[w] = xl; }
        __syncthreads();
        if (w == 0) {
            int a = wk[lane], b = wl[lane];
            for (int off = 1; off < 32; off <<= 1) {
                const int ya = __shfl_up_sync(0xffffffffu, a, off), yb = __shfl_up_sync(0xffffffffu, b, off);
                if (lane >= off) { a += ya; b += yb; }
            }
            wk[lane] = a;
            wl[lane] = b;
        }
        __syncthreads();
        const int ek = (w ? wk[w - 1] : 0) + xk - tk, el = (w ? wl[w - 1] : 0) + xl - tl;
        const int totK = wk[31], totL = wl[31];
        const int ii[2] = {i0, i1}, kk[2] = {k0, k1}, ll[2] = {l0, l1};
        for (int e = 0; e < 2; ++e) {
            if (!kk[e]) continue;
            const int i = ii[e];
            const int pos = ek + (e ? k0 : 0);
            if (ll[e]) {
                const int j = snn[i];
                const int id = next - (el + (e ? l0 : 0));
                float4 u0, u1;
                ploc_write_node(id, idA[i], cbA[2 * i], cbA[2 * i + 1], idA[j], cbA[2 * j],
                                cbA[2 * j + 1], nodes, box, u0, u1);
                idB[pos] = id;
                cbB[2 * pos] = u0;
                cbB[2 * pos + 1] = u1;
            } else {
                idB[pos] = idA[i];
                cbB[2 * pos] = cbA[2 * i];
                cbB[2 * pos + 1] = cbA[2 * i + 1];
            }
        }
        __syncthreads();
        N = totK;
        next -= totL;
        float4* tc = cbA; cbA = cbB; cbB = tc;
        int* ti = idA; idA = idB; idB = ti;
    }
    if (tid == 0 && (N != 1 || next != -1 || idA[0] != 0)) *err = 1;
}

// Scratch of the clustering build, carved from S->ploc_tmp
struct PlocBufs {
    float4* cb[2];       // cluster boxes (2 float4 each), ping-pong
    int* ids[2];         // cluster node ids, ping-pong
    int* nn;             // nearest neighbour of each position
    int2* blk;           // per-block (kept, merges) totals, then their prefix sums
    int* cnt;            // clusters at the start of round it
    int* nxt;            // next internal node id at the start of round it
    int* err;            // set by the finish unless it ends with the root as node 0
    int nb;              // 256-position blocks of the first round
};

mrs_status ploc_bufs(mrs_scene_s* S, PlocBufs& b)
{
    const int ns = S->ns;
    b.nb = (ns + 255) / 256;
    const size_t need = (size_t)ns * (2 * sizeof(int) + 4 * sizeof(float4) + sizeof(int)) +
                        (size_t)b.nb * sizeof(int2) + 2 * (kPlocIters + kPlocBatch + 2) * sizeof(int) +
                        sizeof(int) + 1024;
    mrs_status rc = S->ploc_tmp.ensure(need);
    if (rc != MRS_OK) return rc;
    char* p = S->ploc_tmp.as<char>();
    b.cb[0] = (float4*)p; p += (size_t)ns * 2 * sizeof(float4);
    b.cb[1] = (float4*)p; p += (size_t)ns * 2 * sizeof(float4);
    b.ids[0] = (int*)p; p += (size_t)ns * sizeof(int);
    b.ids[1] = (int*)p; p += (size_t)ns * sizeof(int);
    b.nn = (int*)p; p += (size_t)ns * sizeof(int);
    b.blk = (int2*)(((uintptr_t)p + 7) & ~(uintptr_t)7); p = (char*)(b.blk + b.nb);
    b.cnt = (int*)p; p += (kPlocIters + kPlocBatch + 2) * sizeof(int);
    b.nxt = (int*)p; p += (kPlocIters + kPlocBatch + 2) * sizeof(int);
    b.err = (int*)p;
    static bool attr_set[64] = {false};
    int dev = 0;
    MRS_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index %d out of range", dev); return MRS_ERR_CUDA; }
    if (!attr_set[dev]) {
        MRS_CHECK(cudaFuncSetAttribute(k_ploc_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPlocFinishSmem));
        attr_set[dev] = true;
    }
    return MRS_OK;
}

// rounds it0 .. it0 + kPlocBatch - 1 (4 kernels each)
void ploc_rounds(mrs_scene_s* S, const PlocBufs& b, int it0, cudaStream_t st)
{
    for (int it = it0; it < it0 + kPlocBatch; ++it) {
        const int a = it & 1;
        k_ploc_nn<<<b.nb, 256, 0, st>>>(b.cb[a], b.cnt, it, b.nn);
        k_ploc_count<<<b.nb, 256, 0, st>>>(b.nn, b.cnt, it, b.blk);
        k_ploc_scan<<<1, 1024, 0, st>>>(b.blk, b.cnt, b.nxt, it);
        k_ploc_compact<<<b.nb, 256, 0, st>>>(b.ids[a], b.cb[a], b.nn, b.blk, b.cnt, b.nxt, it,
                                             b.ids[a ^ 1], b.cb[a ^ 1], S->nodes, S->box);
    }
}

void ploc_finish(mrs_scene_s* S, const PlocBufs& b, int it, cudaStream_t st)
{
    k_ploc_finish<<<1, 1024, kPlocFinishSmem, st>>>(b.ids[it & 1], b.cb[it & 1], b.cnt, b.nxt, it,
                                                    S->nodes, S->box, b.err);
}

// the usual clustering build (after k_leaves): init, kPlocBatch rounds when
// the tree has more than kPlocCap leaves, the finish, the error word to the
// host (S->class_host[0]); returns the kernels enqueued
int ploc_enqueue(mrs_scene_s* S, const PlocBufs& b, cudaStream_t st)
{
    const int ns = S->ns;
    k_ploc_init<<<blocks_for(ns, kBlock), kBlock, 0, st>>>(ns, S->box, b.ids[0], b.cb[0], b.cnt, b.nxt,
                                                           b.err);
    const int it_g = ns > kPlocCap ? kPlocBatch : 0;
    if (it_g) ploc_rounds(S, b, 0, st);
    ploc_finish(S, b, it_g, st);
    cudaMemcpyAsync(S->class_host, b.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    return 2 + 4 * it_g;
}

// after ploc_enqueue reported an error: more rounds if more than kPlocCap
// clusters were left, kPlocBatch at a time with a count read-back after each
// batch, then the finish again.  MRS_ERR_CAPACITY: no root within the bound
// (the caller builds the radix tree instead).
mrs_status ploc_continue(mrs_scene_s* S, const PlocBufs& b, cudaStream_t st)
{
    const int it_g = S->ns > kPlocCap ? kPlocBatch : 0;
    MRS_CHECK(cudaMemcpyAsync(S->class_host, b.cnt + it_g, sizeof(int), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    int n_now = S->class_host[0];
    if (n_now <= kPlocCap) return MRS_ERR_CAPACITY;
    int it = it_g;
    while (n_now > kPlocCap) {
        if (it >= kPlocIters) return MRS_ERR_CAPACITY;
        ploc_rounds(S, b, it, st);
        MRS_LAUNCHED(4 * kPlocBatch);
        it += kPlocBatch;
        MRS_CHECK(cudaMemcpyAsync(S->class_host, b.cnt + it, sizeof(int), cudaMemcpyDeviceToHost, st));
        MRS_CHECK(cudaStreamSynchronize(st));
        n_now = S->class_host[0];
    }
    MRS_CHECK(cudaMemsetAsync(b.err, 0, sizeof(int), st));
    ploc_finish(S, b, it, st);
    MRS_LAUNCHED(1);
    MRS_CHECK(cudaMemcpyAsync(S->class_host, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    return S->class_host[0] ? MRS_ERR_CAPACITY : MRS_OK;
}

// ---- hierarchical clustering (the render tree in one launch) -----------------
// The same locally-ordered clustering, restricted to the subtrees of the
// radix tree over the sorted keys and run bottom-up in one launch (Benthin et
// al., "H-PLOC: Hierarchical Parallel Locally-Ordered Clustering for Bounding
// Volume Hierarchy Construction", HPG 2024), on the agglomerative walk of
// Apetrei ("Fast and Simple Agglomerative LBVH Construction", 2014):
//  * thread k starts at leaf k with the range [k, k].  A range [L, R] is the
//    left child of the split at R if the keys R, R + 1 differ in a lower bit
//    than the keys L - 1, L (smaller XOR of the 64-bit keys), else the right
//    child of the split at L - 1.  At the split, the first thread to arrive
//    leaves its end of the range (atomic exchange) and stops; the second takes
//    the union and goes on.  Every split is met twice, no thread waits.
//  * a range of at most kHKeep leaves holds them as its clusters.  When the
//    second thread reaches a larger range, or the root, its warp takes the
//    children's clusters (at most kHKeep each, so at most one per lane) and
//    runs clustering rounds on them -- every cluster's nearest neighbour
//    among all others by union surface area (ties as in the global rounds,
//    by the pair hash of the clusters' lanes), mutual pairs merge -- until at most
//    kHKeep are left (one at the root).  They are stored at the range's first
//    positions with their count, for the next level.
// Node ids come from the split positions: a subtree of the radix tree over
// leaves L .. R owns the ids L .. R - 1 (its splits) and passes the ones its
// merges left unused up with its clusters, in ascending order.  Where two
// children meet, the ids at hand are the left child's unused ones, the split
// itself, then the right child's (ascending again); merges take them from the
// top down.  A subtree other than the root keeps at least two clusters, so it
// leaves its smallest id unused: id 0 reaches the root and goes to its last
// merge, the root of the tree.  The numbering is a function of the tree.
// Surface-area cost on the 200k-triangle procedural scene: 22.4, against 22.1
// for the global rounds and 27.6 for the radix tree.
constexpr int kHKeep = 16;      // clusters a subtree keeps (a warp merges at most 2 kHKeep)
constexpr int kHLevels = 128;   // bound on the walk (the radix tree of 64-bit keys is < 64 deep)

__device__ __forceinline__ uint64_t key_xor(const uint32_t* __restrict__ code,
                                            const int* __restrict__ order, int i)
{
    const uint64_t a = ((uint64_t)__ldg(code + i) << 32) | (uint32_t)__ldg(order + i);
    const uint64_t b = ((uint64_t)__ldg(code + i + 1) << 32) | (uint32_t)__ldg(order + i + 1);
    return a ^ b;
}

__device__ __forceinline__ float4 shfl4(float4 v, int src)
{
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

struct HClusterArgs {
    const uint32_t* code;   // sorted Morton codes [ns]
    const int* order;       // triangle of each sorted position [ns]
    const float* leaf_box;  // S->box: leaf k's box at (ns - 1 + k) * 6
    int* other;             // [ns - 1] zeroed: the range end left at each split, + 1
    int* cids;              // [ns] cluster node ids of the ranges that merged
    float4* cbox;           // [2 ns] their boxes; the count of a range's clusters in
                            // the .w of its first entry's second float4
    int* uid;               // [ns] the unused node ids of a merged range, ascending
    int* err;               // set if a bound was hit (not reached by a valid input)
    float4* nodes;
    float* box;
    int ns;
};

// a pair's entry in the matrix: its union's half area, at most FLT_MAX (+inf
// marks "no pair": an overflowing or NaN area -- huge or non-finite
// coordinates -- must still order the pair, so that every round merges)
__device__ __forceinline__ float pair_area(float4 a0, float4 a1, float4 b0, float4 b1)
{
    return fminf(union_half_area(a0, a1, b0, b1), FLT_MAX);
}

// Per-warp scratch of a merge: the union areas of the warp's cluster pairs
struct HWarpScratch {
    float D[32][33];        // half surface area of cluster i's and j's union (+inf: none)
    float4 kb[64];          // a round's merged boxes, by lane
    int kp[32];             // and each lane's nearest neighbour
};

// One warp merges the clusters of range [L, R] (split after p); see above.
// Lane j < 16 holds the left child's j-th cluster, lane 16 + j the right
// child's; a cluster keeps its lane (its position) through the rounds.  The
// pairs' union areas are computed once; a round then takes each cluster's
// nearest neighbour from its row and, for every merge, recomputes the merged
// cluster's row and column (the other pairs' areas do not change).
__device__ void hcluster_merge(const HClusterArgs& a, int L, int R, int p, HWarpScratch& sc)
{
    const int lane = threadIdx.x & 31, ns = a.ns;
    const bool root = L == 0 && R == ns - 1;
    const int sl = p - L + 1, sr = R - p;
    const bool in_left = lane < 16;
    const int j16 = lane & 15, sz = in_left ? sl : sr, first = in_left ? L : p + 1;
    int id = -1, cnt = 0, un = first + j16;
    float4 b0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), b1 = b0;
    __syncwarp();
    if (sz <= kHKeep) {
        // a child of at most kHKeep leaves: its leaves, all its splits unused
        if (j16 < sz) {
            id = ns - 1 + first + j16;
            const float* bx = a.leaf_box + (size_t)id * 6;
            b0 = make_float4(bx[0], bx[1], bx[2], bx[3]);
            b1 = make_float4(bx[4], bx[5], 0.0f, 0.0f);
        }
    } else {
        // a merged child keeps at most kHKeep clusters (and one id fewer) at
        // its first positions
        const int q = first + j16;
        id = __ldcg(a.cids + q);
        b0 = __ldcg(a.cbox + 2 * q);
        b1 = __ldcg(a.cbox + 2 * q + 1);
        un = __ldcg(a.uid + q);
        cnt = __float_as_int(b1.w);
        b1.w = 0.0f;
    }
    const int cl = __shfl_sync(0xffffffffu, cnt, 0), cr = __shfl_sync(0xffffffffu, cnt, 16);
    const int nl = sl <= kHKeep ? sl : cl, nr = sr <= kHKeep ? sr : cr;
    if (nl < 1 || nl > min(sl, kHKeep) || nr < 1 || nr > min(sr, kHKeep)) {
        if (lane == 0) atomicExch(a.err, 1);
        return;
    }
    const int c0 = nl + nr;
    // the ids at hand, lane k holding the k-th: left's unused, p, right's unused
    {
        const int src = lane < nl - 1 ? lane : 16 + (lane - nl);
        const int v = __shfl_sync(0xffffffffu, un, src & 31);
        un = lane < nl - 1 ? v : lane == nl - 1 ? p : lane < c0 - 1 ? v : -1;
    }
    unsigned alive = __ballot_sync(0xffffffffu, j16 < (in_left ? nl : nr));
    bool mine = (alive >> lane) & 1u;
    int c = c0;
    const int target = root ? 1 : kHKeep;
    int m = 0;   // merges so far
    if (c > target) {
        // all pairs (i, i + d), d = 1 .. 16, each evaluated once
        sc.D[lane][lane] = INFINITY;
        for (int d = 1; d <= 16; ++d) {
            const int j = (lane + d) & 31;
            const float4 o0 = shfl4(b0, j);
            const float o1x = __shfl_sync(0xffffffffu, b1.x, j), o1y = __shfl_sync(0xffffffffu, b1.y, j);
            const float u = mine && ((alive >> j) & 1u)
                                ? pair_area(b0, b1, o0, make_float4(o1x, o1y, 0.0f, 0.0f))
                                : INFINITY;
            sc.D[lane][j] = u;
            sc.D[j][lane] = u;
        }
        __syncwarp();
    }
    for (int round = 0; c > target && round < 2 * kHKeep; ++round) {
        // nearest neighbour: smallest area, then pair hash, then position (the
        // hashes only where a row has a tie for its smallest area)
        float best = INFINITY;
        int bj = -1;
        bool tie = false;
        if (mine) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float v = sc.D[lane][j];
                tie = v == best ? true : (v < best ? false : tie);
                bj = v < best ? j : bj;
                best = fminf(best, v);
            }
        }
        if (__any_sync(0xffffffffu, tie && best != INFINITY)) {
            if (tie && best != INFINITY) {
                for (int j = bj + 1; j < 32; ++j)
                    if (sc.D[lane][j] == best && pair_key(lane, j) < pair_key(lane, bj)) bj = j;
            }
        }
        const int back = __shfl_sync(0xffffffffu, bj, bj >= 0 ? bj : lane);
        const bool mutual = bj >= 0 && back == lane;
        const bool lead = mutual && lane < bj;
        const unsigned lm = __ballot_sync(0xffffffffu, lead);
        const int src = lead ? bj : lane;
        const int pid = __shfl_sync(0xffffffffu, id, src);
        const float4 p0 = shfl4(b0, src), p1 = shfl4(b1, src);
        // merge t takes the (t + 1)-th largest id at hand
        const int t = m + __popc(lm & ((1u << lane) - 1u));
        const int nid = __shfl_sync(0xffffffffu, un, lead ? c0 - 2 - t : 0);
        if (lead) {
            float4 u0, u1;
            ploc_write_node(nid, id, b0, b1, pid, p0, p1, a.nodes, a.box, u0, u1);
            id = nid;
            b0 = u0;
            b1 = u1;
        }
        m += __popc(lm);
        c -= __popc(lm);
        alive &= ~__ballot_sync(0xffffffffu, mutual && lane > bj);
        mine = (alive >> lane) & 1u;
        __syncwarp();
        // merged clusters: new row and column; the partners' columns closed
        if (lead) {
            sc.kb[2 * lane] = b0;
            sc.kb[2 * lane + 1] = b1;
        }
        sc.kp[lane] = bj;
        __syncwarp();
        for (unsigned mm = lm; mm; mm &= mm - 1) {
            const int k = __ffs(mm) - 1;
            const float u = mine && lane != k ? pair_area(sc.kb[2 * k], sc.kb[2 * k + 1], b0, b1)
                                              : INFINITY;
            sc.D[k][lane] = u;
            sc.D[lane][k] = u;
            sc.D[lane][sc.kp[k]] = INFINITY;
        }
        __syncwarp();
    }
    if (c > target && lane == 0) atomicExch(a.err, 1);
    // the surviving clusters, in position order, and the c - 1 smallest ids,
    // still unused, to the range's first positions (over the children's:
    // every lane's loads are done)
    __syncwarp();
    if (mine) {
        const int q = L + __popc(alive & ((1u << lane) - 1u));
        a.cids[q] = id;
        a.cbox[2 * q] = b0;
        a.cbox[2 * q + 1] = make_float4(b1.x, b1.y, 0.0f, __int_as_float(q == L ? c : 0));
    }
    if (lane < c - 1) a.uid[L + lane] = un;
    // published by the release of this warp's next exchange at a split
    __syncwarp();
}

// atomic exchange at GPU scope: acquire-release (publishes what the warp
// stored before it), or acquire only (nothing new to publish)
__device__ __forceinline__ int exch_acq_rel(int* p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int exch_acquire(int* p, int v)
{
    int old;
    asm volatile("atom.acquire.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__global__ void __launch_bounds__(128) k_hcluster(const HClusterArgs a)
{
    __shared__ HWarpScratch s_w[4];
    const int w = threadIdx.x >> 5, ns = a.ns;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int L = k, R = k;
    bool active = k < ns;
    bool fresh = false;   // this lane's range merged since its last exchange
    for (int level = 0; level < kHLevels; ++level) {
        if (!__any_sync(0xffffffffu, active)) return;
        int p = 0;
        bool up = false;
        if (active) {
            const bool is_left = L == 0 ||
                                 (R != ns - 1 && key_xor(a.code, a.order, R) < key_xor(a.code, a.order, L - 1));
            p = is_left ? R : L - 1;
            // releases what this warp stored for the range (if it merged: a
            // range of leaves only has the previous kernel's data), acquires
            // the sibling's
            const int v = (is_left ? L : R) + 1;
            const int prev = fresh ? exch_acq_rel(a.other + p, v) : exch_acquire(a.other + p, v);
            if (prev == 0) {
                active = false;
            } else {
                if (is_left) R = prev - 1;
                else L = prev - 1;
                up = true;
            }
        }
        const bool root = up && L == 0 && R == ns - 1;
        unsigned need = __ballot_sync(0xffffffffu, up && (R - L + 1 > kHKeep || root));
        fresh = (need >> (threadIdx.x & 31)) & 1u;
        while (need) {
            const int q = __ffs(need) - 1;
            need &= need - 1;
            const int qL = __shfl_sync(0xffffffffu, L, q), qR = __shfl_sync(0xffffffffu, R, q);
            const int qp = __shfl_sync(0xffffffffu, p, q);
            hcluster_merge(a, qL, qR, qp, s_w[w]);
        }
        if (root) active = false;
    }
    if (active) atomicExch(a.err, 1);
}

// Scratch of the one-launch clustering build, carved from S->ploc_tmp
struct HClusterBufs {
    int* cids;
    float4* cbox;
    int* uid;
    int* err;
};

mrs_status hcluster_bufs(mrs_scene_s* S, HClusterBufs& b)
{
    const int ns = S->ns;
    const size_t need = (size_t)ns * (2 * sizeof(float4) + 2 * sizeof(int)) + 4 * sizeof(int) + 64;
    mrs_status rc = S->ploc_tmp.ensure(need);
    if (rc != MRS_OK) return rc;
    char* p = S->ploc_tmp.as<char>();
    b.cbox = (float4*)p; p += (size_t)ns * 2 * sizeof(float4);
    b.cids = (int*)p; p += (size_t)ns * sizeof(int);
    b.uid = (int*)p; p += (size_t)ns * sizeof(int);
    b.err = (int*)p;
    return MRS_OK;
}

// after k_leaves (which zeroes S->visit, the splits' exchange words)
int hcluster_enqueue(mrs_scene_s* S, const HClusterBufs& b, cudaStream_t st)
{
    const int ns = S->ns;
    cudaMemsetAsync(b.err, 0, sizeof(int), st);
    HClusterArgs a;
    a.code = S->skeys;
    a.order = S->order;
    a.leaf_box = S->box;
    a.other = S->visit;
    a.cids = b.cids;
    a.cbox = b.cbox;
    a.uid = b.uid;
    a.err = b.err;
    a.nodes = S->nodes;
    a.box = S->box;
    a.ns = ns;
    k_hcluster<<<blocks_for(ns, 128), 128, 0, st>>>(a);
    return 1;
}

// The traversal structure: an LBVH over the scene's compact triangles (ns of
// them, S->small_idx) plus the large triangles (S->big_idx) that every ray
// tests exhaustively first -- large triangles (a ground plane, walls) would
// otherwise inflate the boxes of the tree's upper levels.  The closest hit is
// the same either way (smallest t, ties to the smaller triangle index).
// The radix tree over the sorted leaves (after k_leaves): topology, then the
// bottom-up refit that writes the traversal nodes; returns the kernels enqueued
int karras_enqueue(mrs_scene_s* S, cudaStream_t st)
{
    const int ns = S->ns;
    k_karras<<<blocks_for(ns - 1, kBlock), kBlock, 0, st>>>(S->skeys, S->order, ns, S->left, S->right,
                                                           S->parent);
    k_refit<<<blocks_for(ns, kBlock), kBlock, 0, st>>>(ns, S->left, S->right, S->parent, S->box,
                                                       S->visit, S->nodes);
    return 2;
}

// The whole build is one CUDA graph per scene (captured again when the tree
// size, the tree kind or a scratch buffer changes): some 20 short kernels for
// the LBVH, a hundred for the clustering tree, whose host-side launch cost
// would otherwise be most of the build.  The clustering build then reads its
// error word back (one synchronisation) and, past kPlocBatch rounds or if
// clustering gave up, goes on by direct launches.
mrs_status build_lbvh(mrs_scene_s* S, cudaStream_t st)
{
    const int n = S->n, ns = S->ns, nb = n - ns;
    S->tree_built = S->tree;     // without internal nodes either kind is the same tree
    if (n <= 0) return MRS_OK;
    int nparts = 2 * sm_count();
    int ntiles = blocks_for(ns > 0 ? ns : 1, kTile);
    size_t need = sizeof(float) * 6 * nparts + sizeof(uint32_t) * 256 * (size_t)ntiles +
                  (sizeof(uint32_t) + sizeof(int)) * 2 * (size_t)(ns > 0 ? ns : 1) + 256;
    mrs_status s = S->sort_tmp.ensure(need);
    if (s != MRS_OK) return s;
    const bool cluster = ns > 1 && S->tree == MRS_TREE_CLUSTER;
    const bool hcluster = ns > 1 && S->tree == MRS_TREE_HCLUSTER;
    PlocBufs pb;
    if (cluster && (s = ploc_bufs(S, pb)) != MRS_OK) return s;
    HClusterBufs hb;
    if (hcluster && (s = hcluster_bufs(S, hb)) != MRS_OK) return s;
    char* p = S->sort_tmp.as<char>();
    float* part = (float*)p; p += sizeof(float) * 6 * nparts;
    uint32_t* counts = (uint32_t*)p; p += sizeof(uint32_t) * 256 * (size_t)ntiles;
    uint32_t* ka = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)ns;
    uint32_t* kb = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)ns;
    int* va = (int*)p; p += sizeof(int) * (size_t)ns;
    int* vb = (int*)p;

    // every kernel of the build on stream c; returns how many
    auto enqueue = [&](cudaStream_t c, bool with_cluster) -> int {
        int kernels = 0;
        if (ns > 0) {
            k_bounds_partial<<<nparts, kBlock, 0, c>>>(S->V, ns, part, S->small_idx);
            k_morton<<<min(blocks_for(ns, kBlock), 8 * sm_count()), kBlock, 0, c>>>(
                S->V, ns, part, nparts, nullptr, ka, va, S->small_idx);
            kernels += 2;
            // 30-bit codes: digits at bits 0, 8, 16, 24 (4 passes, ends back in ka/va)
            for (int pass = 0; pass < 4; ++pass) {
                int shift = pass * 8;
                uint32_t* kin = (pass & 1) ? kb : ka;
                uint32_t* kout = (pass & 1) ? ka : kb;
                int* vin = (pass & 1) ? vb : va;
                int* vout = (pass & 1) ? va : vb;
                k_sort_hist<<<ntiles, kBlock, 0, c>>>(kin, ns, shift, counts, ntiles);
                k_sort_scan<<<1, 1024, 0, c>>>(counts, 256 * ntiles);
                k_sort_scatter<<<ntiles, kBlock, 0, c>>>(kin, vin, kout, vout, ns, shift, counts, ntiles);
                kernels += 3;
            }
            cudaMemcpyAsync(S->skeys, ka, sizeof(uint32_t) * ns, cudaMemcpyDeviceToDevice, c);
            cudaMemcpyAsync(S->order, va, sizeof(int) * ns, cudaMemcpyDeviceToDevice, c);
            k_leaves<<<blocks_for(ns, kBlock), kBlock, 0, c>>>(S->V, S->tri_mat, S->tri_light, S->order,
                                                               ns, S->tris, S->tri_ml, S->box, S->visit);
            kernels += 1;
            if (with_cluster) kernels += ploc_enqueue(S, pb, c);
            else if (hcluster) kernels += hcluster_enqueue(S, hb, c);
            else if (ns > 1) kernels += karras_enqueue(S, c);
        }
        if (nb > 0) {
            k_big_leaves<<<blocks_for(nb, kBlock), kBlock, 0, c>>>(S->V, S->tri_mat, S->tri_light,
                                                                   S->big_idx, ns, nb, S->order,
                                                                   S->tris, S->tri_ml);
            kernels += 1;
        }
        return kernels;
    };

    // inside the caller's own stream capture (a captured frame) the kernels go
    // straight into it; the clustering tree of grid-wide rounds, which reads a
    // word back, is not available there and the radix tree is built
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MRS_CHECK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        MRS_LAUNCHED(enqueue(st, false));
        if (ns > 1) S->tree_built = hcluster ? MRS_TREE_HCLUSTER : MRS_TREE_LBVH;
        return cuda_status(cudaGetLastError(), "lbvh launch");
    }

    const BuildKey key{n, ns, ns > 1 ? S->tree : 0, S->sort_tmp.p,
                       cluster || hcluster ? S->ploc_tmp.p : nullptr};
    if (!S->build_exec || !(key == S->build_key)) {
        if (S->build_exec) { cudaGraphExecDestroy(S->build_exec); S->build_exec = nullptr; }
        // captured on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured), launched on the caller's
        if (!S->cap_stream) MRS_CHECK(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
        MRS_CHECK(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int kernels = enqueue(S->cap_stream, cluster);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(S->cap_stream, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&S->build_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) { S->build_exec = nullptr; return cuda_status(e, "build graph"); }
        S->build_key = key;
        S->build_kernels = kernels;
    }
    cudaEvent_t lbvh_a = prof_on() ? prof_record(st) : nullptr;
    MRS_CHECK(cudaGraphLaunch(S->build_exec, st));
    MRS_LAUNCHED(S->build_kernels);
    if (cluster) {
        MRS_CHECK(cudaStreamSynchronize(st));
        mrs_status pc = S->class_host[0] ? ploc_continue(S, pb, st) : MRS_OK;
        if (pc == MRS_ERR_CAPACITY) {
            S->tree_built = MRS_TREE_LBVH;
            MRS_LAUNCHED(karras_enqueue(S, st));
        } else if (pc != MRS_OK) {
            return pc;
        }
    } else if (ns > 1) {
        S->tree_built = hcluster ? MRS_TREE_HCLUSTER : MRS_TREE_LBVH;
    }
    if (lbvh_a) prof_push(PK_LBVH, lbvh_a, prof_record(st));
    return cuda_status(cudaGetLastError(), "lbvh launch");
}

// Large triangles: AABB extent >= 1/4 of the centroid bounds' largest extent,
// at most kMaxBig of them (else none).  They are tested before the tree by
// every ray; the others go into the LBVH.  Classified on the device: centroid
// bounds of all triangles, a flag and a per-block count, one scan, and a
// stable scatter (both index lists in increasing triangle order); only the two
// counts come back to the host, which sizes the build's launches with them.
constexpr int kMaxBig = 64;

// largest extent of the centroid bounds from the block partials (warp 0)
__device__ float bounds_extent(const float* __restrict__ part, int nparts)
{
    __shared__ float s_L;
    if (threadIdx.x < 32) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b = threadIdx.x; b < nparts; b += 32)
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], part[6 * b + a]);
                hi[a] = fmaxf(hi[a], part[6 * b + 3 + a]);
            }
        for (int off = 16; off > 0; off >>= 1)
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
            }
        if (threadIdx.x == 0) {
            float L = 0.0f;
            for (int a = 0; a < 3; ++a) L = fmaxf(L, hi[a] - lo[a]);
            s_L = L;
        }
    }
    __syncthreads();
    return s_L;
}

// flag[i] = triangle i is large; cnt[block] = large triangles of the block
__global__ void k_class_count(const float* __restrict__ V, int n, const float* __restrict__ part,
                              int nparts, uint8_t* __restrict__ flag, uint32_t* __restrict__ cnt)
{
    const float L = bounds_extent(part, nparts);
    const int i = blockIdx.x * kBlock + threadIdx.x;
    bool big = false;
    if (i < n) {
        const float* p = V + (size_t)i * 9;
        float e = 0.0f;
        for (int a = 0; a < 3; ++a)
            e = fmaxf(e, fmaxf(fmaxf(p[a], p[3 + a]), p[6 + a]) - fminf(fminf(p[a], p[3 + a]), p[6 + a]));
        big = L > 0.0f && e >= 0.25f * L;
        flag[i] = big ? 1 : 0;
    }
    const int c = __syncthreads_count(big);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint32_t)c;
}

// small_idx / big_idx in increasing triangle order (off: exclusive scan of the
// block counts, off[nblk] = total); more than kMaxBig large ones: none large.
// counts[0] = small, counts[1] = large
__global__ void k_class_scatter(const uint8_t* __restrict__ flag, int n, const uint32_t* __restrict__ off,
                                int nblk, int* __restrict__ small_idx, int* __restrict__ big_idx,
                                int* __restrict__ counts)
{
    __shared__ uint32_t wsum[kBlock / 32];
    const uint32_t total = off[nblk];
    const bool none = total > (uint32_t)kMaxBig;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const bool big = !none && i < n && flag[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, big);
    if (lane == 0) wsum[warp] = (uint32_t)__popc(m);
    __syncthreads();
    uint32_t before = off[blockIdx.x] + (uint32_t)__popc(m & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (none) before = 0;
    if (i < n) {
        if (big) big_idx[before] = i;
        else small_idx[i - (int)before] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts[0] = none ? n : n - (int)total;
        counts[1] = none ? 0 : (int)total;
    }
}

mrs_status classify_on_device(mrs_scene_s* S, cudaStream_t st)
{
    const int n = S->n;
    const int nparts = 2 * sm_count();
    const int nblk = (n + kBlock - 1) / kBlock;
    size_t need = sizeof(float) * 6 * nparts + sizeof(uint32_t) * ((size_t)nblk + 1) + 16 + (size_t)n + 256;
    mrs_status s = S->class_tmp.ensure(need);
    if (s != MRS_OK) return s;
    char* p = S->class_tmp.as<char>();
    float* part = (float*)p; p += sizeof(float) * 6 * nparts;
    uint32_t* cnt = (uint32_t*)p; p += sizeof(uint32_t) * ((size_t)nblk + 1);
    p = (char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    int* counts = (int*)p; p += 16;
    uint8_t* flag = (uint8_t*)p;
    if (!S->class_host) MRS_CHECK(cudaMallocHost((void**)&S->class_host, 2 * sizeof(int)));
    k_bounds_partial<<<nparts, kBlock, 0, st>>>(S->V, n, part);
    MRS_LAUNCHED(1);
    MRS_CHECK(cudaMemsetAsync(cnt + nblk, 0, sizeof(uint32_t), st));
    k_class_count<<<nblk, kBlock, 0, st>>>(S->V, n, part, nparts, flag, cnt);
    MRS_LAUNCHED(1);
    k_sort_scan<<<1, 1024, 0, st>>>(cnt, nblk + 1);
    MRS_LAUNCHED(1);
    k_class_scatter<<<nblk, kBlock, 0, st>>>(flag, n, cnt, nblk, S->small_idx, S->big_idx, counts);
    MRS_LAUNCHED(1);
    MRS_CHECK(cudaMemcpyAsync(S->class_host, counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MRS_CHECK(cudaStreamSynchronize(st));
    S->ns = S->class_host[0];
    return MRS_OK;
}

void free_scene(mrs_scene_s* S)
{
    void* ptrs[] = {S->V, S->tri_mat, S->tri_light, S->mats, S->lights, S->morton, S->skeys,
                    S->order, S->left, S->right, S->parent, S->visit, S->box, S->nodes,
                    S->tris, S->tri_ml, S->small_idx, S->big_idx};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    S->sort_tmp.release();
    if (S->build_exec) cudaGraphExecDestroy(S->build_exec);
    if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
    S->ploc_tmp.release();
    S->export_tmp.release();
    S->class_tmp.release();
    S->arena.release();
    if (S->class_host) cudaFreeHost(S->class_host);
    delete S;
}

// ---- LBVH build without allocation --------------------------------------
// For callers that cannot allocate device memory (see mrs_lbvh_build_static in
// mrs.h), all scratch of the build lives in one file-scope device array sized
// for MRS_LBVH_STATIC_MAX_TRIS triangles:
//   centroid-bound partials | digit counts | keys a/b | values a/b | parent | visit
constexpr int kStaticMaxTris = MRS_LBVH_STATIC_MAX_TRIS;
constexpr int kStaticParts = 512;
constexpr int kStaticTiles = (kStaticMaxTris + kTile - 1) / kTile;
constexpr size_t kStaticBytes = sizeof(float) * 6 * kStaticParts +
                                sizeof(uint32_t) * 256 * kStaticTiles +
                                sizeof(uint32_t) * 4 * (size_t)kStaticMaxTris +
                                sizeof(int) * 3 * (size_t)kStaticMaxTris;
static __device__ __align__(256) unsigned char g_lbvh_static[kStaticBytes];

// leaf boxes of the sorted triangles; zeroes the refit visit counters (the
// static scratch keeps the previous call's contents)
__global__ void k_static_leaves(const float* __restrict__ V, const int* __restrict__ order, int n,
                                float* __restrict__ box, int* __restrict__ visit)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n - 1) visit[k] = 0;
    if (k >= n) return;
    const float* p = V + (size_t)order[k] * 9;
    float* b = box + (size_t)(n - 1 + k) * 6;
    for (int a = 0; a < 3; ++a) {
        b[a] = fminf(fminf(p[a], p[3 + a]), p[6 + a]);
        b[3 + a] = fmaxf(fmaxf(p[a], p[3 + a]), p[6 + a]);
    }
}

// bottom-up box refit (second arrival at a parent computes its box)
__global__ void k_static_refit(int n, const int* __restrict__ left, const int* __restrict__ right,
                               const int* __restrict__ parent, float* box, int* visit)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int node = parent[(n - 1) + k];
    bool wrote = false;
    while (node >= 0) {
        if ((wrote ? add_acq_rel(&visit[node], 1) : add_acquire(&visit[node], 1)) == 0) return;
        wrote = true;
        const volatile float* bl = box + (size_t)left[node] * 6;
        const volatile float* br = box + (size_t)right[node] * 6;
        float* b = box + (size_t)node * 6;
        for (int a = 0; a < 3; ++a) {
            b[a] = fminf(bl[a], br[a]);
            b[3 + a] = fmaxf(bl[3 + a], br[3 + a]);
        }
        node = parent[node];
    }
}

// device address of g_lbvh_static for the current device, looked up once per
// device (the symbol's host-side name is not a device address)
mrs_status static_scratch(unsigned char** out)
{
    static std::mutex mu;
    static unsigned char* addr[64] = {nullptr};
    int dev = 0;
    MRS_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index %d out of range", dev); return MRS_ERR_CUDA; }
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_lbvh_static);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_lbvh_static)");
        addr[dev] = (unsigned char*)p;
    }
    *out = addr[dev];
    return MRS_OK;
}

template <class T> mrs_status dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cuda_status(cudaMalloc((void**)p, sizeof(T) * count), "cudaMalloc");
}

}  // namespace
}  // namespace mrs

using namespace mrs;

extern "C" const char* mrs_last_error(void) { return mrs::last_error(); }

extern "C" uint64_t mrs_kernel_launches(void) { return mrs::launch_counter().load(); }


extern "C" mrs_status mrs_profile_enable(int32_t on)
{
    mrs::prof().on = on != 0;
    return MRS_OK;
}

extern "C" mrs_status mrs_profile_read(int32_t kernel, double* total_ms, int64_t* launches)
{
    MRS_ARG(kernel >= 0 && kernel < mrs::PK_COUNT, "kernel id out of range");
    MRS_ARG(total_ms && launches, "NULL output");
    std::lock_guard<std::mutex> g(mrs::prof().mu);
    auto& v = mrs::prof().ev[kernel];
    double tot = 0;
    for (auto& pr : v) {
        MRS_CHECK(cudaEventSynchronize(pr.second));
        float ms = 0;
        MRS_CHECK(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    *total_ms = tot;
    *launches = (int64_t)v.size();
    v.clear();
    return MRS_OK;
}

extern "C" const char* mrs_status_string(mrs_status s)
{
    switch (s) {
    case MRS_OK: return "ok";
    case MRS_ERR_ARG: return "invalid argument";
    case MRS_ERR_OOM: return "out of device memory";
    case MRS_ERR_CUDA: return "CUDA error";
    case MRS_ERR_TIMEOUT: return "device wait timed out";
    case MRS_ERR_CAPACITY: return "capacity exceeded";
    case MRS_ERR_STATE: return "invalid handle state";
    case MRS_ERR_FORMAT: return "invalid checkpoint file";
    case MRS_ERR_IO: return "file I/O error";
    default: return "unknown status";
    }
}

extern "C" mrs_status mrs_build_scene_seeded(uint64_t seed, int32_t kind,
                                             const mrs_scene_params* params, void* stream,
                                             mrs_scene* out)
{
    MRS_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MRS_ARG(kind == MRS_SCENE_CORNELL || kind == MRS_SCENE_PROCEDURAL, "unknown scene kind");
    synth_scene_params p;
    synth_default_params(&p);
    if (params) {
        p.n_spheres = params->n_spheres;
        p.n_large = params->n_large;
        p.sphere_subdiv = params->sphere_subdiv;
        p.aspect = params->aspect;
    }
    const int sk = kind == MRS_SCENE_CORNELL ? SYNTH_CORNELL : SYNTH_PROCEDURAL;
    int32_t nt = 0, nm = 0, nl = 0;
    MRS_ARG(synth_scene_counts(sk, &p, &nt, &nm, &nl) == 0, "scene parameters out of range");
    std::vector<float> V((size_t)nt * 9), mats((size_t)nm * 8), lights((size_t)nl * 12 + 1);
    std::vector<int32_t> tri_mat(nt), tri_light(nt);
    float env[3], cam[12];
    if (synth_scene_generate(seed, sk, &p, V.data(), tri_mat.data(), tri_light.data(), mats.data(),
                             lights.data(), env, cam) != 0) {
        set_error("scene generation failed");
        return MRS_ERR_ARG;
    }
    return mrs_build_scene(V.data(), nt, tri_mat.data(), tri_light.data(), mats.data(), nm,
                           lights.data(), nl, env, cam, stream, out);
}

extern "C" mrs_status mrs_build_scene(const float* V, int32_t n, const int32_t* tri_mat,
                                      const int32_t* tri_light, const float* mats,
                                      int32_t n_mats, const float* lights, int32_t n_lights,
                                      const float* env, const float* cam, void* stream,
                                      mrs_scene* out)
{
    MRS_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    MRS_ARG(n >= 0 && n <= (1 << 28), "n_tris out of range [0, 2^28]");
    MRS_ARG(n == 0 || (V && tri_mat && tri_light), "triangle arrays are NULL");
    MRS_ARG(n_mats >= 0 && (n_mats == 0 || mats), "mats");
    MRS_ARG(n_lights >= 0 && (n_lights == 0 || lights), "lights");
    MRS_ARG(env && cam, "env/cam NULL");
    for (int i = 0; i < n; ++i) {
        MRS_ARG(tri_mat[i] >= 0 && tri_mat[i] < n_mats, "tri_mat index out of range");
        MRS_ARG(tri_light[i] >= -1 && tri_light[i] < n_lights, "tri_light index out of range");
    }
    for (int m = 0; m < n_mats; ++m) {
        float t = mats[m * 8];
        MRS_ARG(t == 0.0f || t == 1.0f, "material type must be 0 or 1");
        MRS_ARG(t == 0.0f || mats[m * 8 + 4] > 0.0f, "GGX alpha must be > 0");
    }
    cudaStream_t st = (cudaStream_t)stream;
    mrs_scene_s* S = new mrs_scene_s();
    S->n = n; S->n_mats = n_mats; S->n_lights = n_lights;
    memcpy(S->env, env, sizeof(S->env));
    memcpy(S->cam, cam, sizeof(S->cam));
    mrs_status s = MRS_OK;
#define TRY(x) do { if (s == MRS_OK) s = (x); } while (0)
    TRY(dalloc(&S->V, (size_t)n * 9));
    TRY(dalloc(&S->tri_mat, n));
    TRY(dalloc(&S->tri_light, n));
    TRY(dalloc(&S->mats, (size_t)n_mats * 8));
    TRY(dalloc(&S->lights, (size_t)n_lights * 12));
    TRY(dalloc(&S->morton, n));
    TRY(dalloc(&S->skeys, n));
    TRY(dalloc(&S->order, n));
    TRY(dalloc(&S->left, n > 1 ? n - 1 : 1));
    TRY(dalloc(&S->right, n > 1 ? n - 1 : 1));
    TRY(dalloc(&S->parent, n > 0 ? 2 * (size_t)n - 1 : 1));
    TRY(dalloc(&S->visit, n > 1 ? n - 1 : 1));
    TRY(dalloc(&S->box, n > 0 ? (2 * (size_t)n - 1) * 6 : 6));
    TRY(dalloc(&S->nodes, n > 1 ? 4 * (size_t)(n - 1) : 4));
    TRY(dalloc(&S->tris, 3 * (size_t)(n > 0 ? n : 1)));
    TRY(dalloc(&S->tri_ml, n > 0 ? n : 1));
    TRY(dalloc(&S->small_idx, n > 0 ? n : 1));
    TRY(dalloc(&S->big_idx, kMaxBig));
    if (n > 0) {
        TRY(cuda_status(cudaMemcpyAsync(S->V, V, sizeof(float) * 9 * (size_t)n, cudaMemcpyHostToDevice, st), "copy V"));
        TRY(cuda_status(cudaMemcpyAsync(S->tri_mat, tri_mat, sizeof(int) * n, cudaMemcpyHostToDevice, st), "copy tri_mat"));
        TRY(cuda_status(cudaMemcpyAsync(S->tri_light, tri_light, sizeof(int) * n, cudaMemcpyHostToDevice, st), "copy tri_light"));
    }
    if (n_mats > 0)
        TRY(cuda_status(cudaMemcpyAsync(S->mats, mats, sizeof(float) * 8 * n_mats, cudaMemcpyHostToDevice, st), "copy mats"));
    if (n_lights > 0)
        TRY(cuda_status(cudaMemcpyAsync(S->lights, lights, sizeof(float) * 12 * n_lights, cudaMemcpyHostToDevice, st), "copy lights"));
    if (n > 0) TRY(classify_on_device(S, st));
    TRY(build_lbvh(S, st));
    TRY(cuda_status(cudaStreamSynchronize(st), "build_scene sync"));
#undef TRY
    if (s != MRS_OK) { free_scene(S); return s; }
    *out = S;
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_rebuild(mrs_scene S, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    return build_lbvh(S, (cudaStream_t)stream);
}

extern "C" mrs_status mrs_scene_set_tree(mrs_scene S, int32_t kind, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(kind == MRS_TREE_LBVH || kind == MRS_TREE_CLUSTER || kind == MRS_TREE_HCLUSTER,
            "kind must be MRS_TREE_LBVH, MRS_TREE_CLUSTER or MRS_TREE_HCLUSTER");
    S->tree = kind;
    cudaStream_t st = (cudaStream_t)stream;
    mrs_status rc = build_lbvh(S, st);
    if (rc != MRS_OK) return rc;
    MRS_CHECK(cudaStreamSynchronize(st));
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_get_tree(mrs_scene S, int32_t* kind)
{
    MRS_ARG(S != nullptr && kind != nullptr, "NULL argument");
    *kind = S->tree_built;
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_export_nodes(mrs_scene S, float* nodes, int64_t n_floats,
                                             int32_t* order, int32_t* n_tree)
{
    MRS_ARG(S != nullptr && n_tree != nullptr, "NULL argument");
    const int ns = S->ns;
    *n_tree = ns;
    MRS_CHECK(cudaDeviceSynchronize());
    if (nodes && ns > 1) {
        MRS_ARG(n_floats >= 16 * (int64_t)(ns - 1), "n_floats must be >= 16 (ns - 1)");
        MRS_CHECK(cudaMemcpy(nodes, S->nodes, sizeof(float4) * 4 * (size_t)(ns - 1), cudaMemcpyDeviceToHost));
    }
    if (order && ns > 0)
        MRS_CHECK(cudaMemcpy(order, S->order, sizeof(int) * (size_t)ns, cudaMemcpyDeviceToHost));
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_update_vertices(mrs_scene S, const float* V, int32_t n,
                                                void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(n == S->n, "n must equal the scene's triangle count");
    MRS_ARG(n == 0 || V != nullptr, "V is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0) {
        MRS_CHECK(cudaMemcpyAsync(S->V, V, sizeof(float) * 9 * (size_t)n, cudaMemcpyHostToDevice, st));
        mrs_status s = classify_on_device(S, st);
        if (s != MRS_OK) return s;
    }
    return build_lbvh(S, st);
}

extern "C" mrs_status mrs_free_scene(mrs_scene S)
{
    if (!S) return MRS_OK;
    cudaDeviceSynchronize();
    free_scene(S);
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_export_bvh(mrs_scene S, uint32_t* morton, int32_t* order,
                                           int32_t* left, int32_t* right, float* box,
                                           void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = S->n;
    if (n == 0) return MRS_OK;
    // the LBVH over all n triangles, built by the same kernels
    const int nparts = 2 * sm_count();
    const int ntiles = blocks_for(n, kTile);
    size_t need = sizeof(float) * 6 * nparts + sizeof(uint32_t) * 256 * (size_t)ntiles +
                  sizeof(uint32_t) * 5 * (size_t)n + sizeof(int) * 7 * (size_t)n +
                  sizeof(float) * 6 * (2 * (size_t)n) + 1024;
    mrs_status rc = S->export_tmp.ensure(need);
    if (rc != MRS_OK) return rc;
    char* p = S->export_tmp.as<char>();
    float* part = (float*)p; p += sizeof(float) * 6 * nparts;
    uint32_t* counts = (uint32_t*)p; p += sizeof(uint32_t) * 256 * (size_t)ntiles;
    uint32_t* codes = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)n;
    uint32_t* ka = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)n;
    uint32_t* kb = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)n;
    int* va = (int*)p; p += sizeof(int) * (size_t)n;
    int* vb = (int*)p; p += sizeof(int) * (size_t)n;
    int* ord = (int*)p; p += sizeof(int) * (size_t)n;
    int* lft = (int*)p; p += sizeof(int) * (size_t)n;
    int* rgt = (int*)p; p += sizeof(int) * (size_t)n;
    int* par = (int*)p; p += sizeof(int) * 2 * (size_t)n;
    int* vis = (int*)p; p += sizeof(int) * (size_t)n;
    float* bx = (float*)p;
    k_bounds_partial<<<nparts, kBlock, 0, st>>>(S->V, n, part);
    MRS_LAUNCHED(1);
    k_morton<<<min(blocks_for(n, kBlock), 8 * sm_count()), kBlock, 0, st>>>(S->V, n, part, nparts,
                                                                        codes, ka, va);
    MRS_LAUNCHED(1);
    for (int pass = 0; pass < 4; ++pass) {
        int shift = pass * 8;
        uint32_t* kin = (pass & 1) ? kb : ka;
        uint32_t* kout = (pass & 1) ? ka : kb;
        int* vin = (pass & 1) ? vb : va;
        int* vout = (pass & 1) ? va : vb;
        k_sort_hist<<<ntiles, kBlock, 0, st>>>(kin, n, shift, counts, ntiles);
        MRS_LAUNCHED(1);
        k_sort_scan<<<1, 1024, 0, st>>>(counts, 256 * ntiles);
        MRS_LAUNCHED(1);
        k_sort_scatter<<<ntiles, kBlock, 0, st>>>(kin, vin, kout, vout, n, shift, counts, ntiles);
        MRS_LAUNCHED(1);
    }
    MRS_CHECK(cudaMemcpyAsync(ord, va, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (n > 1) {
        k_karras<<<blocks_for(n - 1, kBlock), kBlock, 0, st>>>(ka, ord, n, lft, rgt, par);
        MRS_LAUNCHED(1);
    }
    k_static_leaves<<<blocks_for(n, kBlock), kBlock, 0, st>>>(S->V, ord, n, bx, vis);
    MRS_LAUNCHED(1);
    if (n > 1) {
        k_static_refit<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, lft, rgt, par, bx, vis);
        MRS_LAUNCHED(1);
    }
    MRS_CHECK(cudaGetLastError());
    if (morton) MRS_CHECK(cudaMemcpyAsync(morton, codes, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (order) MRS_CHECK(cudaMemcpyAsync(order, ord, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (n > 1 && left) MRS_CHECK(cudaMemcpyAsync(left, lft, 4 * (size_t)(n - 1), cudaMemcpyDeviceToDevice, st));
    if (n > 1 && right) MRS_CHECK(cudaMemcpyAsync(right, rgt, 4 * (size_t)(n - 1), cudaMemcpyDeviceToDevice, st));
    if (box) MRS_CHECK(cudaMemcpyAsync(box, bx, 24 * (2 * (size_t)n - 1), cudaMemcpyDeviceToDevice, st));
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_set_wave(mrs_scene S, int64_t max_paths)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(max_paths >= 1 && max_paths <= (int64_t(1) << 30), "wave size out of range [1, 2^30]");
    S->wave_paths = max_paths;
    return MRS_OK;
}

extern "C" mrs_status mrs_scene_set_tail(mrs_scene S, int32_t bounce)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(bounce >= -1 && bounce <= 64, "tail bounce out of range [-1, 64]");
    S->tail_bounce = bounce;
    return MRS_OK;
}

extern "C" mrs_status mrs_lbvh_build_static(const float* V, int32_t n, uint32_t* morton,
                                            int32_t* order, int32_t* left, int32_t* right,
                                            float* box, void* stream)
{
    MRS_ARG(n >= 0, "n_tris < 0");
    if (n > MRS_LBVH_STATIC_MAX_TRIS) {
        set_error("n_tris = %d exceeds MRS_LBVH_STATIC_MAX_TRIS = %d (static scratch capacity)",
                  n, MRS_LBVH_STATIC_MAX_TRIS);
        return MRS_ERR_CAPACITY;
    }
    if (n == 0) return MRS_OK;
    MRS_ARG(V && morton && order && box, "NULL pointer");
    MRS_ARG(n == 1 || (left && right), "left/right are NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    mrs_status s = static_scratch(&base);
    if (s != MRS_OK) return s;
    const int nparts = 2 * sm_count() < kStaticParts ? 2 * sm_count() : kStaticParts;
    const int ntiles = blocks_for(n, kTile);
    unsigned char* p = base;
    float* part = (float*)p; p += sizeof(float) * 6 * kStaticParts;
    uint32_t* counts = (uint32_t*)p; p += sizeof(uint32_t) * 256 * kStaticTiles;
    uint32_t* ka = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)kStaticMaxTris;
    uint32_t* kb = (uint32_t*)p; p += sizeof(uint32_t) * (size_t)kStaticMaxTris;
    int* va = (int*)p; p += sizeof(int) * (size_t)kStaticMaxTris;
    int* vb = (int*)p; p += sizeof(int) * (size_t)kStaticMaxTris;
    int* parent = (int*)p; p += sizeof(int) * 2 * (size_t)kStaticMaxTris;
    int* visit = (int*)p;

    k_bounds_partial<<<nparts, kBlock, 0, st>>>(V, n, part);
    MRS_LAUNCHED(1);
    k_morton<<<min(blocks_for(n, kBlock), 8 * sm_count()), kBlock, 0, st>>>(V, n, part, nparts,
                                                                        morton, ka, va);
    MRS_LAUNCHED(1);
    for (int pass = 0; pass < 4; ++pass) {
        int shift = pass * 8;
        uint32_t* kin = (pass & 1) ? kb : ka;
        uint32_t* kout = (pass & 1) ? ka : kb;
        int* vin = (pass & 1) ? vb : va;
        int* vout = (pass & 1) ? va : vb;
        k_sort_hist<<<ntiles, kBlock, 0, st>>>(kin, n, shift, counts, ntiles);
        MRS_LAUNCHED(1);
        k_sort_scan<<<1, 1024, 0, st>>>(counts, 256 * ntiles);
        MRS_LAUNCHED(1);
        k_sort_scatter<<<ntiles, kBlock, 0, st>>>(kin, vin, kout, vout, n, shift, counts, ntiles);
        MRS_LAUNCHED(1);
    }
    MRS_CHECK(cudaMemcpyAsync(order, va, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (n > 1) {
        k_karras<<<blocks_for(n - 1, kBlock), kBlock, 0, st>>>(ka, order, n, left, right, parent);
        MRS_LAUNCHED(1);
    }
    k_static_leaves<<<blocks_for(n, kBlock), kBlock, 0, st>>>(V, order, n, box, visit);
    MRS_LAUNCHED(1);
    if (n > 1) {
        k_static_refit<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, left, right, parent, box, visit);
        MRS_LAUNCHED(1);
    }
    return cuda_status(cudaGetLastError(), "static lbvh launch");
}
