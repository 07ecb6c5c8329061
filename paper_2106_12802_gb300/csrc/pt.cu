// Wavefront Monte Carlo path tracer: produces the LRHS / HRLS radiance and
// the albedo / normal / depth render layers of the multi-resolution sampling
// method (Sec. 1, Sec. 3.2-3.3).  Per wave of paths:
//   raygen -> for each bounce: traverse (closest hit) -> shade (emission, NEE
//   shadow-ray setup, BSDF sampling, roulette, warp-ballot compaction) ->
//   traverse_shadow (any hit, adds the unoccluded NEE term) -> accumulate
//   (per-pixel Kahan sums in sample order).
//
// Compiled with --fmad=false and IEEE div/sqrt: every float operation is a
// single correctly rounded binary32 operation in the order written, which is
// what makes the per-bounce ray counts and the radiance reproducible
// bit-for-bit by an independent CPU implementation of the same estimator.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mrs {
namespace {

constexpr float PI_F = 3.14159265358979323846f;
constexpr float INV_PI_F = 0.318309886183790671538f;
constexpr float RAY_EPS = 1e-4f;
constexpr float SHADOW_FRAC = 0.999f;
constexpr float T_INF = 1e30f;
constexpr int kThreads = 256;
// traversal stack: the radix tree over 64-bit keys is at most 63 deep; the
// clustering trees have no bound by construction (measured at most 63 deep)
constexpr int kStack = 128;

// ---- Philox4x32-10 (Salmon et al., SC'11) ----------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ float4 draws(uint32_t pixel, uint32_t sample, uint32_t bounce,
                                        uint32_t group, uint2 key)
{
    uint4 o = philox(make_uint4(pixel, sample, bounce, group), key);
    return make_float4(u01(o.x), u01(o.y), u01(o.z), u01(o.w));
}

// ---- float3 algebra, left-to-right evaluation -------------------------------
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 normalize(V3 a) { float inv = 1.0f / sqrtf(dot(a, a)); return a * inv; }
__device__ __forceinline__ V3 madd(V3 a, V3 b, float s)
{
    return {a.x + b.x * s, a.y + b.y * s, a.z + b.z * s};
}
__device__ __forceinline__ float maxc(V3 a) { return fmaxf(fmaxf(a.x, a.y), a.z); }

// cos / sin of 2 pi u: quadrant from 4u, Taylor polynomials (Horner) on
// [0, pi/2) truncated after x^14 / x^13
__device__ __forceinline__ void sincos2pi(float u, float& c, float& s)
{
    float t = u * 4.0f;
    int q = (int)t;
    if (q > 3) q = 3;
    float f = t - (float)q;
    float x = f * 1.57079632679489661923f;
    float x2 = x * x;
    float sp = (float)(1.0 / 6227020800.0);
    sp = (float)(-1.0 / 39916800.0) + x2 * sp;
    sp = (float)(1.0 / 362880.0) + x2 * sp;
    sp = (float)(-1.0 / 5040.0) + x2 * sp;
    sp = (float)(1.0 / 120.0) + x2 * sp;
    sp = (float)(-1.0 / 6.0) + x2 * sp;
    sp = 1.0f + x2 * sp;
    float sn = x * sp;
    float cp = (float)(-1.0 / 87178291200.0);
    cp = (float)(1.0 / 479001600.0) + x2 * cp;
    cp = (float)(-1.0 / 3628800.0) + x2 * cp;
    cp = (float)(1.0 / 40320.0) + x2 * cp;
    cp = (float)(-1.0 / 720.0) + x2 * cp;
    cp = (float)(1.0 / 24.0) + x2 * cp;
    cp = -0.5f + x2 * cp;
    float cs = 1.0f + x2 * cp;
    if (q == 0) { c = cs; s = sn; }
    else if (q == 1) { c = -sn; s = cs; }
    else if (q == 2) { c = -cs; s = -sn; }
    else { c = sn; s = -cs; }
}

// ---- scene access -----------------------------------------------------------
struct SceneView {
    int n, ns, n_lights;   // triangles; of them in the LBVH (positions 0..ns-1); lights
    const float4* __restrict__ nodes;
    const float4* __restrict__ tris;
    const int2* __restrict__ tri_ml;
    const float* __restrict__ mats;
    const float* __restrict__ lights;
};

// Moller-Trumbore against a sorted triangle record; t in (0, tmax) or -1
__device__ __forceinline__ float intersect(V3 o, V3 d, const float4* tri, float tmax, int& prim)
{
    float4 a = __ldg(tri), b = __ldg(tri + 1), c = __ldg(tri + 2);
    prim = __float_as_int(a.w);
    V3 v0 = mk(a.x, a.y, a.z), e1 = mk(b.x, b.y, b.z), e2 = mk(c.x, c.y, c.z);
    V3 p = cross(d, e2);
    float det = dot(e1, p);
    if (det == 0.0f) return -1.0f;
    float inv = 1.0f / det;
    V3 s = o - v0;
    float u = dot(s, p) * inv;
    if (u < 0.0f || u > 1.0f) return -1.0f;
    V3 q = cross(s, e1);
    float v = dot(d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return -1.0f;
    float t = dot(e2, q) * inv;
    if (!(t > 0.0f) || !(t < tmax)) return -1.0f;
    return t;
}

// conservative slab test; returns entry distance or +inf on a miss
__device__ __forceinline__ float slab(float lx, float ly, float lz, float hx, float hy, float hz,
                                      V3 o, V3 inv, float tmax)
{
    float t0x = (lx - o.x) * inv.x, t1x = (hx - o.x) * inv.x;
    float t0y = (ly - o.y) * inv.y, t1y = (hy - o.y) * inv.y;
    float t0z = (lz - o.z) * inv.z, t1z = (hz - o.z) * inv.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    return tn <= tf * 1.0000005f ? tn : INFINITY;
}

// closest hit (ties to the smaller triangle index) or any hit below tmax
template <bool kAny, bool kCount = false>
__device__ int traverse(const SceneView& S, V3 o, V3 d, float tmax, float& t_out,
                        unsigned long long* nvisit = nullptr, unsigned long long* ntest = nullptr)
{
    const int n = S.ns;
    int best = -1, best_prim = 0x7fffffff;
    float bt = tmax;
    // large triangles (positions ns .. S.n-1) first: a hit there bounds the
    // tree traversal below
    for (int k = n; k < S.n; ++k) {
        int prim;
        if (kCount) ++*ntest;
        float t = intersect(o, d, S.tris + 3 * k, kAny ? tmax : T_INF, prim);
        if (t > 0.0f) {
            if (kAny) { t_out = t; return k; }
            if (t < bt || (t == bt && prim < best_prim)) { bt = t; best = k; best_prim = prim; }
        }
    }
    if (n == 0) {
        if (best >= 0) t_out = bt;
        return best;
    }
    if (n == 1) {
        int prim;
        if (kCount) ++*ntest;
        float t = intersect(o, d, S.tris, kAny ? tmax : T_INF, prim);
        if (t > 0.0f) {
            if (kAny) { t_out = t; return 0; }
            if (t < bt || (t == bt && prim < best_prim)) { bt = t; best = 0; best_prim = prim; }
        }
        if (best >= 0) t_out = bt;
        return best;
    }
    V3 inv = mk(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int stack[kStack];
    int sp = 0;
    int node = 0;
    while (true) {
        if (node < n - 1) {
            if (kCount) ++*nvisit;
            const float4* nd = S.nodes + 4 * node;
            float4 a = __ldg(nd), b = __ldg(nd + 1), c = __ldg(nd + 2), e = __ldg(nd + 3);
            float t0 = slab(a.x, a.y, a.z, a.w, b.x, b.y, o, inv, bt);
            float t1 = slab(b.z, b.w, c.x, c.y, c.z, c.w, o, inv, bt);
            int c0 = __float_as_int(e.x), c1 = __float_as_int(e.y);
            bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
            if (h0 && h1) {
                int nearc = t0 <= t1 ? c0 : c1, farc = t0 <= t1 ? c1 : c0;
                if (sp < kStack) stack[sp++] = farc;
                node = nearc;
                continue;
            }
            if (h0) { node = c0; continue; }
            if (h1) { node = c1; continue; }
        } else {
            int k = node - (n - 1), prim;
            if (kCount) ++*ntest;
            float t = intersect(o, d, S.tris + 3 * k, kAny ? tmax : T_INF, prim);
            if (t > 0.0f) {
                if (kAny) { t_out = t; return k; }
                if (t < bt || (t == bt && prim < best_prim)) { bt = t; best = k; best_prim = prim; }
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    if (best >= 0) t_out = bt;
    return best;
}

// ---- materials --------------------------------------------------------------
struct Mat { int type; V3 albedo; float alpha; V3 Le; };
__device__ __forceinline__ Mat material(const float* mats, int m)
{
    const float* p = mats + 8 * m;
    Mat r;
    r.type = (int)__ldg(p);
    r.albedo = mk(__ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
    r.alpha = __ldg(p + 4);
    r.Le = mk(__ldg(p + 5), __ldg(p + 6), __ldg(p + 7));
    return r;
}

__device__ __forceinline__ void basis(V3 n, V3& t, V3& b)
{
    float sign = copysignf(1.0f, n.z);
    float a = -1.0f / (sign + n.z);
    float bb = n.x * n.y * a;
    t = mk(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    b = mk(bb, sign + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ V3 to_local(V3 w, V3 t, V3 b, V3 n) { return mk(dot(w, t), dot(w, b), dot(w, n)); }
__device__ __forceinline__ V3 to_world(V3 w, V3 t, V3 b, V3 n)
{
    return mk(t.x * w.x + b.x * w.y + n.x * w.z, t.y * w.x + b.y * w.y + n.y * w.z,
              t.z * w.x + b.z * w.y + n.z * w.z);
}
__device__ __forceinline__ V3 cosine_sample(float u1, float u2)
{
    float r = sqrtf(u1), c, s;
    sincos2pi(u2, c, s);
    return mk(r * c, r * s, sqrtf(fmaxf(0.0f, 1.0f - u1)));
}
__device__ __forceinline__ float ggx_lambda(V3 w, float a2)
{
    float tan2 = (w.x * w.x + w.y * w.y) / (w.z * w.z);
    return (sqrtf(1.0f + a2 * tan2) - 1.0f) * 0.5f;
}
__device__ __forceinline__ float ggx_D(float hz, float a2)
{
    float den = hz * hz * (a2 - 1.0f) + 1.0f;
    return a2 / (PI_F * den * den);
}
__device__ __forceinline__ V3 schlick(V3 F0, float cosh)
{
    float m = fmaxf(0.0f, 1.0f - cosh);
    float m2 = m * m;
    float m5 = m2 * m2 * m;
    return mk(F0.x + (1.0f - F0.x) * m5, F0.y + (1.0f - F0.y) * m5, F0.z + (1.0f - F0.z) * m5);
}
__device__ V3 bsdf_eval(const Mat& m, V3 wo, V3 wi, float& pdf)
{
    if (m.type == 0) {
        pdf = wi.z * INV_PI_F;
        return m.albedo * INV_PI_F;
    }
    float a2 = m.alpha * m.alpha;
    V3 h = normalize(wo + wi);
    float D = ggx_D(h.z, a2);
    float lo = ggx_lambda(wo, a2), li = ggx_lambda(wi, a2);
    float G1 = 1.0f / (1.0f + lo);
    float G2 = 1.0f / ((1.0f + lo) + li);
    V3 F = schlick(m.albedo, dot(wo, h));
    float k = (D * G2) / ((4.0f * wo.z) * wi.z);
    pdf = (G1 * D) / (4.0f * wo.z);
    return F * k;
}
__device__ bool bsdf_sample(const Mat& m, V3 wo, float u1, float u2, V3& wi, V3& weight, float& pdf)
{
    if (m.type == 0) {
        wi = cosine_sample(u1, u2);
        if (!(wi.z > 0.0f)) return false;
        pdf = wi.z * INV_PI_F;
        weight = m.albedo;
        return true;
    }
    float al = m.alpha, a2 = al * al;
    V3 Vh = normalize(mk(al * wo.x, al * wo.y, wo.z));
    float lensq = Vh.x * Vh.x + Vh.y * Vh.y;
    V3 T1 = mk(1.0f, 0.0f, 0.0f);
    if (lensq > 0.0f) { float il = 1.0f / sqrtf(lensq); T1 = mk(-Vh.y * il, Vh.x * il, 0.0f); }
    V3 T2 = cross(Vh, T1);
    float r = sqrtf(u1), c, s;
    sincos2pi(u2, c, s);
    float t1 = r * c, t2 = r * s;
    float sv = 0.5f * (1.0f + Vh.z);
    t2 = (1.0f - sv) * sqrtf(1.0f - t1 * t1) + sv * t2;
    float q = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
    V3 Nh = mk(T1.x * t1 + T2.x * t2 + Vh.x * q, T1.y * t1 + T2.y * t2 + Vh.y * q,
               T1.z * t1 + T2.z * t2 + Vh.z * q);
    V3 h = normalize(mk(al * Nh.x, al * Nh.y, fmaxf(0.0f, Nh.z)));
    float k = 2.0f * dot(wo, h);
    wi = mk(k * h.x - wo.x, k * h.y - wo.y, k * h.z - wo.z);
    if (!(wi.z > 0.0f)) return false;
    float lo = ggx_lambda(wo, a2), li = ggx_lambda(wi, a2);
    float g = (1.0f + lo) / ((1.0f + lo) + li);
    V3 F = schlick(m.albedo, dot(wo, h));
    weight = F * g;
    float D = ggx_D(h.z, a2);
    pdf = ((1.0f / (1.0f + lo)) * D) / (4.0f * wo.z);
    return true;
}

// ---- wave kernels -----------------------------------------------------------
// One render job's part of a wave: its scene, camera and image, and the
// samples of its pixels that the wave holds -- paths path_off .. path_off +
// n_paths - 1, path path_off + q being sample s0 + q % kk of the job's
// (window) pixel q / kk
struct JobView {
    SceneView S;
    float env[3];
    float cam[12];
    int W, H, max_depth, rr_start;   // W x H: the whole image (camera, RNG pixel ids)
    int win_x0, win_y0, win_w;       // the rendered window of it (its width); whole image:
    bool windowed;                   // 0, 0, W and windowed = false
    int grid;            // camera sampling grid (1 = whole pixel footprint)
    int s0;              // first sample index of the wave
    int kk;              // samples per pixel in the wave
    int path_off;        // the job's first path in the wave
    int n_paths;         // its paths in the wave (= kk * pixels)
    uint2 key;
};

struct WaveParams {
    JobView J;           // the job of a one-job wave (a single render)
    PathSoA P;
    int layers;          // record the first-hit lobe (diffuse / specular / variance layers)
    int64_t wh;          // pixels of the job (accumulation)
    int n_paths;         // paths in the wave (every job's)
    uint32_t* cnt;       // [max_depth + 2] extension rays per bounce
    uint32_t* scnt;      // [max_depth + 1] shadow rays per bounce
    unsigned long long* stats;   // counting variant: node visits / triangle tests (closest, shadow)
};

// A batched wave holds several jobs (different scenes, images, sample
// counts); their table travels as a kernel parameter.  The job of path p is
// the one wave job (OneJob) or the table entry whose paths contain p
// (ManyJobs: binary search over path_off).
constexpr int kMaxWaveJobs = 32;
struct JobTable {
    int n;
    JobView J[kMaxWaveJobs];
};
struct OneJob {
    const JobView& J;
    __device__ __forceinline__ const JobView& operator()(int) const { return J; }
};
struct ManyJobs {
    const JobTable& T;
    __device__ __forceinline__ const JobView& operator()(int p) const
    {
        int lo = 0, hi = T.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (T.J[mid].path_off <= p) lo = mid;
            else hi = mid - 1;
        }
        return T.J[lo];
    }
};

// image pixel id of the job's path q (relative to path_off; the Philox
// counter's pixel): sample q % kk of window pixel q / kk
__device__ __forceinline__ int pixel_of(const JobView& J, int q)
{
    const int lp = q / J.kk;
    if (!J.windowed) return lp;
    return (J.win_y0 + lp / J.win_w) * J.W + (J.win_x0 + lp % J.win_w);
}

template <class Jobs>
__device__ __forceinline__ void raygen_body(const WaveParams& w, const Jobs& jobs)
{
    const PathSoA& P = w.P;
    if (blockIdx.x == 0 && threadIdx.x == 0) w.cnt[0] = (uint32_t)w.n_paths;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < w.n_paths; p += gridDim.x * blockDim.x) {
        const JobView& J = jobs(p);
        const int q = p - J.path_off;
        int pix = pixel_of(J, q);
        int sample = J.s0 + q % J.kk;
        int px = pix % J.W, py = pix / J.W;
        float4 g1 = draws((uint32_t)pix, (uint32_t)sample, 0u, 1u, J.key);
        const float* cam = J.cam;
        // grid g > 1: only the centre sub-pixel (g px + g/2, g py + g/2) of the
        // pixel's g x g block is sampled (nearest-neighbour downsampling of a
        // g-times finer image: the low-resolution renders of Sec. 3); g = 1 is
        // the whole pixel footprint, the same operations as without a grid
        const int g = J.grid;
        float sx = ((float)(px * g + g / 2) + g1.z) / (float)(J.W * g);
        float sy = ((float)(py * g + g / 2) + g1.w) / (float)(J.H * g);
        float a = 2.0f * sx - 1.0f, bq = 1.0f - 2.0f * sy;
        V3 d = normalize(mk(cam[3] + cam[6] * a + cam[9] * bq, cam[4] + cam[7] * a + cam[10] * bq,
                            cam[5] + cam[8] * a + cam[11] * bq));
        P.ox[p] = cam[0]; P.oy[p] = cam[1]; P.oz[p] = cam[2];
        P.dx[p] = d.x; P.dy[p] = d.y; P.dz[p] = d.z;
        P.bx[p] = 1.0f; P.by[p] = 1.0f; P.bz[p] = 1.0f;
        P.Lx[p] = 0.0f; P.Ly[p] = 0.0f; P.Lz[p] = 0.0f;
        P.pdf_b[p] = 0.0f; P.pdf_e[p] = 0.0f;
        P.ax[p] = 0.0f; P.ay[p] = 0.0f; P.az[p] = 0.0f;
        P.nx[p] = 0.0f; P.ny[p] = 0.0f; P.nz[p] = 0.0f; P.dep[p] = 0.0f;
        if (w.layers) P.lobe[p] = 0;
    }
}

template <bool kCount, class Jobs>
__device__ __forceinline__ void trace_body(const WaveParams& w, const Jobs& jobs, int b)
{
    unsigned long long nv = 0, nt = 0;
    const PathSoA& P = w.P;
    const int count = (int)*(volatile uint32_t*)&w.cnt[b];
    const int* q = (b & 1) ? P.q1 : P.q0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        int p = b == 0 ? i : q[i];
        V3 o = mk(P.ox[p], P.oy[p], P.oz[p]), d = mk(P.dx[p], P.dy[p], P.dz[p]);
        float t = -1.0f;
        int k = traverse<false, kCount>(jobs(p).S, o, d, T_INF, t, &nv, &nt);
        P.hit_t[p] = t;
        P.hit_id[p] = k;
    }
    if (kCount) { atomicAdd(&w.stats[0], nv); atomicAdd(&w.stats[1], nt); }
}

// warp-aggregated append: returns this lane's slot (valid only where flag)
__device__ __forceinline__ int warp_append(bool flag, uint32_t* counter)
{
    unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    return (int)(base + __popc(m & ((1u << lane) - 1u)));
}

// Per-bounce constants of the shading step
struct ShadeConst {
    V3 env;
    bool env_on;
    int n_choices;
    float pick;
};
__device__ __forceinline__ ShadeConst shade_const(const JobView& J)
{
    ShadeConst c;
    c.env = mk(J.env[0], J.env[1], J.env[2]);
    c.env_on = c.env.x > 0.0f || c.env.y > 0.0f || c.env.z > 0.0f;
    c.n_choices = J.S.n_lights + (c.env_on ? 1 : 0);
    c.pick = c.n_choices > 0 ? 1.0f / (float)c.n_choices : 0.0f;
    return c;
}

// The shading step of path p at bounce b (its hit in P.hit_id / P.hit_t):
// emission / environment with MIS, first-hit layers, next-event estimation
// (shadow ray and its contribution left in P.sd* / P.sc*), BSDF sampling and
// roulette.  cont: the path continues to bounce b + 1; shadow: a shadow ray
// was set up.  Shared by the wavefront kernel and the tail kernel, so that a
// path's arithmetic does not depend on which one shades it.
__device__ __forceinline__ void shade_path(const WaveParams& w, const JobView& J,
                                           const ShadeConst& sc0, int b, int p, bool& cont,
                                           bool& shadow)
{
    const PathSoA& P = w.P;
    const SceneView& S = J.S;
    const V3 env = sc0.env;
    const bool env_on = sc0.env_on;
    const int n_choices = sc0.n_choices;
    const float pick = sc0.pick;
    V3 o = mk(P.ox[p], P.oy[p], P.oz[p]), d = mk(P.dx[p], P.dy[p], P.dz[p]);
    V3 beta = mk(P.bx[p], P.by[p], P.bz[p]);
    V3 L = mk(P.Lx[p], P.Ly[p], P.Lz[p]);
    float pdf_b = P.pdf_b[p], pdf_e = P.pdf_e[p];
    int k = P.hit_id[p];
    float t = P.hit_t[p];
    do {
        if (k < 0) {
            if (env_on) {
                float wgt = 1.0f;
                if (b > 0 && pdf_e > 0.0f)
                    wgt = (pdf_b * pdf_b) / (pdf_b * pdf_b + pdf_e * pdf_e);
                L = mk(L.x + beta.x * env.x * wgt, L.y + beta.y * env.y * wgt,
                       L.z + beta.z * env.z * wgt);
            }
            break;
        }
        const float4* tr = S.tris + 3 * k;
        float4 ta = __ldg(tr), tb = __ldg(tr + 1), tc = __ldg(tr + 2);
        int2 ml = __ldg(S.tri_ml + k);
        V3 p3 = madd(o, d, t);
        V3 ng = normalize(cross(mk(tb.x, tb.y, tb.z), mk(tc.x, tc.y, tc.z)));
        float cos_o = dot(d, ng);
        V3 ns = cos_o > 0.0f ? ng * -1.0f : ng;
        Mat m = material(S.mats, ml.x);
        if (b == 0) {
            P.ax[p] = m.albedo.x; P.ay[p] = m.albedo.y; P.az[p] = m.albedo.z;
            P.nx[p] = ns.x; P.ny[p] = ns.y; P.nz[p] = ns.z; P.dep[p] = t;
            if (w.layers) P.lobe[p] = m.type == 0 ? 1 : 2;
        }
        if ((m.Le.x > 0.0f || m.Le.y > 0.0f || m.Le.z > 0.0f) && cos_o < 0.0f) {
            float wgt = 1.0f;
            int li = ml.y;
            if (b > 0 && li >= 0) {
                const float* lq = S.lights + 12 * li;
                V3 ln = cross(mk(__ldg(lq + 3), __ldg(lq + 4), __ldg(lq + 5)),
                              mk(__ldg(lq + 6), __ldg(lq + 7), __ldg(lq + 8)));
                float area = sqrtf(dot(ln, ln));
                float pl = pick * (t * t) / (-cos_o * area);
                wgt = (pdf_b * pdf_b) / (pdf_b * pdf_b + pl * pl);
            }
            L = mk(L.x + beta.x * m.Le.x * wgt, L.y + beta.y * m.Le.y * wgt,
                   L.z + beta.z * m.Le.z * wgt);
        }
        if (b == J.max_depth) break;
        if (!(m.albedo.x > 0.0f || m.albedo.y > 0.0f || m.albedo.z > 0.0f)) break;

        const int qj = p - J.path_off;
        int pix = pixel_of(J, qj);
        uint32_t sample = (uint32_t)(J.s0 + qj % J.kk);
        float4 g0 = draws((uint32_t)pix, sample, (uint32_t)b, 0u, J.key);
        float4 g1 = draws((uint32_t)pix, sample, (uint32_t)b, 1u, J.key);
        V3 T, B;
        basis(ns, T, B);
        V3 wo = to_local(d * -1.0f, T, B, ns);
        V3 org = madd(p3, ns, RAY_EPS);
        P.ox[p] = org.x; P.oy[p] = org.y; P.oz[p] = org.z;

        if (n_choices > 0) {
            int kl = (int)(g1.x * (float)n_choices);
            if (kl > n_choices - 1) kl = n_choices - 1;
            if (kl < S.n_lights) {
                const float* lq = S.lights + 12 * kl;
                V3 p0 = mk(__ldg(lq), __ldg(lq + 1), __ldg(lq + 2));
                V3 e1 = mk(__ldg(lq + 3), __ldg(lq + 4), __ldg(lq + 5));
                V3 e2 = mk(__ldg(lq + 6), __ldg(lq + 7), __ldg(lq + 8));
                V3 Le = mk(__ldg(lq + 9), __ldg(lq + 10), __ldg(lq + 11));
                V3 x = madd(madd(p0, e1, g0.z), e2, g0.w);
                V3 ln = cross(e1, e2);
                float area = sqrtf(dot(ln, ln));
                V3 nl = ln * (1.0f / area);
                V3 dl = x - org;
                float d2 = dot(dl, dl);
                float dist = sqrtf(d2);
                V3 wi = dl * (1.0f / dist);
                float cos_l = -dot(wi, nl), cos_s = dot(wi, ns);
                if (cos_l > 0.0f && cos_s > 0.0f) {
                    float pb;
                    V3 f = bsdf_eval(m, wo, to_local(wi, T, B, ns), pb);
                    float pl = pick * d2 / (cos_l * area);
                    float wgt = (pl * pl) / (pl * pl + pb * pb);
                    float sc = (cos_s / pl) * wgt;
                    P.scx[p] = beta.x * f.x * Le.x * sc;
                    P.scy[p] = beta.y * f.y * Le.y * sc;
                    P.scz[p] = beta.z * f.z * Le.z * sc;
                    P.sdx[p] = wi.x; P.sdy[p] = wi.y; P.sdz[p] = wi.z;
                    P.stmax[p] = dist * SHADOW_FRAC;
                    shadow = true;
                }
            } else {
                V3 wl = cosine_sample(g0.z, g0.w);
                if (wl.z > 0.0f) {
                    V3 wi = normalize(to_world(wl, T, B, ns));
                    float pb;
                    V3 f = bsdf_eval(m, wo, wl, pb);
                    float pe = pick * wl.z * INV_PI_F;
                    float wgt = (pe * pe) / (pe * pe + pb * pb);
                    float sc = (wl.z / pe) * wgt;
                    P.scx[p] = beta.x * f.x * env.x * sc;
                    P.scy[p] = beta.y * f.y * env.y * sc;
                    P.scz[p] = beta.z * f.z * env.z * sc;
                    P.sdx[p] = wi.x; P.sdy[p] = wi.y; P.sdz[p] = wi.z;
                    P.stmax[p] = T_INF;
                    shadow = true;
                }
            }
        }

        V3 wl, wt;
        float pb;
        if (!bsdf_sample(m, wo, g0.x, g0.y, wl, wt, pb)) break;
        beta = mk(beta.x * wt.x, beta.y * wt.y, beta.z * wt.z);
        pdf_b = pb;
        pdf_e = env_on ? pick * wl.z * INV_PI_F : 0.0f;
        if (!(maxc(beta) > 0.0f)) break;
        if (b >= J.rr_start) {
            float qq = fminf(0.95f, maxc(beta));
            if (g1.y >= qq) break;
            beta = mk(beta.x / qq, beta.y / qq, beta.z / qq);
        }
        V3 nd = normalize(to_world(wl, T, B, ns));
        P.dx[p] = nd.x; P.dy[p] = nd.y; P.dz[p] = nd.z;
        P.bx[p] = beta.x; P.by[p] = beta.y; P.bz[p] = beta.z;
        P.pdf_b[p] = pdf_b; P.pdf_e[p] = pdf_e;
        cont = true;
    } while (0);
    P.Lx[p] = L.x; P.Ly[p] = L.y; P.Lz[p] = L.z;
}

template <class Jobs>
__device__ __forceinline__ void shade_body(const WaveParams& w, const Jobs& jobs, int b)
{
    const PathSoA& P = w.P;
    const int count = (int)*(volatile uint32_t*)&w.cnt[b];
    const int* q = (b & 1) ? P.q1 : P.q0;
    int* qn = (b & 1) ? P.q0 : P.q1;
    const int stride = gridDim.x * blockDim.x;
    const int end = (count + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) {
        bool cont = false, shadow = false;
        int p = 0;
        if (i < count) {
            p = b == 0 ? i : q[i];
            const JobView& J = jobs(p);
            shade_path(w, J, shade_const(J), b, p, cont, shadow);
        }
        int slot = warp_append(cont, &w.cnt[b + 1]);
        if (cont) qn[slot] = p;
        int sslot = warp_append(shadow, &w.scnt[b]);
        if (shadow) P.qs[sslot] = p;
    }
}

template <bool kCount, class Jobs>
__device__ __forceinline__ void shadow_body(const WaveParams& w, const Jobs& jobs, int b)
{
    unsigned long long nv = 0, nt = 0;
    const PathSoA& P = w.P;
    const int count = (int)*(volatile uint32_t*)&w.scnt[b];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        int p = P.qs[i];
        V3 o = mk(P.ox[p], P.oy[p], P.oz[p]), d = mk(P.sdx[p], P.sdy[p], P.sdz[p]);
        float t;
        if (traverse<true, kCount>(jobs(p).S, o, d, P.stmax[p], t, &nv, &nt) < 0) {
            P.Lx[p] = P.Lx[p] + P.scx[p];
            P.Ly[p] = P.Ly[p] + P.scy[p];
            P.Lz[p] = P.Lz[p] + P.scz[p];
        }
    }
    if (kCount) { atomicAdd(&w.stats[2], nv); atomicAdd(&w.stats[3], nt); }
}

// The late bounces in one launch: each thread takes a path of queue q_b0,
// follows it to its end (closest hit, shading, shadow ray, next bounce) and
// then takes the next one.  Late bounces hold few paths, so one launch per
// step would wait for each step's slowest ray; here a path's steps run back
// to back.  Every path meets the same operations in the same order as in the
// wavefront kernels (trace, shade, shadow; a path's state lives in P), so
// its radiance is bit-identical; the per-bounce counts are the same numbers,
// gathered per block in shared memory.  cnt[kWorkSlot] hands out the paths.
// 32 registers and 8 blocks per SM, as the traversal kernels: with 64
// registers (4 blocks) the tail ran 2-7% slower despite no spills.
constexpr int kWorkSlot = 63;
template <bool kCount, class Jobs>
__device__ __forceinline__ void tail_body(const WaveParams& w, const Jobs& jobs, int b0,
                                          int max_depth)
{
    __shared__ uint32_t s_cnt[64], s_scnt[64];
    for (int j = threadIdx.x; j < 64; j += blockDim.x) { s_cnt[j] = 0u; s_scnt[j] = 0u; }
    __syncthreads();
    unsigned long long nv = 0, nt = 0, sv = 0, stt = 0;
    const PathSoA& P = w.P;
    const int count = (int)*(volatile uint32_t*)&w.cnt[b0];
    const int* q = (b0 & 1) ? P.q1 : P.q0;
    const int lane = threadIdx.x & 31;
    int p = -1, b = b0;
    bool drained = false;   // warp-uniform: the queue has been handed out
    for (;;) {
        // refill: lanes without a path take consecutive queue slots
        const bool want = p < 0;
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (m && !drained) {
            const int leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&w.cnt[kWorkSlot], (uint32_t)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            drained = base + (uint32_t)__popc(m) >= (uint32_t)count;
            if (want) {
                const uint32_t i = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                if (i < (uint32_t)count) { p = b0 == 0 ? (int)i : q[i]; b = b0; }
            }
        }
        if (!__any_sync(0xffffffffu, p >= 0)) break;
        if (p < 0) continue;
        const JobView& J = jobs(p);
        V3 o = mk(P.ox[p], P.oy[p], P.oz[p]), d = mk(P.dx[p], P.dy[p], P.dz[p]);
        float t = -1.0f;
        const int k = traverse<false, kCount>(J.S, o, d, T_INF, t, &nv, &nt);
        P.hit_t[p] = t;
        P.hit_id[p] = k;
        bool cont = false, shadow = false;
        shade_path(w, J, shade_const(J), b, p, cont, shadow);
        if (shadow) {
            atomicAdd(&s_scnt[b], 1u);
            V3 so = mk(P.ox[p], P.oy[p], P.oz[p]), sd = mk(P.sdx[p], P.sdy[p], P.sdz[p]);
            float ts;
            if (traverse<true, kCount>(J.S, so, sd, P.stmax[p], ts, &sv, &stt) < 0) {
                P.Lx[p] = P.Lx[p] + P.scx[p];
                P.Ly[p] = P.Ly[p] + P.scy[p];
                P.Lz[p] = P.Lz[p] + P.scz[p];
            }
        }
        if (cont) { atomicAdd(&s_cnt[b + 1], 1u); ++b; }
        else p = -1;
    }
    __syncthreads();
    for (int j = b0 + threadIdx.x; j <= max_depth + 1; j += blockDim.x) {
        if (j > b0 && s_cnt[j]) atomicAdd(&w.cnt[j], s_cnt[j]);
        if (j <= max_depth && s_scnt[j]) atomicAdd(&w.scnt[j], s_scnt[j]);
    }
    if (kCount) {
        atomicAdd(&w.stats[0], nv); atomicAdd(&w.stats[1], nt);
        atomicAdd(&w.stats[2], sv); atomicAdd(&w.stats[3], stt);
        atomicAdd(&w.stats[4], nv); atomicAdd(&w.stats[5], nt);
        atomicAdd(&w.stats[6], sv); atomicAdd(&w.stats[7], stt);
    }
}

// The kernels: a one-job wave (a render) and a batched wave (a table of jobs)
__global__ void __launch_bounds__(kThreads) k_raygen(const __grid_constant__ WaveParams w)
{
    raygen_body(w, OneJob{w.J});
}
__global__ void __launch_bounds__(kThreads)
    k_raygen_b(const __grid_constant__ WaveParams w, const __grid_constant__ JobTable T)
{
    raygen_body(w, ManyJobs{T});
}
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 8) k_trace(const __grid_constant__ WaveParams w, int b)
{
    trace_body<kCount>(w, OneJob{w.J}, b);
}
__global__ void __launch_bounds__(kThreads, 8)
    k_trace_b(const __grid_constant__ WaveParams w, const __grid_constant__ JobTable T, int b)
{
    trace_body<false>(w, ManyJobs{T}, b);
}
__global__ void __launch_bounds__(kThreads) k_shade(const __grid_constant__ WaveParams w, int b)
{
    shade_body(w, OneJob{w.J}, b);
}
__global__ void __launch_bounds__(kThreads)
    k_shade_b(const __grid_constant__ WaveParams w, const __grid_constant__ JobTable T, int b)
{
    shade_body(w, ManyJobs{T}, b);
}
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 8) k_shadow(const __grid_constant__ WaveParams w, int b)
{
    shadow_body<kCount>(w, OneJob{w.J}, b);
}
__global__ void __launch_bounds__(kThreads, 8)
    k_shadow_b(const __grid_constant__ WaveParams w, const __grid_constant__ JobTable T, int b)
{
    shadow_body<false>(w, ManyJobs{T}, b);
}
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 8) k_tail(const __grid_constant__ WaveParams w, int b0)
{
    tail_body<kCount>(w, OneJob{w.J}, b0, w.J.max_depth);
}
__global__ void __launch_bounds__(kThreads, 8)
    k_tail_b(const __grid_constant__ WaveParams w, const __grid_constant__ JobTable T, int b0,
             int max_depth)
{
    tail_body<false>(w, ManyJobs{T}, b0, max_depth);
}

// Path p of a wave is sample p % kk of pixel p / kk: a pixel's samples are
// consecutive paths, so a warp's camera rays leave through one or a few
// pixels (coherent bounce-0 traversal and shading).  The accumulation reads
// each pixel's kk consecutive samples, V at a time (one 16-byte load per
// field when kk is a multiple of 4: a warp's loads are then contiguous).
template <int V> struct Vec;
template <> struct Vec<1> {
    float v[1];
    __device__ __forceinline__ void load(const float* p) { v[0] = p[0]; }
    __device__ __forceinline__ void load_int(const int* p) { v[0] = __int_as_float(p[0]); }
};
template <> struct Vec<4> {
    float v[4];
    __device__ __forceinline__ void load(const float* p)
    {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ __forceinline__ void load_int(const int* p)
    {
        const int4 q = *reinterpret_cast<const int4*>(p);
        v[0] = __int_as_float(q.x); v[1] = __int_as_float(q.y);
        v[2] = __int_as_float(q.z); v[3] = __int_as_float(q.w);
    }
};

// per pixel: add this wave's samples in sample order (Kahan for radiance)
template <int V>
__global__ void __launch_bounds__(kThreads) k_accumulate(const __grid_constant__ WaveParams w,
                                                          float* acc, int kk)
{
    const PathSoA& P = w.P;
    const int64_t poff = w.J.path_off;
    const int64_t wh = w.wh;
    for (int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pix < wh;
         pix += (int64_t)gridDim.x * blockDim.x) {
        float* a = acc + 13 * pix;
        float s0 = a[0], s1 = a[1], s2 = a[2], c0 = a[3], c1 = a[4], c2 = a[5];
        float ax = a[6], ay = a[7], az = a[8], nx = a[9], ny = a[10], nz = a[11], ds = a[12];
        for (int sb = 0; sb < kk; sb += V) {
            const int64_t p = poff + pix * kk + sb;
            Vec<V> Lx, Ly, Lz, Ax, Ay, Az, Nx, Ny, Nz, D;
            Lx.load(P.Lx + p); Ly.load(P.Ly + p); Lz.load(P.Lz + p);
            Ax.load(P.ax + p); Ay.load(P.ay + p); Az.load(P.az + p);
            Nx.load(P.nx + p); Ny.load(P.ny + p); Nz.load(P.nz + p);
            D.load(P.dep + p);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                float y, t;
                y = Lx.v[j] - c0; t = s0 + y; c0 = (t - s0) - y; s0 = t;
                y = Ly.v[j] - c1; t = s1 + y; c1 = (t - s1) - y; s1 = t;
                y = Lz.v[j] - c2; t = s2 + y; c2 = (t - s2) - y; s2 = t;
                ax = ax + Ax.v[j]; ay = ay + Ay.v[j]; az = az + Az.v[j];
                nx = nx + Nx.v[j]; ny = ny + Ny.v[j]; nz = nz + Nz.v[j];
                ds = ds + D.v[j];
            }
        }
        a[0] = s0; a[1] = s1; a[2] = s2; a[3] = c0; a[4] = c1; a[5] = c2;
        a[6] = ax; a[7] = ay; a[8] = az; a[9] = nx; a[10] = ny; a[11] = nz; a[12] = ds;
    }
}

// extra layers, only when requested: per pixel the diffuse and specular sums
// (each sample's radiance to the layer of its first-hit lobe) and the sum of
// squares for the variance, plain FP32 sums in sample order
template <int V>
__global__ void __launch_bounds__(kThreads) k_accumulate_layers(const __grid_constant__ WaveParams w,
                                                                 float* acc2, int kk)
{
    const PathSoA& P = w.P;
    const int64_t poff = w.J.path_off;
    const int64_t wh = w.wh;
    for (int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pix < wh;
         pix += (int64_t)gridDim.x * blockDim.x) {
        float* e = acc2 + 9 * pix;
        float d0 = e[0], d1 = e[1], d2 = e[2], p0 = e[3], p1 = e[4], p2 = e[5];
        float q0 = e[6], q1 = e[7], q2 = e[8];
        for (int sb = 0; sb < kk; sb += V) {
            const int64_t p = poff + pix * kk + sb;
            Vec<V> Lx, Ly, Lz, Lo;
            Lx.load(P.Lx + p); Ly.load(P.Ly + p); Lz.load(P.Lz + p);
            Lo.load_int(P.lobe + p);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float lx = Lx.v[j], ly = Ly.v[j], lz = Lz.v[j];
                const int lobe = __float_as_int(Lo.v[j]);
                d0 = d0 + (lobe == 1 ? lx : 0.0f); d1 = d1 + (lobe == 1 ? ly : 0.0f);
                d2 = d2 + (lobe == 1 ? lz : 0.0f);
                p0 = p0 + (lobe == 2 ? lx : 0.0f); p1 = p1 + (lobe == 2 ? ly : 0.0f);
                p2 = p2 + (lobe == 2 ? lz : 0.0f);
                q0 = q0 + lx * lx; q1 = q1 + ly * ly; q2 = q2 + lz * lz;
            }
        }
        e[0] = d0; e[1] = d1; e[2] = d2; e[3] = p0; e[4] = p1; e[5] = p2;
        e[6] = q0; e[7] = q1; e[8] = q2;
    }
}

__global__ void k_counts(const uint32_t* cnt, const uint32_t* scnt, int nb, uint64_t* counts,
                         uint64_t* shadow_counts)
{
    int b = threadIdx.x;
    if (b >= nb) return;
    if (counts) counts[b] += cnt[b];
    if (shadow_counts) shadow_counts[b] += scnt[b];
}

__global__ void k_resolve(const float* __restrict__ acc, const float* __restrict__ acc2, int64_t wh,
                          int spp, float* radiance, float* albedo, float* normal, float* depth,
                          float* diffuse, float* specular, float* variance)
{
    float fs = (float)spp;
    for (int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pix < wh;
         pix += (int64_t)gridDim.x * blockDim.x) {
        const float* a = acc + 13 * pix;
        radiance[3 * pix] = a[0] / fs; radiance[3 * pix + 1] = a[1] / fs; radiance[3 * pix + 2] = a[2] / fs;
        if (albedo) { albedo[3 * pix] = a[6] / fs; albedo[3 * pix + 1] = a[7] / fs; albedo[3 * pix + 2] = a[8] / fs; }
        if (normal) { normal[3 * pix] = a[9] / fs; normal[3 * pix + 1] = a[10] / fs; normal[3 * pix + 2] = a[11] / fs; }
        if (depth) depth[pix] = a[12] / fs;
        if (!acc2) continue;
        const float* e = acc2 + 9 * pix;
        if (diffuse) for (int c = 0; c < 3; ++c) diffuse[3 * pix + c] = e[c] / fs;
        if (specular) for (int c = 0; c < 3; ++c) specular[3 * pix + c] = e[3 + c] / fs;
        if (variance) {
            // sample variance of the pixel mean: (sum L^2 - (sum L)^2 / N) / (N (N - 1))
            for (int c = 0; c < 3; ++c) {
                float v = 0.0f;
                if (spp > 1) {
                    v = (e[6 + c] - a[c] * a[c] / fs) / (fs * (fs - 1.0f));
                    if (!(v > 0.0f)) v = 0.0f;
                }
                variance[3 * pix + c] = v;
            }
        }
    }
}

__global__ void k_cast(SceneView S, const float* orig, const float* dir, int n, int* prim, float* tout)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        V3 o = mk(orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]);
        V3 d = mk(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
        float t = -1.0f;
        int k = traverse<false>(S, o, d, T_INF, t);
        if (k >= 0) {
            prim[i] = __float_as_int(__ldg(S.tris + 3 * k).w);
            tout[i] = t;
        } else {
            prim[i] = -1;
            tout[i] = -1.0f;
        }
    }
}

__global__ void k_philox(const uint32_t* triples, int n, uint2 key, float* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (uint32_t g = 0; g < 2; ++g) {
        float4 u = draws(triples[3 * i], triples[3 * i + 1], triples[3 * i + 2], g, key);
        out[8 * i + 4 * g] = u.x; out[8 * i + 4 * g + 1] = u.y;
        out[8 * i + 4 * g + 2] = u.z; out[8 * i + 4 * g + 3] = u.w;
    }
}

SceneView view(const mrs_scene_s* S)
{
    return SceneView{S->n, S->ns, S->n_lights, S->nodes, S->tris, S->tri_ml, S->mats, S->lights};
}

// persistent grid of the tail kernel: as many blocks as fit on the GPU at once
int tail_grid(bool counting)
{
    static int g[2] = {0, 0};
    int& v = g[counting ? 1 : 0];
    if (!v) {
        int per_sm = 0;
        if (counting)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail<true>, kThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail<false>, kThreads, 0);
        v = sm_count() * (per_sm < 1 ? 1 : per_sm);
    }
    return v;
}

int tail_grid_batch()
{
    static int v = 0;
    if (!v) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail_b, kThreads, 0);
        v = sm_count() * (per_sm < 1 ? 1 : per_sm);
    }
    return v;
}

inline int grid_for(int64_t n)
{
    int64_t g = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace mrs

using namespace mrs;

static mrs_status render_impl(mrs_scene S, Buf& arena, int64_t wave_paths, int32_t tail,
                              int32_t W, int32_t H,
                              int32_t spp, int32_t max_depth, int32_t rr_start, uint64_t seed,
                              int32_t grid,
                              float* radiance, float* albedo, float* normal, float* depth,
                              float* diffuse, float* specular, float* variance,
                              uint64_t* counts, uint64_t* shadow_counts,
                              unsigned long long* stats, void* stream, const int32_t* win = nullptr)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(W >= 1 && W <= 16384 && H >= 1 && H <= 16384, "W, H must be in [1, 16384]");
    MRS_ARG(spp >= 1 && spp <= 65536, "spp must be in [1, 65536]");
    MRS_ARG(max_depth >= 0 && max_depth <= 32, "max_depth must be in [0, 32]");
    MRS_ARG(radiance != nullptr, "radiance is NULL");
    MRS_ARG(grid >= 1 && grid <= 64, "grid must be in [1, 64]");
    MRS_ARG((int64_t)W * grid <= 65536 && (int64_t)H * grid <= 65536, "W * grid, H * grid must be <= 65536");
    int32_t wx0 = 0, wy0 = 0, ww = W, wh_ = H;
    if (win) {
        wx0 = win[0]; wy0 = win[1]; ww = win[2]; wh_ = win[3];
        MRS_ARG(ww >= 1 && wh_ >= 1 && wx0 >= 0 && wy0 >= 0 && wx0 + ww <= W && wy0 + wh_ <= H,
                "window must lie inside the W x H image");
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t wh = (int64_t)ww * wh_;
    int64_t k = wave_paths / wh;
    if (k < 1) k = 1;
    if (k > spp) k = spp;
    MRS_ARG(k * wh <= (int64_t(1) << 31) - 1, "wave too large");
    const int64_t P = k * wh;
    const int nb = max_depth + 1;
    // arena: 34 float / int arrays of P paths, accumulator 13 * wh, counters,
    // then (extra layers only) accumulator 9 * wh
    const int kArrays = 34;
    const bool layers = diffuse || specular || variance;
    size_t arr = ((size_t)P * 4 + 255) & ~(size_t)255;
    size_t off_cnt = arr * kArrays + (size_t)wh * 13 * 4 + 256;
    size_t off_acc2 = off_cnt + 4 * 2 * 64;
    size_t need = off_acc2 + (layers ? (size_t)wh * 9 * 4 : 0);
    mrs_status s = arena.ensure(need);
    if (s != MRS_OK) return s;
    char* base = arena.as<char>();
    float* f[kArrays];
    for (int i = 0; i < kArrays; ++i) f[i] = (float*)(base + arr * i);
    PathSoA soa;
    float** fields[] = {&soa.ox, &soa.oy, &soa.oz, &soa.dx, &soa.dy, &soa.dz, &soa.bx, &soa.by,
                        &soa.bz, &soa.Lx, &soa.Ly, &soa.Lz, &soa.pdf_b, &soa.pdf_e, &soa.hit_t,
                        &soa.sdx, &soa.sdy, &soa.sdz, &soa.stmax, &soa.scx, &soa.scy, &soa.scz,
                        &soa.ax, &soa.ay, &soa.az, &soa.nx, &soa.ny, &soa.nz, &soa.dep};
    int fi = 0;
    for (float** fp : fields) *fp = f[fi++];
    soa.hit_id = (int*)f[fi++];
    soa.q0 = (int*)f[fi++];
    soa.q1 = (int*)f[fi++];
    soa.qs = (int*)f[fi++];
    soa.lobe = (int*)f[fi++];
    float* acc = (float*)(base + arr * kArrays);
    uint32_t* cnt = (uint32_t*)(base + off_cnt);
    uint32_t* scnt = cnt + 64;
    float* acc2 = layers ? (float*)(base + off_acc2) : nullptr;

    WaveParams w;
    w.J.S = view(S);
    w.P = soa;
    memcpy(w.J.env, S->env, sizeof(w.J.env));
    memcpy(w.J.cam, S->cam, sizeof(w.J.cam));
    w.J.W = W; w.J.H = H; w.J.max_depth = max_depth;
    w.J.win_x0 = wx0; w.J.win_y0 = wy0; w.J.win_w = ww;
    w.J.windowed = ww != W || wh_ != H;
    w.J.grid = grid;
    w.layers = layers ? 1 : 0;
    w.J.rr_start = rr_start < 0 ? 0x7fffffff : rr_start;
    w.J.path_off = 0;
    w.wh = wh;
    w.J.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    w.cnt = cnt;
    w.scnt = scnt;
    w.stats = stats;

    MRS_CHECK(cudaMemsetAsync(acc, 0, (size_t)wh * 13 * 4, st));
    if (acc2) MRS_CHECK(cudaMemsetAsync(acc2, 0, (size_t)wh * 9 * 4, st));
    if (counts) MRS_CHECK(cudaMemsetAsync(counts, 0, sizeof(uint64_t) * nb, st));
    if (shadow_counts) MRS_CHECK(cudaMemsetAsync(shadow_counts, 0, sizeof(uint64_t) * nb, st));
    for (int s0 = 0; s0 < spp; s0 += (int)k) {
        int kk = (int)((spp - s0) < k ? (spp - s0) : k);
        w.J.s0 = s0;
        w.J.kk = kk;
        w.J.n_paths = (int)(kk * wh);
        w.n_paths = w.J.n_paths;
        MRS_CHECK(cudaMemsetAsync(cnt, 0, 4 * 2 * 64, st));
        int g = grid_for(w.n_paths);
        MRS_TIMED(PK_RAYGEN, st, k_raygen<<<g, kThreads, 0, st>>>(w));
        MRS_LAUNCHED(1);
        // first bounce of the tail kernel: by default bounce 1 (on the 200k-
        // triangle scene at 1024^2, 4 and 16 spp, with and without roulette,
        // and 256^2 at 64 spp, tails from bounce 0-3 beat the wavefront alone;
        // from bounce 1 by 3-5% more than from bounce 2, the next best)
        const int b_tail = tail >= 0 ? tail : 1;
        for (int b = 0; b <= max_depth && b < b_tail; ++b) {
            if (stats) MRS_TIMED(PK_TRACE, st, k_trace<true><<<g, kThreads, 0, st>>>(w, b));
            else MRS_TIMED(PK_TRACE, st, k_trace<false><<<g, kThreads, 0, st>>>(w, b));
            MRS_LAUNCHED(1);
            MRS_TIMED(PK_SHADE, st, k_shade<<<g, kThreads, 0, st>>>(w, b));
            MRS_LAUNCHED(1);
            if (stats) MRS_TIMED(PK_SHADOW, st, k_shadow<true><<<g, kThreads, 0, st>>>(w, b));
            else MRS_TIMED(PK_SHADOW, st, k_shadow<false><<<g, kThreads, 0, st>>>(w, b));
            MRS_LAUNCHED(1);
        }
        if (b_tail <= max_depth) {
            const int gt = tail_grid(stats != nullptr);
            if (stats) MRS_TIMED(PK_TAIL, st, k_tail<true><<<gt, kThreads, 0, st>>>(w, b_tail));
            else MRS_TIMED(PK_TAIL, st, k_tail<false><<<gt, kThreads, 0, st>>>(w, b_tail));
            MRS_LAUNCHED(1);
        }
        // 16-byte sample loads when every pixel's run of kk samples starts on
        // a 16-byte boundary (the arrays are 256-byte aligned)
        const bool v4 = kk % 4 == 0;
        if (v4) MRS_TIMED(PK_ACCUM, st, k_accumulate<4><<<grid_for(wh), kThreads, 0, st>>>(w, acc, kk));
        else MRS_TIMED(PK_ACCUM, st, k_accumulate<1><<<grid_for(wh), kThreads, 0, st>>>(w, acc, kk));
        MRS_LAUNCHED(1);
        if (acc2) {
            if (v4)
                MRS_TIMED(PK_ACCUM, st, k_accumulate_layers<4><<<grid_for(wh), kThreads, 0, st>>>(w, acc2, kk));
            else
                MRS_TIMED(PK_ACCUM, st, k_accumulate_layers<1><<<grid_for(wh), kThreads, 0, st>>>(w, acc2, kk));
            MRS_LAUNCHED(1);
        }
        if (counts || shadow_counts) {
            k_counts<<<1, 64, 0, st>>>(cnt, scnt, nb, counts, shadow_counts);
            MRS_LAUNCHED(1);
        }
    }
    k_resolve<<<grid_for(wh), kThreads, 0, st>>>(acc, acc2, wh, spp, radiance, albedo, normal, depth,
                                                 diffuse, specular, variance);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "render launch");
}

extern "C" mrs_status mrs_render(mrs_scene S, int32_t W, int32_t H, int32_t spp, int32_t max_depth,
                                 int32_t rr_start, uint64_t seed, float* radiance, float* albedo,
                                 float* normal, float* depth, uint64_t* counts,
                                 uint64_t* shadow_counts, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    return render_impl(S, S->arena, S->wave_paths, S->tail_bounce, W, H, spp, max_depth, rr_start, seed, 1, radiance,
                       albedo, normal, depth, nullptr, nullptr, nullptr, counts, shadow_counts,
                       nullptr, stream);
}

extern "C" mrs_status mrs_ctx_create(mrs_ctx* out)
{
    MRS_ARG(out != nullptr, "out is NULL");
    *out = new mrs_ctx_s();
    return MRS_OK;
}

extern "C" mrs_status mrs_ctx_free(mrs_ctx ctx)
{
    if (!ctx) return MRS_OK;
    cudaDeviceSynchronize();
    ctx->arena.release();
    delete ctx;
    return MRS_OK;
}

extern "C" mrs_status mrs_ctx_set_wave(mrs_ctx ctx, int64_t max_paths)
{
    MRS_ARG(ctx != nullptr, "ctx is NULL");
    MRS_ARG(max_paths >= 1 && max_paths <= (int64_t(1) << 30), "wave size out of range [1, 2^30]");
    ctx->wave_paths = max_paths;
    return MRS_OK;
}

extern "C" mrs_status mrs_ctx_set_tail(mrs_ctx ctx, int32_t bounce)
{
    MRS_ARG(ctx != nullptr, "ctx is NULL");
    MRS_ARG(bounce >= -1 && bounce <= 64, "tail bounce out of range [-1, 64]");
    ctx->tail_bounce = bounce;
    return MRS_OK;
}

extern "C" mrs_status mrs_render_ctx(mrs_ctx ctx, mrs_scene S, int32_t W, int32_t H, int32_t spp,
                                     int32_t max_depth, int32_t rr_start, uint64_t seed,
                                     float* radiance, float* albedo, float* normal, float* depth,
                                     uint64_t* counts, uint64_t* shadow_counts, void* stream)
{
    MRS_ARG(ctx != nullptr, "ctx is NULL");
    MRS_ARG(S != nullptr, "scene is NULL");
    return render_impl(S, ctx->arena, ctx->wave_paths, ctx->tail_bounce, W, H, spp, max_depth, rr_start, seed, 1,
                       radiance, albedo, normal, depth, nullptr, nullptr, nullptr, counts,
                       shadow_counts, nullptr, stream);
}

extern "C" mrs_status mrs_render_grid(mrs_ctx ctx, mrs_scene S, int32_t W, int32_t H, int32_t spp,
                                      int32_t max_depth, int32_t rr_start, uint64_t seed,
                                      int32_t grid, float* radiance, float* albedo, float* normal,
                                      float* depth, uint64_t* counts, uint64_t* shadow_counts,
                                      void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    Buf& arena = ctx ? ctx->arena : S->arena;
    int64_t wave = ctx ? ctx->wave_paths : S->wave_paths;
    int32_t tail = ctx ? ctx->tail_bounce : S->tail_bounce;
    return render_impl(S, arena, wave, tail, W, H, spp, max_depth, rr_start, seed, grid, radiance, albedo,
                       normal, depth, nullptr, nullptr, nullptr, counts, shadow_counts, nullptr,
                       stream);
}

extern "C" mrs_status mrs_render_layers(mrs_ctx ctx, mrs_scene S, int32_t W, int32_t H, int32_t spp,
                                        int32_t max_depth, int32_t rr_start, uint64_t seed,
                                        int32_t grid, const mrs_render_out* out, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(out != nullptr, "out is NULL");
    Buf& arena = ctx ? ctx->arena : S->arena;
    int64_t wave = ctx ? ctx->wave_paths : S->wave_paths;
    int32_t tail = ctx ? ctx->tail_bounce : S->tail_bounce;
    return render_impl(S, arena, wave, tail, W, H, spp, max_depth, rr_start, seed, grid, out->radiance,
                       out->albedo, out->normal, out->depth, out->diffuse, out->specular,
                       out->variance, out->counts, out->shadow_counts, nullptr, stream);
}

extern "C" mrs_status mrs_render_window(mrs_ctx ctx, mrs_scene S, int32_t W, int32_t H, int32_t x0,
                                        int32_t y0, int32_t w, int32_t h, int32_t spp,
                                        int32_t max_depth, int32_t rr_start, uint64_t seed,
                                        int32_t grid, const mrs_render_out* out, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(out != nullptr, "out is NULL");
    Buf& arena = ctx ? ctx->arena : S->arena;
    int64_t wave = ctx ? ctx->wave_paths : S->wave_paths;
    int32_t tail = ctx ? ctx->tail_bounce : S->tail_bounce;
    const int32_t win[4] = {x0, y0, w, h};
    return render_impl(S, arena, wave, tail, W, H, spp, max_depth, rr_start, seed, grid, out->radiance,
                       out->albedo, out->normal, out->depth, out->diffuse, out->specular,
                       out->variance, out->counts, out->shadow_counts, nullptr, stream, win);
}

namespace mrs {
namespace {

// one job's chunk of samples: samples s0 .. s0 + kk - 1 of every pixel
struct Chunk { int job, s0, kk; int64_t paths; };

mrs_status render_batch_impl(mrs_ctx ctx, const mrs_render_job* jobs, int32_t n_jobs,
                             cudaStream_t st)
{
    MRS_ARG(ctx != nullptr, "ctx is NULL (a batch keeps its path state in a render context)");
    MRS_ARG(jobs != nullptr && n_jobs >= 1 && n_jobs <= 4096, "n_jobs must be in [1, 4096]");
    for (int j = 0; j < n_jobs; ++j) {
        const mrs_render_job& J = jobs[j];
        MRS_ARG(J.scene != nullptr, "job scene is NULL");
        MRS_ARG(J.W >= 1 && J.W <= 16384 && J.H >= 1 && J.H <= 16384, "job W, H must be in [1, 16384]");
        MRS_ARG(J.spp >= 1 && J.spp <= 65536, "job spp must be in [1, 65536]");
        MRS_ARG(J.max_depth >= 0 && J.max_depth <= 32, "job max_depth must be in [0, 32]");
        MRS_ARG(J.grid >= 1 && J.grid <= 64, "job grid must be in [1, 64]");
        MRS_ARG((int64_t)J.W * J.grid <= 65536 && (int64_t)J.H * J.grid <= 65536,
                "job W * grid, H * grid must be <= 65536");
        MRS_ARG(J.radiance != nullptr, "job radiance is NULL");
    }
    const int64_t cap = ctx->wave_paths;
    // chunks: as many samples per pixel as fit the wave (at least one), in
    // sample order; then waves: consecutive chunks up to the capacity (a job
    // never has two chunks in one wave: two would exceed it)
    std::vector<Chunk> chunks;
    int64_t total_px = 0;
    std::vector<int64_t> acc_off(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const int64_t wh = (int64_t)jobs[j].W * jobs[j].H;
        acc_off[j] = total_px;
        total_px += wh;
        int64_t k = cap / wh;
        if (k < 1) k = 1;
        if (k > jobs[j].spp) k = jobs[j].spp;
        MRS_ARG(k * wh <= (int64_t(1) << 31) - 1, "wave too large");
        for (int s0 = 0; s0 < jobs[j].spp; s0 += (int)k) {
            const int kk = (int)((jobs[j].spp - s0) < k ? (jobs[j].spp - s0) : k);
            chunks.push_back({j, s0, kk, kk * wh});
        }
    }
    std::vector<std::pair<size_t, size_t>> waves;   // chunk ranges [a, b)
    int64_t pmax = 0;
    for (size_t a = 0; a < chunks.size();) {
        size_t b = a + 1;
        int64_t n = chunks[a].paths;
        while (b < chunks.size() && (int)(b - a) < kMaxWaveJobs && n + chunks[b].paths <= cap &&
               n + chunks[b].paths <= (int64_t(1) << 31) - 1) {
            n += chunks[b].paths;
            ++b;
        }
        waves.push_back({a, b});
        if (n > pmax) pmax = n;
        a = b;
    }
    // arena: the path arrays of the largest wave, then every job's accumulator
    const int kArrays = 34;
    size_t arr = ((size_t)pmax * 4 + 255) & ~(size_t)255;
    size_t off_acc = arr * kArrays;
    size_t off_cnt = off_acc + (((size_t)total_px * 13 * 4 + 255) & ~(size_t)255);
    mrs_status rc = ctx->arena.ensure(off_cnt + 4 * 2 * 64);
    if (rc != MRS_OK) return rc;
    char* base = ctx->arena.as<char>();
    float* f[kArrays];
    for (int i = 0; i < kArrays; ++i) f[i] = (float*)(base + arr * i);
    PathSoA soa;
    float** fields[] = {&soa.ox, &soa.oy, &soa.oz, &soa.dx, &soa.dy, &soa.dz, &soa.bx, &soa.by,
                        &soa.bz, &soa.Lx, &soa.Ly, &soa.Lz, &soa.pdf_b, &soa.pdf_e, &soa.hit_t,
                        &soa.sdx, &soa.sdy, &soa.sdz, &soa.stmax, &soa.scx, &soa.scy, &soa.scz,
                        &soa.ax, &soa.ay, &soa.az, &soa.nx, &soa.ny, &soa.nz, &soa.dep};
    int fi = 0;
    for (float** fp : fields) *fp = f[fi++];
    soa.hit_id = (int*)f[fi++];
    soa.q0 = (int*)f[fi++];
    soa.q1 = (int*)f[fi++];
    soa.qs = (int*)f[fi++];
    soa.lobe = (int*)f[fi++];
    float* acc = (float*)(base + off_acc);
    uint32_t* cnt = (uint32_t*)(base + off_cnt);
    uint32_t* scnt = cnt + 64;
    MRS_CHECK(cudaMemsetAsync(acc, 0, (size_t)total_px * 13 * 4, st));

    auto job_view = [&](const Chunk& c, int64_t path_off) {
        const mrs_render_job& J = jobs[c.job];
        JobView v;
        memset(&v, 0, sizeof(v));
        v.S = view(J.scene);
        memcpy(v.env, J.scene->env, sizeof(v.env));
        memcpy(v.cam, J.scene->cam, sizeof(v.cam));
        v.W = J.W; v.H = J.H; v.max_depth = J.max_depth;
        v.rr_start = J.rr_start < 0 ? 0x7fffffff : J.rr_start;
        v.win_x0 = 0; v.win_y0 = 0; v.win_w = J.W; v.windowed = false;
        v.grid = J.grid;
        v.s0 = c.s0; v.kk = c.kk;
        v.path_off = (int)path_off; v.n_paths = (int)c.paths;
        v.key = make_uint2((uint32_t)J.seed, (uint32_t)(J.seed >> 32));
        return v;
    };
    const int32_t tail = ctx->tail_bounce;
    const int b_tail = tail >= 0 ? tail : 1;
    for (const auto& wv : waves) {
        JobTable T;
        memset(&T, 0, sizeof(T));
        T.n = (int)(wv.second - wv.first);
        int64_t off = 0;
        int maxd = 0;
        for (size_t c = wv.first; c < wv.second; ++c) {
            T.J[c - wv.first] = job_view(chunks[c], off);
            off += chunks[c].paths;
            maxd = std::max(maxd, jobs[chunks[c].job].max_depth);
        }
        WaveParams w;
        memset(&w, 0, sizeof(w));
        w.J = T.J[0];
        w.P = soa;
        w.layers = 0;
        w.n_paths = (int)off;
        w.cnt = cnt;
        w.scnt = scnt;
        w.stats = nullptr;
        MRS_CHECK(cudaMemsetAsync(cnt, 0, 4 * 2 * 64, st));
        const int g = grid_for(off);
        MRS_TIMED(PK_RAYGEN, st, k_raygen_b<<<g, kThreads, 0, st>>>(w, T));
        MRS_LAUNCHED(1);
        for (int b = 0; b <= maxd && b < b_tail; ++b) {
            MRS_TIMED(PK_TRACE, st, k_trace_b<<<g, kThreads, 0, st>>>(w, T, b));
            MRS_TIMED(PK_SHADE, st, k_shade_b<<<g, kThreads, 0, st>>>(w, T, b));
            MRS_TIMED(PK_SHADOW, st, k_shadow_b<<<g, kThreads, 0, st>>>(w, T, b));
            MRS_LAUNCHED(3);
        }
        if (b_tail <= maxd) {
            MRS_TIMED(PK_TAIL, st, k_tail_b<<<tail_grid_batch(), kThreads, 0, st>>>(w, T, b_tail, maxd));
            MRS_LAUNCHED(1);
        }
        // each chunk's samples into its job's accumulator, in sample order
        for (size_t c = wv.first; c < wv.second; ++c) {
            const Chunk& ch = chunks[c];
            WaveParams wc = w;
            wc.J = T.J[c - wv.first];
            wc.wh = (int64_t)jobs[ch.job].W * jobs[ch.job].H;
            float* a = acc + acc_off[ch.job] * 13;
            const bool v4 = ch.kk % 4 == 0 && wc.J.path_off % 4 == 0;
            if (v4) MRS_TIMED(PK_ACCUM, st, k_accumulate<4><<<grid_for(wc.wh), kThreads, 0, st>>>(wc, a, ch.kk));
            else MRS_TIMED(PK_ACCUM, st, k_accumulate<1><<<grid_for(wc.wh), kThreads, 0, st>>>(wc, a, ch.kk));
            MRS_LAUNCHED(1);
        }
    }
    for (int j = 0; j < n_jobs; ++j) {
        const int64_t wh = (int64_t)jobs[j].W * jobs[j].H;
        k_resolve<<<grid_for(wh), kThreads, 0, st>>>(acc + acc_off[j] * 13, nullptr, wh, jobs[j].spp,
                                                     jobs[j].radiance, jobs[j].albedo, jobs[j].normal,
                                                     jobs[j].depth, nullptr, nullptr, nullptr);
        MRS_LAUNCHED(1);
    }
    return cuda_status(cudaGetLastError(), "batch render launch");
}

}  // namespace
}  // namespace mrs

extern "C" mrs_status mrs_render_batch(mrs_ctx ctx, const mrs_render_job* jobs, int32_t n_jobs,
                                       void* stream)
{
    return render_batch_impl(ctx, jobs, n_jobs, (cudaStream_t)stream);
}

extern "C" mrs_status mrs_render_stats(mrs_scene S, int32_t W, int32_t H, int32_t spp,
                                       int32_t max_depth, int32_t rr_start, uint64_t seed,
                                       float* radiance, uint64_t* stats, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(stats != nullptr, "stats is NULL");
    MRS_CHECK(cudaMemsetAsync(stats, 0, 8 * sizeof(uint64_t), (cudaStream_t)stream));
    return render_impl(S, S->arena, S->wave_paths, S->tail_bounce, W, H, spp, max_depth, rr_start, seed, 1, radiance,
                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                       (unsigned long long*)stats, stream);
}

extern "C" mrs_status mrs_cast(mrs_scene S, const float* orig, const float* dir, int32_t n,
                               int32_t* prim, float* t, void* stream)
{
    MRS_ARG(S != nullptr, "scene is NULL");
    MRS_ARG(n >= 0, "n_rays < 0");
    if (n == 0) return MRS_OK;
    MRS_ARG(orig && dir && prim && t, "NULL buffer");
    k_cast<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(view(S), orig, dir, n, prim, t);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "cast launch");
}

extern "C" mrs_status mrs_philox_uniforms(const uint32_t* triples, int32_t n, uint64_t seed,
                                          float* out, void* stream)
{
    MRS_ARG(n >= 0, "n < 0");
    if (n == 0) return MRS_OK;
    MRS_ARG(triples && out, "NULL buffer");
    k_philox<<<(n + kThreads - 1) / kThreads, kThreads, 0, (cudaStream_t)stream>>>(
        triples, n, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), out);
    MRS_LAUNCHED(1);
    return cuda_status(cudaGetLastError(), "philox launch");
}
