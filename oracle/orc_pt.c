/*
 * CPU oracle for the renderer: Philox4x32-10, Morton codes + binary radix
 * tree (LBVH), closest-hit / any-hit ray casting, and a per-pixel Monte Carlo
 * path tracer that produces the radiance + albedo/normal/depth buffers of the
 * multi-resolution sampling method (LRHS and HRLS renders, Sec. 1 and
 * Sec. 3.2-3.3 of the paper; the paper renders with Blender Cycles, so the
 * integrator below follows the textbook estimator with the free choices fixed
 * in the design notes).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU
 * reference that the CUDA path is checked against.  It shares no code with
 * the CUDA library; only tests, the smoke check and the bench's CPU-baseline
 * leg may load it.  Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 * -ffp-contract=off matters: every float operation below is a single IEEE
 * binary32 operation (+ - * / sqrt are correctly rounded), in the order
 * written, so that the CUDA path can reproduce it bit for bit.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors of Salmon et al.
 * (SC'11); closest hit == brute force on random triangle soups; radix tree
 * invariants; white furnace L = Le * sum_{k<=D} rho^k; diffuse plane under a
 * uniform sky L = rho * L_sky; 1/sqrt(N) error decay with spp.  Materials:
 * the GGX pdf integrates to 1 (quadrature over half vectors), the sampler
 * draws from it (chi-square), its weight is f cos / pdf and its mean the
 * directional albedo, reciprocity, the Fresnel limit of a near mirror.
 * Direct lighting: a Lambertian plane under two quad lights and an
 * environment equals Lambert's closed form (projected solid angles of the
 * quads) with MIS, light sampling alone and BSDF sampling alone, and the
 * three agree on rough GGX planes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Round: multiply words 0 and 2 by the two
 * multipliers, mix high halves with the other words and the key; the key is
 * bumped by the two Weyl constants between rounds.                        */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform float in [0,1): top 24 bits of the word times 2^-24 (exact) */
static float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

/* draw block: counter (pixel, sample, bounce, group), key (seed lo, seed hi).
 * group 0 -> dims 0..3 = bsdf u1, bsdf u2, light u, light v
 * group 1 -> dims 4..7 = light pick, roulette, pixel jitter x, pixel jitter y */
static void draws(uint32_t pixel, uint32_t sample, uint32_t bounce, uint32_t group,
                  const uint32_t key[2], float u[4])
{
    uint32_t c[4] = {pixel, sample, bounce, group}, o[4];
    orc_philox4x32_10(c, key, o);
    for (int i = 0; i < 4; ++i) u[i] = u01(o[i]);
}

void orc_philox_uniforms(uint32_t pixel, uint32_t sample, uint32_t bounce, uint64_t seed,
                         float* out8)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    draws(pixel, sample, bounce, 0, key, out8);
    draws(pixel, sample, bounce, 1, key, out8 + 4);
}

/* ------------------------------------------------------------------------ */
/* small vector algebra; every expression is evaluated left to right        */
/* ------------------------------------------------------------------------ */
typedef struct { float x, y, z; } v3;
static v3 mk(float x, float y, float z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, float s) { return mk(a.x * s, a.y * s, a.z * s); }
static v3 mul(v3 a, v3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
static float dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static v3 normalize(v3 a) { float inv = 1.0f / sqrtf(dot(a, a)); return scl(a, inv); }
/* a + b * s, per component (one multiply, one add) */
static v3 madd(v3 a, v3 b, float s) { return mk(a.x + b.x * s, a.y + b.y * s, a.z + b.z * s); }
static float maxc(v3 a) { return fmaxf(fmaxf(a.x, a.y), a.z); }

#define PI_F 3.14159265358979323846f
#define INV_PI_F 0.318309886183790671538f
#define RAY_EPS 1e-4f
#define SHADOW_FRAC 0.999f
#define T_INF 1e30f

/* cos(2 pi u), sin(2 pi u) for u in [0,1): quadrant from 4u (exact), then
 * Taylor series of cos and sin about 0 on x = f * pi/2 in [0, pi/2), Horner
 * form, truncated after x^14 / x^13 (truncation error < 1e-9). */
static void sincos2pi(float u, float* c, float* s)
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
    switch (q) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
    }
}

void orc_sincos2pi(const float* u, int n, float* c, float* s)
{
    for (int i = 0; i < n; ++i) sincos2pi(u[i], c + i, s + i);
}

/* ------------------------------------------------------------------------ */
/* scene + LBVH                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;                 /* triangles */
    const float* V;        /* [n][3][3] */
    const int32_t* tri_mat;
    const int32_t* tri_light;
    const float* mats;     /* [m][8] */
    const float* lights;   /* [l][12] */
    int n_lights;
    v3 env;
    const float* cam;      /* [12] */
    /* LBVH */
    uint32_t* morton;      /* input order */
    int32_t* order;        /* sorted position -> prim */
    int32_t* left;         /* [n-1] child id: < n-1 internal, else leaf (n-1 + sorted pos) */
    int32_t* right;
    float* box;            /* [(2n-1)][6] lo xyz, hi xyz; node ids as above */
} scene_t;

static v3 vtx(const scene_t* S, int prim, int k)
{
    const float* p = S->V + (size_t)prim * 9 + k * 3;
    return mk(p[0], p[1], p[2]);
}

static uint32_t expand10(uint32_t v)
{
    /* spread the low 10 bits so that bit i lands at bit 3i */
    uint32_t r = 0;
    for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

/* Morton codes of triangle centroids ((v0+v1)+v2) * (1/3) in the centroid
 * bounding box, 10 bits per axis, x in the highest bit of each triple. */
void orc_morton(const float* V, int n, uint32_t* codes)
{
    if (n <= 0) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float* c = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            const float* p = V + (size_t)i * 9;
            float v = ((p[a] + p[3 + a]) + p[6 + a]) * 0.333333343267f;
            c[i * 3 + a] = v;
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    float sc[3];
    for (int a = 0; a < 3; ++a) {
        float ext = hi[a] - lo[a];
        sc[a] = ext > 0.0f ? 1024.0f / ext : 0.0f;
    }
    for (int i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            float f = (c[i * 3 + a] - lo[a]) * sc[a];
            if (!(f > 0.0f)) f = 0.0f;
            uint32_t u = (uint32_t)f;
            q[a] = u > 1023u ? 1023u : u;
        }
        codes[i] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    }
    free(c);
}

static const uint32_t* g_sort_codes;
static int cmp_prim(const void* a, const void* b)
{
    int32_t i = *(const int32_t*)a, j = *(const int32_t*)b;
    uint32_t ci = g_sort_codes[i], cj = g_sort_codes[j];
    if (ci != cj) return ci < cj ? -1 : 1;
    return i < j ? -1 : (i > j);   /* (code, prim) is the 64-bit key */
}

static int clz64(uint64_t x)
{
    int n = 0;
    if (x == 0) return 64;
    while (!(x & 0x8000000000000000ull)) { x <<= 1; ++n; }
    return n;
}

/* Build the binary radix tree over the sorted 64-bit keys (code << 32 | prim)
 * top down: a node covering sorted range [first, last] splits after the last
 * key that shares more than the range's common prefix; the child covering
 * [first, s] is internal node s (or leaf s if first == s), the child covering
 * [s+1, last] is internal node s+1 (or leaf s+1 if s+1 == last).  This is the
 * node numbering of Karras (HPG 2012, "Maximizing parallelism in the
 * construction of BVHs, octrees and k-d trees"): root = 0, every internal node
 * is named after one end of its range.  The tree is unique for unique keys. */
static void build_tree(scene_t* S)
{
    int n = S->n;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    for (int i = 0; i < n; ++i)
        key[i] = ((uint64_t)S->morton[S->order[i]] << 32) | (uint32_t)S->order[i];
    if (n >= 2) {
        int* stk = (int*)malloc(sizeof(int) * 3 * ((size_t)n + 128));
        int sp = 0;
        stk[sp++] = 0; stk[sp++] = 0; stk[sp++] = n - 1;   /* node, first, last */
        while (sp) {
            int last = stk[--sp], first = stk[--sp], node = stk[--sp];
            int common = clz64(key[first] ^ key[last]);
            int s = first;   /* largest index in [first, last-1] sharing > common bits with first */
            for (int k = first; k < last; ++k)
                if (clz64(key[first] ^ key[k]) > common) s = k;
            int L = (s == first) ? (n - 1) + s : s;
            int R = (s + 1 == last) ? (n - 1) + s + 1 : s + 1;
            S->left[node] = L;
            S->right[node] = R;
            if (s != first) { stk[sp++] = s; stk[sp++] = first; stk[sp++] = s; }
            if (s + 1 != last) { stk[sp++] = s + 1; stk[sp++] = s + 1; stk[sp++] = last; }
        }
        free(stk);
    }
    free(key);
    /* leaf boxes, then internal boxes by a post-order walk */
    for (int i = 0; i < n; ++i) {
        float* b = S->box + (size_t)(n - 1 + i) * 6;
        int prim = S->order[i];
        for (int a = 0; a < 3; ++a) {
            float v0 = S->V[(size_t)prim * 9 + a], v1 = S->V[(size_t)prim * 9 + 3 + a],
                  v2 = S->V[(size_t)prim * 9 + 6 + a];
            b[a] = fminf(fminf(v0, v1), v2);
            b[3 + a] = fmaxf(fmaxf(v0, v1), v2);
        }
    }
    if (n >= 2) {
        int* stk = (int*)malloc(sizeof(int) * 6 * ((size_t)n + 128));
        int sp = 0;
        stk[sp++] = 0; stk[sp++] = 0;
        while (sp) {
            int state = stk[--sp], node = stk[--sp];
            if (node >= n - 1) continue;
            if (state == 0) {
                stk[sp++] = node; stk[sp++] = 1;
                stk[sp++] = S->left[node]; stk[sp++] = 0;
                stk[sp++] = S->right[node]; stk[sp++] = 0;
            } else {
                float* b = S->box + (size_t)node * 6;
                const float* l = S->box + (size_t)S->left[node] * 6;
                const float* r = S->box + (size_t)S->right[node] * 6;
                for (int a = 0; a < 3; ++a) {
                    b[a] = fminf(l[a], r[a]);
                    b[3 + a] = fmaxf(l[3 + a], r[3 + a]);
                }
            }
        }
        free(stk);
    }
}

static int scene_init(scene_t* S, const float* V, int n, const int32_t* tri_mat,
                      const int32_t* tri_light, const float* mats, const float* lights,
                      int n_lights, const float* env, const float* cam)
{
    memset(S, 0, sizeof(*S));
    S->n = n; S->V = V; S->tri_mat = tri_mat; S->tri_light = tri_light; S->mats = mats;
    S->lights = lights; S->n_lights = n_lights; S->cam = cam;
    S->env = env ? mk(env[0], env[1], env[2]) : mk(0, 0, 0);
    if (n <= 0) return 0;
    S->morton = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    S->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    S->left = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
    S->right = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
    S->box = (float*)malloc(sizeof(float) * 6 * (size_t)(2 * n - 1));
    if (!S->morton || !S->order || !S->left || !S->right || !S->box) return -1;
    orc_morton(V, n, S->morton);
    for (int i = 0; i < n; ++i) S->order[i] = i;
    g_sort_codes = S->morton;
    qsort(S->order, (size_t)n, sizeof(int32_t), cmp_prim);
    build_tree(S);
    return 0;
}

static void scene_free(scene_t* S)
{
    free(S->morton); free(S->order); free(S->left); free(S->right); free(S->box);
}

/* LBVH export for tests: morton[n] (input order), order[n], left/right[n-1],
 * box[(2n-1)*6].  Returns 0 on success. */
int orc_lbvh(const float* V, int n, uint32_t* morton, int32_t* order, int32_t* left,
             int32_t* right, float* box)
{
    scene_t S;
    if (scene_init(&S, V, n, NULL, NULL, NULL, NULL, 0, NULL, NULL)) { scene_free(&S); return -1; }
    if (n > 0) {
        memcpy(morton, S.morton, sizeof(uint32_t) * (size_t)n);
        memcpy(order, S.order, sizeof(int32_t) * (size_t)n);
        if (n > 1) {
            memcpy(left, S.left, sizeof(int32_t) * (size_t)(n - 1));
            memcpy(right, S.right, sizeof(int32_t) * (size_t)(n - 1));
        }
        memcpy(box, S.box, sizeof(float) * 6 * (size_t)(2 * n - 1));
    }
    scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ray casting                                                               */
/* ------------------------------------------------------------------------ */

/* Moller-Trumbore; returns t in (0, tmax) or -1 */
static float intersect(v3 o, v3 d, v3 v0, v3 e1, v3 e2, float tmax)
{
    v3 p = cross(d, e2);
    float det = dot(e1, p);
    if (det == 0.0f) return -1.0f;
    float inv = 1.0f / det;
    v3 s = sub(o, v0);
    float u = dot(s, p) * inv;
    if (u < 0.0f || u > 1.0f) return -1.0f;
    v3 q = cross(s, e1);
    float v = dot(d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return -1.0f;
    float t = dot(e2, q) * inv;
    if (!(t > 0.0f) || !(t < tmax)) return -1.0f;
    return t;
}

static float tri_hit(const scene_t* S, int prim, v3 o, v3 d, float tmax)
{
    v3 v0 = vtx(S, prim, 0);
    return intersect(o, d, v0, sub(vtx(S, prim, 1), v0), sub(vtx(S, prim, 2), v0), tmax);
}

/* conservative slab test (far distance widened by 4 ulp) */
static int box_hit(const float* b, v3 o, v3 inv, float tmax)
{
    float t0x = (b[0] - o.x) * inv.x, t1x = (b[3] - o.x) * inv.x;
    float t0y = (b[1] - o.y) * inv.y, t1y = (b[4] - o.y) * inv.y;
    float t0z = (b[2] - o.z) * inv.z, t1z = (b[5] - o.z) * inv.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    return tn <= tf * 1.0000005f;
}

/* closest hit: smallest t, ties to the smaller triangle index */
static int closest(const scene_t* S, v3 o, v3 d, float* t_out)
{
    int n = S->n, best = -1;
    float bt = T_INF;
    if (n == 0) return -1;
    if (n == 1) {
        float t = tri_hit(S, 0, o, d, T_INF);
        if (t > 0.0f) { *t_out = t; return 0; }
        return -1;
    }
    v3 inv = mk(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int stk[128];
    int sp = 0;
    stk[sp++] = 0;
    while (sp) {
        int node = stk[--sp];
        if (!box_hit(S->box + (size_t)node * 6, o, inv, bt)) continue;
        if (node >= n - 1) {
            int prim = S->order[node - (n - 1)];
            float t = tri_hit(S, prim, o, d, T_INF);
            if (t > 0.0f && (t < bt || (t == bt && prim < best))) { bt = t; best = prim; }
        } else {
            stk[sp++] = S->right[node];
            stk[sp++] = S->left[node];
        }
    }
    if (best >= 0) *t_out = bt;
    return best;
}

static int occluded(const scene_t* S, v3 o, v3 d, float tmax)
{
    int n = S->n;
    if (n == 0) return 0;
    if (n == 1) return tri_hit(S, 0, o, d, tmax) > 0.0f;
    v3 inv = mk(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int stk[128];
    int sp = 0;
    stk[sp++] = 0;
    while (sp) {
        int node = stk[--sp];
        if (!box_hit(S->box + (size_t)node * 6, o, inv, tmax)) continue;
        if (node >= n - 1) {
            if (tri_hit(S, S->order[node - (n - 1)], o, d, tmax) > 0.0f) return 1;
        } else {
            stk[sp++] = S->right[node];
            stk[sp++] = S->left[node];
        }
    }
    return 0;
}

/* batch ray casts for tests: prim_out[i] = closest prim or -1, t_out[i] */
int orc_cast(const float* V, int n, const float* orig, const float* dir, int nr, int brute,
             int32_t* prim_out, float* t_out)
{
    scene_t S;
    if (!brute && scene_init(&S, V, n, NULL, NULL, NULL, NULL, 0, NULL, NULL)) { scene_free(&S); return -1; }
    for (int r = 0; r < nr; ++r) {
        v3 o = mk(orig[3 * r], orig[3 * r + 1], orig[3 * r + 2]);
        v3 d = mk(dir[3 * r], dir[3 * r + 1], dir[3 * r + 2]);
        int best = -1;
        float bt = T_INF;
        if (brute) {
            S.n = n; S.V = V;
            for (int p = 0; p < n; ++p) {
                float t = tri_hit(&S, p, o, d, T_INF);
                if (t > 0.0f && (t < bt || (t == bt && p < best))) { bt = t; best = p; }
            }
        } else {
            best = closest(&S, o, d, &bt);
        }
        prim_out[r] = best;
        t_out[r] = best >= 0 ? bt : -1.0f;
    }
    if (!brute) scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* materials                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { int type; v3 albedo; float alpha; v3 Le; } mat_t;

static mat_t material(const scene_t* S, int prim)
{
    const float* m = S->mats + (size_t)S->tri_mat[prim] * 8;
    mat_t r;
    r.type = (int)m[0];
    r.albedo = mk(m[1], m[2], m[3]);
    r.alpha = m[4];
    r.Le = mk(m[5], m[6], m[7]);
    return r;
}

/* orthonormal basis around unit n (Duff et al., JCGT 2017) */
static void basis(v3 n, v3* t, v3* b)
{
    float sign = copysignf(1.0f, n.z);
    float a = -1.0f / (sign + n.z);
    float bb = n.x * n.y * a;
    *t = mk(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    *b = mk(bb, sign + n.y * n.y * a, -n.y);
}

static v3 to_local(v3 w, v3 t, v3 b, v3 n) { return mk(dot(w, t), dot(w, b), dot(w, n)); }
static v3 to_world(v3 w, v3 t, v3 b, v3 n)
{
    return mk(t.x * w.x + b.x * w.y + n.x * w.z, t.y * w.x + b.y * w.y + n.y * w.z,
              t.z * w.x + b.z * w.y + n.z * w.z);
}

static v3 cosine_sample(float u1, float u2)
{
    float r = sqrtf(u1), c, s;
    sincos2pi(u2, &c, &s);
    return mk(r * c, r * s, sqrtf(fmaxf(0.0f, 1.0f - u1)));
}

/* Smith height-correlated Lambda for GGX: (sqrt(1 + a^2 tan^2) - 1) / 2 */
static float ggx_lambda(v3 w, float a2)
{
    float tan2 = (w.x * w.x + w.y * w.y) / (w.z * w.z);
    return (sqrtf(1.0f + a2 * tan2) - 1.0f) * 0.5f;
}

static float ggx_D(float hz, float a2)
{
    float den = hz * hz * (a2 - 1.0f) + 1.0f;
    return a2 / (PI_F * den * den);
}

static v3 schlick(v3 F0, float cosh)
{
    float m = fmaxf(0.0f, 1.0f - cosh);
    float m2 = m * m;
    float m5 = m2 * m2 * m;
    return mk(F0.x + (1.0f - F0.x) * m5, F0.y + (1.0f - F0.y) * m5, F0.z + (1.0f - F0.z) * m5);
}

/* BSDF value f (without cosine) and sampling pdf for local wo, wi (z > 0) */
static v3 bsdf_eval(const mat_t* m, v3 wo, v3 wi, float* pdf)
{
    if (m->type == 0) {
        *pdf = wi.z * INV_PI_F;
        return scl(m->albedo, INV_PI_F);
    }
    float a2 = m->alpha * m->alpha;
    v3 h = normalize(add(wo, wi));
    float D = ggx_D(h.z, a2);
    float lo = ggx_lambda(wo, a2), li = ggx_lambda(wi, a2);
    float G1 = 1.0f / (1.0f + lo);
    float G2 = 1.0f / ((1.0f + lo) + li);
    v3 F = schlick(m->albedo, dot(wo, h));
    float k = (D * G2) / ((4.0f * wo.z) * wi.z);
    *pdf = (G1 * D) / (4.0f * wo.z);
    return scl(F, k);
}

/* sample wi; returns 0 if the sample is below the surface.  weight = f cos / pdf */
static int bsdf_sample(const mat_t* m, v3 wo, float u1, float u2, v3* wi, v3* weight, float* pdf)
{
    if (m->type == 0) {
        *wi = cosine_sample(u1, u2);
        if (!(wi->z > 0.0f)) return 0;
        *pdf = wi->z * INV_PI_F;
        *weight = m->albedo;
        return 1;
    }
    /* GGX visible-normal sampling (Heitz, JCGT 2018) */
    float al = m->alpha, a2 = al * al;
    v3 Vh = normalize(mk(al * wo.x, al * wo.y, wo.z));
    float lensq = Vh.x * Vh.x + Vh.y * Vh.y;
    v3 T1 = mk(1.0f, 0.0f, 0.0f);
    if (lensq > 0.0f) { float il = 1.0f / sqrtf(lensq); T1 = mk(-Vh.y * il, Vh.x * il, 0.0f); }
    v3 T2 = cross(Vh, T1);
    float r = sqrtf(u1), c, s;
    sincos2pi(u2, &c, &s);
    float t1 = r * c, t2 = r * s;
    float sv = 0.5f * (1.0f + Vh.z);
    t2 = (1.0f - sv) * sqrtf(1.0f - t1 * t1) + sv * t2;
    float q = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
    v3 Nh = mk(T1.x * t1 + T2.x * t2 + Vh.x * q, T1.y * t1 + T2.y * t2 + Vh.y * q,
               T1.z * t1 + T2.z * t2 + Vh.z * q);
    v3 h = normalize(mk(al * Nh.x, al * Nh.y, fmaxf(0.0f, Nh.z)));
    float k = 2.0f * dot(wo, h);
    *wi = mk(k * h.x - wo.x, k * h.y - wo.y, k * h.z - wo.z);
    if (!(wi->z > 0.0f)) return 0;
    float lo = ggx_lambda(wo, a2), li = ggx_lambda(*wi, a2);
    float g = (1.0f + lo) / ((1.0f + lo) + li);   /* G2 / G1(wo) */
    v3 F = schlick(m->albedo, dot(wo, h));
    *weight = scl(F, g);
    float D = ggx_D(h.z, a2);
    *pdf = ((1.0f / (1.0f + lo)) * D) / (4.0f * wo.z);
    return 1;
}

/* Test hooks: the BSDF of one material (a row of the scene's material table:
 * type, albedo rgb, alpha, Le rgb) over n pairs of local directions (shading
 * normal = +z).  eval: f (without the cosine) and the sampling pdf of wi;
 * sample: wi, weight = f cos / pdf, pdf and ok (0 = sample below the surface,
 * then the other outputs are 0) for uniforms u [n][2]. */
void orc_bsdf_eval_batch(const float* mat8, const float* wo, const float* wi, int n, float* f,
                         float* pdf)
{
    mat_t m;
    m.type = (int)mat8[0];
    m.albedo = mk(mat8[1], mat8[2], mat8[3]);
    m.alpha = mat8[4];
    m.Le = mk(mat8[5], mat8[6], mat8[7]);
    for (int i = 0; i < n; ++i) {
        v3 o = mk(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]);
        v3 w = mk(wi[3 * i], wi[3 * i + 1], wi[3 * i + 2]);
        v3 r = bsdf_eval(&m, o, w, pdf + i);
        f[3 * i] = r.x; f[3 * i + 1] = r.y; f[3 * i + 2] = r.z;
    }
}

void orc_bsdf_sample_batch(const float* mat8, const float* wo, const float* u, int n, float* wi,
                           float* weight, float* pdf, int32_t* ok)
{
    mat_t m;
    m.type = (int)mat8[0];
    m.albedo = mk(mat8[1], mat8[2], mat8[3]);
    m.alpha = mat8[4];
    m.Le = mk(mat8[5], mat8[6], mat8[7]);
    for (int i = 0; i < n; ++i) {
        v3 o = mk(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]);
        v3 w = mk(0, 0, 0), wt = mk(0, 0, 0);
        float p = 0.0f;
        ok[i] = bsdf_sample(&m, o, u[2 * i], u[2 * i + 1], &w, &wt, &p);
        if (!ok[i]) { w = mk(0, 0, 0); wt = mk(0, 0, 0); p = 0.0f; }
        wi[3 * i] = w.x; wi[3 * i + 1] = w.y; wi[3 * i + 2] = w.z;
        weight[3 * i] = wt.x; weight[3 * i + 1] = wt.y; weight[3 * i + 2] = wt.z;
        pdf[i] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* the path tracer                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int W, H, spp, max_depth, rr_start;
    int grid;   /* camera sampling grid: 1 = whole pixel footprint */
    uint32_t key[2];
    int estimator;   /* ORC_EST_* below */
} rparams_t;

/* Direct-lighting estimator.  ORC_EST_MIS is the renderer's: next-event
 * estimation and BSDF sampling combined by the power heuristic.  The two
 * single-technique estimators exist only to test that combination: with
 * ORC_EST_LIGHT every light and the environment are reached only through
 * next-event estimation (weight 1; BSDF-sampled hits on them add nothing),
 * with ORC_EST_BSDF only through BSDF sampling (no shadow rays; weight 1).
 * All three are unbiased for the same integral, so their means must agree;
 * a light pdf, an MIS weight or a BSDF pdf that is wrong breaks that. */
#define ORC_EST_MIS 0
#define ORC_EST_LIGHT 1
#define ORC_EST_BSDF 2
static int g_estimator = ORC_EST_MIS;

void orc_set_estimator(int mode) { g_estimator = mode; }

/* one path; returns radiance, writes first-hit aux (albedo, shading normal,
   depth, lobe = 1 Lambertian / 2 GGX / 0 no hit), counts rays per bounce */
static v3 trace_path(const scene_t* S, const rparams_t* P, int px, int py, int sample,
                     v3* alb, v3* nrm, float* depth, int* lobe, uint64_t* counts,
                     uint64_t* shadow_counts)
{
    uint32_t pixel = (uint32_t)(py * P->W + px);
    float g1[4];
    draws(pixel, (uint32_t)sample, 0u, 1u, P->key, g1);
    const float* cam = S->cam;
    v3 eye = mk(cam[0], cam[1], cam[2]), fwd = mk(cam[3], cam[4], cam[5]);
    v3 rgt = mk(cam[6], cam[7], cam[8]), up = mk(cam[9], cam[10], cam[11]);
    /* grid g > 1: the pixel stands for a g x g block of a g-times finer image
       and its samples cover only that block's sub-pixel (g*px + g/2,
       g*py + g/2): nearest-neighbour downsampling of the finer image, the
       low-resolution renders of Sec. 3, "Low Resolution Image Generation"
       (rays of the low-resolution image on a sparse grid).  g = 1
       is the ordinary box footprint of the pixel. */
    const int g = P->grid;
    float sx = ((float)(px * g + g / 2) + g1[2]) / (float)(P->W * g);
    float sy = ((float)(py * g + g / 2) + g1[3]) / (float)(P->H * g);
    float a = 2.0f * sx - 1.0f, bq = 1.0f - 2.0f * sy;
    v3 o = eye;
    v3 d = normalize(mk(fwd.x + rgt.x * a + up.x * bq, fwd.y + rgt.y * a + up.y * bq,
                        fwd.z + rgt.z * a + up.z * bq));
    v3 beta = mk(1.0f, 1.0f, 1.0f), L = mk(0.0f, 0.0f, 0.0f);
    float pdf_b = 0.0f, pdf_e = 0.0f;
    int env_on = S->env.x > 0.0f || S->env.y > 0.0f || S->env.z > 0.0f;
    int n_choices = S->n_lights + (env_on ? 1 : 0);
    float pick = n_choices > 0 ? 1.0f / (float)n_choices : 0.0f;
    *alb = mk(0, 0, 0); *nrm = mk(0, 0, 0); *depth = 0.0f; *lobe = 0;

    for (int b = 0; b <= P->max_depth; ++b) {
        counts[b] += 1;
        float t;
        int prim = closest(S, o, d, &t);
        if (prim < 0) {
            if (env_on) {
                float w = 1.0f;
                if (b > 0 && P->estimator == ORC_EST_LIGHT) w = 0.0f;
                else if (b > 0 && P->estimator == ORC_EST_MIS && pdf_e > 0.0f)
                    w = (pdf_b * pdf_b) / (pdf_b * pdf_b + pdf_e * pdf_e);
                L = mk(L.x + beta.x * S->env.x * w, L.y + beta.y * S->env.y * w,
                       L.z + beta.z * S->env.z * w);
            }
            break;
        }
        v3 p = madd(o, d, t);
        v3 v0 = vtx(S, prim, 0);
        v3 ng = normalize(cross(sub(vtx(S, prim, 1), v0), sub(vtx(S, prim, 2), v0)));
        float cos_o = dot(d, ng);
        v3 ns = cos_o > 0.0f ? scl(ng, -1.0f) : ng;
        mat_t m = material(S, prim);
        if (b == 0) { *alb = m.albedo; *nrm = ns; *depth = t; *lobe = m.type == 0 ? 1 : 2; }
        if ((m.Le.x > 0.0f || m.Le.y > 0.0f || m.Le.z > 0.0f) && cos_o < 0.0f) {
            float w = 1.0f;
            int li = S->tri_light[prim];
            if (b > 0 && li >= 0 && P->estimator == ORC_EST_LIGHT) {
                w = 0.0f;
            } else if (b > 0 && li >= 0 && P->estimator == ORC_EST_MIS) {
                const float* lq = S->lights + (size_t)li * 12;
                v3 ln = cross(mk(lq[3], lq[4], lq[5]), mk(lq[6], lq[7], lq[8]));
                float area = sqrtf(dot(ln, ln));
                float pl = pick * (t * t) / (-cos_o * area);
                w = (pdf_b * pdf_b) / (pdf_b * pdf_b + pl * pl);
            }
            L = mk(L.x + beta.x * m.Le.x * w, L.y + beta.y * m.Le.y * w, L.z + beta.z * m.Le.z * w);
        }
        if (b == P->max_depth) break;
        if (!(m.albedo.x > 0.0f || m.albedo.y > 0.0f || m.albedo.z > 0.0f)) break;

        float g0[4];
        draws(pixel, (uint32_t)sample, (uint32_t)b, 0u, P->key, g0);
        if (b > 0) draws(pixel, (uint32_t)sample, (uint32_t)b, 1u, P->key, g1);
        v3 T, B;
        basis(ns, &T, &B);
        v3 wo = to_local(scl(d, -1.0f), T, B, ns);
        v3 org = madd(p, ns, RAY_EPS);

        /* next-event estimation: one light (or the environment), power-heuristic MIS */
        if (n_choices > 0 && P->estimator != ORC_EST_BSDF) {
            int k = (int)(g1[0] * (float)n_choices);
            if (k > n_choices - 1) k = n_choices - 1;
            if (k < S->n_lights) {
                const float* lq = S->lights + (size_t)k * 12;
                v3 p0 = mk(lq[0], lq[1], lq[2]), e1 = mk(lq[3], lq[4], lq[5]);
                v3 e2 = mk(lq[6], lq[7], lq[8]), Le = mk(lq[9], lq[10], lq[11]);
                v3 x = madd(madd(p0, e1, g0[2]), e2, g0[3]);
                v3 ln = cross(e1, e2);
                float area = sqrtf(dot(ln, ln));
                v3 nl = scl(ln, 1.0f / area);
                v3 dl = sub(x, org);
                float d2 = dot(dl, dl);
                float dist = sqrtf(d2);
                v3 wi = scl(dl, 1.0f / dist);
                float cos_l = -dot(wi, nl), cos_s = dot(wi, ns);
                if (cos_l > 0.0f && cos_s > 0.0f) {
                    float pb;
                    v3 f = bsdf_eval(&m, wo, to_local(wi, T, B, ns), &pb);
                    float pl = pick * d2 / (cos_l * area);
                    float w = P->estimator == ORC_EST_LIGHT ? 1.0f : (pl * pl) / (pl * pl + pb * pb);
                    float sc = (cos_s / pl) * w;
                    v3 c = mk(beta.x * f.x * Le.x * sc, beta.y * f.y * Le.y * sc,
                              beta.z * f.z * Le.z * sc);
                    shadow_counts[b] += 1;
                    if (!occluded(S, org, wi, dist * SHADOW_FRAC)) L = add(L, c);
                }
            } else {
                v3 wl = cosine_sample(g0[2], g0[3]);
                if (wl.z > 0.0f) {
                    v3 wi = normalize(to_world(wl, T, B, ns));
                    float pb;
                    v3 f = bsdf_eval(&m, wo, wl, &pb);
                    float pe = pick * wl.z * INV_PI_F;
                    float w = P->estimator == ORC_EST_LIGHT ? 1.0f : (pe * pe) / (pe * pe + pb * pb);
                    float sc = (wl.z / pe) * w;
                    v3 c = mk(beta.x * f.x * S->env.x * sc, beta.y * f.y * S->env.y * sc,
                              beta.z * f.z * S->env.z * sc);
                    shadow_counts[b] += 1;
                    if (!occluded(S, org, wi, T_INF)) L = add(L, c);
                }
            }
        }

        /* continue the path by BSDF sampling */
        v3 wl, wt;
        float pb;
        if (!bsdf_sample(&m, wo, g0[0], g0[1], &wl, &wt, &pb)) break;
        beta = mul(beta, wt);
        pdf_b = pb;
        pdf_e = env_on ? pick * wl.z * INV_PI_F : 0.0f;
        if (!(maxc(beta) > 0.0f)) break;
        if (b >= P->rr_start) {
            float q = fminf(0.95f, maxc(beta));
            if (g1[1] >= q) break;
            beta = mk(beta.x / q, beta.y / q, beta.z / q);
        }
        o = org;
        d = normalize(to_world(wl, T, B, ns));
    }
    return L;
}

/*
 * Render W x H at spp samples per pixel.  Per pixel, samples are accumulated
 * in sample order with Kahan-compensated float sums; radiance = sum / spp.
 * Aux buffers (albedo, facing normal, depth of the first hit; zero on a miss)
 * are plain float sums in sample order divided by spp.  counts[b] /
 * shadow_counts[b] (max_depth+1 entries each, may be NULL) receive the number
 * of extension / shadow rays cast at bounce b.  Only rows row0, row0 +
 * row_step, ... below row1 are rendered (output row i = image row row0 + i
 * row_step): a bounded sample for timing.  threads <= 0 -> all cores.
 */
int orc_render(const float* V, int n, const int32_t* tri_mat, const int32_t* tri_light,
               const float* mats, const float* lights, int n_lights, const float* env,
               const float* cam, int W, int H, int spp, int max_depth, int rr_start,
               int grid, uint64_t seed, int row0, int row1, int row_step, int threads,
               float* radiance, float* albedo, float* normal, float* depth,
               float* diffuse, float* specular, float* variance,
               uint64_t* counts, uint64_t* shadow_counts)
{
    if (W <= 0 || H <= 0 || spp <= 0 || max_depth < 0 || max_depth > 62) return -1;
    if (grid < 1 || grid > 64) return -1;
    if (row1 <= 0 || row1 > H) row1 = H;
    if (row0 < 0) row0 = 0;
    if (row_step < 1) row_step = 1;
    const int nrows = row1 > row0 ? (row1 - row0 + row_step - 1) / row_step : 0;
    scene_t S;
    if (scene_init(&S, V, n, tri_mat, tri_light, mats, lights, n_lights, env, cam)) {
        scene_free(&S);
        return -2;
    }
    rparams_t P = {W, H, spp, max_depth, rr_start, grid, {(uint32_t)seed, (uint32_t)(seed >> 32)},
                   g_estimator};
    int nb = max_depth + 1;
    uint64_t tot[64] = {0}, stot[64] = {0};
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        uint64_t cnt[64] = {0}, scnt[64] = {0};
#pragma omp for schedule(dynamic, 1)
        for (int ri = 0; ri < nrows; ++ri) {
            const int py = row0 + ri * row_step;
            for (int px = 0; px < W; ++px) {
                float s0 = 0, s1 = 0, s2 = 0, c0 = 0, c1 = 0, c2 = 0;
                v3 as = mk(0, 0, 0), ns = mk(0, 0, 0);
                v3 dsum = mk(0, 0, 0), ssum = mk(0, 0, 0), q = mk(0, 0, 0);
                float ds = 0;
                for (int s = 0; s < spp; ++s) {
                    v3 a, nn;
                    float dd;
                    int lobe;
                    v3 Ls = trace_path(&S, &P, px, py, s, &a, &nn, &dd, &lobe, cnt, scnt);
                    /* extra layers (Sec. 4: diffuse, specular, variance) in
                       sample order: the sample's radiance goes to the layer of
                       its first hit's lobe; q sums squares for the variance */
                    v3 zero = mk(0, 0, 0);
                    dsum = add(dsum, lobe == 1 ? Ls : zero);
                    ssum = add(ssum, lobe == 2 ? Ls : zero);
                    q = add(q, mul(Ls, Ls));
                    /* Kahan: y = x - c; t = s + y; c = (t - s) - y; s = t */
                    float y, t;
                    y = Ls.x - c0; t = s0 + y; c0 = (t - s0) - y; s0 = t;
                    y = Ls.y - c1; t = s1 + y; c1 = (t - s1) - y; s1 = t;
                    y = Ls.z - c2; t = s2 + y; c2 = (t - s2) - y; s2 = t;
                    as = add(as, a);
                    ns = add(ns, nn);
                    ds = ds + dd;
                }
                size_t i = (size_t)ri * W + px;
                float fs = (float)spp;
                if (radiance) { radiance[3 * i] = s0 / fs; radiance[3 * i + 1] = s1 / fs; radiance[3 * i + 2] = s2 / fs; }
                if (albedo) { albedo[3 * i] = as.x / fs; albedo[3 * i + 1] = as.y / fs; albedo[3 * i + 2] = as.z / fs; }
                if (normal) { normal[3 * i] = ns.x / fs; normal[3 * i + 1] = ns.y / fs; normal[3 * i + 2] = ns.z / fs; }
                if (depth) depth[i] = ds / fs;
                if (diffuse) { diffuse[3 * i] = dsum.x / fs; diffuse[3 * i + 1] = dsum.y / fs; diffuse[3 * i + 2] = dsum.z / fs; }
                if (specular) { specular[3 * i] = ssum.x / fs; specular[3 * i + 1] = ssum.y / fs; specular[3 * i + 2] = ssum.z / fs; }
                if (variance) {
                    /* sample variance of the pixel mean, per channel:
                       (sum L^2 - (sum L)^2 / N) / (N (N - 1)), 0 for N = 1,
                       floored at 0 (rounding) */
                    float m[3] = {s0, s1, s2}, qq[3] = {q.x, q.y, q.z};
                    for (int c = 0; c < 3; ++c) {
                        float v = 0.0f;
                        if (spp > 1) {
                            v = (qq[c] - m[c] * m[c] / fs) / (fs * (fs - 1.0f));
                            if (!(v > 0.0f)) v = 0.0f;
                        }
                        variance[3 * i + c] = v;
                    }
                }
            }
        }
#pragma omp critical
        for (int b = 0; b < nb; ++b) { tot[b] += cnt[b]; stot[b] += scnt[b]; }
    }
    if (counts) for (int b = 0; b < nb; ++b) counts[b] = tot[b];
    if (shadow_counts) for (int b = 0; b < nb; ++b) shadow_counts[b] = stot[b];
    scene_free(&S);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
