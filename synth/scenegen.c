/*
 * Seeded synthetic scenes (see scenegen.h): the Cornell box of the small
 * path-tracing workload and the procedural field of noise-displaced
 * icospheres of the large ones.  The paper renders Blender scenes (Sec. 3.1);
 * these procedural stand-ins replace its dataset.
 *
 * Random numbers: one splitmix64 stream (Steele, Lea, Flood, OOPSLA 2014)
 * per scene, seeded from the scene seed; uniforms in [0, 1) are its top 53
 * bits times 2^-53.  Geometry is built in double precision and rounded once
 * to float.
 */
#include "scenegen.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double x, y, z; } d3;
static d3 mk(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 scl(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 cross(d3 a, d3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static d3 normalize(d3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }

/* ---- random numbers ------------------------------------------------------ */
typedef struct { uint64_t s; } rng_t;

static uint64_t next64(rng_t* r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double u01(rng_t* r) { return (double)(next64(r) >> 11) * (1.0 / 9007199254740992.0); }
static double uniform(rng_t* r, double a, double b) { return a + (b - a) * u01(r); }

/* ---- icospheres ---------------------------------------------------------- */
typedef struct { int nv, nf; double* v; int* f; } mesh_t;

static void mesh_free(mesh_t* m)
{
    free(m->v);
    free(m->f);
    m->v = NULL;
    m->f = NULL;
}

/* edge -> midpoint vertex, open addressing over keys (lo << 32 | hi) + 1 */
typedef struct { uint64_t* key; int* val; uint64_t mask; } edge_map_t;

static int midpoint(edge_map_t* em, mesh_t* m, int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    uint64_t k = (((uint64_t)lo << 32) | (uint64_t)hi) + 1;
    uint64_t h = (k * 0x9E3779B97F4A7C15ull) >> 20;
    for (;; ++h) {
        uint64_t i = h & em->mask;
        if (em->key[i] == k) return em->val[i];
        if (em->key[i] == 0) {
            d3 va = mk(m->v[3 * a], m->v[3 * a + 1], m->v[3 * a + 2]);
            d3 vb = mk(m->v[3 * b], m->v[3 * b + 1], m->v[3 * b + 2]);
            d3 p = normalize(scl(add(va, vb), 0.5));
            int id = m->nv++;
            m->v[3 * id] = p.x; m->v[3 * id + 1] = p.y; m->v[3 * id + 2] = p.z;
            em->key[i] = k;
            em->val[i] = id;
            return id;
        }
    }
}

/* unit icosphere with 20 * 4^subdiv outward-wound faces: the icosahedron,
 * then `subdiv` times every face split into four at its edge midpoints
 * (pushed out to the sphere) */
static int icosphere(int subdiv, mesh_t* m)
{
    static const int F0[20][3] = {
        {0, 11, 5}, {0, 5, 1}, {0, 1, 7}, {0, 7, 10}, {0, 10, 11},
        {1, 5, 9}, {5, 11, 4}, {11, 10, 2}, {10, 7, 6}, {7, 1, 8},
        {3, 9, 4}, {3, 4, 2}, {3, 2, 6}, {3, 6, 8}, {3, 8, 9},
        {4, 9, 5}, {2, 4, 11}, {6, 2, 10}, {8, 6, 7}, {9, 8, 1},
    };
    const double t = (1.0 + sqrt(5.0)) / 2.0;
    const double V0[12][3] = {
        {-1, t, 0}, {1, t, 0}, {-1, -t, 0}, {1, -t, 0}, {0, -1, t}, {0, 1, t},
        {0, -1, -t}, {0, 1, -t}, {t, 0, -1}, {t, 0, 1}, {-t, 0, -1}, {-t, 0, 1},
    };
    int nf_final = 20, nv_final = 12;
    for (int s = 0; s < subdiv; ++s) { nv_final += 3 * nf_final / 2; nf_final *= 4; }
    m->v = (double*)malloc(sizeof(double) * 3 * (size_t)nv_final);
    m->f = (int*)malloc(sizeof(int) * 3 * (size_t)nf_final);
    int* tmp = (int*)malloc(sizeof(int) * 3 * (size_t)nf_final);
    uint64_t cap = 1;
    while (cap < (uint64_t)(3 * nf_final)) cap <<= 1;
    edge_map_t em = {(uint64_t*)malloc(sizeof(uint64_t) * cap), (int*)malloc(sizeof(int) * cap),
                     cap - 1};
    if (!m->v || !m->f || !tmp || !em.key || !em.val) {
        free(tmp); free(em.key); free(em.val); mesh_free(m);
        return -1;
    }
    m->nv = 12;
    m->nf = 20;
    for (int i = 0; i < 12; ++i) {
        d3 p = normalize(mk(V0[i][0], V0[i][1], V0[i][2]));
        m->v[3 * i] = p.x; m->v[3 * i + 1] = p.y; m->v[3 * i + 2] = p.z;
    }
    memcpy(m->f, F0, sizeof(F0));
    for (int s = 0; s < subdiv; ++s) {
        memset(em.key, 0, sizeof(uint64_t) * cap);
        int nf = 0;
        for (int j = 0; j < m->nf; ++j) {
            int a = m->f[3 * j], b = m->f[3 * j + 1], c = m->f[3 * j + 2];
            int ab = midpoint(&em, m, a, b), bc = midpoint(&em, m, b, c), ca = midpoint(&em, m, c, a);
            int q[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
            memcpy(tmp + 3 * nf, q, sizeof(q));
            nf += 4;
        }
        memcpy(m->f, tmp, sizeof(int) * 3 * (size_t)nf);
        m->nf = nf;
    }
    free(tmp); free(em.key); free(em.val);
    return 0;
}

/* ---- value noise --------------------------------------------------------- */
/* integer lattice hash -> [0, 1) (splitmix-style finaliser) */
static double hash3(int64_t ix, int64_t iy, int64_t iz, uint64_t salt)
{
    uint64_t h = ((uint64_t)ix * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)iy * 0xC2B2AE3D27D4EB4Full) ^
                 ((uint64_t)iz * 0x165667B19E3779F9ull) ^ (salt * 0xD6E8FEB86659FD93ull);
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 32;
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

/* trilinear value noise in [0, 1] with the smoothstep fade f^2 (3 - 2 f) */
static double value_noise(d3 p, uint64_t salt)
{
    double fl[3] = {floor(p.x), floor(p.y), floor(p.z)};
    double f[3] = {p.x - fl[0], p.y - fl[1], p.z - fl[2]};
    int64_t i[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        i[a] = (int64_t)fl[a] + (1 << 20);
        w[a] = f[a] * f[a] * (3.0 - 2.0 * f[a]);
    }
    double acc = 0.0;
    for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
            for (int dz = 0; dz < 2; ++dz) {
                double h = hash3(i[0] + dx, i[1] + dy, i[2] + dz, salt);
                double wx = dx ? w[0] : 1.0 - w[0];
                double wy = dy ? w[1] : 1.0 - w[1];
                double wz = dz ? w[2] : 1.0 - w[2];
                acc += h * wx * wy * wz;
            }
    return acc;
}

/* ---- scene builder ------------------------------------------------------- */
typedef struct {
    float* V; int32_t* tri_mat; int32_t* tri_light; float* mats; float* lights;
    int nt, nm, nl;
} builder_t;

static void put_tri(builder_t* b, d3 p0, d3 p1, d3 p2, int mat, int light)
{
    float* v = b->V + 9 * (size_t)b->nt;
    d3 p[3] = {p0, p1, p2};
    for (int k = 0; k < 3; ++k) {
        v[3 * k] = (float)p[k].x; v[3 * k + 1] = (float)p[k].y; v[3 * k + 2] = (float)p[k].z;
    }
    b->tri_mat[b->nt] = mat;
    b->tri_light[b->nt] = light;
    b->nt++;
}

static int material(builder_t* b, int kind, d3 albedo, double alpha, d3 Le)
{
    float* m = b->mats + 8 * (size_t)b->nm;
    m[0] = (float)kind;
    m[1] = (float)albedo.x; m[2] = (float)albedo.y; m[3] = (float)albedo.z;
    m[4] = (float)alpha;
    m[5] = (float)Le.x; m[6] = (float)Le.y; m[7] = (float)Le.z;
    return b->nm++;
}

/* two triangles covering p0 + [0,1] e1 + [0,1] e2, geometric normal along
 * cross(e1, e2) */
static void quad(builder_t* b, d3 p0, d3 e1, d3 e2, int mat, int light)
{
    d3 a = p0, c1 = add(p0, e1), c2 = add(add(p0, e1), e2), d = add(p0, e2);
    put_tri(b, a, c1, c2, mat, light);
    put_tri(b, a, c2, d, mat, light);
}

static void quad_light(builder_t* b, d3 p0, d3 e1, d3 e2, d3 Le)
{
    int li = b->nl++;
    float* l = b->lights + 12 * (size_t)li;
    d3 q[4] = {p0, e1, e2, Le};
    for (int k = 0; k < 4; ++k) {
        l[3 * k] = (float)q[k].x; l[3 * k + 1] = (float)q[k].y; l[3 * k + 2] = (float)q[k].z;
    }
    int m = material(b, 0, mk(0, 0, 0), 1.0, Le);
    quad(b, p0, e1, e2, m, li);
}

/* pinhole camera: eye, forward, right * th * aspect, up * th with th =
 * tan(fov / 2) given directly */
static void camera(d3 eye, d3 target, d3 up, double th, double aspect, float* cam)
{
    d3 fwd = normalize(sub(target, eye));
    d3 right = normalize(cross(fwd, up));
    d3 upv = cross(right, fwd);
    d3 q[4] = {eye, fwd, scl(right, th * aspect), scl(upv, th)};
    for (int k = 0; k < 4; ++k) {
        cam[3 * k] = (float)q[k].x; cam[3 * k + 1] = (float)q[k].y; cam[3 * k + 2] = (float)q[k].z;
    }
}

#define TAN_20_DEG 0.36397023426620236   /* Cornell camera: 40 degree field of view */

void synth_default_params(synth_scene_params* p)
{
    p->n_spheres = 64;
    p->n_large = 31;
    p->sphere_subdiv = 4;
    p->aspect = 1.0f;
}

static int sphere_tris(int subdiv) { int n = 20; for (int s = 0; s < subdiv; ++s) n *= 4; return n; }

static int valid(int32_t kind, const synth_scene_params* p)
{
    if (kind == SYNTH_CORNELL) return p->sphere_subdiv >= 0 && p->sphere_subdiv <= 6 &&
                                      p->aspect > 0.0f && p->aspect <= 16.0f;
    if (kind == SYNTH_PROCEDURAL) return p->n_spheres >= 1 && p->n_spheres <= 4096 &&
                                         p->n_large >= 0 && p->n_large <= p->n_spheres &&
                                         p->aspect > 0.0f && p->aspect <= 16.0f;
    return 0;
}

int synth_scene_counts(int32_t kind, const synth_scene_params* p, int32_t* n_tris,
                       int32_t* n_mats, int32_t* n_lights)
{
    synth_scene_params d;
    if (!p) { synth_default_params(&d); p = &d; }
    if (!valid(kind, p) || !n_tris || !n_mats || !n_lights) return -1;
    if (kind == SYNTH_CORNELL) {
        *n_tris = 10 + 2 + 2 * sphere_tris(p->sphere_subdiv);
        *n_mats = 6;
        *n_lights = 1;
    } else {
        *n_tris = 2 + p->n_large * sphere_tris(4) + (p->n_spheres - p->n_large) * sphere_tris(3) + 6;
        *n_mats = 1 + p->n_spheres + 3;
        *n_lights = 3;
    }
    return 0;
}

static void add_sphere(builder_t* b, const mesh_t* m, d3 center, double r, int mat)
{
    for (int j = 0; j < m->nf; ++j) {
        d3 p[3];
        for (int k = 0; k < 3; ++k) {
            const double* v = m->v + 3 * (size_t)m->f[3 * j + k];
            p[k] = add(scl(mk(v[0], v[1], v[2]), r), center);
        }
        put_tri(b, p[0], p[1], p[2], mat, -1);
    }
}

/* Cornell box: box x in [-1, 1], y in [0, 2], z in [-1, 1]; white 0.75,
 * red / green 0.6 walls; a 0.5 x 0.5 light of Le 15 under the ceiling; a
 * Lambertian and a GGX (alpha 0.3) sphere of radius 0.25; camera on the
 * z axis looking down -z */
static int cornell(builder_t* b, const synth_scene_params* p, float* env, float* cam)
{
    int white = material(b, 0, mk(0.75, 0.75, 0.75), 1.0, mk(0, 0, 0));
    int red = material(b, 0, mk(0.6, 0.05, 0.05), 1.0, mk(0, 0, 0));
    int green = material(b, 0, mk(0.05, 0.6, 0.05), 1.0, mk(0, 0, 0));
    quad(b, mk(-1, 0, -1), mk(0, 0, 2), mk(2, 0, 0), white, -1);   /* floor, +y */
    quad(b, mk(-1, 2, -1), mk(2, 0, 0), mk(0, 0, 2), white, -1);   /* ceiling, -y */
    quad(b, mk(-1, 0, -1), mk(2, 0, 0), mk(0, 2, 0), white, -1);   /* back wall, +z */
    quad(b, mk(-1, 0, -1), mk(0, 2, 0), mk(0, 0, 2), red, -1);     /* left wall, +x */
    quad(b, mk(1, 0, -1), mk(0, 0, 2), mk(0, 2, 0), green, -1);    /* right wall, -x */
    /* e1 along +x, e2 along +z: cross = -y, the light faces down */
    quad_light(b, mk(-0.25, 1.98, -0.25), mk(0.5, 0, 0), mk(0, 0, 0.5), mk(15, 15, 15));
    mesh_t m;
    if (icosphere(p->sphere_subdiv, &m)) return -1;
    int lam = material(b, 0, mk(0.75, 0.75, 0.75), 1.0, mk(0, 0, 0));
    int ggx = material(b, 1, mk(0.75, 0.75, 0.75), 0.3, mk(0, 0, 0));
    add_sphere(b, &m, mk(-0.4, 0.25, -0.3), 0.25, lam);
    add_sphere(b, &m, mk(0.4, 0.25, 0.2), 0.25, ggx);
    mesh_free(&m);
    env[0] = env[1] = env[2] = 0.0f;
    camera(mk(0, 1, 3.4), mk(0, 1, 0), mk(0, 1, 0), TAN_20_DEG, p->aspect, cam);
    return 0;
}

typedef struct { double r; int i; } rank_t;
static int by_radius_desc(const void* a, const void* b)
{
    const rank_t* x = (const rank_t*)a;
    const rank_t* y = (const rank_t*)b;
    if (x->r != y->r) return x->r > y->r ? -1 : 1;
    return x->i - y->i;
}

/* procedural field: ground quad 30 x 30 (Lambert 0.5); n_spheres icospheres
 * of radius U(0.1, 1) resting on the ground at U(-10, 10)^2, displaced by
 * value noise of amplitude 0.2 r, the n_large largest (ties by index) at
 * subdivision 4 and the rest at 3; 50/50 Lambert / GGX with alpha
 * U(0.05, 1) and albedo U(0.1, 0.9) per channel; 3 quad lights of size
 * U(1, 3)^2 at height U(4, 8) facing down with Le U(5, 20); environment 0.5 */
static int procedural(uint64_t seed, builder_t* b, const synth_scene_params* p, float* env,
                      float* cam)
{
    const int n = p->n_spheres;
    rng_t r = {seed * 0x9E3779B97F4A7C15ull ^ 0x6D72735F73636E65ull};
    double* radius = (double*)malloc(sizeof(double) * n);
    double* pos = (double*)malloc(sizeof(double) * 2 * n);
    int* kind = (int*)malloc(sizeof(int) * n);
    double* alpha = (double*)malloc(sizeof(double) * n);
    double* alb = (double*)malloc(sizeof(double) * 3 * n);
    uint64_t* salt = (uint64_t*)malloc(sizeof(uint64_t) * n);
    rank_t* order = (rank_t*)malloc(sizeof(rank_t) * n);
    char* large = (char*)calloc(n, 1);
    mesh_t m3 = {0, 0, NULL, NULL}, m4 = {0, 0, NULL, NULL};
    int rc = -1;
    if (!radius || !pos || !kind || !alpha || !alb || !salt || !order || !large) goto done;
    if (icosphere(3, &m3) || icosphere(4, &m4)) goto done;
    for (int i = 0; i < n; ++i) radius[i] = uniform(&r, 0.1, 1.0);
    for (int i = 0; i < 2 * n; ++i) pos[i] = uniform(&r, -10.0, 10.0);
    for (int i = 0; i < n; ++i) kind[i] = (int)(next64(&r) >> 63);
    for (int i = 0; i < n; ++i) alpha[i] = uniform(&r, 0.05, 1.0);
    for (int i = 0; i < 3 * n; ++i) alb[i] = uniform(&r, 0.1, 0.9);
    for (int i = 0; i < n; ++i) salt[i] = next64(&r) >> 33;
    for (int i = 0; i < n; ++i) { order[i].r = radius[i]; order[i].i = i; }
    qsort(order, n, sizeof(rank_t), by_radius_desc);
    for (int k = 0; k < p->n_large; ++k) large[order[k].i] = 1;

    int ground = material(b, 0, mk(0.5, 0.5, 0.5), 1.0, mk(0, 0, 0));
    quad(b, mk(-15, 0, -15), mk(0, 0, 30), mk(30, 0, 0), ground, -1);   /* normal +y */
    for (int i = 0; i < n; ++i) {
        const mesh_t* m = large[i] ? &m4 : &m3;
        double rad = radius[i];
        d3 c = mk(pos[2 * i], rad, pos[2 * i + 1]);
        int mat = material(b, kind[i], mk(alb[3 * i], alb[3 * i + 1], alb[3 * i + 2]), alpha[i],
                           mk(0, 0, 0));
        for (int j = 0; j < m->nf; ++j) {
            d3 q[3];
            for (int k = 0; k < 3; ++k) {
                const double* v = m->v + 3 * (size_t)m->f[3 * j + k];
                d3 u = mk(v[0], v[1], v[2]);
                double disp = 1.0 + 0.2 * (2.0 * value_noise(scl(u, 2.5), salt[i]) - 1.0);
                q[k] = add(scl(u, disp * rad), c);
            }
            put_tri(b, q[0], q[1], q[2], mat, -1);
        }
    }
    for (int l = 0; l < 3; ++l) {
        double sx = uniform(&r, 1.0, 3.0), sz = uniform(&r, 1.0, 3.0);
        double cx = uniform(&r, -8.0, 8.0), cy = uniform(&r, 4.0, 8.0), cz = uniform(&r, -8.0, 8.0);
        double le = uniform(&r, 5.0, 20.0);
        d3 p0 = mk(cx - 0.5 * sx, cy, cz - 0.5 * sz);
        /* e1 along +x, e2 along +z: cross = -y, the light faces down */
        quad_light(b, p0, mk(sx, 0, 0), mk(0, 0, sz), mk(le, le, le));
    }
    env[0] = env[1] = env[2] = 0.5f;
    /* 45 degree field of view: tan(22.5 degrees) = sqrt(2) - 1 */
    camera(mk(0, 6, 18), mk(0, 0.5, 0), mk(0, 1, 0), sqrt(2.0) - 1.0, p->aspect, cam);
    rc = 0;
done:
    mesh_free(&m3);
    mesh_free(&m4);
    free(radius); free(pos); free(kind); free(alpha); free(alb); free(salt); free(order);
    free(large);
    return rc;
}

int synth_scene_generate(uint64_t seed, int32_t kind, const synth_scene_params* p, float* V,
                         int32_t* tri_mat, int32_t* tri_light, float* mats, float* lights,
                         float* env, float* cam)
{
    synth_scene_params d;
    if (!p) { synth_default_params(&d); p = &d; }
    int32_t nt, nm, nl;
    if (synth_scene_counts(kind, p, &nt, &nm, &nl)) return -1;
    if (!V || !tri_mat || !tri_light || !mats || !env || !cam || (nl > 0 && !lights)) return -1;
    builder_t b = {V, tri_mat, tri_light, mats, lights, 0, 0, 0};
    int rc = kind == SYNTH_CORNELL ? cornell(&b, p, env, cam) : procedural(seed, &b, p, env, cam);
    if (rc) return rc;
    return (b.nt == nt && b.nm == nm && b.nl == nl) ? 0 : -1;
}
