/*
 * scenegen.h -- seeded synthetic scenes, the shared input generator of the
 * renderer (its CPU reference and its CUDA library both consume what these
 * functions write).  A scene is described by flat arrays:
 *
 *   V          float [n_tris][3][3]  triangle vertices v0, v1, v2
 *   tri_mat    int32 [n_tris]        material index
 *   tri_light  int32 [n_tris]        quad light the triangle belongs to, or -1
 *   mats       float [n_mats][8]     type (0 Lambert, 1 GGX), albedo rgb,
 *                                    GGX alpha, emitted radiance rgb (one-sided,
 *                                    along cross(v1 - v0, v2 - v0))
 *   lights     float [n_lights][12]  quad lights p0, e1, e2, Le (emitting along
 *                                    normalize(cross(e1, e2)))
 *   env        float [3]             constant environment radiance
 *   cam        float [12]            eye, forward, right * tan(fov/2) * aspect,
 *                                    up * tan(fov/2)
 *
 * The arithmetic is integer and IEEE double (+ - * / sqrt, floor) rounded once
 * to float, with no other libm call, so that a seed gives the same scene on
 * every host.  Compile with -ffp-contract=off.  The generator holds no
 * rendering arithmetic.
 */
#ifndef SYNTH_SCENEGEN_H
#define SYNTH_SCENEGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYNTH_CORNELL 0      /* Cornell box: 5 quads, 2 icospheres, 1 quad light */
#define SYNTH_PROCEDURAL 1   /* noise-displaced icospheres on a ground plane */

typedef struct {
    int32_t n_spheres;       /* procedural: spheres (default 64) */
    int32_t n_large;         /* procedural: the n_large largest use subdivision 4, the
                                rest 3 (default 31) */
    int32_t sphere_subdiv;   /* Cornell: icosphere subdivision of both spheres (default 4) */
    float aspect;            /* image width / height of the camera (default 1) */
} synth_scene_params;

/* Fills *p with the defaults above. */
void synth_default_params(synth_scene_params* p);

/* Array sizes of a scene (0 on success, -1 on an invalid kind or parameter:
 * n_spheres in [1, 4096], n_large in [0, n_spheres], sphere_subdiv in [0, 6],
 * aspect in (0, 16]). */
int synth_scene_counts(int32_t kind, const synth_scene_params* p, int32_t* n_tris,
                       int32_t* n_mats, int32_t* n_lights);

/* Writes the scene of (seed, kind, p) into caller arrays sized by
 * synth_scene_counts (lights may be NULL when n_lights is 0).  Returns 0, or
 * -1 on invalid arguments. */
int synth_scene_generate(uint64_t seed, int32_t kind, const synth_scene_params* p, float* V,
                         int32_t* tri_mat, int32_t* tri_light, float* mats, float* lights,
                         float* env, float* cam);

#ifdef __cplusplus
}
#endif
#endif /* SYNTH_SCENEGEN_H */
