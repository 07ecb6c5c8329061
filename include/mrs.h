/*
 * mrs.h -- C ABI of the multi-resolution sampling renderer for GB300 (sm_103a).
 *
 * The method (Hou et al., "Fast Monte Carlo Rendering via Multi-Resolution
 * Sampling", Sec. 1 and Sec. 4) renders the same view twice -- a
 * low-resolution image at a high sample count (LRHS) and a high-resolution
 * image at a low sample count (HRLS, with albedo / normal / depth layers,
 * Sec. 3.2 and Sec. 4) -- and fuses them with a convolutional network into the
 * high-resolution estimate I_SR (problem statement of Sec. 4).
 *
 * Conventions for every entry point:
 *  - Image pointers are DEVICE pointers owned by the caller, float32, NHWC,
 *    C-contiguous ([N][H][W][C]; N = 1 where no batch argument exists).
 *  - Scene and parameter arrays passed by HOST pointer are copied in before
 *    the call returns; the caller may free them afterwards.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously unless the entry point says it synchronises.
 *  - Arguments are validated before anything is launched; on an invalid
 *    argument the call returns MRS_ERR_ARG and has no effect.  CUDA errors are
 *    mapped to MRS_ERR_CUDA (the CUDA error string is kept for
 *    mrs_last_error()).  No entry point aborts the process.
 *  - Handles (mrs_scene, mrs_net) own all device memory they allocate; it is
 *    released by the matching mrs_*_free call.  A handle may be used from one
 *    stream at a time.
 *  - There is no CPU fallback: without a CUDA device every call that computes
 *    returns MRS_ERR_CUDA.
 */
#ifndef MRS_H
#define MRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mrs_status;
#define MRS_OK 0
#define MRS_ERR_ARG (-1)       /* invalid argument (null pointer, size, range) */
#define MRS_ERR_OOM (-2)       /* device allocation failed */
#define MRS_ERR_CUDA (-3)      /* a CUDA runtime/driver call failed */
#define MRS_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up */
#define MRS_ERR_CAPACITY (-5)  /* a size exceeds a documented capacity */
#define MRS_ERR_STATE (-6)     /* handle used in the wrong state */
#define MRS_ERR_FORMAT (-7)    /* a file is not a valid checkpoint (magic, size, checksum) */
#define MRS_ERR_IO (-8)        /* a file could not be opened, read or written */

typedef struct mrs_scene_s* mrs_scene;
typedef struct mrs_net_s* mrs_net;
typedef struct mrs_ctx_s* mrs_ctx;

/* Human-readable name of a status code (static string). */
const char* mrs_status_string(mrs_status s);
/* Last error detail recorded by this thread (static per-thread buffer). */
const char* mrs_last_error(void);
/* Number of CUDA kernels this library has launched in this process so far
 * (instrumentation for benchmarks; no paper counterpart). */
uint64_t mrs_kernel_launches(void);

/* ------------------------------------------------------------------------
 * Scene + LBVH.  The renderer that produces LRHS and HRLS (Sec. 1, Sec. 3.2)
 * needs a ray-casting structure; the paper renders with Blender Cycles and
 * does not specify one, so this library builds a linear BVH on the GPU:
 * 30-bit Morton codes of triangle centroids (10 bits per axis, x highest) in
 * the centroid bounding box, a stable radix sort of (code, triangle index),
 * the binary radix tree of Karras (HPG 2012) over the 64-bit keys
 * code << 32 | index, and a bottom-up refit of the boxes.  The renders
 * traverse that tree, or (mrs_scene_set_tree, MRS_TREE_CLUSTER) one built over
 * the same sorted leaves by locally-ordered agglomerative clustering: about
 * 20% lower surface-area cost, 6-8% faster renders, about 3x the build time;
 * the closest hit is the same with either.
 *
 * V          host, float [n_tris][3][3]   triangle vertices
 * tri_mat    host, int32 [n_tris]         material index (0 <= m < n_mats)
 * tri_light  host, int32 [n_tris]         light index (0 <= l < n_lights) or -1
 * mats       host, float [n_mats][8]      type (0 Lambert, 1 GGX), albedo rgb,
 *                                         GGX alpha, emitted radiance rgb
 *                                         (one-sided, along cross(v1-v0, v2-v0))
 * lights     host, float [n_lights][12]   quad lights p0, e1, e2, Le (may be
 *                                         NULL when n_lights == 0)
 * env        host, float [3]              constant environment radiance
 * cam        host, float [12]             eye, forward, right*tan(fov/2)*aspect,
 *                                         up*tan(fov/2)
 * n_tris may be 0 (every ray misses).  The LBVH is built on `stream` before
 * the call returns (the call synchronises `stream`).
 * ------------------------------------------------------------------------ */
mrs_status mrs_build_scene(const float* V, int32_t n_tris, const int32_t* tri_mat,
                           const int32_t* tri_light, const float* mats, int32_t n_mats,
                           const float* lights, int32_t n_lights, const float* env,
                           const float* cam, void* stream, mrs_scene* out);

/* Seeded scene + LBVH: the scene is generated on the host from (seed, kind,
 * params) -- the workloads this library is measured on; the paper's scenes
 * are Blender scenes (Sec. 3.1) that these procedural stand-ins replace --
 * and then built exactly as mrs_build_scene builds the arrays it is given.
 *   MRS_SCENE_CORNELL     Cornell box: 5 Lambertian quads (white 0.75,
 *                         red / green 0.6), a Lambert and a GGX (alpha 0.3)
 *                         icosphere of radius 0.25 (subdivision
 *                         params->sphere_subdiv), one 0.5 x 0.5 quad light of
 *                         Le 15; no environment; seed unused
 *   MRS_SCENE_PROCEDURAL  ground quad 30 x 30 (Lambert 0.5) with
 *                         params->n_spheres icospheres of radius U(0.1, 1)
 *                         displaced by value noise (amplitude 0.2 r), the
 *                         n_large largest at subdivision 4 and the rest at 3,
 *                         50/50 Lambert / GGX with alpha U(0.05, 1) and albedo
 *                         U(0.1, 0.9); 3 downward quad lights of Le U(5, 20);
 *                         environment 0.5 (the defaults give 200,968 triangles)
 * params (HOST, may be NULL: n_spheres 64, n_large 31, sphere_subdiv 4,
 * aspect 1) -- n_spheres in [1, 4096], n_large in [0, n_spheres],
 * sphere_subdiv in [0, 6], aspect (camera width / height) in (0, 16], else
 * MRS_ERR_ARG.  Random numbers are one splitmix64 stream seeded from `seed`;
 * the generator uses integer and IEEE arithmetic only, so a seed gives the
 * same scene on every host.  Synchronises `stream` like mrs_build_scene. */
#define MRS_SCENE_CORNELL 0
#define MRS_SCENE_PROCEDURAL 1
typedef struct {
    int32_t n_spheres;
    int32_t n_large;
    int32_t sphere_subdiv;
    float aspect;
} mrs_scene_params;
mrs_status mrs_build_scene_seeded(uint64_t seed, int32_t kind, const mrs_scene_params* params,
                                  void* stream, mrs_scene* out);

/* Re-run the GPU build (Morton codes, sort, render tree) over the scene's
 * resident triangles on `stream`; with MRS_TREE_CLUSTER the build reads its
 * error word back, which synchronises `stream`. */
mrs_status mrs_scene_rebuild(mrs_scene scene, void* stream);

/* The render tree (the nodes mrs_render, mrs_cast and the path tracer walk):
 *   MRS_TREE_LBVH     the Karras radix tree with refitted boxes (the default:
 *                     the cheapest build)
 *   MRS_TREE_CLUSTER  locally-ordered agglomerative clustering (Meister and
 *                     Bittner, TVCG 2018) over the Morton-sorted leaves, search
 *                     radius 16: each round, every cluster picks the neighbour
 *                     within 16 positions whose union box has the smallest
 *                     surface area (ties by a hash of the position pair),
 *                     mutual pairs merge, the list is compacted (for scenes
 *                     built once and rendered many times)
 *   MRS_TREE_HCLUSTER the same clustering inside the subtrees of the radix
 *                     tree, bottom-up in one launch (Benthin et al., HPG 2024,
 *                     on the agglomerative walk of Apetrei, 2014): a subtree
 *                     keeps at most 16 clusters; where two children meet with
 *                     more, one warp merges mutual nearest pairs among all of
 *                     them until 16 are left (one at the root).  Nearly the
 *                     global rounds' surface-area cost, no read-back, also
 *                     inside a caller's stream capture.  Node ids are a
 *                     function of the tree (the radix tree's split
 *                     positions), the same on every rebuild.  A frame that
 *                     rebuilds its tree every step runs fastest over it.
 * set_tree records the choice and rebuilds the tree on `stream` (synchronised).
 * get_tree returns the kind in use: MRS_TREE_LBVH also when clustering was
 * asked for but did not finish within its bound of 72 grid-wide rounds plus
 * 2048 single-block rounds (then the radix tree was built instead).  The
 * choice stays with the scene for later rebuilds. */
#define MRS_TREE_LBVH 0
#define MRS_TREE_CLUSTER 1
#define MRS_TREE_HCLUSTER 2
mrs_status mrs_scene_set_tree(mrs_scene scene, int32_t kind, void* stream);
mrs_status mrs_scene_get_tree(mrs_scene scene, int32_t* kind);
/* The render tree's nodes: n_tree (HOST) receives ns, the triangles in the
 * tree (the rest are the large triangles every ray tests first); nodes (HOST,
 * may be NULL) float [ns - 1][16] when n_floats >= 16 (ns - 1): per internal
 * node i (node 0 the root) the boxes of its two children (lo xyz, hi xyz of
 * the first, then of the second) and the children's ids as int32 bits in
 * floats 12 and 13 (an id below ns - 1 is an internal node, ns - 1 + k the
 * leaf of triangle order[k]); order (HOST, may be NULL) int32 [ns] the
 * triangle of each leaf.  Synchronises the device. */
mrs_status mrs_scene_export_nodes(mrs_scene scene, float* nodes, int64_t n_floats, int32_t* order,
                                  int32_t* n_tree);

/* Replace the triangle vertices (HOST float [n][3][3], n equal to the scene's
 * triangle count; materials and lights unchanged) and rebuild the render
 * tree on `stream` (an animated scene's per-frame update).  The large /
 * small split and the clustering build read counts back, so the call
 * synchronises `stream`. */
mrs_status mrs_scene_update_vertices(mrs_scene scene, const float* V, int32_t n, void* stream);

mrs_status mrs_free_scene(mrs_scene scene);

/* Copy the LBVH to caller DEVICE buffers (any may be NULL):
 * morton [n] (input order), order [n] (sorted position -> triangle index),
 * left/right [n-1] (child id: < n-1 internal node, >= n-1 leaf n-1+position),
 * box [(2n-1)][6] (lo xyz, hi xyz; internal nodes first, then leaves). */
mrs_status mrs_scene_export_bvh(mrs_scene scene, uint32_t* morton, int32_t* order,
                                int32_t* left, int32_t* right, float* box, void* stream);

/* LBVH build that allocates nothing.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc (or any allocating library
 * routine) -- code running inside another allocator's callback, under a
 * memory-reservation regime that forbids new device allocations, or in a
 * hard real-time frame loop where an allocation could stall.  It builds the
 * LBVH over all n triangles, bit-identical to what mrs_scene_export_bvh
 * returns for a scene of the same triangles (not the tree mrs_render
 * traverses, which leaves the few scene-sized triangles out of the LBVH and
 * tests them apart), from device inputs into device outputs, with all
 * scratch memory (about 7.5 MB) in one static device array inside
 * libmrs.so; every GPU that loads the library keeps that array until the
 * process exits.
 *
 * V      device float [n][3][3] triangle vertices
 * morton device uint32 [n], order device int32 [n], left/right device int32
 *        [n-1] (may be NULL when n == 1), box device float [(2n-1)][6]: the same
 *        layouts as mrs_scene_export_bvh.
 * n must be <= MRS_LBVH_STATIC_MAX_TRIS, else MRS_ERR_CAPACITY with a message.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture.  The kept
 * address does not survive cudaDeviceReset (or an unload of the library):
 * do not call this entry point on a device after resetting it.  Calls share
 * the one array: two calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and corrupt each other;
 * serialise them.  Work is enqueued on `stream`. */
#define MRS_LBVH_STATIC_MAX_TRIS 262144
mrs_status mrs_lbvh_build_static(const float* V, int32_t n, uint32_t* morton, int32_t* order,
                                 int32_t* left, int32_t* right, float* box, void* stream);

/* Closest hit of n_rays rays through the LBVH: orig/dir device float [n][3];
 * prim device int32 [n] (triangle index, -1 on miss), t device float [n]
 * (-1 on miss).  Ties in t go to the smaller triangle index. */
mrs_status mrs_cast(mrs_scene scene, const float* orig, const float* dir, int32_t n_rays,
                    int32_t* prim, float* t, void* stream);

/* ------------------------------------------------------------------------
 * Monte Carlo path tracing (Sec. 1: the LRHS and HRLS renders; Sec. 3.2:
 * auxiliary render layers).  Unidirectional path tracing with next-event
 * estimation to the quad lights and the environment, power-heuristic MIS,
 * Lambert and GGX (visible-normal sampling, Smith height-correlated masking)
 * materials, Russian roulette from bounce rr_start on (p = min(0.95, max
 * throughput channel)).  max_depth is the number of scattering events
 * (0 = emission only).  Random numbers: Philox4x32-10 with counter
 * (pixel, sample, bounce, group) and key (seed lo, seed hi); group 0 gives
 * BSDF u1, u2, light u, v; group 1 light pick, roulette, pixel jitter x, y.
 *
 * Per pixel, the per-sample radiance is summed in sample order with Kahan
 * compensation in float32 and divided by spp.  Aux layers are the first-hit
 * albedo, the normal facing the camera, and the hit distance (0 on a miss),
 * averaged over samples.  An image at 1/s resolution through the same camera
 * covers the same frustum: each of its pixels jitters over its whole
 * footprint (the LRHS render).
 *
 * radiance device float [H][W][3] (required); albedo, normal [H][W][3] and
 * depth [H][W] device (may be NULL); counts / shadow_counts device uint64
 * [max_depth+1] (may be NULL): extension / shadow rays cast at each bounce.
 * rr_start < 0 disables Russian roulette.  Limits: W, H in [1, 16384],
 * spp in [1, 65536], max_depth in [0, 32].  Allocates its path-state arena
 * inside the scene handle on first use (grown on demand).
 * ------------------------------------------------------------------------ */
mrs_status mrs_render(mrs_scene scene, int32_t W, int32_t H, int32_t spp, int32_t max_depth,
                      int32_t rr_start, uint64_t seed, float* radiance, float* albedo,
                      float* normal, float* depth, uint64_t* counts, uint64_t* shadow_counts,
                      void* stream);

/* The same render with instrumented traversal: stats device uint64[8] receives
 * BVH node visits and triangle tests of the closest-hit traversals, then of
 * the shadow (any-hit) traversals (entries 0-3, all bounces), then the part
 * of those four done inside the tail kernel (entries 4-7; see
 * mrs_scene_set_tail).  The radiance equals mrs_render's.  For measuring
 * algorithmic work (roofline accounting); no paper counterpart. */
mrs_status mrs_render_stats(mrs_scene scene, int32_t W, int32_t H, int32_t spp, int32_t max_depth,
                            int32_t rr_start, uint64_t seed, float* radiance, uint64_t* stats,
                            void* stream);

/* Per-kernel CUDA-event timing: when enabled, the library records an event
 * pair on the launching stream around each launch of the kernels below, and
 * mrs_profile_read (which synchronises on those events) returns and clears
 * the total milliseconds and launch count of one kernel family:
 * 0 closest-hit traversal, 1 shade, 2 shadow traversal, 3 ray generation,
 * 4 accumulation, 5 render-tree build (whole, any kind), 6 tensor-core conv, 7 SIMT conv,
 * 8 fusion input, 9 metrics, 10 training kernels (other than 11),
 * 11 tensor-core weight gradient, 12 the render's tail kernel (the late
 * bounces' traversal, shading and shadow rays in one launch).
 * Instrumentation only. */
mrs_status mrs_profile_enable(int32_t on);
mrs_status mrs_profile_read(int32_t kernel, double* total_ms, int64_t* launches);

/* Failure-detection self-test (no paper counterpart): launches a kernel whose
 * bounded device-side wait (the kind every tensor-core kernel uses on its
 * mbarriers) waits for an event that never happens.  The wait must give up
 * after limit_us microseconds (1 .. 100000), raise the kernel's error word
 * and return; the call then returns MRS_ERR_TIMEOUT and the CUDA context
 * stays usable.  Synchronises `stream`. */
mrs_status mrs_selftest_wait_timeout(int32_t limit_us, void* stream);

/* Render contexts.  mrs_render keeps its path state in the scene handle, so
 * renders of one scene are serialised; a context owns its own path-state
 * arena, so renders of the same scene through different contexts may run
 * concurrently on different streams (e.g. the LRHS and HRLS renders of a
 * frame, whose low-occupancy last bounces then overlap).  mrs_render_ctx takes
 * the arguments of mrs_render; the arena is allocated on first use and grown
 * on demand (make the first call before any stream capture). */
mrs_status mrs_ctx_create(mrs_ctx* out);
mrs_status mrs_ctx_free(mrs_ctx ctx);
mrs_status mrs_ctx_set_wave(mrs_ctx ctx, int64_t max_paths_per_wave);
mrs_status mrs_render_ctx(mrs_ctx ctx, mrs_scene scene, int32_t W, int32_t H, int32_t spp,
                          int32_t max_depth, int32_t rr_start, uint64_t seed, float* radiance,
                          float* albedo, float* normal, float* depth, uint64_t* counts,
                          uint64_t* shadow_counts, void* stream);

/* Render on a sparse camera-sampling grid (the paper's low-resolution images,
 * Sec. 3 "Low Resolution Image Generation": nearest-neighbour downsampling
 * of a `grid`-times finer render, i.e. rays on a sparse grid): pixel (x, y)
 * of the W x H image draws all its samples inside the single sub-pixel
 * (grid*x + grid/2, grid*y + grid/2) of the (grid*W) x (grid*H) image, instead
 * of over its whole footprint.  grid = 1 is exactly mrs_render.  ctx may be
 * NULL (the scene's own path state, as mrs_render) or a render context (as
 * mrs_render_ctx).  grid in [1, 64], W*grid and H*grid <= 65536; other
 * arguments as in mrs_render. */
mrs_status mrs_render_grid(mrs_ctx ctx, mrs_scene scene, int32_t W, int32_t H, int32_t spp,
                           int32_t max_depth, int32_t rr_start, uint64_t seed, int32_t grid,
                           float* radiance, float* albedo, float* normal, float* depth,
                           uint64_t* counts, uint64_t* shadow_counts, void* stream);

/* Every output of a render, including the extra HRLS layers of Sec. 4
 * (device pointers, all [H][W][3] float except depth [H][W] and the
 * uint64[max_depth + 1] ray counts; only radiance is required, NULL skips a
 * layer):
 *   diffuse / specular: mean over samples of the radiance of the samples whose
 *     first hit is Lambertian / GGX (samples that see the environment
 *     directly count in neither: radiance = diffuse + specular + that part);
 *   variance: per channel, the sample variance of the pixel mean,
 *     (sum L^2 - (sum L)^2 / N) / (N (N - 1)) with the compensated sum of L,
 *     0 when N = 1, floored at 0. */
typedef struct {
    float* radiance;
    float* albedo;
    float* normal;
    float* depth;
    float* diffuse;
    float* specular;
    float* variance;
    uint64_t* counts;
    uint64_t* shadow_counts;
} mrs_render_out;
/* mrs_render_grid with all outputs; the extra layers cost a per-path lobe
 * record and a second per-pixel accumulator, only when requested. */
mrs_status mrs_render_layers(mrs_ctx ctx, mrs_scene scene, int32_t W, int32_t H, int32_t spp,
                             int32_t max_depth, int32_t rr_start, uint64_t seed, int32_t grid,
                             const mrs_render_out* out, void* stream);

/* A window of an image: the pixels [x0, x0 + w) x [y0, y0 + h) of the W x H
 * render of mrs_render_layers (same camera, same per-pixel random numbers:
 * every output pixel, layer and count is bit-identical to that pixel of the
 * whole-image render), with outputs [h][w][...].  For rendering crops
 * (training examples at the full image's pixel scale) without the rest of
 * the image.  The window must lie inside the image (else MRS_ERR_ARG). */
mrs_status mrs_render_window(mrs_ctx ctx, mrs_scene scene, int32_t W, int32_t H, int32_t x0,
                             int32_t y0, int32_t w, int32_t h, int32_t spp, int32_t max_depth,
                             int32_t rr_start, uint64_t seed, int32_t grid,
                             const mrs_render_out* out, void* stream);

/* Many renders in one pass (serving many frames of different scenes, sizes
 * and sample counts): each job is the render mrs_render_grid would produce
 * for its arguments (radiance and the albedo / normal / depth layers; every
 * output bit-identical to that call's), but the jobs' paths share waves:
 * each job's samples are cut into chunks that fit the context's wave size
 * (mrs_ctx_set_wave, whole samples of every pixel, at least one), and
 * consecutive chunks of up to 32 jobs fill one wave, whose ray generation,
 * bounce-0 traversal / shading / shadow rays and persistent tail kernel
 * are one launch each over all of its jobs (the jobs' scenes, cameras and
 * seeds travel as a table in the launch).  Each chunk's samples are then
 * added to its job's per-pixel sums in sample order, so chunking changes
 * nothing.  Per-bounce ray counts are not reported per job.  ctx is
 * required (its arena holds the largest wave's path state and every job's
 * accumulator; make the first call of a size before any stream capture).
 * jobs HOST array [n_jobs] (1 .. 4096), read before the call returns; each
 * job's radiance (required) and albedo, normal, depth (may be NULL) are
 * device buffers as for mrs_render; grid as mrs_render_grid; other
 * arguments as mrs_render. */
typedef struct {
    mrs_scene scene;
    int32_t W, H, spp, max_depth, rr_start;
    uint64_t seed;
    int32_t grid;
    float* radiance;
    float* albedo;
    float* normal;
    float* depth;
} mrs_render_job;
mrs_status mrs_render_batch(mrs_ctx ctx, const mrs_render_job* jobs, int32_t n_jobs, void* stream);

/* Paths per wave for subsequent mrs_render calls on this scene (rounded to
 * whole samples of the image; default 16M paths).  For tests and tuning. */
mrs_status mrs_scene_set_wave(mrs_scene scene, int64_t max_paths_per_wave);

/* First bounce that the renders of this scene (mrs_scene_set_tail: those
 * without a context) or of this context (mrs_ctx_set_tail) shade in the tail
 * kernel instead of one launch per step: every bounce b >= `bounce` of a
 * path runs in a single persistent launch that takes each path left in the
 * queue of bounce `bounce` to its end.  The result is bit-identical either
 * way (same per-path operations, same counts); only the launch structure
 * changes.  -1 (default): bounce 1; any value > max_depth: no tail.  Range
 * [-1, 64], else MRS_ERR_ARG. */
mrs_status mrs_scene_set_tail(mrs_scene scene, int32_t bounce);
mrs_status mrs_ctx_set_tail(mrs_ctx ctx, int32_t bounce);

/* The 8 Philox uniforms of each (pixel, sample, bounce) triple given in
 * `triples` (device uint32 [n][3]) for key = seed: out device float [n][8]. */
mrs_status mrs_philox_uniforms(const uint32_t* triples, int32_t n, uint64_t seed, float* out,
                               void* stream);


/* ------------------------------------------------------------------------
 * Fusion network (Sec. 4: I_SR is estimated from I_LRHS and I_HRLS + layers).
 * Architecture (all-high-resolution variant): bilinear x s upsampling of LRHS
 * (half-pixel centres, edge clamp), concatenation with HRLS RGB, albedo and
 * normal (12 channels), conv3x3 12->64 + ReLU, 8 residual blocks
 * h + conv3x3(relu(conv3x3(h))), conv3x3 64->3, plus the upsampled LRHS.
 * All kernels 3x3 with zero padding; 64 feature channels (Sec. 4,
 * "Implement details").
 *
 * Parameters: MRS_NET_NPARAMS float32 values; for each of the 18 convs in
 * forward order, weight [Cout][3][3][Cin] then bias [Cout].
 * ------------------------------------------------------------------------ */
#define MRS_NET_NPARAMS 599555
/* The same network with the extra HRLS layers of Sec. 4 as nine more input
 * channels (21 in all): after the 12 above come diffuse RGB, specular RGB and
 * log(1 + max(variance, 0)) per channel (the log is this library's reading:
 * the variance spans orders of magnitude).  Only the first conv grows, to
 * weight [64][3][3][21]. */
#define MRS_NET_NPARAMS_EXTRA 604739
#define MRS_NET_EXTRA_CHANNELS 9
#define MRS_PREC_FP32 0   /* FP32 SIMT convolutions (reference precision) */
#define MRS_PREC_BF16 1   /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
#define MRS_PREC_FP8 2    /* FP8-E4M3 operands, per-output-channel weight scales */

/* params: HOST float [n_params], copied in as the FP32 master weights; Adam
 * moments start at zero.  n_params = MRS_NET_NPARAMS makes the 12-channel
 * network, MRS_NET_NPARAMS_EXTRA the 21-channel one (extra HRLS layers);
 * anything else is MRS_ERR_ARG.  All later parameter arrays of the handle
 * (set/get params, grads, state) have that many values. */
mrs_status mrs_net_create(const float* params, int32_t n_params, mrs_net* out);
mrs_status mrs_net_free(mrs_net net);
/* Input channels of the net's first conv: 12 or 21 (HOST int32 out). */
mrs_status mrs_net_input_channels(mrs_net net, int32_t* channels);
/* Replace / read the FP32 master weights (HOST float [MRS_NET_NPARAMS]);
 * set also resets the Adam state.  Both synchronise the device. */
mrs_status mrs_net_set_params(mrs_net net, const float* params);
mrs_status mrs_net_get_params(mrs_net net, float* params);

/* I_SR = net(LRHS, HRLS, albedo, normal).  lrhs device [N][h][w][3]; hrls,
 * albedo, normal device [N][H][W][3] with H = scale*h, W = scale*w;
 * out device [N][H][W][3].  scale in {1, 2, 4, 8}; precision one of
 * MRS_PREC_*.  Activation workspace lives in the net handle (grown on
 * demand).  Limits: N*H*W <= 2^27 pixels. */
mrs_status mrs_fuse(mrs_net net, const float* lrhs, const float* hrls, const float* albedo,
                    const float* normal, int32_t N, int32_t H, int32_t W, int32_t scale,
                    int32_t precision, float* out, void* stream);
/* mrs_fuse with the extra HRLS layers as input (Sec. 4: the HRLS carries
 * albedo, normal, diffuse, specular and variance layers).  extra device
 * [N][H][W][9] = diffuse RGB, specular RGB, variance RGB as mrs_render_layers
 * writes them; it must be non-NULL exactly for a 21-channel net (else
 * MRS_ERR_ARG); mrs_fuse is this call with extra = NULL. */
mrs_status mrs_fuse_extra(mrs_net net, const float* lrhs, const float* hrls, const float* albedo,
                          const float* normal, const float* extra, int32_t N, int32_t H, int32_t W,
                          int32_t scale, int32_t precision, float* out, void* stream);

/* One training step of the fusion network (learned part of the method; the
 * paper trains with a robust loss and SGD, Sec. 4 "Loss function" and
 * "Implement details" -- this library uses L1 on log(1 + radiance) with Adam):
 * forward with every activation kept, the net's loss (mrs_net_set_loss;
 * default mean |slog(y) - slog(target)| with slog(x) = sign(x) log1p(|x|),
 * log(1 + radiance) for x >= 0) over N*H*W*3 values (reduced in float64),
 * full backward
 * (transposed convolutions with flipped taps, ReLU masks, dW / db
 * reductions), and one bias-corrected Adam update (beta1 0.9, beta2 0.999,
 * eps 1e-8) of the FP32 master weights.  LRHS, HRLS and the target are
 * clipped at 100 first (firefly clipping of the training data, Sec. 3.2).
 * Image arguments as in mrs_fuse plus target device [N][H][W][3].
 * precision MRS_PREC_FP32: every convolution in FP32 (SIMT);
 * MRS_PREC_BF16: forward, transposed and weight-gradient convolutions on
 * the tensor cores with BF16 activations and activation gradients, FP32
 * accumulation, FP32 dW / db reductions and FP32 master weights.  loss_out (HOST, may be NULL) receives
 * the loss before the update; when non-NULL the call synchronises `stream`.
 * Limit: N*H*W <= 2^22 pixels. */
mrs_status mrs_train_step(mrs_net net, const float* lrhs, const float* hrls, const float* albedo,
                          const float* normal, const float* target, int32_t N, int32_t H,
                          int32_t W, int32_t scale, float lr, int32_t precision, double* loss_out,
                          void* stream);
/* mrs_train_step with the extra HRLS layers (device [N][H][W][9], as in
 * mrs_fuse_extra; non-NULL exactly for a 21-channel net).  Their diffuse and
 * specular radiance is clipped at 100 like the HRLS; the variance is not. */
mrs_status mrs_train_step_extra(mrs_net net, const float* lrhs, const float* hrls,
                                const float* albedo, const float* normal, const float* extra,
                                const float* target, int32_t N, int32_t H, int32_t W, int32_t scale,
                                float lr, int32_t precision, double* loss_out, void* stream);
/* Gradient of the last mrs_train_step (HOST float [n_params]; synchronises). */
mrs_status mrs_net_get_grads(mrs_net net, float* grads);
/* Checkpoint / resume: FP32 master weights, Adam moments (HOST float
 * [MRS_NET_NPARAMS] each) and the Adam step count.  Both synchronise. */
mrs_status mrs_net_get_state(mrs_net net, float* params, float* adam_m, float* adam_v,
                             int64_t* step);
mrs_status mrs_net_set_state(mrs_net net, const float* params, const float* adam_m,
                             const float* adam_v, int64_t step);

/* Checkpoint / resume to a file (the paper keeps the best model during
 * training, Sec. 4 "Implement details"; the file format is this library's).
 * mrs_net_save writes the FP32 master weights, both Adam moments, the Adam
 * step, the training loss (kind and beta) and the caller's `seed` (e.g. the
 * data-sampling seed, returned by mrs_net_load so that a resumed run draws
 * the same batches) to `path`: a 64-byte little-endian header
 *   "MRSNETv2", uint32 64, uint32 2, int64 n_params, int64 step,
 *   uint64 seed, int32 input channels (12 / 21), int32 loss, float beta,
 *   uint32 0, uint64 FNV-1a-64 checksum of the payload
 * then params, adam_m, adam_v as float32 [n_params] each.  The file is
 * written to `path`.tmp and renamed over `path`.  mrs_net_load restores such
 * a file into a net of the same parameter count (MRS_ERR_FORMAT on a wrong
 * magic, version, size, loss or checksum, or trailing bytes; MRS_ERR_IO if
 * the file cannot be read; the net is left unchanged on any error); seed
 * (HOST, may be NULL) receives the stored seed.  Both synchronise the
 * device.  Resuming from a file continues bit-identically to a run that was
 * never interrupted. */
mrs_status mrs_net_save(mrs_net net, const char* path, uint64_t seed);
mrs_status mrs_net_load(mrs_net net, const char* path, uint64_t* seed);

/* A net with seeded initial weights instead of caller-given ones:
 * input_channels 12 (MRS_NET_NPARAMS) or 21 (MRS_NET_NPARAMS_EXTRA); every
 * conv weight zero-mean with the Kaiming variance 2 / (9 Cin), drawn as the
 * sum of 12 splitmix64 uniforms minus 6 (integer and IEEE arithmetic only:
 * the same seed gives the same weights on every host); the second conv of
 * each residual block scaled by resid_gain (in [0, 1]); the 3-channel head
 * and every bias zero, so the untrained net outputs the upsampled LRHS
 * exactly (training starts from the method without the network). */
mrs_status mrs_net_create_seeded(int32_t input_channels, uint64_t init_seed, float resid_gain,
                                 mrs_net* out);

/* Image error metrics of x against ref (device float, n values each, both in
 * scene-linear space), reduced in float64 on the GPU (Sec. 5):
 * out[0] = PSNR of the sRGB images (Eq. cvt_color, peak 1; +inf if equal),
 * out[1] = RelMSE with lambda1, lambda2, out[2] = MSE (linear).
 * out is a HOST double[3]; the call synchronises `stream`. */
mrs_status mrs_image_metrics(const float* x, const float* ref, int64_t n, double lambda1,
                             double lambda2, double* out, void* stream);

/* Fallback gate of the hybrid renderer: D = RelMSE(box_s(fused), LRHS)
 * (lambda1 = 0.5, lambda2 = 0.01), box_s = mean over s x s blocks.  If
 * D > tau, out = plain (the plain high-resolution render), else out = fused.
 * fused, plain, out device [N][H][W][3]; lrhs device [N][h][w][3]; plain may
 * equal NULL only if the caller accepts out = fused regardless (then
 * *used_plain reports the decision without copying).  used_plain and D are
 * HOST pointers (may be NULL); the call synchronises `stream`. */
mrs_status mrs_gate(const float* fused, const float* lrhs, const float* plain, int32_t N,
                    int32_t H, int32_t W, int32_t scale, double tau, float* out,
                    int32_t* used_plain, double* D, void* stream);

/* The same gate without any host synchronisation (capturable in a CUDA
 * graph): the decision stays on the device.  used_plain is a DEVICE int32[2]:
 * [0] = 1 if D > tau, [1] = 1 if `out` received the plain render (plain given
 * and D > tau); D (DEVICE double, may be NULL) receives D.  out receives
 * plain or fused accordingly (out may alias fused).  The first call allocates
 * a small reduction buffer (make it before any stream capture); concurrent
 * calls from several threads are serialised. */
mrs_status mrs_gate_async(const float* fused, const float* lrhs, const float* plain, int32_t N,
                          int32_t H, int32_t W, int32_t scale, double tau, float* out,
                          int32_t* used_plain, double* D, void* stream);

/* One 3x3 convolution with zero padding (a single layer of the network, for
 * testing and tuning): x device float [N][H][W][cin], w HOST float
 * [cout][3][3][cin], b HOST float [cout], out device float [N][H][W][cout];
 * relu != 0 applies max(0, .).  precision MRS_PREC_FP32 computes in FP32;
 * MRS_PREC_BF16 / MRS_PREC_FP8 round x and w to the operand type and
 * accumulate in FP32 on the tensor cores (cout <= 64; cin <= 64 for FP8,
 * cin <= 1024 for BF16: past 64 input channels one launch accumulates the
 * 64-channel chunks in tensor memory). */
mrs_status mrs_conv3x3(const float* x, int32_t N, int32_t H, int32_t W, int32_t cin,
                       int32_t cout, const float* w, const float* b, int32_t relu,
                       int32_t precision, float* out, void* stream);

/* Tuning of the tensor-core convolution (for autotuners; no paper
 * counterpart): the depth of its ring of input rows in shared memory,
 * i.e. how many rows the TMA producer may load ahead of the MMAs, for every
 * later launch in the process.  0 (the default) takes the most that fits
 * the shared memory beside the weights and staging slots; 3 .. 12 asks for
 * that many (capped at what fits).  Results do not depend on it. */
mrs_status mrs_conv_set_ring(int32_t stages);

/* Training loss of mrs_train_step (a property of the net, default
 * MRS_LOSS_L1LOG):
 *   MRS_LOSS_L1LOG  mean |slog(y) - slog(t)|, slog(x) = sign(x) log(1 + |x|)
 *                   (L1 on log(1 + radiance), extended oddly below 0)
 *   MRS_LOSS_ROBUST the robust loss l_r of Sec. 3 ("Loss function"): mean over
 *                   pixel-channel values of |y - t| / (beta + |y - t|); the
 *                   paper uses beta = 0.1
 * with t the target clipped at 100 in both cases.  beta must be positive and
 * finite (ignored by MRS_LOSS_L1LOG).  Host-side setting, no device work. */
#define MRS_LOSS_L1LOG 0
#define MRS_LOSS_ROBUST 1
mrs_status mrs_net_set_loss(mrs_net net, int32_t loss, float beta);

/* Weight and bias gradients of one 3x3 convolution with zero padding (the
 * backward pass of mrs_conv3x3 with respect to its parameters, the training
 * step's contraction): x device float [N][H][W][cin], dy device float
 * [N][H][W][cout] (the gradient of the output), dw HOST float
 * [cout][3][3][cin] = sum over pixels of dy[p][o] * x[p + (ky-1, kx-1)][c]
 * (zero outside the image), db HOST float [cout] = sum over pixels of
 * dy[p][o].  cin, cout in [1, 64].  MRS_PREC_FP32 computes in FP32 on the
 * SIMT cores; MRS_PREC_BF16 rounds x and dy to BF16 and accumulates in FP32
 * on the tensor cores.  Partial sums are reduced in a fixed order
 * (deterministic).  Synchronises `stream`; MRS_ERR_TIMEOUT if a device wait
 * gave up. */
mrs_status mrs_conv3x3_wgrad(const float* x, const float* dy, int32_t N, int32_t H, int32_t W,
                             int32_t cin, int32_t cout, int32_t precision, float* dw, float* db,
                             void* stream);

/* Input gradient of one 3x3 convolution with zero padding (the transposed
 * convolution of the training step's backward pass), with the three
 * epilogues that step applies:
 *   g[p][c] = sum over o, ky, kx of dy[p - (ky - 1, kx - 1)][o] * w[o][ky][kx][c]
 *             (zero outside the image)
 *   MRS_DGRAD_LINEAR     out = g
 *   MRS_DGRAD_RELU_MASK  out = aux > 0 ? g : 0   (aux = the ReLU output the
 *                        gradient flows back through)
 *   MRS_DGRAD_RESIDUAL   out = aux + g          (aux = the gradient already
 *                        reaching this tensor along a residual skip)
 * dy device float [N][H][W][cout]; w HOST float [cout][3][3][cin] (the forward
 * layer's weights); aux device float [N][H][W][cin] (NULL for
 * MRS_DGRAD_LINEAR); out device float [N][H][W][cin].  cin, cout in
 * [1, 64]; N*H*W <= 2^26.  MRS_PREC_FP32 runs the FP32 step's SIMT
 * transposed conv; MRS_PREC_BF16 the BF16 step's tensor-core one: dy, w and
 * aux rounded to BF16, FP32 accumulation, the result rounded to BF16 (as the
 * step stores it) and returned widened to float.  For testing each backward
 * layer of mrs_train_step on its own.  Synchronises `stream`;
 * MRS_ERR_TIMEOUT if a device wait gave up. */
#define MRS_DGRAD_LINEAR 0
#define MRS_DGRAD_RELU_MASK 1
#define MRS_DGRAD_RESIDUAL 2
mrs_status mrs_conv3x3_dgrad(const float* dy, int32_t N, int32_t H, int32_t W, int32_t cin,
                             int32_t cout, const float* w, int32_t mode, const float* aux,
                             int32_t precision, float* out, void* stream);

/* ------------------------------------------------------------------------
 * The method's own fusion network (Sec. 4, Fig. network): a two-encoder-one-
 * decoder network that works at the LRHS resolution.
 *   F_LRHS = ReLU(H_lrhs(I_LRHS))            3x3 conv 3 -> 64 at h x w
 *   F0_HRLS = ReLU(H_hrls(I_HRLS))           3x3 conv C_h -> 64 at H x W
 *   F_HRLS = DSF^D(F0_HRLS)                  D = log2(scale) deshuffle layers
 *                                            (stride 2, no weights)
 *   F_0 = ReLU(fuse(F_LRHS || F_HRLS))       1x1 conv 64 + 64 scale^2 -> 64
 *   F_g = RDB_5(...RDB_1(F_{g-1})) + F_{g-1} g = 1..3 (Eq. RDG)
 *   F_DF = F_3 + F_0                         (Eq. F_DF)
 *   I_SR = H_Rec(UP(F_DF))                   UP: D x (3x3 conv 64 -> 256 +
 *                                            ReLU, shuffle x2); H_Rec 3x3
 *                                            conv 64 -> 3
 * A residual dense block RDB has three dense 3x3 convs (64 c -> 64 over the
 * concatenation [F_in, F_1 .. F_{c-1}], ReLU) and a 3x3 local-fusion conv
 * (256 -> 64, ReLU); RDB(F_in) = F_in + fusion.  I_HRLS = HRLS RGB, albedo,
 * normal (C_h = 9) or those plus diffuse, specular and log(1 + variance)
 * (C_h = 18).  Deshuffle channel 4c + 2dy + dx holds input channel c of
 * pixel (2y + dy, 2x + dx); the shuffle is its inverse.
 * Parameters (float32, HOST): for each conv in the order above (H_lrhs,
 * H_hrls, fuse, per group per block convs 1-4, the D upsampling convs,
 * H_Rec) the weight [Cout][k][k][Cin] then the bias [Cout]; count from
 * mrs_rdn_nparams.
 * ------------------------------------------------------------------------ */
typedef struct mrs_rdn_s* mrs_rdn;
/* Parameter count for scale in {2, 4, 8} and hr_channels in {9, 18}. */
mrs_status mrs_rdn_nparams(int32_t scale, int32_t hr_channels, int64_t* n);
/* Copies the parameters in (FP32 master copy and packed BF16 tensor-core
 * weights); n_params must equal mrs_rdn_nparams(scale, hr_channels). */
mrs_status mrs_rdn_create(int32_t scale, int32_t hr_channels, const float* params,
                          int64_t n_params, mrs_rdn* out);
mrs_status mrs_rdn_free(mrs_rdn rdn);
/* I_SR of N frames.  lrhs device [N][H/scale][W/scale][3]; hrls, albedo,
 * normal device [N][H][W][3]; extra device [N][H][W][9] (diffuse, specular,
 * variance as mrs_render_layers writes them) exactly when hr_channels = 18,
 * else NULL; out device [N][H][W][3].  precision MRS_PREC_FP32 (SIMT,
 * reference precision) or MRS_PREC_BF16 (tensor cores: BF16 activations and
 * weights, FP32 accumulation, a conv over more than 64 input channels
 * accumulates its 64-channel chunks in FP32).  Workspace lives in the handle
 * (grown on demand).  Limit: N*H*W <= 2^26. */
mrs_status mrs_rdn_fuse(mrs_rdn rdn, const float* lrhs, const float* hrls, const float* albedo,
                        const float* normal, const float* extra, int32_t N, int32_t H, int32_t W,
                        int32_t precision, float* out, void* stream);
/* MRS_ERR_TIMEOUT (and the error word cleared) if a tensor-core wait of an
 * earlier mrs_rdn_fuse gave up; synchronises the device. */
mrs_status mrs_rdn_check(mrs_rdn rdn);

/* One training step of the network (Sec. 4 "Implement details": trained
 * with Adam; the loss l_r of Sec. 3 "Loss function", or the L1-log loss):
 * the forward of mrs_rdn_fuse keeping every block's concatenation and every
 * ReLU output, the loss of I_SR against min(target, 100) (firefly clipping of
 * the training target, Sec. 3.2; the inputs are used as given) over N*H*W*3
 * values reduced in float64, the backward of every step in reverse
 * (transposed convolutions with flipped taps, ReLU masks from the stored
 * outputs, deshuffle / shuffle exchanged, the dense concatenations' gradients
 * summed per part, the block, group and Eq. F_DF skips adding theirs; dW / db
 * reduced in a fixed order), and one bias-corrected Adam update (beta1 0.9,
 * beta2 0.999, eps 1e-8) of the FP32 weights at learning rate lr (>= 0).
 * precision:
 *   MRS_PREC_FP32  SIMT, the same forward arithmetic in the same order as
 *                  mrs_rdn_fuse's FP32 path (`out` equals it bit for bit)
 *   MRS_PREC_BF16  tensor cores: the BF16 forward (a block's output is its
 *                  input plus its local-fusion ReLU output summed in FP32 and
 *                  rounded once, so not bit-equal to mrs_rdn_fuse's BF16
 *                  output), input gradients as convolutions with the
 *                  transposed, tap-flipped BF16 weights, weight gradients per
 *                  64 x 64 tile reduced in FP32, BF16 activation gradients
 * Images as in mrs_rdn_fuse plus target device [N][H][W][3].  loss one of
 * MRS_LOSS_L1LOG / MRS_LOSS_ROBUST (beta > 0 for the latter).  out (device
 * [N][H][W][3], may be NULL) receives I_SR of the forward; loss_out (HOST,
 * may be NULL) the mean loss, which synchronises `stream` (and then
 * MRS_ERR_TIMEOUT if a BF16 step's tensor-core wait gave up).  The first step
 * allocates the gradient and Adam moments (3 x n_params floats, moments
 * zero); the workspace (FP32: about 20 KB per LR pixel plus 1.3 KB per HR
 * pixel; BF16: about 11 KB per LR pixel plus 0.8 KB per HR pixel) lives in
 * the handle.  A later MRS_PREC_BF16 mrs_rdn_fuse repacks its BF16 weights
 * from the updated FP32 ones.  A BF16 step copies the batch into the
 * handle's staging buffers; the first step of a shape (N, H, W, loss, beta)
 * runs its launches directly and records them as a CUDA graph that later
 * steps of that shape replay (bit-identical; not while mrs_profile_enable is
 * on).  Limit: N*H*W <= 2^24. */
mrs_status mrs_rdn_train_step(mrs_rdn rdn, const float* lrhs, const float* hrls,
                              const float* albedo, const float* normal, const float* extra,
                              const float* target, int32_t N, int32_t H, int32_t W, int32_t loss,
                              float beta, float lr, int32_t precision, float* out,
                              double* loss_out, void* stream);
/* The gradient of the last training step (HOST float [n_params], parameter
 * layout).  MRS_ERR_ARG before the first step.  Synchronises the device. */
mrs_status mrs_rdn_get_grads(mrs_rdn rdn, float* grads, int64_t n_params);
/* Training state: FP32 weights, Adam moments (HOST float [n_params] each;
 * adam_m / adam_v may be NULL, and read as zero before the first step) and
 * the Adam step count (may be NULL).  set_state with NULL moments zeroes
 * them.  Both synchronise the device. */
mrs_status mrs_rdn_get_state(mrs_rdn rdn, float* params, float* adam_m, float* adam_v,
                             int64_t n_params, int64_t* step);
mrs_status mrs_rdn_set_state(mrs_rdn rdn, const float* params, const float* adam_m,
                             const float* adam_v, int64_t n_params, int64_t step);

#ifdef __cplusplus
}
#endif
#endif /* MRS_H */
