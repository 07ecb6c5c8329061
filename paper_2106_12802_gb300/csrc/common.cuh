// Shared helpers of the CUDA library: status mapping, error detail, the
// scene handle layout, and the float3 algebra used by the renderer kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/mrs.h"

#include <atomic>

namespace mrs {

void set_error(const char* fmt, ...);

// number of kernels this library has launched (process-wide)
std::atomic<unsigned long long>& launch_counter();
#define MRS_LAUNCHED(n) (::mrs::launch_counter().fetch_add((n), std::memory_order_relaxed))

// Optional per-kernel CUDA-event timing (off unless mrs_profile_enable(1)):
// events are recorded on the launching stream around each timed launch.
enum ProfKernel {
    PK_TRACE = 0, PK_SHADE, PK_SHADOW, PK_RAYGEN, PK_ACCUM, PK_LBVH, PK_CONV_TC, PK_CONV_SIMT,
    PK_INPUT, PK_METRICS, PK_TRAIN, PK_WGRAD_TC, PK_TAIL, PK_COUNT
};
bool prof_on();
cudaEvent_t prof_record(cudaStream_t st);
void prof_push(int kernel, cudaEvent_t a, cudaEvent_t b);
#define MRS_TIMED(kid, st, ...)                                             \
    do {                                                                    \
        cudaEvent_t _mrs_a = ::mrs::prof_on() ? ::mrs::prof_record(st) : nullptr; \
        __VA_ARGS__;                                                        \
        if (_mrs_a) ::mrs::prof_push((kid), _mrs_a, ::mrs::prof_record(st)); \
    } while (0)

inline mrs_status cuda_status(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return MRS_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MRS_ERR_OOM : MRS_ERR_CUDA;
}

#define MRS_CHECK(call)                                                     \
    do {                                                                    \
        mrs_status _s = ::mrs::cuda_status((call), #call);                  \
        if (_s != MRS_OK) return _s;                                        \
    } while (0)

#define MRS_ARG(cond, msg)                                                  \
    do {                                                                    \
        if (!(cond)) {                                                      \
            ::mrs::set_error("invalid argument: %s", msg);                  \
            return MRS_ERR_ARG;                                             \
        }                                                                   \
    } while (0)

// Device buffer that grows on demand (never shrinks until freed).
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    mrs_status ensure(size_t need)
    {
        if (need <= bytes) return MRS_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (need == 0) return MRS_OK;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) { p = nullptr; return cuda_status(e, "cudaMalloc"); }
        bytes = need;
        return MRS_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// SM count of the current device, looked up once per device (every thread
// that races on a first lookup stores the same value)
inline int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace mrs

namespace mrs {
// what a captured tree-build graph depends on besides the scene's own arrays
struct BuildKey {
    int n = -1, ns = -1, tree = -1;
    void* sort_buf = nullptr;
    void* ploc_buf = nullptr;
    bool operator==(const BuildKey& o) const
    {
        return n == o.n && ns == o.ns && tree == o.tree && sort_buf == o.sort_buf &&
               ploc_buf == o.ploc_buf;
    }
};
}  // namespace mrs

// Scene handle: triangle soup, materials, lights, camera and the LBVH, all
// resident on the device, plus the render arena.
struct mrs_scene_s {
    int n = 0, n_mats = 0, n_lights = 0;
    float env[3] = {0, 0, 0};
    float cam[12] = {0};
    // inputs (input order)
    float* V = nullptr;          // [n][9]
    int* tri_mat = nullptr;      // [n]
    int* tri_light = nullptr;    // [n]
    float* mats = nullptr;       // [n_mats][8]
    float* lights = nullptr;     // [n_lights][12]
    // LBVH
    uint32_t* morton = nullptr;  // [n] input order
    uint32_t* skeys = nullptr;   // [n] sorted codes
    int* order = nullptr;        // [n] position -> triangle: BVH leaves 0..ns-1, large ns..n-1
    int ns = 0;                  // triangles in the LBVH (the rest are tested exhaustively)
    int* small_idx = nullptr;    // [ns] triangles of the LBVH, in input order
    int* big_idx = nullptr;      // [n - ns] large triangles, in input order
    int* left = nullptr;         // [n-1]
    int* right = nullptr;        // [n-1]
    int* parent = nullptr;       // [2n-1]
    int* visit = nullptr;        // [n-1]
    float* box = nullptr;        // [2n-1][6]
    float4* nodes = nullptr;     // [n-1][4]: child boxes + child ids
    float4* tris = nullptr;      // [n][3]: (v0, prim bits), (e1, 0), (e2, 0) in sorted order
    int2* tri_ml = nullptr;      // [n]: material, light in sorted order
    mrs::Buf sort_tmp;           // radix-sort scratch
    mrs::Buf ploc_tmp;           // clustering-build scratch
    cudaGraphExec_t build_exec = nullptr;  // the tree build as one graph (see build_lbvh)
    mrs::BuildKey build_key;               // ... for these sizes, tree kind and buffers
    int build_kernels = 0;                 // ... holding this many kernels
    cudaStream_t cap_stream = nullptr;     // stream the graph is captured on
    int32_t tree = MRS_TREE_LBVH;          // render tree to build (MRS_TREE_*)
    int32_t tree_built = MRS_TREE_LBVH;    // the one built (the LBVH if clustering gave up)
    mrs::Buf class_tmp;          // large / small classification scratch
    int* class_host = nullptr;   // pinned [2]: small and large triangle counts
    mrs::Buf export_tmp;         // full-scene LBVH built on export
    mrs::Buf arena;              // render path state
    int64_t wave_paths = int64_t(1) << 24;
    int32_t tail_bounce = -1;    // first bounce of the tail kernel (-1: bounce 1)
};

// Render context: a path-state arena of its own, so that several renders of
// the same scene can run concurrently on different streams.
struct mrs_ctx_s {
    mrs::Buf arena;
    int64_t wave_paths = int64_t(1) << 24;
    int32_t tail_bounce = -1;
};

// Layout of the render arena for a wave of P paths (floats unless noted).
namespace mrs {
struct PathSoA {
    float *ox, *oy, *oz, *dx, *dy, *dz;   // ray
    float *bx, *by, *bz;                  // throughput
    float *Lx, *Ly, *Lz;                  // path radiance
    float *pdf_b, *pdf_e;                 // MIS pdfs of the last BSDF sample
    float* hit_t;
    int* hit_id;                          // sorted leaf position or -1
    float *sdx, *sdy, *sdz, *stmax;       // shadow ray direction and extent
    float *scx, *scy, *scz;               // unoccluded shadow contribution
    float *ax, *ay, *az, *nx, *ny, *nz, *dep;   // first-hit aux
    int* lobe;                            // first-hit lobe (1 Lambertian, 2 GGX, 0 none); layers only
    int *q0, *q1, *qs;                    // queues (cur / next / shadow)
};
}  // namespace mrs
