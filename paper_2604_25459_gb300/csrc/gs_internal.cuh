// Internal declarations shared by the CUDA translation units of libgsbatch.
//
// Device data layout (all in HBM, owned by the scene):
//   Gaussians, background first then link-major (global index g):
//     p0[g] = {mean.x, mean.y, mean.z, opacity}
//     p1[g] = {F00, F01, F02, F10}      F = R diag(exp(s)), the factor of the 3D
//     p2[g] = {F11, F12, F20, F21}      covariance F F^T in the frame the mean lives
//     p3[g] = {F22, qstar, tr, link}    in (world for the background, link frame for
//                                       link Gaussians); qstar = 2 ln(255 o) (< 0
//                                       culls), tr = trace(F F^T), link = 0 for the
//                                       background, l+1 for link l (int bits)
//     sh plane-major: plane p holds values 4p..4p+3 (f32) or 8p..8p+7 (bf16/f16)
//     of the flattened [coefficient][channel] vector, for every g: sh[p][g].
//   Per wave of envs (local env index el, G Gaussians, T tiles):
//     xf[el][L+1]        link transforms composed with the camera (+ camera
//                        centre in the link frame for the SH view direction)
//     r0..r3[el*G + g]   projected record of (el, g), valid where the bit is set in
//     mask[el][g/32]     (bit g%32)
//     counts[el][t], off_local[el][t], cursor[el][t]   per (env, tile) intersections
//     env_base[el]       exclusive scan of per-env intersection totals (+ total)
//     pairs[...]         u64 keys (depth bits << 32 | g), bucketed by (env, tile)
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gsbatch.h"

namespace gsb {

enum : uint32_t {
    kStBadPose = 1u,     // zero or non-finite link pose quaternion
    kStBadScene = 2u,    // zero or non-finite Gaussian quaternion at scene build
    kStOverflow = 4u,    // a bucket exceeded what the kernels can address
};

// Row-major rigid transform camera <- frame, plus the camera centre in that frame.
struct __align__(16) LinkXf {
    float4 r0;  // R00 R01 R02 t0
    float4 r1;  // R10 R11 R12 t1
    float4 r2;  // R20 R21 R22 t2
    float4 o;   // camera centre in the frame (x,y,z), unused
};

struct DevGaussians {
    int64_t n = 0;
    int64_t n_bg = 0;
    int n_links = 0;
    int sh_degree = 3;
    gs_dtype dtype = GS_F32;
    int sh_planes = 0;
    float4* p0 = nullptr;
    float4* p1 = nullptr;
    float4* p2 = nullptr;
    float4* p3 = nullptr;
    void* sh = nullptr;  // sh_planes * n * 16 bytes
};

inline int sh_values(int degree) { return 3 * (degree + 1) * (degree + 1); }
inline int sh_planes_for(int degree, gs_dtype dt) {
    int v = sh_values(degree);
    return dt == GS_F32 ? (v + 3) / 4 : (v + 7) / 8;
}

struct ProjParams {
    int64_t G;
    const float4* p0;
    const float4* p1;
    const float4* p2;
    const float4* p3;
    const void* sh;
    const LinkXf* xf;        // [We][L+1]
    const gs_camera* cams;   // [We]
    int L1;                  // n_links + 1
    int We;
    int env_group;
    float4* r0;
    float4* r1;
    float4* r2;
    uint4* r3;
    uint32_t* mask;          // [We][mask_words]
    int64_t mask_words;
    float2* dbg_hxy;         // nullable, [We][G]
};

struct BinParams {
    int64_t G;
    int64_t mask_words;
    const uint32_t* mask;
    const uint4* r3;
    int e_begin;             // first env (wave-local) handled by this launch
    int tile_w, tile_h, ntx, T;
    uint32_t* counts;        // [We][T]
    const uint32_t* off_local;
    const unsigned long long* env_base;
    unsigned long long pair_base;   // env_base[e_begin], subtracted from absolute offsets
    uint32_t* cursor;        // [We][T]
    unsigned long long* pairs;
    int words_per_block;
};

struct CompParams {
    int64_t G;
    const float4* r0;
    const float4* r1;
    const float4* r2;
    const uint32_t* counts;
    const uint32_t* off_local;
    const unsigned long long* env_base;
    unsigned long long pair_base;
    const unsigned long long* pairs;
    unsigned long long* dbg_sorted;  // nullable: receives the full depth-ordered lists
    unsigned long long* neval;       // nullable: composited (pixel, Gaussian) pair counter
    int e_begin;
    int W, H, tile_w, tile_h, ntx, T;
    float* rgb;     // [We][H][W][3] for the wave (env el at el*H*W*3)
    float* depth;
    float* alpha;   // nullable
    uint32_t* status;
};

// Launchers (return cudaGetLastError()).
cudaError_t launch_prep(const float* mean, const float* quat, const void* log_scale, const void* opacity,
                        const void* sh, int64_t n, int64_t dst_offset, int link_of_first, const int64_t* link_offsets,
                        int n_links, const DevGaussians& D, uint32_t* status, cudaStream_t st);
cudaError_t launch_link_table(const float* poses, const gs_camera* cams, int We, int n_links, LinkXf* out,
                              uint32_t* status, cudaStream_t st);
cudaError_t launch_project(const DevGaussians& D, const ProjParams& P, dim3 grid, cudaStream_t st);
cudaError_t launch_count(const BinParams& P, int n_envs, cudaStream_t st, size_t smem);
cudaError_t launch_scan(const uint32_t* counts, uint32_t* off_local, unsigned long long* env_total,
                        unsigned long long* env_base, int We, int T, cudaStream_t st);
cudaError_t launch_scatter(const BinParams& P, int n_envs, cudaStream_t st, size_t smem);
cudaError_t launch_composite(const CompParams& P, int n_envs, cudaStream_t st);

// Depth-ordered window held in shared memory by the compositor.  Smaller
// windows sort less in tiles that terminate early, larger ones re-scan long
// buckets less often; 768 measured best on the 2048 x 640x480 workload
// (1024: +2 %, 512: +4 %, 2048: +19 % compositing time).
constexpr int kCompCap = 768;

// Read-only view of a scene's device data for entry points outside gs_api.cu.
struct SceneView {
    int device;
    DevGaussians D;
    uint32_t* status;
    int tile_w, tile_h;
};
SceneView scene_view(gs_scene s);
// Set the thread-local message returned by gs_last_error and return st.
gs_status report(gs_status st, const char* msg);

}  // namespace gsb
