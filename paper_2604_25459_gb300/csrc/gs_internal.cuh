// Internal declarations shared by the CUDA translation units of libgsbatch.
//
// Device data layout (all in HBM):
//   Gaussians (scene-owned), background first (in the scene's Morton storage
//   order of the means) then link-major (storage index g):
//     p0[g] = {mean.x, mean.y, mean.z, opacity}
//     p1[g] = {F00, F01, F02, F10}      F = R diag(exp(s)), the factor of the 3D
//     p2[g] = {F11, F12, F20, F21}      covariance F F^T in the frame the mean lives
//     p3[g] = {F22, qstar, tr, link}    in (world for the background, link frame for
//                                       link Gaussians); qstar = 2 ln(255 o) (< 0
//                                       culls), tr = trace(F F^T), link = 0 for the
//                                       background, l+1 for link l (int bits)
//     sh plane-major: plane p holds values 4p..4p+3 (f32) or 8p..8p+7 (bf16/f16)
//     of the flattened [coefficient][channel] vector, for every g: sh[p][g].
//   Per wave of envs (scratch), env el described by EnvInfo envs[el]:
//     record slots: local index j = g for background Gaussians (padded to a
//       multiple of 32), then the env's link Gaussians in storage order; slot
//       (el, j) is slot s = envs[el].rec_base + j, valid where bit j%32 of
//       mask[envs[el].mask_base + j/32] is set; its first three 16-byte words
//       r0, r1, r2 lie side by side at float4 index kRecStride s of one array
//       (the compositor gathers all three: two 32-byte sectors instead of
//       three half-used ones), its fourth word r3 at index s of another (the
//       binning reads only r3, coalesced across a warp).  Keys are (depth bits << 32 |
//       i) with i the caller's local index (background: its index before the
//       Morton reordering; links: j), so equal depths order by global index;
//       the compositor maps i back to the record slot j.
//     xf[envs[el].xf_base + f]  frame f = 0 background, f = 1 + (l - link_begin)
//     counts/off_local/cursor[envs[el].tile_base + t]  per (env, tile)
//     env_base[el]              exclusive scan of per-env intersection totals
//     pairs[...]                u64 keys bucketed by (env, tile)
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gsbatch.h"

namespace gsb {

// float4 stride between the r0 (r1, r2) words of consecutive record slots
// (r1 = r0 + 1, r2 = r0 + 2 in one array; see the layout above)
constexpr int kRecStride = 3;

// Stores the r0, r1, r2 words of a warp's 32 consecutive record slots
// (slot0 = the slot of lane 0) from the warp's staging buffer st (96 float4:
// word w of lane l at 3 l + w), with coalesced stores: lane l writes float4
// l, l + 32 and l + 64 of the slots' interleaved region, each where its record
// ((l + 32 k) / 3) is visible in m.  Direct per-lane stores at the 48-byte
// stride would write half sectors.  Call with every lane of the warp, after
// the lanes' staging writes and a __syncwarp().
__device__ __forceinline__ void store_records(float4* r0, size_t slot0, const float4* st, uint32_t m, int lane) {
    static_assert(kRecStride == 3, "three 16-byte words per record slot");
    float4* dst = r0 + (size_t)kRecStride * slot0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = lane + 32 * k;
        if ((m >> (i / 3)) & 1u) dst[i] = st[i];
    }
}

enum : uint32_t {
    kStBadPose = 1u,     // zero or non-finite link pose quaternion
    kStBadScene = 2u,    // zero or non-finite Gaussian quaternion at scene build
    kStOverflow = 4u,    // intersection keys beyond the capacity (planned launches) or a corrupted bucket
    kStBadRay = 8u,      // a ray direction outside its sensor's binning grid (or zero)
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

// One environment of a wave.
struct EnvInfo {
    unsigned long long rec_base;   // first record slot
    unsigned long long mask_base;  // first visibility word
    unsigned long long pix_base;   // first pixel of the env's image in the outputs
    long long pose_base;           // index (units of 7 floats) of the pose of link_begin
    unsigned int tile_base;        // first (env, tile) counter of the wave
    unsigned int n_local;          // record slots: padded background + the env's link Gaussians
    int xf_base;                   // first link-table entry
    int link_begin, n_links;       // links of the scene rendered in this env
    int W, H, ntx, T;              // image and tile grid
    int pad;
    long long g_link0;             // storage (= caller's) index of the env's first link Gaussian (slot bg_slots)
    float lim[4];                  // camera guard band: 1.3 cx/fx, 1.3 (W-cx)/fx, 1.3 cy/fy, 1.3 (H-cy)/fy
};

// A projection block: up to 256 consecutive Gaussians (thread t takes global
// index g_first + t, record slot local_first + t) for envs [e0, e1) of a wave;
// link frame of Gaussian with link field li is xf[envs[e].xf_base + li - lb].
struct ProjBlock {
    long long g_first;
    unsigned int local_first;  // multiple of 32
    int n;
    int e0, e1;
    int lb;
    int frame0;  // 1: every Gaussian of the block is background (link frame 0)
};

struct ProjParams {
    int64_t n_gauss;  // SH plane stride
    const float4* p0;
    const float4* p1;
    const float4* p2;
    const float4* p3;
    const void* sh;
    const ProjBlock* blocks;
    const EnvInfo* envs;
    const gs_camera* cams;  // per env of the wave
    const LinkXf* xf;
    float4* r0;
    float4* r1;
    float4* r2;
    uint4* r3;
    uint32_t* mask;
    float2* dbg_hxy;  // nullable, per record slot
    unsigned long long* nvis;  // nullable: visible (env, Gaussian) pair counter
    unsigned long long* nfp64; // nullable: counter of (env, Gaussian) pairs whose conic took the FP64 branch
    const gs_lidar* lidars;    // LiDAR projection only: per env of the wave
    const int* bg_index;       // nullable: caller's index of the background Gaussian in slot j (into r3.w)
    float cell_pad;            // LiDAR: grid boxes widened by this many cells (arbitrary rays: a ray
                               // anywhere in a cell, not only at its centre)
};

struct BinParams {
    const EnvInfo* envs;
    const uint32_t* mask;
    const uint4* r3;
    int e_begin;             // first env (wave-local) handled by this launch
    int tile_w, tile_h;
    int words_per_block;
    uint32_t* counts;
    const uint32_t* off_local;
    const unsigned long long* env_base;
    unsigned long long pair_base;   // env_base[e_begin], subtracted from absolute offsets
    unsigned long long pair_cap;    // keys the pair buffer holds
    uint32_t* cursor;
    unsigned long long* pairs;
    uint32_t* status;
    // Keys carry the caller's local index of the Gaussian, so equal depths
    // order by it: camera records hold it in r3.w (index_in_r3), LiDAR
    // records are mapped through bg_index (nullable: caller's index of the
    // background Gaussian in storage slot j < n_bg)
    int index_in_r3;
    const int* bg_index;
    unsigned int n_bg;
    int wrap;  // LiDAR: a box with x0 > x1 covers columns [x0, cols) and [0, x1]
    // nullable, per env of the wave: (smallest depth bits, ~largest depth bits)
    // of the env's visible records, taken by the count pass with atomicMin on
    // both words (set to all ones before it)
    uint2* zr;
};

struct CompParams {
    const EnvInfo* envs;
    int e_begin, e_end;              // envs of this launch (wave-local)
    unsigned int item_begin, item_end;  // (env, tile) items: envs[e_begin].tile_base .. envs[e_end].tile_base
    int chunk;                       // items claimed per atomic
    unsigned int* work;              // work counter (zeroed before the launch)
    const float4* r0;
    const float4* r1;
    const float4* r2;
    // nullable, per env of the wave: the depth-bit range of its keys (see
    // BinParams::zr); long buckets are partitioned over it instead of over
    // their own key range, which saves a pass over their keys
    const uint2* zr;
    const uint32_t* counts;
    const uint32_t* off_local;
    const unsigned long long* env_base;
    unsigned long long pair_base;
    unsigned long long pair_cap;
    const unsigned long long* pairs;
    unsigned long long* spill;       // nullable: spill_cap keys per CTA for partitioning long buckets
    unsigned int spill_cap;          // kCompCap <= spill_cap <= kSpillMax
    unsigned int spill_ctas;         // regions in spill: the launch uses at most this many CTAs
    unsigned long long* dbg_sorted;  // nullable: receives the full depth-ordered lists
    unsigned long long* neval;       // nullable: composited (pixel, Gaussian) pair counter
    int tile_w, tile_h;
    int quad;       // 16x16 or 8x8 camera tiles: per-quadrant splat lists (k_composite's QUAD form)
    float* rgb;     // images at envs[e].pix_base (x3 for rgb); unused when rgb8 is set
    float* depth;   // unused when depth16 is set
    float* alpha;   // nullable
    uint8_t* rgb8;        // nullable: observation RGB, 8 bits per channel, at pix_base (x3)
    uint16_t* depth16;    // nullable: observation depth, IEEE half bits, at pix_base
    const gs_appearance* appear;  // nullable: per env (wave-local index) for rgb8
    float* score;         // nullable: contribution pass (no images): score[g] += sum of alpha T
    unsigned int nbp;     // background slots (slot j < nbp is the background Gaussian stored at j)
    const int* bg_index;  // nullable: caller's index of the background Gaussian in slot j (contribution pass)
    const int* bg_slot;   // nullable: keys carry the caller's background index i < n_bg; its record slot is bg_slot[i]
    unsigned int n_bg;
    const gs_lidar* lidars;  // nullable: LiDAR scan (range in depth, hit in alpha), per env of the wave
    const uint4* r3;         // LiDAR scan: records' fourth word (|g2|)
    uint32_t* status;
    // Arbitrary rays (set with lidars): items are (env, tile, chunk of <= 256
    // rays); outputs are indexed by ray, at envs[e].pix_base + ray.
    const float* ray_dirs;         // [wave env][n_rays][3], sensor frame
    const uint32_t* ray_cell;      // [wave env][n_rays]: tile << 8 | cell in tile (row-major 16x16)
    const uint32_t* ray_list;      // [wave env][n_rays]: ray indices grouped by tile
    const uint32_t* ray_cnt;       // per (env, tile) at tile_base: rays in the tile
    const uint32_t* ray_off;       // per (env, tile): first entry of the tile in the env's ray_list
    const uint32_t* item_off;      // per (env, tile): first item of the tile within its env
    const unsigned long long* item_base;  // per wave env (+1): first item of the env
    int n_rays;
};

// Launchers (return cudaGetLastError()).
// Input Gaussian i is stored at dst_offset + (place ? place[i] : i).
cudaError_t launch_prep(const float* mean, const float* quat, const void* log_scale, const void* opacity,
                        const void* sh, int64_t n, int64_t dst_offset, const int64_t* place, int link_mode,
                        const int64_t* link_offsets, int n_links, const DevGaussians& D, uint32_t* status,
                        cudaStream_t st);
// n_items = sum over envs of (1 + n_links); envs[We].xf_base must hold n_items.
cudaError_t launch_link_table(const float* poses, const gs_camera* cams, const EnvInfo* envs, int We, int n_items,
                              LinkXf* out, uint32_t* status, cudaStream_t st);
cudaError_t launch_project(const DevGaussians& D, const ProjParams& P, int n_blocks, cudaStream_t st);
// LiDAR records: r0 = (b, o), r1 = (g0, x-range), r2 = (g1, y-range), r3 =
// (x-range, y-range, distance bits, |g2| bits) with g_k the rows of
// diag(e^-s) R^T in the sensor frame and b = G mu; ranges over the
// (azimuth, beam) grid.
cudaError_t launch_project_lidar(const ProjParams& P, int n_blocks, cudaStream_t st);
// Arbitrary rays, per wave: the cell of every ray on its sensor's binning
// grid (zero and out-of-grid directions flagged and left out) and the rays per
// (env, tile); then the rays grouped by tile and the compositor's items
// (chunks of at most kRayChunk rays per tile).  ray_cnt and ray_cur are zeroed
// by the caller.
constexpr int kRayChunk = 256;
cudaError_t launch_ray_count(const float* dirs, const gs_lidar* lidars, const EnvInfo* envs, int We, int n_rays,
                             uint32_t* cell, uint32_t* cnt, uint32_t* status, cudaStream_t st);
cudaError_t launch_ray_scatter(const EnvInfo* envs, int We, int n_rays, const uint32_t* cell, const uint32_t* off,
                               uint32_t* cur, uint32_t* list, const uint32_t* cnt, uint32_t* item_cnt,
                               unsigned int tiles, cudaStream_t st);
// grid.x covers the largest env's mask words; max_T sizes the shared histogram
cudaError_t launch_count(const BinParams& P, int n_envs, int max_words, int max_T, cudaStream_t st);
cudaError_t launch_scan(const EnvInfo* envs, const uint32_t* counts, uint32_t* off_local,
                        unsigned long long* env_total, unsigned long long* env_base, int We, cudaStream_t st);
cudaError_t launch_scatter(const BinParams& P, int n_envs, int max_words, int max_T, cudaStream_t st);
// grid = persistent CTAs; returns the grid size used through *ctas
cudaError_t launch_composite(const CompParams& P, cudaStream_t st, int* ctas);
// Most CTAs a compositing launch of this tile shape uses on the current
// device (resident CTAs per SM x SMs): the number of spill regions to provide.
cudaError_t composite_max_ctas(int tile_w, int tile_h, int* ctas);

constexpr int kWordsPerBlock = 256;  // binning block: 8 warps x 32 visibility words (8192 slots)

// Depth-ordered window held in shared memory by the compositor.  Smaller
// windows sort less in tiles that terminate early, larger ones re-scan long
// buckets less often; 768 measured best on the 2048 x 640x480 workload
// (1024: +2 %, 512: +4 %, 2048: +19 % compositing time).
constexpr int kCompCap = 768;
constexpr int kBins = 2048;         // key ranges of the long-bucket partition
constexpr int kSpillMax = 32768;    // keys per CTA in the spill region, at most
// Plain renders use the compositor's quadrant form (QUAD) on 16x16 or 8x8 tiles when
// no image of the wave has more pixels than this (measured crossover on the
// room workload: faster at 320x240 and below, slower at 640x480).
constexpr int kQuadMaxPixels = 320 * 240;

// Read-only view of a scene's device data for entry points outside gs_api.cu.
struct SceneView {
    int device;
    DevGaussians D;
    uint32_t* status;
    int tile_w, tile_h;
    const int* bg_index;  // nullable: caller's index of the background Gaussian in storage slot j
    const int* bg_slot;   // nullable: storage slot of the caller's background Gaussian i
};
SceneView scene_view(gs_scene s);
// Set the thread-local message returned by gs_last_error and return st.
gs_status report(gs_status st, const char* msg);

// Host-side construction of a wave's tables (shared by all entry points).
struct EnvSpec {        // one env as requested by the caller
    const gs_camera* cam;
    int link_begin, link_end;
    long long pose_offset;    // pose index of link_begin
    long long pixel_offset;   // first pixel of the image
};
int64_t bg_slots(int64_t n_bg);  // background slots padded to 32
// Fills envs (n+1 entries; the last holds the totals in rec_base, mask_base,
// tile_base and xf_base) and appends projection blocks; returns totals through
// the EnvInfo sentinel.  link_offsets: host copy of the scene's link offsets.
void build_wave_tables(const DevGaussians& D, const int64_t* link_offsets, const EnvSpec* specs, int n, int tile_w,
                       int tile_h, long long pix_rebase, EnvInfo* envs, ProjBlock* blocks, int* n_blocks,
                       int max_blocks);
int count_wave_blocks(const DevGaussians& D, const int64_t* link_offsets, const EnvSpec* specs, int n);

}  // namespace gsb
