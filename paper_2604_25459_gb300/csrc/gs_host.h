// Host-side internals of libgsbatch shared by its C ABI translation units
// (gs_api.cu: scenes, renders and plans; gs_server.cu: the request loop):
// error reporting, device buffers, the scene object and the launch of one
// wave of environments.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gs_internal.cuh"

namespace gsb {

// The calling thread's last error message (what gs_last_error() returns).
extern thread_local std::string g_err;

// Records a printf-style message for gs_last_error() (per thread) and returns st.
gs_status fail(gs_status st, const char* fmt, ...);
// A CUDA error as GS_ERR_OOM (allocation) or GS_ERR_CUDA, recorded like fail().
gs_status cuda_fail(cudaError_t e, const char* what);

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)
#define ST(call)                        \
    do {                                \
        gs_status s_ = (call);          \
        if (s_ != GS_OK) return s_;     \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t need) {
        if (need == 0) need = 16;
        if (need <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, need);
        if (e == cudaSuccess) bytes = need;
        else p = nullptr;
        return e;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// Device scratch of a render: one set per scene (eager calls) and one per plan.
struct Scratch {
    DevBuf envs, blocks, cams, xf, r012, r3, mask, counts, off, cursor, env_total, env_base, pairs, dbg_hxy,
        dbg_sorted, work, spill, zr;  // r012: records' r0, r1, r2 interleaved (kRecStride); zr: depth ranges
    DevBuf* all[18] = {&envs,   &blocks,    &cams,     &xf,    &r012,   &r3,         &mask, &counts, &off,
                       &cursor, &env_total, &env_base, &pairs, &dbg_hxy, &dbg_sorted, &work, &spill, &zr};
    void release() {
        for (DevBuf* b : all) b->release();
    }
    int64_t bytes() const {
        int64_t n = 0;
        for (const DevBuf* b : all) n += (int64_t)b->bytes;
        return n;
    }
};

// Tile shapes the compositor is built for.
bool valid_tile(int tw, int th);

}  // namespace gsb

struct gs_scene_s {
    int device = 0;
    gsb::DevGaussians D;
    gsb::DevBuf g0, g1, g2, g3, gsh;
    std::vector<int64_t> link_offsets{0};  // host copy, n_links + 1 entries
    bool have_format = false;               // dtype / degree fixed by the first non-empty set
    uint32_t* status = nullptr;
    int tile_w = 16, tile_h = 16;
    int64_t budget = 64ll << 30;
    int max_wave = 0;
    int debug = 0;
    gsb::Scratch sc;
    gsb::DevBuf stage_rgb[2], stage_depth[2], stage_alpha[2], poses;
    unsigned long long* pinned = nullptr;
    size_t pinned_n = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    // host tables of the last wave (debug hooks)
    std::vector<gsb::EnvInfo> last_envs;
    int last_e0 = -1, last_We = 0, last_ea = 0, last_eb = 0;
    unsigned long long last_pair_base = 0;
    gs_stats stats{};
    // profiling (per-phase CUDA events on the render stream) and counters
    int profile = 0;
    struct Mark {
        int phase;
        int kernels;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[GS_PHASES] = {0};
    int64_t prof_launches[GS_PHASES] = {0};
    int counters = 0;
    gsb::DevBuf neval;
    gsb::DevBuf appear;  // appearance parameters copied from the host (observation form)
    gsb::DevBuf lidar_tab;  // the current wave's LiDAR sensors
    // arbitrary-ray scans: per ray its cell, the rays grouped by tile, per
    // (env, tile) ray counts, offsets, cursors, item counts and offsets, per
    // env the scans' totals and bases
    gsb::DevBuf ray_cell, ray_list, ray_cnt, ray_off, ray_cur, item_cnt, item_off, ray_tot, ray_base, item_tot,
        item_base;
    // storage order of the background: bg_order[k] is the caller's index of
    // the background Gaussian stored at position k; device copies of it
    // (bg_index) and of its inverse (bg_slot), int32
    std::vector<long long> bg_order;
    gsb::DevBuf bg_index, bg_slot;
    // host staging of tables
    std::vector<gsb::EnvInfo> h_envs;
    std::vector<gsb::ProjBlock> h_blocks;
    std::vector<gs_camera> h_cams;
};

namespace gsb {

struct WaveIO {
    const float* poses;   // device, indexed by the specs' pose offsets
    float* rgb;           // device outputs, indexed by pixel offsets minus pix_rebase
    float* depth;
    float* alpha;
    long long pix_rebase;
    uint32_t* status = nullptr;  // device status word of this wave (NULL: the scene's)
    uint8_t* rgb8 = nullptr;     // observation form (replaces rgb / depth when set)
    uint16_t* depth16 = nullptr;
    const gs_appearance* appear = nullptr;  // device, indexed by the wave's env
    float* score = nullptr;      // contribution pass (no images)
    const gs_lidar* lidars = nullptr;  // LiDAR scan: device table of the wave's sensors
    const float* ray_dirs = nullptr;   // with lidars: arbitrary rays [wave env][n_rays][3] (sensor frame)
    int n_rays = 0;
};

struct WaveTables {       // device copies of one wave's tables
    const EnvInfo* envs;
    const ProjBlock* blocks;
    const gs_camera* cams;
    int We, n_blocks, xf_items, max_words, max_T;
    unsigned long long recs, words, tiles;
    const EnvInfo* host_envs;  // We + 1 host entries
};

// Validates one camera (env index e for the message).
gs_status check_cam(const gs_camera& c, int e);

// Fixed scratch bytes of one env (records, visibility, tile counters, link table).
size_t env_bytes(gs_scene s, const EnvSpec& sp, int tw, int th, bool debug);

// Builds the tables of specs[e0, e1) and uploads them into the given device
// buffers on st (synchronously when sync_copy).
gs_status upload_tables(gs_scene s, const std::vector<EnvSpec>& specs, int e0, int e1, int tw, int th,
                        long long pix_rebase, DevBuf& d_envs, DevBuf& d_blocks, DevBuf& d_cams, cudaStream_t st,
                        bool sync_copy, WaveTables* wt);

// Launches one wave on st: link table, projection, binning, compositing.
// cap == 0: eager (reads the intersection totals back, grows the key buffer);
// cap > 0: planned (no host sync; keys beyond cap dropped and flagged).
// quad: the compositor's quadrant form on 16x16 or 8x8 camera tiles: 1 on,
// 0 off, -1 when no image of the wave exceeds kQuadMaxPixels.
gs_status run_wave(gs_scene s, Scratch& sc, const WaveTables& wt, const WaveIO& io, int tw, int th, int chunk,
                   unsigned long long cap, cudaStream_t st, bool timers, int64_t* launches,
                   unsigned long long* total_out, int quad = -1);

}  // namespace gsb
