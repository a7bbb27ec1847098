// gs_render_batch_noalloc: the batched render with its working memory in a
// fixed, file-scope device array instead of memory the library allocates.
//
// Some callers must not allocate device memory while they render: a process
// whose device memory is already handed out to another allocator (a training
// framework that reserved the GPU at start-up), code that runs where a
// cudaMalloc/cudaFree would stall or is not permitted (cudaFree synchronises
// the device; allocation inside host callbacks is forbidden), or a control
// loop that must not take the latency of a first-time allocation.  For them
// this entry point renders with the same kernels as gs_render_batch, but every
// intermediate (link table, projected records, masks, per-tile counts and
// offsets, intersection keys) lives in g_scratch below.
//
// The array is kNoAllocBytes per device, reserved in every process that loads
// the library until it exits.  All calls (from any scene or thread) on one
// device share it, and it keeps whatever the last call left: the counters that
// must start at zero are cleared on the stream by each call, and calls whose
// work overlaps on the GPU (different streams, or threads) race on it.
#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace gsb {
namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;  // 32 MiB of working memory per device
constexpr int kMaxWave = 256;                   // environments per internal wave
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

gs_status failf(gs_status st, const char* fmt, long long a = 0, long long b = 0, long long c = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b, c);
    return report(st, buf);
}

// Device address of g_scratch on the current device, looked up once per device.
// The host-side name g_scratch is only a stand-in: its address must come from
// cudaGetSymbolAddress with the device current.
gs_status scratch_on(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return failf(GS_ERR_UNSUPPORTED, "device %lld out of range", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress(no-allocation scratch): %s", cudaGetErrorString(e));
            return report(GS_ERR_CUDA, buf);
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return GS_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxBlocks = 16384;  // projection blocks per wave (host tables are static too)
EnvSpec h_specs[kMaxWave];
EnvInfo h_envs[kMaxWave + 1];
ProjBlock h_blocks[kMaxBlocks];

struct Layout {
    size_t envs, blocks, cams, xf, r012, r3, mask, counts, off, cursor, env_total, env_base, work, pairs;
};

Layout layout(int We, int nb, int xf_items, unsigned long long recs, unsigned long long words,
              unsigned long long tiles) {
    Layout y{};
    size_t o = 0;
    y.envs = o;      o = up256(o + sizeof(EnvInfo) * ((size_t)We + 1));
    y.blocks = o;    o = up256(o + sizeof(ProjBlock) * (size_t)(nb > 0 ? nb : 1));
    y.cams = o;      o = up256(o + sizeof(gs_camera) * (size_t)We);
    y.xf = o;        o = up256(o + sizeof(LinkXf) * (size_t)xf_items);
    y.r012 = o;      o = up256(o + recs * 16 * kRecStride);
    y.r3 = o;        o = up256(o + recs * 16);
    y.mask = o;      o = up256(o + words * 4);
    y.counts = o;    o = up256(o + tiles * 4);
    y.off = o;       o = up256(o + tiles * 4);
    y.cursor = o;    o = up256(o + tiles * 4);
    y.env_total = o; o = up256(o + (size_t)We * 8);
    y.env_base = o;  o = up256(o + ((size_t)We + 1) * 8);
    y.work = o;      o = up256(o + 16);
    y.pairs = o;
    return y;
}

#define NA_CK(call, what)                                                        \
    do {                                                                         \
        const cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) {                                                 \
            char b_[256];                                                        \
            snprintf(b_, sizeof b_, "%s: %s", what, cudaGetErrorString(e_));     \
            return report(GS_ERR_CUDA, b_);                                      \
        }                                                                        \
    } while (0)

}  // namespace
}  // namespace gsb

using namespace gsb;

extern "C" gs_status gs_render_batch_noalloc(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                             float* rgb, float* depth, float* alpha, void* cuda_stream) {
    if (!s) return report(GS_ERR_INVALID, "null scene");
    if (n_envs < 0) return report(GS_ERR_INVALID, "negative n_envs");
    if (n_envs == 0) return GS_OK;
    if (!cams || !rgb || !depth) return report(GS_ERR_INVALID, "null cams, rgb or depth");
    const SceneView v = scene_view(s);
    const int L = v.D.n_links;
    if (L > 0 && !link_poses) return report(GS_ERR_INVALID, "null link_poses for a scene with links");
    const int W = cams[0].width, H = cams[0].height;
    for (int e = 0; e < n_envs; ++e) {
        const gs_camera& c = cams[e];
        if (c.width != W || c.height != H) return failf(GS_ERR_INVALID, "camera %lld: resolution differs", e);
        if (W < 1 || H < 1 || W > 16384 || H > 16384)
            return failf(GS_ERR_INVALID, "camera %lld: width/height out of [1, 16384]", e);
        if (!(c.fx > 0 && c.fy > 0 && c.near_plane > 0) || !isfinite(c.fx) || !isfinite(c.fy) ||
            !isfinite(c.cx) || !isfinite(c.cy) || !isfinite(c.near_plane))
            return failf(GS_ERR_INVALID, "camera %lld: intrinsics or near plane invalid", e);
        const double qn = (double)c.q_cw[0] * c.q_cw[0] + (double)c.q_cw[1] * c.q_cw[1] +
                          (double)c.q_cw[2] * c.q_cw[2] + (double)c.q_cw[3] * c.q_cw[3];
        if (!(qn > 0) || !isfinite(qn) || !isfinite(c.t_cw[0] + c.t_cw[1] + c.t_cw[2]))
            return failf(GS_ERR_INVALID, "camera %lld: pose invalid", e);
    }
    const int tw = v.tile_w, th = v.tile_h;
    const int ntx = (W + tw - 1) / tw, nty = (H + th - 1) / th, T = ntx * nty;
    if (T > 16384) return failf(GS_ERR_UNSUPPORTED, "%lld tiles per image exceed 16384", T);
    NA_CK(cudaSetDevice(v.device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t px = (size_t)W * H;
    const int64_t G = v.D.n;
    if (G == 0) {
        NA_CK(cudaMemsetAsync(rgb, 0, (size_t)n_envs * px * 12, st), "clear rgb");
        NA_CK(cudaMemsetAsync(depth, 0, (size_t)n_envs * px * 4, st), "clear depth");
        if (alpha) NA_CK(cudaMemsetAsync(alpha, 0, (size_t)n_envs * px * 4, st), "clear alpha");
        return GS_OK;
    }
    unsigned char* base = nullptr;
    gs_status r = scratch_on(v.device, &base);
    if (r != GS_OK) return r;
    std::lock_guard<std::mutex> lk(g_setup_mu);  // the static host tables below are shared too
    const int64_t n_local = bg_slots(v.D.n_bg) + (v.D.n - v.D.n_bg);
    const unsigned long long words1 = (unsigned long long)(n_local + 31) / 32;
    // largest wave whose fixed part leaves at least a quarter of the array for keys
    int We = n_envs < kMaxWave ? n_envs : kMaxWave;
    auto fixed = [&](int w) {
        return layout(w, kMaxBlocks, w * (1 + L), (unsigned long long)w * n_local, words1 * w,
                      (unsigned long long)w * T).pairs;
    };
    while (We > 0 && fixed(We) > kNoAllocBytes / 4 * 3) --We;
    if (We == 0)
        return failf(GS_ERR_UNSUPPORTED,
                     "scene too large for the no-allocation path: one env needs %lld bytes of records, the fixed "
                     "scratch holds %lld (use gs_render_batch)",
                     (long long)fixed(1), (long long)kNoAllocBytes);
    int64_t link_offs[2] = {0, v.D.n - v.D.n_bg};  // all links of a uniform batch, as one contiguous range
    for (int e0 = 0; e0 < n_envs; e0 += We) {
        const int Wn = n_envs - e0 < We ? n_envs - e0 : We;
        for (int e = 0; e < Wn; ++e)
            h_specs[e] = EnvSpec{cams + e0 + e, 0, L, (long long)(e0 + e) * L, (long long)e * (long long)px};
        // the link range [0, L) of every env maps to link Gaussians [0, n_link_gaussians)
        DevGaussians D1 = v.D;
        D1.n_links = L;
        int nb = 0;
        // build_wave_tables reads link_offsets[link_begin] and [link_end]; give it a
        // table where index 0 is 0 and index L is the link Gaussian count
        static int64_t lo_table[4097];
        if (L > 4096) return report(GS_ERR_UNSUPPORTED, "more than 4096 links on the no-allocation path");
        for (int l = 0; l <= L; ++l) lo_table[l] = l == L ? link_offs[1] : 0;
        build_wave_tables(D1, lo_table, h_specs, Wn, tw, th, 0, h_envs, h_blocks, &nb, kMaxBlocks);
        if (nb > kMaxBlocks)
            return failf(GS_ERR_UNSUPPORTED, "%lld projection blocks exceed the no-allocation table of %lld", nb,
                         kMaxBlocks);
        const EnvInfo& sen = h_envs[Wn];
        const Layout y = layout(Wn, nb, sen.xf_base, sen.rec_base, sen.mask_base, sen.tile_base);
        int max_words = 0, max_T = 0;
        for (int e = 0; e < Wn; ++e) {
            max_words = max_words > (int)((h_envs[e].n_local + 31) / 32) ? max_words : (int)((h_envs[e].n_local + 31) / 32);
            max_T = max_T > h_envs[e].T ? max_T : h_envs[e].T;
        }
        EnvInfo* d_envs = reinterpret_cast<EnvInfo*>(base + y.envs);
        ProjBlock* d_blocks = reinterpret_cast<ProjBlock*>(base + y.blocks);
        gs_camera* d_cams = reinterpret_cast<gs_camera*>(base + y.cams);
        LinkXf* xf = reinterpret_cast<LinkXf*>(base + y.xf);
        NA_CK(cudaMemcpyAsync(d_envs, h_envs, sizeof(EnvInfo) * ((size_t)Wn + 1), cudaMemcpyHostToDevice, st),
              "copy env table");
        NA_CK(cudaMemcpyAsync(d_blocks, h_blocks, sizeof(ProjBlock) * (size_t)nb, cudaMemcpyHostToDevice, st),
              "copy block table");
        NA_CK(cudaMemcpyAsync(d_cams, cams + e0, sizeof(gs_camera) * (size_t)Wn, cudaMemcpyHostToDevice, st),
              "copy cams");
        NA_CK(launch_link_table(link_poses, d_cams, d_envs, Wn, sen.xf_base, xf, v.status, st), "link table");
        ProjParams P{};
        P.n_gauss = v.D.n;
        P.p0 = v.D.p0;
        P.p1 = v.D.p1;
        P.p2 = v.D.p2;
        P.p3 = v.D.p3;
        P.sh = v.D.sh;
        P.blocks = d_blocks;
        P.envs = d_envs;
        P.cams = d_cams;
        P.xf = xf;
        P.r0 = reinterpret_cast<float4*>(base + y.r012);
        P.r1 = P.r0 + 1;
        P.r2 = P.r0 + 2;
        P.r3 = reinterpret_cast<uint4*>(base + y.r3);
        P.mask = reinterpret_cast<uint32_t*>(base + y.mask);
        P.dbg_hxy = nullptr;
        P.bg_index = v.bg_index;
        NA_CK(launch_project(v.D, P, nb, st), "projection");
        uint32_t* counts = reinterpret_cast<uint32_t*>(base + y.counts);
        uint32_t* off = reinterpret_cast<uint32_t*>(base + y.off);
        uint32_t* cursor = reinterpret_cast<uint32_t*>(base + y.cursor);
        auto* env_total = reinterpret_cast<unsigned long long*>(base + y.env_total);
        auto* env_base = reinterpret_cast<unsigned long long*>(base + y.env_base);
        NA_CK(cudaMemsetAsync(counts, 0, (size_t)sen.tile_base * 4, st), "clear counts");
        BinParams B{};
        B.envs = d_envs;
        B.mask = P.mask;
        B.r3 = P.r3;
        B.e_begin = 0;
        B.tile_w = tw;
        B.tile_h = th;
        B.index_in_r3 = 1;
        B.bg_index = v.bg_index;
        B.n_bg = (unsigned)v.D.n_bg;
        B.words_per_block = kWordsPerBlock;
        B.counts = counts;
        B.off_local = off;
        B.env_base = env_base;
        B.cursor = cursor;
        B.status = v.status;
        NA_CK(launch_count(B, Wn, max_words, max_T, st), "count");
        NA_CK(launch_scan(d_envs, counts, off, env_total, env_base, Wn, st), "scan");
        unsigned long long eb[kMaxWave + 1];
        NA_CK(cudaMemcpyAsync(eb, env_base, sizeof(unsigned long long) * (Wn + 1), cudaMemcpyDeviceToHost, st),
              "read totals");
        NA_CK(cudaStreamSynchronize(st), "sync totals");
        const unsigned long long need = eb[Wn] * 8ull;
        if (y.pairs + need > kNoAllocBytes)
            return failf(GS_ERR_UNSUPPORTED,
                         "no-allocation scratch too small: %lld intersection keys need %lld bytes, %lld are free "
                         "(use gs_render_batch)",
                         (long long)eb[Wn], (long long)need, (long long)(kNoAllocBytes - y.pairs));
        NA_CK(cudaMemsetAsync(cursor, 0, (size_t)sen.tile_base * 4, st), "clear cursors");
        B.pair_base = 0;
        B.pair_cap = (kNoAllocBytes - y.pairs) / 8;
        B.pairs = reinterpret_cast<unsigned long long*>(base + y.pairs);
        NA_CK(launch_scatter(B, Wn, max_words, max_T, st), "scatter");
        CompParams C{};
        C.envs = d_envs;
        C.e_begin = 0;
        C.e_end = Wn;
        C.item_begin = 0;
        C.item_end = sen.tile_base;
        C.chunk = 1;
        C.bg_slot = v.bg_slot;
        C.n_bg = (unsigned)v.D.n_bg;
        C.work = reinterpret_cast<unsigned int*>(base + y.work);
        C.r0 = P.r0;
        C.r1 = P.r1;
        C.r2 = P.r2;
        C.counts = counts;
        C.off_local = off;
        C.env_base = env_base;
        C.pair_base = 0;
        C.pair_cap = B.pair_cap;
        C.pairs = B.pairs;
        C.dbg_sorted = nullptr;
        C.neval = nullptr;
        C.tile_w = tw;
        C.tile_h = th;
        C.rgb = rgb + (size_t)e0 * px * 3;
        C.depth = depth + (size_t)e0 * px;
        C.alpha = alpha ? alpha + (size_t)e0 * px : nullptr;
        C.status = v.status;
        NA_CK(cudaMemsetAsync(C.work, 0, 4, st), "clear work counter");
        int ctas = 0;
        NA_CK(launch_composite(C, st, &ctas), "composite");
    }
    return GS_OK;
}
