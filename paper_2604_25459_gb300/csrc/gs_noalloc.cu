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

struct Layout {
    size_t cams, xf, r0, r1, r2, r3, mask, counts, off, cursor, env_total, env_base, pairs, end_fixed;
};

Layout layout(int We, int64_t G, int L, int64_t mask_words, int T) {
    Layout y{};
    size_t o = 0;
    y.cams = o;      o = up256(o + (size_t)We * sizeof(gs_camera));
    y.xf = o;        o = up256(o + (size_t)We * (L + 1) * sizeof(LinkXf));
    y.r0 = o;        o = up256(o + (size_t)We * G * 16);
    y.r1 = o;        o = up256(o + (size_t)We * G * 16);
    y.r2 = o;        o = up256(o + (size_t)We * G * 16);
    y.r3 = o;        o = up256(o + (size_t)We * G * 16);
    y.mask = o;      o = up256(o + (size_t)We * mask_words * 4);
    y.counts = o;    o = up256(o + (size_t)We * T * 4);
    y.off = o;       o = up256(o + (size_t)We * T * 4);
    y.cursor = o;    o = up256(o + (size_t)We * T * 4);
    y.env_total = o; o = up256(o + (size_t)We * 8);
    y.env_base = o;  o = up256(o + (size_t)(We + 1) * 8);
    y.pairs = o;
    y.end_fixed = o;
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
    const int ntx = (W + v.tile_w - 1) / v.tile_w, nty = (H + v.tile_h - 1) / v.tile_h, T = ntx * nty;
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
    const int64_t mask_words = (G + 31) / 32;
    // largest wave whose fixed part leaves at least a quarter of the array for keys
    int We = n_envs < kMaxWave ? n_envs : kMaxWave;
    while (We > 0 && layout(We, G, L, mask_words, T).end_fixed > kNoAllocBytes / 4 * 3) --We;
    if (We == 0)
        return failf(GS_ERR_UNSUPPORTED,
                     "scene too large for the no-allocation path: one env needs %lld bytes of records, the fixed "
                     "scratch holds %lld (use gs_render_batch)",
                     (long long)layout(1, G, L, mask_words, T).end_fixed, (long long)kNoAllocBytes);
    const Layout y = layout(We, G, L, mask_words, T);
    const size_t pose_floats = (size_t)L * 7;
    unsigned long long eb[kMaxWave + 1];
    for (int e0 = 0; e0 < n_envs; e0 += We) {
        const int Wn = n_envs - e0 < We ? n_envs - e0 : We;
        gs_camera* cams_dev = reinterpret_cast<gs_camera*>(base + y.cams);
        LinkXf* xf = reinterpret_cast<LinkXf*>(base + y.xf);
        NA_CK(cudaMemcpyAsync(cams_dev, cams + e0, (size_t)Wn * sizeof(gs_camera), cudaMemcpyHostToDevice, st),
              "copy cams");
        NA_CK(launch_link_table(L > 0 ? link_poses + (size_t)e0 * pose_floats : nullptr, cams_dev, Wn, L, xf,
                                v.status, st),
              "link table");
        ProjParams P{};
        P.G = G;
        P.p0 = v.D.p0;
        P.p1 = v.D.p1;
        P.p2 = v.D.p2;
        P.p3 = v.D.p3;
        P.sh = v.D.sh;
        P.xf = xf;
        P.cams = cams_dev;
        P.L1 = L + 1;
        P.We = Wn;
        P.r0 = reinterpret_cast<float4*>(base + y.r0);
        P.r1 = reinterpret_cast<float4*>(base + y.r1);
        P.r2 = reinterpret_cast<float4*>(base + y.r2);
        P.r3 = reinterpret_cast<uint4*>(base + y.r3);
        P.mask = reinterpret_cast<uint32_t*>(base + y.mask);
        P.mask_words = mask_words;
        P.dbg_hxy = nullptr;
        const unsigned gx = (unsigned)((G + 255) / 256);
        int gy = (int)((4864 + gx - 1) / gx);
        if (gy < 1) gy = 1;
        if (gy > Wn) gy = Wn;
        P.env_group = (Wn + gy - 1) / gy;
        gy = (Wn + P.env_group - 1) / P.env_group;
        NA_CK(launch_project(v.D, P, dim3(gx, (unsigned)gy), st), "projection");
        uint32_t* counts = reinterpret_cast<uint32_t*>(base + y.counts);
        uint32_t* off = reinterpret_cast<uint32_t*>(base + y.off);
        uint32_t* cursor = reinterpret_cast<uint32_t*>(base + y.cursor);
        auto* env_total = reinterpret_cast<unsigned long long*>(base + y.env_total);
        auto* env_base = reinterpret_cast<unsigned long long*>(base + y.env_base);
        NA_CK(cudaMemsetAsync(counts, 0, (size_t)Wn * T * 4, st), "clear counts");
        BinParams B{};
        B.G = G;
        B.mask_words = mask_words;
        B.mask = P.mask;
        B.r3 = P.r3;
        B.e_begin = 0;
        B.tile_w = v.tile_w;
        B.tile_h = v.tile_h;
        B.ntx = ntx;
        B.T = T;
        B.counts = counts;
        B.off_local = off;
        B.env_base = env_base;
        B.cursor = cursor;
        B.words_per_block = 256;  // 8 warps x 32 mask words (8192 Gaussians)
        NA_CK(launch_count(B, Wn, st, (size_t)T * 4), "count");
        NA_CK(launch_scan(counts, off, env_total, env_base, Wn, T, st), "scan");
        NA_CK(cudaMemcpyAsync(eb, env_base, sizeof(unsigned long long) * (Wn + 1), cudaMemcpyDeviceToHost, st),
              "read totals");
        NA_CK(cudaStreamSynchronize(st), "sync totals");
        const unsigned long long need = eb[Wn] * 8ull;
        if (y.pairs + need > kNoAllocBytes)
            return failf(GS_ERR_UNSUPPORTED,
                         "no-allocation scratch too small: %lld intersection keys need %lld bytes, %lld are free "
                         "(use gs_render_batch)",
                         (long long)eb[Wn], (long long)need, (long long)(kNoAllocBytes - y.pairs));
        NA_CK(cudaMemsetAsync(cursor, 0, (size_t)Wn * T * 4, st), "clear cursors");
        B.pair_base = 0;
        B.pairs = reinterpret_cast<unsigned long long*>(base + y.pairs);
        NA_CK(launch_scatter(B, Wn, st, (size_t)T * 8), "scatter");
        CompParams C{};
        C.G = G;
        C.r0 = P.r0;
        C.r1 = P.r1;
        C.r2 = P.r2;
        C.counts = counts;
        C.off_local = off;
        C.env_base = env_base;
        C.pair_base = 0;
        C.pairs = B.pairs;
        C.dbg_sorted = nullptr;
        C.neval = nullptr;
        C.e_begin = 0;
        C.W = W;
        C.H = H;
        C.tile_w = v.tile_w;
        C.tile_h = v.tile_h;
        C.ntx = ntx;
        C.T = T;
        C.rgb = rgb + (size_t)e0 * px * 3;
        C.depth = depth + (size_t)e0 * px;
        C.alpha = alpha ? alpha + (size_t)e0 * px : nullptr;
        C.status = v.status;
        NA_CK(launch_composite(C, Wn, st), "composite");
    }
    return GS_OK;
}
