// C ABI of libgsbatch: scenes, batched rendering (uniform, uneven, planned
// under a CUDA graph), status, profiling and debug hooks; the request loop
// (gs_server_*) is in gs_server.cu.
//
// The call sequence follows the paper's loop (Sec. III-A "Data Flow"): poses
// from the physics step -> RLGK (Sec. III-C) -> batch 3DGS renderer (Sec.
// III-C "Throughput Scaling") -> RGB + depth per environment.  Every step of
// the render runs in the kernels of gs_project.cu, gs_bin.cu and
// gs_composite.cu; this file validates arguments, plans waves of environments
// against the scratch budget and orders the launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gs_host.h"

using namespace gsb;

namespace gsb {

thread_local std::string g_err;

gs_status fail(gs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

gs_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(GS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool valid_tile(int tw, int th) {
    return (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 16 && th == 16) || (tw == 32 && th == 8) ||
           (tw == 32 && th == 16);
}

}  // namespace gsb

struct gs_plan_s {
    gs_scene s = nullptr;
    std::vector<gs_env> envs;
    std::vector<gs_camera> cams;
    int flags = 0;
    int tile_w = 16, tile_h = 16, chunk = 1;
    int quad = 0;  // compositor's quadrant form (16x16 tiles), chosen by the autotuner
    Scratch sc;
    struct Wave {
        int e0, e1;
        DevBuf envs, blocks, cams;
        int n_blocks = 0, xf_items = 0, max_words = 0, max_T = 0;
        unsigned long long recs = 0, words = 0, tiles = 0;
        unsigned long long cap = 0;  // intersection-key capacity
    };
    std::vector<Wave> waves;
    bool tuned = false;
    int tuned_candidates = 0;
    double tuned_ms = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* cap_ptrs[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    uint32_t* pinned_status = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
    int regrows = 0;
};

namespace gsb {

// ------------------------------------------------------------------ scene upload

gs_status check_view(const gs_gaussians* g, const char* name) {
    if (!g) return fail(GS_ERR_INVALID, "%s: null gs_gaussians", name);
    if (g->n < 0) return fail(GS_ERR_INVALID, "%s: negative n", name);
    if (g->n > 0x7FFFFFF0ll) return fail(GS_ERR_UNSUPPORTED, "%s: more than 2^31-16 Gaussians", name);
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(GS_ERR_INVALID, "%s: sh_degree must be 0..3", name);
    if (g->dtype != GS_F32 && g->dtype != GS_BF16 && g->dtype != GS_F16)
        return fail(GS_ERR_INVALID, "%s: unknown dtype", name);
    if (g->n > 0 && (!g->mean || !g->quat || !g->log_scale || !g->opacity || !g->sh))
        return fail(GS_ERR_INVALID, "%s: null attribute pointer", name);
    return GS_OK;
}

size_t elem_size(gs_dtype d) { return d == GS_F32 ? 4 : 2; }

// Copy a view's arrays to the device (if they are host arrays) and run the
// preparation kernel into D[dst, dst + n).
// Storage order of a background: the Morton (Z-order) position of each mean
// in the set's bounding box, 10 bits per axis, equal codes in the caller's
// order.  The projection runs one thread per Gaussian, so a warp then holds
// Gaussians that lie close together and mostly agree on which environments
// see them (in the caller's order a warp mixes a few visible Gaussians with
// many culled ones in nearly every environment).  Returns order[k] = caller's
// index of the Gaussian stored at position k.
std::vector<long long> spatial_order(const float* mean, int64_t n) {
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const float t = mean[3 * i + k];
            if (std::isfinite(t)) {
                lo[k] = std::min(lo[k], t);
                hi[k] = std::max(hi[k], t);
            }
        }
    auto spread = [](uint32_t x) {  // bit b of x to bit 3b
        x &= 0x3ffu;
        x = (x | (x << 16)) & 0x030000ffu;
        x = (x | (x << 8)) & 0x0300f00fu;
        x = (x | (x << 4)) & 0x030c30c3u;
        x = (x | (x << 2)) & 0x09249249u;
        return x;
    };
    std::vector<uint32_t> code((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c = 0;
        for (int k = 0; k < 3; ++k) {
            const float t = mean[3 * i + k];
            uint32_t q = 0;
            if (std::isfinite(t) && hi[k] > lo[k]) {
                const double f = (double)(t - lo[k]) / ((double)hi[k] - (double)lo[k]) * 1023.0;
                q = (uint32_t)std::min(1023.0, std::max(0.0, f));
            }
            c |= spread(q) << k;
        }
        code[(size_t)i] = c;
    }
    std::vector<long long> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](long long a, long long b) { return code[(size_t)a] < code[(size_t)b]; });
    return order;
}

gs_status prep_view(gs_scene s, const gs_gaussians* g, int64_t dst, int link_mode, const int64_t* link_offsets_host,
                    int n_links, const int64_t* place_host = nullptr) {
    const int64_t n = g->n;
    if (n == 0) return GS_OK;
    const size_t es = elem_size(g->dtype);
    const size_t nv = (size_t)sh_values(g->sh_degree);
    const size_t sz_mean = n * 12, sz_quat = n * 16, sz_ls = n * 3 * es, sz_op = n * es, sz_sh = n * nv * es;
    std::vector<void*> tmp;
    auto upload = [&](const void* src, size_t bytes, const void** out) -> cudaError_t {
        if (g->on_device) {
            *out = src;
            return cudaSuccess;
        }
        void* d = nullptr;
        cudaError_t e = cudaMalloc(&d, bytes);
        if (e != cudaSuccess) return e;
        tmp.push_back(d);
        *out = d;
        return cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
    };
    const void *mean, *quat, *ls, *op, *sh;
    const int64_t* offs = nullptr;
    cudaError_t e = upload(g->mean, sz_mean, &mean);
    if (e == cudaSuccess) e = upload(g->quat, sz_quat, &quat);
    if (e == cudaSuccess) e = upload(g->log_scale, sz_ls, &ls);
    if (e == cudaSuccess) e = upload(g->opacity, sz_op, &op);
    if (e == cudaSuccess) e = upload(g->sh, sz_sh, &sh);
    if (e == cudaSuccess && link_mode) {
        void* d = nullptr;
        e = cudaMalloc(&d, sizeof(int64_t) * (n_links + 1));
        if (e == cudaSuccess) {
            tmp.push_back(d);
            e = cudaMemcpy(d, link_offsets_host, sizeof(int64_t) * (n_links + 1), cudaMemcpyHostToDevice);
            offs = static_cast<const int64_t*>(d);
        }
    }
    const int64_t* place = nullptr;
    if (e == cudaSuccess && place_host) {
        void* d = nullptr;
        e = cudaMalloc(&d, sizeof(int64_t) * (size_t)n);
        if (e == cudaSuccess) {
            tmp.push_back(d);
            e = cudaMemcpy(d, place_host, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice);
            place = static_cast<const int64_t*>(d);
        }
    }
    if (e == cudaSuccess)
        e = launch_prep(static_cast<const float*>(mean), static_cast<const float*>(quat), ls, op, sh, n, dst, place,
                        link_mode, offs, n_links, s->D, s->status, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    for (void* p : tmp) cudaFree(p);
    if (e != cudaSuccess) return cuda_fail(e, "scene upload");
    uint32_t st = 0;
    CK(cudaMemcpy(&st, s->status, 4, cudaMemcpyDeviceToHost), "status read");
    if (st & kStBadScene) {
        CK(cudaMemset(s->status, 0, 4), "status clear");
        return fail(GS_ERR_INVALID, "Gaussian set holds a zero or non-finite quaternion or scale");
    }
    return GS_OK;
}

// Uploads a background in its storage order (spatial_order) and keeps the order.
gs_status place_background(gs_scene s, const gs_gaussians* g) {
    const int64_t n = g->n;
    s->bg_order.clear();
    if (n == 0) return GS_OK;
    std::vector<float> host_mean;
    const float* mean = g->mean;
    if (g->on_device) {
        host_mean.resize((size_t)n * 3);
        CK(cudaMemcpy(host_mean.data(), g->mean, (size_t)n * 12, cudaMemcpyDeviceToHost), "copy means");
        mean = host_mean.data();
    }
    std::vector<long long> order = spatial_order(mean, n);
    std::vector<int64_t> place((size_t)n);
    std::vector<int> index32((size_t)n), slot32((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        place[(size_t)order[(size_t)k]] = k;
        index32[(size_t)k] = (int)order[(size_t)k];
        slot32[(size_t)order[(size_t)k]] = (int)k;
    }
    CK(s->bg_index.ensure(sizeof(int) * (size_t)n), "alloc storage order");
    CK(s->bg_slot.ensure(sizeof(int) * (size_t)n), "alloc storage order");
    CK(cudaMemcpy(s->bg_index.p, index32.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice),
       "copy storage order");
    CK(cudaMemcpy(s->bg_slot.p, slot32.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice),
       "copy storage order");
    ST(prep_view(s, g, 0, 0, nullptr, 0, place.data()));
    s->bg_order.swap(order);
    return GS_OK;
}

gs_status alloc_gaussians(int64_t n, DevBuf& a, DevBuf& b, DevBuf& c, DevBuf& d, DevBuf& sh, int planes) {
    const size_t m = (size_t)(n > 0 ? n : 1);
    CK(a.ensure(m * 16), "alloc p0");
    CK(b.ensure(m * 16), "alloc p1");
    CK(c.ensure(m * 16), "alloc p2");
    CK(d.ensure(m * 16), "alloc p3");
    CK(sh.ensure(m * 16 * (size_t)(planes > 0 ? planes : 1)), "alloc sh");
    return GS_OK;
}

// ------------------------------------------------------------------ env validation

gs_status check_cam(const gs_camera& c, int e) {
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
        return fail(GS_ERR_INVALID, "env %d: width/height must be in [1, 16384]", e);
    if (!(std::isfinite(c.fx) && std::isfinite(c.fy) && c.fx > 0 && c.fy > 0))
        return fail(GS_ERR_INVALID, "env %d: focal lengths must be finite and > 0", e);
    if (!(std::isfinite(c.cx) && std::isfinite(c.cy)))
        return fail(GS_ERR_INVALID, "env %d: principal point must be finite", e);
    if (!(std::isfinite(c.near_plane) && c.near_plane > 0))
        return fail(GS_ERR_INVALID, "env %d: near_plane must be finite and > 0", e);
    double qn = 0;
    for (int k = 0; k < 4; ++k) {
        if (!std::isfinite(c.q_cw[k])) return fail(GS_ERR_INVALID, "env %d: non-finite camera quaternion", e);
        qn += (double)c.q_cw[k] * c.q_cw[k];
    }
    if (!(qn > 0)) return fail(GS_ERR_INVALID, "env %d: zero camera quaternion", e);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(c.t_cw[k])) return fail(GS_ERR_INVALID, "env %d: non-finite camera translation", e);
    return GS_OK;
}

gs_status check_specs(gs_scene s, const std::vector<EnvSpec>& specs, int tw, int th) {
    for (size_t e = 0; e < specs.size(); ++e) {
        const EnvSpec& sp = specs[e];
        ST(check_cam(*sp.cam, (int)e));
        const int ntx = (sp.cam->width + tw - 1) / tw, nty = (sp.cam->height + th - 1) / th;
        if (ntx * nty > 16384)
            return fail(GS_ERR_UNSUPPORTED, "env %d: %d tiles exceed the 16384 supported (use larger tiles)", (int)e,
                        ntx * nty);
        if (sp.link_begin < 0 || sp.link_end < sp.link_begin || sp.link_end > s->D.n_links)
            return fail(GS_ERR_INVALID, "env %d: link range [%d, %d) outside [0, %d]", (int)e, sp.link_begin,
                        sp.link_end, s->D.n_links);
        if (sp.link_end > sp.link_begin && sp.pose_offset < 0)
            return fail(GS_ERR_INVALID, "env %d: negative pose_offset", (int)e);
        if (sp.pixel_offset < 0) return fail(GS_ERR_INVALID, "env %d: negative pixel_offset", (int)e);
    }
    return GS_OK;
}

// Fixed scratch bytes of one env (records, visibility, tile counters, link table).
size_t env_bytes(gs_scene s, const EnvSpec& sp, int tw, int th, bool debug) {
    const int64_t nlg = s->link_offsets[sp.link_end] - s->link_offsets[sp.link_begin];
    const int64_t n_local = bg_slots(s->D.n_bg) + nlg;
    const int64_t T = (int64_t)((sp.cam->width + tw - 1) / tw) * ((sp.cam->height + th - 1) / th);
    size_t b = (size_t)n_local * 64 + (size_t)((n_local + 31) / 32) * 4 + (size_t)T * 12 + 16 +
               (size_t)(1 + sp.link_end - sp.link_begin) * sizeof(LinkXf) + sizeof(gs_camera) + sizeof(EnvInfo) + 64;
    if (debug) b += (size_t)n_local * 8;
    return b;
}

// Split envs into waves whose fixed scratch fits 60 % of the budget.
gs_status plan_waves(gs_scene s, const std::vector<EnvSpec>& specs, int tw, int th, bool debug, int max_wave,
                     size_t extra_per_env, std::vector<std::pair<int, int>>* waves) {
    waves->clear();
    const double cap = (double)s->budget * 0.6;
    const int E = (int)specs.size();
    // uniform batches: balanced waves of equal size
    bool uniform = true;
    for (int e = 1; e < E && uniform; ++e)
        uniform = specs[e].cam->width == specs[0].cam->width && specs[e].cam->height == specs[0].cam->height &&
                  specs[e].link_begin == specs[0].link_begin && specs[e].link_end == specs[0].link_end;
    if (uniform && E > 0) {
        const double per = (double)(env_bytes(s, specs[0], tw, th, debug) + extra_per_env);
        int64_t wmax = (int64_t)(cap / per);
        if (wmax < 1)
            return fail(GS_ERR_OOM, "one environment needs %.0f bytes of scratch; budget is %lld", per,
                        (long long)s->budget);
        if (max_wave > 0 && wmax > max_wave) wmax = max_wave;
        if (wmax > E) wmax = E;
        const int64_t nw = (E + wmax - 1) / wmax;
        const int We = (int)((E + nw - 1) / nw);
        for (int e0 = 0; e0 < E; e0 += We) waves->push_back({e0, std::min(E, e0 + We)});
        return GS_OK;
    }
    int e0 = 0;
    double acc = 0;
    for (int e = 0; e < E; ++e) {
        const double b = (double)(env_bytes(s, specs[e], tw, th, debug) + extra_per_env);
        if (b > cap) return fail(GS_ERR_OOM, "env %d needs %.0f bytes of scratch; budget is %lld", e, b,
                                 (long long)s->budget);
        if (e > e0 && (acc + b > cap || (max_wave > 0 && e - e0 >= max_wave))) {
            waves->push_back({e0, e});
            e0 = e;
            acc = 0;
        }
        acc += b;
    }
    if (E > e0) waves->push_back({e0, E});
    return GS_OK;
}

// ------------------------------------------------------------------ one wave

// Brackets one phase's launches with events on the render stream when
// profiling is on (eager renders only).
struct PhaseTimer {
    gs_scene s;
    cudaStream_t st;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(gs_scene s_, cudaStream_t st_, int ph, bool on) : s(s_), st(st_), phase(ph) {
        if (on && s->profile) {
            a = take();
            if (a) cudaEventRecord(a, st);
        }
    }
    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        if (!s->event_pool.empty()) {
            e = s->event_pool.back();
            s->event_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }
    void done(int kernels) {
        if (!a) return;
        cudaEvent_t b = take();
        if (!b) return;
        cudaEventRecord(b, st);
        s->marks.push_back({phase, kernels, a, b});
        a = nullptr;
    }
};

// Where a render's images go: float RGB / depth / alpha, or the observation
// form (8-bit RGB after the appearance transform, half depth).
struct Outputs {
    float* rgb = nullptr;
    float* depth = nullptr;
    float* alpha = nullptr;
    uint8_t* rgb8 = nullptr;
    uint16_t* depth16 = nullptr;
    const gs_appearance* appear = nullptr;
    bool obs() const { return rgb8 != nullptr; }
    size_t rgb_px() const { return obs() ? 3 : 12; }                  // bytes per pixel
    size_t depth_px() const { return obs() ? (depth16 ? 2 : 0) : 4; }
};

// Build and upload the tables of specs[e0, e1) into the given device buffers.
gs_status upload_tables(gs_scene s, const std::vector<EnvSpec>& specs, int e0, int e1, int tw, int th,
                        long long pix_rebase, DevBuf& d_envs, DevBuf& d_blocks, DevBuf& d_cams, cudaStream_t st,
                        bool sync_copy, WaveTables* wt) {
    const int We = e1 - e0;
    const EnvSpec* sp = specs.data() + e0;
    const int nb = count_wave_blocks(s->D, s->link_offsets.data(), sp, We);
    s->h_envs.resize((size_t)We + 1);
    s->h_blocks.resize((size_t)std::max(nb, 1));
    s->h_cams.resize((size_t)We);
    int nb2 = 0;
    build_wave_tables(s->D, s->link_offsets.data(), sp, We, tw, th, pix_rebase, s->h_envs.data(), s->h_blocks.data(),
                      &nb2, nb);
    int max_words = 0, max_T = 0;
    for (int e = 0; e < We; ++e) {
        s->h_cams[e] = *sp[e].cam;
        max_words = std::max(max_words, (int)((s->h_envs[e].n_local + 31) / 32));
        max_T = std::max(max_T, s->h_envs[e].T);
    }
    CK(d_envs.ensure(sizeof(EnvInfo) * ((size_t)We + 1)), "alloc env table");
    CK(d_blocks.ensure(sizeof(ProjBlock) * (size_t)std::max(nb, 1)), "alloc block table");
    CK(d_cams.ensure(sizeof(gs_camera) * (size_t)We), "alloc cameras");
    if (sync_copy) {
        CK(cudaMemcpy(d_envs.p, s->h_envs.data(), sizeof(EnvInfo) * ((size_t)We + 1), cudaMemcpyHostToDevice),
           "copy env table");
        CK(cudaMemcpy(d_blocks.p, s->h_blocks.data(), sizeof(ProjBlock) * (size_t)nb, cudaMemcpyHostToDevice),
           "copy block table");
        CK(cudaMemcpy(d_cams.p, s->h_cams.data(), sizeof(gs_camera) * (size_t)We, cudaMemcpyHostToDevice),
           "copy cameras");
    } else {  // pageable sources: the copies are staged before the calls return
        CK(cudaMemcpyAsync(d_envs.p, s->h_envs.data(), sizeof(EnvInfo) * ((size_t)We + 1), cudaMemcpyHostToDevice,
                           st),
           "copy env table");
        CK(cudaMemcpyAsync(d_blocks.p, s->h_blocks.data(), sizeof(ProjBlock) * (size_t)nb, cudaMemcpyHostToDevice,
                           st),
           "copy block table");
        CK(cudaMemcpyAsync(d_cams.p, s->h_cams.data(), sizeof(gs_camera) * (size_t)We, cudaMemcpyHostToDevice, st),
           "copy cameras");
    }
    const EnvInfo& sen = s->h_envs[We];
    *wt = WaveTables{d_envs.as<EnvInfo>(), d_blocks.as<ProjBlock>(), d_cams.as<gs_camera>(), We, nb, sen.xf_base,
                     max_words, max_T, sen.rec_base, sen.mask_base, sen.tile_base, s->h_envs.data()};
    return GS_OK;
}

// Launch one wave.  Eager (cap == 0): reads the wave's intersection totals back
// (host sync), grows the key buffer and splits the wave into sub-waves that
// fit the budget.  Planned (cap > 0): no host sync; keys beyond cap are dropped
// and flagged in the status word.
gs_status run_wave(gs_scene s, Scratch& sc, const WaveTables& wt, const WaveIO& io, int tw, int th, int chunk,
                   unsigned long long cap, cudaStream_t st, bool timers, int64_t* launches,
                   unsigned long long* total_out, int quad) {
    const int We = wt.We;
    bool use_quad = false;
    if (((tw == 16 && th == 16) || (tw == 8 && th == 8)) && !io.lidars && !io.score) {
        if (quad < 0) {
            long long most = 0;
            for (int e = 0; e < We; ++e)
                most = std::max(most, (long long)wt.host_envs[e].W * wt.host_envs[e].H);
            use_quad = most <= kQuadMaxPixels;
        } else {
            use_quad = quad != 0;
        }
    }
    CK(sc.xf.ensure(sizeof(LinkXf) * (size_t)std::max(wt.xf_items, 1)), "alloc link table");
    CK(sc.r012.ensure(wt.recs * 16 * kRecStride), "alloc records");
    CK(sc.r3.ensure(wt.recs * 16), "alloc records");
    CK(sc.mask.ensure(wt.words * 4), "alloc masks");
    CK(sc.counts.ensure(wt.tiles * 4), "alloc counts");
    CK(sc.zr.ensure((size_t)We * 8), "alloc depth ranges");
    CK(sc.off.ensure(wt.tiles * 4), "alloc offsets");
    CK(sc.cursor.ensure(wt.tiles * 4), "alloc cursors");
    CK(sc.env_total.ensure((size_t)We * 8), "alloc totals");
    CK(sc.env_base.ensure(((size_t)We + 1) * 8), "alloc bases");
    CK(sc.work.ensure(16), "alloc work counter");
    int spill_ctas = 0;  // per-CTA regions for partitioning long buckets
    CK(composite_max_ctas(tw, th, &spill_ctas), "compositor occupancy");
    CK(sc.spill.ensure((size_t)spill_ctas * kSpillMax * 8), "alloc spill");
    const bool debug = s->debug && cap == 0;
    if (debug) CK(sc.dbg_hxy.ensure(wt.recs * 8), "alloc debug");
    uint32_t* const status = io.status ? io.status : s->status;

    // A1: link composition
    PhaseTimer t1(s, st, GS_PHASE_LINK, timers);
    CK(launch_link_table(io.poses, wt.cams, wt.envs, We, wt.xf_items, sc.xf.as<LinkXf>(), status, st),
       "link table");
    t1.done(1);
    ++*launches;
    // A2: projection
    ProjParams P{};
    P.n_gauss = s->D.n;
    P.p0 = s->D.p0;
    P.p1 = s->D.p1;
    P.p2 = s->D.p2;
    P.p3 = s->D.p3;
    P.sh = s->D.sh;
    P.blocks = wt.blocks;
    P.envs = wt.envs;
    P.cams = wt.cams;
    P.xf = sc.xf.as<LinkXf>();
    P.r0 = sc.r012.as<float4>();
    P.r1 = P.r0 + 1;
    P.r2 = P.r0 + 2;
    P.r3 = sc.r3.as<uint4>();
    P.mask = sc.mask.as<uint32_t>();
    P.dbg_hxy = debug ? sc.dbg_hxy.as<float2>() : nullptr;
    P.nvis = (s->counters && cap == 0) ? s->neval.as<unsigned long long>() + 1 : nullptr;
    P.nfp64 = (s->counters && cap == 0) ? s->neval.as<unsigned long long>() + 2 : nullptr;
    P.lidars = io.lidars;
    P.cell_pad = io.ray_dirs ? 0.51f : 0.0f;  // a ray anywhere in its cell (+ rounding)
    P.bg_index = s->bg_order.empty() ? nullptr : s->bg_index.as<int>();
    PhaseTimer t2(s, st, GS_PHASE_PROJECT, timers);
    if (io.lidars) CK(launch_project_lidar(P, wt.n_blocks, st), "LiDAR projection");
    else CK(launch_project(s->D, P, wt.n_blocks, st), "projection");
    t2.done(1);
    ++*launches;
    // A3: counts + scan
    CK(cudaMemsetAsync(sc.counts.p, 0, wt.tiles * 4, st), "memset counts");
    CK(cudaMemsetAsync(sc.zr.p, 0xff, (size_t)We * 8, st), "memset depth ranges");
    BinParams B{};
    B.envs = wt.envs;
    B.mask = P.mask;
    B.r3 = P.r3;
    B.e_begin = 0;
    B.tile_w = tw;
    B.tile_h = th;
    B.words_per_block = kWordsPerBlock;
    B.counts = sc.counts.as<uint32_t>();
    B.off_local = sc.off.as<uint32_t>();
    B.env_base = sc.env_base.as<unsigned long long>();
    B.cursor = sc.cursor.as<uint32_t>();
    B.status = status;
    B.index_in_r3 = io.lidars ? 0 : 1;  // LiDAR records keep |g2| in r3.w
    B.wrap = io.lidars ? 1 : 0;         // LiDAR boxes may wrap across azimuth 0
    B.bg_index = s->bg_order.empty() ? nullptr : s->bg_index.as<int>();
    B.n_bg = (unsigned)s->D.n_bg;
    B.zr = sc.zr.as<uint2>();
    PhaseTimer t3(s, st, GS_PHASE_COUNT, timers);
    CK(launch_count(B, We, wt.max_words, wt.max_T, st), "count");
    t3.done(1);
    ++*launches;
    PhaseTimer t4(s, st, GS_PHASE_SCAN, timers);
    CK(launch_scan(wt.envs, sc.counts.as<uint32_t>(), sc.off.as<uint32_t>(), sc.env_total.as<unsigned long long>(),
                   sc.env_base.as<unsigned long long>(), We, st),
       "scan");
    t4.done(2);
    *launches += 2;
    CK(cudaMemsetAsync(sc.cursor.p, 0, wt.tiles * 4, st), "memset cursors");
    // arbitrary rays: cells, rays grouped by tile, compositor items (eager only)
    std::vector<unsigned long long> items;
    if (io.ray_dirs) {
        if (cap != 0) return fail(GS_ERR_UNSUPPORTED, "arbitrary-ray scans are not planned");
        const size_t nr = (size_t)We * (size_t)io.n_rays;
        CK(s->ray_cell.ensure(nr * 4), "alloc ray cells");
        CK(s->ray_list.ensure(nr * 4), "alloc ray lists");
        for (DevBuf* b : {&s->ray_cnt, &s->ray_off, &s->ray_cur, &s->item_cnt, &s->item_off})
            CK(b->ensure(wt.tiles * 4), "alloc ray tables");
        for (DevBuf* b : {&s->ray_tot, &s->item_tot}) CK(b->ensure((size_t)We * 8), "alloc ray totals");
        for (DevBuf* b : {&s->ray_base, &s->item_base}) CK(b->ensure((size_t)(We + 1) * 8), "alloc ray bases");
        CK(cudaMemsetAsync(s->ray_cnt.p, 0, wt.tiles * 4, st), "memset ray counts");
        CK(cudaMemsetAsync(s->ray_cur.p, 0, wt.tiles * 4, st), "memset ray cursors");
        PhaseTimer tr(s, st, GS_PHASE_SCAN, timers);
        CK(launch_ray_count(io.ray_dirs, io.lidars, wt.envs, We, io.n_rays, s->ray_cell.as<uint32_t>(),
                            s->ray_cnt.as<uint32_t>(), status, st),
           "ray cells");
        CK(launch_scan(wt.envs, s->ray_cnt.as<uint32_t>(), s->ray_off.as<uint32_t>(),
                       s->ray_tot.as<unsigned long long>(), s->ray_base.as<unsigned long long>(), We, st),
           "ray scan");
        CK(launch_ray_scatter(wt.envs, We, io.n_rays, s->ray_cell.as<uint32_t>(), s->ray_off.as<uint32_t>(),
                              s->ray_cur.as<uint32_t>(), s->ray_list.as<uint32_t>(), s->ray_cnt.as<uint32_t>(),
                              s->item_cnt.as<uint32_t>(), (unsigned)wt.tiles, st),
           "ray lists");
        CK(launch_scan(wt.envs, s->item_cnt.as<uint32_t>(), s->item_off.as<uint32_t>(),
                       s->item_tot.as<unsigned long long>(), s->item_base.as<unsigned long long>(), We, st),
           "item scan");
        tr.done(7);
        *launches += 7;
        items.resize((size_t)We + 1);
        CK(cudaMemcpyAsync(items.data(), s->item_base.p, sizeof(unsigned long long) * (We + 1),
                           cudaMemcpyDeviceToHost, st),
           "read items");
    }

    // sub-waves of envs whose keys fit (eager), or the whole wave (planned)
    std::vector<unsigned long long> ebv;
    const unsigned long long* eb = nullptr;
    unsigned long long cap_keys = cap;
    if (cap == 0) {
        if ((size_t)(We + 1) > s->pinned_n) {
            if (s->pinned) cudaFreeHost(s->pinned);
            s->pinned = nullptr;
            s->pinned_n = 0;
            CK(cudaMallocHost((void**)&s->pinned, sizeof(unsigned long long) * (We + 1)), "alloc pinned");
            s->pinned_n = (size_t)We + 1;
        }
        CK(cudaMemcpyAsync(s->pinned, sc.env_base.p, sizeof(unsigned long long) * (We + 1), cudaMemcpyDeviceToHost,
                           st),
           "read totals");
        CK(cudaStreamSynchronize(st), "sync totals");
        eb = s->pinned;
        if (total_out) *total_out = eb[We];
        s->stats.intersections += (int64_t)eb[We];
        double cap_d = (double)s->budget * 0.4;
        const size_t key_bytes = debug ? 16 : 8;
        cap_keys = (unsigned long long)(cap_d / key_bytes);
    } else {
        ebv.assign(2, 0);
        ebv[1] = cap;
    }
    int ea = 0;
    while (ea < We) {
        int ebd = We;
        unsigned long long npairs = cap;
        unsigned long long base = 0;
        if (cap == 0) {
            ebd = ea + 1;
            if (eb[ebd] - eb[ea] > cap_keys)
                return fail(GS_ERR_OOM, "environment %d has %llu intersections, beyond the scratch budget", ea,
                            (unsigned long long)(eb[ebd] - eb[ea]));
            while (ebd < We && eb[ebd + 1] - eb[ea] <= cap_keys) ++ebd;
            npairs = eb[ebd] - eb[ea];
            base = eb[ea];
            const size_t want = (size_t)(npairs > 0 ? npairs : 1) * 8;
            if (want > sc.pairs.bytes) {
                size_t grow = want + want / 4;
                if (grow > (size_t)cap_keys * 8) grow = want;
                CK(cudaStreamSynchronize(st), "sync before growth");
                CK(sc.pairs.ensure(grow), "alloc intersection keys");
            }
            if (debug) CK(sc.dbg_sorted.ensure(sc.pairs.bytes), "alloc debug lists");
        } else {
            CK(sc.pairs.ensure((size_t)cap * 8), "alloc intersection keys");
        }
        B.e_begin = ea;
        B.pair_base = base;
        B.pair_cap = cap == 0 ? (unsigned long long)(sc.pairs.bytes / 8) : cap;
        B.pairs = sc.pairs.as<unsigned long long>();
        PhaseTimer t5(s, st, GS_PHASE_SCATTER, timers);
        CK(launch_scatter(B, ebd - ea, wt.max_words, wt.max_T, st), "scatter");
        t5.done(1);
        ++*launches;
        CompParams C{};
        C.envs = wt.envs;
        C.e_begin = ea;
        C.e_end = ebd;
        C.item_begin = wt.host_envs[ea].tile_base;
        C.item_end = wt.host_envs[ebd].tile_base;
        if (io.ray_dirs) {  // items are chunks of rays (see run_wave's ray binning)
            C.item_begin = (unsigned)items[(size_t)ea];
            C.item_end = (unsigned)items[(size_t)ebd];
            C.ray_dirs = io.ray_dirs;
            C.ray_cell = s->ray_cell.as<uint32_t>();
            C.ray_list = s->ray_list.as<uint32_t>();
            C.ray_cnt = s->ray_cnt.as<uint32_t>();
            C.ray_off = s->ray_off.as<uint32_t>();
            C.item_off = s->item_off.as<uint32_t>();
            C.item_base = s->item_base.as<unsigned long long>();
            C.n_rays = io.n_rays;
        }
        C.chunk = chunk;
        C.work = sc.work.as<unsigned int>();
        C.r0 = P.r0;
        C.r1 = P.r1;
        C.r2 = P.r2;
        C.zr = sc.zr.as<uint2>();
        C.counts = sc.counts.as<uint32_t>();
        C.off_local = sc.off.as<uint32_t>();
        C.env_base = sc.env_base.as<unsigned long long>();
        C.pair_base = base;
        C.pair_cap = B.pair_cap;
        C.pairs = B.pairs;
        C.spill = sc.spill.as<unsigned long long>();
        C.spill_cap = kSpillMax;
        C.spill_ctas = (unsigned)spill_ctas;
        C.dbg_sorted = debug ? sc.dbg_sorted.as<unsigned long long>() : nullptr;
        C.neval = (s->counters && cap == 0) ? s->neval.as<unsigned long long>() : nullptr;
        C.tile_w = tw;
        C.tile_h = th;
        C.quad = use_quad ? 1 : 0;
        C.rgb = io.rgb;
        C.depth = io.depth;
        C.alpha = io.alpha;
        C.rgb8 = io.rgb8;
        C.depth16 = io.depth16;
        C.appear = io.appear;
        C.score = io.score;
        C.nbp = (unsigned)bg_slots(s->D.n_bg);
        C.bg_index = s->bg_order.empty() ? nullptr : s->bg_index.as<int>();
        C.bg_slot = s->bg_order.empty() ? nullptr : s->bg_slot.as<int>();
        C.n_bg = (unsigned)s->D.n_bg;
        C.lidars = io.lidars;
        C.r3 = P.r3;
        C.status = status;
        CK(cudaMemsetAsync(sc.work.p, 0, 4, st), "memset work counter");
        int ctas = 0;
        PhaseTimer t6(s, st, GS_PHASE_COMPOSITE, timers);
        CK(launch_composite(C, st, &ctas), "composite");
        t6.done(1);
        ++*launches;
        if (cap == 0) {
            s->last_ea = ea;
            s->last_eb = ebd;
            s->last_pair_base = base;
        }
        ea = ebd;
    }
    return GS_OK;
}

// ------------------------------------------------------------------ eager renders

enum class Out { Device, Host };

gs_status render_specs(gs_scene s, const std::vector<EnvSpec>& specs, const float* poses_dev, const Outputs& o,
                       cudaStream_t st, Out mode, int64_t pix_per_env_host) {
    float* const rgb = o.rgb;
    float* const depth = o.depth;
    float* const alpha = o.alpha;
    const int tw = s->tile_w, th = s->tile_h;
    ST(check_specs(s, specs, tw, th));
    CK(cudaSetDevice(s->device), "set device");
    s->stats.waves = 0;
    s->stats.kernel_launches = 0;
    s->stats.intersections = 0;
    const int E = (int)specs.size();
    size_t extra = 0;
    if (mode == Out::Host) extra = (size_t)pix_per_env_host * (o.rgb_px() + o.depth_px() + (alpha ? 4 : 0)) * 2;
    std::vector<std::pair<int, int>> waves;
    ST(plan_waves(s, specs, tw, th, s->debug != 0, s->max_wave, extra, &waves));
    int64_t launches = 0;
    if (mode == Out::Device) {
        for (auto& w : waves) {
            WaveTables wt{};
            ST(upload_tables(s, specs, w.first, w.second, tw, th, 0, s->sc.envs, s->sc.blocks, s->sc.cams, st, false,
                             &wt));
            s->last_envs.assign(wt.host_envs, wt.host_envs + wt.We + 1);
            WaveIO io{poses_dev, rgb, depth, alpha, 0};
            io.rgb8 = o.rgb8;
            io.depth16 = o.depth16;
            io.appear = o.appear ? o.appear + w.first : nullptr;
            ST(run_wave(s, s->sc, wt, io, tw, th, 1, 0, st, true, &launches, nullptr));
            s->last_e0 = w.first;
            s->last_We = wt.We;
            s->stats.waves++;
        }
    } else {
        // host buffers: wave outputs in device staging, copied out on a second
        // stream while the next wave renders
        if (!s->copy_stream) CK(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "copy stream");
        int maxw = 0;
        for (auto& w : waves) maxw = std::max(maxw, w.second - w.first);
        const size_t px = (size_t)pix_per_env_host;
        for (int k = 0; k < 2; ++k) {
            if (!s->ev_done[k]) CK(cudaEventCreateWithFlags(&s->ev_done[k], cudaEventDisableTiming), "event");
            if (!s->ev_copied[k]) CK(cudaEventCreateWithFlags(&s->ev_copied[k], cudaEventDisableTiming), "event");
            CK(s->stage_rgb[k].ensure((size_t)maxw * px * o.rgb_px()), "alloc staging");
            CK(s->stage_depth[k].ensure((size_t)maxw * px * std::max<size_t>(o.depth_px(), 1)), "alloc staging");
            if (alpha) CK(s->stage_alpha[k].ensure((size_t)maxw * px * 4), "alloc staging");
        }
        int wave = 0;
        for (auto& w : waves) {
            const int k = wave & 1;
            const int We = w.second - w.first;
            const long long rebase = specs[w.first].pixel_offset;
            if (wave >= 2) CK(cudaStreamWaitEvent(st, s->ev_copied[k], 0), "wait copy");
            WaveTables wt{};
            ST(upload_tables(s, specs, w.first, w.second, tw, th, rebase, s->sc.envs, s->sc.blocks, s->sc.cams, st,
                             false, &wt));
            s->last_envs.assign(wt.host_envs, wt.host_envs + wt.We + 1);
            WaveIO io{poses_dev, s->stage_rgb[k].as<float>(), s->stage_depth[k].as<float>(),
                      alpha ? s->stage_alpha[k].as<float>() : nullptr, rebase};
            if (o.obs()) {
                io.rgb = nullptr;
                io.depth = nullptr;
                io.rgb8 = s->stage_rgb[k].as<uint8_t>();
                io.depth16 = o.depth16 ? s->stage_depth[k].as<uint16_t>() : nullptr;
                io.appear = o.appear ? o.appear + w.first : nullptr;
            }
            ST(run_wave(s, s->sc, wt, io, tw, th, 1, 0, st, true, &launches, nullptr));
            s->last_e0 = w.first;
            s->last_We = We;
            CK(cudaEventRecord(s->ev_done[k], st), "record");
            CK(cudaStreamWaitEvent(s->copy_stream, s->ev_done[k], 0), "wait render");
            if (o.obs()) {
                CK(cudaMemcpyAsync(o.rgb8 + (size_t)rebase * 3, s->stage_rgb[k].p, (size_t)We * px * 3,
                                   cudaMemcpyDeviceToHost, s->copy_stream),
                   "copy rgb out");
                if (o.depth16)
                    CK(cudaMemcpyAsync(o.depth16 + rebase, s->stage_depth[k].p, (size_t)We * px * 2,
                                       cudaMemcpyDeviceToHost, s->copy_stream),
                       "copy depth out");
            } else {
                CK(cudaMemcpyAsync(rgb + (size_t)rebase * 3, s->stage_rgb[k].p, (size_t)We * px * 12,
                                   cudaMemcpyDeviceToHost, s->copy_stream),
                   "copy rgb out");
                CK(cudaMemcpyAsync(depth + rebase, s->stage_depth[k].p, (size_t)We * px * 4, cudaMemcpyDeviceToHost,
                                   s->copy_stream),
                   "copy depth out");
            }
            if (alpha)
                CK(cudaMemcpyAsync(alpha + rebase, s->stage_alpha[k].p, (size_t)We * px * 4, cudaMemcpyDeviceToHost,
                                   s->copy_stream),
                   "copy alpha out");
            CK(cudaEventRecord(s->ev_copied[k], s->copy_stream), "record");
            s->stats.waves++;
            ++wave;
        }
        CK(cudaStreamSynchronize(s->copy_stream), "sync copies");
        CK(cudaStreamSynchronize(st), "sync render");
    }
    s->stats.kernel_launches = launches;
    (void)E;
    return GS_OK;
}

gs_status clear_outputs(float* rgb, float* depth, float* alpha, size_t px, cudaStream_t st, bool host) {
    if (!rgb) return GS_OK;  // observation form: cleared by clear_obs
    if (host) {
        memset(rgb, 0, px * 12);
        memset(depth, 0, px * 4);
        if (alpha) memset(alpha, 0, px * 4);
        return GS_OK;
    }
    CK(cudaMemsetAsync(rgb, 0, px * 12, st), "clear rgb");
    CK(cudaMemsetAsync(depth, 0, px * 4, st), "clear depth");
    if (alpha) CK(cudaMemsetAsync(alpha, 0, px * 4, st), "clear alpha");
    return GS_OK;
}

// Device address of a page-locked host buffer (true, *dev set), true for
// NULL (nothing to write), false for memory the device cannot address as is.
template <typename T>
bool device_view(T* host, T** dev) {
    if (!host) {
        *dev = nullptr;
        return true;
    }
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();  // pageable memory may report an error: not direct
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = static_cast<T*>(a.devicePointer);
    return true;
}

// An empty scene in the observation form: every pixel of env e is the
// appearance transform of black (the same value in all three channels), depth 0.
gs_status clear_obs(const Outputs& o, int E, size_t px, const gs_appearance* appear_host, cudaStream_t st, bool host) {
    for (int e = 0; e < E; ++e) {
        float v = 0.0f;  // black through the transform: clamp(0.5 + brightness - 0.5 contrast)
        if (appear_host) v = std::fma(std::fma(0.0f, 1.0f, -0.5f), appear_host[e].contrast, 0.5f + appear_host[e].brightness);
        v = std::fmin(std::fmax(v, 0.0f), 1.0f);
        const int q = (int)std::nearbyint(v * 255.0f);
        uint8_t* dst = o.rgb8 + (size_t)e * px * 3;
        if (host) memset(dst, q, px * 3);
        else CK(cudaMemsetAsync(dst, q, px * 3, st), "clear rgb");
    }
    if (o.depth16) {
        if (host) memset(o.depth16, 0, (size_t)E * px * 2);
        else CK(cudaMemsetAsync(o.depth16, 0, (size_t)E * px * 2, st), "clear depth");
    }
    return GS_OK;
}

gs_status render_uniform(gs_scene s, int E, const float* link_poses, const gs_camera* cams, float* rgb, float* depth,
                         float* alpha, void* stream, bool host_mode, const Outputs* obs = nullptr) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (E < 0) return fail(GS_ERR_INVALID, "negative n_envs");
    if (E == 0) return GS_OK;
    if (!cams) return fail(GS_ERR_INVALID, "null cams");
    if (!obs && (!rgb || !depth)) return fail(GS_ERR_INVALID, "null rgb or depth output");
    if (obs && !obs->rgb8) return fail(GS_ERR_INVALID, "null rgb8 output");
    const int L = s->D.n_links;
    if (L > 0 && !link_poses) return fail(GS_ERR_INVALID, "null link_poses with %d links", L);
    const int W = cams[0].width, H = cams[0].height;
    for (int e = 0; e < E; ++e) {
        if (cams[e].width != W || cams[e].height != H)
            return fail(GS_ERR_INVALID, "camera %d: resolution %dx%d differs from camera 0 (%dx%d)", e,
                        cams[e].width, cams[e].height, W, H);
        ST(check_cam(cams[e], e));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(s->device), "set device");
    const long long px = (long long)W * H;
    Outputs o;
    if (obs) {
        o = *obs;
    } else {
        o.rgb = rgb;
        o.depth = depth;
        o.alpha = alpha;
    }
    std::vector<gs_appearance> ap_host;
    if (o.obs() && o.appear) {  // the appearance parameters on both sides of the bus
        ap_host.resize((size_t)E);
        if (host_mode) {
            memcpy(ap_host.data(), o.appear, sizeof(gs_appearance) * (size_t)E);
            CK(s->appear.ensure(sizeof(gs_appearance) * (size_t)E), "alloc appearance");
            CK(cudaMemcpyAsync(s->appear.p, o.appear, sizeof(gs_appearance) * (size_t)E, cudaMemcpyHostToDevice, st),
               "copy appearance");
            o.appear = s->appear.as<gs_appearance>();
        } else if (s->D.n == 0) {
            CK(cudaMemcpy(ap_host.data(), o.appear, sizeof(gs_appearance) * (size_t)E, cudaMemcpyDeviceToHost),
               "read appearance");
        }
    }
    if (s->D.n == 0) {
        if (o.obs()) return clear_obs(o, E, (size_t)px, ap_host.empty() ? nullptr : ap_host.data(), st, host_mode);
        return clear_outputs(rgb, depth, alpha, (size_t)E * px, st, host_mode);
    }
    std::vector<EnvSpec> specs((size_t)E);
    for (int e = 0; e < E; ++e) specs[e] = EnvSpec{cams + e, 0, L, (long long)e * L, (long long)e * px};
    const float* poses_dev = link_poses;
    if (host_mode && L > 0) {
        CK(s->poses.ensure((size_t)E * L * 28), "alloc poses");
        CK(cudaMemcpyAsync(s->poses.p, link_poses, (size_t)E * L * 28, cudaMemcpyHostToDevice, st), "copy poses");
        poses_dev = s->poses.as<float>();
    }
    if (host_mode) {
        // Pinned (page-locked) host outputs are mapped into the device's
        // address space: the compositor then stores the images straight into
        // them and no staging copy is needed; other host memory goes through
        // device staging and copies.
        Outputs m = o;
        const bool direct = device_view(o.rgb, &m.rgb) && device_view(o.depth, &m.depth) &&
                            device_view(o.alpha, &m.alpha) && device_view(o.rgb8, &m.rgb8) &&
                            device_view(o.depth16, &m.depth16);
        if (direct) {
            ST(render_specs(s, specs, poses_dev, m, st, Out::Device, px));
            CK(cudaStreamSynchronize(st), "sync render");
            return GS_OK;
        }
    }
    return render_specs(s, specs, poses_dev, o, st, host_mode ? Out::Host : Out::Device, px);
}

gs_status specs_from_envs(gs_scene s, int n, const gs_env* envs, std::vector<EnvSpec>* specs) {
    specs->resize((size_t)n);
    for (int e = 0; e < n; ++e) {
        const gs_env& v = envs[e];
        (*specs)[e] = EnvSpec{&v.cam, v.link_begin, v.link_end, (long long)v.pose_offset, (long long)v.pixel_offset};
    }
    (void)s;
    return GS_OK;
}

// ------------------------------------------------------------------ plans

gs_status plan_release_graph(gs_plan p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    return GS_OK;
}

// Build the plan's per-wave tables for the current tile shape (uploaded once).
gs_status plan_tables(gs_plan p, const std::vector<EnvSpec>& specs) {
    gs_scene s = p->s;
    std::vector<std::pair<int, int>> ranges;
    ST(plan_waves(s, specs, p->tile_w, p->tile_h, false, s->max_wave, 0, &ranges));
    std::vector<unsigned long long> caps;
    for (auto& w : p->waves) caps.push_back(w.cap);
    for (auto& w : p->waves) {
        w.envs.release();
        w.blocks.release();
        w.cams.release();
    }
    p->waves.clear();
    p->waves.resize(ranges.size());
    for (size_t i = 0; i < ranges.size(); ++i) {
        auto& w = p->waves[i];
        w.e0 = ranges[i].first;
        w.e1 = ranges[i].second;
        WaveTables wt{};
        ST(upload_tables(s, specs, w.e0, w.e1, p->tile_w, p->tile_h, 0, w.envs, w.blocks, w.cams, nullptr, true, &wt));
        w.n_blocks = wt.n_blocks;
        w.xf_items = wt.xf_items;
        w.max_words = wt.max_words;
        w.max_T = wt.max_T;
        w.recs = wt.recs;
        w.words = wt.words;
        w.tiles = wt.tiles;
        w.cap = i < caps.size() ? caps[i] : 0;
    }
    return GS_OK;
}

WaveTables plan_wave_tables(gs_plan p, size_t i, std::vector<EnvInfo>& host) {
    auto& w = p->waves[i];
    return WaveTables{w.envs.as<EnvInfo>(), w.blocks.as<ProjBlock>(), w.cams.as<gs_camera>(), w.e1 - w.e0,
                      w.n_blocks, w.xf_items, w.max_words, w.max_T, w.recs, w.words, w.tiles, host.data()};
}

// Eager pass over all waves (host syncs); records each wave's key total.
gs_status plan_eager(gs_plan p, const std::vector<EnvSpec>& specs, const float* poses, float* rgb, float* depth,
                     float* alpha, cudaStream_t st, std::vector<unsigned long long>* totals) {
    gs_scene s = p->s;
    totals->clear();
    int64_t launches = 0;
    for (size_t i = 0; i < p->waves.size(); ++i) {
        auto& w = p->waves[i];
        std::vector<EnvInfo> host((size_t)(w.e1 - w.e0) + 1);
        int nb = 0;
        std::vector<ProjBlock> dummy(1);
        build_wave_tables(s->D, s->link_offsets.data(), specs.data() + w.e0, w.e1 - w.e0, p->tile_w, p->tile_h, 0,
                          host.data(), dummy.data(), &nb, 0);
        WaveTables wt = plan_wave_tables(p, i, host);
        unsigned long long tot = 0;
        ST(run_wave(s, p->sc, wt, WaveIO{poses, rgb, depth, alpha, 0}, p->tile_w, p->tile_h, p->chunk, 0, st, false,
                    &launches, &tot, p->quad));
        totals->push_back(tot);
    }
    return GS_OK;
}

// Enqueue all waves in planned mode (no host sync) on st.
gs_status plan_enqueue(gs_plan p, const std::vector<EnvSpec>& specs, const float* poses, float* rgb, float* depth,
                       float* alpha, cudaStream_t st) {
    gs_scene s = p->s;
    int64_t launches = 0;
    for (size_t i = 0; i < p->waves.size(); ++i) {
        auto& w = p->waves[i];
        std::vector<EnvInfo> host((size_t)(w.e1 - w.e0) + 1);
        int nb = 0;
        std::vector<ProjBlock> dummy(1);
        build_wave_tables(s->D, s->link_offsets.data(), specs.data() + w.e0, w.e1 - w.e0, p->tile_w, p->tile_h, 0,
                          host.data(), dummy.data(), &nb, 0);
        WaveTables wt = plan_wave_tables(p, i, host);
        ST(run_wave(s, p->sc, wt, WaveIO{poses, rgb, depth, alpha, 0}, p->tile_w, p->tile_h, p->chunk, w.cap, st,
                    false, &launches, nullptr, p->quad));
    }
    return GS_OK;
}

}  // namespace gsb

gsb::SceneView gsb::scene_view(gs_scene s) {
    const bool perm = !s->bg_order.empty();
    return SceneView{s->device, s->D, s->status, s->tile_w, s->tile_h, perm ? s->bg_index.as<int>() : nullptr,
                     perm ? s->bg_slot.as<int>() : nullptr};
}

gs_status gsb::report(gs_status st, const char* msg) {
    g_err = msg;
    return st;
}

extern "C" {

const char* gs_last_error(void) { return g_err.c_str(); }

const char* gs_version(void) { return "gsbatch 0.2 (sm_103a)"; }

gs_status gs_scene_create(const gs_gaussians* background, gs_scene* out) {
    if (!out) return fail(GS_ERR_INVALID, "null output handle");
    *out = nullptr;
    gs_status v = check_view(background, "background");
    if (v != GS_OK) return v;
    gs_scene s = new gs_scene_s();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->status, 4);
    if (e == cudaSuccess) e = cudaMemset(s->status, 0, 4);
    if (e != cudaSuccess) {
        gs_scene_destroy(s);
        return cuda_fail(e, "scene create");
    }
    s->D.n = background->n;
    s->D.n_bg = background->n;
    s->D.n_links = 0;
    s->D.sh_degree = background->sh_degree;
    s->D.dtype = background->dtype;
    s->D.sh_planes = sh_planes_for(s->D.sh_degree, s->D.dtype);
    s->have_format = background->n > 0;
    gs_status r = alloc_gaussians(s->D.n, s->g0, s->g1, s->g2, s->g3, s->gsh, s->D.sh_planes);
    if (r == GS_OK) {
        s->D.p0 = s->g0.as<float4>();
        s->D.p1 = s->g1.as<float4>();
        s->D.p2 = s->g2.as<float4>();
        s->D.p3 = s->g3.as<float4>();
        s->D.sh = s->gsh.p;
        r = place_background(s, background);
    }
    if (r != GS_OK) {
        std::string msg = g_err;
        gs_scene_destroy(s);
        g_err = msg;
        return r;
    }
    s->stats.n_gaussians = s->D.n;
    *out = s;
    return GS_OK;
}

gs_status gs_scene_attach_links(gs_scene s, int n_links, const int64_t* link_offsets, const gs_gaussians* lg) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (n_links < 0) return fail(GS_ERR_INVALID, "negative n_links");
    if (n_links > 0 && !link_offsets) return fail(GS_ERR_INVALID, "null link_offsets");
    gs_gaussians empty{};
    empty.sh_degree = s->D.sh_degree;
    empty.dtype = s->D.dtype;
    if (!lg) {
        if (n_links > 0) return fail(GS_ERR_INVALID, "null link_gaussians");
        lg = &empty;
    }
    gs_status v = check_view(lg, "link_gaussians");
    if (v != GS_OK) return v;
    if (n_links > 0) {
        if (link_offsets[0] != 0) return fail(GS_ERR_INVALID, "link_offsets[0] must be 0");
        for (int l = 0; l < n_links; ++l)
            if (link_offsets[l + 1] < link_offsets[l]) return fail(GS_ERR_INVALID, "link_offsets must not decrease");
        if (link_offsets[n_links] != lg->n)
            return fail(GS_ERR_INVALID, "link_offsets[n_links] (%lld) != link_gaussians->n (%lld)",
                        (long long)link_offsets[n_links], (long long)lg->n);
    } else if (lg->n != 0) {
        return fail(GS_ERR_INVALID, "link Gaussians given with n_links = 0");
    }
    if (s->D.n_bg + lg->n > 0x7FFFFFF0ll) return fail(GS_ERR_UNSUPPORTED, "more than 2^31-16 Gaussians in total");
    if (lg->n > 0) {
        if (s->have_format && (lg->dtype != s->D.dtype || lg->sh_degree != s->D.sh_degree))
            return fail(GS_ERR_INVALID, "link Gaussians must use the background's dtype and sh_degree");
    }
    CK(cudaSetDevice(s->device), "set device");
    DevGaussians N = s->D;
    if (lg->n > 0 && !s->have_format) {
        N.dtype = lg->dtype;
        N.sh_degree = lg->sh_degree;
        N.sh_planes = sh_planes_for(N.sh_degree, N.dtype);
    }
    N.n = s->D.n_bg + lg->n;
    N.n_links = n_links;
    DevBuf a, b, c, d, sh;
    gs_status r = alloc_gaussians(N.n, a, b, c, d, sh, N.sh_planes);
    if (r != GS_OK) {
        a.release(); b.release(); c.release(); d.release(); sh.release();
        return r;
    }
    N.p0 = a.as<float4>();
    N.p1 = b.as<float4>();
    N.p2 = c.as<float4>();
    N.p3 = d.as<float4>();
    N.sh = sh.p;
    const int64_t nb = s->D.n_bg;
    cudaError_t e = cudaSuccess;
    if (nb > 0) {
        e = cudaMemcpy(N.p0, s->D.p0, nb * 16, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(N.p1, s->D.p1, nb * 16, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(N.p2, s->D.p2, nb * 16, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(N.p3, s->D.p3, nb * 16, cudaMemcpyDeviceToDevice);
        for (int pl = 0; pl < N.sh_planes && e == cudaSuccess; ++pl)
            e = cudaMemcpy(static_cast<char*>(N.sh) + (size_t)pl * N.n * 16,
                           static_cast<char*>(s->D.sh) + (size_t)pl * s->D.n * 16, nb * 16, cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) {
        a.release(); b.release(); c.release(); d.release(); sh.release();
        return cuda_fail(e, "copy background");
    }
    DevGaussians old = s->D;
    s->D = N;
    r = prep_view(s, lg, nb, 1, link_offsets, n_links);
    if (r != GS_OK) {
        s->D = old;
        a.release(); b.release(); c.release(); d.release(); sh.release();
        return r;
    }
    s->g0.release(); s->g1.release(); s->g2.release(); s->g3.release(); s->gsh.release();
    s->g0 = a; s->g1 = b; s->g2 = c; s->g3 = d; s->gsh = sh;
    s->link_offsets.assign(link_offsets ? link_offsets : nullptr, link_offsets ? link_offsets + n_links + 1 : nullptr);
    if (s->link_offsets.empty()) s->link_offsets.assign(1, 0);
    if (lg->n > 0) s->have_format = true;
    s->stats.n_gaussians = s->D.n;
    return GS_OK;
}

gs_status gs_render_batch(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                          float* depth, float* alpha, void* cuda_stream) {
    return render_uniform(s, n_envs, link_poses, cams, rgb, depth, alpha, cuda_stream, false);
}

gs_status gs_render_batch_host(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                               float* depth, float* alpha, void* cuda_stream) {
    return render_uniform(s, n_envs, link_poses, cams, rgb, depth, alpha, cuda_stream, true);
}

namespace {

// Batch-LiDAR scans on the sensors' (azimuth, beam) grids; with ray_dirs,
// along the given rays instead (the grid then only bins them).
gs_status lidar_scan(gs_scene s, int n_envs, const float* link_poses, const gs_lidar* sensors, const float* ray_dirs,
                     int n_rays, float* range, float* hit, void* cuda_stream) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (n_envs < 0) return fail(GS_ERR_INVALID, "negative n_envs");
    if (n_envs == 0) return GS_OK;
    if (!sensors || !range) return fail(GS_ERR_INVALID, "null sensors or range output");
    if (ray_dirs && (n_rays < 1 || n_rays > (1 << 24)))
        return fail(GS_ERR_INVALID, "n_rays %d outside [1, 2^24]", n_rays);
    const int L = s->D.n_links;
    if (L > 0 && !link_poses) return fail(GS_ERR_INVALID, "null link_poses with %d links", L);
    const int rows = sensors[0].rows, cols = sensors[0].cols;
    std::vector<gs_camera> cams((size_t)n_envs);
    for (int e = 0; e < n_envs; ++e) {
        const gs_lidar& l = sensors[e];
        if (l.rows != rows || l.cols != cols)
            return fail(GS_ERR_INVALID, "sensor %d: %dx%d rays differ from sensor 0 (%dx%d)", e, l.rows, l.cols, rows,
                        cols);
        if (l.rows <= 0 || l.cols <= 0 || l.rows > 65535 || l.cols > 65535)
            return fail(GS_ERR_INVALID, "sensor %d: bad ray grid %dx%d", e, l.rows, l.cols);
        if (!(l.elev_min < l.elev_max) || !(l.elev_min > -1.5707963f) || !(l.elev_max < 1.5707963f))
            return fail(GS_ERR_INVALID, "sensor %d: elevation range must lie in (-pi/2, pi/2)", e);
        if (!(l.near_range > 0.0f) || !std::isfinite(l.near_range))
            return fail(GS_ERR_INVALID, "sensor %d: near_range must be > 0", e);
        if (!std::isfinite(l.az_min) || !std::isfinite(l.az_max) || !(l.az_min < l.az_max) ||
            !((double)l.az_max - (double)l.az_min <= 6.283186))  // 2 pi, with the rounding of float(2 pi)
            return fail(GS_ERR_INVALID, "sensor %d: azimuth window must satisfy az_min < az_max <= az_min + 2 pi", e);
        // the pose travels to the link-table kernel as a camera of the grid's size
        gs_camera& c = cams[e];
        c.fx = c.fy = 1.0f;
        c.cx = 0.5f * (float)cols;
        c.cy = 0.5f * (float)rows;
        c.width = cols;
        c.height = rows;
        for (int k = 0; k < 4; ++k) c.q_cw[k] = l.q_ws[k];
        for (int k = 0; k < 3; ++k) c.t_cw[k] = l.t_ws[k];
        c.near_plane = l.near_range;
        ST(check_cam(c, e));
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaSetDevice(s->device), "set device");
    const size_t px = ray_dirs ? (size_t)n_rays : (size_t)rows * cols;  // outputs per env
    if (s->D.n == 0 || ray_dirs) {  // rays outside their grid (and an empty scene) read 0
        CK(cudaMemsetAsync(range, 0, (size_t)n_envs * px * 4, st), "clear range");
        if (hit) CK(cudaMemsetAsync(hit, 0, (size_t)n_envs * px * 4, st), "clear hit");
        if (s->D.n == 0) return GS_OK;
    }
    const int tw = 16, th = 16;
    std::vector<EnvSpec> specs((size_t)n_envs);
    for (int e = 0; e < n_envs; ++e) specs[e] = EnvSpec{&cams[e], 0, L, (long long)e * L, (long long)e * (long long)px};
    ST(check_specs(s, specs, tw, th));
    std::vector<std::pair<int, int>> waves;
    ST(plan_waves(s, specs, tw, th, false, s->max_wave, 0, &waves));
    int64_t launches = 0;
    for (auto& w : waves) {
        const int We = w.second - w.first;
        CK(s->lidar_tab.ensure(sizeof(gs_lidar) * (size_t)We), "alloc sensors");
        CK(cudaMemcpyAsync(s->lidar_tab.p, sensors + w.first, sizeof(gs_lidar) * (size_t)We, cudaMemcpyHostToDevice,
                           st),
           "copy sensors");
        WaveTables wt{};
        ST(upload_tables(s, specs, w.first, w.second, tw, th, 0, s->sc.envs, s->sc.blocks, s->sc.cams, st, false,
                         &wt));
        WaveIO io{link_poses, nullptr, range, hit, 0};
        io.lidars = s->lidar_tab.as<gs_lidar>();
        if (ray_dirs) {
            io.ray_dirs = ray_dirs + (size_t)w.first * (size_t)n_rays * 3;
            io.n_rays = n_rays;
        }
        ST(run_wave(s, s->sc, wt, io, tw, th, 1, 0, st, true, &launches, nullptr));
        s->stats.waves++;
    }
    s->stats.kernel_launches = launches;
    return GS_OK;
}

}  // namespace

gs_status gs_render_lidar(gs_scene s, int n_envs, const float* link_poses, const gs_lidar* sensors, float* range,
                          float* hit, void* cuda_stream) {
    return lidar_scan(s, n_envs, link_poses, sensors, nullptr, 0, range, hit, cuda_stream);
}

gs_status gs_render_rays(gs_scene s, int n_envs, const float* link_poses, const gs_lidar* sensors, int n_rays,
                         const float* ray_dirs, float* range, float* hit, void* cuda_stream) {
    if (!ray_dirs) return fail(GS_ERR_INVALID, "null ray_dirs");
    return lidar_scan(s, n_envs, link_poses, sensors, ray_dirs, n_rays, range, hit, cuda_stream);
}

gs_status gs_scene_contribution(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                float* scores, void* cuda_stream) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (n_envs < 0) return fail(GS_ERR_INVALID, "negative n_envs");
    if (n_envs == 0 || s->D.n == 0) return GS_OK;
    if (!cams || !scores) return fail(GS_ERR_INVALID, "null cams or scores");
    const int L = s->D.n_links;
    if (L > 0 && !link_poses) return fail(GS_ERR_INVALID, "null link_poses with %d links", L);
    for (int e = 0; e < n_envs; ++e) ST(check_cam(cams[e], e));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaSetDevice(s->device), "set device");
    const int tw = 16, th = 16;  // the contribution pass bins and composites on 16x16 tiles
    std::vector<EnvSpec> specs((size_t)n_envs);
    for (int e = 0; e < n_envs; ++e) specs[e] = EnvSpec{cams + e, 0, L, (long long)e * L, 0};
    ST(check_specs(s, specs, tw, th));
    std::vector<std::pair<int, int>> waves;
    ST(plan_waves(s, specs, tw, th, false, s->max_wave, 0, &waves));
    int64_t launches = 0;
    for (auto& w : waves) {
        WaveTables wt{};
        ST(upload_tables(s, specs, w.first, w.second, tw, th, 0, s->sc.envs, s->sc.blocks, s->sc.cams, st, false,
                         &wt));
        WaveIO io{link_poses, nullptr, nullptr, nullptr, 0};
        io.score = scores;
        ST(run_wave(s, s->sc, wt, io, tw, th, 1, 0, st, false, &launches, nullptr));
    }
    return GS_OK;
}

gs_status gs_render_batch_obs(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                              const gs_appearance* appearance, uint8_t* rgb8, uint16_t* depth16, void* cuda_stream) {
    Outputs o;
    o.rgb8 = rgb8;
    o.depth16 = depth16;
    o.appear = appearance;
    return render_uniform(s, n_envs, link_poses, cams, nullptr, nullptr, nullptr, cuda_stream, false, &o);
}

gs_status gs_render_batch_obs_host(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                   const gs_appearance* appearance, uint8_t* rgb8, uint16_t* depth16,
                                   void* cuda_stream) {
    Outputs o;
    o.rgb8 = rgb8;
    o.depth16 = depth16;
    o.appear = appearance;
    return render_uniform(s, n_envs, link_poses, cams, nullptr, nullptr, nullptr, cuda_stream, true, &o);
}

gs_status gs_render_batch_v(gs_scene s, int n_envs, const gs_env* envs, const float* link_poses, float* rgb,
                            float* depth, float* alpha, void* cuda_stream) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (n_envs < 0) return fail(GS_ERR_INVALID, "negative n_envs");
    if (n_envs == 0) return GS_OK;
    if (!envs || !rgb || !depth) return fail(GS_ERR_INVALID, "null envs, rgb or depth");
    bool any_links = false;
    for (int e = 0; e < n_envs; ++e) any_links |= envs[e].link_end > envs[e].link_begin;
    if (any_links && !link_poses) return fail(GS_ERR_INVALID, "null link_poses");
    std::vector<EnvSpec> specs;
    ST(specs_from_envs(s, n_envs, envs, &specs));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaSetDevice(s->device), "set device");
    if (s->D.n == 0) {
        ST(check_specs(s, specs, s->tile_w, s->tile_h));
        for (int e = 0; e < n_envs; ++e) {
            const size_t px = (size_t)envs[e].cam.width * envs[e].cam.height;
            ST(clear_outputs(rgb + envs[e].pixel_offset * 3, depth + envs[e].pixel_offset,
                             alpha ? alpha + envs[e].pixel_offset : nullptr, px, st, false));
        }
        return GS_OK;
    }
    Outputs o;
    o.rgb = rgb;
    o.depth = depth;
    o.alpha = alpha;
    return render_specs(s, specs, link_poses, o, st, Out::Device, 0);
}

gs_status gs_plan_create(gs_scene s, int n_envs, const gs_env* envs, int flags, gs_plan* out) {
    if (!out) return fail(GS_ERR_INVALID, "null output handle");
    *out = nullptr;
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (n_envs <= 0 || !envs) return fail(GS_ERR_INVALID, "a plan needs n_envs > 0 environments");
    gs_plan p = new gs_plan_s();
    p->s = s;
    p->flags = flags;
    p->envs.assign(envs, envs + n_envs);
    // Render low-resolution envs first: their tiles have the longest buckets,
    // so the persistent compositor claims them early instead of finishing on
    // them.  Outputs are placed by pixel_offset, so the order is not visible.
    std::stable_sort(p->envs.begin(), p->envs.end(), [](const gs_env& a, const gs_env& b) {
        const int64_t pa = (int64_t)a.cam.width * a.cam.height, pb = (int64_t)b.cam.width * b.cam.height;
        if (pa != pb) return pa < pb;
        if (a.link_begin != b.link_begin) return a.link_begin < b.link_begin;
        return a.link_end < b.link_end;
    });
    p->tile_w = s->tile_w;
    p->tile_h = s->tile_h;
    std::vector<EnvSpec> specs;
    specs_from_envs(s, n_envs, p->envs.data(), &specs);
    gs_status r = check_specs(s, specs, 8, 8);
    if (r == GS_OK) r = check_specs(s, specs, p->tile_w, p->tile_h);
    if (r != GS_OK) {
        delete p;
        return r;
    }
    cudaSetDevice(s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->pinned_status, 4);
    if (e != cudaSuccess) {
        gs_plan_destroy(p);
        return cuda_fail(e, "plan create");
    }
    *p->pinned_status = 0;
    *out = p;
    return GS_OK;
}

gs_status gs_plan_launch(gs_plan p, const float* link_poses, float* rgb, float* depth, float* alpha,
                         void* cuda_stream) {
    if (!p) return fail(GS_ERR_INVALID, "null plan");
    if (!rgb || !depth) return fail(GS_ERR_INVALID, "null rgb or depth");
    gs_scene s = p->s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaSetDevice(s->device), "set device");
    std::vector<EnvSpec> specs;
    specs_from_envs(s, (int)p->envs.size(), p->envs.data(), &specs);
    bool any_links = false;
    for (auto& v : p->envs) any_links |= v.link_end > v.link_begin;
    if (any_links && !link_poses) return fail(GS_ERR_INVALID, "null link_poses");
    if (s->D.n == 0) {
        for (auto& v : p->envs)
            ST(clear_outputs(rgb + v.pixel_offset * 3, depth + v.pixel_offset, alpha ? alpha + v.pixel_offset : nullptr,
                             (size_t)v.cam.width * v.cam.height, st, false));
        return GS_OK;
    }
    // a previous planned launch that overflowed its key capacity: regrow and re-plan
    if (p->tuned && p->launched && cudaEventQuery(p->done) == cudaSuccess && (*p->pinned_status & kStOverflow)) {
        // re-measure with the current poses (an eager, host-synchronising pass)
        *p->pinned_status = 0;
        CK(cudaMemsetAsync(s->status, 0, 4, st), "status clear");
        std::vector<unsigned long long> tot;
        ST(plan_eager(p, specs, link_poses, rgb, depth, alpha, st, &tot));
        for (size_t i = 0; i < p->waves.size() && i < tot.size(); ++i)
            p->waves[i].cap = std::max(p->waves[i].cap, tot[i] + tot[i] / 4 + 4096);
        plan_release_graph(p);
        p->regrows++;
    }
    if (!p->tuned) {
        // eager warm-up: autotune (tile shape x claim size) and size the key capacity
        struct Cand {
            int tw, th, chunk, quad;
        };
        std::vector<Cand> cands;
        if (p->flags & GS_PLAN_AUTOTUNE) {
            const int shapes[5][2] = {{16, 16}, {32, 8}, {16, 8}, {8, 8}, {32, 16}};
            for (auto& sh : shapes)
                for (int ch : {1, 4}) {
                    cands.push_back({sh[0], sh[1], ch, 0});
                    if (sh[0] == sh[1]) cands.push_back({sh[0], sh[1], ch, 1});  // quadrant form: 16x16, 8x8
                }
        } else {
            cands.push_back({p->tile_w, p->tile_h, 1, 0});
        }
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a), "event");
        CK(cudaEventCreate(&b), "event");
        double best = 1e30;
        Cand bestc = cands[0];
        std::vector<unsigned long long> best_tot;
        for (const Cand& c : cands) {
            if (check_specs(s, specs, c.tw, c.th) != GS_OK) continue;
            p->tile_w = c.tw;
            p->tile_h = c.th;
            p->chunk = c.chunk;
            p->quad = c.quad;
            ST(plan_tables(p, specs));
            std::vector<unsigned long long> tot;
            ST(plan_eager(p, specs, link_poses, rgb, depth, alpha, st, &tot));  // warm (sizes buffers)
            CK(cudaEventRecord(a, st), "record");
            ST(plan_eager(p, specs, link_poses, rgb, depth, alpha, st, &tot));
            CK(cudaEventRecord(b, st), "record");
            CK(cudaEventSynchronize(b), "sync");
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, a, b), "elapsed");
            if (ms < best) {
                best = ms;
                bestc = c;
                best_tot = tot;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        p->tile_w = bestc.tw;
        p->tile_h = bestc.th;
        p->chunk = bestc.chunk;
        p->quad = bestc.quad;
        p->tuned_candidates = (int)cands.size();
        p->tuned_ms = best;
        ST(plan_tables(p, specs));
        for (size_t i = 0; i < p->waves.size(); ++i) {
            const unsigned long long t = i < best_tot.size() ? best_tot[i] : 0;
            p->waves[i].cap = t + t / 4 + 4096;  // headroom for pose-dependent growth
        }
        p->sc.pairs.release();
        p->tuned = true;
        plan_release_graph(p);
    }
    const void* ptrs[4] = {link_poses, rgb, depth, alpha};
    const bool same = memcmp(ptrs, p->cap_ptrs, sizeof ptrs) == 0;
    if (!(p->flags & GS_PLAN_GRAPH)) {
        ST(plan_enqueue(p, specs, link_poses, rgb, depth, alpha, st));
        CK(cudaMemcpyAsync(p->pinned_status, s->status, 4, cudaMemcpyDeviceToHost, st), "status copy");
    } else {
        if (!p->exec || !same) {
            plan_release_graph(p);
            // grow every buffer the graph will reference before capturing it
            ST(plan_enqueue(p, specs, link_poses, rgb, depth, alpha, st));
            CK(cudaStreamSynchronize(st), "sync");
            CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            gs_status r = plan_enqueue(p, specs, link_poses, rgb, depth, alpha, p->cap_stream);
            cudaError_t ce = cudaMemcpyAsync(p->pinned_status, s->status, 4, cudaMemcpyDeviceToHost, p->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t ee = cudaStreamEndCapture(p->cap_stream, &g);
            if (r != GS_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            CK(ce, "status copy");
            CK(ee, "end capture");
            p->graph = g;
            CK(cudaGraphInstantiate(&p->exec, g, 0), "instantiate graph");
            memcpy(p->cap_ptrs, ptrs, sizeof ptrs);
        }
        CK(cudaGraphLaunch(p->exec, st), "graph launch");
    }
    CK(cudaEventRecord(p->done, st), "record");
    p->launched = true;
    return GS_OK;
}

gs_status gs_plan_get_info(gs_plan p, gs_plan_info* out) {
    if (!p || !out) return fail(GS_ERR_INVALID, "null argument");
    gs_plan_info i{};
    i.tile_w = p->tile_w;
    i.tile_h = p->tile_h;
    i.chunk = p->chunk;
    i.quad = p->quad;
    i.waves = (int)p->waves.size();
    i.graph = p->exec != nullptr;
    i.tuned_candidates = p->tuned_candidates;
    i.tuned_ms = p->tuned_ms;
    i.regrows = p->regrows;
    for (auto& w : p->waves) i.key_capacity += (int64_t)w.cap;
    i.scratch_bytes = p->sc.bytes();
    *out = i;
    return GS_OK;
}

void gs_plan_destroy(gs_plan p) {
    if (!p) return;
    if (p->s) cudaSetDevice(p->s->device);
    cudaDeviceSynchronize();
    plan_release_graph(p);
    for (auto& w : p->waves) {
        w.envs.release();
        w.blocks.release();
        w.cams.release();
    }
    p->sc.release();
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->done) cudaEventDestroy(p->done);
    if (p->pinned_status) cudaFreeHost(p->pinned_status);
    delete p;
}

gs_status gs_scene_set_tile(gs_scene s, int tw, int th) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (!valid_tile(tw, th)) return fail(GS_ERR_INVALID, "tile %dx%d not one of 8x8, 16x8, 16x16, 32x8, 32x16", tw, th);
    s->tile_w = tw;
    s->tile_h = th;
    return GS_OK;
}

gs_status gs_scene_set_budget(gs_scene s, int64_t bytes) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (bytes < (1ll << 20)) return fail(GS_ERR_INVALID, "budget below 1 MiB");
    s->budget = bytes;
    return GS_OK;
}

gs_status gs_scene_set_wave(gs_scene s, int max_envs) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (max_envs < 0) return fail(GS_ERR_INVALID, "negative wave size");
    s->max_wave = max_envs;
    return GS_OK;
}

gs_status gs_scene_set_debug(gs_scene s, int enable) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    s->debug = enable ? 1 : 0;
    return GS_OK;
}

gs_status gs_scene_sync_status(gs_scene s, void* cuda_stream) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    CK(cudaSetDevice(s->device), "set device");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)), "sync");
    uint32_t st = 0;
    CK(cudaMemcpy(&st, s->status, 4, cudaMemcpyDeviceToHost), "status read");
    CK(cudaMemset(s->status, 0, 4), "status clear");
    if (st == 0) return GS_OK;
    std::string m = "device status:";
    if (st & kStBadPose) m += " zero or non-finite link pose;";
    if (st & kStBadScene) m += " bad Gaussian quaternion;";
    if (st & kStOverflow) m += " intersection keys beyond capacity (planned launch) or corrupted bucket;";
    g_err = m;
    return GS_ERR_DEVICE;
}

gs_status gs_scene_set_counters(gs_scene s, int enable) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    s->counters = enable ? 1 : 0;
    if (s->counters) {
        CK(cudaSetDevice(s->device), "set device");
        CK(s->neval.ensure(24), "alloc counters");
        CK(cudaMemset(s->neval.p, 0, 24), "clear counters");
    }
    return GS_OK;
}

gs_status gs_scene_set_profile(gs_scene s, int enable) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    s->profile = enable ? 1 : 0;
    return GS_OK;
}

gs_status gs_scene_get_timings(gs_scene s, gs_timings* out, int reset) {
    if (!s || !out) return fail(GS_ERR_INVALID, "null argument");
    CK(cudaSetDevice(s->device), "set device");
    for (auto& m : s->marks) {
        CK(cudaEventSynchronize(m.b), "wait profile event");
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, m.a, m.b), "profile elapsed");
        s->prof_ms[m.phase] += ms;
        s->prof_launches[m.phase] += m.kernels;
        s->event_pool.push_back(m.a);
        s->event_pool.push_back(m.b);
    }
    s->marks.clear();
    for (int k = 0; k < GS_PHASES; ++k) {
        out->ms[k] = s->prof_ms[k];
        out->launches[k] = s->prof_launches[k];
        if (reset) {
            s->prof_ms[k] = 0;
            s->prof_launches[k] = 0;
        }
    }
    return GS_OK;
}

gs_status gs_scene_get_stats(gs_scene s, gs_stats* out) {
    if (!s || !out) return fail(GS_ERR_INVALID, "null argument");
    s->stats.n_gaussians = s->D.n;
    int64_t bytes = s->sc.bytes();
    const DevBuf* bufs[] = {&s->stage_rgb[0], &s->stage_rgb[1], &s->stage_depth[0], &s->stage_depth[1],
                            &s->stage_alpha[0], &s->stage_alpha[1], &s->poses};
    for (const DevBuf* b : bufs) bytes += (int64_t)b->bytes;
    s->stats.scratch_bytes = bytes;
    s->stats.composited = 0;
    s->stats.visible = 0;
    s->stats.fp64_conics = 0;
    if (s->counters && s->neval.p) {
        CK(cudaSetDevice(s->device), "set device");
        CK(cudaDeviceSynchronize(), "sync");
        unsigned long long c[3] = {0, 0, 0};
        CK(cudaMemcpy(c, s->neval.p, 24, cudaMemcpyDeviceToHost), "read counters");
        s->stats.composited = (int64_t)c[0];
        s->stats.visible = (int64_t)c[1];
        s->stats.fp64_conics = (int64_t)c[2];
    }
    *out = s->stats;
    return GS_OK;
}

gs_status gs_debug_copy_records(gs_scene s, int env, uint8_t* visible, float* u, float* v, float* hx, float* hy,
                                float* z, float* opacity, float* conic, float* rgb, int32_t* range) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (s->last_e0 < 0 || env < s->last_e0 || env >= s->last_e0 + s->last_We)
        return fail(GS_ERR_INVALID, "env %d is not in the last wave rendered", env);
    if (!s->debug || !s->sc.dbg_hxy.p) return fail(GS_ERR_INVALID, "debug was not enabled for the last render");
    CK(cudaSetDevice(s->device), "set device");
    CK(cudaDeviceSynchronize(), "sync");
    const EnvInfo& E = s->last_envs[env - s->last_e0];
    const int64_t n_local = E.n_local, nbp = bg_slots(s->D.n_bg);
    const int64_t lg0 = s->D.n_bg + s->link_offsets[E.link_begin];
    std::vector<uint32_t> mask((n_local + 31) / 32);
    std::vector<float4> a(n_local), b(n_local), c(n_local);
    std::vector<float2> h(n_local);
    CK(cudaMemcpy(mask.data(), s->sc.mask.as<uint32_t>() + E.mask_base, mask.size() * 4, cudaMemcpyDeviceToHost),
       "copy");
    const float4* rec = s->sc.r012.as<float4>() + (size_t)kRecStride * E.rec_base;
    const size_t pitch = 16 * kRecStride;
    CK(cudaMemcpy2D(a.data(), 16, rec, pitch, 16, n_local, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy2D(b.data(), 16, rec + 1, pitch, 16, n_local, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy2D(c.data(), 16, rec + 2, pitch, 16, n_local, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(h.data(), s->sc.dbg_hxy.as<float2>() + E.rec_base, n_local * 8, cudaMemcpyDeviceToHost), "copy");
    if (visible) memset(visible, 0, (size_t)s->D.n);
    for (int64_t j = 0; j < n_local; ++j) {
        if (j >= s->D.n_bg && j < nbp) continue;  // padding slots
        const int64_t g = j < s->D.n_bg ? s->bg_order[(size_t)j] : lg0 + (j - nbp);
        const bool vis = (mask[j >> 5] >> (j & 31)) & 1u;
        if (visible) visible[g] = vis ? 1 : 0;
        if (!vis) continue;
        if (u) u[g] = a[j].x;
        if (v) v[g] = a[j].y;
        if (opacity) opacity[g] = a[j].z;
        if (z) z[g] = a[j].w;
        if (conic) {  // records hold L with L^T L = conic * 0.5 log2(e) (upper triangular)
            const double k2 = 0.72134752044448170;
            const double l00 = b[j].x, l01 = b[j].y, l11 = b[j].z;
            conic[3 * g] = (float)(l00 * l00 / k2);
            conic[3 * g + 1] = (float)(l00 * l01 / k2);
            conic[3 * g + 2] = (float)((l01 * l01 + l11 * l11) / k2);
        }
        if (rgb) {
            rgb[3 * g] = c[j].x;
            rgb[3 * g + 1] = c[j].y;
            rgb[3 * g + 2] = c[j].z;
        }
        if (hx) hx[g] = h[j].x;
        if (hy) hy[g] = h[j].y;
        if (range) {
            uint32_t rx, ry;
            float fx = b[j].w, fy = c[j].w;
            memcpy(&rx, &fx, 4);
            memcpy(&ry, &fy, 4);
            range[4 * g] = (int32_t)(rx & 0xffffu);
            range[4 * g + 1] = (int32_t)(rx >> 16);
            range[4 * g + 2] = (int32_t)(ry & 0xffffu);
            range[4 * g + 3] = (int32_t)(ry >> 16);
        }
    }
    return GS_OK;
}

gs_status gs_debug_copy_tiles(gs_scene s, int env, uint32_t* counts, int64_t n_counts, uint32_t* lists,
                              int64_t n_lists) {
    if (!s || !counts) return fail(GS_ERR_INVALID, "null argument");
    if (s->last_e0 < 0 || env < s->last_e0 || env >= s->last_e0 + s->last_We)
        return fail(GS_ERR_INVALID, "env %d is not in the last wave rendered", env);
    const int el = env - s->last_e0;
    const EnvInfo& E = s->last_envs[el];
    if (n_counts < E.T) return fail(GS_ERR_INVALID, "counts holds %lld < %d tiles", (long long)n_counts, E.T);
    CK(cudaSetDevice(s->device), "set device");
    CK(cudaDeviceSynchronize(), "sync");
    CK(cudaMemcpy(counts, s->sc.counts.as<uint32_t>() + E.tile_base, (size_t)E.T * 4, cudaMemcpyDeviceToHost),
       "copy counts");
    if (!lists) return GS_OK;
    if (!s->debug || !s->sc.dbg_sorted.p) return fail(GS_ERR_INVALID, "debug was not enabled for the last render");
    if (el < s->last_ea || el >= s->last_eb)
        return fail(GS_ERR_INVALID, "env %d is not in the last sub-wave rendered", env);
    unsigned long long base = 0, total = 0;
    CK(cudaMemcpy(&base, s->sc.env_base.as<unsigned long long>() + el, 8, cudaMemcpyDeviceToHost), "copy base");
    CK(cudaMemcpy(&total, s->sc.env_base.as<unsigned long long>() + el + 1, 8, cudaMemcpyDeviceToHost), "copy base");
    total -= base;
    if ((unsigned long long)n_lists < total)
        return fail(GS_ERR_INVALID, "lists holds %lld < %llu entries", (long long)n_lists, total);
    std::vector<unsigned long long> keys(total > 0 ? total : 1);
    if (total > 0)
        CK(cudaMemcpy(keys.data(), s->sc.dbg_sorted.as<unsigned long long>() + (base - s->last_pair_base), total * 8,
                      cudaMemcpyDeviceToHost),
           "copy lists");
    const int64_t nbp = bg_slots(s->D.n_bg), lg0 = s->D.n_bg + s->link_offsets[E.link_begin];
    for (unsigned long long i = 0; i < total; ++i) {
        const int64_t j = (int64_t)(keys[i] & 0xffffffffull);
        lists[i] = (uint32_t)(j < s->D.n_bg ? j : lg0 + (j - nbp));  // keys carry the caller's index
    }
    return GS_OK;
}

gs_status gs_scene_get_order(gs_scene s, int64_t* order, int64_t n) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    const int64_t nb = s->D.n_bg;
    if (nb == 0) return GS_OK;
    if (!order) return fail(GS_ERR_INVALID, "null order");
    if (n < nb) return fail(GS_ERR_INVALID, "order holds %lld < %lld entries", (long long)n, (long long)nb);
    for (int64_t k = 0; k < nb; ++k) order[k] = (int64_t)s->bg_order[(size_t)k];
    return GS_OK;
}

void gs_scene_destroy(gs_scene s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&s->g0, &s->g1, &s->g2, &s->g3, &s->gsh, &s->stage_rgb[0], &s->stage_rgb[1],
                      &s->stage_depth[0], &s->stage_depth[1], &s->stage_alpha[0], &s->stage_alpha[1], &s->poses,
                      &s->neval, &s->appear, &s->lidar_tab, &s->bg_index, &s->bg_slot, &s->ray_cell,
                      &s->ray_list, &s->ray_cnt, &s->ray_off, &s->ray_cur, &s->item_cnt, &s->item_off,
                      &s->ray_tot, &s->ray_base, &s->item_tot, &s->item_base};
    for (DevBuf* b : bufs) b->release();
    s->sc.release();
    for (auto& m : s->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->status) cudaFree(s->status);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    for (int k = 0; k < 2; ++k) {
        if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
        if (s->ev_copied[k]) cudaEventDestroy(s->ev_copied[k]);
    }
    delete s;
}

}  // extern "C"
