// C ABI of libgsbatch: scenes, batched rendering, status and debug hooks.
//
// The call sequence follows the paper's loop (Sec. III-A "Data Flow"): poses
// from the physics step -> RLGK (Sec. III-C) -> batch 3DGS renderer (Sec.
// III-C "Throughput Scaling") -> RGB + depth per environment.  Every step of
// the render runs in the kernels of gs_project.cu, gs_bin.cu and
// gs_composite.cu; this file validates arguments, plans waves of
// environments against the scratch budget and orders the launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gs_internal.cuh"

using namespace gsb;

namespace {

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

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
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

}  // namespace

struct gs_scene_s {
    int device = 0;
    DevGaussians D;
    DevBuf g0, g1, g2, g3, gsh;
    bool have_format = false;  // dtype / degree fixed by the first non-empty set
    uint32_t* status = nullptr;
    int tile_w = 16, tile_h = 16;
    int64_t budget = 64ll << 30;
    int max_wave = 0;
    int debug = 0;
    // scratch
    DevBuf xf, cams, poses, r0, r1, r2, r3, mask, counts, off, cursor, env_total, env_base, pairs, dbg_hxy,
        dbg_sorted;
    DevBuf stage_rgb[2], stage_depth[2], stage_alpha[2];
    unsigned long long* pinned = nullptr;
    size_t pinned_n = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    // what the last render left for the debug hooks
    int last_e0 = -1, last_We = 0, last_ea = 0, last_eb = 0, last_W = 0, last_H = 0, last_T = 0;
    unsigned long long last_pair_base = 0;
    int64_t last_pairs = 0;
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
    DevBuf neval;
};

namespace {

gs_status check_view(const gs_gaussians* g, const char* name) {
    if (!g) return fail(GS_ERR_INVALID, "%s: null gs_gaussians", name);
    if (g->n < 0) return fail(GS_ERR_INVALID, "%s: negative n", name);
    if (g->n > 0xFFFFFFF0ll) return fail(GS_ERR_UNSUPPORTED, "%s: more than 2^32-16 Gaussians", name);
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
gs_status prep_view(gs_scene s, const gs_gaussians* g, int64_t dst, int link_mode, const int64_t* link_offsets_host,
                    int n_links) {
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
    if (e == cudaSuccess)
        e = launch_prep(static_cast<const float*>(mean), static_cast<const float*>(quat), ls, op, sh, n, dst, link_mode,
                        offs, n_links, s->D, s->status, 0);
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

gs_status alloc_gaussians(gs_scene s, int64_t n, DevBuf& a, DevBuf& b, DevBuf& c, DevBuf& d, DevBuf& sh,
                          int planes) {
    const size_t m = (size_t)(n > 0 ? n : 1);
    CK(a.ensure(m * 16), "alloc p0");
    CK(b.ensure(m * 16), "alloc p1");
    CK(c.ensure(m * 16), "alloc p2");
    CK(d.ensure(m * 16), "alloc p3");
    CK(sh.ensure(m * 16 * (size_t)(planes > 0 ? planes : 1)), "alloc sh");
    (void)s;
    return GS_OK;
}

gs_status check_cams(const gs_camera* cams, int E, int* W, int* H) {
    for (int e = 0; e < E; ++e) {
        const gs_camera& c = cams[e];
        if (e == 0) {
            *W = c.width;
            *H = c.height;
        }
        if (c.width != *W || c.height != *H)
            return fail(GS_ERR_INVALID, "camera %d: resolution %dx%d differs from camera 0 (%dx%d)", e, c.width,
                        c.height, *W, *H);
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
            return fail(GS_ERR_INVALID, "camera %d: width/height must be in [1, 16384]", e);
        if (!(std::isfinite(c.fx) && std::isfinite(c.fy) && c.fx > 0 && c.fy > 0))
            return fail(GS_ERR_INVALID, "camera %d: focal lengths must be finite and > 0", e);
        if (!(std::isfinite(c.cx) && std::isfinite(c.cy)))
            return fail(GS_ERR_INVALID, "camera %d: principal point must be finite", e);
        if (!(std::isfinite(c.near_plane) && c.near_plane > 0))
            return fail(GS_ERR_INVALID, "camera %d: near_plane must be finite and > 0", e);
        double qn = 0;
        for (int k = 0; k < 4; ++k) {
            if (!std::isfinite(c.q_cw[k])) return fail(GS_ERR_INVALID, "camera %d: non-finite quaternion", e);
            qn += (double)c.q_cw[k] * c.q_cw[k];
        }
        if (!(qn > 0)) return fail(GS_ERR_INVALID, "camera %d: zero quaternion", e);
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(c.t_cw[k])) return fail(GS_ERR_INVALID, "camera %d: non-finite translation", e);
    }
    return GS_OK;
}

struct Plan {
    int64_t G;
    int L, W, H, ntx, nty, T;
    int64_t mask_words;
    size_t per_env;
    int We;  // envs per wave
};

// Brackets one phase's launches with events on the render stream when
// profiling is on.
struct PhaseTimer {
    gs_scene s;
    cudaStream_t st;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(gs_scene s_, cudaStream_t st_, int ph) : s(s_), st(st_), phase(ph) {
        if (s->profile) {
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

gs_status make_plan(gs_scene s, int E, int W, int H, bool host_mode, Plan* p) {
    p->G = s->D.n;
    p->L = s->D.n_links;
    p->W = W;
    p->H = H;
    p->ntx = (W + s->tile_w - 1) / s->tile_w;
    p->nty = (H + s->tile_h - 1) / s->tile_h;
    p->T = p->ntx * p->nty;
    if (p->T > 16384)
        return fail(GS_ERR_UNSUPPORTED, "%d tiles per image exceed the 16384 supported (use larger tiles)", p->T);
    p->mask_words = (p->G + 31) / 32;
    size_t per = (size_t)p->G * 64 + (size_t)p->mask_words * 4 + (size_t)p->T * 12 + 16 + (size_t)(p->L + 1) * 64;
    if (s->debug) per += (size_t)p->G * 8;
    if (host_mode) per += (size_t)W * H * 20 * 2;  // two staging sets of rgb + depth + alpha
    p->per_env = per;
    int64_t wmax = (int64_t)((double)s->budget * 0.6 / (double)per);
    if (wmax < 1) return fail(GS_ERR_OOM, "one environment needs %zu bytes of scratch; budget is %lld", per,
                              (long long)s->budget);
    if (s->max_wave > 0 && wmax > s->max_wave) wmax = s->max_wave;
    if (wmax > E) wmax = E;
    const int64_t nw = (E + wmax - 1) / wmax;
    p->We = (int)((E + nw - 1) / nw);
    return GS_OK;
}

}  // namespace

namespace {

// Render envs [e0, e0+We) whose poses/cams are already on the device; the
// wave's outputs go to rgb/depth/alpha (device, wave-local env indexing).
gs_status render_wave(gs_scene s, const Plan& p, int e0, int We, const float* poses_dev, const gs_camera* cams_dev,
                      float* rgb, float* depth, float* alpha, cudaStream_t st, int64_t* launches) {
    const int64_t G = p.G;
    const size_t nrec = (size_t)We * (size_t)G;
    CK(s->xf.ensure((size_t)We * (p.L + 1) * sizeof(LinkXf)), "alloc link table");
    CK(s->r0.ensure(nrec * 16), "alloc records");
    CK(s->r1.ensure(nrec * 16), "alloc records");
    CK(s->r2.ensure(nrec * 16), "alloc records");
    CK(s->r3.ensure(nrec * 16), "alloc records");
    CK(s->mask.ensure((size_t)We * p.mask_words * 4), "alloc masks");
    CK(s->counts.ensure((size_t)We * p.T * 4), "alloc counts");
    CK(s->off.ensure((size_t)We * p.T * 4), "alloc offsets");
    CK(s->cursor.ensure((size_t)We * p.T * 4), "alloc cursors");
    CK(s->env_total.ensure((size_t)We * 8), "alloc totals");
    CK(s->env_base.ensure((size_t)(We + 1) * 8), "alloc bases");
    if (s->debug) CK(s->dbg_hxy.ensure(nrec * 8), "alloc debug");
    if ((size_t)(We + 1) > s->pinned_n) {
        if (s->pinned) cudaFreeHost(s->pinned);
        s->pinned = nullptr;
        s->pinned_n = 0;
        CK(cudaMallocHost((void**)&s->pinned, sizeof(unsigned long long) * (We + 1)), "alloc pinned");
        s->pinned_n = (size_t)We + 1;
    }

    // A1: link composition
    PhaseTimer t1(s, st, GS_PHASE_LINK);
    CK(launch_link_table(poses_dev, cams_dev, We, p.L, s->xf.as<LinkXf>(), s->status, st), "link table");
    t1.done(1);
    ++*launches;
    // A2: projection
    ProjParams P{};
    P.G = G;
    P.p0 = s->D.p0;
    P.p1 = s->D.p1;
    P.p2 = s->D.p2;
    P.p3 = s->D.p3;
    P.sh = s->D.sh;
    P.xf = s->xf.as<LinkXf>();
    P.cams = cams_dev;
    P.L1 = p.L + 1;
    P.We = We;
    P.r0 = s->r0.as<float4>();
    P.r1 = s->r1.as<float4>();
    P.r2 = s->r2.as<float4>();
    P.r3 = s->r3.as<uint4>();
    P.mask = s->mask.as<uint32_t>();
    P.mask_words = p.mask_words;
    P.dbg_hxy = s->debug ? s->dbg_hxy.as<float2>() : nullptr;
    const unsigned gx = (unsigned)((G + 255) / 256);
    int gy = (int)((4864 + gx - 1) / gx);
    if (gy < 1) gy = 1;
    if (gy > We) gy = We;
    P.env_group = (We + gy - 1) / gy;
    gy = (We + P.env_group - 1) / P.env_group;
    PhaseTimer t2(s, st, GS_PHASE_PROJECT);
    CK(launch_project(s->D, P, dim3(gx, (unsigned)gy), st), "projection");
    t2.done(1);
    ++*launches;
    // A3: counts + scan
    CK(cudaMemsetAsync(s->counts.p, 0, (size_t)We * p.T * 4, st), "memset counts");
    BinParams B{};
    B.G = G;
    B.mask_words = p.mask_words;
    B.mask = s->mask.as<uint32_t>();
    B.r3 = s->r3.as<uint4>();
    B.e_begin = 0;
    B.tile_w = s->tile_w;
    B.tile_h = s->tile_h;
    B.ntx = p.ntx;
    B.T = p.T;
    B.counts = s->counts.as<uint32_t>();
    B.off_local = s->off.as<uint32_t>();
    B.env_base = s->env_base.as<unsigned long long>();
    B.cursor = s->cursor.as<uint32_t>();
    B.words_per_block = 256;  // 8 warps x 32 mask words (8192 Gaussians)
    const size_t smem1 = (size_t)p.T * 4, smem2 = (size_t)p.T * 8;
    PhaseTimer t3(s, st, GS_PHASE_COUNT);
    CK(launch_count(B, We, st, smem1), "count");
    t3.done(1);
    ++*launches;
    PhaseTimer t4(s, st, GS_PHASE_SCAN);
    CK(launch_scan(s->counts.as<uint32_t>(), s->off.as<uint32_t>(), s->env_total.as<unsigned long long>(),
                   s->env_base.as<unsigned long long>(), We, p.T, st),
       "scan");
    t4.done(2);
    *launches += 2;
    CK(cudaMemcpyAsync(s->pinned, s->env_base.p, sizeof(unsigned long long) * (We + 1), cudaMemcpyDeviceToHost, st),
       "read totals");
    CK(cudaStreamSynchronize(st), "sync totals");
    const unsigned long long* eb = s->pinned;
    s->stats.intersections += (int64_t)eb[We];
    CK(cudaMemsetAsync(s->cursor.p, 0, (size_t)We * p.T * 4, st), "memset cursors");

    // A4 + A5 per sub-wave of envs whose intersection lists fit the budget
    const double fixed = (double)p.per_env * We;
    double cap_d = (double)s->budget - fixed;
    if (cap_d < (double)s->budget * 0.25) cap_d = (double)s->budget * 0.25;
    const size_t key_bytes = s->debug ? 16 : 8;
    const unsigned long long cap_keys = (unsigned long long)(cap_d / key_bytes);
    int ea = 0;
    while (ea < We) {
        int ebd = ea + 1;
        if (eb[ebd] - eb[ea] > cap_keys)
            return fail(GS_ERR_OOM, "environment %d has %llu intersections, beyond the scratch budget", e0 + ea,
                        (unsigned long long)(eb[ebd] - eb[ea]));
        while (ebd < We && eb[ebd + 1] - eb[ea] <= cap_keys) ++ebd;
        const unsigned long long npairs = eb[ebd] - eb[ea];
        size_t want = (size_t)(npairs > 0 ? npairs : 1) * 8;
        if (want > s->pairs.bytes) {
            size_t grow = want + want / 4;
            if (grow > (size_t)cap_keys * 8) grow = want;
            CK(cudaStreamSynchronize(st), "sync before growth");
            CK(s->pairs.ensure(grow), "alloc intersection keys");
        }
        if (s->debug) CK(s->dbg_sorted.ensure(s->pairs.bytes), "alloc debug lists");
        B.e_begin = ea;
        B.pair_base = eb[ea];
        B.pairs = s->pairs.as<unsigned long long>();
        PhaseTimer t5(s, st, GS_PHASE_SCATTER);
        CK(launch_scatter(B, ebd - ea, st, smem2), "scatter");
        t5.done(1);
        ++*launches;
        CompParams C{};
        C.G = G;
        C.r0 = s->r0.as<float4>();
        C.r1 = s->r1.as<float4>();
        C.r2 = s->r2.as<float4>();
        C.counts = s->counts.as<uint32_t>();
        C.off_local = s->off.as<uint32_t>();
        C.env_base = s->env_base.as<unsigned long long>();
        C.pair_base = eb[ea];
        C.pairs = s->pairs.as<unsigned long long>();
        C.dbg_sorted = s->debug ? s->dbg_sorted.as<unsigned long long>() : nullptr;
        C.e_begin = ea;
        C.W = p.W;
        C.H = p.H;
        C.tile_w = s->tile_w;
        C.tile_h = s->tile_h;
        C.ntx = p.ntx;
        C.T = p.T;
        C.rgb = rgb;
        C.depth = depth;
        C.alpha = alpha;
        C.status = s->status;
        C.neval = s->counters ? s->neval.as<unsigned long long>() : nullptr;
        PhaseTimer t6(s, st, GS_PHASE_COMPOSITE);
        CK(launch_composite(C, ebd - ea, st), "composite");
        t6.done(1);
        ++*launches;
        s->last_ea = ea;
        s->last_eb = ebd;
        s->last_pair_base = eb[ea];
        s->last_pairs = (int64_t)npairs;
        ea = ebd;
    }
    s->last_e0 = e0;
    s->last_We = We;
    s->last_W = p.W;
    s->last_H = p.H;
    s->last_T = p.T;
    return GS_OK;
}

gs_status render_common(gs_scene s, int E, const float* link_poses, const gs_camera* cams, float* rgb, float* depth,
                        float* alpha, void* stream, bool host_mode) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (E < 0) return fail(GS_ERR_INVALID, "negative n_envs");
    if (E == 0) return GS_OK;
    if (!cams) return fail(GS_ERR_INVALID, "null cams");
    if (!rgb || !depth) return fail(GS_ERR_INVALID, "null rgb or depth output");
    if (s->D.n_links > 0 && !link_poses) return fail(GS_ERR_INVALID, "null link_poses with %d links", s->D.n_links);
    int W = 0, H = 0;
    gs_status vs = check_cams(cams, E, &W, &H);
    if (vs != GS_OK) return vs;
    Plan p{};
    vs = make_plan(s, E, W, H, host_mode, &p);
    if (vs != GS_OK) return vs;
    CK(cudaSetDevice(s->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s->stats.waves = 0;
    s->stats.kernel_launches = 0;
    s->stats.intersections = 0;
    const size_t px = (size_t)W * H;
    if (p.G == 0) {
        // no Gaussians: black, transparent, depth 0
        if (host_mode) {
            memset(rgb, 0, (size_t)E * px * 12);
            memset(depth, 0, (size_t)E * px * 4);
            if (alpha) memset(alpha, 0, (size_t)E * px * 4);
        } else {
            CK(cudaMemsetAsync(rgb, 0, (size_t)E * px * 12, st), "clear rgb");
            CK(cudaMemsetAsync(depth, 0, (size_t)E * px * 4, st), "clear depth");
            if (alpha) CK(cudaMemsetAsync(alpha, 0, (size_t)E * px * 4, st), "clear alpha");
        }
        return GS_OK;
    }
    CK(s->cams.ensure((size_t)E * sizeof(gs_camera)), "alloc cams");
    CK(cudaMemcpyAsync(s->cams.p, cams, (size_t)E * sizeof(gs_camera), cudaMemcpyHostToDevice, st), "copy cams");
    const gs_camera* cams_dev = s->cams.as<gs_camera>();
    const float* poses_dev = link_poses;
    const size_t pose_floats = (size_t)p.L * 7;
    if (host_mode && p.L > 0) {
        CK(s->poses.ensure((size_t)E * pose_floats * 4), "alloc poses");
        CK(cudaMemcpyAsync(s->poses.p, link_poses, (size_t)E * pose_floats * 4, cudaMemcpyHostToDevice, st),
           "copy poses");
        poses_dev = s->poses.as<float>();
    }
    int64_t launches = 0;
    if (!host_mode) {
        for (int e0 = 0; e0 < E; e0 += p.We) {
            const int We = E - e0 < p.We ? E - e0 : p.We;
            gs_status r = render_wave(s, p, e0, We, poses_dev ? poses_dev + (size_t)e0 * pose_floats : nullptr,
                                      cams_dev + e0, rgb + (size_t)e0 * px * 3, depth + (size_t)e0 * px,
                                      alpha ? alpha + (size_t)e0 * px : nullptr, st, &launches);
            if (r != GS_OK) return r;
            s->stats.waves++;
        }
    } else {
        if (!s->copy_stream) CK(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (int k = 0; k < 2; ++k) {
            if (!s->ev_done[k]) CK(cudaEventCreateWithFlags(&s->ev_done[k], cudaEventDisableTiming), "event");
            if (!s->ev_copied[k]) CK(cudaEventCreateWithFlags(&s->ev_copied[k], cudaEventDisableTiming), "event");
            CK(s->stage_rgb[k].ensure((size_t)p.We * px * 12), "alloc staging");
            CK(s->stage_depth[k].ensure((size_t)p.We * px * 4), "alloc staging");
            if (alpha) CK(s->stage_alpha[k].ensure((size_t)p.We * px * 4), "alloc staging");
        }
        int wave = 0;
        for (int e0 = 0; e0 < E; e0 += p.We, ++wave) {
            const int We = E - e0 < p.We ? E - e0 : p.We;
            const int k = wave & 1;
            if (wave >= 2) CK(cudaStreamWaitEvent(st, s->ev_copied[k], 0), "wait copy");
            gs_status r = render_wave(s, p, e0, We, poses_dev ? poses_dev + (size_t)e0 * pose_floats : nullptr,
                                      cams_dev + e0, s->stage_rgb[k].as<float>(), s->stage_depth[k].as<float>(),
                                      alpha ? s->stage_alpha[k].as<float>() : nullptr, st, &launches);
            if (r != GS_OK) return r;
            CK(cudaEventRecord(s->ev_done[k], st), "record");
            CK(cudaStreamWaitEvent(s->copy_stream, s->ev_done[k], 0), "wait render");
            CK(cudaMemcpyAsync(rgb + (size_t)e0 * px * 3, s->stage_rgb[k].p, (size_t)We * px * 12,
                               cudaMemcpyDeviceToHost, s->copy_stream),
               "copy rgb out");
            CK(cudaMemcpyAsync(depth + (size_t)e0 * px, s->stage_depth[k].p, (size_t)We * px * 4,
                               cudaMemcpyDeviceToHost, s->copy_stream),
               "copy depth out");
            if (alpha)
                CK(cudaMemcpyAsync(alpha + (size_t)e0 * px, s->stage_alpha[k].p, (size_t)We * px * 4,
                                   cudaMemcpyDeviceToHost, s->copy_stream),
                   "copy alpha out");
            CK(cudaEventRecord(s->ev_copied[k], s->copy_stream), "record");
            s->stats.waves++;
        }
        CK(cudaStreamSynchronize(s->copy_stream), "sync copies");
        CK(cudaStreamSynchronize(st), "sync render");
    }
    s->stats.kernel_launches = launches;
    return GS_OK;
}

}  // namespace

gsb::SceneView gsb::scene_view(gs_scene s) {
    return SceneView{s->device, s->D, s->status, s->tile_w, s->tile_h};
}

gs_status gsb::report(gs_status st, const char* msg) {
    g_err = msg;
    return st;
}

extern "C" {

const char* gs_last_error(void) { return g_err.c_str(); }

const char* gs_version(void) { return "gsbatch 0.1 (sm_103a)"; }

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
    gs_status r = alloc_gaussians(s, s->D.n, s->g0, s->g1, s->g2, s->g3, s->gsh, s->D.sh_planes);
    if (r == GS_OK) {
        s->D.p0 = s->g0.as<float4>();
        s->D.p1 = s->g1.as<float4>();
        s->D.p2 = s->g2.as<float4>();
        s->D.p3 = s->g3.as<float4>();
        s->D.sh = s->gsh.p;
        r = prep_view(s, background, 0, 0, nullptr, 0);
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
    if (s->D.n_bg + lg->n > 0xFFFFFFF0ll) return fail(GS_ERR_UNSUPPORTED, "more than 2^32-16 Gaussians in total");
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
    gs_status r = alloc_gaussians(s, N.n, a, b, c, d, sh, N.sh_planes);
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
    if (lg->n > 0) s->have_format = true;
    s->stats.n_gaussians = s->D.n;
    return GS_OK;
}

gs_status gs_render_batch(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                          float* depth, float* alpha, void* cuda_stream) {
    return render_common(s, n_envs, link_poses, cams, rgb, depth, alpha, cuda_stream, false);
}

gs_status gs_render_batch_host(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                               float* depth, float* alpha, void* cuda_stream) {
    return render_common(s, n_envs, link_poses, cams, rgb, depth, alpha, cuda_stream, true);
}

gs_status gs_scene_set_tile(gs_scene s, int tw, int th) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    const bool ok = (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 16 && th == 16) || (tw == 32 && th == 8);
    if (!ok) return fail(GS_ERR_INVALID, "tile %dx%d not one of 8x8, 16x8, 16x16, 32x8", tw, th);
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
    if (st & kStOverflow) m += " capacity overflow;";
    g_err = m;
    return GS_ERR_DEVICE;
}

gs_status gs_scene_get_stats(gs_scene s, gs_stats* out) {
    if (!s || !out) return fail(GS_ERR_INVALID, "null argument");
    s->stats.n_gaussians = s->D.n;
    int64_t bytes = 0;
    const DevBuf* bufs[] = {&s->xf, &s->cams, &s->poses, &s->r0, &s->r1, &s->r2, &s->r3, &s->mask, &s->counts,
                            &s->off, &s->cursor, &s->env_total, &s->env_base, &s->pairs, &s->dbg_hxy,
                            &s->dbg_sorted, &s->stage_rgb[0], &s->stage_rgb[1], &s->stage_depth[0],
                            &s->stage_depth[1], &s->stage_alpha[0], &s->stage_alpha[1]};
    for (const DevBuf* b : bufs) bytes += (int64_t)b->bytes;
    s->stats.scratch_bytes = bytes;
    s->stats.composited = 0;
    if (s->counters && s->neval.p) {
        CK(cudaSetDevice(s->device), "set device");
        CK(cudaDeviceSynchronize(), "sync");
        unsigned long long c = 0;
        CK(cudaMemcpy(&c, s->neval.p, 8, cudaMemcpyDeviceToHost), "read counter");
        s->stats.composited = (int64_t)c;
    }
    *out = s->stats;
    return GS_OK;
}

gs_status gs_scene_set_counters(gs_scene s, int enable) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    s->counters = enable ? 1 : 0;
    if (s->counters) {
        CK(cudaSetDevice(s->device), "set device");
        CK(s->neval.ensure(8), "alloc counter");
        CK(cudaMemset(s->neval.p, 0, 8), "clear counter");
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

gs_status gs_debug_copy_records(gs_scene s, int env, uint8_t* visible, float* u, float* v, float* hx, float* hy,
                                float* z, float* opacity, float* conic, float* rgb, int32_t* range) {
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (s->last_e0 < 0 || env < s->last_e0 || env >= s->last_e0 + s->last_We)
        return fail(GS_ERR_INVALID, "env %d is not in the last wave rendered", env);
    if (!s->debug || !s->dbg_hxy.p) return fail(GS_ERR_INVALID, "debug was not enabled for the last render");
    CK(cudaSetDevice(s->device), "set device");
    CK(cudaDeviceSynchronize(), "sync");
    const int el = env - s->last_e0;
    const int64_t G = s->D.n;
    const size_t base = (size_t)el * G;
    std::vector<uint32_t> mask((G + 31) / 32);
    std::vector<float4> a(G), b(G), c(G);
    std::vector<float2> h(G);
    CK(cudaMemcpy(mask.data(), s->mask.as<uint32_t>() + (size_t)el * mask.size(), mask.size() * 4,
                  cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(a.data(), s->r0.as<float4>() + base, G * 16, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(b.data(), s->r1.as<float4>() + base, G * 16, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(c.data(), s->r2.as<float4>() + base, G * 16, cudaMemcpyDeviceToHost), "copy");
    CK(cudaMemcpy(h.data(), s->dbg_hxy.as<float2>() + base, G * 8, cudaMemcpyDeviceToHost), "copy");
    for (int64_t g = 0; g < G; ++g) {
        const bool vis = (mask[g >> 5] >> (g & 31)) & 1u;
        if (visible) visible[g] = vis ? 1 : 0;
        if (!vis) continue;
        if (u) u[g] = a[g].x;
        if (v) v[g] = a[g].y;
        if (opacity) opacity[g] = a[g].z;
        if (z) z[g] = a[g].w;
        if (conic) {  // records hold L with L^T L = conic * 0.5 log2(e) (upper triangular)
            const double k2 = 0.72134752044448170;
            const double l00 = b[g].x, l01 = b[g].y, l11 = b[g].z;
            conic[3 * g] = (float)(l00 * l00 / k2);
            conic[3 * g + 1] = (float)(l00 * l01 / k2);
            conic[3 * g + 2] = (float)((l01 * l01 + l11 * l11) / k2);
        }
        if (rgb) {
            rgb[3 * g] = c[g].x;
            rgb[3 * g + 1] = c[g].y;
            rgb[3 * g + 2] = c[g].z;
        }
        if (hx) hx[g] = h[g].x;
        if (hy) hy[g] = h[g].y;
        if (range) {
            uint32_t rx, ry;
            float fx = b[g].w, fy = c[g].w;
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
    if (n_counts < s->last_T) return fail(GS_ERR_INVALID, "counts holds %lld < %d tiles", (long long)n_counts,
                                          s->last_T);
    CK(cudaSetDevice(s->device), "set device");
    CK(cudaDeviceSynchronize(), "sync");
    CK(cudaMemcpy(counts, s->counts.as<uint32_t>() + (size_t)el * s->last_T, (size_t)s->last_T * 4,
                  cudaMemcpyDeviceToHost), "copy counts");
    if (!lists) return GS_OK;
    if (!s->debug || !s->dbg_sorted.p) return fail(GS_ERR_INVALID, "debug was not enabled for the last render");
    if (el < s->last_ea || el >= s->last_eb)
        return fail(GS_ERR_INVALID, "env %d is not in the last sub-wave rendered", env);
    unsigned long long base = 0, total = 0;
    CK(cudaMemcpy(&base, s->env_base.as<unsigned long long>() + el, 8, cudaMemcpyDeviceToHost), "copy base");
    CK(cudaMemcpy(&total, s->env_base.as<unsigned long long>() + el + 1, 8, cudaMemcpyDeviceToHost), "copy base");
    total -= base;
    if ((unsigned long long)n_lists < total) return fail(GS_ERR_INVALID, "lists holds %lld < %llu entries",
                                                         (long long)n_lists, total);
    std::vector<unsigned long long> keys(total > 0 ? total : 1);
    if (total > 0)
        CK(cudaMemcpy(keys.data(), s->dbg_sorted.as<unsigned long long>() + (base - s->last_pair_base), total * 8,
                      cudaMemcpyDeviceToHost), "copy lists");
    for (unsigned long long i = 0; i < total; ++i) lists[i] = (uint32_t)(keys[i] & 0xffffffffull);
    return GS_OK;
}

void gs_scene_destroy(gs_scene s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&s->g0, &s->g1, &s->g2, &s->g3, &s->gsh, &s->xf, &s->cams, &s->poses, &s->r0, &s->r1, &s->r2,
                      &s->r3, &s->mask, &s->counts, &s->off, &s->cursor, &s->env_total, &s->env_base, &s->pairs,
                      &s->dbg_hxy, &s->dbg_sorted, &s->stage_rgb[0], &s->stage_rgb[1], &s->stage_depth[0],
                      &s->stage_depth[1], &s->stage_alpha[0], &s->stage_alpha[1]};
    for (DevBuf* b : bufs) b->release();
    s->neval.release();
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
