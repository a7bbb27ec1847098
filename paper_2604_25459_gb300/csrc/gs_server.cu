// The request loop of libgsbatch (gs_server_* in gsbatch.h), the serving
// form of the renderer: scenes and per-env state (camera, output image) stay
// resident; requests carry poses and an arrival time; a scheduler thread
// admits arrived requests into per-scene batches as stream slots and the HBM
// budget allow, launches each batch on its own CUDA stream (so batches overlap
// on the device) and records the completion time with a host callback on that
// stream.  Batches render through run_wave, like every other render.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "gs_host.h"

using namespace gsb;

struct gs_server_s {
    gs_server_config cfg{};
    int device = 0;
    struct SceneRec {
        gs_scene s;
        DevBuf rgb, depth;       // resident output images of the scene's envs
        int64_t px = 0;          // pixels allocated so far
    };
    std::vector<std::unique_ptr<SceneRec>> scenes;
    struct EnvRec {
        int scene;
        gs_camera cam;
        int link_begin, link_end;
        int64_t pix_off;
        bool busy = false;
    };
    std::vector<EnvRec> envs;
    struct Req {
        int env;
        double arrival;
        std::vector<float> poses;
        double admit = -1, done = -1;
        int status = 0;
    };
    std::deque<Req> reqs;  // element addresses stay valid while submit appends
    std::deque<int64_t> scheduled;  // not yet arrived, by arrival time
    std::deque<int64_t> pending;    // arrived, not admitted
    std::deque<int64_t> completed;  // done, not yet polled
    struct Slot {
        cudaStream_t st = nullptr;
        Scratch sc;
        DevBuf poses, dstat;          // link poses; the batch's device status word
        float* h_poses = nullptr;     // pinned staging of the poses
        size_t h_cap = 0;
        unsigned long long* h_meta = nullptr;  // pinned: [0] status word, [1..n+1] key offsets per env
        size_t meta_cap = 0;
        bool busy = false;
        bool eager = false;           // the batch in flight sizes its keys exactly (host sync)
        bool failed = false;          // its launch failed (requests carry the status)
        int scene = -1;
        std::vector<int64_t> batch;   // request ids, in launch order
        std::vector<const Req*> rq;   // the same requests (taken under the lock: launches run without it)
        double bytes = 0;
        std::atomic<int> done{0};
        double t_done = 0;
        std::chrono::steady_clock::time_point t0;
    };
    std::vector<std::unique_ptr<Slot>> slots;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<bool> stop{false};
    bool started = false;
    std::chrono::steady_clock::time_point t0;
    double inflight_bytes = 0;
    gs_server_stats stats{};
    std::map<std::tuple<int, int, int>, double> keys_ema;  // (scene, W, H) -> intersections per env
    std::map<std::tuple<int, int, int>, double> keys_max;  // (scene, W, H) -> most seen for one env
    std::string error;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void CUDART_CB server_slot_done(void* p) {
    auto* sl = static_cast<gs_server_s::Slot*>(p);
    sl->t_done = std::chrono::duration<double>(std::chrono::steady_clock::now() - sl->t0).count();
    sl->done.store(1, std::memory_order_release);
}

// Estimated intersections of an env (running average for its scene and
// resolution), or -1 before any batch of that kind has run.
double keys_estimate(gs_server sv, const gs_server_s::EnvRec& ev) {
    auto it = sv->keys_ema.find({ev.scene, ev.cam.width, ev.cam.height});
    return it != sv->keys_ema.end() ? it->second : -1.0;
}

double request_bytes(gs_server sv, const gs_server_s::EnvRec& ev) {
    gs_scene s = sv->scenes[ev.scene]->s;
    EnvSpec sp{&ev.cam, ev.link_begin, ev.link_end, 0, 0};
    const int tw = sv->cfg.tile_w, th = sv->cfg.tile_h;
    double keys = keys_estimate(sv, ev);
    if (keys < 0) keys = (double)(sv->scenes[ev.scene]->s->D.n);  // first of its kind: about one key per Gaussian
    return (double)env_bytes(s, sp, tw, th, false) + keys * 8.0 * 1.3;
}

// Launch one batch (requests of one scene, in sl.batch) on its slot.  Called
// by the scheduler thread with the lock released.  The batch is ordered by
// ascending pixel count: low-resolution envs have the longest tile buckets,
// so their tiles are claimed first.  Planned mode (keys capacity from the
// running estimates, no host sync) unless the batch has an env of a kind not
// seen before or sl.eager is set; a planned batch whose keys overflowed is
// relaunched eagerly by the scheduler.
gs_status server_launch(gs_server sv, gs_server_s::Slot& sl) {
    auto& sr = *sv->scenes[sl.scene];
    gs_scene s = sr.s;
    const int L = s->D.n_links;
    auto& batch = sl.batch;
    const size_t n = batch.size();
    {
        std::vector<size_t> ord(n);
        for (size_t i = 0; i < n; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
            const gs_camera& a = sv->envs[sl.rq[x]->env].cam;
            const gs_camera& b = sv->envs[sl.rq[y]->env].cam;
            return (int64_t)a.width * a.height < (int64_t)b.width * b.height;
        });
        std::vector<int64_t> ids(n);
        std::vector<const gs_server_s::Req*> rqs(n);
        for (size_t i = 0; i < n; ++i) {
            ids[i] = batch[ord[i]];
            rqs[i] = sl.rq[ord[i]];
        }
        batch.swap(ids);
        sl.rq.swap(rqs);
    }
    const size_t pose_floats = std::max<size_t>(1, n * (size_t)L * 7);
    if (pose_floats > sl.h_cap) {
        if (sl.h_poses) cudaFreeHost(sl.h_poses);
        sl.h_poses = nullptr;
        sl.h_cap = 0;
        CK(cudaMallocHost((void**)&sl.h_poses, pose_floats * 4), "alloc pinned poses");
        sl.h_cap = pose_floats;
    }
    if (n + 2 > sl.meta_cap) {
        if (sl.h_meta) cudaFreeHost(sl.h_meta);
        sl.h_meta = nullptr;
        sl.meta_cap = 0;
        CK(cudaMallocHost((void**)&sl.h_meta, (n + 2) * 8), "alloc pinned batch info");
        sl.meta_cap = n + 2;
    }
    CK(sl.poses.ensure(pose_floats * 4), "alloc poses");
    CK(sl.dstat.ensure(8), "alloc status");
    std::vector<EnvSpec> specs(n);
    double est = 0, spread = 0;  // sum of the running averages; the largest (most seen - average)
    bool known = true;
    for (size_t i = 0; i < n; ++i) {
        const auto& rq = *sl.rq[i];
        const auto& ev = sv->envs[rq.env];
        const int nl = ev.link_end - ev.link_begin;
        if (nl > 0) memcpy(sl.h_poses + i * (size_t)L * 7, rq.poses.data(), sizeof(float) * nl * 7);
        specs[i] = EnvSpec{&ev.cam, ev.link_begin, ev.link_end, (long long)i * L, (long long)ev.pix_off};
        const double k = keys_estimate(sv, ev);
        if (k < 0) known = false;
        est += k;
        auto mt = sv->keys_max.find({ev.scene, ev.cam.width, ev.cam.height});
        if (mt != sv->keys_max.end()) spread = std::max(spread, mt->second - k);
    }
    const bool eager = sl.eager || !known;
    sl.eager = eager;
    if (L > 0)
        CK(cudaMemcpyAsync(sl.poses.p, sl.h_poses, n * (size_t)L * 28, cudaMemcpyHostToDevice, sl.st), "copy poses");
    CK(cudaMemsetAsync(sl.dstat.p, 0, 4, sl.st), "clear status");
    WaveTables wt{};
    ST(upload_tables(s, specs, 0, (int)n, sv->cfg.tile_w, sv->cfg.tile_h, 0, sl.sc.envs, sl.sc.blocks, sl.sc.cams,
                     sl.st, false, &wt));
    int64_t launches = 0;
    unsigned long long keys = 0;
    // capacity: 25% over the averages, plus room for one env at the most seen
    // of its kind (what a batch of a few envs needs)
    const unsigned long long cap = eager ? 0ull : (unsigned long long)(est * 1.25 + spread) + 65536ull;
    WaveIO io{sl.poses.as<float>(), sr.rgb.as<float>(), sr.depth.as<float>(), nullptr, 0, sl.dstat.as<uint32_t>()};
    ST(run_wave(s, sl.sc, wt, io, sv->cfg.tile_w, sv->cfg.tile_h, 1, cap, sl.st, false, &launches, &keys));
    CK(cudaMemcpyAsync(sl.h_meta, sl.dstat.p, 4, cudaMemcpyDeviceToHost, sl.st), "read status");
    CK(cudaMemcpyAsync(sl.h_meta + 1, sl.sc.env_base.p, (n + 1) * 8, cudaMemcpyDeviceToHost, sl.st), "read keys");
    sl.t0 = sv->t0;
    CK(cudaLaunchHostFunc(sl.st, server_slot_done, &sl), "completion callback");
    return GS_OK;
}

// A finished batch (lock held): update the key estimates from its exact
// per-env intersection counts; true if it must be relaunched eagerly.
bool server_batch_done(gs_server sv, gs_server_s::Slot& sl, uint32_t* status_out) {
    const uint32_t st = (uint32_t)(sl.h_meta[0] & 0xffffffffu);
    const unsigned long long* base = sl.h_meta + 1;
    for (size_t i = 0; i < sl.batch.size(); ++i) {
        const auto& ev = sv->envs[sv->reqs[sl.batch[i]].env];
        const double k = (double)(base[i + 1] - base[i]);
        const std::tuple<int, int, int> kind{ev.scene, ev.cam.width, ev.cam.height};
        auto it = sv->keys_ema.find(kind);
        if (it == sv->keys_ema.end()) sv->keys_ema[kind] = k;
        else it->second = 0.9 * it->second + 0.1 * k;
        double& mx = sv->keys_max[kind];
        mx = std::max(mx, k);
    }
    *status_out = st;
    return (st & kStOverflow) && !sl.eager;
}

void server_loop(gs_server sv) {
    cudaSetDevice(sv->device);
    while (!sv->stop.load()) {
        bool worked = false;
        std::vector<gs_server_s::Slot*> launch, relaunch;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            const double t = sv->now();
            while (!sv->scheduled.empty() && sv->reqs[sv->scheduled.front()].arrival <= t) {
                sv->pending.push_back(sv->scheduled.front());
                sv->scheduled.pop_front();
            }
            // completions
            for (auto& sl : sv->slots) {
                if (sl->busy && sl->done.load(std::memory_order_acquire)) {
                    uint32_t dst = 0;
                    if (sl->failed) {
                        dst = 0;  // the requests already carry the launch's status
                    } else if (server_batch_done(sv, *sl, &dst)) {
                        sl->done.store(0);  // keys overflowed the estimate: render it again, exactly
                        sl->eager = true;
                        sv->stats.retried++;
                        relaunch.push_back(sl.get());
                        worked = true;
                        continue;
                    }
                    for (int64_t id : sl->batch) {
                        auto& rq = sv->reqs[id];
                        rq.done = sl->t_done;
                        if (rq.status == 0 && dst != 0) rq.status = (int)GS_ERR_DEVICE;
                        sv->envs[rq.env].busy = false;
                        sv->completed.push_back(id);
                        sv->stats.completed++;
                    }
                    sv->inflight_bytes -= sl->bytes;
                    sl->busy = false;
                    sl->batch.clear();
                    sl->rq.clear();
                    worked = true;
                }
            }
            // admission: per-scene batches of arrived requests whose env is idle
            int inflight = 0;
            for (auto& sl : sv->slots) inflight += sl->busy ? 1 : 0;
            for (auto& slp : sv->slots) {
                if (slp->busy || sv->pending.empty()) continue;
                int scene = -1;
                std::vector<int64_t> batch;
                double bytes = 0;
                std::deque<int64_t> keep;
                std::vector<char> taken(sv->envs.size(), 0);
                while (!sv->pending.empty()) {
                    const int64_t id = sv->pending.front();
                    sv->pending.pop_front();
                    auto& rq = sv->reqs[id];
                    auto& ev = sv->envs[rq.env];
                    const bool fits_scene = scene < 0 || ev.scene == scene;
                    const double b = request_bytes(sv, ev);
                    // a batch holds at most budget / slots (a slot's scratch keeps its
                    // high-water mark, so the slots together stay within the budget);
                    // the batches in flight together at most the budget; a request
                    // larger than that runs alone when nothing else is in flight
                    const double budget = (double)sv->cfg.budget_bytes;
                    const bool fits_budget =
                        batch.empty() ? (sv->inflight_bytes + b <= budget || inflight == 0)
                                      : (bytes + b <= budget / sv->cfg.max_inflight &&
                                         sv->inflight_bytes + bytes + b <= budget);
                    if (!ev.busy && !taken[rq.env] && fits_scene && fits_budget &&
                        (int)batch.size() < sv->cfg.max_batch_envs) {
                        scene = ev.scene;
                        batch.push_back(id);
                        bytes += b;
                        taken[rq.env] = 1;
                    } else {
                        keep.push_back(id);
                    }
                }
                sv->pending.swap(keep);
                if (batch.empty()) break;
                for (int64_t id : batch) {
                    sv->reqs[id].admit = sv->now();
                    sv->envs[sv->reqs[id].env].busy = true;
                }
                slp->busy = true;
                slp->done.store(0);
                slp->eager = false;
                slp->failed = false;
                slp->scene = scene;
                slp->batch = batch;
                slp->rq.clear();
                for (int64_t id : batch) slp->rq.push_back(&sv->reqs[id]);
                slp->bytes = bytes;
                sv->inflight_bytes += bytes;
                sv->stats.batches++;
                sv->stats.peak_inflight_bytes = std::max(sv->stats.peak_inflight_bytes, (int64_t)sv->inflight_bytes);
                ++inflight;
                sv->stats.max_concurrent = std::max(sv->stats.max_concurrent, inflight);
                sv->stats.max_batch = std::max(sv->stats.max_batch, (int)batch.size());
                launch.push_back(slp.get());
            }
        }
        for (auto* l : relaunch) launch.push_back(l);
        for (auto* l : launch) {
            gs_status st = server_launch(sv, *l);
            worked = true;
            if (st != GS_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->error = g_err;
                for (int64_t id : l->batch) sv->reqs[id].status = (int)st;
                // completes once the stream has drained, so the loop does not stall;
                // the requests carry the status
                cudaStreamSynchronize(l->st);
                l->failed = true;
                l->t_done = sv->now();
                l->done.store(1);
            }
        }
        if (!worked) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

gs_status gs_server_create(const gs_server_config* cfg, gs_server* out) {
    if (!out || !cfg) return fail(GS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (cfg->budget_bytes < (1ll << 20)) return fail(GS_ERR_INVALID, "budget below 1 MiB");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 64) return fail(GS_ERR_INVALID, "max_inflight must be 1..64");
    if (cfg->max_batch_envs < 1) return fail(GS_ERR_INVALID, "max_batch_envs must be >= 1");
    if (!valid_tile(cfg->tile_w, cfg->tile_h)) return fail(GS_ERR_INVALID, "unsupported tile shape");
    gs_server sv = new gs_server_s();
    sv->cfg = *cfg;
    cudaGetDevice(&sv->device);
    for (int k = 0; k < cfg->max_inflight; ++k) {
        auto sl = std::make_unique<gs_server_s::Slot>();
        cudaError_t e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            gs_server_destroy(sv);
            return cuda_fail(e, "server stream");
        }
        sv->slots.push_back(std::move(sl));
    }
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv;
    return GS_OK;
}

gs_status gs_server_add_scene(gs_server sv, gs_scene s, int* scene_id) {
    if (!sv || !s || !scene_id) return fail(GS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->started) return fail(GS_ERR_INVALID, "scenes must be added before gs_server_start");
    auto sr = std::make_unique<gs_server_s::SceneRec>();
    sr->s = s;
    sv->scenes.push_back(std::move(sr));
    *scene_id = (int)sv->scenes.size() - 1;
    return GS_OK;
}

gs_status gs_server_add_env(gs_server sv, int scene_id, const gs_camera* cam, int link_begin, int link_end,
                            int* env_id) {
    if (!sv || !cam || !env_id) return fail(GS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->started) return fail(GS_ERR_INVALID, "envs must be added before gs_server_start");
    if (scene_id < 0 || scene_id >= (int)sv->scenes.size()) return fail(GS_ERR_INVALID, "unknown scene %d", scene_id);
    gs_scene s = sv->scenes[scene_id]->s;
    ST(check_cam(*cam, (int)sv->envs.size()));
    if (link_begin < 0 || link_end < link_begin || link_end > s->D.n_links)
        return fail(GS_ERR_INVALID, "link range [%d, %d) outside [0, %d]", link_begin, link_end, s->D.n_links);
    const int ntx = (cam->width + sv->cfg.tile_w - 1) / sv->cfg.tile_w;
    const int nty = (cam->height + sv->cfg.tile_h - 1) / sv->cfg.tile_h;
    if (ntx * nty > 16384) return fail(GS_ERR_UNSUPPORTED, "more than 16384 tiles");
    gs_server_s::EnvRec ev{scene_id, *cam, link_begin, link_end, sv->scenes[scene_id]->px, false};
    sv->scenes[scene_id]->px += (int64_t)cam->width * cam->height;
    sv->envs.push_back(ev);
    *env_id = (int)sv->envs.size() - 1;
    return GS_OK;
}

gs_status gs_server_start(gs_server sv) {
    if (!sv) return fail(GS_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->started) return GS_OK;
    CK(cudaSetDevice(sv->device), "set device");
    for (auto& sr : sv->scenes) {  // resident per-env outputs
        CK(sr->rgb.ensure((size_t)std::max<int64_t>(sr->px, 1) * 12), "alloc env images");
        CK(sr->depth.ensure((size_t)std::max<int64_t>(sr->px, 1) * 4), "alloc env depth");
        CK(cudaMemset(sr->rgb.p, 0, sr->rgb.bytes), "clear");
        CK(cudaMemset(sr->depth.p, 0, sr->depth.bytes), "clear");
    }
    sv->t0 = std::chrono::steady_clock::now();
    std::sort(sv->scheduled.begin(), sv->scheduled.end(),
              [&](int64_t a, int64_t b) { return sv->reqs[a].arrival < sv->reqs[b].arrival; });
    sv->started = true;
    sv->stop = false;
    sv->worker = std::thread(server_loop, sv);
    return GS_OK;
}

gs_status gs_server_submit(gs_server sv, int env_id, const float* poses, double arrival_s, int64_t* request_id) {
    if (!sv) return fail(GS_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (env_id < 0 || env_id >= (int)sv->envs.size()) return fail(GS_ERR_INVALID, "unknown env %d", env_id);
    const auto& ev = sv->envs[env_id];
    const int nl = ev.link_end - ev.link_begin;
    if (nl > 0 && !poses) return fail(GS_ERR_INVALID, "env %d renders %d links: poses required", env_id, nl);
    gs_server_s::Req rq;
    rq.env = env_id;
    rq.arrival = arrival_s >= 0 ? arrival_s : (sv->started ? sv->now() : 0.0);
    if (nl > 0) rq.poses.assign(poses, poses + (size_t)nl * 7);
    sv->reqs.push_back(std::move(rq));
    const int64_t id = (int64_t)sv->reqs.size() - 1;
    // keep `scheduled` ordered by arrival (appends are usually in order)
    auto pos = sv->scheduled.end();
    while (pos != sv->scheduled.begin() && sv->reqs[*(pos - 1)].arrival > sv->reqs[id].arrival) --pos;
    sv->scheduled.insert(pos, id);
    sv->stats.submitted++;
    if (request_id) *request_id = id;
    sv->cv.notify_all();
    return GS_OK;
}

gs_status gs_server_cancel(gs_server sv, int64_t request_id) {
    if (!sv) return fail(GS_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (request_id < 0 || request_id >= (int64_t)sv->reqs.size())
        return fail(GS_ERR_INVALID, "unknown request %lld", (long long)request_id);
    for (std::deque<int64_t>* q : {&sv->scheduled, &sv->pending}) {
        auto it = std::find(q->begin(), q->end(), request_id);
        if (it == q->end()) continue;
        q->erase(it);
        auto& rq = sv->reqs[request_id];
        rq.status = 1;
        rq.done = sv->started ? sv->now() : 0.0;
        sv->completed.push_back(request_id);
        sv->stats.cancelled++;
        return GS_OK;
    }
    return fail(GS_ERR_INVALID, "request %lld already admitted or finished", (long long)request_id);
}

gs_status gs_server_poll(gs_server sv, gs_request_result* out, int max_results, int* n_out) {
    if (!sv || !n_out || (max_results > 0 && !out)) return fail(GS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    int n = 0;
    while (n < max_results && !sv->completed.empty()) {
        const int64_t id = sv->completed.front();
        sv->completed.pop_front();
        const auto& rq = sv->reqs[id];
        out[n++] = gs_request_result{id, rq.env, rq.status, rq.arrival, rq.admit, rq.done};
    }
    *n_out = n;
    return GS_OK;
}

gs_status gs_server_drain(gs_server sv, double timeout_s) {
    if (!sv) return fail(GS_ERR_INVALID, "null server");
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (!sv->error.empty()) {
                g_err = sv->error;
                return GS_ERR_CUDA;
            }
            if (sv->stats.completed + sv->stats.cancelled >= sv->stats.submitted) break;
        }
        if (std::chrono::steady_clock::now() > t_end) return fail(GS_ERR_TIMEOUT, "requests still in flight");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    // every batch has completed: the scenes' device status words are final
    for (auto& sr : sv->scenes) ST(gs_scene_sync_status(sr->s, nullptr));
    return GS_OK;
}

double gs_server_now(gs_server sv) {
    if (!sv) return -1.0;
    std::lock_guard<std::mutex> lk(sv->mu);
    return sv->started ? sv->now() : 0.0;
}

gs_status gs_server_get_stats(gs_server sv, gs_server_stats* out) {
    if (!sv || !out) return fail(GS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    return GS_OK;
}

gs_status gs_server_env_output(gs_server sv, int env_id, float** rgb, float** depth) {
    if (!sv || !rgb || !depth) return fail(GS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (env_id < 0 || env_id >= (int)sv->envs.size()) return fail(GS_ERR_INVALID, "unknown env %d", env_id);
    if (!sv->started) return fail(GS_ERR_INVALID, "server not started");
    const auto& ev = sv->envs[env_id];
    auto& sr = *sv->scenes[ev.scene];
    *rgb = sr.rgb.as<float>() + ev.pix_off * 3;
    *depth = sr.depth.as<float>() + ev.pix_off;
    return GS_OK;
}

void gs_server_destroy(gs_server sv) {
    if (!sv) return;
    sv->stop = true;
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    for (auto& sl : sv->slots) {
        if (sl->st) cudaStreamSynchronize(sl->st);
        sl->sc.release();
        sl->poses.release();
        sl->dstat.release();
        if (sl->h_poses) cudaFreeHost(sl->h_poses);
        if (sl->h_meta) cudaFreeHost(sl->h_meta);
        if (sl->st) cudaStreamDestroy(sl->st);
    }
    for (auto& sr : sv->scenes) {
        sr->rgb.release();
        sr->depth.release();
    }
    delete sv;
}

}  // extern "C"
