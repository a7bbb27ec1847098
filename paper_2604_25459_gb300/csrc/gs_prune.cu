// gs_scene_prune: pruning as a scene transform.  The paper prunes its
// Gaussians for speed and memory (Sec. III-C, "Batch Renderer Optimization":
// about 30 % of a static scene kept, and up to 90 % fewer on dynamic objects)
// without giving the criterion; here the caller's per-Gaussian scores (for
// instance gs_scene_contribution's summed blending weights) rank the
// Gaussians, and the top fraction of the background and of every link's
// cluster is kept.
//
// Selection runs on the device: every Gaussian gets the unique 64-bit key
// (descending score bits << 32 | index within its group), and a radix
// selection over 8-bit digits (eight passes, all groups at once, the host
// choosing each group's digit from the pass's histograms) finds each group's
// k-th smallest key; a Gaussian is kept when its key is at most that.  The new
// scene is gathered on the device from the source scene's stored attributes,
// so the kept Gaussians render exactly as they did in the source scene.
#include <cmath>
#include <cstring>
#include <vector>

#include "gs_host.h"

namespace gsb {
namespace {

// Score of Gaussian g (caller's order) -> key that orders by descending score,
// then ascending index i within the group.  Returns false for a NaN score.
__device__ __forceinline__ bool prune_key(float score, uint32_t i, unsigned long long& key) {
    uint32_t b = __float_as_uint(score);
    if ((b & 0x7fffffffu) > 0x7f800000u) return false;  // NaN
    if (b == 0x80000000u) b = 0u;                        // -0 ranks as +0
    const uint32_t up = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending float order
    key = ((unsigned long long)(~up) << 32) | i;
    return true;
}

// Group of Gaussian g: 0 background, 1 + l for link l (offs: the link
// Gaussians' offsets within the link part, n_links + 1 entries).
__device__ __forceinline__ int prune_group(long long g, long long n_bg, const long long* offs, int n_links,
                                           uint32_t& i) {
    if (g < n_bg) {
        i = (uint32_t)g;
        return 0;
    }
    const long long r = g - n_bg;
    int lo = 0, hi = n_links - 1;  // last l with offs[l] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= r) lo = mid; else hi = mid - 1;
    }
    i = (uint32_t)(r - offs[lo]);
    return 1 + lo;
}

// One radix-selection pass: per group, the histogram of digit (key >> shift) &
// 255 over the keys that match the group's prefix so far.
__global__ void __launch_bounds__(256) k_prune_hist(const float* scores, long long n, long long n_bg,
                                                    const long long* offs, int n_links,
                                                    const unsigned long long* prefix, const unsigned long long* mask,
                                                    int shift, uint32_t* hist, uint32_t* bad) {
    const long long g = (long long)blockIdx.x * 256 + threadIdx.x;
    if (g >= n) return;
    uint32_t i;
    const int grp = prune_group(g, n_bg, offs, n_links, i);
    unsigned long long key;
    if (!prune_key(scores[g], i, key)) {
        atomicOr(bad, 1u);
        return;
    }
    if ((key & mask[grp]) == prefix[grp]) atomicAdd(hist + (size_t)grp * 256 + ((key >> shift) & 255ull), 1u);
}

// keep[g] = 1 when the key is at most the group's threshold (thr valid only
// where the group keeps at least one).
__global__ void __launch_bounds__(256) k_prune_mark(const float* scores, long long n, long long n_bg,
                                                    const long long* offs, int n_links,
                                                    const unsigned long long* thr, const uint32_t* keep_any,
                                                    uint8_t* keep) {
    const long long g = (long long)blockIdx.x * 256 + threadIdx.x;
    if (g >= n) return;
    uint32_t i;
    const int grp = prune_group(g, n_bg, offs, n_links, i);
    unsigned long long key = ~0ull;
    const bool ok = prune_key(scores[g], i, key);
    keep[g] = (uint8_t)(ok && keep_any[grp] && key <= thr[grp]);
}

// Gather of stored attributes: dst storage position m <- src storage position map[m].
__global__ void __launch_bounds__(256) k_prune_gather(DevGaussians src, DevGaussians dst, const long long* map) {
    const long long m = (long long)blockIdx.x * 256 + threadIdx.x;
    if (m >= dst.n) return;
    const long long k = map[m];
    dst.p0[m] = src.p0[k];
    dst.p1[m] = src.p1[k];
    dst.p2[m] = src.p2[k];
    dst.p3[m] = src.p3[k];
    const float4* ss = static_cast<const float4*>(src.sh);
    float4* ds = static_cast<float4*>(dst.sh);
    for (int p = 0; p < dst.sh_planes; ++p) ds[(size_t)p * dst.n + m] = ss[(size_t)p * src.n + k];
}

}  // namespace
}  // namespace gsb

using namespace gsb;

extern "C" gs_status gs_scene_prune(gs_scene s, const float* scores, double keep_bg, double keep_links,
                                    gs_scene* out, int64_t* kept, int64_t kept_cap) {
    if (!out) return fail(GS_ERR_INVALID, "null output handle");
    *out = nullptr;
    if (!s) return fail(GS_ERR_INVALID, "null scene");
    if (!scores && s->D.n > 0) return fail(GS_ERR_INVALID, "null scores");
    if (!(keep_bg >= 0.0 && keep_bg <= 1.0) || !(keep_links >= 0.0 && keep_links <= 1.0))
        return fail(GS_ERR_INVALID, "keep fractions must lie in [0, 1]");
    const long long n = s->D.n, nb = s->D.n_bg;
    const int L = s->D.n_links, G = 1 + L;
    // how many each group keeps: ceil(fraction x size)
    std::vector<long long> gsize((size_t)G), gkeep((size_t)G);
    gsize[0] = nb;
    for (int l = 0; l < L; ++l) gsize[(size_t)l + 1] = s->link_offsets[(size_t)l + 1] - s->link_offsets[(size_t)l];
    long long total = 0;
    for (int q = 0; q < G; ++q) {
        const double f = q == 0 ? keep_bg : keep_links;
        gkeep[(size_t)q] = std::min(gsize[(size_t)q], (long long)std::ceil(f * (double)gsize[(size_t)q]));
        total += gkeep[(size_t)q];
    }
    if (kept && kept_cap < total)
        return fail(GS_ERR_INVALID, "kept holds %lld < %lld entries", (long long)kept_cap, total);
    CK(cudaSetDevice(s->device), "set device");

    // radix selection of every group's threshold key
    DevBuf d_offs, d_prefix, d_mask, d_hist, d_bad, d_thr, d_any, d_keep, d_map;
    std::vector<long long> offs_host(s->link_offsets.begin(), s->link_offsets.end());
    if (offs_host.empty()) offs_host.assign(1, 0);
    CK(d_offs.ensure(offs_host.size() * 8), "alloc prune tables");
    CK(cudaMemcpy(d_offs.p, offs_host.data(), offs_host.size() * 8, cudaMemcpyHostToDevice), "copy offsets");
    CK(d_prefix.ensure((size_t)G * 8), "alloc prune tables");
    CK(d_mask.ensure((size_t)G * 8), "alloc prune tables");
    CK(d_hist.ensure((size_t)G * 256 * 4), "alloc prune tables");
    CK(d_bad.ensure(4), "alloc prune tables");
    CK(cudaMemset(d_bad.p, 0, 4), "clear flag");
    std::vector<unsigned long long> prefix((size_t)G, 0ull), mask((size_t)G, 0ull);
    std::vector<long long> remaining(gkeep);
    std::vector<uint32_t> hist((size_t)G * 256);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    for (int shift = 56; shift >= 0 && n > 0; shift -= 8) {
        CK(cudaMemcpy(d_prefix.p, prefix.data(), (size_t)G * 8, cudaMemcpyHostToDevice), "copy prefixes");
        CK(cudaMemcpy(d_mask.p, mask.data(), (size_t)G * 8, cudaMemcpyHostToDevice), "copy masks");
        CK(cudaMemset(d_hist.p, 0, (size_t)G * 256 * 4), "clear histograms");
        k_prune_hist<<<blocks, 256>>>(scores, n, nb, d_offs.as<long long>(), L, d_prefix.as<unsigned long long>(),
                                      d_mask.as<unsigned long long>(), shift, d_hist.as<uint32_t>(),
                                      d_bad.as<uint32_t>());
        CK(cudaGetLastError(), "prune histogram");
        CK(cudaMemcpy(hist.data(), d_hist.p, hist.size() * 4, cudaMemcpyDeviceToHost), "read histograms");
        for (int q = 0; q < G; ++q) {
            if (remaining[(size_t)q] <= 0) continue;  // keeps nothing: no threshold needed
            long long cum = 0;
            int d = 0;
            for (; d < 256; ++d) {
                const long long c = hist[(size_t)q * 256 + d];
                if (cum + c >= remaining[(size_t)q]) break;
                cum += c;
            }
            if (d == 256) return fail(GS_ERR_CUDA, "prune selection lost keys (group %d)", q);
            remaining[(size_t)q] -= cum;
            prefix[(size_t)q] |= (unsigned long long)d << shift;
            mask[(size_t)q] |= 255ull << shift;
        }
    }
    uint32_t bad = 0;
    CK(cudaMemcpy(&bad, d_bad.p, 4, cudaMemcpyDeviceToHost), "read flag");
    if (bad) return fail(GS_ERR_INVALID, "scores hold a NaN");
    std::vector<uint32_t> any((size_t)G);
    for (int q = 0; q < G; ++q) any[(size_t)q] = gkeep[(size_t)q] > 0;
    CK(d_thr.ensure((size_t)G * 8), "alloc prune tables");
    CK(d_any.ensure((size_t)G * 4), "alloc prune tables");
    CK(d_keep.ensure((size_t)(n > 0 ? n : 1)), "alloc keep flags");
    CK(cudaMemcpy(d_thr.p, prefix.data(), (size_t)G * 8, cudaMemcpyHostToDevice), "copy thresholds");
    CK(cudaMemcpy(d_any.p, any.data(), (size_t)G * 4, cudaMemcpyHostToDevice), "copy thresholds");
    std::vector<uint8_t> keep((size_t)(n > 0 ? n : 1), 0);
    if (n > 0) {
        k_prune_mark<<<blocks, 256>>>(scores, n, nb, d_offs.as<long long>(), L, d_thr.as<unsigned long long>(),
                                      d_any.as<uint32_t>(), d_keep.as<uint8_t>());
        CK(cudaGetLastError(), "prune marks");
        CK(cudaMemcpy(keep.data(), d_keep.p, (size_t)n, cudaMemcpyDeviceToHost), "read keep flags");
    }

    // new caller indices (kept Gaussians in their original order, per part)
    std::vector<long long> newidx((size_t)(n > 0 ? n : 1), -1);
    long long nb2 = 0, nl2 = 0;
    for (long long g = 0; g < nb; ++g)
        if (keep[(size_t)g]) newidx[(size_t)g] = nb2++;
    std::vector<int64_t> offs2((size_t)L + 1, 0);
    for (int l = 0; l < L; ++l) {
        for (long long r = offs_host[(size_t)l]; r < offs_host[(size_t)l + 1]; ++r)
            if (keep[(size_t)(nb + r)]) newidx[(size_t)(nb + r)] = nb2 + nl2++;
        offs2[(size_t)l + 1] = nl2;
    }
    if (nb2 + nl2 != total) return fail(GS_ERR_CUDA, "prune kept %lld, expected %lld", nb2 + nl2, total);
    // storage: the kept background in the source's storage order, then the links
    std::vector<long long> map((size_t)(total > 0 ? total : 1));
    std::vector<long long> order2;
    order2.reserve((size_t)nb2);
    long long m = 0;
    for (long long k = 0; k < nb; ++k) {
        const long long g = s->bg_order.empty() ? k : s->bg_order[(size_t)k];
        if (keep[(size_t)g]) {
            map[(size_t)m++] = k;
            order2.push_back(newidx[(size_t)g]);
        }
    }
    for (long long r = 0; r < n - nb; ++r)
        if (keep[(size_t)(nb + r)]) map[(size_t)m++] = nb + r;
    if (kept) {
        for (long long g = 0; g < n; ++g)
            if (newidx[(size_t)g] >= 0) kept[newidx[(size_t)g]] = g;
    }

    gs_scene t = new gs_scene_s();
    auto bail = [&](gs_status st) {
        std::string msg = g_err;
        gs_scene_destroy(t);
        g_err = msg;
        return st;
    };
    t->device = s->device;
    cudaError_t e = cudaMalloc((void**)&t->status, 4);
    if (e == cudaSuccess) e = cudaMemset(t->status, 0, 4);
    if (e != cudaSuccess) return bail(cuda_fail(e, "scene create"));
    t->D = s->D;
    t->D.n = total;
    t->D.n_bg = nb2;
    const size_t cnt = (size_t)(total > 0 ? total : 1);
    for (DevBuf* b : {&t->g0, &t->g1, &t->g2, &t->g3}) {
        e = b->ensure(cnt * 16);
        if (e != cudaSuccess) return bail(cuda_fail(e, "alloc pruned scene"));
    }
    e = t->gsh.ensure(cnt * 16 * (size_t)(t->D.sh_planes > 0 ? t->D.sh_planes : 1));
    if (e != cudaSuccess) return bail(cuda_fail(e, "alloc pruned scene"));
    t->D.p0 = t->g0.as<float4>();
    t->D.p1 = t->g1.as<float4>();
    t->D.p2 = t->g2.as<float4>();
    t->D.p3 = t->g3.as<float4>();
    t->D.sh = t->gsh.p;
    if (total > 0) {
        e = d_map.ensure((size_t)total * 8);
        if (e == cudaSuccess) e = cudaMemcpy(d_map.p, map.data(), (size_t)total * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            k_prune_gather<<<(unsigned)((total + 255) / 256), 256>>>(s->D, t->D, d_map.as<long long>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return bail(cuda_fail(e, "gather pruned scene"));
    }
    t->link_offsets.assign(offs2.begin(), offs2.end());
    t->have_format = s->have_format;
    t->tile_w = s->tile_w;
    t->tile_h = s->tile_h;
    t->budget = s->budget;
    if (nb2 > 0) {
        std::vector<int> index32((size_t)nb2), slot32((size_t)nb2);
        for (long long k = 0; k < nb2; ++k) {
            index32[(size_t)k] = (int)order2[(size_t)k];
            slot32[(size_t)order2[(size_t)k]] = (int)k;
        }
        e = t->bg_index.ensure(sizeof(int) * (size_t)nb2);
        if (e == cudaSuccess) e = t->bg_slot.ensure(sizeof(int) * (size_t)nb2);
        if (e == cudaSuccess)
            e = cudaMemcpy(t->bg_index.p, index32.data(), sizeof(int) * (size_t)nb2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(t->bg_slot.p, slot32.data(), sizeof(int) * (size_t)nb2, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(cuda_fail(e, "pruned storage order"));
        t->bg_order.assign(order2.begin(), order2.end());
    }
    t->stats.n_gaussians = t->D.n;
    *out = t;
    return GS_OK;
}
