// Host-side tables of a wave: per-env offsets (EnvInfo) and the projection
// block list.  Every entry point (uniform batch, uneven batch, plans, the
// allocation-free path) describes its environments with EnvSpec and gets the
// same tables, so the kernels see one layout.
#include "gs_internal.cuh"

namespace gsb {

int64_t bg_slots(int64_t n_bg) { return (n_bg + 31) & ~int64_t(31); }

namespace {

// Envs per projection block: enough blocks to fill the GPU (>= 4864 of 256
// threads), as few env groups as possible so each Gaussian's attributes are
// read by few blocks.
int env_group(int64_t chunks, int n_envs) {
    int64_t gy = (4864 + chunks - 1) / chunks;
    if (gy < 1) gy = 1;
    if (gy > n_envs) gy = n_envs;
    return (int)((n_envs + gy - 1) / gy);
}

template <typename Emit>
void walk_blocks(const DevGaussians& D, const int64_t* link_offsets, const EnvSpec* specs, int n, Emit&& emit) {
    const int64_t nbp = bg_slots(D.n_bg);
    if (D.n_bg > 0 && n > 0) {
        const int64_t chunks = (D.n_bg + 255) / 256;
        const int eg = env_group(chunks, n);
        for (int e0 = 0; e0 < n; e0 += eg) {
            const int e1 = e0 + eg < n ? e0 + eg : n;
            for (int64_t c = 0; c < chunks; ++c) {
                const int64_t rem = D.n_bg - c * 256;
                emit(ProjBlock{c * 256, (unsigned)(c * 256), (int)(rem < 256 ? rem : 256), e0, e1, 0, 1});
            }
        }
    }
    int e = 0;
    while (e < n) {
        const int lb = specs[e].link_begin, le = specs[e].link_end;
        int e_end = e + 1;
        while (e_end < n && specs[e_end].link_begin == lb && specs[e_end].link_end == le) ++e_end;
        const int64_t r0 = link_offsets ? link_offsets[lb] : 0, r1 = link_offsets ? link_offsets[le] : 0;
        const int64_t nlg = r1 - r0;
        if (nlg > 0) {
            const int64_t chunks = (nlg + 255) / 256;
            const int eg = env_group(chunks, e_end - e);
            for (int a = e; a < e_end; a += eg) {
                const int b = a + eg < e_end ? a + eg : e_end;
                for (int64_t c = 0; c < chunks; ++c) {
                    const int64_t rem = nlg - c * 256;
                    emit(ProjBlock{D.n_bg + r0 + c * 256, (unsigned)(nbp + c * 256), (int)(rem < 256 ? rem : 256), a,
                                   b, lb, 0});
                }
            }
        }
        e = e_end;
    }
}

}  // namespace

int count_wave_blocks(const DevGaussians& D, const int64_t* link_offsets, const EnvSpec* specs, int n) {
    int nb = 0;
    walk_blocks(D, link_offsets, specs, n, [&](const ProjBlock&) { ++nb; });
    return nb;
}

void build_wave_tables(const DevGaussians& D, const int64_t* link_offsets, const EnvSpec* specs, int n, int tile_w,
                       int tile_h, long long pix_rebase, EnvInfo* envs, ProjBlock* blocks, int* n_blocks,
                       int max_blocks) {
    const int64_t nbp = bg_slots(D.n_bg);
    unsigned long long rec = 0, mask = 0;
    unsigned int tiles = 0;
    int xf = 0;
    for (int e = 0; e < n; ++e) {
        const EnvSpec& sp = specs[e];
        const int W = sp.cam->width, H = sp.cam->height;
        const int ntx = (W + tile_w - 1) / tile_w, nty = (H + tile_h - 1) / tile_h;
        const int nl = sp.link_end - sp.link_begin;
        const int64_t nlg = link_offsets ? link_offsets[sp.link_end] - link_offsets[sp.link_begin] : 0;
        EnvInfo& ei = envs[e];
        ei.rec_base = rec;
        ei.mask_base = mask;
        ei.pix_base = (unsigned long long)(sp.pixel_offset - pix_rebase);
        ei.pose_base = sp.pose_offset;
        ei.tile_base = tiles;
        ei.n_local = (unsigned)(nbp + nlg);
        ei.xf_base = xf;
        ei.link_begin = sp.link_begin;
        ei.n_links = nl;
        ei.W = W;
        ei.H = H;
        ei.ntx = ntx;
        ei.T = ntx * nty;
        ei.pad = 0;
        ei.g_link0 = D.n_bg + (link_offsets ? link_offsets[sp.link_begin] : 0);
        // guard-band limits of the EWA Jacobian (IEEE float division, as on the device)
        const gs_camera& c = *sp.cam;
        ei.lim[0] = 1.3f * c.cx / c.fx;
        ei.lim[1] = 1.3f * ((float)W - c.cx) / c.fx;
        ei.lim[2] = 1.3f * c.cy / c.fy;
        ei.lim[3] = 1.3f * ((float)H - c.cy) / c.fy;
        rec += ei.n_local;
        mask += (ei.n_local + 31) / 32;
        tiles += (unsigned)ei.T;
        xf += 1 + nl;
    }
    EnvInfo& s = envs[n];
    s = EnvInfo{};
    s.rec_base = rec;
    s.mask_base = mask;
    s.tile_base = tiles;
    s.xf_base = xf;
    int nb = 0;
    walk_blocks(D, link_offsets, specs, n, [&](const ProjBlock& b) {
        if (nb < max_blocks) blocks[nb] = b;
        ++nb;
    });
    *n_blocks = nb;
}

}  // namespace gsb
