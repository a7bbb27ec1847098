// Batch-LiDAR projection: every (env, Gaussian) of a wave against the env's
// LiDAR (a rotating one, or a solid-state one with a narrower azimuth window).  The paper's Batch-LiDAR ray-casts the 3DGS scene with its
// moving links (Sec. III-E, Table II); here a scan is rendered like an image
// over the (azimuth, beam) grid: this kernel writes, per visible pair, the
// Gaussian's ray-space factors in the sensor frame and a conservative grid box
// of the rays it can reach, and the binning kernels and the compositor (its
// LiDAR form) do the rest.
//
// A Gaussian with covariance F F^T, F = R diag(e^s) (columns f_k = e^{s_k} r_k),
// has q(x) = sum_k (g_k . (x - mu))^2 with g_k = f_k / |f_k|^2 = e^{-s_k} r_k.
// Along a ray t d: a_k = g_k . d and b_k = g_k . mu give q(t) = |t a - b|^2.
// Since q(x) >= |x - mu|^2 / max_k e^{2 s_k} = |x - mu|^2 / max_k |f_k|^2, every
// point with alpha >= 1/255 (q <= q*) lies within r = sqrt(q*) max_k |f_k| of
// mu: the rays that can reach it lie within the cone of half-angle
// asin(r / |mu|).  The cone bounds the elevations; the azimuths are the exact
// range of the ellipsoid's shadow on the sensor's xy-plane where that is
// tighter (see below).
//
// Arbitrary rays (non-repetitive scan patterns) reuse the grid as a binning
// structure: each ray falls in one cell of its sensor's (azimuth, beam) grid,
// the Gaussians' grid boxes are widened by half a cell (so they hold every
// cell that a direction inside the cone can fall in, not only the cells whose
// centres lie inside it), and the compositor walks a tile's keys for the rays
// of that tile.
//
// A cone across the window's first column (azimuth 0 of a full turn) reaches
// the first and the last columns: its box is stored wrapped, x0 > x1 meaning
// columns [x0, cols) and [0, x1], which the binning kernels and the
// compositor's LiDAR forms read as two ranges (a box over every column
// between them would put the Gaussian in every tile of its rows).
#include "gs_internal.cuh"

namespace gsb {

namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr float kHalfPi = 1.5707963267948966f;

// Inclusive grid range [lo, hi] of the centres c_k = (k + 1/2) step + origin
// within [a, b]; false if none.
__device__ __forceinline__ bool grid_range(float a, float b, float origin, float step, int n, int& lo, int& hi) {
    float l = ceilf((a - origin) / step - 0.5f);
    float h = floorf((b - origin) / step - 0.5f);
    l = fmaxf(l, 0.0f);
    h = fminf(h, (float)(n - 1));
    if (!(l <= h)) return false;
    lo = (int)l;
    hi = (int)h;
    return true;
}

}  // namespace

__global__ void __launch_bounds__(256) k_project_lidar(ProjParams P) {
    const ProjBlock blk = P.blocks[blockIdx.x];
    const int t = threadIdx.x;
    const bool act = t < blk.n;
    const int lane = t & 31;
    const long long g = blk.g_first + t;
    const unsigned int local = blk.local_first + (unsigned)t;
    const bool warp_live = (t - lane) < blk.n;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    if (act) {
        a0 = __ldg(P.p0 + g);
        a1 = __ldg(P.p1 + g);
        a2 = __ldg(P.p2 + g);
        a3 = __ldg(P.p3 + g);
    }
    const int li = __float_as_int(a3.w) - blk.lb;
    const float qstar = a3.y;
    const bool live = act && qstar >= 0.0f;
    // support radius (metres): sqrt(q*) times the largest scale (the longest column of F)
    float fmax2 = 0.0f;
    {
        const float F[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x};  // row-major
#pragma unroll
        for (int k = 0; k < 3; ++k)
            fmax2 = fmaxf(fmax2, F[k] * F[k] + F[3 + k] * F[3 + k] + F[6 + k] * F[6 + k]);
    }
    const float reach = sqrtf(fmaxf(qstar, 0.0f) * fmax2) * 1.001f + 1e-6f;
    for (int el = blk.e0; el < blk.e1; ++el) {
        bool vis = false;
        const EnvInfo* E = P.envs + el;
        if (live) {
            const LinkXf* Xp = P.xf + __ldg(&E->xf_base) + li;
            const float4 r0 = __ldg(&Xp->r0), r1 = __ldg(&Xp->r1), r2 = __ldg(&Xp->r2);
            const float mx = r0.x * a0.x + r0.y * a0.y + r0.z * a0.z + r0.w;
            const float my = r1.x * a0.x + r1.y * a0.y + r1.z * a0.z + r1.w;
            const float mz = r2.x * a0.x + r2.y * a0.y + r2.z * a0.z + r2.w;
            const float dist = sqrtf(mx * mx + my * my + mz * mz);
            const gs_lidar* L = P.lidars + el;
            const int rows = __ldg(&L->rows), cols = __ldg(&L->cols);
            const float em = __ldg(&L->elev_min), eM = __ldg(&L->elev_max);
            const float near = __ldg(&L->near_range);
            if (dist + reach > near) {
                int i0 = 0, i1 = cols - 1, j0 = 0, j1 = rows - 1;
                bool any = true;
                if (reach < dist) {
                    const float rho = asinf(fminf(1.0f, reach / dist)) * 1.001f + 1e-5f;
                    const float thc = asinf(fmaxf(-1.0f, fminf(1.0f, mz / dist)));
                    const float estep = (eM - em) / (float)rows;
                    any = grid_range(thc - rho - P.cell_pad * estep, thc + rho + P.cell_pad * estep, em, estep, rows,
                                     j0, j1);
                    if (any && fabsf(thc) + rho < kHalfPi) {
                        // azimuth half-widths below / above the centre: the cone's, and
                        // where tighter the exact range of the Gaussian's shadow on the
                        // xy-plane (azimuth depends on x and y only, so every ray that
                        // meets {q <= q*} lies between the shadow's tangents from the
                        // sensor).  In the frame of the centre direction e (normal n), with
                        // S the shadow's covariance there and d the centre's distance, a
                        // tangent y = k x solves k^2 (d^2 - q* s11) + 2 q* s12 k - q* s22 = 0.
                        float dlo = asinf(fminf(1.0f, sinf(rho) / cosf(thc))) * 1.001f + 1e-5f, dhi = dlo;
                        {
                            const float d2 = mx * mx + my * my;
                            const float id = rsqrtf(fmaxf(d2, 1e-30f));
                            const float ex = mx * id, ey = my * id;
                            const float Fm[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x};
                            float s11 = 0.0f, s12 = 0.0f, s22 = 0.0f;
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const float fx = r0.x * Fm[k] + r0.y * Fm[3 + k] + r0.z * Fm[6 + k];
                                const float fy = r1.x * Fm[k] + r1.y * Fm[3 + k] + r1.z * Fm[6 + k];
                                const float pe = fx * ex + fy * ey, pn = fy * ex - fx * ey;
                                s11 += pe * pe;
                                s12 += pe * pn;
                                s22 += pn * pn;
                            }
                            const float al = d2 - qstar * s11;
                            if (al > 0.01f * d2) {  // the sensor well outside the shadow along e
                                const float disc = sqrtf(qstar * qstar * s12 * s12 + al * qstar * s22);
                                dhi = fminf(dhi, atanf((disc - qstar * s12) / al) * 1.001f + 1e-5f);
                                dlo = fminf(dlo, atanf((disc + qstar * s12) / al) * 1.001f + 1e-5f);
                            }
                        }
                        // azimuth relative to the window start, within one turn: [0, 2 pi)
                        const float az0 = __ldg(&L->az_min), step = (__ldg(&L->az_max) - az0) / (float)cols;
                        float rel = atan2f(my, mx) - az0;
                        rel -= kTwoPi * floorf(rel / kTwoPi);
                        const float lo = rel - dlo - P.cell_pad * step, hi = rel + dhi + P.cell_pad * step;
                        // the cone's azimuths in this turn, and their copy one turn away
                        // when the cone crosses 0
                        int a0, a1, b0 = 0, b1 = -1;
                        const bool ina = grid_range(lo, hi, 0.0f, step, cols, a0, a1);
                        bool inb = false;
                        if (lo < 0.0f) inb = grid_range(lo + kTwoPi, hi + kTwoPi, 0.0f, step, cols, b0, b1);
                        else if (hi >= kTwoPi) inb = grid_range(lo - kTwoPi, hi - kTwoPi, 0.0f, step, cols, b0, b1);
                        if (ina && inb) {
                            // two ranges, one from column 0 and one to the last
                            // column: stored as a wrapped box i0 > i1 (columns
                            // [i0, cols) and [0, i1]) unless they meet
                            const int l1 = a0 <= b0 ? a1 : b1, h0 = a0 <= b0 ? b0 : a0;
                            if (h0 <= l1 + 1) {
                                i0 = 0;
                                i1 = cols - 1;
                            } else {
                                i0 = h0;
                                i1 = l1;
                            }
                        } else if (ina) {
                            i0 = a0;
                            i1 = a1;
                        } else if (inb) {
                            i0 = b0;
                            i1 = b1;
                        } else {
                            any = false;
                        }
                    }
                }
                if (any) {
                    // sensor-frame columns of F, then g_k = f_k / |f_k|^2 and b = G mu
                    float f[3][3];
                    const float F[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x};  // row-major
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        f[k][0] = r0.x * F[k] + r0.y * F[3 + k] + r0.z * F[6 + k];
                        f[k][1] = r1.x * F[k] + r1.y * F[3 + k] + r1.z * F[6 + k];
                        f[k][2] = r2.x * F[k] + r2.y * F[3 + k] + r2.z * F[6 + k];
                    }
                    float gk[3][3], b[3], glen2 = 0.0f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float n2 = f[k][0] * f[k][0] + f[k][1] * f[k][1] + f[k][2] * f[k][2];
                        const float inv = 1.0f / n2;
                        gk[k][0] = f[k][0] * inv;
                        gk[k][1] = f[k][1] * inv;
                        gk[k][2] = f[k][2] * inv;
                        b[k] = gk[k][0] * mx + gk[k][1] * my + gk[k][2] * mz;
                        if (k == 2) glen2 = inv;  // |g_2|^2 = 1 / |f_2|^2
                    }
                    const uint32_t rx = (uint32_t)i0 | ((uint32_t)i1 << 16);
                    const uint32_t ry = (uint32_t)j0 | ((uint32_t)j1 << 16);
                    const size_t ri = (size_t)__ldg(&E->rec_base) + local;
                    // direct stores at the records' 48-byte stride (staging them for
                    // coalesced stores, as the camera projection does, measured slower
                    // here, where most warps see many visible Gaussians per env)
                    P.r0[kRecStride * ri] = make_float4(b[0], b[1], b[2], a0.w);
                    P.r1[kRecStride * ri] = make_float4(gk[0][0], gk[0][1], gk[0][2], __uint_as_float(rx));
                    P.r2[kRecStride * ri] = make_float4(gk[1][0], gk[1][1], gk[1][2], __uint_as_float(ry));
                    P.r3[ri] = make_uint4(rx, ry, __float_as_uint(dist), __float_as_uint(sqrtf(glen2)));
                    vis = true;
                }
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, vis);
        if (lane == 0 && warp_live) P.mask[(size_t)__ldg(&E->mask_base) + (local >> 5)] = m;
    }
}

cudaError_t launch_project_lidar(const ProjParams& P, int n_blocks, cudaStream_t st) {
    if (n_blocks == 0) return cudaSuccess;
    k_project_lidar<<<n_blocks, 256, 0, st>>>(P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- arbitrary rays

// Cell of ray r of wave env el: azimuth phi = atan2(y, x) and elevation
// asin(z / |d|); column floor(((phi - az_min) mod 2 pi) / step) within the
// window, row floor((theta - elev_min) / estep).  grid: (rays / 256, envs).
__global__ void __launch_bounds__(256) k_ray_count(const float* __restrict__ dirs, const gs_lidar* lidars,
                                                   const EnvInfo* envs, int n_rays, uint32_t* cell, uint32_t* cnt,
                                                   uint32_t* status) {
    const int el = blockIdx.y;
    const int r = blockIdx.x * 256 + threadIdx.x;
    if (r >= n_rays) return;
    const size_t k = (size_t)el * n_rays + r;
    const float dx = dirs[3 * k], dy = dirs[3 * k + 1], dz = dirs[3 * k + 2];
    const gs_lidar* L = lidars + el;
    const EnvInfo& E = envs[el];
    const float n = sqrtf(dx * dx + dy * dy + dz * dz);
    bool ok = n > 0.0f && isfinite(n);
    int i = 0, j = 0;
    if (ok) {
        const float em = __ldg(&L->elev_min), eM = __ldg(&L->elev_max);
        const float az0 = __ldg(&L->az_min), span = __ldg(&L->az_max) - az0;
        const float th = asinf(fmaxf(-1.0f, fminf(1.0f, dz / n)));
        float rel = atan2f(dy, dx) - az0;
        rel -= kTwoPi * floorf(rel / kTwoPi);
        const float fi = floorf(rel / (span / (float)E.W));
        const float fj = floorf((th - em) / ((eM - em) / (float)E.H));
        ok = rel < span && fi >= 0.0f && fi < (float)E.W && fj >= 0.0f && fj < (float)E.H;
        i = (int)fi;
        j = (int)fj;
    }
    if (!ok) {
        cell[k] = 0xffffffffu;
        atomicOr(status, kStBadRay);
        return;
    }
    const int t = (j >> 4) * E.ntx + (i >> 4);
    cell[k] = ((uint32_t)t << 8) | ((uint32_t)(j & 15) << 4) | (uint32_t)(i & 15);
    atomicAdd(cnt + E.tile_base + t, 1u);
}

// Rays grouped by tile: list[el][off[tile] + rank] = r.
__global__ void __launch_bounds__(256) k_ray_scatter(const EnvInfo* envs, int n_rays, const uint32_t* cell,
                                                     const uint32_t* off, uint32_t* cur, uint32_t* list) {
    const int el = blockIdx.y;
    const int r = blockIdx.x * 256 + threadIdx.x;
    if (r >= n_rays) return;
    const size_t k = (size_t)el * n_rays + r;
    const uint32_t c = cell[k];
    if (c == 0xffffffffu) return;
    const unsigned int tb = envs[el].tile_base;
    const uint32_t t = c >> 8;
    const uint32_t pos = off[tb + t] + atomicAdd(cur + tb + t, 1u);
    list[(size_t)el * n_rays + pos] = (uint32_t)r;
}

// Compositor items per (env, tile): chunks of at most kRayChunk rays.
__global__ void __launch_bounds__(256) k_ray_items(const EnvInfo* envs, int We, const uint32_t* cnt,
                                                   uint32_t* item_cnt) {
    const unsigned int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= envs[We].tile_base) return;
    item_cnt[i] = (cnt[i] + (uint32_t)kRayChunk - 1u) / (uint32_t)kRayChunk;
}

cudaError_t launch_ray_count(const float* dirs, const gs_lidar* lidars, const EnvInfo* envs, int We, int n_rays,
                             uint32_t* cell, uint32_t* cnt, uint32_t* status, cudaStream_t st) {
    if (We == 0 || n_rays == 0) return cudaSuccess;
    k_ray_count<<<dim3((unsigned)((n_rays + 255) / 256), (unsigned)We), 256, 0, st>>>(dirs, lidars, envs, n_rays,
                                                                                      cell, cnt, status);
    return cudaGetLastError();
}

cudaError_t launch_ray_scatter(const EnvInfo* envs, int We, int n_rays, const uint32_t* cell, const uint32_t* off,
                               uint32_t* cur, uint32_t* list, const uint32_t* cnt, uint32_t* item_cnt,
                               unsigned int tiles, cudaStream_t st) {
    if (We == 0 || n_rays == 0) return cudaSuccess;
    k_ray_scatter<<<dim3((unsigned)((n_rays + 255) / 256), (unsigned)We), 256, 0, st>>>(envs, n_rays, cell, off,
                                                                                        cur, list);
    k_ray_items<<<(tiles + 255) / 256, 256, 0, st>>>(envs, We, cnt, item_cnt);
    return cudaGetLastError();
}

}  // namespace gsb
