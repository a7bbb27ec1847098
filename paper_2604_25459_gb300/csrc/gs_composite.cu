// Per-tile front-to-back alpha compositing with early termination (step A5).
//
// The 3DGS forward pass (paper Sec. II-B; the batch renderer of Sec. III-C
// "Throughput Scaling" is built on it) blends, per pixel, the splats whose
// alpha = min(0.99, o exp(-q/2)) reaches 1/255, in depth order, until the
// transmittance would drop below 1e-4; Sec. III-A asks for RGB and depth.
//
// Persistent CTAs claim (env, tile) items; each warp owns an 8x8 pixel
// subtile and each lane two of its pixels.  The tile's bucket of keys (depth
// bits << 32 | the caller's local index of the Gaussian) is consumed in depth
// windows of at most kCompCap keys: a short bucket is one window; a long one
// is first partitioned into kBins ranges of the env's depth range through the
// CTA's spill region, and windows are runs of ranges, so sorting stops at the
// window where every pixel has terminated.  Each window is sorted in shared
// memory (a counting sort by depth ranges, or LSD radix passes when the depths
// crowd, then index order within equal depths), its keys mapped to record
// slots, and composited in batches whose records are staged in shared memory;
// warps test 32 splats at a time against their subtile with one ballot (box,
// then the exact ellipse for large splats) and walk the overlapping ones two
// at a time, every lane evaluating both at its pixels with no branch inside a
// step.  Besides the image form the kernel has an observation
// form (8-bit colour after per-env appearance, half depth), a contribution
// form (per-Gaussian blending weights, for pruning) and a LiDAR form (rays of
// an (azimuth, beam) grid, Gaussians evaluated in ray space).
#include "gs_internal.cuh"
#include <type_traits>

namespace gsb {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int NT>
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
        v = o > v ? o : v;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long m = red[0];
    for (int w = 1; w < NT / 32; ++w) m = red[w] > m ? red[w] : m;
    __syncthreads();
    return m;
}

template <int NT>
__device__ __forceinline__ uint32_t block_or_u32(uint32_t v, uint32_t* red) {
    v = __reduce_or_sync(0xffffffffu, v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    uint32_t m = 0;
    for (int w = 0; w < NT / 32; ++w) m |= red[w];
    __syncthreads();
    return m;
}

// Exclusive scan of one value per thread; red holds NT/32 words.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += red[w];
    __syncthreads();
    return before + x - v;
}

// Radix counters are addressed through cidx: one spare 32-bit word after every
// 16 counters, so that the raking read of 16 consecutive counters per thread
// hits 32 different banks across a warp.
__device__ __forceinline__ int cidx(int e) { return e + ((e >> 4) << 1); }

constexpr int kSortBins = 1024;  // depth ranges of the window counting sort

// f(i, L[i]) for every i in [0, len) of this thread (i = tid + k NT), with up
// to U loads of L in flight per thread.
template <int NT, int U, typename F>
__device__ __forceinline__ void for_keys(const unsigned long long* L, uint32_t len, F&& f) {
    for (uint32_t i0 = threadIdx.x; i0 < len; i0 += NT * U) {
        unsigned long long k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + (uint32_t)(u * NT);
            k[u] = i < len ? L[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + (uint32_t)(u * NT);
            if (i < len) f(i, k[u]);
        }
    }
}

// Block-wide min and max of one u32 per thread; red holds 32 words.
template <int NT>
__device__ __forceinline__ void block_minmax_u32(uint32_t& mn, uint32_t& mx, uint32_t* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) {
        red[warp] = mn;
        red[16 + warp] = mx;
    }
    __syncthreads();
    mn = red[0];
    mx = red[16];
    for (int w = 1; w < NT / 32; ++w) {
        mn = red[w] < mn ? red[w] : mn;
        mx = red[16 + w] > mx ? red[16 + w] : mx;
    }
    __syncthreads();
}

// Sort keys[0, n) into tmp when the window's depths spread out: a counting
// sort by kSortBins equal ranges of the depth bits, then an insertion sort of
// each range by whole keys (equal depths fall in index order).  Applies when
// no range holds more than 32 keys; returns tmp then, else nullptr with keys
// untouched.  [zmin, zmax] bounds the window's depth bits (the window's
// producer takes them while loading it).  c32 (kSortBins u32) holds zeros on
// entry unless `dirty` is set (it is cleared here then); a successful sort
// leaves it zeroed again (each thread clears its own ranges after the last
// barrier; the next reader comes after the caller's next barriers).  red: 32 u32.
template <int NT>
__device__ unsigned long long* bin_sort(const unsigned long long* keys, unsigned long long* tmp, uint32_t* c32,
                                        uint32_t* red, int n, uint32_t zmin, uint32_t zmax, bool& dirty) {
    constexpr int PER = kSortBins / NT;
    static_assert(kSortBins % NT == 0, "ranges per thread");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t span = zmax - zmin;
    const int shift = (span >> 10) ? 22 - __clz(span) : 0;  // span >> shift < kSortBins
    if (dirty) {
        for (int b = tid; b < kSortBins; b += NT) c32[b] = 0u;
        __syncthreads();
        dirty = false;
    }
    for (int i = tid; i < n; i += NT) atomicAdd(&c32[((uint32_t)(keys[i] >> 32) - zmin) >> shift], 1u);
    __syncthreads();
    uint32_t loc[PER];
    uint32_t sum = 0;
    bool crowded = false;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        loc[j] = c32[tid * PER + j];
        sum += loc[j];
        crowded |= loc[j] > 32u;
    }
    // exclusive scan of the per-thread sums; the warps' totals carry a crowded
    // range in bit 31 (a window holds at most kCompCap keys)
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    const bool wc = __any_sync(0xffffffffu, crowded);
    if (lane == 31) red[warp] = x | (wc ? 0x80000000u : 0u);
    __syncthreads();
    uint32_t before = 0;
    bool any = false;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint32_t r = red[w];
        if (w < warp) before += r & 0x7fffffffu;
        any |= (r >> 31) != 0u;
    }
    __syncthreads();  // red is reused
    if (any) {
        dirty = true;  // c32 keeps the counts
        return nullptr;
    }
    uint32_t run = before + x - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        c32[tid * PER + j] = run;
        run += loc[j];
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
        const unsigned long long k = keys[i];
        const uint32_t pos = atomicAdd(&c32[((uint32_t)(k >> 32) - zmin) >> shift], 1u);
        tmp[pos] = k;
    }
    __syncthreads();
    // range b is now [c32[b-1], c32[b]) (c32 holds each range's end); the
    // ranges are interleaved over the threads, so a cluster of crowded
    // neighbouring ranges (a window's depths bunch up) spreads over many
    // threads instead of the few that hold them in the blocked layout
#pragma unroll 1
    for (int b = tid; b < kSortBins; b += NT) {
        const int e = (int)c32[b];
        const int a = b ? (int)c32[b - 1] : 0;
        for (int x = a + 1; x < e; ++x) {
            const unsigned long long k = tmp[x];
            int y = x - 1;
            while (y >= a && tmp[y] > k) {
                tmp[y + 1] = tmp[y];
                --y;
            }
            tmp[y + 1] = k;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) c32[tid * PER + j] = 0u;
    return tmp;
}

// Sort keys[0, n) ascending by the full 64-bit key (depth bits high, global
// index low; all distinct), n <= kCompCap.  bin_sort when the depths spread
// out; otherwise LSD radix passes of 4 bits over the depth bits that differ
// inside the window give a stable order by depth, and runs of equal depth are
// then ordered by index.  Returns the array that holds the result (keys or
// tmp).  cnt: cidx(16*NT) u16 and at least kSortBins u32 (see bin_sort for
// zmin, zmax and dirty); red: 32 u32.
template <int NT>
__device__ unsigned long long* window_sort(unsigned long long* keys, unsigned long long* tmp, uint16_t* cnt,
                                           uint32_t* red, int n, uint32_t zmin, uint32_t zmax, bool& dirty) {
    if (unsigned long long* r = bin_sort<NT>(keys, tmp, reinterpret_cast<uint32_t*>(cnt), red, n, zmin, zmax, dirty))
        return r;
    const int tid = threadIdx.x;
    const int I = (n + NT - 1) / NT;  // keys per thread, blocked arrangement
    const int b0 = tid * I;
    const uint32_t z0 = (uint32_t)(keys[0] >> 32);
    uint32_t zx = 0;
    for (int i = 0; i < I; ++i) {
        const int idx = b0 + i;
        if (idx < n) zx |= (uint32_t)(keys[idx] >> 32) ^ z0;
    }
    zx = block_or_u32<NT>(zx, red);
    const int nbits = zx ? 32 - __clz(zx) : 0;
    unsigned long long* src = keys;
    unsigned long long* dst = tmp;
    for (int shift = 0; shift < nbits; shift += 4) {
        const int s = 32 + shift;
#pragma unroll
        for (int d = 0; d < 16; ++d) cnt[cidx(d * NT + tid)] = 0;
        for (int i = 0; i < I; ++i) {
            const int idx = b0 + i;
            if (idx < n) {
                const int d = (int)((src[idx] >> s) & 15ull);
                cnt[cidx(d * NT + tid)] += 1;
            }
        }
        __syncthreads();
        // exclusive scan over (digit, thread) in row-major order
        uint32_t loc[16];
        uint32_t sum = 0;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            loc[e] = cnt[cidx(tid * 16 + e)];
            sum += loc[e];
        }
        uint32_t run = block_excl_scan_u32<NT>(sum, red);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            cnt[cidx(tid * 16 + e)] = (uint16_t)run;
            run += loc[e];
        }
        __syncthreads();
        for (int i = 0; i < I; ++i) {
            const int idx = b0 + i;
            if (idx < n) {
                const unsigned long long k = src[idx];
                const int d = (int)((k >> s) & 15ull);
                const uint32_t pos = cnt[cidx(d * NT + tid)];
                cnt[cidx(d * NT + tid)] = (uint16_t)(pos + 1);
                dst[pos] = k;
            }
        }
        __syncthreads();
        unsigned long long* t = src;
        src = dst;
        dst = t;
    }
    // runs of equal depth: order by the low (index) half
    bool tie = false;
    for (int i = 0; i < I; ++i) {
        const int idx = b0 + i;
        if (idx + 1 < n && (src[idx] >> 32) == (src[idx + 1] >> 32)) tie = true;
    }
    if (__syncthreads_or(tie)) {
        for (int i = 0; i < I; ++i) {
            const int idx = b0 + i;
            const bool head = idx + 1 < n && (src[idx] >> 32) == (src[idx + 1] >> 32) &&
                              (idx == 0 || (src[idx - 1] >> 32) != (src[idx] >> 32));
            if (head) {
                int e = idx + 1;
                while (e + 1 < n && (src[e + 1] >> 32) == (src[idx] >> 32)) ++e;
                for (int a = idx + 1; a <= e; ++a) {  // insertion sort of the run [idx, e]
                    const unsigned long long k = src[a];
                    int b = a - 1;
                    while (b >= idx && src[b] > k) {
                        src[b + 1] = src[b];
                        --b;
                    }
                    src[b + 1] = k;
                }
            }
        }
        __syncthreads();
    }
    return src;
}

// One pixel's blend step for a splat whose alpha is `al` (already >= 1/255);
// returns the weight w = alpha T added (0 when the step stops instead):
// T' = T (1 - alpha), evaluated as T - w; stop (splat not added) when
// T' < 1e-4.  The arithmetic is pinned to explicit round-to-nearest operations
// so every tile shape and every pixel slot evaluates exactly the same.
__device__ __forceinline__ float blend(float al, const float4& C, float z, float& T, float& r, float& g, float& b,
                                       float& d, bool& done) {
    const float w = __fmul_rn(al, T);
    const float Tn = __fsub_rn(T, w);
    if (Tn < 1e-4f) {
        done = true;
        return 0.0f;
    }
    r = __fmaf_rn(w, C.x, r);
    g = __fmaf_rn(w, C.y, g);
    b = __fmaf_rn(w, C.z, b);
    d = __fmaf_rn(w, z, d);
    T = Tn;
    return w;
}

// Warp sum of one float per lane.
__device__ __forceinline__ float warp_sum(float v) {
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Sum of one float per lane over each group of eight lanes.
__device__ __forceinline__ float group_sum(float v) {
    for (int d = 4; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// alpha = min(0.99, o exp(-q/2)) = min(0.99, 2^(log2 o - (l00 dx + l01 dy)^2 - (l11 dy)^2))
// where B = (l00, l01, l11) is the conic's upper Cholesky factor scaled by
// sqrt(log2(e)/2): q is evaluated as a sum of two squares.  Evaluated at a
// lane's two pixel centres (fpx, fpy.x) and (fpx, fpy.y) with the paired FP32
// instructions of sm_100+ (two round-to-nearest operations per instruction).
// CLAMP = false leaves out the 0.99 cap, for splats of opacity <= 0.98 (their
// alpha stays below it).
template <bool CLAMP = true>
__device__ __forceinline__ float2 splat_alpha2(const float4& A, const float4& B, float fpx, float2 fpy) {
    const float dx = fpx - A.x;
    const float2 dy = __fadd2_rn(fpy, make_float2(-A.y, -A.y));
    const float bx = __fmul_rn(B.x, dx);
    const float2 t = __ffma2_rn(make_float2(B.y, B.y), dy, make_float2(bx, bx));
    const float2 s = __fmul2_rn(make_float2(B.z, B.z), dy);
    // camera splats are staged with A.z = log2(o), folded into the exponent:
    // alpha = 2^(log2 o - t^2 - s^2), two paired FMAs before the ex2
    const float2 pw =
        __ffma2_rn(make_float2(-t.x, -t.y), t, __ffma2_rn(make_float2(-s.x, -s.y), s, make_float2(A.z, A.z)));
    const float2 a = make_float2(ex2_approx(pw.x), ex2_approx(pw.y));
    if constexpr (!CLAMP) return a;
    return make_float2(fminf(0.99f, a.x), fminf(0.99f, a.y));
}

// blend() for a lane's two pixels at once: pixel k takes the splat where uk
// is set.  A pixel that does not take it keeps its state exactly (its weight
// is 0, and fma(0, c, x) = x for the finite, non-negative sums here).  Returns
// the sum of the two weights added.
__device__ __forceinline__ float blend2(float2 al, bool u0, bool u1, const float4& C, float z, float2& T, float2& r,
                                        float2& g, float2& b, float2& d, bool& done0, bool& done1) {
    const float2 am = make_float2(u0 ? al.x : 0.0f, u1 ? al.y : 0.0f);
    const float2 x = __fmul2_rn(am, T);
    const float2 Tn = __fadd2_rn(T, make_float2(-x.x, -x.y));
    const bool s0 = u0 && Tn.x < 1e-4f, s1 = u1 && Tn.y < 1e-4f;
    done0 = done0 || s0;
    done1 = done1 || s1;
    const float2 w = make_float2(s0 ? 0.0f : x.x, s1 ? 0.0f : x.y);
    r = __ffma2_rn(w, make_float2(C.x, C.x), r);
    g = __ffma2_rn(w, make_float2(C.y, C.y), g);
    b = __ffma2_rn(w, make_float2(C.z, C.z), b);
    d = __ffma2_rn(w, make_float2(z, z), d);
    T = make_float2(s0 ? T.x : Tn.x, s1 ? T.y : Tn.y);
    return w.x + w.y;
}

// Whether a splat can reach alpha >= 1/255 at any pixel centre of the 8x8
// subtile whose first centre is (x0, y0): the minimum of its quadratic form
// q = (l00 dx + l01 dy)^2 + (l11 dy)^2 over the rectangle spanned by the
// centres, against log2(255 o) (B.w).  q is convex, so with the splat centre
// outside the rectangle the minimum lies on an edge, where it is the clamped
// stationary point of a 1D quadratic.  The test only skips splats that no
// pixel of the subtile blends: it keeps a relative margin of 1e-3 plus 1e-3
// on the threshold, far above the rounding of q here and in the blend loop.
__device__ __forceinline__ bool reaches_rect(const float4& A, const float4& B, float x0, float y0) {
    const float ax = x0 - A.x, bx = ax + 7.0f;  // dx range
    const float ay = y0 - A.y, by = ay + 7.0f;  // dy range
    if (ax <= 0.0f && bx >= 0.0f && ay <= 0.0f && by >= 0.0f) return true;
    const float l00 = B.x, l01 = B.y, l11 = B.z;
    auto q = [&](float dx, float dy) {
        const float t = fmaf(l01, dy, l00 * dx);
        const float u = l11 * dy;
        return fmaf(t, t, u * u);
    };
    // vertical edges dx = const: stationary dy = -l00 l01 dx / (l01^2 + l11^2);
    // horizontal edges dy = const: stationary dx = -l01 dy / l00.  Fast
    // divisions: q is evaluated exactly at whatever point is used, and a
    // stationary point off by a few ulp raises q only to second order.
    const float kv = __fdividef(-l00 * l01, fmaf(l01, l01, l11 * l11));
    const float kh = __fdividef(-l01, l00);
    const float q1 = q(ax, fminf(fmaxf(kv * ax, ay), by));
    const float q2 = q(bx, fminf(fmaxf(kv * bx, ay), by));
    const float q3 = q(fminf(fmaxf(kh * ay, ax), bx), ay);
    const float q4 = q(fminf(fmaxf(kh * by, ax), bx), by);
    const float qmin = fminf(fminf(q1, q2), fminf(q3, q4));
    return qmin <= fmaf(B.w, 1.001f, 1e-3f);
}

// Persistent CTAs of TW*TH/2 threads claim (env, tile) items from a work
// counter, `chunk` consecutive items at a time (items run env-major, tiles
// row-major, so envs of any resolution mix in one launch).  For an item the
// CTA covers the TW x TH tile: warp w owns an 8x8 subtile and each lane two
// pixels of it, (x, y) and (x, y + 4), whose blend chains are independent.
//
// A bucket of at most kCompCap keys is sorted in shared memory at once.  A
// longer bucket is first partitioned, in one counting pass, into kBins equal
// key ranges written in range order to the CTA's spill region (spill_cap
// keys); window w then holds the bins that start in [w H, (w+1) H) with
// H = kCompCap / 2, so every window is at most kCompCap keys unless one bin is
// larger than H; such a window (and a bucket longer than spill_cap, or any
// long bucket when there is no spill region) is cut into windows by radix
// selection over its keys instead.
// SC: contribution pass (pruning support): instead of writing images, add
// each blended (pixel, splat) weight alpha T to score[global index], summed
// per warp and splat before one atomic add.
// MODE 1: LiDAR scan (records of k_project_lidar; each "pixel" is a ray of
// the (azimuth, beam) grid, the Gaussian evaluated at its closest approach).
// MODE 2: the camera form that also counts composited (pixel, splat) pairs
// into P.neval (MODE 0 leaves the count out of its blend loop).
// MODE 3: LiDAR along arbitrary rays: an item is a chunk of at most 256 rays
// of one grid tile (16x16 tiles only); the chunk's rays are counting-sorted by
// cell so that each warp takes 64 neighbouring rays, and the warp's culling
// box is the bounding box of its rays' cells instead of a subtile.
// QUAD: each group of eight lanes owns a 4x4 quadrant of the warp's subtile
// and walks only the splats whose box reaches that quadrant, dropping it once
// the quadrant's pixels have terminated.  Small splats (low resolutions)
// reach one quadrant, so the groups then advance through different splats at
// once; large ones reach all four and the extra votes only cost (measured on
// the 2048-env room workload: 64x64 -21 %, 128x128 -15 %, 320x240 -3 %,
// 640x480 +1.4 % compositing time).  Every pixel still composites the same
// splats in the same order, so the images are identical either way.  Every
// bucket is long at those resolutions, so the quadrant form also fills each
// window of a partitioned bucket up to the cap and keeps several keys in
// flight per thread in the partition passes (64x64 and 128x128 -6 to -7 %;
// neither paid at 640x480).
template <int TW, int TH, bool SC = false, int MODE = 0, bool QUAD = false>
__global__ void __launch_bounds__(TW* TH / 2, (TW * TH >= 512 ? 4 : (TW * TH >= 256 ? 8 : 12))) k_composite(CompParams P) {
    constexpr int NT = TW * TH / 2;
    constexpr int NB = NT;  // splats staged per batch (one per thread)
    constexpr int CAP = kCompCap;
    constexpr int HALF = kCompCap / 2;
    constexpr int UB = (CAP * 8 > NB * 64) ? CAP * 8 : NB * 64;
    constexpr int CB = (18 * NT * 2 > kSortBins * 4) ? 18 * NT * 2 : kSortBins * 4;  // >= selection histogram
    constexpr int NW = NT / 32;
    constexpr bool CNT = MODE != 0 || SC;  // count composited pairs
    constexpr bool LID = MODE == 1 || MODE == 3;  // LiDAR records and ray evaluation
    static_assert(MODE != 3 || 2 * NT == kRayChunk, "ray chunks: two rays per thread");
    static_assert(CAP * 8 + UB >= kBins * 4, "bin counters alias the key and staging buffers");
    static_assert(kBins % NT == 0, "bins per thread");
    __shared__ __align__(16) unsigned char kbuf[CAP * 8 + UB];  // window keys | sort scratch, staged records
    __shared__ __align__(16) unsigned char cbuf[CB];            // radix counters | selection histogram
    __shared__ uint32_t red[32];
    __shared__ unsigned long long redl[2 * (NW > 0 ? NW : 1)];
    __shared__ unsigned long long sel_lo, sel_hi, sel_khi;
    __shared__ uint32_t sel_wn, sel_cnt;
    __shared__ int sel_state;
    __shared__ uint32_t s_ws[kSpillMax / (kCompCap / 2) + 2];  // window starts in the spill region
    __shared__ uint32_t s_zr[2 * (NW > 0 ? NW : 1)];             // per warp: depth bounds of a loaded window
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(kbuf);
    unsigned char* ubuf = kbuf + CAP * 8;
    unsigned long long* tmp = reinterpret_cast<unsigned long long*>(ubuf);
    float4* sA = reinterpret_cast<float4*>(ubuf);  // u, v, o, z
    float4* sB = sA + NB;                          // scaled conic factor l00, l01, l11
    float4* sC = sB + NB;                          // r, g, b
    int4* sR = reinterpret_cast<int4*>(sC + NB);   // x0, x1 - x0, y0, y1 - y0
    uint16_t* cnt = reinterpret_cast<uint16_t*>(cbuf);
    uint32_t* hist = reinterpret_cast<uint32_t*>(cbuf);
    __shared__ uint32_t sG[SC ? NB : 1];  // contribution pass: slot of each staged splat
    __shared__ float4 sD[LID ? NB : 1];  // LiDAR: third row of G of each staged splat
    uint32_t* bins = reinterpret_cast<uint32_t*>(kbuf);  // partition counters (between windows only)

    __shared__ unsigned int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool dbg = P.dbg_sorted != nullptr;
    unsigned long long* spill =
        P.spill ? P.spill + (size_t)blockIdx.x * P.spill_cap : nullptr;  // this CTA's region
    bool c32_dirty = true;  // the window sort's counters (cbuf) need clearing before use
    int el = P.e_begin;  // env of the current item, cached across items (uniform in the CTA)
    unsigned int e_lo = P.envs[el].tile_base, e_hi = e_lo + (unsigned)P.envs[el].T;
    if (tid == 0) s_item = atomicAdd(P.work, (unsigned)P.chunk);
    __syncthreads();
    for (;;) {
    const unsigned int first = P.item_begin + s_item;
    if (first >= P.item_end) break;
    const unsigned int last = min(first + (unsigned)P.chunk, P.item_end);
    for (unsigned int item = first; item < last; ++item) {
    int t;
    uint32_t rchunk = 0;  // MODE 3: chunk of the tile's rays
    if constexpr (MODE == 3) {
        int lo = P.e_begin, hi = P.e_end - 1;  // env: last e with item_base[e] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&P.item_base[mid]) <= (unsigned long long)item) lo = mid; else hi = mid - 1;
        }
        el = lo;
        e_lo = P.envs[el].tile_base;
        e_hi = e_lo + (unsigned)P.envs[el].T;
        const uint32_t li = item - (uint32_t)__ldg(&P.item_base[el]);
        int a = 0, b = P.envs[el].T - 1;  // tile: last t with item_off[t] <= li (empty tiles come before)
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (__ldg(&P.item_off[e_lo + mid]) <= li) a = mid; else b = mid - 1;
        }
        t = a;
        rchunk = li - __ldg(&P.item_off[e_lo + t]);
    } else {
        if (item < e_lo || item >= e_hi) {
            int lo = P.e_begin, hi = P.e_end - 1;  // env: last e with tile_base <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&P.envs[mid].tile_base) <= item) lo = mid; else hi = mid - 1;
            }
            el = lo;
            e_lo = P.envs[el].tile_base;
            e_hi = e_lo + (unsigned)P.envs[el].T;
        }
        t = (int)(item - e_lo);
    }
    const EnvInfo* Ep = P.envs + el;
    const int W = __ldg(&Ep->W), H = __ldg(&Ep->H), ntx = __ldg(&Ep->ntx);
    const unsigned int tile_base = e_lo;
    const unsigned int n_local = __ldg(&Ep->n_local);
    const unsigned long long pix_base = __ldg(&Ep->pix_base);
    const int tx = t % ntx, ty = t / ntx;
    constexpr int SWX = TW / 8;
    int wx0 = tx * TW + (warp % SWX) * 8, wy0 = ty * TH + (warp / SWX) * 8;
    int wx1 = wx0 + 7, wy1 = wy0 + 7;
    // QUAD: lanes in groups of eight, group q = lane / 8 owning the 4x4 quadrant
    // (q & 1, q >> 1) of the warp's subtile, each lane a column and rows r, r + 2;
    // otherwise lane = column (lane % 8) and rows lane / 8, lane / 8 + 4
    const int grp = lane >> 3, l8 = lane & 7;
    const int px = QUAD ? wx0 + 4 * (grp & 1) + (l8 & 3) : wx0 + (lane & 7);
    const int py0 = QUAD ? wy0 + 4 * (grp >> 1) + (l8 >> 2) : wy0 + (lane >> 3);
    const int py1 = QUAD ? py0 + 2 : py0 + 4;
    bool in0 = px < W && py0 < H, in1 = px < W && py1 < H;
    const float fpx = (float)px + 0.5f, fpy0 = (float)py0 + 0.5f, fpy1 = (float)py1 + 0.5f;
    float3 dir0 = make_float3(0.f, 0.f, 0.f), dir1 = dir0;  // LiDAR: the lane's two rays
    int cx0 = px, cy0 = py0, cx1 = px, cy1 = py1;           // LiDAR: their grid cells
    int ray0 = -1, ray1 = -1;                               // MODE 3: their indices
    float near_range = 0.0f;
    if constexpr (MODE == 1) {
        const gs_lidar* Ld = P.lidars + el;
        const float em = __ldg(&Ld->elev_min), eM = __ldg(&Ld->elev_max);
        const float az0 = __ldg(&Ld->az_min), span = __ldg(&Ld->az_max) - az0;
        const float phi = az0 + span * fpx / (float)W;
        const float th0 = em + (eM - em) * fpy0 / (float)H, th1 = em + (eM - em) * fpy1 / (float)H;
        float sp, cp, s0, c0, s1, c1;
        sincosf(phi, &sp, &cp);
        sincosf(th0, &s0, &c0);
        sincosf(th1, &s1, &c1);
        dir0 = make_float3(c0 * cp, c0 * sp, s0);
        dir1 = make_float3(c1 * cp, c1 * sp, s1);
        near_range = __ldg(&Ld->near_range);
    }
    if constexpr (MODE == 3) {
        // the chunk's rays, counting-sorted by cell (row-major in the tile)
        uint32_t* cellh = reinterpret_cast<uint32_t*>(kbuf);  // 256 counters
        uint32_t* srt = cellh + 256;                          // 256 ray indices
        const size_t renv = (size_t)el * (size_t)P.n_rays;
        const uint32_t rc = __ldg(&P.ray_cnt[e_lo + t]);
        const uint32_t nr = min((uint32_t)kRayChunk, rc - rchunk * (uint32_t)kRayChunk);
        const size_t lbase = renv + __ldg(&P.ray_off[e_lo + t]) + (size_t)rchunk * kRayChunk;
        for (int c = tid; c < 256; c += NT) cellh[c] = 0u;
        __syncthreads();
        uint32_t rr[2], cc[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint32_t k = (uint32_t)(tid + u * NT);
            rr[u] = k < nr ? __ldg(&P.ray_list[lbase + k]) : 0xffffffffu;
            cc[u] = k < nr ? (__ldg(&P.ray_cell[renv + rr[u]]) & 255u) : 0u;
            if (k < nr) atomicAdd(&cellh[cc[u]], 1u);
        }
        __syncthreads();
        const uint32_t h0 = cellh[2 * tid], h1 = cellh[2 * tid + 1];
        const uint32_t ex = block_excl_scan_u32<NT>(h0 + h1, red);
        cellh[2 * tid] = ex;
        cellh[2 * tid + 1] = ex + h0;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (rr[u] != 0xffffffffu) srt[atomicAdd(&cellh[cc[u]], 1u)] = rr[u];
        __syncthreads();
        const uint32_t s0 = (uint32_t)(warp * 64 + lane), s1 = s0 + 32u;
        ray0 = s0 < nr ? (int)srt[s0] : -1;
        ray1 = s1 < nr ? (int)srt[s1] : -1;
        __syncthreads();  // kbuf holds the windows from here on
        in0 = ray0 >= 0;
        in1 = ray1 >= 0;
        near_range = __ldg(&P.lidars[el].near_range);
        auto take = [&](int r, int& ci, int& cj, float3& d) {
            const uint32_t c = __ldg(&P.ray_cell[renv + (uint32_t)r]) & 255u;
            ci = tx * 16 + (int)(c & 15u);
            cj = ty * 16 + (int)(c >> 4);
            const float* v = P.ray_dirs + (renv + (uint32_t)r) * 3;
            const float x = v[0], y = v[1], z = v[2];
            const float inv = 1.0f / sqrtf(x * x + y * y + z * z);
            d = make_float3(x * inv, y * inv, z * inv);
        };
        if (in0) take(ray0, cx0, cy0, dir0);
        if (in1) take(ray1, cx1, cy1, dir1);
        // the warp's culling box: the cells of its rays
        const int big = 1 << 30;
        wx0 = __reduce_min_sync(0xffffffffu, min(in0 ? cx0 : big, in1 ? cx1 : big));
        wy0 = __reduce_min_sync(0xffffffffu, min(in0 ? cy0 : big, in1 ? cy1 : big));
        wx1 = __reduce_max_sync(0xffffffffu, max(in0 ? cx0 : -big, in1 ? cx1 : -big));
        wy1 = __reduce_max_sync(0xffffffffu, max(in0 ? cy0 : -big, in1 ? cy1 : -big));
    }
    // LiDAR: alpha and t* of a staged Gaussian (b, o | g0 | g1 | g2) on each
    // of the lane's two rays d: u = G d, q = |u x b|^2 / |u|^2, t* = u.b / |u|^2,
    // with paired FP32 instructions (the reciprocal of |u|^2 by the fast
    // division, ~2 ulp, far inside the scan's tolerance).
    auto ray_eval2 = [&](const float4& A, const float4& B, const float4& C, const float4& D, float2& al,
                         float2& ts) {
        const float2 dx = make_float2(dir0.x, dir1.x), dy = make_float2(dir0.y, dir1.y),
                     dz = make_float2(dir0.z, dir1.z);
        auto dot = [&](const float4& G) {
            return __ffma2_rn(make_float2(G.z, G.z), dz,
                              __ffma2_rn(make_float2(G.y, G.y), dy, __fmul2_rn(make_float2(G.x, G.x), dx)));
        };
        const float2 u0 = dot(B), u1 = dot(C), u2 = dot(D);
        const float2 aa = __ffma2_rn(u2, u2, __ffma2_rn(u1, u1, __fmul2_rn(u0, u0)));
        const float2 ab = __ffma2_rn(u2, make_float2(A.z, A.z),
                                     __ffma2_rn(u1, make_float2(A.y, A.y), __fmul2_rn(u0, make_float2(A.x, A.x))));
        const float2 c0 = __ffma2_rn(u1, make_float2(A.z, A.z), __fmul2_rn(u2, make_float2(-A.y, -A.y)));
        const float2 c1 = __ffma2_rn(u2, make_float2(A.x, A.x), __fmul2_rn(u0, make_float2(-A.z, -A.z)));
        const float2 c2 = __ffma2_rn(u0, make_float2(A.y, A.y), __fmul2_rn(u1, make_float2(-A.x, -A.x)));
        const float2 cc = __ffma2_rn(c2, c2, __ffma2_rn(c1, c1, __fmul2_rn(c0, c0)));
        const float2 inv = make_float2(__fdividef(1.0f, aa.x), __fdividef(1.0f, aa.y));
        const float2 q = __fmul2_rn(cc, inv);
        ts = __fmul2_rn(ab, inv);
        const float k = -0.72134752044448170f;  // -log2(e) / 2
        al.x = ts.x > near_range ? fminf(0.99f, A.w * ex2_approx(k * q.x)) : 0.0f;
        al.y = ts.y > near_range ? fminf(0.99f, A.w * ex2_approx(k * q.y)) : 0.0f;
    };
    bool done0 = !in0, done1 = !in1;
    // the lane's two pixels: .x = (px, py0), .y = (px, py1)
    float2 Tp = make_float2(1.0f, 1.0f), rp = make_float2(0.0f, 0.0f), gp = rp, bp = rp, dp = rp;
    const float2 fpy = make_float2(fpy0, fpy1);
    uint32_t ncomp = 0;

    uint32_t n = P.counts[tile_base + t];
    const unsigned long long start = P.env_base[el] - P.pair_base + P.off_local[tile_base + t];
    if (start + n > P.pair_cap) {  // keys past a planned capacity were dropped: render nothing
        n = 0;
        if (tid == 0) atomicOr(P.status, kStOverflow);
    }
    const unsigned long long* Lk = P.pairs + start;
    const size_t recbase = (size_t)__ldg(&Ep->rec_base);
    // contribution pass: record slot -> global Gaussian index
    const long long g_link0 = SC ? __ldg(&Ep->g_link0) : 0ll;
    auto score_index = [&](uint32_t j) -> long long {
        if (j < P.nbp) return P.bg_index ? (long long)__ldg(P.bg_index + j) : (long long)j;
        return g_link0 + (long long)(j - P.nbp);
    };
    bool finished = false;
    uint32_t win_zmin = 0u, win_zmax = 0xffffffffu;  // depth-bit bounds of the loaded window
    // A window producer's last pass: the block-wide depth bounds of the keys
    // it loaded, folded into the barrier that ends the load.
    auto end_load = [&](uint32_t zl, uint32_t zh) {
        zl = __reduce_min_sync(0xffffffffu, zl);
        zh = __reduce_max_sync(0xffffffffu, zh);
        if (lane == 0) {
            s_zr[warp] = zl;
            s_zr[NW + warp] = zh;
        }
        __syncthreads();
        win_zmin = s_zr[0];
        win_zmax = s_zr[NW];
        for (int w = 1; w < NW; ++w) {
            win_zmin = min(win_zmin, s_zr[w]);
            win_zmax = max(win_zmax, s_zr[NW + w]);
        }
    };

    // Sort keys[0, wn) (the next wn keys in depth order) and composite them;
    // `before` keys of the bucket precede them.  Sets `finished` once every
    // pixel of the tile has terminated.
    auto run_window = [&](uint32_t wn, uint32_t before) {
        const unsigned long long* sorted =
            window_sort<NT>(keys, tmp, cnt, red, (int)wn, win_zmin, win_zmax, c32_dirty);
        if (dbg)
            for (uint32_t i = tid; i < wn; i += NT) P.dbg_sorted[start + before + i] = sorted[i];
        // Move the sorted window home (from the scratch half) and, where keys
        // carry the caller's background index, swap in the record slot.
        if (sorted != keys || P.bg_slot) {
            for (uint32_t i = tid; i < wn; i += NT) {
                unsigned long long k = sorted[i];
                const uint32_t g = (uint32_t)(k & 0xffffffffull);
                if (P.bg_slot && g < P.n_bg) k = (k & 0xffffffff00000000ull) | (uint32_t)__ldg(P.bg_slot + g);
                keys[i] = k;
            }
            __syncthreads();
        }

        for (uint32_t b = 0; b < wn; b += NB) {
            const int cnt_b = (int)min((uint32_t)NB, wn - b);
            for (int s = tid; s < cnt_b; s += NT) {
                const uint32_t g = (uint32_t)(keys[b + s] & 0xffffffffull);
                if (g < n_local) {
                    const size_t ri = recbase + g;
                    const float4 q0 = P.r0[kRecStride * ri];
                    const float4 q1 = P.r1[kRecStride * ri];
                    const float4 q2 = P.r2[kRecStride * ri];
                    const uint32_t rx = __float_as_uint(q1.w), ry = __float_as_uint(q2.w);
                    sA[s] = LID ? q0 : make_float4(q0.x, q0.y, log2f(q0.z), q0.w);  // camera: log2(o)
                    if constexpr (LID) {
                        // g2 = |g2| (g0 x g1) / (|g0| |g1|): the rows of G are orthogonal
                        const float glen2 = __uint_as_float(P.r3[ri].w);
                        const float cx = q1.y * q2.z - q1.z * q2.y, cy = q1.z * q2.x - q1.x * q2.z,
                                    cz = q1.x * q2.y - q1.y * q2.x;
                        const float k = glen2 * rsqrtf((q1.x * q1.x + q1.y * q1.y + q1.z * q1.z) *
                                                       (q2.x * q2.x + q2.y * q2.y + q2.z * q2.z));
                        sB[s] = make_float4(q1.x, q1.y, q1.z, 0.0f);
                        sD[s] = make_float4(cx * k, cy * k, cz * k, 0.0f);
                    } else {
                        // alpha >= 1/255 iff q <= w (w only feeds the subtile cull, whose
                        // 1e-3 margin dwarfs the error of the fast logarithm)
                        sB[s] = make_float4(q1.x, q1.y, q1.z, __log2f(255.0f * q0.z));
                    }
                    sC[s] = q2;
                    int bx0 = (int)(rx & 0xffffu), bx1 = (int)(rx >> 16);
                    if (LID && bx0 > bx1) {
                        // a LiDAR box across azimuth 0 (columns [x0, cols) and
                        // [0, x1]): the hull of its parts in this tile's columns
                        // [ta, tb], the high part [max(x0, ta), tb] when x0 <= tb
                        // and the low part [ta, min(x1, tb)] when x1 >= ta
                        const int ta = tx * TW, tb = ta + TW - 1;
                        const int h0 = max(bx0, ta), l1 = min(bx1, tb);
                        bx0 = bx1 >= ta ? ta : h0;
                        bx1 = h0 <= tb ? tb : l1;
                    }
                    sR[s] = make_int4(bx0, bx1 - bx0, (int)(ry & 0xffffu), (int)((ry >> 16) - (ry & 0xffffu)));
                    if constexpr (SC) sG[s] = g;
                } else {  // never happens for a well-formed bucket; stage an empty range
                    sA[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sB[s] = sA[s];
                    sC[s] = sA[s];
                    if constexpr (!LID) sA[s].z = -126.0f;  // log2 of a vanishing opacity
                    sR[s] = make_int4(1 << 20, -1, 1 << 20, -1);
                    atomicOr(P.status, kStOverflow);
                }
            }
            __syncthreads();
            if (!__all_sync(0xffffffffu, done0 && done1)) {
                for (int c = 0; c < cnt_b; c += 32) {
                    const int j = c + lane;
                    bool ov = false;
                    if constexpr (!LID) {
                        // camera splats: box, then the exact ellipse for large ones
                        // (a box under 24 px in width + height is kept as it is: it
                        // overstates the ellipse least), evaluated by every lane
                        const int jj = j < cnt_b ? j : c;
                        const int4 R = sR[jj];
                        ov = j < cnt_b && R.x <= wx1 && R.x + R.y >= wx0 && R.z <= wy1 && R.z + R.w >= wy0;
                        const bool rr = reaches_rect(sA[jj], sB[jj], (float)wx0 + 0.5f, (float)wy0 + 0.5f);
                        ov = ov && (R.y + R.w < 24 || rr);
                    } else if (j < cnt_b) {
                        const int4 R = sR[j];
                        ov = R.x <= wx1 && R.x + R.y >= wx0 && R.z <= wy1 && R.z + R.w >= wy0;
                    }
                    uint32_t m;
                    if constexpr (QUAD) {
                        // per quadrant: the splats whose box reaches it
                        bool qa = false, qb = false, qc = false, qd = false;
                        if (ov) {
                            const int4 R = sR[j];
                            const bool c0 = R.x <= wx0 + 3, c1 = R.x + R.y >= wx0 + 4;
                            const bool r0 = R.z <= wy0 + 3, r1 = R.z + R.w >= wy0 + 4;
                            qa = c0 && r0;
                            qb = c1 && r0;
                            qc = c0 && r1;
                            qd = c1 && r1;
                        }
                        const uint32_t ma = __ballot_sync(0xffffffffu, qa), mb = __ballot_sync(0xffffffffu, qb);
                        const uint32_t mc = __ballot_sync(0xffffffffu, qc), md = __ballot_sync(0xffffffffu, qd);
                        const uint32_t dm = __ballot_sync(0xffffffffu, done0 && done1);
                        m = grp == 0 ? ma : (grp == 1 ? mb : (grp == 2 ? mc : md));
                        if (((dm >> (8 * grp)) & 0xffu) == 0xffu) m = 0u;
                    } else {
                        m = __ballot_sync(0xffffffffu, ov);
                    }
                    float2 score_pair = make_float2(0.0f, 0.0f);  // contribution pass only
                    // Camera splats of opacity <= 0.98 never reach the 0.99 cap of
                    // alpha (o 2^-q with q >= 0), so a chunk without brighter splats
                    // walks a copy of the loop without the cap (non-quadrant form;
                    // the quadrant form measured slower with the extra vote).
                    bool clamp_chunk = true;
                    if constexpr (!LID && !QUAD)  // staged log2(o) > log2(0.98)
                        clamp_chunk = __any_sync(0xffffffffu, j < cnt_b && sA[j].z > -0.029146346f);
                    auto walk = [&](auto clamp_tag) {
                    constexpr bool CL = decltype(clamp_tag)::value;
                    // two splats per iteration: their four alpha evaluations are
                    // independent; the blends then run in depth order
                    while (QUAD ? __any_sync(0xffffffffu, m != 0u) : m != 0u) {
                        const bool one = !QUAD || m != 0u;
                        const int k1 = one ? __ffs(m) - 1 : 0;
                        m &= m - 1u;
                        const bool two = m != 0u;
                        const int k2 = two ? __ffs(m) - 1 : k1;
                        if (two) m &= m - 1u;
                        const int j1 = c + k1, j2 = c + k2;
                        // Camera pixels skip the per-pixel box test: a pixel outside a
                        // splat's support box has q > q* (1 + 2e-4), so its alpha falls
                        // below 1/255 and the alpha test alone rejects it.  LiDAR rays
                        // keep the test (their grid box is a looser cone bound and a ray
                        // evaluation costs more).
                        bool h10 = one && !done0, h11 = one && !done1, h20 = two && !done0, h21 = two && !done1;
                        if constexpr (MODE == 1) {
                            const int4 R1 = sR[j1];
                            const int4 R2 = sR[j2];
                            const bool x1 = (unsigned)(px - R1.x) <= (unsigned)R1.y;
                            const bool x2 = (unsigned)(px - R2.x) <= (unsigned)R2.y;
                            h10 = h10 && x1 && (unsigned)(py0 - R1.z) <= (unsigned)R1.w;
                            h11 = h11 && x1 && (unsigned)(py1 - R1.z) <= (unsigned)R1.w;
                            h20 = h20 && x2 && (unsigned)(py0 - R2.z) <= (unsigned)R2.w;
                            h21 = h21 && x2 && (unsigned)(py1 - R2.z) <= (unsigned)R2.w;
                        } else if constexpr (MODE == 3) {
                            const int4 R1 = sR[j1];
                            const int4 R2 = sR[j2];
                            auto inb = [](const int4& R, int x, int y) {
                                return (unsigned)(x - R.x) <= (unsigned)R.y && (unsigned)(y - R.z) <= (unsigned)R.w;
                            };
                            h10 = h10 && inb(R1, cx0, cy0);
                            h11 = h11 && inb(R1, cx1, cy1);
                            h20 = h20 && inb(R2, cx0, cy0);
                            h21 = h21 && inb(R2, cx1, cy1);
                        }
                        // Grid scans evaluate every lane's rays (no divergent branch, so
                        // the vote below sees every lane); along arbitrary rays the
                        // per-ray boxes cull so much that the branch pays.
                        if (MODE == 1 || (MODE == 3 && (h10 || h11 || h20 || h21))) {
                            const float4 A1 = sA[j1], B1 = sB[j1], C1 = sC[j1], D1 = sD[LID ? j1 : 0];
                            const float4 A2 = sA[j2], B2 = sB[j2], C2 = sC[j2], D2 = sD[LID ? j2 : 0];
                            float2 al1, ts1, al2, ts2;
                            ray_eval2(A1, B1, C1, D1, al1, ts1);
                            ray_eval2(A2, B2, C2, D2, al2, ts2);
                            const float a10 = al1.x, a11 = al1.y, a20 = al2.x, a21 = al2.y;
                            const float t10 = ts1.x, t11 = ts1.y, t20 = ts2.x, t21 = ts2.y;
                            const float4 none = make_float4(0.f, 0.f, 0.f, 0.f);
                            bool voted = false;  // both splats blended by the vote path below
                            if constexpr (MODE == 1) {
                                // as in the camera form: both splats with selects unless a ray stops
                                const bool u10 = h10 && a10 >= (1.0f / 255.0f), u11 = h11 && a11 >= (1.0f / 255.0f);
                                const float2 am1 = make_float2(u10 ? a10 : 0.0f, u11 ? a11 : 0.0f);
                                const float2 x1 = __fmul2_rn(am1, Tp);
                                const float2 Tn1 = __fadd2_rn(Tp, make_float2(-x1.x, -x1.y));
                                const bool v20 = h20 && a20 >= (1.0f / 255.0f), v21 = h21 && a21 >= (1.0f / 255.0f);
                                const float2 am2 = make_float2(v20 ? a20 : 0.0f, v21 ? a21 : 0.0f);
                                const float2 x2 = __fmul2_rn(am2, Tn1);
                                const float2 Tn2 = __fadd2_rn(Tn1, make_float2(-x2.x, -x2.y));
                                const bool stop = Tn2.x < 1e-4f || Tn2.y < 1e-4f;  // Tn2 <= Tn1
                                if (!__any_sync(0xffffffffu, stop)) {
                                    if constexpr (CNT) ncomp += (uint32_t)u10 + (uint32_t)u11 + (uint32_t)v20 + (uint32_t)v21;
                                    dp = __ffma2_rn(x1, ts1, dp);
                                    dp = __ffma2_rn(x2, ts2, dp);
                                    Tp = Tn2;
                                    voted = true;
                                }
                            }
                            if (!voted) {
                                if (h10 && a10 >= (1.0f / 255.0f)) {
                                    if constexpr (CNT) ++ncomp;
                                    blend(a10, none, t10, Tp.x, rp.x, gp.x, bp.x, dp.x, done0);
                                }
                                if (h11 && a11 >= (1.0f / 255.0f)) {
                                    if constexpr (CNT) ++ncomp;
                                    blend(a11, none, t11, Tp.y, rp.y, gp.y, bp.y, dp.y, done1);
                                }
                                if (h20 && !done0 && a20 >= (1.0f / 255.0f)) {
                                    if constexpr (CNT) ++ncomp;
                                    blend(a20, none, t20, Tp.x, rp.x, gp.x, bp.x, dp.x, done0);
                                }
                                if (h21 && !done1 && a21 >= (1.0f / 255.0f)) {
                                    if constexpr (CNT) ++ncomp;
                                    blend(a21, none, t21, Tp.y, rp.y, gp.y, bp.y, dp.y, done1);
                                }
                            }
                        } else if constexpr (!LID) {
                            const float4 A1 = sA[j1], B1 = sB[j1];
                            const float4 A2 = sA[j2], B2 = sB[j2];
                            const float2 a1 = splat_alpha2<CL>(A1, B1, fpx, fpy);
                            const float2 a2 = splat_alpha2<CL>(A2, B2, fpx, fpy);
                            const bool u10 = h10 && a1.x >= (1.0f / 255.0f);
                            const bool u11 = h11 && a1.y >= (1.0f / 255.0f);
                            float w1 = 0.0f, w2 = 0.0f;
                            // Both splats' blends with plain selects while no pixel of the
                            // warp stops at either (the common case); else one splat at a
                            // time with the stop rule.  Either way the arithmetic is that
                            // of blend2, so the images do not depend on the path taken.
                            // Every lane of the warp reaches the vote: the camera path has
                            // no divergent branch around it (branches here measured slower
                            // than evaluating every lane's pixels).
                            const float2 am1 = make_float2(u10 ? a1.x : 0.0f, u11 ? a1.y : 0.0f);
                            const float2 x1 = __fmul2_rn(am1, Tp);
                            const float2 Tn1 = __fadd2_rn(Tp, make_float2(-x1.x, -x1.y));
                            const bool v20 = h20 && a2.x >= (1.0f / 255.0f);
                            const bool v21 = h21 && a2.y >= (1.0f / 255.0f);
                            const float2 am2 = make_float2(v20 ? a2.x : 0.0f, v21 ? a2.y : 0.0f);
                            const float2 x2 = __fmul2_rn(am2, Tn1);
                            const float2 Tn2 = __fadd2_rn(Tn1, make_float2(-x2.x, -x2.y));
                            // Tn2 = Tn1 - am2 Tn1 <= Tn1 (am2 >= 0, rounding is monotone),
                            // so a pixel that stops at either splat has Tn2 < 1e-4
                            const bool stop = Tn2.x < 1e-4f || Tn2.y < 1e-4f;
                            if (!__any_sync(0xffffffffu, stop)) {
                                if constexpr (CNT) ncomp += (uint32_t)u10 + (uint32_t)u11 + (uint32_t)v20 + (uint32_t)v21;
                                const float4 C1 = sC[j1], C2 = sC[j2];
                                rp = __ffma2_rn(x1, make_float2(C1.x, C1.x), rp);
                                gp = __ffma2_rn(x1, make_float2(C1.y, C1.y), gp);
                                bp = __ffma2_rn(x1, make_float2(C1.z, C1.z), bp);
                                dp = __ffma2_rn(x1, make_float2(A1.w, A1.w), dp);
                                rp = __ffma2_rn(x2, make_float2(C2.x, C2.x), rp);
                                gp = __ffma2_rn(x2, make_float2(C2.y, C2.y), gp);
                                bp = __ffma2_rn(x2, make_float2(C2.z, C2.z), bp);
                                dp = __ffma2_rn(x2, make_float2(A2.w, A2.w), dp);
                                Tp = Tn2;
                                w1 = x1.x + x1.y;
                                w2 = x2.x + x2.y;
                            } else {
                                if constexpr (CNT) ncomp += (uint32_t)u10 + (uint32_t)u11;
                                w1 = blend2(a1, u10, u11, sC[j1], A1.w, Tp, rp, gp, bp, dp, done0, done1);
                                const bool u20 = h20 && !done0 && a2.x >= (1.0f / 255.0f);
                                const bool u21 = h21 && !done1 && a2.y >= (1.0f / 255.0f);
                                if constexpr (CNT) ncomp += (uint32_t)u20 + (uint32_t)u21;
                                w2 = blend2(a2, u20, u21, sC[j2], A2.w, Tp, rp, gp, bp, dp, done0, done1);
                            }
                            if constexpr (SC) score_pair = make_float2(w1, w2);
                        }
                        if constexpr (SC) {  // warp-uniform: every lane reaches this point
                            // the lanes that walk the same splats add their weights
                            const float s1 = QUAD ? group_sum(score_pair.x) : warp_sum(score_pair.x);
                            const float s2 = QUAD ? group_sum(score_pair.y) : warp_sum(score_pair.y);
                            score_pair = make_float2(0.0f, 0.0f);
                            if (QUAD ? l8 == 0 : lane == 0) {
                                if (one && s1 > 0.0f) atomicAdd(P.score + score_index(sG[j1]), s1);
                                if (two && s2 > 0.0f) atomicAdd(P.score + score_index(sG[j2]), s2);
                            }
                        }
                    }
                    };
                    if constexpr (LID || QUAD) walk(std::true_type{});
                    else if (clamp_chunk) walk(std::true_type{});
                    else walk(std::false_type{});
                    if (__all_sync(0xffffffffu, done0 && done1)) break;
                }
            }
            const bool all = __syncthreads_and(done0 && done1) != 0;
            if (all && !dbg) {
                finished = true;
                break;
            }
        }
    };

    // Smallest and largest of the keys L[0, len) (block-wide).
    auto key_range = [&](const unsigned long long* L, uint32_t len, unsigned long long& mn,
                         unsigned long long& mx) {
        unsigned long long a = ~0ull, b = 0;
        auto take = [&](uint32_t, unsigned long long k) {
            a = k < a ? k : a;
            b = k > b ? k : b;
        };
        if constexpr (QUAD) for_keys<NT, 4>(L, len, take);  // long buckets are the rule there
        else for (uint32_t i = tid; i < len; i += NT) take(i, L[i]);
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, d);
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, d);
            a = oa < a ? oa : a;
            b = ob > b ? ob : b;
        }
        if (lane == 0) {
            redl[warp] = a;
            redl[NW + warp] = b;
        }
        __syncthreads();
        mn = redl[0];
        mx = redl[NW];
        for (int w = 1; w < NW; ++w) {
            mn = redl[w] < mn ? redl[w] : mn;
            mx = redl[NW + w] > mx ? redl[NW + w] : mx;
        }
        __syncthreads();
    };

    // Radix-select, among the keys of L[0, len) inside [lo, hi], the smallest
    // ones: on success khi is such that the keys in [lo, khi) number wn, with
    // 0 < wn <= cap (8-bit digits of the key range; distinct keys are always
    // isolated within eight levels).  False means a corrupted bucket.
    auto select = [&](const unsigned long long* L, uint32_t len, unsigned long long lo0, unsigned long long hi0,
                      uint32_t cap, unsigned long long& khi, uint32_t& wn) -> bool {
        c32_dirty = true;  // hist shares the window sort's counters
        if (tid == 0) {
            sel_lo = lo0;
            sel_hi = hi0;
            sel_state = 0;
        }
        __syncthreads();
        for (int level = 0; level < 10; ++level) {
            const unsigned long long lo = sel_lo, hi = sel_hi;
            const unsigned long long x = lo ^ hi;
            const int hb = x ? 63 - __clzll((long long)x) : 0;
            const int shift = hb > 7 ? hb - 7 : 0;
            for (int i = tid; i < 256; i += NT) hist[i] = 0;
            __syncthreads();
            for (uint32_t i = tid; i < len; i += NT) {
                const unsigned long long k = L[i];
                if (k >= lo && k <= hi) atomicAdd(&hist[(k >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                const unsigned long long pre = (lo >> (shift + 8)) << (shift + 8);
                int d = 0;
                while (d < 255 && hist[d] == 0) ++d;
                if (hist[d] > cap) {
                    const unsigned long long blo = pre | ((unsigned long long)d << shift);
                    const unsigned long long bhi = blo | ((1ull << shift) - 1ull);
                    sel_lo = blo > lo ? blo : lo;
                    sel_hi = bhi < hi ? bhi : hi;
                } else {
                    uint32_t cum = 0;
                    while (d < 256 && cum + hist[d] <= cap) {
                        cum += hist[d];
                        ++d;
                    }
                    // window ends just before digit d (or after hi when all digits fit)
                    unsigned long long kh;
                    if (d >= 256) {
                        kh = hi + 1ull;
                    } else {
                        kh = pre | ((unsigned long long)d << shift);
                        if (kh > hi + 1ull) kh = hi + 1ull;
                    }
                    sel_khi = kh;
                    sel_wn = cum;
                    sel_state = 1;
                }
            }
            __syncthreads();
            if (sel_state) break;
        }
        const bool ok = sel_state != 0 && sel_wn > 0;
        khi = sel_khi;
        wn = sel_wn;
        __syncthreads();  // the shared selection state is rewritten by the next call
        return ok;
    };

    // Window producer: fills keys[0, wn) with the next wn keys of the bucket
    // in depth order (unsorted) and returns wn, 0 when the bucket is done.
    // Short buckets are one window; long ones are partitioned run by run into
    // the spill region (see above), and a segment that needs it (an oversized
    // window, or the whole bucket without a spill region) is cut by selection.
    unsigned long long klo = 0, kmax = 0;
    uint32_t processed = 0;  // keys of the bucket in runs started so far
    int w = 0, nw = 0;       // next window of the current run
    const unsigned long long* seg = nullptr;
    uint32_t seg_len = 0, seg_used = 0;
    unsigned long long seg_lo = 0, seg_hi = 0;
    bool started = false;
    auto next_window = [&]() -> uint32_t {
        if (n <= (uint32_t)CAP) {
            if (started || n == 0) return 0u;
            started = true;
            uint32_t zl = 0xffffffffu, zh = 0u;
            for_keys<NT, 6>(Lk, n, [&](uint32_t i, unsigned long long k) {
                keys[i] = k;
                const uint32_t z = (uint32_t)(k >> 32);
                zl = min(zl, z);
                zh = max(zh, z);
            });
            end_load(zl, zh);
            return n;
        }
        if (!started) {
            started = true;
            if (spill && P.zr) {  // the env's depth range bounds every key of its buckets
                const uint2 r = P.zr[el];
                klo = (unsigned long long)r.x << 32;
                kmax = ((unsigned long long)~r.y << 32) | 0xffffffffull;
            } else {
                key_range(Lk, n, klo, kmax);
            }
            if (!spill) {
                seg = Lk;
                seg_len = n;
                seg_lo = klo;
                seg_hi = kmax;
                processed = n;
            }
        }
        for (;;) {
            if (seg_used < seg_len) {  // cut the segment by selection
                unsigned long long kh;
                uint32_t wn;
                if (seg_len - seg_used <= (uint32_t)CAP) {
                    kh = seg_hi + 1ull;
                    wn = seg_len - seg_used;
                } else if (!select(seg, seg_len, seg_lo, seg_hi, CAP, kh, wn)) {
                    if (tid == 0) atomicOr(P.status, kStOverflow);
                    return 0u;
                }
                if (tid == 0) sel_cnt = 0;
                __syncthreads();
                uint32_t zl = 0xffffffffu, zh = 0u;
                for_keys<NT, 4>(seg, seg_len, [&](uint32_t, unsigned long long k) {
                    if (k >= seg_lo && k < kh) {
                        const uint32_t slot = atomicAdd(&sel_cnt, 1u);
                        if (slot < (uint32_t)CAP) keys[slot] = k;
                        const uint32_t z = (uint32_t)(k >> 32);
                        zl = min(zl, z);
                        zh = max(zh, z);
                    }
                });
                end_load(zl, zh);
                seg_used += wn;
                seg_lo = kh;
                return wn;
            }
            if (w < nw) {  // the next window of the partitioned run
                const uint32_t a = s_ws[w], b = s_ws[w + 1];
                ++w;
                if (b <= a) continue;
                if (b - a <= (uint32_t)CAP) {
                    uint32_t zl = 0xffffffffu, zh = 0u;
                    for_keys<NT, 6>(spill + a, b - a, [&](uint32_t i, unsigned long long k) {
                        keys[i] = k;
                        const uint32_t z = (uint32_t)(k >> 32);
                        zl = min(zl, z);
                        zh = max(zh, z);
                    });
                    end_load(zl, zh);
                    return b - a;
                }
                seg = spill + a;  // a bin of more than HALF keys
                seg_len = b - a;
                seg_used = 0;
                key_range(seg, seg_len, seg_lo, seg_hi);
                continue;
            }
            if (processed >= n) return 0u;
            // the next run of at most spill_cap keys, [klo, kh), partitioned
            // into kBins key ranges in the spill region
            unsigned long long kh;
            uint32_t m;
            if (n - processed <= P.spill_cap) {
                kh = kmax + 1ull;
                m = n - processed;
            } else if (!select(Lk, n, klo, kmax, P.spill_cap, kh, m)) {
                if (tid == 0) atomicOr(P.status, kStOverflow);
                return 0u;
            }
            const unsigned long long span = kh - 1ull - klo;
            const int shift = (span >> 11) ? 53 - __clzll((long long)span) : 0;  // span >> shift < kBins
            for (int i = tid; i < kBins; i += NT) bins[i] = 0;
            __syncthreads();
            auto count_key = [&](uint32_t, unsigned long long k) {
                if (k >= klo && k < kh) atomicAdd(&bins[(uint32_t)((k - klo) >> shift)], 1u);
            };
            if constexpr (QUAD) for_keys<NT, 4>(Lk, n, count_key);
            else for (uint32_t i = tid; i < n; i += NT) count_key(i, Lk[i]);
            __syncthreads();
            constexpr int PER = kBins / NT;
            uint32_t loc = 0, big = 0;
#pragma unroll 4
            for (int j = 0; j < PER; ++j) {
                const uint32_t c = bins[tid * PER + j];
                loc += c;
                if constexpr (QUAD) big = c > big ? c : big;
            }
            // window stride: a window holds the bins that start in one stride of
            // keys, so it is at most stride + the largest bin; the quadrant form
            // (low resolutions: every bucket long) fills windows up to the cap
            uint32_t stride = HALF;
            if constexpr (QUAD) {
                uint32_t none = 0;
                block_minmax_u32<NT>(none, big, red);
                if (big <= (uint32_t)HALF) stride = (uint32_t)CAP - big;
            }
            uint32_t run = block_excl_scan_u32<NT>(loc, red);
#pragma unroll 4
            for (int j = 0; j < PER; ++j) {
                const uint32_t c = bins[tid * PER + j];
                bins[tid * PER + j] = run;
                run += c;
            }
            __syncthreads();
            // window v: the bins that start in [v stride, (v+1) stride)
            nw = (int)((m + stride - 1) / stride);
            for (int v = tid; v <= nw; v += NT) {
                uint32_t x = m;
                if (v == 0) {
                    x = 0;
                } else if (v < nw) {
                    const uint32_t target = (uint32_t)v * stride;
                    int lo = 0, hi = kBins;  // first bin whose start >= target
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (bins[mid] >= target) hi = mid; else lo = mid + 1;
                    }
                    x = lo < kBins ? bins[lo] : m;
                }
                s_ws[v] = x;
            }
            __syncthreads();
            auto place = [&](uint32_t, unsigned long long k) {
                if (k >= klo && k < kh) {
                    const uint32_t pos = atomicAdd(&bins[(uint32_t)((k - klo) >> shift)], 1u);
                    spill[pos] = k;
                }
            };
            if constexpr (QUAD) for_keys<NT, 4>(Lk, n, place);
            else for (uint32_t i = tid; i < n; i += NT) place(i, Lk[i]);
            __syncthreads();
            w = 0;
            processed += m;
            klo = kh;
        }
    };

    uint32_t before = 0;  // keys of the bucket composited so far (windows come in depth order)
    while (!finished) {
        const uint32_t wn = next_window();
        if (wn == 0) break;
        run_window(wn, before);
        before += wn;
    }

    if (CNT && P.neval) {
        uint32_t c = ncomp;
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0 && c) atomicAdd(P.neval, (unsigned long long)c);
    }
    // Outputs.  Observation form (rgb8 / depth16): the clamped colour goes
    // through the env's appearance transform (exposure gain 2^e, contrast c
    // about 0.5, brightness offset b), is clamped again and rounded to 8 bits;
    // depth is rounded to half precision.
    float gain = 1.0f, con = 1.0f, bri = 0.0f;
    if (P.rgb8 && P.appear) {
        const gs_appearance ap = P.appear[el];
        gain = exp2f(ap.exposure);
        con = ap.contrast;
        bri = ap.brightness;
    }
    auto store = [&](int py, float T, float r, float g, float b, float d) {
        const size_t pix = pix_base + (size_t)py * W + px;
        const float cr = fminf(fmaxf(r, 0.0f), 1.0f), cg = fminf(fmaxf(g, 0.0f), 1.0f),
                    cb = fminf(fmaxf(b, 0.0f), 1.0f);
        const float a = 1.0f - T;
        const float dep = a > 0.0f ? d / a : 0.0f;
        if (P.rgb8) {
            auto q = [&](float v) {
                // no appearance given: the identity, exactly ((v - 0.5) + 0.5 would round)
                if (P.appear) v = fmaf(fmaf(v, gain, -0.5f), con, 0.5f + bri);
                return (uint8_t)__float2int_rn(fminf(fmaxf(v, 0.0f), 1.0f) * 255.0f);
            };
            P.rgb8[3 * pix] = q(cr);
            P.rgb8[3 * pix + 1] = q(cg);
            P.rgb8[3 * pix + 2] = q(cb);
        } else {
            P.rgb[3 * pix] = cr;
            P.rgb[3 * pix + 1] = cg;
            P.rgb[3 * pix + 2] = cb;
        }
        if (P.depth16) P.depth16[pix] = __half_as_ushort(__float2half_rn(dep));
        else if (P.depth) P.depth[pix] = dep;
        if (P.alpha) P.alpha[pix] = a;
    };
    if (MODE == 3) {  // range and hit per ray, at the ray's index
        if (in0) {
            const size_t o = pix_base + (size_t)ray0;
            const float a = 1.0f - Tp.x;
            P.depth[o] = a > 0.0f ? dp.x / a : 0.0f;
            if (P.alpha) P.alpha[o] = a;
        }
        if (in1) {
            const size_t o = pix_base + (size_t)ray1;
            const float a = 1.0f - Tp.y;
            P.depth[o] = a > 0.0f ? dp.y / a : 0.0f;
            if (P.alpha) P.alpha[o] = a;
        }
    } else if (MODE == 1) {  // range and hit per ray
        if (in0) {
            const size_t pix = pix_base + (size_t)py0 * W + px;
            const float a = 1.0f - Tp.x;
            P.depth[pix] = a > 0.0f ? dp.x / a : 0.0f;
            if (P.alpha) P.alpha[pix] = a;
        }
        if (in1) {
            const size_t pix = pix_base + (size_t)py1 * W + px;
            const float a = 1.0f - Tp.y;
            P.depth[pix] = a > 0.0f ? dp.y / a : 0.0f;
            if (P.alpha) P.alpha[pix] = a;
        }
    } else if (!SC) {
        if (in0) store(py0, Tp.x, rp.x, gp.x, bp.x, dp.x);
        if (in1) store(py1, Tp.y, rp.y, gp.y, bp.y, dp.y);
    }
    __syncthreads();  // shared staging is reused by the next item
    }  // items of the claim
    if (tid == 0) s_item = atomicAdd(P.work, (unsigned)P.chunk);  // every thread has read the last claim
    __syncthreads();
    }  // claims
}

template <int TW, int TH, bool SC = false, int MODE = 0, bool QUAD = false>
static cudaError_t resident_ctas(int* out) {
    constexpr int NT = TW * TH / 2;
    static int per_sm[64] = {0};  // resident CTAs per SM, per device
    static int sms[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
        int ps = 0, n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_composite<TW, TH, SC, MODE, QUAD>, NT, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sms[dev] = n;
        per_sm[dev] = ps < 1 ? 1 : ps;
    }
    *out = per_sm[dev] * sms[dev];
    return cudaSuccess;
}

template <int TW, int TH, bool SC = false, int MODE = 0, bool QUAD = false>
static cudaError_t launch_tiles(const CompParams& P, cudaStream_t st, int* ctas) {
    constexpr int NT = TW * TH / 2;
    int full = 0;
    cudaError_t e = resident_ctas<TW, TH, SC, MODE, QUAD>(&full);
    if (e != cudaSuccess) return e;
    const unsigned items = P.item_end - P.item_begin;
    unsigned grid = (unsigned)full;
    const unsigned claims = (items + P.chunk - 1) / P.chunk;
    if (grid > claims) grid = claims;
    if (P.spill && grid > P.spill_ctas) grid = P.spill_ctas;
    if (grid == 0) grid = 1;
    *ctas = (int)grid;
    k_composite<TW, TH, SC, MODE, QUAD><<<grid, NT, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_composite(const CompParams& P, cudaStream_t st, int* ctas) {
    *ctas = 0;
    if (P.item_end <= P.item_begin) return cudaSuccess;
    if (P.spill && (P.spill_cap < (unsigned)kCompCap || P.spill_cap > (unsigned)kSpillMax || P.spill_ctas == 0))
        return cudaErrorInvalidValue;
    // LiDAR scans run on 16x16 tiles only; grid scans in the quadrant form (a
    // Gaussian's cone box spans few cells: rotating -3.7 %, solid-state -13 %
    // compositing time on the 2048-env room)
    if (P.lidars) {
        if (P.tile_w != 16 || P.tile_h != 16 || P.score) return cudaErrorInvalidValue;
        if (P.ray_list) return launch_tiles<16, 16, false, 3>(P, st, ctas);
        return launch_tiles<16, 16, false, 1, true>(P, st, ctas);
    }
    if (P.score) {  // the contribution pass runs on 16x16 tiles only
        if (P.tile_w != 16 || P.tile_h != 16) return cudaErrorInvalidValue;
        return launch_tiles<16, 16, true>(P, st, ctas);
    }
    if (P.quad && P.tile_w == 16 && P.tile_h == 16) {  // quadrant lists (16x16 and 8x8 camera tiles)
        if (P.neval) return launch_tiles<16, 16, false, 2, true>(P, st, ctas);
        return launch_tiles<16, 16, false, 0, true>(P, st, ctas);
    }
    if (P.quad && P.tile_w == 8 && P.tile_h == 8) {
        if (P.neval) return launch_tiles<8, 8, false, 2, true>(P, st, ctas);
        return launch_tiles<8, 8, false, 0, true>(P, st, ctas);
    }
    if (P.neval) {  // counting pass
        if (P.tile_w == 16 && P.tile_h == 16) return launch_tiles<16, 16, false, 2>(P, st, ctas);
        if (P.tile_w == 32 && P.tile_h == 16) return launch_tiles<32, 16, false, 2>(P, st, ctas);
        if (P.tile_w == 8 && P.tile_h == 8) return launch_tiles<8, 8, false, 2>(P, st, ctas);
        if (P.tile_w == 16 && P.tile_h == 8) return launch_tiles<16, 8, false, 2>(P, st, ctas);
        return launch_tiles<32, 8, false, 2>(P, st, ctas);
    }
    if (P.tile_w == 16 && P.tile_h == 16) return launch_tiles<16, 16>(P, st, ctas);
    if (P.tile_w == 32 && P.tile_h == 16) return launch_tiles<32, 16>(P, st, ctas);
    if (P.tile_w == 8 && P.tile_h == 8) return launch_tiles<8, 8>(P, st, ctas);
    if (P.tile_w == 16 && P.tile_h == 8) return launch_tiles<16, 8>(P, st, ctas);
    return launch_tiles<32, 8>(P, st, ctas);
}

cudaError_t composite_max_ctas(int tile_w, int tile_h, int* ctas) {
    if (tile_w == 16 && tile_h == 16) {
        int a = 0, b = 0;
        cudaError_t e = resident_ctas<16, 16>(&a);
        if (e == cudaSuccess) e = resident_ctas<16, 16, false, 0, true>(&b);
        *ctas = a > b ? a : b;
        return e;
    }
    if (tile_w == 8 && tile_h == 8) {
        int a = 0, b = 0;
        cudaError_t e = resident_ctas<8, 8>(&a);
        if (e == cudaSuccess) e = resident_ctas<8, 8, false, 0, true>(&b);
        *ctas = a > b ? a : b;
        return e;
    }
    if (tile_w == 32 && tile_h == 16) return resident_ctas<32, 16>(ctas);
    if (tile_w == 8 && tile_h == 8) return resident_ctas<8, 8>(ctas);
    if (tile_w == 16 && tile_h == 8) return resident_ctas<16, 8>(ctas);
    return resident_ctas<32, 8>(ctas);
}

}  // namespace gsb
