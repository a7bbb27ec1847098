// (env, tile) intersection counting, prefix scan and bucketed scatter of
// depth keys (steps A3 and A4).  The renderer of the paper (Sec. III-C
// "Throughput Scaling", built on gsplat) bins projected splats into screen
// tiles before compositing; this file is that binning, designed for many envs.
//
// Each splat's support box [i0,i1]x[j0,j1] (pixels) touches the tiles
// [i0/tw, i1/tw] x [j0/th, j1/th].  Counting and scattering first aggregate in
// a shared-memory histogram per (env, block of Gaussians), so global atomics
// are one per touched tile per block rather than one per intersection.  The
// order inside a bucket is arbitrary; the compositor orders each bucket by the
// unique key (depth bits << 32 | the caller's local index of the Gaussian).
#include "gs_internal.cuh"

namespace gsb {

// Tile widths and heights are powers of two (8, 16 or 32; the API rejects
// other shapes), and box coordinates are non-negative, so the tile of a pixel
// coordinate is a shift of it: sx = log2(tile width), sy = log2(tile height).
__device__ __forceinline__ void tile_span(uint32_t rx, uint32_t ry, int sx, int sy, int& tx0, int& tx1, int& ty0,
                                          int& ty1) {
    tx0 = (int)((rx & 0xffffu) >> sx);
    tx1 = (int)((rx >> 16) >> sx);
    ty0 = (int)((ry & 0xffffu) >> sy);
    ty1 = (int)((ry >> 16) >> sy);
}

// f(t) for every tile t of a record's span: rows ty0..ty1 of the columns
// tx0..tx1 in one flat loop (lanes with spans of different shapes then diverge
// only by their tile counts).  WRAP (LiDAR waves): a box with x0 > x1 covers
// the columns [x0, cols) and [0, x1] (a cone across azimuth 0), so its tile
// columns run tx0..ntx-1 and then 0..tx1.
template <bool WRAP, typename F>
__device__ __forceinline__ void for_span(uint32_t rx, uint32_t ry, int sx, int sy, int ntx, F&& f) {
    int tx0, tx1, ty0, ty1;
    tile_span(rx, ry, sx, sy, tx0, tx1, ty0, ty1);
    if (WRAP && (rx & 0xffffu) > (rx >> 16)) {
        const int nx = min(ntx, ntx - tx0 + tx1 + 1);
        const int n = nx * (ty1 - ty0 + 1);
        int tx = tx0, row = ty0 * ntx, c = 0;
        for (int k = 0; k < n; ++k) {
            f(row + tx);
            if (++c == nx) {
                c = 0;
                tx = tx0;
                row += ntx;
            } else if (++tx == ntx) {
                tx = 0;
            }
        }
        return;
    }
    const int n = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    int tx = tx0, t = ty0 * ntx + tx0;
    for (int k = 0; k < n; ++k) {
        f(t);
        if (tx == tx1) {
            tx = tx0;
            t += ntx - (tx1 - tx0);
        } else {
            ++tx;
            ++t;
        }
    }
}

// The visible record slots of mask words [w0, w1) of one env, one word per
// thread (w1 - w0 <= blockDim.x), listed block-wide in slot order in lst (at
// most 32 (w1 - w0) entries, slots relative to 32 w0); returns their number.
// One list per block spreads the visible records evenly over its warps,
// however unevenly visibility clusters in the storage order, and the scatter
// walks the same list in both of its passes.  wtot: one u32 per warp.
__device__ __forceinline__ int block_visible(const uint32_t* mask, int64_t w0, int64_t w1, uint16_t* lst,
                                             uint32_t* wtot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t w = w0 + threadIdx.x;
    uint32_t m = w < w1 ? __ldg(mask + w) : 0u;
    const uint32_t c = __popc(m);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int i = 0; i < nw; ++i) {
        const uint32_t t = wtot[i];
        if (i < warp) before += t;
        total += t;
    }
    uint32_t pos = before + incl - c;
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1u;
        lst[pos++] = (uint16_t)(threadIdx.x * 32 + bit);
    }
    __syncthreads();
    return (int)total;
}

// Rebuilds a block's tile histogram of env el's visible records (the block's
// list from block_visible, records 32 w0 + lst[i]) in hist[0, T).  Neighbouring
// threads take neighbouring records of the list.
// With RANGE, also the smallest and largest depth bits (r3.z) of the records
// this thread visits, into zl and zh.
template <bool WRAP, bool RANGE = false>
__device__ __forceinline__ void block_histogram(const BinParams& P, const EnvInfo& E, int64_t w0, const uint16_t* lst,
                                                int nvis, uint32_t* hist, uint32_t* zl = nullptr,
                                                uint32_t* zh = nullptr) {
    const uint4* r3 = P.r3 + E.rec_base;
    const int sx = __ffs(P.tile_w) - 1, sy = __ffs(P.tile_h) - 1;
    for (int i = threadIdx.x; i < nvis; i += blockDim.x) {
        const uint4 q = r3[w0 * 32 + lst[i]];
        if constexpr (RANGE) {
            *zl = min(*zl, q.z);
            *zh = max(*zh, q.z);
        }
        for_span<WRAP>(q.x, q.y, sx, sy, E.ntx, [&](int t) { atomicAdd(&hist[t], 1u); });
    }
}

// grid: (blocks over the largest env's visibility words, envs); block 256;
// dynamic smem: max T u32.  Blocks past their env's words exit at once.
template <bool WRAP>
__global__ void __launch_bounds__(256) k_count(BinParams P) {
    extern __shared__ uint32_t hist[];
    __shared__ uint16_t wbuf[32 * kWordsPerBlock];
    __shared__ uint32_t wtot[32];
    const int el = P.e_begin + blockIdx.y;
    const EnvInfo E = P.envs[el];
    const int64_t words = (E.n_local + 31) / 32;
    const int64_t w0 = (int64_t)blockIdx.x * P.words_per_block;
    if (w0 >= words) return;
    const int64_t w1 = min(w0 + (int64_t)P.words_per_block, words);
    for (int t = threadIdx.x; t < E.T; t += blockDim.x) hist[t] = 0;
    const int nvis = block_visible(P.mask + E.mask_base, w0, w1, wbuf, wtot);
    uint32_t zl = 0xffffffffu, zh = 0u;
    block_histogram<WRAP, true>(P, E, w0, wbuf, nvis, hist, &zl, &zh);
    if (P.zr) {  // the env's depth-bit range: one atomic pair per warp
        zl = __reduce_min_sync(0xffffffffu, zl);
        zh = __reduce_max_sync(0xffffffffu, zh);
        if ((threadIdx.x & 31) == 0 && zl <= zh) {
            atomicMin(&P.zr[el].x, zl);
            atomicMin(&P.zr[el].y, ~zh);
        }
    }
    __syncthreads();
    uint32_t* cnt = P.counts + E.tile_base;
    for (int t = threadIdx.x; t < E.T; t += blockDim.x) {
        const uint32_t h = hist[t];
        if (h) atomicAdd(cnt + t, h);
    }
}

static cudaError_t opt_in_smem(const void* fn, size_t smem) {
    if (smem <= 16 * 1024) return cudaSuccess;  // plus 16 KB of static shared memory
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static_assert(kWordsPerBlock <= 256, "binning blocks: one visibility word per thread of 256");

cudaError_t launch_count(const BinParams& P, int n_envs, int max_words, int max_T, cudaStream_t st) {
    if (n_envs == 0 || max_words == 0) return cudaSuccess;
    const size_t smem = (size_t)max_T * 4;
    const void* fn = P.wrap ? (const void*)k_count<true> : (const void*)k_count<false>;
    cudaError_t e = opt_in_smem(fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((max_words + P.words_per_block - 1) / P.words_per_block), (unsigned)n_envs);
    if (P.wrap) k_count<true><<<grid, 256, smem, st>>>(P);
    else k_count<false><<<grid, 256, smem, st>>>(P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scan

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T& block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    const T before = warp == 0 ? T(0) : warp_tot[warp - 1];
    block_total = warp_tot[nw - 1];
    __syncthreads();
    return before + x - v;
}

// per env: off_local[t] = sum_{t' < t} counts[t'], env_total = sum
__global__ void __launch_bounds__(1024) k_scan_env(const EnvInfo* envs, const uint32_t* counts, uint32_t* off_local,
                                                   unsigned long long* env_total) {
    __shared__ uint32_t wt[32];
    const int el = blockIdx.x;
    const int T = envs[el].T;
    const uint32_t* c = counts + envs[el].tile_base;
    uint32_t* o = off_local + envs[el].tile_base;
    uint32_t carry = 0;
    for (int base = 0; base < T; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const uint32_t v = t < T ? c[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(v, wt, tot);
        if (t < T) o[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) env_total[el] = carry;
}

// env_base[e] = sum_{e' < e} env_total[e'], env_base[We] = total
__global__ void __launch_bounds__(1024) k_scan_base(const unsigned long long* env_total, unsigned long long* env_base,
                                                    int We) {
    __shared__ unsigned long long wt[32];
    unsigned long long carry = 0;
    for (int base = 0; base < We; base += blockDim.x) {
        const int e = base + threadIdx.x;
        const unsigned long long v = e < We ? env_total[e] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan<unsigned long long>(v, wt, tot);
        if (e < We) env_base[e] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) env_base[We] = carry;
}

cudaError_t launch_scan(const EnvInfo* envs, const uint32_t* counts, uint32_t* off_local,
                        unsigned long long* env_total, unsigned long long* env_base, int We, cudaStream_t st) {
    if (We == 0) return cudaSuccess;
    k_scan_env<<<We, 1024, 0, st>>>(envs, counts, off_local, env_total);
    k_scan_base<<<1, 1024, 0, st>>>(env_total, env_base, We);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scatter
// Same partition and visiting order as k_count.  Pass 1 rebuilds the block's
// histogram, then one global atomic per touched tile reserves the block's range
// of that bucket; pass 2 writes each key at (bucket start + block range +
// shared cursor).  A key past the pair buffer's capacity (possible only for a
// launch planned with a fixed capacity) is dropped and flagged.

template <bool WRAP>
__global__ void __launch_bounds__(256, 6) k_scatter(BinParams P) {  // <= 42 registers: 6 CTAs/SM
    extern __shared__ uint32_t sm[];
    __shared__ uint16_t wbuf[32 * kWordsPerBlock];
    __shared__ uint32_t wtot[32];
    const int el = P.e_begin + blockIdx.y;
    const EnvInfo E = P.envs[el];
    const int64_t words = (E.n_local + 31) / 32;
    const int64_t w0 = (int64_t)blockIdx.x * P.words_per_block;
    if (w0 >= words) return;
    const int64_t w1 = min(w0 + (int64_t)P.words_per_block, words);
    uint32_t* hist = sm;
    uint32_t* base = sm + E.T;
    for (int t = threadIdx.x; t < E.T; t += blockDim.x) hist[t] = 0;
    const int nvis = block_visible(P.mask + E.mask_base, w0, w1, wbuf, wtot);
    block_histogram<WRAP>(P, E, w0, wbuf, nvis, hist);
    __syncthreads();
    uint32_t* cur = P.cursor + E.tile_base;
    const uint32_t* off = P.off_local + E.tile_base;
    const unsigned long long eb = P.env_base[el] - P.pair_base;
    for (int t = threadIdx.x; t < E.T; t += blockDim.x) {
        const uint32_t h = hist[t];
        if (h) base[t] = off[t] + atomicAdd(cur + t, h);
        hist[t] = 0;
    }
    __syncthreads();
    const uint4* r3 = P.r3 + E.rec_base;
    const int sx = __ffs(P.tile_w) - 1, sy = __ffs(P.tile_h) - 1;
    bool dropped = false;
    for (int iv = threadIdx.x; iv < nvis; iv += blockDim.x) {
        const int64_t j = w0 * 32 + wbuf[iv];
        const uint4 q = r3[j];
        const uint32_t i = P.index_in_r3 ? q.w
                           : ((P.bg_index && j < (int64_t)P.n_bg) ? (uint32_t)__ldg(P.bg_index + j) : (uint32_t)j);
        const unsigned long long key = ((unsigned long long)q.z << 32) | (unsigned long long)i;
        for_span<WRAP>(q.x, q.y, sx, sy, E.ntx, [&](int t) {
            const uint32_t k = atomicAdd(&hist[t], 1u);
            const unsigned long long pos = eb + base[t] + k;
            if (pos < P.pair_cap) P.pairs[pos] = key;
            else dropped = true;
        });
    }
    if (__syncthreads_or(dropped) && threadIdx.x == 0) atomicOr(P.status, kStOverflow);
}

cudaError_t launch_scatter(const BinParams& P, int n_envs, int max_words, int max_T, cudaStream_t st) {
    if (n_envs == 0 || max_words == 0) return cudaSuccess;
    size_t smem = (size_t)max_T * 8;
    // Large images (at least half a 640x480 frame per env): at most 4 CTAs per
    // SM, by padding the shared memory (29 KB dynamic + 16 KB static + the
    // per-CTA reserve: 5 no longer fit).  Measured on the 2048-env room
    // workload at 640x480: 6 CTAs/SM (what 40 registers allow) 20.7 ms, 5: 19.9,
    // 4: 18.7, 3: 18.6 ms per step; at 320x240 and 128x128 six are fastest
    // (6.8 vs 8.0 ms and 5.1 vs 6.2 ms with 4).
    if ((long long)max_T * P.tile_w * P.tile_h >= 640ll * 480 / 2 && smem < (size_t)29 * 1024) smem = 29 * 1024;
    const void* fn = P.wrap ? (const void*)k_scatter<true> : (const void*)k_scatter<false>;
    cudaError_t e = opt_in_smem(fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((max_words + P.words_per_block - 1) / P.words_per_block), (unsigned)n_envs);
    if (P.wrap) k_scatter<true><<<grid, 256, smem, st>>>(P);
    else k_scatter<false><<<grid, 256, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace gsb
