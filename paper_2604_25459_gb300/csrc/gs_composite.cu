// Per-tile front-to-back alpha compositing with early termination (step A5).
//
// The 3DGS forward pass (paper Sec. II-B; the batch renderer of Sec. III-C
// "Throughput Scaling" is built on it) blends, per pixel, the splats whose
// alpha = min(0.99, o exp(-q/2)) reaches 1/255, in depth order, until the
// transmittance would drop below 1e-4; Sec. III-A asks for RGB and depth.
//
// One CTA renders one (env, tile); each warp owns an 8x4 pixel subtile.
// The tile's bucket of keys (depth bits << 32 | global index) is consumed in
// depth windows of at most kCompCap keys: a window is chosen by a radix
// histogram over the bucket (so the long buckets of dense robot tiles are
// never sorted past the point where every pixel has terminated), gathered into
// shared memory, bitonic-sorted, and composited in batches whose records are
// staged in shared memory.  Warps test 32 splats at a time against their
// subtile with one ballot and then evaluate only the overlapping ones.
#include "gs_internal.cuh"

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
__device__ __forceinline__ void bitonic_sort(unsigned long long* keys, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += NT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH) k_composite(CompParams P) {
    constexpr int NT = TW * TH;
    constexpr int CAP = kCompCap;
    __shared__ unsigned long long keys[CAP];
    __shared__ float4 s0[NT];
    __shared__ float4 s1[NT];
    __shared__ float4 s2[NT];
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long red[NT / 32];
    __shared__ unsigned long long sel_lo, sel_hi, sel_khi;
    __shared__ uint32_t sel_wn, sel_cnt;
    __shared__ int sel_state;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int el = P.e_begin + blockIdx.y;
    const int t = blockIdx.x;
    const int tx = t % P.ntx, ty = t / P.ntx;
    constexpr int SWX = TW / 8;
    const int wx0 = tx * TW + (warp % SWX) * 8, wy0 = ty * TH + (warp / SWX) * 4;
    const int wx1 = wx0 + 7, wy1 = wy0 + 3;
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool inside = px < P.W && py < P.H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    bool done = !inside;
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, dz = 0.0f;
    uint32_t ncomp = 0;

    const uint32_t n = P.counts[(size_t)el * P.T + t];
    const unsigned long long start = P.env_base[el] - P.pair_base + P.off_local[(size_t)el * P.T + t];
    const unsigned long long* Lk = P.pairs + start;
    const size_t recbase = (size_t)el * P.G;
    const bool dbg = P.dbg_sorted != nullptr;
    constexpr float kA = -0.72134752044448170f;  // -0.5 log2(e)
    constexpr float kB = -1.44269504088896341f;  // -log2(e)

    unsigned long long kmax = 0;
    if (n > (uint32_t)CAP) {
        unsigned long long m = 0;
        for (uint32_t i = tid; i < n; i += NT) {
            const unsigned long long k = Lk[i];
            m = k > m ? k : m;
        }
        kmax = block_max_u64<NT>(m, red);
    }

    unsigned long long klo = 0;
    uint32_t processed = 0;
    bool finished = false;
    while (processed < n && !finished) {
        uint32_t wn;
        unsigned long long khi;
        if (n - processed <= (uint32_t)CAP) {
            wn = n - processed;
            khi = ~0ull;
        } else {
            // radix-select a window [klo, khi) of at most CAP keys
            if (tid == 0) {
                sel_lo = klo;
                sel_hi = kmax;
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
                for (uint32_t i = tid; i < n; i += NT) {
                    const unsigned long long k = Lk[i];
                    if (k >= lo && k <= hi) atomicAdd(&hist[(k >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    const unsigned long long pre = (shift + 8 >= 64) ? 0ull : (lo >> (shift + 8)) << (shift + 8);
                    int d0 = 0;
                    while (d0 < 255 && hist[d0] == 0) ++d0;
                    if (hist[d0] > (uint32_t)CAP) {
                        const unsigned long long blo = pre | ((unsigned long long)d0 << shift);
                        const unsigned long long bhi = blo | ((1ull << shift) - 1ull);
                        sel_lo = blo > lo ? blo : lo;
                        sel_hi = bhi < hi ? bhi : hi;
                    } else {
                        uint32_t cum = 0;
                        int d = d0;
                        while (d < 256 && cum + hist[d] <= (uint32_t)CAP) {
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
            // keys are unique, so eight 8-bit levels always isolate a window; anything
            // else means a corrupted bucket: flag it and stop instead of spinning
            khi = sel_state ? sel_khi : klo;
            wn = sel_state ? sel_wn : 0u;
        }
        if (wn == 0) {
            if (tid == 0) atomicOr(P.status, kStOverflow);
            break;
        }
        // gather the window into shared memory
        if (processed == 0 && n <= (uint32_t)CAP) {
            for (uint32_t i = tid; i < n; i += NT) keys[i] = Lk[i];
        } else {
            if (tid == 0) sel_cnt = 0;
            __syncthreads();
            for (uint32_t i = tid; i < n; i += NT) {
                const unsigned long long k = Lk[i];
                if (k >= klo && k < khi) {
                    const uint32_t slot = atomicAdd(&sel_cnt, 1u);
                    if (slot < (uint32_t)CAP) keys[slot] = k;
                }
            }
        }
        int n2 = 1;
        while (n2 < (int)wn) n2 <<= 1;
        for (int i = (int)wn + tid; i < n2; i += NT) keys[i] = ~0ull;
        __syncthreads();
        bitonic_sort<NT>(keys, n2);
        if (dbg)
            for (uint32_t i = tid; i < wn; i += NT) P.dbg_sorted[start + processed + i] = keys[i];

        for (uint32_t b = 0; b < wn; b += NT) {
            const int cnt = (int)min((uint32_t)NT, wn - b);
            if (tid < cnt) {
                const uint32_t g = (uint32_t)(keys[b + tid] & 0xffffffffull);
                if (g < (uint64_t)P.G) {
                    const size_t ri = recbase + g;
                    const float4 q0 = P.r0[ri];
                    const float4 q1 = P.r1[ri];
                    const float4 q2 = P.r2[ri];
                    s0[tid] = q0;
                    s1[tid] = make_float4(q1.x * kA, q1.y * kB, q1.z * kA, q1.w);
                    s2[tid] = q2;
                } else {  // never happens for a well-formed bucket; stage an empty range
                    s0[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                    s1[tid] = make_float4(0.f, 0.f, 0.f, __uint_as_float(1u));
                    s2[tid] = make_float4(0.f, 0.f, 0.f, __uint_as_float(1u));
                    atomicOr(P.status, kStOverflow);
                }
            }
            __syncthreads();
            if (!__all_sync(0xffffffffu, done)) {
                for (int c = 0; c < cnt; c += 32) {
                    const int j = c + lane;
                    bool ov = false;
                    if (j < cnt) {
                        const uint32_t rx = __float_as_uint(s1[j].w), ry = __float_as_uint(s2[j].w);
                        ov = (int)(rx & 0xffffu) <= wx1 && (int)(rx >> 16) >= wx0 && (int)(ry & 0xffffu) <= wy1 &&
                             (int)(ry >> 16) >= wy0;
                    }
                    uint32_t m = __ballot_sync(0xffffffffu, ov);
                    while (m) {
                        const int k = __ffs(m) - 1;
                        m &= m - 1u;
                        const int jj = c + k;
                        const float4 A = s0[jj];
                        const float4 B = s1[jj];
                        const uint32_t rx = __float_as_uint(B.w);
                        const float4 Cc = s2[jj];
                        const uint32_t ry = __float_as_uint(Cc.w);
                        if (!done && px >= (int)(rx & 0xffffu) && px <= (int)(rx >> 16) && py >= (int)(ry & 0xffffu) &&
                            py <= (int)(ry >> 16)) {
                            const float dx = fpx - A.x, dy = fpy - A.y;
                            const float pw = B.x * dx * dx + B.y * dx * dy + B.z * dy * dy;
                            const float al = fminf(0.99f, A.z * ex2_approx(pw));
                            if (al >= (1.0f / 255.0f)) {
                                ++ncomp;
                                const float Tn = T * (1.0f - al);
                                if (Tn < 1e-4f) {
                                    done = true;
                                } else {
                                    const float w = al * T;
                                    cr += w * Cc.x;
                                    cg += w * Cc.y;
                                    cb += w * Cc.z;
                                    dz += w * A.w;
                                    T = Tn;
                                }
                            }
                        }
                    }
                    if (__all_sync(0xffffffffu, done)) break;
                }
            }
            const bool all = __syncthreads_and(done) != 0;
            if (all && !dbg) {
                finished = true;
                break;
            }
        }
        processed += wn;
        klo = khi;
    }

    if (P.neval) {
        uint32_t c = ncomp;
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0 && c) atomicAdd(P.neval, (unsigned long long)c);
    }
    if (inside) {
        const size_t pix = ((size_t)el * P.H + py) * P.W + px;
        P.rgb[3 * pix] = fminf(fmaxf(cr, 0.0f), 1.0f);
        P.rgb[3 * pix + 1] = fminf(fmaxf(cg, 0.0f), 1.0f);
        P.rgb[3 * pix + 2] = fminf(fmaxf(cb, 0.0f), 1.0f);
        const float a = 1.0f - T;
        P.depth[pix] = a > 0.0f ? dz / a : 0.0f;
        if (P.alpha) P.alpha[pix] = a;
    }
}

cudaError_t launch_composite(const CompParams& P, int n_envs, cudaStream_t st) {
    if (n_envs == 0) return cudaSuccess;
    dim3 grid((unsigned)P.T, (unsigned)n_envs);
    if (P.tile_w == 16 && P.tile_h == 16)
        k_composite<16, 16><<<grid, 256, 0, st>>>(P);
    else if (P.tile_w == 8 && P.tile_h == 8)
        k_composite<8, 8><<<grid, 64, 0, st>>>(P);
    else if (P.tile_w == 16 && P.tile_h == 8)
        k_composite<16, 8><<<grid, 128, 0, st>>>(P);
    else
        k_composite<32, 8><<<grid, 256, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace gsb
