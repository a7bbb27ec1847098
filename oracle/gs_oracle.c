/* CPU oracle for batched 3DGS RGB-D rendering -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke entry point and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or constant with the CUDA
 * path: it is a plain, slow restatement of what the renderer computes.
 *
 * Two instantiations of the projection + compositing oracle (see
 * gs_oracle_impl.inc for the step-by-step definition and its sources in the
 * paper): *_f64 in double (the reference for parity) and *_f32 in float (for
 * the precision pin: double and float oracles agree on tiny scenes).
 *
 * or_bin is the binning oracle: given a renderer's projected keys (u, v, hx,
 * hy, float32 depth bits, global index) it recomputes, in float32 with the
 * pixel-range formula below, the (tile) intersection counts and the per-tile
 * lists in (depth bits, global index) order, for bit-exact comparison.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REAL double
#define FN(name) name##_f64
#include "gs_oracle_impl.inc"
#undef REAL
#undef FN

#define REAL float
#define FN(name) name##_f32
#include "gs_oracle_impl.inc"
#undef REAL
#undef FN

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Pixel range of a support box in float32:
 *   i0 = max(0, ceil((u - hx) - 0.5)), i1 = min(W-1, floor((u + hx) - 0.5)),
 * evaluated left to right; returns 0 when the range is empty. */
static int px_range(float u, float h, int W, int* lo, int* hi)
{
    float a = ceilf(u - h - 0.5f);
    float b = floorf(u + h - 0.5f);
    if (!(a <= b)) return 0;
    if (a < 0.0f) a = 0.0f;
    if (b > (float)(W - 1)) b = (float)(W - 1);
    if (a > b) return 0;
    *lo = (int)a;
    *hi = (int)b;
    return 1;
}

typedef struct {
    uint32_t z;
    uint32_t g;
} zkey_t;

static int cmp_zkey(const void* a, const void* b)
{
    const zkey_t* x = (const zkey_t*)a;
    const zkey_t* y = (const zkey_t*)b;
    if (x->z != y->z) return x->z < y->z ? -1 : 1;
    return (x->g > y->g) - (x->g < y->g);
}

/* counts[tiles] (tiles = ceil(W/tw) * ceil(H/th), row-major); when lists is
 * non-NULL it receives, per tile in order, the global indices sorted by
 * (zbits, gidx), at offsets given by the exclusive scan of counts.
 * Returns the total number of (record, tile) intersections. */
int64_t or_bin(int64_t n, const float* u, const float* v, const float* hx, const float* hy, const uint32_t* zbits,
               const uint32_t* gidx, int W, int H, int tw, int th, int64_t* counts, uint32_t* lists)
{
    int ntx = (W + tw - 1) / tw, nty = (H + th - 1) / th;
    int64_t ntiles = (int64_t)ntx * nty;
    memset(counts, 0, sizeof(int64_t) * (size_t)ntiles);
    for (int64_t r = 0; r < n; ++r) {
        int i0, i1, j0, j1;
        if (!px_range(u[r], hx[r], W, &i0, &i1) || !px_range(v[r], hy[r], H, &j0, &j1)) continue;
        for (int ty = j0 / th; ty <= j1 / th; ++ty)
            for (int tx = i0 / tw; tx <= i1 / tw; ++tx) counts[(int64_t)ty * ntx + tx]++;
    }
    int64_t total = 0;
    for (int64_t t = 0; t < ntiles; ++t) total += counts[t];
    if (!lists) return total;
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntiles + 1));
    off[0] = 0;
    for (int64_t t = 0; t < ntiles; ++t) off[t + 1] = off[t] + counts[t];
    zkey_t* tmp = (zkey_t*)malloc(sizeof(zkey_t) * (size_t)(total > 0 ? total : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntiles + 1));
    memcpy(fill, off, sizeof(int64_t) * (size_t)ntiles);
    for (int64_t r = 0; r < n; ++r) {
        int i0, i1, j0, j1;
        if (!px_range(u[r], hx[r], W, &i0, &i1) || !px_range(v[r], hy[r], H, &j0, &j1)) continue;
        for (int ty = j0 / th; ty <= j1 / th; ++ty)
            for (int tx = i0 / tw; tx <= i1 / tw; ++tx) {
                int64_t t = (int64_t)ty * ntx + tx;
                tmp[fill[t]].z = zbits[r];
                tmp[fill[t]].g = gidx[r];
                fill[t]++;
            }
    }
    for (int64_t t = 0; t < ntiles; ++t) {
        qsort(tmp + off[t], (size_t)counts[t], sizeof(zkey_t), cmp_zkey);
        for (int64_t k = off[t]; k < off[t + 1]; ++k) lists[k] = tmp[k].g;
    }
    free(fill);
    free(tmp);
    free(off);
    return total;
}
