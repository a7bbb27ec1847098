// Scene preparation, link composition (RLGK) and EWA projection + SH colour.
//
// Paper: Sec. III-C "RLGK" binds Gaussian clusters to rigid links (step A1
// here composes each link pose with the env's camera); Sec. II-B cites the 3DGS
// forward pass that the batch renderer of Sec. III-C "Throughput Scaling"
// builds on (step A2: projection of every (env, Gaussian) to a 2D conic with
// view-dependent SH colour).
#include "gs_internal.cuh"

namespace gsb {

// ------------------------------------------------------------------ helpers

template <int DT>
__device__ __forceinline__ float load_val(const void* p, int64_t i) {
    if constexpr (DT == GS_F32) {
        return static_cast<const float*>(p)[i];
    } else if constexpr (DT == GS_BF16) {
        return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    } else {
        return __half2float(static_cast<const __half*>(p)[i]);
    }
}

// Rotation matrix (row-major) of the normalised quaternion (w,x,y,z).
template <typename T>
__device__ __forceinline__ bool quat_rot(T w, T x, T y, T z, T* R) {
    T nn = w * w + x * x + y * y + z * z;
    if (!(nn > T(0)) || !isfinite(nn)) {
        R[0] = 1; R[1] = 0; R[2] = 0; R[3] = 0; R[4] = 1; R[5] = 0; R[6] = 0; R[7] = 0; R[8] = 1;
        return false;
    }
    T inv = T(1) / sqrt(nn);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    return true;
}

// ------------------------------------------------------------------ scene preparation
// Once per Gaussian: the factor F = R diag(exp(s)) of the 3DGS covariance
// Sigma = F F^T (FP32), trace(Sigma), the support
// threshold q* = 2 ln(255 o) and the link the Gaussian rides on.

struct PrepArgs {
    const float* mean;
    const float* quat;
    const void* log_scale;
    const void* opacity;
    const void* sh;
    int64_t n;
    int64_t dst;          // first destination index
    const int64_t* place;  // nullable: input i goes to dst + place[i] (the scene's storage order)
    int link_mode;        // 0: background (link 0), 1: binary search in link_offsets
    const int64_t* link_offsets;
    int n_links;
    int64_t n_total;
    float4* p0;
    float4* p1;
    float4* p2;
    float4* p3;
    void* shp;
    int sh_values;
    int sh_planes;
    uint32_t* status;
};

template <int DT>
__global__ void k_prep(PrepArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int64_t g = A.dst + (A.place ? A.place[i] : i);
    float R[9];
    bool ok = quat_rot<float>(A.quat[4 * i], A.quat[4 * i + 1], A.quat[4 * i + 2], A.quat[4 * i + 3], R);
    float sc[3];
    for (int k = 0; k < 3; ++k) sc[k] = expf(load_val<DT>(A.log_scale, 3 * i + k));
    float F[9];  // F = R diag(exp(s)), covariance F F^T
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) F[3 * r + c] = R[3 * r + c] * sc[c];
    const float tr = sc[0] * sc[0] + sc[1] * sc[1] + sc[2] * sc[2];
    const float o = load_val<DT>(A.opacity, i);
    float qstar = -1.0f;
    if (o >= 1.0f / 255.0f && isfinite(o)) qstar = 2.0f * logf(255.0f * o);
    if (!ok || !isfinite(tr)) {
        atomicOr(A.status, kStBadScene);
        qstar = -1.0f;
    }
    int link = 0;
    if (A.link_mode) {
        int lo = 0, hi = A.n_links - 1;
        while (lo < hi) {  // last l with link_offsets[l] <= i
            int mid = (lo + hi + 1) >> 1;
            if (A.link_offsets[mid] <= i) lo = mid; else hi = mid - 1;
        }
        link = lo + 1;
    }
    A.p0[g] = make_float4(A.mean[3 * i], A.mean[3 * i + 1], A.mean[3 * i + 2], o);
    A.p1[g] = make_float4(F[0], F[1], F[2], F[3]);
    A.p2[g] = make_float4(F[4], F[5], F[6], F[7]);
    A.p3[g] = make_float4(F[8], qstar, tr, __int_as_float(link));
    if constexpr (DT == GS_F32) {
        float* dst = static_cast<float*>(A.shp);
        for (int p = 0; p < A.sh_planes; ++p)
            for (int c = 0; c < 4; ++c) {
                const int f = 4 * p + c;
                dst[((size_t)p * A.n_total + g) * 4 + c] =
                    f < A.sh_values ? static_cast<const float*>(A.sh)[i * A.sh_values + f] : 0.0f;
            }
    } else {
        uint16_t* dst = static_cast<uint16_t*>(A.shp);
        const uint16_t* src = static_cast<const uint16_t*>(A.sh);
        for (int p = 0; p < A.sh_planes; ++p)
            for (int c = 0; c < 8; ++c) {
                const int f = 8 * p + c;
                dst[((size_t)p * A.n_total + g) * 8 + c] = f < A.sh_values ? src[i * A.sh_values + f] : (uint16_t)0;
            }
    }
}

cudaError_t launch_prep(const float* mean, const float* quat, const void* log_scale, const void* opacity,
                        const void* sh, int64_t n, int64_t dst_offset, const int64_t* place, int link_mode,
                        const int64_t* link_offsets, int n_links, const DevGaussians& D, uint32_t* status,
                        cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    PrepArgs A{mean, quat, log_scale, opacity, sh, n, dst_offset, place, link_mode, link_offsets, n_links, D.n,
               D.p0, D.p1, D.p2, D.p3, D.sh, sh_values(D.sh_degree), D.sh_planes, status};
    dim3 grid((unsigned)((n + 255) / 256));
    switch (D.dtype) {
        case GS_F32: k_prep<GS_F32><<<grid, 256, 0, st>>>(A); break;
        case GS_BF16: k_prep<GS_BF16><<<grid, 256, 0, st>>>(A); break;
        default: k_prep<GS_F16><<<grid, 256, 0, st>>>(A); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ A1: link composition (RLGK)
// For env e and frame f (f = 0: background/world, f = 1 + l - link_begin: link l):
//   M = [R_c R_l | R_c t_l + t_c]  (camera <- link), o = -M_R^T M_t (camera
//   centre in the link frame, so that normalize(mu - o) is the view direction
//   rotated into the link frame).

__global__ void k_link_table(const float* poses, const gs_camera* cams, const EnvInfo* envs, int We, int n_items,
                             LinkXf* out, uint32_t* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_items) return;
    int lo = 0, hi = We - 1;  // env: last e with envs[e].xf_base <= idx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (envs[mid].xf_base <= idx) lo = mid; else hi = mid - 1;
    }
    const int e = lo, f = idx - envs[e].xf_base;
    const gs_camera& c = cams[e];
    float Rc[9];
    quat_rot<float>(c.q_cw[0], c.q_cw[1], c.q_cw[2], c.q_cw[3], Rc);
    const float tc[3] = {c.t_cw[0], c.t_cw[1], c.t_cw[2]};
    float M[9], t[3];
    if (f == 0) {
        for (int k = 0; k < 9; ++k) M[k] = Rc[k];
        for (int k = 0; k < 3; ++k) t[k] = tc[k];
    } else {
        const float* P = poses + (size_t)(envs[e].pose_base + (f - 1)) * 7;
        float Rl[9];
        bool ok = quat_rot<float>(P[0], P[1], P[2], P[3], Rl);
        float tl[3] = {P[4], P[5], P[6]};
        if (!ok || !isfinite(tl[0] + tl[1] + tl[2])) {
            atomicOr(status, kStBadPose);
            tl[0] = tl[1] = tl[2] = 0.0f;
        }
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j)
                M[3 * i + j] = Rc[3 * i] * Rl[j] + Rc[3 * i + 1] * Rl[3 + j] + Rc[3 * i + 2] * Rl[6 + j];
            t[i] = Rc[3 * i] * tl[0] + Rc[3 * i + 1] * tl[1] + Rc[3 * i + 2] * tl[2] + tc[i];
        }
    }
    float o[3];
    for (int j = 0; j < 3; ++j) o[j] = -(M[j] * t[0] + M[3 + j] * t[1] + M[6 + j] * t[2]);
    LinkXf X;
    X.r0 = make_float4(M[0], M[1], M[2], t[0]);
    X.r1 = make_float4(M[3], M[4], M[5], t[1]);
    X.r2 = make_float4(M[6], M[7], M[8], t[2]);
    X.o = make_float4(o[0], o[1], o[2], 0.0f);
    out[idx] = X;
}

cudaError_t launch_link_table(const float* poses, const gs_camera* cams, const EnvInfo* envs, int We, int n_items,
                              LinkXf* out, uint32_t* status, cudaStream_t st) {
    if (n_items == 0 || We == 0) return cudaSuccess;
    k_link_table<<<(n_items + 127) / 128, 128, 0, st>>>(poses, cams, envs, We, n_items, out, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ A2: projection

// 2D covariance of one Gaussian before the 0.3 px^2 low-pass, in factored
// form: M = J W F (2x3) with W the rotation part of X, J the EWA Jacobian at
// the guard-band-clamped centre and F the Gaussian's covariance factor, so
// Sigma_2 = M M^T.  Returns A = |m0|^2, B = m0.m1, C = |m1|^2 and
// K = |m0 x m1|^2 = AC - B^2 (Lagrange's identity): computed as a cross
// product, K carries no cancellation from A, B and C themselves.
template <typename T>
__device__ __forceinline__ void ewa_factor(const LinkXf& X, const float4& a0, const float4& a1, const float4& a2,
                                           const float4& a3, float fx, float fy, float limxn, float limxp,
                                           float limyn, float limyp, T& A, T& B, T& C, T& K) {
    const T mx = (T)X.r0.x * a0.x + (T)X.r0.y * a0.y + (T)X.r0.z * a0.z + (T)X.r0.w;
    const T my = (T)X.r1.x * a0.x + (T)X.r1.y * a0.y + (T)X.r1.z * a0.z + (T)X.r1.w;
    const T mz = (T)X.r2.x * a0.x + (T)X.r2.y * a0.y + (T)X.r2.z * a0.z + (T)X.r2.w;
    const T iz = T(1) / mz;
    T tx = mx * iz, ty = my * iz;
    tx = tx < -(T)limxn ? -(T)limxn : (tx > (T)limxp ? (T)limxp : tx);
    ty = ty < -(T)limyn ? -(T)limyn : (ty > (T)limyp ? (T)limyp : ty);
    const T j00 = (T)fx * iz, j02 = -(T)fx * tx * iz;
    const T j11 = (T)fy * iz, j12 = -(T)fy * ty * iz;
    const T w0x = j00 * X.r0.x + j02 * X.r2.x, w0y = j00 * X.r0.y + j02 * X.r2.y, w0z = j00 * X.r0.z + j02 * X.r2.z;
    const T w1x = j11 * X.r1.x + j12 * X.r2.x, w1y = j11 * X.r1.y + j12 * X.r2.y, w1z = j11 * X.r1.z + j12 * X.r2.z;
    // F row-major: (F00 F01 F02 | F10 F11 F12 | F20 F21 F22)
    const T f00 = a1.x, f01 = a1.y, f02 = a1.z, f10 = a1.w, f11 = a2.x, f12 = a2.y, f20 = a2.z, f21 = a2.w,
            f22 = a3.x;
    const T m0x = w0x * f00 + w0y * f10 + w0z * f20;
    const T m0y = w0x * f01 + w0y * f11 + w0z * f21;
    const T m0z = w0x * f02 + w0y * f12 + w0z * f22;
    const T m1x = w1x * f00 + w1y * f10 + w1z * f20;
    const T m1y = w1x * f01 + w1y * f11 + w1z * f21;
    const T m1z = w1x * f02 + w1y * f12 + w1z * f22;
    A = m0x * m0x + m0y * m0y + m0z * m0z;
    B = m0x * m1x + m0y * m1y + m0z * m1z;
    C = m1x * m1x + m1y * m1y + m1z * m1z;
    const T kx = m0y * m1z - m0z * m1y, ky = m0z * m1x - m0x * m1z, kz = m0x * m1y - m0y * m1x;
    K = kx * kx + ky * ky + kz * kz;
}

// Near-degenerate 2D covariance (a thin Gaussian seen edge-on): the factor,
// its products and the scaled conic factor in FP64.  Kept out of line so the
// common FP32 path does not carry its registers.
__device__ __noinline__ void conic_factor_fp64(const LinkXf& X, const float4& a0, const float4& a1, const float4& a2,
                                               const float4& a3, float fx, float fy, float limxn, float limxp,
                                               float limyn, float limyp, float& l00, float& l01, float& l11, float& cA,
                                               float& cC) {
    constexpr double kS = 0.84932180028801907;  // sqrt(0.5 log2(e))
    double dA, dB, dC, dK;
    ewa_factor<double>(X, a0, a1, a2, a3, fx, fy, limxn, limxp, limyn, limyp, dA, dB, dC, dK);
    const double eA = dA + 0.3, eC = dC + 0.3;
    const double det = dK + 0.3 * (dA + dC) + 0.09;
    const double rc = 1.0 / sqrt(eC);
    l00 = (float)(kS * sqrt(eC / det));
    l01 = (float)(-kS * dB * rc / sqrt(det));
    l11 = (float)(kS * rc);
    cA = (float)eA;
    cC = (float)eC;
}

// Real SH basis through degree D in the 3DGS order (k = l*l + l + m), with the
// Condon-Shortley phase.  Constants: sqrt(1/(4 pi)), sqrt(3/(4 pi)),
// sqrt(15/(4 pi)), sqrt(5/(16 pi)), sqrt(15/(16 pi)), sqrt(35/(32 pi)),
// sqrt(105/(4 pi)), sqrt(21/(32 pi)), sqrt(7/(16 pi)), sqrt(105/(16 pi)).
template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = 0.28209479177387814f;
    if constexpr (D >= 1) {
        Y[1] = -0.4886025119029199f * y;
        Y[2] = 0.4886025119029199f * z;
        Y[3] = -0.4886025119029199f * x;
    }
    if constexpr (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (xx - yy);
        if constexpr (D >= 3) {
            Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
            Y[10] = 2.890611442640554f * x * y * z;
            Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);
            Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
            Y[14] = 1.445305721320277f * z * (xx - yy);
            Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
        }
    }
}

// Colour max(0, sum_k Y_k sh_k + 0.5) per channel for Gaussian g.  The
// coefficients are consumed plane by plane as they arrive (flattened value f
// = 3k + channel), so only the basis and three sums stay live; each channel
// accumulates in ascending k.
template <int D, int DT>
__device__ __forceinline__ void sh_colour(const void* base, int64_t n, int64_t g, float x, float y, float z,
                                          float& r, float& gr, float& b) {
    constexpr int NV = 3 * (D + 1) * (D + 1);
    float Y[16];
    sh_basis<D>(x, y, z, Y);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (DT == GS_F32) {
        constexpr int NP = (NV + 3) / 4;
        const float4* P = static_cast<const float4*>(base);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const float4 v = __ldg(P + (size_t)p * n + g);
            const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int f = 4 * p + h;
                if (f < NV) acc[f % 3] += Y[f / 3] * w[h];
            }
        }
    } else {
        constexpr int NP = (NV + 7) / 8;
        const uint4* P = static_cast<const uint4*>(base);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const uint4 v = __ldg(P + (size_t)p * n + g);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int f = 8 * p + h;
                if (f < NV) {
                    const uint16_t bits = (uint16_t)(w[h >> 1] >> (16 * (h & 1)));
                    float val;
                    if constexpr (DT == GS_BF16)
                        val = __uint_as_float((uint32_t)bits << 16);
                    else
                        val = __half2float(__ushort_as_half(bits));
                    acc[f % 3] += Y[f / 3] * val;
                }
            }
        }
    }
    r = fmaxf(acc[0] + 0.5f, 0.0f);
    gr = fmaxf(acc[1] + 0.5f, 0.0f);
    b = fmaxf(acc[2] + 0.5f, 0.0f);
}

// Pixel range [lo, hi] of a support interval centred at c with half extent h:
// lo = max(0, ceil((c - h) - 0.5)), hi = min(n-1, floor((c + h) - 0.5)).
__device__ __forceinline__ bool pixel_range(float c, float h, int n, int& lo, int& hi) {
    float a = ceilf(c - h - 0.5f);
    float b = floorf(c + h - 0.5f);
    if (!(a <= b)) return false;
    a = fmaxf(a, 0.0f);
    b = fminf(b, (float)(n - 1));
    if (a > b) return false;
    lo = (int)a;
    hi = (int)b;
    return true;
}

constexpr int kProjStageEnvs = 256;  // envs per shared-memory chunk of a projection block

template <int D, int DT>
__global__ void __launch_bounds__(256, 3) k_project(ProjParams P) {
    constexpr int NV = 3 * (D + 1) * (D + 1);
    const ProjBlock blk = P.blocks[blockIdx.x];
    const int t = threadIdx.x;
    const bool act = t < blk.n;
    const int lane = t & 31;
    const long long g = blk.g_first + t;
    const unsigned int local = blk.local_first + (unsigned)t;
    const bool warp_live = (t - lane) < blk.n;  // the warp owns visibility word local/32
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    if (act) {
        a0 = __ldg(P.p0 + g);
        a1 = __ldg(P.p1 + g);
        a2 = __ldg(P.p2 + g);
        a3 = __ldg(P.p3 + g);
    }
    const int li = __float_as_int(a3.w) - blk.lb;  // frame offset within the env's link table
    const float qstar = a3.y;
    const bool live = act && qstar >= 0.0f;
    const float trace = a3.z;  // trace(Sigma) >= its largest eigenvalue (rotation-invariant)
    // the caller's local index (the key's tie order): background slots map
    // through the storage order, link slots are their own
    const uint32_t key_index = (blk.frame0 && P.bg_index && act) ? (uint32_t)__ldg(P.bg_index + local) : local;
    // Every block stages, per env of a chunk, the camera, guard-band limits
    // and table offsets in shared memory; background blocks (one link frame
    // for every thread) also stage the frame's z row.  The many culled (env,
    // Gaussian) pairs then wait on shared loads instead of chains of table
    // loads, and the visible ones read their camera from shared memory.
    __shared__ float4 s_r2[kProjStageEnvs];     // background blocks: frame 0's z row
    __shared__ float4 s_cam[kProjStageEnvs];    // fx, fy, cx, cy
    __shared__ float4 s_lim[kProjStageEnvs];    // guard-band limits
    __shared__ int4 s_misc[kProjStageEnvs];     // W, H, xf_base, near plane (bits)
    __shared__ unsigned long long s_mb[kProjStageEnvs];  // visibility-word base
    __shared__ unsigned long long s_rb[kProjStageEnvs];  // record base
    __shared__ float4 s_rec[8][3 * 32];                  // per warp: the records of an env, before their store
    const bool frame0 = blk.frame0 != 0;
    for (int c0 = blk.e0; c0 < blk.e1; c0 += kProjStageEnvs) {
    const int c1 = min(c0 + kProjStageEnvs, blk.e1);
    __syncthreads();  // the previous chunk's entries are no longer read
    for (int i = t; i < c1 - c0; i += blockDim.x) {
        const EnvInfo* Ei = P.envs + c0 + i;
        const gs_camera* ci = P.cams + c0 + i;
        const int xb = __ldg(&Ei->xf_base);
        if (frame0) s_r2[i] = __ldg(&P.xf[xb].r2);
        s_cam[i] = make_float4(__ldg(&ci->fx), __ldg(&ci->fy), __ldg(&ci->cx), __ldg(&ci->cy));
        s_lim[i] = make_float4(__ldg(&Ei->lim[0]), __ldg(&Ei->lim[1]), __ldg(&Ei->lim[2]), __ldg(&Ei->lim[3]));
        s_misc[i] = make_int4(__ldg(&ci->width), __ldg(&ci->height), xb, __float_as_int(__ldg(&ci->near_plane)));
        s_mb[i] = __ldg(&Ei->mask_base);
        s_rb[i] = __ldg(&Ei->rec_base);
    }
    __syncthreads();
    for (int el = c0; el < c1; ++el) {
        bool vis = false;
        const int ei = el - c0;
        if (live) {
            const int4 misc = s_misc[ei];
            const LinkXf* Xp = P.xf + misc.z + li;
            // depth first: most (env, Gaussian) pairs stop at the near-plane test,
            // so only the z row of the transform and the near plane are read here
            LinkXf X;
            const float near = __int_as_float(misc.w);
            X.r2 = frame0 ? s_r2[ei] : __ldg(&Xp->r2);
            const float mz = X.r2.x * a0.x + X.r2.y * a0.y + X.r2.z * a0.z + X.r2.w;
            if (mz > near) {
                X.r0 = __ldg(&Xp->r0);
                X.r1 = __ldg(&Xp->r1);
                const float mx = X.r0.x * a0.x + X.r0.y * a0.y + X.r0.z * a0.z + X.r0.w;
                const float my = X.r1.x * a0.x + X.r1.y * a0.y + X.r1.z * a0.z + X.r1.w;
                const float4 cam = s_cam[ei], lim = s_lim[ei];
                const float fx = cam.x, fy = cam.y, cx = cam.z, cy = cam.w;
                const int W = misc.x, H = misc.y;
                const float limxn = lim.x, limxp = lim.y;  // per env, from the tables
                const float limyn = lim.z, limyp = lim.w;
                const float iz = 1.0f / mz;
                const float u = fx * mx * iz + cx;
                const float v = fy * my * iz + cy;
                // Conservative cull: the support half extent is at most
                // sqrt(q* (|J_row|^2 tr(Sigma) + 0.3)) with |J_row|^2 <= (f/z)^2 (1 + lim^2).
                // The test is on squares: a centre at distance d outside [0.5, W - 0.5]
                // may reach the image when d <= 1 + 1.001 sqrt(S), i.e. when d <= 1 or
                // (d - 1)^2 <= 1.002001 S (and likewise in y).
                const float lx = fmaxf(limxn, limxp), ly = fmaxf(limyn, limyp);
                const float fz = fx * iz, fzy = fy * iz;
                const float sx = qstar * (fz * fz * (1.0f + lx * lx) * trace + 0.3f);
                const float sy = qstar * (fzy * fzy * (1.0f + ly * ly) * trace + 0.3f);
                const float ex = fmaxf(fmaxf(0.5f - u, u - ((float)W - 0.5f)), 1.0f) - 1.0f;
                const float ey = fmaxf(fmaxf(0.5f - v, v - ((float)H - 0.5f)), 1.0f) - 1.0f;
                const bool maybe = ex * ex <= 1.002001f * sx && ey * ey <= 1.002001f * sy;
                if (maybe) {
                    // Sigma_2 = M M^T + 0.3 I; det = K + 0.3 (A + C) + 0.09 is a sum of
                    // non-negative terms.  The conic enters the compositor as its
                    // upper Cholesky factor L (L^T L = conic, l11 = 1/sqrt(C + 0.3)),
                    // scaled by sqrt(log2(e)/2) so that alpha = o 2^-(|L d|^2), a sum of
                    // two squares with no cancellation for thin splats.
                    constexpr float kS = 0.84932180028801907f;  // sqrt(0.5 log2(e))
                    float A, B, C, K;
                    ewa_factor<float>(X, a0, a1, a2, a3, fx, fy, limxn, limxp, limyn, limyp, A, B, C, K);
                    float cA, cC, l00, l01, l11;
                    if (K >= 0x1p-10f * A * C) {
                        cA = A + 0.3f;
                        cC = C + 0.3f;
                        const float det = K + 0.3f * (A + C) + 0.09f;
                        // reciprocal square roots (MUFU, <= 2 ulp): the support box below
                        // keeps its IEEE square roots and a 1e-4 margin over this ellipse
                        const float rc = rsqrtf(cC), rd = rsqrtf(det);
                        l00 = kS * (cC * rc) * rd;
                        l01 = -kS * B * rc * rd;
                        l11 = kS * rc;
                    } else {
                        conic_factor_fp64(X, a0, a1, a2, a3, fx, fy, limxn, limxp, limyn, limyp, l00, l01, l11, cA,
                                          cC);
                        if (P.nfp64) atomicAdd(P.nfp64, 1ull);
                    }
                    const bool ok = true;
                    const float hx = sqrtf(qstar * cA) * 1.0001f;
                    const float hy = sqrtf(qstar * cC) * 1.0001f;
                    int i0, i1, j0, j1;
                    if (ok && pixel_range(u, hx, W, i0, i1) && pixel_range(v, hy, H, j0, j1)) {
                        // SH coefficients are re-read per visible env (L1/L2 hits) and
                        // streamed into the colour sums
                        const float4 O = __ldg(&Xp->o);
                        float dx = a0.x - O.x, dy = a0.y - O.y, dz = a0.z - O.z;
                        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
                        dx *= inv;
                        dy *= inv;
                        dz *= inv;
                        float r, gg, b;
                        sh_colour<D, DT>(P.sh, P.n_gauss, g, dx, dy, dz, r, gg, b);
                        const uint32_t rx = (uint32_t)i0 | ((uint32_t)i1 << 16);
                        const uint32_t ry = (uint32_t)j0 | ((uint32_t)j1 << 16);
                        const size_t ri = (size_t)s_rb[ei] + local;
                        float4* sr = s_rec[t >> 5] + 3 * lane;
                        sr[0] = make_float4(u, v, a0.w, mz);
                        sr[1] = make_float4(l00, l01, l11, __uint_as_float(rx));
                        sr[2] = make_float4(r, gg, b, __uint_as_float(ry));
                        P.r3[ri] = make_uint4(rx, ry, __float_as_uint(mz), key_index);
                        if (P.dbg_hxy) P.dbg_hxy[ri] = make_float2(hx, hy);
                        vis = true;
                    }
                }
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, vis);
        if (m) {  // warp-uniform
            __syncwarp();
            store_records(P.r0, (size_t)s_rb[ei] + local - lane, s_rec[t >> 5], m, lane);
            __syncwarp();  // s_rec is rewritten for the next env
        }
        if (lane == 0 && warp_live) {
            const unsigned long long mb = s_mb[ei];
            P.mask[(size_t)mb + (local >> 5)] = m;
            if (P.nvis && m) atomicAdd(P.nvis, (unsigned long long)__popc(m));
        }
    }
    }  // env chunks
}

template <int D>
static void launch_project_d(const DevGaussians& Dg, const ProjParams& P, int n_blocks, cudaStream_t st) {
    switch (Dg.dtype) {
        case GS_F32: k_project<D, GS_F32><<<n_blocks, 256, 0, st>>>(P); break;
        case GS_BF16: k_project<D, GS_BF16><<<n_blocks, 256, 0, st>>>(P); break;
        default: k_project<D, GS_F16><<<n_blocks, 256, 0, st>>>(P); break;
    }
}

cudaError_t launch_project(const DevGaussians& Dg, const ProjParams& P, int n_blocks, cudaStream_t st) {
    if (n_blocks == 0) return cudaSuccess;
    switch (Dg.sh_degree) {
        case 0: launch_project_d<0>(Dg, P, n_blocks, st); break;
        case 1: launch_project_d<1>(Dg, P, n_blocks, st); break;
        case 2: launch_project_d<2>(Dg, P, n_blocks, st); break;
        default: launch_project_d<3>(Dg, P, n_blocks, st); break;
    }
    return cudaGetLastError();
}

}  // namespace gsb
