// Measured plain-ALU rates of the device: FP32 FMA lane-ops/s and MUFU ex2
// lane-ops/s.  The compositor is bound by these two pipes (its alpha is one
// ex2 and about twenty FMA-class operations per (pixel, splat) pair), so they
// are the denominators of its roofline next to the rate derived from SM count
// and clock.  Not part of a render.
#include "gs_internal.cuh"

namespace gsb {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-6f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_ex2(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 1e-6f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a[k]));
                a[k] = y;  // stays in (0.5, 1): 2^-x maps [0.5, 1] into itself
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gsb

using namespace gsb;

extern "C" gs_status gs_measure_alu_peak(double* fma_lane_ops_per_s, double* ex2_lane_ops_per_s, void* cuda_stream) {
    if (!fma_lane_ops_per_s || !ex2_lane_ops_per_s) return report(GS_ERR_INVALID, "null output");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return report(GS_ERR_CUDA, "device query failed");
    const int blocks = sms * 8, threads = 256;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return report(GS_ERR_OOM, "alloc");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double rates[2] = {0.0, 0.0};
    const int iters[2] = {4096, 1024};
    gs_status rc = GS_OK;
    for (int which = 0; which < 2 && rc == GS_OK; ++which) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // first run warms up; the best of the rest counts
            cudaEventRecord(e0, st);
            if (which == 0) k_ffma<<<blocks, threads, 0, st>>>(out, iters[0], 0.999999f, 1e-7f);
            else k_ex2<<<blocks, threads, 0, st>>>(out, iters[1]);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                rc = report(GS_ERR_CUDA, "microbenchmark launch failed");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double ops = (double)blocks * threads * iters[which] * 16.0 * kChains;
        rates[which] = ops / (best * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != GS_OK) return rc;
    *fma_lane_ops_per_s = rates[0];
    *ex2_lane_ops_per_s = rates[1];
    return GS_OK;
}
