// dse_peaks.cu -- arithmetic-rate microbenchmark (include/dse_peaks.h): the
// measured FP64 FMA, FP32 FMA and special-function-unit rates that the
// arithmetic roofline of the quadrature kernels divides by.
#include <cuda_runtime.h>

#include "dse.h"
#include "dse_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

// Sink for the chains' results: written only if a value is impossible, so that
// the compiler keeps every operation (no allocation needed).
__device__ double g_peak_sink;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// D = A B + D for one 8x8x4 FP64 tile of the warp (a and b: this thread's
// elements of A and B, d: its two of D).
__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

// iters x kUnroll x kChains operations per thread (for DMMA, matrix products:
// 8 FMAs per thread each).
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_alu_peak(int iters, double seed) {
    const double t = seed + 1e-9 * threadIdx.x;
    if (KIND == DSE_PEAK_FP64_FMA) {
        double a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = t + i;
        const double b = 0.9999999, c = 1e-7;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        if (s == -1.0) g_peak_sink = s;
    } else if (KIND == DSE_PEAK_FP64_DMMA) {
        double d[kChains][2];
#pragma unroll
        for (int i = 0; i < kChains; ++i) d[i][0] = d[i][1] = t + i;
        const double a = 1e-4 * (1.0 + 1e-3 * (threadIdx.x & 31)), b = 1e-4;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kChains; ++i) dmma_8x8x4(d[i][0], d[i][1], a, b);
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += d[i][0] + d[i][1];
        if (s == -1.0) g_peak_sink = s;
    } else if (KIND == DSE_PEAK_FP32X2_FMA) {
        float2 a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = make_float2((float)t + i, (float)t - i);
        const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b, c);
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
        if (s == -1.0f) g_peak_sink = s;
    } else if (KIND == DSE_PEAK_FP32_FMA) {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (float)t + i;
        const float b = 0.9999999f, c = 1e-7f;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        if (s == -1.0f) g_peak_sink = s;
    } else {
        // x -> 2^-x keeps x in [0.5, 1]; x -> lg2(x) + 2 keeps x in [1, 2]
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = KIND == DSE_PEAK_MUFU_EX2 ? 0.75f : 1.5f + 0.01f * i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kChains; ++i)
                    a[i] = KIND == DSE_PEAK_MUFU_EX2 ? ex2_approx(-a[i]) : lg2_approx(a[i]) + 1.0f;
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        if (s == -1.0f) g_peak_sink = s;
    }
}

template <int KIND>
cudaError_t run(int grid, int iters, cudaStream_t s) {
    k_alu_peak<KIND><<<grid, kThreads, 0, s>>>(iters, 1.0);
    return cudaGetLastError();
}

cudaError_t launch(int kind, int grid, int iters, cudaStream_t s) {
    switch (kind) {
        case DSE_PEAK_FP64_FMA: return run<DSE_PEAK_FP64_FMA>(grid, iters, s);
        case DSE_PEAK_FP32_FMA: return run<DSE_PEAK_FP32_FMA>(grid, iters, s);
        case DSE_PEAK_MUFU_EX2: return run<DSE_PEAK_MUFU_EX2>(grid, iters, s);
        case DSE_PEAK_FP64_DMMA: return run<DSE_PEAK_FP64_DMMA>(grid, iters, s);
        case DSE_PEAK_FP32X2_FMA: return run<DSE_PEAK_FP32X2_FMA>(grid, iters, s);
        default: return run<DSE_PEAK_MUFU_LG2>(grid, iters, s);
    }
}

int occupancy(int kind) {
    int nb = 0;
    cudaError_t e;
    switch (kind) {
        case DSE_PEAK_FP64_FMA:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_FP64_FMA>, kThreads, 0);
            break;
        case DSE_PEAK_FP32_FMA:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_FP32_FMA>, kThreads, 0);
            break;
        case DSE_PEAK_MUFU_EX2:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_MUFU_EX2>, kThreads, 0);
            break;
        case DSE_PEAK_FP64_DMMA:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_FP64_DMMA>, kThreads, 0);
            break;
        case DSE_PEAK_FP32X2_FMA:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_FP32X2_FMA>, kThreads, 0);
            break;
        default:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alu_peak<DSE_PEAK_MUFU_LG2>, kThreads, 0);
            break;
    }
    return e == cudaSuccess ? nb : 0;
}

// duration of one launch of `iters` iterations, in ms
cudaError_t timed(int kind, int grid, int iters, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch(kind, grid, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e;
}

}  // namespace

extern "C" int dse_alu_peak(int kind, double target_ms, void* stream, double* ops_per_s, double* ms) {
    if (kind < DSE_PEAK_FP64_FMA || kind > DSE_PEAK_FP32X2_FMA || !ops_per_s || !(target_ms >= 1.0) ||
        !(target_ms <= 5000.0))
        return DSE_ERR_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return DSE_ERR_CUDA;
    const int per_sm = occupancy(kind);
    if (per_sm <= 0) return DSE_ERR_CUDA;
    const int grid = nsm * per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return DSE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DSE_ERR_CUDA;
    }
    // warm-up and calibration: grow the launch until it takes >= 2 ms, then
    // scale it to target_ms
    int iters = 16;
    float t = 0.0f;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < 24 && e == cudaSuccess; ++round) {
        e = timed(kind, grid, iters, s, e0, e1, &t);
        if (e != cudaSuccess || t >= 2.0f || iters > (1 << 24)) break;
        iters *= 4;
    }
    if (e == cudaSuccess) {
        const double scale = target_ms / (t > 0.0f ? t : 1.0f);
        double want = iters * scale;
        if (want < 1.0) want = 1.0;
        if (want > 2.0e9) want = 2.0e9;
        iters = (int)want;
        e = timed(kind, grid, iters, s, e0, e1, &t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    const double ops = (double)grid * kThreads * (double)iters * kUnroll * kChains *
                       (kind == DSE_PEAK_FP64_DMMA ? 8 : kind == DSE_PEAK_FP32X2_FMA ? 2 : 1);
    *ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
    return DSE_OK;
}
