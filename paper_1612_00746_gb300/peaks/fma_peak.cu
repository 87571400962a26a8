// FMA-chain microbenchmark: the FP32 and FP64 arithmetic peaks of the GPU,
// measured under load, as the denominators of the ALU rooflines that the
// benchmark reports (the stencil kernels are bound by FP32 FMA issue, the
// FP64 comparison path by the FP64 pipe).
//
// Every thread runs CH independent dependent chains acc = acc * a + b for
// `iters` rounds; a and b are run-time values, so nothing folds.  Three
// kinds: packed FP32 pairs (fma.rn.f32x2, the instruction the stencil
// kernels use), scalar FP32 and FP64.  The grid is a whole number of waves
// of resident blocks on every SM.  The host entry point calibrates the
// number of rounds so that one timed launch takes about `seconds`, and
// returns the rate in FMA lane-operations per second (x2 for flop/s).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) fma2_kernel(float a, float b, long long iters, float *sink) {
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
    const float2 va = make_float2(a, a), vb = make_float2(b, b);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], va, vb);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) fma_kernel(float a, float b, long long iters, float *sink) {
    float acc[2 * kChains];
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) acc[c] = threadIdx.x * 1e-3f + c;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < 2 * kChains; ++c) acc[c] = fmaf(acc[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) s += acc[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_kernel(double a, double b, long long iters, float *sink) {
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678) sink[threadIdx.x] = (float)s;
}

// FMA lane-operations of one thread per round of the outer loop: 8 x CH
// packed pairs (two each), 8 x 2CH scalar FP32, 8 x CH FP64.
long long lane_ops_per_round(int kind) { return kind == 2 ? 8LL * kChains : 16LL * kChains; }

int launch(int kind, int blocks, long long iters, float *sink, cudaStream_t s) {
    if (kind == 0)
        fma2_kernel<<<blocks, kThreads, 0, s>>>(0.999999f, 1e-6f, iters, sink);
    else if (kind == 1)
        fma_kernel<<<blocks, kThreads, 0, s>>>(0.999999f, 1e-6f, iters, sink);
    else
        dfma_kernel<<<blocks, kThreads, 0, s>>>(0.999999999, 1e-9, iters, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace

extern "C" {

/*
 * Measure an arithmetic peak of the current device.  kind 0: packed FP32
 * pairs (fma.rn.f32x2), 1: scalar FP32 fma, 2: FP64 fma.  Runs one launch
 * of about `seconds` (0.05..20) after a calibration launch and writes the
 * rate in FMA lane-operations per second to *ops_per_s and the timed
 * duration to *elapsed_s.  Returns 0, 1 for a bad argument, 3 for a CUDA
 * failure.  Allocates and frees a 1 KB sink.  Synchronizes the device.
 */
int fma_peak_measure(int kind, double seconds, double *ops_per_s, double *elapsed_s) {
    if (kind < 0 || kind > 2 || !ops_per_s || !(seconds >= 0.05 && seconds <= 20.0)) return 1;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
    const void *fn = kind == 0 ? (const void *)fma2_kernel : (kind == 1 ? (const void *)fma_kernel : (const void *)dfma_kernel);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1) return 3;
    const int blocks = sms * per_sm;
    float *sink = nullptr;
    if (cudaMalloc(&sink, 1024) != cudaSuccess) return 3;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int st = 0;
    long long iters = kind == 2 ? 64 : 4096;
    float ms = 0.f;
    // calibrate: grow the round count until a launch takes >= 20 ms
    for (int t = 0; t < 24 && st == 0; ++t) {
        cudaEventRecord(e0, 0);
        st = launch(kind, blocks, iters, sink, 0);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = 3;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms >= 20.f) break;
        iters *= 4;
    }
    if (st == 0) {
        iters = (long long)((double)iters * seconds * 1e3 / ms);
        if (iters < 1) iters = 1;
        cudaEventRecord(e0, 0);
        st = launch(kind, blocks, iters, sink, 0);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = 3;
        cudaEventElapsedTime(&ms, e0, e1);
    }
    if (st == 0) {
        const double lane_ops = (double)blocks * kThreads * (double)iters * (double)lane_ops_per_round(kind);
        *ops_per_s = lane_ops / (ms * 1e-3);
        if (elapsed_s) *elapsed_s = ms * 1e-3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

}  // extern "C"
