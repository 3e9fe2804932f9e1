// scmd_peak.cu -- md_fp32_peak: the FP32 lane-operation rate this device sustains, measured.
//
// The pair passes are bound by FP32 SIMT arithmetic, so their roofline denominator is the FP32
// pipe's rate. Besides the figure derived from the unit counts (SMs x 128 FP32 lanes x the
// maximum SM clock), this measures what FFMA chains actually reach on every SM: each thread runs
// 8 independent multiply-add chains (enough to hide the FMA latency at 16 warps per SM), a
// launch covers every SM twice, and CUDA events time `reps` back-to-back launches.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/scmd.h"
#include "scmd_internal.cuh"

namespace {

constexpr int kChains = 8;    // independent FFMA chains per thread
constexpr int kUnroll = 16;   // FFMA per chain per loop iteration
constexpr int kIters = 4096;  // loop iterations per thread
constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads) k_ffma(float* sink, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) sink[0] = s;  // never true for these operands; keeps the chains live
}

}  // namespace

extern "C" md_status md_fp32_peak(int32_t reps, double* measured, double* derived) {
    scmd::set_thread_error("");
    if (reps < 1 || !measured || !derived) {
        scmd::set_thread_error("md_fp32_peak: reps must be >= 1 and both outputs non-NULL");
        return MD_ERR_INVALID;
    }
    int dev = 0, sms = 0, khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    float* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&sink), sizeof(float), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 2 * sms;
    if (e == cudaSuccess) {
        k_ffma<<<blocks, kThreads, 0, s>>>(sink, 0.999f, 0.001f);  // warm-up (clock ramp)
        k_ffma<<<blocks, kThreads, 0, s>>>(sink, 0.999f, 0.001f);
        e = cudaEventRecord(e0, s);
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        k_ffma<<<blocks, kThreads, 0, s>>>(sink, 0.999f, 0.001f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (sink) cudaFreeAsync(sink, s);
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess || ms <= 0.f) {
        char buf[200];
        snprintf(buf, sizeof buf, "md_fp32_peak: %s", e != cudaSuccess ? cudaGetErrorString(e) : "no elapsed time");
        scmd::set_thread_error(buf);
        return MD_ERR_CUDA;
    }
    const double ops = (double)reps * blocks * kThreads * (double)kIters * kUnroll * kChains;
    *measured = ops / (ms * 1e-3);
    *derived = (double)sms * 128.0 * (double)khz * 1e3;
    return MD_OK;
}
