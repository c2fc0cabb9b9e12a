// npm_peaks.cu -- measured throughput of the units the hot path leans on:
// FP32 FMA (packed two-lane and scalar), the MUFU exponential, random
// 32-byte sector reads from L2, and random FP32 (scalar, 2- and 4-wide
// vector) atomic adds into L2. The roofline
// of each kernel is the minimum over its HBM, L2, tensor and ALU/MUFU bounds;
// HBM and tensor peaks are copy and GEMM measurements, these are the rest.
//
// Every kernel runs a fixed number of iterations over in-bounds addresses
// (power-of-two buffer, masked indices); nothing waits on anything.
#include <cuda_runtime.h>
#include <stdint.h>

#include "npm_handle.h"

namespace {

constexpr int kThreads = 256;
constexpr int kIters = 2048;
constexpr size_t kBufBytes = size_t(64) << 20;  // L2-resident (129 MB L2)
constexpr uint32_t kBufFloats = uint32_t(kBufBytes / 4);

// Sixteen independent packed two-lane FMA chains per thread.
__global__ void __launch_bounds__(kThreads) k_fma(float seed, float* sink) {
    float2 acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = make_float2(seed + i, seed - i);
    const float2 a = make_float2(0.999f, 1.001f), b = make_float2(1e-3f, -1e-3f);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = __ffma2_rn(acc[i], a, b);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += acc[i].x + acc[i].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains live
}

// Sixteen independent scalar FMA chains per thread.
__global__ void __launch_bounds__(kThreads) k_fma1(float seed, float* sink) {
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = seed + i;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = fmaf(acc[i], 0.999f, 1e-3f);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += acc[i];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

// Eight independent chains of x <- 2^(-x) on the MUFU unit.
__global__ void __launch_bounds__(kThreads) k_mufu(float seed, float* sink) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed * (i + 1) * 1e-3f;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[i]) : "f"(-x[i]));
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__device__ __forceinline__ uint32_t hash32(uint32_t v) {
    v ^= v >> 16;
    v *= 0x7feb352du;
    v ^= v >> 15;
    v *= 0x846ca68bu;
    v ^= v >> 16;
    return v;
}

// Random sector reads, L2 only (ld.global.cg): one float per 32-byte
// sector, eight loads in flight per thread.
__global__ void __launch_bounds__(kThreads) k_l2_read(const float* __restrict__ buf, float* sink, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.0f;
    for (int it = 0; it < iters; ++it) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t sector = hash32(tid * 0x9E3779B9u + (uint32_t)(it * 8 + i)) & (kBufFloats / 8 - 1);
            v[i] = __ldcg(buf + sector * 8);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s += v[i];
    }
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

// Random atomic adds without return (reductions in L2): W = 1 scalar,
// W = 2 and 4 vector.
template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_atomic(float* __restrict__ buf, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t slot = hash32(tid * 0x9E3779B9u + (uint32_t)(it * 8 + i)) & (kBufFloats / 8 - 1);
            if constexpr (W == 1)
                atomicAdd(buf + slot * 8, 1.0f);
            else if constexpr (W == 2)
                atomicAdd(reinterpret_cast<float2*>(buf + slot * 8), make_float2(1.0f, 1.0f));
            else
                atomicAdd(reinterpret_cast<float4*>(buf + slot * 8), make_float4(1.0f, 1.0f, 1.0f, 1.0f));
        }
    }
}

template <typename F>
float best_ms(F launch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps) {
    launch();  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.0f && ms < best) best = ms;
    }
    return best;
}

}  // namespace

extern "C" npm_status npm_measure_unit_peaks(npm_unit_peaks* out, void* stream) {
    if (!out) return npm::set_error(NPM_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    float* buf = nullptr;
    float* sink = nullptr;
    if (cudaMalloc(&buf, kBufBytes) != cudaSuccess || cudaMalloc(&sink, kThreads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        return npm::set_error(NPM_ERR_OOM, "cannot allocate the measurement buffer");
    }
    cudaMemsetAsync(buf, 0, kBufBytes, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * (2048 / kThreads);
    const double threads = (double)blocks * kThreads;

    const float ms_fma = best_ms([&] { k_fma<<<blocks, kThreads, 0, st>>>(1.0f, sink); }, st, e0, e1, 3);
    const float ms_fma1 = best_ms([&] { k_fma1<<<blocks, kThreads, 0, st>>>(1.0f, sink); }, st, e0, e1, 3);
    const float ms_mufu = best_ms([&] { k_mufu<<<blocks, kThreads, 0, st>>>(1.0f, sink); }, st, e0, e1, 3);
    const int mem_iters = 64;
    const float ms_rd = best_ms([&] { k_l2_read<<<blocks, kThreads, 0, st>>>(buf, sink, mem_iters); }, st, e0, e1, 3);
    const float ms_at1 = best_ms([&] { k_l2_atomic<1><<<blocks, kThreads, 0, st>>>(buf, mem_iters); }, st, e0, e1, 3);
    const float ms_at2 = best_ms([&] { k_l2_atomic<2><<<blocks, kThreads, 0, st>>>(buf, mem_iters); }, st, e0, e1, 3);
    const float ms_at4 = best_ms([&] { k_l2_atomic<4><<<blocks, kThreads, 0, st>>>(buf, mem_iters); }, st, e0, e1, 3);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (err != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(err));

    const double accesses = threads * mem_iters * 8.0;
    out->fp32_fma_tflops = threads * kIters * 16.0 * 2.0 * 2.0 / (ms_fma * 1e-3) / 1e12;
    out->fp32_fma_scalar_tflops = threads * kIters * 16.0 * 2.0 / (ms_fma1 * 1e-3) / 1e12;
    out->mufu_gops = threads * kIters * 8.0 / (ms_mufu * 1e-3) / 1e9;
    out->l2_sector_read_gbs = accesses * 32.0 / (ms_rd * 1e-3) / 1e9;
    out->l2_atomic_gops = accesses / (ms_at1 * 1e-3) / 1e9;
    out->l2_atomic_v2_gops = accesses / (ms_at2 * 1e-3) / 1e9;
    out->l2_atomic_v4_gops = accesses / (ms_at4 * 1e-3) / 1e9;
    out->sm_count = sms;
    out->max_sm_clock_mhz = clk_khz / 1000.0;
    return NPM_OK;
}
