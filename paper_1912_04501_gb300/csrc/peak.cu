// CUDA-core FMA throughput of the device, measured: the denominators of the
// near sums' rooflines (their pairs are FMA/MUL/ADD work, not tensor-core or
// memory work).  Three kernels of independent FMA chains -- scalar
// fma.rn.f32, packed fma.rn.f32x2 (two lanes per instruction) and
// fma.rn.f64 -- each launched as a full-occupancy grid of a few milliseconds
// and timed with CUDA events; the best of three launches counts, at 2 flops
// per FMA lane.
// No counterpart in the paper (a measurement aid, like bie_profile).
#include <algorithm>

#include "bie_internal.cuh"

namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kInner = 64;    // unrolled FMA rounds per loop trip
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_ffma(int trips, float a, float b, float* __restrict__ sink) {
    float acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int i = 0; i < kInner; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[k]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_ffma2(int trips, float a, float b, float* __restrict__ sink) {
    bie::f32x2 acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = bie::pk2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    const bie::f32x2 a2 = bie::pk2(a, a), b2 = bie::pk2(b, b);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int i = 0; i < kInner; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[k]) : "l"(a2), "l"(b2));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        bie::upk2(acc[k], lo, hi);
        s += lo + hi;
    }
    if (s == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_dfma(int trips, double a, double b, double* __restrict__ sink) {
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int i = 0; i < kInner; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[k]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == 12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int bie_alu_peak(int32_t device, void* stream, double* ffma_tflops, double* ffma2_tflops,
                            double* dfma_tflops) {
    if (device < 0) return BIE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return BIE_ECUDA;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return BIE_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma, kThreads, 0) != cudaSuccess || per_sm <= 0)
        return BIE_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sms * per_sm;
    const int trips = 1024;  // 1024 x 64 x 8 FMAs per thread: a few ms per launch
    const double lanes = (double)blocks * kThreads * trips * kInner * kChains;
    double* sink = nullptr;  // never written (the guard value is never met); a valid pointer all the same
    if (cudaMalloc((void**)&sink, (size_t)blocks * kThreads * sizeof(double)) != cudaSuccess) return BIE_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BIE_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = BIE_ECUDA;
    double best[3] = {0, 0, 0};
    for (int kind = 0; kind < 3 && !rc; ++kind) {
        // the FP64 pipe is far narrower: fewer trips keep that launch short
        const int tr = kind == 2 ? trips / 64 : trips;
        for (int rep = 0; rep < 4 && !rc; ++rep) {  // one warm-up, three timed
            cudaEventRecord(e0, st);
            if (kind == 0)
                k_ffma<<<blocks, kThreads, 0, st>>>(tr, 0.999f, 1e-4f, reinterpret_cast<float*>(sink));
            else if (kind == 1)
                k_ffma2<<<blocks, kThreads, 0, st>>>(tr, 0.999f, 1e-4f, reinterpret_cast<float*>(sink));
            else
                k_dfma<<<blocks, kThreads, 0, st>>>(tr, 0.999, 1e-4, sink);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = BIE_ECUDA;
                break;
            }
            const double flops = 2.0 * lanes * (kind == 1 ? 2.0 : 1.0) * tr / trips;
            if (rep > 0 && ms > 0) best[kind] = std::max(best[kind], flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    if (ffma_tflops) *ffma_tflops = best[0];
    if (ffma2_tflops) *ffma2_tflops = best[1];
    if (dfma_tflops) *dfma_tflops = best[2];
    return BIE_OK;
}
