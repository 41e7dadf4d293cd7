// FP32 FMA throughput microbenchmark: the denominator of the coding passes'
// roofline.  Those passes are bound by FP32 fused multiply-adds (their
// arithmetic intensity is far above the HBM ridge), so their achieved
// FLOP/s is compared with what this GPU really sustains for FP32 FMAs, in
// the instruction forms the coders use: scalar fma.rn.f32 and packed
// fma.rn.f32x2.  Nothing here changes a clock or any other GPU setting; the
// SM clock is whatever the GPU runs at during the timing.
#include <algorithm>

#include "ctx.cuh"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kUnroll = 8;     // FMA rounds per loop trip

__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
    asm volatile("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// Each thread runs kChains independent packed chains d = a*d + b (2 FMAs per
// instruction, 4 FLOP); iters * kUnroll rounds.  |a| < 1 keeps d bounded.
__global__ void __launch_bounds__(256) fma2_peak_kernel(float a, float b, int iters, float* out) {
    const unsigned long long A = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
    const unsigned long long B = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
    unsigned long long d[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v = (float)(threadIdx.x + c);
        d[c] = ((unsigned long long)__float_as_uint(v + 0.5f) << 32) | __float_as_uint(v);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) fma2(d[c], A, B);
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc += __uint_as_float((unsigned)(d[c] & 0xffffffffu)) + __uint_as_float((unsigned)(d[c] >> 32));
    if (out && acc == 1234.5f) out[blockIdx.x] = acc;   // keeps the chains live (out is null)
}

// The same with scalar FMAs (2 FLOP per instruction), 2 * kChains chains so
// that the FLOP per thread match the packed kernel.
__global__ void __launch_bounds__(256) fma1_peak_kernel(float a, float b, int iters, float* out) {
    float d[2 * kChains];
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) d[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 2 * kChains; ++c) asm volatile("fma.rn.f32 %0, %1, %0, %2;" : "+f"(d[c]) : "f"(a), "f"(b));
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) acc += d[c];
    if (out && acc == 1234.5f) out[blockIdx.x] = acc;
}

}  // namespace

extern "C" int sdl_fp32_fma_peak(int packed, double* tflops_out, double* ms_out, void* stream) {
    if (!tflops_out || (packed != 0 && packed != 1)) return SDL_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SDL_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = sms * 8;   // 64 warps per SM
    const int iters = 2048;
    const double flops = (double)blocks * threads * iters * kUnroll * kChains * 4.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SDL_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SDL_ERR_CUDA;
    }
    float best = 1e30f;
    int rc = SDL_OK;
    for (int rep = 0; rep < 12 && rc == SDL_OK; ++rep) {
        cudaEventRecord(e0, st);
        if (packed)
            fma2_peak_kernel<<<blocks, threads, 0, st>>>(0.999f, 1e-3f, iters, nullptr);
        else
            fma1_peak_kernel<<<blocks, threads, 0, st>>>(0.999f, 1e-3f, iters, nullptr);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = SDL_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep >= 2) best = std::min(best, ms);   // the first two launches warm up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SDL_OK) return rc;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return SDL_OK;
}
