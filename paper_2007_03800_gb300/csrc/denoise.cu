// Patch-based denoising around the sparse coder (the experiment of Sec. IV):
// gather every stride-1 p x p patch of an image with its mean removed, put
// the coded patches back by averaging overlapping reconstructions, and the
// PSNR and SSIM of the result.
#include <algorithm>
#include <cmath>

#include "ctx.cuh"

using namespace sdl;

namespace {

constexpr unsigned kFull = 0xffffffffu;

// One warp per patch k (top-left corner (r, c), raster order over the
// (H-p+1) x (W-p+1) corners); element (a, b) goes to patches[k*p*p + a + p*b].
__global__ void extract_patches_kernel(const float* __restrict__ img, int H, int W, int p,
                                       float* __restrict__ patches, float* __restrict__ means,
                                       long long N) {
    const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const int wc = W - p + 1;
    const int r = (int)(k / wc), c = (int)(k % wc);
    const int pp = p * p;
    float s = 0.f;
    for (int e = lane; e < pp; e += 32) {
        const int a = e % p, b = e / p;
        s += img[(size_t)(r + a) * W + (c + b)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    const float mean = s / (float)pp;
    float* dst = patches + (size_t)k * pp;
    for (int e = lane; e < pp; e += 32) {
        const int a = e % p, b = e / p;
        dst[e] = img[(size_t)(r + a) * W + (c + b)] - mean;
    }
    if (lane == 0) means[k] = mean;
}

// Reconstructed patch k (mean added back): one warp per patch.
__global__ void reconstruct_patches_kernel(const int32_t* __restrict__ support,
                                           const float* __restrict__ coef,
                                           const float* __restrict__ means, long long N, int s,
                                           const float* __restrict__ D1, int n1,
                                           const float* __restrict__ D2, int n2, int p,
                                           float* __restrict__ rec) {
    const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const int pp = p * p;
    int q = -1;
    float x = 0.f;
    if (lane < s) {
        q = support[k * s + lane];
        x = coef[k * s + lane];
    }
    const float mean = means[k];
    for (int e = lane; e < pp; e += 32) {
        const int a = e % p, b = e / p;
        float v = mean;
        for (int l = 0; l < s; ++l) {
            const int ql = __shfl_sync(kFull, q, l);
            const float xl = __shfl_sync(kFull, x, l);
            if (ql >= 0 && ql < n1 * n2) {
                const int i = ql % n1, j = ql / n1;
                v = fmaf(xl * D1[a + p * i], D2[b + p * j], v);
            }
        }
        rec[(size_t)k * pp + e] = v;
    }
}

// Output pixel = average of the reconstructions of every patch covering it,
// summed in a fixed (r, c) order: deterministic.
__global__ void average_patches_kernel(const float* __restrict__ rec, int H, int W, int p,
                                       float* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const int wc = W - p + 1;
    const int r0 = max(0, y - p + 1), r1 = min(y, H - p);
    const int c0 = max(0, x - p + 1), c1 = min(x, W - p);
    const int pp = p * p;
    float s = 0.f;
    for (int r = r0; r <= r1; ++r)
        for (int c = c0; c <= c1; ++c) {
            const long long k = (long long)r * wc + c;
            s += rec[(size_t)k * pp + (y - r) + p * (x - c)];
        }
    out[(size_t)y * W + x] = s / (float)((r1 - r0 + 1) * (c1 - c0 + 1));
}

// PSNR = 10 log10(peak^2 / MSE): one CTA, compensated FP32 per thread,
// fixed-order FP64 combination.
__global__ void __launch_bounds__(1024) psnr_kernel(const float* __restrict__ a,
                                                    const float* __restrict__ b, long long count,
                                                    float peak, float* __restrict__ out) {
    __shared__ double part[32];
    float sum = 0.f, comp = 0.f;
    for (long long e = threadIdx.x; e < count; e += blockDim.x) {
        const float d = a[e] - b[e];
        const float y = d * d - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    double v = (double)sum - (double)comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        const double mse = tot / (double)count;
        out[0] = (float)(10.0 * log10((double)peak * peak / mse));
    }
}

// SSIM index (Wang, Bovik, Sheikh, Simoncelli 2004) of x against ref: one
// thread per window position inside the image (valid region), 11 x 11
// Gaussian window (sigma 1.5, normalised to sum 1), per-block sums in FP64
// combined in a fixed order by ssim_finish_kernel.
constexpr int kSsimWin = 11;
constexpr float kSsimSigma = 1.5f;
constexpr int kSsimThreads = 256;

__global__ void __launch_bounds__(kSsimThreads)
    ssim_kernel(const float* __restrict__ x, const float* __restrict__ y, int H, int W,
                float peak, double* __restrict__ part) {
    __shared__ float w[kSsimWin * kSsimWin];
    __shared__ double red[kSsimThreads / 32];
    constexpr int G = kSsimWin;
    if (threadIdx.x < G * G) {
        const int u = threadIdx.x / G - G / 2, v = threadIdx.x % G - G / 2;
        w[threadIdx.x] = expf(-(float)(u * u + v * v) / (2.f * kSsimSigma * kSsimSigma));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int e = 0; e < G * G; ++e) t += (double)w[e];
        red[0] = t;
    }
    __syncthreads();
    const float inv = (float)(1.0 / red[0]);
    __syncthreads();
    if (threadIdx.x < G * G) w[threadIdx.x] *= inv;
    __syncthreads();
    const int wc = W - G + 1;
    const long long P = (long long)(H - G + 1) * wc;
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double val = 0.0;
    if (k < P) {
        const int r = (int)(k / wc), c = (int)(k % wc);
        float mx = 0.f, my = 0.f;
        for (int a = 0; a < G; ++a)
            for (int b = 0; b < G; ++b) {
                const float wt = w[a * G + b];
                mx = fmaf(wt, x[(size_t)(r + a) * W + c + b], mx);
                my = fmaf(wt, y[(size_t)(r + a) * W + c + b], my);
            }
        float vx = 0.f, vy = 0.f, cxy = 0.f;
        for (int a = 0; a < G; ++a)
            for (int b = 0; b < G; ++b) {
                const float wt = w[a * G + b];
                const float dx = x[(size_t)(r + a) * W + c + b] - mx;
                const float dy = y[(size_t)(r + a) * W + c + b] - my;
                vx = fmaf(wt * dx, dx, vx);
                vy = fmaf(wt * dy, dy, vy);
                cxy = fmaf(wt * dx, dy, cxy);
            }
        const double C1 = (0.01 * peak) * (0.01 * peak), C2 = (0.03 * peak) * (0.03 * peak);
        val = ((2.0 * mx * my + C1) * (2.0 * cxy + C2)) /
              (((double)mx * mx + (double)my * my + C1) * ((double)vx + vy + C2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(kFull, val, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int e = 0; e < kSsimThreads / 32; ++e) t += red[e];
        part[blockIdx.x] = t;
    }
}

__global__ void ssim_finish_kernel(const double* __restrict__ part, int nblocks, long long P,
                                   float* __restrict__ out) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += part[b];
        out[0] = (float)(t / (double)P);
    }
}

}  // namespace

extern "C" {

int sdl_extract_patches(const float* image, int H, int W, int p, float* patches, float* means,
                        void* stream) {
    if (!image || !patches || !means || p < 1 || H < p || W < p) return SDL_ERR_ARG;
    const long long N = (long long)(H - p + 1) * (W - p + 1);
    const int threads = 256;
    const long long blocks = (N * 32 + threads - 1) / threads;
    extract_patches_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        image, H, W, p, patches, means, N);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int sdl_patch_average(sdl_ctx* c, const int32_t* support, const float* coef, const float* means,
                      int s_max, const float* D1, int n1, const float* D2, int n2, int p, int H,
                      int W, float* image_out, void* stream) {
    if (!c || !support || !coef || !means || !D1 || !D2 || !image_out) return SDL_ERR_ARG;
    if (p < 1 || H < p || W < p || s_max < 1 || s_max > 32 || n1 < 1 || n2 < 1) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = (long long)(H - p + 1) * (W - p + 1);
    const size_t need = (size_t)N * p * p;
    if (need > c->cap_rec) {
        if (c->rec) cudaFree(c->rec);
        c->rec = nullptr;
        c->cap_rec = 0;
        if (cudaMalloc(&c->rec, need * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return SDL_ERR_WORKSPACE;
        }
        c->cap_rec = need;
    }
    const int threads = 256;
    const long long blocks = (N * 32 + threads - 1) / threads;
    reconstruct_patches_kernel<<<(unsigned)blocks, threads, 0, st>>>(support, coef, means, N, s_max,
                                                                     D1, n1, D2, n2, p, c->rec);
    average_patches_kernel<<<dim3((W + 127) / 128, H), 128, 0, st>>>(c->rec, H, W, p, image_out);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int sdl_ssim(sdl_ctx* c, const float* x, const float* ref, int H, int W, float peak, float* out,
             void* stream) {
    if (!c || !x || !ref || !out || H < kSsimWin || W < kSsimWin || !(peak > 0.f))
        return SDL_ERR_ARG;
    DeviceGuard g(c->device);
    const long long P = (long long)(H - kSsimWin + 1) * (W - kSsimWin + 1);
    const int nblocks = (int)((P + kSsimThreads - 1) / kSsimThreads);
    if ((size_t)nblocks > c->cap_ssim) {
        if (c->ssim_part) cudaFree(c->ssim_part);
        c->ssim_part = nullptr;
        c->cap_ssim = 0;
        if (cudaMalloc(&c->ssim_part, sizeof(double) * nblocks) != cudaSuccess) {
            cudaGetLastError();
            return SDL_ERR_WORKSPACE;
        }
        c->cap_ssim = nblocks;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ssim_kernel<<<nblocks, kSsimThreads, 0, st>>>(x, ref, H, W, peak, c->ssim_part);
    ssim_finish_kernel<<<1, 32, 0, st>>>(c->ssim_part, nblocks, P, out);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int sdl_psnr(const float* x, const float* ref, int64_t count, float peak, float* out,
             void* stream) {
    if (!x || !ref || !out || count < 1 || !(peak > 0.f)) return SDL_ERR_ARG;
    psnr_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(x, ref, count, peak, out);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // extern "C"
