// Precision extension: the correlations C0 = D1^T Y_k D2 of every signal as
// ONE BF16 tensor-core GEMM, and the normal-equation solve in FP64.
//
// Correlations: with the column-order vec of Sec. I, C0_k = (D2 (x) D1)^T vec(Y_k),
// so C0 for all signals is Yvec (N x p1p2) times the Kronecker dictionary
// (p1p2 x n1n2): A = vec(Y_k) rows (BF16), B = rows of (D2 (x) D1)^T (BF16),
// FP32 accumulation in tensor memory (tc_gemm.cu).  Each entry is within
// 2^-7 (1 + small) ||Y_k||_F of the FP32 value (BF16 rounding of both
// operands, unit-norm Kronecker atoms, Cauchy-Schwarz); the coding kernel
// re-scores in FP32 every entry that close to the running maximum, so its
// picks are the FP32 picks.
#include <cuda_bf16.h>

#include "ctx.cuh"

using namespace sdl;

namespace {

__global__ void y_to_bf16_kernel(const float* __restrict__ Y, long long N, int P, int Kp,
                                 __nv_bfloat16* __restrict__ Yb) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * Kp) return;
    const long long k = e / Kp;
    const int c = (int)(e - k * Kp);
    Yb[e] = __float2bfloat16_rn(c < P ? Y[k * P + c] : 0.f);
}

// row q = i + n1*j of (D2 (x) D1)^T: entry (a + p1*b) = D1[a, i] D2[b, j]
__global__ void kron_bf16_kernel(const float* __restrict__ D1, int p1, int n1,
                                 const float* __restrict__ D2, int p2, int n2, int Kp,
                                 __nv_bfloat16* __restrict__ KT) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)n1 * n2 * Kp;
    if (e >= total) return;
    const int q = (int)(e / Kp), c = (int)(e - (long long)q * Kp);
    float v = 0.f;
    if (c < p1 * p2) {
        const int i = q % n1, j = q / n1, aa = c % p1, b = c / p1;
        v = D1[aa + p1 * i] * D2[b + p2 * j];
    }
    KT[e] = __float2bfloat16_rn(v);
}

}  // namespace

namespace sdl {

// Yb must hold N x Kp BF16 (Kp = p1p2 rounded up to 8); filled when fill_y.
int tc_correlations(const float* Y, long long N, int p1, int p2, const float* D1, int n1,
                    const float* D2, int n2, __nv_bfloat16* Yb, bool fill_y, __nv_bfloat16* KT,
                    float* C0, int* err, cudaStream_t st) {
    const int P = p1 * p2, Kp = (P + 7) & ~7, Q = n1 * n2;
    if (fill_y)
        y_to_bf16_kernel<<<(unsigned)((N * Kp + 255) / 256), 256, 0, st>>>(Y, N, P, Kp, Yb);
    kron_bf16_kernel<<<(unsigned)(((long long)Q * Kp + 255) / 256), 256, 0, st>>>(D1, p1, n1, D2, p2,
                                                                                  n2, Kp, KT);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return tc_gemm(Yb, Kp, KT, Kp, (int)N, Q, Kp, 1.f, nullptr, 0, C0, Q, 0, nullptr, 0, nullptr,
                   0, nullptr, 0, err, st);
}

}  // namespace sdl
