// Precision extension: the correlations C0 = D1^T Y_k D2 of every signal on
// the BF16 tensor cores, and the normal-equation solve in FP64.
//
// Correlations: with the column-order vec of Sec. I, C0_k = (D2 (x) D1)^T vec(Y_k),
// so C0 for all signals is Yvec (N x p1p2) times the Kronecker dictionary
// (p1p2 x n1n2).  Both operands are split into BF16 high and low parts
// (y = yh + yl + ey, |ey| <= 2^-16 |y|; likewise k), and the three products
// yh kh + yh kl + yl kh run as ONE tensor-core GEMM with FP32 accumulation in
// tensor memory (tc_gemm.cu, three operand pairs in one accumulator).  The
// dropped terms are at most (3 + 2^-6) 2^-16 |y||k| per product, the FP32
// products of D1 and D2 entries add 2^-24 |y||k|, and the 3 p1p2 FP32
// additions at most 3 p1p2 2^-23 of the sum of |terms|; with unit-norm
// Kronecker atoms and Cauchy-Schwarz every entry is within
//   c0_split_err_rel(p1 p2) * ||Y_k||_F
// of its exact value.  The coding kernel re-scores in FP32 every entry within
// three times that of the approximate maximum, so its picks are the FP32 picks.
#include <cuda_bf16.h>

#include "ctx.cuh"

using namespace sdl;

namespace {

// hi/lo BF16 split of Y (rows padded to Kp with zeros)
__global__ void y_split_kernel(const float* __restrict__ Y, long long N, int P, int Kp,
                               __nv_bfloat16* __restrict__ Yh, __nv_bfloat16* __restrict__ Yl) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= N * Kp) return;
    const long long k = e / Kp;
    const int c = (int)(e - k * Kp);
    const float y = c < P ? Y[k * P + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(y);
    Yh[e] = h;
    Yl[e] = __float2bfloat16_rn(y - __bfloat162float(h));
}

// row q = i + n1*j of (D2 (x) D1)^T: entry (a + p1*b) = D1[a, i] D2[b, j], split
__global__ void kron_split_kernel(const float* __restrict__ D1, int p1, int n1,
                                  const float* __restrict__ D2, int p2, int n2, int Kp,
                                  __nv_bfloat16* __restrict__ Kh, __nv_bfloat16* __restrict__ Kl) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)n1 * n2 * Kp;
    if (e >= total) return;
    const int q = (int)(e / Kp), c = (int)(e - (long long)q * Kp);
    float v = 0.f;
    if (c < p1 * p2) {
        const int i = q % n1, j = q / n1, aa = c % p1, b = c / p1;
        v = D1[aa + p1 * i] * D2[b + p2 * j];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Kh[e] = h;
    Kl[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

}  // namespace

namespace sdl {

float c0_split_err_rel(int p1p2) {
    const int Kp = (p1p2 + 7) & ~7;
    return (float)((3.0 + 1.0 / 64) * 0x1p-16 + 0x1p-24 + 3.0 * Kp * 0x1p-23);
}

// Yb must hold 2 x N x Kp BF16 (Kp = p1p2 rounded up to 8), KT 2 x n1n2 x Kp;
// Yb is filled when fill_y.
int tc_correlations(const float* Y, long long N, int p1, int p2, const float* D1, int n1,
                    const float* D2, int n2, __nv_bfloat16* Yb, bool fill_y, __nv_bfloat16* KT,
                    float* C0, int* err, cudaStream_t st) {
    const int P = p1 * p2, Kp = (P + 7) & ~7, Q = n1 * n2;
    __nv_bfloat16* Yh = Yb;
    __nv_bfloat16* Yl = Yb + (size_t)N * Kp;
    __nv_bfloat16* Kh = KT;
    __nv_bfloat16* Kl = KT + (size_t)Q * Kp;
    if (fill_y)
        y_split_kernel<<<(unsigned)((N * Kp + 255) / 256), 256, 0, st>>>(Y, N, P, Kp, Yh, Yl);
    kron_split_kernel<<<(unsigned)(((long long)Q * Kp + 255) / 256), 256, 0, st>>>(D1, p1, n1, D2,
                                                                                   p2, n2, Kp, Kh, Kl);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    const void* A[3] = {Yh, Yh, Yl};
    const void* B[3] = {Kh, Kl, Kh};
    return tc_gemm_terms(A, Kp, B, Kp, 3, (int)N, Q, Kp, 1.f, nullptr, 0, C0, Q, 0, nullptr, 0,
                         nullptr, 0, nullptr, 0, err, st);
}

}  // namespace sdl
