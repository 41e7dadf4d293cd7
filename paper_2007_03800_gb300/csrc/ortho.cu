// Orthonormal variant of Algorithm 1 (Remark 1): square orthonormal
// dictionaries (n1 = p1, n2 = p2), codes X_k = T_s(D1^T Y_k D2) (the s
// largest |entries|, no pursuit), and orthogonal-Procrustes updates
// D1 = U V^T of B1 = sum_k Y_k D2 X_k^T (D2 = U2 V2^T of B2 = sum_k Y_k^T D1 X_k).
// B1 and B2 are the sums of the general update (Corollary 1, Result 1); the
// printed SVD argument of Remark 1 carries an extra sum X X^T factor, which
// the trace maximisation behind the Procrustes problem does not have.
//
//   ortho_code_sq_kernel  square shapes compiled ahead (8, 12, 16): a
//                      half-warp per signal with register-blocked Z and C;
//   ortho_code_kernel  any other shape, one warp per signal: Y staged in shared memory,
//                      Z = Y D2, C = D1^T Z, s rounds of warp argmax with
//                      masking (ties to the smallest q), the code, and B1 or
//                      B2 accumulated in warp-private shared memory, combined
//                      in warp order per CTA (deterministic slots);
//   procrustes_kernel  one CTA: one-sided Jacobi SVD of B in FP32 (column
//                      pairs in round-robin order, one warp per pair),
//                      D = U V^T, the objective change 2 (tr(D_old^T B) -
//                      sum sigma) and the RMSE.
#include <algorithm>
#include <cmath>

#include "ctx.cuh"

using namespace sdl;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kOrthoMaxP = 32;       // p1, p2 <= 32
constexpr int kOrthoWarps = 8;       // warps (signals in flight) per CTA
constexpr float kRankRel = 1e-6f;    // smallest / largest singular value (FP32 level)
constexpr float kJacobiTol = 1e-7f;  // rotate while |a_i . a_j| > tol ||a_i|| ||a_j||
constexpr int kMaxSweeps = 30;

__host__ __device__ constexpr int al4(int x) { return (x + 3) & ~3; }

// shared memory (floats): D1 (p1 x n1 column-major), D2 row-major (p2 x n2),
// then per warp Y | Z | C | accumulator (p x n of the side) | 2 energies
struct OrthoLayout {
    int d1, d2, warp0, y, z, c, acc, en, wstride, total;
    __host__ __device__ OrthoLayout(int p1, int p2, int side, int wpc) {
        const int n1 = p1, n2 = p2;
        d1 = 0;
        d2 = d1 + al4(p1 * n1);
        warp0 = d2 + al4(p2 * n2);
        y = 0;
        z = y + al4(p1 * p2);
        c = z + al4(p1 * n2);
        acc = c + al4(n1 * n2);
        const int nacc = side == kSideD1 ? p1 * n1 : side == kSideD2 ? p2 * n2 : 0;
        en = acc + al4(nacc);
        wstride = en + 4;
        total = warp0 + wpc * wstride;
    }
};

template <int SIDE>
__global__ void __launch_bounds__(kOrthoWarps * 32)
    ortho_code_kernel(const float* __restrict__ Y, int p1, int p2, long long N,
                      const float* __restrict__ D1, const float* __restrict__ D2, int s, float eps2,
                      int32_t* __restrict__ support, float* __restrict__ coef,
                      int32_t* __restrict__ nnz, float* __restrict__ res_energy,
                      float* __restrict__ part_f, double* __restrict__ part_d, int* err) {
    extern __shared__ __align__(16) float sm[];
    const int n1 = p1, n2 = p2, P = p1 * p2, Q = n1 * n2;
    const int wpc = blockDim.x >> 5;
    const OrthoLayout L(p1, p2, SIDE, wpc);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* D1s = sm + L.d1;
    float* D2r = sm + L.d2;
    float* wb = sm + L.warp0 + w * L.wstride;
    float* Ys = wb + L.y;
    float* Zs = wb + L.z;
    float* Cs = wb + L.c;
    float* acc = wb + L.acc;
    const int nacc = SIDE == kSideD1 ? p1 * n1 : SIDE == kSideD2 ? p2 * n2 : 0;

    for (int e = threadIdx.x; e < p1 * n1; e += blockDim.x) D1s[e] = D1[e];
    for (int e = threadIdx.x; e < p2 * n2; e += blockDim.x) {
        const int b = e / n2, j = e - b * n2;
        D2r[e] = D2[b + p2 * j];
    }
    for (int e = lane; e < nacc; e += 32) acc[e] = 0.f;
    __syncthreads();

    float e_res = 0.f, e_res_c = 0.f, e_y = 0.f, e_y_c = 0.f;   // compensated sums (lane 0)
    const long long stride = (long long)gridDim.x * wpc;
    for (long long k = (long long)blockIdx.x * wpc + w; k < N; k += stride) {
        // ---- Y_k and ||Y_k||^2
        float ss = 0.f;
        for (int e = lane; e < P; e += 32) {
            const float v = Y[(size_t)k * P + e];
            Ys[e] = v;
            ss = fmaf(v, v, ss);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
        __syncwarp();
        const bool finite = isfinite(ss);
        int cnt = 0;
        float E2 = ss;
        int my_q = -1;
        float my_x = 0.f;
        // a signal already within the error target keeps no entry: skip its correlations
        if (finite && !(eps2 > 0.f && ss <= eps2)) {
            // ---- Z = Y D2 (p1 x n2), C = D1^T Z (entry q = i + n1 j)
            for (int e = lane; e < p1 * n2; e += 32) {
                const int a = e / n2, j = e - a * n2;
                float z = 0.f;
                for (int b = 0; b < p2; ++b) z = fmaf(Ys[a + p1 * b], D2r[b * n2 + j], z);
                Zs[e] = z;
            }
            __syncwarp();
            for (int q = lane; q < Q; q += 32) {
                const int i = q % n1, j = q / n1;
                float c = 0.f;
                for (int a = 0; a < p1; ++a) c = fmaf(D1s[a + p1 * i], Zs[a * n2 + j], c);
                Cs[q] = c;
            }
            __syncwarp();
            // ---- T_s: s rounds of argmax |C| over unmasked entries (with an
            // error-driven stop before a round once ||R||^2 <= eps^2)
            for (int t = 0; t < s; ++t) {
                if (eps2 > 0.f && E2 <= eps2) break;
                float best = 0.f;
                int bq = 0x7fffffff;
                for (int q = lane; q < Q; q += 32) {
                    const float v = fabsf(Cs[q]);
                    if (v > best) { best = v; bq = q; }   // NaN (masked) never wins
                }
                const unsigned M = __reduce_max_sync(kFull, __float_as_uint(best));
                if (M == 0u) break;   // every remaining entry is 0
                const unsigned cand = (__float_as_uint(best) == M) ? (unsigned)bq : 0xffffffffu;
                const int q = (int)__reduce_min_sync(kFull, cand);
                const float x = Cs[q];
                __syncwarp();
                if (lane == 0) Cs[q] = __int_as_float(0x7fc00000);
                if (lane == t) {
                    my_q = q;
                    my_x = x;
                }
                E2 = fmaf(-x, x, E2);
                cnt = t + 1;
                __syncwarp();
            }
        }
        // ---- emit the code (lane l holds pick l)
        if (support && lane < s) {
            support[(size_t)k * s + lane] = lane < cnt ? my_q : -1;
            coef[(size_t)k * s + lane] = lane < cnt ? my_x : 0.f;
        }
        if (lane == 0) {
            if (nnz) nnz[k] = cnt;
            if (res_energy) res_energy[k] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
            if (!finite) record_error(err, SDL_ERR_NONFINITE);
        }
        // ---- fused partial sums (warp-private accumulators)
        if constexpr (SIDE == kSideD1) {
            // B1[a, i_l] += x_l Z[a, j_l]
            for (int l = 0; l < cnt; ++l) {
                const int ql = __shfl_sync(kFull, my_q, l);
                const float xl = __shfl_sync(kFull, my_x, l);
                const int il = ql % n1, jl = ql / n1;
                for (int a = lane; a < p1; a += 32) acc[a * n1 + il] = fmaf(xl, Zs[a * n2 + jl], acc[a * n1 + il]);
                __syncwarp();
            }
        } else if constexpr (SIDE == kSideD2) {
            // B2[b, j_l] += x_l (Y^T D1)[b, i_l]
            for (int l = 0; l < cnt; ++l) {
                const int ql = __shfl_sync(kFull, my_q, l);
                const float xl = __shfl_sync(kFull, my_x, l);
                const int il = ql % n1, jl = ql / n1;
                for (int b = lane; b < p2; b += 32) {
                    float wv = 0.f;
                    for (int a = 0; a < p1; ++a) wv = fmaf(Ys[a + p1 * b], D1s[a + p1 * il], wv);
                    acc[b * n2 + jl] = fmaf(xl, wv, acc[b * n2 + jl]);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && finite) {
            const float ye = fmaxf(E2, 0.f) - e_res_c;
            const float te = e_res + ye;
            e_res_c = (te - e_res) - ye;
            e_res = te;
            const float yy = ss - e_y_c;
            const float ty = e_y + yy;
            e_y_c = (ty - e_y) - yy;
            e_y = ty;
        }
        __syncwarp();
    }
    if constexpr (SIDE != kCodeOnly) {
        float* en = wb + L.en;
        if (lane == 0) {
            en[0] = e_res - e_res_c;
            en[1] = e_y - e_y_c;
        }
        __syncthreads();
        // combine the warps' accumulators in warp order into this CTA's slot
        float* dst = part_f + (size_t)blockIdx.x * nacc;
        for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
            float v = 0.f;
            for (int ww = 0; ww < wpc; ++ww) v += sm[L.warp0 + ww * L.wstride + L.acc + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int ww = 0; ww < wpc; ++ww) d += (double)sm[L.warp0 + ww * L.wstride + L.en + threadIdx.x];
            part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = d;
        }
    }
}

// Square shapes compiled ahead (P = p1 = p2 in {8, 12, 16}): a half-warp
// (16 lanes, a 4 x 4 lane grid) per signal, each lane owning an R x R block
// (R = P / 4) of Z = Y D2 and of C = D1^T Z in registers, so each shared-memory
// operand load feeds R multiply-adds.  Same selection, codes and partial sums
// as ortho_code_kernel; the two half-warps of a warp code different signals
// and keep separate accumulators, combined in a fixed order.
constexpr int kHalfTeams = 2 * kOrthoWarps;   // signals in flight per CTA

template <int P>
struct SqLayout {
    static constexpr int PP = P * P, LDZ = P + 1;
    static constexpr int d1r = 0;                       // D1 row-major (a, i)
    static constexpr int d2r = d1r + al4(PP);           // D2 row-major (b, j)
    static constexpr int team0 = d2r + al4(PP);
    static constexpr int y = 0, z = al4(PP), acc = z + al4(P * LDZ), en = acc + al4(PP);
    static constexpr int tstride = en + 4;
    static constexpr int total = team0 + kHalfTeams * tstride;
};

template <int P, int SIDE>
__global__ void __launch_bounds__(kOrthoWarps * 32)
    ortho_code_sq_kernel(const float* __restrict__ Y, long long N, const float* __restrict__ D1,
                         const float* __restrict__ D2, int s, float eps2, int32_t* __restrict__ support,
                         float* __restrict__ coef, int32_t* __restrict__ nnz,
                         float* __restrict__ res_energy, float* __restrict__ part_f,
                         double* __restrict__ part_d, int* err) {
    using L = SqLayout<P>;
    constexpr int R = P / 4, PP = P * P, LDZ = L::LDZ;
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, half = lane >> 4, l16 = lane & 15;
    const int team = (threadIdx.x >> 5) * 2 + half;
    const unsigned hm = 0xffffu << (16 * half);
    const int li = l16 & 3, lj = l16 >> 2, i0 = li * R, j0 = lj * R;
    float* D1r = sm + L::d1r;
    float* D2r = sm + L::d2r;
    float* tb = sm + L::team0 + team * L::tstride;
    float* Ys = tb + L::y;
    float* Zs = tb + L::z;
    float* acc = tb + L::acc;
    for (int e = threadIdx.x; e < PP; e += blockDim.x) {
        const int r = e / P, c = e - r * P;
        D1r[e] = D1[r + P * c];
        D2r[e] = D2[r + P * c];
    }
    if constexpr (SIDE != kCodeOnly)
        for (int e = l16; e < PP; e += 16) acc[e] = 0.f;
    __syncthreads();

    float e_res = 0.f, e_res_c = 0.f, e_y = 0.f, e_y_c = 0.f;
    const long long stride = (long long)gridDim.x * kHalfTeams;
    // the next signal of this half-warp is loaded into registers while the
    // current one is coded
    constexpr int NV = (PP + 15) / 16;
    float yn[NV];
    {
        const long long k0 = (long long)blockIdx.x * kHalfTeams + team;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int e = l16 + 16 * v;
            yn[v] = (k0 < N && e < PP) ? __ldg(Y + (size_t)k0 * PP + e) : 0.f;
        }
    }
    for (long long k = (long long)blockIdx.x * kHalfTeams + team; k < N; k += stride) {
        float ss = 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int e = l16 + 16 * v;
            if (e < PP) {
                Ys[e] = yn[v];
                ss = fmaf(yn[v], yn[v], ss);
            }
        }
        const long long kn = k + stride;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int e = l16 + 16 * v;
            yn[v] = (kn < N && e < PP) ? __ldg(Y + (size_t)kn * PP + e) : 0.f;
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(hm, ss, o);
        __syncwarp(hm);
        const bool finite = isfinite(ss);
        int cnt = 0;
        float E2 = ss;
        int my_q = -1;
        float my_x = 0.f;
        // a signal already within the error target keeps no entry: skip its correlations
        if (finite && !(eps2 > 0.f && ss <= eps2)) {
            // Z block: rows i0.., cols j0.. of Y D2
            float z[R][R];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) z[r][c] = 0.f;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                float u[R], v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) u[r] = Ys[(i0 + r) + P * b];
#pragma unroll
                for (int c = 0; c < R; ++c) v[c] = D2r[b * P + j0 + c];
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c) z[r][c] = fmaf(u[r], v[c], z[r][c]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) Zs[(i0 + r) * LDZ + j0 + c] = z[r][c];
            __syncwarp(hm);
            // C block: C[i][j] = sum_a D1[a][i] Z[a][j]
            float cv[R][R];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) cv[r][c] = 0.f;
#pragma unroll
            for (int aa = 0; aa < P; ++aa) {
                float u[R], v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) u[r] = D1r[aa * P + i0 + r];
#pragma unroll
                for (int c = 0; c < R; ++c) v[c] = Zs[aa * LDZ + j0 + c];
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c) cv[r][c] = fmaf(u[r], v[c], cv[r][c]);
            }
            // T_s: s rounds of (max |C|, smallest q) over the half-warp, with
            // the error-driven stop
            for (int t = 0; t < s; ++t) {
                if (eps2 > 0.f && E2 <= eps2) break;
                float best = 0.f, bestv = 0.f;
                int bq = 0x7fffffff;
#pragma unroll
                for (int c = 0; c < R; ++c)
#pragma unroll
                    for (int r = 0; r < R; ++r) {           // increasing q = i + P j
                        const float v = fabsf(cv[r][c]);
                        if (v > best) { best = v; bestv = cv[r][c]; bq = (i0 + r) + P * (j0 + c); }
                    }
                const unsigned M = __reduce_max_sync(hm, __float_as_uint(best));
                if (M == 0u) break;
                const unsigned cand = (__float_as_uint(best) == M) ? (unsigned)bq : 0xffffffffu;
                const int q = (int)__reduce_min_sync(hm, cand);
                const int qi = q % P, qj = q / P;
                const int owner = (qi / R) + 4 * (qj / R) + 16 * half;
                const float x = __shfl_sync(hm, bestv, owner);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c)
                        if (i0 + r == qi && j0 + c == qj) cv[r][c] = __int_as_float(0x7fc00000);
                if (l16 == t) {
                    my_q = q;
                    my_x = x;
                }
                E2 = fmaf(-x, x, E2);
                cnt = t + 1;
            }
        }
        if (support && l16 < s) {
            support[(size_t)k * s + l16] = l16 < cnt ? my_q : -1;
            coef[(size_t)k * s + l16] = l16 < cnt ? my_x : 0.f;
        }
        if (l16 == 0) {
            if (nnz) nnz[k] = cnt;
            if (res_energy) res_energy[k] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
            if (!finite) record_error(err, SDL_ERR_NONFINITE);
        }
        if constexpr (SIDE == kSideD1) {
            // B1[a, i_l] += x_l Z[a, j_l], lane a
            for (int l = 0; l < cnt; ++l) {
                const int ql = __shfl_sync(hm, my_q, l + 16 * half);
                const float xl = __shfl_sync(hm, my_x, l + 16 * half);
                const int il = ql % P, jl = ql / P;
                if (l16 < P) acc[l16 * P + il] = fmaf(xl, Zs[l16 * LDZ + jl], acc[l16 * P + il]);
                __syncwarp(hm);
            }
        } else if constexpr (SIDE == kSideD2) {
            // B2[b, j_l] += x_l (Y^T D1)[b, i_l], lane b
            for (int l = 0; l < cnt; ++l) {
                const int ql = __shfl_sync(hm, my_q, l + 16 * half);
                const float xl = __shfl_sync(hm, my_x, l + 16 * half);
                const int il = ql % P, jl = ql / P;
                if (l16 < P) {
                    float wv = 0.f;
#pragma unroll
                    for (int aa = 0; aa < P; ++aa) wv = fmaf(Ys[aa + P * l16], D1r[aa * P + il], wv);
                    acc[l16 * P + jl] = fmaf(xl, wv, acc[l16 * P + jl]);
                }
                __syncwarp(hm);
            }
        }
        if (l16 == 0 && finite) {
            const float ye = fmaxf(E2, 0.f) - e_res_c;
            const float te = e_res + ye;
            e_res_c = (te - e_res) - ye;
            e_res = te;
            const float yy = ss - e_y_c;
            const float ty = e_y + yy;
            e_y_c = (ty - e_y) - yy;
            e_y = ty;
        }
        __syncwarp(hm);
    }
    if constexpr (SIDE != kCodeOnly) {
        if (l16 == 0) {
            tb[L::en] = e_res - e_res_c;
            tb[L::en + 1] = e_y - e_y_c;
        }
        __syncthreads();
        float* dst = part_f + (size_t)blockIdx.x * PP;
        for (int e = threadIdx.x; e < PP; e += blockDim.x) {
            float v = 0.f;
            for (int tt = 0; tt < kHalfTeams; ++tt) v += sm[L::team0 + tt * L::tstride + L::acc + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int tt = 0; tt < kHalfTeams; ++tt)
                d += (double)sm[L::team0 + tt * L::tstride + L::en + threadIdx.x];
            part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = d;
        }
    }
}

template <int P, int SIDE>
int launch_sq(const float* Y, long long N, const float* D1, const float* D2, int s, float eps2,
              int32_t* support, float* coef, int32_t* nnz, float* res, float* part_f,
              double* part_d, int max_slots, int* err, int num_sms, cudaStream_t st) {
    const size_t bytes = sizeof(float) * (size_t)SqLayout<P>::total;
    auto kern = ortho_code_sq_kernel<P, SIDE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kOrthoWarps * 32, bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    bps = std::max(1, std::min(bps, 8));
    const long long need = (N + kHalfTeams - 1) / kHalfTeams;
    long long grid = std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
    if (SIDE != kCodeOnly) grid = std::min<long long>(grid, max_slots);
    kern<<<(int)grid, kOrthoWarps * 32, bytes, st>>>(Y, N, D1, D2, s, eps2, support, coef, nnz,
                                                     res, part_f, part_d, err);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return SIDE == kCodeOnly ? 0 : (int)grid;
}

template <int P>
int launch_sq_side(const float* Y, long long N, const float* D1, const float* D2, int s, float eps2,
                   int32_t* support, float* coef, int32_t* nnz, float* res, float* part_f,
                   double* part_d, int max_slots, int side, int* err, int num_sms,
                   cudaStream_t st) {
    switch (side) {
        case kCodeOnly:
            return launch_sq<P, kCodeOnly>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                           max_slots, err, num_sms, st);
        case kSideD1:
            return launch_sq<P, kSideD1>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                         max_slots, err, num_sms, st);
        default:
            return launch_sq<P, kSideD2>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                         max_slots, err, num_sms, st);
    }
}

// One CTA, 32 * ceil(m/2) threads (m = n rounded up to even): one-sided
// Jacobi SVD of B (p x n row-major, p = n) in FP32 and D = U V^T.  B itself
// is an FP32 sum, so FP32 rotations add no error beyond its own (FP64 is a
// narrow, long-latency pipe on this part: a 12 x 12 FP64 Jacobi took ~0.3 ms).
//   red_f = B, red_d[0] = objective before (sum of residual energies with
//   the old dictionary and these codes).  The old D must be orthonormal: then
//   f(D) = sum ||Y||^2 - 2 tr(D^T B) + sum ||X||^2, and the change is
//   -2 (sum sigma - tr(D_old^T B)) (accumulated in FP64).
__global__ void procrustes_kernel(const float* __restrict__ red_f, const double* __restrict__ red_d,
                                  float* D, int n, double inv_count, double* objective_out,
                                  double* rmse_out, int* err) {
    extern __shared__ __align__(16) float smf[];
    const int m = (n + 1) & ~1;             // even number of columns (a zero column pads)
    float* A = smf;                          // m columns of length n (column-major)
    float* V = A + m * n;                    // m x m (column-major)
    float* sig = V + m * m;                  // m
    int* sched = reinterpret_cast<int*>(sig + m);   // (m - 1) x m/2 column pairs
    __shared__ int s_fail, s_rot;
    __shared__ double s_tr, s_sig;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_fail = 0;
        s_tr = 0.0;
        s_sig = 0.0;
    }
    __syncthreads();
    for (int e = tid; e < m * n; e += nth) {
        const int c = e / n, r = e - c * n;
        const float v = c < n ? red_f[r * n + c] : 0.f;
        A[e] = v;
        if (!isfinite(v)) s_fail = SDL_ERR_NONFINITE;
    }
    for (int e = tid; e < m * m; e += nth) V[e] = (e / m == e % m) ? 1.f : 0.f;
    // tr(D_old^T B)
    if (warp == 0) {
        double t = 0.0;
        for (int e = lane; e < n * n; e += 32) {
            const int r = e / n, c = e - r * n;
            t += (double)D[r + n * c] * (double)red_f[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (lane == 0) s_tr = t;
    }
    __syncthreads();
    // round-robin tournament: in round r, positions w and m-1-w meet; position
    // 0 is fixed and the others rotate (every pair meets once per sweep)
    for (int e = tid; e < (m - 1) * (m / 2); e += nth) {
        const int round = e / (m / 2), w = e - round * (m / 2);
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (m - 1); };
        int ci = player(w), cj = player(m - 1 - w);
        if (ci > cj) {
            const int t = ci;
            ci = cj;
            cj = t;
        }
        sched[e] = ci | (cj << 16);
    }
    __syncthreads();
    // sweeps: m - 1 rounds of m/2 disjoint column pairs
    for (int sweep = 0; sweep < kMaxSweeps && s_fail == 0; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < m - 1; ++round) {
            const int pr = sched[round * (m / 2) + warp];
            const int ci = pr & 0xffff, cj = pr >> 16;
            float al = 0.f, be = 0.f, ga = 0.f;
            for (int r = lane; r < n; r += 32) {
                const float x = A[ci * n + r], y = A[cj * n + r];
                al = fmaf(x, x, al);
                be = fmaf(y, y, be);
                ga = fmaf(x, y, ga);
            }
            if (n > 16) {
                al += __shfl_xor_sync(kFull, al, 16);
                be += __shfl_xor_sync(kFull, be, 16);
                ga += __shfl_xor_sync(kFull, ga, 16);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                al += __shfl_xor_sync(kFull, al, o);
                be += __shfl_xor_sync(kFull, be, o);
                ga += __shfl_xor_sync(kFull, ga, o);
            }
            // rotate while ga^2 > tol^2 al be; the angle only needs to be
            // approximate (fast reciprocal / square root): a rotation is
            // orthogonal for any (c, s) with c^2 + s^2 = 1 to rounding
            if (ga != 0.f && ga * ga > kJacobiTol * kJacobiTol * al * be) {
                const float zeta = __fdividef(be - al, 2.f * ga);
                float t;
                if (fabsf(zeta) < 1e18f) {
                    const float q = fmaf(zeta, zeta, 1.f);
                    t = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + q * rsqrtf(q));
                } else {
                    t = __fdividef(0.5f, zeta);
                }
                const float c = rsqrtf(fmaf(t, t, 1.f)), sn = c * t;
                for (int r = lane; r < n; r += 32) {
                    const float x = A[ci * n + r], y = A[cj * n + r];
                    A[ci * n + r] = c * x - sn * y;
                    A[cj * n + r] = sn * x + c * y;
                }
                for (int r = lane; r < m; r += 32) {
                    const float x = V[ci * m + r], y = V[cj * m + r];
                    V[ci * m + r] = c * x - sn * y;
                    V[cj * m + r] = sn * x + c * y;
                }
                if (lane == 0) atomicAdd(&s_rot, 1);
            }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (rot == 0) break;
    }
    for (int c = tid; c < m; c += nth) {
        float t = 0.f;
        for (int r = 0; r < n; ++r) t = fmaf(A[c * n + r], A[c * n + r], t);
        sig[c] = sqrtf(t);
    }
    __syncthreads();
    if (tid == 0 && s_fail == 0) {
        float smax = 0.f, smin = INFINITY;
        int pad = m != n ? 1 : 0;   // the padding column carries one zero singular value
        double ssum = 0.0;
        for (int c = 0; c < m; ++c) {
            smax = fmaxf(smax, sig[c]);
            ssum += (double)sig[c];
        }
        for (int c = 0; c < m; ++c) {
            if (pad && sig[c] == 0.f) {
                pad = 0;
                continue;
            }
            smin = fminf(smin, sig[c]);
        }
        if (!(smax > 0.f) || !(smin > kRankRel * smax)) s_fail = SDL_ERR_SINGULAR;
        s_sig = ssum;
    }
    __syncthreads();
    const bool ok = s_fail == 0;
    if (ok) {
        for (int e = tid; e < n * n; e += nth) {
            const int r = e / n, c = e - r * n;   // D[r, c] = sum_i U[r, i] V[c, i]
            float d = 0.f;
            for (int i = 0; i < m; ++i)
                if (sig[i] > 0.f) d = fmaf(A[i * n + r] / sig[i], V[i * m + c], d);
            D[r + n * c] = d;
        }
    }
    if (tid == 0) {
        if (!ok) record_error(err, s_fail);
        const double before = red_d[0];
        const double after = ok ? before - 2.0 * (s_sig - s_tr) : before;
        if (objective_out) {
            objective_out[0] = before;
            objective_out[1] = after;
        }
        if (rmse_out) rmse_out[0] = sqrt(fmax(after, 0.0) * inv_count);
    }
}

size_t code_smem(int p1, int p2, int side, int wpc) {
    return sizeof(float) * (size_t)OrthoLayout(p1, p2, side, wpc).total;
}

template <int SIDE>
int launch_ortho_code_impl(const float* Y, int p1, int p2, long long N, const float* D1,
                           const float* D2, int s, float eps2, int32_t* support, float* coef, int32_t* nnz,
                           float* res, float* part_f, double* part_d, int max_slots, int* err,
                           int num_sms, cudaStream_t st) {
    const size_t bytes = code_smem(p1, p2, SIDE, kOrthoWarps);
    auto kern = ortho_code_kernel<SIDE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kOrthoWarps * 32, bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    bps = std::max(1, std::min(bps, 8));
    const long long need = (N + kOrthoWarps - 1) / kOrthoWarps;
    long long grid = std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
    if (SIDE != kCodeOnly) grid = std::min<long long>(grid, max_slots);
    kern<<<(int)grid, kOrthoWarps * 32, bytes, st>>>(Y, p1, p2, N, D1, D2, s, eps2, support, coef,
                                                     nnz, res, part_f, part_d, err);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return SIDE == kCodeOnly ? 0 : (int)grid;
}

}  // namespace

namespace sdl {

bool ortho_shape_supported(int p1, int p2, int s) {
    return p1 >= 1 && p2 >= 1 && p1 <= kOrthoMaxP && p2 <= kOrthoMaxP && s >= 1 && s <= 32 &&
           s <= p1 * p2;
}

int launch_ortho_code(const float* Y, int p1, int p2, long long N, const float* D1,
                      const float* D2, int s, float eps2, int32_t* support, float* coef, int32_t* nnz,
                      float* res, float* part_f, double* part_d, int max_slots, int side,
                      int* err, int num_sms, cudaStream_t st) {
    // compiled square shapes (s <= 16: the half-warp holds one pick per lane)
    if (p1 == p2 && s <= 16 && (p1 == 8 || p1 == 12 || p1 == 16)) {
        if (p1 == 8)
            return launch_sq_side<8>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                     max_slots, side, err, num_sms, st);
        if (p1 == 12)
            return launch_sq_side<12>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                      max_slots, side, err, num_sms, st);
        return launch_sq_side<16>(Y, N, D1, D2, s, eps2, support, coef, nnz, res, part_f, part_d,
                                  max_slots, side, err, num_sms, st);
    }
    switch (side) {
        case kCodeOnly:
            return launch_ortho_code_impl<kCodeOnly>(Y, p1, p2, N, D1, D2, s, eps2, support, coef, nnz,
                                                     res, part_f, part_d, max_slots, err, num_sms, st);
        case kSideD1:
            return launch_ortho_code_impl<kSideD1>(Y, p1, p2, N, D1, D2, s, eps2, support, coef, nnz,
                                                   res, part_f, part_d, max_slots, err, num_sms, st);
        case kSideD2:
            return launch_ortho_code_impl<kSideD2>(Y, p1, p2, N, D1, D2, s, eps2, support, coef, nnz,
                                                   res, part_f, part_d, max_slots, err, num_sms, st);
        default:
            return SDL_ERR_ARG;
    }
}

int launch_procrustes(const float* red_f, const double* red_d, float* D, int n, double inv_count,
                      double* objective_out, double* rmse_out, int* err, cudaStream_t st) {
    const int m = (n + 1) & ~1;
    const size_t bytes = sizeof(float) * ((size_t)m * n + (size_t)m * m + m) +
                         sizeof(int) * (size_t)(m - 1) * (m / 2);
    if (cudaFuncSetAttribute(procrustes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return SDL_ERR_CUDA;
    procrustes_kernel<<<1, 32 * (m / 2), bytes, st>>>(red_f, red_d, D, n, inv_count, objective_out,
                                                      rmse_out, err);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // namespace sdl

// ------------------------------------------------------------------ C ABI
extern "C" {

int sdl_ortho_sparse_code(sdl_ctx* c, const float* Y, int p1, int p2, int64_t N, const float* D1,
                          const float* D2, int s, float eps, int32_t* support, float* coef,
                          int32_t* nnz, float* res_energy, void* stream) {
    if (!c || N < 0 || (N > 0 && (!Y || !D1 || !D2 || !support || !coef || !nnz)))
        return SDL_ERR_ARG;
    if (!ortho_shape_supported(p1, p2, s)) return SDL_ERR_ARG;
    if (N == 0) return SDL_OK;
    DeviceGuard g(c->device);
    Trace tr(c, kOrthoCode, (cudaStream_t)stream);
    const int rc = launch_ortho_code(Y, p1, p2, N, D1, D2, s, eps > 0.f ? eps * eps : 0.f, support,
                                     coef, nnz, res_energy,
                                     nullptr, nullptr, 0, kCodeOnly, c->err, c->num_sms,
                                     (cudaStream_t)stream);
    return rc < 0 ? rc : SDL_OK;
}

int sdl_ortho_iterate(sdl_ctx* c, const float* Y, int p1, int p2, int64_t N, float* D1, float* D2,
                      int s, float eps, int32_t* support, float* coef, int32_t* nnz,
                      double* rmse_out, void* stream) {
    if (!c || N < 1 || !Y || !D1 || !D2 || !support || !coef || !nnz) return SDL_ERR_ARG;
    if (!ortho_shape_supported(p1, p2, s)) return SDL_ERR_ARG;
    DeviceGuard g(c->device);
    int rc = ctx_workspace(c, p1, p2, p1, p2);
    if (rc != SDL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int max_slots = max_partial_slots(c->num_sms);
    const double inv_count = 1.0 / ((double)p1 * p2 * (double)N);
    for (int side = kSideD1; side <= kSideD2; ++side) {
        const int p = side == kSideD1 ? p1 : p2;
        int slots;
        {
            Trace tr(c, kOrthoCode, st);
            slots = launch_ortho_code(Y, p1, p2, N, D1, D2, s, eps > 0.f ? eps * eps : 0.f,
                                      side == kSideD2 ? support : nullptr,
                                      coef, nnz, nullptr, c->part_f, c->part_d, max_slots, side,
                                      c->err, c->num_sms, st);
        }
        if (slots < 0) return slots;
        {
            Trace tr(c, kReduce, st);
            launch_reduce_partials(c->part_f, c->part_d, slots, p * p, c->red_f, c->red_d, st);
        }
        Trace tr(c, kProcrustes, st);
        rc = launch_procrustes(c->red_f, c->red_d, side == kSideD1 ? D1 : D2, p, inv_count, nullptr,
                               rmse_out ? rmse_out + (side - kSideD1) : nullptr, c->err, st);
        if (rc != SDL_OK) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // extern "C"
