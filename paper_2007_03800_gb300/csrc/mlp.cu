// Learned support proposal: a two-layer network (p1*p2 -> hidden, GELU ->
// n1*n2 scores) trained on the GPU on (signal, 2D-OMP support) pairs, whose
// top-k scores shortlist the atom pairs that 2D-OMP then searches.
//
//   x = vec(Y)/||Y||,  h = GELU(W1 x + b1),  z = W2 h + b2
//   loss = mean_b sum_q softplus(z) - t z   (t: multi-hot OMP support)
//
// Forward and backward run as tcgen05 GEMMs (tc_gemm.cu) with fused
// epilogues; this file holds the element-wise kernels (input scaling, the
// loss gradient, bias-gradient reductions, Adam), the warp top-k, the
// shortlist 2D-OMP kernel with its fallback test, and the deterministic
// compaction of the fallback signals.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <utility>
#include <vector>

#include "ctx.cuh"

using namespace sdl;
using bf16 = __nv_bfloat16;

struct sdl_mlp {
    sdl_ctx* ctx = nullptr;
    int P = 0, H = 0, Q = 0, Kp = 0, Bmax = 0, step = 0;
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
    float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2;
    float *gW1, *gb1, *gW2, *gb2;
    bf16 *W1b, *W2b, *W2Tb;
    bf16 *Xb, *XTb, *Hb, *HTb, *dZb, *dZTb, *dPreTb;
    float *pre, *Z, *lossp;
    char* mem = nullptr;
};

namespace {

constexpr unsigned kFull = 0xffffffffu;

// x = vec(Y_k)/||Y_k|| as BF16 rows (zero padded to Kp), optional transposed copy
__global__ void prep_input_kernel(const float* __restrict__ Y, long long N, int P, int Kp,
                                  bf16* __restrict__ X, int ldx, bf16* __restrict__ XT, int ldt) {
    const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const float* y = Y + (size_t)k * P;
    float ss = 0.f;
    for (int e = lane; e < P; e += 32) ss = fmaf(y[e], y[e], ss);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
    const float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
    for (int e = lane; e < Kp; e += 32) {
        const bf16 v = __float2bfloat16_rn(e < P ? y[e] * inv : 0.f);
        X[(size_t)k * ldx + e] = v;
        if (XT) XT[(size_t)e * ldt + k] = v;
    }
}

// dz = (sigmoid(z) - t) * scale, loss terms softplus(z) - t z; one block per row
__global__ void bce_kernel(const float* __restrict__ Z, int ldz, const int32_t* __restrict__ sup,
                           int s, int Q, float scale, bf16* __restrict__ dZ, int lddz,
                           bf16* __restrict__ dZT, int lddt, float* __restrict__ lossp) {
    __shared__ int ssup[32];
    __shared__ float red[32];
    const int b = blockIdx.x;
    if (threadIdx.x < s) ssup[threadIdx.x] = sup[(size_t)b * s + threadIdx.x];
    __syncthreads();
    float acc = 0.f;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        float t = 0.f;
        for (int l = 0; l < s; ++l) t = (ssup[l] == q) ? 1.f : t;
        const float z = Z[(size_t)b * ldz + q];
        acc += fmaxf(z, 0.f) - t * z + log1pf(expf(-fabsf(z)));
        const float g = (1.f / (1.f + expf(-z)) - t) * scale;
        const bf16 gb = __float2bfloat16_rn(g);
        dZ[(size_t)b * lddz + q] = gb;
        dZT[(size_t)q * lddt + b] = gb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        lossp[b] = t;
    }
}

// out[r] = sum_c M[r, c] (BF16 rows), one warp per row, fixed order
__global__ void rowsum_kernel(const bf16* __restrict__ M, int ld, int R, int C,
                              float* __restrict__ out) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    float acc = 0.f;
    for (int c = lane; c < C; c += 32) acc += __bfloat162float(M[(size_t)r * ld + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) out[r] = acc;
}

__global__ void sum_kernel(const float* __restrict__ x, int n, float scale, float* __restrict__ out) {
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += 32) acc += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (threadIdx.x == 0) out[0] = acc * scale;
}

// Adam on FP32 master weights; refresh the BF16 copy (and its transpose)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int rows, int cols,
                            float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                            bf16* __restrict__ pb, bf16* __restrict__ pbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pn = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pn;
    const bf16 b = __float2bfloat16_rn(pn);
    if (pb) pb[i] = b;
    if (pbT) pbT[(size_t)(i % cols) * rows + i / cols] = b;
}

__global__ void to_bf16_kernel(const float* __restrict__ p, int rows, int cols,
                               bf16* __restrict__ pb, bf16* __restrict__ pbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const bf16 b = __float2bfloat16_rn(p[i]);
    if (pb) pb[i] = b;
    if (pbT) pbT[(size_t)(i % cols) * rows + i / cols] = b;
}

// ---------------------------------------------------------------- top-k
// order-preserving 16-bit key of a float (larger float -> larger key)
__device__ __forceinline__ unsigned key16(float f) {
    unsigned u = __float_as_uint(f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return u >> 16;
}

// Per signal: the k1 best scores (the shortlist) and the next k2 - k1 (the
// fallback check set), ranked by 16-bit key then by smaller pair index; each
// of the two sets is written in increasing pair index.
// One warp per signal; lane holds scores q = lane + 32 e.
template <int EQ>
__global__ void topk_kernel(const float* __restrict__ Z, int ldz, long long N, int Q, int k1,
                            int k2, int32_t* __restrict__ out) {
    const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    unsigned key[EQ];
#pragma unroll
    for (int e = 0; e < EQ; ++e) {
        const int q = lane + 32 * e;
        const float z = (q < Q) ? Z[(size_t)k * ldz + q] : 0.f;
        key[e] = (q < Q && z == z) ? key16(z) + 1u : 0u;   // 0 = no entry (past Q, or NaN)
    }
    auto count_ge = [&](unsigned t) {
        int c = 0;
#pragma unroll
        for (int e = 0; e < EQ; ++e) c += key[e] >= t ? 1 : 0;
        return (int)__reduce_add_sync(kFull, (unsigned)c);
    };
    // largest threshold with at least kk keys >= it
    auto threshold = [&](int kk) {
        unsigned t = 0;
        for (int bit = 16; bit >= 0; --bit) {
            const unsigned c = t | (1u << bit);
            if (count_ge(c) >= kk) t = c;
        }
        return t;
    };
    // membership masks of the top-kk set (ties at the threshold by smaller q)
    auto select = [&](int kk) {
        const unsigned t = threshold(kk);
        unsigned mask = 0;
        int above = 0;
#pragma unroll
        for (int e = 0; e < EQ; ++e) {
            if (key[e] > t) mask |= 1u << e;
            above += key[e] > t ? 1 : 0;
        }
        int need = kk - (int)__reduce_add_sync(kFull, (unsigned)above);
#pragma unroll
        for (int e = 0; e < EQ; ++e) {      // q = lane + 32 e ascending: e outer, lane inner
            const bool eq = key[e] == t && t > 0;
            const unsigned bal = __ballot_sync(kFull, eq);
            const int rank = __popc(bal & ((1u << lane) - 1u));
            if (eq && rank < need) mask |= 1u << e;
            need -= min(need, __popc(bal));
        }
        return mask;
    };
    const unsigned m1 = select(k1);
    const unsigned m2 = k2 > k1 ? select(k2) & ~m1 : 0u;   // no check set: one bisection
    int base = 0;
    int32_t* o = out + (size_t)k * k2;
    for (int pass = 0; pass < 2; ++pass) {
        const unsigned msk = pass == 0 ? m1 : m2;
        if (pass == 1) base = k1;
        int written = 0;
#pragma unroll
        for (int e = 0; e < EQ; ++e) {
            const bool on = (msk >> e) & 1u;
            const unsigned bal = __ballot_sync(kFull, on);
            if (on) o[base + written + __popc(bal & ((1u << lane) - 1u))] = lane + 32 * e;
            written += __popc(bal);
        }
        const int lim = pass == 0 ? k1 : k2;
        for (int p = base + written + lane; p < lim; p += 32) o[p] = -1;   // fewer valid scores
    }
}

// ---------------------------------------------------------------- shortlist OMP
// fallback test: a signal whose final residual correlates with some
// unselected pair more strongly than this fraction of its weakest greedy
// score is coded again by the full coder
constexpr float kCheckMargin = 0.7f;
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// 2D-OMP restricted to the k1 shortlisted pairs (lane l owns candidate l),
// the same greedy rule, Cholesky and energy identity as the full coder.
// Fallback test: after the last pick, the residual's correlation with every
// pair not picked, C0 - sum_l x_l G1[:, i_l] G2[j_l, :]; if one exceeds
// kCheckMargin x the weakest pick's score at its step, plain 2D-OMP might
// have taken a pair the shortlist missed: the signal is flagged.
template <int P1, int P2, int N1, int N2, int S>
__global__ void __launch_bounds__(256) shortlist_omp_kernel(
    const float* __restrict__ Y, long long N, const float* __restrict__ D1,
    const float* __restrict__ D2, const float* __restrict__ G1, const float* __restrict__ G2,
    const int32_t* __restrict__ cand, int k1, int k2, int32_t* __restrict__ support,
    float* __restrict__ coef, int32_t* __restrict__ nnz, float* __restrict__ res_energy,
    int32_t* __restrict__ flag) {
    constexpr int PP = P1 * P2;
    __shared__ float D1c[N1 * P1];       // column i contiguous
    __shared__ float D2r[P2 * N2];       // row b contiguous
    __shared__ float G1s[N1 * N1], G2s[N2 * N2];
    __shared__ float Ysh[8][PP];
    __shared__ float Zsh[8][P1 * N2];
    for (int e = threadIdx.x; e < N1 * P1; e += blockDim.x) D1c[e] = D1[e];
    for (int e = threadIdx.x; e < P2 * N2; e += blockDim.x) {
        const int b = e / N2, j = e % N2;
        D2r[e] = D2[b + P2 * j];
    }
    for (int e = threadIdx.x; e < N1 * N1; e += blockDim.x) G1s[e] = G1[e];
    for (int e = threadIdx.x; e < N2 * N2; e += blockDim.x) G2s[e] = G2[e];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* Ys = Ysh[w];
    float* Zs = Zsh[w];
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long k = (long long)blockIdx.x * (blockDim.x >> 5) + w; k < N; k += stride) {
        float ss = 0.f;
        for (int e = lane; e < PP; e += 32) {
            const float v = Y[(size_t)k * PP + e];
            Ys[e] = v;
            ss = fmaf(v, v, ss);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
        __syncwarp();
        for (int e = lane; e < P1 * N2; e += 32) {
            const int a = e / N2, j = e % N2;
            float z = 0.f;
#pragma unroll
            for (int b = 0; b < P2; ++b) z = fmaf(Ys[a + P1 * b], D2r[b * N2 + j], z);
            Zs[e] = z;
        }
        __syncwarp();
        // lane's shortlist candidate
        const int q = lane < k1 ? cand[(size_t)k * k2 + lane] : -1;
        const int ci = q >= 0 ? q % N1 : 0, cj = q >= 0 ? q / N1 : 0;
        float c0 = 0.f;
#pragma unroll
        for (int a = 0; a < P1; ++a) c0 = fmaf(D1c[ci * P1 + a], Zs[a * N2 + cj], c0);
        if (q < 0) c0 = __int_as_float(0x7fc00000);
        int si[S], sj[S];
        float xs[S], yv[S], Lrow[S], Lcol[S];
#pragma unroll
        for (int m = 0; m < S; ++m) {
            si[m] = 0; sj[m] = 0; xs[m] = 0.f; yv[m] = 0.f; Lrow[m] = 0.f; Lcol[m] = 0.f;
        }
        float myinvd = 0.f, myy = 0.f, myx = 0.f;
        int myi = 0, myj = 0, cnt = 0;
        float E2 = ss, weakest = INFINITY;
        bool go = isfinite(ss);
        sfor<0, S>([&](auto tc) {
            constexpr int t = decltype(tc)::value;
            if (!go) return;
            float sc = c0;
#pragma unroll
            for (int l = 0; l < t; ++l)
                sc = fmaf(-xs[l] * G1s[ci * N1 + si[l]], G2s[sj[l] * N2 + cj], sc);
            const float v = fabsf(sc);
            const float vv = (v == v) ? v : 0.f;             // masked / padding lanes: NaN
            const unsigned M = __reduce_max_sync(kFull, __float_as_uint(vv));
            if (M == 0u) { go = false; return; }
            const unsigned cq = (__float_as_uint(vv) == M && q >= 0) ? (unsigned)q : 0xffffffffu;
            const unsigned qs = __reduce_min_sync(kFull, cq);
            const int owner = __ffs(__ballot_sync(kFull, (unsigned)q == qs)) - 1;
            const float b = __shfl_sync(kFull, c0, owner);
            if (lane == owner) c0 = __int_as_float(0x7fc00000);
            const int it = (int)(qs % N1), jt = (int)(qs / N1);
            float r = 0.f;
            if (lane < t) r = G1s[it * N1 + myi] * G2s[jt * N2 + myj];
            const float Att = G1s[it * N1 + it] * G2s[jt * N2 + jt];
            float ww = 0.f, wy = 0.f;
#pragma unroll
            for (int m = 0; m < t; ++m) {
                const float wm = __shfl_sync(kFull, r * myinvd, m);
                r = fmaf(-Lrow[m], wm, r);
                ww = fmaf(wm, wm, ww);
                wy = fmaf(wm, yv[m], wy);
                if (lane == t) Lrow[m] = wm;
                if (lane == m) Lcol[t] = wm;
            }
            const float d = Att - ww;
            if (!(d > kPivotRel * Att)) { go = false; return; }
            const float inv = rsqrtf(d);
            const float yt = (b - wy) * inv;
            yv[t] = yt;
            si[t] = it;
            sj[t] = jt;
            if (lane == t) {
                Lrow[t] = d * inv;
                myinvd = inv;
                myy = yt;
                myi = it;
                myj = jt;
            }
            float rb = myy;
#pragma unroll
            for (int kk = t; kk >= 0; --kk) {
                const float xk = __shfl_sync(kFull, rb * myinvd, kk);
                rb = fmaf(-Lcol[kk], xk, rb);
                xs[kk] = xk;
            }
            E2 = fmaf(-yt, yt, E2);
            weakest = fminf(weakest, __uint_as_float(M));
            cnt = t + 1;
        });
#pragma unroll
        for (int m = 0; m < S; ++m)
            if (lane == m) myx = xs[m];
        // fallback test over every pair not picked (lane takes q = lane + 32 e)
        float ve = 0.f;
        if (cnt == S) {
            for (int qq = lane; qq < N1 * N2; qq += 32) {
                const int i = qq % N1, j = qq / N1;
                bool picked = false;
#pragma unroll
                for (int l = 0; l < S; ++l) picked |= (si[l] == i && sj[l] == j);
                if (picked) continue;
                float sce = 0.f;
#pragma unroll
                for (int a = 0; a < P1; ++a) sce = fmaf(D1c[i * P1 + a], Zs[a * N2 + j], sce);
#pragma unroll
                for (int l = 0; l < S; ++l) sce = fmaf(-xs[l] * G1s[i * N1 + si[l]], G2s[sj[l] * N2 + j], sce);
                ve = fmaxf(ve, fabsf(sce));
            }
        }
        const float maxe = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(ve)));
        const bool fb = !isfinite(ss) || (cnt == S && maxe > kCheckMargin * weakest);
        if (lane < S) {
            support[(size_t)k * S + lane] = lane < cnt ? myi + N1 * myj : -1;
            coef[(size_t)k * S + lane] = lane < cnt ? myx : 0.f;
        }
        if (lane == 0) {
            nnz[k] = cnt;
            if (res_energy) res_energy[k] = fmaxf(E2, 0.f);
            flag[k] = fb ? 1 : 0;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- compaction
constexpr int kScanBlock = 1024;

__global__ void count_flags_kernel(const int32_t* __restrict__ flag, long long N,
                                   int* __restrict__ blockcnt) {
    __shared__ int wsum[32];
    const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
    const int f = (i < N && flag[i]) ? 1 : 0;
    const int c = __popc(__ballot_sync(kFull, f));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) t += wsum[w];
        blockcnt[blockIdx.x] = t;
    }
}

__global__ void scan_counts_kernel(int* __restrict__ blockcnt, int nblocks, int* __restrict__ total) {
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < nblocks; ++b) {
            const int c = blockcnt[b];
            blockcnt[b] = run;
            run += c;
        }
        total[0] = run;
    }
}

__global__ void write_index_kernel(const int32_t* __restrict__ flag, long long N,
                                   const int* __restrict__ blockoff, int32_t* __restrict__ idx) {
    __shared__ int woff[32];
    const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int f = (i < N && flag[i]) ? 1 : 0;
    const unsigned bal = __ballot_sync(kFull, f);
    if (lane == 0) woff[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int ww = 0; ww < kScanBlock / 32; ++ww) {
            const int c = woff[ww];
            woff[ww] = run;
            run += c;
        }
    }
    __syncthreads();
    if (f) idx[blockoff[blockIdx.x] + woff[w] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
}

// ---------------------------------------------------------------- RMSE guard
// The plain coder judges the learned one on a strided sample of the signals:
// if the learned codes' RMSE there exceeds the plain coder's by more than 1 %,
// every signal is coded again by the plain coder.
constexpr double kGuardRmseRatio = 1.01;
constexpr int kGuardThreads = 1024;
constexpr long long kGuardMinSample = 4096;

__global__ void sample_index_kernel(int32_t* __restrict__ idx, int m, long long stride,
                                    int* __restrict__ count) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m) idx[r] = (int32_t)(r * stride);
    if (r == 0) *count = m;
}

// fixed-order FP64 sums of the two residual energies over the sample
__global__ void __launch_bounds__(kGuardThreads)
    guard_kernel(const float* __restrict__ plainE, const float* __restrict__ learnedE,
                 const int32_t* __restrict__ idx, int m, long long N, int P, int* __restrict__ recode_count,
                 int32_t* __restrict__ n_fallback, float* __restrict__ guard_out) {
    __shared__ double sp[kGuardThreads / 32], sl[kGuardThreads / 32];
    double a = 0.0, b = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        a += (double)plainE[r];
        b += (double)learnedE[idx[r]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFull, a, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sp[threadIdx.x >> 5] = a;
        sl[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kGuardThreads / 32; ++w) {
            ta += sp[w];
            tb += sl[w];
        }
        const bool fail = tb > kGuardRmseRatio * kGuardRmseRatio * ta;
        *recode_count = fail ? (int)N : 0;
        if (fail) *n_fallback = (int32_t)N;
        if (guard_out) {
            const double scale = 1.0 / ((double)m * P);
            guard_out[0] = (float)sqrt(tb * scale);
            guard_out[1] = (float)sqrt(ta * scale);
            guard_out[2] = fail ? 1.f : 0.f;
        }
    }
}

__global__ void mark_all_kernel(const int* __restrict__ recode_count, long long N,
                                int32_t* __restrict__ idx, int32_t* __restrict__ fallback) {
    if (*recode_count == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        idx[i] = (int32_t)i;
        fallback[i] = 1;
    }
}

template <class T>
T* carve(char*& p, size_t n) {
    T* r = reinterpret_cast<T*>(p);
    p += (n * sizeof(T) + 255) & ~size_t(255);
    return r;
}

int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

extern "C" {

int sdl_mlp_create(sdl_ctx* c, int p1, int p2, int n1, int n2, int hidden, int max_batch,
                   sdl_mlp** out) {
    if (!out) return SDL_ERR_ARG;
    *out = nullptr;
    if (!c || p1 < 1 || p2 < 1 || n1 < 1 || n2 < 1 || hidden < 8 || hidden % 8 ||
        max_batch < 8 || max_batch % 8 || (long long)n1 * n2 > 1024 || (long long)n1 * n2 % 8)
        return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    sdl_mlp* m = new (std::nothrow) sdl_mlp();
    if (!m) return SDL_ERR_WORKSPACE;
    m->ctx = c;
    m->P = p1 * p2;
    m->Kp = (m->P + 7) & ~7;
    m->H = hidden;
    m->Q = n1 * n2;
    m->Bmax = max_batch;
    const size_t H = m->H, Kp = m->Kp, Q = m->Q, B = m->Bmax;
    const size_t nf = 4 * (H * Kp + H + Q * H + Q) + 1024;     // params, m, v, grads
    const size_t bytes = (nf * 4 + (H * Kp + 2 * Q * H) * 2 + (2 * B * Kp + 2 * B * H + 2 * B * Q + B * H) * 2 +
                          (B * H + B * Q + B) * 4) + 64 * 256;
    if (cudaMalloc(&m->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return SDL_ERR_WORKSPACE;
    }
    cudaMemset(m->mem, 0, bytes);
    char* p = m->mem;
    m->W1 = carve<float>(p, H * Kp); m->b1 = carve<float>(p, H);
    m->W2 = carve<float>(p, Q * H); m->b2 = carve<float>(p, Q);
    m->mW1 = carve<float>(p, H * Kp); m->vW1 = carve<float>(p, H * Kp);
    m->mb1 = carve<float>(p, H); m->vb1 = carve<float>(p, H);
    m->mW2 = carve<float>(p, Q * H); m->vW2 = carve<float>(p, Q * H);
    m->mb2 = carve<float>(p, Q); m->vb2 = carve<float>(p, Q);
    m->gW1 = carve<float>(p, H * Kp); m->gb1 = carve<float>(p, H);
    m->gW2 = carve<float>(p, Q * H); m->gb2 = carve<float>(p, Q);
    m->W1b = carve<bf16>(p, H * Kp); m->W2b = carve<bf16>(p, Q * H); m->W2Tb = carve<bf16>(p, H * Q);
    m->Xb = carve<bf16>(p, B * Kp); m->XTb = carve<bf16>(p, Kp * B);
    m->Hb = carve<bf16>(p, B * H); m->HTb = carve<bf16>(p, H * B);
    m->dZb = carve<bf16>(p, B * Q); m->dZTb = carve<bf16>(p, Q * B);
    m->dPreTb = carve<bf16>(p, H * B);
    m->pre = carve<float>(p, B * H); m->Z = carve<float>(p, B * Q); m->lossp = carve<float>(p, B);
    if ((size_t)(p - m->mem) > bytes) {
        cudaFree(m->mem);
        delete m;
        return SDL_ERR_WORKSPACE;
    }
    *out = m;
    return SDL_OK;
}

int sdl_mlp_destroy(sdl_mlp* m) {
    if (!m) return SDL_OK;
    DeviceGuard guard(m->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(m->mem);
    delete m;
    return SDL_OK;
}

// Host FP32 arrays: W1 [hidden x p1p2], b1 [hidden], W2 [n1n2 x hidden], b2 [n1n2].
// Either direction is synchronous; Adam moments and the step count are reset on set.
int sdl_mlp_set_weights(sdl_mlp* m, const float* W1, const float* b1, const float* W2,
                        const float* b2) {
    if (!m || !W1 || !b1 || !W2 || !b2) return SDL_ERR_ARG;
    DeviceGuard guard(m->ctx->device);
    std::vector<float> w1((size_t)m->H * m->Kp, 0.f);
    for (int h = 0; h < m->H; ++h)
        for (int e = 0; e < m->P; ++e) w1[(size_t)h * m->Kp + e] = W1[(size_t)h * m->P + e];
    const size_t H = m->H, Kp = m->Kp, Q = m->Q;
    if (cudaMemcpy(m->W1, w1.data(), H * Kp * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->b1, b1, H * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->W2, W2, Q * H * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->b2, b2, Q * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return SDL_ERR_CUDA;
    for (float* z : {m->mW1, m->vW1, m->gW1}) cudaMemset(z, 0, H * Kp * 4);
    for (float* z : {m->mb1, m->vb1, m->gb1}) cudaMemset(z, 0, H * 4);
    for (float* z : {m->mW2, m->vW2, m->gW2}) cudaMemset(z, 0, Q * H * 4);
    for (float* z : {m->mb2, m->vb2, m->gb2}) cudaMemset(z, 0, Q * 4);
    m->step = 0;
    to_bf16_kernel<<<blocks_for(H * Kp, 256), 256>>>(m->W1, (int)H, (int)Kp, m->W1b, nullptr);
    to_bf16_kernel<<<blocks_for(Q * H, 256), 256>>>(m->W2, (int)Q, (int)H, m->W2b, m->W2Tb);
    return cudaDeviceSynchronize() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int sdl_mlp_get_weights(sdl_mlp* m, float* W1, float* b1, float* W2, float* b2) {
    if (!m) return SDL_ERR_ARG;
    DeviceGuard guard(m->ctx->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return SDL_ERR_CUDA;
    const size_t H = m->H, Kp = m->Kp, Q = m->Q;
    if (W1) {
        std::vector<float> w1(H * Kp);
        if (cudaMemcpy(w1.data(), m->W1, H * Kp * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SDL_ERR_CUDA;
        for (size_t h = 0; h < H; ++h)
            for (int e = 0; e < m->P; ++e) W1[h * m->P + e] = w1[h * Kp + e];
    }
    if (b1 && cudaMemcpy(b1, m->b1, H * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    if (W2 && cudaMemcpy(W2, m->W2, Q * H * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    if (b2 && cudaMemcpy(b2, m->b2, Q * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    return SDL_OK;
}

// Forward + loss + backward for one batch (gradients left in the network's
// gradient buffers); optionally the Adam step.  Y: B signals (layout of
// sdl_iterate), support: B x s OMP supports (the labels).
static int mlp_batch(sdl_mlp* m, const float* Y, const int32_t* support, int s, int B, bool update,
                     float lr, float* loss_out, cudaStream_t st) {
    sdl_ctx* c = m->ctx;
    const int H = m->H, Kp = m->Kp, Q = m->Q, Bm = m->Bmax;
    int rc;
    {
        Trace tr(c, kMlp, st);
        prep_input_kernel<<<blocks_for((long long)B * 32, 256), 256, 0, st>>>(Y, B, m->P, Kp, m->Xb,
                                                                             Kp, m->XTb, Bm);
        if ((rc = tc_gemm(m->Xb, Kp, m->W1b, Kp, B, H, Kp, 1.f, m->b1, 1, nullptr, 0, 0, m->Hb, H,
                          m->HTb, Bm, m->pre, H, c->err, st)))
            return rc;
        if ((rc = tc_gemm(m->Hb, H, m->W2b, H, B, Q, H, 1.f, m->b2, 0, m->Z, Q, 0, nullptr, 0,
                          nullptr, 0, nullptr, 0, c->err, st)))
            return rc;
        bce_kernel<<<B, 256, 0, st>>>(m->Z, Q, support, s, Q, 1.f / (float)B, m->dZb, Q, m->dZTb,
                                      Bm, m->lossp);
        // dW2 = dZ^T H ; dPre = (dZ W2) * GELU'(pre) ; dW1 = dPre^T X
        if ((rc = tc_gemm(m->dZTb, Bm, m->HTb, Bm, Q, H, B, 1.f, nullptr, 0, m->gW2, H, 0, nullptr,
                          0, nullptr, 0, nullptr, 0, c->err, st)))
            return rc;
        if ((rc = tc_gemm(m->dZb, Q, m->W2Tb, Q, B, H, Q, 1.f, nullptr, 2, nullptr, 0, 0, nullptr,
                          0, m->dPreTb, Bm, nullptr, 0, c->err, st, m->pre, H)))
            return rc;
        if ((rc = tc_gemm(m->dPreTb, Bm, m->XTb, Bm, H, Kp, B, 1.f, nullptr, 0, m->gW1, Kp, 0,
                          nullptr, 0, nullptr, 0, nullptr, 0, c->err, st)))
            return rc;
        rowsum_kernel<<<blocks_for((long long)Q * 32, 256), 256, 0, st>>>(m->dZTb, Bm, Q, B, m->gb2);
        rowsum_kernel<<<blocks_for((long long)H * 32, 256), 256, 0, st>>>(m->dPreTb, Bm, H, B, m->gb1);
        if (loss_out) sum_kernel<<<1, 32, 0, st>>>(m->lossp, B, 1.f / (float)B, loss_out);
    }
    if (update) {
        Trace tr(c, kAdam, st);
        m->step += 1;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float bc1 = 1.f - powf(b1, (float)m->step), bc2 = 1.f - powf(b2, (float)m->step);
        adam_kernel<<<blocks_for((long long)H * Kp, 256), 256, 0, st>>>(
            m->W1, m->gW1, m->mW1, m->vW1, H, Kp, lr, b1, b2, eps, bc1, bc2, m->W1b, nullptr);
        adam_kernel<<<blocks_for(H, 256), 256, 0, st>>>(m->b1, m->gb1, m->mb1, m->vb1, 1, H, lr, b1,
                                                         b2, eps, bc1, bc2, nullptr, nullptr);
        adam_kernel<<<blocks_for((long long)Q * H, 256), 256, 0, st>>>(
            m->W2, m->gW2, m->mW2, m->vW2, Q, H, lr, b1, b2, eps, bc1, bc2, m->W2b, m->W2Tb);
        adam_kernel<<<blocks_for(Q, 256), 256, 0, st>>>(m->b2, m->gb2, m->mb2, m->vb2, 1, Q, lr, b1,
                                                         b2, eps, bc1, bc2, nullptr, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int sdl_mlp_train_step(sdl_mlp* m, const float* Y, const int32_t* support, int s, int B, float lr,
                       float* loss_out, void* stream) {
    if (!m || !Y || !support || s < 1 || s > 32 || B < 8 || B % 8 || B > m->Bmax || !(lr > 0.f))
        return SDL_ERR_ARG;
    DeviceGuard guard(m->ctx->device);
    return mlp_batch(m, Y, support, s, B, true, lr, loss_out, (cudaStream_t)stream);
}

int sdl_mlp_gradients(sdl_mlp* m, const float* Y, const int32_t* support, int s, int B,
                      float* loss_out, float* gW1, float* gb1, float* gW2, float* gb2,
                      void* stream) {
    if (!m || !Y || !support || s < 1 || s > 32 || B < 8 || B % 8 || B > m->Bmax) return SDL_ERR_ARG;
    DeviceGuard guard(m->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = mlp_batch(m, Y, support, s, B, false, 0.f, loss_out, st);
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SDL_ERR_CUDA;
    const size_t H = m->H, Kp = m->Kp, Q = m->Q;
    if (gW1) {
        std::vector<float> g(H * Kp);
        if (cudaMemcpy(g.data(), m->gW1, H * Kp * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
        for (size_t h = 0; h < H; ++h)
            for (int e = 0; e < m->P; ++e) gW1[h * m->P + e] = g[h * Kp + e];
    }
    if (gb1 && cudaMemcpy(gb1, m->gb1, H * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    if (gW2 && cudaMemcpy(gW2, m->gW2, Q * H * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    if (gb2 && cudaMemcpy(gb2, m->gb2, Q * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SDL_ERR_CUDA;
    return SDL_OK;
}

// Scores of N signals (device FP32 N x n1n2), processed in chunks of max_batch.
int sdl_mlp_forward(sdl_mlp* m, const float* Y, int64_t N, float* scores, void* stream) {
    if (!m || (N > 0 && (!Y || !scores)) || N < 0) return SDL_ERR_ARG;
    DeviceGuard guard(m->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    sdl_ctx* c = m->ctx;
    const int H = m->H, Kp = m->Kp, Q = m->Q;
    Trace tr(c, kMlp, st);
    for (int64_t r0 = 0; r0 < N; r0 += m->Bmax) {
        const int B = (int)std::min<int64_t>(m->Bmax, N - r0);
        prep_input_kernel<<<blocks_for((long long)B * 32, 256), 256, 0, st>>>(
            Y + (size_t)r0 * m->P, B, m->P, Kp, m->Xb, Kp, nullptr, 0);
        int rc = tc_gemm(m->Xb, Kp, m->W1b, Kp, B, H, Kp, 1.f, m->b1, 1, nullptr, 0, 0, m->Hb, H,
                         nullptr, 0, nullptr, 0, c->err, st);
        if (!rc)
            rc = tc_gemm(m->Hb, H, m->W2b, H, B, Q, H, 1.f, m->b2, 0, scores + (size_t)r0 * Q, Q, 0,
                         nullptr, 0, nullptr, 0, nullptr, 0, c->err, st);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // extern "C"

// ------------------------------------------------------------ learned coder
namespace {

template <int P1, int P2, int N1, int N2, int S>
int launch_shortlist(const float* Y, long long N, const float* D1, const float* D2, const float* G1,
                     const float* G2, const int32_t* cand, int k1, int k2, int32_t* support,
                     float* coef, int32_t* nnz, float* res, int32_t* flag, int num_sms,
                     cudaStream_t st) {
    const long long need = (N + 7) / 8;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * 8));
    shortlist_omp_kernel<P1, P2, N1, N2, S><<<grid, 256, 0, st>>>(Y, N, D1, D2, G1, G2, cand, k1, k2,
                                                                  support, coef, nnz, res, flag);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // namespace

extern "C" int sdl_sparse_code_learned(sdl_ctx* c, sdl_mlp* m, const float* Y, int p1, int p2,
                                       int64_t N, const float* D1, int n1, const float* D2, int n2,
                                       int s_max, int k, int32_t* support, float* coef,
                                       int32_t* nnz, float* res_energy, int32_t* fallback,
                                       int32_t* n_fallback, float* guard_out, void* stream) {
    if (!c || !m || m->ctx != c || !Y || !D1 || !D2 || !support || !coef || !nnz || !fallback ||
        !n_fallback || N < 1 || N > 0x7fffffffLL)
        return SDL_ERR_ARG;
    if (m->P != p1 * p2 || m->Q != n1 * n2 || k < 1 || k > 32) return SDL_ERR_ARG;
    const bool shape_a = p1 == 12 && p2 == 12 && n1 == 24 && n2 == 24 && s_max == 6;
    const bool shape_b = p1 == 8 && p2 == 8 && n1 == 16 && n2 == 16 && s_max == 4;
    if (!shape_a && !shape_b) return SDL_ERR_UNSUPPORTED;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int k2 = k, Q = m->Q;     // the shortlist only: the fallback test scans every pair
    // workspace: scores of one chunk, candidates, Grams, scan buffers, index list
    const long long chunk = m->Bmax;
    const int nblk = (int)((N + kScanBlock - 1) / kScanBlock);
    const long long m_s = std::min<long long>(N, std::max<long long>(kGuardMinSample, N / 16));
    const long long stride_s = N / m_s;
    const size_t need = sizeof(float) * (size_t)chunk * Q + sizeof(int32_t) * (size_t)N * k2 +
                        sizeof(float) * (size_t)(n1 * n1 + n2 * n2) + sizeof(int) * (nblk + 8) +
                        sizeof(int32_t) * (size_t)N + sizeof(int32_t) * (size_t)m_s +
                        sizeof(float) * (size_t)m_s + sizeof(float) * (size_t)N + 10 * 256;
    if (need > c->cap_learn) {
        if (c->learn) cudaFree(c->learn);
        c->learn = nullptr;
        c->cap_learn = 0;
        if (cudaMalloc(&c->learn, need) != cudaSuccess) {
            cudaGetLastError();
            return SDL_ERR_WORKSPACE;
        }
        c->cap_learn = need;
    }
    char* p = c->learn;
    float* scores = carve<float>(p, (size_t)chunk * Q);
    int32_t* cand = carve<int32_t>(p, (size_t)N * k2);
    float* G1 = carve<float>(p, (size_t)n1 * n1);
    float* G2 = carve<float>(p, (size_t)n2 * n2);
    int* blockcnt = carve<int>(p, nblk + 8);
    int32_t* idx = carve<int32_t>(p, (size_t)N);
    int32_t* idx_s = carve<int32_t>(p, (size_t)m_s);
    float* plainE = carve<float>(p, (size_t)m_s);
    float* learnedE = res_energy ? res_energy : carve<float>(p, (size_t)N);
    int* cnt_s = carve<int>(p, 2);
    int rc;
    {
        Trace tr(c, kGram, st);
        launch_gram2(D1, p1, n1, G1, D2, p2, n2, G2, st);
    }
    // 1. scores and shortlists, chunk by chunk
    for (int64_t r0 = 0; r0 < N; r0 += chunk) {
        const int B = (int)std::min<int64_t>(chunk, N - r0);
        if ((rc = sdl_mlp_forward(m, Y + (size_t)r0 * p1 * p2, B, scores, stream))) return rc;
        Trace tr(c, kTopk, st);
        if (Q <= 256)
            topk_kernel<8><<<blocks_for((long long)B * 32, 256), 256, 0, st>>>(
                scores, Q, B, Q, k, k2, cand + (size_t)r0 * k2);
        else if (Q <= 576)
            topk_kernel<18><<<blocks_for((long long)B * 32, 256), 256, 0, st>>>(
                scores, Q, B, Q, k, k2, cand + (size_t)r0 * k2);
        else
            topk_kernel<32><<<blocks_for((long long)B * 32, 256), 256, 0, st>>>(
                scores, Q, B, Q, k, k2, cand + (size_t)r0 * k2);
    }
    // 2. 2D-OMP on the shortlists, with the fallback test
    {
        Trace tr(c, kShortlist, st);
        rc = shape_a ? launch_shortlist<12, 12, 24, 24, 6>(Y, N, D1, D2, G1, G2, cand, k, k2, support,
                                                          coef, nnz, learnedE, fallback,
                                                          c->num_sms, st)
                     : launch_shortlist<8, 8, 16, 16, 4>(Y, N, D1, D2, G1, G2, cand, k, k2, support,
                                                        coef, nnz, learnedE, fallback, c->num_sms,
                                                        st);
        if (rc) return rc;
    }
    // 3. compact the flagged signals (fixed order) and re-code them with the full coder
    count_flags_kernel<<<nblk, kScanBlock, 0, st>>>(fallback, N, blockcnt);
    scan_counts_kernel<<<1, 32, 0, st>>>(blockcnt, nblk, n_fallback);
    write_index_kernel<<<nblk, kScanBlock, 0, st>>>(fallback, N, blockcnt, idx);
    PassArgs a{};
    a.Y = Y;
    a.p1 = p1;
    a.p2 = p2;
    a.N = N;
    a.D1 = D1;
    a.D2 = D2;
    a.G1 = G1;
    a.G2 = G2;
    a.n1 = n1;
    a.n2 = n2;
    a.s = s_max;
    a.support = support;
    a.coef = coef;
    a.nnz = nnz;
    a.res_energy = learnedE;
    a.n_slots = 1;
    a.err = c->err;
    a.idx = idx;
    a.idx_count = n_fallback;
    {
        Trace tr(c, kCode, st);
        rc = launch_code_pass_fast(a, kCodeOnly, st, c->num_sms);
        if (rc < 0) return rc;
    }
    // 4. the plain coder on the strided sample (residual energies only)
    sample_index_kernel<<<blocks_for(m_s, 256), 256, 0, st>>>(idx_s, (int)m_s, stride_s, cnt_s);
    PassArgs g = a;
    g.support = nullptr;
    g.coef = nullptr;
    g.nnz = nullptr;
    g.res_energy = plainE;
    g.idx = idx_s;
    g.idx_count = cnt_s;
    g.idx_compact = 1;
    {
        Trace tr(c, kCode, st);
        rc = launch_code_pass_fast(g, kCodeOnly, st, c->num_sms);
        if (rc < 0) return rc;
    }
    // 5. RMSE guard; when it trips, every signal is coded again by the plain coder
    guard_kernel<<<1, kGuardThreads, 0, st>>>(plainE, learnedE, idx_s, (int)m_s, N, p1 * p2,
                                              cnt_s + 1, n_fallback, guard_out);
    mark_all_kernel<<<std::max(1, std::min(blocks_for(N, 256), c->num_sms * 8)), 256, 0, st>>>(
        cnt_s + 1, N, idx, fallback);
    a.idx_count = cnt_s + 1;
    {
        Trace tr(c, kCode, st);
        rc = launch_code_pass_fast(a, kCodeOnly, st, c->num_sms);
    }
    return rc < 0 ? rc : SDL_OK;
}

// The two shortlist steps of sdl_sparse_code_learned on their own (before
// any fallback), so that each can be checked against a reference.
extern "C" int sdl_learned_shortlists(sdl_ctx* c, const float* scores, int64_t N, int Q, int k1,
                                      int k2, int32_t* cand, void* stream) {
    if (!c || N < 0 || N > 0x7fffffffLL || Q < 1 || Q > 1024 || k1 < 1 || k2 < k1 || k2 > Q)
        return SDL_ERR_ARG;
    if (N == 0) return SDL_OK;
    if (!scores || !cand) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    Trace tr(c, kTopk, st);
    const int blocks = blocks_for(N * 32, 256);
    if (Q <= 256)
        topk_kernel<8><<<blocks, 256, 0, st>>>(scores, Q, N, Q, k1, k2, cand);
    else if (Q <= 576)
        topk_kernel<18><<<blocks, 256, 0, st>>>(scores, Q, N, Q, k1, k2, cand);
    else
        topk_kernel<32><<<blocks, 256, 0, st>>>(scores, Q, N, Q, k1, k2, cand);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

extern "C" int sdl_sparse_code_shortlist(sdl_ctx* c, const float* Y, int p1, int p2, int64_t N,
                                         const float* D1, int n1, const float* D2, int n2,
                                         int s_max, const int32_t* cand, int k1, int k2,
                                         int32_t* support, float* coef, int32_t* nnz,
                                         float* res_energy, int32_t* flag, void* stream) {
    if (!c || !D1 || !D2 || N < 0 || N > 0x7fffffffLL || k1 < 1 || k1 > 32 || k2 < k1)
        return SDL_ERR_ARG;
    const bool shape_a = p1 == 12 && p2 == 12 && n1 == 24 && n2 == 24 && s_max == 6;
    const bool shape_b = p1 == 8 && p2 == 8 && n1 == 16 && n2 == 16 && s_max == 4;
    if (!shape_a && !shape_b) return SDL_ERR_UNSUPPORTED;
    if (N == 0) return SDL_OK;
    if (!Y || !cand || !support || !coef || !nnz || !flag) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ctx_workspace(c, p1, p2, n1, n2);
    if (rc) return rc;
    {
        Trace tr(c, kGram, st);
        launch_gram2(D1, p1, n1, c->G1, D2, p2, n2, c->G2, st);
    }
    Trace tr(c, kShortlist, st);
    return shape_a ? launch_shortlist<12, 12, 24, 24, 6>(Y, N, D1, D2, c->G1, c->G2, cand, k1, k2,
                                                         support, coef, nnz, res_energy, flag,
                                                         c->num_sms, st)
                   : launch_shortlist<8, 8, 16, 16, 4>(Y, N, D1, D2, c->G1, c->G2, cand, k1, k2,
                                                       support, coef, nnz, res_energy, flag,
                                                       c->num_sms, st);
}
