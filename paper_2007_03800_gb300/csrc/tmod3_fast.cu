// Three-mode coding pass (Remark 3) specialised at compile time: one warp per
// signal Y_k (p1 x p2 x p3, column-order vec), atom triples q = i + n1 j +
// n1 n2 l, s greedy steps fully unrolled.  Same method and results (within
// rounding) as the generic code3_kernel; what changes is the schedule:
//   * the n1 x n2 x n3 correlation tensor is split over a LI x LJ x LL lane
//     grid, RI x RJ x RL entries per lane, kept in registers during a step;
//   * C0 = Y x_3 D3^T x_1 D1^T x_2 D2^T: the first two contractions are
//     formed cooperatively in shared memory (T1[a][b, l], then T2[i, b, l]),
//     the last one on each lane's own block;
//   * each step re-applies the earlier picks as rank-1 three-way updates
//     -x_m G1[:, i_m] o G2[:, j_m] o G3[:, l_m] with vector loads of the
//     lane's blocks of the three Gram rows;
//   * the argmax is four compare/select chains per lane and two redux.sync;
//   * every lane computes the Cholesky update of the pick (identical values),
//     lane 0 keeps the factor in shared memory (it holds no registers while the
//     scores are live);
//   * the next signal is loaded into registers while the current one is coded.
// The partial sums of the mode-k update go to warp-private accumulators with
// the generic kernel's layout, so the same reduction and solve follow.
#include <algorithm>
#include <cmath>
#include <utility>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr unsigned kAll = 0xffffffffu;
__host__ __device__ constexpr int r4(int x) { return (x + 3) & ~3; }

template <int P1_, int P2_, int P3_, int N1_, int N2_, int N3_, int S_, int LI_, int LJ_>
struct Shape3F {
    static constexpr int P1 = P1_, P2 = P2_, P3 = P3_, N1 = N1_, N2 = N2_, N3 = N3_, S = S_;
    static constexpr int LI = LI_, LJ = LJ_, LL = 32 / (LI_ * LJ_);
    static constexpr int RI = N1_ / LI_, RJ = N2_ / LJ_, RL = N3_ / LL;
    static constexpr int E = RI * RJ * RL;
    static constexpr int PP = P1_ * P2_ * P3_, Q = N1_ * N2_ * N3_;
    static constexpr int EP = ((r4(E) / 4) % 2 == 0) ? r4(E) + 4 : r4(E);   // lane stride, odd x 4
    static constexpr int YPL = PP / 32;                                     // Y floats per lane
    static constexpr int WPC = 8;                                           // warps per CTA
    static_assert(LI * LJ * LL == 32, "lane grid");
    static_assert(RI * LI == N1 && RJ * LJ == N2 && RL * LL == N3, "blocks tile the tensor");
    static_assert(RI == 4 && N1 % 4 == 0 && (RJ == 4 || RJ == 2) && (RL == 1 || RL == 2 || RL == 4),
                  "vector loads of the Gram rows");
    static_assert(P1 <= 16 && P2 <= 16 && P3 <= 16 && S <= 16 && S <= PP && S <= Q, "sizes");
    static_assert(YPL == 2 || YPL % 4 == 0, "signal loads");
};

template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

template <int R>
__device__ __forceinline__ void ld(float (&v)[R], const float* p) {
    if constexpr (R == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (R == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = p[0];
    }
}

// d = a * b + c on two lanes at once (fma.rn.f32x2, each half as fmaf)
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    const unsigned long long A = ((unsigned long long)__float_as_uint(a1) << 32) | __float_as_uint(a0);
    const unsigned long long B = ((unsigned long long)__float_as_uint(b1) << 32) | __float_as_uint(b0);
    const unsigned long long C = ((unsigned long long)__float_as_uint(d1) << 32) | __float_as_uint(d0);
    unsigned long long D;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(C));
    d0 = __uint_as_float((unsigned)(D & 0xffffffffu));
    d1 = __uint_as_float((unsigned)(D >> 32));
}

// blk[c * R + r] += a[r] * b[c]  (R even: packed along r)
template <int R, int C>
__device__ __forceinline__ void rank1(float* blk, const float (&a)[R], const float (&b)[C]) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int r = 0; r < R; r += 2) ffma2(blk[c * R + r], blk[c * R + r + 1], a[r], a[r + 1], b[c], b[c]);
}

template <class Sh>
struct Layout3F {
    static constexpr int P1 = Sh::P1, P2 = Sh::P2, P3 = Sh::P3, N1 = Sh::N1, N2 = Sh::N2, N3 = Sh::N3;
    // shared part (floats, 16-byte aligned regions): rows of D1, D2, D3, the Grams
    static constexpr int d1 = 0;                        // P1 x N1
    static constexpr int d2 = d1 + r4(P1 * N1);         // P2 x N2
    static constexpr int d3 = d2 + r4(P2 * N2);         // P3 x N3
    static constexpr int g1 = d3 + r4(P3 * N3);         // N1 x N1
    static constexpr int g2 = g1 + r4(N1 * N1);         // N2 x N2
    static constexpr int g3 = g2 + r4(N2 * N2);         // N3 x N3
    static constexpr int acc = g3 + r4(N3 * N3);
    __host__ __device__ static constexpr int nf(int mode) {
        return mode == 1 ? N1 * N1 + P1 * N1 : mode == 2 ? N2 * N2 + P2 * N2 : mode == 3 ? N3 * N3 + P3 * N3 : 0;
    }
    __host__ __device__ static constexpr int acce(int mode) { return acc + r4(nf(mode)) * Sh::WPC; }
    __host__ __device__ static constexpr int warp0(int mode) { return acce(mode) + r4(2 * Sh::WPC); }
    // per warp: Y, T1 (P1 x P2 N3), T2 (N1 P2 N3), C0 blocks, Cholesky state
    static constexpr int w_y = 0;
    static constexpr int w_t1 = w_y + r4(Sh::PP);
    static constexpr int w_t2 = w_t1 + r4(P1 * P2 * N3);
    static constexpr int w_c0 = w_t2 + r4(N1 * P2 * N3);
    static constexpr int w_l = w_c0 + 32 * Sh::EP;
    static constexpr int w_iv = w_l + r4(Sh::S * (Sh::S + 1) / 2);
    static constexpr int w_yv = w_iv + r4(Sh::S);
    static constexpr int w_stride = w_yv + r4(Sh::S);
    __host__ __device__ static constexpr int total(int mode) { return warp0(mode) + Sh::WPC * w_stride; }
};

template <class Sh, int MODE>
__global__ void __launch_bounds__(Sh::WPC * 32, 2)
    code3_fast_kernel(const float* __restrict__ Y, long long N, const float* __restrict__ D1,
                      const float* __restrict__ D2, const float* __restrict__ D3,
                      const float* __restrict__ G1, const float* __restrict__ G2,
                      const float* __restrict__ G3, int32_t* __restrict__ support,
                      float* __restrict__ coef, int32_t* __restrict__ nnz,
                      float* __restrict__ res_energy, float* __restrict__ part_f,
                      double* __restrict__ part_d, int* err) {
    using L = Layout3F<Sh>;
    constexpr int P1 = Sh::P1, P2 = Sh::P2, P3 = Sh::P3, N1 = Sh::N1, N2 = Sh::N2, N3 = Sh::N3;
    constexpr int S = Sh::S, RI = Sh::RI, RJ = Sh::RJ, RL = Sh::RL, E = Sh::E, PP = Sh::PP;
    constexpr int LI = Sh::LI, LJ = Sh::LJ, N12 = N1 * N2, P12 = P1 * P2;
    extern __shared__ __align__(16) float sm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = lane % LI, lj = (lane / LI) % LJ, ll = lane / (LI * LJ);
    const int i0 = li * RI, j0 = lj * RJ, l0 = ll * RL;
    float* sD1 = sm + L::d1;
    float* sD2 = sm + L::d2;
    float* sD3 = sm + L::d3;
    float* sG1 = sm + L::g1;
    float* sG2 = sm + L::g2;
    float* sG3 = sm + L::g3;
    constexpr int nf = L::nf(MODE);
    float* wacc = sm + L::acc + w * r4(nf);
    float* acce = sm + L::acce(MODE);
    float* wb = sm + L::warp0(MODE) + w * L::w_stride;
    float* Ys = wb + L::w_y;
    float* T1 = wb + L::w_t1;    // T1[a * P2 N3 + b + P2 l] = sum_c Y[a, b, c] D3[c, l]
    float* T2 = wb + L::w_t2;    // T2[i + N1 (b + P2 l)] = sum_a D1[a, i] T1[a, b, l]
    float* C0s = wb + L::w_c0;
    float* myc0 = C0s + lane * Sh::EP;
    float* Lsm = wb + L::w_l;
    float* ivsm = wb + L::w_iv;
    float* yvsm = wb + L::w_yv;

    for (int e = threadIdx.x; e < P1 * N1; e += blockDim.x) sD1[e] = D1[(e / N1) + P1 * (e % N1)];
    for (int e = threadIdx.x; e < P2 * N2; e += blockDim.x) sD2[e] = D2[(e / N2) + P2 * (e % N2)];
    for (int e = threadIdx.x; e < P3 * N3; e += blockDim.x) sD3[e] = D3[(e / N3) + P3 * (e % N3)];
    for (int e = threadIdx.x; e < N1 * N1; e += blockDim.x) sG1[e] = G1[e];
    for (int e = threadIdx.x; e < N2 * N2; e += blockDim.x) sG2[e] = G2[e];
    for (int e = threadIdx.x; e < N3 * N3; e += blockDim.x) sG3[e] = G3[e];
    for (int e = threadIdx.x; e < (L::warp0(MODE) - L::acc); e += blockDim.x) sm[L::acc + e] = 0.f;
    __syncthreads();

    // the signal's floats this lane loads (vector chunks, coalesced)
    float yr[Sh::YPL];
    auto load_y = [&](long long k) {
        const float* src = Y + (size_t)k * PP;
        if constexpr (Sh::YPL == 2) {
            const float2 t = *reinterpret_cast<const float2*>(src + 2 * lane);
            yr[0] = t.x; yr[1] = t.y;
        } else {
#pragma unroll
            for (int c = 0; c < Sh::YPL / 4; ++c) {
                const float4 t = *reinterpret_cast<const float4*>(src + 128 * c + 4 * lane);
                yr[4 * c] = t.x; yr[4 * c + 1] = t.y; yr[4 * c + 2] = t.z; yr[4 * c + 3] = t.w;
            }
        }
    };
    auto store_y = [&]() {
        if constexpr (Sh::YPL == 2) {
            *reinterpret_cast<float2*>(Ys + 2 * lane) = make_float2(yr[0], yr[1]);
        } else {
#pragma unroll
            for (int c = 0; c < Sh::YPL / 4; ++c)
                *reinterpret_cast<float4*>(Ys + 128 * c + 4 * lane) =
                    make_float4(yr[4 * c], yr[4 * c + 1], yr[4 * c + 2], yr[4 * c + 3]);
        }
    };

    float w_energy = 0.f, w_energy_c = 0.f, w_ynorm = 0.f, w_ynorm_c = 0.f;
    const long long stride = (long long)gridDim.x * Sh::WPC;
    long long k = (long long)blockIdx.x * Sh::WPC + w;
    if (k < N) load_y(k);
    for (; k < N; k += stride) {
        __syncwarp();
        store_y();
        float ss = 0.f;
#pragma unroll
        for (int e = 0; e < Sh::YPL; ++e) ss = fmaf(yr[e], yr[e], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kAll, ss, o);
        if (k + stride < N) load_y(k + stride);   // in flight while this signal is coded
        __syncwarp();
        const bool finite = isfinite(ss);
        int cnt = 0, myq = 0;
        float E2 = ss, myx = 0.f;
        int qs[S];
        float xs[S];
#pragma unroll
        for (int m = 0; m < S; ++m) {
            qs[m] = 0;
            xs[m] = 0.f;
        }
        if (finite) {
            // ---- T1 = Y x_3 D3^T
            for (int e = lane; e < P12 * N3; e += 32) {
                const int ab = e % P12, l = e / P12;
                float t = 0.f;
#pragma unroll
                for (int c = 0; c < P3; ++c) t = fmaf(Ys[ab + P12 * c], sD3[c * N3 + l], t);
                T1[(ab % P1) * (P2 * N3) + ab / P1 + P2 * l] = t;
            }
            __syncwarp();
            // ---- T2 = T1 x_1 D1^T
            for (int e = lane; e < N1 * P2 * N3; e += 32) {
                const int i = e % N1, bl = e / N1;
                float t = 0.f;
#pragma unroll
                for (int a = 0; a < P1; ++a) t = fmaf(sD1[a * N1 + i], T1[a * (P2 * N3) + bl], t);
                T2[e] = t;
            }
            __syncwarp();
            // ---- C0 = T2 x_2 D2^T on the lane's block, entry e = (rl RJ + rj) RI + ri
            float c0[E];
#pragma unroll
            for (int e = 0; e < E; ++e) c0[e] = 0.f;
#pragma unroll
            for (int b = 0; b < P2; ++b) {
                float v[RJ];
                ld<RJ>(v, sD2 + b * N2 + j0);
#pragma unroll
                for (int rl = 0; rl < RL; ++rl) {
                    float u[RI];
                    ld<RI>(u, T2 + i0 + N1 * (b + P2 * (l0 + rl)));
                    rank1<RI, RJ>(c0 + rl * RJ * RI, u, v);
                }
            }
#pragma unroll
            for (int e = 0; e < E; e += 4)
                *reinterpret_cast<float4*>(myc0 + e) = make_float4(c0[e], c0[e + 1], c0[e + 2], c0[e + 3]);
            __syncwarp();

            // ---- greedy steps
            const int qbase = i0 + N1 * j0 + N12 * l0;
            bool go = true;
            sfor<0, S>([&](auto tc) {
                constexpr int t = decltype(tc)::value;
                if (!go) return;
                float sc[E];
                if constexpr (t == 0) {
#pragma unroll
                    for (int e = 0; e < E; ++e) sc[e] = c0[e];
                } else {
#pragma unroll
                    for (int e = 0; e < E; e += 4) {
                        const float4 x4 = *reinterpret_cast<const float4*>(myc0 + e);
                        sc[e] = x4.x; sc[e + 1] = x4.y; sc[e + 2] = x4.z; sc[e + 3] = x4.w;
                    }
                }
                // C = C0 - sum_m x_m G1[:, i_m] o G2[:, j_m] o G3[:, l_m]
#pragma unroll
                for (int m = 0; m < t; ++m) {
                    const int qm = qs[m];
                    const int im = qm % N1, jm = (qm / N1) % N2, lm = qm / N12;
                    float u[RI], v[RJ], wl[RL], vw[RJ * RL];
                    ld<RI>(u, sG1 + im * N1 + i0);
                    ld<RJ>(v, sG2 + jm * N2 + j0);
                    ld<RL>(wl, sG3 + lm * N3 + l0);
#pragma unroll
                    for (int rl = 0; rl < RL; ++rl) {
                        const float wx = -xs[m] * wl[rl];
#pragma unroll
                        for (int rj = 0; rj < RJ; ++rj) vw[rl * RJ + rj] = v[rj] * wx;
                    }
                    rank1<RI, RJ * RL>(sc, u, vw);
                }
                // argmax |C|, ties to the smallest q: four chains (entries e = 4k + ch
                // in increasing q), merged by (value, q)
                float bv[4] = {0.f, 0.f, 0.f, 0.f};
                int bqv[4] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
#pragma unroll
                for (int rl = 0; rl < RL; ++rl)
#pragma unroll
                    for (int rj = 0; rj < RJ; ++rj)
#pragma unroll
                        for (int ri = 0; ri < RI; ++ri) {
                            const int e = (rl * RJ + rj) * RI + ri;
                            const float v = fabsf(sc[e]);
                            if (v > bv[e & 3]) { bv[e & 3] = v; bqv[e & 3] = qbase + ri + N1 * rj + N12 * rl; }
                        }
#pragma unroll
                for (int ch = 1; ch < 4; ch += 2)
                    if (bv[ch] > bv[ch - 1] || (bv[ch] == bv[ch - 1] && bqv[ch] < bqv[ch - 1])) {
                        bv[ch - 1] = bv[ch];
                        bqv[ch - 1] = bqv[ch];
                    }
                if (bv[2] > bv[0] || (bv[2] == bv[0] && bqv[2] < bqv[0])) {
                    bv[0] = bv[2];
                    bqv[0] = bqv[2];
                }
                // the Cholesky state of steps 0..t-1
                constexpr int kOld = t * (t + 1) / 2;
                float Lo[kOld > 0 ? kOld : 1], io[t > 0 ? t : 1], yo[t > 0 ? t : 1];
#pragma unroll
                for (int m = 0; m < kOld; ++m) Lo[m] = Lsm[m];
#pragma unroll
                for (int m = 0; m < t; ++m) {
                    io[m] = ivsm[m];
                    yo[m] = yvsm[m];
                }
                const unsigned bb = __float_as_uint(bv[0]);
                const unsigned M = __reduce_max_sync(kAll, bb);
                if (M == 0u) { go = false; return; }           // every remaining score is 0
                const int q = (int)__reduce_min_sync(kAll, bb == M ? (unsigned)bqv[0] : 0xffffffffu);
                const int it = q % N1, jt = (q / N1) % N2, lt = q / N12;
                const int owner = it / RI + LI * (jt / RJ) + LI * LJ * (lt / RL);
                float* cq = C0s + owner * Sh::EP + ((lt % RL) * RJ + jt % RJ) * RI + it % RI;
                const float b = *cq;
                __syncwarp();
                if (lane == 0) *cq = __int_as_float(0x7fc00000);   // mask the pick
                // ---- Cholesky row t: w = L^{-1} a, a_m = A[t, m]
                const float Att = sG1[it * N1 + it] * sG2[jt * N2 + jt] * sG3[lt * N3 + lt];
                float wr[t > 0 ? t : 1];
                float ww = 0.f, wy = 0.f;
#pragma unroll
                for (int m = 0; m < t; ++m) {
                    const int qm = qs[m];
                    const int im = qm % N1, jm = (qm / N1) % N2, lm = qm / N12;
                    float am = sG1[it * N1 + im] * sG2[jt * N2 + jm] * sG3[lt * N3 + lm];
#pragma unroll
                    for (int l = 0; l < m; ++l) am = fmaf(-Lo[m * (m + 1) / 2 + l], wr[l], am);
                    wr[m] = am * io[m];
                    ww = fmaf(wr[m], wr[m], ww);
                    wy = fmaf(wr[m], yo[m], wy);
                }
                const float d = Att - ww;
                if (!(d > kPivotRel * Att)) { go = false; return; }
                const float inv = rsqrtf(d);
                const float yt = (b - wy) * inv;
                // ---- x = L^{-T} y
                float xn[t + 1];
                xn[t] = yt * inv;
#pragma unroll
                for (int kk = t - 1; kk >= 0; --kk) {
                    float v = yo[kk];
#pragma unroll
                    for (int l = kk + 1; l < t; ++l) v = fmaf(-Lo[l * (l + 1) / 2 + kk], xn[l], v);
                    v = fmaf(-wr[kk], xn[t], v);
                    xn[kk] = v * io[kk];
                }
#pragma unroll
                for (int kk = 0; kk <= t; ++kk) xs[kk] = xn[kk];
                qs[t] = q;
                if (lane == t) myq = q;
                E2 = fmaf(-yt, yt, E2);
                cnt = t + 1;
                if (lane == 0) {
#pragma unroll
                    for (int m = 0; m < t; ++m) Lsm[kOld + m] = wr[m];
                    ivsm[t] = inv;
                    yvsm[t] = yt;
                }
                __syncwarp();   // the masked entry and the new row are visible to the next step
            });
#pragma unroll
            for (int m = 0; m < S; ++m)
                if (lane == m) myx = xs[m];
        }

        // ---- emit the code (lane m holds pick m)
        if (support && lane < S) {
            support[(size_t)k * S + lane] = lane < cnt ? myq : -1;
            coef[(size_t)k * S + lane] = lane < cnt ? myx : 0.f;
        }
        if (lane == 0) {
            if (nnz) nnz[k] = cnt;
            if (res_energy) res_energy[k] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
            if (!finite) record_error(err, SDL_ERR_NONFINITE);
        }

        // ---- partial sums of the mode-k update (Remark 3 -> Corollary 1)
        if constexpr (MODE != 0) {
            constexpr int nk = MODE == 1 ? N1 : MODE == 2 ? N2 : N3;
            constexpr int pk = MODE == 1 ? P1 : MODE == 2 ? P2 : P3;
            float* accP = wacc;
            float* accB = wacc + nk * nk;
            // P_k[u_m, u_m'] += x_m x_m' (product of the other two Gram entries)
#pragma unroll
            for (int e0 = 0; e0 < S * S; e0 += 32) {
                const int e = e0 + lane;
                const int m = e / S, m2 = e % S;
                const int qa = __shfl_sync(kAll, myq, m & 31), qb = __shfl_sync(kAll, myq, m2);
                const float xa = __shfl_sync(kAll, myx, m & 31), xb = __shfl_sync(kAll, myx, m2);
                if (m < cnt && m2 < cnt) {
                    const int ia = qa % N1, ja = (qa / N1) % N2, la = qa / N12;
                    const int ib = qb % N1, jb = (qb / N1) % N2, lb = qb / N12;
                    float f = xa * xb;
                    int u, v;
                    if constexpr (MODE == 1) {
                        f *= sG2[ja * N2 + jb] * sG3[la * N3 + lb];
                        u = ia; v = ib;
                    } else if constexpr (MODE == 2) {
                        f *= sG1[ia * N1 + ib] * sG3[la * N3 + lb];
                        u = ja; v = jb;
                    } else {
                        f *= sG1[ia * N1 + ib] * sG2[ja * N2 + jb];
                        u = la; v = lb;
                    }
                    atomicAdd(&accP[u * nk + v], f);
                }
            }
            // B_k[r, u_m] += x_m (Y contracted with the other two atoms of pick m)
#pragma unroll
            for (int e0 = 0; e0 < S * pk; e0 += 32) {
                const int e = e0 + lane;
                const int m = e / pk, r = e % pk;
                const int qm = __shfl_sync(kAll, myq, m & 31);
                const float xm = __shfl_sync(kAll, myx, m & 31);
                if (m < cnt) {
                    const int im = qm % N1, jm = (qm / N1) % N2, lm = qm / N12;
                    float t = 0.f;
                    int um;
                    if constexpr (MODE == 1) {          // r = a: sum_b D2[b, j_m] T1[a, b, l_m]
#pragma unroll
                        for (int bb2 = 0; bb2 < P2; ++bb2)
                            t = fmaf(sD2[bb2 * N2 + jm], T1[r * (P2 * N3) + bb2 + P2 * lm], t);
                        um = im;
                    } else if constexpr (MODE == 2) {   // r = b: sum_a D1[a, i_m] T1[a, b, l_m]
#pragma unroll
                        for (int a = 0; a < P1; ++a)
                            t = fmaf(sD1[a * N1 + im], T1[a * (P2 * N3) + r + P2 * lm], t);
                        um = jm;
                    } else {                            // r = c: sum_b D2[b, j_m] sum_a D1[a, i_m] Y[a, b, c]
#pragma unroll
                        for (int bb2 = 0; bb2 < P2; ++bb2) {
                            float ua = 0.f;
#pragma unroll
                            for (int a = 0; a < P1; ++a)
                                ua = fmaf(Ys[a + P1 * bb2 + P12 * r], sD1[a * N1 + im], ua);
                            t = fmaf(ua, sD2[bb2 * N2 + jm], t);
                        }
                        um = lm;
                    }
                    atomicAdd(&accB[r * nk + um], xm * t);
                }
            }
        }
        if (lane == 0 && finite) {
            const float ye = fmaxf(E2, 0.f) - w_energy_c;
            const float te = w_energy + ye;
            w_energy_c = (te - w_energy) - ye;
            w_energy = te;
            const float yy = ss - w_ynorm_c;
            const float ty = w_ynorm + yy;
            w_ynorm_c = (ty - w_ynorm) - yy;
            w_ynorm = ty;
        }
    }

    if constexpr (MODE != 0) {
        if (lane == 0) {
            acce[2 * w] = w_energy - w_energy_c;
            acce[2 * w + 1] = w_ynorm - w_ynorm_c;
        }
        __syncthreads();
        float* dst = part_f + (size_t)blockIdx.x * nf;
        for (int e = threadIdx.x; e < nf; e += blockDim.x) {
            float v = 0.f;
            for (int ww = 0; ww < Sh::WPC; ++ww) v += sm[L::acc + ww * r4(nf) + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int ww = 0; ww < Sh::WPC; ++ww) d += (double)acce[2 * ww + threadIdx.x];
            part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = d;
        }
    }
}

template <class Sh>
int launch_fast3(int mode, const float* Y, long long N, const float* D1, const float* D2,
                 const float* D3, const float* G1, const float* G2, const float* G3,
                 int32_t* support, float* coef, int32_t* nnz, float* res, float* part_f,
                 double* part_d, int max_slots, int* err, int num_sms, cudaStream_t st) {
    using L = Layout3F<Sh>;
    const size_t bytes = sizeof(float) * (size_t)L::total(mode);
    auto run = [&](auto kern) -> int {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess)
            return SDL_ERR_CUDA;
        int bps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, Sh::WPC * 32, bytes) != cudaSuccess)
            return SDL_ERR_CUDA;
        bps = std::max(1, std::min(bps, 8));
        const long long need = (N + Sh::WPC - 1) / Sh::WPC;
        long long grid = std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
        if (mode != 0) grid = std::min<long long>(grid, max_slots);
        kern<<<(int)grid, Sh::WPC * 32, bytes, st>>>(Y, N, D1, D2, D3, G1, G2, G3, support, coef, nnz,
                                                     res, part_f, part_d, err);
        if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
        return mode == 0 ? 0 : (int)grid;
    };
    switch (mode) {
        case 0: return run(code3_fast_kernel<Sh, 0>);
        case 1: return run(code3_fast_kernel<Sh, 1>);
        case 2: return run(code3_fast_kernel<Sh, 2>);
        default: return run(code3_fast_kernel<Sh, 3>);
    }
}

// Compiled shapes: <p1, p2, p3, n1, n2, n3, s, LI, LJ>
using F3cube = Shape3F<4, 4, 16, 8, 8, 16, 8, 2, 2>;   // 4 x 4 pixels x 16 bands
using F3small = Shape3F<4, 4, 4, 8, 8, 8, 4, 2, 2>;

template <class Sh>
bool is_shape(int p1, int p2, int p3, int n1, int n2, int n3, int s) {
    return p1 == Sh::P1 && p2 == Sh::P2 && p3 == Sh::P3 && n1 == Sh::N1 && n2 == Sh::N2 &&
           n3 == Sh::N3 && s == Sh::S;
}

}  // namespace

int launch_code3_fast(int mode, const float* Y, int p1, int p2, int p3, int n1, int n2, int n3,
                      long long N, const float* D1, const float* D2, const float* D3,
                      const float* G1, const float* G2, const float* G3, int s, int32_t* support,
                      float* coef, int32_t* nnz, float* res, float* part_f, double* part_d,
                      int max_slots, int* err, int num_sms, cudaStream_t st) {
    if ((reinterpret_cast<uintptr_t>(Y) & 15u) != 0) return SDL_ERR_UNSUPPORTED;
    if (is_shape<F3cube>(p1, p2, p3, n1, n2, n3, s))
        return launch_fast3<F3cube>(mode, Y, N, D1, D2, D3, G1, G2, G3, support, coef, nnz, res,
                                    part_f, part_d, max_slots, err, num_sms, st);
    if (is_shape<F3small>(p1, p2, p3, n1, n2, n3, s))
        return launch_fast3<F3small>(mode, Y, N, D1, D2, D3, G1, G2, G3, support, coef, nnz, res,
                                     part_f, part_d, max_slots, err, num_sms, st);
    return SDL_ERR_UNSUPPORTED;
}

}  // namespace sdl
