// 2D-OMP coding passes with the TMOD partial sums fused into their epilogue.
//
// One *team* (one warp, or TW warps for large pair grids) codes one signal at
// a time; a CTA holds several teams that share the dictionaries, their Gram
// matrices and the CTA-private partial-sum accumulators in shared memory.
//
// Per signal (Sec. III step 1, 2D-OMP == 1D OMP on D2 (x) D1, Sec. II):
//   Z   = Y_k D2                       (p1 x n2, shared memory)
//   C0  = D1^T Z                       (n1 x n2, registers: thread (li, lj)
//                                       owns rows li*RI.. and cols lj*RJ..)
//   for t = 0..s-1:
//     C   = C0 - sum_l x_l G1[:, i_l] G2[j_l, :]     (correlation of the
//           residual with every pair, Gram domain, G1 = D1^T D1, G2 = D2^T D2)
//     q   = argmax |C| over unselected pairs, ties -> smallest q = i + n1*j
//     extend the Cholesky factor of A[l,l'] = G1[i_l,i_l'] G2[j_l,j_l'] by
//     one row, y_t = (b_t - w.y)/L_tt with b = C0 at the support, and
//     x = L^{-T} y (one lane per row, shuffles between lanes)
//     ||R||^2 = ||Y||^2 - ||y||^2   (least-squares energy identity)
//   epilogue (Algorithm 1 steps 1 / 3, Gram shortcut of Sec. III):
//     D1 side: B1[:, i_l] += x_l Z[:, j_l],  P[i_l, i_m] += x_l x_m G2[j_l, j_m]
//     D2 side: B2[:, j_l] += x_l Y^T d1_{i_l}, M[j_l, j_m] += x_l x_m G1[i_l, i_m]
// Selected pairs are masked by poisoning their C0 entry with NaN: fmaxf skips
// NaN, so a selected pair can never win the argmax again.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int align4(int x) { return (x + 3) & ~3; }

// Lane grid LI x LJ of a team of TW warps, each thread an RI x RJ block of the
// n1 x n2 scores; CTA threads per block (the teams it holds: CTA / (32 TW)).
template <int LI_, int LJ_, int RI_, int RJ_, int TW_, int CTA_ = 256>
struct Tile {
    static constexpr int LI = LI_, LJ = LJ_, RI = RI_, RJ = RJ_, TW = TW_, CTA = CTA_;
    static constexpr int T = 32 * TW;
    static constexpr int N1P = LI * RI, N2P = LJ * RJ;
    static_assert(LI * LJ == T, "the lane grid must cover the team");
};

// Shared-memory layout of a coding CTA, in floats (identical on host and device).
struct Layout {
    int d1r, d2r, g1, g2, acc, accd, team0, team_stride;
    int slab_L, slab_invd, slab_y, slab_x, slab_b, slab_si, slab_sj, slab_misc;
    int total;  // floats
    __host__ __device__ Layout(int p1, int p2, int N1P, int N2P, int s, int nf_smem, int tpc) {
        d1r = 0;
        d2r = d1r + align4(p1 * N1P);
        g1 = d2r + align4(p2 * N2P);
        g2 = g1 + align4(N1P * N1P);
        acc = g2 + align4(N2P * N2P);
        accd = acc + align4(nf_smem);       // 2 doubles = 4 floats, 16-byte aligned
        team0 = accd + 4;
        // team region: Y (p1*p2) | Z (p1*N2P), or W = D1^T Y (N1P*p2) when
        // C0 comes from the tensor cores | slab
        int ys = align4(p1 * p2), zs = align4(p1 * N2P > N1P * p2 ? p1 * N2P : N1P * p2);
        slab_L = ys + zs;
        slab_invd = slab_L + s * s;
        slab_y = slab_invd + s;
        slab_x = slab_y + s;
        slab_b = slab_x + s;
        slab_si = slab_b + s;
        slab_sj = slab_si + s;
        slab_misc = slab_sj + s;
        team_stride = align4(slab_misc + 32);
        total = team0 + tpc * team_stride;
    }
};

template <int TW>
__device__ __forceinline__ void team_sync(int team) {
    if constexpr (TW == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TW * 32) : "memory");
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Team-wide reductions through per-warp slots in the slab scratch area.
template <int TW>
__device__ __forceinline__ unsigned team_max_u32(unsigned v, unsigned* scratch, int wit, int lane,
                                                 int team) {
    v = __reduce_max_sync(kFull, v);
    if constexpr (TW == 1) {
        return v;
    } else {
        if (lane == 0) scratch[wit] = v;
        team_sync<TW>(team);
        unsigned r = scratch[0];
#pragma unroll
        for (int w = 1; w < TW; ++w) r = max(r, scratch[w]);
        return r;
    }
}

template <int TW>
__device__ __forceinline__ unsigned team_min_u32(unsigned v, unsigned* scratch, int wit, int lane,
                                                 int team) {
    v = __reduce_min_sync(kFull, v);
    if constexpr (TW == 1) {
        return v;
    } else {
        if (lane == 0) scratch[wit] = v;
        team_sync<TW>(team);
        unsigned r = scratch[0];
#pragma unroll
        for (int w = 1; w < TW; ++w) r = min(r, scratch[w]);
        return r;
    }
}

// The team's smallest candidate pair index and the C0 value its owner holds:
// each warp's minimum (candidates are distinct pair indices, so one lane
// holds it) with its value, then the minimum over the warps.  Returns q
// (0xffffffff when no thread has a candidate) and sets b.
template <int TW>
__device__ __forceinline__ unsigned team_min_pick(unsigned cand, float bc, float& b, unsigned* scratch,
                                                  float* bscratch, int wit, int lane, int team) {
    static_assert(TW <= 6, "one value slot per warp");
    const unsigned wmin = __reduce_min_sync(kFull, cand);
    const unsigned holder = __ballot_sync(kFull, cand == wmin && wmin != 0xffffffffu);
    const float wb = __shfl_sync(kFull, bc, holder ? __ffs(holder) - 1 : 0);
    if constexpr (TW == 1) {
        b = wb;
        return wmin;
    } else {
        if (lane == 0) {
            scratch[wit] = wmin;
            bscratch[wit] = wb;
        }
        team_sync<TW>(team);
        unsigned r = scratch[0];
        float rb = bscratch[0];
#pragma unroll
        for (int w = 1; w < TW; ++w)
            if (scratch[w] < r) {
                r = scratch[w];
                rb = bscratch[w];
            }
        b = rb;
        return r;
    }
}

template <int TW>
__device__ __forceinline__ float team_sum_f32(float v, float* scratch, int wit, int lane, int team) {
    v = warp_sum(v);
    if constexpr (TW == 1) {
        return v;
    } else {
        if (lane == 0) scratch[wit] = v;
        team_sync<TW>(team);
        float r = 0.f;
#pragma unroll
        for (int w = 0; w < TW; ++w) r += scratch[w];
        return r;
    }
}

// blk[r][c] += a[r] * b[c] over an R x C register block, packed in pairs along
// c with fma.rn.f32x2 when C is even (each half rounds exactly as fmaf)
template <int R, int C>
__device__ __forceinline__ void rank1_rc(float (&blk)[R][C], const float (&a)[R], const float (&b)[C]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if constexpr (C % 2 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                const unsigned long long A =
                    ((unsigned long long)__float_as_uint(a[r]) << 32) | __float_as_uint(a[r]);
                const unsigned long long B =
                    ((unsigned long long)__float_as_uint(b[c + 1]) << 32) | __float_as_uint(b[c]);
                const unsigned long long Cc =
                    ((unsigned long long)__float_as_uint(blk[r][c + 1]) << 32) | __float_as_uint(blk[r][c]);
                unsigned long long D;
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(Cc));
                blk[r][c] = __uint_as_float((unsigned)(D & 0xffffffffu));
                blk[r][c + 1] = __uint_as_float((unsigned)(D >> 32));
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) blk[r][c] = fmaf(a[r], b[c], blk[r][c]);
        }
    }
}

// R consecutive floats from shared memory, as float4 / float2 loads when R
// allows: every block a thread reads starts at a multiple of its own length
// within rows whose lengths (N1P, N2P) and region offsets are multiples of 4
template <int R>
__device__ __forceinline__ void ldv(float (&v)[R], const float* p) {
    if constexpr (R % 4 == 0) {
#pragma unroll
        for (int k = 0; k < R; k += 4) {
            const float4 t = *reinterpret_cast<const float4*>(p + k);
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
    } else if constexpr (R % 2 == 0) {
#pragma unroll
        for (int k = 0; k < R; k += 2) {
            const float2 t = *reinterpret_cast<const float2*>(p + k);
            v[k] = t.x; v[k + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = p[k];
    }
}

// FP32 re-scoring of one correlation: w_i . d2_j over p2 terms (w_i contiguous,
// d2_j with stride ld), four interleaved partial sums so the loads and
// multiply-adds overlap.  Kept out of line: it runs for a few flagged entries
// per step, and inlining it into the unrolled per-entry loops only inflates
// register pressure.
__device__ __noinline__ float rescore_dot(const float* __restrict__ w, const float* __restrict__ d,
                                          int ld, int p2) {
    float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
    int b = 0;
    for (; b + 4 <= p2; b += 4) {
        e0 = fmaf(w[b], d[b * ld], e0);
        e1 = fmaf(w[b + 1], d[(b + 1) * ld], e1);
        e2 = fmaf(w[b + 2], d[(b + 2) * ld], e2);
        e3 = fmaf(w[b + 3], d[(b + 3) * ld], e3);
    }
    for (; b < p2; ++b) e0 = fmaf(w[b], d[b * ld], e0);
    return (e0 + e1) + (e2 + e3);
}

// misc area of the slab (32 words): [0,8) max scratch, [8,16) min scratch,
// [16,24) sum scratch, 25 = accept flag, [26,32) the C0 value of each warp's
// smallest candidate.
enum { kMiscMax = 0, kMiscMin = 8, kMiscSum = 16, kMiscOk = 25, kMiscPickB = 26 };

// Signal and dictionary sizes fixed at compile time (0: taken from the call),
// so that the contraction, re-scoring and epilogue loops of a frequent shape
// unroll with constant bounds and strides.
template <int P1, int P2, int N1, int N2, int S>
struct FixedSizes {
    static constexpr int p1 = P1, p2 = P2, n1 = N1, n2 = N2, s = S;
};
using RuntimeSizes = FixedSizes<0, 0, 0, 0, 0>;

template <class Tl, int SIDE, class FS = RuntimeSizes>
__global__ void __launch_bounds__(Tl::CTA) code_pass_kernel(PassArgs a) {
    constexpr int T = Tl::T, TW = Tl::TW, RI = Tl::RI, RJ = Tl::RJ;
    constexpr int LI = Tl::LI, N1P = Tl::N1P, N2P = Tl::N2P;
    extern __shared__ __align__(16) float smem[];

    const int p1 = FS::p1 ? FS::p1 : a.p1, p2 = FS::p2 ? FS::p2 : a.p2;
    const int n1 = FS::n1 ? FS::n1 : a.n1, n2 = FS::n2 ? FS::n2 : a.n2;
    const int s = FS::s ? FS::s : a.s;
    const int p1p2 = p1 * p2;
    const int tpc = blockDim.x / T;
    const int team = threadIdx.x / T;
    const int tau = threadIdx.x % T;
    const int lane = threadIdx.x & 31;
    const int wit = tau >> 5;
    const int li = tau % LI, lj = tau / LI;
    const int i0 = li * RI, j0 = lj * RJ;

    // which partial sums, and where they accumulate
    const int nacc = (SIDE == kSideD1) ? n1 : n2;
    const int pacc = (SIDE == kSideD1) ? p1 : p2;
    const int nf = (SIDE == kCodeOnly) ? 0 : nacc * nacc + pacc * nacc;
    const Layout L(p1, p2, N1P, N2P, s, a.acc_in_smem ? nf : 0, tpc);

    float* D1r = smem + L.d1r;          // D1 row-major p1 x N1P
    float* D2r = smem + L.d2r;          // D2 row-major p2 x N2P
    float* G1s = smem + L.g1;           // G1 column-major N1P x N1P (symmetric)
    float* G2s = smem + L.g2;
    double* accd = reinterpret_cast<double*>(smem + L.accd);
    float* acc = nullptr;
    if constexpr (SIDE != kCodeOnly) {
        acc = a.acc_in_smem ? smem + L.acc : a.part_f + (size_t)(blockIdx.x % a.n_slots) * nf;
    }
    float* tb = smem + L.team0 + team * L.team_stride;
    float* Ys = tb;
    float* Zs = tb + align4(p1p2);
    float* Ls = tb + L.slab_L;
    float* invd = tb + L.slab_invd;
    float* yv = tb + L.slab_y;
    float* xv = tb + L.slab_x;
    int* si = reinterpret_cast<int*>(tb + L.slab_si);
    int* sj = reinterpret_cast<int*>(tb + L.slab_sj);
    unsigned* misc = reinterpret_cast<unsigned*>(tb + L.slab_misc);
    float* miscf = reinterpret_cast<float*>(misc);

    for (int e = threadIdx.x; e < p1 * N1P; e += blockDim.x) {
        int r = e / N1P, i = e - r * N1P;
        D1r[e] = (i < n1) ? a.D1[r + p1 * i] : 0.f;
    }
    for (int e = threadIdx.x; e < p2 * N2P; e += blockDim.x) {
        int r = e / N2P, j = e - r * N2P;
        D2r[e] = (j < n2) ? a.D2[r + p2 * j] : 0.f;
    }
    for (int e = threadIdx.x; e < N1P * N1P; e += blockDim.x) {
        int c = e / N1P, r = e - c * N1P;
        G1s[e] = (r < n1 && c < n1) ? a.G1[r * n1 + c] : 0.f;
    }
    for (int e = threadIdx.x; e < N2P * N2P; e += blockDim.x) {
        int c = e / N2P, r = e - c * N2P;
        G2s[e] = (r < n2 && c < n2) ? a.G2[r * n2 + c] : 0.f;
    }
    if constexpr (SIDE != kCodeOnly) {
        if (a.acc_in_smem)
            for (int e = threadIdx.x; e < nf; e += blockDim.x) acc[e] = 0.f;
        if (threadIdx.x < 2) accd[threadIdx.x] = 0.0;
    }
    __syncthreads();

    double team_energy = 0.0, team_ynorm = 0.0;
    const long long stride = (long long)gridDim.x * tpc;
    for (long long k = (long long)blockIdx.x * tpc + team; k < a.N; k += stride) {
        // ---- stage Y_k, ||Y_k||^2
        const float* Yk = a.Y + (size_t)k * p1p2;
        float ss = 0.f;
        for (int e = tau; e < p1p2; e += T) {
            float v = __ldg(Yk + e);
            Ys[e] = v;
            ss = fmaf(v, v, ss);
        }
        ss = team_sum_f32<TW>(ss, miscf + kMiscSum, wit, lane, team);
        team_sync<TW>(team);
        const bool finite = isfinite(ss);
        if (!finite && tau == 0) record_error(a.err, SDL_ERR_NONFINITE);

        int cnt = 0;
        float E = ss;
        // a signal already within the error target takes no atom: skip its correlations
        if (finite && !(a.eps2 > 0.f && ss <= a.eps2)) {
            float c0[RI][RJ];
            unsigned long long exact = ~0ull;  // bit r*RJ+c: c0 entry is an FP32 value
            static_assert(RI * RJ <= 64, "one flag bit per entry");
            const float bound = a.c0ext ? a.c0_err_rel * sqrtf(ss) : 0.f;
            if (!a.c0ext) {
                // ---- Z = Y D2 (p1 x N2P, row-major).  When p1 is a multiple
                // of 4, a thread forms 4 x 4 blocks: per b one float4 of Y's
                // column b and one of D2's row b, 16 independent FMA chains
                // (each entry still sums over b in order, as the scalar form)
                if ((p1 & 3) == 0) {
                    const int nbj = N2P / 4, nb = (p1 / 4) * nbj;
                    for (int e = tau; e < nb; e += T) {
                        const int a0 = (e / nbj) * 4, j0z = (e % nbj) * 4;
                        float z[4][4];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) z[r][c] = 0.f;
                        for (int b = 0; b < p2; ++b) {
                            const float4 y4 = *reinterpret_cast<const float4*>(Ys + a0 + p1 * b);
                            const float4 d4 = *reinterpret_cast<const float4*>(D2r + b * N2P + j0z);
                            const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
                            const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
                            rank1_rc<4, 4>(z, yv, dv);
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            *reinterpret_cast<float4*>(Zs + (a0 + r) * N2P + j0z) =
                                make_float4(z[r][0], z[r][1], z[r][2], z[r][3]);
                    }
                } else {
                    for (int e = tau; e < p1 * N2P; e += T) {
                        int r = e / N2P, j = e - r * N2P;
                        float z = 0.f;
                        for (int b = 0; b < p2; ++b) z = fmaf(Ys[r + p1 * b], D2r[b * N2P + j], z);
                        Zs[e] = z;
                    }
                }
                team_sync<TW>(team);
                // ---- C0 = D1^T Z on this thread's (RI x RJ) block
#pragma unroll
                for (int r = 0; r < RI; ++r)
#pragma unroll
                    for (int c = 0; c < RJ; ++c) c0[r][c] = 0.f;
                for (int aa = 0; aa < p1; ++aa) {
                    float u[RI], v[RJ];
                    ldv<RI>(u, D1r + aa * N1P + i0);
                    ldv<RJ>(v, Zs + aa * N2P + j0);
                    rank1_rc<RI, RJ>(c0, u, v);
                }
            } else {
                // ---- C0 from the tensor-core correlations (approximate)
                const float* cg = a.c0ext + (size_t)k * a.ldc0;
#pragma unroll
                for (int r = 0; r < RI; ++r)
#pragma unroll
                    for (int c = 0; c < RJ; ++c)
                        c0[r][c] = (i0 + r < n1 && j0 + c < n2) ? cg[(i0 + r) + n1 * (j0 + c)] : 0.f;
                if (bound > 0.f) {
                    exact = 0ull;
                    // W = D1^T Y (n1 x p2, row i contiguous) in the Z area:
                    // a re-scored entry is then w_i . d2_j, p2 FMAs
                    float* Ws = Zs;
                    for (int e = tau; e < n1 * p2; e += T) {
                        const int i = e / p2, b = e - i * p2;
                        float w = 0.f;
                        for (int aa = 0; aa < p1; ++aa) w = fmaf(D1r[aa * N1P + i], Ys[aa + p1 * b], w);
                        Ws[e] = w;
                    }
                    team_sync<TW>(team);
                }
            }
#pragma unroll
            for (int r = 0; r < RI; ++r)
#pragma unroll
                for (int c = 0; c < RJ; ++c)
                    if (i0 + r >= n1 || j0 + c >= n2) c0[r][c] = __int_as_float(0x7fc00000);

            // ---- greedy steps
            for (int t = 0; t < s; ++t) {
                if (a.eps2 > 0.f && E <= a.eps2) break;
                float sc[RI][RJ];
#pragma unroll
                for (int r = 0; r < RI; ++r)
#pragma unroll
                    for (int c = 0; c < RJ; ++c) sc[r][c] = c0[r][c];
                for (int l = 0; l < t; ++l) {
                    const int il = si[l], jl = sj[l];
                    const float xl = xv[l];
                    float u[RI], v[RJ];
                    ldv<RI>(u, G1s + il * N1P + i0);
                    ldv<RJ>(v, G2s + jl * N2P + j0);
#pragma unroll
                    for (int c = 0; c < RJ; ++c) v[c] *= -xl;
                    rank1_rc<RI, RJ>(sc, u, v);
                }
                float m = 0.f;
#pragma unroll
                for (int r = 0; r < RI; ++r)
#pragma unroll
                    for (int c = 0; c < RJ; ++c) m = fmaxf(m, fabsf(sc[r][c]));
                unsigned Mu = team_max_u32<TW>(__float_as_uint(m), misc + kMiscMax, wit, lane, team);
                if (bound > 0.f) {
                    // FP32 re-scoring, one pass: every approximate entry within
                    // 3*bound of the approximate maximum Mu gets its FP32
                    // correlation (d1_i^T Y) d2_j.  The entry at Mu is among them
                    // and its FP32 score is >= Mu - bound - e (e: FP32 rounding,
                    // far below bound); an entry left approximate has |score| <
                    // Mu - 3*bound, so its FP32 score is < Mu - 2*bound + e.  The
                    // new maximum is therefore an FP32 value and the pick is the
                    // pick over FP32 scores.
                    const float thr = __uint_as_float(Mu) - 3.f * bound;
                    unsigned did = 0;
#pragma unroll
                    for (int r = 0; r < RI; ++r)
#pragma unroll
                        for (int c = 0; c < RJ; ++c) {
                            const int e = r * RJ + c;
                            if (!((exact >> e) & 1ull) && fabsf(sc[r][c]) >= thr) {
                                const int i = i0 + r, j = j0 + c;
                                const float ex = rescore_dot(Zs + i * p2, D2r + j, N2P, p2);
                                sc[r][c] = ex - (c0[r][c] - sc[r][c]);
                                c0[r][c] = ex;
                                exact |= 1ull << e;
                                ++did;
                            }
                        }
                    if (a.rescored && did) atomicAdd(a.rescored, (unsigned long long)did);
                    m = 0.f;
#pragma unroll
                    for (int r = 0; r < RI; ++r)
#pragma unroll
                        for (int c = 0; c < RJ; ++c) m = fmaxf(m, fabsf(sc[r][c]));
                    Mu = team_max_u32<TW>(__float_as_uint(m), misc + kMiscSum, wit, lane, team);
                }
                if (Mu == 0u) break;  // every remaining score is exactly 0
                const float Mf = __uint_as_float(Mu);
                unsigned cand = 0xffffffffu;
                float bc = 0.f;   // C0 at this thread's candidate
                // only a thread whose own maximum is the team's holds a
                // candidate: the others (mostly whole warps) skip the search
                if (m == Mf) {
#pragma unroll
                    for (int r = 0; r < RI; ++r)
#pragma unroll
                        for (int c = 0; c < RJ; ++c) {
                            const unsigned qe = (unsigned)(i0 + r + n1 * (j0 + c));
                            if (fabsf(sc[r][c]) == Mf && qe < cand) {
                                cand = qe;
                                bc = c0[r][c];
                            }
                        }
                }
                // the pick and b_t = C0[q] arrive together; the owner masks it
                float b;
                const unsigned q = team_min_pick<TW>(cand, bc, b, misc + kMiscMin, miscf + kMiscPickB,
                                                     wit, lane, team);
                const int it = (int)(q % (unsigned)n1), jt = (int)(q / (unsigned)n1);
                const int owner = it / RI + LI * (jt / RJ);
                const int rt = it % RI, ct = jt % RJ;
                if (tau == owner) {
#pragma unroll
                    for (int r = 0; r < RI; ++r)
#pragma unroll
                        for (int c = 0; c < RJ; ++c)
                            if (r == rt && c == ct) c0[r][c] = __int_as_float(0x7fc00000);
                }
                // ---- Cholesky row + solves, warp 0 of the team
                if (wit == 0) {
                    float al = 0.f;
                    if (lane < t) al = G1s[si[lane] * N1P + it] * G2s[sj[lane] * N2P + jt];
                    const float Att = G1s[it * N1P + it] * G2s[jt * N2P + jt];
                    float rr = al, ww = 0.f, wy = 0.f;
                    for (int mm = 0; mm < t; ++mm) {
                        const float wm = __shfl_sync(kFull, rr, mm) * invd[mm];
                        if (lane == mm) Ls[t * s + mm] = wm;
                        if (lane > mm && lane < t) rr = fmaf(-Ls[lane * s + mm], wm, rr);
                        ww = fmaf(wm, wm, ww);
                        wy = fmaf(wm, yv[mm], wy);
                    }
                    const float d = Att - ww;
                    const bool ok = d > kPivotRel * Att;
                    if (ok) {
                        const float Ltt = sqrtf(d);
                        const float inv = 1.f / Ltt;
                        const float yt = (b - wy) * inv;
                        if (lane == 0) {
                            Ls[t * s + t] = Ltt;
                            invd[t] = inv;
                            yv[t] = yt;
                            si[t] = it;
                            sj[t] = jt;
                        }
                        __syncwarp();
                        // back substitution x = L^{-T} y over rows 0..t
                        float xr = (lane <= t) ? yv[lane] : 0.f;
                        for (int kk = t; kk >= 0; --kk) {
                            const float xk = __shfl_sync(kFull, xr, kk) * invd[kk];
                            if (lane == kk) xv[kk] = xk;
                            if (lane < kk) xr = fmaf(-Ls[kk * s + lane], xk, xr);
                        }
                    }
                    if (lane == 0) misc[kMiscOk] = ok ? 1u : 0u;
                }
                team_sync<TW>(team);
                if (misc[kMiscOk] == 0u) break;
                const float yt = yv[t];
                E = fmaf(-yt, yt, E);
                cnt = t + 1;
            }
        }

        // ---- emit the code
        if (a.support) {
            for (int l = tau; l < s; l += T) {
                a.support[(size_t)k * s + l] = (l < cnt) ? si[l] + n1 * sj[l] : -1;
                a.coef[(size_t)k * s + l] = (l < cnt) ? xv[l] : 0.f;
            }
        }
        if (tau == 0) {
            if (a.nnz) a.nnz[k] = cnt;
            if (a.res_energy) a.res_energy[k] = finite ? fmaxf(E, 0.f) : __int_as_float(0x7fc00000);
        }

        // ---- fused partial sums of the dictionary update
        if constexpr (SIDE == kSideD1) {
            float* accP = acc;
            float* accB = acc + n1 * n1;
            for (int e = tau; e < p1 * cnt; e += T) {
                const int l = e / p1, r = e - l * p1;
                float z;
                if (a.c0ext) {   // no Z stage ran: (Y D2)[r, j_l] here
                    z = 0.f;
                    for (int b = 0; b < p2; ++b) z = fmaf(Ys[r + p1 * b], D2r[b * N2P + sj[l]], z);
                } else {
                    z = Zs[r * N2P + sj[l]];
                }
                atomicAdd(&accB[r * n1 + si[l]], xv[l] * z);
            }
            for (int e = tau; e < cnt * cnt; e += T) {
                const int l = e / cnt, m2 = e - l * cnt;
                atomicAdd(&accP[si[l] * n1 + si[m2]], xv[l] * xv[m2] * G2s[sj[l] * N2P + sj[m2]]);
            }
        } else if constexpr (SIDE == kSideD2) {
            float* accM = acc;
            float* accB = acc + n2 * n2;
            // B2[b, j_l] += x_l (Y^T d1_{i_l})[b]
            if ((p1 & 3) == 0 && p1 <= 16) {
                // a thread keeps column b of Y in registers for every pick it takes
                const int LG = T / p2 > 1 ? T / p2 : 1;
                for (int e = tau; e < p2 * LG; e += T) {
                    const int bb = e % p2, g = e / p2;
                    float yc[16];
#pragma unroll
                    for (int r = 0; r < 16; r += 4) {
                        const float4 v = r < p1 ? *reinterpret_cast<const float4*>(Ys + p1 * bb + r)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                        yc[r] = v.x; yc[r + 1] = v.y; yc[r + 2] = v.z; yc[r + 3] = v.w;
                    }
                    for (int l = g; l < cnt; l += LG) {
                        const int il = si[l];
                        float w = 0.f;
#pragma unroll
                        for (int r = 0; r < 16; ++r)
                            if (r < p1) w = fmaf(yc[r], D1r[r * N1P + il], w);
                        atomicAdd(&accB[bb * n2 + sj[l]], xv[l] * w);
                    }
                }
            } else {
                for (int e = tau; e < p2 * cnt; e += T) {
                    const int l = e / p2, bb = e - l * p2;
                    const int il = si[l];
                    float w = 0.f;
                    for (int r = 0; r < p1; ++r) w = fmaf(Ys[r + p1 * bb], D1r[r * N1P + il], w);
                    atomicAdd(&accB[bb * n2 + sj[l]], xv[l] * w);
                }
            }
            for (int e = tau; e < cnt * cnt; e += T) {
                const int l = e / cnt, m2 = e - l * cnt;
                atomicAdd(&accM[sj[l] * n2 + sj[m2]], xv[l] * xv[m2] * G1s[si[l] * N1P + si[m2]]);
            }
        }
        if (tau == 0 && finite) {
            team_energy += (double)fmaxf(E, 0.f);
            team_ynorm += (double)ss;
        }
        team_sync<TW>(team);  // slab and Y/Z buffers are reused by the next signal
    }

    if constexpr (SIDE != kCodeOnly) {
        if (tau == 0) {
            atomicAdd(&accd[0], team_energy);
            atomicAdd(&accd[1], team_ynorm);
        }
        __syncthreads();
        if (a.acc_in_smem) {
            float* dst = a.part_f + (size_t)blockIdx.x * nf;
            for (int e = threadIdx.x; e < nf; e += blockDim.x) dst[e] = acc[e];
            if (threadIdx.x < 2) a.part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = accd[threadIdx.x];
        } else if (threadIdx.x < 2) {
            atomicAdd(&a.part_d[(size_t)(blockIdx.x % a.n_slots) * 2 + threadIdx.x], accd[threadIdx.x]);
        }
    }
}

// Accumulation-only pass for the stand-alone dictionary updates: codes are
// given, so each warp forms the partial sums of one signal at a time, plus
// the exact residual energy ||Y_k - D1 X_k D2^T||^2 of the objective before
// the update.
struct AccLayout {
    int d1, d2, g, acc, accd, warp0, warp_stride, total;
    __host__ __device__ AccLayout(int p1, int p2, int n1, int n2, int ng, int s, int nf, int wpc) {
        d1 = 0;
        d2 = d1 + align4(p1 * n1);
        g = d2 + align4(p2 * n2);
        acc = g + align4(ng * ng);
        accd = acc + align4(nf);
        warp0 = accd + 4;
        warp_stride = align4(p1 * p2) + align4(3 * s);
        total = warp0 + wpc * warp_stride;
    }
};

template <int SIDE>
__global__ void __launch_bounds__(256) accumulate_kernel(PassArgs a) {
    extern __shared__ __align__(16) float smem[];
    const int p1 = a.p1, p2 = a.p2, n1 = a.n1, n2 = a.n2, s = a.s;
    const int p1p2 = p1 * p2;
    const int wpc = blockDim.x / 32;
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int ng = (SIDE == kSideD1) ? n2 : n1;       // Gram used by the shortcut
    const int nacc = (SIDE == kSideD1) ? n1 : n2;
    const int pacc = (SIDE == kSideD1) ? p1 : p2;
    const int nf = nacc * nacc + pacc * nacc;
    const AccLayout L(p1, p2, n1, n2, ng, s, a.acc_in_smem ? nf : 0, wpc);
    float* D1s = smem + L.d1;   // column-major p1 x n1
    float* D2s = smem + L.d2;   // column-major p2 x n2
    float* Gs = smem + L.g;     // row-major ng x ng
    double* accd = reinterpret_cast<double*>(smem + L.accd);
    float* acc = a.acc_in_smem ? smem + L.acc : a.part_f + (size_t)(blockIdx.x % a.n_slots) * nf;
    float* Ys = smem + L.warp0 + w * L.warp_stride;
    float* xv = Ys + align4(p1p2);
    int* si = reinterpret_cast<int*>(xv + s);
    int* sj = si + s;
    const float* Gsrc = (SIDE == kSideD1) ? a.G2 : a.G1;

    for (int e = threadIdx.x; e < p1 * n1; e += blockDim.x) D1s[e] = a.D1[e];
    for (int e = threadIdx.x; e < p2 * n2; e += blockDim.x) D2s[e] = a.D2[e];
    for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) Gs[e] = Gsrc[e];
    if (a.acc_in_smem)
        for (int e = threadIdx.x; e < nf; e += blockDim.x) acc[e] = 0.f;
    if (threadIdx.x < 2) accd[threadIdx.x] = 0.0;
    __syncthreads();

    double warp_energy = 0.0, warp_ynorm = 0.0;
    const long long stride = (long long)gridDim.x * wpc;
    for (long long k = (long long)blockIdx.x * wpc + w; k < a.N; k += stride) {
        const float* Yk = a.Y + (size_t)k * p1p2;
        for (int e = lane; e < p1p2; e += 32) Ys[e] = __ldg(Yk + e);
        // compact the used slots of X_k
        int q = -1;
        float x = 0.f;
        if (lane < s) {
            q = a.in_support[(size_t)k * s + lane];
            x = a.in_coef[(size_t)k * s + lane];
        }
        const bool valid = (lane < s) && q >= 0 && q < n1 * n2 && x != 0.f;
        const unsigned vm = __ballot_sync(kFull, valid);
        const int cnt = __popc(vm);
        if (valid) {
            const int pos = __popc(vm & ((1u << lane) - 1u));
            xv[pos] = x;
            si[pos] = q % n1;
            sj[pos] = q / n1;
        }
        __syncwarp();
        // exact residual energy with the current dictionaries
        float e2 = 0.f, y2 = 0.f;
        for (int e = lane; e < p1p2; e += 32) {
            const int r = e % p1, bb = e / p1;
            float rec = 0.f;
            for (int l = 0; l < cnt; ++l) rec = fmaf(xv[l] * D1s[r + p1 * si[l]], D2s[bb + p2 * sj[l]], rec);
            const float res = Ys[e] - rec;
            e2 = fmaf(res, res, e2);
            y2 = fmaf(Ys[e], Ys[e], y2);
        }
        e2 = warp_sum(e2);
        y2 = warp_sum(y2);
        if (!isfinite(y2)) {
            if (lane == 0) record_error(a.err, SDL_ERR_NONFINITE);
            __syncwarp();
            continue;
        }
        if constexpr (SIDE == kSideD1) {
            float* accP = acc;
            float* accB = acc + n1 * n1;
            for (int e = lane; e < p1 * cnt; e += 32) {
                const int l = e / p1, r = e - l * p1;
                const float* d2 = D2s + p2 * sj[l];
                float z = 0.f;
                for (int bb = 0; bb < p2; ++bb) z = fmaf(Ys[r + p1 * bb], d2[bb], z);
                atomicAdd(&accB[r * n1 + si[l]], xv[l] * z);
            }
            for (int e = lane; e < cnt * cnt; e += 32) {
                const int l = e / cnt, m2 = e - l * cnt;
                atomicAdd(&accP[si[l] * n1 + si[m2]], xv[l] * xv[m2] * Gs[sj[l] * n2 + sj[m2]]);
            }
        } else {
            float* accM = acc;
            float* accB = acc + n2 * n2;
            for (int e = lane; e < p2 * cnt; e += 32) {
                const int l = e / p2, bb = e - l * p2;
                const float* d1 = D1s + p1 * si[l];
                float z = 0.f;
                for (int r = 0; r < p1; ++r) z = fmaf(Ys[r + p1 * bb], d1[r], z);
                atomicAdd(&accB[bb * n2 + sj[l]], xv[l] * z);
            }
            for (int e = lane; e < cnt * cnt; e += 32) {
                const int l = e / cnt, m2 = e - l * cnt;
                atomicAdd(&accM[sj[l] * n2 + sj[m2]], xv[l] * xv[m2] * Gs[si[l] * n1 + si[m2]]);
            }
        }
        if (lane == 0) {
            warp_energy += (double)e2;
            warp_ynorm += (double)y2;
        }
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&accd[0], warp_energy);
        atomicAdd(&accd[1], warp_ynorm);
    }
    __syncthreads();
    if (a.acc_in_smem) {
        float* dst = a.part_f + (size_t)blockIdx.x * nf;
        for (int e = threadIdx.x; e < nf; e += blockDim.x) dst[e] = acc[e];
        if (threadIdx.x < 2) a.part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = accd[threadIdx.x];
    } else if (threadIdx.x < 2) {
        atomicAdd(&a.part_d[(size_t)(blockIdx.x % a.n_slots) * 2 + threadIdx.x], accd[threadIdx.x]);
    }
}

constexpr int kMaxSmem = 200 * 1024;
constexpr int kCtaSlotsPerSm = 8;
constexpr int kGlobalSlots = 64;

// plan_only: return the partial-sum slots the launch would write, launch nothing
template <class Tl, int SIDE, class FS = RuntimeSizes>
int launch_code_impl(const PassArgs& a0, cudaStream_t st, int num_sms, bool plan_only = false) {
    PassArgs a = a0;
    const int nacc = (SIDE == kSideD1) ? a.n1 : a.n2;
    const int pacc = (SIDE == kSideD1) ? a.p1 : a.p2;
    const int nf = (SIDE == kCodeOnly) ? 0 : nacc * nacc + pacc * nacc;
    int tpc = Tl::CTA / Tl::T;
    a.acc_in_smem = 1;
    size_t bytes = 0;
    for (;;) {
        bytes = sizeof(float) * (size_t)Layout(a.p1, a.p2, Tl::N1P, Tl::N2P, a.s,
                                               a.acc_in_smem ? nf : 0, tpc).total;
        if ((int)bytes <= kMaxSmem) break;
        if (a.acc_in_smem && nf > 0) {
            a.acc_in_smem = 0;  // accumulate into global slots instead
        } else if (tpc > 1) {
            --tpc;
        } else {
            return SDL_ERR_UNSUPPORTED;
        }
    }
    auto kern = code_pass_kernel<Tl, SIDE, FS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    const int threads = tpc * Tl::T;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, bytes) != cudaSuccess)
        return SDL_ERR_CUDA;
    bps = std::max(1, std::min(bps, kCtaSlotsPerSm));
    const long long need = (a.N + tpc - 1) / tpc;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
    int slots = 0;
    if (SIDE != kCodeOnly) {
        slots = a.acc_in_smem ? grid : std::min(grid, kGlobalSlots);
        if (plan_only) return slots;
        if (!a.acc_in_smem) {
            a.n_slots = slots;
            if (cudaMemsetAsync(a.part_f, 0, sizeof(float) * (size_t)slots * nf, st) != cudaSuccess ||
                cudaMemsetAsync(a.part_d, 0, sizeof(double) * 2 * (size_t)slots, st) != cudaSuccess)
                return SDL_ERR_CUDA;
        }
    } else if (plan_only) {
        return 0;
    }
    kern<<<grid, threads, bytes, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return slots;
}

template <int SIDE>
int launch_acc_impl(const PassArgs& a0, cudaStream_t st, int num_sms) {
    PassArgs a = a0;
    const int ng = (SIDE == kSideD1) ? a.n2 : a.n1;
    const int nacc = (SIDE == kSideD1) ? a.n1 : a.n2;
    const int pacc = (SIDE == kSideD1) ? a.p1 : a.p2;
    const int nf = nacc * nacc + pacc * nacc;
    int wpc = 8;
    a.acc_in_smem = 1;
    size_t bytes = 0;
    for (;;) {
        bytes = sizeof(float) *
                (size_t)AccLayout(a.p1, a.p2, a.n1, a.n2, ng, a.s, a.acc_in_smem ? nf : 0, wpc).total;
        if ((int)bytes <= kMaxSmem) break;
        if (a.acc_in_smem) {
            a.acc_in_smem = 0;
        } else if (wpc > 1) {
            --wpc;
        } else {
            return SDL_ERR_UNSUPPORTED;
        }
    }
    auto kern = accumulate_kernel<SIDE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, wpc * 32, bytes) != cudaSuccess)
        return SDL_ERR_CUDA;
    bps = std::max(1, std::min(bps, kCtaSlotsPerSm));
    const long long need = (a.N + wpc - 1) / wpc;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
    int slots;
    if (a.acc_in_smem) {
        slots = grid;
    } else {
        slots = std::min(grid, kGlobalSlots);
        a.n_slots = slots;
        if (cudaMemsetAsync(a.part_f, 0, sizeof(float) * (size_t)slots * nf, st) != cudaSuccess ||
            cudaMemsetAsync(a.part_d, 0, sizeof(double) * 2 * (size_t)slots, st) != cudaSuccess)
            return SDL_ERR_CUDA;
    }
    kern<<<grid, wpc * 32, bytes, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return slots;
}

// Compiled tile shapes: (lane grid LI x LJ, per-thread block RI x RJ, warps).
using Tile16 = Tile<4, 8, 4, 2, 1>;      // n1, n2 <= 16
using Tile24 = Tile<4, 8, 6, 3, 1>;      // n1, n2 <= 24
using Tile32 = Tile<4, 8, 8, 4, 1>;      // n1, n2 <= 32
// n1 <= 32, n2 <= 128: FP32 correlations on six four-warp teams per 768-thread
// CTA (24 warps per SM at 80 registers, 8 x 4 blocks); correlations from the
// tensor cores with FP32 re-scoring on four per 512-thread CTA (16 warps at
// 128 registers, 4 x 8 blocks), where the re-scoring needs the registers
using Tile32x128 = Tile<4, 32, 8, 4, 4, 768>;
using Tile32x128R = Tile<8, 16, 4, 8, 4, 512>;
using Tile128x32 = Tile<16, 8, 8, 4, 4>; // n1 <= 128, n2 <= 32
using Tile64 = Tile<8, 16, 8, 4, 4>;     // n1, n2 <= 64

template <int SIDE>
int dispatch_code(const PassArgs& a, cudaStream_t st, int num_sms, bool plan_only = false) {
    const int n1 = a.n1, n2 = a.n2;
    if (n1 <= 16 && n2 <= 16) return launch_code_impl<Tile16, SIDE>(a, st, num_sms, plan_only);
    if (n1 <= 24 && n2 <= 24) return launch_code_impl<Tile24, SIDE>(a, st, num_sms, plan_only);
    if (n1 <= 32 && n2 <= 32) return launch_code_impl<Tile32, SIDE>(a, st, num_sms, plan_only);
    if (n1 <= 32 && n2 <= 128) {
        auto run = [&](auto tl) {
            using Tl = decltype(tl);
            // the hyperspectral-shaped problem (16 x 64 signals, 32 x 128
            // atoms, and s = 10) with its sizes fixed at compile time
            if (a.p1 == 16 && a.p2 == 64 && n1 == 32 && n2 == 128) {
                if (a.s == 10)
                    return launch_code_impl<Tl, SIDE, FixedSizes<16, 64, 32, 128, 10>>(a, st, num_sms,
                                                                                      plan_only);
                return launch_code_impl<Tl, SIDE, FixedSizes<16, 64, 32, 128, 0>>(a, st, num_sms,
                                                                                 plan_only);
            }
            return launch_code_impl<Tl, SIDE>(a, st, num_sms, plan_only);
        };
        return a.c0ext ? run(Tile32x128R{}) : run(Tile32x128{});
    }
    if (n1 <= 128 && n2 <= 32) return launch_code_impl<Tile128x32, SIDE>(a, st, num_sms, plan_only);
    if (n1 <= 64 && n2 <= 64) return launch_code_impl<Tile64, SIDE>(a, st, num_sms, plan_only);
    return SDL_ERR_UNSUPPORTED;
}

}  // namespace

bool code_shape_supported(int p1, int p2, int n1, int n2, int s) {
    if (p1 < 1 || p2 < 1 || n1 < 1 || n2 < 1 || s < 1) return false;
    if (p1 > kMaxP || p2 > kMaxP || p1 * p2 > 1024) return false;
    if (s > kMaxS || s > p1 * p2 || s > n1 * n2) return false;
    const bool tile = (n1 <= 32 && n2 <= 128) || (n1 <= 128 && n2 <= 32) || (n1 <= 64 && n2 <= 64);
    return tile;
}

int max_partial_slots(int num_sms) { return std::max(num_sms * kCtaSlotsPerSm, kGlobalSlots); }

int launch_code_pass(const PassArgs& a, int side, cudaStream_t st, int num_sms) {
    // the specialised kernels fetch signals with 16-byte TMA bulk copies; the
    // tensor-core correlation path runs on the generic kernel
    if (!a.c0ext && (reinterpret_cast<uintptr_t>(a.Y) & 15u) == 0) {
        const int r = launch_code_pass_fast(a, side, st, num_sms);
        if (r != SDL_ERR_UNSUPPORTED) return r;
    }
    switch (side) {
        case kCodeOnly: return dispatch_code<kCodeOnly>(a, st, num_sms);
        case kSideD1: return dispatch_code<kSideD1>(a, st, num_sms);
        case kSideD2: return dispatch_code<kSideD2>(a, st, num_sms);
        default: return SDL_ERR_ARG;
    }
}

int launch_code_pass_generic(const PassArgs& a, int side, cudaStream_t st, int num_sms,
                             bool plan_only) {
    switch (side) {
        case kCodeOnly: return dispatch_code<kCodeOnly>(a, st, num_sms, plan_only);
        case kSideD1: return dispatch_code<kSideD1>(a, st, num_sms, plan_only);
        case kSideD2: return dispatch_code<kSideD2>(a, st, num_sms, plan_only);
        default: return SDL_ERR_ARG;
    }
}

int launch_accumulate_pass(const PassArgs& a, int side, cudaStream_t st, int num_sms) {
    switch (side) {
        case kSideD1: return launch_acc_impl<kSideD1>(a, st, num_sms);
        case kSideD2: return launch_acc_impl<kSideD2>(a, st, num_sms);
        default: return SDL_ERR_ARG;
    }
}

}  // namespace sdl
