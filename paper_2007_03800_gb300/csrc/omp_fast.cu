// 2D-OMP coding pass specialised at compile time for the common pair shapes
// (one warp per signal), with the TMOD partial sums fused into its epilogue.
//
// Same method and results as code_pass_kernel (omp_pass.cu); what changes is
// the schedule:
//   * every shape (p1, p2, n1, n2) and the step count s are template
//     constants, so the s greedy steps are fully unrolled and the selected
//     pairs, the coefficients, the Cholesky factor and y live in registers;
//   * lane l keeps row l of L (forward solve) and column l of L (back solve),
//     so both triangular solves are one shuffle + one FMA per row;
//   * the argmax is one compare/select pass per entry plus two redux.sync;
//   * the next signal of each warp is fetched by a TMA bulk copy
//     (cp.async.bulk, mbarrier completion) while the current one is coded;
//   * shared-memory rows of D1, G1, G2 and Z are padded so that each lane's
//     block of the n1 x n2 correlation matrix loads with 64/128-bit accesses.
// Correlation C0 = D1^T (Y D2): Z = Y D2 is formed cooperatively (a ZA x ZB
// block per lane) into shared memory, then each lane contracts its RI x RJ
// block.  The D2-side pass associates the other way, C0 = (D1^T Y) D2, because
// its partial sum B2 = sum (Y^T D1) X takes rows of W = D1^T Y.  Every tiling
// of a shape forms each entry with the same FMA chains, so all tilings give
// bit-identical results.  Scores are recomputed from C0 every step (Gram
// domain):
//   C = C0 - sum_l x_l G1[:, i_l] G2[j_l, :].
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr long long kWaitCycles = 1ll << 31;  // bounded mbarrier wait: about one second

__host__ __device__ constexpr int pad_vec(int r) { return r <= 2 ? r : ((r + 3) & ~3); }
__host__ __device__ constexpr int al4(int x) { return (x + 3) & ~3; }

template <int P1_, int P2_, int N1_, int N2_, int S_, int LI_, int RI_, int RJ_, int ZA_, int ZB_,
          int WI_, int WB_, int WPC_, int MINB_>
struct Shape {
    static constexpr int P1 = P1_, P2 = P2_, N1 = N1_, N2 = N2_, S = S_;
    static constexpr bool kHalf = false;
    static constexpr int WPC = WPC_;     // warps (= signals in flight) per CTA
    static constexpr int SPC = WPC_;     // signals in flight per CTA
    static constexpr int MINB = MINB_;   // CTAs per SM the register budget must allow
    static constexpr int LI = LI_, LJ = 32 / LI_, RI = RI_, RJ = RJ_, E = RI_ * RJ_;
    static constexpr int RIP = pad_vec(RI_), RJP = pad_vec(RJ_);
    static constexpr int LD1 = LI * RIP, LD2 = LJ * RJP;     // padded row strides
    static constexpr int ZA = ZA_, ZB = ZB_;
    static constexpr int ZLA = P1_ / ZA_, ZLB = N2_ / ZB_;   // Z-stage lane grid
    static constexpr int WI = WI_, WB = WB_;
    static constexpr int WLI = N1_ / WI_, WLB = P2_ / WB_;   // W-stage lane grid
    static constexpr int PP = P1_ * P2_;
    // lane stride of the C0 blocks in shared memory: an odd multiple of 4
    // floats, so the 8 lanes of a 128-bit load phase hit distinct banks
    static constexpr int EP = ((al4(E) / 4) % 2 == 0) ? al4(E) + 4 : al4(E);
    static_assert(LI * RI == N1 && LJ * RJ == N2, "lane grid must tile n1 x n2 exactly");
    static_assert(ZLA * ZA == P1 && ZLB * ZB == N2 && ZLA * ZLB <= 32, "Z tiling");
    static_assert(WLI * WI == N1 && WLB * WB == P2 && WLI * WLB <= 32, "W tiling");
    static_assert(S <= 32 && S <= P1 * P2 && S <= N1 * N2, "s");
    static_assert((PP * 4) % 16 == 0, "TMA bulk copies need 16-byte multiples");
};

// Two signals per warp: lanes 0-15 code one signal, lanes 16-31 another, each
// half on a 16-lane grid LI x LJ of RI x RJ blocks of the n1 x n2 correlation
// matrix.  The per-signal scalar work (pick decoding, the Cholesky recurrences
// and both triangular solves, which every lane of a signal replicates) is then
// issued once for two signals.  The first contraction is Z = Y D2 (ZA x ZB
// block per lane) for coding and the D1-side pass, and W = D1^T Y (WI x WB
// block per lane) for the D2-side pass, whose partial sum B2 takes rows of W.
// Both halves run every greedy step together (a half that has stopped only
// stops changing its state), so the maxima and picks of the two halves are
// reduced with full-warp redux.sync.  A lane updates and scans its block in two
// row halves (four argmax chains in all), and the Cholesky state lives in
// shared memory, so that registers hold half a score block at a time.
template <int P1_, int P2_, int N1_, int N2_, int S_, int LI_, int RI_, int RJ_, int ZA_, int ZB_,
          int WI_, int WB_, int WPC_, int MINB_>
struct HalfShape {
    static constexpr bool kHalf = true;
    static constexpr int P1 = P1_, P2 = P2_, N1 = N1_, N2 = N2_, S = S_;
    static constexpr int WPC = WPC_, MINB = MINB_;
    static constexpr int SPC = 2 * WPC_;
    static constexpr int LI = LI_, LJ = 16 / LI_, RI = RI_, RJ = RJ_, E = RI_ * RJ_;
    static constexpr int RIP = pad_vec(RI_), RJP = pad_vec(RJ_);
    static constexpr int LD1 = LI * RIP, LD2 = LJ * RJP;
    static constexpr int ZA = ZA_, ZB = ZB_, ZLA = P1_ / ZA_, ZLB = N2_ / ZB_;
    static constexpr int WI = WI_, WB = WB_, WLI = N1_ / WI_, WLB = P2_ / WB_;
    static constexpr int PP = P1_ * P2_;
    static constexpr int EP = ((al4(E) / 4) % 2 == 0) ? al4(E) + 4 : al4(E);
    static_assert(16 % LI_ == 0 && LI * RI == N1 && LJ * RJ == N2, "lane grid must tile n1 x n2 exactly");
    static_assert(ZLA * ZA == P1 && ZLB * ZB == N2 && ZLA * ZLB == 16 && ZA % 2 == 0, "Z tiling");
    static_assert(WLI * WI == N1 && WLB * WB == P2 && WLI * WLB == 16 && WI % 2 == 0, "W tiling");
    static_assert(P1 % 2 == 0 && N1 % 2 == 0 && P1 <= 16 && P2 <= 16, "row pairs, epilogue lanes");
    static_assert(RI_ % 4 == 0 && RIP == RI_, "two even row halves per lane block, unpadded rows");
    static_assert(E % 4 == 0, "C0 blocks stored as float4");
    static_assert(S <= 16 && S <= P1 * P2 && S <= N1 * N2, "s");
    static_assert((PP * 4) % 16 == 0, "TMA bulk copies need 16-byte multiples");
};

// padded position of correlation row i / column j inside the SMEM row layouts
template <class Sh> __device__ __forceinline__ int pos1(int i) {
    return (i / Sh::RI) * Sh::RIP + i % Sh::RI;
}
template <class Sh> __device__ __forceinline__ int pos2(int j) {
    return (j / Sh::RJ) * Sh::RJP + j % Sh::RJ;
}

template <int R>
__device__ __forceinline__ void vload(float (&v)[R], const float* p) {
    if constexpr (R % 4 == 0) {
#pragma unroll
        for (int k = 0; k < R; k += 4) {
            const float4 t = *reinterpret_cast<const float4*>(p + k);
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
    } else if constexpr (R == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (R == 3) {
        const float4 t = *reinterpret_cast<const float4*>(p);   // 4th lane is padding
        v[0] = t.x; v[1] = t.y; v[2] = t.z;
    } else if constexpr (R == 6) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        const float2 u = *reinterpret_cast<const float2*>(p + 4);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; v[4] = u.x; v[5] = u.y;
    } else {
        // 16-byte-aligned p: float4 chunks, then a float2 / float tail
#pragma unroll
        for (int k = 0; k + 4 <= R; k += 4) {
            const float4 t = *reinterpret_cast<const float4*>(p + k);
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
        constexpr int k0 = R & ~3;
        if constexpr (R - k0 >= 2) {
            const float2 t = *reinterpret_cast<const float2*>(p + k0);
            v[k0] = t.x; v[k0 + 1] = t.y;
        }
        if constexpr ((R - k0) & 1) v[R - 1] = p[R - 1];
    }
}

// d = a * b + c on two FP32 lanes at once (one packed fma.rn.f32x2: each half
// rounds exactly as fmaf, so results are bit-identical to two scalar FMAs)
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    const unsigned long long A = ((unsigned long long)__float_as_uint(a1) << 32) | __float_as_uint(a0);
    const unsigned long long B = ((unsigned long long)__float_as_uint(b1) << 32) | __float_as_uint(b0);
    const unsigned long long C = ((unsigned long long)__float_as_uint(d1) << 32) | __float_as_uint(d0);
    unsigned long long D;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(C));
    d0 = __uint_as_float((unsigned)(D & 0xffffffffu));
    d1 = __uint_as_float((unsigned)(D >> 32));
}

// block[c * R + r] += a[r] * b[c] for an R x C register block, packed in
// pairs along r when R is even
template <int R, int C>
__device__ __forceinline__ void rank1_update(float* blk, const float (&a)[R], const float (&b)[C]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if constexpr (R % 2 == 0) {
#pragma unroll
            for (int r = 0; r < R; r += 2)
                ffma2(blk[c * R + r], blk[c * R + r + 1], a[r], a[r + 1], b[c], b[c]);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) blk[c * R + r] = fmaf(a[r], b[c], blk[c * R + r]);
        }
    }
}

// R floats (R even) from an 8-byte-aligned address
template <int R>
__device__ __forceinline__ void vload2(float (&v)[R], const float* p) {
    static_assert(R % 2 == 0, "pairs");
#pragma unroll
    for (int k = 0; k < R; k += 2) {
        const float2 t = *reinterpret_cast<const float2*>(p + k);
        v[k] = t.x;
        v[k + 1] = t.y;
    }
}

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------- mbarrier / TMA
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// arrive (this thread) and expect `bytes` of asynchronous transactions
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy completing on `bar`
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// bounded wait for phase `parity` of `bar` (SM clock); false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    while (clock64() - t0 < kWaitCycles) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------------ layout
template <class Sh>
struct FastLayout {
    // floats; every region starts 16-byte aligned
    static constexpr int d1r = 0;                                   // P1 x LD1
    static constexpr int d1w = d1r + al4(Sh::P1 * Sh::LD1);         // P1 x N1 (rows of D1)
    static constexpr int d2r = d1w + al4(Sh::P1 * Sh::N1);          // P2 x N2
    static constexpr int d2p = d2r + al4(Sh::P2 * Sh::N2);          // P2 x LD2
    static constexpr int g1 = d2p + al4(Sh::P2 * Sh::LD2);          // N1 x LD1
    static constexpr int g2 = g1 + al4(Sh::N1 * Sh::LD1);           // N2 x LD2
    static constexpr int acc = g2 + al4(Sh::N2 * Sh::LD2);
    __host__ __device__ static constexpr int nf(int side) {
        return side == kSideD1 ? Sh::N1 * Sh::N1 + Sh::P1 * Sh::N1
               : side == kSideD2 ? Sh::N2 * Sh::N2 + Sh::P2 * Sh::N2 : 0;
    }
    // warp-private accumulators: WPC x nf floats (summed in warp order at the end)
    __host__ __device__ static constexpr int accw(int side) { return al4(nf(side)) * Sh::WPC; }
    // per-warp energy sums: WPC x 2 floats
    __host__ __device__ static constexpr int acce(int side) { return acc + accw(side); }
    __host__ __device__ static constexpr int warp0(int side) { return acce(side) + al4(2 * Sh::WPC); }
    // per warp: mbarriers (4 floats), Y double buffer, Z or W, the C0 blocks
    // of the 32 lanes (lane-major, stride EP: conflict-free 128-bit loads)
    static constexpr int EP = Sh::EP;
    static constexpr int w_bar = 0;
    static constexpr int w_y = 4;
    static constexpr int TZ = Sh::P1 * Sh::LD2, TW = Sh::P2 * Sh::LD1;
    static constexpr int w_z = w_y + 2 * al4(Sh::PP);
    static constexpr int w_c0 = w_z + al4(TZ > TW ? TZ : TW);
    // with s >= 8 the Cholesky state (rows of L, 1/L_tt, y) sits in shared
    // memory rather than in every lane's registers
    static constexpr bool kSmemChol = Sh::S >= 8;
    static constexpr int w_chol = w_c0 + 32 * EP;
    static constexpr int n_chol = kSmemChol ? al4(Sh::S * (Sh::S + 1) / 2) + 2 * al4(Sh::S) : 0;
    static constexpr int w_stride = w_chol + n_chol;
    __host__ __device__ static constexpr int total(int side, int wpc) { return warp0(side) + wpc * w_stride; }
};

// Body of the coding pass for one CTA: `cta` of `n_ctas` CTAs working on the
// signals of problem `a` (grid-stride over warps), partial sums to `slot`.
template <class Sh, int SIDE>
__device__ __forceinline__ void code_fast_body(const PassArgs& a, int cta, int n_ctas, int slot) {
    using L = FastLayout<Sh>;
    constexpr int P1 = Sh::P1, P2 = Sh::P2, N1 = Sh::N1, N2 = Sh::N2, S = Sh::S;
    constexpr int RI = Sh::RI, RJ = Sh::RJ, E = Sh::E, LI = Sh::LI;
    constexpr int LD1 = Sh::LD1, LD2 = Sh::LD2, RIP = Sh::RIP, RJP = Sh::RJP;
    constexpr int PP = Sh::PP;
    constexpr unsigned kBytes = PP * 4;
    extern __shared__ __align__(16) float smem[];

    // the shape's warps code signals; a CTA of the multi-problem kernel may
    // have more (warps w >= WPC only join the CTA-wide set-up and combine)
    constexpr int wpc = Sh::WPC;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool wact = w < wpc;
    const int li = lane % LI, lj = lane / LI;
    constexpr bool kW = (SIDE == kSideD2);   // C0 = (D1^T Y) D2 rather than D1^T (Y D2)
    float* D1r = smem + L::d1r;
    float* D1w = smem + L::d1w;
    float* D2r = smem + L::d2r;
    float* D2p = smem + L::d2p;
    float* G1s = smem + L::g1;
    float* G2s = smem + L::g2;
    float* acc = smem + L::acc;
    float* acce = smem + L::acce(SIDE);
    float* wb = smem + L::warp0(SIDE) + w * L::w_stride;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(wb + L::w_bar);
    float* Ybuf = wb + L::w_y;
    float* Zs = wb + L::w_z;
    float* C0s = wb + L::w_c0;
    float* myc0 = C0s + lane * L::EP;
    constexpr int nf = L::nf(SIDE);
    constexpr int nfa = al4(nf);
    float* wacc = acc + w * nfa;     // this warp's private accumulators

    // ---- CTA set-up: padded copies of D1, D2, G1, G2; zero accumulators
    for (int e = threadIdx.x; e < P1 * LD1; e += blockDim.x) {
        const int r = e / LD1, pp = e % LD1;
        const int blk = pp / RIP, off = pp % RIP;
        D1r[e] = (off < RI) ? a.D1[r + P1 * (blk * RI + off)] : 0.f;
    }
    for (int e = threadIdx.x; e < P1 * N1; e += blockDim.x) {
        const int r = e / N1, i = e % N1;
        D1w[e] = a.D1[r + P1 * i];
    }
    for (int e = threadIdx.x; e < P2 * N2; e += blockDim.x) {
        const int r = e / N2, j = e % N2;
        D2r[e] = a.D2[r + P2 * j];
    }
    for (int e = threadIdx.x; e < P2 * LD2; e += blockDim.x) {
        const int r = e / LD2, pp = e % LD2;
        const int blk = pp / RJP, off = pp % RJP;
        D2p[e] = (off < RJ) ? a.D2[r + P2 * (blk * RJ + off)] : 0.f;
    }
    for (int e = threadIdx.x; e < N1 * LD1; e += blockDim.x) {
        const int c = e / LD1, pp = e % LD1;
        const int blk = pp / RIP, off = pp % RIP;
        G1s[e] = (off < RI) ? a.G1[c * N1 + blk * RI + off] : 0.f;
    }
    for (int e = threadIdx.x; e < N2 * LD2; e += blockDim.x) {
        const int c = e / LD2, pp = e % LD2;
        const int blk = pp / RJP, off = pp % RJP;
        G2s[e] = (off < RJ) ? a.G2[c * N2 + blk * RJ + off] : 0.f;
    }
    if constexpr (SIDE != kCodeOnly) {
        for (int e = threadIdx.x; e < L::accw(SIDE) + al4(2 * Sh::WPC); e += blockDim.x) acc[e] = 0.f;
    }
    for (int e = threadIdx.x; e < wpc * L::w_stride; e += blockDim.x)
        smem[L::warp0(SIDE) + e] = 0.f;   // Z padding columns stay 0
    __syncthreads();

    const long long stride = (long long)n_ctas * wpc;
    // positions j index either the signals themselves or a list of signals
    const long long count = a.idx ? (long long)*a.idx_count : a.N;
    long long j = wact ? (long long)cta * wpc + w : count;
    long long k = (a.idx && j < count) ? (long long)a.idx[j] : j;
    if (wact && lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (lane == 0 && j < count) {
        mbar_arrive_tx(&bar[0], kBytes);
        tma_load_1d(Ybuf, a.Y + (size_t)k * PP, kBytes, &bar[0]);
    }
    unsigned phase0 = 0, phase1 = 0;
    // per-warp residual-energy and ||Y||^2 sums: compensated FP32 (the FP64
    // pipe is slow on this part), widened to FP64 once per warp
    float w_energy = 0.f, w_energy_c = 0.f, w_ynorm = 0.f, w_ynorm_c = 0.f;
    bool alive = true;
    int pending = 0;

    for (int it = 0; j < count && alive; ++it, j += stride) {
        k = a.idx ? (long long)a.idx[j] : j;
        const int buf = it & 1;
        float* Ys = Ybuf + buf * al4(PP);
        const bool got = mbar_wait(&bar[buf], buf ? phase1 : phase0);
        if (!__all_sync(kFull, got)) {
            if (lane == 0) record_error(a.err, SDL_ERR_TIMEOUT);
            alive = false;
            pending = buf;
            break;
        }
        if (buf) phase1 ^= 1u; else phase0 ^= 1u;
        // prefetch this warp's next signal into the other buffer
        const long long jn = j + stride;
        if (lane == 0 && jn < count) {
            const long long kn = a.idx ? (long long)a.idx[jn] : jn;
            fence_proxy_async();
            mbar_arrive_tx(&bar[buf ^ 1], kBytes);
            tma_load_1d(Ybuf + (buf ^ 1) * al4(PP), a.Y + (size_t)kn * PP, kBytes, &bar[buf ^ 1]);
        }

        // ---- ||Y||^2
        float ss = 0.f;
#pragma unroll
        for (int e = lane; e < PP; e += 32) ss = fmaf(Ys[e], Ys[e], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
        const bool finite = isfinite(ss);
        if (finite && a.eps2 > 0.f && ss <= a.eps2) {
            // already within the error target: an empty code, no correlations
            const long long ko = (a.idx && a.idx_compact) ? j : k;
            if (a.support && lane < S) {
                a.support[(size_t)ko * S + lane] = -1;
                a.coef[(size_t)ko * S + lane] = 0.f;
            }
            if (lane == 0) {
                if (a.nnz) a.nnz[ko] = 0;
                if (a.res_energy) a.res_energy[ko] = ss;
                const float ye = ss - w_energy_c;
                const float te = w_energy + ye;
                w_energy_c = (te - w_energy) - ye;
                w_energy = te;
                const float yy = ss - w_ynorm_c;
                const float ty = w_ynorm + yy;
                w_ynorm_c = (ty - w_ynorm) - yy;
                w_ynorm = ty;
            }
            __syncwarp();
            continue;
        }

        int cnt = 0;
        float E2 = ss;
        int myi = 0, myj = 0;
        float myx = 0.f;
        if (finite) {
            // ---- Z = Y D2 (ZA x ZB block per lane) or W = D1^T Y (WI x WB block per lane)
            if constexpr (kW) {
                if (lane < Sh::WLI * Sh::WLB) {
                    const int wi = lane % Sh::WLI, wb = lane / Sh::WLI;
                    const int i0 = wi * Sh::WI, b0 = wb * Sh::WB;
                    float wv[Sh::WI * Sh::WB];
#pragma unroll
                    for (int e = 0; e < Sh::WI * Sh::WB; ++e) wv[e] = 0.f;
#pragma unroll
                    for (int aa = 0; aa < P1; ++aa) {
                        float dv[Sh::WI], yw[Sh::WB];
#pragma unroll
                        for (int r = 0; r < Sh::WI; ++r) dv[r] = D1w[aa * N1 + i0 + r];
#pragma unroll
                        for (int c = 0; c < Sh::WB; ++c) yw[c] = Ys[(b0 + c) * P1 + aa];
                        rank1_update<Sh::WI, Sh::WB>(wv, dv, yw);
                    }
#pragma unroll
                    for (int c = 0; c < Sh::WB; ++c)
#pragma unroll
                        for (int r = 0; r < Sh::WI; ++r) Zs[(b0 + c) * LD1 + pos1<Sh>(i0 + r)] = wv[c * Sh::WI + r];
                }
            } else if (lane < Sh::ZLA * Sh::ZLB) {
                const int za = lane % Sh::ZLA, zb = lane / Sh::ZLA;
                const int a0 = za * Sh::ZA, j0 = zb * Sh::ZB;
                float z[Sh::ZA][Sh::ZB];
#pragma unroll
                for (int r = 0; r < Sh::ZA; ++r)
#pragma unroll
                    for (int c = 0; c < Sh::ZB; ++c) z[r][c] = 0.f;
#pragma unroll
                for (int b = 0; b < P2; ++b) {
                    float yv[Sh::ZA], dv[Sh::ZB];
#pragma unroll
                    for (int r = 0; r < Sh::ZA; ++r) yv[r] = Ys[b * P1 + a0 + r];
#pragma unroll
                    for (int c = 0; c < Sh::ZB; ++c) dv[c] = D2r[b * N2 + j0 + c];
#pragma unroll
                    for (int r = 0; r < Sh::ZA; ++r)
#pragma unroll
                        for (int c = 0; c < Sh::ZB; ++c) z[r][c] = fmaf(yv[r], dv[c], z[r][c]);
                }
#pragma unroll
                for (int r = 0; r < Sh::ZA; ++r)
#pragma unroll
                    for (int c = 0; c < Sh::ZB; ++c) Zs[(a0 + r) * LD2 + pos2<Sh>(j0 + c)] = z[r][c];
            }
            __syncwarp();
            // ---- C0 = D1^T Z or W D2 on the lane's RI x RJ block (flat index e = c*RI + r)
            float c0[E];
#pragma unroll
            for (int e = 0; e < E; ++e) c0[e] = 0.f;
            if constexpr (!kW) {
#pragma unroll
                for (int aa = 0; aa < P1; ++aa) {
                    float u[RI], v[RJ];
                    vload<RI>(u, D1r + aa * LD1 + li * RIP);
                    vload<RJ>(v, Zs + aa * LD2 + lj * RJP);
                    rank1_update<RI, RJ>(c0, u, v);
                }
            } else {
#pragma unroll
                for (int bb = 0; bb < P2; ++bb) {
                    float u[RI], v[RJ];
                    vload<RI>(u, Zs + bb * LD1 + li * RIP);
                    vload<RJ>(v, D2p + bb * LD2 + lj * RJP);
                    rank1_update<RI, RJ>(c0, u, v);
                }
            }

            // keep C0 in shared memory: re-read once per step, masked by one store
#pragma unroll
            for (int e = 0; e < E; e += 4) {
                if (e + 4 <= E) {
                    *reinterpret_cast<float4*>(myc0 + e) = make_float4(c0[e], c0[e + 1], c0[e + 2], c0[e + 3]);
                } else {
#pragma unroll
                    for (int k2 = e; k2 < E; ++k2) myc0[k2] = c0[k2];
                }
            }
            __syncwarp();

            // ---- greedy steps, fully unrolled.  Every lane computes the whole
            // Cholesky update (packed rows of L and 1/L_tt), so both triangular
            // solves run without shuffles; the factor stays in registers, or
            // (s >= 8) in shared memory, written by lane 0, so that it holds no
            // registers while the scores are live.
            constexpr bool kSC = L::kSmemChol;
            constexpr int kR = kSC ? 1 : S, kRL = kSC ? 1 : S * (S + 1) / 2;
            float* Lsm = wb + L::w_chol;
            float* ivsm = Lsm + al4(S * (S + 1) / 2);
            float* yvsm = ivsm + al4(S);
            int si[S], sj[S];
            float xs[S], yv[kR], Lf[kRL], invd[kR];
#pragma unroll
            for (int m = 0; m < S; ++m) {
                si[m] = 0; sj[m] = 0; xs[m] = 0.f;
            }
#pragma unroll
            for (int m = 0; m < kR; ++m) {
                yv[m] = 0.f; invd[m] = 0.f;
            }
#pragma unroll
            for (int m = 0; m < kRL; ++m) Lf[m] = 0.f;
            bool go = true;
            const int qbase = li * RI + N1 * (lj * RJ);
            static_for<0, S>([&](auto tc) {
                constexpr int t = decltype(tc)::value;
                if (!go) return;
                if (a.eps2 > 0.f && E2 <= a.eps2) { go = false; return; }
                float sc[E];
                if constexpr (t == 0) {
#pragma unroll
                    for (int e = 0; e < E; ++e) sc[e] = c0[e];
                } else {
                    vload<E>(sc, myc0);
                }
#pragma unroll
                for (int l = 0; l < t; ++l) {
                    float u[RI], v[RJ];
                    vload<RI>(u, G1s + si[l] * LD1 + li * RIP);
                    vload<RJ>(v, G2s + sj[l] * LD2 + lj * RJP);
                    const float nx = -xs[l];
#pragma unroll
                    for (int c = 0; c < RJ; ++c) v[c] *= nx;
                    rank1_update<RI, RJ>(sc, u, v);
                }
                // argmax |sc|, ties to the smallest q: two interleaved chains
                // (even and odd entries in increasing q), merged by (value, q)
                float best = 0.f, best1 = 0.f;
                int bq = 0x7fffffff, bq1 = 0x7fffffff;
#pragma unroll
                for (int c = 0; c < RJ; ++c)
#pragma unroll
                    for (int r = 0; r < RI; ++r) {
                        const float v = fabsf(sc[c * RI + r]);
                        if ((c * RI + r) & 1) {
                            if (v > best1) { best1 = v; bq1 = qbase + r + N1 * c; }
                        } else {
                            if (v > best) { best = v; bq = qbase + r + N1 * c; }
                        }
                    }
                if (best1 > best || (best1 == best && bq1 < bq)) { best = best1; bq = bq1; }
                const unsigned M = __reduce_max_sync(kFull, __float_as_uint(best));
                if (M == 0u) { go = false; return; }
                const unsigned cand = (__float_as_uint(best) == M) ? (unsigned)bq : 0xffffffffu;
                const int q = (int)__reduce_min_sync(kFull, cand);
                const int it_ = q % N1, jt = q / N1;
                const int owner = it_ / RI + LI * (jt / RJ);
                float* cq = C0s + owner * L::EP + (jt % RJ) * RI + it_ % RI;
                const float b = *cq;
                __syncwarp();
                if (lane == 0) *cq = __int_as_float(0x7fc00000);   // mask the pick
                // ---- Cholesky row t:  w = L^{-1} a,  L_tt = sqrt(A_tt - w.w),
                // a_m = G1[i_t, i_m] G2[j_t, j_m] (the same value in every lane)
                const float* g1t = G1s + it_ * LD1;
                const float* g2t = G2s + jt * LD2;
                const float Att = g1t[pos1<Sh>(it_)] * g2t[pos2<Sh>(jt)];
                float ww = 0.f, wy = 0.f;
                float yt;
                if constexpr (kSC) {
                    // the state of steps 0..t-1 from shared memory; the same
                    // recurrences and FMA order as the register form below
                    constexpr int kOld = t * (t + 1) / 2;
                    float Lo[kOld > 0 ? kOld : 1], io[t > 0 ? t : 1], yo[t > 0 ? t : 1];
#pragma unroll
                    for (int m = 0; m < kOld; ++m) Lo[m] = Lsm[m];
#pragma unroll
                    for (int m = 0; m < t; ++m) {
                        io[m] = ivsm[m];
                        yo[m] = yvsm[m];
                    }
                    float wr[t > 0 ? t : 1];   // row t of L
#pragma unroll
                    for (int m = 0; m < t; ++m) {
                        float am = g1t[pos1<Sh>(si[m])] * g2t[pos2<Sh>(sj[m])];
#pragma unroll
                        for (int l = 0; l < m; ++l) am = fmaf(-Lo[m * (m + 1) / 2 + l], wr[l], am);
                        wr[m] = am * io[m];
                        ww = fmaf(wr[m], wr[m], ww);
                        wy = fmaf(wr[m], yo[m], wy);
                    }
                    const float d = Att - ww;
                    if (!(d > kPivotRel * Att)) { go = false; return; }
                    const float inv = rsqrtf(d);
                    yt = (b - wy) * inv;
                    si[t] = it_;
                    sj[t] = jt;
                    if (lane == t) {
                        myi = it_;
                        myj = jt;
                    }
                    // ---- x = L^{-T} y (rows t..0)
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
                    if (lane == 0) {
#pragma unroll
                        for (int m = 0; m < t; ++m) Lsm[kOld + m] = wr[m];
                        ivsm[t] = inv;
                        yvsm[t] = yt;
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < t; ++m) {
                        float am = g1t[pos1<Sh>(si[m])] * g2t[pos2<Sh>(sj[m])];
#pragma unroll
                        for (int l = 0; l < m; ++l) am = fmaf(-Lf[m * (m + 1) / 2 + l], Lf[t * (t + 1) / 2 + l], am);
                        const float wm = am * invd[m];
                        Lf[t * (t + 1) / 2 + m] = wm;
                        ww = fmaf(wm, wm, ww);
                        wy = fmaf(wm, yv[m], wy);
                    }
                    const float d = Att - ww;
                    if (!(d > kPivotRel * Att)) { go = false; return; }
                    const float inv = rsqrtf(d);
                    yt = (b - wy) * inv;
                    yv[t] = yt;
                    si[t] = it_;
                    sj[t] = jt;
                    invd[t] = inv;
                    if (lane == t) {
                        myi = it_;
                        myj = jt;
                    }
                    // ---- x = L^{-T} y (rows t..0)
#pragma unroll
                    for (int kk = t; kk >= 0; --kk) {
                        float v = yv[kk];
#pragma unroll
                        for (int l = kk + 1; l <= t; ++l) v = fmaf(-Lf[l * (l + 1) / 2 + kk], xs[l], v);
                        xs[kk] = v * invd[kk];
                    }
                }
                E2 = fmaf(-yt, yt, E2);
                cnt = t + 1;
                __syncwarp();   // the masked C0 entry is visible to the next step
            });
#pragma unroll
            for (int m = 0; m < S; ++m)
                if (lane == m) myx = xs[m];
        }

        // ---- emit the code (lane l holds pick l)
        const long long ko = (a.idx && a.idx_compact) ? j : k;
        if (a.support && lane < S) {
            a.support[(size_t)ko * S + lane] = (lane < cnt) ? myi + N1 * myj : -1;
            a.coef[(size_t)ko * S + lane] = (lane < cnt) ? myx : 0.f;
        }
        if (lane == 0) {
            if (a.nnz) a.nnz[ko] = cnt;
            if (a.res_energy) a.res_energy[ko] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
            if (!finite) record_error(a.err, SDL_ERR_NONFINITE);
        }

        // ---- fused partial sums into this warp's private accumulators (no
        // other warp touches them, and the warps are combined in a fixed
        // order at the end); terms are spread over the lanes as (pick, row)
        // and (pick, pick) pairs
        if constexpr (SIDE == kSideD1) {
            float* wP = wacc;
            float* wB = wacc + N1 * N1;
#pragma unroll
            for (int e0 = 0; e0 < P1 * S; e0 += 32) {
                const int e = e0 + lane;
                const int l = e / P1, r = e % P1;
                const int il = __shfl_sync(kFull, myi, l & 31), jl = __shfl_sync(kFull, myj, l & 31);
                const float xl = __shfl_sync(kFull, myx, l & 31);
                if (l < cnt) atomicAdd(&wB[r * N1 + il], xl * Zs[r * LD2 + pos2<Sh>(jl)]);
            }
#pragma unroll
            for (int e0 = 0; e0 < S * S; e0 += 32) {
                const int e = e0 + lane;
                const int l = e / S, m = e % S;
                const int il = __shfl_sync(kFull, myi, l & 31), im = __shfl_sync(kFull, myi, m);
                const int jl = __shfl_sync(kFull, myj, l & 31), jm = __shfl_sync(kFull, myj, m);
                const float xl = __shfl_sync(kFull, myx, l & 31), xm = __shfl_sync(kFull, myx, m);
                if (l < cnt && m < cnt)
                    atomicAdd(&wP[il * N1 + im], xl * xm * G2s[jl * LD2 + pos2<Sh>(jm)]);
            }
        } else if constexpr (SIDE == kSideD2) {
            float* wM = wacc;
            float* wB = wacc + N2 * N2;
            // B2[b, j_l] += x_l W[i_l, b]
#pragma unroll
            for (int e0 = 0; e0 < P2 * S; e0 += 32) {
                const int e = e0 + lane;
                const int l = e / P2, bb = e % P2;
                const int il = __shfl_sync(kFull, myi, l & 31), jl = __shfl_sync(kFull, myj, l & 31);
                const float xl = __shfl_sync(kFull, myx, l & 31);
                if (l < cnt) atomicAdd(&wB[bb * N2 + jl], xl * Zs[bb * LD1 + pos1<Sh>(il)]);
            }
#pragma unroll
            for (int e0 = 0; e0 < S * S; e0 += 32) {
                const int e = e0 + lane;
                const int l = e / S, m = e % S;
                const int il = __shfl_sync(kFull, myi, l & 31), im = __shfl_sync(kFull, myi, m);
                const int jl = __shfl_sync(kFull, myj, l & 31), jm = __shfl_sync(kFull, myj, m);
                const float xl = __shfl_sync(kFull, myx, l & 31), xm = __shfl_sync(kFull, myx, m);
                if (l < cnt && m < cnt)
                    atomicAdd(&wM[jl * N2 + jm], xl * xm * G1s[il * LD1 + pos1<Sh>(im)]);
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
        __syncwarp();
    }
    if (!alive && lane == 0) {
        // give the copy that timed out a last bounded chance to land before the
        // CTA's shared memory is released
        mbar_wait(&bar[pending], pending ? phase1 : phase0);
    }

    if constexpr (SIDE != kCodeOnly) {
        if (wact && lane == 0) {
            acce[2 * w] = w_energy - w_energy_c;
            acce[2 * w + 1] = w_ynorm - w_ynorm_c;
        }
        __syncthreads();
        // combine the warps' accumulators in warp order
        float* dst = a.part_f + (size_t)slot * nf;
        for (int e = threadIdx.x; e < nf; e += blockDim.x) {
            float v = 0.f;
            for (int ww = 0; ww < wpc; ++ww) v += acc[ww * nfa + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int ww = 0; ww < wpc; ++ww) d += (double)acce[2 * ww + threadIdx.x];
            a.part_d[(size_t)slot * 2 + threadIdx.x] = d;
        }
    }
}

// ------------------------------------------------------------ two signals per warp
template <class Sh>
struct HalfLayout {
    static constexpr int P1 = Sh::P1, P2 = Sh::P2, N1 = Sh::N1, N2 = Sh::N2;
    // floats; every region starts 16-byte aligned
    static constexpr int d1r = 0;                                  // P1 x LD1: rows of D1, lane blocks
    static constexpr int d1w = d1r + al4(P1 * Sh::LD1);            // P1 x N1: rows of D1
    static constexpr int d2r = d1w + al4(P1 * N1);                 // P2 x N2: rows of D2
    static constexpr int d2p = d2r + al4(P2 * N2);                 // P2 x LD2: rows of D2, lane blocks
    static constexpr int g1 = d2p + al4(P2 * Sh::LD2);             // N1 x LD1
    static constexpr int g2 = g1 + al4(N1 * Sh::LD1);              // N2 x LD2
    static constexpr int acc = g2 + al4(N2 * Sh::LD2);
    __host__ __device__ static constexpr int nf(int side) {
        return side == kSideD1 ? N1 * N1 + P1 * N1 : side == kSideD2 ? N2 * N2 + P2 * N2 : 0;
    }
    // warp-private accumulators (both halves of a warp add into them)
    __host__ __device__ static constexpr int accw(int side) { return al4(nf(side)) * Sh::WPC; }
    // per-half energy sums: 2 WPC x 2 floats
    __host__ __device__ static constexpr int acce(int side) { return acc + accw(side); }
    __host__ __device__ static constexpr int half0(int side) { return acce(side) + al4(4 * Sh::WPC); }
    // per half: mbarrier, Y (one buffer: the next signal is fetched into it as
    // soon as the first contraction has read it), Z or W, the C0 blocks of the
    // 16 lanes (lane-major, stride EP)
    static constexpr int TZ = P1 * Sh::LD2, TW = P2 * Sh::LD1;
    static constexpr int h_bar = 0;
    static constexpr int h_y = 4;
    static constexpr int h_t = h_y + al4(Sh::PP);
    static constexpr int h_c0 = h_t + al4(TZ > TW ? TZ : TW);
    // Cholesky state: packed rows of L, 1/L_tt, y
    static constexpr int h_chol = h_c0 + 16 * Sh::EP;
    static constexpr int h_stride = h_chol + al4(Sh::S * (Sh::S + 1) / 2) + 2 * al4(Sh::S);
    __host__ __device__ static constexpr int total(int side, int wpc) {
        return half0(side) + 2 * wpc * h_stride;
    }
};

template <class Sh, int SIDE>
__device__ __forceinline__ void code_half_body(const PassArgs& a, int cta, int n_ctas, int slot) {
    using L = HalfLayout<Sh>;
    constexpr int P1 = Sh::P1, P2 = Sh::P2, N1 = Sh::N1, N2 = Sh::N2, S = Sh::S;
    constexpr int RI = Sh::RI, RJ = Sh::RJ, E = Sh::E, LI = Sh::LI;
    constexpr int LD1 = Sh::LD1, LD2 = Sh::LD2, RIP = Sh::RIP, RJP = Sh::RJP;
    constexpr int PP = Sh::PP;
    constexpr unsigned kBytes = PP * 4;
    constexpr bool kW = (SIDE == kSideD2);   // C0 = (D1^T Y) D2 rather than D1^T (Y D2)
    extern __shared__ __align__(16) float smem[];

    const int wpc = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = lane >> 4, hl = lane & 15;
    const unsigned hm = 0xffffu << (16 * h);
    const int li = hl % LI, lj = hl / LI;
    float* D1r = smem + L::d1r;
    float* D1w = smem + L::d1w;
    float* D2r = smem + L::d2r;
    float* D2p = smem + L::d2p;
    float* G1s = smem + L::g1;
    float* G2s = smem + L::g2;
    float* acc = smem + L::acc;
    float* acce = smem + L::acce(SIDE);
    float* hb = smem + L::half0(SIDE) + (2 * w + h) * L::h_stride;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(hb + L::h_bar);
    float* Ys = hb + L::h_y;
    float* Ts = hb + L::h_t;    // Z (rows a, lane-block columns j) or W (rows b, lane-block columns i)
    float* C0s = hb + L::h_c0;
    float* myc0 = C0s + hl * Sh::EP;
    float* Lsm = hb + L::h_chol;
    float* ivsm = Lsm + al4(S * (S + 1) / 2);
    float* yvsm = ivsm + al4(S);
    constexpr int nf = L::nf(SIDE);
    constexpr int nfa = al4(nf);
    float* wacc = acc + w * nfa;

    // ---- CTA set-up
    for (int e = threadIdx.x; e < P1 * LD1; e += blockDim.x) {
        const int r = e / LD1, pp = e % LD1;
        const int blk = pp / RIP, off = pp % RIP;
        D1r[e] = (off < RI) ? a.D1[r + P1 * (blk * RI + off)] : 0.f;
    }
    for (int e = threadIdx.x; e < P1 * N1; e += blockDim.x) {
        const int r = e / N1, i = e % N1;
        D1w[e] = a.D1[r + P1 * i];
    }
    for (int e = threadIdx.x; e < P2 * N2; e += blockDim.x) {
        const int r = e / N2, j = e % N2;
        D2r[e] = a.D2[r + P2 * j];
    }
    for (int e = threadIdx.x; e < P2 * LD2; e += blockDim.x) {
        const int r = e / LD2, pp = e % LD2;
        const int blk = pp / RJP, off = pp % RJP;
        D2p[e] = (off < RJ) ? a.D2[r + P2 * (blk * RJ + off)] : 0.f;
    }
    for (int e = threadIdx.x; e < N1 * LD1; e += blockDim.x) {
        const int c = e / LD1, pp = e % LD1;
        const int blk = pp / RIP, off = pp % RIP;
        G1s[e] = (off < RI) ? a.G1[c * N1 + blk * RI + off] : 0.f;
    }
    for (int e = threadIdx.x; e < N2 * LD2; e += blockDim.x) {
        const int c = e / LD2, pp = e % LD2;
        const int blk = pp / RJP, off = pp % RJP;
        G2s[e] = (off < RJ) ? a.G2[c * N2 + blk * RJ + off] : 0.f;
    }
    if constexpr (SIDE != kCodeOnly) {
        for (int e = threadIdx.x; e < L::accw(SIDE) + al4(4 * Sh::WPC); e += blockDim.x) acc[e] = 0.f;
    }
    for (int e = threadIdx.x; e < 2 * wpc * L::h_stride; e += blockDim.x) smem[L::half0(SIDE) + e] = 0.f;
    __syncthreads();

    // Positions: this warp takes pairs (jb, jb + 1), jb = first, first + stride,
    // ...; half h codes position jb + h.  The trip count is the same for both
    // halves (half 1 idles when only jb is left), so the warp meets at every
    // full-warp synchronisation point.
    const long long stride = (long long)n_ctas * wpc * 2;
    const long long count = a.idx ? (long long)*a.idx_count : a.N;
    const long long first = ((long long)cta * wpc + w) * 2;
    if (hl == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    bool inflight = first + h < count;   // a copy into Ys is outstanding
    if (hl == 0 && inflight) {
        const long long k0 = a.idx ? (long long)a.idx[first + h] : first + h;
        mbar_arrive_tx(bar, kBytes);
        tma_load_1d(Ys, a.Y + (size_t)k0 * PP, kBytes, bar);
    }
    unsigned phase = 0;
    float w_energy = 0.f, w_energy_c = 0.f, w_ynorm = 0.f, w_ynorm_c = 0.f;
    bool alive = true;

    for (long long jb = first; jb < count && alive; jb += stride) {
        const long long jj = jb + h;
        const bool act = jj < count;
        const long long k = act ? (a.idx ? (long long)a.idx[jj] : jj) : 0;
        bool got = true;
        if (act) got = mbar_wait(bar, phase);
        if (!__all_sync(kFull, got)) {
            if (lane == 0) record_error(a.err, SDL_ERR_TIMEOUT);
            alive = false;
            break;
        }
        if (act) {
            phase ^= 1u;
            inflight = false;
        }

        // ---- ||Y||^2, with the partial sums and the combining order of a full warp
        float ss = 0.f;
        if (act) {
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int e = hl; e < PP; e += 32) lo = fmaf(Ys[e], Ys[e], lo);
#pragma unroll
            for (int e = hl + 16; e < PP; e += 32) hi = fmaf(Ys[e], Ys[e], hi);
            ss = lo + hi;
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
        const bool finite = act && isfinite(ss);
        // a signal already within the error target takes no atom: skip its correlations
        const bool work = finite && !(a.eps2 > 0.f && ss <= a.eps2);

        // ---- first contraction: Z = Y D2 or W = D1^T Y (packed FMAs along row pairs)
        if (work) {
            if constexpr (!kW) {
                const int za = hl % Sh::ZLA, zb = hl / Sh::ZLA;
                const int a0 = za * Sh::ZA, jz = zb * Sh::ZB;
                float z[Sh::ZA * Sh::ZB];
#pragma unroll
                for (int e = 0; e < Sh::ZA * Sh::ZB; ++e) z[e] = 0.f;
#pragma unroll
                for (int b = 0; b < P2; ++b) {
                    float yv[Sh::ZA], dv[Sh::ZB];
                    vload2<Sh::ZA>(yv, Ys + b * P1 + a0);
#pragma unroll
                    for (int c = 0; c < Sh::ZB; ++c) dv[c] = D2r[b * N2 + jz + c];
                    rank1_update<Sh::ZA, Sh::ZB>(z, yv, dv);
                }
#pragma unroll
                for (int c = 0; c < Sh::ZB; ++c)
#pragma unroll
                    for (int r = 0; r < Sh::ZA; ++r) Ts[(a0 + r) * LD2 + pos2<Sh>(jz + c)] = z[c * Sh::ZA + r];
            } else {
                const int wi = hl % Sh::WLI, wb = hl / Sh::WLI;
                const int i0 = wi * Sh::WI, b0 = wb * Sh::WB;
                float wv[Sh::WI * Sh::WB];
#pragma unroll
                for (int e = 0; e < Sh::WI * Sh::WB; ++e) wv[e] = 0.f;
#pragma unroll
                for (int aa = 0; aa < P1; ++aa) {
                    float dv[Sh::WI], yv[Sh::WB];
                    vload2<Sh::WI>(dv, D1w + aa * N1 + i0);
#pragma unroll
                    for (int c = 0; c < Sh::WB; ++c) yv[c] = Ys[(b0 + c) * P1 + aa];
                    rank1_update<Sh::WI, Sh::WB>(wv, dv, yv);
                }
#pragma unroll
                for (int c = 0; c < Sh::WB; ++c)
#pragma unroll
                    for (int r = 0; r < Sh::WI; ++r) Ts[(b0 + c) * LD1 + pos1<Sh>(i0 + r)] = wv[c * Sh::WI + r];
            }
        }
        __syncwarp(hm);   // Y is consumed: fetch this half's next signal into it
        {
            const long long jn = jj + stride;
            if (act && jn < count) {
                inflight = true;
                if (hl == 0) {
                    const long long kn = a.idx ? (long long)a.idx[jn] : jn;
                    fence_proxy_async();
                    mbar_arrive_tx(bar, kBytes);
                    tma_load_1d(Ys, a.Y + (size_t)kn * PP, kBytes, bar);
                }
            }
        }

        int cnt = 0;
        float E2 = ss;
        int myi = 0, myj = 0;
        float myx = 0.f;
        int si[S], sj[S];
        float xs[S];
#pragma unroll
        for (int m = 0; m < S; ++m) {
            si[m] = 0; sj[m] = 0; xs[m] = 0.f;
        }
        if (__any_sync(kFull, work)) {
            // ---- C0 on the lane's RI x RJ block (flat index e = c*RI + r)
            float c0[E];
#pragma unroll
            for (int e = 0; e < E; ++e) c0[e] = 0.f;
            if constexpr (!kW) {
#pragma unroll
                for (int aa = 0; aa < P1; ++aa) {
                    float u[RI], v[RJ];
                    vload<RI>(u, D1r + aa * LD1 + li * RIP);
                    vload<RJ>(v, Ts + aa * LD2 + lj * RJP);
                    rank1_update<RI, RJ>(c0, u, v);
                }
            } else {
#pragma unroll
                for (int bb = 0; bb < P2; ++bb) {
                    float u[RI], v[RJ];
                    vload<RI>(u, Ts + bb * LD1 + li * RIP);
                    vload<RJ>(v, D2p + bb * LD2 + lj * RJP);
                    rank1_update<RI, RJ>(c0, u, v);
                }
            }
#pragma unroll
            for (int e = 0; e < E; e += 4)
                *reinterpret_cast<float4*>(myc0 + e) = make_float4(c0[e], c0[e + 1], c0[e + 2], c0[e + 3]);
            __syncwarp(hm);

            // ---- greedy steps: every lane of a half computes the whole Cholesky
            // update of its signal (identical values), lane 0 stores it
            bool go = work;
            const int qbase = li * RI + N1 * (lj * RJ);
            static_for<0, S>([&](auto tc) {
                constexpr int t = decltype(tc)::value;
                const bool live = go && !(a.eps2 > 0.f && E2 <= a.eps2);
                if (!__any_sync(kFull, live)) {   // both halves done: skip the remaining steps
                    go = false;
                    return;
                }
                // scores in two row halves of the lane's block (RH x RJ each), so
                // that only half the block is live at once, in a loop that is not
                // unrolled (half the code, for the instruction cache); C0 comes
                // from shared memory, so no register array is indexed by the
                // half.  Each half scans two argmax chains (alternate rows, each
                // in increasing q), merged by (value, q) into the running best.
                constexpr int RH = RI / 2, EH = RH * RJ;
                float bv[1] = {0.f};
                int bqv[1] = {0x7fffffff};
#pragma unroll 1
                for (int hh = 0; hh < 2; ++hh) {
                    float sc[EH];   // sc[c*RH + r] = score of row hh*RH + r, column c
#pragma unroll
                    for (int c = 0; c < RJ; ++c)
#pragma unroll
                        for (int r = 0; r < RH; r += 2) {
                            const float2 x2 = *reinterpret_cast<const float2*>(myc0 + c * RI + hh * RH + r);
                            sc[c * RH + r] = x2.x;
                            sc[c * RH + r + 1] = x2.y;
                        }
#pragma unroll
                    for (int l = 0; l < t; ++l) {
                        float u[RH], v[RJ];
                        vload2<RH>(u, G1s + si[l] * LD1 + li * RIP + hh * RH);
                        vload<RJ>(v, G2s + sj[l] * LD2 + lj * RJP);
                        const float nx = -xs[l];
#pragma unroll
                        for (int c = 0; c < RJ; ++c) v[c] *= nx;
                        rank1_update<RH, RJ>(sc, u, v);
                    }
                    float be = 0.f, bo = 0.f;
                    int qe = 0x7fffffff, qo = 0x7fffffff;
                    const int qh = qbase + hh * RH;
#pragma unroll
                    for (int c = 0; c < RJ; ++c)
#pragma unroll
                        for (int r = 0; r < RH; ++r) {
                            const float v = fabsf(sc[c * RH + r]);
                            if (r & 1) {
                                if (v > bo) { bo = v; qo = qh + r + N1 * c; }
                            } else {
                                if (v > be) { be = v; qe = qh + r + N1 * c; }
                            }
                        }
                    if (bo > be || (bo == be && qo < qe)) {
                        be = bo;
                        qe = qo;
                    }
                    if (be > bv[0] || (be == bv[0] && qe < bqv[0])) {
                        bv[0] = be;
                        bqv[0] = qe;
                    }
                }
                // the Cholesky state of steps 0..t-1 (shared memory, so that it
                // holds no registers while the scores are live)
                constexpr int kOld = t * (t + 1) / 2;
                float Lo[kOld > 0 ? kOld : 1], io[t > 0 ? t : 1], yo[t > 0 ? t : 1];
#pragma unroll
                for (int m = 0; m < kOld; ++m) Lo[m] = Lsm[m];
#pragma unroll
                for (int m = 0; m < t; ++m) {
                    io[m] = ivsm[m];
                    yo[m] = yvsm[m];
                }
                // each half's maximum and smallest q holding it, by full-warp
                // reductions in which the other half contributes the identity
                const unsigned bb = live ? __float_as_uint(bv[0]) : 0u;
                const unsigned m0 = __reduce_max_sync(kFull, h ? 0u : bb);
                const unsigned m1 = __reduce_max_sync(kFull, h ? bb : 0u);
                const unsigned M = h ? m1 : m0;
                const bool pick = live && M != 0u;
                const unsigned cand = (pick && bb == M) ? (unsigned)bqv[0] : 0xffffffffu;
                const unsigned q0 = __reduce_min_sync(kFull, h ? 0xffffffffu : cand);
                const unsigned q1 = __reduce_min_sync(kFull, h ? cand : 0xffffffffu);
                const int q = pick ? (int)(h ? q1 : q0) : 0;
                const int it_ = q % N1, jt = q / N1;
                const int owner = it_ / RI + LI * (jt / RJ);
                float* cq = C0s + owner * Sh::EP + (jt % RJ) * RI + it_ % RI;
                const float b = *cq;
                __syncwarp();
                if (hl == 0 && pick) *cq = __int_as_float(0x7fc00000);   // mask the pick
                // ---- Cholesky row t (row t of a half that does not keep this
                // pick is never read again)
                const float* g1t = G1s + it_ * LD1;
                const float* g2t = G2s + jt * LD2;
                const float Att = g1t[pos1<Sh>(it_)] * g2t[pos2<Sh>(jt)];
                float wr[t > 0 ? t : 1];   // row t of L
                float ww = 0.f, wy = 0.f;
#pragma unroll
                for (int m = 0; m < t; ++m) {
                    float am = g1t[pos1<Sh>(si[m])] * g2t[pos2<Sh>(sj[m])];
#pragma unroll
                    for (int l = 0; l < m; ++l) am = fmaf(-Lo[m * (m + 1) / 2 + l], wr[l], am);
                    wr[m] = am * io[m];
                    ww = fmaf(wr[m], wr[m], ww);
                    wy = fmaf(wr[m], yo[m], wy);
                }
                const float d = Att - ww;
                const bool ok = pick && (d > kPivotRel * Att);
                const float inv = rsqrtf(d);
                const float yt = (b - wy) * inv;
                si[t] = it_;
                sj[t] = jt;
                if (hl == t && ok) {
                    myi = it_;
                    myj = jt;
                }
                // ---- x = L^{-T} y, kept only by a half that keeps the pick
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
                for (int kk = 0; kk <= t; ++kk) xs[kk] = ok ? xn[kk] : xs[kk];
                if (hl == 0) {
#pragma unroll
                    for (int m = 0; m < t; ++m) Lsm[kOld + m] = wr[m];
                    ivsm[t] = inv;
                    yvsm[t] = yt;
                }
                E2 = ok ? fmaf(-yt, yt, E2) : E2;
                cnt = ok ? t + 1 : cnt;
                go = ok;
                __syncwarp();   // the masked C0 entry is visible to the next step
            });
#pragma unroll
            for (int m = 0; m < S; ++m)
                if (hl == m) myx = xs[m];
        }

        // ---- emit the code (lane hl of the half holds pick hl)
        if (act) {
            const long long ko = (a.idx && a.idx_compact) ? jj : k;
            if (a.support && hl < S) {
                a.support[(size_t)ko * S + hl] = (hl < cnt) ? myi + N1 * myj : -1;
                a.coef[(size_t)ko * S + hl] = (hl < cnt) ? myx : 0.f;
            }
            if (hl == 0) {
                if (a.nnz) a.nnz[ko] = cnt;
                if (a.res_energy) a.res_energy[ko] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
                if (!finite) record_error(a.err, SDL_ERR_NONFINITE);
            }
        }

        // ---- fused partial sums into the warp's private accumulators; both
        // halves run these adds together, so their order is fixed
        __syncwarp();
        if constexpr (SIDE == kSideD1) {
            float* wP = wacc;
            float* wB = wacc + N1 * N1;
            // B1[r, i_l] += x_l Z[r, j_l]  (lane = r)
#pragma unroll
            for (int l = 0; l < S; ++l)
                if (l < cnt && hl < P1) atomicAdd(&wB[hl * N1 + si[l]], xs[l] * Ts[hl * LD2 + pos2<Sh>(sj[l])]);
            // P[i_l, i_m] += x_l x_m G2[j_l, j_m]  (lane = m)
            const int pj = pos2<Sh>(myj);
#pragma unroll
            for (int l = 0; l < S; ++l)
                if (l < cnt && hl < cnt) atomicAdd(&wP[si[l] * N1 + myi], xs[l] * myx * G2s[sj[l] * LD2 + pj]);
        } else if constexpr (SIDE == kSideD2) {
            float* wM = wacc;
            float* wB = wacc + N2 * N2;
            // B2[b, j_l] += x_l W[i_l, b]  (lane = b)
#pragma unroll
            for (int l = 0; l < S; ++l)
                if (l < cnt && hl < P2) atomicAdd(&wB[hl * N2 + sj[l]], xs[l] * Ts[hl * LD1 + pos1<Sh>(si[l])]);
            // M[j_l, j_m] += x_l x_m G1[i_l, i_m]  (lane = m)
            const int pi = pos1<Sh>(myi);
#pragma unroll
            for (int l = 0; l < S; ++l)
                if (l < cnt && hl < cnt) atomicAdd(&wM[sj[l] * N2 + myj], xs[l] * myx * G1s[si[l] * LD1 + pi]);
        }
        if (hl == 0 && finite) {
            const float ye = fmaxf(E2, 0.f) - w_energy_c;
            const float te = w_energy + ye;
            w_energy_c = (te - w_energy) - ye;
            w_energy = te;
            const float yy = ss - w_ynorm_c;
            const float ty = w_ynorm + yy;
            w_ynorm_c = (ty - w_ynorm) - yy;
            w_ynorm = ty;
        }
        __syncwarp();
    }
    if (!alive && hl == 0 && inflight) {
        // give the copy that timed out a last bounded chance to land before the
        // CTA's shared memory is released
        mbar_wait(bar, phase);
    }

    if constexpr (SIDE != kCodeOnly) {
        if (hl == 0) {
            acce[2 * (2 * w + h)] = w_energy - w_energy_c;
            acce[2 * (2 * w + h) + 1] = w_ynorm - w_ynorm_c;
        }
        __syncthreads();
        const int wpc_all = blockDim.x >> 5;
        float* dst = a.part_f + (size_t)slot * nf;
        for (int e = threadIdx.x; e < nf; e += blockDim.x) {
            float v = 0.f;
            for (int ww = 0; ww < wpc_all; ++ww) v += acc[ww * nfa + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int hh = 0; hh < 2 * wpc_all; ++hh) d += (double)acce[2 * hh + threadIdx.x];
            a.part_d[(size_t)slot * 2 + threadIdx.x] = d;
        }
    }
}

template <class Sh>
using LayoutFor = std::conditional_t<Sh::kHalf, HalfLayout<Sh>, FastLayout<Sh>>;

template <class Sh, int SIDE>
__device__ __forceinline__ void code_body(const PassArgs& a, int cta, int n_ctas, int slot) {
    if constexpr (Sh::kHalf) code_half_body<Sh, SIDE>(a, cta, n_ctas, slot);
    else code_fast_body<Sh, SIDE>(a, cta, n_ctas, slot);
}

template <class Sh, int SIDE>
__global__ void __launch_bounds__(Sh::WPC * 32, Sh::MINB) code_fast_kernel(PassArgs a) {
    code_body<Sh, SIDE>(a, blockIdx.x, gridDim.x, blockIdx.x);
}

constexpr int kMaxCtasPerSm = 8;

template <class Sh, int SIDE>
int launch_fast_impl(const PassArgs& a, cudaStream_t st, int num_sms, int ctas_per_sm) {
    using L = LayoutFor<Sh>;
    constexpr int kWarpsPerCta = Sh::WPC;
    const size_t bytes = sizeof(float) * (size_t)L::total(SIDE, kWarpsPerCta);
    auto kern = code_fast_kernel<Sh, SIDE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kWarpsPerCta * 32, bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    bps = std::max(1, std::min(bps, kMaxCtasPerSm));
    if (ctas_per_sm > 0) bps = std::min(bps, ctas_per_sm);
    const long long need = (a.N + Sh::SPC - 1) / Sh::SPC;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
    kern<<<grid, kWarpsPerCta * 32, bytes, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    return SIDE == kCodeOnly ? 0 : grid;
}

template <class Sh>
int launch_fast_side(const PassArgs& a, int side, cudaStream_t st, int num_sms, int ctas_per_sm) {
    switch (side) {
        case kCodeOnly: return launch_fast_impl<Sh, kCodeOnly>(a, st, num_sms, ctas_per_sm);
        case kSideD1: return launch_fast_impl<Sh, kSideD1>(a, st, num_sms, ctas_per_sm);
        case kSideD2: return launch_fast_impl<Sh, kSideD2>(a, st, num_sms, ctas_per_sm);
        default: return SDL_ERR_ARG;
    }
}

// Compiled shapes: <p1, p2, n1, n2, s, LI, RI, RJ, ZA, ZB, WI, WB, warps/CTA, min CTAs/SM>.
// Two lane tilings of the n1 x n2 correlation block per problem shape; the
// batch autotuner times both.
using F8x16s4 = Shape<8, 8, 16, 16, 4, 4, 4, 2, 2, 2, 2, 2, 8, 3>;
using F8x16s4b = Shape<8, 8, 16, 16, 4, 8, 2, 4, 2, 2, 2, 2, 8, 2>;
using F12x24s6 = Shape<12, 12, 24, 24, 6, 4, 6, 3, 3, 3, 3, 3, 8, 2>;
using F12x24s6b = Shape<12, 12, 24, 24, 6, 8, 3, 6, 3, 3, 3, 3, 8, 2>;
// 16x32: 6 warps per CTA, so that two CTAs' shared memory (partial-sum copies,
// C0 blocks, Y buffers) fits an SM
using F16x32s8 = Shape<16, 16, 32, 32, 8, 4, 8, 4, 4, 4, 4, 4, 6, 2>;
using F16x32s8b = Shape<16, 16, 32, 32, 8, 8, 4, 8, 4, 4, 4, 4, 6, 2>;
// two signals per warp: <p1, p2, n1, n2, s, LI, RI, RJ, ZA, ZB, WI, WB, warps/CTA, min CTAs/SM>
using H8x16s4 = HalfShape<8, 8, 16, 16, 4, 4, 4, 4, 2, 4, 4, 2, 8, 2>;
using H12x24s6 = HalfShape<12, 12, 24, 24, 6, 2, 12, 3, 6, 3, 6, 3, 8, 2>;

enum FastId { k8x16a = 0, k8x16b, k12x24a, k12x24b, k16x32a, k16x32b, k8x16h, k12x24h, kNumFast };

struct FastKey {
    int p1, p2, n1, n2, s;
};
constexpr FastKey kFastKeys[kNumFast] = {{8, 8, 16, 16, 4},  {8, 8, 16, 16, 4},
                                         {12, 12, 24, 24, 6}, {12, 12, 24, 24, 6},
                                         {16, 16, 32, 32, 8}, {16, 16, 32, 32, 8},
                                         {8, 8, 16, 16, 4},  {12, 12, 24, 24, 6}};

template <class F>
int with_shape(int id, F&& f) {
    switch (id) {
        case k8x16a: return f(F8x16s4{});
        case k8x16b: return f(F8x16s4b{});
        case k12x24a: return f(F12x24s6{});
        case k12x24b: return f(F12x24s6b{});
        case k16x32a: return f(F16x32s8{});
        case k16x32b: return f(F16x32s8b{});
        case k8x16h: return f(H8x16s4{});
        case k12x24h: return f(H12x24s6{});
        default: return SDL_ERR_UNSUPPORTED;
    }
}

// Persistent multi-problem pass: CTAs [cta_begin[g], cta_begin[g+1]) code the
// signals of problem g with its compiled shape; each problem writes one
// partial-sum slot per CTA into its own buffers.
template <int SIDE>
__global__ void __launch_bounds__(256, 2)
    code_multi_kernel(const PassArgs* __restrict__ groups, const int* __restrict__ cta_begin,
                      const int* __restrict__ shape, int G, int spread) {
    // position of this CTA: with spread = R SMs and W = gridDim / R waves, CTA
    // b = w R + r takes position r W + w (a bijection of 0..gridDim-1)
    int b = (int)blockIdx.x;
    if (spread > 0 && (int)gridDim.x % spread == 0) {
        const int waves = (int)gridDim.x / spread;
        b = (b % spread) * waves + b / spread;
    }
    int g = 0;
    while (g + 1 < G && b >= cta_begin[g + 1]) ++g;
    const int cta = b - cta_begin[g];
    const int n = cta_begin[g + 1] - cta_begin[g];
    const PassArgs a = groups[g];
    switch (shape[g]) {
        case k8x16a: code_fast_body<F8x16s4, SIDE>(a, cta, n, cta); break;
        case k8x16b: code_fast_body<F8x16s4b, SIDE>(a, cta, n, cta); break;
        case k12x24a: code_fast_body<F12x24s6, SIDE>(a, cta, n, cta); break;
        case k12x24b: code_fast_body<F12x24s6b, SIDE>(a, cta, n, cta); break;
        case k16x32a: code_fast_body<F16x32s8, SIDE>(a, cta, n, cta); break;
        case k16x32b: code_fast_body<F16x32s8b, SIDE>(a, cta, n, cta); break;
        case k8x16h: code_half_body<H8x16s4, SIDE>(a, cta, n, cta); break;
        case k12x24h: code_half_body<H12x24s6, SIDE>(a, cta, n, cta); break;
        default: break;
    }
}

template <int SIDE>
int launch_multi_impl(const PassArgs* d_groups, const int* d_cta_begin, const int* d_shape, int G,
                      int total_ctas, size_t smem, cudaStream_t st, int spread) {
    auto kern = code_multi_kernel<SIDE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    kern<<<total_ctas, 256, smem, st>>>(d_groups, d_cta_begin, d_shape, G, spread);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // namespace

int launch_code_pass_grid(const PassArgs& a, int side, int shape_id, int grid, cudaStream_t st) {
    if (grid < 1) return SDL_ERR_ARG;
    return with_shape(shape_id, [&](auto sh) -> int {
        using Sh = decltype(sh);
        const size_t bytes = sizeof(float) * (size_t)LayoutFor<Sh>::total(side, Sh::WPC);
        auto go = [&](auto kern) -> int {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess)
                return SDL_ERR_CUDA;
            kern<<<grid, Sh::WPC * 32, bytes, st>>>(a);
            return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
        };
        switch (side) {
            case kCodeOnly: return go(code_fast_kernel<Sh, kCodeOnly>);
            case kSideD1: return go(code_fast_kernel<Sh, kSideD1>);
            case kSideD2: return go(code_fast_kernel<Sh, kSideD2>);
            default: return SDL_ERR_ARG;
        }
    });
}

int fast_variant_ctas_per_sm(int shape_id, int side) {
    return with_shape(shape_id, [&](auto sh) -> int {
        using Sh = decltype(sh);
        const size_t bytes = sizeof(float) * (size_t)LayoutFor<Sh>::total(side, Sh::WPC);
        int bps = 0;
        auto occ = [&](auto kern) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, Sh::WPC * 32, bytes) != cudaSuccess) {
                cudaGetLastError();
                bps = 0;
            }
        };
        if (side == kCodeOnly) occ(code_fast_kernel<Sh, kCodeOnly>);
        else if (side == kSideD1) occ(code_fast_kernel<Sh, kSideD1>);
        else occ(code_fast_kernel<Sh, kSideD2>);
        return bps;
    });
}

int fast_variant_warps(int shape_id) {
    return with_shape(shape_id, [&](auto sh) { return decltype(sh)::WPC; });
}

int fast_shape_variants(int p1, int p2, int n1, int n2, int s, int* ids, int max_ids) {
    int k = 0;
    for (int id = 0; id < kNumFast; ++id) {
        const FastKey& f = kFastKeys[id];
        if (f.p1 == p1 && f.p2 == p2 && f.n1 == n1 && f.n2 == n2 && f.s == s && k < max_ids)
            ids[k++] = id;
    }
    return k;
}

size_t fast_smem_bytes(int shape_id, int side) {
    const int r = with_shape(shape_id, [&](auto sh) {
        using Sh = decltype(sh);
        return (int)(sizeof(float) * (size_t)LayoutFor<Sh>::total(side, Sh::WPC));
    });
    return r < 0 ? 0 : (size_t)r;
}

int launch_code_pass_variant(const PassArgs& a, int side, int shape_id, int ctas_per_sm,
                             cudaStream_t st, int num_sms) {
    return with_shape(shape_id, [&](auto sh) {
        return launch_fast_side<decltype(sh)>(a, side, st, num_sms, ctas_per_sm);
    });
}

int launch_code_multi(const PassArgs* d_groups, const int* d_cta_begin, const int* d_shape, int G,
                      int total_ctas, size_t smem, int side, cudaStream_t st, int spread) {
    switch (side) {
        case kCodeOnly: return launch_multi_impl<kCodeOnly>(d_groups, d_cta_begin, d_shape, G, total_ctas, smem, st, spread);
        case kSideD1: return launch_multi_impl<kSideD1>(d_groups, d_cta_begin, d_shape, G, total_ctas, smem, st, spread);
        case kSideD2: return launch_multi_impl<kSideD2>(d_groups, d_cta_begin, d_shape, G, total_ctas, smem, st, spread);
        default: return SDL_ERR_ARG;
    }
}

int multi_ctas_per_sm(size_t smem, int side) {
    int bps = 0;
    cudaError_t e = cudaSuccess;
    auto occ = [&](auto kern) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, smem);
    };
    if (side == kCodeOnly) occ(code_multi_kernel<kCodeOnly>);
    else if (side == kSideD1) occ(code_multi_kernel<kSideD1>);
    else occ(code_multi_kernel<kSideD2>);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return bps;
}

int launch_code_pass_fast(const PassArgs& a, int side, cudaStream_t st, int num_sms) {
    int ids[kNumFast];
    const int n = fast_shape_variants(a.p1, a.p2, a.n1, a.n2, a.s, ids, kNumFast);
    if (n == 0) return SDL_ERR_UNSUPPORTED;
    // a tiling pinned for this shape, else the first compiled variant
    for (int v = 0; v < n; ++v)
        if (a.tiling - 1 == ids[v]) return launch_code_pass_variant(a, side, ids[v], a.tiling_cps, st, num_sms);
    return launch_code_pass_variant(a, side, ids[0], 0, st, num_sms);
}

}  // namespace sdl
