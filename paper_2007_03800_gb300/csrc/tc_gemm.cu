// BF16 tensor-core GEMM for sm_103a: C = alpha * sum_t A_t B_t^T (+ bias,
// activation), A_t (M x K) and B_t (N x K) row-major with K contiguous,
// FP32 accumulation; t runs over 1 to 3 operand pairs summed into one
// accumulator (the split-precision products of the correlation path).
//
// Blackwell path, persistent and warp-specialised (one CTA per SM, 192
// threads):
//   warp 0  TMA producer: operand tiles by cp.async.bulk.tensor (128-byte
//           swizzle) into a shared-memory ring of 6 stages (4 at BN = 256)
//           guarded by mbarriers;
//   warp 1  MMA issuer: one thread issues tcgen05.mma (128 x BN x 16, BN =
//           256 when N is a multiple of 256 and the 256-wide tiles fill the
//           SMs, else 128) into one of two
//           BN-column FP32 accumulators in tensor memory (all 512 columns at
//           BN = 256: the wider tile halves the operand bytes each FLOP needs
//           from L2);
//           tcgen05.commit releases ring stages and hands a finished
//           accumulator to the epilogue;
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//           lanes 32 (w % 4) .. +31 = output rows), bias / GELU / GELU'
//           and the outputs.  The FP32 and BF16 row-major outputs leave by
//           TMA: each warp writes its 32 x 32 block into one of two swizzled
//           shared-memory slots and one lane issues cp.async.bulk.tensor (a
//           tensor reduce-add when accumulating), so the stores neither cost
//           the warp an instruction per row nor wait on it.  The other
//           outputs (transposed BF16, pre-activation, the GELU' product) go
//           through a per-warp 32 x 33 shared-memory transpose as coalesced
//           128-byte row segments.
// With two accumulators the epilogue of one tile overlaps the main loop of
// the next.  Tiles are visited m-block-major, so CTAs running at the same
// time share A rows and the whole of B in L2.
// Every wait is bounded (clock-based limit) and also ends when another role
// has failed: the CTA then records SDL_ERR_TIMEOUT, lets its copies land and
// frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ctx.cuh"

using namespace sdl;

namespace {

constexpr int BM = 128, BK = 64, UMMA_K = 16;
// shared-memory ring depth: as many stages as fit beside the epilogue's staging
__host__ __device__ constexpr int stages_for(int BN) { return BN == 256 ? 4 : 6; }
constexpr int kMaxTerms = 3;
constexpr int kThreads = 192;
constexpr int kEpiWarps = 4;
constexpr int kStageLd = 33;                  // epilogue transpose row stride (floats)
constexpr int kSlot = 4096;                   // one TMA output slot: 32 rows x 128 B
constexpr int kEpiBytes = kEpiWarps * 2 * kSlot;   // both epilogue forms share this area
static_assert(kEpiWarps * 32 * kStageLd * 4 <= kEpiBytes, "transpose staging must fit");
constexpr int TILE_A = BM * BK * 2;           // bytes
constexpr long long kWaitCycles = 1ll << 31;  // about one second at 2 GHz

struct Epi {
    float alpha;
    const float* bias;   // [N] or null
    int act;             // 0 none, 1 GELU (erf form), 2 times GELU'(gin)
    float* C;            // FP32 output or null
    int ldc;
    int accumulate;      // C += result
    __nv_bfloat16* Cb;   // BF16 copy or null
    int ldcb;
    __nv_bfloat16* Ct;   // BF16 transposed copy (Ct[n * ldct + m]) or null
    int ldct;
    int tma;             // C and Cb leave through the tensor maps Maps::c / Maps::cb
    float* pre;          // FP32 pre-activation (alpha*acc + bias) or null
    int ldpre;
    const float* gin;    // act 2: multiply by GELU'(gin[m, n])
    int ldgin;
};

struct Maps {
    CUtensorMap a[kMaxTerms];
    CUtensorMap b[kMaxTerms];
    CUtensorMap c;    // FP32 output, 32 x 32 boxes, 128-byte swizzle
    CUtensorMap cb;   // BF16 output, 32 x 32 boxes, 64-byte swizzle
};

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait; false on timeout or when *fail is set by another role
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* fail) {
    const uint32_t a = saddr(b);
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test(a, parity)) return true;
        if (*fail) return false;
        if (clock64() - t0 > kWaitCycles) {
            *fail = 1;
            return false;
        }
    }
}
// bounded wait used only to let copies land before exit
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity) {
    const uint32_t a = saddr(b);
    const long long t0 = clock64();
    while (!mbar_test(a, parity) && clock64() - t0 < kWaitCycles) {
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}
// 32 x 32 output block from shared memory to global (clipped at the tensor's
// edges); a reduce-add into global when `add`
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src,
                                             bool add) {
    if (add)
        asm volatile(
            "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                reinterpret_cast<uint64_t>(map)),
            "r"(x), "r"(y), "r"(saddr(src))
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                reinterpret_cast<uint64_t>(map)),
            "r"(x), "r"(y), "r"(saddr(src))
            : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major operand tile, 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t a = (saddr(p) & 0x3FFFFu) >> 4;
    return a | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major
template <int BN>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

// 64 consecutive accumulator columns of this thread's TMEM lane (one load
// per 64 columns: the load's latency is paid half as often as with 32); the
// wait follows at once, so v is complete when the call returns
__device__ __forceinline__ void tmem_ld64(uint32_t ta, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
        "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, "
        "%19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, "
        "%36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, "
        "%53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63 "
        "}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
          "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
          "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]),
          "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]),
          "=r"(v[62]), "=r"(v[63])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ Maps maps, int terms, int M, int N, int K, Epi epi,
                   int* err) {
    constexpr int TILE_B = BN * BK * 2;
    constexpr int STAGES = stages_for(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~uintptr_t(1023));
    uint8_t* sA = base;
    uint8_t* sB = base + STAGES * TILE_A;
    // epilogue area (1024-byte aligned): two TMA slots per warp, or the
    // transpose staging of the other outputs
    uint8_t* epi_area = sB + STAGES * TILE_B;
    float* stage_all = reinterpret_cast<float*>(epi_area);
    uint64_t* full = reinterpret_cast<uint64_t*>(epi_area + kEpiBytes);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;      // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;       // [2] epilogue -> MMA
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    __shared__ int s_fail;
    volatile int* fail = &s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K + BK - 1) / BK;
    const int ksteps = nk * terms;             // k-blocks per tile, all terms
    const int nt = (N + BN - 1) / BN;
    const long long tiles = (long long)((M + BM - 1) / BM) * nt;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            long long g = 0;   // k-blocks issued so far (ring position)
            for (long long t = blockIdx.x; t < tiles && !*fail; t += gridDim.x) {
                const int m0 = (int)(t / nt) * BM, n0 = (int)(t % nt) * BN;
                for (int ks = 0; ks < ksteps; ++ks) {
                    const int s = (int)(g % STAGES);
                    const long long use = g / STAGES;
                    if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), fail)) break;
                    const int term = ks / nk, kb = ks - term * nk;
                    mbar_arrive_tx(&full[s], TILE_A + TILE_B);
                    tma_load_2d(sA + s * TILE_A, &maps.a[term], kb * BK, m0, &full[s]);
                    tma_load_2d(sB + s * TILE_B, &maps.b[term], kb * BK, n0, &full[s]);
                    ++g;
                }
            }
            if (*fail) {
                // let the copies in flight land before shared memory is released
                for (long long h = g - STAGES > 0 ? g - STAGES : 0; h < g; ++h)
                    mbar_drain(&full[h % STAGES], (uint32_t)((h / STAGES) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = instr_desc<BN>();
            long long g = 0;
            int i = 0;   // local tile counter
            for (long long t = blockIdx.x; t < tiles && !*fail; t += gridDim.x, ++i) {
                const int b = i & 1, use_b = i >> 1;
                if (use_b > 0 && !mbar_wait(&acc_empty[b], (uint32_t)((use_b - 1) & 1), fail)) break;
                tc_fence_after();
                const uint32_t acc_addr = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int ks = 0; ks < ksteps; ++ks, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1), fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                        const uint64_t ad = smem_desc(sA + s * TILE_A + kk * UMMA_K * 2);
                        const uint64_t bd = smem_desc(sB + s * TILE_B + kk * UMMA_K * 2);
                        const uint32_t accum = (ks > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                acc_addr),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(saddr(&empty[s]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        saddr(&acc_full[b]))
                    : "memory");
            }
        }
    } else {
        // ---- epilogue warps
        const int quarter = warp & 3;              // TMEM lanes this warp may access
        float* stage = stage_all + (warp - 2) * 32 * kStageLd;
        uint8_t* slots = epi_area + (warp - 2) * 2 * kSlot;
        int slot = 0;
        int i = 0;
        for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int b = i & 1, use_b = i >> 1;
            int got = 0;
            if (lane == 0) got = mbar_wait(&acc_full[b], (uint32_t)(use_b & 1), fail) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            tc_fence_after();
            const int m0 = (int)(t / nt) * BM, n0 = (int)(t % nt) * BN;
            const int row0 = m0 + quarter * 32;    // first output row of this warp
            const int m = row0 + lane;
            for (int c64 = 0; c64 < BN; c64 += 64) {
                uint32_t v[64];
                tmem_ld64(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c64), v);
                if (c64 + 64 == BN) {
                    // the whole accumulator has been read: hand it back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
                }
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int c0 = c64 + 32 * h;   // this 32-column block
                float x[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + c0 + j;
                    x[j] = epi.alpha * __uint_as_float(v[32 * h + j]);
                    if (epi.bias && n < N) x[j] += epi.bias[n];
                }
                if (epi.tma) {
                    // act is 0 or 1 here, no pre-activation or transposed copy
                    if (epi.act == 1) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            x[j] = 0.5f * x[j] * (1.f + erff(x[j] * 0.70710678118654752f));
                    }
                    if (n0 + c0 >= N || row0 >= M) continue;   // block wholly outside C
                    // a slot is rewritten only after the store issued from it two
                    // stores ago has read it
                    auto next_slot = [&]() {
                        uint8_t* buf = slots + slot * kSlot;
                        slot ^= 1;
                        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                        __syncwarp();
                        return buf;
                    };
                    auto issue = [&](const CUtensorMap* map, const uint8_t* buf, bool add) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) tma_store_2d(map, n0 + c0, row0, buf, add);
                    };
                    if (epi.C) {
                        // row `lane` is 128 B; its 16-byte chunk k sits at k ^ (lane & 7)
                        uint8_t* buf = next_slot();
                        float4* row = reinterpret_cast<float4*>(buf + lane * 128);
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            row[k ^ (lane & 7)] =
                                make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
                        issue(&maps.c, buf, epi.accumulate != 0);
                    }
                    if (epi.Cb) {
                        // row `lane` is 64 B; its 16-byte chunk k sits at k ^ ((lane >> 1) & 3)
                        uint8_t* buf = next_slot();
                        uint4* row = reinterpret_cast<uint4*>(buf + lane * 64);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const __nv_bfloat162 pr =
                                    __floats2bfloat162_rn(x[8 * k + 2 * h], x[8 * k + 2 * h + 1]);
                                w[h] = *reinterpret_cast<const uint32_t*>(&pr);
                            }
                            row[k ^ ((lane >> 1) & 3)] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                        issue(&maps.cb, buf, false);
                    }
                    continue;
                }
                // row-major [m, n] block (32 rows of this warp x 32 columns),
                // stored (or added) one coalesced row segment at a time
                auto store_rows = [&](float* dst, int ld, int accumulate) {
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 32; ++j) stage[lane * kStageLd + j] = x[j];
                    __syncwarp();
                    const int n = n0 + c0 + lane;
                    if (accumulate) {
                        // all 32 old values first (independent loads), then the stores
                        float old[32];
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr) {
                            const int mm = row0 + rr;
                            old[rr] = (mm < M && n < N) ? dst[(size_t)mm * ld + n] : 0.f;
                        }
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr) {
                            const int mm = row0 + rr;
                            if (mm < M && n < N)
                                dst[(size_t)mm * ld + n] = old[rr] + stage[rr * kStageLd + lane];
                        }
                    } else {
                        for (int rr = 0; rr < 32; ++rr) {
                            const int mm = row0 + rr;
                            if (mm < M && n < N) dst[(size_t)mm * ld + n] = stage[rr * kStageLd + lane];
                        }
                    }
                };
                if (epi.pre) store_rows(epi.pre, epi.ldpre, 0);
                if (epi.act == 1) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        x[j] = 0.5f * x[j] * (1.f + erff(x[j] * 0.70710678118654752f));
                } else if (epi.act == 2) {
                    // chain rule through GELU: d/du [u Phi(u)] = Phi(u) + u phi(u); the
                    // gin block arrives through the transpose buffer
                    __syncwarp();
                    const int n = n0 + c0 + lane;
                    for (int rr = 0; rr < 32; ++rr) {
                        const int mm = row0 + rr;
                        stage[rr * kStageLd + lane] =
                            (mm < M && n < N) ? epi.gin[(size_t)mm * epi.ldgin + n] : 0.f;
                    }
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float u = stage[lane * kStageLd + j];
                        const float Phi = 0.5f * (1.f + erff(u * 0.70710678118654752f));
                        const float phi = 0.3989422804014327f * expf(-0.5f * u * u);
                        x[j] *= Phi + u * phi;
                    }
                }
                if (epi.C) store_rows(epi.C, epi.ldc, epi.accumulate);
                if (epi.Cb) {
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 32; ++j) stage[lane * kStageLd + j] = x[j];
                    __syncwarp();
                    const int n = n0 + c0 + lane;
                    for (int rr = 0; rr < 32; ++rr) {
                        const int mm = row0 + rr;
                        if (mm < M && n < N)
                            epi.Cb[(size_t)mm * epi.ldcb + n] =
                                __float2bfloat16_rn(stage[rr * kStageLd + lane]);
                    }
                }
                if (epi.Ct && m < M) {
                    // transposed: for a fixed column the lanes write consecutive m
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < N) epi.Ct[(size_t)n * epi.ldct + m] = __float2bfloat16_rn(x[j]);
                    }
                }
              }
            }
        }
        // the output stores have left shared memory and are complete
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) record_error(err, SDL_ERR_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * BN)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// rows x cols bf16 matrix, row stride ld (elements), box box_rows rows x 64 cols
int make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return SDL_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SDL_OK : SDL_ERR_ARG;
}

constexpr size_t smem_bytes(int BN) {
    return 1024 + (size_t)stages_for(BN) * (TILE_A + BN * BK * 2) + kEpiBytes + 256;
}
static_assert(smem_bytes(256) <= 232448 && smem_bytes(128) <= 232448, "shared memory per CTA");

// output map: rows x cols matrix of 4-byte (f32) or 2-byte (bf16) elements,
// row stride ld elements, 32 x 32 boxes swizzled to match the epilogue's slots
int make_out_map(CUtensorMap* map, void* ptr, int rows, int cols, int ld, bool bf16) {
    auto fn = encode_fn();
    if (!fn) return SDL_ERR_CUDA;
    const size_t es = bf16 ? 2 : 4;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    const cuuint32_t box[2] = {32u, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SDL_OK : SDL_ERR_ARG;
}

// Encoded tensor maps, remembered per host thread: a training loop calls the
// same GEMMs on the same buffers thousands of times, and encoding two to four
// maps per call is host time on a launch-bound path.  A map depends only on
// the arguments of its encoding, which form the key.
struct MapKey {
    const void* ptr;
    int rows, cols, ld, box_rows, kind;   // kind 0: operand, 1: FP32 out, 2: BF16 out
    bool operator==(const MapKey& o) const {
        return ptr == o.ptr && rows == o.rows && cols == o.cols && ld == o.ld &&
               box_rows == o.box_rows && kind == o.kind;
    }
};
constexpr int kMapCache = 32;
struct MapCache {
    MapKey key[kMapCache];
    CUtensorMap map[kMapCache];
    int used = 0, next = 0;
};
thread_local MapCache t_maps;

template <class Encode>
int cached_map(CUtensorMap* out, const MapKey& k, Encode encode) {
    MapCache& c = t_maps;
    for (int i = 0; i < c.used; ++i)
        if (c.key[i] == k) {
            *out = c.map[i];
            return SDL_OK;
        }
    const int rc = encode(out);
    if (rc != SDL_OK) return rc;
    const int slot = c.used < kMapCache ? c.used++ : c.next;
    c.next = (slot + 1) % kMapCache;
    c.key[slot] = k;
    c.map[slot] = *out;
    return SDL_OK;
}

int sm_count() {
    static int count[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!count[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        count[dev] = n;
    }
    return count[dev];
}

}  // namespace

namespace sdl {
int tc_gemm_terms(const void* const* A, int lda, const void* const* B, int ldb, int terms, int M,
                  int N, int K, float alpha, const float* bias, int act, float* C, int ldc,
                  int accumulate, void* Cb, int ldcb, void* Ct, int ldct, float* pre, int ldpre,
                  int* err, cudaStream_t st, const float* gin, int ldgin) {
    if (!A || !B || terms < 1 || terms > kMaxTerms || M < 1 || N < 1 || K < 1) return SDL_ERR_ARG;
    if (act == 2 && !gin) return SDL_ERR_ARG;
    if ((lda % 8) || (ldb % 8) || lda < K || ldb < K) return SDL_ERR_ARG;
    // 128 x 256 tiles when N is a multiple of 256 and there are enough of them
    // to fill the SMs, else 128 x 128 (a small output with a long K, such as a
    // weight gradient, keeps twice the CTAs busy)
    const long long mb = (M + BM - 1) / BM;
    const int bn = (N % 256 == 0 && mb * (N / 256) >= sm_count()) ? 256 : 128;
    Maps maps;
    std::memset(&maps, 0, sizeof(maps));
    int rc;
    for (int t = 0; t < terms; ++t) {
        if (!A[t] || !B[t] || (reinterpret_cast<uintptr_t>(A[t]) & 15u) ||
            (reinterpret_cast<uintptr_t>(B[t]) & 15u))
            return SDL_ERR_ARG;
        if ((rc = cached_map(&maps.a[t], MapKey{A[t], M, K, lda, BM, 0}, [&](CUtensorMap* m) {
                 return make_map(m, A[t], M, K, lda, BM);
             })) != SDL_OK)
            return rc;
        if ((rc = cached_map(&maps.b[t], MapKey{B[t], N, K, ldb, bn, 0}, [&](CUtensorMap* m) {
                 return make_map(m, B[t], N, K, ldb, bn);
             })) != SDL_OK)
            return rc;
    }
    Epi e;
    e.alpha = alpha;
    e.bias = bias;
    e.act = act;
    e.C = C;
    e.ldc = ldc;
    e.accumulate = accumulate;
    e.Cb = static_cast<__nv_bfloat16*>(Cb);
    e.ldcb = ldcb;
    e.Ct = static_cast<__nv_bfloat16*>(Ct);
    e.ldct = ldct;
    e.pre = pre;
    e.ldpre = ldpre;
    e.gin = gin;
    e.ldgin = ldgin;
    // C and Cb leave by TMA when they are the only outputs and their rows
    // start and end on 16-byte boundaries (a tensor store clips the row at
    // 16-byte granularity: a row of 13 BF16 values would also get 3 values of
    // its padding); otherwise every output takes the transpose path
    bool tma = (C || Cb) && !pre && !Ct && act != 2;
    if (C)
        tma = tma && !(reinterpret_cast<uintptr_t>(C) & 15u) && ldc % 4 == 0 && N % 4 == 0 &&
              ldc >= N;
    if (Cb)
        tma = tma && !(reinterpret_cast<uintptr_t>(Cb) & 15u) && ldcb % 8 == 0 && N % 8 == 0 &&
              ldcb >= N;
    if (tma && C)
        tma = cached_map(&maps.c, MapKey{C, M, N, ldc, 32, 1}, [&](CUtensorMap* m) {
                  return make_out_map(m, C, M, N, ldc, false);
              }) == SDL_OK;
    if (tma && Cb)
        tma = cached_map(&maps.cb, MapKey{Cb, M, N, ldcb, 32, 2}, [&](CUtensorMap* m) {
                  return make_out_map(m, Cb, M, N, ldcb, true);
              }) == SDL_OK;
    e.tma = tma ? 1 : 0;
    auto launch = [&](auto kern, int BN) -> int {
        const size_t bytes = smem_bytes(BN);
        // the shared-memory opt-in is set once per device and tile width
        static bool attr_set[2][64] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return SDL_ERR_CUDA;
        bool& done = attr_set[BN == 256][dev & 63];
        if (!done || dev >= 64) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess)
                return SDL_ERR_CUDA;
            done = dev < 64;
        }
        const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
        const int grid = (int)std::min<long long>(tiles, sm_count());
        kern<<<grid, kThreads, bytes, st>>>(maps, terms, M, N, K, e, err);
        return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
    };
    return bn == 256 ? launch(tc_gemm_kernel<256>, 256) : launch(tc_gemm_kernel<128>, 128);
}

int tc_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float alpha,
            const float* bias, int act, float* C, int ldc, int accumulate, void* Cb, int ldcb,
            void* Ct, int ldct, float* pre, int ldpre, int* err, cudaStream_t st,
            const float* gin, int ldgin) {
    const void* a[1] = {A};
    const void* b[1] = {B};
    return tc_gemm_terms(a, lda, b, ldb, 1, M, N, K, alpha, bias, act, C, ldc, accumulate, Cb,
                         ldcb, Ct, ldct, pre, ldpre, err, st, gin, ldgin);
}
}  // namespace sdl

extern "C" int sdl_gemm_bf16(sdl_ctx* c, const void* A, int lda, const void* B, int ldb, int M,
                             int N, int K, float alpha, const float* bias, int act, float* C,
                             int ldc, int accumulate, void* Cb, int ldcb, void* Ct, int ldct,
                             float* pre, int ldpre, void* stream) {
    if (!c) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    if (act == 2) return SDL_ERR_ARG;   // the GELU-derivative mode is internal
    return tc_gemm(A, lda, B, ldb, M, N, K, alpha, bias, act, C, ldc, accumulate, Cb, ldcb, Ct,
                   ldct, pre, ldpre, c->err, (cudaStream_t)stream, nullptr, 0);
}

extern "C" int sdl_gemm_bf16_terms(sdl_ctx* c, const void* const* A, int lda,
                                   const void* const* B, int ldb, int terms, int M, int N, int K,
                                   float alpha, const float* bias, int act, float* C, int ldc,
                                   int accumulate, void* Cb, int ldcb, void* Ct, int ldct,
                                   float* pre, int ldpre, void* stream) {
    if (!c) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    if (act == 2) return SDL_ERR_ARG;
    return sdl::tc_gemm_terms(A, lda, B, ldb, terms, M, N, K, alpha, bias, act, C, ldc,
                              accumulate, Cb, ldcb, Ct, ldct, pre, ldpre, c->err,
                              (cudaStream_t)stream, nullptr, 0);
}
