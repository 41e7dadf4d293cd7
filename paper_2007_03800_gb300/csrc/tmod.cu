// Tensor-MOD dictionary update: reduction of the per-CTA partial sums, the
// small normal-equation solve with atom normalisation (Corollary 1 for D1,
// Result 1 for D2), the W^{-1} rescale of the codes, and the Gram matrices.
#include <algorithm>
#include <type_traits>
#include <cmath>

#include <cstdint>

#include "sdl_internal.cuh"

namespace sdl {
namespace {


// G = D^T D (row-major n x n) for a column-major p x n dictionary.
__global__ void gram_kernel(const float* __restrict__ D, int p, int n, float* __restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e / n, j = e - i * n;
    const float* di = D + (size_t)p * i;
    const float* dj = D + (size_t)p * j;
    float g = 0.f;
    for (int a = 0; a < p; ++a) g = fmaf(di[a], dj[a], g);
    G[e] = g;
}

// Gram matrices of several dictionaries in one launch (block ranges per entry).
__global__ void gram_multi_kernel(const GramDesc* __restrict__ d, int G) {
    int g = 0;
    while (g + 1 < G && (int)blockIdx.x >= d[g + 1].block_begin) ++g;
    const GramDesc q = d[g];
    const int e = (blockIdx.x - q.block_begin) * blockDim.x + threadIdx.x;
    if (e >= q.n * q.n) return;
    const int i = e / q.n, j = e - i * q.n;
    float acc = 0.f;
    for (int a = 0; a < q.p; ++a) acc = fmaf(q.D[(size_t)q.p * i + a], q.D[(size_t)q.p * j + a], acc);
    q.G[e] = acc;
}

// Both Gram matrices in one launch: blocks [0, b1) for D1, the rest for D2.
__global__ void gram2_kernel(const float* __restrict__ D1, int p1, int n1, float* __restrict__ G1,
                             int b1, const float* __restrict__ D2, int p2, int n2,
                             float* __restrict__ G2) {
    const bool first = blockIdx.x < b1;
    const float* D = first ? D1 : D2;
    const int p = first ? p1 : p2, n = first ? n1 : n2;
    float* G = first ? G1 : G2;
    const int e = (first ? blockIdx.x : blockIdx.x - b1) * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e / n, j = e - i * n;
    float g = 0.f;
    for (int a = 0; a < p; ++a) g = fmaf(D[(size_t)p * i + a], D[(size_t)p * j + a], g);
    G[e] = g;
}

// Fixed-order compensated sum of the partial-sum slots, no floating-point
// atomics (deterministic for a given slot count).  A block owns 32 entries;
// warp w sums slots w, w+16, w+32, ... (coalesced 128-byte rows) in eight
// interleaved compensated sums, so that eight loads per lane are in flight,
// then warp 0 adds the 16 warp sums in order.
constexpr int kReduceWarps = 16;
constexpr int kReduceIlp = 8;

__device__ __forceinline__ void reduce_body(const float* __restrict__ part_f,
                                            const double* __restrict__ part_d, int n_slots,
                                            int nf, float* __restrict__ red_f,
                                            double* __restrict__ red_d, int blk) {
    __shared__ float ws[kReduceWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blk * 32 + lane;
    float sum[kReduceIlp], comp[kReduceIlp];
#pragma unroll
    for (int u = 0; u < kReduceIlp; ++u) sum[u] = comp[u] = 0.f;
    if (e < nf) {
        int c = warp;
        for (; c + (kReduceIlp - 1) * kReduceWarps < n_slots; c += kReduceIlp * kReduceWarps) {
            float v[kReduceIlp];
#pragma unroll
            for (int u = 0; u < kReduceIlp; ++u) v[u] = part_f[(size_t)(c + u * kReduceWarps) * nf + e];
#pragma unroll
            for (int u = 0; u < kReduceIlp; ++u) {
                const float y = v[u] - comp[u];
                const float t = sum[u] + y;
                comp[u] = (t - sum[u]) - y;
                sum[u] = t;
            }
        }
        for (; c < n_slots; c += kReduceWarps) {
            const float y = part_f[(size_t)c * nf + e] - comp[0];
            const float t = sum[0] + y;
            comp[0] = (t - sum[0]) - y;
            sum[0] = t;
        }
    }
    float wsum = 0.f;
#pragma unroll
    for (int u = 0; u < kReduceIlp; ++u) wsum += sum[u] - comp[u];
    ws[warp][lane] = wsum;
    __syncthreads();
    if (warp == 0 && e < nf) {
        float tot = 0.f, c2 = 0.f;
#pragma unroll
        for (int w = 0; w < kReduceWarps; ++w) {
            const float y = ws[w][lane] - c2;
            const float t = tot + y;
            c2 = (t - tot) - y;
            tot = t;
        }
        red_f[e] = tot;
    }
    if (blk == 0 && warp < 2) {
        // the two FP64 sums: lanes stride over the slots, then a fixed shuffle tree
        double d = 0.0;
        for (int c = lane; c < n_slots; c += 32) d += part_d[(size_t)c * 2 + warp];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) red_d[warp] = d;
    }
}

__global__ void __launch_bounds__(kReduceWarps * 32)
    reduce_partials_kernel(const float* __restrict__ part_f, const double* __restrict__ part_d,
                           int n_slots, int nf, float* __restrict__ red_f,
                           double* __restrict__ red_d) {
    reduce_body(part_f, part_d, n_slots, nf, red_f, red_d, blockIdx.x);
}

// Reductions of several problems in one launch; d[g].block_begin is the first
// block of problem g (ascending), blocks of a problem cover its nf entries.
__global__ void __launch_bounds__(kReduceWarps * 32)
    reduce_multi_kernel(const ReduceDesc* __restrict__ d, int G) {
    int g = 0;
    while (g + 1 < G && (int)blockIdx.x >= d[g + 1].block_begin) ++g;
    const ReduceDesc r = d[g];
    reduce_body(r.part_f, r.part_d, r.n_slots, r.nf, r.red_f, r.red_d, blockIdx.x - r.block_begin);
}

// One CTA: the normal-equation solve of a dictionary update with atom
// normalisation (Corollary 1 for D1, Result 1 for D2).
//   red_f = [P (n x n, row-major) | B (p x n, row-major)], red_d[0] = objective
//   before the update (sum of residual energies with the old dictionary).
// Only the used atoms (diag(P) > 0) take part; unused atoms keep their column.
//   1. P_u^{-1} by in-place Gauss-Jordan elimination without pivoting: for an
//      SPD matrix the k-th pivot is the k-th Cholesky pivot squared, so the
//      same relative-pivot test flags a singular P;
//   2. D* = B_u P_u^{-1} (rows of the right-hand side times the inverse);
//   3. objective after = before + sum_a Delta_a (P (D*_a + D_old_a) - 2 B_a),
//      Delta = D* - D_old by rows a: the change of the least-squares objective
//      of Result 1 for ANY D*, so an inexact solve (an ill-conditioned P)
//      enters only to second order, unlike before - tr(Delta P Delta^T),
//      which holds at the exact minimiser only;
//   4. norms of the columns of D*, D <- D* diag(1/norm), optional G = D^T D.
// Every step is a data-parallel sweep, one barrier per pivot.  On any
// failure D is left untouched and the norms are set to 1.
constexpr int kSolveThreads = 512;       // n > 32
constexpr int kSolveThreadsSmall = 256;  // n <= 32

// f(integral_constant<int, i>) for i = B .. E-1, unrolled at compile time
template <int B, int E, class F>
__device__ __forceinline__ void unrolled_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        unrolled_for<B + 1, E>(f);
    }
}

// In-place Gauss-Jordan inverse of the nu x nu matrix A (stride lda) without
// pivoting, the matrix held in registers: thread (ti, tj) of a TI x TJ grid
// owns rows ti + TI r and columns tj + TJ c (r < RI, c < RJ), so a warp reads
// consecutive columns.  Only the pivot row and column go through shared
// memory (rc: two buffers of row | column, 4 nu floats), published by their
// owners after each update: one barrier per pivot.  Every element takes the
// same operations as the shared-memory form:
//   a_rc - (a_rk / p) a_kc,  a_kc / p,  -a_rk / p,  1 / p.
// Pivots run as k = t + TI r (r outer and unrolled, t inner), so pivot k sits
// in register row r and, with TJ a multiple of TI, in register column
// r / (TJ / TI): no register array is indexed at run time.
// Returns false (everywhere) at the first pivot that fails the relative test.
template <int TI, int TJ, int RI, int RJ>
__device__ bool gj_inverse_regs(float* A, int lda, int nu, const float* d0, float* rc) {
    static_assert(TJ % TI == 0, "pivot columns must follow the row blocks");
    constexpr int M = TJ / TI;
    const int tid = threadIdx.x, ti = tid / TJ, tj = tid % TJ;
    float a[RI][RJ];
#pragma unroll
    for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < RJ; ++c) {
            const int R = ti + TI * r, C = tj + TJ * c;
            a[r][c] = (R < nu && C < nu) ? A[R * lda + C] : 0.f;
        }
    // buffer b: pivot row at rc + 2 nu b, pivot column at rc + 2 nu b + nu;
    // the owners of row / column kn (register row rr, register column cc)
    // write them there
    auto publish = [&](int kn, auto rrc, auto ccc) {
        constexpr int rr = decltype(rrc)::value, cc = decltype(ccc)::value;
        float* rown = rc + 2 * nu * (kn & 1);
        float* coln = rown + nu;
        if (ti == kn % TI)
#pragma unroll
            for (int c = 0; c < RJ; ++c)
                if (tj + TJ * c < nu) rown[tj + TJ * c] = a[rr][c];
        if (tj == kn % TJ)
#pragma unroll
            for (int r = 0; r < RI; ++r)
                if (ti + TI * r < nu) coln[ti + TI * r] = a[r][cc];
    };
    publish(0, std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{});
    __syncthreads();
    bool ok = true, done = false;
    unrolled_for<0, RI>([&](auto rcst) {
        constexpr int r0 = decltype(rcst)::value;
        if (done) return;
        for (int t = 0; t < TI; ++t) {
            const int k = t + TI * r0;
            if (k >= nu) {
                done = true;
                break;
            }
            const float* rowk = rc + 2 * nu * (k & 1);
            const float* colk = rowk + nu;
            const float piv = colk[k];
            if (!(piv > kSolvePivotRel * d0[k])) {
                ok = false;
                done = true;
                break;
            }
            const float inv = 1.f / piv;
            float cr[RI], rw[RJ];
#pragma unroll
            for (int r = 0; r < RI; ++r) cr[r] = colk[min(ti + TI * r, nu - 1)];
#pragma unroll
            for (int c = 0; c < RJ; ++c) rw[c] = rowk[min(tj + TJ * c, nu - 1)];
#pragma unroll
            for (int r = 0; r < RI; ++r) {
                const int R = ti + TI * r;
                const float f = cr[r] * inv;
#pragma unroll
                for (int c = 0; c < RJ; ++c) {
                    const int C = tj + TJ * c;
                    float v;
                    if (R != k) v = (C != k) ? fmaf(-f, rw[c], a[r][c]) : cr[r] * -inv;
                    else v = (C != k) ? rw[c] * inv : inv;
                    a[r][c] = v;
                }
            }
            const int kn = k + 1;
            if (kn < nu) {
                if (t + 1 < TI) {
                    publish(kn, std::integral_constant<int, r0>{}, std::integral_constant<int, r0 / M>{});
                } else if constexpr (r0 + 1 < RI) {
                    publish(kn, std::integral_constant<int, r0 + 1>{},
                            std::integral_constant<int, (r0 + 1) / M>{});
                }
            }
            __syncthreads();
        }
    });
    if (ok)
#pragma unroll
        for (int r = 0; r < RI; ++r)
#pragma unroll
            for (int c = 0; c < RJ; ++c) {
                const int R = ti + TI * r, C = tj + TJ * c;
                if (R < nu && C < nu) A[R * lda + C] = a[r][c];
            }
    return ok;
}

// out[a][c] = init(a, c) + sum_k Lf(a, k) Rf(k, c) for a < m, c < nu, k in
// increasing order (each entry one FMA chain, as a plain loop), in 4 x 4
// register blocks: thread (ta, tc) of a TA x TC grid takes rows ta + TA i and
// columns tc + TC j, so a warp reads one row of L and consecutive columns of
// R.  `emit` receives (a, c, value).
template <int TA, int TC, class Lf, class Rf, class Init, class Emit>
__device__ __forceinline__ void block_product(int m, int nu, int kn, Lf lf, Rf rf, Init init,
                                              Emit emit) {
    const int tid = threadIdx.x, ta = tid / TC, tc = tid % TC;
    for (int ab = 0; ab < m; ab += 4 * TA)
        for (int cb = 0; cb < nu; cb += 4 * TC) {
            float acc[4][4];
            int ai[4], ci[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ai[i] = min(ab + ta + TA * i, m - 1);
                ci[i] = min(cb + tc + TC * i, nu - 1);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = init(ai[i], ci[j]);
            for (int k = 0; k < kn; ++k) {
                float l[4], r[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) l[i] = lf(ai[i], k);
#pragma unroll
                for (int j = 0; j < 4; ++j) r[j] = rf(k, ci[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(l[i], r[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int a = ab + ta + TA * i, c = cb + tc + TC * j;
                    if (a < m && c < nu) emit(a, c, acc[i][j]);
                }
        }
}

// kLarge: the n > 32 instantiation (the 8 x 4 register Gauss-Jordan and the
// blocked products); the n <= 32 one stays small, since each solve runs once
// from a cold instruction cache.
template <bool kLarge>
__device__ __forceinline__ void solve_body(const float* __restrict__ red_f,
                                           const double* __restrict__ red_d, float* D, int p,
                                           int n, float* __restrict__ norms, double inv_count,
                                           double* objective_out, double* rmse_out, int* err,
                                           float* G_out, int keep_p) {
    extern __shared__ __align__(16) float sm[];
    // keep_p: a copy of P_u stays in shared memory for the objective term
    // (else P_u is read again into A once the inverse has been used)
    keep_p &= 1;
    const int lda = n | 1;                          // odd row strides: fewer bank conflicts
    float* A = sm;                                  // nu x nu (stride lda): P_u, then its inverse
    float* A2 = A + n * lda;                        // pivot rows | columns, two buffers (4n)
    float* Bc = A2 + 4 * n;                         // p x nu right-hand sides (stride lda)
    float* X = Bc + p * lda;                        // p x nu, D* rows (stride lda)
    float* Dn = X + p * lda;                        // p x n, old then new D (stride lda)
    float* P0 = Dn + p * lda;                       // nu x nu copy of P_u (stride lda), if kept
    float* nrm = P0 + (keep_p ? n * lda : 0);       // n
    float* d0 = nrm + n;                            // n
    int* idx = reinterpret_cast<int*>(d0 + n);      // n
    __shared__ int s_nu, s_fail;
    __shared__ double s_red[kSolveThreads / 32];

    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    const float* P = red_f;
    const float* B = red_f + n * n;

    if (tid < 32) {
        int base = 0, fail = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const float dl = (i < n) ? P[i * n + i] : 0.f;
            if (i < n && !isfinite(dl)) fail = SDL_ERR_NONFINITE;
            const unsigned um = __ballot_sync(0xffffffffu, i < n && dl > 0.f);
            if (i < n && dl > 0.f) {
                const int pos = base + __popc(um & ((1u << lane) - 1u));
                idx[pos] = i;
                d0[pos] = dl;
            }
            base += __popc(um);
        }
        fail = __reduce_or_sync(0xffffffffu, fail);
        if (lane == 0) {
            s_nu = base;
            s_fail = fail;
        }
    }
    __syncthreads();
    const int nu = s_nu;
    // every loop below maps rows to warps and columns to lanes (no index division)
    int bad = 0;
#pragma unroll 4
    for (int r = warp; r < nu; r += nw)
        for (int c = lane; c < nu; c += 32) {
            const float v = P[idx[r] * n + idx[c]];
            A[r * lda + c] = v;
            if (keep_p) P0[r * lda + c] = v;
            if (!isfinite(v)) bad = SDL_ERR_NONFINITE;
        }
#pragma unroll 4
    for (int r = warp; r < p; r += nw)
        for (int c = lane; c < nu; c += 32) {
            const float v = B[r * n + idx[c]];
            Bc[r * lda + c] = v;
            if (!isfinite(v)) bad = SDL_ERR_NONFINITE;
        }
#pragma unroll 4
    for (int c = warp; c < n; c += nw)
        for (int r = lane; r < p; r += 32) Dn[r * lda + c] = D[r + p * c];
    if (bad) s_fail = bad;
    __syncthreads();

    // 1. Gauss-Jordan inverse of the used block, held in registers (one
    //    barrier per pivot); every thread sees the same pivot, so a failed
    //    pivot test ends the loop everywhere
    if (s_fail == 0) {
        bool ok;
        bool regs = false;
        if constexpr (kLarge) {
            if (nth == kSolveThreads && nu <= 128) {
                ok = gj_inverse_regs<16, 32, 8, 4>(A, lda, nu, d0, A2);
                regs = true;
            }
        } else {
            if (nth == kSolveThreadsSmall && nu <= 32) {
                ok = gj_inverse_regs<16, 16, 2, 2>(A, lda, nu, d0, A2);
                regs = true;
            }
        }
        if (!regs) {
            // any other size: in place through shared memory, the saved pivot
            // row and column in A2 (two barriers per pivot)
            ok = true;
            float* rowk = A2;
            float* colk = A2 + n;
            for (int k = 0; k < nu; ++k) {
                const float piv = A[k * lda + k];
                if (!(piv > kSolvePivotRel * d0[k])) {
                    ok = false;
                    break;
                }
                const float inv = 1.f / piv;
                for (int c = tid; c < nu; c += nth) {
                    rowk[c] = A[k * lda + c];
                    colk[c] = A[c * lda + k];
                }
                __syncthreads();
                for (int r = warp; r < nu; r += nw) {
                    float* ar = A + r * lda;
                    const float ark = colk[r];
                    const float f = ark * inv;
                    for (int c = lane; c < nu; c += 32) {
                        float v;
                        if (r != k) v = (c != k) ? fmaf(-f, rowk[c], ar[c]) : ark * -inv;
                        else v = (c != k) ? rowk[c] * inv : inv;
                        ar[c] = v;
                    }
                }
                __syncthreads();
            }
        }
        if (!ok && tid == 0) s_fail = SDL_ERR_SINGULAR;
    }
    __syncthreads();
    const float* Ain = A;
    const bool ok_inv = (s_fail == 0);
    double part = 0.0;
    if (ok_inv) {
        // 2. D* rows: D*[a][c] = sum_k B[a][k] P_u^{-1}[k][c].  Few entries
        //    (p nu <= 2 threads): one chain per thread; else 4 x 4 blocks
        const bool blocked = kLarge && nth == kSolveThreads && p * nu > 2 * nth;
        if constexpr (kLarge) {
            if (blocked)
            block_product<16, 32>(
                p, nu, nu, [&](int a, int k) { return Bc[a * lda + k]; },
                [&](int k, int c) { return Ain[k * lda + c]; }, [](int, int) { return 0.f; },
                [&](int a, int c, float v) { X[a * lda + c] = v; });
        }
        if (!blocked) {
            for (int a = warp; a < p; a += nw)
                for (int c = lane; c < nu; c += 32) {
                    float x = 0.f;
#pragma unroll 4
                    for (int k = 0; k < nu; ++k) x = fmaf(Bc[a * lda + k], Ain[k * lda + c], x);
                    X[a * lda + c] = x;
                }
        }
        __syncthreads();
        // 3. objective change: for row a and used atom c,
        //    w = -2 B[a][c] + sum_k P_u[c][k] (D_old[a][idx k] + D*[a][k]),
        //    the sum in increasing k; P_u from the kept copy, or read again
        //    into A (the inverse is no longer needed)
        const float* Pu = P0;
        if (!keep_p) {
#pragma unroll 4
            for (int r = warp; r < nu; r += nw)
                for (int c = lane; c < nu; c += 32) A[r * lda + c] = P[idx[r] * n + idx[c]];
            __syncthreads();
            Pu = A;
        }
        if constexpr (kLarge) {
            if (blocked)
            block_product<16, 32>(
                p, nu, nu, [&](int a, int k) { return Dn[a * lda + idx[k]] + X[a * lda + k]; },
                [&](int k, int c) { return Pu[c * lda + k]; },
                [&](int a, int c) { return -2.f * Bc[a * lda + c]; },
                [&](int a, int c, float w) {
                    part += (double)(X[a * lda + c] - Dn[a * lda + idx[c]]) * (double)w;
                });
        }
        if (!blocked) {
            for (int a = warp; a < p; a += nw)
                for (int c = lane; c < nu; c += 32) {
                    float w = -2.f * Bc[a * lda + c];
                    const float* prow = Pu + c * lda;
#pragma unroll 4
                    for (int k = 0; k < nu; ++k) w = fmaf(prow[k], Dn[a * lda + idx[k]] + X[a * lda + k], w);
                    part += (double)(X[a * lda + c] - Dn[a * lda + idx[c]]) * (double)w;
                }
        }
        // 4. column norms of D*
        for (int c = tid; c < nu; c += nth) {
            float ss = 0.f;
            for (int a = 0; a < p; ++a) ss = fmaf(X[a * lda + c], X[a * lda + c], ss);
            const float nr = sqrtf(ss);
            nrm[c] = nr;
            if (!(nr > 0.f) || !isfinite(nr)) s_fail = SDL_ERR_SINGULAR;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    const bool ok = (s_fail == 0);
    for (int i = tid; i < n; i += nth) norms[i] = 1.f;
    __syncthreads();
    if (ok) {
        for (int c = tid; c < nu; c += nth) norms[idx[c]] = nrm[c];
        for (int c = warp; c < nu; c += nw)
            for (int a = lane; a < p; a += 32) {
                const float v = X[a * lda + c] / nrm[c];
                Dn[a * lda + idx[c]] = v;
                D[a + p * idx[c]] = v;
            }
        __syncthreads();
        if (G_out) {
            for (int i = warp; i < n; i += nw)
                for (int j = lane; j < n; j += 32) {
                    float g = 0.f;
                    for (int a = 0; a < p; ++a) g = fmaf(Dn[a * lda + i], Dn[a * lda + j], g);
                    G_out[i * n + j] = g;
                }
        }
    }
    if (tid == 0) {
        double change = 0.0;
        for (int w = 0; w < nth / 32; ++w) change += s_red[w];
        if (!ok) record_error(err, s_fail);
        const double before = red_d[0];
        const double after = ok ? before + change : before;
        if (objective_out) {
            objective_out[0] = before;
            objective_out[1] = after;
        }
        if (rmse_out) rmse_out[0] = sqrt(fmax(after, 0.0) * inv_count);
    }
}

template <bool kLarge>
__global__ void __launch_bounds__(kSolveThreads)
    solve_kernel(const float* __restrict__ red_f, const double* __restrict__ red_d, float* D, int p,
                 int n, float* __restrict__ norms, double inv_count, double* objective_out,
                 double* rmse_out, int* err, float* G_out, int keep_p) {
    solve_body<kLarge>(red_f, red_d, D, p, n, norms, inv_count, objective_out, rmse_out, err,
                       G_out, keep_p);
}

// One CTA per problem.
template <bool kLarge>
__global__ void __launch_bounds__(kSolveThreads) solve_multi_kernel(const SolveDesc* __restrict__ d,
                                                                    int* err) {
    const SolveDesc q = d[blockIdx.x];
    solve_body<kLarge>(q.red_f, q.red_d, q.D, q.p, q.n, q.norms, q.inv_count, q.objective_out, q.rmse_out,
               err, q.G_out, q.keep_p);
}

// FP64 version of solve_kernel (precision extension): the same steps with
// the normal matrix, its inverse, D*, the objective change and the column
// norms in double precision (inputs are the FP32 partial sums).
constexpr int kSolve64Threads = 512;
// FP64 elimination of the FP32 normal matrix: a pivot is rejected only when
// it is at the level of the FP64 rounding of the diagonal (the FP32 solve
// rejects at 1e-7, its own rounding level)
constexpr double kSolvePivotRel64 = 1e-12;

__global__ void __launch_bounds__(kSolve64Threads)
    solve64_kernel(const float* __restrict__ red_f, const double* __restrict__ red_d, float* D,
                   int p, int n, float* __restrict__ norms, double inv_count,
                   double* objective_out, double* rmse_out, int* err, float* G_out) {
    extern __shared__ __align__(16) double smd[];
    const int lda = n | 1;
    double* A = smd;                        // nu x nu (stride lda)
    double* X = A + (size_t)n * lda;        // p x nu right-hand sides -> D* rows
    double* tmp = X + (size_t)p * lda;      // one row per warp
    double* d0 = tmp + (size_t)(kSolve64Threads / 32) * lda;
    double* nrm = d0 + n;
    int* idx = reinterpret_cast<int*>(nrm + n);
    __shared__ int s_nu, s_fail;
    __shared__ double s_red[kSolve64Threads / 32];
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = nth >> 5;
    const float* P = red_f;
    const float* B = red_f + n * n;
    if (tid < 32) {
        int base = 0, fail = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const float dl = (i < n) ? P[i * n + i] : 0.f;
            if (i < n && !isfinite(dl)) fail = SDL_ERR_NONFINITE;
            const unsigned um = __ballot_sync(0xffffffffu, i < n && dl > 0.f);
            if (i < n && dl > 0.f) {
                const int pos = base + __popc(um & ((1u << lane) - 1u));
                idx[pos] = i;
                d0[pos] = dl;
            }
            base += __popc(um);
        }
        fail = __reduce_or_sync(0xffffffffu, fail);
        if (lane == 0) {
            s_nu = base;
            s_fail = fail;
        }
    }
    __syncthreads();
    const int nu = s_nu;
    for (int e = tid; e < nu * nu; e += nth) {
        const int r = e / nu, c = e - r * nu;
        A[r * lda + c] = (double)P[idx[r] * n + idx[c]];
    }
    for (int e = tid; e < p * nu; e += nth) {
        const int r = e / nu, c = e - r * nu;
        X[r * lda + c] = (double)B[r * n + idx[c]];
    }
    __syncthreads();
    for (int k = 0; k < nu && s_fail == 0; ++k) {
        const double piv = A[k * lda + k];
        if (!(piv > kSolvePivotRel64 * d0[k])) {
            __syncthreads();
            if (tid == 0) s_fail = SDL_ERR_SINGULAR;
            __syncthreads();
            break;
        }
        const double inv = 1.0 / piv;
        for (int e = tid; e < nu * nu; e += nth) {
            const int i = e / nu, j = e - i * nu;
            if (i != k && j != k) A[i * lda + j] -= A[i * lda + k] * inv * A[k * lda + j];
        }
        __syncthreads();
        for (int e = tid; e < 2 * nu; e += nth) {
            if (e < nu) {
                if (e != k) A[k * lda + e] *= inv;
            } else if (e - nu != k) {
                A[(e - nu) * lda + k] *= -inv;
            }
        }
        if (tid == 0) A[k * lda + k] = inv;
        __syncthreads();
    }
    const bool ok_inv = s_fail == 0;
    double part = 0.0;
    if (ok_inv) {
        // D* rows: X[a, :] <- X[a, :] A^{-1}, one warp per row through a copy
        for (int a = warp; a < p; a += nw) {
            double* t = tmp + warp * lda;
            for (int c = lane; c < nu; c += 32) t[c] = X[a * lda + c];
            __syncwarp();
            for (int c = lane; c < nu; c += 32) {
                double x = 0.0;
                for (int k = 0; k < nu; ++k) x += t[k] * A[k * lda + c];
                X[a * lda + c] = x;
            }
            __syncwarp();
        }
        __syncthreads();
        // objective change (as in solve_body), P, B and D_old read back in FP32
        for (int e = tid; e < p * nu; e += nth) {
            const int a = e / nu, c = e - a * nu;
            double w = -2.0 * (double)B[a * n + idx[c]];
            const float* prow = P + (size_t)idx[c] * n;
            for (int k = 0; k < nu; ++k)
                w += (double)prow[idx[k]] * ((double)D[a + p * idx[k]] + X[a * lda + k]);
            part += w * (X[a * lda + c] - (double)D[a + p * idx[c]]);
        }
        for (int c = tid; c < nu; c += nth) {
            double ss = 0.0;
            for (int a = 0; a < p; ++a) ss += X[a * lda + c] * X[a * lda + c];
            nrm[c] = sqrt(ss);
            if (!(nrm[c] > 0.0) || !isfinite(nrm[c])) s_fail = SDL_ERR_SINGULAR;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    const bool ok = s_fail == 0;
    for (int i = tid; i < n; i += nth) norms[i] = 1.f;
    __syncthreads();
    if (ok) {
        for (int c = tid; c < nu; c += nth) norms[idx[c]] = (float)nrm[c];
        for (int e = tid; e < p * nu; e += nth) {
            const int a = e / nu, c = e - a * nu;
            D[a + p * idx[c]] = (float)(X[a * lda + c] / nrm[c]);
        }
        __syncthreads();
        if (G_out) {
            for (int e = tid; e < n * n; e += nth) {
                const int i = e / n, j = e - i * n;
                float g = 0.f;
                for (int a = 0; a < p; ++a) g = fmaf(D[a + p * i], D[a + p * j], g);
                G_out[e] = g;
            }
        }
    }
    if (tid == 0) {
        double change = 0.0;
        for (int w = 0; w < nw; ++w) change += s_red[w];
        if (!ok) record_error(err, s_fail);
        const double before = red_d[0];
        const double after = ok ? before + change : before;
        if (objective_out) {
            objective_out[0] = before;
            objective_out[1] = after;
        }
        if (rmse_out) rmse_out[0] = sqrt(fmax(after, 0.0) * inv_count);
    }
}

// X <- W^{-1} X: slot l of every code times the norm of its D1 atom (side 1,
// Corollary 1) or D2 atom (side 2, Result 1).  The norms are staged in shared
// memory; with 16-byte aligned arrays a thread takes four slots at a time.
constexpr int kRescaleMaxN = 128;

__device__ __forceinline__ float rescale_one(int q, float x, int n1, int nq, bool d1,
                                             const float* sn) {
    if (q < 0 || q >= nq) return x;
    return x * sn[d1 ? q % n1 : q / n1];
}

__device__ __forceinline__ void rescale_body(const int32_t* __restrict__ support,
                                             float* __restrict__ coef, long long count, int n1,
                                             int n2, int side, const float* __restrict__ norms,
                                             long long first, long long step) {
    __shared__ float sn_s[kRescaleMaxN];
    const bool d1 = side == kSideD1;
    const int n = d1 ? n1 : n2;
    const bool staged = n <= kRescaleMaxN;
    if (staged)
        for (int a = threadIdx.x; a < n; a += blockDim.x) sn_s[a] = norms[a];
    __syncthreads();
    const float* sn = staged ? sn_s : norms;
    const int nq = n1 * n2;
    const bool vec = ((reinterpret_cast<uintptr_t>(support) | reinterpret_cast<uintptr_t>(coef)) & 15u) == 0;
    long long done = 0;
    if (vec) {
        const long long n4 = count / 4;
        const int4* s4 = reinterpret_cast<const int4*>(support);
        float4* c4 = reinterpret_cast<float4*>(coef);
        for (long long g = first; g < n4; g += step) {
            const int4 q = s4[g];
            float4 x = c4[g];
            x.x = rescale_one(q.x, x.x, n1, nq, d1, sn);
            x.y = rescale_one(q.y, x.y, n1, nq, d1, sn);
            x.z = rescale_one(q.z, x.z, n1, nq, d1, sn);
            x.w = rescale_one(q.w, x.w, n1, nq, d1, sn);
            c4[g] = x;
        }
        done = n4 * 4;
    }
    for (long long e = done + first; e < count; e += step) coef[e] = rescale_one(support[e], coef[e], n1, nq, d1, sn);
}

__global__ void rescale_kernel(const int32_t* __restrict__ support, float* __restrict__ coef,
                               long long count, int n1, int n2, int side,
                               const float* __restrict__ norms) {
    rescale_body(support, coef, count, n1, n2, side, norms,
                 blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// Code rescale of several problems: blockIdx.y = problem.
__global__ void rescale_multi_kernel(const RescaleDesc* __restrict__ d) {
    const RescaleDesc q = d[blockIdx.y];
    rescale_body(q.support, q.coef, q.count, q.n1, q.n2, q.side, q.norms,
                 blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

}  // namespace

size_t solve_smem_bytes(int p, int n, int* keep_p) {
    const size_t lda = (size_t)(n | 1);
    // A, the two pivot row | column buffers, B, D*, D and the n-vectors
    const size_t base = (size_t)n * lda + 4 * (size_t)n + 3 * (size_t)p * lda + 3 * (size_t)n;
    const size_t limit = 200 * 1024 / sizeof(float);
    // a kept copy of P for the objective term when it fits
    const int keep = base + (size_t)n * lda <= limit ? 1 : 0;
    if (keep_p) *keep_p = keep;
    return sizeof(float) * (base + (keep ? (size_t)n * lda : 0));
}

int launch_multi_update_kernels(int which, const void* d_desc, int G, int blocks, size_t smem,
                                int* err, cudaStream_t st) {
    switch (which) {
        case 0:
            gram_multi_kernel<<<blocks, 256, 0, st>>>(static_cast<const GramDesc*>(d_desc), G);
            break;
        case 1:
            reduce_multi_kernel<<<blocks, kReduceWarps * 32, 0, st>>>(
                static_cast<const ReduceDesc*>(d_desc), G);
            break;
        case 2:
        case 4: {
            // 4: some problem has n > 32
            auto kern = which == 4 ? solve_multi_kernel<true> : solve_multi_kernel<false>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return SDL_ERR_CUDA;
            kern<<<G, which == 4 ? kSolveThreads : kSolveThreadsSmall, smem, st>>>(
                static_cast<const SolveDesc*>(d_desc), err);
            break;
        }
        case 3:
            rescale_multi_kernel<<<dim3(std::max(1, blocks), G), 256, 0, st>>>(
                static_cast<const RescaleDesc*>(d_desc));
            break;
        default: return SDL_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

void launch_gram(const float* D, int p, int n, float* G, cudaStream_t st) {
    const int threads = 256;
    gram_kernel<<<(n * n + threads - 1) / threads, threads, 0, st>>>(D, p, n, G);
}

void launch_gram2(const float* D1, int p1, int n1, float* G1, const float* D2, int p2, int n2,
                  float* G2, cudaStream_t st) {
    const int threads = 256;
    const int b1 = (n1 * n1 + threads - 1) / threads, b2 = (n2 * n2 + threads - 1) / threads;
    gram2_kernel<<<b1 + b2, threads, 0, st>>>(D1, p1, n1, G1, b1, D2, p2, n2, G2);
}

void launch_reduce_partials(const float* part_f, const double* part_d, int n_slots, int nf,
                            float* red_f, double* red_d, cudaStream_t st) {
    const int blocks = std::max(1, (nf + 31) / 32);
    reduce_partials_kernel<<<blocks, kReduceWarps * 32, 0, st>>>(part_f, part_d, n_slots, nf,
                                                                 red_f, red_d);
}

int launch_solve64(const float* red_f, const double* red_d, float* D, int p, int n, float* norms,
                   double inv_count, double* objective_out, double* rmse_out, int* err,
                   cudaStream_t st, float* G_out) {
    const size_t lda = (size_t)(n | 1);
    const size_t bytes = sizeof(double) * ((size_t)n * lda + (size_t)p * lda +
                                           (size_t)(kSolve64Threads / 32) * lda + 2 * (size_t)n) +
                         sizeof(int) * (size_t)n;
    if (bytes > 227 * 1024) return SDL_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(solve64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return SDL_ERR_CUDA;
    solve64_kernel<<<1, kSolve64Threads, bytes, st>>>(red_f, red_d, D, p, n, norms, inv_count,
                                                      objective_out, rmse_out, err, G_out);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

int launch_solve(const float* red_f, const double* red_d, float* D, int p, int n, float* norms,
                 double inv_count, double* objective_out, double* rmse_out, int* err,
                 cudaStream_t st, float* G_out) {
    // keep a copy of P in shared memory for the objective term when it fits
    int keep_p = 0;
    const size_t bytes = solve_smem_bytes(p, n, &keep_p);
    auto kern = n > 32 ? solve_kernel<true> : solve_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return SDL_ERR_CUDA;
    kern<<<1, n > 32 ? kSolveThreads : kSolveThreadsSmall, bytes, st>>>(red_f, red_d, D, p, n, norms, inv_count, objective_out,
                                            rmse_out, err, G_out, keep_p);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

void launch_rescale(const int32_t* support, float* coef, long long count, int n1, int n2,
                    int side, const float* norms, cudaStream_t st) {
    if (count <= 0) return;
    const int threads = 256;
    const long long blocks = std::min<long long>((count / 4 + threads - 1) / threads + 1, 152 * 16);
    rescale_kernel<<<(int)blocks, threads, 0, st>>>(support, coef, count, n1, n2, side, norms);
}

}  // namespace sdl
