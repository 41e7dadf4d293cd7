// Three-mode generalisation (Remark 3): signals Y_k (p1 x p2 x p3, column-order
// vec, first index fastest), dictionaries D1 (p1 x n1), D2 (p2 x n2), D3
// (p3 x n3), sparse cores over atom triples q = i + n1 j + n1 n2 l (the column
// of D3 (x) D2 (x) D1).
//
//   code3_kernel<MODE>  one warp per signal: C0 = Y x_1 D1^T x_2 D2^T x_3 D3^T
//                       by three mode contractions in shared memory, greedy
//                       pursuit over triples in the Gram domain
//                       (C = C0 - sum_m x_m G1[:, i_m] o G2[:, j_m] o G3[:, l_m]),
//                       the Cholesky re-fit kept by lane 0 in shared memory, and
//                       for MODE k the partial sums of the mode-k update
//                       (Remark 3 -> Corollary 1):
//                         P_k[u_m, u_m'] += x_m x_m' prod_{other modes} G[.., ..]
//                         B_k[:, u_m]    += x_m (Y contracted with the other two atoms)
//                       in warp-private accumulators combined in warp order;
//   rescale3_kernel     the coefficients of every pick times the norm of its
//                       mode-k atom (X <- X W_k^{-1}).
// The reduction and the normal-equation solve are the two-mode kernels.  Shapes
// compiled in tmod3_fast.cu take the specialised coder instead.
#include <algorithm>
#include <cmath>

#include "ctx.cuh"

using namespace sdl;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxP3 = 16;          // each p_k <= 16
constexpr int kMaxQ3 = 1024;        // n1 n2 n3 <= 1024
constexpr int kMaxS3 = 16;
constexpr int kMaxWarps3 = 4;
constexpr size_t kMaxSmem3 = 200 * 1024;

__host__ __device__ constexpr int a4(int x) { return (x + 3) & ~3; }

struct Shape3 {
    int p1, p2, p3, n1, n2, n3;
    __host__ __device__ int P() const { return p1 * p2 * p3; }
    __host__ __device__ int Q() const { return n1 * n2 * n3; }
    __host__ __device__ int nf(int mode) const {
        const int n = mode == 1 ? n1 : mode == 2 ? n2 : n3;
        const int p = mode == 1 ? p1 : mode == 2 ? p2 : p3;
        return mode == 0 ? 0 : n * n + p * n;
    }
};

// shared memory (floats): D1 | D2 | D3 (column-major) | G1 | G2 | G3 | per warp:
// Y | W1 (n1 p2 p3) | W2 (n1 n2 p3) | C0 (Q) | L (s x s) | y (s) | x (s) | q (s) |
// acc (nf) | misc (4)
struct Layout3 {
    int d1, d2, d3, g1, g2, g3, warp0, y, w1, w2, c0, L, yv, x, q, acc, misc, wstride, total;
    __host__ __device__ Layout3(const Shape3& h, int s, int nf, int wpc) {
        d1 = 0;
        d2 = d1 + a4(h.p1 * h.n1);
        d3 = d2 + a4(h.p2 * h.n2);
        g1 = d3 + a4(h.p3 * h.n3);
        g2 = g1 + a4(h.n1 * h.n1);
        g3 = g2 + a4(h.n2 * h.n2);
        warp0 = g3 + a4(h.n3 * h.n3);
        y = 0;
        w1 = y + a4(h.P());
        w2 = w1 + a4(h.n1 * h.p2 * h.p3);
        c0 = w2 + a4(h.n1 * h.n2 * h.p3);
        L = c0 + a4(h.Q());
        yv = L + a4(s * s);
        x = yv + a4(s);
        q = x + a4(s);
        acc = q + a4(s);
        misc = acc + a4(nf);
        wstride = misc + 4;
        total = warp0 + wpc * wstride;
    }
};

template <int MODE>
__global__ void __launch_bounds__(kMaxWarps3 * 32)
    code3_kernel(const float* __restrict__ Y, Shape3 h, long long N, const float* __restrict__ D1,
                 const float* __restrict__ D2, const float* __restrict__ D3,
                 const float* __restrict__ G1, const float* __restrict__ G2,
                 const float* __restrict__ G3, int s, int32_t* __restrict__ support,
                 float* __restrict__ coef, int32_t* __restrict__ nnz,
                 float* __restrict__ res_energy, float* __restrict__ part_f,
                 double* __restrict__ part_d, int* err) {
    extern __shared__ __align__(16) float sm[];
    const int wpc = blockDim.x >> 5;
    const int nf = h.nf(MODE);
    const Layout3 L(h, s, nf, wpc);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p1 = h.p1, p2 = h.p2, p3 = h.p3, n1 = h.n1, n2 = h.n2, n3 = h.n3;
    const int P = h.P(), Q = h.Q(), n12 = n1 * n2;
    float* sD1 = sm + L.d1;
    float* sD2 = sm + L.d2;
    float* sD3 = sm + L.d3;
    float* sG1 = sm + L.g1;
    float* sG2 = sm + L.g2;
    float* sG3 = sm + L.g3;
    float* wb = sm + L.warp0 + w * L.wstride;
    float* Ys = wb + L.y;
    float* W1 = wb + L.w1;    // [i + n1 (b + p2 c)]
    float* W2 = wb + L.w2;    // [i + n1 (j + n2 c)]
    float* C0 = wb + L.c0;    // [q], picked entries masked with NaN
    float* Ls = wb + L.L;     // row-major s x s Cholesky factor
    float* yv = wb + L.yv;    // forward-substitution values y = L^{-1} b
    float* xs = wb + L.x;     // coefficients of the current fit
    int* qs = reinterpret_cast<int*>(wb + L.q);
    float* acc = wb + L.acc;  // [P_k (n x n) | B_k (p x n)]
    for (int e = threadIdx.x; e < p1 * n1; e += blockDim.x) sD1[e] = D1[e];
    for (int e = threadIdx.x; e < p2 * n2; e += blockDim.x) sD2[e] = D2[e];
    for (int e = threadIdx.x; e < p3 * n3; e += blockDim.x) sD3[e] = D3[e];
    for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) sG1[e] = G1[e];
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) sG2[e] = G2[e];
    for (int e = threadIdx.x; e < n3 * n3; e += blockDim.x) sG3[e] = G3[e];
    for (int e = lane; e < nf; e += 32) acc[e] = 0.f;
    __syncthreads();

    double e_res = 0.0, e_y = 0.0;   // lane 0: this warp's sums
    const long long stride = (long long)gridDim.x * wpc;
    for (long long k = (long long)blockIdx.x * wpc + w; k < N; k += stride) {
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
        float E2 = ss;   // residual energy ||Y||^2 - ||y||^2 (lane 0's copy is used)
        if (finite) {
            // ---- C0 by three mode contractions
            for (int e = lane; e < n1 * p2 * p3; e += 32) {
                const int i = e % n1, bc = e / n1;
                float t = 0.f;
                for (int a = 0; a < p1; ++a) t = fmaf(sD1[a + p1 * i], Ys[a + p1 * bc], t);
                W1[e] = t;
            }
            __syncwarp();
            for (int e = lane; e < n12 * p3; e += 32) {
                const int i = e % n1, j = (e / n1) % n2, c = e / n12;
                float t = 0.f;
                for (int b = 0; b < p2; ++b) t = fmaf(sD2[b + p2 * j], W1[i + n1 * (b + p2 * c)], t);
                W2[e] = t;
            }
            __syncwarp();
            for (int q = lane; q < Q; q += 32) {
                const int ij = q % n12, l = q / n12;
                float t = 0.f;
                for (int c = 0; c < p3; ++c) t = fmaf(sD3[c + p3 * l], W2[ij + n12 * c], t);
                C0[q] = t;
            }
            __syncwarp();
            // ---- greedy steps
            for (int t = 0; t < s; ++t) {
                float best = 0.f;
                int bq = 0x7fffffff;
                for (int q = lane; q < Q; q += 32) {          // increasing q per lane
                    const int i = q % n1, j = (q / n1) % n2, l = q / n12;
                    float v = C0[q];
                    for (int m = 0; m < t; ++m) {
                        const int qm = qs[m];
                        const int im = qm % n1, jm = (qm / n1) % n2, lm = qm / n12;
                        v = fmaf(-xs[m] * sG1[i * n1 + im], sG2[j * n2 + jm] * sG3[l * n3 + lm], v);
                    }
                    v = fabsf(v);                              // NaN (picked) never wins
                    if (v > best) { best = v; bq = q; }
                }
                const unsigned Mx = __reduce_max_sync(kFull, __float_as_uint(best));
                if (Mx == 0u) break;                           // every remaining score is 0
                const unsigned cand = (__float_as_uint(best) == Mx) ? (unsigned)bq : 0xffffffffu;
                const int qt = (int)__reduce_min_sync(kFull, cand);
                int ok = 0;
                if (lane == 0) {
                    const float b = C0[qt];
                    C0[qt] = __int_as_float(0x7fc00000);
                    const int it = qt % n1, jt = (qt / n1) % n2, lt = qt / n12;
                    // row t of the Cholesky factor: w = L^{-1} a, a_m = A[t, m]
                    float ww = 0.f;
                    for (int m = 0; m < t; ++m) {
                        const int qm = qs[m];
                        const int im = qm % n1, jm = (qm / n1) % n2, lm = qm / n12;
                        float a = sG1[it * n1 + im] * sG2[jt * n2 + jm] * sG3[lt * n3 + lm];
                        for (int m2 = 0; m2 < m; ++m2) a = fmaf(-Ls[m * s + m2], Ls[t * s + m2], a);
                        const float wm = a / Ls[m * s + m];
                        Ls[t * s + m] = wm;
                        ww = fmaf(wm, wm, ww);
                    }
                    const float Att = sG1[it * n1 + it] * sG2[jt * n2 + jt] * sG3[lt * n3 + lt];
                    const float d = Att - ww;
                    if (d > kPivotRel * Att) {
                        ok = 1;
                        const float Ltt = sqrtf(d);
                        Ls[t * s + t] = Ltt;
                        float wy = 0.f;
                        for (int m = 0; m < t; ++m) wy = fmaf(Ls[t * s + m], yv[m], wy);
                        const float ytv = (b - wy) / Ltt;
                        yv[t] = ytv;
                        qs[t] = qt;
                        // x = L^{-T} y over the t + 1 picks
                        for (int r = t; r >= 0; --r) {
                            float v = yv[r];
                            for (int m = r + 1; m <= t; ++m) v = fmaf(-Ls[m * s + r], xs[m], v);
                            xs[r] = v / Ls[r * s + r];
                        }
                        E2 = fmaf(-ytv, ytv, E2);
                    }
                }
                ok = __shfl_sync(kFull, ok, 0);
                __syncwarp();
                if (!ok) break;
                cnt = t + 1;
            }
        }
        // ---- emit the code
        if (support && lane < s) {
            support[(size_t)k * s + lane] = lane < cnt ? qs[lane] : -1;
            coef[(size_t)k * s + lane] = lane < cnt ? xs[lane] : 0.f;
        }
        if (lane == 0) {
            if (nnz) nnz[k] = cnt;
            if (res_energy) res_energy[k] = finite ? fmaxf(E2, 0.f) : __int_as_float(0x7fc00000);
            if (!finite) record_error(err, SDL_ERR_NONFINITE);
            if (finite) {
                e_res += (double)fmaxf(E2, 0.f);
                e_y += (double)ss;
            }
        }
        // ---- partial sums of the mode-k update
        if constexpr (MODE != 0) {
            const int nk = MODE == 1 ? n1 : MODE == 2 ? n2 : n3;
            float* accP = acc;
            float* accB = acc + nk * nk;
            // P_k: pairs (m, m') over the lanes
            for (int e = lane; e < cnt * cnt; e += 32) {
                const int m = e / cnt, m2 = e - m * cnt;
                const int qa = qs[m], qb = qs[m2];
                const int ia = qa % n1, ja = (qa / n1) % n2, la = qa / n12;
                const int ib = qb % n1, jb = (qb / n1) % n2, lb = qb / n12;
                float f = xs[m] * xs[m2];
                int u, v;
                if (MODE == 1) {
                    f *= sG2[ja * n2 + jb] * sG3[la * n3 + lb];
                    u = ia;
                    v = ib;
                } else if (MODE == 2) {
                    f *= sG1[ia * n1 + ib] * sG3[la * n3 + lb];
                    u = ja;
                    v = jb;
                } else {
                    f *= sG1[ia * n1 + ib] * sG2[ja * n2 + jb];
                    u = la;
                    v = lb;
                }
                atomicAdd(&accP[u * nk + v], f);
            }
            // B_k: one pick at a time, lanes over the rows of mode k
            for (int m = 0; m < cnt; ++m) {
                const int qm = qs[m];
                const int im = qm % n1, jm = (qm / n1) % n2, lm = qm / n12;
                const float xm = xs[m];
                if (MODE == 1) {
                    for (int a = lane; a < p1; a += 32) {
                        float t = 0.f;
                        for (int c = 0; c < p3; ++c) {
                            float u = 0.f;
                            for (int b = 0; b < p2; ++b) u = fmaf(Ys[a + p1 * (b + p2 * c)], sD2[b + p2 * jm], u);
                            t = fmaf(u, sD3[c + p3 * lm], t);
                        }
                        accB[a * nk + im] = fmaf(xm, t, accB[a * nk + im]);
                    }
                } else if (MODE == 2) {
                    for (int b = lane; b < p2; b += 32) {
                        float t = 0.f;
                        for (int c = 0; c < p3; ++c) {
                            float u = 0.f;
                            for (int a = 0; a < p1; ++a) u = fmaf(Ys[a + p1 * (b + p2 * c)], sD1[a + p1 * im], u);
                            t = fmaf(u, sD3[c + p3 * lm], t);
                        }
                        accB[b * nk + jm] = fmaf(xm, t, accB[b * nk + jm]);
                    }
                } else {
                    for (int c = lane; c < p3; c += 32) {
                        float t = 0.f;
                        for (int b = 0; b < p2; ++b) {
                            float u = 0.f;
                            for (int a = 0; a < p1; ++a) u = fmaf(Ys[a + p1 * (b + p2 * c)], sD1[a + p1 * im], u);
                            t = fmaf(u, sD2[b + p2 * jm], t);
                        }
                        accB[c * nk + lm] = fmaf(xm, t, accB[c * nk + lm]);
                    }
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
    if constexpr (MODE != 0) {
        double* ed = reinterpret_cast<double*>(wb + L.misc);   // 16-byte aligned (a4 offsets)
        if (lane == 0) {
            ed[0] = e_res;
            ed[1] = e_y;
        }
        __syncthreads();
        float* dst = part_f + (size_t)blockIdx.x * nf;
        for (int e = threadIdx.x; e < nf; e += blockDim.x) {
            float v = 0.f;
            for (int ww = 0; ww < wpc; ++ww) v += sm[L.warp0 + ww * L.wstride + L.acc + e];
            dst[e] = v;
        }
        if (threadIdx.x < 2) {
            double d = 0.0;
            for (int ww = 0; ww < wpc; ++ww)
                d += reinterpret_cast<const double*>(sm + L.warp0 + ww * L.wstride + L.misc)[threadIdx.x];
            part_d[(size_t)blockIdx.x * 2 + threadIdx.x] = d;
        }
    }
}

__global__ void rescale3_kernel(const int32_t* __restrict__ support, float* __restrict__ coef,
                                long long count, int n1, int n2, int mode,
                                const float* __restrict__ norms) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = support[e];
        if (q < 0) continue;
        const int atom = mode == 1 ? q % n1 : mode == 2 ? (q / n1) % n2 : q / (n1 * n2);
        coef[e] *= norms[atom];
    }
}

size_t smem3(const Shape3& h, int s, int mode, int wpc) {
    return sizeof(float) * (size_t)Layout3(h, s, h.nf(mode), wpc).total;
}

int launch_code3(int mode, const float* Y, const Shape3& h, long long N, const float* D1,
                 const float* D2, const float* D3, const float* G1, const float* G2,
                 const float* G3, int s, int32_t* support, float* coef, int32_t* nnz, float* res,
                 float* part_f, double* part_d, int max_slots, int* err, int num_sms,
                 cudaStream_t st) {
    const int rf = launch_code3_fast(mode, Y, h.p1, h.p2, h.p3, h.n1, h.n2, h.n3, N, D1, D2, D3, G1,
                                     G2, G3, s, support, coef, nnz, res, part_f, part_d, max_slots,
                                     err, num_sms, st);
    if (rf != SDL_ERR_UNSUPPORTED) return rf;
    int wpc = kMaxWarps3;
    while (wpc > 1 && smem3(h, s, mode, wpc) > kMaxSmem3) --wpc;
    const size_t bytes = smem3(h, s, mode, wpc);
    if (bytes > kMaxSmem3) return SDL_ERR_UNSUPPORTED;
    auto launch = [&](auto kern) -> int {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess)
            return SDL_ERR_CUDA;
        int bps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, wpc * 32, bytes) != cudaSuccess)
            return SDL_ERR_CUDA;
        bps = std::max(1, std::min(bps, 8));
        const long long need = (N + wpc - 1) / wpc;
        long long grid = std::max<long long>(1, std::min<long long>(need, (long long)num_sms * bps));
        if (mode != 0) grid = std::min<long long>(grid, max_slots);
        kern<<<(int)grid, wpc * 32, bytes, st>>>(Y, h, N, D1, D2, D3, G1, G2, G3, s, support, coef,
                                                 nnz, res, part_f, part_d, err);
        if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
        return mode == 0 ? 0 : (int)grid;
    };
    switch (mode) {
        case 0: return launch(code3_kernel<0>);
        case 1: return launch(code3_kernel<1>);
        case 2: return launch(code3_kernel<2>);
        default: return launch(code3_kernel<3>);
    }
}

bool shape3_ok(const Shape3& h, int s) {
    const int ps[3] = {h.p1, h.p2, h.p3}, ns[3] = {h.n1, h.n2, h.n3};
    for (int k = 0; k < 3; ++k)
        if (ps[k] < 1 || ps[k] > kMaxP3 || ns[k] < 1 || ns[k] > kMaxQ3) return false;
    return h.Q() <= kMaxQ3 && h.P() <= 1024 && s >= 1 && s <= kMaxS3 && s <= h.P() && s <= h.Q();
}

// G buffer of the context: G1 (n1^2) | G2 (n2^2) | G3 (n3^2) | spare (n3^2)
int grams3(sdl_ctx* c, const float* D1, int p1, int n1, const float* D2, int p2, int n2,
           const float* D3, int p3, int n3, float** G1, float** G2, float** G3, cudaStream_t st) {
    const size_t need = (size_t)n1 * n1 + (size_t)n2 * n2 + 2 * (size_t)n3 * n3;
    if (need > c->cap_g3) {
        if (c->G3) cudaFree(c->G3);
        c->G3 = nullptr;
        c->cap_g3 = 0;
        if (cudaMalloc(&c->G3, need * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return SDL_ERR_WORKSPACE;
        }
        c->cap_g3 = need;
    }
    *G1 = c->G3;
    *G2 = *G1 + (size_t)n1 * n1;
    *G3 = *G2 + (size_t)n2 * n2;
    Trace tr(c, kGram, st);
    launch_gram2(D1, p1, n1, *G1, D2, p2, n2, *G2, st);
    launch_gram2(D3, p3, n3, *G3, D3, p3, n3, *G3 + (size_t)n3 * n3, st);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int sdl_sparse_code3(sdl_ctx* c, const float* Y, int p1, int p2, int p3, int64_t N,
                     const float* D1, int n1, const float* D2, int n2, const float* D3, int n3,
                     int s, int32_t* support, float* coef, int32_t* nnz, float* res_energy,
                     void* stream) {
    const Shape3 h{p1, p2, p3, n1, n2, n3};
    if (!c || N < 0 || !shape3_ok(h, s)) return SDL_ERR_ARG;
    if (N == 0) return SDL_OK;
    if (!Y || !D1 || !D2 || !D3 || !support || !coef || !nnz) return SDL_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    float *G1, *G2, *G3;
    int rc = grams3(c, D1, p1, n1, D2, p2, n2, D3, p3, n3, &G1, &G2, &G3, st);
    if (rc != SDL_OK) return rc;
    Trace tr(c, kCode, st);
    rc = launch_code3(0, Y, h, N, D1, D2, D3, G1, G2, G3, s, support, coef, nnz, res_energy,
                      nullptr, nullptr, 0, c->err, c->num_sms, st);
    return rc < 0 ? rc : SDL_OK;
}

int sdl_iterate3(sdl_ctx* c, const float* Y, int p1, int p2, int p3, int64_t N, float* D1, int n1,
                 float* D2, int n2, float* D3, int n3, int s, int32_t* support, float* coef,
                 int32_t* nnz, double* rmse_out, void* stream) {
    const Shape3 h{p1, p2, p3, n1, n2, n3};
    if (!c || N < 1 || !Y || !D1 || !D2 || !D3 || !support || !coef || !nnz || !shape3_ok(h, s))
        return SDL_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = ctx_workspace(c, p1, p2, n1, n2)) != SDL_OK) return rc;
    if ((rc = ctx_workspace(c, p3, p3, n3, n3)) != SDL_OK) return rc;
    float *G1, *G2, *G3;
    if ((rc = grams3(c, D1, p1, n1, D2, p2, n2, D3, p3, n3, &G1, &G2, &G3, st)) != SDL_OK) return rc;
    const int max_slots = max_partial_slots(c->num_sms);
    const double inv_count = 1.0 / ((double)h.P() * (double)N);
    float* Ds[3] = {D1, D2, D3};
    float* Gs[3] = {G1, G2, G3};
    const int ps[3] = {p1, p2, p3}, ns[3] = {n1, n2, n3};
    for (int mode = 1; mode <= 3; ++mode) {
        int slots;
        {
            Trace tr(c, mode == 1 ? kCodeD1 : kCodeD2, st);
            const bool last = mode == 3;
            slots = launch_code3(mode, Y, h, N, D1, D2, D3, G1, G2, G3, s,
                                 last ? support : nullptr, coef, last ? nnz : nullptr, nullptr,
                                 c->part_f, c->part_d, max_slots, c->err, c->num_sms, st);
        }
        if (slots < 0) return slots;
        const int nfk = h.nf(mode);
        {
            Trace tr(c, kReduce, st);
            launch_reduce_partials(c->part_f, c->part_d, slots, nfk, c->red_f, c->red_d, st);
        }
        Trace tr(c, kSolve, st);
        rc = launch_solve(c->red_f, c->red_d, Ds[mode - 1], ps[mode - 1], ns[mode - 1], c->norms,
                          inv_count, nullptr, rmse_out ? rmse_out + (mode - 1) : nullptr, c->err,
                          st, Gs[mode - 1]);
        if (rc != SDL_OK) return rc;
    }
    {
        Trace tr(c, kRescale, st);
        const long long count = N * (long long)s;
        rescale3_kernel<<<(int)std::min<long long>((count + 255) / 256, 4096), 256, 0, st>>>(
            support, coef, count, n1, n2, 3, c->norms);
    }
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}

}  // extern "C"
