// Tensor-MOD dictionary update: reduction of the per-CTA partial sums, the
// small normal-equation solve with atom normalisation (Corollary 1 for D1,
// Result 1 for D2), the W^{-1} rescale of the codes, and the Gram matrices.
#include <algorithm>
#include <cmath>

#include "sdl_internal.cuh"

namespace sdl {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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
// warp w sums slots w, w+8, w+16, ... (coalesced 128-byte rows), then warp 0
// adds the 8 warp sums in order.
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(kReduceWarps * 32)
    reduce_partials_kernel(const float* __restrict__ part_f, const double* __restrict__ part_d,
                           int n_slots, int nf, float* __restrict__ red_f,
                           double* __restrict__ red_d) {
    __shared__ float ws[kReduceWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float sum = 0.f, comp = 0.f;
    if (e < nf) {
        for (int c = warp; c < n_slots; c += kReduceWarps) {
            const float y = part_f[(size_t)c * nf + e] - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
    }
    ws[warp][lane] = sum - comp;
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
    if (blockIdx.x == 0 && threadIdx.x < 2) {
        double d = 0.0;
        for (int c = 0; c < n_slots; ++c) d += part_d[(size_t)c * 2 + threadIdx.x];
        red_d[threadIdx.x] = d;
    }
}

// Single-warp version of solve_kernel (below) for n <= 32: lane i owns row i
// of the Cholesky factor, lane a owns right-hand side a; only __syncwarp.
// Also writes G = D_new^T D_new (row-major) when G_out != NULL.
__global__ void __launch_bounds__(32)
    solve_small_kernel(const float* __restrict__ red_f, const double* __restrict__ red_d, float* D,
                       int p, int n, float* __restrict__ norms, double inv_count,
                       float* objective_out, float* rmse_out, int* err, float* G_out) {
    extern __shared__ __align__(16) float sm[];
    const int ldb = n | 1;                   // odd strides: lanes hit distinct banks
    float* A = sm;                           // nu x nu (row stride n), becomes L
    float* Bc = A + n * n;                   // p rows of stride ldb: RHS -> D* rows
    float* Dn = Bc + p * ldb;                // p rows of stride ldb: old, then new D
    float* invL = Dn + p * ldb;              // n
    float* nrm = invL + n;                   // n
    int* idx = reinterpret_cast<int*>(nrm + n);   // n
    const int lane = threadIdx.x;
    const float* P = red_f;
    const float* B = red_f + n * n;

    bool bad = false;
    float dl = 0.f;
    if (lane < n) {
        dl = P[lane * n + lane];
        bad = !isfinite(dl);
    }
    const unsigned um = __ballot_sync(kFull, lane < n && dl > 0.f);
    const int nu = __popc(um);
    if (lane < n && dl > 0.f) idx[__popc(um & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    for (int e = lane; e < nu * nu; e += 32) {
        const int r = e / nu, c = e - r * nu;
        const float v = P[idx[r] * n + idx[c]];
        A[r * n + c] = v;
        bad |= !isfinite(v);
    }
    for (int e = lane; e < p * nu; e += 32) {
        const int r = e / nu, c = e - r * nu;
        const float v = B[r * n + idx[c]];
        Bc[r * ldb + c] = v;
        bad |= !isfinite(v);
    }
    for (int e = lane; e < p * n; e += 32) {
        const int r = e % p, c = e / p;
        Dn[r * ldb + c] = D[r + p * c];
    }
    int fail = __any_sync(kFull, bad) ? SDL_ERR_NONFINITE : 0;
    __syncwarp();
    // Cholesky, lane i updates row i
    for (int k = 0; k < nu && !fail; ++k) {
        const float akk = A[k * n + k];
        const float d0 = P[idx[k] * n + idx[k]];
        if (!(akk > kSolvePivotRel * d0)) {
            fail = SDL_ERR_SINGULAR;
            break;
        }
        const float Lkk = sqrtf(akk), inv = 1.f / Lkk;
        __syncwarp();
        if (lane == k) {
            A[k * n + k] = Lkk;
            invL[k] = inv;
        }
        if (lane > k && lane < nu) A[lane * n + k] *= inv;
        __syncwarp();
        if (lane > k && lane < nu) {
            const float lik = A[lane * n + k];
            for (int j = k + 1; j <= lane; ++j) A[lane * n + j] = fmaf(-lik, A[j * n + k], A[lane * n + j]);
        }
        __syncwarp();
    }
    double trace = 0.0;
    if (!fail) {
        float acc = 0.f;
        for (int a = lane; a < p; a += 32) {
            float* row = Bc + a * ldb;
            for (int k = 0; k < nu; ++k) {          // L z = b
                float z = row[k];
                for (int j = 0; j < k; ++j) z = fmaf(-A[k * n + j], row[j], z);
                row[k] = z * invL[k];
            }
            for (int k = nu - 1; k >= 0; --k) {     // L^T x = z
                float x = row[k];
                for (int j = k + 1; j < nu; ++j) x = fmaf(-A[j * n + k], row[j], x);
                row[k] = x * invL[k];
            }
            for (int i = 0; i < nu; ++i) {          // ||L^T delta||^2
                float v = 0.f;
                for (int k = i; k < nu; ++k) v = fmaf(A[k * n + i], Dn[a * ldb + idx[k]] - row[k], v);
                acc = fmaf(v, v, acc);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        trace = (double)acc;
        __syncwarp();
        bool zero = false;
        for (int c = lane; c < nu; c += 32) {
            float ss = 0.f;
            for (int a = 0; a < p; ++a) ss = fmaf(Bc[a * ldb + c], Bc[a * ldb + c], ss);
            nrm[c] = sqrtf(ss);
            zero |= !(nrm[c] > 0.f) || !isfinite(nrm[c]);
        }
        if (__any_sync(kFull, zero)) fail = SDL_ERR_SINGULAR;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) norms[i] = 1.f;
    __syncwarp();
    if (!fail) {
        for (int c = lane; c < nu; c += 32) norms[idx[c]] = nrm[c];
        for (int e = lane; e < p * nu; e += 32) {
            const int a = e / nu, c = e - a * nu;
            const float v = Bc[a * ldb + c] / nrm[c];
            Dn[a * ldb + idx[c]] = v;
            D[a + p * idx[c]] = v;
        }
        __syncwarp();
        if (G_out) {
            for (int e = lane; e < n * n; e += 32) {
                const int i = e / n, j = e - i * n;
                float g = 0.f;
                for (int a = 0; a < p; ++a) g = fmaf(Dn[a * ldb + i], Dn[a * ldb + j], g);
                G_out[e] = g;
            }
        }
    }
    if (lane == 0) {
        if (fail) record_error(err, fail);
        const double before = red_d[0];
        const double after = fail ? before : before - trace;
        if (objective_out) {
            objective_out[0] = (float)before;
            objective_out[1] = (float)after;
        }
        if (rmse_out) rmse_out[0] = (float)sqrt(fmax(after, 0.0) * inv_count);
    }
}

// One CTA: D* = B P^{-1} on the used atoms (diag(P) > 0), unit-norm columns,
// the objective after the update, and the column norms for the code rescale.
//   red_f = [P (n x n, row-major) | B (p x n, row-major)], red_d[0] = objective
//   before the update (sum of residual energies with the old dictionary).
// Objective after = before - tr(Delta P Delta^T), Delta = D_old - D*, which
// is ||L^T delta_a||^2 summed over the rows a (P = L L^T).  On any failure the
// dictionary is left untouched and the norms are set to 1.
constexpr int kSolveThreads = 512;

__global__ void __launch_bounds__(kSolveThreads)
    solve_kernel(const float* __restrict__ red_f, const double* __restrict__ red_d, float* D, int p,
                 int n, float* __restrict__ norms, double inv_count, float* objective_out,
                 float* rmse_out, int* err) {
    extern __shared__ __align__(16) float sm[];
    float* A = sm;                       // nu x nu, becomes L (lower)
    float* Bc = A + n * n;               // p x nu right-hand sides, become D* rows
    float* Dold = Bc + p * n;            // p x n row-major
    float* diag0 = Dold + p * n;         // n
    float* invL = diag0 + n;             // n
    int* idx = reinterpret_cast<int*>(invL + n);   // n
    __shared__ int s_nu, s_fail;
    __shared__ double s_trace;

    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    const float* P = red_f;
    const float* B = red_f + n * n;

    if (tid == 0) {
        int nu = 0, fail = 0;
        for (int i = 0; i < n; ++i) {
            const float d = P[i * n + i];
            if (!isfinite(d)) fail = SDL_ERR_NONFINITE;
            if (d > 0.f) idx[nu++] = i;
        }
        s_nu = nu;
        s_fail = fail;
        s_trace = 0.0;
    }
    __syncthreads();
    const int nu = s_nu;
    for (int e = tid; e < nu * nu; e += nth) {
        const int r = e / nu, c = e - r * nu;
        const float v = P[idx[r] * n + idx[c]];
        A[e] = v;
        if (!isfinite(v)) s_fail = SDL_ERR_NONFINITE;
    }
    for (int e = tid; e < p * nu; e += nth) {
        const int r = e / nu, c = e - r * nu;
        const float v = B[r * n + idx[c]];
        Bc[e] = v;
        if (!isfinite(v)) s_fail = SDL_ERR_NONFINITE;
    }
    for (int e = tid; e < p * n; e += nth) {
        const int r = e / n, c = e - r * n;
        Dold[e] = D[r + p * c];
    }
    for (int c = tid; c < nu; c += nth) diag0[c] = P[idx[c] * n + idx[c]];
    __syncthreads();

    // right-looking Cholesky of the used block
    if (s_fail == 0) {
        for (int k = 0; k < nu; ++k) {
            if (tid == 0) {
                const float piv = A[k * nu + k];
                if (!(piv > kSolvePivotRel * diag0[k])) s_fail = SDL_ERR_SINGULAR;
                const float Lkk = sqrtf(fmaxf(piv, 1e-30f));
                A[k * nu + k] = Lkk;
                invL[k] = 1.f / Lkk;
            }
            __syncthreads();
            const float il = invL[k];
            for (int i = k + 1 + tid; i < nu; i += nth) A[i * nu + k] *= il;
            __syncthreads();
            const int m = nu - k - 1;
            for (int e = tid; e < m * m; e += nth) {
                const int i = k + 1 + e / m, j = k + 1 + e % m;
                if (j <= i) A[i * nu + j] = fmaf(-A[i * nu + k], A[j * nu + k], A[i * nu + j]);
            }
            __syncthreads();
        }
    }
    const bool ok_chol = (s_fail == 0);
    // solve L L^T x = b for every right-hand-side row (one warp per row)
    if (ok_chol) {
        for (int a = warp; a < p; a += nwarps) {
            float* row = Bc + a * nu;
            for (int k = 0; k < nu; ++k) {
                __syncwarp();
                const float zk = row[k] * invL[k];
                __syncwarp();
                if (lane == 0) row[k] = zk;
                for (int i = k + 1 + lane; i < nu; i += 32) row[i] = fmaf(-A[i * nu + k], zk, row[i]);
            }
            for (int k = nu - 1; k >= 0; --k) {
                __syncwarp();
                const float xk = row[k] * invL[k];
                __syncwarp();
                if (lane == 0) row[k] = xk;
                for (int i = lane; i < k; i += 32) row[i] = fmaf(-A[k * nu + i], xk, row[i]);
            }
            __syncwarp();
            // ||L^T delta||^2 with delta = D_old[a, used] - D*[a, :]
            float acc = 0.f;
            for (int i = lane; i < nu; i += 32) {
                float v = 0.f;
                for (int k = i; k < nu; ++k)
                    v = fmaf(A[k * nu + i], Dold[a * n + idx[k]] - row[k], v);
                acc = fmaf(v, v, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (lane == 0) atomicAdd(&s_trace, (double)acc);
        }
    }
    __syncthreads();
    // column norms of D*; a zero or non-finite norm fails the update
    if (ok_chol) {
        for (int c = tid; c < nu; c += nth) {
            float ss = 0.f;
            for (int a = 0; a < p; ++a) ss = fmaf(Bc[a * nu + c], Bc[a * nu + c], ss);
            const float nr = sqrtf(ss);
            diag0[c] = nr;
            if (!(nr > 0.f) || !isfinite(nr)) s_fail = SDL_ERR_SINGULAR;
        }
    }
    __syncthreads();
    const bool ok = (s_fail == 0);
    for (int i = tid; i < n; i += nth) norms[i] = 1.f;
    __syncthreads();
    if (ok) {
        for (int c = tid; c < nu; c += nth) norms[idx[c]] = diag0[c];
        for (int e = tid; e < p * nu; e += nth) {
            const int a = e / nu, c = e - a * nu;
            D[a + p * idx[c]] = Bc[e] / diag0[c];
        }
    }
    if (tid == 0) {
        if (!ok) record_error(err, s_fail);
        const double before = red_d[0];
        const double after = ok ? before - s_trace : before;
        if (objective_out) {
            objective_out[0] = (float)before;
            objective_out[1] = (float)after;
        }
        if (rmse_out) rmse_out[0] = (float)sqrt(fmax(after, 0.0) * inv_count);
    }
}

// X <- W^{-1} X: slot l of every code times the norm of its D1 atom (side 1,
// Corollary 1) or D2 atom (side 2, Result 1).
__global__ void rescale_kernel(const int32_t* __restrict__ support, float* __restrict__ coef,
                               long long count, int n1, int n2, int side,
                               const float* __restrict__ norms) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = support[e];
        if (q < 0 || q >= n1 * n2) continue;
        const int atom = (side == kSideD1) ? q % n1 : q / n1;
        coef[e] *= norms[atom];
    }
}

}  // namespace

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

int launch_solve(const float* red_f, const double* red_d, float* D, int p, int n, float* norms,
                 double inv_count, float* objective_out, float* rmse_out, int* err,
                 cudaStream_t st, float* G_out) {
    if (n <= 32) {
        const int ldb = n | 1;
        const size_t bytes = sizeof(float) * ((size_t)n * n + 2 * (size_t)p * ldb + 3 * (size_t)n);
        if (cudaFuncSetAttribute(solve_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return SDL_ERR_CUDA;
        solve_small_kernel<<<1, 32, bytes, st>>>(red_f, red_d, D, p, n, norms, inv_count,
                                                 objective_out, rmse_out, err, G_out);
        return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
    }
    const size_t bytes = sizeof(float) * ((size_t)n * n + 2 * (size_t)p * n + 3 * (size_t)n);
    if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return SDL_ERR_CUDA;
    solve_kernel<<<1, kSolveThreads, bytes, st>>>(red_f, red_d, D, p, n, norms, inv_count,
                                                  objective_out, rmse_out, err);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    if (G_out) launch_gram(D, p, n, G_out, st);   // Gram of the (possibly unchanged) D
    return SDL_OK;
}

void launch_rescale(const int32_t* support, float* coef, long long count, int n1, int n2,
                    int side, const float* norms, cudaStream_t st) {
    if (count <= 0) return;
    const int threads = 256;
    const long long blocks = std::min<long long>((count + threads - 1) / threads, 152 * 16);
    rescale_kernel<<<(int)blocks, threads, 0, st>>>(support, coef, count, n1, n2, side, norms);
}

}  // namespace sdl
