// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sdl.h"

namespace sdl {

// Degenerate-pick rule of the greedy step: the new Cholesky pivot^2 must
// exceed this fraction of the new pair's Gram diagonal.
constexpr float kPivotRel = 1e-6f;
// Singular-normal-matrix rule of the dictionary solves (relative pivot).
constexpr float kSolvePivotRel = 1e-7f;
// Hard limit of the per-signal register Cholesky (one lane per row).
constexpr int kMaxS = 32;
// Largest dictionary dimension handled by the update solve.
constexpr int kMaxN = 128;
constexpr int kMaxP = 64;

// Which partial sums a coding pass accumulates next to the codes.
enum Side : int {
    kCodeOnly = 0,   // sparse coding only
    kSideD1 = 1,     // P = sum X G2 X^T, B1 = sum (Y D2) X^T  (Corollary 1)
    kSideD2 = 2      // M = sum X^T G1 X, B2 = sum (Y^T D1) X  (Result 1)
};

// Arguments of a coding / accumulation pass (device pointers).
struct PassArgs {
    const float* Y;
    int p1, p2;
    long long N;
    const float* D1;      // p1 x n1 column-major
    const float* D2;      // p2 x n2 column-major
    const float* G1;      // n1 x n1 (symmetric)
    const float* G2;      // n2 x n2
    int n1, n2;
    int s;                // slots per signal (s_max)
    float eps2;           // > 0: error-driven stop at ||R||^2 <= eps2
    int32_t* support;     // may be null (codes not stored)
    float* coef;
    int32_t* nnz;
    float* res_energy;    // may be null
    const int32_t* in_support;   // accumulation-only pass: given codes
    const float* in_coef;
    float* part_f;        // partial sums: [slot][n*n + p*n]
    double* part_d;       // [slot][2]: residual energy, ||Y||^2
    int acc_in_smem;      // 1: CTA-private shared accumulators, slot = CTA
    int n_slots;          // global-accumulator mode: slots (CTA % n_slots)
    int* err;
    const int32_t* idx;   // optional: code only the signals idx[0 .. *idx_count)
    const int* idx_count; //   (specialised kernels only; device count)
    int idx_compact;      // with idx: outputs at list position j, not at idx[j]
    // optional correlations C0 from outside (BF16 tensor-core path), N x ldc0
    // FP32 with entry q = i + n1*j, each within c0_err_rel * ||Y_k|| of the
    // FP32 value; entries near the running maximum are re-scored in FP32
    // (generic kernel only; c0_err_rel = 0: no re-scoring)
    const float* c0ext;
    int ldc0;
    float c0_err_rel;
    unsigned long long* rescored;   // optional counter of re-scored entries
    // host side only: compiled tiling of the specialised coder (id + 1; 0 =
    // the first tiling compiled for the shape) and CTAs per SM (0 = as many
    // as fit)
    int tiling;
    int tiling_cps;
};

// Host launchers (omp_pass.cu).  They return the number of partial-sum
// slots written (to be reduced), or a negative sdl_error.
int launch_code_pass(const PassArgs& a, int side, cudaStream_t st, int num_sms);
// The generic kernel alone (any supported shape, Y at any alignment); with
// plan_only it returns the slot count the launch would write and launches
// nothing (a batch sizes its reductions with it before capturing the graph).
int launch_code_pass_generic(const PassArgs& a, int side, cudaStream_t st, int num_sms,
                             bool plan_only = false);
int launch_accumulate_pass(const PassArgs& a, int side, cudaStream_t st, int num_sms);
// omp_fast.cu: compile-time-shape kernels; SDL_ERR_UNSUPPORTED when no
// specialisation matches (the caller then uses the generic kernel).
int launch_code_pass_fast(const PassArgs& a, int side, cudaStream_t st, int num_sms);
// Compiled tilings ("shape ids") for a problem shape; returns how many.
int fast_shape_variants(int p1, int p2, int n1, int n2, int s, int* ids, int max_ids);
// warps per CTA of a compiled tiling (the persistent multi-problem kernel runs
// 8-warp CTAs, so only those tilings can join a batch)
int fast_variant_warps(int shape_id);
// one compiled tiling on exactly `grid` CTAs (a one-problem batch runs its
// passes this way), and the CTAs per SM that tiling's kernel fits
int launch_code_pass_grid(const PassArgs& a, int side, int shape_id, int grid, cudaStream_t st);
int fast_variant_ctas_per_sm(int shape_id, int side);
size_t fast_smem_bytes(int shape_id, int side);
// One problem with a given tiling; ctas_per_sm > 0 caps the resident CTAs per SM.
int launch_code_pass_variant(const PassArgs& a, int side, int shape_id, int ctas_per_sm,
                             cudaStream_t st, int num_sms);
// Several problems in one persistent launch (device arrays of G entries,
// cta_begin has G+1); smem = the largest per-problem requirement.  spread > 0
// (the SM count, total_ctas a multiple of it): CTAs b and b + spread take
// neighbouring positions, so that the CTAs an SM holds at once mostly run the
// same problem's code.
int launch_code_multi(const PassArgs* d_groups, const int* d_cta_begin, const int* d_shape, int G,
                      int total_ctas, size_t smem, int side, cudaStream_t st, int spread = 0);
int multi_ctas_per_sm(size_t smem, int side);
bool code_shape_supported(int p1, int p2, int n1, int n2, int s);
// Upper bound of the partial-sum slots any pass may use for these sizes.
int max_partial_slots(int num_sms);
// tmod3_fast.cu: three-mode coding pass specialised at compile time for the
// compiled shapes (SDL_ERR_UNSUPPORTED otherwise or for a Y not 16-byte
// aligned); returns the partial-sum slots written (mode 1-3) or 0 (mode 0)
int launch_code3_fast(int mode, const float* Y, int p1, int p2, int p3, int n1, int n2, int n3,
                      long long N, const float* D1, const float* D2, const float* D3,
                      const float* G1, const float* G2, const float* G3, int s, int32_t* support,
                      float* coef, int32_t* nnz, float* res, float* part_f, double* part_d,
                      int max_slots, int* err, int num_sms, cudaStream_t st);

// tmod.cu
void launch_gram(const float* D, int p, int n, float* G, cudaStream_t st);
void launch_reduce_partials(const float* part_f, const double* part_d, int n_slots,
                            int nf, float* red_f, double* red_d, cudaStream_t st);
void launch_gram2(const float* D1, int p1, int n1, float* G1, const float* D2, int p2, int n2,
                  float* G2, cudaStream_t st);
// G_out (may be NULL): receives the Gram matrix of D after the update.
int launch_solve(const float* red_f, const double* red_d, float* D, int p, int n,
                 float* norms, double inv_count, double* objective_out, double* rmse_out,
                 int* err, cudaStream_t st, float* G_out = nullptr);

void launch_rescale(const int32_t* support, float* coef, long long count, int n1, int n2,
                    int side, const float* norms, cudaStream_t st);

// Descriptors of the batched (several problems per launch) update kernels.
struct GramDesc {
    const float* D;
    int p, n;
    float* G;
    int block_begin;
};
struct ReduceDesc {
    const float* part_f;
    const double* part_d;
    int n_slots, nf;
    float* red_f;
    double* red_d;
    int block_begin;
};
struct SolveDesc {
    const float* red_f;
    const double* red_d;
    float* D;
    int p, n;
    float* norms;
    double inv_count;
    double* objective_out;
    double* rmse_out;
    float* G_out;
    int keep_p;
};
struct RescaleDesc {
    const int32_t* support;
    float* coef;
    long long count;
    int n1, n2, side;
    const float* norms;
};
// which: 0 gram, 1 reduce, 2 solve (one CTA per problem; 4 when some problem
// has n > 32), 3 rescale.
int launch_multi_update_kernels(int which, const void* d_desc, int G, int blocks, size_t smem,
                                int* err, cudaStream_t st);
size_t solve_smem_bytes(int p, int n, int* keep_p);
int launch_solve64(const float* red_f, const double* red_d, float* D, int p, int n, float* norms,
                   double inv_count, double* objective_out, double* rmse_out, int* err,
                   cudaStream_t st, float* G_out);
}  // namespace sdl
#include <cuda_bf16.h>
namespace sdl {
// precision.cu: C0 of N signals by one split-BF16 tensor-core GEMM (FP32 out,
// N x n1n2); every entry within c0_split_err_rel(p1 p2) ||Y_k||_F of exact
float c0_split_err_rel(int p1p2);
int tc_correlations(const float* Y, long long N, int p1, int p2, const float* D1, int n1,
                    const float* D2, int n2, __nv_bfloat16* Yb, bool fill_y, __nv_bfloat16* KT,
                    float* C0, int* err, cudaStream_t st);

// tc_gemm.cu: C = alpha A B^T (+bias, GELU) on tcgen05 tensor cores, BF16 in,
// FP32 accumulate; optional FP32 / BF16 / transposed-BF16 / pre-activation outputs.
int tc_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float alpha,
            const float* bias, int act, float* C, int ldc, int accumulate, void* Cb, int ldcb,
            void* Ct, int ldct, float* pre, int ldpre, int* err, cudaStream_t st,
            const float* gin = nullptr, int ldgin = 0);
// The same with the sum of `terms` (1..3) operand pairs in one accumulator:
// C = alpha sum_t A[t] B[t]^T (...), all pairs with the shapes and strides given.
int tc_gemm_terms(const void* const* A, int lda, const void* const* B, int ldb, int terms, int M,
                  int N, int K, float alpha, const float* bias, int act, float* C, int ldc,
                  int accumulate, void* Cb, int ldcb, void* Ct, int ldct, float* pre, int ldpre,
                  int* err, cudaStream_t st, const float* gin = nullptr, int ldgin = 0);

// Record the first device-side error (first writer wins).
__device__ __forceinline__ void record_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace sdl
