/*
 * sdl.h - C ABI of the GB300 separable dictionary learning library.
 *
 * The library learns a pair dictionary (D1, D2) for 2D signals,
 * Y_k ~= D1 X_k D2^T with s-sparse X_k, by the Tensor-MOD alternation of
 * Rusu & Irofti, "Efficient and Parallel Separable Dictionary Learning"
 * (arXiv 2007.03800): 2D-OMP sparse coding (Sec. III step 1) followed by the
 * closed-form least-squares dictionary updates of Corollary 1 (D1) and
 * Result 1 (D2), one iteration being the main loop of Algorithm 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Y   : float32, p1 x p2 x N, each signal column-major and signals back to
 *          back: element (a, b, k) at Y[a + p1*b + p1*p2*k].
 *  - D1  : float32 p1 x n1 column-major (D1[a + p1*i]); D2 likewise p2 x n2.
 *          Dictionaries passed in are expected to have unit-norm columns
 *          (the constraint of Eq. (1)); outputs always do.
 *  - Sparse codes X_k are stored per signal as s_max slots in pick order:
 *          support[k*s_max + l]  int32 pair index q = i + n1*j  (the column of
 *                                D2 (x) D1 under column-order vec, Sec. I),
 *                                -1 in unused slots;
 *          coef[k*s_max + l]     float32 value of X_k[i, j] (0 in unused slots);
 *          nnz[k]                int32 number of used slots.
 *  - Every pointer argument is a DEVICE pointer owned by the caller, unless
 *    stated otherwise; the library never frees or retains caller memory.
 *    Buffers must not overlap unless an argument is documented in/out.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream: they return after
 *    enqueueing.  A negative return value is an argument or launch error
 *    detected on the host, and then nothing was enqueued.  Errors found on
 *    the device (non-finite data, a singular normal matrix) are recorded in
 *    the context and reported by sdl_status().
 *  - Supported shapes: 1 <= p1, p2 <= 64, p1*p2 <= 1024; n1, n2 >= 1 with
 *    (n1, n2) inside one of the compiled tile shapes (see
 *    sdl_shape_supported); 1 <= s_max <= min(p1*p2, n1*n2, 32).
 *  - Precision: FP32 arithmetic throughout.  Tie rule of the greedy step:
 *    the largest |correlation|, ties to the smallest q.  A pick whose new
 *    Cholesky pivot^2 <= 1e-6 * A_tt, or whose best score is exactly 0,
 *    stops that signal early (nnz < s_max).
 *  - A context is not thread-safe: calls sharing one context must be issued
 *    from one host thread and on streams ordered with each other.
 */
#ifndef SDL_GB300_H
#define SDL_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdl_ctx sdl_ctx;

enum sdl_error {
    SDL_OK = 0,
    SDL_ERR_ARG = -1,          /* invalid argument (null pointer, bad size)   */
    SDL_ERR_CUDA = -2,         /* a CUDA runtime call failed                  */
    SDL_ERR_NONFINITE = -3,    /* NaN/Inf in Y or in a normal matrix          */
    SDL_ERR_SINGULAR = -4,     /* normal matrix P or M not positive definite  */
    SDL_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up          */
    SDL_ERR_WORKSPACE = -6,    /* workspace allocation failed                 */
    SDL_ERR_UNSUPPORTED = -7,  /* shape outside the compiled tile shapes      */
    SDL_ERR_CAPACITY = -8      /* problem too large for the static scratch    */
};

/* Create a context on CUDA device `device` (the device is made current).
 * The context owns only its workspace (partial sums, Gram matrices, scale
 * factors, the device error word), grown on demand.  Returns SDL_OK and sets
 * *ctx, or a negative code and sets *ctx = NULL. */
int sdl_create(sdl_ctx** ctx, int device);

/* Free the context and its workspace (synchronises the device first).
 * NULL is accepted and ignored. */
int sdl_destroy(sdl_ctx* ctx);

/* Human-readable name of an error code (static string). */
const char* sdl_strerror(int code);

/* Synchronise `stream`, then return the first device-side error recorded by
 * work enqueued through `ctx` since the previous sdl_status call (SDL_OK if
 * none) and clear it.  Also reports pending CUDA errors as SDL_ERR_CUDA. */
int sdl_status(sdl_ctx* ctx, void* stream);

/* 1 if (p1, p2, n1, n2, s_max) is handled by a compiled kernel shape, else 0. */
int sdl_shape_supported(int p1, int p2, int n1, int n2, int s_max);

/* Pre-size the context workspace for problems up to these sizes, so that
 * later calls allocate nothing (needed before capturing calls into a CUDA
 * graph).  Synchronous. */
int sdl_reserve(sdl_ctx* ctx, int p1, int p2, int n1, int n2, int s_max);

/*
 * sdl_sparse_code - 2D-OMP of all N signals (Sec. III step 1; the greedy
 * pursuit over atom pairs d1_i d2_j^T that is equivalent to 1D OMP on
 * D2 (x) D1, Sec. II), with a full least-squares re-fit after every pick.
 *
 *   eps <= 0 : exactly s_max picks per signal (fewer only at a degenerate
 *              pick, see above);
 *   eps >  0 : error-driven mode of the denoising experiments (Sec. IV):
 *              before every pick, stop once ||R_k||_F <= eps; at most s_max.
 *
 * Outputs support/coef (N*s_max), nnz (N) and, if res_energy != NULL,
 * res_energy[k] = ||Y_k - D1 X_k D2^T||_F^2 (FP32, from the least-squares
 * energy identity).  N = 0 enqueues nothing.  Signals containing NaN/Inf get
 * nnz = 0 and raise SDL_ERR_NONFINITE in sdl_status.
 */
int sdl_sparse_code(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                    const float* D1, int n1, const float* D2, int n2,
                    int s_max, float eps,
                    int32_t* support, float* coef, int32_t* nnz,
                    float* res_energy, void* stream);

/*
 * sdl_update_D1 - optimal left dictionary for fixed codes (Corollary 1):
 *   T_k = X_k D2^T,  P = sum_k T_k T_k^T (n1 x n1),  B1 = sum_k Y_k T_k^T,
 *   D1* = B1 P^{-1},  W1 = diag(1/||d1*_i||),  D1 <- D1* W1,  X_k <- W1^{-1} X_k.
 * P is accumulated through the Gram shortcut of Sec. III,
 * T_k T_k^T = X_k (D2^T D2) X_k^T.
 *
 *   D1   in/out: replaced by the normalised optimum on success; left
 *        unchanged if the update fails on the device (see sdl_status).
 *   coef in/out: rescaled by W1^{-1} (slot l times ||d1*_{i_l}||).
 *   objective_out: NULL or device double[2] = {objective of Eq. (1) before,
 *        after} the update: sums over all signals kept in FP64 (the FP32
 *        per-signal energies are added in compensated FP32 per warp and in
 *        FP64 across warps; "after" uses the exact change identity of the
 *        update, so the solve error enters only to second order).
 * Atoms used by no signal (zero row/column of P) are kept unchanged and the
 * normal equations are solved on the used atoms.
 */
int sdl_update_D1(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                  float* D1, int n1, const float* D2, int n2, int s_max,
                  const int32_t* support, float* coef,
                  double* objective_out, void* stream);

/*
 * sdl_update_D2 - optimal right dictionary for fixed codes (Result 1):
 *   Z_k = D1 X_k,  M = sum_k Z_k^T Z_k (n2 x n2),  B2 = sum_k Y_k^T Z_k,
 *   D2* = B2 M^{-1} (the transpose of the printed (D2*)^T = M^{-1} sum Z^T Y),
 *   W2 = diag(1/||d2*_j||),  D2 <- D2* W2,  X_k <- X_k W2^{-1}.
 * Same argument rules as sdl_update_D1, mirrored.
 */
int sdl_update_D2(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                  const float* D1, int n1, float* D2, int n2, int s_max,
                  const int32_t* support, float* coef,
                  double* objective_out, void* stream);

/*
 * sdl_iterate - one iteration of Algorithm 1 on one GPU:
 *   1. 2D-OMP of all signals with (D1, D2), accumulating P and B1 on the fly;
 *   2. D1 update (Corollary 1);
 *   3. 2D-OMP again with the new D1, accumulating M and B2;
 *   4. D2 update (Result 1), and X_k <- X_k W2^{-1}.
 * D1, D2 in/out.  support/coef/nnz receive the codes of step 3 rescaled as
 * in step 4, consistent with the returned dictionaries.  rmse_out: NULL or
 * device double[2] = RMSE ||Y - D1 X D2^T||_F / sqrt(p1 p2 N) right after step
 * 2 and right after step 4.  eps as in sdl_sparse_code.
 */
int sdl_iterate(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                float* D1, int n1, float* D2, int n2, int s_max, float eps,
                int32_t* support, float* coef, int32_t* nnz,
                double* rmse_out, void* stream);

/*
 * Batching: several independent dictionary-learning problems ("groups") that
 * differ in signal size, dictionary size, sparsity and stopping rule, run
 * together.  This is the GB300 counterpart of the paper's many-worker setting
 * (Algorithm 1 with its data split over nodes): each coding pass of all groups
 * is ONE persistent launch, each update stage (Gram, reduction, solve,
 * rescale) is one launch for all groups, and with SDL_BATCH_GRAPH the whole
 * iteration is captured once into a CUDA graph and replayed.
 *
 * A group is described like the arguments of sdl_iterate (all device
 * pointers, owned by the caller, which must keep them valid and unmoved for
 * the batch's lifetime).  A group with a compiled specialised shape,
 * (p1, p2, n1, n2, s_max) in {(8,8,16,16,4), (12,12,24,24,6), (16,16,32,32,8)},
 * and Y 16-byte aligned joins the persistent multi-problem launch.  Any other
 * group that sdl_sparse_code supports (n1 <= 32 and n2 <= 128, n1 <= 128 and
 * n2 <= 32, or both <= 64) is coded by the generic kernel in a launch of its
 * own within the same iteration (and graph); its update stages still share
 * the one launch per stage.  Other shapes: SDL_ERR_UNSUPPORTED.  eps > 0 gives
 * the group an error-driven stop (Sec. IV), per group.
 */
typedef struct sdl_group {
    const float* Y;      /* p1 x p2 x N signals (layout as in sdl_iterate)   */
    int p1, p2;
    int64_t N;           /* >= 1                                              */
    float* D1;           /* p1 x n1, in/out                                   */
    int n1;
    float* D2;           /* p2 x n2, in/out                                   */
    int n2;
    int s_max;
    float eps;
    int32_t* support;    /* N x s_max outputs of the codes                    */
    float* coef;
    int32_t* nnz;
    float* res_energy;   /* N, may be NULL                                    */
} sdl_group;

#define SDL_BATCH_AUTOTUNE 1  /* time each group's compiled lane tilings and
                                 split the CTAs between groups by measured cost;
                                 the context remembers the result for batches
                                 of the same groups (shapes, N, s_max, eps)
                                 and reuses it                                  */
#define SDL_BATCH_GRAPH 2     /* capture one iteration into a CUDA graph       */
#define SDL_BATCH_RETUNE 4    /* with AUTOTUNE: time again even if remembered  */

typedef struct sdl_batch sdl_batch;

/* Validate the groups, allocate the batch workspace, autotune (if asked) by
 * timing coding passes on the groups' own data (writes only workspace), build
 * the launch descriptors and capture the graph.  Synchronous on `stream`. */
int sdl_batch_create(sdl_ctx* ctx, const sdl_group* groups, int n_groups, int flags,
                     void* stream, sdl_batch** out);

/* 2D-OMP of every group's signals in one persistent launch (codes only). */
int sdl_batch_sparse_code(sdl_batch* batch, void* stream);

/* One Algorithm-1 iteration of every group (graph replay when captured).
 * rmse_out: NULL or device double[2 * n_groups], for group g the RMSE after
 * its D1 update (2g) and after its D2 update (2g + 1). */
int sdl_batch_iterate(sdl_batch* batch, double* rmse_out, void* stream);

/* Host arrays of n_groups (each may be NULL): chosen tiling id (-1 for a
 * group coded by the generic kernel), CTAs given to the group in the
 * multi-problem launch (0 for those), and the measured (autotune) or
 * modelled cost of one of its coding passes in microseconds.  Returns
 * n_groups. */
int sdl_batch_tuning(const sdl_batch* batch, int* shape_id, int* ctas, float* cost_us);

/* Every measurement the autotuner took (empty without SDL_BATCH_AUTOTUNE): for
 * entry e, the group, the tiling id, the CTAs per SM and the time of one D1-side
 * coding pass of that group alone in microseconds.  Host arrays of max_entries
 * (each may be NULL); returns the number of entries (which may exceed
 * max_entries: only the first max_entries are written), SDL_ERR_ARG on a NULL
 * batch or a negative max_entries. */
int sdl_batch_tuning_log(const sdl_batch* batch, int* group, int* shape_id, int* ctas_per_sm,
                         float* cost_us, int max_entries);

/* Synchronise the device and free the batch (NULL accepted). */
int sdl_batch_destroy(sdl_batch* batch);

/*
 * Patch-based denoising (Sec. IV): the sparse coder applied to every
 * overlapping patch of a noisy image, the image rebuilt by averaging.
 *
 * sdl_extract_patches - every stride-1 p x p patch of an H x W row-major FP32
 *   image, raster order of the top-left corner (k = r*(W-p+1) + c), each with
 *   its mean removed: patches[k*p*p + a + p*b] = img[(r+a)*W + c+b] - means[k].
 *   N = (H-p+1)(W-p+1) patches; patches holds N*p*p floats, means N.
 */
int sdl_extract_patches(const float* image, int H, int W, int p, float* patches,
                        float* means, void* stream);

/*
 * sdl_patch_average - rebuild the image from coded patches: pixel (y, x) is
 *   the plain average, over every patch k covering it, of
 *   means[k] + (D1 X_k D2^T)[y - r, x - c]   (D1 p x n1, D2 p x n2).
 *   Codes as written by the coders (N x s_max slots).  The reconstructed
 *   patches go through a context-owned workspace of N*p*p floats.  Output
 *   image_out: H*W floats, row-major.  Deterministic (fixed summation order).
 */
int sdl_patch_average(sdl_ctx* ctx, const int32_t* support, const float* coef,
                      const float* means, int s_max, const float* D1, int n1,
                      const float* D2, int n2, int p, int H, int W, float* image_out,
                      void* stream);

/* sdl_ssim - mean SSIM index (Wang, Bovik, Sheikh, Simoncelli 2004; the index
 * of Table III) of image x against ref (H x W row-major device floats, H, W
 * >= 11) over every 11 x 11 window position inside the image, Gaussian window
 * weights (sigma 1.5, normalised to sum 1), C1 = (0.01 peak)^2,
 * C2 = (0.03 peak)^2; written to device float out[0].  Deterministic (fixed
 * summation order); per-block sums use a context workspace. */
int sdl_ssim(sdl_ctx* ctx, const float* x, const float* ref, int H, int W, float peak,
             float* out, void* stream);

/* sdl_psnr - 10 log10(peak^2 / MSE(x, ref)) over `count` floats, written to
 * device float out[0]. */
int sdl_psnr(const float* x, const float* ref, int64_t count, float peak, float* out,
             void* stream);

/*
 * sdl_gemm_bf16 - the library's tensor-core GEMM (used by the support-
 * proposal network and the BF16 correlation path):
 *   out = act(alpha * A B^T + bias),   A: M x K, B: N x K, both BF16 row-major
 *   with K contiguous (leading dimensions lda, ldb in elements, multiples of
 *   8, pointers 16-byte aligned), FP32 accumulation on tcgen05 tensor cores.
 *   act: 0 none, 1 GELU (0.5 x (1 + erf(x / sqrt 2))); bias: NULL or FP32 [N].
 * Outputs (each optional, NULL to skip): C FP32 (C += out when accumulate),
 * Cb BF16 copy, Ct BF16 transposed copy (Ct[n*ldct + m]), pre FP32 values
 * before the activation.  A device-side timeout is reported by sdl_status.
 */
int sdl_gemm_bf16(sdl_ctx* ctx, const void* A, int lda, const void* B, int ldb, int M, int N,
                  int K, float alpha, const float* bias, int act, float* C, int ldc,
                  int accumulate, void* Cb, int ldcb, void* Ct, int ldct, float* pre,
                  int ldpre, void* stream);

/*
 * sdl_gemm_bf16_terms - the same GEMM over the sum of `terms` (1 to 3)
 *   operand pairs in one FP32 accumulator:
 *   out = act(alpha * sum_t A[t] B[t]^T + bias).
 * A and B are HOST arrays of `terms` device pointers; every A[t] is M x K
 * with leading dimension lda and every B[t] is N x K with ldb (the rules of
 * sdl_gemm_bf16 apply to each).  This is the split-BF16 correlation product
 * hi*hi + hi*lo + lo*hi of the BF16 precision mode.  SDL_ERR_ARG for terms
 * outside 1..3 or a null or misaligned pointer.
 */
int sdl_gemm_bf16_terms(sdl_ctx* ctx, const void* const* A, int lda, const void* const* B,
                        int ldb, int terms, int M, int N, int K, float alpha, const float* bias,
                        int act, float* C, int ldc, int accumulate, void* Cb, int ldcb, void* Ct,
                        int ldct, float* pre, int ldpre, void* stream);

/*
 * Precision modes (an extension beyond the paper; default SDL_PREC_FP32).
 *  SDL_PREC_BF16_CORR: the correlations C0 = D1^T Y_k D2 of a coding pass come
 *    from ONE tensor-core GEMM of the vectorised signals with the Kronecker
 *    dictionary D2 (x) D1 (Sec. I): both operands split into BF16 high and
 *    low parts, the three products hi*hi + hi*lo + lo*hi summed in one FP32
 *    accumulator.  Every entry is within
 *    e(p1 p2) = (3 + 1/64) 2^-16 + 2^-24 + 3 Kp 2^-23 (Kp = p1 p2 rounded up
 *    to 8) times ||Y_k||_F of its exact value; at every greedy step each
 *    entry within 3 e ||Y_k||_F of the approximate maximum is re-scored in
 *    FP32 ((d1_i^T Y_k) d2_j, from the rows of D1^T Y_k formed once per
 *    signal), so the maximum is an FP32 score and the picks are FP32 picks.  The Gram-domain updates, the Cholesky
 *    factor and the partial sums stay FP32.  Uses N x n1n2 FP32 and
 *    2 (N + n1n2) x Kp BF16 of workspace.
 *  SDL_PREC_NO_RESCORE: with BF16_CORR, skip the re-scoring (pure BF16 picks;
 *    for precision studies).
 *  SDL_PREC_FP64_SOLVE: the normal-equation solves, the objective change and
 *    the atom renormalisation in FP64 (partial sums stay FP32); a pivot is
 *    rejected (SDL_ERR_SINGULAR) below 1e-12 of its diagonal entry instead of
 *    the FP32 solve's 1e-7.
 */
#define SDL_PREC_FP32 0
#define SDL_PREC_BF16_CORR 1
#define SDL_PREC_NO_RESCORE 2
#define SDL_PREC_FP64_SOLVE 4
int sdl_set_precision(sdl_ctx* ctx, int flags);

/* ---- Tilings of the specialised coder (Algorithm 1, step "sparse coding").
 * The shapes (p1, p2, n1, n2, s) = (8, 8, 16, 16, 4), (12, 12, 24, 24, 6) and
 * (16, 16, 32, 32, 8) have coders compiled for several tilings: one signal per
 * warp on two lane grids, and for the first two shapes also two signals per
 * warp (each half-warp codes one signal).  Every tiling of a shape forms each correlation, update and solve
 * with the same FMA chains, so the codes (support, coef, nnz) do not depend on
 * the tiling; the TMOD partial sums are added in a tiling-dependent order.
 *
 * sdl_tilings: the tiling ids compiled for the shape (host array of max_ids,
 *   may be NULL); returns their number (0: no specialised coder, the generic
 *   kernel runs), SDL_ERR_ARG for max_ids < 0.
 * sdl_set_tiling: pin `tiling` (one of those ids) and ctas_per_sm (0 = as many
 *   CTAs per SM as fit, else 1..8) for the shape in this context; tiling < 0
 *   unpins.  SDL_ERR_UNSUPPORTED if the shape has no such tiling.
 * sdl_tune_tiling: time one D1-side coding pass (Y p1 x p2 x N and D1, D2 as
 *   in sdl_iterate, device pointers, Y 16-byte aligned; nothing is written but
 *   workspace) with every tiling at 1 and 2 CTAs per SM, pin the fastest and
 *   return its id in *tiling_out (may be NULL).  Synchronises the stream.
 *   SDL_ERR_UNSUPPORTED if the shape has no specialised coder or Y is not
 *   16-byte aligned.
 * sdl_tune_log: the measurements of the last sdl_tune_tiling (tiling id, CTAs
 *   per SM, microseconds per pass; host arrays of max_entries, each may be
 *   NULL); returns the number of entries. */
int sdl_tilings(int p1, int p2, int n1, int n2, int s, int* ids, int max_ids);
int sdl_set_tiling(sdl_ctx* ctx, int p1, int p2, int n1, int n2, int s, int tiling, int ctas_per_sm);
int sdl_tune_tiling(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N, const float* D1, int n1,
                    const float* D2, int n2, int s, int* tiling_out, void* stream);
int sdl_tune_log(const sdl_ctx* ctx, int* tiling, int* ctas_per_sm, float* cost_us, int max_entries);

/* Number of correlation entries re-scored in FP32 since the previous call
 * (synchronises the device). */
int sdl_precision_stats(sdl_ctx* ctx, uint64_t* rescored_entries);

/*
 * Learned support proposal (an extension beyond the paper).  A two-layer
 * network scores every atom pair of a signal,
 *   x = vec(Y)/||Y||_F,  h = GELU(W1 x + b1),  z = W2 h + b2  (z: n1*n2 scores),
 * with BF16 weights/activations and FP32 accumulation on tcgen05 tensor cores.
 * It is trained on (signal, 2D-OMP support) pairs with the mean over the
 * batch of the summed binary cross-entropy with logits and Adam (FP32 master
 * weights; beta1 0.9, beta2 0.999, eps 1e-8).
 */
typedef struct sdl_mlp sdl_mlp;

/* Network for p1 x p2 signals and n1 x n2 pairs (n1*n2 <= 1024, a multiple
 * of 8), `hidden` units (multiple of 8), batches of up to max_batch (multiple
 * of 8) signals.  Weights start at zero: set them with sdl_mlp_set_weights. */
int sdl_mlp_create(sdl_ctx* ctx, int p1, int p2, int n1, int n2, int hidden, int max_batch,
                   sdl_mlp** out);
int sdl_mlp_destroy(sdl_mlp* mlp);

/* HOST FP32 arrays: W1 [hidden x p1p2] (row-major, input index = column-order
 * vec of Y), b1 [hidden], W2 [n1n2 x hidden], b2 [n1n2].  Synchronous.
 * set resets the Adam moments and step count. */
int sdl_mlp_set_weights(sdl_mlp* mlp, const float* W1, const float* b1, const float* W2,
                        const float* b2);
int sdl_mlp_get_weights(sdl_mlp* mlp, float* W1, float* b1, float* W2, float* b2);

/* One Adam step on a batch: Y (device, B signals laid out as for
 * sdl_iterate), support (device, B x s pair indices, -1 = none) = the labels,
 * B a multiple of 8 <= max_batch.  loss_out: NULL or device float[1]. */
int sdl_mlp_train_step(sdl_mlp* mlp, const float* Y, const int32_t* support, int s, int B,
                       float lr, float* loss_out, void* stream);

/* Loss and gradients of a batch without updating (gradient check): HOST
 * FP32 outputs shaped like the weights (each may be NULL).  Synchronous. */
int sdl_mlp_gradients(sdl_mlp* mlp, const float* Y, const int32_t* support, int s, int B,
                      float* loss_out, float* gW1, float* gb1, float* gW2, float* gb2,
                      void* stream);

/* Scores of N signals: device FP32 N x n1n2. */
int sdl_mlp_forward(sdl_mlp* mlp, const float* Y, int64_t N, float* scores, void* stream);

/*
 * sdl_sparse_code_learned - 2D-OMP on learned shortlists, with the full coder
 * as the fallback:
 *   1. the network scores all pairs; the k best (1 <= k <= 32) form the
 *      shortlist;
 *   2. 2D-OMP (same greedy rule, re-fit and stopping as sdl_sparse_code,
 *      fixed s_max) searches only the shortlist;
 *   3. a signal is flagged when it took s_max picks and some pair it did not
 *      pick correlates with the final residual more strongly than 0.7 x the
 *      weakest greedy score of its picks, or its data is not finite; flagged
 *      signals are coded again by the full coder;
 *   4. the full coder also codes a strided sample of max(4096, N/16) signals
 *      (all of them when N is smaller) and judges the learned codes there: if
 *      their RMSE on the sample exceeds the full coder's by more than 1 %,
 *      every signal is coded again by the full coder (fallback[] all 1,
 *      n_fallback = N).
 * Outputs as sdl_sparse_code plus fallback[N] (1 = re-coded), device
 * int n_fallback[1] and guard_out: NULL or device float[3] = {RMSE of the
 * learned codes on the sample (after step 3), RMSE of the full coder there,
 * 1 if step 4 re-coded everything else 0}.  N <= 2^31 - 1.  Compiled for
 * (p1,p2,n1,n2,s_max) = (12,12,24,24,6) and (8,8,16,16,4); the network must
 * match the shape.
 */
int sdl_sparse_code_learned(sdl_ctx* ctx, sdl_mlp* mlp, const float* Y, int p1, int p2,
                            int64_t N, const float* D1, int n1, const float* D2, int n2,
                            int s_max, int k, int32_t* support, float* coef, int32_t* nnz,
                            float* res_energy, int32_t* fallback, int32_t* n_fallback,
                            float* guard_out, void* stream);

/*
 * The first two steps of sdl_sparse_code_learned on their own (no fallback),
 * for callers that bring their own scores and for checking each step.
 *
 * sdl_learned_shortlists - per signal, rank the N x Q device FP32 scores
 * (row k at scores + k*Q) by the order-preserving 16-bit key of each score
 * (its upper 16 bits after flipping negative values, so that a larger float
 * never has a smaller key), ties to the smaller pair index q; NaN scores never
 * rank.  cand (device int32, N x k2): the k1 best pairs, then the next k2 - k1
 * (the check set), each of the two sets in increasing q and padded with -1
 * where fewer scores are valid.
 * 1 <= k1 <= k2 <= Q <= 1024.
 */
int sdl_learned_shortlists(sdl_ctx* ctx, const float* scores, int64_t N, int Q, int k1, int k2,
                           int32_t* cand, void* stream);

/*
 * sdl_sparse_code_shortlist - 2D-OMP whose greedy step looks only at the
 * first k1 pairs of cand[k] (k2 entries per signal, -1 = none): the largest
 * |correlation| over unselected candidates, ties to the smallest q, with the
 * re-fit, energy identity and stopping rules of sdl_sparse_code (fixed
 * s_max).  flag[k] = 1 when the signal's data is not finite, or when it took
 * s_max picks and some pair it did not pick (any of the n1 n2) correlates
 * with its final residual more strongly than 0.7 x the smallest best-score
 * among its picks (the learned coder's fallback test); else 0.  cand has k2
 * entries per signal (only the first k1 are searched).  res_energy may be
 * NULL.  1 <= k1 <= 32, k2 >= k1.  Compiled for (p1,p2,n1,n2,s_max) =
 * (12,12,24,24,6) and (8,8,16,16,4).
 */
int sdl_sparse_code_shortlist(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                              const float* D1, int n1, const float* D2, int n2, int s_max,
                              const int32_t* cand, int k1, int k2, int32_t* support, float* coef,
                              int32_t* nnz, float* res_energy, int32_t* flag, void* stream);

/*
 * Orthonormal variant (Remark 1): square orthonormal dictionaries
 * (n1 = p1, n2 = p2, D^T D = I), codes X_k = T_s(D1^T Y_k D2) (the s largest
 * |entries|, ties to the smallest q = i + p1 j; a signal keeps fewer when the
 * remaining entries are exactly 0), and orthogonal-Procrustes updates
 * D1 = U V^T of B1 = sum_k Y_k D2 X_k^T = U S V^T, D2 = U2 V2^T of
 * B2 = sum_k Y_k^T D1 X_k (the trace-maximisation reading of the garbled SVD
 * argument printed in Remark 1).  1 <= p1, p2 <= 32, 1 <= s <= min(32, p1 p2).
 * Layouts as sdl_sparse_code (D1 p1 x p1, D2 p2 x p2 column-major).
 *
 * eps > 0: error-driven, a signal stops before keeping another entry once
 * ||Y_k - D1 X_k D2^T||_F <= eps (the residual energy of orthonormal
 * dictionaries is ||Y_k||^2 - sum of the kept entries squared), at most s;
 * eps <= 0: s entries.
 *
 * sdl_ortho_sparse_code - the thresholded codes only (res_energy may be NULL).
 */
int sdl_ortho_sparse_code(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N,
                          const float* D1, const float* D2, int s, float eps, int32_t* support,
                          float* coef, int32_t* nnz, float* res_energy, void* stream);

/*
 * sdl_ortho_iterate - one iteration of Algorithm 1 - Orthonormal: codes with
 * (D1, D2), D1 by Procrustes (a one-sided Jacobi SVD of the FP32 sum B, in
 * FP32), codes again with the new D1, D2 by Procrustes.  D1, D2 in/out (must
 * be orthonormal on entry); support/coef/nnz receive the second codes.
 * rmse_out: NULL or device double[2], the RMSE right after each update (with
 * the codes of the preceding coding pass).  A numerically rank-deficient B
 * (smallest singular value <= 1e-6 of the largest) records SDL_ERR_SINGULAR
 * and leaves that dictionary unchanged.  N >= 1.
 */
int sdl_ortho_iterate(sdl_ctx* ctx, const float* Y, int p1, int p2, int64_t N, float* D1,
                      float* D2, int s, float eps, int32_t* support, float* coef, int32_t* nnz,
                      double* rmse_out, void* stream);

/*
 * Three-mode generalisation (Remark 3): signals Y_k of shape p1 x p2 x p3
 * (element (a, b, c) at a + p1 b + p1 p2 c + p1 p2 p3 k), dictionaries D1
 * (p1 x n1), D2 (p2 x n2), D3 (p3 x n3) column-major with unit columns, codes
 * over atom triples q = i + n1 j + n1 n2 l (the column of D3 (x) D2 (x) D1).
 * Limits: 1 <= p_m <= 16, p1 p2 p3 <= 1024, n1 n2 n3 <= 1024,
 * 1 <= s <= min(16, p1 p2 p3, n1 n2 n3).
 *
 * sdl_sparse_code3 - greedy pursuit over atom triples (argmax |correlation|
 * over unselected triples, ties to the smallest q, full least-squares re-fit,
 * the degenerate-pick rule of sdl_sparse_code), fixed s.
 */
int sdl_sparse_code3(sdl_ctx* ctx, const float* Y, int p1, int p2, int p3, int64_t N,
                     const float* D1, int n1, const float* D2, int n2, const float* D3, int n3,
                     int s, int32_t* support, float* coef, int32_t* nnz, float* res_energy,
                     void* stream);

/*
 * sdl_iterate3 - one iteration of the three-mode algorithm: for mode k = 1,
 * 2, 3 in turn, code all signals with the current dictionaries and update
 * D_k by Corollary 1 applied to the mode-k unfolding
 * Y_(k) = D_k X_(k) T_k^T (T_k the Kronecker product of the other two
 * dictionaries), with the column normalisation.  D1, D2, D3 in/out;
 * support/coef/nnz receive the codes of the third pass rescaled by W3^{-1};
 * rmse_out: NULL or device double[3], the RMSE right after each update.
 * Singular normal matrices follow sdl_update_D1.  N >= 1.
 */
int sdl_iterate3(sdl_ctx* ctx, const float* Y, int p1, int p2, int p3, int64_t N, float* D1,
                 int n1, float* D2, int n2, float* D3, int n3, int s, int32_t* support,
                 float* coef, int32_t* nnz, double* rmse_out, void* stream);

/*
 * sdl_sparse_code_static - the sparse coder of sdl_sparse_code with no
 * context and no device allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory once running
 * (an application that serves all GPU memory from its own pre-sized pool, or
 * a latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation and its possible failure under memory pressure) and for
 * callers that cannot keep a library context.
 *
 * Arguments, layouts and results are those of sdl_sparse_code (the caller
 * still provides Y, D1, D2 and the output buffers).  The only scratch, the
 * Gram matrices D1^T D1 and D2^T D2, lives in one file-scope device array of
 * 8192 floats (32 KiB) that every GPU which loads the library holds until
 * the process exits; hence n1*n1 + n2*n2 <= 8192, else SDL_ERR_CAPACITY and
 * nothing is enqueued.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Every call on a device shares the one array, which keeps the contents
 *    of the last call (each call rewrites both Gram matrices before reading
 *    them).  Calls whose work overlaps on the GPU (different streams, no
 *    ordering between them) race on the array and give wrong codes.
 *  - Device-side errors (a signal with NaN/Inf, which also gets nnz = 0; a
 *    bounded wait for a signal copy that gave up, after which the remaining
 *    signals of that warp are not coded) go to a second file-scope device
 *    word shared by every allocation-free call on the device, kept until
 *    sdl_static_status reads it.
 *  - The device addresses of both arrays are cached per device ordinal; a
 *    cudaDeviceReset of that device invalidates them (reload the library).
 */
int sdl_sparse_code_static(const float* Y, int p1, int p2, int64_t N,
                           const float* D1, int n1, const float* D2, int n2,
                           int s_max, float eps,
                           int32_t* support, float* coef, int32_t* nnz,
                           float* res_energy, void* stream);

/* Synchronise `stream`, then return the first device-side error recorded by
 * allocation-free calls on the current device since the previous
 * sdl_static_status (SDL_OK if none) and clear it.  Allocates nothing. */
int sdl_static_status(void* stream);

/*
 * sdl_fp32_fma_peak - FP32 fused multiply-add throughput of the current
 * device, the denominator of the coding passes' roofline (those passes are
 * bound by FP32 FMAs; the paper has no counterpart).  Times 12 launches of a
 * kernel in which every thread runs 8 independent chains of packed
 * fma.rn.f32x2 (packed = 1) or 16 chains of scalar fma.rn.f32 (packed = 0),
 * 64 warps per SM, with CUDA events on `stream`, and returns the best of the
 * last 10 in TFLOP/s (2 FLOP per multiply-add) and, if ms_out != NULL, its
 * duration.  Changes no clock or other GPU setting.  Synchronous.
 */
int sdl_fp32_fma_peak(int packed, double* tflops_out, double* ms_out, void* stream);

/*
 * Tracing: per-kernel device time and launch counts.  The paper reports only
 * wall-clock times (Tables I, II, IV); this hook gives the per-kernel split.
 *
 * Kernel kinds (index into the arrays of sdl_profile_collect):
 *   0 gram          G = D^T D of a dictionary
 *   1 code          2D-OMP pass without partial sums (sdl_sparse_code)
 *   2 code_D1       2D-OMP pass fused with the P, B1 partial sums
 *   3 code_D2       2D-OMP pass fused with the M, B2 partial sums
 *   4 accum_D1      partial sums of given codes, D1 side
 *   5 accum_D2      partial sums of given codes, D2 side
 *   6 reduce        fixed-order reduction of the partial-sum slots
 *   7 solve         normal-equation solve + atom normalisation
 *   8 rescale       X <- W^{-1} X
 *   9 memset        zeroing of global accumulation slots
 *  10 batch_graph   one replay of a batch's captured iteration graph
 *                   (its kernels are counted under their own kinds too)
 *  11 mlp           support-network forward / backward (GEMMs + element-wise)
 *  12 adam          support-network parameter update
 *  13 topk          shortlist selection from the network's scores
 *  14 shortlist     2D-OMP restricted to the shortlists, with the fallback test
 *  15 tc_corr       tensor-core correlations (precision extension)
 *  16 ortho_code    thresholded coding pass of the orthonormal variant
 *  17 procrustes    Procrustes update of the orthonormal variant
 */
#define SDL_NUM_KERNEL_KINDS 18

/* Failure-detection self-test: enqueue one tiny kernel that waits, bounded
 * by max_cycles SM clock cycles (1 .. 2^31, about one second at most), on an
 * mbarrier that nothing completes, exactly as the library's waiting kernels
 * do; when the bound runs out it records SDL_ERR_TIMEOUT in the context (read
 * by sdl_status) and returns.  The context stays usable. */
int sdl_selftest_timeout(sdl_ctx* ctx, long long max_cycles, void* stream);

/* Enable (1) or disable (0) event timing of every kernel this context
 * enqueues.  Launch counts are kept either way.  Host-side, synchronous. */
int sdl_profile_enable(sdl_ctx* ctx, int enable);

/* Synchronise the device, then write for each kind k < max_kinds the total
 * device milliseconds (total_ms[k], 0 when timing is off) and the number of
 * launches (launches[k]) since the previous call, and reset both.  Host
 * arrays; either may be NULL.  Returns SDL_NUM_KERNEL_KINDS or an error. */
int sdl_profile_collect(sdl_ctx* ctx, double* total_ms, int64_t* launches, int max_kinds);

/* Name of a kernel kind (static string), "?" when out of range. */
const char* sdl_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* SDL_GB300_H */
