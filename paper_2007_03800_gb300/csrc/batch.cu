// Batched problems ("groups") with different signal and dictionary shapes,
// sparsities and stopping rules, coded and updated together: one persistent
// multi-problem launch per coding pass, one launch per update stage for all
// groups, and the whole Algorithm-1 iteration captured once into a CUDA graph
// that is replayed every iteration.  An autotuner times the compiled lane
// tilings of every group and splits the CTAs between groups by measured cost.
// A group whose shape has no compiled tiling (for instance 16 x 64 signals
// with 32 x 128 atoms) is coded by the generic kernel in a launch of its own
// inside the same iteration; its update stages join the others'.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

#include "ctx.cuh"

using namespace sdl;

struct sdl_batch {
    sdl_ctx* ctx = nullptr;
    int G = 0;
    std::vector<sdl_group> groups;
    std::vector<int> shape;        // compiled tiling per group (-1: generic kernel)
    std::vector<int> generic;      // groups coded by the generic kernel
    std::vector<int> gslots[3];    // their partial-sum slots per pass side
    int n_fast = 0;                // groups in the multi-problem kernel
    std::vector<int> cta_begin;    // G + 1 prefix of CTAs per group
    std::vector<float> cost_us;    // time of one fused pass of the group alone
    int single_cps = 0;            // one group: the CTAs per SM the autotuner chose
    // every (group, tiling, CTAs per SM, cost) the autotuner measured
    std::vector<int> log_group, log_shape, log_cps;
    std::vector<float> log_cost;
    int total_ctas = 0;
    size_t smem[3] = {0, 0, 0};    // multi-kernel dynamic smem per side
    size_t solve_smem[2] = {0, 0};
    bool solve_large[2] = {false, false};   // some group's n on this side is > 32
    int gram_blocks = 0, red_blocks[2] = {0, 0}, rescale_blocks = 0;
    // device memory: one allocation, carved up
    char* dmem = nullptr;
    PassArgs* d_args[3] = {nullptr, nullptr, nullptr};
    int* d_cta_begin = nullptr;
    int* d_shape = nullptr;
    GramDesc* d_gram = nullptr;
    ReduceDesc* d_red[2] = {nullptr, nullptr};
    SolveDesc* d_solve[2] = {nullptr, nullptr};
    RescaleDesc* d_rescale = nullptr;
    double* rmse_stage = nullptr;
    std::vector<PassArgs> args[3];
    std::vector<float*> G1, G2, red_f, norms;
    std::vector<double*> red_d, part_d;
    std::vector<float*> part_f;
    cudaGraphExec_t graph = nullptr;
};

namespace {

constexpr int kSlotsPerSm = 8;   // partial-sum slots reserved per SM and group
constexpr int kMultiWarps = 8;   // warps per CTA of the persistent multi-problem kernel

// A coding pass of every group: one persistent multi-problem launch, or for a
// single group its tiling's own kernel on the same CTAs (no other problem's
// code shares its register allocation).
int code_pass(const sdl_batch* b, int side, cudaStream_t st) {
    int rc = SDL_OK;
    if (b->n_fast > 0) {
        rc = b->G == 1 ? launch_code_pass_grid(b->args[side][0], side, b->shape[0], b->total_ctas, st)
                       : launch_code_multi(b->d_args[side], b->d_cta_begin, b->d_shape, b->G,
                                           b->total_ctas, b->smem[side], side, st, b->ctx->num_sms);
        if (rc != SDL_OK) return rc;
    }
    for (size_t i = 0; i < b->generic.size(); ++i) {
        const int r = launch_code_pass_generic(b->args[side][b->generic[i]], side, st, b->ctx->num_sms);
        if (r < 0) return r;
        if (r != b->gslots[side][i]) return SDL_ERR_CUDA;   // the planned reduction would miss slots
    }
    return SDL_OK;
}


size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

double model_cost(const sdl_group& g) {
    // FLOP model of one coding pass (used when not autotuning)
    const double c0 = 2.0 * std::min((double)g.p1 * g.p2 * g.n2 + (double)g.n1 * g.p1 * g.n2,
                                     (double)g.n1 * g.p1 * g.p2 + (double)g.n1 * g.p2 * g.n2);
    const double upd = (double)g.n1 * g.n2 * g.s_max * (g.s_max - 1);
    return (double)g.N * (c0 + upd);
}

int enqueue_iteration(sdl_batch* b, cudaStream_t st, bool trace) {
    sdl_ctx* c = b->ctx;
    int rc;
    auto run = [&](int kind, auto&& f) {
        if (trace) {
            Trace tr(c, kind, st);
            return f();
        }
        return f();
    };
    const int G = b->G;
    rc = run(kGram, [&] {
        return launch_multi_update_kernels(0, b->d_gram, 2 * G, b->gram_blocks, 0, c->err, st);
    });
    if (rc) return rc;
    for (int side = kSideD1; side <= kSideD2; ++side) {
        const int si = side - 1;
        rc = run(side == kSideD1 ? kCodeD1 : kCodeD2, [&] { return code_pass(b, side, st); });
        if (rc) return rc;
        rc = run(kReduce, [&] {
            return launch_multi_update_kernels(1, b->d_red[si], G, b->red_blocks[si], 0, c->err, st);
        });
        if (rc) return rc;
        rc = run(kSolve, [&] {
            return launch_multi_update_kernels(b->solve_large[si] ? 4 : 2, b->d_solve[si], G, G,
                                               b->solve_smem[si], c->err, st);
        });
        if (rc) return rc;
    }
    return run(kRescale, [&] {
        return launch_multi_update_kernels(3, b->d_rescale, G, b->rescale_blocks, 0, c->err, st);
    });
}

// A group is valid with at least one compiled tiling the multi-problem kernel
// can run (Y 16-byte aligned), or else a shape the generic kernel supports
// (*generic set, *n_ids = 0).
bool valid_group(const sdl_group& g, int* shape_ids, int* n_ids, bool* generic) {
    *n_ids = 0;
    *generic = false;
    if (!g.Y || !g.D1 || !g.D2 || !g.support || !g.coef || !g.nnz || g.N < 1) return false;
    if ((reinterpret_cast<uintptr_t>(g.Y) & 15u) == 0) {
        int all[16];
        const int n = fast_shape_variants(g.p1, g.p2, g.n1, g.n2, g.s_max, all, 16);
        for (int v = 0; v < n && *n_ids < 8; ++v)
            if (fast_variant_warps(all[v]) <= kMultiWarps) shape_ids[(*n_ids)++] = all[v];
    }
    if (*n_ids > 0) return true;
    *generic = code_shape_supported(g.p1, g.p2, g.n1, g.n2, g.s_max);
    return *generic;
}

void destroy(sdl_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->dmem) cudaFree(b->dmem);
    delete b;
}

}  // namespace

extern "C" {

int sdl_batch_create(sdl_ctx* c, const sdl_group* groups, int n_groups, int flags, void* stream,
                     sdl_batch** out) {
    if (!out) return SDL_ERR_ARG;
    *out = nullptr;
    if (!c || !groups || n_groups < 1 || n_groups > 64) return SDL_ERR_ARG;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    sdl_batch* b = new (std::nothrow) sdl_batch();
    if (!b) return SDL_ERR_WORKSPACE;
    b->ctx = c;
    b->G = n_groups;
    b->groups.assign(groups, groups + n_groups);
    const int G = n_groups;
    std::vector<std::vector<int>> variants(G);
    for (int g = 0; g < G; ++g) {
        int ids[8], n = 0;
        bool gen = false;
        if (!valid_group(groups[g], ids, &n, &gen)) {
            destroy(b);
            return SDL_ERR_UNSUPPORTED;
        }
        variants[g].assign(ids, ids + n);
        if (gen) b->generic.push_back(g);
    }
    b->n_fast = G - (int)b->generic.size();

    // ---- device memory
    const int max_slots = c->num_sms * kSlotsPerSm;
    size_t bytes = 0;
    auto take = [&](size_t n) {
        const size_t off = bytes;
        bytes += align256(n);
        return off;
    };
    std::vector<size_t> o_g1(G), o_g2(G), o_pf(G), o_pd(G), o_rf(G), o_rd(G), o_nr(G);
    for (int g = 0; g < G; ++g) {
        const sdl_group& q = groups[g];
        const size_t nf = std::max<size_t>((size_t)q.n1 * q.n1 + (size_t)q.p1 * q.n1,
                                           (size_t)q.n2 * q.n2 + (size_t)q.p2 * q.n2);
        o_g1[g] = take(sizeof(float) * q.n1 * q.n1);
        o_g2[g] = take(sizeof(float) * q.n2 * q.n2);
        o_pf[g] = take(sizeof(float) * nf * max_slots);
        o_pd[g] = take(sizeof(double) * 2 * max_slots);
        o_rf[g] = take(sizeof(float) * nf);
        o_rd[g] = take(sizeof(double) * 2);
        o_nr[g] = take(sizeof(float) * std::max(q.n1, q.n2));
    }
    const size_t o_args = take(sizeof(PassArgs) * 3 * G);
    const size_t o_cb = take(sizeof(int) * (G + 1));
    const size_t o_sh = take(sizeof(int) * G);
    const size_t o_gram = take(sizeof(GramDesc) * 2 * G);
    const size_t o_red = take(sizeof(ReduceDesc) * 2 * G);
    const size_t o_sol = take(sizeof(SolveDesc) * 2 * G);
    const size_t o_res = take(sizeof(RescaleDesc) * G);
    const size_t o_rmse = take(sizeof(double) * 2 * G);
    if (cudaMalloc(&b->dmem, bytes) != cudaSuccess) {
        cudaGetLastError();
        destroy(b);
        return SDL_ERR_WORKSPACE;
    }
    for (int g = 0; g < G; ++g) {
        b->G1.push_back(reinterpret_cast<float*>(b->dmem + o_g1[g]));
        b->G2.push_back(reinterpret_cast<float*>(b->dmem + o_g2[g]));
        b->part_f.push_back(reinterpret_cast<float*>(b->dmem + o_pf[g]));
        b->part_d.push_back(reinterpret_cast<double*>(b->dmem + o_pd[g]));
        b->red_f.push_back(reinterpret_cast<float*>(b->dmem + o_rf[g]));
        b->red_d.push_back(reinterpret_cast<double*>(b->dmem + o_rd[g]));
        b->norms.push_back(reinterpret_cast<float*>(b->dmem + o_nr[g]));
    }
    for (int side = 0; side < 3; ++side)
        b->d_args[side] = reinterpret_cast<PassArgs*>(b->dmem + o_args) + side * G;
    b->d_cta_begin = reinterpret_cast<int*>(b->dmem + o_cb);
    b->d_shape = reinterpret_cast<int*>(b->dmem + o_sh);
    b->d_gram = reinterpret_cast<GramDesc*>(b->dmem + o_gram);
    b->d_red[0] = reinterpret_cast<ReduceDesc*>(b->dmem + o_red);
    b->d_red[1] = b->d_red[0] + G;
    b->d_solve[0] = reinterpret_cast<SolveDesc*>(b->dmem + o_sol);
    b->d_solve[1] = b->d_solve[0] + G;
    b->d_rescale = reinterpret_cast<RescaleDesc*>(b->dmem + o_res);
    b->rmse_stage = reinterpret_cast<double*>(b->dmem + o_rmse);

    // ---- per-group pass arguments
    for (int side = 0; side < 3; ++side) b->args[side].resize(G);
    for (int g = 0; g < G; ++g) {
        const sdl_group& q = groups[g];
        PassArgs a;
        std::memset(&a, 0, sizeof(a));
        a.Y = q.Y;
        a.p1 = q.p1;
        a.p2 = q.p2;
        a.N = q.N;
        a.D1 = q.D1;
        a.D2 = q.D2;
        a.G1 = b->G1[g];
        a.G2 = b->G2[g];
        a.n1 = q.n1;
        a.n2 = q.n2;
        a.s = q.s_max;
        a.eps2 = q.eps > 0.f ? q.eps * q.eps : 0.f;
        a.part_f = b->part_f[g];
        a.part_d = b->part_d[g];
        a.acc_in_smem = 1;
        a.n_slots = 1;
        a.err = c->err;
        b->args[kSideD1][g] = a;                 // pass 1: partial sums only
        a.support = q.support;
        a.coef = q.coef;
        a.nnz = q.nnz;
        a.res_energy = q.res_energy;
        b->args[kCodeOnly][g] = a;               // sparse coding only
        b->args[kSideD2][g] = a;                 // pass 2: codes + partial sums
    }
    // slots the generic groups' passes will write (their reductions are sized now)
    for (int side = 0; side < 3; ++side)
        for (int g : b->generic) {
            const int r = launch_code_pass_generic(b->args[side][g], side, st, c->num_sms, true);
            if (r < 0 || r > max_slots) {
                destroy(b);
                return r < 0 ? r : SDL_ERR_UNSUPPORTED;
            }
            b->gslots[side].push_back(r);
        }
    // Gram matrices of the given dictionaries, needed by the autotuning passes
    std::vector<GramDesc> gram(2 * G);
    int blk = 0;
    for (int g = 0; g < G; ++g) {
        const sdl_group& q = groups[g];
        gram[2 * g] = GramDesc{q.D1, q.p1, q.n1, b->G1[g], blk};
        blk += (q.n1 * q.n1 + 255) / 256;
        gram[2 * g + 1] = GramDesc{q.D2, q.p2, q.n2, b->G2[g], blk};
        blk += (q.n2 * q.n2 + 255) / 256;
    }
    b->gram_blocks = blk;
    if (cudaMemcpyAsync(b->d_gram, gram.data(), sizeof(GramDesc) * 2 * G, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        launch_multi_update_kernels(0, b->d_gram, 2 * G, b->gram_blocks, 0, c->err, st) != SDL_OK) {
        cudaGetLastError();
        destroy(b);
        return SDL_ERR_CUDA;
    }

    // ---- tiling and CTA split
    b->shape.resize(G);
    b->cost_us.resize(G);
    // remembered tunings are keyed by every group's shape, count and error
    // target (its bit pattern; 0 for a fixed s), which set the groups' costs
    std::vector<long long> tkey;
    for (int g = 0; g < G; ++g) {
        const sdl_group& q = groups[g];
        uint32_t eps_bits = 0;
        if (q.eps > 0.f) std::memcpy(&eps_bits, &q.eps, sizeof eps_bits);
        for (long long v : {(long long)q.p1, (long long)q.p2, (long long)q.n1, (long long)q.n2,
                            (long long)q.s_max, (long long)q.N, (long long)eps_bits})
            tkey.push_back(v);
    }
    const sdl_ctx::BatchTune* known = nullptr;
    if ((flags & SDL_BATCH_AUTOTUNE) && !(flags & SDL_BATCH_RETUNE))
        for (const auto& t : c->batch_tunes)
            if (t.key == tkey) known = &t;
    if (known) {
        b->shape = known->shape;
        b->cost_us = known->cost_us;
        b->single_cps = known->single_cps;
        b->log_group = known->log_group;
        b->log_shape = known->log_shape;
        b->log_cps = known->log_cps;
        b->log_cost = known->log_cost;
    } else if (flags & SDL_BATCH_AUTOTUNE) {
        // each candidate is timed in the multi-problem kernel that will run it
        // (its register allocation is not the single-problem kernel's): group g
        // alone, as a one-group launch on num_sms x cps CTAs
        if (cudaMemcpyAsync(b->d_args[kSideD1], b->args[kSideD1].data(), sizeof(PassArgs) * G,
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            destroy(b);
            return SDL_ERR_CUDA;
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int g = 0; g < G; ++g) {
            float best = 1e30f;
            int best_cps = 2;
            b->cost_us[g] = (float)(model_cost(groups[g]) * 1e-6);
            if (variants[g].empty()) {   // generic kernel: nothing to tune
                b->shape[g] = -1;
                continue;
            }
            b->shape[g] = variants[g][0];
            for (int v : variants[g]) {
                const size_t sm_v = fast_smem_bytes(v, kSideD1);
                int fit = G == 1 ? fast_variant_ctas_per_sm(v, kSideD1) : multi_ctas_per_sm(sm_v, kSideD1);
                for (int sd = 0; sd < 3 && G == 1; ++sd) fit = std::min(fit, fast_variant_ctas_per_sm(v, sd));
                for (int cps = 1; cps <= std::min(2, fit); ++cps) {
                    const int grid = c->num_sms * cps;
                    if (G > 1) {
                        const int hb[3] = {0, grid, v};   // cta_begin[0..1], shape[0]
                        if (cudaMemcpy(b->d_cta_begin, hb, sizeof(int) * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
                            cudaMemcpy(b->d_shape, hb + 2, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
                            continue;
                    }
                    auto pass = [&] {
                        if (G == 1) return launch_code_pass_grid(b->args[kSideD1][g], kSideD1, v, grid, st);
                        return launch_code_multi(b->d_args[kSideD1] + g, b->d_cta_begin, b->d_shape, 1,
                                                 grid, sm_v, kSideD1, st);
                    };
                    if (pass() != SDL_OK) continue;
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < 3; ++r) pass();
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    const float us = ms * 1000.f / 3.f;
                    b->log_group.push_back(g);
                    b->log_shape.push_back(v);
                    b->log_cps.push_back(cps);
                    b->log_cost.push_back(us);
                    if (us < best) {
                        best = us;
                        b->shape[g] = v;
                        best_cps = cps;
                    }
                }
            }
            if (best < 1e30f) b->cost_us[g] = best;
            if (G == 1) b->single_cps = best_cps;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        sdl_ctx::BatchTune t{tkey, b->shape, b->cost_us, b->single_cps,
                             b->log_group, b->log_shape, b->log_cps, b->log_cost};
        bool replaced = false;
        for (auto& old : c->batch_tunes)
            if (old.key == tkey) {
                old = t;
                replaced = true;
            }
        if (!replaced) c->batch_tunes.push_back(std::move(t));
    } else {
        for (int g = 0; g < G; ++g) {
            b->shape[g] = variants[g].empty() ? -1 : variants[g][0];
            b->cost_us[g] = (float)(model_cost(groups[g]) * 1e-6);
        }
    }
    // the multi-problem kernel's groups (generic ones take no CTAs in it)
    std::vector<int> fast;
    for (int g = 0; g < G; ++g)
        if (!variants[g].empty()) fast.push_back(g);
    const int F = (int)fast.size();
    for (int side = 0; side < 3; ++side) {
        size_t m = 0;
        for (int g : fast) m = std::max(m, fast_smem_bytes(b->shape[g], side));
        b->smem[side] = m;
    }
    int cps = 2;
    for (int side = 0; side < 3 && F > 0; ++side)
        cps = std::min(cps, std::max(1, G == 1 ? fast_variant_ctas_per_sm(b->shape[0], side)
                                               : multi_ctas_per_sm(b->smem[side], side)));
    if (G == 1 && b->single_cps > 0) cps = std::min(cps, b->single_cps);
    int total = F > 0 ? c->num_sms * cps : 0;
    std::vector<int> n_cta(G, 0);
    if (F > 0) {
        std::vector<long long> cap(G, 0);
        double csum = 0.0;
        for (int g : fast) {
            cap[g] = std::max<long long>(1, (groups[g].N + 7) / 8);
            csum += b->cost_us[g];
        }
        int used = 0;
        std::vector<double> frac(G, 0.0);
        for (int g : fast) {
            const double want = std::max(1.0, total * b->cost_us[g] / std::max(csum, 1e-30));
            n_cta[g] = (int)std::min<long long>(cap[g], (long long)std::floor(want));
            n_cta[g] = std::max(1, n_cta[g]);
            frac[g] = want - std::floor(want);
            used += n_cta[g];
        }
        // hand out what is left by largest remainder (fixed order on ties)
        std::vector<int> order = fast;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return frac[x] > frac[y]; });
        for (int k = 0; used < total && k < 4 * F; ++k) {
            const int g = order[k % F];
            if (n_cta[g] < cap[g] && n_cta[g] < max_slots) {
                ++n_cta[g];
                ++used;
            }
        }
        total = 0;
        for (int g : fast) {
            n_cta[g] = std::min(n_cta[g], max_slots);
            total += n_cta[g];
        }
    }
    b->total_ctas = total;
    b->cta_begin.assign(G + 1, 0);
    for (int g = 0; g < G; ++g) b->cta_begin[g + 1] = b->cta_begin[g] + n_cta[g];

    // ---- update-stage descriptors
    std::vector<ReduceDesc> red(2 * G);
    std::vector<SolveDesc> sol(2 * G);
    std::vector<RescaleDesc> res(G);
    for (int si = 0; si < 2; ++si) {
        int rb = 0;
        size_t sm = 0;
        for (int g = 0; g < G; ++g) {
            const sdl_group& q = groups[g];
            const int p = si == 0 ? q.p1 : q.p2, n = si == 0 ? q.n1 : q.n2;
            const int nf = n * n + p * n;
            int slots = n_cta[g];
            for (size_t i = 0; i < b->generic.size(); ++i)
                if (b->generic[i] == g) slots = b->gslots[si + 1][i];
            red[si * G + g] = ReduceDesc{b->part_f[g], b->part_d[g], slots, nf, b->red_f[g],
                                         b->red_d[g], rb};
            rb += (nf + 31) / 32;
            int keep = 0;
            sm = std::max(sm, solve_smem_bytes(p, n, &keep));
            if (n > 32) b->solve_large[si] = true;
            SolveDesc d;
            d.red_f = b->red_f[g];
            d.red_d = b->red_d[g];
            d.D = si == 0 ? q.D1 : q.D2;
            d.p = p;
            d.n = n;
            d.norms = b->norms[g];
            d.inv_count = 1.0 / ((double)q.p1 * q.p2 * (double)q.N);
            d.objective_out = nullptr;
            d.rmse_out = b->rmse_stage + 2 * g + si;
            d.G_out = si == 0 ? b->G1[g] : nullptr;
            d.keep_p = keep;
            sol[si * G + g] = d;
        }
        b->red_blocks[si] = rb;
        b->solve_smem[si] = sm;
    }
    long long maxcount = 0;
    for (int g = 0; g < G; ++g) {
        const sdl_group& q = groups[g];
        res[g] = RescaleDesc{q.support, q.coef, q.N * (long long)q.s_max, q.n1, q.n2, kSideD2,
                             b->norms[g]};
        maxcount = std::max(maxcount, res[g].count);
    }
    b->rescale_blocks = (int)std::min<long long>((maxcount / 4 + 255) / 256 + 1, (long long)c->num_sms * 4);
    std::vector<PassArgs> all_args(3 * G);
    for (int side = 0; side < 3; ++side)
        std::copy(b->args[side].begin(), b->args[side].end(), all_args.begin() + side * G);
    if (cudaMemcpyAsync(b->d_args[0], all_args.data(), sizeof(PassArgs) * 3 * G,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_cta_begin, b->cta_begin.data(), sizeof(int) * (G + 1),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_shape, b->shape.data(), sizeof(int) * G, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_red[0], red.data(), sizeof(ReduceDesc) * 2 * G, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_solve[0], sol.data(), sizeof(SolveDesc) * 2 * G,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_rescale, res.data(), sizeof(RescaleDesc) * G, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        destroy(b);
        return SDL_ERR_CUDA;
    }

    // ---- one captured graph per iteration
    if (flags & SDL_BATCH_GRAPH) {
        cudaStream_t cs;
        cudaGraph_t graph = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            destroy(b);
            return SDL_ERR_CUDA;
        }
        int rc = SDL_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = SDL_ERR_CUDA;
        } else {
            rc = enqueue_iteration(b, cs, false);
            if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rc = SDL_ERR_CUDA;
        }
        if (rc == SDL_OK && cudaGraphInstantiate(&b->graph, graph, 0) != cudaSuccess) rc = SDL_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (rc != SDL_OK) {
            cudaGetLastError();
            destroy(b);
            return rc;
        }
    }
    *out = b;
    return SDL_OK;
}

int sdl_batch_destroy(sdl_batch* b) {
    if (!b) return SDL_OK;
    DeviceGuard guard(b->ctx->device);
    cudaDeviceSynchronize();
    destroy(b);
    return SDL_OK;
}

int sdl_batch_sparse_code(sdl_batch* b, void* stream) {
    if (!b) return SDL_ERR_ARG;
    sdl_ctx* c = b->ctx;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    {
        Trace tr(c, kGram, st);
        rc = launch_multi_update_kernels(0, b->d_gram, 2 * b->G, b->gram_blocks, 0, c->err, st);
    }
    if (rc) return rc;
    Trace tr(c, kCode, st);
    return code_pass(b, kCodeOnly, st);
}

int sdl_batch_iterate(sdl_batch* b, double* rmse_out, void* stream) {
    if (!b) return SDL_ERR_ARG;
    sdl_ctx* c = b->ctx;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = SDL_OK;
    if (b->graph) {
        {
            Trace tr(c, kBatchGraph, st);
            if (cudaGraphLaunch(b->graph, st) != cudaSuccess) rc = SDL_ERR_CUDA;
        }
        const int code_launches = (b->n_fast > 0 ? 1 : 0) + (int)b->generic.size();
        c->launches[kGram] += 1;
        c->launches[kCodeD1] += code_launches;
        c->launches[kCodeD2] += code_launches;
        c->launches[kReduce] += 2;
        c->launches[kSolve] += 2;
        c->launches[kRescale] += 1;
    } else {
        rc = enqueue_iteration(b, st, true);
    }
    if (rc != SDL_OK) return rc;
    if (rmse_out && cudaMemcpyAsync(rmse_out, b->rmse_stage, sizeof(double) * 2 * b->G,
                                    cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SDL_ERR_CUDA;
    return SDL_OK;
}

int sdl_batch_tuning(const sdl_batch* b, int* shape_id, int* ctas, float* cost_us) {
    if (!b) return SDL_ERR_ARG;
    for (int g = 0; g < b->G; ++g) {
        if (shape_id) shape_id[g] = b->shape[g];
        if (ctas) ctas[g] = b->cta_begin[g + 1] - b->cta_begin[g];
        if (cost_us) cost_us[g] = b->cost_us[g];
    }
    return b->G;
}

int sdl_batch_tuning_log(const sdl_batch* b, int* group, int* shape_id, int* ctas_per_sm,
                         float* cost_us, int max_entries) {
    if (!b || max_entries < 0) return SDL_ERR_ARG;
    const int n = (int)b->log_cost.size();
    for (int e = 0; e < n && e < max_entries; ++e) {
        if (group) group[e] = b->log_group[e];
        if (shape_id) shape_id[e] = b->log_shape[e];
        if (ctas_per_sm) ctas_per_sm[e] = b->log_cps[e];
        if (cost_us) cost_us[e] = b->log_cost[e];
    }
    return n;
}

}  // extern "C"
