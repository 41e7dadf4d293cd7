// The library context and its host-side helpers (shared by the C ABI
// translation units).
#pragma once

#include <vector>

#include "sdl_internal.cuh"

struct sdl_ctx {
    int device = 0;
    int num_sms = 0;
    int* err = nullptr;          // device error word
    float* G1 = nullptr;         // Gram matrices of the current dictionaries
    float* G2 = nullptr;
    float* part_f = nullptr;     // partial-sum slots
    double* part_d = nullptr;
    float* red_f = nullptr;      // reduced sums
    double* red_d = nullptr;
    float* norms = nullptr;      // column norms of the last solve
    float* rec = nullptr;        // reconstructed patches (patch averaging)
    size_t cap_rec = 0;
    char* learn = nullptr;       // learned-coder workspace
    size_t cap_learn = 0;
    double* ssim_part = nullptr; // per-block SSIM sums
    size_t cap_ssim = 0;
    float* G3 = nullptr;         // three-mode Gram matrices (G1 | G2 | G3 | spare)
    size_t cap_g3 = 0;
    // precision extension
    int prec = 0;                // SDL_PREC_* flags
    void* Yb = nullptr;          // BF16 signals (N x Kp)
    void* KT = nullptr;          // BF16 Kronecker dictionary rows (n1n2 x Kp)
    float* C0 = nullptr;         // tensor-core correlations (N x n1n2)
    size_t cap_yb = 0, cap_kt = 0, cap_c0 = 0;
    unsigned long long* rescored = nullptr;
    size_t cap_g1 = 0, cap_g2 = 0, cap_part = 0, cap_slots = 0, cap_red = 0, cap_redd = 0,
           cap_norms = 0;
    // coder tilings pinned per shape (sdl_tune_tiling / sdl_set_tiling) and
    // the measurements of the last sdl_tune_tiling
    struct Pin {
        int p1, p2, n1, n2, s, id, cps;
    };
    std::vector<Pin> pins;
    struct TuneRec {
        int id, cps;
        float us;
    };
    std::vector<TuneRec> tune_log;
    // batch autotuning results, remembered per group signature (shapes, sizes,
    // stopping rule) so that a batch of the same groups is not re-timed
    struct BatchTune {
        std::vector<long long> key;
        std::vector<int> shape;
        std::vector<float> cost_us;
        int single_cps;
        std::vector<int> log_group, log_shape, log_cps;
        std::vector<float> log_cost;
    };
    std::vector<BatchTune> batch_tunes;
    // tracing: launch counters and (optionally) one event pair per launch
    struct Rec {
        int kind;
        cudaEvent_t beg, end;
    };
    bool timing = false;
    std::vector<Rec> recs;           // event pool, reused
    size_t n_recs = 0;               // records in use
    int64_t launches[SDL_NUM_KERNEL_KINDS] = {};
};

namespace sdl {

enum Kind {
    kGram = 0, kCode, kCodeD1, kCodeD2, kAccD1, kAccD2, kReduce, kSolve, kRescale, kMemset,
    kBatchGraph, kMlp, kAdam, kTopk, kShortlist, kTcCorr, kOrthoCode, kProcrustes
};

// Grow the context's Gram, partial-sum and reduction buffers for a problem
// shape (api.cu).
int ctx_workspace(sdl_ctx* c, int p1, int p2, int n1, int n2);
constexpr size_t kMaxRecs = 1 << 16;

// Bracket one launch of `kind` on `st` with timing events (when enabled).
struct Trace {
    sdl_ctx* c;
    cudaStream_t st;
    sdl_ctx::Rec* rec = nullptr;
    Trace(sdl_ctx* c_, int kind, cudaStream_t st_) : c(c_), st(st_) {
        c->launches[kind] += 1;
        if (!c->timing || c->n_recs >= kMaxRecs) return;
        if (c->n_recs == c->recs.size()) {
            sdl_ctx::Rec r{kind, nullptr, nullptr};
            if (cudaEventCreate(&r.beg) != cudaSuccess || cudaEventCreate(&r.end) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            c->recs.push_back(r);
        }
        rec = &c->recs[c->n_recs++];
        rec->kind = kind;
        cudaEventRecord(rec->beg, st);
    }
    ~Trace() {
        if (rec) cudaEventRecord(rec->end, st);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace sdl
