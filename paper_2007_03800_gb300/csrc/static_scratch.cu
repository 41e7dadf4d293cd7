// sdl_sparse_code_static: the 2D-OMP sparse coder without a context and
// without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running, or cannot hold a library context.  Examples are a host
// application or server that hands out all GPU memory from its own pre-sized
// pool and forbids libraries from calling cudaMalloc, and latency-critical
// loops where cudaMalloc's implicit device synchronisation, and its possible
// failure under memory pressure, are not acceptable.
//
// The only scratch the coder needs beyond the caller's inputs and outputs is
// the two Gram matrices G1 = D1^T D1 and G2 = D2^T D2.  They live in the
// file-scope device array below, which every GPU that loads this library
// holds until the process exits.
#include <atomic>

#include "sdl_internal.cuh"

namespace {

// Capacity of the static scratch, in floats: G1 (n1*n1) and G2 (n2*n2) must
// fit together, i.e. n1*n1 + n2*n2 <= 8192 (32 KiB; covers every pair shape
// up to 64 x 64 atoms per side).
constexpr int kStaticGramFloats = 8192;

static __device__ __align__(256) float g_static_gram[kStaticGramFloats];
// Error word of the allocation-free calls on this device (SDL_OK or the first
// device-side error since it was last read by sdl_static_status).
static __device__ int g_static_err;

constexpr int kMaxDevices = 64;
// Device addresses of g_static_gram and g_static_err per device ordinal,
// looked up once per device (with that device current) on its first call.
// They stay valid for the life of the device's primary context: after a
// cudaDeviceReset of that device the library must be reloaded.
std::atomic<float*> g_static_addr[kMaxDevices];
std::atomic<int*> g_static_err_addr[kMaxDevices];

int static_scratch(int device, float** out, int** err) {
    if (device < 0 || device >= kMaxDevices) return SDL_ERR_ARG;
    float* p = g_static_addr[device].load(std::memory_order_acquire);
    int* e = g_static_err_addr[device].load(std::memory_order_acquire);
    if (!p || !e) {
        void* addr = nullptr;
        void* eaddr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_static_gram) != cudaSuccess || !addr ||
            cudaGetSymbolAddress(&eaddr, g_static_err) != cudaSuccess || !eaddr) {
            cudaGetLastError();
            return SDL_ERR_CUDA;
        }
        p = static_cast<float*>(addr);
        e = static_cast<int*>(eaddr);
        g_static_addr[device].store(p, std::memory_order_release);
        g_static_err_addr[device].store(e, std::memory_order_release);
    }
    *out = p;
    *err = e;
    return SDL_OK;
}

}  // namespace

extern "C" int sdl_sparse_code_static(const float* Y, int p1, int p2, int64_t N, const float* D1,
                                      int n1, const float* D2, int n2, int s_max, float eps,
                                      int32_t* support, float* coef, int32_t* nnz,
                                      float* res_energy, void* stream) {
    using namespace sdl;
    if (p1 < 1 || p2 < 1 || n1 < 1 || n2 < 1 || N < 0 || s_max < 1 || !D1 || !D2)
        return SDL_ERR_ARG;
    if (N > 0 && (!Y || !support || !coef || !nnz)) return SDL_ERR_ARG;
    if (s_max > kMaxS || s_max > p1 * p2 || s_max > n1 * n2) return SDL_ERR_ARG;
    if (!code_shape_supported(p1, p2, n1, n2, s_max)) return SDL_ERR_UNSUPPORTED;
    if ((long long)n1 * n1 + (long long)n2 * n2 > kStaticGramFloats) return SDL_ERR_CAPACITY;
    if (N == 0) return SDL_OK;

    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return SDL_ERR_CUDA;
    }
    float* scratch = nullptr;
    int* err = nullptr;
    int rc = static_scratch(device, &scratch, &err);
    if (rc != SDL_OK) return rc;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return SDL_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float* G1 = scratch;
    float* G2 = scratch + n1 * n1;
    // Both Grams are fully rewritten before the coding pass reads them, so
    // nothing left over from an earlier call is used.
    launch_gram(D1, p1, n1, G1, st);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;
    launch_gram(D2, p2, n2, G2, st);
    if (cudaGetLastError() != cudaSuccess) return SDL_ERR_CUDA;

    PassArgs a{};
    a.Y = Y;
    a.p1 = p1;
    a.p2 = p2;
    a.N = N;
    a.D1 = D1;
    a.D2 = D2;
    a.G1 = G1;
    a.G2 = G2;
    a.n1 = n1;
    a.n2 = n2;
    a.s = s_max;
    a.eps2 = eps > 0.f ? eps * eps : 0.f;
    a.support = support;
    a.coef = coef;
    a.nnz = nnz;
    a.res_energy = res_energy;
    a.n_slots = 1;
    a.err = err;       // read by sdl_static_status
    rc = launch_code_pass(a, kCodeOnly, st, num_sms);
    return rc < 0 ? rc : SDL_OK;
}

extern "C" int sdl_static_status(void* stream) {
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return SDL_ERR_CUDA;
    }
    float* scratch = nullptr;
    int* err = nullptr;
    int rc = static_scratch(device, &scratch, &err);
    if (rc != SDL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int v = SDL_OK;
    if (cudaMemcpyAsync(&v, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SDL_ERR_CUDA;
    }
    return v;
}
