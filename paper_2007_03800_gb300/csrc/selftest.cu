// Failure-detection self-test: exercises the bounded-wait path that every
// waiting kernel of the library uses (an mbarrier wait limited by the SM
// clock, after which the kernel records SDL_ERR_TIMEOUT and returns), on a
// barrier that nothing ever completes.  The GPU stays usable: the kernel
// only spins for the requested number of cycles.
#include "ctx.cuh"

namespace {

__global__ void timeout_probe_kernel(long long max_cycles, int* err) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(&bar));
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // nothing arrives on `bar`: phase 0 never completes
    const long long t0 = clock64();
    bool done = false;
    while (!done && clock64() - t0 < max_cycles) {
        unsigned d;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(d)
            : "r"(a), "r"(0u)
            : "memory");
        done = d != 0;
    }
    if (!done) sdl::record_error(err, SDL_ERR_TIMEOUT);
}

}  // namespace

extern "C" int sdl_selftest_timeout(sdl_ctx* c, long long max_cycles, void* stream) {
    if (!c || max_cycles < 1 || max_cycles > (1ll << 31)) return SDL_ERR_ARG;
    sdl::DeviceGuard g(c->device);
    timeout_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(max_cycles, c->err);
    return cudaGetLastError() == cudaSuccess ? SDL_OK : SDL_ERR_CUDA;
}
