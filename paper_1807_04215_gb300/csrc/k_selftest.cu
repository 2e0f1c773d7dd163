// Self-test of the bounded device-side wait used by the TMA-staged passes: one
// block waits on an mbarrier whose phase never completes (no arrival is ever
// made). The wait gives up after its iteration limit, the kernel records the
// timeout in the status word and returns. Used only by the failure-detection
// test; no GPU fault, trap or unbounded spin is involved.
#include "gridspt_internal.h"

namespace gridspt {

__global__ void k_wait_selftest(int* status) {
    __shared__ uint64_t bar;
    const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    __syncthreads();
    bool done = false;
    for (unsigned it = 0; it < (1u << 14) && !done; ++it) {
        unsigned d;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(d) : "r"(a) : "memory");
        done = d != 0;
        __nanosleep(64);
    }
    if (!done && threadIdx.x == 0) atomicOr(status, kStatusWaitSelftest);
}

cudaError_t launch_wait_selftest(int* status, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

}  // namespace gridspt
