// cluster.cuh -- bounded synchronisation of the CTAs of a thread-block cluster.
#pragma once

#include <cstdint>

namespace cbfm {

__device__ __forceinline__ uint32_t cl_su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t cl_time_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Initialise this CTA's two cluster mbarriers (one arrival per CTA per
// phase).  Step k of a loop synchronises on bar[k & 1], phase parity
// (k >> 1) & 1: a CTA can arrive for step k + 2 only after every CTA has
// arrived for step k + 1, i.e. after every barrier has completed step k, so an
// early arrival is never counted in the wrong phase.  Call from one thread;
// make every CTA's barriers visible (hardware cluster barrier, reached
// unconditionally) before the first arrival.
__device__ __forceinline__ void cl_bar_init(uint64_t *bar, int ncta) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cl_su32(bar)), "r"(ncta) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cl_su32(bar + 1)), "r"(ncta) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// cl_arrive(bar, k, ncta): threads 0 .. ncta-1 each arrive (release,
// cluster scope) for step k on CTA threadIdx.x; call it after a
// __syncthreads that orders the CTA's writes before the arrivals.
// cl_wait(bar, k, ...): thread 0 waits (acquire) for step k, giving up after
// `limit_ns` (sets *abort_flag and *err); all threads call it and see the
// other CTAs' writes made before their arrivals.
__device__ __forceinline__ void cl_arrive(uint64_t *bar, int k, int ncta) {
    if ((int)threadIdx.x < ncta) {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(remote)
                     : "r"(cl_su32(bar + (k & 1))), "r"((int)threadIdx.x));
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
    }
}

__device__ __forceinline__ bool cl_wait(uint64_t *bar, int k, int *abort_flag, int *err,
                                        uint64_t limit_ns = 1000000000ull) {
    if (threadIdx.x == 0) {
        const uint32_t local = cl_su32(bar + (k & 1)), parity = (uint32_t)(k >> 1) & 1u;
        uint32_t ok = 0;
        const uint64_t t0 = cl_time_ns();
        while (true) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(local), "r"(parity)
                : "memory");
            if (ok || cl_time_ns() - t0 > limit_ns) break;
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 1);
        }
    }
    __syncthreads();
    return *(volatile int *)abort_flag == 0;
}

// Whole-cluster synchronisation for step k: every CTA's writes before the
// call are visible to every CTA after it.  All threads call it.
__device__ __forceinline__ bool cl_sync(uint64_t *bar, int k, int ncta, int *abort_flag, int *err,
                                        uint64_t limit_ns = 1000000000ull) {
    __syncthreads();   // the CTA's writes happen before the release-arrivals (cumulative)
    cl_arrive(bar, k, ncta);
    return cl_wait(bar, k, abort_flag, err, limit_ns);
}

}  // namespace cbfm
