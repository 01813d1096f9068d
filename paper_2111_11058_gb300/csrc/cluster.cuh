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

// Initialise this CTA's cluster mbarrier (one arrival per CTA per phase).
// Call from one thread; make every CTA's barrier visible (hardware cluster
// barrier, reached unconditionally) before the first cl_sync.
__device__ __forceinline__ void cl_bar_init(uint64_t *bar, int ncta) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cl_su32(bar)), "r"(ncta) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Cluster-wide synchronisation on the mbarrier `bar` of every CTA (ncta CTAs,
// phase parity `parity`): the CTA's memory writes (shared, distributed shared
// and global) before the call are visible to every CTA of the cluster after
// it.  Thread 0 arrives remotely on each CTA's barrier (release, cluster
// scope) and waits on its own (acquire); the wait gives up after `limit_ns`,
// sets *abort_flag and *err, and returns false.  All threads of the CTA call it.
__device__ __forceinline__ bool cl_sync(uint64_t *bar, uint32_t parity, int ncta, int *abort_flag, int *err,
                                        uint64_t limit_ns = 1000000000ull) {
    __syncthreads();   // the CTA's writes happen before thread 0's release-arrives (cumulative)
    if (threadIdx.x == 0) {
        const uint32_t local = cl_su32(bar);
        for (int r = 0; r < ncta; ++r) {
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
        }
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
    __syncthreads();   // the others' writes, acquired by thread 0, are visible to the CTA
    return *(volatile int *)abort_flag == 0;
}

}  // namespace cbfm
