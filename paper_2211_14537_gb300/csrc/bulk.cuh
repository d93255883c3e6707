// bulk.cuh -- one-dimensional TMA bulk copies global -> shared memory
// (cp.async.bulk) completing on an mbarrier, for the kernels that stage a
// contiguous table or vector before computing on it: one instruction moves the
// whole block, so its latency is paid once instead of once per load loop
// iteration.
//
// Rules of the copy: source and destination 16-byte aligned, size a multiple
// of 16 bytes, at most 2^20 - 1 bytes in flight per barrier phase.  Every wait
// is bounded in wall-clock time (kWaitLimitNs of the global timer): the wait
// returns false, and the caller reports VPX_ERR_TIMEOUT instead of computing.
#pragma once

#include <cstdint>

namespace vpx {

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // one second

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// poll phase `parity` of an mbarrier until it completes (true) or limit_ns of
// wall-clock time pass (false); sleep_ns > 0 backs off between polls
__device__ inline bool mbar_wait_bounded(uint32_t bar_addr, uint32_t parity, unsigned long long limit_ns,
                                         unsigned sleep_ns) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {   // the clock bounds it; the count too
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar_addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return false;
}

__device__ inline uint32_t bulk_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// one thread: initialise the barrier (one arrival per phase)
__device__ inline void bulk_bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bulk_smem_addr(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one thread: announce the bytes of this phase (the arrival of the phase)
__device__ inline void bulk_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bulk_smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// one thread: start a copy that completes `bytes` of the phase's transaction count
__device__ inline void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            bulk_smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(bulk_smem_addr(bar))
        : "memory");
}

// all threads: wait for phase `parity` of the barrier; false on timeout
__device__ inline bool bulk_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_bounded(bulk_smem_addr(bar), parity, kWaitLimitNs, 0);
}

}  // namespace vpx
