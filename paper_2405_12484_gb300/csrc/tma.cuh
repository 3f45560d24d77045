// Bulk asynchronous copies (cp.async.bulk, global -> shared) completed on
// shared-memory mbarriers, with bounded waits, for the streaming kernels of
// sm_103a.  A wait gives up after kWaitNs (1 s) of %globaltimer or, when an
// abort flag is given, as soon as the CTA is marked aborted; the caller then
// reports ERR_TIMEOUT and drains its own copies in flight before it exits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdg {
namespace tma {

constexpr unsigned long long kWaitNs = 1000000000ull;

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

static __device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

static __device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false when it ran out (1 s) or, if `abort` is given, when the
// CTA was marked aborted meanwhile.  Waits for copies still in flight pass no
// abort flag: they must not end early.
static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int* abort = nullptr) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtime_ns();
    for (unsigned k = 1;; ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 63u) == 0) {
            if (abort && *reinterpret_cast<const volatile int*>(abort)) return false;
            if (gtime_ns() - t0 > kWaitNs) return false;
        }
    }
}

static __device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace tma
}  // namespace pdg
