// common.cuh -- device helpers shared by the libsa kernels (sm_103a).
//
// SFU wrappers, integer-weight decoding, warp reductions, shared-memory barriers for the
// bulk-copy engine, and a bounded group barrier for persistent cooperative kernels.
// Every spin-wait here is bounded by a wall-clock limit; on expiry it records an error
// code and returns false so the kernel can drain and exit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sa_internal.h"

namespace sa {

// ---- special-function unit ---------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- weight decoding -----------------------------------------------------------------
// A non-negative integer below 2^23 placed in the mantissa of 2^23 is exact:
// float(k) = bits(0x4B000000 | k) - 2^23.  For a 32-bit word holding two int16 weights
// the byte permute builds both patterns without a conversion instruction.
__device__ __forceinline__ float lo16_to_float(uint32_t word) {
    return __uint_as_float(__byte_perm(word, 0x4B00u, 0x5410u)) - 8388608.0f;
}
__device__ __forceinline__ float hi16_to_float(uint32_t word) {
    return __uint_as_float(__byte_perm(word, 0x4B00u, 0x5432u)) - 8388608.0f;
}
__device__ __forceinline__ float w_to_float(int16_t w) { return (float)w; }
__device__ __forceinline__ float w_to_float(int32_t w) { return (float)w; }

// ---- reductions --------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---- timing --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- global-memory acquire/release -------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier over `nblocks` co-resident blocks (cooperative launch).  bar[0] counts
// arrivals, bar[1] is the generation.  Returns false if the wait exceeded timeout_ns
// or another block already reported an error; *err then holds a kErr* code.
__device__ __forceinline__ bool group_barrier(unsigned* bar, unsigned nblocks, int* err,
                                              uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire(bar + 1);
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            st_release(bar + 1, gen + 1);
        } else {
            uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire(bar + 1) == gen) {
                if ((++spins & 63u) == 0) {
                    if (*(volatile int*)err != 0) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        atomicCAS(err, 0, kErrTimeout);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(20);
            }
        }
        if (*(volatile int*)err != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- shared-memory barriers and the bulk-copy (TMA) engine ----------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
// Invalidate an mbarrier (no pending arrivals or transactions) before re-initialising it.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Arrive on a CTA mbarrier (release at CTA scope: prior shared stores are visible to
// threads that complete a wait on this phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
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
// Bounded wait on phase `parity` of an mbarrier; false on timeout (error recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err,
                                          uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
            atomicCAS(err, 0, kErrTimeout);
            return false;
        }
    }
    return true;
}
// 1-D bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// L2 eviction policy "evict first" for the copies that carry it: lines read that way are
// the first candidates for replacement, so lines read without it stay longer.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                              uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace sa
