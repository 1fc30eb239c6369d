// serve_live.cu -- the server's device-resident request queue: a persistent kernel whose
// blocks take small assignment requests (n <= 512) from a queue in host-mapped memory as
// they are published, scale each on one block (the K rows form of krows.cuh: Sec. 4.1.2
// iteration, Sec. 4.2 stop rule, p continuation of Sec. 4.1) and flag its completion in
// host-mapped memory, so that a request published while others are being scaled starts on
// the first block that frees up, without waiting for a launch.
//
// Protocol (host side in server.cpp):
//   * the host writes the request's descriptor into ring slot q % cap, then publishes it
//     by storing tail = q + 1 (release);
//   * thread 0 of a block claims the next request with a compare-and-swap on the device
//     counter head while head < tail (acquire load of tail, system scope), marks the slot
//     claimed (host-mapped), counts itself busy, reads the descriptor, and after the block
//     has scaled the request writes sweeps and status into the slot and done[slot] = q + 1
//     (release, system scope);
//   * a block leaves once it has seen stop, or has found no request for idle_ns while no
//     block of the queue was busy; the kernel ends when all its blocks have left.  A claimed
//     request is always finished before its block leaves, so a request published but not
//     claimed after every kernel of the queue has ended starts a new launch; one that
//     stays unclaimed while the running blocks are all busy starts a second kernel of the
//     queue on its own stream and slots of K.
// Every wait is on host memory or on the busy count, with a time limit.
#include <cuda_runtime.h>

#include "common.cuh"
#include "krows.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// thread 0: the next published request (its sequence number), or -1 once stop is set, or
// after idle_ns without one while no block of the queue is busy
__device__ int live_claim(const LiveArgs& A) {
    uint64_t t0 = globaltimer_ns();
    for (unsigned spin = 0;; ++spin) {
        if (ld_acquire_sys(A.stop) != 0u) return -1;
        const unsigned t = ld_acquire_sys(A.tail);
        unsigned h = *(volatile unsigned*)A.head;
        while ((int)(t - h) > 0) {
            const unsigned old = atomicCAS(A.head, h, h + 1u);
            if (old == h) {
                atomicAdd(A.busy, 1u);
                st_release_sys(A.claimed + h % A.cap, h + 1u);
                return (int)h;
            }
            h = old;
        }
        const uint64_t now = globaltimer_ns();
        if (now - t0 > A.idle_ns) {
            if (*(volatile unsigned*)A.busy == 0u) return -1;
            t0 = now;   // another block is scaling: stay for the requests that may follow
        }
        __nanosleep(spin < 64u ? 256u : 2048u);
    }
}

// one request on the block, on the narrowest K rows layout that holds its n (the shared
// state of a narrower layout is a prefix of the widest one's)
template <typename WT>
__device__ __forceinline__ void run_one(KrowsSmem<4>& sm, const LiveDesc& d, const LiveArgs& A, float* K,
                                        unsigned slot) {
    const WT* w = (const WT*)d.w;
    if (d.n <= 128)
        krows_instance<WT, 1>(*reinterpret_cast<KrowsSmem<1>*>(&sm), w, d.n, d.ld, A.P, A.n_p, A.tol, A.max_sweeps,
                              K, d.u, d.v, A.sweeps + slot, A.status + slot);
    else if (d.n <= 256)
        krows_instance<WT, 2>(*reinterpret_cast<KrowsSmem<2>*>(&sm), w, d.n, d.ld, A.P, A.n_p, A.tol, A.max_sweeps,
                              K, d.u, d.v, A.sweeps + slot, A.status + slot);
    else
        krows_instance<WT, 4>(sm, w, d.n, d.ld, A.P, A.n_p, A.tol, A.max_sweeps, K, d.u, d.v, A.sweeps + slot,
                              A.status + slot);
}

__global__ void __launch_bounds__(kKrowsThreads, 2) serve_live_kernel(LiveArgs A) {
    __shared__ KrowsSmem<4> sm;
    __shared__ int s_q;
    __shared__ LiveDesc s_d;
    krows_init(sm);
    float* K = A.kscr + (size_t)blockIdx.x * A.kscr_floats;
    for (;;) {
        if (threadIdx.x == 0) {
            s_q = live_claim(A);
            if (s_q >= 0) {
                const volatile LiveDesc* d = A.desc + (unsigned)s_q % A.cap;
                s_d.w = d->w;
                s_d.u = d->u;
                s_d.v = d->v;
                s_d.ld = d->ld;
                s_d.n = d->n;
                s_d.i16 = d->i16;
            }
        }
        __syncthreads();
        const int q = s_q;
        if (q < 0) break;
        const unsigned slot = (unsigned)q % A.cap;
        const LiveDesc d = s_d;
        if (d.i16) run_one<int16_t>(sm, d, A, K, slot);
        else run_one<int32_t>(sm, d, A, K, slot);
        // the potentials (device memory, every thread) before the flag the host reads
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys(A.done + slot, (unsigned)q + 1u);
            atomicSub(A.busy, 1u);
        }
    }
}

}  // namespace

size_t live_slot_floats() { return (size_t)512 * 512; }

sa_status live_launch(const LiveArgs& args, int grid, cudaStream_t st) {
    if (grid <= 0 || args.cap == 0 || args.kscr_floats < live_slot_floats()) {
        set_error("live queue: bad launch arguments");
        return SA_E_INVALID;
    }
    serve_live_kernel<<<grid, kKrowsThreads, 0, st>>>(args);
    count_launch();
    SA_CUDA(cudaGetLastError());
    return SA_OK;
}

}  // namespace sa
