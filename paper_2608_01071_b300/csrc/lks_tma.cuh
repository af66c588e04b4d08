// Tensor-memory-accelerator (TMA) tile loads completing on shared-memory mbarriers (sm_90 and later PTX), with
// waits bounded in time.
//
// The plane-pair kernels fetch a raw tile of a state (4 fields) for each plane: one 4-D tensor copy
// (x, y, z, field) issued by one thread replaces the per-thread 16-byte asynchronous copies, their address
// arithmetic and their completion groups.  The tensor map lives in the kernel's parameter space
// (__grid_constant__); its box is the kernel's raw region, so that the copy lands in the layout the kernels
// index ([field][row][column]).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "lks_common.cuh"

namespace lks {

// Status bit set in Geom::status when a bounded device-side wait expired (reported as LKS_ETIMEOUT).
constexpr unsigned kStatusTimeout = 1u;
// Default limit of one wait, and the limit of the wait for copies still in flight after a timeout (ns).
constexpr unsigned long long kWaitNsDefault = 1000000000ull;
constexpr unsigned long long kDrainNs = 2000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

// Make initialised barriers visible to the asynchronous proxy (the tensor copies that complete on them).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive once and add `bytes` to the transaction count of the current phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with `parity` to complete, for at most `limit_ns`; false when it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(b, parity)) return true;
        if (global_ns() - t0 >= limit_ns) return false;
    }
}

// 4-D tiled copy of the box at (x, y, z, w) into shared memory, completing on barrier b.  x times the element size
// must be a multiple of 16 bytes; dst 128-byte aligned.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int x, int y, int z, int w, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(b))
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* tm) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// Pipeline of raw plane pairs fetched by tensor copies: pair jj completes on barrier jj mod 2 (phase jj / 2).
// One thread of the block issues and waits; a barrier of the block then publishes the data to the other threads.
struct PairTma {
    uint64_t bar[3];  // two pair slots, and one that nothing completes (the diagnostic wait)
    int bad;          // a wait expired: the block leaves

    __device__ __forceinline__ void init() {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        bad = 0;
        mbar_init_fence();
    }
    // the issuing thread: wait for pairs first .. last; on a timeout, wait (kDrainNs at most) for the copies still in flight,
    // record the timeout and mark the block
    __device__ __forceinline__ void wait(int first, int last, const Geom& g) {
        const unsigned long long lim = g.wait_ns ? g.wait_ns : kWaitNsDefault;
        bool ok = !(g.wait_probe && !mbar_wait(&bar[2], 0, lim));
        for (int jj = first; jj <= last; ++jj) {
            uint64_t* b = &bar[jj & 1];
            const unsigned par = (unsigned)(jj >> 1) & 1u;
            if (ok) ok = mbar_wait(b, par, lim);
            if (!ok) mbar_wait(b, par, kDrainNs);
        }
        if (!ok) {
            bad = 1;
            if (g.status != nullptr) atomicOr(g.status, kStatusTimeout);
        }
    }
};

}  // namespace lks
