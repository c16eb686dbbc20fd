// Element operators staged into shared memory by bulk asynchronous copies (cp.async.bulk, the
// TMA's unstructured form) completing on an mbarrier.
//
// A block of the Schur-complement kernels handles EPB consecutive elements, whose S^{-1} blocks
// and node numbers are two contiguous ranges per element in global memory.  One warp issues one
// copy of each per element (to rows padded for FP32 so that the two elements of a warp read
// different banks); the other threads meanwhile issue their own loads (the stage data, the
// traces), and the block then reads the operators from shared memory.  Every wait gives up after
// kStagedWaitCap polls: the block then ORs kStagedWaitCode into the handle's device error word,
// waits (again bounded) for its copies to land and skips its work, so a copy that never completes
// ends the launch with an error the host reads instead of a hang.
#pragma once

#include "schur.h"

namespace hdgdg {

constexpr int kStagedWaitCap = 1 << 22;
constexpr unsigned kStagedWaitCode = 4u;

__device__ __forceinline__ unsigned smem_addr_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void staged_mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void staged_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void staged_bulk_copy(void* smem, const void* gmem, unsigned bytes,
                                                 unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr_u32(smem)),
                 "l"(gmem), "r"(bytes), "r"(smem_addr_u32(bar))
                 : "memory");
}

// true once the mbarrier's first phase has completed, false after kStagedWaitCap polls
__device__ __forceinline__ bool staged_wait_phase0(unsigned long long* bar) {
    for (int k = 0; k < kStagedWaitCap; ++k) {
        unsigned ok = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr_u32(bar))
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int P, int EPB, class A>
struct StagedOps {
    using T = typename A::T;
    static constexpr int Np = P * P;
    static constexpr int PAD = sizeof(T) == 4 ? 16 : 0;   // FP32 rows: the next element 16 banks on
    static constexpr int SLD = Np * Np + PAD, ALD = 4 * Np + PAD;
    static constexpr unsigned BS = Np * Np * sizeof(T), BA = 4 * Np * sizeof(T);
    static constexpr bool kFits = BS % 16 == 0 && BA % 16 == 0 && (SLD * sizeof(T)) % 16 == 0;
    alignas(16) T S[EPB * SLD];
    alignas(16) T aux[EPB * ALD];
    unsigned long long bar;

    // Start the copies of elements e0 .. e0 + ne - 1 (every thread of the block calls it).
    __device__ __forceinline__ void issue(const T* __restrict__ Sg, const T* __restrict__ auxg, int e0, int ne) {
        static_assert(kFits, "staged copies need 16-byte pieces");
        if (threadIdx.x == 0) staged_mbar_init(&bar);
        __syncthreads();
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) staged_expect_tx(&bar, (unsigned)ne * (BS + BA));
            __syncwarp();
            for (int le = threadIdx.x; le < ne; le += 32) {
                staged_bulk_copy(&S[le * SLD], Sg + (size_t)(e0 + le) * Np * Np, BS, &bar);
                staged_bulk_copy(&aux[le * ALD], auxg + (size_t)(e0 + le) * 4 * Np, BA, &bar);
            }
        }
    }

    // Wait for them; false (for the whole block) if the wait ran out -- err then carries the code.
    __device__ __forceinline__ bool wait(unsigned* err) {
        const bool ok = __syncthreads_and(staged_wait_phase0(&bar) ? 1 : 0) != 0;
        if (!ok) {
            if (threadIdx.x == 0 && err) atomicOr(err, kStagedWaitCode);
            (void)staged_wait_phase0(&bar);   // let copies still in flight land before the block leaves
        }
        return ok;
    }

    __device__ __forceinline__ void load_node(SchurNode<A>& nd, int le, int n) const {
        const T* ax = aux + le * ALD;
        nd.rd = ax[n];
        nd.ncx = ax[Np + n];
        nd.ncy = ax[2 * Np + n];
        nd.pb = ax[3 * Np + n];
    }
    // (S^{-1})_{n m} of element le
    __device__ __forceinline__ T srow(int le, int n, int m) const { return S[le * SLD + m * Np + n]; }
};

}  // namespace hdgdg
