// flb_tma.cuh -- Tensor Memory Accelerator copies and mbarriers (sm_90+ PTX),
// used by the pipelined FP32 step kernel. Every wait is bounded: after
// kWaitCycles without progress the caller gets `false` and must record a
// timeout and stop issuing work.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace flb {

constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Count one release of a stage (acquire-release at CTA scope: the thread that
// makes the last release also observes every earlier releaser's reads of the
// stage as complete). Returns the count before this release.
__device__ __forceinline__ uint32_t release_count(uint32_t* cnt) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;"
                 : "=r"(old)
                 : "r"(smem_u32(cnt))
                 : "memory");
    return old;
}

// Orders this thread's view of shared memory before its later asynchronous-proxy
// (tensor copy) accesses: used before a copy into a stage released through a
// counter rather than an mbarrier.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A warp releases a stage: every lane has finished its reads (syncwarp), then
// lane 0 arrives, predicated rather than branched around.
__device__ __forceinline__ void warp_arrive(uint64_t* bar, int lane_id) {
    __syncwarp();
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.eq.s32 p, %1, 0;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_u32(bar)),
        "r"(lane_id)
        : "memory");
}

// try_wait: a thread whose phase has not completed is parked by the hardware
// for up to its own time limit before the call returns false, so a waiting
// warp takes few issue slots from the warps that compute. (A 1 ms suspend-time
// hint measured 0.3-0.5 % slower in the pipelined steps.)
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
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

// Wait for the completion of the phase with the given parity; false after
// `limit` cycles without it.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, kWaitCycles);
}

// Wait for warps that run ahead of the colliding warps (sampler warps, the
// producer) and would otherwise poll for most of a tile: between polls the
// warp sleeps, with the pause doubling from 32 ns up to kSleepMaxNs, so it
// takes almost no issue slots from the colliding warps. False on timeout.
constexpr unsigned kSleepMaxNs = 1024;

__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (!mbar_try_wait(bar, parity)) {
        __nanosleep(ns);
        ns = ns < kSleepMaxNs ? 2 * ns : kSleepMaxNs;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// 2D tiled TMA load of the box at (x, y) into shared memory, completing on bar.
// x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Barrier among the first `count` threads of the CTA (named barrier `id`).
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace flb
