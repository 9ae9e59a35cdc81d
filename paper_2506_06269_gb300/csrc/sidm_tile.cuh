// sidm_tile.cuh -- per-warp staging of one candidate leaf (32 x 16 B or
// 32 x 32 B) into shared memory, and round-to-nearest arithmetic helpers.
//
// Two staging paths with identical results:
//   plain: each lane issues one coalesced 128-bit (or 2 x 128-bit) load;
//   TMA  : lane 0 issues a 1-D bulk asynchronous copy global -> shared
//          (cp.async.bulk ... mbarrier::complete_tx) and the warp waits on the
//          mbarrier phase with an iteration limit; on timeout the status bit
//          SIDM_DEV_WAIT_TIMEOUT is raised instead of hanging.
// Source and destination are 16-byte aligned and the size is a multiple of 16.
#pragma once

#include "sidm_internal.cuh"

namespace sidm {

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float sqrt_ru(float a) { return __fsqrt_ru(a); }
__device__ __forceinline__ double sqrt_ru(double a) { return __dsqrt_ru(a); }

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

constexpr unsigned kWaitLimit = 1u << 22;

// NBUF = 2: the staged tile and a second buffer for its shifted copy;
// NBUF = 1: the caller shifts the tile in place (each lane its own entry).
template <class R, bool TMA, int NBUF = 2>
struct TileStageT {
    using V = typename Vec4<R>::T;
    static constexpr size_t bytes() { return NBUF * 32 * sizeof(V) + 16; }
    unsigned char* base;
    uint32_t phase;
    bool timed_out;
    __device__ explicit TileStageT(unsigned char* b) : base(b), phase(0u), timed_out(false) {}
    __device__ V* raw() const { return (V*)base; }
    __device__ V* shifted() const { return (V*)(base + (NBUF - 1) * 32 * sizeof(V)); }
    __device__ unsigned long long* bar() const { return (unsigned long long*)(base + NBUF * 32 * sizeof(V)); }

    __device__ void init(int lane)
    {
        if constexpr (TMA) {
            if (lane == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar())), "r"(1u) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
        }
        __syncwarp();
    }

    __device__ bool wait(uint32_t ph)
    {
        for (unsigned it = 0; it < kWaitLimit; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok) : "r"(smem_u32(bar())), "r"(ph) : "memory");
            if (ok) return true;
        }
        return false;
    }

    // Stage 32 consecutive V from src; returns the shared copy.
    __device__ const V* load(const V* __restrict__ src, int lane, DevCounters* cnt)
    {
        if constexpr (!TMA) {
            raw()[lane] = src[lane];
            __syncwarp();
            return raw();
        } else {
            __syncwarp();   // every lane is done with the previous contents
            if (lane == 0) {
                const uint32_t nbytes = 32u * (uint32_t)sizeof(V);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(smem_u32(bar())), "r"(nbytes) : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(smem_u32(raw())), "l"(src), "r"(nbytes), "r"(smem_u32(bar())) : "memory");
            }
            if (!wait(phase)) {
                timed_out = true;
                if (lane == 0) raise_status(cnt, SIDM_DEV_WAIT_TIMEOUT);
            }
            phase ^= 1u;
            __syncwarp();
            return raw();
        }
    }

    __device__ void finish(int lane, DevCounters* cnt)
    {
        if constexpr (TMA) {
            // a copy that timed out may still be in flight: wait once more (bounded)
            if (timed_out && !wait(phase ^ 1u) && lane == 0) raise_status(cnt, SIDM_DEV_WAIT_TIMEOUT);
        }
        (void)lane; (void)cnt;
    }
};

template <class R>
using TileStage = TileStageT<R, false>;

}  // namespace sidm
