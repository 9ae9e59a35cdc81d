// sidm_tile.cuh -- per-warp staging of one candidate leaf (32 x 16 B or
// 32 x 32 B) into shared memory, and round-to-nearest arithmetic helpers.
//
// Two staging paths with identical results:
//   plain: each lane issues one coalesced 128-bit (or 2 x 128-bit) load;
//   TMA  : lane 0 issues a 1-D bulk asynchronous copy global -> shared
//          (cp.async.bulk ... mbarrier::complete_tx) and the warp waits on the
//          mbarrier phase for at most kWaitNs of wall-clock time (%globaltimer).
//          On a timeout the status bit SIDM_DEV_WAIT_TIMEOUT is raised, the
//          warp stops arming the barrier and issuing copies, and every later
//          leaf is read with plain loads straight into registers (never into
//          the buffer the late copy may still write); finish() waits, again
//          bounded, for that copy before the CTA may exit.
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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wall-clock limit of one wait on a bulk copy (a 512-byte copy lands in about a
// microsecond), and a backstop on the number of polls
constexpr unsigned long long kWaitNs = 2000000ull;      // 2 ms
constexpr unsigned kWaitPolls = 1u << 24;

// NBUF = 2: the staged tile and a second buffer for its shifted copy;
// NBUF = 1: the caller shifts the tile in place (each lane its own entry).
template <class R, bool TMA, int NBUF = 2>
struct TileStageT {
    using V = typename Vec4<R>::T;
    static constexpr size_t bytes() { return NBUF * 32 * sizeof(V) + 16; }
    unsigned char* base;
    uint32_t phase;
    bool timed_out;      // warp-uniform: a wait gave up; no copy is issued any more
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

    // Wait for phase ph of the barrier, at most kWaitNs; the result is the same
    // in every lane of the warp.
    __device__ bool wait(uint32_t ph)
    {
        const unsigned long long t0 = global_ns();
        bool ok = false;
        for (unsigned it = 0; it < kWaitPolls; ++it) {
            uint32_t r;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(r) : "r"(smem_u32(bar())), "r"(ph) : "memory");
            if (r) { ok = true; break; }
            if (global_ns() - t0 > kWaitNs) break;
        }
        return __all_sync(0xffffffffu, ok);
    }

    // This lane's entry of the 32 consecutive V at src: staged through shared
    // memory by a bulk copy (TMA), or loaded directly (plain path, or a warp
    // whose earlier wait timed out).
    __device__ V load_lane(const V* __restrict__ src, int lane, DevCounters* cnt)
    {
        if constexpr (!TMA) {
            (void)cnt;
            return src[lane];
        } else {
            if (timed_out) return src[lane];
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
                // the copy of this phase may still land later: keep the phase
                // (finish() waits for it) and read this leaf directly
                timed_out = true;
                if (lane == 0) raise_status(cnt, SIDM_DEV_WAIT_TIMEOUT);
                return src[lane];
            }
            phase ^= 1u;
            const V v = raw()[lane];
            __syncwarp();
            return v;
        }
    }

    __device__ void finish(int lane, DevCounters* cnt)
    {
        if constexpr (TMA) {
            // a copy whose wait timed out may still be in flight into this
            // warp's shared memory: wait for it (bounded) before the CTA exits
            if (timed_out && !wait(phase) && lane == 0) raise_status(cnt, SIDM_DEV_WAIT_TIMEOUT);
        }
        (void)lane; (void)cnt;
    }
};

template <class R>
using TileStage = TileStageT<R, false>;

}  // namespace sidm
