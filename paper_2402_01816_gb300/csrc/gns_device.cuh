// gns_device.cuh -- device helpers shared by the library's kernels.
//
// Key encoding (order map): every key is turned into an unsigned 64-bit integer
// whose unsigned order is the requested sort order, so that every comparison in
// every kernel is one integer compare.  The map is a bijection, so the original
// bit pattern is restored exactly on the final write.
//   float64: IEEE 754 totalOrder -- a negative pattern (sign bit set) maps to its
//            complement, a non-negative pattern gets its sign bit set.
//   int64  : flip the sign bit (two's complement order -> unsigned order).
//   descending: complement of the ascending map (the DescLeft target of the
//            "Definition of sorting" chapter: ties still keep input order,
//            because every merge below is stable under this single order).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gns.h"

namespace gns {

constexpr uint64_t kSignBit = 0x8000000000000000ull;
constexpr int MODE_DESC = 1;   // bit 0 of a mode: descending
constexpr int MODE_I64 = 2;    // bit 1 of a mode: int64 keys (else float64)

__device__ __forceinline__ uint64_t encode_key(uint64_t u, int mode)
{
    uint64_t m = (mode & MODE_I64) ? (u ^ kSignBit)
                                   : (u ^ ((uint64_t)((int64_t)u >> 63) | kSignBit));
    return (mode & MODE_DESC) ? ~m : m;
}

__device__ __forceinline__ uint64_t decode_key(uint64_t e, int mode)
{
    uint64_t m = (mode & MODE_DESC) ? ~e : e;
    if (mode & MODE_I64) return m ^ kSignBit;
    return m ^ ((m & kSignBit) ? kSignBit : ~0ull);
}

// ---------------------------------------------------------------------------
// Inter-CTA flags with acquire/release semantics and bounded waits.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Test hook (gns_debug_jitter): a pseudo-random delay of up to max_ns for work
// item `item` of pass `pass`, so that the in-place passes' tickets load in
// perturbed orders and a missing dependency wait shows up as a wrong result.
__device__ __forceinline__ void debug_jitter(uint32_t max_ns, int64_t item, int pass)
{
    if (max_ns == 0) return;
    const uint32_t h = (uint32_t)item * 2654435761u ^ (uint32_t)pass * 40503u;
    __nanosleep((h ^ (h >> 15)) % max_ns);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Spin until *flag == want.  Gives up (returns false) when the call's error word
// is already set by another CTA, or after limit_ns nanoseconds, in which case it
// records err_code in the call's error word.  Never spins unboundedly.
__device__ __forceinline__ bool wait_flag(const int* flag, int want, int* call_err,
                                          uint64_t limit_ns, int err_code)
{
    if (ld_acquire(flag) == want) return true;
    uint64_t t0 = global_ns();
    unsigned sleep_ns = 32;
    for (;;) {
        if (ld_acquire(flag) == want) return true;
        if (ld_relaxed(call_err) != 0) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicCAS(call_err, 0, err_code);
            return false;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 2048) sleep_ns <<= 1;
    }
}

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

}  // namespace gns
