// dev_common.cuh -- device helpers shared by the solver kernels: wall-clock time,
// TMA bulk copies with mbarrier completion and bounded waits, fixed-point conversions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "roi_internal.h"

namespace roi {

// Storage element of a resident array or a projector image: DT 0 = float, 1 = bfloat16,
// 2 = IEEE half (16-bit patterns).  Arithmetic is always float.
template <int DT>
struct Stor {
    using T = unsigned short;
};
template <>
struct Stor<0> {
    using T = float;
};
template <int DT>
__device__ __forceinline__ float to_f32(typename Stor<DT>::T v) {
    if constexpr (DT == 0) {
        return v;
    } else if constexpr (DT == 1) {
        return __uint_as_float((unsigned)v << 16);  // bfloat16 -> float is exact
    } else {
        return __half2float(__ushort_as_half(v));
    }
}
template <int DT>
__device__ __forceinline__ typename Stor<DT>::T from_f32(float x) {  // round to nearest even
    if constexpr (DT == 0) {
        return x;
    } else if constexpr (DT == 1) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
        return __half_as_ushort(__float2half_rn(x));
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: arm the barrier for `bytes` and start the bulk copy global -> shared; the
// caller has ordered earlier generic writes of the destination (fence.proxy.async).
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One thread: fence, arm the barrier for `bytes` and start the bulk copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async;" ::: "memory");
    bulk_copy(dst, src, bytes, bar);
}

// Plain arrival (completes the phase of a barrier initialised with count 1 when no copy
// is due in it).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Asynchronous 4-byte copy global -> shared (zero-filled when !valid, nothing read); the
// issuing thread waits with cp_async_wait_all before it reads the word.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid = true) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits (bounded) for the bulk copy of phase `parity`.  On time-out sets the error flag,
// waits once more (bounded) so no copy is left writing into shared memory, returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long wait_ns, int* err) {
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > wait_ns) {
            atomicExch(err, 1);
            const unsigned long long t1 = global_ns();
            while (!mbar_test(bar, parity) && global_ns() - t1 < wait_ns) {
            }
            return false;
        }
    }
    return true;
}

// Float-float coordinate v in [-2^8, 2^8) to Q.F fixed point.
template <int F>
__device__ __forceinline__ int to_fixed(ff v) {
    const float n = floorf(v.hi);
    const float fr = (v.hi - n) + v.lo;
    return ((int)n << F) + __float2int_rn(fr * (float)(1 << F));
}

// Float-float coordinate v split into its integer part j0 and the Q.22 fixed-point offset
// from j0 (the return value, in [0, 2^22] up to rounding): any grid size fits, and
// (j0 << 22) + offset is what to_fixed<22>(v) gives wherever that does not overflow
// (|v| < 2^9).
__device__ __forceinline__ int split_fixed22(ff v, int& j0) {
    const float n = floorf(v.hi);
    j0 = (int)n;
    const float fr = (v.hi - n) + v.lo;
    return __float2int_rn(fr * 4194304.0f);
}

// The F <= 23 fraction bits of a Q.F number as an integer-valued float in [0, 2^F):
// OR-ing them into the mantissa of 2^23 and subtracting 2^23 is exact (one logic op and
// one add, no conversion instruction).
// a * b + c, rounded once and clamped to [0, 1] (the clamp is a modifier of the FMA, so a
// hat weight max(0, 1 - |d|/w) costs one FMA-pipe instruction and no min/max).
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
    float r;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int F>
__device__ __forceinline__ float frac_int(int q) {
    return __uint_as_float(0x4B000000u | ((unsigned)q & ((1u << F) - 1u))) - 8388608.0f;
}

}  // namespace roi
