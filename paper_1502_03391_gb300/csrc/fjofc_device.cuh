// Device-side building blocks shared by the fJOFC kernels: inline-PTX wrappers for
// mbarriers and TMA (cp.async.bulk.tensor), bounded waits, packed float math and the
// device status block.  sm_100+ only (built for sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "fjofc_internal.h"

namespace fjofc {

// ----------------------------------------------------------------- status block
// Written by the kernels, read by later kernels of the same call and copied to the
// host once at the end of a call.
struct DevStatus {
    int done;          // 1 once the loop has stopped (converged, max_iter, error)
    int error;         // 0 or an FJOFC_ERR_* code raised on the device
    int final_iter;    // index T of the returned iterate X_T
    int timeout_site;  // where a bounded wait gave up (diagnostics)
    double stress;     // sigma(X_T)
    unsigned long long bad;   // input check: smallest ((l n + row) n + col) * 4 + kind of an
                              // invalid Delta entry (kind 1 negative, 2 not finite,
                              // 3 asymmetric), ~0 when none was found
};
constexpr unsigned long long kNoBadEntry = ~0ull;

__device__ __forceinline__ int ld_volatile(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int site) {
    atomicCAS(&st->error, 0, code);
    atomicExch(&st->timeout_site, site);
    atomicExch(&st->done, 1);
}

// ----------------------------------------------------------------- walk order
// The all-pairs pass visits the row-block walks of a modality in alternating long/short
// order (row blocks 0, nRB-1, 1, nRB-2, ...), so that any contiguous range of sub-tiles
// holds the same mix of full and diagonal/ragged (masked) sub-tiles and walk changes.
// walk_off[] is indexed by walk position.
__host__ __device__ __forceinline__ int walk_row(int pos, int nRB) {
    return (pos & 1) ? nRB - 1 - (pos >> 1) : (pos >> 1);
}
__host__ __device__ __forceinline__ int walk_pos(int I, int nRB) {
    return (2 * I < nRB) ? 2 * I : 2 * (nRB - 1 - I) + 1;
}

// ----------------------------------------------------------------- timers / waits
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Upper bound of the device-side waits on mbarriers (TMA and copy completions, which
// take microseconds when healthy); the grid-wide waits of the in-sample loop take their
// bound from the call (fjofc_opts.wait_limit_us, this value by default).  On expiry the
// kernel records FJOFC_ERR_TIMEOUT and returns instead of spinning.
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

// 16-byte asynchronous copy global -> shared through L2 only (cp.async.cg); bytes < 16
// reads that many and zero-fills the rest (0: reads nothing).  Both addresses 16-byte
// aligned.
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(bytes) : "memory");
}
// Arrive on the mbarrier once this thread's earlier cp.async copies have landed (counts
// as one of the barrier's expected arrivals).
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Untiled bulk copy (cp.async.bulk) of `bytes` from global to shared memory, completing on
// the mbarrier `bar` (complete_tx).  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar) : "memory");
}

// Orders this thread's view of global memory written through ordinary stores (by any
// thread, once acquired) before its later asynchronous-proxy reads (bulk copies, TMA).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Invalidate an mbarrier before its memory is initialised again (a CTA that runs several
// problems re-initialises its ring barriers for each one).
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

// Plain arrive (count 1) with the default release semantics at CTA scope: writes made
// before the arrive are visible to threads that observe the phase completion.
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier.  Returns false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// As mbar_wait_bounded, but also gives up early once *abort_flag (shared memory) is set
// by another warp of the CTA that has already timed out.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, const volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
        }
    }
}

// 2-D tiled TMA load of box {x (inner), y} into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}

// 3-D tiled TMA load of box {x, y, z}.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ----------------------------------------------------------------- math helpers
// Hardware reciprocal square root (MUFU); inputs are clamped to >= FLT_MIN by callers.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct DeltaLoad;
template <> struct DeltaLoad<float> {
    static __device__ __forceinline__ float to_f32(float v) { return v; }
};
template <> struct DeltaLoad<__half> {
    static __device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
};
template <> struct DeltaLoad<__nv_bfloat16> {
    static __device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// Loads from the shared state space by 32-bit shared address (the compiler does not know
// that the ring's generic pointers point into shared memory).
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_f1(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// C consecutive Delta values at shared address a (16-byte aligned for float32 C % 4 == 0)
// as float.
template <typename TD, int C>
__device__ __forceinline__ void lds_delta_row(uint32_t a, float (&out)[C]) {
    if constexpr (sizeof(TD) == 4) {
        if constexpr (C % 4 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 4) {
                const float4 v = lds_f4(a + 4 * c);
                out[c] = v.x; out[c + 1] = v.y; out[c + 2] = v.z; out[c + 3] = v.w;
            }
        } else {
            static_assert(C % 2 == 0, "even column count");
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                const float2 v = lds_f2(a + 4 * c);
                out[c] = v.x; out[c + 1] = v.y;
            }
        }
    } else {
        static_assert(C % 2 == 0, "even column count");
#pragma unroll
        for (int c = 0; c < C; c += 2) {
            const uint32_t w = lds_u32(a + 2 * c);
            if constexpr (std::is_same<TD, __half>::value) {
                const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
                out[c] = v.x; out[c + 1] = v.y;
            } else {
                const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
                out[c] = v.x; out[c + 1] = v.y;
            }
        }
    }
}

// Load C consecutive Delta values from shared memory (vectorised) as float.
template <typename TD, int C>
__device__ __forceinline__ void load_delta_row(const TD* p, float (&out)[C]) {
    if constexpr (sizeof(TD) == 4) {
        if constexpr (C % 4 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 4) {
                float4 v = *reinterpret_cast<const float4*>(p + c);
                out[c] = v.x; out[c + 1] = v.y; out[c + 2] = v.z; out[c + 3] = v.w;
            }
        } else if constexpr (C % 2 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                float2 v = *reinterpret_cast<const float2*>(p + c);
                out[c] = v.x; out[c + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c] = reinterpret_cast<const float*>(p)[c];
        }
    } else {
        if constexpr (C % 2 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                if constexpr (std::is_same<TD, __half>::value) {
                    float2 v = __half22float2(*reinterpret_cast<const __half2*>(p + c));
                    out[c] = v.x; out[c + 1] = v.y;
                } else {
                    float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p + c));
                    out[c] = v.x; out[c + 1] = v.y;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c] = DeltaLoad<TD>::to_f32(p[c]);
        }
    }
}

// ----------------------------------------------------------------- float-float sums
// GB300 executes float64 at a small fraction of the float32 rate, so reductions that
// need more than float32 accuracy carry an unevaluated float pair (hi + lo) combined with
// error-free transformations (Knuth's TwoSum); float64 appears only in a few scalars.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    const float e = (a - (s - bp)) + (b - bp);
    return FF{s, e};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    FF s = ff_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return ff_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_add(FF a, float b) {
    FF s = ff_two_sum(a.hi, b);
    s.lo += a.lo;
    return ff_two_sum(s.hi, s.lo);
}
// (a.hi + a.lo) * w as a float-float (TwoProd by fma).
__device__ __forceinline__ FF ff_mul(FF a, float w) {
    const float ph = a.hi * w;
    const float pe = fmaf(a.hi, w, -ph) + a.lo * w;
    return ff_two_sum(ph, pe);
}
// Full-warp float-float sum (xor butterfly: every lane gets the same total).
__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        // combine in a lane-independent order so every lane computes the same value
        v = ((threadIdx.x & o) == 0) ? ff_add(v, w) : ff_add(w, v);
    }
    return v;
}

// Float-float total of v[0], v[stride], ..., v[(count-1)*stride] by one warp: lane l sums
// entries l, l+32, ... (loads issued together), then a fixed-order butterfly.  Used for the
// per-pass totals, identically by the persistent kernel and by K2.
__device__ __forceinline__ FF totals_ff(const float2* v, int stride, int count) {
    const int lane = threadIdx.x & 31;
    FF acc{0.f, 0.f};
    for (int g = lane; g < count; g += 32) {
        const float2 x = __ldcg(v + int64_t(g) * stride);
        acc = ff_add(acc, FF{x.x, x.y});
    }
    return warp_sum_ff(acc);
}

// Full-warp float64 sum (xor butterfly, every lane gets the total).
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace fjofc
