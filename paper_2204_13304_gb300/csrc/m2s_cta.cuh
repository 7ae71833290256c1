// Pieces shared by the CTA wavefront sweeps (k_wave2.cu: 27-point,
// k_wave7.cu: 7-point): tagged mailbox words, and the shared-memory rings
// that carry values between the warps of a CTA.
#pragma once

#include "m2s_internal.cuh"

namespace m2s {
namespace cta {

// ---------------------------------------------------------------------------
// Tagged words.  A value and a 32-bit tag travel in 64-bit words, each
// written with one relaxed 64-bit store (single-copy atomic): a reader that
// sees the expected tag sees the value, with no fence on either side.
// FP32: one word (tag | bits); FP64: two words (tag | low half, tag | high).
// ---------------------------------------------------------------------------
typedef unsigned long long u64;

template <typename T> struct Tagged;
template <> struct Tagged<float> {
    struct W { u64 w; };
    static __device__ __forceinline__ W pack(float v, unsigned tag) {
        return W{((u64)tag << 32) | (u64)__float_as_uint(v)};
    }
    static __device__ __forceinline__ bool unpack(W w, unsigned tag, float* v) {
        *v = __uint_as_float((unsigned)w.w);
        return (unsigned)(w.w >> 32) == tag;
    }
    static __device__ __forceinline__ W zero() { return W{0ull}; }
};
template <> struct Tagged<double> {
    struct W { u64 lo, hi; };
    static __device__ __forceinline__ W pack(double v, unsigned tag) {
        const u64 b = (u64)__double_as_longlong(v);
        return W{((u64)tag << 32) | (b & 0xffffffffull), ((u64)tag << 32) | (b >> 32)};
    }
    static __device__ __forceinline__ bool unpack(W w, unsigned tag, double* v) {
        const u64 b = (w.lo & 0xffffffffull) | ((w.hi & 0xffffffffull) << 32);
        *v = __longlong_as_double((long long)b);
        return (unsigned)(w.lo >> 32) == tag && (unsigned)(w.hi >> 32) == tag;
    }
    static __device__ __forceinline__ W zero() { return W{0ull, 0ull}; }
};

__device__ __forceinline__ void st_relaxed_u64(u64* p, u64 v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u64 ld_relaxed_u64(const u64* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
template <typename T>
__device__ __forceinline__ void mb_store(u64* mb, i64 p, T v, unsigned tag) {
    const typename Tagged<T>::W w = Tagged<T>::pack(v, tag);
    if constexpr (sizeof(T) == 4) {
        st_relaxed_u64(mb + p, w.w);
    } else {
        st_relaxed_u64(mb + 2 * p, w.lo);
        st_relaxed_u64(mb + 2 * p + 1, w.hi);
    }
}
template <typename T>
__device__ __forceinline__ typename Tagged<T>::W mb_load(const u64* mb, i64 p) {
    typename Tagged<T>::W w;
    if constexpr (sizeof(T) == 4) {
        w.w = ld_relaxed_u64(mb + p);
    } else {
        w.lo = ld_relaxed_u64(mb + 2 * p);
        w.hi = ld_relaxed_u64(mb + 2 * p + 1);
    }
    return w;
}

// Ask L2 for the line holding p (no register is written, nothing waits).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// A replayed row keeps its mailbox word in the ring registers of Q and b
// (a row is either computed or replayed, never both).
__device__ __forceinline__ void tw_to_regs(Tagged<float>::W w, float* q, float* b) {
    *q = __uint_as_float((unsigned)w.w);
    *b = __uint_as_float((unsigned)(w.w >> 32));
}
__device__ __forceinline__ Tagged<float>::W regs_to_tw(float q, float b) {
    return Tagged<float>::W{((u64)__float_as_uint(b) << 32) | (u64)__float_as_uint(q)};
}
__device__ __forceinline__ void tw_to_regs(Tagged<double>::W w, double* q, double* b) {
    *q = __longlong_as_double((long long)w.lo);
    *b = __longlong_as_double((long long)w.hi);
}
__device__ __forceinline__ Tagged<double>::W regs_to_tw(double q, double b) {
    return Tagged<double>::W{(u64)__double_as_longlong(q), (u64)__double_as_longlong(b)};
}

// A ring entry read from shared memory as it is now (the producer warp may
// be writing it: each 64-bit half is read once, and its tag tells whether it
// is the entry wanted).
__device__ __forceinline__ Tagged<float>::W ring_load(const Tagged<float>::W* p) {
    Tagged<float>::W r;
    r.w = ((volatile const Tagged<float>::W*)p)->w;
    return r;
}
__device__ __forceinline__ Tagged<double>::W ring_load(const Tagged<double>::W* p) {
    Tagged<double>::W r;
    r.lo = ((volatile const Tagged<double>::W*)p)->lo;
    r.hi = ((volatile const Tagged<double>::W*)p)->hi;
    return r;
}

constexpr int RING = 32;  // steps held by a plane-sum ring

// Shared memory of one CTA: per warp, a ring of tagged plane sums G read by
// the warp above, and the warp's progress (read by the warp below for
// back-pressure only).
template <typename T, int W>
struct CtaShared {
    typename Tagged<T>::W ring[W][RING][32];
    volatile int prog[W];
};


}  // namespace cta
}  // namespace m2s
