// gj_lookback.cuh -- decoupled lookback shared by the single-pass scans.
//
// A tile publishes its aggregate, reads its predecessors' published
// aggregates or inclusive prefixes until it meets a prefix, and publishes its
// own inclusive prefix.  The status of a tile is a flag (ST_A: aggregate
// published, ST_P: inclusive prefix published) and a value, written and read
// as one word, so a reader never pairs a flag with another publication's
// value and no memory fence is needed: 32-bit values share an 8-byte word
// with the flag, 64-bit values take a 16-byte aligned pair moved by one
// vector access.  Every poll is bounded by SPIN_LIMIT; on expiry the kernel
// records ERRF_TIMEOUT and counts the predecessor as a zero prefix, so a
// stuck predecessor can never hang the GPU.
#pragma once

#include "gj_internal.cuh"

namespace gj {

template <class T>
__device__ __forceinline__ T ld_volatile(const T *p) { return *(const volatile T *)p; }

constexpr uint32_t ST_A = 1u, ST_P = 2u;

template <class T> struct TileStatus;
template <> struct TileStatus<uint32_t> {
    using W = unsigned long long;
    static __device__ __forceinline__ void put(W *s, uint32_t f, uint32_t v) {
        atomicExch(s, ((W)f << 32) | v);
    }
    static __device__ __forceinline__ void get(const W *s, uint32_t &f, uint32_t &v) {
        const W w = ld_volatile(s);
        f = (uint32_t)(w >> 32);
        v = (uint32_t)w;
    }
};
template <> struct TileStatus<uint64_t> {
    using W = ulonglong2;
    static __device__ __forceinline__ void put(W *s, uint32_t f, uint64_t v) {
        asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(s), "l"((unsigned long long)f),
                     "l"((unsigned long long)v)
                     : "memory");
    }
    static __device__ __forceinline__ void get(const W *s, uint32_t &f, uint64_t &v) {
        unsigned long long a, b;
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(s) : "memory");
        f = (uint32_t)a;
        v = b;
    }
};

struct AddU32 {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};
struct SatAddU64 {
    __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const { return sat_add(a, b); }
};

// Decoupled lookback by one warp (every lane calls it): publishes the
// tile's aggregate, then reads the status of 32 predecessors at a time
// (lane 31 the nearest), folds everything from the nearest published prefix
// onwards, and moves 32 tiles further back only while all of them hold just
// an aggregate.  Returns the tile's carry-in (the same in every lane) after
// publishing its inclusive prefix.  Op must be associative and commutative
// (the window is folded by a butterfly).
template <class T>
__device__ __forceinline__ void publish_aggregate(typename TileStatus<T>::W *st, uint32_t tile, T agg) {
    TileStatus<T>::put(&st[tile], tile == 0 ? ST_P : ST_A, agg);
}

// The lookback proper, after the tile's aggregate has been published
// (publish_aggregate by one thread, visible before any lane calls this).
template <class T, class Op>
__device__ __forceinline__ T warp_lookback_published(typename TileStatus<T>::W *st, uint32_t tile,
                                                     T agg, int lane, uint32_t *err,
                                                     uint32_t limit = SPIN_LIMIT) {
    Op op;
    if (tile == 0) return T(0);
    T carry = T(0);
    int64_t p = (int64_t)tile - 1;
    for (;;) {
        const int64_t q = p - 31 + lane;
        uint32_t f = ST_P;   // tiles before the first count as a zero prefix
        T v = T(0);
        if (q >= 0) {
            uint32_t spins = 0;
            for (;;) {
                TileStatus<T>::get(&st[q], f, v);
                if (f) break;
                if (++spins > limit) {
                    raise_err(err, ERRF_TIMEOUT);
                    f = ST_P;
                    v = T(0);
                    break;
                }
            }
        }
        const uint32_t pm = __ballot_sync(0xffffffffu, f == ST_P);
        const int hi = pm ? 31 - __clz((int)pm) : 0;
        T x = lane >= hi ? v : T(0);
#pragma unroll
        for (int d = 16; d; d >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, d));
        carry = op(x, carry);
        if (pm) break;
        p -= 32;
    }
    if (lane == 0) TileStatus<T>::put(&st[tile], ST_P, op(carry, agg));
    return carry;
}

template <class T, class Op>
__device__ __forceinline__ T warp_lookback(typename TileStatus<T>::W *st, uint32_t tile, T agg,
                                           int lane, uint32_t *err) {
    if (lane == 0) publish_aggregate<T>(st, tile, agg);
    return warp_lookback_published<T, Op>(st, tile, agg, lane, err);
}

}  // namespace gj
