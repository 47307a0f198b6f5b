// Device helpers shared by the reduce_by_index kernels (hist.cu, hist_part.cu).
#pragma once

#include "common.cuh"

namespace adc {

__device__ __forceinline__ bool in_range(int32_t k, int64_t m) { return (uint32_t)k < (uint64_t)m; }

// Lifted min/max (Fig. 5) as one 64-bit word: order-preserving value bits in
// the high half, the element index in the low half (inverted for max), so that
// the lifted operator -- smaller index wins ties -- is a plain integer min/max.
template <bool MAX> struct Pack {
    static constexpr unsigned long long kEmpty = MAX ? 0ull : ~0ull;
    static __device__ __forceinline__ unsigned long long key(float v, int64_t i) {
        const uint32_t idx = MAX ? (0xffffffffu - (uint32_t)i) : (uint32_t)i;
        return ((unsigned long long)ordered_key(v) << 32) | idx;
    }
    static __device__ __forceinline__ int64_t index(unsigned long long k) {
        const uint32_t lo = (uint32_t)k;
        return MAX ? (int64_t)(0xffffffffu - lo) : (int64_t)lo;
    }
    static __device__ __forceinline__ bool better(unsigned long long a, unsigned long long b) {
        return MAX ? a > b : a < b;
    }
    static __device__ __forceinline__ void update(unsigned long long *p, unsigned long long k) {
        if (better(k, __ldcg(p))) {
            if (MAX) atomicMax(p, k);
            else atomicMin(p, k);
        }
    }
    static __device__ __forceinline__ void update_smem(unsigned long long *p, unsigned long long k) {
        if (better(k, *reinterpret_cast<volatile unsigned long long *>(p))) {
            if (MAX) atomicMax(p, k);
            else atomicMin(p, k);
        }
    }
};

// The un-lifted min/max on order-preserving 32-bit value keys.
template <bool MAX> struct Ord32 {
    static constexpr uint32_t kEmpty = MAX ? 0u : 0xffffffffu;
    static __device__ __forceinline__ bool better(uint32_t a, uint32_t b) { return MAX ? a > b : a < b; }
    static __device__ __forceinline__ void update(uint32_t *p, uint32_t k, bool shared) {
        const uint32_t cur = shared ? *reinterpret_cast<volatile uint32_t *>(p) : __ldcg(p);
        if (better(k, cur)) {
            if (MAX) atomicMax(p, k);
            else atomicMin(p, k);
        }
    }
};

__device__ __forceinline__ float from_ordered(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ double from_ordered(unsigned long long u) {
    return __longlong_as_double(
        (long long)((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u));
}

// Compare-and-swap on the bit pattern of a float / double; returns the old value.
__device__ __forceinline__ float cas_val(float *a, float expect, float val) {
    return __uint_as_float(atomicCAS(reinterpret_cast<unsigned *>(a), __float_as_uint(expect), __float_as_uint(val)));
}
__device__ __forceinline__ double cas_val(double *a, double expect, double val) {
    return __longlong_as_double((long long)atomicCAS(reinterpret_cast<unsigned long long *>(a),
                                                     (unsigned long long)__double_as_longlong(expect),
                                                     (unsigned long long)__double_as_longlong(val)));
}
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }

// Multiplies up to U values into bins base[idx[j]] (global or shared memory)
// with all compare-and-swaps of a round in flight together, so that U
// independent round trips overlap.  Bounded rounds; a give-up sets the error
// word.
template <typename T, int U>
__device__ __forceinline__ void mul_batch(T *base, const int32_t (&idx)[U], const T (&v)[U], const bool (&use)[U],
                                          unsigned *err) {
    T cur[U];
    bool todo[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
        todo[j] = use[j];
        if (todo[j]) cur[j] = *reinterpret_cast<volatile T *>(base + idx[j]);
    }
    for (int round = 0; round < (1 << 20); ++round) {
        bool any = false;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (todo[j]) {
                const T old = cas_val(base + idx[j], cur[j], cur[j] * v[j]);
                if (same_bits(old, cur[j])) {
                    todo[j] = false;
                } else {
                    cur[j] = old;
                    any = true;
                }
            }
        }
        if (!any) return;
    }
    set_error(err, kErrCasLimit);
}

}  // namespace adc
