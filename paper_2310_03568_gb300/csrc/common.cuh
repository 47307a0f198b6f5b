// Device-side building blocks shared by the libadcomb kernels (sm_103a).
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/adcomb.h"

namespace adc {

constexpr int kWarp = 32;

template <typename T> constexpr adc_dtype dt_of() { return sizeof(T) == 8 ? ADC_F64 : ADC_F32; }

// Error bits in the workspace's device error word.
enum : unsigned { kErrTimeout = 1u, kErrCasLimit = 2u };

// Tile-status flags of the decoupled look-back (Merrill & Garland single-pass scan).
enum : unsigned { kFlagNone = 0u, kFlagAgg = 1u, kFlagInc = 2u, kFlagError = 3u };

struct DevCtl {
    unsigned *err;          // device error word (workspace offset 0)
    unsigned *counter;      // dynamic tile counter
    long long spin_limit;   // bound on polling iterations
    long long stall_tile;   // fault-injection: tile that never publishes (-1: off)
    int prefetch;           // range engine: prefetch each range into L2
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_error(unsigned *err, unsigned bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------- scalars --
template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

// Order-preserving maps float -> uint32 and double -> uint64 (IEEE total order
// restricted to non-NaN values, -0.0 folded onto +0.0 so that they tie).
__device__ __forceinline__ uint32_t ordered_key(float v) {
    uint32_t u = __float_as_uint(v);
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t ordered_key(double v) {
    uint64_t u = (uint64_t)__double_as_longlong(v);
    if (u == 0x8000000000000000ull) u = 0ull;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// a / b for the zero-count vjps, where a is often an exact zero (a product
// that underflowed): a zero numerator gives a * b instead, the same signed
// zero, without the division (measured on the * reduce vjp at n = 1e8 with
// an underflowed product: 0.225 -> 0.143 ms).
template <typename T> __device__ __forceinline__ T div_or_zero(T a, T b) { return a == T(0) ? a * b : a / b; }

// ------------------------------------------------------- tuple element types --
template <typename T> struct Pair { T b, c; };        // linFnComp element x -> b + c*x
template <typename T> struct Mat2 { T a, b, c, d; };  // [[a, b], [c, d]]

template <typename T> __device__ __forceinline__ Mat2<T> mat_mul(const Mat2<T> &x, const Mat2<T> &y) {
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
template <typename T> __device__ __forceinline__ Mat2<T> mat_add(const Mat2<T> &x, const Mat2<T> &y) {
    return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d};
}
template <typename T> __device__ __forceinline__ Mat2<T> mat_t(const Mat2<T> &x) { return {x.a, x.c, x.b, x.d}; }
template <typename T> __device__ __forceinline__ Mat2<T> mat_eye() { return {T(1), T(0), T(0), T(1)}; }
template <typename T> __device__ __forceinline__ Mat2<T> mat_zero() { return {T(0), T(0), T(0), T(0)}; }

// Q x Q row-major matrices (the q = 3, 5 matrix-product operators).
template <typename T, int Q> struct MatQ { T a[Q * Q]; };
template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> matq_mul(const MatQ<T, Q> &x, const MatQ<T, Q> &y) {
    MatQ<T, Q> z;
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            T s = x.a[Q * i] * y.a[j];
#pragma unroll
            for (int k = 1; k < Q; ++k) s += x.a[Q * i + k] * y.a[Q * k + j];
            z.a[Q * i + j] = s;
        }
    return z;
}
template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> matq_add(const MatQ<T, Q> &x, const MatQ<T, Q> &y) {
    MatQ<T, Q> z;
#pragma unroll
    for (int i = 0; i < Q * Q; ++i) z.a[i] = x.a[i] + y.a[i];
    return z;
}
template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> matq_t(const MatQ<T, Q> &x) {
    MatQ<T, Q> z;
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < Q; ++j) z.a[Q * i + j] = x.a[Q * j + i];
    return z;
}
template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> matq_eye() {
    MatQ<T, Q> z;
#pragma unroll
    for (int i = 0; i < Q * Q; ++i) z.a[i] = (i % (Q + 1) == 0) ? T(1) : T(0);
    return z;
}
template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> matq_zero() {
    MatQ<T, Q> z;
#pragma unroll
    for (int i = 0; i < Q * Q; ++i) z.a[i] = T(0);
    return z;
}
// The q x q vjp's affine maps L -> v + L c (c a product of transposed elements).
template <typename T, int Q> struct AffQ { MatQ<T, Q> v, c; };
// In-place products for the matrix segment walks (one row of temporaries):
// A <- A B, and A <- A B^T with B given untransposed.
template <typename T, int Q> __device__ __forceinline__ void matq_mul_right(MatQ<T, Q> &A, const MatQ<T, Q> &B) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T r[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            T acc = A.a[Q * i] * B.a[j];
#pragma unroll
            for (int k = 1; k < Q; ++k) acc += A.a[Q * i + k] * B.a[Q * k + j];
            r[j] = acc;
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) A.a[Q * i + j] = r[j];
    }
}
template <typename T, int Q> __device__ __forceinline__ void matq_mul_right_t(MatQ<T, Q> &A, const MatQ<T, Q> &B) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T r[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            T acc = A.a[Q * i] * B.a[Q * j];
#pragma unroll
            for (int k = 1; k < Q; ++k) acc += A.a[Q * i + k] * B.a[Q * j + k];
            r[j] = acc;
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) A.a[Q * i + j] = r[j];
    }
}


// --------------------------------------------------- L2-coherent state I/O --
// Look-back states are plain structs of T; they are read with ld.global.cg
// (L2, bypassing the non-coherent L1) after an acquire load of the flag.
template <typename S> __device__ __forceinline__ S load_cg(const S *p) {
    static_assert(sizeof(S) % 4 == 0, "state must be made of 32-bit words");
    S out;
    const unsigned *src = reinterpret_cast<const unsigned *>(p);
    unsigned *dst = reinterpret_cast<unsigned *>(&out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(S) / 4); ++i) dst[i] = __ldcg(src + i);
    return out;
}

template <typename S> __device__ __forceinline__ S shfl_up(const S &v, int delta) {
    static_assert(sizeof(S) % 4 == 0, "state must be made of 32-bit words");
    S out;
    const unsigned *src = reinterpret_cast<const unsigned *>(&v);
    unsigned *dst = reinterpret_cast<unsigned *>(&out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(S) / 4); ++i) dst[i] = __shfl_up_sync(0xffffffffu, src[i], delta);
    return out;
}

template <typename S> __device__ __forceinline__ S shfl_down(const S &v, int delta) {
    S out;
    const unsigned *src = reinterpret_cast<const unsigned *>(&v);
    unsigned *dst = reinterpret_cast<unsigned *>(&out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(S) / 4); ++i) dst[i] = __shfl_down_sync(0xffffffffu, src[i], delta);
    return out;
}

template <typename S> __device__ __forceinline__ S shfl_idx(const S &v, int lane) {
    S out;
    const unsigned *src = reinterpret_cast<const unsigned *>(&v);
    unsigned *dst = reinterpret_cast<unsigned *>(&out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(S) / 4); ++i) dst[i] = __shfl_sync(0xffffffffu, src[i], lane);
    return out;
}

// v <- combine(v of lane (lane - o), v) where `active`: an Op with a large
// state may provide shfl_combine(v, o, down, active) doing the shuffles and
// the combine piecewise (fewer live registers than the whole shuffled state
// plus the result); down = true takes the value of lane (lane + o) instead.
template <class Op, typename S> constexpr bool has_shfl_combine(long) { return false; }
template <class Op, typename S>
constexpr auto has_shfl_combine(int)
    -> decltype(std::declval<const Op &>().shfl_combine(std::declval<S &>(), 0, true, true), bool()) {
    return true;
}
template <class Op, typename S>
__device__ __forceinline__ void shfl_combine(const Op &op, S &v, int o, bool down, bool active) {
    if constexpr (has_shfl_combine<Op, S>(0)) {
        op.shfl_combine(v, o, down, active);
    } else {
        const S other = down ? shfl_down(v, o) : shfl_up(v, o);
        if (active) v = op.combine(other, v);
    }
}

// Inclusive warp scan in lane order for an associative (not necessarily
// commutative) operator: lane l ends with x_0 . x_1 . ... . x_l.
template <class Op, typename S> __device__ __forceinline__ S warp_inclusive_scan(const Op &op, S v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) shfl_combine(op, v, o, false, lane >= o);
    return v;
}

// Bounded spin on a tile flag until it is non-zero.  Returns the flag, or
// kFlagError when the iteration limit expires.
__device__ __forceinline__ unsigned spin_flag(const unsigned *flag, long long limit) {
    unsigned f = ld_acquire_u32(flag);
    long long it = 0;
    while (f == kFlagNone) {
        if (++it > limit) return kFlagError;
        __nanosleep(64);
        f = ld_acquire_u32(flag);
    }
    return f;
}

// Bounded CAS-based atomic multiply (no native float atomic multiply exists).
__device__ __forceinline__ void atomic_mul(float *addr, float v, unsigned *err) {
    unsigned *a = reinterpret_cast<unsigned *>(addr);
    unsigned old = *a, assumed;
    int it = 0;
    do {
        assumed = old;
        old = atomicCAS(a, assumed, __float_as_uint(__uint_as_float(assumed) * v));
        if (++it > (1 << 20)) { set_error(err, kErrCasLimit); return; }
    } while (assumed != old);
}
__device__ __forceinline__ void atomic_mul(double *addr, double v, unsigned *err) {
    unsigned long long *a = reinterpret_cast<unsigned long long *>(addr);
    unsigned long long old = *a, assumed;
    int it = 0;
    do {
        assumed = old;
        old = atomicCAS(a, assumed, (unsigned long long)__double_as_longlong(__longlong_as_double((long long)assumed) * v));
        if (++it > (1 << 20)) { set_error(err, kErrCasLimit); return; }
    } while (assumed != old);
}

}  // namespace adc
