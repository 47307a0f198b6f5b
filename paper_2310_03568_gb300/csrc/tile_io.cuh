// Per-thread chunk loads/stores: ITEMS consecutive elements starting at c0,
// 128-bit vectorised when the chunk is whole, element-wise at the ragged tail.
#pragma once

#include <string.h>

#include "common.cuh"

namespace adc {

template <typename E, int ITEMS>
__device__ __forceinline__ void load_chunk(const E *__restrict__ p, int64_t c0, int64_t n, E (&st)[ITEMS], E fill) {
    constexpr int BYTES = (int)sizeof(E) * ITEMS;
    if constexpr (BYTES % 16 == 0) {
        if (c0 + ITEMS <= n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(p + c0);
#pragma unroll
            for (int w = 0; w < BYTES / 16; ++w) {
                uint4 v = __ldg(src + w);  // default L2 policy: a second pass may hit L2
                memcpy(reinterpret_cast<char *>(st) + 16 * w, &v, 16);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) st[k] = (c0 + k < n) ? p[c0 + k] : fill;
}

// The same with the evict-first (streaming) policy: data read once, which
// should not displace tables that are gathered from.
template <typename E, int ITEMS>
__device__ __forceinline__ void load_chunk_cs(const E *__restrict__ p, int64_t c0, int64_t n, E (&st)[ITEMS], E fill) {
    constexpr int BYTES = (int)sizeof(E) * ITEMS;
    if constexpr (BYTES % 16 == 0) {
        if (c0 + ITEMS <= n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(p + c0);
#pragma unroll
            for (int w = 0; w < BYTES / 16; ++w) {
                uint4 v = __ldcs(src + w);
                memcpy(reinterpret_cast<char *>(st) + 16 * w, &v, 16);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) st[k] = (c0 + k < n) ? p[c0 + k] : fill;
}

// A read-only gather that asks L2 to keep the line (evict-last): per-bin
// tables that a streaming pass gathers from at random.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ld_keep(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *p, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_keep(const int32_t *p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

template <typename E, int ITEMS>
__device__ __forceinline__ void store_chunk(E *__restrict__ p, int64_t c0, int64_t n, const E (&st)[ITEMS]) {
    constexpr int BYTES = (int)sizeof(E) * ITEMS;
    if constexpr (BYTES % 16 == 0) {
        if (c0 + ITEMS <= n) {
            uint4 *dst = reinterpret_cast<uint4 *>(p + c0);
#pragma unroll
            for (int w = 0; w < BYTES / 16; ++w) {
                uint4 v;
                memcpy(&v, reinterpret_cast<const char *>(st) + 16 * w, 16);
                __stcs(dst + w, v);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (c0 + k < n) p[c0 + k] = st[k];
}

}  // namespace adc
