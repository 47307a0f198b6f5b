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
