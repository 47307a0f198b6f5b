// Range-partitioned single-pass scan with the range staged in shared memory
// by the Tensor Memory Accelerator (1-D bulk copies, mbarrier completion).
//
// Same protocol as k_scan_ranges (claim a range of tiles in start order,
// per-warp tile aggregates, range aggregate, block-wide look-back over
// earlier ranges, rescan), but the range's input arrays are copied into
// shared memory once, by one thread, with cp.async.bulk: the copy engine keeps
// the whole range in flight without registers, both passes read shared memory,
// and nothing is read from DRAM twice.  A thread handles 16 bytes of each
// array per tile (one 128-bit shared load, consecutive threads on consecutive
// 16-byte words: no bank conflicts), so a tile is 4 KB per array.
//
// A staged Op provides, besides the scan interface of scan_engine.cuh:
//   static constexpr int kStreams;      arrays read (1..3), all of n elements
//   using Elem;                         their element type
//   const Elem* stream(int s) const;    the arrays
//   void fetch_staged(const Elem *const (&sm)[kStreams], int64_t lo,
//                     int64_t c0, int64_t n, Raw&) const;
//        like fetch(), reading element c0 + k at sm[s][lo + k]; one element
//        before and after the range is staged too (halos).
#pragma once

#include "common.cuh"
#include "internal.h"
#include "scan_engine.cuh"

namespace adc {

constexpr int kStageGroups = 4;          // mbarriers per range (tiles arrive in groups)
constexpr int kStageMaxTiles = 32;       // tiles per range
// Bytes staged before and after the range (one element at least, 16 at least).
template <typename E> constexpr int64_t stage_halo() { return sizeof(E) > 16 ? (int64_t)sizeof(E) : 16; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Global -> shared bulk copy; addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Bounded wait for phase 0 of a barrier; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, long long limit) {
    long long it = 0;
    while (!mbar_try_wait(bar, 0u)) {
        if (++it > limit) return false;
    }
    return true;
}

// Shared-memory chunk load: 128-bit when whole, element-wise at the ragged end.
template <typename E, int ITEMS>
__device__ __forceinline__ void load_chunk_sm(const E *p, int64_t c0, int64_t n, E (&st)[ITEMS], E fill) {
    constexpr int BYTES = (int)sizeof(E) * ITEMS;
    if constexpr (BYTES % 16 == 0) {
        if (c0 + ITEMS <= n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(p);
#pragma unroll
            for (int w = 0; w < BYTES / 16; ++w) {
                const uint4 v = src[w];
                memcpy(reinterpret_cast<char *>(st) + 16 * w, &v, 16);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) st[k] = (c0 + k < n) ? p[k] : fill;
}

// Bytes of one stream's stage buffer for ranges of `rt` tiles.
template <class Op, int ITEMS> constexpr size_t stage_stream_bytes(int rt) {
    return (size_t)rt * kScanThreads * ITEMS * sizeof(typename Op::Elem) + 2 * stage_halo<typename Op::Elem>();
}
template <class Op, int ITEMS> constexpr size_t stage_smem_bytes(int rt) {
    return (size_t)Op::kStreams * stage_stream_bytes<Op, ITEMS>(rt);
}

template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan_staged(const Op op, const int64_t n, const int64_t num_tiles, const int rt, unsigned long long *__restrict__ aggw,
              unsigned long long *__restrict__ incw, const DevCtl ctl) {
    using S = typename Op::State;
    using E = typename Op::Elem;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int NW = THREADS / kWarp;
    constexpr int K = Tagged<S>::K;
    constexpr int NS = Op::kStreams;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar[kStageGroups];
    __shared__ unsigned s_range;
    __shared__ S s_wt[kStageMaxTiles * NW];
    __shared__ S s_lbv[NW];
    __shared__ int s_lbinc[NW], s_lberr[NW];
    __shared__ S s_range_agg;
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;
    const int64_t NR = (num_tiles + rt - 1) / rt;
    const size_t sb = stage_stream_bytes<Op, ITEMS>(rt);

    if (tid == 0) {
        s_range = atomicAdd(ctl.counter, 1u);
        s_abort = 0;
        for (int g = 0; g < kStageGroups; ++g) mbar_init(&s_bar[g], 1);
        mbar_init_fence();
    }
    __syncthreads();
    const long long r = s_range;
    const int64_t pr = REVERSE ? (NR - 1 - r) : r;          // physical range
    const int64_t t0 = pr * rt;                             // its first physical tile
    const int cnt = (int)((num_tiles - t0) < rt ? (num_tiles - t0) : rt);
    const int64_t e0 = t0 * TILE;                           // first element of the range
    const int64_t e1 = (e0 + (int64_t)cnt * TILE) < n ? (e0 + (int64_t)cnt * TILE) : n;
    const int per_group = (cnt + kStageGroups - 1) / kStageGroups;
    const int groups = (cnt + per_group - 1) / per_group;

    // ---- stage: thread 0 issues the bulk copies, group by group (physical tile order)
    const E *sm_e[NS];  // element e0 of each stream in the stage (read side)
    E *sm_w[NS];        // the same (write side)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        sm_w[s] = reinterpret_cast<E *>(smem_raw + (size_t)s * sb + stage_halo<E>());
        sm_e[s] = sm_w[s];
    }
    if (tid == 0) {
        const int64_t nb = n * (int64_t)sizeof(E);
        for (int g = 0; g < groups; ++g) {
            // bytes [lo, hi) of each stream, plus the halos at the range's ends
            int64_t lo = (e0 + (int64_t)g * per_group * TILE) * (int64_t)sizeof(E);
            int64_t hi = (e0 + (int64_t)(g + 1) * per_group * TILE) * (int64_t)sizeof(E);
            if (g == 0 && lo >= stage_halo<E>()) lo -= stage_halo<E>();
            if (g == groups - 1) hi += stage_halo<E>();
            if (hi > nb) hi = nb;
            const int64_t hi16 = hi & ~(int64_t)15;
            const uint32_t bytes = hi16 > lo ? (uint32_t)(hi16 - lo) : 0u;
            mbar_expect_tx(&s_bar[g], bytes * NS);
            if (bytes) {
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const char *src = reinterpret_cast<const char *>(op.stream(s)) + lo;
                    char *dst = reinterpret_cast<char *>(sm_w[s]) + (lo - e0 * (int64_t)sizeof(E));
                    bulk_g2s(dst, src, bytes, &s_bar[g]);
                }
            }
            // ragged tail (< 16 bytes at the end of the arrays): plain copies
            for (int64_t b = hi16 > lo ? hi16 : lo; b < hi; ++b) {
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    reinterpret_cast<char *>(sm_w[s])[b - e0 * (int64_t)sizeof(E)] =
                        reinterpret_cast<const char *>(op.stream(s))[b];
            }
        }
    }
    __syncthreads();  // the plain tail copies are visible

    auto chunk0 = [&](int i) -> int64_t {  // logical tile i of the range -> this thread's first element
        const int64_t p = REVERSE ? (t0 + cnt - 1 - i) : (t0 + i);
        return p * (int64_t)TILE + (int64_t)jc * ITEMS;
    };
    auto group_of = [&](int i) -> int { return (REVERSE ? (cnt - 1 - i) : i) / per_group; };
    // REVERSE: items of a chunk are combined from the highest index down
    auto thread_agg_dir = [&](const S (&st)[ITEMS]) -> S {
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) a = op.combine(a, st[REVERSE ? ITEMS - 1 - k : k]);
        return a;
    };

    // ---- phase A: warp-tile aggregates, waiting for each group as it is needed
    int waited = -1;
    bool abort = false;
    for (int i = 0; i < cnt; ++i) {
        const int g = group_of(i);
        if (g != waited) {
            // warp-uniform: a lane that gave up takes its whole warp out
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&s_bar[g], ctl.spin_limit))) {
                abort = true;
                break;
            }
            waited = g;
        }
        const int64_t c0 = chunk0(i);
        typename Op::Raw raw;
        op.fetch_staged(sm_e, c0 - e0, c0, n, raw);
        S st[ITEMS];
        typename Op::Aux aux;
        op.build(c0, n, raw, st, aux);
        const S winc = warp_inclusive_scan(op, thread_agg_dir(st));
        if (lane == kWarp - 1) s_wt[i * NW + warp] = winc;
    }
    if (abort) atomicOr(reinterpret_cast<unsigned *>(&s_abort), 1u);
    __syncthreads();
    if (s_abort) {
        // a bulk copy never completed: fail this range, give the copies a last
        // bounded chance to land in this block's memory, and leave
        if (tid == 0) {
            publish_tag(incw + r * K, K, kFlagError);
            set_error(ctl.err, kErrTimeout);
            for (int g = 0; g < groups; ++g) mbar_wait_bounded(&s_bar[g], ctl.spin_limit);
        }
        return;
    }

    // ---- range aggregate
    const int E_ = cnt * NW;
    const int per_lane = (E_ + kWarp - 1) / kWarp;
    S lane_fold = op.identity();
    if (warp == 0) {
        for (int e = lane * per_lane; e < E_ && e < (lane + 1) * per_lane; ++e) lane_fold = op.combine(lane_fold, s_wt[e]);
        S v = lane_fold;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const S other = shfl_down(v, o);
            if (lane + o < kWarp) v = op.combine(v, other);
        }
        if (lane == 0) s_range_agg = v;
    }
    __syncthreads();
    const S range_agg = s_range_agg;

    // ---- look-back over the ranges
    S prefix = op.identity();
    if (r == ctl.stall_tile) {  // fault injection: this range never publishes
        abort = true;
    } else {
        if (tid == 0) publish(aggw + r * K, range_agg, kFlagAgg);
        if (r == 0) {
            if (tid == 0) publish(incw, range_agg, kFlagInc);
        } else {
            long long base = r - 1;
            while (true) {
                const long long tj = base - (long long)kWarp * warp - lane;
                S v = op.identity();
                unsigned f = kFlagInc;
                if (tj >= 0) f = wait_tile(aggw + tj * K, incw + tj * K, &v, ctl.spin_limit);
                const bool err = __any_sync(0xffffffffu, f == kFlagError);
                const unsigned incmask = __ballot_sync(0xffffffffu, f == kFlagInc);
                const int stop = incmask ? (__ffs(incmask) - 1) : (kWarp - 1);
                if (lane > stop) v = op.identity();
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const S other = shfl_down(v, o);
                    if (lane + o < kWarp) v = op.combine(other, v);
                }
                if (lane == 0) {
                    s_lbv[warp] = v;
                    s_lbinc[warp] = incmask != 0;
                    s_lberr[warp] = err;
                }
                __syncthreads();
                bool found = false;
                for (int w = 0; w < NW; ++w) {
                    if (s_lberr[w]) {
                        abort = true;
                        break;
                    }
                    prefix = op.combine(s_lbv[w], prefix);
                    if (s_lbinc[w]) {
                        found = true;
                        break;
                    }
                }
                __syncthreads();
                if (abort || found) break;
                base -= (long long)kWarp * NW;
            }
            if (tid == 0) {
                if (abort) {
                    publish_tag(incw + r * K, K, kFlagError);
                    set_error(ctl.err, kErrTimeout);
                } else {
                    publish(incw + r * K, op.combine(prefix, range_agg), kFlagInc);
                }
            }
        }
    }
    if (abort) return;  // block-uniform; every group was waited for in phase A

    // ---- exclusive prefix of every warp-tile entry (warp 0, in order)
    if (warp == 0) {
        S ex = shfl_up(warp_inclusive_scan(op, lane_fold), 1);
        if (lane == 0) ex = op.identity();
        S run = op.combine(prefix, ex);
        for (int e = lane * per_lane; e < E_ && e < (lane + 1) * per_lane; ++e) {
            const S agg = s_wt[e];
            s_wt[e] = run;
            run = op.combine(run, agg);
        }
    }
    __syncthreads();

    // ---- phase B: rescan from shared memory, store
    for (int i = 0; i < cnt; ++i) {
        const int64_t c0 = chunk0(i);
        typename Op::Raw raw;
        op.fetch_staged(sm_e, c0 - e0, c0, n, raw);
        S st[ITEMS];
        typename Op::Aux aux;
        op.build(c0, n, raw, st, aux);
        S ex = shfl_up(warp_inclusive_scan(op, thread_agg_dir(st)), 1);
        if (lane == 0) ex = op.identity();
        S run = op.combine(s_wt[i * NW + warp], ex);
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int kk = REVERSE ? ITEMS - 1 - k : k;
            run = op.combine(run, st[kk]);
            st[kk] = run;
        }
        op.store(c0, n, st, aux);
    }
    (void)e1;
}

// Tiles per range: about 96 KB of staged input per block (two blocks per SM).
template <class Op, int ITEMS> constexpr int stage_range_tiles() {
    constexpr size_t tile_bytes = (size_t)kScanThreads * ITEMS * sizeof(typename Op::Elem) * Op::kStreams;
    constexpr size_t t = (96 * 1024) / tile_bytes;
    return t < 1 ? 1 : (t > kStageMaxTiles ? kStageMaxTiles : (int)t);
}

template <class Op, int ITEMS, bool REVERSE>
adc_status run_scan_staged(const Op &op, int64_t n, void *ws, int slot, void *region, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    using Sh = ScanShape<Op, ITEMS>;
    const int64_t T = Sh::tiles(n);
    const int rt = g_scan_range_tiles > 0 && g_scan_range_tiles <= kStageMaxTiles ? g_scan_range_tiles
                                                                                  : stage_range_tiles<Op, ITEMS>();
    const int64_t NR = (T + rt - 1) / rt;
    const ScanWs L = scan_ws_layout(T, sizeof(typename Op::State));
    char *w = static_cast<char *>(region);
    if (cudaMemsetAsync(w, 0, L.bytes, s) != cudaSuccess) return ADC_ERR_CUDA;
    const DevCtl ctl = make_ctl(ws, slot);
    const size_t smem = stage_smem_bytes<Op, ITEMS>(rt);
    auto kern = k_scan_staged<Op, kScanThreads, ITEMS, REVERSE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ADC_ERR_CUDA;
    kern<<<(unsigned)NR, kScanThreads, smem, s>>>(op, n, T, rt, reinterpret_cast<unsigned long long *>(w + L.agg_off),
                                                  reinterpret_cast<unsigned long long *>(w + L.inc_off), ctl);
    return check_launch();
}

}  // namespace adc
