// Range-partitioned single-pass scan with the ranges staged in shared memory
// by the Tensor Memory Accelerator (1-D bulk copies, mbarrier completion),
// persistent and double-buffered.
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
#include "tma.cuh"

namespace adc {

constexpr int kStageGroups = 4;          // mbarriers per range (tiles arrive in groups)
constexpr int kStageMaxTiles = 32;       // tiles per range
// Bytes staged before and after the range (one element at least, 16 at least).
template <typename E> constexpr int64_t stage_halo() { return sizeof(E) > 16 ? (int64_t)sizeof(E) : 16; }

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

// Persistent and double-buffered: a cooperative launch makes every block
// resident, so block b can own ranges b, b + G, b + 2G, ... in that order
// (G blocks).  While it scans range r from one stage buffer, the bulk copies
// of range r + G land in the other, so each SM always has a range's loads in
// flight.  Range r's look-back only waits on ranges below r, which are being
// or have been processed by resident blocks, so every wait ends.
template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan_staged(const Op op, const int64_t n, const int64_t num_tiles, const int rt, unsigned long long *__restrict__ aggw,
              unsigned long long *__restrict__ incw, const DevCtl ctl) {
    using S = typename Op::State;
    using E = typename Op::Elem;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int NW = THREADS / kWarp;
    constexpr int K = Tagged<S>::K;
    constexpr int64_t SO = tags_first<S>() ? 1 : K;          // slot offset of a tile
    const int64_t WS = tags_first<S>() ? num_tiles : 1;      // word stride (word-major for large states)
    constexpr int NS = Op::kStreams;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar[2][kStageGroups];
    __shared__ S s_wt[kStageMaxTiles * NW];
    __shared__ S s_lbv[NW];
    __shared__ int s_lbinc[NW], s_lberr[NW];
    __shared__ S s_range_agg;
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;
    const int64_t NR = (num_tiles + rt - 1) / rt;
    const int64_t G = gridDim.x;
    const size_t sb = stage_stream_bytes<Op, ITEMS>(rt);
    const int per_group = (rt + kStageGroups - 1) / kStageGroups;

    // stage pointers: element e0 of the range, per buffer and stream
    auto stage_w = [&](int buf, int s) -> E * {
        return reinterpret_cast<E *>(smem_raw + ((size_t)buf * NS + s) * sb + stage_halo<E>());
    };
    struct Geo {
        int64_t t0, e0;
        int cnt, groups;
    };
    auto geo = [&](int64_t r) -> Geo {
        Geo g;
        const int64_t pr = REVERSE ? (NR - 1 - r) : r;
        g.t0 = pr * rt;
        g.cnt = (int)((num_tiles - g.t0) < rt ? (num_tiles - g.t0) : rt);
        g.e0 = g.t0 * TILE;
        g.groups = (g.cnt + per_group - 1) / per_group;
        return g;
    };
    // thread 0: the bulk copies of range r into buffer buf (plain copies for
    // a ragged end shorter than 16 bytes; a later __syncthreads publishes them)
    auto issue = [&](int64_t r, int buf) {
        const Geo q = geo(r);
        const int64_t nb = n * (int64_t)sizeof(E);
        for (int g = 0; g < q.groups; ++g) {
            int64_t lo = (q.e0 + (int64_t)g * per_group * TILE) * (int64_t)sizeof(E);
            int64_t hi = (q.e0 + (int64_t)(g + 1) * per_group * TILE) * (int64_t)sizeof(E);
            if (g == 0 && lo >= stage_halo<E>()) lo -= stage_halo<E>();
            if (g == q.groups - 1) hi += stage_halo<E>();
            if (hi > nb) hi = nb;
            const int64_t hi16 = hi & ~(int64_t)15;
            const uint32_t bytes = hi16 > lo ? (uint32_t)(hi16 - lo) : 0u;
            mbar_expect_tx(&s_bar[buf][g], bytes * NS);
            const int64_t base = q.e0 * (int64_t)sizeof(E);
            if (bytes) {
#pragma unroll
                for (int st = 0; st < NS; ++st)
                    bulk_g2s(reinterpret_cast<char *>(stage_w(buf, st)) + (lo - base),
                             reinterpret_cast<const char *>(op.stream(st)) + lo, bytes, &s_bar[buf][g]);
            }
            for (int64_t b = hi16 > lo ? hi16 : lo; b < hi; ++b) {
#pragma unroll
                for (int st = 0; st < NS; ++st)
                    reinterpret_cast<char *>(stage_w(buf, st))[b - base] = reinterpret_cast<const char *>(op.stream(st))[b];
            }
        }
        // every barrier of the buffer completes one phase per use, so that the
        // parities stay in step when a short range needs fewer groups
        for (int g = q.groups; g < kStageGroups; ++g) mbar_expect_tx(&s_bar[buf][g], 0u);
    };
    auto thread_agg_dir = [&](const S (&st)[ITEMS]) -> S {
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) a = op.combine(a, st[REVERSE ? ITEMS - 1 - k : k]);
        return a;
    };

    if (tid == 0) {
        for (int b = 0; b < 2; ++b)
            for (int g = 0; g < kStageGroups; ++g) mbar_init(&s_bar[b][g], 1);
        mbar_init_fence();
        s_abort = 0;
        if ((int64_t)blockIdx.x < NR) issue(blockIdx.x, 0);
    }
    __syncthreads();

    bool abort = false;
    int64_t i = 0;
    for (;; ++i) {
        const long long r = (long long)(blockIdx.x + i * G);
        if (r >= NR) break;
        const int buf = (int)(i & 1);
        const uint32_t par = (uint32_t)((i >> 1) & 1);
        __syncthreads();  // iteration i-1 is done with buffer buf ^ 1 (and the tail copies are visible)
        if (tid == 0 && r + G < NR) issue(r + G, buf ^ 1);
        const Geo q = geo(r);
        const E *sm_e[NS];
#pragma unroll
        for (int st = 0; st < NS; ++st) sm_e[st] = stage_w(buf, st);
        auto chunk0 = [&](int t) -> int64_t {
            const int64_t p = REVERSE ? (q.t0 + q.cnt - 1 - t) : (q.t0 + t);
            return p * (int64_t)TILE + (int64_t)jc * ITEMS;
        };
        auto group_of = [&](int t) -> int { return (REVERSE ? (q.cnt - 1 - t) : t) / per_group; };

        // ---- phase A
        int waited = -1;
        for (int t = 0; t < q.cnt; ++t) {
            const int g = group_of(t);
            if (g != waited) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&s_bar[buf][g], par, ctl.spin_limit))) {
                    abort = true;
                    break;
                }
                waited = g;
            }
            const int64_t c0 = chunk0(t);
            typename Op::Raw raw;
            op.fetch_staged(sm_e, c0 - q.e0, c0, n, raw);
            S st[ITEMS];
            typename Op::Aux aux;
            op.build(c0, n, raw, st, aux);
            const S winc = warp_inclusive_scan(op, thread_agg_dir(st));
            if (lane == kWarp - 1) s_wt[t * NW + warp] = winc;
        }
        if (abort) atomicOr(reinterpret_cast<unsigned *>(&s_abort), 1u);
        __syncthreads();
        if (s_abort) {
            abort = true;
            if (tid == 0) {
                publish_tag(incw + r * SO, K, kFlagError, WS);
                set_error(ctl.err, kErrTimeout);
            }
            break;
        }

        // ---- range aggregate
        const int E_ = q.cnt * NW;
        const int per_lane = (E_ + kWarp - 1) / kWarp;
        S lane_fold = op.identity();
        if (warp == 0) {
            for (int e = lane * per_lane; e < E_ && e < (lane + 1) * per_lane; ++e)
                lane_fold = op.combine(lane_fold, s_wt[e]);
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
            if (tid == 0) publish(aggw + r * SO, range_agg, kFlagAgg, WS);
            if (r == 0) {
                if (tid == 0) publish(incw, range_agg, kFlagInc, WS);
            } else {
                long long base = r - 1;
                while (true) {
                    const long long tj = base - (long long)kWarp * warp - lane;
                    S v = op.identity();
                    unsigned f = kFlagInc;
                    if (tj >= 0) f = wait_tile(aggw + tj * SO, incw + tj * SO, &v, ctl.spin_limit, WS);
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
                        publish_tag(incw + r * SO, K, kFlagError, WS);
                        set_error(ctl.err, kErrTimeout);
                    } else {
                        publish(incw + r * SO, op.combine(prefix, range_agg), kFlagInc, WS);
                    }
                }
            }
        }
        if (abort) break;  // block-uniform

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
        for (int t = 0; t < q.cnt; ++t) {
            const int64_t c0 = chunk0(t);
            typename Op::Raw raw;
            op.fetch_staged(sm_e, c0 - q.e0, c0, n, raw);
            S st[ITEMS];
            typename Op::Aux aux;
            op.build(c0, n, raw, st, aux);
            S ex = shfl_up(warp_inclusive_scan(op, thread_agg_dir(st)), 1);
            if (lane == 0) ex = op.identity();
            S run = op.combine(s_wt[t * NW + warp], ex);
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) {
                const int kk = REVERSE ? ITEMS - 1 - k : k;
                run = op.combine(run, st[kk]);
                st[kk] = run;
            }
            op.store(c0, n, st, aux);
        }
    }
    if (abort && tid == 0) {
        // leave no bulk copy in flight into this block's shared memory: give the
        // current range's and the prefetched range's copies a bounded chance to land
        const int buf = (int)(i & 1);
        for (int g = 0; g < kStageGroups; ++g) {
            mbar_wait_bounded(&s_bar[buf][g], (uint32_t)((i >> 1) & 1), ctl.spin_limit);
            if ((long long)(blockIdx.x + (i + 1) * G) < NR)
                mbar_wait_bounded(&s_bar[buf ^ 1][g], (uint32_t)(((i + 1) >> 1) & 1), ctl.spin_limit);
        }
    }
}

// Tiles per range: two stage buffers of about 48 KB of input each per block
// (two blocks per SM).
template <class Op, int ITEMS> constexpr int stage_range_tiles() {
    constexpr size_t tile_bytes = (size_t)kScanThreads * ITEMS * sizeof(typename Op::Elem) * Op::kStreams;
    constexpr size_t t = (48 * 1024) / tile_bytes;
    return t < 1 ? 1 : (t > kStageMaxTiles ? kStageMaxTiles : (int)t);
}

template <class Op, int ITEMS, bool REVERSE>
adc_status run_scan_staged(const Op &op, int64_t n, void *ws, int slot, void *region, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    using Sh = ScanShape<Op, ITEMS>;
    const int64_t T = Sh::tiles(n);
    int rt = g_scan_range_tiles > 0 && g_scan_range_tiles <= kStageMaxTiles ? g_scan_range_tiles
                                                                            : stage_range_tiles<Op, ITEMS>();
    while (rt > 1 && 2 * stage_smem_bytes<Op, ITEMS>(rt) > (size_t)200 * 1024) --rt;  // both buffers fit
    const int64_t NR = (T + rt - 1) / rt;
    const ScanWs L = scan_ws_layout(T, sizeof(typename Op::State));
    char *w = static_cast<char *>(region);
    if (cudaMemsetAsync(w, 0, L.bytes, s) != cudaSuccess) return ADC_ERR_CUDA;
    DevCtl ctl = make_ctl(ws, slot);
    const size_t smem = 2 * stage_smem_bytes<Op, ITEMS>(rt);
    auto kern = k_scan_staged<Op, kScanThreads, ITEMS, REVERSE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ADC_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScanThreads, smem) != cudaSuccess || per_sm < 1)
        return ADC_ERR_CUDA;
    int64_t G = (int64_t)num_sms() * per_sm;
    if (G > NR) G = NR;
    Op o = op;
    int64_t nn = n, tt = T;
    int rr = rt;
    unsigned long long *aggw = reinterpret_cast<unsigned long long *>(w + L.agg_off);
    unsigned long long *incw = reinterpret_cast<unsigned long long *>(w + L.inc_off);
    void *args[] = {&o, &nn, &tt, &rr, &aggw, &incw, &ctl};
    // cooperative: all G blocks resident at once (the static range ownership relies on it)
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3((unsigned)G), dim3(kScanThreads), args,
                                    smem, s) != cudaSuccess)
        return ADC_ERR_CUDA;
    return check_launch();
}

}  // namespace adc
