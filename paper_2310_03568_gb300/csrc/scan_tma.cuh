// Single-pass scan with decoupled look-back, one tile per block, the tile
// staged in shared memory by bulk (TMA) copies.
//
// A tile is kTmaSubTiles sub-tiles of THREADS * ITEMS elements (a thread
// handles 16 bytes of each array per sub-tile, so its shared reads are
// conflict-free); with 16-byte elements and one array it is 32 KB.  A block
// claims its tile by atomic ticket (tiles are handed out in order, so a tile
// only ever waits on tiles that running blocks hold), one thread copies every
// input array of the tile (plus one element on each side) into shared memory,
// and the block
//   phase A   per sub-tile, per-warp aggregates from shared memory;
//   publish   the tile's aggregate, look back (whole block, 256 tiles per
//             step) for its exclusive prefix, publish the inclusive prefix;
//   phase B   rescans from shared memory and stores.
// The data sit in shared memory rather than registers, so several blocks fit
// an SM (about 190 KB of tiles in flight per SM), and while some blocks wait
// on their look-back, others' copies stream in.  Nothing is read twice.
// Every wait is bounded (look-back polls, the tile's mbarrier); on expiry the
// tile publishes ERROR, the error word gets kErrTimeout, and the block waits
// (bounded) for its copy before it leaves.  Same Op interface as
// k_scan_staged (fetch_staged, kStreams, Elem, stream()).
#pragma once

#include "common.cuh"
#include "internal.h"
#include "scan_engine.cuh"
#include "scan_staged.cuh"
#include "tma.cuh"

namespace adc {

constexpr int kTmaSubTiles = 8;  // sub-tiles per tile

template <class Op, int ITEMS> constexpr size_t tma_stream_bytes() {
    return (size_t)kTmaSubTiles * kScanThreads * ITEMS * sizeof(typename Op::Elem) +
           2 * stage_halo<typename Op::Elem>();
}
template <class Op, int ITEMS> constexpr size_t tma_tile_bytes() {
    return (size_t)Op::kStreams * tma_stream_bytes<Op, ITEMS>();
}

template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan_tma(const Op op, const int64_t n, const int64_t num_tiles, unsigned long long *__restrict__ aggw,
           unsigned long long *__restrict__ incw, const DevCtl ctl) {
    using S = typename Op::State;
    using E = typename Op::Elem;
    constexpr int SUB = THREADS * ITEMS;
    constexpr int TILE = kTmaSubTiles * SUB;
    constexpr int NW = THREADS / kWarp;
    constexpr int K = Tagged<S>::K;
    constexpr int64_t SO = tags_first<S>() ? 1 : K;          // slot offset of a tile
    const int64_t WS = tags_first<S>() ? num_tiles : 1;      // word stride (word-major for large states)
    constexpr int NS = Op::kStreams;
    constexpr int NE = kTmaSubTiles * NW;        // (sub-tile, warp) entries in logical order
    constexpr int EPL = (NE + kWarp - 1) / kWarp;  // entries per lane of warp 0
    constexpr int64_t HALO = stage_halo<E>();
    static_assert(16 % sizeof(E) == 0 || sizeof(E) % 16 == 0, "tiles need 16-byte aligned starts and halos");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ unsigned s_tile;
    __shared__ S s_wt[NE];
    __shared__ S s_lbv[NW];
    __shared__ int s_lbinc[NW], s_lberr[NW];
    __shared__ S s_agg;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;
    const size_t sb = tma_stream_bytes<Op, ITEMS>();
    auto stage = [&](int st) -> E * { return reinterpret_cast<E *>(smem_raw + (size_t)st * sb + HALO); };

    if (tid == 0) {
        s_tile = atomicAdd(ctl.counter, 1u);
        mbar_init(&s_bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const long long t = s_tile;
    const int64_t e0 = (REVERSE ? (num_tiles - 1 - t) : t) * (int64_t)TILE;
    if (tid == 0) {
        // the bulk copies of the tile (plain copies for a ragged end shorter
        // than 16 bytes; the __syncthreads after the wait publishes them)
        const int64_t nb = n * (int64_t)sizeof(E);
        int64_t lo = e0 * (int64_t)sizeof(E);
        int64_t hi = (e0 + TILE) * (int64_t)sizeof(E) + HALO;
        if (lo >= HALO) lo -= HALO;
        if (hi > nb) hi = nb;
        const int64_t hi16 = hi & ~(int64_t)15;
        const uint32_t bytes = hi16 > lo ? (uint32_t)(hi16 - lo) : 0u;
        const int64_t base = e0 * (int64_t)sizeof(E);
        mbar_expect_tx(&s_bar, bytes * NS);
        if (bytes) {
#pragma unroll
            for (int st = 0; st < NS; ++st)
                bulk_g2s(reinterpret_cast<char *>(stage(st)) + (lo - base),
                         reinterpret_cast<const char *>(op.stream(st)) + lo, bytes, &s_bar);
        }
        for (int64_t b = hi16 > lo ? hi16 : lo; b < hi; ++b) {
#pragma unroll
            for (int st = 0; st < NS; ++st)
                reinterpret_cast<char *>(stage(st))[b - base] = reinterpret_cast<const char *>(op.stream(st))[b];
        }
    }
    const E *sm[NS];
#pragma unroll
    for (int st = 0; st < NS; ++st) sm[st] = stage(st);
    auto chunk0 = [&](int s) -> int64_t {
        const int ps = REVERSE ? (kTmaSubTiles - 1 - s) : s;
        return e0 + (int64_t)ps * SUB + (int64_t)jc * ITEMS;
    };
    auto thread_agg = [&](const S (&st)[ITEMS]) -> S {
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) a = op.combine(a, st[REVERSE ? ITEMS - 1 - k : k]);
        return a;
    };
    if (!__syncthreads_and(mbar_wait_bounded(&s_bar, 0u, ctl.spin_limit))) {
        if (tid == 0) {
            publish_tag(incw + t * SO, K, kFlagError, WS);
            set_error(ctl.err, kErrTimeout);
            mbar_wait_bounded(&s_bar, 0u, ctl.spin_limit);  // a second chance for the copy to land
        }
        return;
    }

    // ---- phase A: per-warp aggregates of every sub-tile
#pragma unroll
    for (int s = 0; s < kTmaSubTiles; ++s) {
        const int64_t c0 = chunk0(s);
        typename Op::Raw raw;
        op.fetch_staged(sm, c0 - e0, c0, n, raw);
        S st[ITEMS];
        typename Op::Aux aux;
        op.build(c0, n, raw, st, aux);
        const S winc = warp_inclusive_scan(op, thread_agg(st));
        if (lane == kWarp - 1) s_wt[s * NW + warp] = winc;
    }
    __syncthreads();
    // warp 0: lane l folds entries [l * EPL, (l + 1) * EPL), then an ordered reduction
    S lane_fold = op.identity();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < EPL; ++q) {
            const int e = lane * EPL + q;
            if (e < NE) lane_fold = op.combine(lane_fold, s_wt[e]);
        }
        S v = lane_fold;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const S other = shfl_down(v, o);
            if (lane + o < kWarp) v = op.combine(v, other);
        }
        if (lane == 0) s_agg = v;
    }
    __syncthreads();
    const S tile_agg = s_agg;

    // ---- look-back over the tiles
    S prefix = op.identity();
    bool abort = false;
    if (t == ctl.stall_tile) {  // fault injection: this tile never publishes
        abort = true;
    } else {
        if (tid == 0) publish(aggw + t * SO, tile_agg, kFlagAgg, WS);
        if (t == 0) {
            if (tid == 0) publish(incw, tile_agg, kFlagInc, WS);
        } else {
            long long base = t - 1;
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
                for (int o = 1; o < kWarp; o <<= 1) {  // farthest (highest lane) first
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
                    publish_tag(incw + t * SO, K, kFlagError, WS);
                    set_error(ctl.err, kErrTimeout);
                } else {
                    publish(incw + t * SO, op.combine(prefix, tile_agg), kFlagInc, WS);
                }
            }
        }
    }
    if (abort) return;  // block-uniform; the copy has landed

    // ---- exclusive prefix of every (sub-tile, warp) entry (warp 0, in order)
    if (warp == 0) {
        S ex = shfl_up(warp_inclusive_scan(op, lane_fold), 1);
        if (lane == 0) ex = op.identity();
        S run = op.combine(prefix, ex);
#pragma unroll
        for (int q = 0; q < EPL; ++q) {
            const int e = lane * EPL + q;
            if (e < NE) {
                const S agg = s_wt[e];
                s_wt[e] = run;
                run = op.combine(run, agg);
            }
        }
    }
    __syncthreads();

    // ---- phase B: rescan from shared memory, store
#pragma unroll
    for (int s = 0; s < kTmaSubTiles; ++s) {
        const int64_t c0 = chunk0(s);
        typename Op::Raw raw;
        op.fetch_staged(sm, c0 - e0, c0, n, raw);
        S st[ITEMS];
        typename Op::Aux aux;
        op.build(c0, n, raw, st, aux);
        S ex = shfl_up(warp_inclusive_scan(op, thread_agg(st)), 1);
        if (lane == 0) ex = op.identity();
        S run = op.combine(s_wt[s * NW + warp], ex);
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int kk = REVERSE ? ITEMS - 1 - k : k;
            const S exk = run;
            run = op.combine(run, st[kk]);
            st[kk] = exclusive_store<Op>(0) ? exk : run;
        }
        op.store(c0, n, st, aux);
    }
}

template <class Op, int ITEMS, bool REVERSE>
adc_status run_scan_tma(const Op &op, int64_t n, void *ws, int slot, void *region, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    constexpr int64_t TILE = (int64_t)kTmaSubTiles * kScanThreads * ITEMS;
    const int64_t T = (n + TILE - 1) / TILE;
    const ScanWs L = scan_ws_layout(T, sizeof(typename Op::State));
    char *w = static_cast<char *>(region);
    if (cudaMemsetAsync(w, 0, L.bytes, s) != cudaSuccess) return ADC_ERR_CUDA;
    const DevCtl ctl = make_ctl(ws, slot);
    const size_t smem = tma_tile_bytes<Op, ITEMS>();
    auto kern = k_scan_tma<Op, kScanThreads, ITEMS, REVERSE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ADC_ERR_CUDA;
    kern<<<(unsigned)T, kScanThreads, smem, s>>>(op, n, T, reinterpret_cast<unsigned long long *>(w + L.agg_off),
                                               reinterpret_cast<unsigned long long *>(w + L.inc_off), ctl);
    return check_launch();
}

}  // namespace adc
