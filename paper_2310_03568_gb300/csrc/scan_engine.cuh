// Single-pass scan with decoupled look-back (Merrill & Garland), forward or
// reverse, for any associative operator given as an Op class.  One tile per
// block; the tile index comes from an atomic counter, so every tile a block
// waits on belongs to a block that is already running.
//
// An Op provides
//   using State;                         the scanned value
//   struct Raw;                          this thread's loaded data for one tile
//   struct Aux;                          per-thread data carried from build to store
//   State identity() const;
//   State combine(const State& earlier, const State& later) const;   (logical order)
//   void  fetch(int64_t c0, int64_t n, Raw&) const;
//         issues the loads of elements [c0, c0+ITEMS) (and any halo)
//   void  build(int64_t c0, int64_t n, const Raw&, State (&st)[ITEMS], Aux&) const;
//         the elements' states in PHYSICAL order, identity() beyond n
//   void  store(int64_t c0, int64_t n, const State (&inc)[ITEMS], const Aux&) const;
//         receives the inclusive scan values of those elements.
//
// REVERSE scans run in descending index order: tile claim t maps to physical
// tile T-1-t and the scan is inclusive from the right, i.e. a forward scan of
// the reversed array (the reversals of Figs 2, 4 and 7 are index maps here).
//
// Protocol per tile: reduce the tile, publish its aggregate (tag AGG), look
// back over predecessors with the whole block -- each of the 8 warps polls 32
// tiles, so 256 predecessors per step -- until a tile with an inclusive
// prefix (tag INC) is found, publish the inclusive prefix, then rescan the
// tile from registers.  With many tiles in flight the inclusive-prefix
// frontier advances by one look-back window per memory round trip, so the
// window is made wide (256 tiles) and a poll is one round trip (tagged words
// below).  Every wait is bounded: on expiry the
// tile publishes ERROR, the error word gets kErrTimeout and the tile is not
// stored; later tiles see ERROR and stop waiting at once.
#pragma once

#include <atomic>

#include "common.cuh"
#include "internal.h"

namespace adc {

struct NoAux {};

// An Op may ask (static constexpr bool members, detected here) to receive in
// store() the EXCLUSIVE prefix of each item instead of the inclusive one
// (kExclusiveStore: segment ops, whose item is a run of elements that store()
// re-walks from its incoming value), and to be scanned by the per-tile engine
// only (kPerTileOnly: ops whose build() is expensive, which the range engine
// would run twice).
template <class Op> constexpr bool exclusive_store(long) { return false; }
template <class Op> constexpr auto exclusive_store(int) -> decltype(Op::kExclusiveStore, bool()) {
    return Op::kExclusiveStore;
}
template <class Op> constexpr bool per_tile_only(long) { return false; }
template <class Op> constexpr auto per_tile_only(int) -> decltype(Op::kPerTileOnly, bool()) {
    return Op::kPerTileOnly;
}
// A per-tile-only Op may also ask for its own block size (kThreads) and for
// dynamic shared memory (kDynSmem bytes, e.g. to stage its tile).
template <class Op> constexpr int op_threads(long) { return 256; }
template <class Op> constexpr auto op_threads(int) -> decltype(Op::kThreads, int()) { return Op::kThreads; }
template <class Op> constexpr size_t op_dyn_smem(long) { return 0; }
template <class Op> constexpr auto op_dyn_smem(int) -> decltype(Op::kDynSmem, size_t()) { return Op::kDynSmem; }
// A per-tile-only Op may stage its tile in shared memory by bulk copies
// (kBulkStaged): thread 0 calls op.stage_init() (its mbarrier) when it claims
// the tile, op.fetch() has thread 0 issue the copies, and every thread then
// waits through op.staged_wait(limit), bounded, before build().  A wait that
// runs out marks the tile ERROR and records kErrTimeout, as a look-back that
// runs out does; thread 0 then gives the copies a second bounded wait before
// the block leaves.
template <class Op> constexpr bool bulk_staged(long) { return false; }
template <class Op> constexpr auto bulk_staged(int) -> decltype(Op::kBulkStaged, bool()) { return Op::kBulkStaged; }
// Such an Op may also finish its tile after store() (kFinish: e.g. stage a
// further input into space store() has freed): every thread calls
// op.finish(c0, n, limit), which returns false, alike in every thread, if a
// bounded wait in it ran out; the engine then records kErrTimeout.
template <class Op> constexpr bool op_finish(long) { return false; }
template <class Op> constexpr auto op_finish(int) -> decltype(Op::kFinish, bool()) { return Op::kFinish; }
// An Op may ask (kKeepPrefix) the range engine to keep, from phase A, every
// thread's exclusive prefix within its warp for every tile of the range in
// shared memory, so that phase B needs neither the thread folds nor the warp
// scans again: worth it where the combine itself is the bound (fp64 on this
// part's FP64 pipe).  Ranges are then at most keep_tiles<S>() tiles long.
template <class Op> constexpr bool keep_prefix(long) { return false; }
template <class Op> constexpr auto keep_prefix(int) -> decltype(Op::kKeepPrefix, bool()) { return Op::kKeepPrefix; }
template <typename S, int THREADS> constexpr int keep_tiles() {
    return (int)((32 * 1024) / (THREADS * sizeof(S))) < 1 ? 1 : (int)((32 * 1024) / (THREADS * sizeof(S)));
}

// Ops that name their input arrays (kStreams, stream(s), Elem) can have a
// block's range prefetched into L2 by bulk prefetches.
template <class Op> constexpr int op_streams(long) { return 0; }
template <class Op> constexpr auto op_streams(int) -> decltype(Op::kStreams, int()) { return Op::kStreams; }

// L2 prefetch of [p, p + bytes): p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Test and tuning hook: the range engine prefetches each block's range into
// L2 when the block starts (0 off, 1 on).
extern int g_scan_prefetch;

// ---------------------------------------------------- tagged tile status --
// A published tile state S is stored as K = sizeof(S)/4 64-bit words, each
// (tag << 32 | one 32-bit word of S), in two arrays: aggregates (tag AGG) and
// inclusive prefixes (tag INC; ERROR marks a failed tile).  Every word is
// written and read with single-copy-atomic 64-bit accesses, so a reader that
// sees the same non-zero tag in all K words holds a consistent state -- one
// round trip per poll, no separate flag and no acquire/release pair.  Mixed
// tags mean a write in progress: poll again.  The arrays are word-major:
// word k of tile j sits at slot[k * stride + j] (stride = the launch's tile
// count), so a warp polling 32 consecutive tiles reads 256 contiguous bytes
// per word instead of touching 32 lines -- for large states (tags_first);
// small ones keep their K words together (slot[j * K + k]: word-major
// measured slower for them, e.g. the 2x2 per-tile forward 0.19 -> 0.27 ms).
template <typename S> struct Tagged {
    static constexpr int K = sizeof(S) / 4;
    static_assert(sizeof(S) % 4 == 0, "state must be made of 32-bit words");
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Large states (more than 4 words) are read tag first by the look-back (see
// wait_tag); small ones are polled in full, one round trip per poll.
template <typename S> constexpr bool tags_first() { return Tagged<S>::K > 4; }

// A large state's word 0 goes last, as a release: a reader that acquires
// word 0 with the tag then finds every other word in place, so it reads the
// state once (measured: the 3x3 vjp 0.62 -> 0.55 ms).  Small states keep
// relaxed stores only (a release per publish slowed the fp32 * vjp's
// 6000-range scan by a fifth); their readers check every word's tag.
template <typename S>
__device__ __forceinline__ void publish(unsigned long long *slot, const S &v, unsigned tag, int64_t stride) {
    const unsigned *w = reinterpret_cast<const unsigned *>(&v);
    const unsigned long long t = (unsigned long long)tag << 32;
#pragma unroll
    for (int k = Tagged<S>::K - 1; k > 0; --k) st_relaxed_u64(slot + k * stride, t | w[k]);
    if constexpr (tags_first<S>())
        st_release_u64(slot, t | w[0]);
    else
        st_relaxed_u64(slot, t | w[0]);
}
__device__ __forceinline__ void publish_tag(unsigned long long *slot, int K, unsigned tag, int64_t stride) {
    for (int k = 0; k < K; ++k) st_relaxed_u64(slot + k * stride, (unsigned long long)tag << 32);
}

// One poll of tile j: returns kFlagInc / kFlagAgg with the state in *out,
// kFlagError if the tile failed, or kFlagNone if nothing complete is visible.
template <typename S>
__device__ __forceinline__ unsigned poll_tile(const unsigned long long *agg, const unsigned long long *inc, S *out,
                                              int64_t stride) {
    constexpr int K = Tagged<S>::K;
    unsigned long long a[K], b[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        b[k] = ld_relaxed_u64(inc + k * stride);
        a[k] = ld_relaxed_u64(agg + k * stride);
    }
    unsigned *w = reinterpret_cast<unsigned *>(out);
    bool inc_ok = true, agg_ok = true, err = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        inc_ok &= (unsigned)(b[k] >> 32) == kFlagInc;
        agg_ok &= (unsigned)(a[k] >> 32) == kFlagAgg;
        err |= (unsigned)(b[k] >> 32) == kFlagError;
    }
    if (err) return kFlagError;
    if (inc_ok) {
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (unsigned)b[k];
        return kFlagInc;
    }
    if (agg_ok) {
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (unsigned)a[k];
        return kFlagAgg;
    }
    return kFlagNone;
}

// Bounded spin until tile j shows a complete state.
template <typename S>
__device__ __forceinline__ unsigned wait_tile(const unsigned long long *agg, const unsigned long long *inc, S *out,
                                              long long limit, int64_t stride) {
    long long it = 0;
    unsigned f = poll_tile(agg, inc, out, stride);
    while (f == kFlagNone) {
        if (++it > limit) return kFlagError;
        __nanosleep(32);
        f = poll_tile(agg, inc, out, stride);
    }
    return f;
}

// Large states (tags_first): a look-back lane first spins on the two tag
// words of its tile only, and reads the whole state afterwards, only where
// the ordered reduction needs it (at or before the nearest inclusive
// prefix).  Measured on the 3x3 forward (9-word states): polling every state
// in full read 1.7 GB of L2 for 0.18 GB of input; one full poll before the
// tag spin still doubled the kernel's time.
// Bounded spin until tile j shows a tag: kFlagInc, kFlagAgg or kFlagError
// (also on expiry).  Both tag words are loaded together, with acquire (see
// publish).
__device__ __forceinline__ unsigned wait_tag(const unsigned long long *agg, const unsigned long long *inc,
                                             long long limit) {
    long long it = 0;
    while (true) {
        const unsigned tb = (unsigned)(ld_acquire_u64(inc) >> 32);
        const unsigned ta = (unsigned)(ld_acquire_u64(agg) >> 32);
        if (tb == kFlagInc || tb == kFlagError) return tb;
        if (ta == kFlagAgg) return kFlagAgg;
        if (++it > limit) return kFlagError;
        __nanosleep(32);
    }
}
// Reads a state whose first word showed `tag`, spinning (bounded) until every
// word carries it; false on expiry.
template <typename S>
__device__ __forceinline__ bool read_tagged(const unsigned long long *slot, unsigned tag, S *out, long long limit,
                                            int64_t stride) {
    constexpr int K = Tagged<S>::K;
    unsigned *w = reinterpret_cast<unsigned *>(out);
    long long it = 0;
    while (true) {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const unsigned long long v = ld_relaxed_u64(slot + k * stride);
            ok &= (unsigned)(v >> 32) == tag;
            w[k] = (unsigned)v;
        }
        if (ok) return true;
        if (++it > limit) return false;
        __nanosleep(32);
    }
}

template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan(const Op op, const int64_t n, const int64_t num_tiles, unsigned long long *__restrict__ aggw,
       unsigned long long *__restrict__ incw, const DevCtl ctl) {
    using S = typename Op::State;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int NW = THREADS / kWarp;
    constexpr int K = Tagged<S>::K;
    constexpr int64_t SO = tags_first<S>() ? 1 : K;          // slot offset of a tile
    const int64_t WS = tags_first<S>() ? num_tiles : 1;      // word stride (word-major for large states)
    static_assert(NW <= kWarp, "block too large");
    __shared__ unsigned s_tile;
    __shared__ S s_warp[NW];   // per-warp totals, then per-warp exclusive prefixes
    __shared__ S s_lbv[NW];    // look-back: each warp's combined window
    __shared__ int s_lbinc[NW], s_lberr[NW];
    __shared__ S s_total;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;

    // One tile per block, claimed when the block starts: its aggregate is
    // published one load latency after the claim, so no tile a successor
    // waits on is ever held back behind other work.
    if (tid == 0) {
        s_tile = atomicAdd(ctl.counter, 1u);
        if constexpr (bulk_staged<Op>(0)) op.stage_init();
    }
    __syncthreads();
    const long long t = s_tile;
    {
        const int64_t p = REVERSE ? (num_tiles - 1 - t) : t;
        const int64_t c0 = p * (int64_t)TILE + (int64_t)jc * ITEMS;
        typename Op::Raw raw;
        op.fetch(c0, n, raw);
        if constexpr (bulk_staged<Op>(0)) {
            if (!__syncthreads_and(op.staged_wait(ctl.spin_limit))) {
                if (tid == 0) {
                    publish_tag(incw + t * SO, K, kFlagError, WS);
                    set_error(ctl.err, kErrTimeout);
                    op.staged_wait(ctl.spin_limit);
                }
                return;
            }
        }
        S st[ITEMS];
        typename Op::Aux aux;
        op.build(c0, n, raw, st, aux);

        if (t != ctl.stall_tile) {  // fault injection: this tile never publishes
            // ---- tile reduction and its publication as an aggregate
            S a = op.identity();
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) a = op.combine(a, st[REVERSE ? ITEMS - 1 - k : k]);
            const S winc = warp_inclusive_scan(op, a);
            if (lane == kWarp - 1) s_warp[warp] = winc;
            __syncthreads();
            S wexc = shfl_up(winc, 1);
            if (lane == 0) wexc = op.identity();
            if (warp == 0) {
                const S w = (lane < NW) ? s_warp[lane] : op.identity();
                const S wi = warp_inclusive_scan(op, w);
                S wex = shfl_up(wi, 1);
                if (lane == 0) wex = op.identity();
                const S total = shfl_idx(wi, NW - 1);
                if (lane == 0) {
                    s_total = total;
                    publish(aggw + t * SO, total, kFlagAgg, WS);
                    if (t == 0) publish(incw, total, kFlagInc, WS);
                }
                if (lane < NW) s_warp[lane] = wex;
            }
            // ---- block-wide look-back: 32 x NW predecessors per step
            S prefix = op.identity();
            bool abort = false;
            if (t > 0) {
                long long base = t - 1;
                while (true) {
                    const long long tj = base - (long long)kWarp * warp - lane;  // warp 0 lane 0: nearest
                    S v = op.identity();
                    unsigned f = kFlagInc;
                    if constexpr (tags_first<S>()) {
                        if (tj >= 0) f = wait_tag(aggw + tj * SO, incw + tj * SO, ctl.spin_limit);
                    } else {
                        if (tj >= 0) f = wait_tile(aggw + tj * SO, incw + tj * SO, &v, ctl.spin_limit, WS);
                    }
                    const unsigned incmask = __ballot_sync(0xffffffffu, f == kFlagInc);
                    const int stop = incmask ? (__ffs(incmask) - 1) : (kWarp - 1);
                    bool bad = f == kFlagError;
                    if constexpr (tags_first<S>()) {
                        if (tj >= 0 && lane <= stop && !bad)
                            bad = !read_tagged(f == kFlagInc ? incw + tj * SO : aggw + tj * SO, f, &v, ctl.spin_limit, WS);
                    }
                    const bool err = __any_sync(0xffffffffu, bad);
                    if (lane > stop) v = op.identity();
#pragma unroll
                    for (int o = 1; o < kWarp; o <<= 1)  // ordered: farthest (highest lane) first
                        shfl_combine(op, v, o, true, lane + o < kWarp);
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
                        publish(incw + t * SO, op.combine(prefix, s_total), kFlagInc, WS);
                    }
                }
            } else {
                __syncthreads();  // s_warp prefixes written by warp 0 are visible
            }
            if (!abort) {
                S run = op.combine(op.combine(prefix, s_warp[warp]), wexc);
#pragma unroll
                for (int k = 0; k < ITEMS; ++k) {
                    const int kk = REVERSE ? ITEMS - 1 - k : k;
                    const S ex = run;
                    run = op.combine(run, st[kk]);
                    st[kk] = exclusive_store<Op>(0) ? ex : run;
                }
                op.store(c0, n, st, aux);
                if constexpr (op_finish<Op>(0)) {
                    if (!op.finish(c0, n, ctl.spin_limit) && tid == 0) set_error(ctl.err, kErrTimeout);
                }
            }
        }
    }
}

// Block-wide exclusive scan of one state per thread in thread order; returns
// this thread's exclusive value and (through *total) the block's aggregate.
// Contains two __syncthreads().
template <class Op, int THREADS, typename S>
__device__ __forceinline__ S block_scan_excl(const Op &op, const S &a, S *s_warp, S *total) {
    constexpr int NW = THREADS / kWarp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S winc = warp_inclusive_scan(op, a);
    if (lane == kWarp - 1) s_warp[warp] = winc;
    __syncthreads();
    S wexc = shfl_up(winc, 1);
    if (lane == 0) wexc = op.identity();
    S before = op.identity(), all = op.identity();
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (w < warp) before = op.combine(before, s_warp[w]);
        all = op.combine(all, s_warp[w]);
    }
    __syncthreads();
    *total = all;
    return op.combine(before, wexc);
}

// ------------------------------------------------- range-partitioned scan --
// For large n.  Each block claims (atomic counter, so every block it waits on
// is running) a contiguous range of tiles.  Phase A streams the range once;
// every warp reduces its part of each tile in order and keeps the result in
// shared memory (no block barrier per tile: the warps stream independently).
// The block then folds these warp-tile aggregates into its range aggregate,
// publishes it and looks back over the other ranges -- a few hundred, so the
// look-back is short -- and turns the warp-tile aggregates into exclusive
// prefixes.  Phase B streams the range again in REVERSE tile order, so the
// tiles read last in phase A (still in L2) come first, and each warp rescans
// its part of a tile from its prefix, again without block barriers.
// Traffic: the input twice (less what L2 keeps), the output once.  Same Op
// interface as k_scan.
// Tiles whose loads the range engine keeps in flight per thread: about 64
// bytes of input each (1 for the 64-byte tiles, up to 4 for 16-byte ones).
template <class Op, int ITEMS> constexpr int range_prefetch() {
    constexpr int per = (int)sizeof(typename Op::Raw);
    return per >= 64 ? 1 : (64 / per > 4 ? 4 : (64 / per < 1 ? 1 : 64 / per));
}

template <typename S> constexpr int range_max_tiles() {
    return (int)((32 * 1024) / (8 * sizeof(S))) < 256 ? (int)((32 * 1024) / (8 * sizeof(S))) : 256;
}

template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan_ranges(const Op op, const int64_t n, const int64_t num_tiles, unsigned long long *__restrict__ aggw,
              unsigned long long *__restrict__ incw, const DevCtl ctl) {
    using S = typename Op::State;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int NW = THREADS / kWarp;
    constexpr int K = Tagged<S>::K;
    constexpr int64_t SO = tags_first<S>() ? 1 : K;          // slot offset of a tile
    const int64_t WS = tags_first<S>() ? num_tiles : 1;      // word stride (word-major for large states)
    constexpr bool KEEP = keep_prefix<Op>(0);
    constexpr int KT = KEEP ? keep_tiles<S, THREADS>() : 1;
    constexpr int MT = KEEP ? KT : range_max_tiles<S>();  // KEEP ranges are at most KT tiles
    __shared__ unsigned s_range;
    __shared__ S s_wt[MT * NW];  // warp-tile aggregates, then their exclusive prefixes
    __shared__ S s_tp[KT * THREADS];  // KEEP: each thread's exclusive prefix in its warp, per tile
    __shared__ S s_lbv[NW];
    __shared__ int s_lbinc[NW], s_lberr[NW];
    __shared__ S s_range_agg;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;
    if (tid == 0) s_range = atomicAdd(ctl.counter, 1u);
    __syncthreads();
    const long long r = s_range;
    const long long G = gridDim.x;
    const int64_t per = num_tiles / G, extra = num_tiles % G;
    const int64_t t0 = r * per + (r < extra ? r : extra);
    const int cnt = (int)(per + (r < extra ? 1 : 0));
    auto chunk0 = [&](int64_t t) -> int64_t {
        const int64_t p = REVERSE ? (num_tiles - 1 - t) : t;
        return p * (int64_t)TILE + (int64_t)jc * ITEMS;
    };
    auto thread_agg = [&](const S (&st)[ITEMS]) -> S {
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) a = op.combine(a, st[REVERSE ? ITEMS - 1 - k : k]);
        return a;
    };
    if constexpr (op_streams<Op>(0) > 0) {
        // the range's input into L2 in 64 KB pieces, so that both phases read
        // it from there (the range is whole tiles: every piece starts on a
        // 16-byte boundary; a ragged end shorter than 16 bytes is not prefetched)
        if (ctl.prefetch && tid < op_streams<Op>(0) && cnt > 0) {
            using E = typename Op::Elem;
            const int64_t p0 = REVERSE ? (num_tiles - t0 - cnt) : t0;  // first physical tile
            int64_t lo = p0 * (int64_t)TILE * (int64_t)sizeof(E);
            int64_t hi = (p0 + cnt) * (int64_t)TILE * (int64_t)sizeof(E);
            const int64_t nb = n * (int64_t)sizeof(E);
            if (hi > nb) hi = nb & ~(int64_t)15;
            const char *base = reinterpret_cast<const char *>(op.stream(tid));
            for (; lo < hi; lo += 65536) prefetch_l2_bulk(base + lo, (uint32_t)(hi - lo < 65536 ? hi - lo : 65536));
        }
    }

    // ---- phase A: warp-tile aggregates; the loads of PF tiles in flight
    // (PF > 1 where a thread's tile is small: about 64 bytes in flight each)
    constexpr int PF = range_prefetch<Op, ITEMS>();
    typename Op::Raw raw[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q)
        if (q < cnt) op.fetch(chunk0(t0 + q), n, raw[q]);
    for (int i0 = 0; i0 < cnt; i0 += PF) {
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int i = i0 + q;
            if (i < cnt) {
                S st[ITEMS];
                typename Op::Aux aux;
                op.build(chunk0(t0 + i), n, raw[q], st, aux);
                if (i + PF < cnt) op.fetch(chunk0(t0 + i + PF), n, raw[q]);
                const S winc = warp_inclusive_scan(op, thread_agg(st));
                if (lane == kWarp - 1) s_wt[i * NW + warp] = winc;
                if constexpr (KEEP) {
                    S ex = shfl_up(winc, 1);
                    if (lane == 0) ex = op.identity();
                    s_tp[i * THREADS + tid] = ex;
                }
            }
        }
    }
    __syncthreads();

    // ---- range aggregate: warp 0 folds the cnt*NW entries in order
    const int E = cnt * NW;
    const int per_lane = (E + kWarp - 1) / kWarp;
    S lane_fold = op.identity();
    if (warp == 0) {
        for (int e = lane * per_lane; e < E && e < (lane + 1) * per_lane; ++e) lane_fold = op.combine(lane_fold, s_wt[e]);
        S v = lane_fold;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {  // ordered reduction: lane 0 ends with lanes 0..31 in order
            const S other = shfl_down(v, o);
            if (lane + o < kWarp) v = op.combine(v, other);
        }
        if (lane == 0) s_range_agg = v;
    }
    __syncthreads();
    const S range_agg = s_range_agg;

    // ---- look-back over the ranges
    bool abort = false;
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
                    publish_tag(incw + r * SO, K, kFlagError, WS);
                    set_error(ctl.err, kErrTimeout);
                } else {
                    publish(incw + r * SO, op.combine(prefix, range_agg), kFlagInc, WS);
                }
            }
        }
    }
    if (abort) return;  // block-uniform

    // ---- exclusive prefix of every warp-tile entry (warp 0, in order)
    if (warp == 0) {
        S ex = shfl_up(warp_inclusive_scan(op, lane_fold), 1);
        if (lane == 0) ex = op.identity();
        S run = op.combine(prefix, ex);
        for (int e = lane * per_lane; e < E && e < (lane + 1) * per_lane; ++e) {
            const S agg = s_wt[e];
            s_wt[e] = run;
            run = op.combine(run, agg);
        }
    }
    __syncthreads();

    // ---- phase B: rescan, last tile of phase A first; warps independent
#pragma unroll
    for (int q = 0; q < PF; ++q)
        if (q < cnt) op.fetch(chunk0(t0 + cnt - 1 - q), n, raw[q]);
    for (int j0 = 0; j0 < cnt; j0 += PF) {
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int j = j0 + q;
            if (j < cnt) {
                const int i = cnt - 1 - j;
                S st[ITEMS];
                typename Op::Aux aux;
                const int64_t c0 = chunk0(t0 + i);
                op.build(c0, n, raw[q], st, aux);
                if (j + PF < cnt) op.fetch(chunk0(t0 + i - PF), n, raw[q]);
                S ex;
                if constexpr (KEEP) {
                    ex = s_tp[i * THREADS + tid];
                } else {
                    ex = shfl_up(warp_inclusive_scan(op, thread_agg(st)), 1);
                    if (lane == 0) ex = op.identity();
                }
                S run = op.combine(s_wt[i * NW + warp], ex);
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
    }
}

// Layout of one scan launch's region of the workspace: tagged aggregates and
// tagged inclusive prefixes, 8 bytes per 32-bit state word, both zeroed before
// the launch (tag 0 = nothing published).
struct ScanWs {
    size_t agg_off, inc_off, bytes;
};

inline ScanWs scan_ws_layout(int64_t num_tiles, size_t state_bytes) {
    ScanWs w;
    const size_t words = (size_t)num_tiles * (state_bytes / 4) * 8;
    w.agg_off = 0;
    w.inc_off = align_up(words, 256);
    w.bytes = align_up(w.inc_off + words, 256);
    return w;
}

constexpr int kScanThreads = 256;

template <class Op, int ITEMS> struct ScanShape {
    static constexpr int TILE = op_threads<Op>(0) * ITEMS;
    static int64_t tiles(int64_t n) { return (n + TILE - 1) / TILE; }
    static size_t region(int64_t n) { return scan_ws_layout(tiles(n), sizeof(typename Op::State)).bytes; }
};

// Resident blocks per SM of one range-scan instantiation (cached per device).
template <class Op, int ITEMS, bool REVERSE> int ranges_blocks_per_sm() {
    // Host threads may call at once: the entries are atomics (every writer
    // stores the same value).
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int b = cache[dev].load(std::memory_order_relaxed);
    if (b == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan_ranges<Op, kScanThreads, ITEMS, REVERSE>,
                                                          kScanThreads, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        cache[dev].store(b, std::memory_order_relaxed);
    }
    return b;
}

// An Op may ask for ranges of a fixed number of tiles (static constexpr int
// kRangeTiles) instead of one range per resident block: worth it when its
// phase-B re-read from DRAM costs more than the extra look-backs (measured).
template <class Op> constexpr int range_tiles_hint(long) { return 0; }
template <class Op> constexpr auto range_tiles_hint(int) -> decltype(Op::kRangeTiles, int()) { return Op::kRangeTiles; }

// Engine selection for tests and measurements: 0 automatic, 1 per-tile
// look-back only, 2 range-partitioned where it applies.
extern int g_scan_engine;
extern int g_scan_range_tiles;

// Queue one scan.  `ws` is the call's workspace (error word and counter slot
// `slot` in its header); `region` holds this launch's tile flags and states.
template <class Op, int ITEMS, bool REVERSE>
adc_status run_scan(const Op &op, int64_t n, void *ws, int slot, void *region, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    using Sh = ScanShape<Op, ITEMS>;
    const int64_t T = Sh::tiles(n);
    const ScanWs L = scan_ws_layout(T, sizeof(typename Op::State));
    char *w = static_cast<char *>(region);
    if (cudaMemsetAsync(w, 0, L.bytes, s) != cudaSuccess) return ADC_ERR_CUDA;
    const DevCtl ctl = make_ctl(ws, slot);
    if constexpr (per_tile_only<Op>(0)) {
        constexpr int TH = op_threads<Op>(0);
        constexpr size_t dyn = op_dyn_smem<Op>(0);
        if constexpr (dyn > 0) {
            if (cudaFuncSetAttribute(k_scan<Op, TH, ITEMS, REVERSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dyn) != cudaSuccess)
                return ADC_ERR_CUDA;
        }
        k_scan<Op, TH, ITEMS, REVERSE><<<(unsigned)T, TH, dyn, s>>>(
            op, n, T, reinterpret_cast<unsigned long long *>(w + L.agg_off),
            reinterpret_cast<unsigned long long *>(w + L.inc_off), ctl);
        return check_launch();
    } else {
    const int64_t G = (int64_t)num_sms() * ranges_blocks_per_sm<Op, ITEMS, REVERSE>();
    // Ranges: one per resident block by default; a tuned count launches more,
    // smaller ranges (blocks claim them in start order, so the look-back only
    // ever waits on running blocks).
    int64_t R = G;
    int rt = g_scan_range_tiles > 0 ? g_scan_range_tiles : range_tiles_hint<Op>(0);
    if constexpr (keep_prefix<Op>(0)) {  // one range per resident block, at most the kept tiles long
        constexpr int KT = keep_tiles<typename Op::State, kScanThreads>();
        if (rt <= 0) rt = (int)((T + G - 1) / G);
        if (rt > KT) rt = KT;
    }
    if (rt > 0) R = (T + rt - 1) / rt;
    if (R > T) R = T;
    const bool ranges = T <= (int64_t)range_max_tiles<typename Op::State>() * R &&
                        (g_scan_engine == 2 || g_scan_engine == 5 || (g_scan_engine == 0 && T >= 4 * G));
    if (ranges) {
        k_scan_ranges<Op, kScanThreads, ITEMS, REVERSE><<<(unsigned)R, kScanThreads, 0, s>>>(
            op, n, T, reinterpret_cast<unsigned long long *>(w + L.agg_off),
            reinterpret_cast<unsigned long long *>(w + L.inc_off), ctl);
        return check_launch();
    }
    k_scan<Op, kScanThreads, ITEMS, REVERSE><<<(unsigned)T, kScanThreads, 0, s>>>(
        op, n, T, reinterpret_cast<unsigned long long *>(w + L.agg_off),
        reinterpret_cast<unsigned long long *>(w + L.inc_off), ctl);
    return check_launch();
    }
}

}  // namespace adc
