// Single-pass scan with decoupled look-back (Merrill & Garland), forward or
// reverse, for any associative operator given as an Op class.
//
// An Op provides
//   using State;                         the scanned value
//   struct Aux;                          per-thread data carried from load to store
//   State identity() const;
//   State combine(const State& earlier, const State& later) const;   (logical order)
//   void  load (int64_t c0, int64_t n, State (&st)[ITEMS], Aux&) const;
//         fills st with the elements [c0, c0+ITEMS) in PHYSICAL order,
//         identity() beyond n
//   void  store(int64_t c0, int64_t n, const State (&inc)[ITEMS], const Aux&) const;
//         receives the inclusive scan values of those elements.
//
// REVERSE scans run in descending index order: tile claim t maps to physical
// tile T-1-t and the scan is inclusive from the right, i.e. a forward scan of
// the reversed array (the reversals of Figs 2, 4 and 7 are index maps here).
//
// Protocol per tile: claim a tile index from an atomic counter (so every tile
// a block waits on is already resident or finished), reduce the tile, publish
// its aggregate (flag AGG), look back over predecessors with one warp, 32
// tiles per step, until a tile with an inclusive prefix (flag INC) is found,
// publish the inclusive prefix, then rescan the tile from registers.  Every
// wait is bounded: on expiry the tile publishes ERROR, the error word gets
// kErrTimeout and the block leaves without storing.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace adc {

template <class Op, int THREADS, int ITEMS, bool REVERSE>
__global__ void __launch_bounds__(THREADS)
k_scan(const Op op, const int64_t n, const int64_t num_tiles, unsigned *__restrict__ flags,
       typename Op::State *__restrict__ agg, typename Op::State *__restrict__ inc, const DevCtl ctl) {
    using S = typename Op::State;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int NW = THREADS / kWarp;
    static_assert(NW <= kWarp, "block too large");
    __shared__ unsigned s_tile;
    __shared__ int s_abort;
    __shared__ S s_warp[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_tile = atomicAdd(ctl.counter, 1u);
        s_abort = 0;
    }
    __syncthreads();
    const long long t = s_tile;
    if (t == ctl.stall_tile) return;  // fault injection: this tile never publishes

    const int64_t p = REVERSE ? (num_tiles - 1 - t) : t;
    const int jc = REVERSE ? (THREADS - 1 - tid) : tid;
    const int64_t c0 = p * (int64_t)TILE + (int64_t)jc * ITEMS;

    S st[ITEMS];
    typename Op::Aux aux;
    op.load(c0, n, st, aux);

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
        const S total = shfl_idx(wi, NW - 1);
        S wex = shfl_up(wi, 1);
        if (lane == 0) wex = op.identity();
        S prefix = op.identity();
        bool abort = false;
        if (t == 0) {
            if (lane == 0) {
                inc[0] = total;
                st_release_u32(&flags[0], kFlagInc);
            }
        } else {
            if (lane == 0) {
                agg[t] = total;
                st_release_u32(&flags[t], kFlagAgg);
            }
            long long base = t - 1;
            S run = op.identity();
            while (true) {
                const long long tj = base - lane;  // lane 0: nearest predecessor
                unsigned f = kFlagInc;
                if (tj >= 0) f = spin_flag(&flags[tj], ctl.spin_limit);
                if (__any_sync(0xffffffffu, f == kFlagError)) {
                    abort = true;
                    break;
                }
                S v = op.identity();
                if (tj >= 0) v = (f == kFlagInc) ? load_cg(&inc[tj]) : load_cg(&agg[tj]);
                const unsigned incmask = __ballot_sync(0xffffffffu, f == kFlagInc);
                const int stop = incmask ? (__ffs(incmask) - 1) : (kWarp - 1);
                if (lane > stop) v = op.identity();
                // ordered reduction: farthest (highest lane) first
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const S other = shfl_down(v, o);
                    if (lane + o < kWarp) v = op.combine(other, v);
                }
                v = shfl_idx(v, 0);
                run = op.combine(v, run);
                if (incmask) break;
                base -= kWarp;
            }
            if (abort) {
                if (lane == 0) {
                    st_release_u32(&flags[t], kFlagError);
                    set_error(ctl.err, kErrTimeout);
                    s_abort = 1;
                }
            } else {
                prefix = run;
                if (lane == 0) {
                    inc[t] = op.combine(prefix, total);
                    st_release_u32(&flags[t], kFlagInc);
                }
            }
        }
        if (lane < NW) s_warp[lane] = op.combine(prefix, wex);
    }
    __syncthreads();
    if (s_abort) return;

    S run = op.combine(s_warp[warp], wexc);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int kk = REVERSE ? ITEMS - 1 - k : k;
        run = op.combine(run, st[kk]);
        st[kk] = run;
    }
    op.store(c0, n, st, aux);
}

// Layout of one scan launch's region of the workspace: [flags][agg][inc].
struct ScanWs {
    size_t flags_off, agg_off, inc_off, bytes;
};

inline ScanWs scan_ws_layout(int64_t num_tiles, size_t state_bytes) {
    ScanWs w;
    w.flags_off = 0;
    w.agg_off = align_up(w.flags_off + (size_t)num_tiles * 4, 256);
    w.inc_off = align_up(w.agg_off + (size_t)num_tiles * state_bytes, 256);
    w.bytes = align_up(w.inc_off + (size_t)num_tiles * state_bytes, 256);
    return w;
}

constexpr int kScanThreads = 256;

template <class Op, int ITEMS> struct ScanShape {
    static constexpr int TILE = kScanThreads * ITEMS;
    static int64_t tiles(int64_t n) { return (n + TILE - 1) / TILE; }
    static size_t region(int64_t n) { return scan_ws_layout(tiles(n), sizeof(typename Op::State)).bytes; }
};

// Queue one scan.  `ws` is the call's workspace (error word and counter slot
// `slot` in its header); `region` holds this launch's tile flags and states.
template <class Op, int ITEMS, bool REVERSE>
adc_status run_scan(const Op &op, int64_t n, void *ws, int slot, void *region, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    using Sh = ScanShape<Op, ITEMS>;
    const int64_t T = Sh::tiles(n);
    const ScanWs L = scan_ws_layout(T, sizeof(typename Op::State));
    char *w = static_cast<char *>(region);
    if (cudaMemsetAsync(w, 0, L.agg_off, s) != cudaSuccess) return ADC_ERR_CUDA;
    const DevCtl ctl = make_ctl(ws, slot);
    k_scan<Op, kScanThreads, ITEMS, REVERSE><<<(unsigned)T, kScanThreads, 0, s>>>(
        op, n, T, reinterpret_cast<unsigned *>(w + L.flags_off),
        reinterpret_cast<typename Op::State *>(w + L.agg_off), reinterpret_cast<typename Op::State *>(w + L.inc_off),
        ctl);
    return check_launch();
}

}  // namespace adc
