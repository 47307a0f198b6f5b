// General reduce_by_index (Sec. 4.1, Fig. 4) for the non-commutative
// linFnComp operator: a stable sort of [0..n-1] by key, a gather of the values,
// then segmented scans over the sorted values.
//
// Sort.  Keys outside [0, m) are mapped to the bucket m, which sorts last and
// is ignored.  With B = m + 1 <= 2048 buckets the sort is ONE stable counting
// pass; larger m uses LSD passes of 8-bit digits.  A pass is
//   count   : per tile of 4096 keys, a shared-memory count per bucket, stored
//             bucket-major so that
//   scan    : one exclusive +-scan (the decoupled-look-back engine) gives
//             every (bucket, tile) its output offset, and
//   scatter : each warp ranks its 512 keys in order (match-any within a round
//             of 32, per-warp running counts in shared memory), warps are
//             offset in order, and every element is written to
//             offset + rank: stable by construction.
// The last pass also gathers the values into sorted order.
//
// Forward: one forward segmented scan over the sorted values whose store
// writes hist[k] = hist0[k] . (segment total) at each segment end.
// vjp (Fig. 4): the forward segmented exclusive scan gives l_i (and the
// per-bin totals for hist0's adjoint); a reverse segmented exclusive scan
// gives r_i and, fused into its store, the map
//   vbar = d(hist0[k] . l_i . v_i . r_i)/d v_i ^T histbar[k]
// scattered back through the permutation (0 for out-of-range keys).
// Flags are computed on the fly from neighbouring sorted keys (never stored):
// segment start = (i == 0 || k[i-1] != k[i]), end = (i == n-1 || k[i+1] != k[i]),
// which is the reading of Fig. 4's flag_rev as "reversed position starts a
// segment iff the original position ends one".
#include "block_scan.cuh"
#include "common.cuh"
#include "internal.h"
#include "scan_engine.cuh"
#include "tile_io.cuh"

namespace adc {

constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;               // 8 warps x 16 rounds x 32 keys
constexpr int kSortRounds = kSortTile / kSortThreads;
constexpr int kMaxSingleBuckets = 2048;

struct SortPass {
    int shift;      // digit = (key >> shift) & mask
    unsigned mask;  // all ones for the single counting pass
    int buckets;    // number of digit values
};

__device__ __forceinline__ int32_t mapped_key(int32_t k, int64_t m) {
    return ((uint32_t)k < (uint64_t)m) ? k : (int32_t)m;
}

// ------------------------------------------------------------------ count --
__global__ void __launch_bounds__(kSortThreads)
k_sort_count(const int32_t *__restrict__ keys, const int64_t n, const int64_t m, const int first, const SortPass P,
             const int64_t T, int32_t *__restrict__ counts) {
    extern __shared__ int32_t s_cnt[];
    for (int b = threadIdx.x; b < P.buckets; b += kSortThreads) s_cnt[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) {
            const int32_t k = first ? mapped_key(__ldcs(keys + i), m) : __ldcs(keys + i);
            atomicAdd(&s_cnt[((uint32_t)k >> P.shift) & P.mask], 1);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < P.buckets; b += kSortThreads) counts[(int64_t)b * T + blockIdx.x] = s_cnt[b];
}

// Exclusive +-scan of the bucket-major count matrix.
template <int ITEMS> struct ExclAddI32 {
    using State = int32_t;
    struct Aux { int32_t own[ITEMS]; };
    struct Raw { int32_t v[ITEMS]; };
    const int32_t *in;
    int32_t *out;
    __device__ int32_t identity() const { return 0; }
    __device__ int32_t combine(int32_t a, int32_t b) const { return a + b; }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const { load_chunk(in, c0, n, r.v, 0); }
    __device__ void build(int64_t, int64_t, const Raw &r, int32_t (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            st[k] = r.v[k];
            aux.own[k] = r.v[k];
        }
    }
    __device__ void store(int64_t c0, int64_t n, const int32_t (&st)[ITEMS], const Aux &aux) const {
        int32_t o[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) o[k] = st[k] - aux.own[k];
        store_chunk(out, c0, n, o);
    }
};
constexpr int kCountItems = 16;

// ---------------------------------------------------------------- scatter --
template <typename V>
__global__ void __launch_bounds__(kSortThreads)
k_sort_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ perm_in, const int64_t n, const int64_t m,
               const int first, const SortPass P, const int64_t T, const int32_t *__restrict__ offsets,
               int32_t *__restrict__ keys_out, int32_t *__restrict__ perm_out, const V *__restrict__ vals,
               V *__restrict__ vals_out) {
    extern __shared__ int32_t s_w[];  // [8 warps][buckets]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kSortThreads / kWarp;
    for (int j = threadIdx.x; j < NW * P.buckets; j += kSortThreads) s_w[j] = 0;
    __syncthreads();
    int32_t *wc = s_w + warp * P.buckets;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (kSortTile / NW);
    const unsigned lt = (1u << lane) - 1u;
    int32_t kk[kSortRounds], dg[kSortRounds], rk[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + (int64_t)r * kWarp + lane;
        int32_t k = 0, d = P.buckets;  // past the end: a digit value no bucket has
        if (i < n) {
            k = first ? mapped_key(__ldcs(keys + i), m) : __ldcs(keys + i);
            d = ((uint32_t)k >> P.shift) & P.mask;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = __popc(peers & lt);
        const int cnt = __popc(peers);
        int prior = 0;
        if (d < P.buckets) prior = wc[d];
        __syncwarp();
        if (d < P.buckets && before == 0) wc[d] = prior + cnt;
        __syncwarp();
        kk[r] = k;
        dg[r] = d;
        rk[r] = prior + before;
    }
    __syncthreads();
    // warp offsets within the tile, plus the tile's global offset per bucket
    for (int b = threadIdx.x; b < P.buckets; b += kSortThreads) {
        int32_t run = offsets[(int64_t)b * T + blockIdx.x];
        for (int w = 0; w < NW; ++w) {
            const int32_t c = s_w[w * P.buckets + b];
            s_w[w * P.buckets + b] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + (int64_t)r * kWarp + lane;
        if (i < n) {
            const int32_t dest = wc[dg[r]] + rk[r];
            const int32_t src = first ? (int32_t)i : __ldcs(perm_in + i);
            keys_out[dest] = kk[r];
            perm_out[dest] = src;
            if (vals_out) vals_out[dest] = vals[src];
        }
    }
}

// ------------------------------------------------------- segmented scans --
template <typename T> struct SegS {
    Pair<T> v;
    uint32_t f;
    uint32_t pad;
};

template <typename T> __device__ __forceinline__ Pair<T> lin(const Pair<T> &a, const Pair<T> &b) {
    return {b.b + b.c * a.b, b.c * a.c};  // (b1,c1) . (b2,c2) = (b2 + c2*b1, c2*c1)
}
template <typename T> __device__ __forceinline__ Pair<T> lin_id() { return {T(0), T(1)}; }

// d(l . v . r)/dv ^T g for linFnComp.
template <typename T> __device__ __forceinline__ Pair<T> lin_adj(const Pair<T> &l, const Pair<T> &r, const Pair<T> &g) {
    return {r.c * g.b, r.c * (l.b * g.b + l.c * g.c)};
}

// Forward segmented EXCLUSIVE scan: element i carries v_{i-1} (identity at a
// segment start), so the inclusive value at i is l_i.  The store writes l_i
// (vjp) and, at segment ends, the segment total to hist / xs.
template <typename T, int ITEMS> struct SegFwd {
    using State = SegS<T>;
    struct Aux {
        int32_t k[ITEMS];
        int32_t knext;
        Pair<T> v[ITEMS];
    };
    const int32_t *sk;
    const Pair<T> *sv;
    const Pair<T> *h0;
    int64_t m;
    Pair<T> *hist;  // forward: hist[k] = h0[k] . total (may be null)
    Pair<T> *xs;    // vjp: per-bin totals (may be null)
    Pair<T> *lout;  // vjp: l_i (may be null)
    __device__ State identity() const { return {lin_id<T>(), 0u, 0u}; }
    __device__ State combine(const State &a, const State &b) const {
        return {b.f ? b.v : lin(a.v, b.v), a.f | b.f, 0u};
    }
    struct Raw {
        int32_t k[ITEMS];
        int32_t kprev, knext;
        Pair<T> v[ITEMS];
        Pair<T> vprev;
    };
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(sk, c0, n, r.k, (int32_t)0);
        load_chunk(sv, c0, n, r.v, lin_id<T>());
        r.kprev = (c0 > 0 && c0 <= n) ? sk[c0 - 1] : -1;
        r.vprev = (c0 > 0 && c0 <= n) ? sv[c0 - 1] : lin_id<T>();
        r.knext = (c0 + ITEMS < n) ? sk[c0 + ITEMS] : -1;
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
        aux.knext = r.knext;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            aux.k[j] = r.k[j];
            aux.v[j] = r.v[j];
            const bool start = (c0 + j == 0) || ((j == 0 ? r.kprev : r.k[j - 1]) != r.k[j]);
            const Pair<T> prev = (j == 0) ? r.vprev : r.v[j - 1];
            st[j] = (c0 + j < n) ? State{start ? lin_id<T>() : prev, start ? 1u : 0u, 0u} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        if (lout) {
            Pair<T> l[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) l[j] = st[j].v;
            store_chunk(lout, c0, n, l);
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (c0 + j >= n) break;
            const int32_t k = aux.k[j];
            const int32_t kn = (j + 1 < ITEMS) ? aux.k[j + 1] : aux.knext;
            const bool end = (c0 + j == n - 1) || (kn != k);
            if (end && k < m) {
                const Pair<T> tot = lin(st[j].v, aux.v[j]);
                if (xs) xs[k] = tot;
                if (hist) hist[k] = h0 ? lin(h0[k], tot) : tot;
            }
        }
    }
};

// Reverse segmented EXCLUSIVE scan (logical order = decreasing index):
// element i carries v_{i+1} (identity at a segment end), so the inclusive
// value at i is r_i = v_{i+1} . ... . v_end.  Fused map + scatter in store.
template <typename T, int ITEMS> struct SegRev {
    using State = SegS<T>;
    struct Aux {
        int32_t k[ITEMS];
        int32_t knext;
        Pair<T> v[ITEMS];
    };
    const int32_t *sk;
    const Pair<T> *sv;
    const int32_t *perm;
    const Pair<T> *lbuf;
    const Pair<T> *h0;
    const Pair<T> *hb;
    Pair<T> *vbar;
    int64_t m;
    int accumulate;
    __device__ State identity() const { return {lin_id<T>(), 0u, 0u}; }
    // logical combine: `e` is physically before `acc`
    __device__ State combine(const State &acc, const State &e) const {
        return {e.f ? e.v : lin(e.v, acc.v), acc.f | e.f, 0u};
    }
    struct Raw {
        int32_t k[ITEMS];
        int32_t knext;
        Pair<T> v[ITEMS];
        Pair<T> vnext;
    };
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(sk, c0, n, r.k, (int32_t)0);
        load_chunk(sv, c0, n, r.v, lin_id<T>());
        r.knext = (c0 + ITEMS < n) ? sk[c0 + ITEMS] : -1;
        r.vnext = (c0 + ITEMS < n) ? sv[c0 + ITEMS] : lin_id<T>();
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
        aux.knext = r.knext;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            aux.k[j] = r.k[j];
            aux.v[j] = r.v[j];
            const int32_t kn = (j + 1 < ITEMS) ? r.k[j + 1] : r.knext;
            const bool end = (c0 + j == n - 1) || (kn != r.k[j]);
            const Pair<T> nxt = (j + 1 < ITEMS) ? r.v[j + 1] : r.vnext;
            st[j] = (c0 + j < n) ? State{end ? lin_id<T>() : nxt, end ? 1u : 0u, 0u} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        Pair<T> l[ITEMS];
        int32_t p[ITEMS];
        load_chunk(lbuf, c0, n, l, lin_id<T>());
        load_chunk(perm, c0, n, p, (int32_t)0);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (c0 + j >= n) break;
            const int32_t k = aux.k[j];
            Pair<T> g{T(0), T(0)};
            if (k < m) {
                const Pair<T> lp = h0 ? lin(h0[k], l[j]) : l[j];
                g = lin_adj(lp, st[j].v, hb[k]);
            }
            Pair<T> *dst = vbar + p[j];
            if (accumulate) {
                const Pair<T> o = *dst;
                *dst = {o.b + g.b, o.c + g.c};
            } else {
                *dst = g;
            }
        }
    }
};

template <typename T>
__global__ void k_lin_init(Pair<T> *__restrict__ a, const Pair<T> *__restrict__ src, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        a[j] = src ? src[j] : Pair<T>{T(0), T(1)};
}

// hist0bar[j] = d(h0 . xs)/d h0 ^T histbar[j]
template <typename T>
__global__ void k_lin_h0bar(const Pair<T> *__restrict__ xs, const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ h0b,
                            const int64_t m, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const Pair<T> g = lin_adj(lin_id<T>(), xs[j], hb[j]);
        h0b[j] = accumulate ? Pair<T>{h0b[j].b + g.b, h0b[j].c + g.c} : g;
    }
}

// ================================================================== host ==
template <typename T> struct SegItems { static constexpr int v = 16 / sizeof(T) >= 4 ? 4 : 2; };

static void plan_passes(int64_t m, SortPass *passes, int *np) {
    const int64_t B = m + 1;
    if (B <= kMaxSingleBuckets) {
        passes[0] = {0, 0xffffffffu, (int)B};
        *np = 1;
        return;
    }
    int bits = 0;
    while (((int64_t)1 << bits) < B) ++bits;
    int k = 0;
    for (int sh = 0; sh < bits; sh += 8) passes[k++] = {sh, 0xffu, 256};
    *np = k;
}

struct GenLayout {
    size_t counts, offsets, scanreg, keys_tmp, perm_tmp, lbuf, xs, segreg, bytes;
};

static GenLayout gen_layout(size_t sb, int64_t n, int64_t m) {
    SortPass P[4];
    int np;
    plan_passes(m, P, &np);
    int maxb = 0;
    for (int i = 0; i < np; ++i) maxb = P[i].buckets > maxb ? P[i].buckets : maxb;
    const int64_t T = (n + kSortTile - 1) / kSortTile;
    const int64_t cn = (int64_t)maxb * (T > 0 ? T : 1);
    GenLayout L;
    size_t o = kWsHeader;
    L.counts = o;
    o = align_up(o + cn * 4, 256);
    L.offsets = o;
    o = align_up(o + cn * 4, 256);
    L.scanreg = o;
    o = align_up(o + ScanShape<ExclAddI32<kCountItems>, kCountItems>::region(cn), 256);
    L.keys_tmp = o;
    o = align_up(o + (size_t)n * 4, 256);
    L.perm_tmp = o;
    o = align_up(o + (size_t)n * 4, 256);
    L.lbuf = o;
    o = align_up(o + (size_t)n * 2 * sb, 256);
    L.xs = o;
    o = align_up(o + (size_t)m * 2 * sb, 256);
    L.segreg = o;
    // both segmented scans use the same tile shape and state
    const size_t seg = sb == 8 ? ScanShape<SegFwd<double, SegItems<double>::v>, SegItems<double>::v>::region(n)
                               : ScanShape<SegFwd<float, SegItems<float>::v>, SegItems<float>::v>::region(n);
    o = align_up(o + seg, 256);
    L.bytes = o;
    return L;
}

// m <= 2047 fp32 / 1023 fp64 (and not forced to the global sort): the hierarchical path of
// hist_lin.cu; otherwise the global stable radix sort below.
static bool use_local(adc_dtype dt, int64_t m) { return linh_applicable(dt, m) && hist_forced_strategy() != 2; }

size_t histgen_ws_bytes(adc_dtype dt, int64_t n, int64_t m) {
    if (use_local(dt, m)) return linh_ws_bytes(dt, n, m);
    return gen_layout(dt == ADC_F64 ? 8 : 4, n, m).bytes;
}

// saved: perm [n] i32, sorted keys [n] i32, sorted values [n] pairs
size_t histgen_saved_bytes(adc_dtype dt, int64_t n, int64_t m) {
    if (use_local(dt, m)) return linh_saved_bytes(dt, n, m);
    const size_t sb = dt == ADC_F64 ? 8 : 4;
    return align_up((size_t)n * 4, 256) * 2 + (size_t)n * 2 * sb + 256;
}

struct SavedPtrs {
    int32_t *perm, *skeys;
    void *svals;
};
static SavedPtrs saved_ptrs(void *saved, int64_t n) {
    char *s = static_cast<char *>(saved);
    const size_t a = align_up((size_t)n * 4, 256);
    return {reinterpret_cast<int32_t *>(s), reinterpret_cast<int32_t *>(s + a), s + 2 * a};
}

template <typename T>
static adc_status sort_by_key(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const SavedPtrs &out,
                              void *ws, const GenLayout &L, cudaStream_t s) {
    SortPass P[4];
    int np;
    plan_passes(m, P, &np);
    char *w = static_cast<char *>(ws);
    const int64_t NT = (n + kSortTile - 1) / kSortTile;
    int32_t *counts = reinterpret_cast<int32_t *>(w + L.counts);
    int32_t *offs = reinterpret_cast<int32_t *>(w + L.offsets);
    // ping-pong so that the last pass lands in `out`
    int32_t *kb[2] = {reinterpret_cast<int32_t *>(w + L.keys_tmp), out.skeys};
    int32_t *pb[2] = {reinterpret_cast<int32_t *>(w + L.perm_tmp), out.perm};
    const int32_t *kin = keys;
    const int32_t *pin = nullptr;
    for (int p = 0; p < np; ++p) {
        const int dst = ((np - 1 - p) % 2 == 0) ? 1 : 0;
        const bool last = p == np - 1;
        const size_t cs = (size_t)P[p].buckets * 4;
        k_sort_count<<<(unsigned)NT, kSortThreads, cs, s>>>(kin, n, m, p == 0, P[p], NT, counts);
        ExclAddI32<kCountItems> ex{counts, offs};
        adc_status st = run_scan<ExclAddI32<kCountItems>, kCountItems, false>(ex, (int64_t)P[p].buckets * NT, ws, 2 + p,
                                                                              w + L.scanreg, s);
        if (st != ADC_OK) return st;
        const size_t ss = (size_t)P[p].buckets * 4 * (kSortThreads / kWarp);
        if (ss > 48 * 1024 &&
            cudaFuncSetAttribute(k_sort_scatter<Pair<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss) !=
                cudaSuccess)
            return ADC_ERR_CUDA;
        k_sort_scatter<Pair<T>><<<(unsigned)NT, kSortThreads, ss, s>>>(
            kin, pin, n, m, p == 0, P[p], NT, offs, kb[dst], pb[dst], vals,
            last ? static_cast<Pair<T> *>(out.svals) : nullptr);
        if ((st = check_launch()) != ADC_OK) return st;
        kin = kb[dst];
        pin = pb[dst];
    }
    return ADC_OK;
}

template <typename T>
static adc_status gen_fwd_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const Pair<T> *h0,
                            Pair<T> *hist, void *saved, void *ws, cudaStream_t s) {
    const GenLayout L = gen_layout(sizeof(T), n, m);
    const SavedPtrs sp = saved_ptrs(saved, n);
    const unsigned gm = (unsigned)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096);
    k_lin_init<T><<<gm > 0 ? gm : 1, 256, 0, s>>>(hist, h0, m);
    adc_status st = check_launch();
    if (st != ADC_OK || n == 0) return st;
    if ((st = sort_by_key<T>(n, m, keys, vals, sp, ws, L, s)) != ADC_OK) return st;
    constexpr int I = SegItems<T>::v;
    SegFwd<T, I> op{sp.skeys, static_cast<const Pair<T> *>(sp.svals), h0, m, hist, nullptr, nullptr};
    return run_scan<SegFwd<T, I>, I, false>(op, n, ws, 10, static_cast<char *>(ws) + L.segreg, s);
}

template <typename T>
static adc_status gen_vjp_t(int64_t n, int64_t m, const Pair<T> *h0, const void *saved, const Pair<T> *hb,
                            Pair<T> *vb, Pair<T> *h0b, int acc, void *ws, cudaStream_t s) {
    const GenLayout L = gen_layout(sizeof(T), n, m);
    const SavedPtrs sp = saved_ptrs(const_cast<void *>(saved), n);
    char *w = static_cast<char *>(ws);
    Pair<T> *xs = reinterpret_cast<Pair<T> *>(w + L.xs);
    Pair<T> *lbuf = reinterpret_cast<Pair<T> *>(w + L.lbuf);
    const unsigned gm = (unsigned)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096);
    k_lin_init<T><<<gm > 0 ? gm : 1, 256, 0, s>>>(xs, nullptr, m);
    adc_status st = check_launch();
    if (st != ADC_OK) return st;
    constexpr int I = SegItems<T>::v;
    if (n > 0) {
        SegFwd<T, I> fw{sp.skeys, static_cast<const Pair<T> *>(sp.svals), h0, m, nullptr, xs, lbuf};
        if ((st = run_scan<SegFwd<T, I>, I, false>(fw, n, ws, 10, w + L.segreg, s)) != ADC_OK) return st;
        SegRev<T, I> rv{sp.skeys, static_cast<const Pair<T> *>(sp.svals), sp.perm, lbuf, h0, hb, vb, m, acc};
        if ((st = run_scan<SegRev<T, I>, I, true>(rv, n, ws, 11, w + L.segreg, s)) != ADC_OK) return st;
    }
    if (h0b) {
        k_lin_h0bar<T><<<gm > 0 ? gm : 1, 256, 0, s>>>(xs, hb, h0b, m, acc);
        return check_launch();
    }
    return ADC_OK;
}

// Exclusive +-scan of an int32 array (count matrices of the partitioned passes).
size_t excl_scan_i32_region(int64_t n) { return ScanShape<ExclAddI32<kCountItems>, kCountItems>::region(n); }

adc_status excl_scan_i32(const int32_t *in, int32_t *out, int64_t n, void *ws, int slot, void *region,
                         cudaStream_t s) {
    ExclAddI32<kCountItems> ex{in, out};
    return run_scan<ExclAddI32<kCountItems>, kCountItems, false>(ex, n, ws, slot, region, s);
}

adc_status histgen_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                       void *hist, void *saved, void *ws, cudaStream_t s) {
    if (use_local(dt, m)) return linh_fwd(dt, n, m, keys, vals, hist0, hist, saved, ws, s);
    if (dt == ADC_F64)
        return gen_fwd_t<double>(n, m, keys, static_cast<const Pair<double> *>(vals),
                                 static_cast<const Pair<double> *>(hist0), static_cast<Pair<double> *>(hist), saved, ws,
                                 s);
    return gen_fwd_t<float>(n, m, keys, static_cast<const Pair<float> *>(vals), static_cast<const Pair<float> *>(hist0),
                            static_cast<Pair<float> *>(hist), saved, ws, s);
}

adc_status histgen_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                       const void *hist, const void *saved, const void *histbar, void *valsbar, void *hist0bar,
                       int accumulate, void *ws, cudaStream_t s) {
    (void)hist;
    if (use_local(dt, m)) return linh_vjp(dt, n, m, keys, vals, saved, histbar, valsbar, hist0bar, accumulate, s);
    if (dt == ADC_F64)
        return gen_vjp_t<double>(n, m, static_cast<const Pair<double> *>(hist0), saved,
                                 static_cast<const Pair<double> *>(histbar), static_cast<Pair<double> *>(valsbar),
                                 static_cast<Pair<double> *>(hist0bar), accumulate, ws, s);
    return gen_vjp_t<float>(n, m, static_cast<const Pair<float> *>(hist0), saved,
                            static_cast<const Pair<float> *>(histbar), static_cast<Pair<float> *>(valsbar),
                            static_cast<Pair<float> *>(hist0bar), accumulate, ws, s);
}

}  // namespace adc
