// General reduce_by_index for the non-commutative linFnComp operator with up
// to a few thousand bins (Sec. 4.1, Fig. 4).  The paper sorts the elements by
// bin (stable), then runs segmented scans; here the stable sort is done
// hierarchically so that no pass moves the whole input more than once:
//   1. per chunk of kLChunk elements (one block): a stable counting sort of the
//      chunk by bin in shared memory (warp ranks from per-bit ballots, per-warp
//      bin counters, so equal bins keep index order), then a segmented fold per
//      bin -> the chunk's partial P[bin][chunk] (identity where the bin is
//      absent);
//   2. across chunks, per bin, two segmented scans of the small [m][chunks]
//      matrix with the look-back engine: L[bin][c] = hist0 . P[bin][0..c-1]
//      and R[bin][c] = P[bin][c+1..]; hist = L . P at the last chunk, and the
//      bin total A = P[bin][0] . R[bin][0] (for hist0bar);
//   3. vjp: per chunk again the stable local sort, in-chunk segmented
//      exclusive prefix and suffix, l_i = L . prefix_i, r_i = suffix_i . R, and
//      vbar_i = d(l_i . v_i . r_i)/dv_i ^T histbar[k_i], put back in element
//      order in shared memory and written coalesced.
// Within every bin the values meet in index order, as the sequential
// definition requires; only the bracketing differs (associativity).
// Residuals: L, R and A (about 2 * 8 * m * n / kLChunk bytes) instead of the
// global sort's permutation, sorted keys and sorted values (16 bytes/element).
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"
#include "scan_engine.cuh"
#include "tile_io.cuh"

namespace adc {

constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / kWarp;
// Bins fit 16 bits, and the vjp's shared memory (per-warp counters, the
// sorted chunk, prefixes, per-bin L, R, histbar) fits one block: 2047 bins for
// fp32, 1023 for fp64.
template <typename T> constexpr int64_t lmax_bins() { return sizeof(T) == 4 ? 2047 : 1023; }
template <typename T> struct LChunk {
    static constexpr int kRounds = sizeof(T) == 4 ? 16 : 8;     // rounds of 32 elements per warp
    static constexpr int kSize = kLThreads * kRounds;           // elements per chunk (block)
    static constexpr int kSpan = kRounds;                       // sorted positions per thread
    static constexpr int kPad = kSize + kSize / 16;             // padded shared arrays
};
// Sorted position -> padded shared index: one spare slot every 16, so that a
// thread walking 16 consecutive positions does not collide with its neighbours.
__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }
__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) / 16 * 16; }

template <typename T> __device__ __forceinline__ Pair<T> lf(const Pair<T> &a, const Pair<T> &b) {
    return {b.b + b.c * a.b, b.c * a.c};  // (b1,c1) . (b2,c2) = (b2 + c2*b1, c2*c1)
}
template <typename T> __device__ __forceinline__ Pair<T> lf_id() { return {T(0), T(1)}; }
// d(l . v . r)/dv ^T g for linFnComp
template <typename T> __device__ __forceinline__ Pair<T> lf_adj(const Pair<T> &l, const Pair<T> &r, const Pair<T> &g) {
    return {r.c * g.b, r.c * (l.b * g.b + l.c * g.c)};
}

// Segmented-scan state: flag = a segment boundary lies inside.
template <typename T> struct LSeg {
    Pair<T> v;
    uint32_t f;
    uint32_t pad;
};
template <typename T> struct LSegFwdOp {  // physical order: a before b
    __device__ LSeg<T> identity() const { return {lf_id<T>(), 0u, 0u}; }
    __device__ LSeg<T> combine(const LSeg<T> &a, const LSeg<T> &b) const {
        return {b.f ? b.v : lf(a.v, b.v), a.f | b.f, 0u};
    }
};
template <typename T> struct LSegRevOp {  // logical order decreasing index: e lies physically before acc
    __device__ LSeg<T> identity() const { return {lf_id<T>(), 0u, 0u}; }
    __device__ LSeg<T> combine(const LSeg<T> &acc, const LSeg<T> &e) const {
        return {e.f ? e.v : lf(e.v, acc.v), acc.f | e.f, 0u};
    }
};

// Block-wide exclusive scan of one state per thread, in thread order (fwd) or
// reverse thread order (rev).  Two __syncthreads().
template <class Op, typename S, bool REV>
__device__ __forceinline__ S lblock_excl(const Op &op, const S &a, S *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // reverse order = a forward scan over mirrored lanes and warps
    const int vl = REV ? (kWarp - 1 - lane) : lane;
    const int vw = REV ? (kLWarps - 1 - warp) : warp;
    S x = a;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const S up = REV ? shfl_down(x, o) : shfl_up(x, o);
        if (vl >= o) x = op.combine(up, x);
    }
    if (vl == kWarp - 1) s_w[vw] = x;
    S ex = REV ? shfl_down(x, 1) : shfl_up(x, 1);
    if (vl == 0) ex = op.identity();
    __syncthreads();
    S before = op.identity();
#pragma unroll
    for (int w = 0; w < kLWarps; ++w)
        if (w < vw) before = op.combine(before, s_w[w]);
    __syncthreads();
    return op.combine(before, ex);
}

// ------------------------------------------------------------ chunk pass --
// VJP = false: writes P[bin * nc + chunk].  VJP = true: writes vbar.
template <typename T, bool VJP>
__global__ void __launch_bounds__(kLThreads)
k_linh_chunk(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals, const int64_t n, const int m,
             const int64_t nc, Pair<T> *__restrict__ P, const Pair<T> *__restrict__ L, const Pair<T> *__restrict__ R,
             const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ vbar, const int accumulate) {
    using C = LChunk<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [shared region: per-warp counters, then fwd bin totals / vjp outputs] [values] [bins] [vjp: src, prefixes]
    const size_t region = (size_t)kLWarps * m * 4 > (VJP ? (size_t)C::kSize * sizeof(Pair<T>) : (size_t)m * sizeof(Pair<T>))
                              ? (size_t)kLWarps * m * 4
                              : (VJP ? (size_t)C::kSize * sizeof(Pair<T>) : (size_t)m * sizeof(Pair<T>));
    int32_t *s_cnt = reinterpret_cast<int32_t *>(smem_raw);
    Pair<T> *s_tot = reinterpret_cast<Pair<T> *>(smem_raw);  // fwd, after placement
    Pair<T> *s_out = reinterpret_cast<Pair<T> *>(smem_raw);  // vjp, after placement
    Pair<T> *s_val = reinterpret_cast<Pair<T> *>(smem_raw + al16(region));
    uint16_t *s_bin = reinterpret_cast<uint16_t *>(s_val + C::kPad);
    uint16_t *s_src = s_bin + C::kPad;
    Pair<T> *s_pre = reinterpret_cast<Pair<T> *>(smem_raw + al16(region) + (size_t)C::kPad * sizeof(Pair<T>) +
                                                 al16((size_t)C::kPad * 4));
    Pair<T> *s_lrh = s_pre + C::kPad;  // vjp: L, R and histbar of every bin for this chunk
    __shared__ int32_t s_part[kLWarps];
    __shared__ LSeg<T> s_seg[kLWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    const int64_t base = c * C::kSize;
    const int len = (int)((n - base) < (int64_t)C::kSize ? (n - base) : (int64_t)C::kSize);  // may be <= 0 when n = 0
    for (int j = tid; j < kLWarps * m; j += kLThreads) s_cnt[j] = 0;
    __syncthreads();

    // ---- stable ranks: warp w owns elements [w * 32 * kRounds, ...), rounds in order
    int32_t *wc = s_cnt + warp * m;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t pk[C::kRounds];  // bin << 16 | rank within (warp, bin); bin == m: absent
    int32_t kk[C::kRounds];
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {  // all loads in flight before the first use
        const int t = warp * (kWarp * C::kRounds) + r * kWarp + lane;
        kk[r] = t < len ? __ldcs(keys + base + t) : -1;
    }
    const int nbits = 32 - __clz(m);  // bits of the bin values 0..m (m: absent)
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int d = in_range(kk[r], m) ? kk[r] : m;
        // lanes holding the same bin: intersect one ballot per bit of d
        unsigned peers = 0xffffffffu;
        for (int bit = 0; bit < nbits; ++bit) {
            const unsigned b = __ballot_sync(0xffffffffu, (d >> bit) & 1);
            peers &= ((d >> bit) & 1) ? b : ~b;
        }
        const int before = __popc(peers & lt);
        int prior = 0;
        if (d < m) prior = wc[d];
        __syncwarp();
        if (d < m && before == 0) wc[d] = prior + __popc(peers);
        __syncwarp();
        pk[r] = ((uint32_t)d << 16) | (uint32_t)(prior + before);
    }
    __syncthreads();

    // ---- bin starts: exclusive scan over bins of the per-bin totals, warps in order within a bin
    const int per = (m + kLThreads - 1) / kLThreads;
    const int b0 = tid * per, b1 = (b0 + per < m) ? b0 + per : m;
    int32_t sum = 0;
    for (int b = b0; b < b1; ++b)
        for (int w = 0; w < kLWarps; ++w) sum += s_cnt[w * m + b];
    int32_t inc = sum;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == kWarp - 1) s_part[warp] = inc;
    __syncthreads();
    int32_t run = inc - sum, V = 0;
#pragma unroll
    for (int w = 0; w < kLWarps; ++w) {
        if (w < warp) run += s_part[w];
        V += s_part[w];
    }
    for (int b = b0; b < b1; ++b)
        for (int w = 0; w < kLWarps; ++w) {
            const int32_t x = s_cnt[w * m + b];
            s_cnt[w * m + b] = run;
            run += x;
        }
    __syncthreads();

    // ---- placement (values read here, once, coalesced, all in flight together)
    Pair<T> vv[C::kRounds];
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int t = warp * (kWarp * C::kRounds) + r * kWarp + lane;
        if ((int)(pk[r] >> 16) < m) vv[r] = vals[base + t];
    }
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int t = warp * (kWarp * C::kRounds) + r * kWarp + lane;
        const int d = (int)(pk[r] >> 16);
        if (d < m) {
            const int p = pad16(s_cnt[warp * m + d] + (int)(pk[r] & 0xffffu));
            s_val[p] = vv[r];
            s_bin[p] = (uint16_t)d;
            if (VJP) s_src[p] = (uint16_t)t;
        }
    }
    __syncthreads();
    if (!VJP) {
        for (int j = tid; j < m; j += kLThreads) s_tot[j] = lf_id<T>();
    } else {
        for (int j = tid; j < C::kSize; j += kLThreads) s_out[j] = Pair<T>{T(0), T(0)};
        for (int j = tid; j < m; j += kLThreads) {
            s_lrh[3 * j] = L[(int64_t)j * nc + c];
            s_lrh[3 * j + 1] = R[(int64_t)j * nc + c];
            s_lrh[3 * j + 2] = hb[j];
        }
    }
    __syncthreads();

    // ---- forward segmented walk over this thread's sorted positions
    const int p0 = tid * C::kSpan;
    const LSegFwdOp<T> fop;
    LSeg<T> agg = fop.identity();
#pragma unroll
    for (int j = 0; j < C::kSpan; ++j) {
        const int p = p0 + j;
        if (p < V) {
            const int q = pad16(p);
            const bool head = p == 0 || s_bin[q] != s_bin[pad16(p - 1)];
            agg = fop.combine(agg, LSeg<T>{s_val[q], head ? 1u : 0u, 0u});
        }
    }
    const LSeg<T> carry = lblock_excl<LSegFwdOp<T>, LSeg<T>, false>(fop, agg, s_seg);
    Pair<T> acc = carry.v;
#pragma unroll
    for (int j = 0; j < C::kSpan; ++j) {
        const int p = p0 + j;
        if (p < V) {
            const int q = pad16(p);
            const int bin = s_bin[q];
            if (p == 0 || bin != s_bin[pad16(p - 1)]) acc = lf_id<T>();
            if (VJP) s_pre[q] = acc;  // exclusive in-chunk prefix of this bin
            acc = lf(acc, s_val[q]);
            if (!VJP && (p == V - 1 || bin != s_bin[pad16(p + 1)])) s_tot[bin] = acc;
        }
    }
    if (!VJP) {
        __syncthreads();
        for (int j = tid; j < m; j += kLThreads) P[(int64_t)j * nc + c] = s_tot[j];
        return;
    }

    // ---- vjp: reverse segmented walk (suffixes), then the map
    const LSegRevOp<T> rop;
    LSeg<T> ragg = rop.identity();
#pragma unroll
    for (int j = C::kSpan - 1; j >= 0; --j) {
        const int p = p0 + j;
        if (p < V) {
            const int q = pad16(p);
            const bool tail = p == V - 1 || s_bin[q] != s_bin[pad16(p + 1)];
            ragg = rop.combine(ragg, LSeg<T>{s_val[q], tail ? 1u : 0u, 0u});
        }
    }
    const LSeg<T> rcarry = lblock_excl<LSegRevOp<T>, LSeg<T>, true>(rop, ragg, s_seg);
    Pair<T> racc = rcarry.v;
#pragma unroll
    for (int j = C::kSpan - 1; j >= 0; --j) {
        const int p = p0 + j;
        if (p < V) {
            const int q = pad16(p);
            const int bin = s_bin[q];
            if (p == V - 1 || bin != s_bin[pad16(p + 1)]) racc = lf_id<T>();
            const Pair<T> l = lf(s_lrh[3 * bin], s_pre[q]);
            const Pair<T> rr = lf(racc, s_lrh[3 * bin + 1]);
            s_out[s_src[q]] = lf_adj(l, rr, s_lrh[3 * bin + 2]);
            racc = lf(s_val[q], racc);
        }
    }
    __syncthreads();
    for (int t = tid; t < len; t += kLThreads) {
        const Pair<T> g = s_out[t];
        if (accumulate) {
            const Pair<T> o = vbar[base + t];
            vbar[base + t] = Pair<T>{o.b + g.b, o.c + g.c};
        } else {
            vbar[base + t] = g;
        }
    }
}

// ------------------------------------------------------- column scans --
// Over the [m][nc] matrix P (bin-major).  Forward: element (bin, c) carries
// hist0[bin] at c = 0 (a segment start) and P[bin][c-1] otherwise, so the
// inclusive value is L[bin][c]; at the last chunk hist[bin] = L . P.
template <typename T, int ITEMS> struct ColFwd {
    using State = LSeg<T>;
    struct Aux {
        Pair<T> v[ITEMS];
    };
    struct Raw {
        Pair<T> v[ITEMS];
        Pair<T> vprev;
    };
    const Pair<T> *P;
    const Pair<T> *h0;
    Pair<T> *Lout;
    Pair<T> *hist;
    int64_t nc;
    __device__ State identity() const { return {lf_id<T>(), 0u, 0u}; }
    __device__ State combine(const State &a, const State &b) const { return {b.f ? b.v : lf(a.v, b.v), a.f | b.f, 0u}; }
    __device__ void fetch(int64_t c0, int64_t N, Raw &r) const {
        load_chunk(P, c0, N, r.v, lf_id<T>());
        r.vprev = (c0 > 0 && c0 <= N) ? P[c0 - 1] : lf_id<T>();
    }
    __device__ void build(int64_t c0, int64_t N, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
        int64_t bin = c0 / nc, cc = c0 - bin * nc;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            aux.v[j] = r.v[j];
            const bool head = cc == 0;
            const Pair<T> q = head ? (h0 ? h0[bin] : lf_id<T>()) : (j == 0 ? r.vprev : r.v[j - 1]);
            st[j] = (c0 + j < N) ? State{q, head ? 1u : 0u, 0u} : identity();
            if (++cc == nc) {
                cc = 0;
                ++bin;
            }
        }
    }
    __device__ void store(int64_t c0, int64_t N, const State (&st)[ITEMS], const Aux &aux) const {
        Pair<T> o[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) o[j] = st[j].v;
        store_chunk(Lout, c0, N, o);
        int64_t bin = c0 / nc, cc = c0 - bin * nc;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (c0 + j < N && cc == nc - 1) hist[bin] = lf(st[j].v, aux.v[j]);
            if (++cc == nc) {
                cc = 0;
                ++bin;
            }
        }
    }
};

// Reverse (logical order = decreasing index): element (bin, c) carries
// P[bin][c+1], identity at the last chunk (a segment start in this order), so
// the inclusive value is R[bin][c]; at c = 0 the bin total A = P[bin][0] . R.
template <typename T, int ITEMS> struct ColRev {
    using State = LSeg<T>;
    struct Aux {
        Pair<T> v[ITEMS];
    };
    struct Raw {
        Pair<T> v[ITEMS];
        Pair<T> vnext;
    };
    const Pair<T> *P;
    Pair<T> *Rout;
    Pair<T> *A;
    int64_t nc;
    __device__ State identity() const { return {lf_id<T>(), 0u, 0u}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {e.f ? e.v : lf(e.v, acc.v), acc.f | e.f, 0u};
    }
    __device__ void fetch(int64_t c0, int64_t N, Raw &r) const {
        load_chunk(P, c0, N, r.v, lf_id<T>());
        r.vnext = (c0 + ITEMS < N) ? P[c0 + ITEMS] : lf_id<T>();
    }
    __device__ void build(int64_t c0, int64_t N, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
        int64_t bin = c0 / nc, cc = c0 - bin * nc;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            aux.v[j] = r.v[j];
            const bool head = cc == nc - 1;
            const Pair<T> q = head ? lf_id<T>() : (j + 1 < ITEMS ? r.v[j + 1] : r.vnext);
            st[j] = (c0 + j < N) ? State{q, head ? 1u : 0u, 0u} : identity();
            if (++cc == nc) {
                cc = 0;
                ++bin;
            }
        }
    }
    __device__ void store(int64_t c0, int64_t N, const State (&st)[ITEMS], const Aux &aux) const {
        Pair<T> o[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) o[j] = st[j].v;
        store_chunk(Rout, c0, N, o);
        int64_t bin = c0 / nc, cc = c0 - bin * nc;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (c0 + j < N && cc == 0) A[bin] = lf(aux.v[j], st[j].v);
            if (++cc == nc) {
                cc = 0;
                ++bin;
            }
        }
    }
};

template <typename T> struct ColItems { static constexpr int v = 64 / (2 * (int)sizeof(T)); };

// hist0bar[j] (+)= d(hist0 . A)/d hist0 ^T histbar[j] = A.c * histbar[j]
template <typename T>
__global__ void k_linh_h0bar(const Pair<T> *__restrict__ A, const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ h0b,
                             const int64_t m, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const Pair<T> g = lf_adj(lf_id<T>(), A[j], hb[j]);
        h0b[j] = accumulate ? Pair<T>{h0b[j].b + g.b, h0b[j].c + g.c} : g;
    }
}

// -------------------------------------------------------------------- host --
template <typename T> static int64_t num_chunks(int64_t n) {
    const int64_t c = (n + LChunk<T>::kSize - 1) / LChunk<T>::kSize;
    return c > 0 ? c : 1;
}

struct LinLayout {
    size_t P, fwdreg, revreg, ws_bytes;  // workspace
    size_t L, R, A, saved_bytes;         // residuals
};

template <typename T> static LinLayout lin_layout(int64_t n, int64_t m) {
    LinLayout o;
    const int64_t nc = num_chunks<T>(n);
    const size_t cells = (size_t)m * (size_t)nc * sizeof(Pair<T>);
    constexpr int I = ColItems<T>::v;
    size_t w = kWsHeader;
    o.P = w;
    w = align_up(w + cells, 256);
    o.fwdreg = w;
    w = align_up(w + ScanShape<ColFwd<T, I>, I>::region((int64_t)m * nc), 256);
    o.revreg = w;
    w = align_up(w + ScanShape<ColRev<T, I>, I>::region((int64_t)m * nc), 256);
    o.ws_bytes = w;
    o.L = 0;
    o.R = align_up(cells, 256);
    o.A = 2 * align_up(cells, 256);
    o.saved_bytes = o.A + align_up((size_t)m * sizeof(Pair<T>), 256);
    return o;
}

bool linh_applicable(adc_dtype dt, int64_t m) {
    return m >= 1 && m <= (dt == ADC_F64 ? lmax_bins<double>() : lmax_bins<float>());
}

size_t linh_ws_bytes(adc_dtype dt, int64_t n, int64_t m) {
    return dt == ADC_F64 ? lin_layout<double>(n, m).ws_bytes : lin_layout<float>(n, m).ws_bytes;
}
size_t linh_saved_bytes(adc_dtype dt, int64_t n, int64_t m) {
    return dt == ADC_F64 ? lin_layout<double>(n, m).saved_bytes : lin_layout<float>(n, m).saved_bytes;
}

template <typename T, bool VJP> static size_t chunk_smem(int m) {
    using C = LChunk<T>;
    const size_t a = (size_t)kLWarps * m * 4;
    const size_t b = VJP ? (size_t)C::kSize * sizeof(Pair<T>) : (size_t)m * sizeof(Pair<T>);
    size_t s = al16(a > b ? a : b) + (size_t)C::kPad * sizeof(Pair<T>) + al16((size_t)C::kPad * 4);
    if (VJP) s += (size_t)C::kPad * sizeof(Pair<T>) + (size_t)3 * m * sizeof(Pair<T>);
    return s;
}

template <typename T>
static adc_status linh_fwd_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const Pair<T> *h0,
                             Pair<T> *hist, void *saved, void *ws, cudaStream_t s) {
    const LinLayout Lo = lin_layout<T>(n, m);
    const int64_t nc = num_chunks<T>(n);
    char *w = static_cast<char *>(ws);
    char *sv = static_cast<char *>(saved);
    Pair<T> *P = reinterpret_cast<Pair<T> *>(w + Lo.P);
    Pair<T> *L = reinterpret_cast<Pair<T> *>(sv + Lo.L);
    Pair<T> *R = reinterpret_cast<Pair<T> *>(sv + Lo.R);
    Pair<T> *A = reinterpret_cast<Pair<T> *>(sv + Lo.A);
    const size_t smem = chunk_smem<T, false>((int)m);
    if (cudaFuncSetAttribute(k_linh_chunk<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return ADC_ERR_CUDA;
    k_linh_chunk<T, false><<<(unsigned)nc, kLThreads, smem, s>>>(keys, vals, n, (int)m, nc, P, nullptr, nullptr,
                                                                 nullptr, nullptr, 0);
    adc_status st = check_launch();
    if (st != ADC_OK) return st;
    constexpr int I = ColItems<T>::v;
    const int64_t N = m * nc;
    ColFwd<T, I> fw{P, h0, L, hist, nc};
    if ((st = run_scan<ColFwd<T, I>, I, false>(fw, N, ws, 24, w + Lo.fwdreg, s)) != ADC_OK) return st;
    ColRev<T, I> rv{P, R, A, nc};
    return run_scan<ColRev<T, I>, I, true>(rv, N, ws, 25, w + Lo.revreg, s);
}

template <typename T>
static adc_status linh_vjp_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const void *saved,
                             const Pair<T> *hb, Pair<T> *vb, Pair<T> *h0b, int acc, cudaStream_t s) {
    const LinLayout Lo = lin_layout<T>(n, m);
    const int64_t nc = num_chunks<T>(n);
    const char *sv = static_cast<const char *>(saved);
    const Pair<T> *L = reinterpret_cast<const Pair<T> *>(sv + Lo.L);
    const Pair<T> *R = reinterpret_cast<const Pair<T> *>(sv + Lo.R);
    const Pair<T> *A = reinterpret_cast<const Pair<T> *>(sv + Lo.A);
    if (n > 0) {
        const size_t smem = chunk_smem<T, true>((int)m);
        if (cudaFuncSetAttribute(k_linh_chunk<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return ADC_ERR_CUDA;
        k_linh_chunk<T, true><<<(unsigned)nc, kLThreads, smem, s>>>(keys, vals, n, (int)m, nc, nullptr, L, R, hb, vb,
                                                                    acc);
    }
    if (h0b) {
        const int64_t g = (m + 255) / 256;
        k_linh_h0bar<T><<<(unsigned)(g < 1024 ? g : 1024), 256, 0, s>>>(A, hb, h0b, m, acc);
    }
    return check_launch();
}

adc_status linh_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                    void *hist, void *saved, void *ws, cudaStream_t s) {
    if (dt == ADC_F64)
        return linh_fwd_t<double>(n, m, keys, static_cast<const Pair<double> *>(vals),
                                  static_cast<const Pair<double> *>(hist0), static_cast<Pair<double> *>(hist), saved,
                                  ws, s);
    return linh_fwd_t<float>(n, m, keys, static_cast<const Pair<float> *>(vals), static_cast<const Pair<float> *>(hist0),
                             static_cast<Pair<float> *>(hist), saved, ws, s);
}

adc_status linh_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *saved,
                    const void *histbar, void *valsbar, void *hist0bar, int accumulate, cudaStream_t s) {
    if (dt == ADC_F64)
        return linh_vjp_t<double>(n, m, keys, static_cast<const Pair<double> *>(vals), saved,
                                  static_cast<const Pair<double> *>(histbar), static_cast<Pair<double> *>(valsbar),
                                  static_cast<Pair<double> *>(hist0bar), accumulate, s);
    return linh_vjp_t<float>(n, m, keys, static_cast<const Pair<float> *>(vals), saved,
                             static_cast<const Pair<float> *>(histbar), static_cast<Pair<float> *>(valsbar),
                             static_cast<Pair<float> *>(hist0bar), accumulate, s);
}

}  // namespace adc
