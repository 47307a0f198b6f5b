// General reduce_by_index for the non-commutative linFnComp operator with up
// to a few thousand bins (Sec. 4.1, Fig. 4).  The paper sorts the elements by
// bin (stable) and runs segmented scans over the sorted values; what those
// scans compute per element is the fold of its bin's values before it (l_i)
// and after it (r_i), in index order.  Here no element is moved:
//   1. per chunk of kLThreads * R elements (one block; warp w owns the w-th
//      run of 32 * R consecutive elements, R rounds of 32): every warp walks
//      its run in index order and folds each element into its bin's entry of
//      a warp-private table in shared memory.  Within a round, lanes holding
//      the same bin (__match_any_sync peers) update one after another in lane
//      order, so every bin's entry is the ordered fold of the run's values;
//      the block then composes the warp tables per bin in warp order ->
//      P[bin][chunk] (identity where the bin is absent);
//   2. one block per bin composes its row of P in chunk order: the exclusive
//      prefix L[bin][c] = hist0 . P[bin][0..c-1], the exclusive suffix
//      R[bin][c] = P[bin][c+1..], hist = L . P at the last chunk and the bin
//      total A = P[bin][0] . R[bin][0] (for hist0bar);
//   3. vjp, per chunk: the forward walk again, keeping each element's
//      exclusive prefix p_i within its warp run, and a backward walk keeping
//      the product s_i of the c's after it; per bin and warp the block forms
//      what lies before the run (L . earlier runs) and the product of the c's
//      after it (later runs, R), and every element gets
//      vbar_i = d(l_i . v_i . r_i)/dv_i ^T histbar[k_i] with l_i = before . p_i
//      and r_i.c = s_i * after.c.
// Within every bin the values meet in index order, as the sequential
// definition requires; only the bracketing differs (associativity).
// Traffic: the forward reads keys and values once (12 B per fp32 element) and
// moves the [m][chunks] matrices (P, L, R: 8 B per bin and chunk each); the
// vjp reads keys, values, L and R and writes the adjoints once.
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"

namespace adc {

constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / kWarp;
// The vjp's shared memory (per-warp tables of (b, c) and of c, histbar) fits
// one block up to 2047 bins (fp32) / 1023 bins (fp64).
template <typename T> constexpr int64_t lmax_bins() { return sizeof(T) == 4 ? 2047 : 1023; }
template <typename T> struct LChunk {
    static constexpr int kRounds = sizeof(T) == 4 ? 16 : 8;  // rounds of 32 elements per warp
    static constexpr int kRun = kWarp * kRounds;             // elements per warp
    static constexpr int kSize = kLThreads * kRounds;        // elements per chunk (block)
};

template <typename T> __device__ __forceinline__ Pair<T> lf(const Pair<T> &a, const Pair<T> &b) {
    return {b.b + b.c * a.b, b.c * a.c};  // (b1,c1) . (b2,c2) = (b2 + c2*b1, c2*c1)
}
template <typename T> __device__ __forceinline__ Pair<T> lf_id() { return {T(0), T(1)}; }
// d(l . v . r)/dv ^T g for linFnComp
template <typename T> __device__ __forceinline__ Pair<T> lf_adj(const Pair<T> &l, const Pair<T> &r, const Pair<T> &g) {
    return {r.c * g.b, r.c * (l.b * g.b + l.c * g.c)};
}

// One (b, c) element as one 8- or 16-byte streaming load (the array is
// 16-byte aligned, so every element is aligned to its size).
__device__ __forceinline__ Pair<float> ld_pair(const Pair<float> *p) {
    const float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
    return {t.x, t.y};
}
__device__ __forceinline__ Pair<double> ld_pair(const Pair<double> *p) {
    const double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
    return {t.x, t.y};
}

// One warp run of a chunk: keys (-1 past n) and values, round r at element
// base + r * 32 + lane, every load issued before the first use.
template <typename T, int R>
__device__ __forceinline__ void load_run(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals,
                                         int64_t base, int64_t n, int m, int32_t (&k)[R], Pair<T> (&v)[R]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = base + r * kWarp + lane;
        k[r] = i < n ? __ldcs(keys + i) : -1;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = base + r * kWarp + lane;
        v[r] = in_range(k[r], m) ? ld_pair(vals + i) : lf_id<T>();
    }
}

// One round of a warp walk: upd() runs for every lane with an in-range key,
// in lane order among lanes that share a key (REV: descending lane order),
// lanes with different keys at once.  Every such lane first writes its lane
// number to its key's byte in `tag` (one byte per bin and warp): when each
// reads its own number back, no two lanes share a key and all update in one
// step; otherwise __match_any_sync groups the lanes and the groups advance
// one rank per step.  Warp-wide: all lanes call it.
template <bool REV, class F>
__device__ __forceinline__ void ordered_round(int32_t key, bool ok, uint8_t *tag, F &&upd) {
    const int lane = threadIdx.x & 31;
    if (ok) tag[key] = (uint8_t)lane;
    __syncwarp();
    const bool alone = !ok || tag[key] == (uint8_t)lane;
    if (__all_sync(0xffffffffu, alone)) {
        if (ok) upd();
    } else {
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? key : -1);
        const unsigned ahead = REV ? (peers & ~((2u << lane) - 1u)) : (peers & ((1u << lane) - 1u));
        const int rank = __popc(ahead);
        for (int q = 0; __any_sync(0xffffffffu, ok && rank >= q); ++q) {
            if (ok && rank == q) upd();
            __syncwarp();
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------ chunk fold --
// P[bin * nc + chunk] = ordered fold of the chunk's values of that bin.
template <typename T>
__global__ void __launch_bounds__(kLThreads)
k_linh_fold(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals, const int64_t n, const int m,
            const int64_t nc, Pair<T> *__restrict__ P) {
    using C = LChunk<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Pair<T> *s_tab = reinterpret_cast<Pair<T> *>(smem_raw);              // [kLWarps][m]
    uint8_t *s_tag = reinterpret_cast<uint8_t *>(s_tab + (size_t)kLWarps * m);  // [kLWarps][m]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    Pair<T> *tab = s_tab + (size_t)warp * m;
    uint8_t *tag = s_tag + (size_t)warp * m;
    int32_t k[C::kRounds];
    Pair<T> v[C::kRounds];
    load_run<T, C::kRounds>(keys, vals, c * C::kSize + (int64_t)warp * C::kRun, n, m, k, v);
    for (int j = lane; j < m; j += kWarp) tab[j] = lf_id<T>();
    __syncwarp();
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int32_t key = k[r];
        const Pair<T> x = v[r];
        ordered_round<false>(key, in_range(key, m), tag, [&] { tab[key] = lf(tab[key], x); });
    }
    __syncthreads();
    for (int j = tid; j < m; j += kLThreads) {
        Pair<T> acc = s_tab[j];
#pragma unroll
        for (int w = 1; w < kLWarps; ++w) acc = lf(acc, s_tab[(size_t)w * m + j]);
        P[(int64_t)j * nc + c] = acc;
    }
}

// ------------------------------------------------------------- bin rows --
// Block-wide exclusive scan of one state per thread in thread order (REV:
// reverse thread order) for linFnComp; two __syncthreads().
template <typename T, bool REV>
__device__ __forceinline__ Pair<T> lblock_excl(Pair<T> a, Pair<T> *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int vl = REV ? (kWarp - 1 - lane) : lane;
    const int vw = REV ? (kLWarps - 1 - warp) : warp;
    // REV: a forward scan over mirrored lanes and warps with the operands
    // swapped (later elements come first in logical order)
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const Pair<T> up = REV ? shfl_down(a, o) : shfl_up(a, o);
        if (vl >= o) a = REV ? lf(a, up) : lf(up, a);
    }
    if (vl == kWarp - 1) s_w[vw] = a;
    Pair<T> ex = REV ? shfl_down(a, 1) : shfl_up(a, 1);
    if (vl == 0) ex = lf_id<T>();
    __syncthreads();
    Pair<T> before = lf_id<T>();
#pragma unroll
    for (int w = 0; w < kLWarps; ++w)
        if (w < vw) before = REV ? lf(s_w[w], before) : lf(before, s_w[w]);
    __syncthreads();
    return REV ? lf(ex, before) : lf(before, ex);
}

// One block per bin j: L[j][c], R[j][c], hist[j], A[j] from the row P[j][.].
// The row goes through shared memory in segments of RI entries per thread
// (loads and stores coalesced); within a segment thread t composes its RI
// consecutive entries and a block scan gives what lies before (L) or after
// (R) them.  A row that fits one segment is loaded once: the reverse pass
// reuses each thread's entries from registers (fp32 takes 16 entries per
// thread, so rows of up to 4096 chunks, n <= 16.7M, are one segment).
template <typename T> constexpr int row_items() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T>
__global__ void __launch_bounds__(kLThreads)
k_linh_rows(const Pair<T> *__restrict__ P, const Pair<T> *__restrict__ h0, const int64_t nc,
            Pair<T> *__restrict__ L, Pair<T> *__restrict__ R, Pair<T> *__restrict__ hist, Pair<T> *__restrict__ A) {
    constexpr int RI = row_items<T>();
    constexpr int SEG = kLThreads * RI;
    __shared__ Pair<T> s_seg[SEG];
    __shared__ Pair<T> s_w[kLWarps];
    __shared__ Pair<T> s_tot;
    const int tid = threadIdx.x;
    const int64_t j = blockIdx.x;
    const Pair<T> *row = P + j * nc;
    const bool one = nc <= SEG;  // the whole row in one segment
    Pair<T> v[RI], agg = lf_id<T>();
    // forward: L = hist0 . the entries before
    Pair<T> carry = h0 ? h0[j] : lf_id<T>();
    for (int64_t s0 = 0; s0 < nc; s0 += SEG) {
        const int len = (int)((nc - s0) < SEG ? (nc - s0) : SEG);
        for (int e = tid; e < len; e += kLThreads) s_seg[e] = row[s0 + e];
        __syncthreads();
        agg = lf_id<T>();
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            const int idx = tid * RI + k;
            v[k] = idx < len ? s_seg[idx] : lf_id<T>();
            agg = lf(agg, v[k]);
        }
        const Pair<T> ex = lblock_excl<T, false>(agg, s_w);
        if (tid == kLThreads - 1) s_tot = lf(ex, agg);
        Pair<T> run = lf(carry, ex);
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            const int idx = tid * RI + k;
            if (idx < len) {
                s_seg[idx] = run;
                run = lf(run, v[k]);
            }
        }
        __syncthreads();
        for (int e = tid; e < len; e += kLThreads) L[j * nc + s0 + e] = s_seg[e];
        carry = lf(carry, s_tot);
        __syncthreads();
    }
    if (tid == 0) hist[j] = carry;
    // reverse: R = the entries after, from the last segment down
    Pair<T> rcarry = lf_id<T>();
    for (int64_t s0 = (nc - 1) / SEG * SEG; s0 >= 0; s0 -= SEG) {
        const int len = (int)((nc - s0) < SEG ? (nc - s0) : SEG);
        if (!one) {  // a single segment's entries are still in v
            for (int e = tid; e < len; e += kLThreads) s_seg[e] = row[s0 + e];
            __syncthreads();
            agg = lf_id<T>();
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                const int idx = tid * RI + k;
                v[k] = idx < len ? s_seg[idx] : lf_id<T>();
                agg = lf(agg, v[k]);
            }
        }
        const Pair<T> rex = lblock_excl<T, true>(agg, s_w);  // the later threads' entries
        if (tid == 0) s_tot = lf(agg, rex);
        Pair<T> rrun = lf(rex, rcarry);
#pragma unroll
        for (int k = RI - 1; k >= 0; --k) {
            const int idx = tid * RI + k;
            if (idx < len) {
                s_seg[idx] = rrun;
                rrun = lf(v[k], rrun);
            }
        }
        __syncthreads();
        for (int e = tid; e < len; e += kLThreads) R[j * nc + s0 + e] = s_seg[e];
        rcarry = lf(s_tot, rcarry);
        __syncthreads();
    }
    if (tid == 0) A[j] = rcarry;  // P[j][0] . R[j][0]: the bin's whole fold
}

// ------------------------------------------------------------------- vjp --
template <typename T>
__global__ void __launch_bounds__(kLThreads, 2)
k_linh_vjp(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals, const int64_t n, const int m,
           const int64_t nc, const Pair<T> *__restrict__ L, const Pair<T> *__restrict__ R,
           const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ vbar, const int accumulate) {
    using C = LChunk<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Pair<T> *s_tab = reinterpret_cast<Pair<T> *>(smem_raw);  // [kLWarps][m]: folds, then (before . g, after.c)
    Pair<T> *s_g = s_tab + (size_t)kLWarps * m;              // [m] histbar
    T *s_q = reinterpret_cast<T *>(s_g + m);                  // [kLWarps][m] products of c (backward walk)
    uint8_t *s_tag = reinterpret_cast<uint8_t *>(s_q + (size_t)kLWarps * m);  // [kLWarps][m]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    const int64_t base = c * C::kSize + (int64_t)warp * C::kRun;
    Pair<T> *tab = s_tab + (size_t)warp * m;
    T *qt = s_q + (size_t)warp * m;
    uint8_t *tag = s_tag + (size_t)warp * m;
    int32_t k[C::kRounds];
    Pair<T> v[C::kRounds];
    load_run<T, C::kRounds>(keys, vals, base, n, m, k, v);
    for (int j = lane; j < m; j += kWarp) {
        tab[j] = lf_id<T>();
        qt[j] = T(1);
    }
    for (int j = tid; j < m; j += kLThreads) s_g[j] = hb[j];
    __syncwarp();
    // forward walk: p_i = the run's fold of i's bin before i
    Pair<T> p[C::kRounds];
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int32_t key = k[r];
        const Pair<T> x = v[r];
        Pair<T> pr = lf_id<T>();
        ordered_round<false>(key, in_range(key, m), tag, [&] {
            pr = tab[key];
            tab[key] = lf(pr, x);
        });
        p[r] = pr;
    }
    // backward walk: s_i = product of the c's of i's bin after i in the run
    T sv[C::kRounds];
#pragma unroll
    for (int r = C::kRounds - 1; r >= 0; --r) {
        const int32_t key = k[r];
        const T xc = v[r].c;
        T sr = T(1);
        ordered_round<true>(key, in_range(key, m), tag, [&] {
            sr = qt[key];
            qt[key] = xc * sr;
        });
        sv[r] = sr;
    }
    __syncthreads();
    // per bin and warp run: u = <L . earlier runs, g> and the product of the
    // c's after the run (later runs, then R)
    for (int j = tid; j < m; j += kLThreads) {
        const Pair<T> g = s_g[j];
        Pair<T> before = L[(int64_t)j * nc + c];
        T fc[kLWarps], u[kLWarps];
#pragma unroll
        for (int w = 0; w < kLWarps; ++w) {
            const Pair<T> f = s_tab[(size_t)w * m + j];
            u[w] = g.b * before.b + g.c * before.c;
            fc[w] = f.c;
            before = lf(before, f);
        }
        T after = R[(int64_t)j * nc + c].c;
#pragma unroll
        for (int w = kLWarps - 1; w >= 0; --w) {
            s_tab[(size_t)w * m + j] = Pair<T>{u[w], after};
            after = fc[w] * after;
        }
    }
    __syncthreads();
    // vbar_i = (rc g.b, rc <l_i, g>) with l_i = before . p_i, rc = s_i * after
#pragma unroll
    for (int r = 0; r < C::kRounds; ++r) {
        const int64_t i = base + r * kWarp + lane;
        if (i >= n) continue;
        Pair<T> out{T(0), T(0)};
        if (in_range(k[r], m)) {
            const Pair<T> ua = tab[k[r]];
            const Pair<T> g = s_g[k[r]];
            const T rc = sv[r] * ua.c;
            out = Pair<T>{rc * g.b, rc * (g.b * p[r].b + p[r].c * ua.b)};
        }
        if (accumulate) {
            const Pair<T> o = vbar[i];
            out = Pair<T>{o.b + out.b, o.c + out.c};
        }
        vbar[i] = out;
    }
}

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
    size_t P, ws_bytes;                  // workspace
    size_t L, R, A, saved_bytes;         // residuals
};

template <typename T> static LinLayout lin_layout(int64_t n, int64_t m) {
    LinLayout o;
    const int64_t nc = num_chunks<T>(n);
    const size_t cells = (size_t)m * (size_t)nc * sizeof(Pair<T>);
    o.P = kWsHeader;
    o.ws_bytes = align_up(kWsHeader + cells, 256);
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

template <typename T> static size_t fold_smem(int64_t m) { return (size_t)kLWarps * m * (sizeof(Pair<T>) + 1); }
template <typename T> static size_t vjp_smem(int64_t m) {
    return (size_t)(kLWarps + 1) * m * sizeof(Pair<T>) + (size_t)kLWarps * m * (sizeof(T) + 1);
}

template <typename T>
static adc_status linh_fwd_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const Pair<T> *h0,
                             Pair<T> *hist, void *saved, void *ws, cudaStream_t s) {
    const LinLayout Lo = lin_layout<T>(n, m);
    const int64_t nc = num_chunks<T>(n);
    char *sv = static_cast<char *>(saved);
    Pair<T> *P = reinterpret_cast<Pair<T> *>(static_cast<char *>(ws) + Lo.P);
    const size_t smem = fold_smem<T>(m);
    if (cudaFuncSetAttribute(k_linh_fold<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ADC_ERR_CUDA;
    k_linh_fold<T><<<(unsigned)nc, kLThreads, smem, s>>>(keys, vals, n, (int)m, nc, P);
    k_linh_rows<T><<<(unsigned)m, kLThreads, 0, s>>>(P, h0, nc, reinterpret_cast<Pair<T> *>(sv + Lo.L),
                                                     reinterpret_cast<Pair<T> *>(sv + Lo.R), hist,
                                                     reinterpret_cast<Pair<T> *>(sv + Lo.A));
    return check_launch();
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
        const size_t smem = vjp_smem<T>(m);
        if (cudaFuncSetAttribute(k_linh_vjp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return ADC_ERR_CUDA;
        k_linh_vjp<T><<<(unsigned)nc, kLThreads, smem, s>>>(keys, vals, n, (int)m, nc, L, R, hb, vb, acc);
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
