// Bulk-staged segment forms of the q x q matrix-product scans (Sec. 5.3.4:
// the forward P_i = P_{i-1} M_i and the vjp with the RBDS Jacobian M_{i+1}^T,
// f_i(L) = Ybar_i + L M_{i+1}^T, Mbar_i = P_{i-1}^T lambda_i).
//
// An engine item is a run of SEG consecutive matrices; a block's tile is TH
// runs.  The per-tile engine (k_scan, kBulkStaged) has thread 0 bring the
// tile of every array the walk reads into shared memory with one bulk (TMA)
// copy per array, all on one mbarrier, while the other threads wait; the
// threads then walk their runs in shared memory (build: the run's state;
// store: the re-walk from the run's exclusive prefix, the results written in
// place), and the block copies the results out with consecutive 16-byte
// stores (the vjp's third input, y, needed only for its last step, follows
// in finish() into the space its re-walk freed).  Why: a q x q element is
// 36 / 100 bytes (fp32), so a thread that
// walks its own run in global memory makes every warp access touch 32
// different lines, and the loads of a tile are spread over a long dependent
// walk; a bulk copy puts the whole tile in flight at once and the walks run
// at shared-memory latency.
//
// Geometry: SEG * q * q is odd, so 32 consecutive runs start in 32 distinct
// banks (conflict-free walks for 4- and 8-byte words); TH is whole warps (a
// multiple of 4), so a tile (TH * SEG elements) is whole 16-byte words and every
// tile starts 16-byte aligned (the API requires 16-byte aligned arrays).
// Elements outside the array are never read from it: the vjp's x_n (after the
// last element) and y_{-1} (before the first) are the identity, written into
// the stage by thread 0.  Every wait on a copy is bounded (the engine's spin
// limit); a block whose wait runs out gives the copy a second bounded wait
// before it leaves, and the call reports a timeout.
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "scan_engine.cuh"
#include "tma.cuh"

namespace adc {

template <typename T, int Q, int TH, int SEG> struct MMQGeom {
    static constexpr int QQ = Q * Q;
    static constexpr int64_t B = (int64_t)QQ * sizeof(T);  // bytes per element
    static constexpr int64_t H = (B + 15) / 16 * 16;       // one element, in whole 16-byte words
    static constexpr int TE = TH * SEG;                    // elements per tile
    static constexpr int64_t TB = (int64_t)TE * B;         // bytes per tile of one array
    static_assert(TB % 16 == 0, "a tile must be whole 16-byte words");
    static_assert((SEG * QQ) % 2 == 1, "runs need an odd word stride");
    static_assert(TH % 32 == 0, "whole warps");
};

// One array's span of a tile: bytes [lo, hi) of the array, clamped to
// [0, nb); the 16-byte-aligned body [lo, body) goes by one bulk copy, the
// ragged end [body, hi) (under 16 bytes, whole 4-byte words) by plain copies.
struct StageSpan {
    int64_t lo, body, hi;
    __device__ StageSpan(int64_t l, int64_t h, int64_t nb) {
        lo = l < 0 ? 0 : l;
        hi = h > nb ? nb : h;
        if (hi < lo) hi = lo;
        body = lo + ((hi - lo) & ~(int64_t)15);
    }
    __device__ uint32_t bulk_bytes() const { return (uint32_t)(body - lo); }
    // dst holds byte `org` of the array at its start
    __device__ void issue(char *dst, const char *src, int64_t org, unsigned long long *bar) const {
        if (body > lo) bulk_g2s(dst + (lo - org), src + lo, (uint32_t)(body - lo), bar);
        for (int64_t b = body; b < hi; b += 4)
            *reinterpret_cast<uint32_t *>(dst + (b - org)) = *reinterpret_cast<const uint32_t *>(src + b);
    }
};

template <typename T, int Q> __device__ __forceinline__ void put_eye(T *p) {
#pragma unroll
    for (int i = 0; i < Q * Q; ++i) p[i] = (i % (Q + 1) == 0) ? T(1) : T(0);
}

template <typename T, int Q> __device__ __forceinline__ MatQ<T, Q> ld_matq(const T *p) {
    MatQ<T, Q> m;
#pragma unroll
    for (int i = 0; i < Q * Q; ++i) m.a[i] = p[i];
    return m;
}

// 16 bytes of T as one vector (float4 / double2) for the copy-out.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using V = float4;
    static __device__ __forceinline__ V add(V a, V b) { return {a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w}; }
};
template <> struct Vec16<double> {
    using V = double2;
    static __device__ __forceinline__ V add(V a, V b) { return {a.x + b.x, a.y + b.y}; }
};

// The block copies `bytes` (a multiple of sizeof(T)) from the stage to dst,
// adding to dst's contents when accumulate is set: 16-byte words, then the
// ragged end element by element.  dst is 16-byte aligned.
template <typename T, int TH>
__device__ __forceinline__ void copy_out(T *dst, const T *src, int64_t bytes, bool accumulate) {
    using V = typename Vec16<T>::V;
    constexpr int PER = 16 / (int)sizeof(T);
    const int64_t nv = bytes / 16;
    V *dv = reinterpret_cast<V *>(dst);
    const V *sv = reinterpret_cast<const V *>(src);
    if (accumulate) {
        for (int64_t v = threadIdx.x; v < nv; v += TH) dv[v] = Vec16<T>::add(dv[v], sv[v]);
    } else {
        for (int64_t v = threadIdx.x; v < nv; v += TH) dv[v] = sv[v];
    }
    const int64_t ne = bytes / (int64_t)sizeof(T);
    for (int64_t e = nv * PER + threadIdx.x; e < ne; e += TH) dst[e] = accumulate ? dst[e] + src[e] : src[e];
}

// Shared-memory base of the stage (dynamic shared memory; its first 16
// bytes hold the tile's mbarrier).
__device__ __forceinline__ char *mmq_stage_base() {
    extern __shared__ __align__(16) unsigned char mmq_dyn[];
    return reinterpret_cast<char *>(mmq_dyn);
}
__device__ __forceinline__ unsigned long long *mmq_stage_bar() {
    return reinterpret_cast<unsigned long long *>(mmq_stage_base());
}

// Forward: a run's state is the product of its elements; store() re-walks
// the run from its exclusive prefix, writing P_i over the staged M_i.
// Stage: [mbarrier: 16 B][x: TB].
template <typename T, int Q, int TH, int SEG> struct StagedFwdMMQ {
    using G = MMQGeom<T, Q, TH, SEG>;
    using E = MatQ<T, Q>;
    using State = E;
    using Aux = NoAux;
    struct Raw {};
    static constexpr bool kExclusiveStore = true;
    static constexpr bool kPerTileOnly = true;
    static constexpr bool kBulkStaged = true;
    static constexpr int kThreads = TH;
    static constexpr size_t kOffX = 16;
    static constexpr size_t kDynSmem = kOffX + G::TB;
    const E *x;
    E *y;
    int64_t n;  // elements (the engine counts runs)
    __device__ State identity() const { return matq_eye<T, Q>(); }
    __device__ State combine(const State &a, const State &b) const { return matq_mul(a, b); }
    __device__ void stage_init() const {
        mbar_init(mmq_stage_bar(), 1);
        mbar_init_fence();
    }
    __device__ bool staged_wait(long long limit) const { return mbar_wait_bounded(mmq_stage_bar(), 0u, limit); }
    // c0 is this thread's run; the tile's runs start at (c0 / TH) * TH
    __device__ void fetch(int64_t c0, int64_t, Raw &) const {
        if (threadIdx.x != 0) return;
        const int64_t o = (c0 / TH) * (int64_t)G::TB;
        const StageSpan sx(o, o + G::TB, n * G::B);
        mbar_expect_tx(mmq_stage_bar(), sx.bulk_bytes());
        sx.issue(mmq_stage_base() + kOffX, reinterpret_cast<const char *>(x), o, mmq_stage_bar());
    }
    __device__ void build(int64_t c0, int64_t items, const Raw &, State (&st)[1], Aux &) const {
        E s = matq_eye<T, Q>();
        if (c0 < items) {
            const T *sx = reinterpret_cast<const T *>(mmq_stage_base() + kOffX) + (int)(c0 % TH) * SEG * G::QQ;
            const int64_t lo = c0 * SEG;
            const int cnt = (int)((lo + SEG < n) ? SEG : n - lo);
            for (int k = 0; k < cnt; ++k) matq_mul_right(s, ld_matq<T, Q>(sx + k * G::QQ));
        }
        st[0] = s;
    }
    __device__ void store(int64_t c0, int64_t items, const State (&ex)[1], const Aux &) const {
        T *sx = reinterpret_cast<T *>(mmq_stage_base() + kOffX);
        if (c0 < items) {
            T *mine = sx + (int)(c0 % TH) * SEG * G::QQ;
            const int64_t lo = c0 * SEG;
            const int cnt = (int)((lo + SEG < n) ? SEG : n - lo);
            E run = ex[0];
            for (int k = 0; k < cnt; ++k) {
                matq_mul_right(run, ld_matq<T, Q>(mine + k * G::QQ));
#pragma unroll
                for (int q = 0; q < G::QQ; ++q) mine[k * G::QQ + q] = run.a[q];  // this thread's own slots
            }
        }
        __syncthreads();  // every run's prefixes are in the stage
        const int64_t e0 = (c0 / TH) * (int64_t)G::TE;
        const int64_t ne = (n - e0 < G::TE) ? n - e0 : G::TE;
        copy_out<T, TH>(reinterpret_cast<T *>(y + e0), sx, ne * G::B, false);
    }
};

// vjp (reverse): the run's state composes f_i(L) = Ybar_i + L M_{i+1}^T from
// its last element down; the re-walk applies lambda_i = Ybar_i + lambda_{i+1}
// M_{i+1}^T from the incoming lambda and writes lambda_i over the staged
// Ybar_i.  y is needed only for the last step, Mbar_i = P_{i-1}^T lambda_i:
// finish() bulk-copies the tile's y (one element before it included) into
// the x stage the re-walk has freed, and the block then forms Mbar_i one
// element per thread (odd word strides again) and copies it out.  Two arrays
// in shared memory instead of three: three blocks fit an SM instead of two.
// Stage: [mbarriers: 16 B][x_e, e = e0 .. e0 + TE (one past the tile), later
//        y_e, e = e0 - 1 .. e0 + TE - 1: TB + H][ybar, then lambda, then Mbar: TB].
template <typename T, int Q, int TH, int SEG> struct StagedVjpMMQ {
    using G = MMQGeom<T, Q, TH, SEG>;
    using E = MatQ<T, Q>;
    using State = AffQ<T, Q>;
    using Aux = NoAux;
    struct Raw {};
    static constexpr bool kExclusiveStore = true;
    static constexpr bool kPerTileOnly = true;
    static constexpr bool kBulkStaged = true;
    static constexpr bool kFinish = true;
    static constexpr int kThreads = TH;
    static constexpr size_t kOffX = 16;
    static constexpr size_t kOffG = kOffX + G::TB + G::H;
    static constexpr size_t kDynSmem = kOffG + G::TB;
    const E *x, *y, *ybar;
    E *xbar;
    int accumulate;
    int64_t n;
    __device__ State identity() const { return {matq_zero<T, Q>(), matq_eye<T, Q>()}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {matq_add(e.v, matq_mul(acc.v, e.c)), matq_mul(acc.c, e.c)};
    }
    // The scans' combine, piecewise: v <- combine(other, v) with `other` the
    // state of lane (lane -/+ o), fetched one row at a time -- new v = v.v +
    // other.v v.c, new c = other.c v.c -- so that about three matrices are
    // live instead of six (the 5x5 fp32 state is 50 words).
    __device__ void shfl_combine(State &s, int o, bool down, bool active) const {
        E nc;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T ov[Q], oc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                ov[j] = down ? __shfl_down_sync(0xffffffffu, s.v.a[Q * i + j], o)
                             : __shfl_up_sync(0xffffffffu, s.v.a[Q * i + j], o);
                oc[j] = down ? __shfl_down_sync(0xffffffffu, s.c.a[Q * i + j], o)
                             : __shfl_up_sync(0xffffffffu, s.c.a[Q * i + j], o);
            }
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                T av = s.v.a[Q * i + j], ac = T(0);
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    av += ov[k] * s.c.a[Q * k + j];
                    ac += oc[k] * s.c.a[Q * k + j];
                }
                nc.a[Q * i + j] = active ? ac : s.c.a[Q * i + j];
                if (active) s.v.a[Q * i + j] = av;  // row i of v is read by no later row
            }
        }
        s.c = nc;
    }
    // two mbarriers: the inputs of build() / store(), then y for finish()
    __device__ unsigned long long *bar(int i) const { return mmq_stage_bar() + i; }
    __device__ void stage_init() const {
        mbar_init(bar(0), 1);
        mbar_init(bar(1), 1);
        mbar_init_fence();
    }
    __device__ bool staged_wait(long long limit) const { return mbar_wait_bounded(bar(0), 0u, limit); }
    __device__ void fetch(int64_t c0, int64_t, Raw &) const {
        if (threadIdx.x != 0) return;
        const int64_t e0 = (c0 / TH) * (int64_t)G::TE;
        const int64_t o = e0 * G::B, nb = n * G::B;
        const StageSpan sx(o, o + G::TB + G::H, nb), sg(o, o + G::TB, nb);
        char *base = mmq_stage_base();
        mbar_expect_tx(bar(0), sx.bulk_bytes() + sg.bulk_bytes());
        sx.issue(base + kOffX, reinterpret_cast<const char *>(x), o, bar(0));
        sg.issue(base + kOffG, reinterpret_cast<const char *>(ybar), o, bar(0));
        // x_n (after the last element) is the identity (bytes no copy above writes)
        if (n - e0 <= G::TE) put_eye<T, Q>(reinterpret_cast<T *>(base + kOffX + (n - e0) * G::B));
    }
    __device__ void build(int64_t c0, int64_t items, const Raw &, State (&st)[1], Aux &) const {
        State s = identity();
        if (c0 < items) {
            const int le = (int)(c0 % TH) * SEG;
            const T *sx = reinterpret_cast<const T *>(mmq_stage_base() + kOffX) + le * G::QQ;
            const T *sg = reinterpret_cast<const T *>(mmq_stage_base() + kOffG) + le * G::QQ;
            const int64_t lo = c0 * SEG;
            const int cnt = (int)((lo + SEG < n) ? SEG : n - lo);
            for (int k = cnt - 1; k >= 0; --k) {
                // s <- f_i o s: v = Ybar_i + v M^T, c = c M^T  (M = x_{i+1})
                const E M = ld_matq<T, Q>(sx + (k + 1) * G::QQ);
                matq_mul_right_t(s.v, M);
                matq_mul_right_t(s.c, M);
#pragma unroll
                for (int q = 0; q < G::QQ; ++q) s.v.a[q] += sg[k * G::QQ + q];
            }
        }
        st[0] = s;
    }
    __device__ void store(int64_t c0, int64_t items, const State (&ex)[1], const Aux &) const {
        if (c0 >= items) return;
        const int le = (int)(c0 % TH) * SEG;
        const T *sx = reinterpret_cast<const T *>(mmq_stage_base() + kOffX) + le * G::QQ;
        T *sg = reinterpret_cast<T *>(mmq_stage_base() + kOffG) + le * G::QQ;
        const int64_t lo = c0 * SEG;
        const int cnt = (int)((lo + SEG < n) ? SEG : n - lo);
        E lam = ex[0].v;
        for (int k = cnt - 1; k >= 0; --k) {
            matq_mul_right_t(lam, ld_matq<T, Q>(sx + (k + 1) * G::QQ));
#pragma unroll
            for (int q = 0; q < G::QQ; ++q) {
                lam.a[q] += sg[k * G::QQ + q];
                sg[k * G::QQ + q] = lam.a[q];  // this thread's own slots
            }
        }
    }
    __device__ bool finish(int64_t c0, int64_t, long long limit) const {
        const int64_t e0 = (c0 / TH) * (int64_t)G::TE;
        const int64_t ne = (n - e0 < G::TE) ? n - e0 : G::TE;
        char *base = mmq_stage_base();
        __syncthreads();  // every re-walk is done with the x stage
        if (threadIdx.x == 0) {
            const int64_t o = e0 * G::B;
            const StageSpan sy(o - G::H, o + G::TB, n * G::B);
            fence_proxy_async_smem();  // the walks' reads of the x stage come before the copy's writes
            mbar_expect_tx(bar(1), sy.bulk_bytes());
            sy.issue(base + kOffX, reinterpret_cast<const char *>(y), o - G::H, bar(1));
            // y_{-1} (before the first element) is the identity
            if (e0 == 0) put_eye<T, Q>(reinterpret_cast<T *>(base + kOffX + G::H - G::B));
        }
        if (!__syncthreads_and(mbar_wait_bounded(bar(1), 0u, limit))) {
            if (threadIdx.x == 0) mbar_wait_bounded(bar(1), 0u, limit);  // a second chance for the copy to land
            return false;
        }
        // Mbar_i = P_{i-1}^T lambda_i, one element per thread, in place of lambda_i
        const T *py = reinterpret_cast<const T *>(base + kOffX + G::H - G::B);  // y_{i-1} at element slot i
        T *sg = reinterpret_cast<T *>(base + kOffG);
        for (int e = threadIdx.x; e < (int)ne; e += TH) {
            const E P = ld_matq<T, Q>(py + e * G::QQ);
            const E lam = ld_matq<T, Q>(sg + e * G::QQ);
#pragma unroll
            for (int r = 0; r < Q; ++r) {
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    T g = P.a[r] * lam.a[j];
#pragma unroll
                    for (int q = 1; q < Q; ++q) g += P.a[Q * q + r] * lam.a[Q * q + j];
                    sg[e * G::QQ + Q * r + j] = g;
                }
            }
        }
        __syncthreads();  // every adjoint is in the stage
        copy_out<T, TH>(reinterpret_cast<T *>(xbar + e0), sg, ne * G::B, accumulate != 0);
        return true;
    }
};

// Block size and run length per (type, q, direction).  Larger tiles mean
// fewer look-backs, which bound these scans, until shared memory (two staged
// arrays for the vjps, one for the forwards) or registers leave fewer than
// two blocks per SM.  Measured at n = 1e7 (3x3) / 4e6 (5x5) fp32 over
// threads x run in {32..384} x {3, 5, 7}: 3x3 forward 384 x 7 (0.22 ms;
// 256 x 7: 0.24, 128 x 7: 0.27), 3x3 vjp 224 x 7 (0.40; 192 x 7: 0.44,
// 128 x 7: 0.51), 5x5 forward 160 x 7 (0.28; 128 x 7: 0.31, 128 x 5: 0.35),
// 5x5 vjp 96 x 5 (1.03; 64 x 7: 1.09, 64 x 5: 1.31).  fp64 (bound by the FP64 pipe) takes tiles of the
// same bytes.
template <typename T, int Q, bool VJP> struct MMQStaged {
    static constexpr int seg = Q == 3 || !VJP ? 7 : 5;
    static constexpr int threads = VJP ? (Q == 3 ? (sizeof(T) == 4 ? 224 : 96) : (sizeof(T) == 4 ? 96 : 32))
                                       : (Q == 3 ? (sizeof(T) == 4 ? 384 : 128) : (sizeof(T) == 4 ? 160 : 64));
};

}  // namespace adc
