// reduce forward passes and vjps (Sec. 3).
//
//  ADD     : y = sum x;                    xbar (+)= ybar            (Sec. 3.2.1)
//  MIN/MAX : lifted (value, index), lowest index wins ties;
//            xbar (+)= ybar at k only                                (Sec. 3.2.2)
//  MUL     : lifted (zero count, product of non-zeros);
//            three-case map of Fig. 3                                (Sec. 3.2.3)
//  LIN/MM2 : general rule (Eq. red-adj, Fig. 2).  The forward pass saves, per
//            tile of the input, the exclusive prefix L_t and suffix R_t of the
//            tile aggregates; the vjp rebuilds l_i and r_i for each element from
//            L_t, R_t and in-tile scans held in registers, so it reads x once and
//            writes xbar once (3x the primal's bytes, against the ~8x of the
//            paper's fused two-scan formulation).
//
// Simple reductions: each block folds a contiguous range of tiles, writes one
// partial, and the last block to finish (threadfence + atomic ticket) combines
// the partials in block order, so results are deterministic for a given n.
#include "block_scan.cuh"
#include "common.cuh"
#include "internal.h"
#include "scan_engine.cuh"
#include "tile_io.cuh"

namespace adc {

constexpr int kRedThreads = 256;

// ------------------------------------------------------------- operators --
template <typename T> struct RAdd {
    using State = T;
    __device__ State identity() const { return T(0); }
    __device__ State combine(State a, State b) const { return a + b; }
    __device__ State lift(T x, int64_t) const { return x; }
};

template <typename T> struct MinMaxS { T v; int32_t i; int32_t pad; };

template <typename T, bool MAX> struct RSel {
    using State = MinMaxS<T>;
    int32_t n;
    __device__ State identity() const { return {MAX ? -Num<T>::inf() : Num<T>::inf(), n, 0}; }
    // Fig. 5's min^L: better value wins, equal values -> smaller index.
    __device__ State combine(const State &a, const State &b) const {
        const bool a_better = MAX ? (a.v > b.v) : (a.v < b.v);
        const bool b_better = MAX ? (b.v > a.v) : (b.v < a.v);
        if (a_better) return a;
        if (b_better) return b;
        return a.i <= b.i ? a : b;
    }
    __device__ State lift(T x, int64_t i) const { return {x, (int32_t)i, 0}; }
};

template <typename T> struct MulS { T p; int32_t z; int32_t pad; };

// Fig. 3's lifted primal: (count of zeros, product of non-zeros) under (+, *).
template <typename T> struct RMul {
    using State = MulS<T>;
    __device__ State identity() const { return {T(1), 0, 0}; }
    __device__ State combine(const State &a, const State &b) const { return {a.p * b.p, a.z + b.z, 0}; }
    __device__ State lift(T x, int64_t) const { return x == T(0) ? State{T(1), 1, 0} : State{x, 0, 0}; }
};

// sumOfProd (Sec. 3.3) on (p, s) = Pair{b: p, c: s}:
// (p1,s1) . (p2,s2) = (p1 + p2 + s1*s2, s1 + s2); associative and commutative.
template <typename T> struct RSop {
    using State = Pair<T>;
    __device__ State identity() const { return {T(0), T(0)}; }
    __device__ State combine(const State &a, const State &b) const { return {a.b + b.b + a.c * b.c, a.c + b.c}; }
    __device__ State lift(const Pair<T> &x, int64_t) const { return x; }
};

// General operators (non-commutative).
template <typename T> struct GLin {
    using State = Pair<T>;
    __device__ State identity() const { return {T(0), T(1)}; }
    __device__ State combine(const State &a, const State &b) const { return {b.b + b.c * a.b, b.c * a.c}; }
};
template <typename T> struct GMM2 {
    using State = Mat2<T>;
    __device__ State identity() const { return mat_eye<T>(); }
    __device__ State combine(const State &a, const State &b) const { return mat_mul(a, b); }
};
template <typename T, int Q> struct GMMQ {
    using State = MatQ<T, Q>;
    __device__ State identity() const { return matq_eye<T, Q>(); }
    __device__ State combine(const State &a, const State &b) const { return matq_mul(a, b); }
};

// ------------------------------------------------------- simple reduction --
// Workspace: [header][ticket u32 @ +8 in header][partials G states]
// The operators here (+, the lifted * and min/max, sumOfProd) are
// commutative, so a thread may take any of the tile's elements: it takes
// 16-byte words t, t + kRedThreads, ..., so that a warp's load covers 512
// contiguous bytes.  The lifted operators get each element's own index.
template <class Op, typename T, int ITEMS>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_simple(const Op op, const T *__restrict__ x, const int64_t n, const int64_t tiles_per_block,
                typename Op::State *__restrict__ part, unsigned *__restrict__ ticket,
                typename Op::State *__restrict__ result) {
    using S = typename Op::State;
    constexpr int TILE = kRedThreads * ITEMS;
    constexpr int WE = 16 / sizeof(T) < ITEMS ? 16 / sizeof(T) : ITEMS;  // elements per word
    constexpr int NWD = ITEMS / WE;                                       // words per thread and tile
    __shared__ S tmp[kRedThreads / kWarp];
    __shared__ bool last;
    const int64_t t0 = (int64_t)blockIdx.x * tiles_per_block;
    S acc = op.identity();
    for (int64_t t = t0; t < t0 + tiles_per_block; ++t) {
        if (t * TILE >= n) break;
        T v[NWD][WE];
#pragma unroll
        for (int j = 0; j < NWD; ++j)
            load_chunk(x, t * TILE + ((int64_t)j * kRedThreads + threadIdx.x) * WE, n, v[j], T{});
#pragma unroll
        for (int j = 0; j < NWD; ++j) {
            const int64_t c0 = t * TILE + ((int64_t)j * kRedThreads + threadIdx.x) * WE;
#pragma unroll
            for (int k = 0; k < WE; ++k)
                if (c0 + k < n) acc = op.combine(acc, op.lift(v[j][k], c0 + k));
        }
    }
    S total;
    block_exclusive_fwd<Op, kRedThreads>(op, acc, tmp, &total);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = total;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last block: combine the partials in block order
    S a = op.identity();
    const int per = (gridDim.x + kRedThreads - 1) / kRedThreads;
    for (int j = 0; j < per; ++j) {
        const int b = threadIdx.x * per + j;
        if (b < (int)gridDim.x) a = op.combine(a, load_cg(&part[b]));
    }
    block_exclusive_fwd<Op, kRedThreads>(op, a, tmp, &total);
    if (threadIdx.x == 0) *result = total;
}

// Finalisers: turn the lifted result into y and the saved residuals.
template <typename T> __global__ void k_fin_add(const T *r, T *y) { *y = *r; }
template <typename T> __global__ void k_fin_sel(const MinMaxS<T> *r, T *y, int32_t *k) {
    *y = r->v;
    *k = r->i;
}
template <typename T> __global__ void k_fin_sop(const Pair<T> *r, Pair<T> *y) { *y = *r; }
template <typename T> __global__ void k_fin_mul(const MulS<T> *r, T *y, int32_t *n0, T *p) {
    *y = r->z > 0 ? T(0) : r->p;
    *n0 = r->z;
    *p = r->p;
}

// ------------------------------------------------------ general reduction --
// Pass 1: the aggregate of every tile, in order.
template <class Op, typename T, int ITEMS>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_tiles(const Op op, const typename Op::State *__restrict__ x, const int64_t n,
               typename Op::State *__restrict__ tpart) {
    using S = typename Op::State;
    constexpr int TILE = kRedThreads * ITEMS;
    __shared__ S tmp[kRedThreads / kWarp];
    const int64_t c0 = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
    S v[ITEMS];
    load_chunk(x, c0, n, v, op.identity());
    S acc = op.identity();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) acc = op.combine(acc, v[k]);
    S total;
    block_exclusive_fwd<Op, kRedThreads>(op, acc, tmp, &total);
    if (threadIdx.x == 0) tpart[blockIdx.x] = total;
}

// Pass 2 (look-back scans over the T tile aggregates): element t carries the
// aggregate of tile t-1, so the inclusive scan at t is the EXCLUSIVE prefix
// L_t; the store of the last element also writes y = L_{T-1} . P_{T-1}.
template <class G, int ITEMS> struct TilePrefix {
    using State = typename G::State;
    using Aux = NoAux;
    struct Raw { State v[ITEMS]; };
    G g;
    const State *tpart;
    State *Lex;
    State *y;
    __device__ State identity() const { return g.identity(); }
    __device__ State combine(const State &a, const State &b) const { return g.combine(a, b); }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int64_t i = c0 + k;
            r.v[k] = (i > 0 && i <= n) ? tpart[i - 1] : g.identity();
        }
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) st[k] = (c0 + k < n) ? r.v[k] : g.identity();
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            if (c0 + k < n) Lex[c0 + k] = st[k];
            if (c0 + k == n - 1) *y = g.combine(st[k], tpart[n - 1]);
        }
    }
};

// Reverse look-back scan: element t carries the aggregate of tile t+1, so the
// inclusive value at t is the EXCLUSIVE suffix R_t.
template <class G, int ITEMS> struct TileSuffix {
    using State = typename G::State;
    using Aux = NoAux;
    struct Raw { State v[ITEMS]; };
    G g;
    const State *tpart;
    State *Rex;
    __device__ State identity() const { return g.identity(); }
    // logical order: `e` lies physically before everything already combined
    __device__ State combine(const State &acc, const State &e) const { return g.combine(e, acc); }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int64_t i = c0 + k;
            r.v[k] = (i + 1 < n) ? tpart[i + 1] : g.identity();
        }
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) st[k] = (c0 + k < n) ? r.v[k] : g.identity();
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k)
            if (c0 + k < n) Rex[c0 + k] = st[k];
    }
};
constexpr int kTileScanItems = 4;

// vjp of the general rule: xbar_i = d(l_i . x_i . r_i)/dx_i ^T ybar.
template <typename T> __device__ __forceinline__ Pair<T> general_adj(const Pair<T> &l, const Pair<T> &r, const Pair<T> &yb) {
    // y = r.b + r.c*(x.b + x.c*l.b), r.c*x.c*l.c
    return {r.c * yb.b, r.c * (l.b * yb.b + l.c * yb.c)};
}
template <typename T> __device__ __forceinline__ Mat2<T> general_adj(const Mat2<T> &l, const Mat2<T> &r, const Mat2<T> &yb) {
    return mat_mul(mat_mul(mat_t(l), yb), mat_t(r));  // L^T Ybar R^T
}
template <typename T, int Q>
__device__ __forceinline__ MatQ<T, Q> general_adj(const MatQ<T, Q> &l, const MatQ<T, Q> &r, const MatQ<T, Q> &yb) {
    return matq_mul(matq_mul(matq_t(l), yb), matq_t(r));  // L^T Ybar R^T
}

template <class Op, typename T, int ITEMS>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_general_vjp(const Op op, const typename Op::State *__restrict__ x, const int64_t n,
                     const typename Op::State *__restrict__ Lex, const typename Op::State *__restrict__ Rex,
                     const typename Op::State *__restrict__ ybar, typename Op::State *__restrict__ xbar,
                     const int accumulate) {
    using S = typename Op::State;
    constexpr int TILE = kRedThreads * ITEMS;
    __shared__ S tmp[kRedThreads / kWarp];
    const int64_t t = blockIdx.x;
    const int64_t c0 = t * TILE + (int64_t)threadIdx.x * ITEMS;
    S v[ITEMS];
    load_chunk(x, c0, n, v, op.identity());
    S acc = op.identity();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) acc = op.combine(acc, v[k]);
    S tot;
    const S pre = block_exclusive_fwd<Op, kRedThreads>(op, acc, tmp, &tot);
    const S suf = block_exclusive_rev<Op, kRedThreads>(op, acc, tmp);
    const S yb = *ybar;
    S l[ITEMS], r[ITEMS];
    S run = op.combine(Lex[t], pre);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        l[k] = run;
        run = op.combine(run, v[k]);
    }
    run = op.combine(suf, Rex[t]);
#pragma unroll
    for (int k = ITEMS - 1; k >= 0; --k) {
        r[k] = run;
        run = op.combine(v[k], run);
    }
    S out[ITEMS];
    if (accumulate) load_chunk(xbar, c0, n, out, op.identity());
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const S g = general_adj(l[k], r[k], yb);
        if (accumulate) {
            const T *gp = reinterpret_cast<const T *>(&g);
            T *op_ = reinterpret_cast<T *>(&out[k]);
#pragma unroll
            for (int c = 0; c < (int)(sizeof(S) / sizeof(T)); ++c) op_[c] += gp[c];
        } else {
            out[k] = g;
        }
    }
    store_chunk(xbar, c0, n, out);
}

// ------------------------------------------------------------- simple vjps --
template <typename T>
__global__ void k_vjp_add(T *__restrict__ xbar, const T *__restrict__ ybar, const int64_t n, const int accumulate) {
    const T yb = __ldg(ybar);
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        T v[V];
        if (accumulate) load_chunk(xbar, i * V, n, v, T(0));
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = accumulate ? v[k] + yb : yb;
        store_chunk(xbar, i * V, n, v);
    }
    for (int64_t i = nv * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        xbar[i] = accumulate ? xbar[i] + yb : yb;
}

template <typename T>
__global__ void k_vjp_sel_fill(T *__restrict__ xbar, const T *__restrict__ ybar, const int32_t *__restrict__ kp,
                               const int64_t n) {
    const T yb = __ldg(ybar);
    const int64_t kk = __ldg(kp);
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        T v[V];
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = (i * V + k == kk) ? yb : T(0);
        store_chunk(xbar, i * V, n, v);
    }
    for (int64_t i = nv * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        xbar[i] = (i == kk) ? yb : T(0);
}

template <typename T>
__global__ void k_vjp_sel_acc(T *__restrict__ xbar, const T *__restrict__ ybar, const int32_t *__restrict__ kp,
                              const int64_t n) {
    const int64_t kk = *kp;
    if (kk >= 0 && kk < n) xbar[kk] += *ybar;
}

// Fig. 3 return sweep.
template <typename T>
__global__ void k_vjp_mul(T *__restrict__ xbar, const T *__restrict__ x, const T *__restrict__ ybar,
                          const int32_t *__restrict__ n0p, const T *__restrict__ pp, const int64_t n,
                          const int accumulate) {
    const T yb = __ldg(ybar);
    const int32_t n0 = __ldg(n0p);
    const T p = __ldg(pp);
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = (n + V - 1) / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto grad = [&](T a) -> T {
        if (n0 == 0) return div_or_zero(p, a) * yb;
        if (n0 == 1 && a == T(0)) return p * yb;
        return T(0);
    };
    // two vectors per thread in flight before any result is needed
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += 2 * stride) {
        const int64_t j = i + stride;
        T a[V], b[V], o[V], q[V];
        load_chunk(x, i * V, n, a, T(1));
        if (j < nv) load_chunk(x, j * V, n, b, T(1));
        if (accumulate) {
            load_chunk(xbar, i * V, n, o, T(0));
            if (j < nv) load_chunk(xbar, j * V, n, q, T(0));
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            o[k] = accumulate ? o[k] + grad(a[k]) : grad(a[k]);
            if (j < nv) q[k] = accumulate ? q[k] + grad(b[k]) : grad(b[k]);
        }
        store_chunk(xbar, i * V, n, o);
        if (j < nv) store_chunk(xbar, j * V, n, q);
    }
}

// --------------------------------------------------------------- planning --
// Sec. 3.3, the invertible-operator rule for sumOfProd: with b_i = y (.)^-1 x_i,
// xbar_i = d(b_i . x)/dx ^T ybar = (ybar.p, ybar.p * b_i.s + ybar.s), b_i.s = y.s - x_i.s.
template <typename T>
__global__ void k_vjp_sop(Pair<T> *__restrict__ xbar, const Pair<T> *__restrict__ x, const Pair<T> *__restrict__ ybar,
                          const Pair<T> *__restrict__ y, const int64_t n, const int accumulate) {
    const Pair<T> yb = *ybar, yy = *y;
    constexpr int V = 16 / sizeof(Pair<T>) > 0 ? 16 / sizeof(Pair<T>) : 1;  // pairs per 128-bit word
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c * V < n; c += stride) {
        Pair<T> xv[V], o[V];
        load_chunk(x, c * V, n, xv, Pair<T>{T(0), T(0)});
        if (accumulate) load_chunk(xbar, c * V, n, o, Pair<T>{T(0), T(0)});
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const Pair<T> g{yb.b, yb.b * (yy.c - xv[k].c) + yb.c};
            o[k] = accumulate ? Pair<T>{o[k].b + g.b, o[k].c + g.c} : g;
        }
        store_chunk(xbar, c * V, n, o);
    }
}

template <typename T> struct RedItems {
    static constexpr int scalar = 64 / sizeof(T);
    static constexpr int pair = 64 / (2 * sizeof(T));  // 16 KB tiles of (b, c) pairs
    static constexpr int mat = 64 / (4 * sizeof(T));   // 16 KB tiles of 2x2 matrices
    static constexpr int mat3 = sizeof(T) == 4 ? 4 : 2; // 144-byte chunks of 3x3 matrices
    static constexpr int mat5 = 1;
};

static bool is_general(adc_op op) {
    return op == ADC_OP_LIN || op == ADC_OP_MM2 || op == ADC_OP_MM3 || op == ADC_OP_MM5;
}

static int64_t simple_grid(int64_t tiles) {
    int64_t g = (int64_t)num_sms() * 4;
    if (tiles < g) g = tiles;
    return g < 1 ? 1 : g;
}

template <typename T> static size_t general_state_bytes(adc_op op) {
    switch (op) {
    case ADC_OP_LIN: return sizeof(Pair<T>);
    case ADC_OP_MM3: return sizeof(MatQ<T, 3>);
    case ADC_OP_MM5: return sizeof(MatQ<T, 5>);
    default: return sizeof(Mat2<T>);
    }
}
template <typename T> static int64_t general_tiles(adc_op op, int64_t n) {
    int items = RedItems<T>::mat;
    if (op == ADC_OP_LIN) items = RedItems<T>::pair;
    if (op == ADC_OP_MM3) items = RedItems<T>::mat3;
    if (op == ADC_OP_MM5) items = RedItems<T>::mat5;
    const int tile = kRedThreads * items;
    return (n + tile - 1) / tile;
}

// Workspace of the general reduce: [header][tile aggregates][two look-back regions].
template <class G> static size_t general_ws(int64_t tiles) {
    using P = TilePrefix<G, kTileScanItems>;
    using Q = TileSuffix<G, kTileScanItems>;
    const size_t sb = sizeof(typename G::State);
    return kWsHeader + align_up((size_t)(tiles + 1) * sb, 256) + ScanShape<P, kTileScanItems>::region(tiles) +
           ScanShape<Q, kTileScanItems>::region(tiles);
}

template <class G, typename T, int ITEMS>
static adc_status general_fwd(int64_t n, const void *xv, void *yv, void *saved, void *ws, cudaStream_t s) {
    using S = typename G::State;
    constexpr int TILE = kRedThreads * ITEMS;
    const int64_t tiles = n > 0 ? (n + TILE - 1) / TILE : 1;  // n == 0: one tile of identities
    char *w = static_cast<char *>(ws);
    S *tpart = reinterpret_cast<S *>(w + kWsHeader);
    char *reg1 = w + kWsHeader + align_up((size_t)(tiles + 1) * sizeof(S), 256);
    char *reg2 = reg1 + ScanShape<TilePrefix<G, kTileScanItems>, kTileScanItems>::region(tiles);
    S *Lex = static_cast<S *>(saved);
    S *Rex = Lex + tiles;
    k_reduce_tiles<G, T, ITEMS><<<(unsigned)tiles, kRedThreads, 0, s>>>(G{}, static_cast<const S *>(xv), n, tpart);
    adc_status st = check_launch();
    if (st != ADC_OK) return st;
    TilePrefix<G, kTileScanItems> pre{G{}, tpart, Lex, static_cast<S *>(yv)};
    if ((st = run_scan<decltype(pre), kTileScanItems, false>(pre, tiles, ws, 2, reg1, s)) != ADC_OK) return st;
    TileSuffix<G, kTileScanItems> suf{G{}, tpart, Rex};
    return run_scan<decltype(suf), kTileScanItems, true>(suf, tiles, ws, 3, reg2, s);
}

template <typename T> static size_t red_ws_t(adc_op op, int64_t n) {
    if (is_general(op)) {
        const int64_t tiles = general_tiles<T>(op, n) > 0 ? general_tiles<T>(op, n) : 1;
        switch (op) {
        case ADC_OP_LIN: return general_ws<GLin<T>>(tiles);
        case ADC_OP_MM3: return general_ws<GMMQ<T, 3>>(tiles);
        case ADC_OP_MM5: return general_ws<GMMQ<T, 5>>(tiles);
        default: return general_ws<GMM2<T>>(tiles);
        }
    }
    const int items = op == ADC_OP_SOP ? RedItems<T>::pair : RedItems<T>::scalar;
    const int64_t tiles = (n + kRedThreads * items - 1) / (kRedThreads * items);
    return kWsHeader + (size_t)(simple_grid(tiles) + 1) * 32 + 256;
}

size_t reduce_ws_bytes(adc_op op, adc_dtype dt, int64_t n) {
    if (op > ADC_OP_MM5 || op < ADC_OP_ADD) return 0;
    return dt == ADC_F64 ? red_ws_t<double>(op, n) : red_ws_t<float>(op, n);
}

template <typename T> static size_t red_saved_t(adc_op op, int64_t n) {
    switch (op) {
    case ADC_OP_ADD: return 16;
    case ADC_OP_MIN:
    case ADC_OP_MAX: return 16;
    case ADC_OP_MUL: return 16;
    case ADC_OP_SOP: return 16;
    case ADC_OP_LIN:
    case ADC_OP_MM2:
    case ADC_OP_MM3:
    case ADC_OP_MM5: return 2 * (size_t)(general_tiles<T>(op, n) > 0 ? general_tiles<T>(op, n) : 1) * general_state_bytes<T>(op);
    default: return 0;
    }
}

size_t reduce_saved_bytes(adc_op op, adc_dtype dt, int64_t n) {
    return dt == ADC_F64 ? red_saved_t<double>(op, n) : red_saved_t<float>(op, n);
}

template <class Op, typename T, int ITEMS>
static adc_status launch_simple(const Op &op, const T *x, int64_t n, void *ws, cudaStream_t s,
                                typename Op::State **result) {
    constexpr int TILE = kRedThreads * ITEMS;
    const int64_t tiles = (n + TILE - 1) / TILE;
    const int64_t G = simple_grid(tiles);
    const int64_t tpb = tiles > 0 ? (tiles + G - 1) / G : 0;
    char *w = static_cast<char *>(ws);
    auto *part = reinterpret_cast<typename Op::State *>(w + kWsHeader);
    *result = part + G;
    k_reduce_simple<Op, T, ITEMS><<<(unsigned)G, kRedThreads, 0, s>>>(op, x, n, tpb, part, counter_slot(ws, 1),
                                                                       *result);
    return check_launch();
}

template <typename T>
static adc_status red_fwd_t(adc_op op, int64_t n, const void *xv, void *yv, void *saved, void *ws, cudaStream_t s) {
    constexpr int I = RedItems<T>::scalar;
    const T *x = static_cast<const T *>(xv);
    T *y = static_cast<T *>(yv);
    adc_status st;
    switch (op) {
    case ADC_OP_ADD: {
        RAdd<T> o;
        T *r;
        if ((st = launch_simple<RAdd<T>, T, I>(o, x, n, ws, s, &r)) != ADC_OK) return st;
        k_fin_add<T><<<1, 1, 0, s>>>(r, y);
        return check_launch();
    }
    case ADC_OP_MIN:
    case ADC_OP_MAX: {
        MinMaxS<T> *r;
        if (op == ADC_OP_MIN) {
            RSel<T, false> o{(int32_t)n};
            if ((st = launch_simple<RSel<T, false>, T, I>(o, x, n, ws, s, &r)) != ADC_OK) return st;
        } else {
            RSel<T, true> o{(int32_t)n};
            if ((st = launch_simple<RSel<T, true>, T, I>(o, x, n, ws, s, &r)) != ADC_OK) return st;
        }
        k_fin_sel<T><<<1, 1, 0, s>>>(r, y, static_cast<int32_t *>(saved));
        return check_launch();
    }
    case ADC_OP_MUL: {
        RMul<T> o;
        MulS<T> *r;
        if ((st = launch_simple<RMul<T>, T, I>(o, x, n, ws, s, &r)) != ADC_OK) return st;
        k_fin_mul<T><<<1, 1, 0, s>>>(r, y, static_cast<int32_t *>(saved),
                                     reinterpret_cast<T *>(static_cast<char *>(saved) + 8));
        return check_launch();
    }
    case ADC_OP_SOP: {
        RSop<T> o;
        Pair<T> *r;
        if ((st = launch_simple<RSop<T>, Pair<T>, RedItems<T>::pair>(o, static_cast<const Pair<T> *>(xv), n, ws, s,
                                                                     &r)) != ADC_OK)
            return st;
        k_fin_sop<T><<<1, 1, 0, s>>>(r, static_cast<Pair<T> *>(yv));
        return check_launch();
    }
    case ADC_OP_LIN:
        return general_fwd<GLin<T>, T, RedItems<T>::pair>(n, xv, yv, saved, ws, s);
    case ADC_OP_MM2:
        return general_fwd<GMM2<T>, T, RedItems<T>::mat>(n, xv, yv, saved, ws, s);
    case ADC_OP_MM3:
        return general_fwd<GMMQ<T, 3>, T, RedItems<T>::mat3>(n, xv, yv, saved, ws, s);
    case ADC_OP_MM5:
        return general_fwd<GMMQ<T, 5>, T, RedItems<T>::mat5>(n, xv, yv, saved, ws, s);
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status reduce_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *saved, void *ws,
                      cudaStream_t s) {
    return dt == ADC_F64 ? red_fwd_t<double>(op, n, x, y, saved, ws, s) : red_fwd_t<float>(op, n, x, y, saved, ws, s);
}

static unsigned elementwise_grid(int64_t work) {
    int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename T>
static adc_status red_vjp_t(adc_op op, int64_t n, const void *xv, const void *yv, const void *saved,
                            const void *ybar, void *xbar, int acc, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    constexpr int V = 16 / sizeof(T);
    switch (op) {
    case ADC_OP_ADD:
        k_vjp_add<T><<<elementwise_grid(n / V + 1), 256, 0, s>>>(static_cast<T *>(xbar), static_cast<const T *>(ybar), n, acc);
        return check_launch();
    case ADC_OP_MIN:
    case ADC_OP_MAX:
        if (acc)
            k_vjp_sel_acc<T><<<1, 1, 0, s>>>(static_cast<T *>(xbar), static_cast<const T *>(ybar),
                                             static_cast<const int32_t *>(saved), n);
        else
            k_vjp_sel_fill<T><<<elementwise_grid(n / V + 1), 256, 0, s>>>(
                static_cast<T *>(xbar), static_cast<const T *>(ybar), static_cast<const int32_t *>(saved), n);
        return check_launch();
    case ADC_OP_MUL:
        k_vjp_mul<T><<<elementwise_grid((n + V - 1) / V), 256, 0, s>>>(
            static_cast<T *>(xbar), static_cast<const T *>(xv), static_cast<const T *>(ybar),
            static_cast<const int32_t *>(saved), reinterpret_cast<const T *>(static_cast<const char *>(saved) + 8), n,
            acc);
        return check_launch();
    case ADC_OP_SOP: {
        constexpr int PV = 16 / sizeof(Pair<T>) > 0 ? 16 / sizeof(Pair<T>) : 1;
        k_vjp_sop<T><<<elementwise_grid((n + PV - 1) / PV), 256, 0, s>>>(
            static_cast<Pair<T> *>(xbar), static_cast<const Pair<T> *>(xv), static_cast<const Pair<T> *>(ybar),
            static_cast<const Pair<T> *>(yv), n, acc);
        return check_launch();
    }
    case ADC_OP_LIN:
    case ADC_OP_MM2: {
        const int64_t Tn = general_tiles<T>(op, n);
        const size_t sb = general_state_bytes<T>(op);
        const char *sv = static_cast<const char *>(saved);
        if (op == ADC_OP_LIN) {
            using S = Pair<T>;
            k_reduce_general_vjp<GLin<T>, T, RedItems<T>::pair><<<(unsigned)Tn, kRedThreads, 0, s>>>(
                GLin<T>{}, static_cast<const S *>(xv), n, reinterpret_cast<const S *>(sv),
                reinterpret_cast<const S *>(sv + Tn * sb), static_cast<const S *>(ybar), static_cast<S *>(xbar), acc);
        } else {
            using S = Mat2<T>;
            k_reduce_general_vjp<GMM2<T>, T, RedItems<T>::mat><<<(unsigned)Tn, kRedThreads, 0, s>>>(
                GMM2<T>{}, static_cast<const S *>(xv), n, reinterpret_cast<const S *>(sv),
                reinterpret_cast<const S *>(sv + Tn * sb), static_cast<const S *>(ybar), static_cast<S *>(xbar), acc);
        }
        return check_launch();
    }
    case ADC_OP_MM3: {
        using S = MatQ<T, 3>;
        const int64_t Tn = general_tiles<T>(op, n);
        const char *sv = static_cast<const char *>(saved);
        k_reduce_general_vjp<GMMQ<T, 3>, T, RedItems<T>::mat3><<<(unsigned)Tn, kRedThreads, 0, s>>>(
            GMMQ<T, 3>{}, static_cast<const S *>(xv), n, reinterpret_cast<const S *>(sv),
            reinterpret_cast<const S *>(sv + Tn * sizeof(S)), static_cast<const S *>(ybar), static_cast<S *>(xbar),
            acc);
        return check_launch();
    }
    case ADC_OP_MM5: {
        using S = MatQ<T, 5>;
        const int64_t Tn = general_tiles<T>(op, n);
        const char *sv = static_cast<const char *>(saved);
        k_reduce_general_vjp<GMMQ<T, 5>, T, RedItems<T>::mat5><<<(unsigned)Tn, kRedThreads, 0, s>>>(
            GMMQ<T, 5>{}, static_cast<const S *>(xv), n, reinterpret_cast<const S *>(sv),
            reinterpret_cast<const S *>(sv + Tn * sizeof(S)), static_cast<const S *>(ybar), static_cast<S *>(xbar),
            acc);
        return check_launch();
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status reduce_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *saved,
                      const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s) {
    (void)ws;
    return dt == ADC_F64 ? red_vjp_t<double>(op, n, x, y, saved, ybar, xbar, accumulate, s)
                         : red_vjp_t<float>(op, n, x, y, saved, ybar, xbar, accumulate, s);
}

}  // namespace adc
