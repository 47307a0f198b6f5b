// Scan forward passes (Sec. 5.1) and their vjps (Fig. 7, with the RBDS
// specialisation of Sec. 5.3.4 where the Jacobians allow it), each one
// decoupled-look-back launch.
//
// vjp: the backward recurrence lambda_i = ybar_i + lambda_{i+1} * J_{i+1} with
// J_{i+1} = d(y_i . x_{i+1}) / d y_i is solved as a reverse scan whose element
// is the affine map f_i(lambda) = ybar_i + lambda * J_{i+1} and whose operator
// is composition -- the paper's lin_o of Fig. 7, written in the order the
// reverse scan consumes elements.  The final map
// xbar_i = d(y_{i-1} . x_i)/dx_i ^T lambda_i (y_{-1} = e) is fused into the
// store, so a vjp reads x, y, ybar once and writes xbar once.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "scan_engine.cuh"
#include "scan_mmq.cuh"
#include "scan_tma.cuh"
#include "scan_staged.cuh"
#include "tile_io.cuh"

namespace adc {

// One streamed array: the thread's chunk, loaded in fetch() and read in build().
template <typename E, int ITEMS> struct Chunk { E v[ITEMS]; };

// A streamed array plus its neighbour on one side (x_{i+1} beyond the chunk,
// or y_{i-1} before it).
template <typename E, int ITEMS> struct HaloChunk {
    E v[ITEMS];
    E halo;
};

template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_next(const E *x, int64_t c0, int64_t n, HaloChunk<E, ITEMS> &r, E fill) {
    load_chunk(x, c0, n, r.v, fill);
    r.halo = (c0 + ITEMS < n) ? x[c0 + ITEMS] : fill;
}
template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_prev(const E *y, int64_t c0, int64_t n, HaloChunk<E, ITEMS> &r, E e) {
    load_chunk(y, c0, n, r.v, e);
    r.halo = (c0 > 0 && c0 - 1 < n) ? y[c0 - 1] : e;
}
// The same two fetches from a shared-memory stage (sm[lo + k] is element c0 + k,
// and the stage holds one element on each side of its range).
template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_next_sm(const E *sm, int64_t lo, int64_t c0, int64_t n, HaloChunk<E, ITEMS> &r,
                                              E fill) {
    load_chunk_sm(sm + lo, c0, n, r.v, fill);
    r.halo = (c0 + ITEMS < n) ? sm[lo + ITEMS] : fill;
}
template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_prev_sm(const E *sm, int64_t lo, int64_t c0, int64_t n, HaloChunk<E, ITEMS> &r,
                                              E e) {
    load_chunk_sm(sm + lo, c0, n, r.v, e);
    r.halo = (c0 > 0 && c0 - 1 < n) ? sm[lo - 1] : e;
}
// One chunk with one element on each side: v[k] = y[c0 + k], prev = y[c0 - 1],
// next = y[c0 + ITEMS] (fill outside [0, n)).
template <typename E, int ITEMS> struct Halo2Chunk {
    E v[ITEMS];
    E prev, next;
};
template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_both(const E *y, int64_t c0, int64_t n, Halo2Chunk<E, ITEMS> &r, E fill) {
    load_chunk(y, c0, n, r.v, fill);
    r.prev = (c0 > 0 && c0 - 1 < n) ? y[c0 - 1] : fill;
    r.next = (c0 + ITEMS < n) ? y[c0 + ITEMS] : fill;
}
template <typename E, int ITEMS>
__device__ __forceinline__ void fetch_both_sm(const E *sm, int64_t lo, int64_t c0, int64_t n, Halo2Chunk<E, ITEMS> &r,
                                              E fill) {
    load_chunk_sm(sm + lo, c0, n, r.v, fill);
    r.prev = (c0 > 0 && c0 - 1 < n) ? sm[lo - 1] : fill;
    r.next = (c0 + ITEMS < n) ? sm[lo + ITEMS] : fill;
}
// xs[k] = x[c0 + k + 1]  and  ys[k] = y[c0 + k - 1]
template <typename E, int ITEMS> __device__ __forceinline__ E next_of(const HaloChunk<E, ITEMS> &r, int k) {
    return (k + 1 < ITEMS) ? r.v[k + 1] : r.halo;
}
template <typename E, int ITEMS> __device__ __forceinline__ E prev_of(const HaloChunk<E, ITEMS> &r, int k) {
    return k > 0 ? r.v[k - 1] : r.halo;
}

// ------------------------------------------------------------ forward ops --
// One input array, scanned as is; the state is the element type.
template <typename E, int ITEMS, class Derived> struct PlainScan {
    using State = E;
    using Aux = NoAux;
    using Raw = Chunk<E, ITEMS>;
    const E *x;
    E *y;
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(x, c0, n, r.v, static_cast<const Derived *>(this)->identity());
    }
    __device__ void build(int64_t, int64_t, const Raw &r, State (&st)[ITEMS], Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) st[k] = r.v[k];
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &) const {
        store_chunk(y, c0, n, st);
    }
    // staged in shared memory (scan_staged.cuh)
    static constexpr int kStreams = 1;
    using Elem = E;
    __device__ const E *stream(int) const { return x; }
    __device__ void fetch_staged(const E *const (&sm)[1], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        load_chunk_sm(sm[0] + lo, c0, n, r.v, static_cast<const Derived *>(this)->identity());
    }
};

template <typename T, int ITEMS> struct FwdAdd : PlainScan<T, ITEMS, FwdAdd<T, ITEMS>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ T identity() const { return T(0); }
    __device__ T combine(T a, T b) const { return a + b; }
};

template <typename T, int ITEMS> struct FwdMul : PlainScan<T, ITEMS, FwdMul<T, ITEMS>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ T identity() const { return T(1); }
    __device__ T combine(T a, T b) const { return a * b; }
};

// min / max scans: the running extremum; the earlier operand wins ties (the
// lifted operator of Fig. 5 with the lowest index first).
template <typename T, int ITEMS, bool MAX> struct FwdSel : PlainScan<T, ITEMS, FwdSel<T, ITEMS, MAX>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ T identity() const { return MAX ? -Num<T>::inf() : Num<T>::inf(); }
    __device__ T combine(T a, T b) const { return (MAX ? (b > a) : (b < a)) ? b : a; }
    // The scan's loop starts from y_0 = x_0, and a NaN never loses as the
    // earlier operand, so a NaN x_0 makes every y_i NaN.  The partial scans
    // here start from the identity, which a NaN cannot beat, so that case is
    // written out: every output is x_0 when x_0 is NaN.
    __device__ void store(int64_t c0, int64_t n, const T (&st)[ITEMS], const NoAux &) const {
        const T x0 = __ldg(this->x);
        T out[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) out[k] = x0 != x0 ? x0 : st[k];
        store_chunk(this->y, c0, n, out);
    }
};

// linFnComp (Fig. 8): (b1,c1) . (b2,c2) = (b2 + c2*b1, c2*c1)
template <typename T, int ITEMS> struct FwdLin : PlainScan<Pair<T>, ITEMS, FwdLin<T, ITEMS>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ Pair<T> identity() const { return {T(0), T(1)}; }
    __device__ Pair<T> combine(const Pair<T> &a, const Pair<T> &b) const { return {b.b + b.c * a.b, b.c * a.c}; }
};

// sumOfProd (Fig. 8): (p1,s1) . (p2,s2) = (p1 + p2 + s1*s2, s1 + s2)
template <typename T, int ITEMS> struct FwdSop : PlainScan<Pair<T>, ITEMS, FwdSop<T, ITEMS>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ Pair<T> identity() const { return {T(0), T(0)}; }
    __device__ Pair<T> combine(const Pair<T> &a, const Pair<T> &b) const {
        return {a.b + b.b + a.c * b.c, a.c + b.c};
    }
};

template <typename T, int ITEMS> struct FwdMM2 : PlainScan<Mat2<T>, ITEMS, FwdMM2<T, ITEMS>> {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    __device__ Mat2<T> identity() const { return mat_eye<T>(); }
    __device__ Mat2<T> combine(const Mat2<T> &a, const Mat2<T> &b) const { return mat_mul(a, b); }
};

// ---------------------------------------------------------------- vjp ops --
// Sec. 5.3.1: the adjoint of a +-scan is a reverse +-scan of ybar.
template <typename T, int ITEMS> struct VjpAdd {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    using State = T;
    using Aux = NoAux;
    using Raw = Chunk<T, ITEMS>;
    const T *ybar;
    T *xbar;
    int accumulate;
    __device__ T identity() const { return T(0); }
    __device__ T combine(T a, T b) const { return a + b; }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const { load_chunk(ybar, c0, n, r.v, T(0)); }
    static constexpr int kStreams = 1;
    using Elem = T;
    __device__ const T *stream(int) const { return ybar; }
    __device__ void fetch_staged(const T *const (&sm)[1], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        load_chunk_sm(sm[0] + lo, c0, n, r.v, T(0));
    }
    __device__ void build(int64_t, int64_t, const Raw &r, T (&st)[ITEMS], Aux &) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) st[k] = r.v[k];
    }
    __device__ void store(int64_t c0, int64_t n, const T (&st)[ITEMS], const Aux &) const {
        if (accumulate) {
            T old[ITEMS], out[ITEMS];
            load_chunk(xbar, c0, n, old, T(0));
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) out[k] = old[k] + st[k];
            store_chunk(xbar, c0, n, out);
        } else {
            store_chunk(xbar, c0, n, st);
        }
    }
};

// Affine map lambda -> v + c * lambda with a scalar (RBDS, q = 1) coefficient.
template <typename T> struct AffS { T v, c; };
template <typename T> struct AffP { T vb, vc, c; };  // 2-vector value (lin)

// Inputs of the recurrence vjps: ybar_i, x_{i+1} (coefficient) and y_{i-1} (map).
template <typename E, int ITEMS> struct VjpRaw {
    Chunk<E, ITEMS> yb;
    HaloChunk<E, ITEMS> x;  // halo = x[c0 + ITEMS]
    HaloChunk<E, ITEMS> y;  // halo = y[c0 - 1]
};

// Product scan: J_{i+1} = x_{i+1}; xbar_i = y_{i-1} * lambda_i.
template <typename T, int ITEMS> struct VjpMul {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    static constexpr int kRangeTiles = sizeof(T) == 4 ? 8 : 0;
    using State = AffS<T>;
    using Raw = VjpRaw<T, ITEMS>;
    struct Aux { T yprev[ITEMS]; };
    const T *x, *y, *ybar;
    T *xbar;
    int accumulate;
    __device__ State identity() const { return {T(0), T(1)}; }
    __device__ State combine(const State &acc, const State &e) const { return {e.v + e.c * acc.v, e.c * acc.c}; }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(ybar, c0, n, r.yb.v, T(0));
        fetch_next(x, c0, n, r.x, T(1));
        fetch_prev(y, c0, n, r.y, T(1));
    }
    static constexpr int kStreams = 3;
    using Elem = T;
    __device__ const T *stream(int s) const { return s == 0 ? ybar : (s == 1 ? x : y); }
    __device__ void fetch_staged(const T *const (&sm)[3], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        load_chunk_sm(sm[0] + lo, c0, n, r.yb.v, T(0));
        fetch_next_sm(sm[1], lo, c0, n, r.x, T(1));
        fetch_prev_sm(sm[2], lo, c0, n, r.y, T(1));
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            aux.yprev[k] = prev_of(r.y, k);
            st[k] = (c0 + k < n) ? State{r.yb.v[k], next_of(r.x, k)} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        T out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, T(0));
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) out[k] = (accumulate ? out[k] : T(0)) + aux.yprev[k] * st[k].v;
        store_chunk(xbar, c0, n, out);
    }
};

// min / max scan (the general rule of Fig. 7 with a scalar Jacobian): the step
// y_{i+1} = y_i . x_{i+1} has d/dy_i = c_{i+1} = [y_i selected] and
// d/dx_{i+1} = 1 - c_{i+1}, so lambda_i = ybar_i + c_{i+1} lambda_{i+1} and
// xbar_i = [x_i selected at step i] lambda_i (x_0 always is).  Both
// selections are read off y alone: x_i wins step i exactly when y_i differs
// from y_{i-1} (a strict win changes the value, a loss or a tie keeps it; two
// NaNs count as equal, as a NaN y_{i-1} is never beaten), so x is not read.
template <typename T> __device__ __forceinline__ bool same_value(T a, T b) { return a == b || (a != a && b != b); }

template <typename T, int ITEMS, bool MAX> struct VjpSel {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    using State = AffS<T>;
    struct Raw {
        Chunk<T, ITEMS> yb;
        Halo2Chunk<T, ITEMS> y;
    };
    struct Aux { T sel[ITEMS]; };
    const T *x, *y, *ybar;
    T *xbar;
    int accumulate;
    __device__ State identity() const { return {T(0), T(1)}; }
    __device__ State combine(const State &acc, const State &e) const { return {e.v + e.c * acc.v, e.c * acc.c}; }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(ybar, c0, n, r.yb.v, T(0));
        fetch_both(y, c0, n, r.y, T(0));
    }
    static constexpr int kStreams = 2;
    using Elem = T;
    __device__ const T *stream(int s) const { return s == 0 ? ybar : y; }
    __device__ void fetch_staged(const T *const (&sm)[2], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        load_chunk_sm(sm[0] + lo, c0, n, r.yb.v, T(0));
        fetch_both_sm(sm[1], lo, c0, n, r.y, T(0));
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int64_t i = c0 + k;
            const T yi = r.y.v[k];
            const T yp = k > 0 ? r.y.v[k - 1] : r.y.prev;
            const T yn = k + 1 < ITEMS ? r.y.v[k + 1] : r.y.next;
            aux.sel[k] = (i == 0 || !same_value(yi, yp)) ? T(1) : T(0);
            const T c = (i + 1 < n && !same_value(yn, yi)) ? T(0) : T(1);
            st[k] = (i < n) ? State{r.yb.v[k], c} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        T out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, T(0));
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const T g = aux.sel[k] * st[k].v;
            out[k] = accumulate ? out[k] + g : g;
        }
        store_chunk(xbar, c0, n, out);
    }
};

// linFnComp scan: J = diag(c_{i+1}, c_{i+1}) (Sec. 5.3.4);
// bbar_i = lambda.b, cbar_i = lambda.b * B_{i-1} + lambda.c * C_{i-1}, (B,C)_{-1} = (0,1).
template <typename T, int ITEMS> struct VjpLin {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    static constexpr int kRangeTiles = sizeof(T) == 4 ? 8 : 0;
    using State = AffP<T>;
    using Raw = VjpRaw<Pair<T>, ITEMS>;
    struct Aux { Pair<T> yprev[ITEMS]; };
    const Pair<T> *x, *y, *ybar;
    Pair<T> *xbar;
    int accumulate;
    __device__ State identity() const { return {T(0), T(0), T(1)}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {e.vb + e.c * acc.vb, e.vc + e.c * acc.vc, e.c * acc.c};
    }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        const Pair<T> e{T(0), T(1)};
        load_chunk(ybar, c0, n, r.yb.v, Pair<T>{T(0), T(0)});
        fetch_next(x, c0, n, r.x, e);
        fetch_prev(y, c0, n, r.y, e);
    }
    static constexpr int kStreams = 3;
    using Elem = Pair<T>;
    __device__ const Pair<T> *stream(int s) const { return s == 0 ? ybar : (s == 1 ? x : y); }
    __device__ void fetch_staged(const Pair<T> *const (&sm)[3], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        const Pair<T> e{T(0), T(1)};
        load_chunk_sm(sm[0] + lo, c0, n, r.yb.v, Pair<T>{T(0), T(0)});
        fetch_next_sm(sm[1], lo, c0, n, r.x, e);
        fetch_prev_sm(sm[2], lo, c0, n, r.y, e);
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            aux.yprev[k] = prev_of(r.y, k);
            st[k] = (c0 + k < n) ? State{r.yb.v[k].b, r.yb.v[k].c, next_of(r.x, k).c} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        Pair<T> out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, Pair<T>{T(0), T(0)});
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const T gb = st[k].vb;
            const T gc = gb * aux.yprev[k].b + st[k].vc * aux.yprev[k].c;
            out[k] = accumulate ? Pair<T>{out[k].b + gb, out[k].c + gc} : Pair<T>{gb, gc};
        }
        store_chunk(xbar, c0, n, out);
    }
};

// sumOfProd scan by the general rule of Fig. 7 (arity 2, Jacobian blocks not
// redundant): the step y_{i+1} = y_i . x_{i+1} has
//   d y_{i+1} / d y_i     = [[1, s(x_{i+1})], [0, 1]],
//   d y_{i+1} / d x_{i+1} = [[1, s(y_i)],     [0, 1]]     (rows p, s; columns p, s),
// so lambda_i = ybar_i + (lambda_{i+1}.p, s(x_{i+1}) lambda_{i+1}.p + lambda_{i+1}.s) and
// xbar_i = (lambda_i.p, s(y_{i-1}) lambda_i.p + lambda_i.s), y_{-1} = (0, 0).
// Unit upper-triangular 2x2 matrices multiply by adding their corner entries,
// so the composed coefficient of lin_o is carried as that one entry (sig):
// the affine map lambda -> v + lambda [[1, sig], [0, 1]] is 3 values, not 2 + 4.
template <typename T> struct AffU { T vp, vs, sig; };

template <typename T, int ITEMS> struct VjpSop {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    static constexpr int kRangeTiles = sizeof(T) == 4 ? 8 : 0;
    using State = AffU<T>;
    using Raw = VjpRaw<Pair<T>, ITEMS>;
    struct Aux { T sprev[ITEMS]; };
    const Pair<T> *x, *y, *ybar;
    Pair<T> *xbar;
    int accumulate;
    __device__ State identity() const { return {T(0), T(0), T(0)}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {e.vp + acc.vp, e.vs + e.sig * acc.vp + acc.vs, acc.sig + e.sig};
    }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        const Pair<T> z{T(0), T(0)};
        load_chunk(ybar, c0, n, r.yb.v, z);
        fetch_next(x, c0, n, r.x, z);
        fetch_prev(y, c0, n, r.y, z);
    }
    static constexpr int kStreams = 3;
    using Elem = Pair<T>;
    __device__ const Pair<T> *stream(int s) const { return s == 0 ? ybar : (s == 1 ? x : y); }
    __device__ void fetch_staged(const Pair<T> *const (&sm)[3], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        const Pair<T> z{T(0), T(0)};
        load_chunk_sm(sm[0] + lo, c0, n, r.yb.v, z);
        fetch_next_sm(sm[1], lo, c0, n, r.x, z);
        fetch_prev_sm(sm[2], lo, c0, n, r.y, z);
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            aux.sprev[k] = prev_of(r.y, k).c;
            st[k] = (c0 + k < n) ? State{r.yb.v[k].b, r.yb.v[k].c, next_of(r.x, k).c} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        Pair<T> out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, Pair<T>{T(0), T(0)});
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const T gp = st[k].vp;
            const T gs = aux.sprev[k] * st[k].vp + st[k].vs;
            out[k] = accumulate ? Pair<T>{out[k].b + gp, out[k].c + gs} : Pair<T>{gp, gs};
        }
        store_chunk(xbar, c0, n, out);
    }
};

// 2x2 matrix-product scan: f_i(L) = Ybar_i + L * M_{i+1}^T;  Mbar_i = P_{i-1}^T * lambda_i, P_{-1} = I.
template <typename T> struct AffM { Mat2<T> v, c; };

template <typename T, int ITEMS> struct VjpMM2 {
    static constexpr bool kKeepPrefix = sizeof(T) == 8;  // fp64: the combine is the bound
    using State = AffM<T>;
    using Raw = VjpRaw<Mat2<T>, ITEMS>;
    struct Aux { Mat2<T> yprev[ITEMS]; };
    const Mat2<T> *x, *y, *ybar;
    Mat2<T> *xbar;
    int accumulate;
    __device__ State identity() const { return {mat_zero<T>(), mat_eye<T>()}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {mat_add(e.v, mat_mul(acc.v, e.c)), mat_mul(acc.c, e.c)};
    }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(ybar, c0, n, r.yb.v, mat_zero<T>());
        fetch_next(x, c0, n, r.x, mat_eye<T>());
        fetch_prev(y, c0, n, r.y, mat_eye<T>());
    }
    static constexpr int kStreams = 3;
    using Elem = Mat2<T>;
    __device__ const Mat2<T> *stream(int s) const { return s == 0 ? ybar : (s == 1 ? x : y); }
    __device__ void fetch_staged(const Mat2<T> *const (&sm)[3], int64_t lo, int64_t c0, int64_t n, Raw &r) const {
        load_chunk_sm(sm[0] + lo, c0, n, r.yb.v, mat_zero<T>());
        fetch_next_sm(sm[1], lo, c0, n, r.x, mat_eye<T>());
        fetch_prev_sm(sm[2], lo, c0, n, r.y, mat_eye<T>());
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            aux.yprev[k] = prev_of(r.y, k);
            st[k] = (c0 + k < n) ? State{r.yb.v[k], mat_t(next_of(r.x, k))} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        Mat2<T> out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, mat_zero<T>());
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const Mat2<T> g = mat_mul(mat_t(aux.yprev[k]), st[k].v);
            out[k] = accumulate ? mat_add(out[k], g) : g;
        }
        store_chunk(xbar, c0, n, out);
    }
};

// q x q matrix-product scans (q = 3, 5): the same forward, and the vjp with
// the RBDS Jacobian M_{i+1}^T (Sec. 5.3.4 for q > 2): f_i(L) = Ybar_i + L M_{i+1}^T,
// Mbar_i = P_{i-1}^T lambda_i.
template <typename T, int Q, int ITEMS>
struct FwdMMQ : PlainScan<MatQ<T, Q>, ITEMS, FwdMMQ<T, Q, ITEMS>> {
    __device__ MatQ<T, Q> identity() const { return matq_eye<T, Q>(); }
    __device__ MatQ<T, Q> combine(const MatQ<T, Q> &a, const MatQ<T, Q> &b) const { return matq_mul(a, b); }
};

template <typename T, int Q, int ITEMS> struct VjpMMQ {
    using E = MatQ<T, Q>;
    using State = AffQ<T, Q>;
    using Raw = VjpRaw<E, ITEMS>;
    struct Aux { E yprev[ITEMS]; };
    const E *x, *y, *ybar;
    E *xbar;
    int accumulate;
    __device__ State identity() const { return {matq_zero<T, Q>(), matq_eye<T, Q>()}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {matq_add(e.v, matq_mul(acc.v, e.c)), matq_mul(acc.c, e.c)};
    }
    __device__ void fetch(int64_t c0, int64_t n, Raw &r) const {
        load_chunk(ybar, c0, n, r.yb.v, matq_zero<T, Q>());
        fetch_next(x, c0, n, r.x, matq_eye<T, Q>());
        fetch_prev(y, c0, n, r.y, matq_eye<T, Q>());
    }
    __device__ void build(int64_t c0, int64_t n, const Raw &r, State (&st)[ITEMS], Aux &aux) const {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            aux.yprev[k] = prev_of(r.y, k);
            st[k] = (c0 + k < n) ? State{r.yb.v[k], matq_t(next_of(r.x, k))} : identity();
        }
    }
    __device__ void store(int64_t c0, int64_t n, const State (&st)[ITEMS], const Aux &aux) const {
        E out[ITEMS];
        if (accumulate) load_chunk(xbar, c0, n, out, matq_zero<T, Q>());
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const E g = matq_mul(matq_t(aux.yprev[k]), st[k].v);
            out[k] = accumulate ? matq_add(out[k], g) : g;
        }
        store_chunk(xbar, c0, n, out);
    }
};

// Segment forms of the q x q matrix scans (q = 3, 5), for states too large
// to hold several per thread: an engine item is a run of SEG consecutive
// elements.  build() streams the run once, composing its state one element
// at a time (one state and one element in registers); the engine scans the
// runs' states and hands store() each run's EXCLUSIVE prefix, from which
// store() re-walks the run.  The re-walk needs only the value part of the
// vjp's affine maps, so it costs one matrix product per element instead of
// two.  Loads are per thread over its own contiguous run (L1 keeps the lines
// between the two walks).
template <typename T, int Q, int SEG> struct SegFwdMMQ {
    using E = MatQ<T, Q>;
    using State = E;
    using Aux = NoAux;
    struct Raw {};
    static constexpr bool kExclusiveStore = true;
    static constexpr bool kPerTileOnly = true;
    const E *x;
    E *y;
    int64_t n;  // elements (the engine counts runs)
    __device__ State identity() const { return matq_eye<T, Q>(); }
    __device__ State combine(const State &a, const State &b) const { return matq_mul(a, b); }
    __device__ void fetch(int64_t, int64_t, Raw &) const {}
    __device__ void build(int64_t c0, int64_t items, const Raw &, State (&st)[1], Aux &) const {
        E s = matq_eye<T, Q>();
        if (c0 < items) {
            const int64_t lo = c0 * SEG, hi = (lo + SEG < n) ? lo + SEG : n;
            for (int64_t i = lo; i < hi; ++i) matq_mul_right(s, x[i]);
        }
        st[0] = s;
    }
    __device__ void store(int64_t c0, int64_t items, const State (&ex)[1], const Aux &) const {
        if (c0 >= items) return;
        const int64_t lo = c0 * SEG, hi = (lo + SEG < n) ? lo + SEG : n;
        E run = ex[0];
        for (int64_t i = lo; i < hi; ++i) {
            matq_mul_right(run, x[i]);
            y[i] = run;
        }
    }
};

// vjp (reverse): the run's state composes f_i(L) = Ybar_i + L M_{i+1}^T from
// its last element down; the re-walk applies lambda_i = Ybar_i + lambda_{i+1}
// M_{i+1}^T from the incoming lambda and writes Mbar_i = P_{i-1}^T lambda_i.
template <typename T, int Q, int SEG> struct SegVjpMMQ {
    using E = MatQ<T, Q>;
    using State = AffQ<T, Q>;
    using Aux = NoAux;
    struct Raw {};
    static constexpr bool kExclusiveStore = true;
    static constexpr bool kPerTileOnly = true;
    const E *x, *y, *ybar;
    E *xbar;
    int accumulate;
    int64_t n;
    __device__ State identity() const { return {matq_zero<T, Q>(), matq_eye<T, Q>()}; }
    __device__ State combine(const State &acc, const State &e) const {
        return {matq_add(e.v, matq_mul(acc.v, e.c)), matq_mul(acc.c, e.c)};
    }
    __device__ void fetch(int64_t, int64_t, Raw &) const {}
    __device__ void build(int64_t c0, int64_t items, const Raw &, State (&st)[1], Aux &) const {
        State s = identity();
        if (c0 < items) {
            const int64_t lo = c0 * SEG, hi = (lo + SEG < n) ? lo + SEG : n;
            for (int64_t i = hi - 1; i >= lo; --i) {
                // s <- f_i o s: v = Ybar_i + v M^T, c = c M^T  (M = x_{i+1}; I past the end)
                if (i + 1 < n) {
                    const E M = x[i + 1];
                    matq_mul_right_t(s.v, M);
                    matq_mul_right_t(s.c, M);
                }
                const E yb = ybar[i];
#pragma unroll
                for (int k = 0; k < Q * Q; ++k) s.v.a[k] += yb.a[k];
            }
        }
        st[0] = s;
    }
    __device__ void store(int64_t c0, int64_t items, const State (&ex)[1], const Aux &) const {
        if (c0 >= items) return;
        const int64_t lo = c0 * SEG, hi = (lo + SEG < n) ? lo + SEG : n;
        E lam = ex[0].v;
        for (int64_t i = hi - 1; i >= lo; --i) {
            if (i + 1 < n) matq_mul_right_t(lam, x[i + 1]);
            const E yb = ybar[i];
#pragma unroll
            for (int k = 0; k < Q * Q; ++k) lam.a[k] += yb.a[k];
            // Mbar_i = P_{i-1}^T lambda_i (P_{-1} = I), row by row
            const E P = i > 0 ? y[i - 1] : matq_eye<T, Q>();
            E *dst = xbar + i;
#pragma unroll
            for (int r = 0; r < Q; ++r) {
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    T g = P.a[r] * lam.a[j];
#pragma unroll
                    for (int k = 1; k < Q; ++k) g += P.a[Q * k + r] * lam.a[Q * k + j];
                    dst->a[Q * r + j] = accumulate ? dst->a[Q * r + j] + g : g;
                }
            }
        }
    }
};

// Elements per run: enough to amortise the engine's per-item scan of a large
// state, few enough that the run's lines stay in L1 between the two walks
// (measured at n = 1e7 / 4e6 fp32: 8 beat 4 and 16 for both q).
template <int Q> struct SegLen { static constexpr int value = 8; };

// -------------------------------------------------------------- launching --
// Items per thread: 64 bytes of each streamed array per thread (32 for the
// three-array vjps), so a tile is 16 KB (8 KB) per array.
template <typename T> struct Items {
    static constexpr int scalar = 64 / sizeof(T);       // add / mul
    static constexpr int pair = 64 / (2 * sizeof(T));   // lin
    static constexpr int mat = 64 / (4 * sizeof(T));    // mm2
    static constexpr int vscalar = 32 / sizeof(T);      // vjp mul
    static constexpr int vpair = 32 / (2 * sizeof(T));  // vjp lin
    static constexpr int vmat = 2;                      // vjp mm2
    // staged engine: 16 bytes of each array per thread per tile
    static constexpr int s_scalar = 16 / sizeof(T);
    static constexpr int s_pair = 16 / (2 * sizeof(T)) > 0 ? 16 / (2 * sizeof(T)) : 1;
    static constexpr int s_mat = 1;
    // q x q matrices: whole 16-byte words per thread where it stays small
    static constexpr int mat3 = sizeof(T) == 4 ? 4 : 2;  // 144 bytes
    static constexpr int mat5 = 1;
    static constexpr int vmatq = 1;
};

// Engines fed by bulk (TMA) copies into shared memory: the range-staged one
// (test hook 3) and the per-tile one (test hook 4).
static bool use_staged(int64_t n, int64_t regular_tile) {
    if (n <= 0) return false;
    if (g_scan_engine == 3 || g_scan_engine == 4) return true;
    (void)regular_tile;
    return false;
}

static size_t max4(size_t a, size_t b, size_t c, size_t d) {
    const size_t ab = a > b ? a : b, cd = c > d ? c : d;
    return ab > cd ? ab : cd;
}

// The bulk-staged matrix segment scans (scan_mmq.cuh) at the run length and
// block size MMQStaged picks.
template <typename T, int Q, bool VJP> using MMQStagedOp =
    typename std::conditional<VJP, StagedVjpMMQ<T, Q, MMQStaged<T, Q, true>::threads, MMQStaged<T, Q, true>::seg>,
                              StagedFwdMMQ<T, Q, MMQStaged<T, Q, false>::threads, MMQStaged<T, Q, false>::seg>>::type;
template <typename T, int Q, bool VJP> static size_t mmq_staged_region(int64_t n) {
    constexpr int L = MMQStaged<T, Q, VJP>::seg;
    return ScanShape<MMQStagedOp<T, Q, VJP>, 1>::region((n + L - 1) / L);
}

template <typename T> static size_t scan_ws_t(adc_op op, int64_t n) {
    using I = Items<T>;
    size_t a = 0, b = 0, c = 0, d = 0;
    switch (op) {
    case ADC_OP_ADD:
        a = ScanShape<FwdAdd<T, I::scalar>, I::scalar>::region(n);
        b = ScanShape<VjpAdd<T, I::scalar>, I::scalar>::region(n);
        break;
    case ADC_OP_MUL:
        a = ScanShape<FwdMul<T, I::scalar>, I::scalar>::region(n);
        b = ScanShape<VjpMul<T, I::vscalar>, I::vscalar>::region(n);
        break;
    case ADC_OP_LIN:
        a = ScanShape<FwdLin<T, I::pair>, I::pair>::region(n);
        b = ScanShape<VjpLin<T, I::vpair>, I::vpair>::region(n);
        break;
    case ADC_OP_MM2:
        a = ScanShape<FwdMM2<T, I::mat>, I::mat>::region(n);
        b = ScanShape<VjpMM2<T, I::vmat>, I::vmat>::region(n);
        break;
    case ADC_OP_MIN:
    case ADC_OP_MAX:
        a = ScanShape<FwdSel<T, I::scalar, false>, I::scalar>::region(n);
        b = ScanShape<VjpSel<T, I::vscalar, false>, I::vscalar>::region(n);
        c = ScanShape<FwdSel<T, I::s_scalar, false>, I::s_scalar>::region(n);
        d = ScanShape<VjpSel<T, I::s_scalar, false>, I::s_scalar>::region(n);
        return kWsHeader + max4(a, b, c, d);
    case ADC_OP_SOP:
        a = ScanShape<FwdSop<T, I::pair>, I::pair>::region(n);
        b = ScanShape<VjpSop<T, I::vpair>, I::vpair>::region(n);
        c = ScanShape<FwdSop<T, I::s_pair>, I::s_pair>::region(n);
        d = ScanShape<VjpSop<T, I::s_pair>, I::s_pair>::region(n);
        return kWsHeader + max4(a, b, c, d);
    case ADC_OP_MM3: {
        const int64_t runs = (n + SegLen<3>::value - 1) / SegLen<3>::value;
        a = ScanShape<FwdMMQ<T, 3, I::mat3>, I::mat3>::region(n);
        b = ScanShape<SegVjpMMQ<T, 3, SegLen<3>::value>, 1>::region(runs);
        c = mmq_staged_region<T, 3, false>(n);
        d = mmq_staged_region<T, 3, true>(n);
        return kWsHeader + max4(a, b, c, d);
    }
    case ADC_OP_MM5: {
        const int64_t runs = (n + SegLen<5>::value - 1) / SegLen<5>::value;
        a = ScanShape<SegFwdMMQ<T, 5, SegLen<5>::value>, 1>::region(runs);
        b = ScanShape<SegVjpMMQ<T, 5, SegLen<5>::value>, 1>::region(runs);
        c = mmq_staged_region<T, 5, false>(n);
        d = mmq_staged_region<T, 5, true>(n);
        return kWsHeader + max4(a, b, c, d);
    }
    default: return 0;
    }
    switch (op) {
    case ADC_OP_ADD:
        c = ScanShape<FwdAdd<T, I::s_scalar>, I::s_scalar>::region(n);
        d = ScanShape<VjpAdd<T, I::s_scalar>, I::s_scalar>::region(n);
        break;
    case ADC_OP_MUL:
        c = ScanShape<FwdMul<T, I::s_scalar>, I::s_scalar>::region(n);
        d = ScanShape<VjpMul<T, I::s_scalar>, I::s_scalar>::region(n);
        break;
    case ADC_OP_LIN:
        c = ScanShape<FwdLin<T, I::s_pair>, I::s_pair>::region(n);
        d = ScanShape<VjpLin<T, I::s_pair>, I::s_pair>::region(n);
        break;
    default:
        c = ScanShape<FwdMM2<T, I::s_mat>, I::s_mat>::region(n);
        d = ScanShape<VjpMM2<T, I::s_mat>, I::s_mat>::region(n);
        break;
    }
    return kWsHeader + max4(a, b, c, d);
}

size_t scan_ws_bytes(adc_op op, adc_dtype dt, int64_t n) {
    return dt == ADC_F64 ? scan_ws_t<double>(op, n) : scan_ws_t<float>(op, n);
}

template <class Op, int ITEMS, bool REVERSE>
static adc_status launch(const Op &o, int64_t n, void *ws, cudaStream_t s) {
    return run_scan<Op, ITEMS, REVERSE>(o, n, ws, 0, static_cast<char *>(ws) + kWsHeader, s);
}
template <class Op, int ITEMS, bool REVERSE>
static adc_status launch_staged(const Op &o, int64_t n, void *ws, cudaStream_t s) {
    if (g_scan_engine == 4) return run_scan_tma<Op, ITEMS, REVERSE>(o, n, ws, 0, static_cast<char *>(ws) + kWsHeader, s);
    return run_scan_staged<Op, ITEMS, REVERSE>(o, n, ws, 0, static_cast<char *>(ws) + kWsHeader, s);
}

// The engines of run_scan with 16 bytes of each array per thread per tile
// (test hook 5): consecutive threads hold consecutive 16-byte words, so a
// warp's load or store covers 512 contiguous bytes.
template <typename T>
static adc_status scan_fwd_items16(adc_op op, int64_t n, const void *x, void *y, void *ws, cudaStream_t s) {
    using I = Items<T>;
    switch (op) {
    case ADC_OP_ADD: {
        FwdAdd<T, I::s_scalar> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::s_scalar, false>(o, n, ws, s);
    }
    case ADC_OP_MUL: {
        FwdMul<T, I::s_scalar> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::s_scalar, false>(o, n, ws, s);
    }
    case ADC_OP_MIN: {
        FwdSel<T, I::s_scalar, false> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::s_scalar, false>(o, n, ws, s);
    }
    case ADC_OP_MAX: {
        FwdSel<T, I::s_scalar, true> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::s_scalar, false>(o, n, ws, s);
    }
    case ADC_OP_LIN: {
        FwdLin<T, I::s_pair> o;
        o.x = static_cast<const Pair<T> *>(x);
        o.y = static_cast<Pair<T> *>(y);
        return launch<decltype(o), I::s_pair, false>(o, n, ws, s);
    }
    case ADC_OP_SOP: {
        FwdSop<T, I::s_pair> o;
        o.x = static_cast<const Pair<T> *>(x);
        o.y = static_cast<Pair<T> *>(y);
        return launch<decltype(o), I::s_pair, false>(o, n, ws, s);
    }
    case ADC_OP_MM2: {
        FwdMM2<T, I::s_mat> o;
        o.x = static_cast<const Mat2<T> *>(x);
        o.y = static_cast<Mat2<T> *>(y);
        return launch<decltype(o), I::s_mat, false>(o, n, ws, s);
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

template <typename T>
static adc_status scan_vjp_items16(adc_op op, int64_t n, const void *x, const void *y, const void *ybar, void *xbar,
                                   int acc, void *ws, cudaStream_t s) {
    using I = Items<T>;
    switch (op) {
    case ADC_OP_ADD: {
        VjpAdd<T, I::s_scalar> o{static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::s_scalar, true>(o, n, ws, s);
    }
    case ADC_OP_MUL: {
        VjpMul<T, I::s_scalar> o{static_cast<const T *>(x), static_cast<const T *>(y), static_cast<const T *>(ybar),
                                 static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::s_scalar, true>(o, n, ws, s);
    }
    case ADC_OP_MIN: {
        VjpSel<T, I::s_scalar, false> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                        static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::s_scalar, true>(o, n, ws, s);
    }
    case ADC_OP_MAX: {
        VjpSel<T, I::s_scalar, true> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                       static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::s_scalar, true>(o, n, ws, s);
    }
    case ADC_OP_LIN: {
        VjpLin<T, I::s_pair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                               static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
        return launch<decltype(o), I::s_pair, true>(o, n, ws, s);
    }
    case ADC_OP_SOP: {
        VjpSop<T, I::s_pair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                               static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
        return launch<decltype(o), I::s_pair, true>(o, n, ws, s);
    }
    case ADC_OP_MM2: {
        VjpMM2<T, I::s_mat> o{static_cast<const Mat2<T> *>(x), static_cast<const Mat2<T> *>(y),
                              static_cast<const Mat2<T> *>(ybar), static_cast<Mat2<T> *>(xbar), acc};
        return launch<decltype(o), I::s_mat, true>(o, n, ws, s);
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

// q x q matrix scans: the bulk-staged segment forms (scan_mmq.cuh; the API
// has checked that every array is 16-byte aligned) unless the engine hook
// asks for the register forms (1: per-tile, 2: ranges where the forward has
// one); hook 6 asks for the staged forms explicitly.
static bool mmq_staged_ok() { return g_scan_engine == 0 || g_scan_engine == 6; }
template <typename T, int Q>
static adc_status mmq_fwd_staged(int64_t n, const void *x, void *y, void *ws, cudaStream_t s) {
    constexpr int L = MMQStaged<T, Q, false>::seg;
    MMQStagedOp<T, Q, false> o{static_cast<const MatQ<T, Q> *>(x), static_cast<MatQ<T, Q> *>(y), n};
    return launch<decltype(o), 1, false>(o, (n + L - 1) / L, ws, s);
}
template <typename T, int Q>
static adc_status mmq_vjp_staged(int64_t n, const void *x, const void *y, const void *ybar, void *xbar, int acc,
                                 void *ws, cudaStream_t s) {
    using M = MatQ<T, Q>;
    constexpr int L = MMQStaged<T, Q, true>::seg;
    MMQStagedOp<T, Q, true> o{static_cast<const M *>(x), static_cast<const M *>(y), static_cast<const M *>(ybar),
                              static_cast<M *>(xbar), acc, n};
    return launch<decltype(o), 1, true>(o, (n + L - 1) / L, ws, s);
}

template <typename T>
static adc_status scan_fwd_t(adc_op op, int64_t n, const void *x, void *y, void *ws, cudaStream_t s) {
    using I = Items<T>;
    if ((op == ADC_OP_MIN || op == ADC_OP_MAX) && g_scan_engine == 4 && n > 0) {
        if (op == ADC_OP_MAX) {
            FwdSel<T, I::s_scalar, true> o;
            o.x = static_cast<const T *>(x);
            o.y = static_cast<T *>(y);
            return launch_staged<decltype(o), I::s_scalar, false>(o, n, ws, s);
        }
        FwdSel<T, I::s_scalar, false> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch_staged<decltype(o), I::s_scalar, false>(o, n, ws, s);
    }
    if (op == ADC_OP_MIN || op == ADC_OP_MAX) {
        if (op == ADC_OP_MAX) {
            FwdSel<T, I::scalar, true> o;
            o.x = static_cast<const T *>(x);
            o.y = static_cast<T *>(y);
            return launch<decltype(o), I::scalar, false>(o, n, ws, s);
        }
        FwdSel<T, I::scalar, false> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::scalar, false>(o, n, ws, s);
    }
    if ((op == ADC_OP_MM3 || op == ADC_OP_MM5) && mmq_staged_ok()) {
        if (op == ADC_OP_MM3) return mmq_fwd_staged<T, 3>(n, x, y, ws, s);
        return mmq_fwd_staged<T, 5>(n, x, y, ws, s);
    }
    if (op == ADC_OP_MM3) {  // the 3x3 forward holds a few matrices per thread without spilling
        FwdMMQ<T, 3, I::mat3> o;
        o.x = static_cast<const MatQ<T, 3> *>(x);
        o.y = static_cast<MatQ<T, 3> *>(y);
        return launch<decltype(o), I::mat3, false>(o, n, ws, s);
    }
    if (op == ADC_OP_MM5) {
        constexpr int L = SegLen<5>::value;
        SegFwdMMQ<T, 5, L> o{static_cast<const MatQ<T, 5> *>(x), static_cast<MatQ<T, 5> *>(y), n};
        return launch<decltype(o), 1, false>(o, (n + L - 1) / L, ws, s);
    }
    if (g_scan_engine == 5 && n > 0) return scan_fwd_items16<T>(op, n, x, y, ws, s);
    if (use_staged(n, 0)) {
        switch (op) {
        case ADC_OP_ADD: {
            FwdAdd<T, I::s_scalar> o;
            o.x = static_cast<const T *>(x);
            o.y = static_cast<T *>(y);
            return launch_staged<decltype(o), I::s_scalar, false>(o, n, ws, s);
        }
        case ADC_OP_MUL: {
            FwdMul<T, I::s_scalar> o;
            o.x = static_cast<const T *>(x);
            o.y = static_cast<T *>(y);
            return launch_staged<decltype(o), I::s_scalar, false>(o, n, ws, s);
        }
        case ADC_OP_LIN: {
            FwdLin<T, I::s_pair> o;
            o.x = static_cast<const Pair<T> *>(x);
            o.y = static_cast<Pair<T> *>(y);
            return launch_staged<decltype(o), I::s_pair, false>(o, n, ws, s);
        }
        case ADC_OP_MM2: {
            FwdMM2<T, I::s_mat> o;
            o.x = static_cast<const Mat2<T> *>(x);
            o.y = static_cast<Mat2<T> *>(y);
            return launch_staged<decltype(o), I::s_mat, false>(o, n, ws, s);
        }
        case ADC_OP_SOP: {
            FwdSop<T, I::s_pair> o;
            o.x = static_cast<const Pair<T> *>(x);
            o.y = static_cast<Pair<T> *>(y);
            return launch_staged<decltype(o), I::s_pair, false>(o, n, ws, s);
        }
        default: return ADC_ERR_UNSUPPORTED;
        }
    }
    switch (op) {
    case ADC_OP_ADD: {
        FwdAdd<T, I::scalar> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::scalar, false>(o, n, ws, s);
    }
    case ADC_OP_MUL: {
        FwdMul<T, I::scalar> o;
        o.x = static_cast<const T *>(x);
        o.y = static_cast<T *>(y);
        return launch<decltype(o), I::scalar, false>(o, n, ws, s);
    }
    case ADC_OP_LIN: {
        FwdLin<T, I::pair> o;
        o.x = static_cast<const Pair<T> *>(x);
        o.y = static_cast<Pair<T> *>(y);
        return launch<decltype(o), I::pair, false>(o, n, ws, s);
    }
    case ADC_OP_MM2: {
        FwdMM2<T, I::mat> o;
        o.x = static_cast<const Mat2<T> *>(x);
        o.y = static_cast<Mat2<T> *>(y);
        return launch<decltype(o), I::mat, false>(o, n, ws, s);
    }
    case ADC_OP_SOP: {
        FwdSop<T, I::pair> o;
        o.x = static_cast<const Pair<T> *>(x);
        o.y = static_cast<Pair<T> *>(y);
        return launch<decltype(o), I::pair, false>(o, n, ws, s);
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status scan_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *ws, cudaStream_t s) {
    return dt == ADC_F64 ? scan_fwd_t<double>(op, n, x, y, ws, s) : scan_fwd_t<float>(op, n, x, y, ws, s);
}

template <typename T>
static adc_status scan_vjp_t(adc_op op, int64_t n, const void *x, const void *y, const void *ybar, void *xbar,
                             int acc, void *ws, cudaStream_t s) {
    using I = Items<T>;
    if ((op == ADC_OP_MIN || op == ADC_OP_MAX) && g_scan_engine == 4 && n > 0) {
        if (op == ADC_OP_MAX) {
            VjpSel<T, I::s_scalar, true> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                           static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
            return launch_staged<decltype(o), I::s_scalar, true>(o, n, ws, s);
        }
        VjpSel<T, I::s_scalar, false> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                        static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch_staged<decltype(o), I::s_scalar, true>(o, n, ws, s);
    }
    if (op == ADC_OP_MIN || op == ADC_OP_MAX) {
        if (op == ADC_OP_MAX) {
            VjpSel<T, I::vscalar, true> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                          static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
            return launch<decltype(o), I::vscalar, true>(o, n, ws, s);
        }
        VjpSel<T, I::vscalar, false> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                       static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::vscalar, true>(o, n, ws, s);
    }
    if ((op == ADC_OP_MM3 || op == ADC_OP_MM5) && mmq_staged_ok()) {
        if (op == ADC_OP_MM3) return mmq_vjp_staged<T, 3>(n, x, y, ybar, xbar, acc, ws, s);
        return mmq_vjp_staged<T, 5>(n, x, y, ybar, xbar, acc, ws, s);
    }
    if (op == ADC_OP_MM3 || op == ADC_OP_MM5) {
        if (op == ADC_OP_MM3) {
            using M = MatQ<T, 3>;
            constexpr int L = SegLen<3>::value;
            SegVjpMMQ<T, 3, L> o{static_cast<const M *>(x), static_cast<const M *>(y), static_cast<const M *>(ybar),
                                 static_cast<M *>(xbar), acc, n};
            return launch<decltype(o), 1, true>(o, (n + L - 1) / L, ws, s);
        }
        using M = MatQ<T, 5>;
        constexpr int L = SegLen<5>::value;
        SegVjpMMQ<T, 5, L> o{static_cast<const M *>(x), static_cast<const M *>(y), static_cast<const M *>(ybar),
                             static_cast<M *>(xbar), acc, n};
        return launch<decltype(o), 1, true>(o, (n + L - 1) / L, ws, s);
    }
    if (g_scan_engine == 5 && n > 0) return scan_vjp_items16<T>(op, n, x, y, ybar, xbar, acc, ws, s);
    if (use_staged(n, 0)) {
        switch (op) {
        case ADC_OP_ADD: {
            VjpAdd<T, I::s_scalar> o{static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
            return launch_staged<decltype(o), I::s_scalar, true>(o, n, ws, s);
        }
        case ADC_OP_MUL: {
            VjpMul<T, I::s_scalar> o{static_cast<const T *>(x), static_cast<const T *>(y),
                                     static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
            return launch_staged<decltype(o), I::s_scalar, true>(o, n, ws, s);
        }
        case ADC_OP_LIN: {
            VjpLin<T, I::s_pair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                                   static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
            return launch_staged<decltype(o), I::s_pair, true>(o, n, ws, s);
        }
        case ADC_OP_MM2: {
            VjpMM2<T, I::s_mat> o{static_cast<const Mat2<T> *>(x), static_cast<const Mat2<T> *>(y),
                                  static_cast<const Mat2<T> *>(ybar), static_cast<Mat2<T> *>(xbar), acc};
            return launch_staged<decltype(o), I::s_mat, true>(o, n, ws, s);
        }
        case ADC_OP_SOP: {
            VjpSop<T, I::s_pair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                                   static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
            return launch_staged<decltype(o), I::s_pair, true>(o, n, ws, s);
        }
        default: return ADC_ERR_UNSUPPORTED;
        }
    }
    switch (op) {
    case ADC_OP_ADD: {
        VjpAdd<T, I::scalar> o{static_cast<const T *>(ybar), static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::scalar, true>(o, n, ws, s);
    }
    case ADC_OP_MUL: {
        VjpMul<T, I::vscalar> o{static_cast<const T *>(x), static_cast<const T *>(y), static_cast<const T *>(ybar),
                                static_cast<T *>(xbar), acc};
        return launch<decltype(o), I::vscalar, true>(o, n, ws, s);
    }
    case ADC_OP_LIN: {
        VjpLin<T, I::vpair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                              static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
        return launch<decltype(o), I::vpair, true>(o, n, ws, s);
    }
    case ADC_OP_MM2: {
        VjpMM2<T, I::vmat> o{static_cast<const Mat2<T> *>(x), static_cast<const Mat2<T> *>(y),
                             static_cast<const Mat2<T> *>(ybar), static_cast<Mat2<T> *>(xbar), acc};
        return launch<decltype(o), I::vmat, true>(o, n, ws, s);
    }
    case ADC_OP_SOP: {
        VjpSop<T, I::vpair> o{static_cast<const Pair<T> *>(x), static_cast<const Pair<T> *>(y),
                              static_cast<const Pair<T> *>(ybar), static_cast<Pair<T> *>(xbar), acc};
        return launch<decltype(o), I::vpair, true>(o, n, ws, s);
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status scan_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *ybar, void *xbar,
                    int accumulate, void *ws, cudaStream_t s) {
    return dt == ADC_F64 ? scan_vjp_t<double>(op, n, x, y, ybar, xbar, accumulate, ws, s)
                         : scan_vjp_t<float>(op, n, x, y, ybar, xbar, accumulate, ws, s);
}

}  // namespace adc
