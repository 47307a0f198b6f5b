// Vectorised operators: reduce, scan and reduce_by_index whose operator is
// map2 (.) over rows of d elements (Sec. 3.2, "Vectorized Operators", the
// Irwim rule; Sec. 5.3, the Iswim rule; the same interchange for
// reduce_by_index).  Each rule interchanges the outer combinator with the
// inner map, so that
//   reduce (map2 .) (replicate d e) x  ==  map (reduce . e) (transpose x)
//   scan   (map2 .) (replicate d e) x  ==  transpose (map (scan . e) (transpose x))
// and the vjp is taken of the right-hand side: d scalar combinators whose
// specialised rules (Sec. 3-5) apply column by column.  Reduce, scan and (for
// + and the fp32 min/max while the [m][d] table fits one block's shared
// memory) reduce_by_index run these column rules in direct form, on the rows
// where they lie; the other reduce_by_index cases transpose the [n][d] and
// [m][d] operands to [d][n] through shared-memory tiles, call the scalar
// kernels on the d contiguous columns and transpose the results back.
// Operators: ADD, MUL, MIN, MAX (scalar elements).
#include <atomic>
#include <cstring>
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"

namespace adc {

// dst[c * dld + r] = src[r * sld + c] for a rows x cols matrix (leading
// dimensions sld >= cols, dld >= rows), through 32 x 32 shared-memory tiles
// (one padding column: conflict-free on both sides).  A flat grid of tiles, so
// neither dimension is limited by the grid's y extent.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T *__restrict__ src, T *__restrict__ dst, const int64_t rows,
                                                    const int64_t cols, const int64_t sld, const int64_t dld,
                                                    const int64_t tiles_c) {
    __shared__ T tile[32][33];
    const int64_t t = blockIdx.x;
    const int64_t r0 = (t / tiles_c) * 32, c0 = (t % tiles_c) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int64_t r = r0 + ty + k, c = c0 + tx;
        if (r < rows && c < cols) tile[ty + k][tx] = src[r * sld + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int64_t c = c0 + ty + k, r = r0 + tx;
        if (r < rows && c < cols) dst[c * dld + r] = tile[tx][ty + k];
    }
}

static adc_status transpose_ld(adc_dtype dt, int64_t rows, int64_t cols, int64_t sld, int64_t dld, const void *src,
                               void *dst, cudaStream_t s) {
    if (rows == 0 || cols == 0) return ADC_OK;
    const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
    if (tr * tc > 0x7fffffffLL) return ADC_ERR_INVALID_ARG;
    if (dt == ADC_F64)
        k_transpose<double><<<(unsigned)(tr * tc), 256, 0, s>>>(static_cast<const double *>(src),
                                                               static_cast<double *>(dst), rows, cols, sld, dld, tc);
    else
        k_transpose<float><<<(unsigned)(tr * tc), 256, 0, s>>>(static_cast<const float *>(src),
                                                              static_cast<float *>(dst), rows, cols, sld, dld, tc);
    return check_launch();
}

adc_status transpose(adc_dtype dt, int64_t rows, int64_t cols, const void *src, void *dst, cudaStream_t s) {
    return transpose_ld(dt, rows, cols, cols, rows, src, dst, s);
}

// Columns of a [d][.] plane start every `ld` elements, ld rounded up to 64 so
// that every column starts on a 256-byte boundary: the scalar kernels load
// 16-byte words and require 16-byte-aligned arrays.
static int64_t plane_ld(int64_t len) { return (len + 63) / 64 * 64; }
// [len][d] row-major -> plane of d columns of stride plane_ld(len), and back
static adc_status to_plane(adc_dtype dt, int64_t len, int64_t d, const void *src, void *plane, cudaStream_t s) {
    return transpose_ld(dt, len, d, d, plane_ld(len), src, plane, s);
}
static adc_status from_plane(adc_dtype dt, int64_t len, int64_t d, const void *plane, void *dst, cudaStream_t s) {
    return transpose_ld(dt, d, len, plane_ld(len), d, plane, dst, s);
}

// OR the error words of the per-column calls into the call's own error word.
__global__ void k_gather_errors(unsigned *err, const char *cols, const int64_t d, const size_t stride) {
    unsigned e = 0;
    for (int64_t c = threadIdx.x; c < d; c += blockDim.x) e |= *reinterpret_cast<const unsigned *>(cols + c * stride);
    if (e) atomicOr(err, e);
}

// ------------------------------------------------------------- workspace --
// The transposed reduce_by_index: [header][2 n-planes [d][n]: vals^T,
// valsbar^T][3 m-planes [d][m]: hist0^T / histbar^T, hist^T, hist0bar^T]
// [d per-column scalar workspaces, each with its own header].
struct VLayout {
    size_t nplane[2], mplane[3], col, col_stride, bytes;
};

static size_t scalar_ws(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    switch (kind) {
    case ADC_REDUCE: return reduce_ws_bytes(op, dt, n);
    case ADC_SCAN: return scan_ws_bytes(op, dt, n);
    default: return hist_ws_bytes(op, dt, n, m);
    }
}
static size_t scalar_saved(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    switch (kind) {
    case ADC_REDUCE: return reduce_saved_bytes(op, dt, n);
    case ADC_SCAN: return 0;
    default: return hist_saved_bytes(op, dt, n, m);
    }
}

static VLayout vlayout(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    VLayout L{};
    const size_t e = dt == ADC_F64 ? 8 : 4;
    size_t o = kWsHeader;
    for (int i = 0; i < 2; ++i) {
        L.nplane[i] = o;
        o = align_up(o + (size_t)d * plane_ld(n) * e, 256);
    }
    for (int i = 0; i < 3; ++i) {
        L.mplane[i] = o;
        o = align_up(o + (size_t)d * plane_ld(m) * e, 256);
    }
    L.col = o;
    L.col_stride = align_up(scalar_ws(ADC_HIST, op, dt, n, m), 256);
    L.bytes = o + (size_t)d * L.col_stride;
    return L;
}

// The direct reduce_by_index (below) applies to + and the lifted fp32 min/max
// when one block's shared memory holds the whole [m][d] table; its workspace
// holds one partial table per block.
constexpr size_t kVHBudget = 200 * 1024;
static bool vhist_direct(adc_op op, adc_dtype dt, int64_t m, int64_t d) {
    const size_t cells = (size_t)m * (size_t)d;
    if (op == ADC_OP_ADD) return cells * (dt == ADC_F64 ? 8 : 4) <= kVHBudget;
    if (op == ADC_OP_MIN || op == ADC_OP_MAX) return dt == ADC_F32 && cells * 8 <= kVHBudget;
    return false;
}
static size_t vhist_direct_ws(int64_t m, int64_t d) {
    return kWsHeader + align_up((size_t)num_sms() * (size_t)m * (size_t)d * 8, 256);
}

// The direct scan (below) keeps two rows of column states (at most 16 bytes
// each) per unit (a warp, or a block when d > 32): the unit folds and their
// exclusive prefixes.
constexpr int kVScanMaxBlocksPerSM = 8;
static size_t vscan_states_bytes(int64_t d, size_t state_bytes = 16) {
    return align_up((size_t)num_sms() * kVScanMaxBlocksPerSM * 8 * (size_t)d * state_bytes, 256);
}
static size_t vscan_direct_ws(int64_t d) { return kWsHeader + 2 * vscan_states_bytes(d); }

size_t vws_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    if (scalar_ws(kind, op, dt, n, m) == 0) return 0;
    if (kind == ADC_REDUCE)  // the direct form: one partial row of column states per block
        return kWsHeader + align_up((size_t)num_sms() * 8 * (size_t)d * 16, 256);
    if (kind == ADC_HIST && vhist_direct(op, dt, m, d)) return vhist_direct_ws(m, d);
    if (kind == ADC_SCAN) return d == 1 ? scan_ws_bytes(op, dt, n) : vscan_direct_ws(d);
    return vlayout(op, dt, n, m, d).bytes;
}
size_t vsaved_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    if (kind == ADC_SCAN) return 16;
    const size_t one = scalar_saved(kind, op, dt, n, m);
    return one ? (size_t)d * align_up(one, 256) : 0;
}

// A column call gets its own workspace, whose header is zeroed as every entry
// point zeroes its own.
struct Cols {
    char *base;
    size_t stride;
    char *ws(int64_t c, cudaStream_t s, bool *ok) const {
        char *w = base + c * stride;
        *ok = cudaMemsetAsync(w, 0, kWsHeader, s) == cudaSuccess;
        return w;
    }
};

static adc_status finish(char *ws, const VLayout &L, int64_t d, cudaStream_t s) {
    k_gather_errors<<<1, 32, 0, s>>>(reinterpret_cast<unsigned *>(ws), ws + L.col, d, L.col_stride);
    return check_launch();
}

// -------------------------------------------------------------- combinators --
// ---------------------------------------------------- reduce, direct form --
// The Irwim rule makes the vectorised reduce d independent column reductions.
// Rather than transposing, the rows are read as they lie: the flat array of
// n*d scalars is strided by S, a multiple of d threads, so each thread meets
// a single column and folds it with that column's lifted operator (Fig. 3's
// zero count and product for *, Fig. 5's lowest-index min/max); each block
// then folds its threads column by column into one partial row, and one more
// kernel folds the partial rows in block order.  Column c's residuals go to
// saved + c * kVColSaved, laid out as the scalar reduce's.
constexpr int kVRedThreads = 256;
constexpr size_t kVColSaved = 256;  // bytes of residuals per column

template <typename T> struct VAdd {
    using State = T;
    __device__ State identity() const { return T(0); }
    __device__ State combine(State a, State b) const { return a + b; }
    __device__ State lift(T x, int64_t) const { return x; }
};
template <typename T> struct VMulS { T p; int32_t z; int32_t pad; };
template <typename T> struct VMul {
    using State = VMulS<T>;
    __device__ State identity() const { return {T(1), 0, 0}; }
    __device__ State combine(const State &a, const State &b) const { return {a.p * b.p, a.z + b.z, 0}; }
    __device__ State lift(T x, int64_t) const { return x == T(0) ? State{T(1), 1, 0} : State{x, 0, 0}; }
};
template <typename T> struct VSelS { T v; int32_t i; int32_t pad; };
template <typename T, bool MAX> struct VSel {
    using State = VSelS<T>;
    int32_t none;  // the index of "no element" (n)
    __device__ State identity() const { return {MAX ? -Num<T>::inf() : Num<T>::inf(), none, 0}; }
    __device__ State combine(const State &a, const State &b) const {
        if (MAX ? (a.v > b.v) : (a.v < b.v)) return a;
        if (MAX ? (b.v > a.v) : (b.v < a.v)) return b;
        return a.i <= b.i ? a : b;  // equal values: the smaller index
    }
    __device__ State lift(T x, int64_t i) const { return {x, (int32_t)i, 0}; }
};

// Active threads of the grid: the largest multiple of d.
__device__ __forceinline__ int64_t vred_active(int64_t d) {
    return ((int64_t)gridDim.x * blockDim.x / d) * d;
}

template <class Op, typename T>
__global__ void __launch_bounds__(kVRedThreads)
k_vred_rows(const Op op, const T *__restrict__ x, const int64_t n, const int64_t d,
            typename Op::State *__restrict__ part) {
    using S = typename Op::State;
    __shared__ S s_st[kVRedThreads];
    const int64_t S_ = vred_active(d);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    S a = op.identity();
    if (gt < S_) {
        // eight loads in flight per thread before they are folded in order
        constexpr int U = 8;
        const int64_t total = n * d, rstep = S_ / d;
        int64_t row = gt / d, f = gt;
        for (; f + (U - 1) * S_ < total; f += U * S_, row += U * rstep) {
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldcs(x + f + u * S_);
#pragma unroll
            for (int u = 0; u < U; ++u) a = op.combine(a, op.lift(v[u], row + u * rstep));
        }
        for (; f < total; f += S_, row += rstep) a = op.combine(a, op.lift(__ldcs(x + f), row));
    }
    s_st[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < d) {
        // this block's threads of column c = (base + t) mod d, in thread order
        const int64_t base = (int64_t)blockIdx.x * blockDim.x;
        const int64_t c = (base + threadIdx.x) % d;
        S r = op.identity();
        for (int t = threadIdx.x; t < kVRedThreads && base + t < S_; t += (int)d) r = op.combine(r, s_st[t]);
        part[(int64_t)blockIdx.x * d + c] = r;
    }
}

// Column c: fold the G partial rows in block order, write y[c] and the residuals.
template <typename T> __device__ __forceinline__ void vred_out(const T &r, T *y, char *, int64_t c) { y[c] = r; }
template <typename T> __device__ __forceinline__ void vred_out(const VMulS<T> &r, T *y, char *sv, int64_t c) {
    y[c] = r.z > 0 ? T(0) : r.p;
    *reinterpret_cast<int32_t *>(sv + c * kVColSaved) = r.z;
    *reinterpret_cast<T *>(sv + c * kVColSaved + 8) = r.p;
}
template <typename T> __device__ __forceinline__ void vred_out(const VSelS<T> &r, T *y, char *sv, int64_t c) {
    y[c] = r.v;
    *reinterpret_cast<int32_t *>(sv + c * kVColSaved) = r.i;
}

template <class Op, typename T>
__global__ void k_vred_final(const Op op, const typename Op::State *__restrict__ part, const int G, const int64_t d,
                             T *__restrict__ y, char *__restrict__ saved) {
    for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
        typename Op::State r = op.identity();
        for (int g = 0; g < G; ++g) r = op.combine(r, part[(int64_t)g * d + c]);
        vred_out(r, y, saved, c);
    }
}

// vjp, elementwise with the same fixed-column striding: xbar[i][c] (+)= the
// scalar rule of column c (Sec. 3.2: broadcast for +; Fig. 3's three cases for
// *; Fig. 5's selected index for min/max).
template <typename T, int OPK>  // OPK: 0 add, 1 mul, 2 min/max
__global__ void __launch_bounds__(kVRedThreads)
k_vred_vjp(const T *__restrict__ x, const T *__restrict__ ybar, const char *__restrict__ saved, T *__restrict__ xbar,
           const int64_t n, const int64_t d, const int accumulate) {
    const int64_t S_ = vred_active(d);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= S_) return;
    const int64_t c = gt % d, total = n * d, rstep = S_ / d;
    const T yb = ybar[c];
    int32_t k = 0;
    T p = T(0);
    if (OPK == 1) {
        k = *reinterpret_cast<const int32_t *>(saved + c * kVColSaved);
        p = *reinterpret_cast<const T *>(saved + c * kVColSaved + 8);
    } else if (OPK == 2) {
        k = *reinterpret_cast<const int32_t *>(saved + c * kVColSaved);
    }
    auto grad = [&](T a, int64_t row) -> T {
        if (OPK == 0) return yb;
        if (OPK == 1) return k == 0 ? div_or_zero(p, a) * yb : ((k == 1 && a == T(0)) ? p * yb : T(0));
        return row == k ? yb : T(0);
    };
    // eight elements per thread and step, their loads issued first
    constexpr int U = 8;
    int64_t row = gt / d, f = gt;
    for (; f + (U - 1) * S_ < total; f += U * S_, row += U * rstep) {
        T a[U], o[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = OPK == 1 ? __ldcs(x + f + u * S_) : T(0);
            o[u] = accumulate ? xbar[f + u * S_] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const T g = grad(a[u], row + u * rstep);
            __stcs(xbar + f + u * S_, accumulate ? o[u] + g : g);
        }
    }
    for (; f < total; f += S_, row += rstep) {
        const T g = grad(OPK == 1 ? __ldcs(x + f) : T(0), row);
        xbar[f] = accumulate ? xbar[f] + g : g;
    }
}

static int vred_grid() { return num_sms() * 8; }

template <typename T>
static adc_status vred_fwd_t(adc_op op, int64_t n, int64_t d, const T *x, T *y, char *saved, char *ws,
                             cudaStream_t s) {
    const int G = vred_grid();
    void *part = ws + kWsHeader;
    switch (op) {
    case ADC_OP_ADD: {
        VAdd<T> o;
        k_vred_rows<<<G, kVRedThreads, 0, s>>>(o, x, n, d, static_cast<T *>(part));
        k_vred_final<<<1, 64, 0, s>>>(o, static_cast<const T *>(part), G, d, y, saved);
        break;
    }
    case ADC_OP_MUL: {
        VMul<T> o;
        k_vred_rows<<<G, kVRedThreads, 0, s>>>(o, x, n, d, static_cast<VMulS<T> *>(part));
        k_vred_final<<<1, 64, 0, s>>>(o, static_cast<const VMulS<T> *>(part), G, d, y, saved);
        break;
    }
    case ADC_OP_MIN: {
        VSel<T, false> o{(int32_t)n};
        k_vred_rows<<<G, kVRedThreads, 0, s>>>(o, x, n, d, static_cast<VSelS<T> *>(part));
        k_vred_final<<<1, 64, 0, s>>>(o, static_cast<const VSelS<T> *>(part), G, d, y, saved);
        break;
    }
    case ADC_OP_MAX: {
        VSel<T, true> o{(int32_t)n};
        k_vred_rows<<<G, kVRedThreads, 0, s>>>(o, x, n, d, static_cast<VSelS<T> *>(part));
        k_vred_final<<<1, 64, 0, s>>>(o, static_cast<const VSelS<T> *>(part), G, d, y, saved);
        break;
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
    return check_launch();
}

adc_status vreduce_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *saved, void *ws,
                       cudaStream_t s) {
    char *sv = static_cast<char *>(saved), *w = static_cast<char *>(ws);
    if (dt == ADC_F64)
        return vred_fwd_t<double>(op, n, d, static_cast<const double *>(x), static_cast<double *>(y), sv, w, s);
    return vred_fwd_t<float>(op, n, d, static_cast<const float *>(x), static_cast<float *>(y), sv, w, s);
}

template <typename T>
static adc_status vred_vjp_t(adc_op op, int64_t n, int64_t d, const T *x, const char *saved, const T *ybar, T *xbar,
                             int acc, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    const int G = vred_grid();
    switch (op) {
    case ADC_OP_ADD: k_vred_vjp<T, 0><<<G, kVRedThreads, 0, s>>>(x, ybar, saved, xbar, n, d, acc); break;
    case ADC_OP_MUL: k_vred_vjp<T, 1><<<G, kVRedThreads, 0, s>>>(x, ybar, saved, xbar, n, d, acc); break;
    case ADC_OP_MIN:
    case ADC_OP_MAX: k_vred_vjp<T, 2><<<G, kVRedThreads, 0, s>>>(x, ybar, saved, xbar, n, d, acc); break;
    default: return ADC_ERR_UNSUPPORTED;
    }
    return check_launch();
}

adc_status vreduce_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *saved,
                       const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s) {
    (void)y;
    (void)ws;
    const char *sv = static_cast<const char *>(saved);
    if (dt == ADC_F64)
        return vred_vjp_t<double>(op, n, d, static_cast<const double *>(x), sv, static_cast<const double *>(ybar),
                                  static_cast<double *>(xbar), accumulate, s);
    return vred_vjp_t<float>(op, n, d, static_cast<const float *>(x), sv, static_cast<const float *>(ybar),
                             static_cast<float *>(xbar), accumulate, s);
}

// ------------------------------------------------------ scan, direct form --
// The Iswim rule makes the vectorised scan d independent column scans (and
// its vjp d column vjps).  Rather than transposing, the rows are scanned where
// they lie, in three launches with no inter-unit waits:
//   1. unit u folds its contiguous range of rows into one state per column;
//   2. per column, the U unit states become exclusive prefixes;
//   3. unit u rescans its range from its prefixes, tile by tile.
// A unit is a warp when d <= 32, else a block of 256 threads.  Its threads
// t < P*d (P = floor(threads / d) parts) own column c = t mod d and part
// p = t / d; a tile is P*RP consecutive rows, part p its RP rows from p*RP
// on, held in registers.  A warp's load then covers whole row segments
// (32 / d parts of d columns), and consecutive rows follow in its next load.
// The tile's part states are combined across parts by shuffles (warp units)
// or a Hillis-Steele scan in shared memory (block units).  Reverse scans
// (the vjps, Sec. 5) run in logical order L = n-1-i.  Traffic: the inputs
// twice, the outputs once.
// An op gives identity(), combine(earlier, later), state(i, f, aux) -- the
// element state of row i at flat offset f = i*d + c, with what its store
// needs in aux -- store(f, inclusive, aux), kRev (a reverse scan) and
// kHaloChunk (its rescan loads a whole chunk through its own vscan_chunk).
constexpr int kVScanThreads = 256;

template <typename T> struct VAff { T v, c; };  // lambda -> v + c * lambda

template <typename T, int K> struct VScanFwd {  // K: 0 add, 1 mul, 2 min, 3 max
    using S = T;
    struct Aux {};
    static constexpr bool kRev = false, kHaloChunk = false;
    const T *__restrict__ x;
    T *__restrict__ y;
    int64_t d;
    __device__ S identity() const {
        return K == 0 ? T(0) : K == 1 ? T(1) : K == 2 ? Num<T>::inf() : -Num<T>::inf();
    }
    __device__ S combine(const S &a, const S &b) const {
        if (K == 0) return a + b;
        if (K == 1) return a * b;
        return (K == 3 ? (b > a) : (b < a)) ? b : a;  // the earlier value wins ties
    }
    __device__ S state(int64_t, int64_t f, Aux &) const { return __ldg(x + f); }
    __device__ void store(int64_t f, const S &inc, const Aux &) const { y[f] = inc; }
    // The state every column's scan starts from.  For min / max the scan's
    // loop starts from y_0 = x_0, and a NaN never loses as the earlier operand,
    // so a NaN in row 0 makes its whole column NaN: starting the column from
    // that NaN (instead of the identity, which a NaN cannot beat) gives it.
    __device__ S initial(int64_t c) const {
        if (K < 2) return identity();
        const T x0 = __ldg(x + c);
        return x0 != x0 ? x0 : identity();
    }
};

// The state column c's scan starts from: the op's initial(c) where it has one.
template <class Op> __device__ __forceinline__ typename Op::S vscan_initial(const Op &op, int64_t c, long) {
    return op.identity();
}
template <class Op>
__device__ __forceinline__ auto vscan_initial(const Op &op, int64_t c, int) -> decltype(op.initial(c)) {
    return op.initial(c);
}

// + scan vjp: xbar_i = sum_{j >= i} ybar_j (a reverse + scan).
template <typename T> struct VScanVjpAdd {
    using S = T;
    struct Aux { T old; };
    static constexpr bool kRev = true, kHaloChunk = false;
    const T *__restrict__ ybar;
    T *__restrict__ xbar;
    int64_t d;
    int accumulate;
    __device__ S identity() const { return T(0); }
    __device__ S combine(const S &a, const S &b) const { return a + b; }
    __device__ S state(int64_t, int64_t f, Aux &a) const {
        a.old = accumulate ? xbar[f] : T(0);
        return __ldg(ybar + f);
    }
    __device__ void store(int64_t f, const S &inc, const Aux &a) const { xbar[f] = accumulate ? a.old + inc : inc; }
};

// * and min / max scan vjps: the recurrence lambda_i = ybar_i + J_{i+1}
// lambda_{i+1} as a reverse scan of affine maps (Sec. 5.1), with
// J_{i+1} = x_{i+1} for * and the 0/1 "y_i selected" for min / max; then
// xbar_i = y_{i-1} lambda_i (*) or [x_i selected at step i] lambda_i.  The
// min / max selections are read off y alone: x_i wins step i exactly when
// y_i differs from y_{i-1} (a strict win changes the value, a loss or a tie
// keeps it; two NaNs count as equal), so x is not read.
template <typename T> __device__ __forceinline__ bool vsame(T a, T b) { return a == b || (a != a && b != b); }

template <typename T, int K> struct VScanVjpAff {  // K: 1 mul, 2 min, 3 max
    using S = VAff<T>;
    struct Aux { T g, old; };
    static constexpr bool kRev = true;
    // fp32 min / max: the rescan loads through vscan_chunk (fp64 would hold
    // too many registers for it)
    static constexpr bool kHaloChunk = K != 1 && sizeof(T) == 4;
    const T *__restrict__ x, *__restrict__ y, *__restrict__ ybar;
    T *__restrict__ xbar;
    int64_t n, d;
    int accumulate;
    __device__ S identity() const { return {T(0), T(1)}; }
    __device__ S combine(const S &acc, const S &e) const { return {e.v + e.c * acc.v, e.c * acc.c}; }
    __device__ S state(int64_t i, int64_t f, Aux &a) const {
        a.old = accumulate ? xbar[f] : T(0);
        if (K == 1) {
            a.g = i > 0 ? __ldg(y + f - d) : T(1);
            return {__ldg(ybar + f), i + 1 < n ? __ldg(x + f + d) : T(1)};
        }
        const T yi = __ldg(y + f);
        a.g = (i == 0 || !vsame(yi, __ldg(y + f - d))) ? T(1) : T(0);
        return {__ldg(ybar + f), (i + 1 < n && !vsame(__ldg(y + f + d), yi)) ? T(0) : T(1)};
    }
    __device__ void store(int64_t f, const S &inc, const Aux &a) const {
        const T g = a.g * inc.v;
        xbar[f] = accumulate ? a.old + g : g;
    }
};

// ---- rows of k equal multi-word elements (tuple scans whose blocks are all
// lin, all sumOfProd or all 2x2 matrix products): the direct form above over
// the k element columns of each row, with the element operator's state.  The
// formulas are the scalar scans' (Sec. 5.3.2-5.3.4 and Fig. 7's general rule
// for sumOfProd), written per element: x_{i+1} and y_{i-1} are the elements
// one row after and before (f + d, f - d).
template <typename E> __device__ __forceinline__ E ld_elem(const E *p) {
    static_assert(sizeof(E) % 8 == 0 && sizeof(E) <= 32, "8-, 16- or 32-byte elements");
    E e;
    if constexpr (sizeof(E) == 8) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        memcpy(&e, &v, 8);
    } else {
        float4 v[sizeof(E) / 16];
#pragma unroll
        for (int q = 0; q < (int)(sizeof(E) / 16); ++q) v[q] = __ldg(reinterpret_cast<const float4 *>(p) + q);
        memcpy(&e, v, sizeof(E));
    }
    return e;
}
template <typename E> __device__ __forceinline__ void st_elem(E *p, const E &e) {
    if constexpr (sizeof(E) == 8) {
        float2 v;
        memcpy(&v, &e, 8);
        *reinterpret_cast<float2 *>(p) = v;
    } else {
        float4 v[sizeof(E) / 16];
        memcpy(v, &e, sizeof(E));
#pragma unroll
        for (int q = 0; q < (int)(sizeof(E) / 16); ++q) reinterpret_cast<float4 *>(p)[q] = v[q];
    }
}

template <typename T> struct ElemLin {  // linFnComp: (b, c): x -> b + c x
    using E = Pair<T>;
    static __device__ E identity() { return {T(0), T(1)}; }
    static __device__ E combine(const E &a, const E &b) { return {b.b + b.c * a.b, b.c * a.c}; }
};
template <typename T> struct ElemSop {  // sumOfProd (Fig. 8)
    using E = Pair<T>;
    static __device__ E identity() { return {T(0), T(0)}; }
    static __device__ E combine(const E &a, const E &b) { return {a.b + b.b + a.c * b.c, a.c + b.c}; }
};
template <typename T> struct ElemMM2 {  // 2x2 matrix product
    using E = Mat2<T>;
    static __device__ E identity() { return mat_eye<T>(); }
    static __device__ E combine(const E &a, const E &b) { return mat_mul(a, b); }
};

template <typename T, class EO> struct VScanFwdE {
    using E = typename EO::E;
    using S = E;
    struct Aux {};
    static constexpr bool kRev = false, kHaloChunk = false;
    const E *__restrict__ x;
    E *__restrict__ y;
    int64_t d;
    __device__ S identity() const { return EO::identity(); }
    __device__ S combine(const S &a, const S &b) const { return EO::combine(a, b); }
    __device__ S state(int64_t, int64_t f, Aux &) const { return ld_elem(x + f); }
    __device__ void store(int64_t f, const S &inc, const Aux &) const { st_elem(y + f, inc); }
};

// lin vjp: lambda_i = ybar_i + c(x_{i+1}) lambda_i+1 (a 2-vector), xbar_i =
// (lambda.b, lambda.b b(y_{i-1}) + lambda.c c(y_{i-1})), y_{-1} = (0, 1).
template <typename T> struct VAffP { T vb, vc, c; };
template <typename T> struct VScanVjpLinE {
    using E = Pair<T>;
    using S = VAffP<T>;
    struct Aux { E yprev, old; };
    static constexpr bool kRev = true, kHaloChunk = false;
    const E *__restrict__ x, *__restrict__ y, *__restrict__ ybar;
    E *__restrict__ xbar;
    int64_t n, d;
    int accumulate;
    __device__ S identity() const { return {T(0), T(0), T(1)}; }
    __device__ S combine(const S &acc, const S &e) const {
        return {e.vb + e.c * acc.vb, e.vc + e.c * acc.vc, e.c * acc.c};
    }
    __device__ S state(int64_t i, int64_t f, Aux &a) const {
        a.old = accumulate ? xbar[f] : E{T(0), T(0)};
        a.yprev = i > 0 ? ld_elem(y + f - d) : E{T(0), T(1)};
        const E yb = ld_elem(ybar + f);
        return {yb.b, yb.c, i + 1 < n ? ld_elem(x + f + d).c : T(1)};
    }
    __device__ void store(int64_t f, const S &inc, const Aux &a) const {
        const T gb = inc.vb, gc = gb * a.yprev.b + inc.vc * a.yprev.c;
        st_elem(xbar + f, accumulate ? E{a.old.b + gb, a.old.c + gc} : E{gb, gc});
    }
};

// sumOfProd vjp by the general rule (unit upper-triangular Jacobians: the
// composed map is (vp, vs, sig)); xbar_i = (lambda.p, s(y_{i-1}) lambda.p + lambda.s).
template <typename T> struct VAffU { T vp, vs, sig; };
template <typename T> struct VScanVjpSopE {
    using E = Pair<T>;
    using S = VAffU<T>;
    struct Aux { T sprev; E old; };
    static constexpr bool kRev = true, kHaloChunk = false;
    const E *__restrict__ x, *__restrict__ y, *__restrict__ ybar;
    E *__restrict__ xbar;
    int64_t n, d;
    int accumulate;
    __device__ S identity() const { return {T(0), T(0), T(0)}; }
    __device__ S combine(const S &acc, const S &e) const {
        return {e.vp + acc.vp, e.vs + e.sig * acc.vp + acc.vs, acc.sig + e.sig};
    }
    __device__ S state(int64_t i, int64_t f, Aux &a) const {
        a.old = accumulate ? xbar[f] : E{T(0), T(0)};
        a.sprev = i > 0 ? ld_elem(y + f - d).c : T(0);
        const E yb = ld_elem(ybar + f);
        return {yb.b, yb.c, i + 1 < n ? ld_elem(x + f + d).c : T(0)};
    }
    __device__ void store(int64_t f, const S &inc, const Aux &a) const {
        const T gp = inc.vp, gs = a.sprev * inc.vp + inc.vs;
        st_elem(xbar + f, accumulate ? E{a.old.b + gp, a.old.c + gs} : E{gp, gs});
    }
};

// 2x2 vjp: f_i(L) = Ybar_i + L M_{i+1}^T, Mbar_i = P_{i-1}^T lambda_i, P_{-1} = I.
template <typename T> struct VAffM { Mat2<T> v, c; };
template <typename T> struct VScanVjpMM2E {
    using E = Mat2<T>;
    using S = VAffM<T>;
    struct Aux { E yprev, old; };
    static constexpr bool kRev = true, kHaloChunk = false;
    const E *__restrict__ x, *__restrict__ y, *__restrict__ ybar;
    E *__restrict__ xbar;
    int64_t n, d;
    int accumulate;
    __device__ S identity() const { return {mat_zero<T>(), mat_eye<T>()}; }
    __device__ S combine(const S &acc, const S &e) const {
        return {mat_add(e.v, mat_mul(acc.v, e.c)), mat_mul(acc.c, e.c)};
    }
    __device__ S state(int64_t i, int64_t f, Aux &a) const {
        a.old = accumulate ? ld_elem(xbar + f) : mat_zero<T>();
        a.yprev = i > 0 ? ld_elem(y + f - d) : mat_eye<T>();
        return {ld_elem(ybar + f), i + 1 < n ? mat_t(ld_elem(x + f + d)) : mat_eye<T>()};
    }
    __device__ void store(int64_t f, const S &inc, const Aux &a) const {
        const E g = mat_mul(mat_t(a.yprev), inc.v);
        st_elem(xbar + f, accumulate ? mat_add(a.old, g) : g);
    }
};

// Block b's logical rows [l0, l1): the G blocks split n as evenly as possible.
__device__ __forceinline__ void vscan_range(int64_t n, int64_t b, int64_t G, int64_t *l0, int64_t *l1) {
    const int64_t per = n / G, extra = n % G;
    *l0 = b * per + (b < extra ? b : extra);
    *l1 = *l0 + per + (b < extra ? 1 : 0);
}

template <class Op> __device__ __forceinline__ int64_t vscan_phys(int64_t L, int64_t n) {
    return Op::kRev ? n - 1 - L : L;
}

// A rescan chunk: column c at logical rows lp .. lp+RP-1, none at or beyond
// hi.  Offsets step by -d / +d from the chunk's first row; whole chunks (the
// common case) run without per-element bounds tests.
template <class Op, int RP>
__device__ __forceinline__ void vscan_load(const Op &op, int64_t lp, int64_t hi, int64_t n, int64_t d, int64_t c,
                                           bool active, typename Op::S (&st)[RP], typename Op::Aux (&aux)[RP]) {
    const int64_t i0 = vscan_phys<Op>(lp, n), f0 = i0 * d + c, step = Op::kRev ? -d : d;
    if (active && lp + RP <= hi) {
#pragma unroll
        for (int k = 0; k < RP; ++k) st[k] = op.state(Op::kRev ? i0 - k : i0 + k, f0 + k * step, aux[k]);
    } else {
#pragma unroll
        for (int k = 0; k < RP; ++k)
            st[k] = (active && lp + k < hi) ? op.state(Op::kRev ? i0 - k : i0 + k, f0 + k * step, aux[k])
                                            : op.identity();
    }
}
// ... and its stores of the inclusive values, r the chunk's incoming prefix.
template <class Op, int RP>
__device__ __forceinline__ void vscan_store(const Op &op, int64_t lp, int64_t hi, int64_t n, int64_t d, int64_t c,
                                            bool active, typename Op::S r, const typename Op::S (&st)[RP],
                                            const typename Op::Aux (&aux)[RP]) {
    const int64_t f0 = vscan_phys<Op>(lp, n) * d + c, step = Op::kRev ? -d : d;
    if (active && lp + RP <= hi) {
#pragma unroll
        for (int k = 0; k < RP; ++k) {
            r = op.combine(r, st[k]);
            op.store(f0 + k * step, r, aux[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < RP; ++k) {
            if (active && lp + k < hi) {
                r = op.combine(r, st[k]);
                op.store(f0 + k * step, r, aux[k]);
            }
        }
    }
}

// The rescan of the min / max scan vjps: they read y at the element and at
// both neighbours; here y is loaded once per row of the chunk (logical rows
// lp .. lp+RP-1, none at or beyond hi) plus a halo row on each side, and the
// neighbours are taken from registers.
template <typename T, int K, int RP>
__device__ __forceinline__ void vscan_chunk(const VScanVjpAff<T, K> &op, int64_t lp, int64_t hi, int64_t n, int64_t c,
                                            bool active, VAff<T> (&st)[RP],
                                            typename VScanVjpAff<T, K>::Aux (&aux)[RP]) {
    static_assert(K == 2 || K == 3, "min / max only");
    const int64_t d = op.d;
    int64_t cnt = hi - lp < RP ? hi - lp : RP;
    if (!active || cnt < 0) cnt = 0;  // nothing is loaded then, not even a halo
    const int64_t i0 = n - 1 - lp;   // physical rows i0, i0-1, ..., i0-cnt+1 (all >= 0)
    // Y[j] = y[i0 + 1 - j]: Y[0] the halo y_{i0+1}, Y[cnt+1] the halo y_{i0-cnt}
    T Y[RP + 2], yb[RP], old[RP];
#pragma unroll
    for (int j = 0; j < RP + 2; ++j) {
        const int64_t iy = i0 + 1 - j;
        Y[j] = (cnt > 0 && j <= cnt + 1 && iy >= 0 && iy < n) ? __ldg(op.y + iy * d + c) : T(0);
    }
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        yb[k] = k < cnt ? __ldg(op.ybar + (i0 - k) * d + c) : T(0);
        old[k] = (k < cnt && op.accumulate) ? op.xbar[(i0 - k) * d + c] : T(0);
    }
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const int64_t i = i0 - k;  // y_{i+1} = Y[k], y_i = Y[k+1], y_{i-1} = Y[k+2]
        aux[k].old = old[k];
        if (k >= cnt) {
            st[k] = op.identity();
            aux[k].g = T(0);
        } else {
            aux[k].g = (i == 0 || !vsame(Y[k + 1], Y[k + 2])) ? T(1) : T(0);
            st[k] = {yb[k], (i + 1 < n && !vsame(Y[k], Y[k + 1])) ? T(0) : T(1)};
        }
    }
}

template <class Op, int RP>
__global__ void __launch_bounds__(kVScanThreads)
k_vscan_fold(const Op op, const int64_t n, const int64_t d, typename Op::S *__restrict__ agg) {
    using S = typename Op::S;
    __shared__ S s_part[kVScanThreads];
    const int t = threadIdx.x;
    const int P = kVScanThreads / (int)d;
    const bool active = t < P * (int)d;
    const int64_t c = t % d, p = t / d;
    int64_t l0, l1;
    vscan_range(n, blockIdx.x, gridDim.x, &l0, &l1);
    S a = op.identity();
    if (active) {
        // part p folds a contiguous piece of the range, RP loads in flight
        const int64_t per = (l1 - l0 + P - 1) / P;
        const int64_t lo = l0 + p * per, hi = lo + per < l1 ? lo + per : l1;
        const int64_t step = Op::kRev ? -d : d;
        int64_t L = lo;
        for (; L + RP <= hi; L += RP) {
            const int64_t i0 = vscan_phys<Op>(L, n), f0 = i0 * d + c;
            S v[RP];
            typename Op::Aux aux;
#pragma unroll
            for (int k = 0; k < RP; ++k) v[k] = op.state(Op::kRev ? i0 - k : i0 + k, f0 + k * step, aux);
#pragma unroll
            for (int k = 0; k < RP; ++k) a = op.combine(a, v[k]);
        }
        for (; L < hi; ++L) {
            typename Op::Aux aux;
            const int64_t i = vscan_phys<Op>(L, n);
            a = op.combine(a, op.state(i, i * d + c, aux));
        }
    }
    s_part[t] = a;
    __syncthreads();
    if (t < d) {
        S r = op.identity();
        for (int q = 0; q < P; ++q) r = op.combine(r, s_part[q * d + t]);
        agg[(int64_t)blockIdx.x * d + t] = r;
    }
}

// One warp per column: the exclusive prefixes of the G block states, in order.
template <class Op>
__global__ void k_vscan_prefix(const Op op, const typename Op::S *__restrict__ agg, const int G, const int64_t d,
                               typename Op::S *__restrict__ pre) {
    using S = typename Op::S;
    const int lane = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int per = (G + kWarp - 1) / kWarp;
    const int g0 = lane * per, g1 = g0 + per < G ? g0 + per : G;
    S v = op.identity();
    for (int g = g0; g < g1; ++g) v = op.combine(v, agg[(int64_t)g * d + c]);
    const S inc = warp_inclusive_scan(op, v);
    S run = shfl_up(inc, 1);
    if (lane == 0) run = op.identity();
    run = op.combine(vscan_initial(op, c, 0), run);
    for (int g = g0; g < g1; ++g) {
        pre[(int64_t)g * d + c] = run;
        run = op.combine(run, agg[(int64_t)g * d + c]);
    }
}

template <class Op, int RP>
__global__ void __launch_bounds__(kVScanThreads)
k_vscan_apply(const Op op, const int64_t n, const int64_t d, const typename Op::S *__restrict__ pre) {
    using S = typename Op::S;
    __shared__ S s_part[kVScanThreads];
    const int t = threadIdx.x;
    const int P = kVScanThreads / (int)d;
    const bool active = t < P * (int)d;
    const int64_t c = t % d, p = t / d;
    int64_t l0, l1;
    vscan_range(n, blockIdx.x, gridDim.x, &l0, &l1);
    S carry = active ? pre[(int64_t)blockIdx.x * d + c] : op.identity();
    for (int64_t lt = l0; lt < l1; lt += (int64_t)P * RP) {
        const int64_t lp = lt + p * RP;
        S st[RP];
        typename Op::Aux aux[RP];
        if constexpr (Op::kHaloChunk)
            vscan_chunk(op, lp, l1, n, c, active, st, aux);
        else
            vscan_load(op, lp, l1, n, d, c, active, st, aux);
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < RP; ++k) a = op.combine(a, st[k]);
        s_part[t] = a;
        __syncthreads();
        // inclusive scan over the parts of each column (Hillis-Steele)
        for (int sh = 1; sh < P; sh <<= 1) {
            const bool h = active && p >= sh;
            S o = op.identity();
            if (h) o = s_part[t - sh * d];
            __syncthreads();
            if (h) {
                a = op.combine(o, a);
                s_part[t] = a;
            }
            __syncthreads();
        }
        S r = (active && p > 0) ? op.combine(carry, s_part[t - d]) : carry;
        const S tile = active ? s_part[(P - 1) * d + c] : op.identity();
        vscan_store(op, lp, l1, n, d, c, active, r, st, aux);
        carry = op.combine(carry, tile);
        __syncthreads();  // s_part is rewritten by the next tile
    }
}

// ---- warp form, d <= 32: every warp is a unit of its own, with a range of
// rows, its parts (P = floor(32 / d)) and their cross-part scan in one warp
// (shuffles by d, 2d, 4d, ...), so no block barrier is ever waited on.
constexpr int kVScanWarps = kVScanThreads / kWarp;
static_assert(kVScanWarps <= 8, "the workspace holds 8 units per resident block");

// Column c's inclusive scan over the warp's parts: lane p*d + c combines the
// states of lanes c, d + c, ..., p*d + c in order (lanes >= P*d never feed
// an active lane: shuffles only read lower lanes).
template <class Op>
__device__ __forceinline__ typename Op::S warp_parts_scan(const Op &op, typename Op::S a, int d, int P) {
    const int lane = threadIdx.x & 31;
    for (int sh = d; sh < P * d; sh <<= 1) {
        const typename Op::S o = shfl_up(a, sh);
        if (lane >= sh) a = op.combine(o, a);
    }
    return a;
}

template <class Op, int RP>
__global__ void __launch_bounds__(kVScanThreads)
k_vscan_wfold(const Op op, const int64_t n, const int64_t d, const int64_t U, typename Op::S *__restrict__ agg) {
    using S = typename Op::S;
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kVScanWarps + (threadIdx.x >> 5);
    if (u >= U) return;  // whole warps
    const int P = kWarp / (int)d;
    const bool active = lane < P * (int)d;
    const int64_t c = lane % d, p = lane / d;
    int64_t l0, l1;
    vscan_range(n, u, U, &l0, &l1);
    S a = op.identity();
    if (active) {
        // part p folds a contiguous piece of the unit, RP loads in flight
        const int64_t per = (l1 - l0 + P - 1) / P;
        const int64_t lo = l0 + p * per, hi = lo + per < l1 ? lo + per : l1;
        const int64_t step = Op::kRev ? -d : d;
        int64_t L = lo;
        for (; L + RP <= hi; L += RP) {
            const int64_t i0 = vscan_phys<Op>(L, n), f0 = i0 * d + c;
            S v[RP];
            typename Op::Aux aux;
#pragma unroll
            for (int k = 0; k < RP; ++k) v[k] = op.state(Op::kRev ? i0 - k : i0 + k, f0 + k * step, aux);
#pragma unroll
            for (int k = 0; k < RP; ++k) a = op.combine(a, v[k]);
        }
        for (; L < hi; ++L) {
            typename Op::Aux aux;
            const int64_t i = vscan_phys<Op>(L, n);
            a = op.combine(a, op.state(i, i * d + c, aux));
        }
    }
    a = warp_parts_scan(op, a, (int)d, P);
    if (active && p == P - 1) agg[u * d + c] = a;
}

// One block per column: the exclusive prefixes of the U unit states, in order.
constexpr int kVPrefixThreads = 1024;
template <class Op>
__global__ void __launch_bounds__(kVPrefixThreads)
k_vscan_wprefix(const Op op, const typename Op::S *__restrict__ agg, const int64_t U, const int64_t d,
                typename Op::S *__restrict__ pre) {
    using S = typename Op::S;
    __shared__ S s_w[kVPrefixThreads / kWarp];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t c = blockIdx.x;
    const int64_t per = (U + kVPrefixThreads - 1) / kVPrefixThreads;
    const int64_t g0 = t * per, g1 = g0 + per < U ? g0 + per : U;
    S v = op.identity();
    for (int64_t g = g0; g < g1; ++g) v = op.combine(v, agg[g * d + c]);
    const S inc = warp_inclusive_scan(op, v);
    if (lane == kWarp - 1) s_w[w] = inc;
    __syncthreads();
    S run = vscan_initial(op, c, 0);
    for (int j = 0; j < w; ++j) run = op.combine(run, s_w[j]);
    S ex = shfl_up(inc, 1);
    if (lane > 0) run = op.combine(run, ex);
    for (int64_t g = g0; g < g1; ++g) {
        pre[g * d + c] = run;
        run = op.combine(run, agg[g * d + c]);
    }
}

template <class Op, int RP>
__global__ void __launch_bounds__(kVScanThreads)
k_vscan_wapply(const Op op, const int64_t n, const int64_t d, const int64_t U, const typename Op::S *__restrict__ pre) {
    using S = typename Op::S;
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kVScanWarps + (threadIdx.x >> 5);
    if (u >= U) return;  // whole warps
    const int P = kWarp / (int)d;
    const bool active = lane < P * (int)d;
    const int64_t c = lane % d, p = lane / d;
    const int last = (P - 1) * (int)d + (int)c;  // the lane with column c's tile total
    int64_t l0, l1;
    vscan_range(n, u, U, &l0, &l1);
    S carry = active ? pre[u * d + c] : op.identity();
    for (int64_t lt = l0; lt < l1; lt += (int64_t)P * RP) {
        const int64_t lp = lt + p * RP;
        S st[RP];
        typename Op::Aux aux[RP];
        if constexpr (Op::kHaloChunk)
            vscan_chunk(op, lp, l1, n, c, active, st, aux);
        else
            vscan_load(op, lp, l1, n, d, c, active, st, aux);
        S a = op.identity();
#pragma unroll
        for (int k = 0; k < RP; ++k) a = op.combine(a, st[k]);
        a = warp_parts_scan(op, a, (int)d, P);
        const S ex = P > 1 ? shfl_up(a, (int)d) : a;  // P is warp-uniform; read for p > 0 only
        const S tile = shfl_idx(a, last);
        S r = p > 0 ? op.combine(carry, ex) : carry;
        vscan_store(op, lp, l1, n, d, c, active, r, st, aux);
        carry = op.combine(carry, tile);
    }
}

// Units of one wave of the rescan kernel: its resident blocks on every SM
// (cached per device) times the units a block holds, fewer for short inputs
// (at least 64 rows a unit).
template <class Op, int RP, bool WARP> static int64_t vscan_units(int64_t n) {
    // Host threads may call at once: the entries are atomics (every writer
    // stores the same value).
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int per_sm = cache[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        int b = 0;
        const void *k = WARP ? (const void *)k_vscan_wapply<Op, RP> : (const void *)k_vscan_apply<Op, RP>;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kVScanThreads, 0) != cudaSuccess || b < 1) b = 1;
        per_sm = b < kVScanMaxBlocksPerSM ? b : kVScanMaxBlocksPerSM;
        cache[dev].store(per_sm, std::memory_order_relaxed);
    }
    const int64_t want = (n + 63) / 64;
    const int64_t cap = (int64_t)num_sms() * per_sm * (WARP ? kVScanWarps : 1);
    return want < 1 ? 1 : want < cap ? want : cap;
}

template <class Op, int RP> static adc_status vscan_run(const Op &op, int64_t n, int64_t d, char *ws, cudaStream_t s) {
    using S = typename Op::S;
    if (n == 0) return ADC_OK;
    S *agg = reinterpret_cast<S *>(ws + kWsHeader);
    S *pre = reinterpret_cast<S *>(ws + kWsHeader + vscan_states_bytes(d, sizeof(S) > 16 ? sizeof(S) : 16));
    if (d <= kWarp) {
        const int64_t U = vscan_units<Op, RP, true>(n);
        const unsigned blocks = (unsigned)((U + kVScanWarps - 1) / kVScanWarps);
        k_vscan_wfold<Op, RP><<<blocks, kVScanThreads, 0, s>>>(op, n, d, U, agg);
        k_vscan_wprefix<Op><<<(unsigned)d, kVPrefixThreads, 0, s>>>(op, agg, U, d, pre);
        k_vscan_wapply<Op, RP><<<blocks, kVScanThreads, 0, s>>>(op, n, d, U, pre);
    } else {
        const int G = (int)vscan_units<Op, RP, false>(n);
        k_vscan_fold<Op, RP><<<G, kVScanThreads, 0, s>>>(op, n, d, agg);
        k_vscan_prefix<Op><<<(unsigned)d, kWarp, 0, s>>>(op, agg, G, d, pre);
        k_vscan_apply<Op, RP><<<G, kVScanThreads, 0, s>>>(op, n, d, pre);
    }
    return check_launch();
}

template <typename T>
static adc_status vscan_fwd_t(adc_op op, int64_t n, int64_t d, const T *x, T *y, char *ws, cudaStream_t s) {
    switch (op) {
    case ADC_OP_ADD: return vscan_run<VScanFwd<T, 0>, 16>({x, y, d}, n, d, ws, s);
    case ADC_OP_MUL: return vscan_run<VScanFwd<T, 1>, 16>({x, y, d}, n, d, ws, s);
    case ADC_OP_MIN: return vscan_run<VScanFwd<T, 2>, 16>({x, y, d}, n, d, ws, s);
    case ADC_OP_MAX: return vscan_run<VScanFwd<T, 3>, 16>({x, y, d}, n, d, ws, s);
    default: return ADC_ERR_UNSUPPORTED;
    }
}

template <typename T>
static adc_status vscan_vjp_t(adc_op op, int64_t n, int64_t d, const T *x, const T *y, const T *ybar, T *xbar,
                              int acc, char *ws, cudaStream_t s) {
    switch (op) {
    case ADC_OP_ADD: return vscan_run<VScanVjpAdd<T>, 8>({ybar, xbar, d, acc}, n, d, ws, s);
    case ADC_OP_MUL: return vscan_run<VScanVjpAff<T, 1>, 8>({x, y, ybar, xbar, n, d, acc}, n, d, ws, s);
    case ADC_OP_MIN: return vscan_run<VScanVjpAff<T, 2>, 8>({x, y, ybar, xbar, n, d, acc}, n, d, ws, s);
    case ADC_OP_MAX: return vscan_run<VScanVjpAff<T, 3>, 8>({x, y, ybar, xbar, n, d, acc}, n, d, ws, s);
    default: return ADC_ERR_UNSUPPORTED;
    }
}

// d = 1 is the scalar scan itself; wider rows take the direct form above.
adc_status vscan_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws, cudaStream_t s) {
    if (d == 1) return scan_fwd(op, dt, n, x, y, ws, s);
    char *w = static_cast<char *>(ws);
    if (dt == ADC_F64)
        return vscan_fwd_t<double>(op, n, d, static_cast<const double *>(x), static_cast<double *>(y), w, s);
    return vscan_fwd_t<float>(op, n, d, static_cast<const float *>(x), static_cast<float *>(y), w, s);
}

adc_status vscan_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                     void *xbar, int accumulate, void *ws, cudaStream_t s) {
    if (d == 1) return scan_vjp(op, dt, n, x, y, ybar, xbar, accumulate, ws, s);
    char *w = static_cast<char *>(ws);
    if (dt == ADC_F64)
        return vscan_vjp_t<double>(op, n, d, static_cast<const double *>(x), static_cast<const double *>(y),
                                   static_cast<const double *>(ybar), static_cast<double *>(xbar), accumulate, w, s);
    return vscan_vjp_t<float>(op, n, d, static_cast<const float *>(x), static_cast<const float *>(y),
                              static_cast<const float *>(ybar), static_cast<float *>(xbar), accumulate, w, s);
}

// Rows of d equal lin / sumOfProd / 2x2 elements (the tuple scans' uniform
// multi-word rows), in the direct form; workspace from velem_ws_bytes.
size_t velem_ws_bytes(adc_op op, adc_dtype dt, int64_t d) {
    const size_t s = dt == ADC_F64 ? 8 : 4;
    const size_t sb = op == ADC_OP_MM2 ? 8 * s : 4 * s;  // the largest state: the vjp's (v, c) / 3 words rounded
    return kWsHeader + 2 * vscan_states_bytes(d, sb > 16 ? sb : 16);
}
template <typename T>
static adc_status velem_fwd_t(adc_op op, int64_t n, int64_t d, const void *x, void *y, char *ws, cudaStream_t s) {
    switch (op) {
    case ADC_OP_LIN:
        return vscan_run<VScanFwdE<T, ElemLin<T>>, 8>(
            {static_cast<const Pair<T> *>(x), static_cast<Pair<T> *>(y), d}, n, d, ws, s);
    case ADC_OP_SOP:
        return vscan_run<VScanFwdE<T, ElemSop<T>>, 8>(
            {static_cast<const Pair<T> *>(x), static_cast<Pair<T> *>(y), d}, n, d, ws, s);
    case ADC_OP_MM2:
        return vscan_run<VScanFwdE<T, ElemMM2<T>>, 4>(
            {static_cast<const Mat2<T> *>(x), static_cast<Mat2<T> *>(y), d}, n, d, ws, s);
    default: return ADC_ERR_UNSUPPORTED;
    }
}
template <typename T>
static adc_status velem_vjp_t(adc_op op, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                              void *xbar, int acc, char *ws, cudaStream_t s) {
    switch (op) {
    case ADC_OP_LIN: {
        using E = Pair<T>;
        return vscan_run<VScanVjpLinE<T>, 4>({static_cast<const E *>(x), static_cast<const E *>(y),
                                              static_cast<const E *>(ybar), static_cast<E *>(xbar), n, d, acc},
                                             n, d, ws, s);
    }
    case ADC_OP_SOP: {
        using E = Pair<T>;
        return vscan_run<VScanVjpSopE<T>, 4>({static_cast<const E *>(x), static_cast<const E *>(y),
                                              static_cast<const E *>(ybar), static_cast<E *>(xbar), n, d, acc},
                                             n, d, ws, s);
    }
    case ADC_OP_MM2: {
        using E = Mat2<T>;
        return vscan_run<VScanVjpMM2E<T>, 2>({static_cast<const E *>(x), static_cast<const E *>(y),
                                              static_cast<const E *>(ybar), static_cast<E *>(xbar), n, d, acc},
                                             n, d, ws, s);
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}
adc_status velem_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws, cudaStream_t s) {
    char *w = static_cast<char *>(ws);
    return dt == ADC_F64 ? velem_fwd_t<double>(op, n, d, x, y, w, s) : velem_fwd_t<float>(op, n, d, x, y, w, s);
}
adc_status velem_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                     void *xbar, int accumulate, void *ws, cudaStream_t s) {
    char *w = static_cast<char *>(ws);
    return dt == ADC_F64 ? velem_vjp_t<double>(op, n, d, x, y, ybar, xbar, accumulate, w, s)
                         : velem_vjp_t<float>(op, n, d, x, y, ybar, xbar, accumulate, w, s);
}

// -------------------------------------------- reduce_by_index, direct form --
// For + (fp32, fp64) and the lifted fp32 min/max, when one block's shared
// memory holds the whole [m][d] table: the same fixed-column striding over the
// row-major values (each thread meets one column c and reads its row's key),
// the element goes to table[key][c] (a float add, or Fig. 5's packed
// value/index key), each block writes its table as a partial row, and a final
// kernel folds the rows in block order per (bin, column) -- decoding min/max,
// folding hist0 in and writing column c's selected indices where the scalar
// entry point keeps them (saved + c * sv).  Other cases take the transposed
// path above.
constexpr int kVHThreads = 1024;


// MODE 0: +, entries T; MODE 1 / 2: min / max, entries packed 64-bit keys.
template <typename T, int MODE> struct VHE { using type = T; };
template <typename T> struct VHE<T, 1> { using type = unsigned long long; };
template <typename T> struct VHE<T, 2> { using type = unsigned long long; };

template <typename T, int MODE>
__global__ void __launch_bounds__(kVHThreads)
k_vhist_rows(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
             const int64_t d, typename VHE<T, MODE>::type *__restrict__ part) {
    using E = typename VHE<T, MODE>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E *tab = reinterpret_cast<E *>(smem_raw);
    const int64_t cells = m * d;
    for (int64_t j = threadIdx.x; j < cells; j += blockDim.x)
        tab[j] = MODE == 0 ? E(0) : (MODE == 2 ? Pack<true>::kEmpty : Pack<false>::kEmpty);
    __syncthreads();
    const int64_t S_ = vred_active(d);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt < S_) {
        const int64_t total = n * d, rstep = S_ / d, c = gt % d;
        auto upd = [&](int32_t k, T v, int64_t row) {
            if (!in_range(k, m)) return;
            E *cell = tab + (int64_t)k * d + c;
            if constexpr (MODE == 0) atomicAdd(cell, v);
            else if constexpr (MODE == 1) Pack<false>::update_smem(cell, Pack<false>::key((float)v, row));
            else Pack<true>::update_smem(cell, Pack<true>::key((float)v, row));
        };
        constexpr int U = 4;  // four rows' loads in flight per thread
        int64_t row = gt / d, f = gt;
        for (; f + (U - 1) * S_ < total; f += U * S_, row += U * rstep) {
            int32_t k[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                k[u] = __ldg(keys + row + u * rstep);
                v[u] = __ldcs(vals + f + u * S_);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) upd(k[u], v[u], row + u * rstep);
        }
        for (; f < total; f += S_, row += rstep) upd(__ldg(keys + row), __ldcs(vals + f), row);
    }
    __syncthreads();
    E *dst = part + (int64_t)blockIdx.x * cells;
    for (int64_t j = threadIdx.x; j < cells; j += blockDim.x) dst[j] = tab[j];
}

template <typename T, int MODE>
__global__ void k_vhist_final(const typename VHE<T, MODE>::type *__restrict__ part, const int G, const int64_t m,
                              const int64_t d, const T *__restrict__ vals, const T *__restrict__ h0, const int64_t n,
                              T *__restrict__ hist, char *__restrict__ saved, const size_t sv) {
    using E = typename VHE<T, MODE>::type;
    const int64_t cells = m * d;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cells; j += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (MODE == 0) {
            T a = T(0);
            for (int g = 0; g < G; ++g) a += part[(int64_t)g * cells + j];
            hist[j] = h0 ? h0[j] + a : a;
        } else {
            constexpr bool MAX = MODE == 2;
            E best = Pack<MAX>::kEmpty;
            for (int g = 0; g < G; ++g) {
                const E k = part[(int64_t)g * cells + j];
                if (Pack<MAX>::better(k, best)) best = k;
            }
            const int64_t c = j % d, bin = j / d;
            float v = MAX ? -Num<float>::inf() : Num<float>::inf();
            int64_t idx = n;
            if (best != Pack<MAX>::kEmpty) {
                idx = Pack<MAX>::index(best);
                v = from_ordered((uint32_t)(best >> 32));
                if (v == 0.0f) v = (float)vals[idx * d + c];  // the key folds -0.0 onto +0.0
            }
            if (h0) {
                const float a = (float)h0[j];
                if (MAX ? (a >= v) : (a <= v)) {
                    v = a;
                    idx = n;
                }
            }
            hist[j] = (T)v;
            if (saved) reinterpret_cast<int32_t *>(saved + c * sv)[bin] = (int32_t)idx;
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
k_vhist_vjp(const int32_t *__restrict__ keys, const char *__restrict__ saved, const size_t sv,
            const T *__restrict__ hb, T *__restrict__ vb, const int64_t n, const int64_t m, const int64_t d,
            const int accumulate) {
    const int64_t S_ = vred_active(d);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= S_) return;
    const int64_t total = n * d, rstep = S_ / d, c = gt % d;
    const int32_t *is = MODE == 0 ? nullptr : reinterpret_cast<const int32_t *>(saved + c * sv);
    int64_t row = gt / d;
    for (int64_t f = gt; f < total; f += S_, row += rstep) {
        const int32_t k = __ldg(keys + row);
        T g = T(0);
        if (in_range(k, m) && (MODE == 0 || __ldg(is + k) == (int32_t)row)) g = __ldg(hb + (int64_t)k * d + c);
        vb[f] = accumulate ? vb[f] + g : g;
    }
}

template <typename T, int MODE>
__global__ void k_vhist_h0bar(const char *__restrict__ saved, const size_t sv, const T *__restrict__ hb,
                              T *__restrict__ h0b, const int64_t m, const int64_t d, const int64_t n,
                              const int accumulate) {
    const int64_t cells = m * d;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cells; j += (int64_t)gridDim.x * blockDim.x) {
        T g = hb[j];
        if (MODE != 0 && reinterpret_cast<const int32_t *>(saved + (j % d) * sv)[j / d] < n) g = T(0);
        h0b[j] = accumulate ? h0b[j] + g : g;
    }
}

template <typename T, int MODE>
static adc_status vhist_direct_fwd(int64_t n, int64_t m, int64_t d, const int32_t *keys, const T *vals, const T *h0,
                                   T *hist, char *saved, size_t sv, char *ws, cudaStream_t s) {
    using E = typename VHE<T, MODE>::type;
    const int G = num_sms();
    E *part = reinterpret_cast<E *>(ws + kWsHeader);
    const size_t smem = (size_t)m * (size_t)d * sizeof(E);
    if (cudaFuncSetAttribute(k_vhist_rows<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return ADC_ERR_CUDA;
    k_vhist_rows<T, MODE><<<G, kVHThreads, smem, s>>>(keys, vals, n, m, d, part);
    const int64_t cells = m * d;
    const unsigned gb = (unsigned)((cells + 255) / 256 < 4096 ? (cells + 255) / 256 : 4096);
    k_vhist_final<T, MODE><<<gb, 256, 0, s>>>(part, G, m, d, vals, h0, n, hist, saved, sv);
    return check_launch();
}

template <typename T, int MODE>
static adc_status vhist_direct_vjp(int64_t n, int64_t m, int64_t d, const int32_t *keys, const char *saved, size_t sv,
                                   const T *hb, T *vb, T *h0b, int acc, cudaStream_t s) {
    if (n > 0) k_vhist_vjp<T, MODE><<<num_sms() * 8, 256, 0, s>>>(keys, saved, sv, hb, vb, n, m, d, acc);
    if (h0b) {
        const int64_t cells = m * d;
        const unsigned gb = (unsigned)((cells + 255) / 256 < 4096 ? (cells + 255) / 256 : 4096);
        k_vhist_h0bar<T, MODE><<<gb, 256, 0, s>>>(saved, sv, hb, h0b, m, d, n, acc);
    }
    return check_launch();
}

adc_status vhist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys, const void *vals,
                     const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s) {
    if (vhist_direct(op, dt, m, d)) {
        const size_t svb = align_up(scalar_saved(ADC_HIST, op, dt, n, m), 256);
        char *sv = static_cast<char *>(saved), *w = static_cast<char *>(ws);
        if (dt == ADC_F64)
            return vhist_direct_fwd<double, 0>(n, m, d, keys, static_cast<const double *>(vals),
                                               static_cast<const double *>(hist0), static_cast<double *>(hist), sv,
                                               svb, w, s);
        const float *v = static_cast<const float *>(vals), *h0 = static_cast<const float *>(hist0);
        float *h = static_cast<float *>(hist);
        if (op == ADC_OP_ADD) return vhist_direct_fwd<float, 0>(n, m, d, keys, v, h0, h, sv, svb, w, s);
        if (op == ADC_OP_MIN) return vhist_direct_fwd<float, 1>(n, m, d, keys, v, h0, h, sv, svb, w, s);
        return vhist_direct_fwd<float, 2>(n, m, d, keys, v, h0, h, sv, svb, w, s);
    }
    const VLayout L = vlayout(op, dt, n, m, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *vt = w + L.nplane[0], *h0t = w + L.mplane[0], *ht = w + L.mplane[1];
    adc_status st = to_plane(dt, n, d, vals, vt, s);
    if (st != ADC_OK) return st;
    if (hist0 && (st = to_plane(dt, m, d, hist0, h0t, s)) != ADC_OK) return st;
    const size_t sv = align_up(scalar_saved(ADC_HIST, op, dt, n, m), 256);
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        if ((st = hist_fwd(op, dt, n, m, keys, vt + (size_t)c * plane_ld(n) * e, hist0 ? h0t + (size_t)c * plane_ld(m) * e : nullptr,
                           ht + (size_t)c * plane_ld(m) * e, saved ? static_cast<char *>(saved) + c * sv : nullptr, cw, s)) !=
            ADC_OK)
            return st;
    }
    if ((st = from_plane(dt, m, d, ht, hist, s)) != ADC_OK) return st;
    return finish(w, L, d, s);
}

adc_status vhist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys, const void *vals,
                     const void *hist0, const void *hist, const void *saved, const void *histbar, void *valsbar,
                     void *hist0bar, int accumulate, void *ws, cudaStream_t s) {
    (void)hist;
    if (vhist_direct(op, dt, m, d)) {
        const size_t svb = align_up(scalar_saved(ADC_HIST, op, dt, n, m), 256);
        const char *sv = static_cast<const char *>(saved);
        if (dt == ADC_F64)
            return vhist_direct_vjp<double, 0>(n, m, d, keys, sv, svb, static_cast<const double *>(histbar),
                                               static_cast<double *>(valsbar), static_cast<double *>(hist0bar),
                                               accumulate, s);
        const float *hb = static_cast<const float *>(histbar);
        float *vb = static_cast<float *>(valsbar), *h0b = static_cast<float *>(hist0bar);
        if (op == ADC_OP_ADD) return vhist_direct_vjp<float, 0>(n, m, d, keys, sv, svb, hb, vb, h0b, accumulate, s);
        if (op == ADC_OP_MIN) return vhist_direct_vjp<float, 1>(n, m, d, keys, sv, svb, hb, vb, h0b, accumulate, s);
        return vhist_direct_vjp<float, 2>(n, m, d, keys, sv, svb, hb, vb, h0b, accumulate, s);
    }
    const VLayout L = vlayout(op, dt, n, m, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *vt = w + L.nplane[0], *vbt = w + L.nplane[1];
    char *hbt = w + L.mplane[0], *h0t = w + L.mplane[1], *h0bt = w + L.mplane[2];
    adc_status st;
    if (vals && (st = to_plane(dt, n, d, vals, vt, s)) != ADC_OK) return st;
    if ((st = to_plane(dt, m, d, histbar, hbt, s)) != ADC_OK) return st;
    if (hist0 && (st = to_plane(dt, m, d, hist0, h0t, s)) != ADC_OK) return st;
    if (accumulate && (st = to_plane(dt, n, d, valsbar, vbt, s)) != ADC_OK) return st;
    if (accumulate && hist0bar && (st = to_plane(dt, m, d, hist0bar, h0bt, s)) != ADC_OK) return st;
    const size_t sv = align_up(scalar_saved(ADC_HIST, op, dt, n, m), 256);
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        if ((st = hist_vjp(op, dt, n, m, keys, vals ? vt + (size_t)c * plane_ld(n) * e : nullptr,
                           hist0 ? h0t + (size_t)c * plane_ld(m) * e : nullptr, nullptr,
                           saved ? static_cast<const char *>(saved) + c * sv : nullptr, hbt + (size_t)c * plane_ld(m) * e,
                           vbt + (size_t)c * plane_ld(n) * e, hist0bar ? h0bt + (size_t)c * plane_ld(m) * e : nullptr, accumulate, cw,
                           s)) != ADC_OK)
            return st;
    }
    if ((st = from_plane(dt, n, d, vbt, valsbar, s)) != ADC_OK) return st;
    if (hist0bar && (st = from_plane(dt, m, d, h0bt, hist0bar, s)) != ADC_OK) return st;
    return finish(w, L, d, s);
}

}  // namespace adc
