// Vectorised operators: reduce, scan and reduce_by_index whose operator is
// map2 (.) over rows of d elements (Sec. 3.2, "Vectorized Operators", the
// Irwim rule; Sec. 5.3, the Iswim rule; the same interchange for
// reduce_by_index).  Each rule interchanges the outer combinator with the
// inner map, so that
//   reduce (map2 .) (replicate d e) x  ==  map (reduce . e) (transpose x)
//   scan   (map2 .) (replicate d e) x  ==  transpose (map (scan . e) (transpose x))
// and the vjp is taken of the right-hand side: d scalar combinators whose
// specialised rules (Sec. 3-5) apply column by column.  Here: tiled
// shared-memory transposes of the [n][d] (or [m][d]) operands to [d][n], d
// calls of the scalar kernels on contiguous rows, and a transpose back of the
// [n][d] / [m][d] results.  Operators: ADD, MUL, MIN, MAX (scalar elements).
#include "common.cuh"
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
// [header][n-planes: [d][n] each][m-planes: [d][m] each][per-column scalar
// workspaces, each with its own header].  Planes per kind: reduce 2 (x^T,
// xbar^T); scan 4 (x^T, y^T, ybar^T, xbar^T); reduce_by_index 2 n-planes
// (vals^T, valsbar^T) and 3 m-planes (hist0^T / histbar^T, hist^T, hist0bar^T).
struct VLayout {
    size_t nplane[4], mplane[3], col, col_stride, bytes;
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

static VLayout vlayout(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    VLayout L{};
    const size_t e = dt == ADC_F64 ? 8 : 4;
    const int np = kind == ADC_SCAN ? 4 : 2, mp = kind == ADC_HIST ? 3 : 0;
    size_t o = kWsHeader;
    for (int i = 0; i < np; ++i) {
        L.nplane[i] = o;
        o = align_up(o + (size_t)d * plane_ld(n) * e, 256);
    }
    for (int i = 0; i < mp; ++i) {
        L.mplane[i] = o;
        o = align_up(o + (size_t)d * plane_ld(m) * e, 256);
    }
    L.col = o;
    L.col_stride = align_up(scalar_ws(kind, op, dt, n, m), 256);
    L.bytes = o + (size_t)d * L.col_stride;
    return L;
}

size_t vws_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    if (scalar_ws(kind, op, dt, n, m) == 0) return 0;
    return vlayout(kind, op, dt, n, m, d).bytes;
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
adc_status vreduce_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *saved, void *ws,
                       cudaStream_t s) {
    const VLayout L = vlayout(ADC_REDUCE, op, dt, n, 0, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *xt = w + L.nplane[0];
    adc_status st = to_plane(dt, n, d, x, xt, s);
    if (st != ADC_OK) return st;
    const size_t sv = align_up(scalar_saved(ADC_REDUCE, op, dt, n, 0), 256);
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        // y is the row of d results; column c's residuals follow column c-1's
        if ((st = reduce_fwd(op, dt, n, xt + (size_t)c * plane_ld(n) * e, static_cast<char *>(y) + c * e,
                             saved ? static_cast<char *>(saved) + c * sv : nullptr, cw, s)) != ADC_OK)
            return st;
    }
    return finish(w, L, d, s);
}

adc_status vreduce_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *saved,
                       const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s) {
    const VLayout L = vlayout(ADC_REDUCE, op, dt, n, 0, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *xt = w + L.nplane[0], *xbt = w + L.nplane[1];
    adc_status st;
    if (x && (st = to_plane(dt, n, d, x, xt, s)) != ADC_OK) return st;
    if (accumulate && (st = to_plane(dt, n, d, xbar, xbt, s)) != ADC_OK) return st;
    const size_t sv = align_up(scalar_saved(ADC_REDUCE, op, dt, n, 0), 256);
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        if ((st = reduce_vjp(op, dt, n, x ? xt + (size_t)c * plane_ld(n) * e : nullptr, static_cast<const char *>(y) + c * e,
                             saved ? static_cast<const char *>(saved) + c * sv : nullptr,
                             static_cast<const char *>(ybar) + c * e, xbt + (size_t)c * plane_ld(n) * e, accumulate, cw, s)) !=
            ADC_OK)
            return st;
    }
    if ((st = from_plane(dt, n, d, xbt, xbar, s)) != ADC_OK) return st;
    return finish(w, L, d, s);
}

adc_status vscan_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws, cudaStream_t s) {
    const VLayout L = vlayout(ADC_SCAN, op, dt, n, 0, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *xt = w + L.nplane[0], *yt = w + L.nplane[1];
    adc_status st = to_plane(dt, n, d, x, xt, s);
    if (st != ADC_OK) return st;
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        if ((st = scan_fwd(op, dt, n, xt + (size_t)c * plane_ld(n) * e, yt + (size_t)c * plane_ld(n) * e, cw, s)) != ADC_OK) return st;
    }
    if ((st = from_plane(dt, n, d, yt, y, s)) != ADC_OK) return st;
    return finish(w, L, d, s);
}

adc_status vscan_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                     void *xbar, int accumulate, void *ws, cudaStream_t s) {
    const VLayout L = vlayout(ADC_SCAN, op, dt, n, 0, d);
    const size_t e = dt == ADC_F64 ? 8 : 4;
    char *w = static_cast<char *>(ws);
    char *xt = w + L.nplane[0], *yt = w + L.nplane[1], *ybt = w + L.nplane[2], *xbt = w + L.nplane[3];
    adc_status st;
    if (op != ADC_OP_ADD) {
        if ((st = to_plane(dt, n, d, x, xt, s)) != ADC_OK) return st;
        if ((st = to_plane(dt, n, d, y, yt, s)) != ADC_OK) return st;
    }
    if ((st = to_plane(dt, n, d, ybar, ybt, s)) != ADC_OK) return st;
    if (accumulate && (st = to_plane(dt, n, d, xbar, xbt, s)) != ADC_OK) return st;
    const Cols cols{w + L.col, L.col_stride};
    for (int64_t c = 0; c < d; ++c) {
        bool ok;
        char *cw = cols.ws(c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        const size_t off = (size_t)c * plane_ld(n) * e;
        if ((st = scan_vjp(op, dt, n, xt + off, yt + off, ybt + off, xbt + off, accumulate, cw, s)) != ADC_OK) return st;
    }
    if ((st = from_plane(dt, n, d, xbt, xbar, s)) != ADC_OK) return st;
    return finish(w, L, d, s);
}

adc_status vhist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys, const void *vals,
                     const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s) {
    const VLayout L = vlayout(ADC_HIST, op, dt, n, m, d);
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
    const VLayout L = vlayout(ADC_HIST, op, dt, n, m, d);
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
