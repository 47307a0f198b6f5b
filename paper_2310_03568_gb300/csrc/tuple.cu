// Tuple scans with block-diagonal Jacobians (Sec. 5.3.3, BDS).  The element is
// a tuple of k blocks; block c is an element of operator ops[c] (arity a_c) and
// the tuple operator applies ops[c] to block c alone, so the Jacobian of every
// step is block-diagonal with k blocks of a_c x a_c.  The BDS rule replaces the
// one reverse scan over (alpha^D, alpha^{D x D}) pairs by k scans over
// (alpha^{a_c}, alpha^{a_c x a_c}); each of them here is block c's own forward
// or vjp launch of scan.cu, so inside a block its specialised rule still
// applies (RBDS for lin and the matrix products, the general rule for
// sumOfProd and min/max).
//
// Two layouts.  Blocks in separate arrays -- the tuple-of-arrays form the
// paper's compiler uses: k scans on the caller's arrays, nothing copied.  Rows
// [n][D] with the blocks side by side: the rows are split into per-block
// planes through shared-memory tiles, each plane is scanned, and the results
// are merged back into rows -- except when every block is the same scalar
// operator (+, *, min, max), where the rows are the vectorised scan of width k
// and its direct form scans them in place.
#include "common.cuh"
#include "internal.h"

namespace adc {

struct TupleDesc {
    int k, D, Dp;                   // blocks, row width, shared-memory row stride (odd)
    int off[kMaxTupleBlocks];       // first column of block c in a row
    int w[kMaxTupleBlocks];         // arity of block c
    float invw[kMaxTupleBlocks];    // 1 / w[c]
    int64_t plane[kMaxTupleBlocks]; // element offset of block c's plane in a plane set
};

// q = f / d for f < 2^14 by a float reciprocal and one correction step (the
// estimate is off by at most one there); an integer division per element
// would dominate these copy kernels.
struct SmallDiv {
    uint32_t d;
    float inv;
    __device__ __forceinline__ uint32_t operator()(uint32_t f) const {
        uint32_t q = __float2uint_rz(__uint2float_rz(f) * inv);
        if (q * d > f) --q;
        else if ((q + 1) * d <= f) ++q;
        return q;
    }
};
__device__ __forceinline__ SmallDiv small_div(int d) { return {(uint32_t)d, 1.0f / (float)d}; }

// 16-byte words of T, for the vectorised halves of the copies.
template <typename T> struct Vec16 {
    static constexpr int V = 16 / (int)sizeof(T);
    T v[V];
};

// Rows [n][D] -> k planes [n][a_c].  A tile of R rows (R a multiple of 4, so
// every tile and every plane run starts on a 16-byte boundary) is read with
// 16-byte loads into shared memory (row stride Dp odd: a column walk is
// conflict-free), then each block's R x a_c run is written out with 16-byte
// stores; the ragged ends element by element.
template <typename T>
__global__ void __launch_bounds__(256) k_tuple_split(const T *__restrict__ x, T *__restrict__ planes,
                                                      const TupleDesc d, const int64_t n, const int R) {
    constexpr int V = Vec16<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const SmallDiv divD = small_div(d.D);
    const int64_t tiles = (n + R - 1) / R;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t r0 = t * R;
        const int rows = (int)((n - r0) < R ? (n - r0) : R);
        const int total = rows * d.D;
        const T *src = x + r0 * d.D;
        for (int fv = threadIdx.x; fv < total / V; fv += blockDim.x) {
            const Vec16<T> u = reinterpret_cast<const Vec16<T> *>(src)[fv];
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int f = fv * V + q, r = (int)divD((uint32_t)f);
                sm[r * d.Dp + (f - r * d.D)] = u.v[q];
            }
        }
        for (int f = (total / V) * V + threadIdx.x; f < total; f += blockDim.x) {
            const int r = (int)divD((uint32_t)f);
            sm[r * d.Dp + (f - r * d.D)] = src[f];
        }
        __syncthreads();
        for (int b = 0; b < d.k; ++b) {
            const int w = d.w[b], o = d.off[b], cnt = rows * w;
            const SmallDiv divw{(uint32_t)w, d.invw[b]};
            T *dst = planes + d.plane[b] + r0 * w;
            for (int jv = threadIdx.x; jv < cnt / V; jv += blockDim.x) {
                Vec16<T> u;
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    const int j = jv * V + q, r = (int)divw((uint32_t)j);
                    u.v[q] = sm[r * d.Dp + o + (j - r * w)];
                }
                reinterpret_cast<Vec16<T> *>(dst)[jv] = u;
            }
            for (int j = (cnt / V) * V + threadIdx.x; j < cnt; j += blockDim.x) {
                const int r = (int)divw((uint32_t)j);
                dst[j] = sm[r * d.Dp + o + (j - r * w)];
            }
        }
        __syncthreads();
    }
}

// k planes -> rows [n][D] (y = rows, or y += rows), the same way round.
template <typename T>
__global__ void __launch_bounds__(256) k_tuple_merge(const T *__restrict__ planes, T *__restrict__ y,
                                                      const TupleDesc d, const int64_t n, const int R,
                                                      const int accumulate) {
    constexpr int V = Vec16<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const SmallDiv divD = small_div(d.D);
    const int64_t tiles = (n + R - 1) / R;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t r0 = t * R;
        const int rows = (int)((n - r0) < R ? (n - r0) : R);
        const int total = rows * d.D;
        for (int b = 0; b < d.k; ++b) {
            const int w = d.w[b], o = d.off[b], cnt = rows * w;
            const SmallDiv divw{(uint32_t)w, d.invw[b]};
            const T *src = planes + d.plane[b] + r0 * w;
            for (int jv = threadIdx.x; jv < cnt / V; jv += blockDim.x) {
                const Vec16<T> u = reinterpret_cast<const Vec16<T> *>(src)[jv];
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    const int j = jv * V + q, r = (int)divw((uint32_t)j);
                    sm[r * d.Dp + o + (j - r * w)] = u.v[q];
                }
            }
            for (int j = (cnt / V) * V + threadIdx.x; j < cnt; j += blockDim.x) {
                const int r = (int)divw((uint32_t)j);
                sm[r * d.Dp + o + (j - r * w)] = src[j];
            }
        }
        __syncthreads();
        T *dst = y + r0 * d.D;
        for (int fv = threadIdx.x; fv < total / V; fv += blockDim.x) {
            Vec16<T> u;
            if (accumulate) u = reinterpret_cast<const Vec16<T> *>(dst)[fv];
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int f = fv * V + q, r = (int)divD((uint32_t)f);
                const T v = sm[r * d.Dp + (f - r * d.D)];
                u.v[q] = accumulate ? u.v[q] + v : v;
            }
            reinterpret_cast<Vec16<T> *>(dst)[fv] = u;
        }
        for (int f = (total / V) * V + threadIdx.x; f < total; f += blockDim.x) {
            const int r = (int)divD((uint32_t)f);
            const T v = sm[r * d.Dp + (f - r * d.D)];
            dst[f] = accumulate ? dst[f] + v : v;
        }
        __syncthreads();
    }
}

// OR the blocks' error words into the call's own.
__global__ void k_tuple_errors(unsigned *err, const char *blocks, const int k, const size_t stride) {
    unsigned e = 0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) e |= *reinterpret_cast<const unsigned *>(blocks + c * stride);
    if (e) atomicOr(err, e);
}

// ------------------------------------------------------------- workspace --
// [header][k block workspaces, each with its own header][rows layout, k > 1:
// four plane sets (x, y, ybar, xbar), each the k planes at 256-byte offsets].
struct TLayout {
    size_t blocks, stride, sets[4], set_bytes, bytes;
    int64_t plane[kMaxTupleBlocks];  // element offsets within a set
};

static TLayout tlayout(int k, const adc_op *ops, adc_dtype dt, int64_t n, bool rows) {
    TLayout L{};
    const size_t e = dt == ADC_F64 ? 8 : 4;
    size_t stride = 0;
    for (int c = 0; c < k; ++c) {
        const size_t b = align_up(scan_ws_bytes(ops[c], dt, n), 256);
        stride = b > stride ? b : stride;
    }
    L.blocks = kWsHeader;
    L.stride = stride;
    size_t o = L.blocks + (size_t)k * stride;
    if (rows && k > 1) {
        size_t p = 0;
        for (int c = 0; c < k; ++c) {
            L.plane[c] = (int64_t)(p / e);
            p = align_up(p + (size_t)n * arity(ops[c]) * e, 256);
        }
        L.set_bytes = p;
        for (int i = 0; i < 4; ++i) {
            L.sets[i] = o;
            o += p;
        }
    }
    L.bytes = o;
    return L;
}

// Rows whose k blocks are all the same scalar operator (+, *, min or max) are
// the vectorised scan of width k: its direct form scans them in place.
static bool uniform_scalar(int k, const adc_op *ops) {
    const adc_op op = ops[0];
    if (op != ADC_OP_ADD && op != ADC_OP_MUL && op != ADC_OP_MIN && op != ADC_OP_MAX) return false;
    for (int c = 1; c < k; ++c)
        if (ops[c] != op) return false;
    return true;
}

// Rows whose k blocks are all lin, all sumOfProd or all 2x2 matrix products
// are k element columns: the vectorised direct form scans them in place too.
static bool uniform_elem(int k, const adc_op *ops) {
    const adc_op op = ops[0];
    if (op != ADC_OP_LIN && op != ADC_OP_SOP && op != ADC_OP_MM2) return false;
    for (int c = 1; c < k; ++c)
        if (ops[c] != op) return false;
    return true;
}

size_t tscan_ws_bytes(int k, const adc_op *ops, adc_dtype dt, int64_t n, bool rows) {
    if (rows && k == 1) return scan_ws_bytes(ops[0], dt, n);
    if (rows && uniform_scalar(k, ops)) return vws_bytes(ADC_SCAN, ops[0], dt, n, 0, k);
    if (rows && uniform_elem(k, ops)) return velem_ws_bytes(ops[0], dt, k);
    return tlayout(k, ops, dt, n, rows).bytes;
}

static char *block_ws(char *ws, const TLayout &L, int c, cudaStream_t s, bool *ok) {
    char *w = ws + L.blocks + (size_t)c * L.stride;
    *ok = cudaMemsetAsync(w, 0, kWsHeader, s) == cudaSuccess;
    return w;
}

static adc_status gather_errors(char *ws, const TLayout &L, int k, cudaStream_t s) {
    k_tuple_errors<<<1, 64, 0, s>>>(reinterpret_cast<unsigned *>(ws), ws + L.blocks, k, L.stride);
    return check_launch();
}

// ------------------------------------------------------- tuple of arrays --
static adc_status fwd_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x, void *const *y,
                             char *ws, const TLayout &L, cudaStream_t s) {
    for (int c = 0; c < k; ++c) {
        bool ok;
        char *w = block_ws(ws, L, c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        const adc_status st = scan_fwd(ops[c], dt, n, x[c], y[c], w, s);
        if (st != ADC_OK) return st;
    }
    return gather_errors(ws, L, k, s);
}

static adc_status vjp_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x,
                             const void *const *y, const void *const *ybar, void *const *xbar, int acc, char *ws,
                             const TLayout &L, cudaStream_t s) {
    for (int c = 0; c < k; ++c) {
        bool ok;
        char *w = block_ws(ws, L, c, s, &ok);
        if (!ok) return ADC_ERR_CUDA;
        const adc_status st = scan_vjp(ops[c], dt, n, x[c], y[c], ybar[c], xbar[c], acc, w, s);
        if (st != ADC_OK) return st;
    }
    return gather_errors(ws, L, k, s);
}

adc_status tscan_fwd_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x, void *const *y,
                            void *ws, cudaStream_t s) {
    const TLayout L = tlayout(k, ops, dt, n, false);
    return fwd_blocks(k, ops, dt, n, x, y, static_cast<char *>(ws), L, s);
}

adc_status tscan_vjp_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x,
                            const void *const *y, const void *const *ybar, void *const *xbar, int accumulate, void *ws,
                            cudaStream_t s) {
    const TLayout L = tlayout(k, ops, dt, n, false);
    return vjp_blocks(k, ops, dt, n, x, y, ybar, xbar, accumulate, static_cast<char *>(ws), L, s);
}

// -------------------------------------------------------------------- rows --
static TupleDesc tdesc(int k, const adc_op *ops, const TLayout &L) {
    TupleDesc d{};
    d.k = k;
    int o = 0;
    for (int c = 0; c < k; ++c) {
        d.off[c] = o;
        d.w[c] = arity(ops[c]);
        d.invw[c] = 1.0f / (float)d.w[c];
        d.plane[c] = L.plane[c];
        o += d.w[c];
    }
    d.D = o;
    d.Dp = o | 1;
    return d;
}

// Rows per tile: 16 KB of shared memory per block (Dp <= 65 scalars: R >= 28),
// a multiple of 4 so that tiles and plane runs start on 16-byte boundaries.
static int tile_rows(const TupleDesc &d, size_t e) { return (int)(16384 / ((size_t)d.Dp * e)) & ~3; }

static unsigned tile_grid(int64_t n, int R) {
    const int64_t tiles = (n + R - 1) / R;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)(tiles < cap ? (tiles < 1 ? 1 : tiles) : cap);
}

template <typename T>
static adc_status split_t(const TupleDesc &d, int64_t n, const void *x, char *set, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    const int R = tile_rows(d, sizeof(T));
    k_tuple_split<T><<<tile_grid(n, R), 256, (size_t)R * d.Dp * sizeof(T), s>>>(static_cast<const T *>(x),
                                                                               reinterpret_cast<T *>(set), d, n, R);
    return check_launch();
}

template <typename T>
static adc_status merge_t(const TupleDesc &d, int64_t n, const char *set, void *y, int acc, cudaStream_t s) {
    if (n == 0) return ADC_OK;
    const int R = tile_rows(d, sizeof(T));
    k_tuple_merge<T><<<tile_grid(n, R), 256, (size_t)R * d.Dp * sizeof(T), s>>>(
        reinterpret_cast<const T *>(set), static_cast<T *>(y), d, n, R, acc);
    return check_launch();
}

static adc_status split(adc_dtype dt, const TupleDesc &d, int64_t n, const void *x, char *set, cudaStream_t s) {
    return dt == ADC_F64 ? split_t<double>(d, n, x, set, s) : split_t<float>(d, n, x, set, s);
}
static adc_status merge(adc_dtype dt, const TupleDesc &d, int64_t n, const char *set, void *y, int acc,
                        cudaStream_t s) {
    return dt == ADC_F64 ? merge_t<double>(d, n, set, y, acc, s) : merge_t<float>(d, n, set, y, acc, s);
}

// Block c's array within a plane set.
static char *plane_ptr(char *set, const TLayout &L, int c, adc_dtype dt) {
    return set + (size_t)L.plane[c] * (dt == ADC_F64 ? 8 : 4);
}

adc_status tscan_fwd_rows(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *x, void *y, void *ws,
                          cudaStream_t s) {
    if (k == 1) return scan_fwd(ops[0], dt, n, x, y, ws, s);  // one block: the rows are its elements
    if (uniform_scalar(k, ops)) return vscan_fwd(ops[0], dt, n, k, x, y, ws, s);
    if (uniform_elem(k, ops)) return n > 0 ? velem_fwd(ops[0], dt, n, k, x, y, ws, s) : ADC_OK;
    char *w = static_cast<char *>(ws);
    const TLayout L = tlayout(k, ops, dt, n, true);
    const TupleDesc d = tdesc(k, ops, L);
    char *xs = w + L.sets[0], *ys = w + L.sets[1];
    adc_status st = split(dt, d, n, x, xs, s);
    if (st != ADC_OK) return st;
    const void *xp[kMaxTupleBlocks];
    void *yp[kMaxTupleBlocks];
    for (int c = 0; c < k; ++c) {
        xp[c] = plane_ptr(xs, L, c, dt);
        yp[c] = plane_ptr(ys, L, c, dt);
    }
    if ((st = fwd_blocks(k, ops, dt, n, xp, yp, w, L, s)) != ADC_OK) return st;
    return merge(dt, d, n, ys, y, 0, s);
}

adc_status tscan_vjp_rows(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *x, const void *y,
                          const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s) {
    if (k == 1) return scan_vjp(ops[0], dt, n, x, y, ybar, xbar, accumulate, ws, s);
    if (uniform_scalar(k, ops)) return vscan_vjp(ops[0], dt, n, k, x, y, ybar, xbar, accumulate, ws, s);
    if (uniform_elem(k, ops)) return n > 0 ? velem_vjp(ops[0], dt, n, k, x, y, ybar, xbar, accumulate, ws, s) : ADC_OK;
    char *w = static_cast<char *>(ws);
    const TLayout L = tlayout(k, ops, dt, n, true);
    const TupleDesc d = tdesc(k, ops, L);
    char *xs = w + L.sets[0], *ys = w + L.sets[1], *ybs = w + L.sets[2], *xbs = w + L.sets[3];
    bool all_add = true;
    for (int c = 0; c < k; ++c) all_add = all_add && ops[c] == ADC_OP_ADD;
    adc_status st;
    if (!all_add) {  // the + rule reads neither x nor y
        if ((st = split(dt, d, n, x, xs, s)) != ADC_OK) return st;
        if ((st = split(dt, d, n, y, ys, s)) != ADC_OK) return st;
    }
    if ((st = split(dt, d, n, ybar, ybs, s)) != ADC_OK) return st;
    const void *xp[kMaxTupleBlocks], *yp[kMaxTupleBlocks], *ybp[kMaxTupleBlocks];
    void *xbp[kMaxTupleBlocks];
    for (int c = 0; c < k; ++c) {
        xp[c] = plane_ptr(xs, L, c, dt);
        yp[c] = plane_ptr(ys, L, c, dt);
        ybp[c] = plane_ptr(ybs, L, c, dt);
        xbp[c] = plane_ptr(xbs, L, c, dt);
    }
    if ((st = vjp_blocks(k, ops, dt, n, xp, yp, ybp, xbp, 0, w, L, s)) != ADC_OK) return st;
    return merge(dt, d, n, xbs, xbar, accumulate, s);
}

}  // namespace adc
