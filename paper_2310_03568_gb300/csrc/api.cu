// libadcomb C ABI: argument validation, workspace checks and dispatch.
// Every entry point validates on the host, zeroes the workspace header (error
// word and launch counters) on the stream, then queues its kernels.
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace adc {

static long long g_spin_limit = 1ll << 22;
static long long g_stall_tile = -1;
int g_scan_engine = 0;
int g_scan_range_tiles = 0;
int g_scan_prefetch = 0;

long long spin_limit() { return g_spin_limit; }

DevCtl make_ctl(void *ws, int slot) {
    DevCtl c;
    c.err = static_cast<unsigned *>(ws);
    c.counter = counter_slot(ws, slot);
    c.spin_limit = g_spin_limit;
    c.stall_tile = g_stall_tile;
    c.prefetch = g_scan_prefetch;
    return c;
}

int num_sms() {
    // Host threads may call at once: the entries are atomics (every writer
    // stores the same value).
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
    int sms = cache[dev].load(std::memory_order_relaxed);
    if (sms == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 132;
        cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

adc_status check_launch() { return cudaGetLastError() == cudaSuccess ? ADC_OK : ADC_ERR_CUDA; }

}  // namespace adc

using namespace adc;

namespace {

bool valid_op(adc_op op) { return op >= ADC_OP_ADD && op <= ADC_OP_MM5; }
bool matrix_op(adc_op op) { return op == ADC_OP_MM2 || op == ADC_OP_MM3 || op == ADC_OP_MM5; }
// Operators a scan can take (sumOfProd's invertible rule is a reduce /
// reduce_by_index rule).
bool scan_op(adc_op op) { return valid_op(op); }
bool valid_dt(adc_dtype dt) { return dt == ADC_F32 || dt == ADC_F64; }
bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Array argument: NULL only when empty; 16-byte aligned otherwise.
bool arr_ok(const void *p, int64_t count) { return count == 0 || (p != nullptr && aligned(p, 16)); }
// Single-element argument: non-NULL, aligned to its scalar type.
bool one_ok(const void *p, adc_dtype dt) { return p != nullptr && aligned(p, dt == ADC_F64 ? 8 : 4); }

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

adc_status prologue(void *ws, size_t ws_bytes, size_t need, cudaStream_t s) {
    if (ws == nullptr || !aligned(ws, 256)) return ADC_ERR_INVALID_ARG;
    if (ws_bytes < need) return ADC_ERR_WORKSPACE;
    if (cudaMemsetAsync(ws, 0, kWsHeader, s) != cudaSuccess) return ADC_ERR_CUDA;
    return ADC_OK;
}

constexpr int64_t kIdxMax = 0x7fffffffll;
constexpr int64_t kMaxVecWidth = 64;  // row width d of the vectorised operators

bool vec_op(adc_op op) { return op == ADC_OP_ADD || op == ADC_OP_MUL || op == ADC_OP_MIN || op == ADC_OP_MAX; }
bool vec_ok(adc_op op, adc_dtype dt, int64_t n, int64_t d) {
    return vec_op(op) && valid_dt(dt) && n >= 0 && n < kIdxMax && d >= 1 && d <= kMaxVecWidth;
}

// Copies and checks the block operators: 1 <= k <= kMaxTupleBlocks, every one a
// scan operator; *width receives the row width sum of arities.
adc_status tuple_ops(int32_t k, const int32_t *codes, adc_dtype dt, int64_t n, adc_op *ops, int64_t *width) {
    if (k < 1 || k > kMaxTupleBlocks || codes == nullptr || !valid_dt(dt) || n < 0) return ADC_ERR_INVALID_ARG;
    int64_t w = 0;
    for (int c = 0; c < k; ++c) {
        if (codes[c] < (int32_t)ADC_OP_ADD || codes[c] > (int32_t)ADC_OP_MM5) return ADC_ERR_INVALID_ARG;
        const adc_op op = static_cast<adc_op>(codes[c]);
        if (!valid_op(op)) return ADC_ERR_INVALID_ARG;
        if (!scan_op(op)) return ADC_ERR_UNSUPPORTED;
        ops[c] = op;
        w += arity(op);
    }
    *width = w;
    return ADC_OK;
}

}  // namespace

extern "C" {

const char *adc_status_string(adc_status s) {
    switch (s) {
    case ADC_OK: return "ok";
    case ADC_ERR_INVALID_ARG: return "invalid argument";
    case ADC_ERR_UNSUPPORTED: return "unsupported operator for this combinator";
    case ADC_ERR_WORKSPACE: return "workspace or saved buffer too small";
    case ADC_ERR_CUDA: return "CUDA error";
    case ADC_ERR_TIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
    }
}

const char *adc_version(void) { return "libadcomb 0.1 (sm_103a)"; }

size_t adc_workspace_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return 0;
    switch (kind) {
    case ADC_REDUCE: return reduce_ws_bytes(op, dt, n);
    case ADC_SCAN:
        if (!scan_op(op)) return 0;
        return scan_ws_bytes(op, dt, n);
    case ADC_HIST:
        if (matrix_op(op) || m < 1 || m > kIdxMax || n > kIdxMax) return 0;
        return hist_ws_bytes(op, dt, n, m);
    default: return 0;
    }
}

size_t adc_saved_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return 0;
    switch (kind) {
    case ADC_REDUCE: return reduce_saved_bytes(op, dt, n);
    case ADC_SCAN: return scan_op(op) ? 16 : 0;  // scans keep no residuals beyond x and y
    case ADC_HIST:
        if (matrix_op(op) || m < 1 || m > kIdxMax || n > kIdxMax) return 0;
        return hist_saved_bytes(op, dt, n, m);
    default: return 0;
    }
}

adc_status adc_reduce_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *saved, void *ws,
                          size_t ws_bytes, void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return ADC_ERR_INVALID_ARG;
    if ((op == ADC_OP_MIN || op == ADC_OP_MAX) && n >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(x, n) || !one_ok(y, dt)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && op != ADC_OP_SOP && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, reduce_ws_bytes(op, dt, n), s);
    if (st != ADC_OK) return st;
    return reduce_fwd(op, dt, n, x, y, saved, ws, s);
}

adc_status adc_reduce_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *saved,
                          const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return ADC_ERR_INVALID_ARG;
    if ((op == ADC_OP_MIN || op == ADC_OP_MAX) && n >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(xbar, n) || !one_ok(ybar, dt)) return ADC_ERR_INVALID_ARG;
    if ((op == ADC_OP_MUL || op == ADC_OP_LIN || matrix_op(op) || op == ADC_OP_SOP) && !arr_ok(x, n))
        return ADC_ERR_INVALID_ARG;
    if (op == ADC_OP_SOP && !one_ok(y, dt)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && op != ADC_OP_SOP && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, reduce_ws_bytes(op, dt, n), s);
    if (st != ADC_OK) return st;
    return reduce_vjp(op, dt, n, x, y, saved, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_scan_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *ws, size_t ws_bytes,
                        void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return ADC_ERR_INVALID_ARG;
    if (!scan_op(op)) return ADC_ERR_UNSUPPORTED;
    if (!arr_ok(x, n) || !arr_ok(y, n)) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, scan_ws_bytes(op, dt, n), s);
    if (st != ADC_OK) return st;
    return scan_fwd(op, dt, n, x, y, ws, s);
}

adc_status adc_scan_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *ybar,
                        void *xbar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0) return ADC_ERR_INVALID_ARG;
    if (!scan_op(op)) return ADC_ERR_UNSUPPORTED;
    if (!arr_ok(ybar, n) || !arr_ok(xbar, n)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && (!arr_ok(x, n) || !arr_ok(y, n))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, scan_ws_bytes(op, dt, n), s);
    if (st != ADC_OK) return st;
    return scan_vjp(op, dt, n, x, y, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_hist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                        const void *hist0, void *hist, void *saved, void *ws, size_t ws_bytes, void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0 || m < 1) return ADC_ERR_INVALID_ARG;
    if (matrix_op(op)) return ADC_ERR_UNSUPPORTED;
    if (n >= kIdxMax || m >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(keys, n) || !arr_ok(vals, n) || !arr_ok(hist, m)) return ADC_ERR_INVALID_ARG;
    if (hist0 != nullptr && !aligned(hist0, 16)) return ADC_ERR_INVALID_ARG;
    // saved == NULL selects the original (un-lifted) primal for MUL/MIN/MAX
    if (op == ADC_OP_LIN && saved == nullptr) return ADC_ERR_INVALID_ARG;
    if (saved != nullptr && !aligned(saved, 16)) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, hist_ws_bytes(op, dt, n, m), s);
    if (st != ADC_OK) return st;
    return hist_fwd(op, dt, n, m, keys, vals, hist0, hist, saved, ws, s);
}

adc_status adc_hist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                        const void *hist0, const void *hist, const void *saved, const void *histbar, void *valsbar,
                        void *hist0bar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    if (!valid_op(op) || !valid_dt(dt) || n < 0 || m < 1) return ADC_ERR_INVALID_ARG;
    if (matrix_op(op)) return ADC_ERR_UNSUPPORTED;
    if (n >= kIdxMax || m >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(histbar, m) || !arr_ok(valsbar, n)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_LIN && !arr_ok(keys, n)) return ADC_ERR_INVALID_ARG;
    if ((op == ADC_OP_MUL || op == ADC_OP_SOP) && !arr_ok(vals, n)) return ADC_ERR_INVALID_ARG;
    if (op == ADC_OP_SOP && (hist == nullptr || !aligned(hist, 16))) return ADC_ERR_INVALID_ARG;
    if ((hist0 != nullptr && !aligned(hist0, 16)) || (hist0bar != nullptr && !aligned(hist0bar, 16)))
        return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && op != ADC_OP_SOP && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, hist_ws_bytes(op, dt, n, m), s);
    if (st != ADC_OK) return st;
    return hist_vjp(op, dt, n, m, keys, vals, hist0, hist, saved, histbar, valsbar, hist0bar, accumulate ? 1 : 0, ws,
                    s);
}

// ------------------------------------------------------ vectorised operators --
adc_status adc_transpose(adc_dtype dt, int64_t rows, int64_t cols, const void *src, void *dst, void *stream) {
    if (!valid_dt(dt) || rows < 0 || cols < 0) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(src, rows * cols) || !arr_ok(dst, rows * cols) || (rows * cols > 0 && src == dst))
        return ADC_ERR_INVALID_ARG;
    return transpose(dt, rows, cols, src, dst, as_stream(stream));
}

size_t adc_vworkspace_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    if (!vec_ok(op, dt, n, d)) return 0;
    if (kind == ADC_HIST && (m < 1 || m >= kIdxMax)) return 0;
    if (kind != ADC_REDUCE && kind != ADC_SCAN && kind != ADC_HIST) return 0;
    return vws_bytes(kind, op, dt, n, m, d);
}

size_t adc_vsaved_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d) {
    if (!vec_ok(op, dt, n, d)) return 0;
    if (kind == ADC_HIST && (m < 1 || m >= kIdxMax)) return 0;
    if (kind != ADC_REDUCE && kind != ADC_SCAN && kind != ADC_HIST) return 0;
    return vsaved_bytes(kind, op, dt, n, m, d);
}

adc_status adc_vreduce_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *saved,
                           void *ws, size_t ws_bytes, void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (!arr_ok(x, n * d) || !arr_ok(y, d)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_REDUCE, op, dt, n, 0, d), s);
    if (st != ADC_OK) return st;
    return vreduce_fwd(op, dt, n, d, x, y, saved, ws, s);
}

adc_status adc_vreduce_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y,
                           const void *saved, const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes,
                           void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (!arr_ok(xbar, n * d) || !arr_ok(ybar, d)) return ADC_ERR_INVALID_ARG;
    if (op == ADC_OP_MUL && !arr_ok(x, n * d)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_REDUCE, op, dt, n, 0, d), s);
    if (st != ADC_OK) return st;
    return vreduce_vjp(op, dt, n, d, op == ADC_OP_MUL ? x : nullptr, y, saved, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_vscan_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws,
                         size_t ws_bytes, void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (!arr_ok(x, n * d) || !arr_ok(y, n * d)) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_SCAN, op, dt, n, 0, d), s);
    if (st != ADC_OK) return st;
    return vscan_fwd(op, dt, n, d, x, y, ws, s);
}

adc_status adc_vscan_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y,
                         const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (!arr_ok(ybar, n * d) || !arr_ok(xbar, n * d)) return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && (!arr_ok(x, n * d) || !arr_ok(y, n * d))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_SCAN, op, dt, n, 0, d), s);
    if (st != ADC_OK) return st;
    return vscan_vjp(op, dt, n, d, x, y, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_vhist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys,
                         const void *vals, const void *hist0, void *hist, void *saved, void *ws, size_t ws_bytes,
                         void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (m < 1 || m >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(keys, n) || !arr_ok(vals, n * d) || !arr_ok(hist, m * d)) return ADC_ERR_INVALID_ARG;
    if ((hist0 != nullptr && !aligned(hist0, 16)) || (saved != nullptr && !aligned(saved, 16)))
        return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_HIST, op, dt, n, m, d), s);
    if (st != ADC_OK) return st;
    return vhist_fwd(op, dt, n, m, d, keys, vals, hist0, hist, saved, ws, s);
}

adc_status adc_vhist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys,
                         const void *vals, const void *hist0, const void *hist, const void *saved, const void *histbar,
                         void *valsbar, void *hist0bar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    if (!vec_ok(op, dt, n, d)) return vec_op(op) ? ADC_ERR_INVALID_ARG : ADC_ERR_UNSUPPORTED;
    if (m < 1 || m >= kIdxMax) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(keys, n) || !arr_ok(histbar, m * d) || !arr_ok(valsbar, n * d)) return ADC_ERR_INVALID_ARG;
    if (op == ADC_OP_MUL && !arr_ok(vals, n * d)) return ADC_ERR_INVALID_ARG;
    if ((hist0 != nullptr && !aligned(hist0, 16)) || (hist0bar != nullptr && !aligned(hist0bar, 16)))
        return ADC_ERR_INVALID_ARG;
    if (op != ADC_OP_ADD && (saved == nullptr || !aligned(saved, 16))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    adc_status st = prologue(ws, ws_bytes, vws_bytes(ADC_HIST, op, dt, n, m, d), s);
    if (st != ADC_OK) return st;
    return vhist_vjp(op, dt, n, m, d, keys, op == ADC_OP_MUL ? vals : nullptr, hist0, hist, saved, histbar, valsbar,
                     hist0bar, accumulate ? 1 : 0, ws, s);
}

// ----------------------------------------------------------- tuple scans --

size_t adc_tscan_workspace_bytes(int32_t k, const int32_t *ops, adc_dtype dt, int64_t n, int32_t rows) {
    adc_op o[kMaxTupleBlocks];
    int64_t w = 0;
    if (tuple_ops(k, ops, dt, n, o, &w) != ADC_OK) return 0;
    if (rows && w > kMaxTupleBlocks) return 0;
    return tscan_ws_bytes(k, o, dt, n, rows != 0);
}

adc_status adc_tscan_fwd(int32_t k, const int32_t *ops, adc_dtype dt, int64_t n, const void *x, void *y, void *ws,
                         size_t ws_bytes, void *stream) {
    adc_op o[kMaxTupleBlocks];
    int64_t w = 0;
    adc_status st = tuple_ops(k, ops, dt, n, o, &w);
    if (st != ADC_OK) return st;
    if (w > kMaxTupleBlocks) return ADC_ERR_INVALID_ARG;
    if (!arr_ok(x, n * w) || !arr_ok(y, n * w)) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if ((st = prologue(ws, ws_bytes, tscan_ws_bytes(k, o, dt, n, true), s)) != ADC_OK) return st;
    return tscan_fwd_rows(k, o, dt, n, x, y, ws, s);
}

adc_status adc_tscan_vjp(int32_t k, const int32_t *ops, adc_dtype dt, int64_t n, const void *x, const void *y,
                         const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes, void *stream) {
    adc_op o[kMaxTupleBlocks];
    int64_t w = 0;
    adc_status st = tuple_ops(k, ops, dt, n, o, &w);
    if (st != ADC_OK) return st;
    if (w > kMaxTupleBlocks) return ADC_ERR_INVALID_ARG;
    bool all_add = true;
    for (int c = 0; c < k; ++c) all_add = all_add && o[c] == ADC_OP_ADD;
    if (!arr_ok(ybar, n * w) || !arr_ok(xbar, n * w)) return ADC_ERR_INVALID_ARG;
    if (!all_add && (!arr_ok(x, n * w) || !arr_ok(y, n * w))) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if ((st = prologue(ws, ws_bytes, tscan_ws_bytes(k, o, dt, n, true), s)) != ADC_OK) return st;
    return tscan_vjp_rows(k, o, dt, n, x, y, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_tscan_fwd_blocks(int32_t k, const int32_t *ops, adc_dtype dt, int64_t n, const void *const *x,
                                void *const *y, void *ws, size_t ws_bytes, void *stream) {
    adc_op o[kMaxTupleBlocks];
    int64_t w = 0;
    adc_status st = tuple_ops(k, ops, dt, n, o, &w);
    if (st != ADC_OK) return st;
    if (x == nullptr || y == nullptr) return ADC_ERR_INVALID_ARG;
    for (int c = 0; c < k; ++c)
        if (!arr_ok(x[c], n) || !arr_ok(y[c], n)) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if ((st = prologue(ws, ws_bytes, tscan_ws_bytes(k, o, dt, n, false), s)) != ADC_OK) return st;
    return tscan_fwd_blocks(k, o, dt, n, x, y, ws, s);
}

adc_status adc_tscan_vjp_blocks(int32_t k, const int32_t *ops, adc_dtype dt, int64_t n, const void *const *x,
                                const void *const *y, const void *const *ybar, void *const *xbar, int accumulate,
                                void *ws, size_t ws_bytes, void *stream) {
    adc_op o[kMaxTupleBlocks];
    int64_t w = 0;
    adc_status st = tuple_ops(k, ops, dt, n, o, &w);
    if (st != ADC_OK) return st;
    if (ybar == nullptr || xbar == nullptr) return ADC_ERR_INVALID_ARG;
    for (int c = 0; c < k; ++c) {
        if (!arr_ok(ybar[c], n) || !arr_ok(xbar[c], n)) return ADC_ERR_INVALID_ARG;
        if (o[c] != ADC_OP_ADD && (x == nullptr || y == nullptr || !arr_ok(x[c], n) || !arr_ok(y[c], n)))
            return ADC_ERR_INVALID_ARG;
    }
    // + blocks read neither x nor y: hand them null arrays when none were given
    const void *xs[kMaxTupleBlocks], *ys[kMaxTupleBlocks];
    for (int c = 0; c < k; ++c) {
        xs[c] = x ? x[c] : nullptr;
        ys[c] = y ? y[c] : nullptr;
    }
    cudaStream_t s = as_stream(stream);
    if ((st = prologue(ws, ws_bytes, tscan_ws_bytes(k, o, dt, n, false), s)) != ADC_OK) return st;
    return tscan_vjp_blocks(k, o, dt, n, xs, ys, ybar, xbar, accumulate ? 1 : 0, ws, s);
}

adc_status adc_check_device_error(const void *ws, size_t ws_bytes, void *stream) {
    if (ws == nullptr || ws_bytes < kWsHeader) return ADC_ERR_INVALID_ARG;
    unsigned word = 0;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return ADC_ERR_CUDA;
    if (cudaMemcpy(&word, ws, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return ADC_ERR_CUDA;
    return word ? ADC_ERR_TIMEOUT : ADC_OK;
}

void adc_set_spin_limit(int64_t iterations) { g_spin_limit = iterations < 1 ? (1ll << 22) : iterations; }

void adc_debug_set_stall_tile(int64_t tile) { g_stall_tile = tile; }

void adc_debug_set_scan_engine(int engine) { g_scan_engine = (engine >= 0 && engine <= 6) ? engine : 0; }
void adc_debug_set_scan_range_tiles(int tiles) { g_scan_range_tiles = tiles > 0 ? tiles : 0; }
void adc_debug_set_scan_prefetch(int on) { g_scan_prefetch = on ? 1 : 0; }

}  // extern "C"
