// Host-side internals shared by the libadcomb translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/adcomb.h"

namespace adc {

struct DevCtl;

// Workspace header, zeroed by every entry point before it queues work:
// [0] device error word, [4 + 4*slot] one counter per launch of the call.
constexpr size_t kWsHeader = 256;
constexpr int kMaxSlots = 48;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

DevCtl make_ctl(void *ws, int slot);
long long spin_limit();  // the polling bound of every device-side wait (adc_set_spin_limit)
inline unsigned *counter_slot(void *ws, int slot) {
    return reinterpret_cast<unsigned *>(static_cast<char *>(ws) + 4 + 4 * slot);
}
int num_sms();

// Returns ADC_ERR_CUDA if the last launch failed.
adc_status check_launch();

inline int arity(adc_op op) {
    switch (op) {
    case ADC_OP_LIN:
    case ADC_OP_SOP: return 2;
    case ADC_OP_MM2: return 4;
    case ADC_OP_MM3: return 9;
    case ADC_OP_MM5: return 25;
    default: return 1;
    }
}
inline size_t elem_bytes(adc_op op, adc_dtype dt) { return (size_t)arity(op) * (dt == ADC_F64 ? 8 : 4); }

// scan.cu
size_t scan_ws_bytes(adc_op op, adc_dtype dt, int64_t n);
adc_status scan_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *ws, cudaStream_t s);
adc_status scan_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *ybar,
                    void *xbar, int accumulate, void *ws, cudaStream_t s);

// reduce.cu
size_t reduce_ws_bytes(adc_op op, adc_dtype dt, int64_t n);
size_t reduce_saved_bytes(adc_op op, adc_dtype dt, int64_t n);
adc_status reduce_fwd(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *saved, void *ws,
                      cudaStream_t s);
adc_status reduce_vjp(adc_op op, adc_dtype dt, int64_t n, const void *x, const void *y, const void *saved,
                      const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s);

// hist.cu
size_t hist_ws_bytes(adc_op op, adc_dtype dt, int64_t n, int64_t m);
size_t hist_saved_bytes(adc_op op, adc_dtype dt, int64_t n, int64_t m);
adc_status hist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s);
adc_status hist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, const void *hist, const void *saved, const void *histbar,
                    void *valsbar, void *hist0bar, int accumulate, void *ws, cudaStream_t s);

// sort.cu (general reduce_by_index through a stable radix sort)
size_t histgen_ws_bytes(adc_dtype dt, int64_t n, int64_t m);
size_t histgen_saved_bytes(adc_dtype dt, int64_t n, int64_t m);
adc_status histgen_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                       const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s);
adc_status histgen_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                       const void *hist0, const void *hist, const void *saved, const void *histbar,
                       void *valsbar, void *hist0bar, int accumulate, void *ws, cudaStream_t s);

size_t excl_scan_i32_region(int64_t n);
adc_status excl_scan_i32(const int32_t *in, int32_t *out, int64_t n, void *ws, int slot, void *region,
                         cudaStream_t s);

// hist_lin.cu (general reduce_by_index, linFnComp, m <= 2047 fp32 / 1023 fp64:
// hierarchical stable sort)
bool linh_applicable(adc_dtype dt, int64_t m);
size_t linh_ws_bytes(adc_dtype dt, int64_t n, int64_t m);
size_t linh_saved_bytes(adc_dtype dt, int64_t n, int64_t m);
adc_status linh_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                    void *hist, void *saved, void *ws, cudaStream_t s);
adc_status linh_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *saved,
                    const void *histbar, void *valsbar, void *hist0bar, int accumulate, cudaStream_t s);
// hist.cu: the strategy forced by the test hook (-1: automatic); for LIN, 2
// forces the global radix-sort path
int hist_forced_strategy();

// vector.cu (vectorised operators: transpose + per-column scalar combinators)
adc_status transpose(adc_dtype dt, int64_t rows, int64_t cols, const void *src, void *dst, cudaStream_t s);
size_t vws_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d);
size_t vsaved_bytes(adc_kind kind, adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d);
adc_status vreduce_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *saved, void *ws,
                       cudaStream_t s);
adc_status vreduce_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *saved,
                       const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s);
adc_status vscan_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws, cudaStream_t s);
// rows of d equal lin / sumOfProd / 2x2 elements, scanned per element column
size_t velem_ws_bytes(adc_op op, adc_dtype dt, int64_t d);
adc_status velem_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, void *y, void *ws, cudaStream_t s);
adc_status velem_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                     void *xbar, int accumulate, void *ws, cudaStream_t s);
adc_status vscan_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t d, const void *x, const void *y, const void *ybar,
                     void *xbar, int accumulate, void *ws, cudaStream_t s);
adc_status vhist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys, const void *vals,
                     const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s);
adc_status vhist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, int64_t d, const int32_t *keys, const void *vals,
                     const void *hist0, const void *hist, const void *saved, const void *histbar, void *valsbar,
                     void *hist0bar, int accumulate, void *ws, cudaStream_t s);

// tuple.cu (tuple scans with block-diagonal Jacobians, Sec. 5.3.3): at most
// kMaxTupleBlocks blocks; in the rows layout at most kMaxTupleBlocks scalars a row
constexpr int kMaxTupleBlocks = 64;
size_t tscan_ws_bytes(int k, const adc_op *ops, adc_dtype dt, int64_t n, bool rows);
adc_status tscan_fwd_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x, void *const *y,
                            void *ws, cudaStream_t s);
adc_status tscan_vjp_blocks(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *const *x,
                            const void *const *y, const void *const *ybar, void *const *xbar, int accumulate, void *ws,
                            cudaStream_t s);
adc_status tscan_fwd_rows(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *x, void *y, void *ws,
                          cudaStream_t s);
adc_status tscan_vjp_rows(int k, const adc_op *ops, adc_dtype dt, int64_t n, const void *x, const void *y,
                          const void *ybar, void *xbar, int accumulate, void *ws, cudaStream_t s);

// hist_sop.cu (sumOfProd reduce_by_index, Sec. 3.3)
adc_status sop_hist_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                        void *hist, cudaStream_t s);
adc_status sop_hist_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                        const void *hist, const void *histbar, void *valsbar, void *hist0bar, int accumulate,
                        cudaStream_t s);

// hist_part.cu (reduce_by_index for tables beyond shared memory: partition by
// bin range, then per-bucket shared-memory tables)
enum PartMode { kPAdd = 0, kPMul = 1, kPMin = 2, kPMax = 3, kPPrimMul = 4, kPPrimMin = 5, kPPrimMax = 6 };
bool part_applicable(int mode, size_t s, int64_t m);
size_t part_ws_bytes(int mode, size_t s, int64_t n, int64_t m);
// Outputs: every mode writes hist (hist0 folded in); MUL also writes the
// residuals n0, p; MIN/MAX (fp32) also the selected index per bin, `is` (n if
// none, or if hist0 won).  n > 0.
adc_status part_fwd(int mode, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, void *hist, int32_t *n0, void *p, int32_t *is, void *ws, size_t ws_off,
                    cudaStream_t s);

}  // namespace adc
