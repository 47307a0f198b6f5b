/*
 * libadcomb -- reverse-mode AD of reduce, scan and reduce-by-index on GB300.
 *
 * C ABI over hand-written sm_103a CUDA kernels.  Every entry point follows a
 * definition of "Reverse-Mode AD of Reduce-by-Index and Scan in Futhark"
 * (arXiv 2310.03568); the citation is given per function.  "vjp" is the
 * paper's vector-Jacobian product (Sec. 2.2): given the adjoint of the result,
 * return the adjoint of the inputs.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  Pointers.  Every array argument is a DEVICE pointer on the current CUDA
 *    device, owned by the caller.  The library never allocates, frees or
 *    synchronises (except adc_check_device_error, which says so); all work is
 *    queued asynchronously on `stream` (a cudaStream_t passed as void*, NULL
 *    means the legacy default stream).  Arrays must be 16-byte aligned.
 *  Element layout.  fp32 (ADC_F32) or fp64 (ADC_F64) as chosen by `dtype`.
 *    Tuple operators use AoS:
 *      ADC_OP_LIN : element (b, c), the function x -> b + c*x; the operator is
 *                   (b1,c1) . (b2,c2) = (b2 + c2*b1, c2*c1)        (Fig. 8, linFnComp)
 *      ADC_OP_MM2 : element (a, b, c, d) = row-major [[a, b], [c, d]];
 *                   X . Y = X * Y                                  (Fig. 8, matMul2x2)
 *    so an element is 1, 2 or 4 scalars ("arity" below).
 *  Keys.  int32; keys outside [0, m) are ignored (Sec. 4) and their values
 *    receive adjoint 0 (Fig. 4).
 *  Workspace.  `ws` is caller-owned device scratch of at least
 *    adc_workspace_bytes(...) bytes; the library zeroes the parts it needs
 *    inside each call (cudaMemsetAsync).  One workspace must not be used by
 *    two calls that may run concurrently.
 *  Saved residuals.  `saved` is caller-owned device memory of at least
 *    adc_saved_bytes(...) bytes, written by a *_fwd call and read by the
 *    matching *_vjp call (the "primal trace" of Sec. 2.2).  Its content is
 *    listed per operator below.
 *  accumulate.  0: the adjoint output is overwritten; 1: the contribution is
 *    added to it (the paper's "+=", Eq. 1).
 *  Errors.  Status codes only; nothing is thrown across the ABI.  Argument
 *    errors are detected on the host before anything is queued.  Device-side
 *    waits are bounded; a wait that expires records ADC_ERR_TIMEOUT in the
 *    workspace, read back by adc_check_device_error.
 *  Edge cases.  n = 0 is valid: a reduce returns the neutral element, a
 *    histogram equals hist0 (or the neutral element), nothing is written to
 *    adjoints of length 0.
 */
#ifndef ADCOMB_H
#define ADCOMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADC_OP_ADD = 0,   /* +                                   */
    ADC_OP_MUL = 1,   /* *  (with zero counting, Fig. 3)     */
    ADC_OP_MIN = 2,   /* min (lifted with the argmin index)  */
    ADC_OP_MAX = 3,   /* max (lifted with the argmax index)  */
    ADC_OP_LIN = 4,   /* linFnComp on (b, c) pairs           */
    ADC_OP_MM2 = 5,   /* 2x2 matrix product                  */
    ADC_OP_SOP = 6,   /* sumOfProd on (p, s) pairs: (p1,s1).(p2,s2) = (p1+p2+s1*s2, s1+s2),
                         associative, commutative and invertible (Sec. 3.3); reduce and
                         reduce_by_index only                                              */
    ADC_OP_MM3 = 7,   /* 3x3 matrix product, row-major (9 elements); reduce and scan      */
    ADC_OP_MM5 = 8    /* 5x5 matrix product, row-major (25 elements); reduce and scan     */
} adc_op;

typedef enum { ADC_F32 = 0, ADC_F64 = 1 } adc_dtype;

typedef enum {
    ADC_OK = 0,
    ADC_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, negative size, bad enum      */
    ADC_ERR_UNSUPPORTED = 2,  /* operator not defined for this combinator (e.g. MM2 histogram) */
    ADC_ERR_WORKSPACE = 3,    /* workspace or saved buffer smaller than required      */
    ADC_ERR_CUDA = 4,         /* a CUDA call or kernel launch failed                  */
    ADC_ERR_TIMEOUT = 5       /* a bounded device-side wait expired                   */
} adc_status;

typedef enum { ADC_REDUCE = 0, ADC_SCAN = 1, ADC_HIST = 2 } adc_kind;

/* Human-readable name of a status code (static string). */
const char *adc_status_string(adc_status s);

/* Library version string (static). */
const char *adc_version(void);

/*
 * Bytes of workspace / saved residuals required by the given call shape.
 * m is ignored for reduce and scan.  Returns 0 for unsupported combinations
 * (the entry point then reports ADC_ERR_UNSUPPORTED).
 */
size_t adc_workspace_bytes(adc_kind kind, adc_op op, adc_dtype dtype, int64_t n, int64_t m);
size_t adc_saved_bytes(adc_kind kind, adc_op op, adc_dtype dtype, int64_t n, int64_t m);

/* ---------------------------------------------------------------- reduce --
 * y = reduce (.) e [x_0 .. x_{n-1}]                              (Sec. 3.1)
 *   x     : [n] elements (arity per op)          y : one element
 *   saved : ADD -- unused
 *           MIN/MAX -- int32 k, the index of the selected element, lowest
 *                   index among equal values, n if none     (Sec. 3.2.2)
 *           MUL -- int32 n0 (number of zeros) then one scalar y>0, the product
 *                  of the non-zeros (Fig. 3's lifted primal)
 *           LIN/MM2/MM3/MM5 -- per-tile exclusive prefix and suffix partials used
 *                  by the general rule (Fig. 2)
 *           SOP -- unused (the invertible-operator rule needs only x and y)
 *   ops: ADD, MUL, MIN, MAX, LIN, MM2, MM3, MM5, SOP.  MIN/MAX need n < 2^31.
 */
adc_status adc_reduce_fwd(adc_op op, adc_dtype dtype, int64_t n, const void *x, void *y,
                          void *saved, void *ws, size_t ws_bytes, void *stream);

/*
 * xbar (+)= d y / d x ^T ybar                                     (Sec. 3)
 *   ADD     : xbar_i = ybar                                      (Sec. 3.2.1)
 *   MIN/MAX : xbar_k = ybar at the saved index k, 0 elsewhere    (Sec. 3.2.2)
 *   MUL     : three-case rule of Fig. 3 (division by x_i when there is no zero)
 *   LIN/MM2 : xbar_i = d(l_i . x_i . r_i)/dx_i ybar with l_i, r_i the exclusive
 *             prefix / suffix (Eq. red-adj, Fig. 2); for MM2 xbar_i = l_i^T ybar r_i^T
 *   MM3/MM5 : the same rule for 3x3 / 5x5 matrices
 *   SOP     : invertible-operator rule (Sec. 3.3): b_i = y (.)^-1 x_i, then
 *             xbar_i = d(b_i . x)/dx at x_i ybar = (ybar.p, ybar.p * (y.s - x_i.s) + ybar.s);
 *             y is required (the fwd call's output)
 *   x, y and saved are the fwd call's input, output and residuals; ybar is one
 *   element in device memory.
 */
adc_status adc_reduce_vjp(adc_op op, adc_dtype dtype, int64_t n, const void *x, const void *y,
                          const void *saved, const void *ybar, void *xbar, int accumulate,
                          void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ scan --
 * Inclusive scan y_i = x_0 . x_1 . ... . x_i                      (Sec. 5.1)
 *   x, y : [n] elements.  ops: ADD, MUL, MIN, MAX (running extremum, the
 *   earlier element wins ties), LIN, MM2, MM3, MM5, SOP.
 */
adc_status adc_scan_fwd(adc_op op, adc_dtype dtype, int64_t n, const void *x, void *y,
                        void *ws, size_t ws_bytes, void *stream);

/*
 * xbar (+)= d y / d x ^T ybar by the rule of Fig. 7: the backward linear
 * recurrence lambda_i = ybar_i + c_{i+1} lambda_{i+1},
 * c_{i+1} = d(y_i . x_{i+1})/d y_i, solved by one reverse scan of linear-function
 * composition, fused with the map xbar_i = d(y_{i-1} . x_i)/d x_i lambda_i
 * (y_{-1} = e).  The Jacobians are block-diagonal with equal blocks (RBDS,
 * Sec. 5.3.4): a scalar c for ADD/MUL/LIN, M_{i+1}^T for MM2/MM3/MM5; for
 * MIN/MAX the scalar c_{i+1} = [y_i selected] is 0 or 1 and
 * xbar_i = [x_i selected] lambda_i (the general arity-1 rule); both are read
 * off y (x_i is selected exactly when y_i differs from y_{i-1}), so MIN/MAX
 * do not read x, although it must be passed.  SOP takes the
 * general arity-2 rule: c_{i+1} = [[1, s(x_{i+1})], [0, 1]] (not block-redundant),
 * composed as the single corner entry because unit upper-triangular matrices
 * multiply by adding it; xbar_i = (lambda.p, s(y_{i-1}) lambda.p + lambda.s).
 *   x, y : the fwd call's input and output; ybar, xbar : [n] elements.
 */
adc_status adc_scan_vjp(adc_op op, adc_dtype dtype, int64_t n, const void *x, const void *y,
                        const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes,
                        void *stream);

/*
 * adc_scan_fwd, for callers that cannot allocate device memory -- for example
 * code running inside an allocator or memory-pool callback (where cudaMalloc
 * would re-enter the allocator), or a plugin handed only fixed input and
 * output buffers.  The paper has no counterpart: this is a packaging of the
 * same scan kernel whose look-back scratch lives in a file-scope device array
 * of 4 MiB held by every GPU that loads the library until the process exits.
 * Every operator adc_scan_fwd accepts (ADD, MUL, MIN, MAX, LIN, MM2, SOP, MM3,
 * MM5), with the same layouts and results; nothing is allocated or freed.
 *   Limit : n must satisfy adc_workspace_bytes(ADC_SCAN, op, dtype, n, 0) <= 4 MiB
 *           (about 1.0e9 fp32 + elements, 2.6e8 fp32 *, 8.9e7 fp32 lin,
 *           1.6e7 fp32 mm2, 8.3e6 fp64 mm2); larger n returns
 *           ADC_ERR_WORKSPACE before any work is queued.  An operator code
 *           outside the enum returns ADC_ERR_INVALID_ARG.
 *   Set-up: the first call on a device, with that device current, looks up the
 *           array's device address; make that first call before capturing a
 *           stream.  The address belongs to the device's context: after
 *           cudaDeviceReset the next call finds a new context id and looks the
 *           address up again (a set-up call again, so again not under capture).
 *   Sharing: all calls on a device use the same array, which keeps the last
 *           call's contents; each call clears what must start at zero.  Calls
 *           that may overlap on the GPU race and must not be issued.
 *   A bounded device wait that expires leaves y incomplete; this entry point
 *   cannot report it (it does not synchronise).
 */
adc_status adc_scan_fwd_noalloc(adc_op op, adc_dtype dtype, int64_t n, const void *x, void *y,
                                void *stream);

/* ------------------------------------------------------- reduce_by_index --
 * hist = reduce_by_index hist0 (.) e keys vals                    (Sec. 4)
 *   keys : [n] int32, vals : [n] elements, hist0 : [m] elements or NULL for the
 *   neutral element, hist : [m] elements (output).
 *   saved : ADD -- unused
 *           MIN/MAX -- int32 is[m]: per bin the index of the selected value
 *                   (lowest index on ties), n when the bin is empty or hist0
 *                   won (hist0 wins ties)             (Sec. 4.2.2, Fig. 5)
 *           MUL -- int32 n0[m] zero counts, then p[m] products of the non-zeros
 *                   (Sec. 4.2.3)
 *           SOP -- unused (the vjp reads hist)
 *           LIN -- for m <= 2047 (fp32) / 1023 (fp64): per (bin, input chunk) the exclusive
 *                   prefix and suffix of the bin's fold across chunks, and
 *                   the bin totals (the chunk-local stable sort is redone in
 *                   the vjp); for larger m: the stable sort permutation, the
 *                   sorted keys and the sorted values (general rule, Fig. 4)
 *   ops: ADD, MUL, MIN, MAX, LIN, SOP (LIN is not commutative: the fold follows
 *   the index order within each bin, computed through a stable sort).  MM2 is
 *   ADC_ERR_UNSUPPORTED, and so are MM3 and MM5.  Requires 1 <= m < 2^31 and n < 2^31.
 *   ADD and SOP keep no residuals (saved may be NULL).
 *   saved == NULL (MUL, MIN, MAX only) computes the ORIGINAL, un-lifted primal
 *   instead -- the plain product per bin with zeros included, or the plain
 *   min/max value -- and keeps no residuals, so no vjp can follow.  This is the
 *   program whose time the AD overhead of Sec. 6.1.4 is measured against.
 */
adc_status adc_hist_fwd(adc_op op, adc_dtype dtype, int64_t n, int64_t m, const int32_t *keys,
                        const void *vals, const void *hist0, void *hist, void *saved, void *ws,
                        size_t ws_bytes, void *stream);

/*
 * valsbar (+)= d hist / d vals ^T histbar and, when hist0bar is not NULL,
 * hist0bar (+)= d hist / d hist0 ^T histbar.
 *   ADD     : valsbar_i = histbar[k_i]                           (Sec. 4.2.1)
 *   MIN/MAX : valsbar[is[j]] = histbar[j]                        (Fig. 5)
 *   MUL     : per-bin zero-count rule                            (Sec. 4.2.3)
 *   LIN     : sorted segmented forward and reverse scans, then
 *             d(l_i . v_i . r_i)/dv_i histbar[k_i], scattered back (Fig. 4)
 *   SOP     : invertible-operator rule per bin (Sec. 3.3, 4): with y = hist[k_i],
 *             valsbar_i = (hb.p, hb.p * (y.s - v_i.s) + hb.s), hb = histbar[k_i];
 *             hist0bar likewise with hist0 in place of v_i.  Needs vals and hist.
 *   hist and saved are the fwd call's output and residuals.
 */
adc_status adc_hist_vjp(adc_op op, adc_dtype dtype, int64_t n, int64_t m, const int32_t *keys,
                        const void *vals, const void *hist0, const void *hist, const void *saved,
                        const void *histbar, void *valsbar, void *hist0bar, int accumulate,
                        void *ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------------------- batched --
 * Many independent instances of  loss = sum_j scan(+)(hist)_j  with
 * hist = reduce_by_index (replicate m 0) (op) keys vals, op in {ADD, MAX}
 * (Sec. 4's definition with an all-zero initial histogram, Sec. 5.1's scan and a
 * +-reduce), evaluated for all instances together in a few persistent launches
 * instead of several launches per instance.  The vjp chains the specialised
 * rules: the adjoint of the sum is a broadcast (Sec. 3.2.1), of the +-scan a
 * reverse +-scan (Sec. 5.3.1), then the gather (Sec. 4.2.1) or the argmax
 * scatter (Fig. 5).
 *
 * Instances are described by adc_instance records.  Keys and values of all
 * instances are concatenated (instance i owns [val_off, val_off + n)); bins
 * likewise ([bin_off, bin_off + m) of hist / scan / is / histbar).  Work is cut
 * into adc_work items (an instance's element range) by adc_batched_plan on the
 * host; the device copy of both tables is passed to the kernels.
 */
typedef struct {
    int64_t n;        /* values of the instance (< 2^31)                        */
    int64_t m;        /* bins (1 <= m < 2^31)                                   */
    int64_t val_off;  /* offset of its first key / value                        */
    int64_t bin_off;  /* offset of its first bin                                */
    int32_t op;       /* ADC_OP_ADD or ADC_OP_MAX                                */
    int32_t pad;
} adc_instance;

typedef struct {
    int32_t inst;     /* instance index                                         */
    int32_t pad;
    int64_t start;    /* first element, relative to the instance                */
    int64_t len;      /* number of elements                                     */
} adc_work;

/*
 * Host-only planning: cuts every instance into items of at most `chunk`
 * elements (largest instances first).  Writes up to `capacity` items to
 * `items` (host memory, may be NULL to count) and returns the number of items,
 * or -1 on invalid arguments.
 */
int64_t adc_batched_plan(const adc_instance *desc, int32_t count, int64_t chunk, adc_work *items,
                         int64_t capacity);

/* Workspace bytes for the batched calls (total_bins = sum of m). */
size_t adc_batched_workspace_bytes(int32_t count, int64_t total_bins);

/*
 * Forward: hist (fp32, [total_bins]), scan (fp32, [total_bins], the inclusive
 * +-scan of each instance's histogram), is (int32, [total_bins]: for MAX
 * instances the selected element's index within the instance, n when the zero
 * initial value won or the bin is empty; unused for ADD), loss_parts (fp32,
 * [count]) and loss (fp32, one value).  desc and items are DEVICE copies.
 * smem_bins: shared-memory table size per block in bins (the instances with
 * more bins use global atomics); 0 picks the default.
 */
adc_status adc_batched_hist_scan_fwd(const adc_instance *desc, int32_t count, const adc_work *items,
                                     int64_t n_items, int64_t total_bins, const int32_t *keys,
                                     const float *vals, float *hist, float *scan, int32_t *is,
                                     float *loss_parts, float *loss, int32_t smem_bins, void *ws,
                                     size_t ws_bytes, void *stream);

/*
 * vjp w.r.t. the values given the loss adjoint (one fp32 value in device
 * memory): valsbar (fp32, [total values]); histbar (fp32, [total_bins]) receives
 * the histogram adjoints on the way.  is comes from the forward call.
 */
adc_status adc_batched_hist_scan_vjp(const adc_instance *desc, int32_t count, const adc_work *items,
                                     int64_t n_items, int64_t total_bins, const int32_t *keys,
                                     const int32_t *is, const float *loss_bar, float *histbar,
                                     float *valsbar, void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------- diagnostics --
 * Waits for `stream`, reads the workspace's device error word and returns
 * ADC_OK or the recorded error (ADC_ERR_TIMEOUT).  This call synchronises.
 */
/* ----------------------------------------------------- vectorised operators --
 * reduce, scan and reduce_by_index whose operator is map2 (.) over rows of d
 * elements, (.) in ADD, MUL, MIN, MAX (Sec. 3.2 "Vectorized Operators": the
 * Irwim rule; Sec. 5.3: the Iswim rule; the same interchange for
 * reduce_by_index).  Computed as the rules rewrite them: d column
 * combinators, each following its operator's specialised scalar rule (zero
 * counting, lowest-index argmin, ...).  reduce, scan, and reduce_by_index
 * with ADD (and fp32 MIN / MAX) while the [m][d] table fits one block's
 * shared memory run on the row-major rows where they lie; the other
 * reduce_by_index cases transpose the operands to [d][n] / [d][m], run the
 * scalar entry point's kernels per column and transpose the results back.
 * Arrays are row-major and 16-byte aligned; 1 <= d <= 64.
 *   vreduce : x [n][d] -> y [d]; saved = d column residuals (adc_vsaved_bytes)
 *   vscan   : x [n][d] -> y [n][d]; the vjp reads ybar [n][d] and, except for
 *             ADD, y (the MIN / MAX selections come from y alone) and x (MUL);
 *             x and y must still be passed for every operator but ADD
 *   vhist   : keys [n], vals [n][d], hist0 [m][d] or NULL -> hist [m][d];
 *             saved == NULL computes the original primal (MUL, MIN, MAX)
 * The workspace (adc_vworkspace_bytes) holds per-block partial states, or
 * for the transposed cases the planes and one scalar workspace per column;
 * a timeout in any column is reported by adc_check_device_error on this
 * workspace.  Other operators: ADC_ERR_UNSUPPORTED.
 */
size_t adc_vworkspace_bytes(adc_kind kind, adc_op op, adc_dtype dtype, int64_t n, int64_t m, int64_t d);
size_t adc_vsaved_bytes(adc_kind kind, adc_op op, adc_dtype dtype, int64_t n, int64_t m, int64_t d);
adc_status adc_vreduce_fwd(adc_op op, adc_dtype dtype, int64_t n, int64_t d, const void *x, void *y, void *saved,
                           void *ws, size_t ws_bytes, void *stream);
adc_status adc_vreduce_vjp(adc_op op, adc_dtype dtype, int64_t n, int64_t d, const void *x, const void *y,
                           const void *saved, const void *ybar, void *xbar, int accumulate, void *ws,
                           size_t ws_bytes, void *stream);
adc_status adc_vscan_fwd(adc_op op, adc_dtype dtype, int64_t n, int64_t d, const void *x, void *y, void *ws,
                         size_t ws_bytes, void *stream);
adc_status adc_vscan_vjp(adc_op op, adc_dtype dtype, int64_t n, int64_t d, const void *x, const void *y,
                         const void *ybar, void *xbar, int accumulate, void *ws, size_t ws_bytes, void *stream);
adc_status adc_vhist_fwd(adc_op op, adc_dtype dtype, int64_t n, int64_t m, int64_t d, const int32_t *keys,
                         const void *vals, const void *hist0, void *hist, void *saved, void *ws, size_t ws_bytes,
                         void *stream);
adc_status adc_vhist_vjp(adc_op op, adc_dtype dtype, int64_t n, int64_t m, int64_t d, const int32_t *keys,
                         const void *vals, const void *hist0, const void *hist, const void *saved,
                         const void *histbar, void *valsbar, void *hist0bar, int accumulate, void *ws,
                         size_t ws_bytes, void *stream);

/* ----------------------------------------------------------- tuple scans --
 * Scans whose element is a tuple of k blocks that combine independently
 * (Sec. 5.3.3, block-diagonal sparsity): block c is an element of operator
 * ops[c] (an adc_op code, arity a_c: 1 for ADD/MUL/MIN/MAX, 2 LIN/SOP, 4 MM2,
 * 9 MM3, 25 MM5) and the tuple operator applies ops[c] to block c alone, so
 * every step's Jacobian is block-diagonal with k blocks of a_c x a_c.  The vjp
 * is the BDS rule: k reverse scans, block c by its own operator's rule (the
 * same results as adc_scan_fwd / adc_scan_vjp on that block).  1 <= k <= 64;
 * ops is a host array of k codes.
 *
 * Rows layout (adc_tscan_fwd / _vjp): x, y, ybar, xbar are [n][D] row-major,
 * D = sum a_c <= 64, block c at columns [sum_{b<c} a_b, + a_c) of every row;
 * 16-byte aligned.  The rows are split into per-block planes in the
 * workspace, scanned, and merged back (k = 1: scanned in place).  In the vjp
 * x and y may be NULL when every block is ADD.
 *
 * Blocks layout (adc_tscan_fwd_blocks / _vjp_blocks): the tuple of arrays --
 * x, y, ybar, xbar are host arrays of k device pointers, entry c an [n][a_c]
 * array (16-byte aligned); nothing is copied.  In the vjp, x and y (or their
 * entries for ADD blocks) may be NULL.
 *
 * Workspace: adc_tscan_workspace_bytes(k, ops, dtype, n, rows) (rows = 1 for
 * the rows layout, 0 for blocks); it holds one scan workspace per block (and
 * the planes for rows); a timeout in any block is reported by
 * adc_check_device_error on it.  Returns 0 for invalid arguments.
 * Errors: ADC_ERR_INVALID_ARG for k, codes, D or arrays out of range;
 * ADC_ERR_WORKSPACE when ws_bytes is too small.
 */
size_t adc_tscan_workspace_bytes(int32_t k, const int32_t *ops, adc_dtype dtype, int64_t n, int32_t rows);
adc_status adc_tscan_fwd(int32_t k, const int32_t *ops, adc_dtype dtype, int64_t n, const void *x, void *y,
                         void *ws, size_t ws_bytes, void *stream);
adc_status adc_tscan_vjp(int32_t k, const int32_t *ops, adc_dtype dtype, int64_t n, const void *x,
                         const void *y, const void *ybar, void *xbar, int accumulate, void *ws,
                         size_t ws_bytes, void *stream);
adc_status adc_tscan_fwd_blocks(int32_t k, const int32_t *ops, adc_dtype dtype, int64_t n,
                                const void *const *x, void *const *y, void *ws, size_t ws_bytes,
                                void *stream);
adc_status adc_tscan_vjp_blocks(int32_t k, const int32_t *ops, adc_dtype dtype, int64_t n,
                                const void *const *x, const void *const *y, const void *const *ybar,
                                void *const *xbar, int accumulate, void *ws, size_t ws_bytes,
                                void *stream);

/*
 * dst = transpose(src) for a rows x cols row-major matrix of dtype elements
 * (the layout change of the rewrites above), through shared-memory tiles.
 * src and dst must not overlap.  Asynchronous on the stream.
 */
adc_status adc_transpose(adc_dtype dtype, int64_t rows, int64_t cols, const void *src, void *dst, void *stream);

adc_status adc_check_device_error(const void *ws, size_t ws_bytes, void *stream);

/*
 * Bound on device-side spin iterations (each iteration polls once and sleeps
 * about 100 ns); default 1 << 22.  Values < 1 restore the default.
 */
void adc_set_spin_limit(int64_t iterations);

/*
 * Fault-injection hook for tests: the scan tile with this claim index
 * publishes nothing, so every tile that looks back across it must give up
 * after the spin limit and report ADC_ERR_TIMEOUT.  -1 (the default) disables.
 */
void adc_debug_set_stall_tile(int64_t tile);

/*
 * Test hook: scan engine selection -- 0 automatic (range-partitioned for large
 * n, per-tile look-back otherwise), 1 per-tile look-back only, 2 range-
 * partitioned wherever it applies, 3 range-partitioned with the range staged
 * in shared memory by bulk (TMA) copies, 4 per-tile look-back with each
 * block's tile staged in shared memory by bulk copies, 5 the range engine with
 * 16 bytes of each array per thread per tile, 6 the bulk-staged segment forms
 * of the q x q matrix scans (ADC_OP_MM3 / ADC_OP_MM5; also what 0 picks for
 * them, while 1 and 2 pick their register forms).  Other values restore 0.
 * In the fault-injection hook
 * above, the "tile" of the range engines is a range.
 */
void adc_debug_set_scan_engine(int engine);

/*
 * Tuning hook: tiles per range of the range-partitioned scan engine.  0 (the
 * default) lets the library choose; a positive value launches
 * ceil(tiles / value) ranges (as long as no range would exceed the engine's
 * per-block limit).  Results do not depend on it beyond rounding order.
 */
void adc_debug_set_scan_range_tiles(int tiles);

/*
 * Tuning hook: 1 makes every block of the range-partitioned scan engine
 * prefetch its range's input into L2 (bulk prefetches) when it starts; 0 (the
 * default) does not.  Results do not depend on it.
 */
void adc_debug_set_scan_prefetch(int on);

/*
 * Tuning hook: elements per thread and step of the batched histogram launch
 * (1, 4 or 8; anything else selects the default, 4).  A step's key and value
 * loads are all issued before its atomic updates.  Results do not depend on it
 * beyond the order of the + atomics.
 */
void adc_debug_set_batched_items(int items);

/*
 * Test hook: force the forward histogram strategy of ADD/MUL/MIN/MAX
 * (0: per-warp shared-memory copies, 1: one shared-memory copy per block,
 * 2: global atomics, 3: per-thread shared-memory tables, 4: partition by bin
 * range into shared-memory-sized buckets, 5: lifted fp32 min/max split over
 * 2-4 block tables, 6: lifted fp32 min/max spread over the shared memory of a
 * 2-8 block cluster, 7: lifted fp32 min/max by per-block value tables and an
 * index pass, 8: lifted fp32 min/max by pairs of blocks holding half the bins
 * as value and index tables, never chosen automatically) where the histogram
 * fits it; -1
 * (default) chooses automatically from m and the operator.  The choice also
 * applies to the original primal (saved == NULL).
 */
void adc_debug_force_hist_strategy(int strategy);

/*
 * Tuning hook: form of the min/max reduce-by-index vjp -- 0 automatic (the
 * bitmap form when bins are sparse, 8m > n; else a zero-fill plus a scatter
 * of the m adjoints), 1 a gather pass over the keys (is[k_i] == i), 2 the
 * zero-fill + scatter, 3 a bitmap of the selected elements (one bit each, set
 * from is[]) and one streaming pass that gathers only for set bits.  Results
 * are identical.
 */
void adc_debug_set_sel_vjp_form(int form);

#ifdef __cplusplus
}
#endif

#endif /* ADCOMB_H */
