// Batched reduce_by_index -> +-scan -> sum over many independent instances,
// forward and vjp, in a few persistent launches.
//
// Forward (per instance i, op ADD or MAX, initial histogram all zero):
//   hist_i  = reduce_by_index (replicate m_i 0) op keys_i vals_i     (Sec. 4)
//   scan_i  = scan (+) hist_i                                        (Sec. 5.1)
//   loss    = sum_i sum_j scan_i[j]                                  (Sec. 3)
// vjp: ybar of the sum is a broadcast (Sec. 3.2.1), the +-scan's adjoint a
// reverse +-scan (Sec. 5.3.1), then the gather of Sec. 4.2.1 (ADD) or the
// argmax scatter of Fig. 5 (MAX; the zero initial value wins ties).
//
// Launches: init (one block per instance) -> histogram (persistent blocks
// pulling (instance, element range) work items from an atomic counter; a
// shared-memory table when the instance's bins fit and the item is long
// enough to amortise it, global atomics otherwise) -> scan + loss (one block
// per instance, deterministic loss from per-instance partials combined in
// instance order by the last block).  Backward: reverse scan of the loss
// adjoint per instance -> per-item gather / zero-fill -> per-instance argmax
// scatter.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace adc {

constexpr int kBHistThreads = 512;
constexpr int kBScanThreads = 1024;
constexpr int32_t kDefaultSmemBins = 8192;

// Packed max key: order-preserving value bits above the inverted index, so a
// 64-bit atomicMax keeps the largest value and, among equal values, the
// smallest index (Fig. 5's lifted operator).
__device__ __forceinline__ unsigned long long bmax_key(float v, int64_t i) {
    return ((unsigned long long)ordered_key(v) << 32) | (0xffffffffu - (uint32_t)i);
}
__device__ __forceinline__ int64_t bmax_index(unsigned long long k) { return (int64_t)(0xffffffffu - (uint32_t)k); }

// Elements per thread and step of the histogram launch (1, 4 or 8; tuning hook).
static int g_batched_ipt = 4;

__global__ void k_b_init(const adc_instance *__restrict__ desc, float *__restrict__ hist,
                         unsigned long long *__restrict__ tab) {
    const adc_instance d = desc[blockIdx.x];
    for (int64_t j = threadIdx.x; j < d.m; j += blockDim.x) {
        if (d.op == ADC_OP_ADD) hist[d.bin_off + j] = 0.f;
        else tab[d.bin_off + j] = 0ull;
    }
}

// IPT elements per thread and step (e = base + j * blockDim.x, j < IPT): the
// step's key and value loads are all issued before its atomics.
template <int IPT, class F>
__device__ __forceinline__ void b_elements(const int32_t *__restrict__ k, const float *__restrict__ v, int64_t len,
                                           int64_t m, F &&update) {
    for (int64_t e0 = threadIdx.x; e0 < len; e0 += (int64_t)IPT * blockDim.x) {
        int32_t kk[IPT];
        float vv[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int64_t e = e0 + (int64_t)j * blockDim.x;
            kk[j] = e < len ? __ldcs(k + e) : -1;
            vv[j] = e < len ? __ldcs(v + e) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            if ((uint32_t)kk[j] < (uint64_t)m) update(kk[j], vv[j], e0 + (int64_t)j * blockDim.x);
    }
}

template <int IPT>
__global__ void __launch_bounds__(kBHistThreads)
k_b_hist(const adc_instance *__restrict__ desc, const adc_work *__restrict__ items, const int64_t n_items,
         const int32_t *__restrict__ keys, const float *__restrict__ vals, float *__restrict__ hist,
         unsigned long long *__restrict__ tab, const int32_t smem_bins, unsigned *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sf = reinterpret_cast<float *>(smem_raw);
    unsigned long long *su = reinterpret_cast<unsigned long long *>(smem_raw);
    __shared__ unsigned s_item;
    while (true) {
        __syncthreads();  // the previous item's flush is done before smem is reused
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t w = s_item;
        if (w >= n_items) return;
        const adc_work it = items[w];
        const adc_instance d = desc[it.inst];
        const int32_t *k = keys + d.val_off + it.start;
        const float *v = vals + d.val_off + it.start;
        const int64_t len = it.len, m = d.m;
        const bool use_smem = m <= smem_bins && 2 * len >= m;
        if (d.op == ADC_OP_ADD) {
            float *g = hist + d.bin_off;
            if (use_smem) {
                for (int64_t j = threadIdx.x; j < m; j += blockDim.x) sf[j] = 0.f;
                __syncthreads();
                b_elements<IPT>(k, v, len, m, [&](int32_t kk, float x, int64_t) { atomicAdd(sf + kk, x); });
                __syncthreads();
                for (int64_t j = threadIdx.x; j < m; j += blockDim.x)
                    if (sf[j] != 0.f) atomicAdd(g + j, sf[j]);
            } else {
                b_elements<IPT>(k, v, len, m, [&](int32_t kk, float x, int64_t) { atomicAdd(g + kk, x); });
            }
        } else {
            unsigned long long *g = tab + d.bin_off;
            if (use_smem) {
                for (int64_t j = threadIdx.x; j < m; j += blockDim.x) su[j] = 0ull;
                __syncthreads();
                b_elements<IPT>(k, v, len, m, [&](int32_t kk, float x, int64_t e) {
                    const unsigned long long key = bmax_key(x, it.start + e);
                    if (key > *reinterpret_cast<volatile unsigned long long *>(su + kk)) atomicMax(su + kk, key);
                });
                __syncthreads();
                for (int64_t j = threadIdx.x; j < m; j += blockDim.x)
                    if (su[j] > __ldcg(g + j)) atomicMax(g + j, su[j]);
            } else {
                b_elements<IPT>(k, v, len, m, [&](int32_t kk, float x, int64_t e) {
                    const unsigned long long key = bmax_key(x, it.start + e);
                    if (key > __ldcg(g + kk)) atomicMax(g + kk, key);
                });
            }
        }
    }
}

// Block-wide inclusive +-scan of one float per thread (1024 threads).
__device__ __forceinline__ float block_incl_sum(float x, float *tmp, float *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        float w = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        tmp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    *total = tmp[31];
    return x + (warp > 0 ? tmp[warp - 1] : 0.f);
}

__device__ __forceinline__ double block_sum_d(double x, double *tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) tmp[warp] = x;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += tmp[w];
    return s;
}

__global__ void __launch_bounds__(kBScanThreads)
k_b_scan_loss(const adc_instance *__restrict__ desc, const int32_t count, const float *__restrict__ vals,
              float *__restrict__ hist, const unsigned long long *__restrict__ tab, float *__restrict__ scan,
              int32_t *__restrict__ is, float *__restrict__ loss_parts, float *__restrict__ loss,
              unsigned *__restrict__ ticket) {
    __shared__ float tmp[32];
    __shared__ double tmpd[32];
    __shared__ bool last;
    const adc_instance d = desc[blockIdx.x];
    float carry = 0.f;
    double acc = 0.0;
    for (int64_t base = 0; base < d.m; base += kBScanThreads) {
        const int64_t j = base + threadIdx.x;
        float h = 0.f;
        if (j < d.m) {
            if (d.op == ADC_OP_ADD) {
                h = hist[d.bin_off + j];
            } else {
                const unsigned long long key = tab[d.bin_off + j];
                int64_t idx = d.n;
                if (key != 0ull) {
                    const int64_t c = bmax_index(key);
                    const float val = vals[d.val_off + c];
                    if (!(0.f >= val)) {  // the zero initial value wins ties
                        h = val;
                        idx = c;
                    }
                }
                hist[d.bin_off + j] = h;
                is[d.bin_off + j] = (int32_t)idx;
            }
        }
        float total;
        const float inc = block_incl_sum(h, tmp, &total) + carry;
        if (j < d.m) {
            scan[d.bin_off + j] = inc;
            acc += (double)inc;
        }
        carry += total;
    }
    const double part = block_sum_d(acc, tmpd);
    if (threadIdx.x == 0) {
        loss_parts[blockIdx.x] = (float)part;
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)count - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) s += (double)__ldcg(loss_parts + i);
    s = block_sum_d(s, tmpd);
    if (threadIdx.x == 0) *loss = (float)s;
}

// histbar_i[j] = sum_{k >= j} lbar  (reverse +-scan of the broadcast loss adjoint)
__global__ void __launch_bounds__(kBScanThreads)
k_b_hbar(const adc_instance *__restrict__ desc, const float *__restrict__ loss_bar, float *__restrict__ histbar) {
    __shared__ float tmp[32];
    const adc_instance d = desc[blockIdx.x];
    const float lb = *loss_bar;
    float carry = 0.f;
    for (int64_t base = 0; base < d.m; base += kBScanThreads) {
        const int64_t j = d.m - 1 - (base + threadIdx.x);  // descending bins
        float total;
        const float inc = block_incl_sum(j >= 0 ? lb : 0.f, tmp, &total) + carry;
        if (j >= 0) histbar[d.bin_off + j] = inc;
        carry += total;
    }
}

// ADD: valsbar_e = histbar[k_e]; MAX: zero-fill (the scatter follows).
__global__ void __launch_bounds__(kBHistThreads)
k_b_vjp_items(const adc_instance *__restrict__ desc, const adc_work *__restrict__ items, const int64_t n_items,
              const int32_t *__restrict__ keys, const float *__restrict__ histbar, float *__restrict__ valsbar,
              unsigned *__restrict__ counter) {
    __shared__ unsigned s_item;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t w = s_item;
        if (w >= n_items) return;
        const adc_work it = items[w];
        const adc_instance d = desc[it.inst];
        const int64_t o = d.val_off + it.start;
        if (d.op == ADC_OP_ADD) {
            for (int64_t e = threadIdx.x; e < it.len; e += blockDim.x) {
                const int32_t kk = __ldcs(keys + o + e);
                valsbar[o + e] = ((uint32_t)kk < (uint64_t)d.m) ? __ldg(histbar + d.bin_off + kk) : 0.f;
            }
        } else {
            for (int64_t e = threadIdx.x; e < it.len; e += blockDim.x) valsbar[o + e] = 0.f;
        }
    }
}

__global__ void k_b_scatter(const adc_instance *__restrict__ desc, const int32_t *__restrict__ is,
                            const float *__restrict__ histbar, float *__restrict__ valsbar) {
    const adc_instance d = desc[blockIdx.x];
    if (d.op != ADC_OP_MAX) return;
    for (int64_t j = threadIdx.x; j < d.m; j += blockDim.x) {
        const int64_t i = is[d.bin_off + j];
        if (i >= 0 && i < d.n) valsbar[d.val_off + i] = histbar[d.bin_off + j];
    }
}

}  // namespace adc

using namespace adc;

namespace {
inline bool al(const void *p, size_t a) { return p != nullptr && reinterpret_cast<uintptr_t>(p) % a == 0; }
size_t ws_need(int64_t total_bins) { return kWsHeader + align_up((size_t)total_bins * 8, 256); }
}  // namespace

extern "C" {

int64_t adc_batched_plan(const adc_instance *desc, int32_t count, int64_t chunk, adc_work *items, int64_t capacity) {
    if (desc == nullptr || count < 1 || chunk < 1) return -1;
    // largest instances first: long items start early and small ones fill the tail
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return desc[a].n > desc[b].n; });
    int64_t k = 0;
    for (int32_t r = 0; r < count; ++r) {
        const adc_instance &d = desc[order[r]];
        if (d.n < 0 || d.m < 1) return -1;
        for (int64_t s = 0; s < d.n; s += chunk) {
            if (items != nullptr && k < capacity) {
                items[k].inst = order[r];
                items[k].pad = 0;
                items[k].start = s;
                items[k].len = (d.n - s < chunk) ? d.n - s : chunk;
            }
            ++k;
        }
    }
    return k;
}

size_t adc_batched_workspace_bytes(int32_t count, int64_t total_bins) {
    if (count < 1 || total_bins < 1) return 0;
    return ws_need(total_bins);
}

adc_status adc_batched_hist_scan_fwd(const adc_instance *desc, int32_t count, const adc_work *items, int64_t n_items,
                                     int64_t total_bins, const int32_t *keys, const float *vals, float *hist,
                                     float *scan, int32_t *is, float *loss_parts, float *loss, int32_t smem_bins,
                                     void *ws, size_t ws_bytes, void *stream) {
    if (count < 1 || n_items < 0 || total_bins < 1 || smem_bins < 0) return ADC_ERR_INVALID_ARG;
    if (!al(desc, 8) || (n_items > 0 && (!al(items, 8) || !al(keys, 4) || !al(vals, 4))) || !al(hist, 4) ||
        !al(scan, 4) || !al(is, 4) || !al(loss_parts, 4) || !al(loss, 4))
        return ADC_ERR_INVALID_ARG;
    if (!al(ws, 256)) return ADC_ERR_INVALID_ARG;
    if (ws_bytes < ws_need(total_bins)) return ADC_ERR_WORKSPACE;
    if (smem_bins == 0) smem_bins = kDefaultSmemBins;
    const size_t smem = (size_t)smem_bins * 8;
    if (smem > 200 * 1024) return ADC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(ws);
    auto *tab = reinterpret_cast<unsigned long long *>(w + kWsHeader);
    if (cudaMemsetAsync(ws, 0, kWsHeader, s) != cudaSuccess) return ADC_ERR_CUDA;
    k_b_init<<<count, 256, 0, s>>>(desc, hist, tab);
    if (n_items > 0) {
        int per_sm = (int)((200 * 1024) / (smem + 1024));
        per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
        const unsigned grid = (unsigned)(num_sms() * per_sm);
        unsigned *ctr = counter_slot(ws, 0);
        auto run = [&](auto kern) -> bool {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return false;
            kern<<<grid, kBHistThreads, smem, s>>>(desc, items, n_items, keys, vals, hist, tab, smem_bins, ctr);
            return true;
        };
        const bool ok = g_batched_ipt == 1 ? run(k_b_hist<1>) : g_batched_ipt == 8 ? run(k_b_hist<8>) : run(k_b_hist<4>);
        if (!ok) return ADC_ERR_CUDA;
    }
    k_b_scan_loss<<<count, kBScanThreads, 0, s>>>(desc, count, vals, hist, tab, scan, is, loss_parts, loss,
                                                   counter_slot(ws, 1));
    return check_launch();
}

adc_status adc_batched_hist_scan_vjp(const adc_instance *desc, int32_t count, const adc_work *items, int64_t n_items,
                                     int64_t total_bins, const int32_t *keys, const int32_t *is, const float *loss_bar,
                                     float *histbar, float *valsbar, void *ws, size_t ws_bytes, void *stream) {
    if (count < 1 || n_items < 0 || total_bins < 1) return ADC_ERR_INVALID_ARG;
    if (!al(desc, 8) || (n_items > 0 && (!al(items, 8) || !al(keys, 4) || !al(valsbar, 4))) || !al(is, 4) ||
        !al(loss_bar, 4) || !al(histbar, 4))
        return ADC_ERR_INVALID_ARG;
    if (!al(ws, 256)) return ADC_ERR_INVALID_ARG;
    if (ws_bytes < kWsHeader) return ADC_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, kWsHeader, s) != cudaSuccess) return ADC_ERR_CUDA;
    k_b_hbar<<<count, kBScanThreads, 0, s>>>(desc, loss_bar, histbar);
    if (n_items > 0)
        k_b_vjp_items<<<num_sms() * 4, kBHistThreads, 0, s>>>(desc, items, n_items, keys, histbar, valsbar,
                                                              counter_slot(ws, 2));
    k_b_scatter<<<count, 256, 0, s>>>(desc, is, histbar, valsbar);
    return check_launch();
}

}  // extern "C"

extern "C" void adc_debug_set_batched_items(int items) {
    g_batched_ipt = (items == 1 || items == 8) ? items : 4;
}
