// reduce_by_index with the specialised operators (Sec. 4.2) and their vjps.
//
// Forward strategies (Sec. 4.2.6 lists the design space; chosen per call):
//   SMEM_WARP : one private sub-histogram per warp in shared memory (8 copies
//               per block), shared-memory atomics, one flush per block into
//               the global result -- for histograms of up to a few KB.
//   SMEM_BLOCK: one sub-histogram per 1024-thread block filling most of the
//               SM's shared memory -- for histograms up to ~200 KB.
//   SPLIT     : lifted min/max tables of 2-4 block tables: S blocks read the
//               same elements, each owns 1/S of the bins in its shared
//               memory, then flushes them (filtered global atomics).
//   CLUSTER   : lifted fp32 min/max tables of 2-8 block tables: the table is
//               spread over the blocks of a thread-block cluster, each element
//               is read once and updates its bin in the owning block's shared
//               memory (local or distributed); each cluster's table is written
//               as a partial row and the rows are reduced per bin.
//   TWOPASS   : lifted fp32 min/max whose packed table exceeds one block but
//               whose 32-bit value table does not: per-block value tables
//               written as partial rows and reduced per bin, then a second
//               pass finds the lowest index holding each bin's value.
//   PART      : for tables beyond shared memory: the elements are first
//               partitioned by bin range so that every range's bins fit one
//               block's shared memory (hist_part.cu) -- no global atomics.
//   GLOBAL    : atomics directly on the global table (L2-resident); for
//               fp64 min/max and tables too large for PART.
// Operators and their atomics:
//   ADD     : native float/double atomic add.
//   MIN/MAX : fp32 value and int32 index packed into one 64-bit key
//             (order-preserving value bits << 32 | index, the index inverted
//             for max) so that Fig. 5's lifted min^L (smaller index wins
//             ties) is ONE native 64-bit atomicMin/atomicMax; a plain read of
//             the current key skips the atomic when it cannot win (the table
//             only moves one way, so a stale read is safe).  fp64 uses two
//             phases: the value by 64-bit atomicMin on its ordered bits, then
//             the lowest index among elements equal to it.
//   MUL     : (zero count, product of non-zeros) per bin (Sec. 4.2.3): integer
//             atomicAdd for zeros, compare-and-swap multiply for the rest.
// The initial histogram is decoupled as in Sec. 4: the atomics build the
// histogram of the values from the neutral element and a finalising map folds
// hist0 in (hist0 wins min/max ties, acting as index -1).
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"
#include "tile_io.cuh"
#include "tma.cuh"

namespace adc {

enum HistStrategy {
    kSmemWarp = 0, kSmemBlock = 1, kGlobal = 2, kSmemThread = 3, kPart = 4, kSplit = 5, kCluster = 6, kTwoPass = 7,
    kPairs = 8
};

// ------------------------------------------------------------ element loop --
// Calls f(key, value, index) for every element, grid-stride over 4-element
// vectors (128-bit key loads), two vectors in flight per thread.
template <typename T, class F>
__device__ __forceinline__ void for_each_elem(const int32_t *__restrict__ keys, const T *__restrict__ vals,
                                              const int64_t n, F &&f) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nv = n / 4;
    int64_t v = gtid;
    for (; v + stride < nv; v += 2 * stride) {
        const int4 k0 = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        const int4 k1 = __ldcs(reinterpret_cast<const int4 *>(keys) + v + stride);
        T a[4], b[4];
        load_chunk(vals, v * 4, n, a, T(0));
        load_chunk(vals, (v + stride) * 4, n, b, T(0));
        f(k0.x, a[0], 4 * v);
        f(k0.y, a[1], 4 * v + 1);
        f(k0.z, a[2], 4 * v + 2);
        f(k0.w, a[3], 4 * v + 3);
        const int64_t w = v + stride;
        f(k1.x, b[0], 4 * w);
        f(k1.y, b[1], 4 * w + 1);
        f(k1.z, b[2], 4 * w + 2);
        f(k1.w, b[3], 4 * w + 3);
    }
    if (v < nv) {
        const int4 k0 = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        T a[4];
        load_chunk(vals, v * 4, n, a, T(0));
        f(k0.x, a[0], 4 * v);
        f(k0.y, a[1], 4 * v + 1);
        f(k0.z, a[2], 4 * v + 2);
        f(k0.w, a[3], 4 * v + 3);
    }
    for (int64_t i = nv * 4 + gtid; i < n; i += stride) f(keys[i], vals[i], i);
}


// Same traversal, but hands the callback groups of up to 8 elements so that
// it can keep 8 independent global atomics in flight.
template <typename T, class F8>
__device__ __forceinline__ void for_each_batch(const int32_t *__restrict__ keys, const T *__restrict__ vals,
                                               const int64_t n, F8 &&f) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nv = n / 4;
    int64_t v = gtid;
    int32_t kk[8];
    T vv[8];
    int64_t ii[8];
    for (; v + stride < nv; v += 2 * stride) {
        const int4 k0 = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        const int4 k1 = __ldcs(reinterpret_cast<const int4 *>(keys) + v + stride);
        T a[4], b[4];
        load_chunk(vals, v * 4, n, a, T(0));
        load_chunk(vals, (v + stride) * 4, n, b, T(0));
        kk[0] = k0.x; kk[1] = k0.y; kk[2] = k0.z; kk[3] = k0.w;
        kk[4] = k1.x; kk[5] = k1.y; kk[6] = k1.z; kk[7] = k1.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            vv[j] = a[j];
            vv[4 + j] = b[j];
            ii[j] = 4 * v + j;
            ii[4 + j] = 4 * (v + stride) + j;
        }
        f(kk, vv, ii, 8);
    }
    if (v < nv) {
        const int4 k0 = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        T a[4];
        load_chunk(vals, v * 4, n, a, T(0));
        kk[0] = k0.x; kk[1] = k0.y; kk[2] = k0.z; kk[3] = k0.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            vv[j] = a[j];
            ii[j] = 4 * v + j;
        }
        f(kk, vv, ii, 4);
    }
    for (int64_t i = nv * 4 + gtid; i < n; i += stride) {
        kk[0] = keys[i];
        vv[0] = vals[i];
        ii[0] = i;
        f(kk, vv, ii, 1);
    }
}

// ===================================================================== ADD ==
template <typename T>
__global__ void k_hist_init(T *__restrict__ h, const T *__restrict__ h0, const int64_t m, const T e) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        h[j] = h0 ? h0[j] : e;
}

template <typename T>
__global__ void __launch_bounds__(1024)
k_hist_add_smem(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                const int R, T *__restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sh = reinterpret_cast<T *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) sh[j] = T(0);
    __syncthreads();
    T *mine = sh + (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (in_range(k, m)) atomicAdd(mine + k, v);
    });
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        T s = T(0);
        for (int r = 0; r < R; ++r) s += sh[(int64_t)r * m + j];
        if (s != T(0)) atomicAdd(hist + j, s);
    }
}

template <typename T>
__global__ void k_hist_add_global(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n,
                                  const int64_t m, T *__restrict__ hist) {
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (in_range(k, m)) atomicAdd(hist + k, v);
    });
}

// ========================================================== MIN/MAX fp32 ==
template <bool MAX>
__global__ void k_pack_init(unsigned long long *__restrict__ tab, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        tab[j] = Pack<MAX>::kEmpty;
}

template <bool MAX>
__global__ void __launch_bounds__(1024)
k_hist_sel_smem(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                const int R, unsigned long long *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *sh = reinterpret_cast<unsigned long long *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) sh[j] = Pack<MAX>::kEmpty;
    __syncthreads();
    unsigned long long *mine = sh + (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t i) {
        if (in_range(k, m)) Pack<MAX>::update_smem(mine + k, Pack<MAX>::key(v, i));
    });
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        unsigned long long b = Pack<MAX>::kEmpty;
        for (int r = 0; r < R; ++r) {
            const unsigned long long c = sh[(int64_t)r * m + j];
            if (Pack<MAX>::better(c, b)) b = c;
        }
        if (b != Pack<MAX>::kEmpty) Pack<MAX>::update(tab + j, b);
    }
}

template <bool MAX>
__global__ void k_hist_sel_global(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n,
                                  const int64_t m, unsigned long long *__restrict__ tab, const int filter) {
    // With many values per bin: 8 reads of the current keys in flight, then
    // only the atomics that can still win.  With few values per bin most
    // updates win anyway: issue the (fire-and-forget) atomic directly.
    for_each_batch(keys, vals, n, [&](const int32_t (&kk)[8], const float (&vv)[8], const int64_t (&ii)[8], int cnt) {
        unsigned long long key[8], cur[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = j < cnt && in_range(kk[j], m);
            key[j] = ok ? Pack<MAX>::key(vv[j], ii[j]) : Pack<MAX>::kEmpty;
            cur[j] = (ok && filter) ? __ldcg(tab + kk[j]) : Pack<MAX>::kEmpty;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (Pack<MAX>::better(key[j], cur[j])) {
                if (MAX) atomicMax(tab + kk[j], key[j]);
                else atomicMin(tab + kk[j], key[j]);
            }
        }
    });
}

// CLUSTER: the table is spread over the CS blocks of a cluster, block r owning
// bins [r*H, r*H + H); every element is read once (the grid strides over all
// of them) and its packed key goes to the owning block's shared memory through
// the cluster's shared window: a read of the current key, then, while it can
// win, a compare-and-swap.
// After a cluster barrier each block writes its bins to the cluster's partial
// row; k_sel_reduce combines the rows.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory offset in block `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ unsigned long long cluster_ld_u64(uint32_t addr) {
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long cluster_cas_u64(uint32_t addr, unsigned long long expect,
                                                          unsigned long long val) {
    unsigned long long prev;
    asm volatile("atom.shared::cluster.cas.b64 %0, [%1], %2, %3;" : "=l"(prev) : "r"(addr), "l"(expect), "l"(val)
                 : "memory");
    return prev;
}
// The lifted min/max update of a bin in a cluster block's table, as a
// compare-and-swap loop from the key read just before (bounded; a give-up
// sets the error word).  64-bit min/max atomics on distributed shared memory
// were measured to lose updates on this part (min.u64 / max.u64 with red and
// with atom), so the update is built on the compare-and-swap, which did not.
template <bool MAX>
__device__ __forceinline__ void cluster_update(uint32_t addr, unsigned long long k, unsigned long long cur,
                                               unsigned *err) {
    for (int it = 0; it < (1 << 20); ++it) {
        if (!Pack<MAX>::better(k, cur)) return;
        const unsigned long long prev = cluster_cas_u64(addr, cur, k);
        if (prev == cur) return;
        cur = prev;
    }
    set_error(err, kErrCasLimit);
}

constexpr int kMaxClusterBlocks = 8;

template <bool MAX>
__global__ void __launch_bounds__(1024)
k_hist_sel_cluster(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                   const int CS, const int64_t H, unsigned long long *__restrict__ rows, unsigned *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *sh = reinterpret_cast<unsigned long long *>(smem_raw);
    const uint32_t rank = cluster_rank();
    const int64_t lo = (int64_t)rank * H;
    const int64_t w = (m - lo) < H ? (m - lo) : H;
    for (int64_t j = threadIdx.x; j < H; j += blockDim.x) sh[j] = Pack<MAX>::kEmpty;
    uint32_t base[kMaxClusterBlocks];
    const uint32_t mine = smem_u32(sh);
#pragma unroll
    for (int q = 0; q < kMaxClusterBlocks; ++q) base[q] = q < CS ? cluster_map(mine, (uint32_t)q) : 0u;
    cluster_barrier();  // every block's table is initialised before anyone writes into it
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t i) {
        if (!in_range(k, m)) return;
        const uint32_t owner = (uint32_t)((int64_t)k / H);
        uint32_t b = base[0];
#pragma unroll
        for (int q = 1; q < kMaxClusterBlocks; ++q)
            if ((uint32_t)q == owner) b = base[q];
        const uint32_t addr = b + (uint32_t)(((int64_t)k - (int64_t)owner * H) * 8);
        cluster_update<MAX>(addr, Pack<MAX>::key(v, i), cluster_ld_u64(addr), err);
    });
    cluster_barrier();  // all updates, local and remote, have landed
    unsigned long long *row = rows + (int64_t)(blockIdx.x / CS) * m + lo;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) row[j] = sh[j];
}

// Per bin, the best key over the C partial rows (in row order), decoded with
// hist0 folded in as in k_hist_sel_final: 32 bins per block across the lanes,
// the rows split over the 32 warps.
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_sel_reduce(const unsigned long long *__restrict__ rows, const int C, const int64_t m,
             const float *__restrict__ vals, const float *__restrict__ h0, const int64_t n,
             float *__restrict__ hist, int32_t *__restrict__ is) {
    __shared__ unsigned long long s_k[32][33];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    unsigned long long best = Pack<MAX>::kEmpty;
    if (j < m)
        for (int c = wp; c < C; c += 32) {
            const unsigned long long k = rows[(int64_t)c * m + j];
            if (Pack<MAX>::better(k, best)) best = k;
        }
    s_k[wp][lane] = best;
    __syncthreads();
    if (wp == 0 && j < m) {
        for (int u = 1; u < 32; ++u)
            if (Pack<MAX>::better(s_k[u][lane], best)) best = s_k[u][lane];
        float v = MAX ? -Num<float>::inf() : Num<float>::inf();
        int64_t idx = n;
        if (best != Pack<MAX>::kEmpty) {
            idx = Pack<MAX>::index(best);
            v = from_ordered((uint32_t)(best >> 32));
            if (v == 0.0f) v = vals[idx];  // the key folds -0.0 onto +0.0
        }
        if (h0) {
            const float a = h0[j];
            if (MAX ? (a >= v) : (a <= v)) {
                v = a;
                idx = n;
            }
        }
        hist[j] = v;
        is[j] = (int32_t)idx;
    }
}

// TWOPASS, pass 1: each block (one per SM) keeps a table of the bins' best
// order-preserving 32-bit value keys in shared memory and writes it as its
// partial row; k_ord_rows_reduce takes the best over the rows per bin.
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_sel_val_rows(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
               uint32_t *__restrict__ rows) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) sh[j] = Ord32<MAX>::kEmpty;
    __syncthreads();
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t) {
        if (in_range(k, m)) Ord32<MAX>::update(sh + k, ordered_key(v), true);
    });
    __syncthreads();
    uint32_t *row = rows + (int64_t)blockIdx.x * m;
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) row[j] = sh[j];
}

// Per bin, the best of the G rows' keys (32 bins across the lanes, the rows
// over the 32 warps); idx gets its "none yet" sentinel for pass 2.
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_ord_rows_reduce(const uint32_t *__restrict__ rows, const int G, const int64_t m, uint32_t *__restrict__ best,
                  uint32_t *__restrict__ idx) {
    __shared__ uint32_t s_k[32][33];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    uint32_t b = Ord32<MAX>::kEmpty;
    if (j < m)
        for (int g = wp; g < G; g += 32) {
            const uint32_t c = rows[(int64_t)g * m + j];
            if (Ord32<MAX>::better(c, b)) b = c;
        }
    s_k[wp][lane] = b;
    __syncthreads();
    if (wp == 0 && j < m) {
        for (int u = 1; u < 32; ++u)
            if (Ord32<MAX>::better(s_k[u][lane], b)) b = s_k[u][lane];
        best[j] = b;
        idx[j] = 0xffffffffu;
    }
}

// TWOPASS, pass 2: with the bins' best keys in shared memory, every element
// holding its bin's best value offers its index; the lowest one stays (the
// lifted operator's tie rule).  Few elements match, so the global atomics are
// few.
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_sel_index_pass(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                 const uint32_t *__restrict__ best, uint32_t *__restrict__ idx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) sh[j] = best[j];
    __syncthreads();
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t i) {
        if (in_range(k, m) && ordered_key(v) == sh[k]) atomicMin(idx + k, (uint32_t)i);
    });
}

// PAIRS (the same range of m): blocks work in pairs, block p of a pair keeping
// bins [p W, p W + w) as a 32-bit value table and a 32-bit index table in
// shared memory; both blocks of a pair read the same elements, the second
// mostly from L2, so the input comes from DRAM once instead of twice.
// Elements go in rounds of 8 per thread, held in registers (the next round's
// loads are issued before this round's barriers):
//   1. each updates its bin's best value; one that makes it strictly better
//      clears the bin's index;
//   2. after a barrier, each holding its bin's best value offers its index
//      (the lowest stays); a barrier closes the round.
// After every round a bin's index is the lowest among the elements seen so
// far that hold its best value -- the lifted operator's result.  Per pair one
// row of values and one of indices; k_sel_pair_rows_reduce folds the rows.
// Forced only: at m = 50,000 it measured 0.31 ms against 0.18 ms for TWOPASS
// (one 1024-thread block per SM, and every round's two barriers stall it).
constexpr uint32_t kNoIndex = 0xffffffffu;
template <bool MAX>
__global__ void __launch_bounds__(1024, 1)
k_sel_pairs(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
            const int64_t W, uint32_t *__restrict__ rows_val, uint32_t *__restrict__ rows_idx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sv = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *si = sv + W;
    const int tid = threadIdx.x;
    const int64_t pair = blockIdx.x >> 1, pairs = gridDim.x >> 1;
    const int64_t lo = (int64_t)(blockIdx.x & 1) * W;
    const int64_t w = (m - lo) < W ? (m - lo) : W;
    for (int64_t j = tid; j < w; j += 1024) {
        sv[j] = Ord32<MAX>::kEmpty;
        si[j] = kNoIndex;
    }
    __syncthreads();
    const int64_t nv = n / 4;                    // whole quads
    const int64_t span = pairs * 1024;           // quads of one half-round over all pairs
    const int64_t rounds = (nv + 2 * span - 1) / (2 * span);
    const int64_t t0 = pair * 1024 + tid;
    const int4 *k4 = reinterpret_cast<const int4 *>(keys);
    const float4 *v4 = reinterpret_cast<const float4 *>(vals);
    auto fetch = [&](int64_t r, int4 (&kq)[2], float4 (&vq)[2]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int64_t v = (2 * r + q) * span + t0;
            if (v < nv) {
                kq[q] = __ldcg(k4 + v);
                vq[q] = __ldcg(v4 + v);
            } else {
                kq[q] = make_int4(-1, -1, -1, -1);
                vq[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    // one round over up to 8 (key, value, index) triples; uniform barriers
    auto round = [&](const int32_t (&kk)[8], const float (&vv)[8], const int64_t (&ii)[8]) {
        uint32_t key[8];
        int b[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t bb = (int64_t)kk[c] - lo;
            const bool mine = in_range(kk[c], m) && bb >= 0 && bb < w;
            b[c] = mine ? (int)bb : -1;
            key[c] = ordered_key(vv[c]);
            if (mine) {
                const uint32_t cur = *reinterpret_cast<volatile uint32_t *>(sv + bb);
                if (Ord32<MAX>::better(key[c], cur)) {
                    const uint32_t old = MAX ? atomicMax(sv + bb, key[c]) : atomicMin(sv + bb, key[c]);
                    if (Ord32<MAX>::better(key[c], old)) si[bb] = kNoIndex;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (b[c] >= 0 && key[c] == sv[b[c]]) atomicMin(si + b[c], (uint32_t)ii[c]);
        __syncthreads();
    };
    int4 kq[2], kn[2];
    float4 vq[2], vn[2];
    if (rounds > 0) fetch(0, kq, vq);
    for (int64_t r = 0; r < rounds; ++r) {
        if (r + 1 < rounds) fetch(r + 1, kn, vn);
        const int32_t kk[8] = {kq[0].x, kq[0].y, kq[0].z, kq[0].w, kq[1].x, kq[1].y, kq[1].z, kq[1].w};
        const float vv[8] = {vq[0].x, vq[0].y, vq[0].z, vq[0].w, vq[1].x, vq[1].y, vq[1].z, vq[1].w};
        int64_t ii[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) ii[c] = 4 * ((2 * r + (c >> 2)) * span + t0) + (c & 3);
        round(kk, vv, ii);
        kq[0] = kn[0];
        kq[1] = kn[1];
        vq[0] = vn[0];
        vq[1] = vn[1];
    }
    // the last n % 4 elements: pair 0 only (every block passes the barriers)
    {
        int32_t kk[8];
        float vv[8];
        int64_t ii[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t i = 4 * nv + c;
            const bool take = pair == 0 && tid == 0 && c < 4 && i < n;
            kk[c] = take ? keys[i] : -1;
            vv[c] = take ? vals[i] : 0.f;
            ii[c] = i;
        }
        round(kk, vv, ii);
    }
    uint32_t *rv = rows_val + pair * m + lo, *ri = rows_idx + pair * m + lo;
    for (int64_t j = tid; j < w; j += 1024) {
        rv[j] = sv[j];
        ri[j] = si[j];
    }
}

// Per bin, over the P pairs' rows: the best value, and the lowest index among
// the rows holding it (32 bins across the lanes, the rows over the 32 warps).
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_sel_pair_rows_reduce(const uint32_t *__restrict__ rows_val, const uint32_t *__restrict__ rows_idx, const int P,
                       const int64_t m, uint32_t *__restrict__ best, uint32_t *__restrict__ idx) {
    __shared__ uint32_t s_v[32][33], s_i[32][33];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    uint32_t bv = Ord32<MAX>::kEmpty, bi = kNoIndex;
    if (j < m)
        for (int g = wp; g < P; g += 32) {
            const uint32_t v = rows_val[(int64_t)g * m + j], i = rows_idx[(int64_t)g * m + j];
            if (Ord32<MAX>::better(v, bv) || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
    s_v[wp][lane] = bv;
    s_i[wp][lane] = bi;
    __syncthreads();
    if (wp == 0 && j < m) {
        for (int u = 1; u < 32; ++u) {
            const uint32_t v = s_v[u][lane], i = s_i[u][lane];
            if (Ord32<MAX>::better(v, bv) || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        best[j] = bv;
        idx[j] = bi;
    }
}

// Decode: the bin's value (a selected zero takes the stored element's sign),
// its index (n if none), hist0 folded in as in k_hist_sel_final.
template <bool MAX>
__global__ void k_sel_twopass_final(const uint32_t *__restrict__ best, const uint32_t *__restrict__ idx,
                                    const float *__restrict__ vals, const float *__restrict__ h0, const int64_t m,
                                    const int64_t n, float *__restrict__ hist, int32_t *__restrict__ is) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        float v = MAX ? -Num<float>::inf() : Num<float>::inf();
        int64_t i = n;
        if (best[j] != Ord32<MAX>::kEmpty) {
            i = idx[j];
            v = from_ordered(best[j]);
            if (v == 0.0f) v = vals[i];
        }
        if (h0) {
            const float a = h0[j];
            if (MAX ? (a >= v) : (a <= v)) {
                v = a;
                i = n;
            }
        }
        hist[j] = v;
        is[j] = (int32_t)i;
    }
}

// SPLIT: blocks come in groups of S that read the same elements; block p of a
// group keeps bins [p*W, (p+1)*W) in shared memory and skips the others.
template <bool MAX>
__global__ void __launch_bounds__(1024)
k_hist_sel_split(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                 const int S, const int64_t W, unsigned long long *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *sh = reinterpret_cast<unsigned long long *>(smem_raw);
    const int64_t group = blockIdx.x / S, groups = gridDim.x / S;
    const int64_t lo = (int64_t)(blockIdx.x % S) * W;
    const int64_t w = (m - lo) < W ? (m - lo) : W;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) sh[j] = Pack<MAX>::kEmpty;
    __syncthreads();
    // the element loop of for_each_elem over the group's virtual grid
    const int64_t gtid = group * blockDim.x + threadIdx.x, stride = groups * blockDim.x;
    const int64_t nv = n / 4;
    auto upd = [&](int32_t k, float v, int64_t i) {
        const int64_t b = (int64_t)k - lo;
        if (in_range(k, m) && b >= 0 && b < w) Pack<MAX>::update_smem(sh + b, Pack<MAX>::key(v, i));
    };
    for (int64_t v = gtid; v < nv; v += stride) {
        const int4 k4 = __ldcg(reinterpret_cast<const int4 *>(keys) + v);
        float a[4];
        load_chunk(vals, v * 4, n, a, 0.f);
        upd(k4.x, a[0], 4 * v);
        upd(k4.y, a[1], 4 * v + 1);
        upd(k4.z, a[2], 4 * v + 2);
        upd(k4.w, a[3], 4 * v + 3);
    }
    for (int64_t i = nv * 4 + gtid; i < n; i += stride) upd(keys[i], vals[i], i);
    __syncthreads();
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x)
        if (sh[j] != Pack<MAX>::kEmpty) Pack<MAX>::update(tab + lo + j, sh[j]);
}

// Decode the packed table, fold hist0 in (it wins ties), write hist and is.
template <bool MAX>
__global__ void k_hist_sel_final(const unsigned long long *__restrict__ tab, const float *__restrict__ vals,
                                 const float *__restrict__ h0, const int64_t m, const int64_t n,
                                 float *__restrict__ hist, int32_t *__restrict__ is) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = tab[j];
        const float neutral = MAX ? -Num<float>::inf() : Num<float>::inf();
        float v = neutral;
        int64_t idx = n;
        if (key != Pack<MAX>::kEmpty) {
            idx = Pack<MAX>::index(key);
            // the key holds the value itself; only a zero needs the stored
            // element (the key folds -0.0 onto +0.0)
            v = from_ordered((uint32_t)(key >> 32));
            if (v == 0.0f) v = vals[idx];
        }
        if (h0) {
            const float a = h0[j];
            if (MAX ? (a >= v) : (a <= v)) {
                v = a;
                idx = n;
            }
        }
        hist[j] = v;
        is[j] = (int32_t)idx;
    }
}

// ========================================================== MIN/MAX fp64 ==
template <bool MAX>
__global__ void k_hist_sel64_value(const int32_t *__restrict__ keys, const double *__restrict__ vals, const int64_t n,
                                   const int64_t m, unsigned long long *__restrict__ tv) {
    for_each_elem(keys, vals, n, [&](int32_t k, double v, int64_t) {
        if (!in_range(k, m)) return;
        const unsigned long long o = ordered_key(v);
        const unsigned long long cur = __ldcg(tv + k);
        if (MAX ? (o > cur) : (o < cur)) {
            if (MAX) atomicMax(tv + k, o);
            else atomicMin(tv + k, o);
        }
    });
}

template <bool MAX>
__global__ void k_hist_sel64_index(const int32_t *__restrict__ keys, const double *__restrict__ vals, const int64_t n,
                                   const int64_t m, const unsigned long long *__restrict__ tv,
                                   unsigned *__restrict__ ti) {
    for_each_elem(keys, vals, n, [&](int32_t k, double v, int64_t i) {
        if (!in_range(k, m)) return;
        if (ordered_key(v) == tv[k] && (unsigned)i < __ldcg(ti + k)) atomicMin(ti + k, (unsigned)i);
    });
}

__global__ void k_sel64_init(unsigned long long *__restrict__ tv, unsigned *__restrict__ ti, const int64_t m,
                             const unsigned long long empty) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        tv[j] = empty;
        ti[j] = 0xffffffffu;
    }
}

template <bool MAX>
__global__ void k_hist_sel64_final(const unsigned *__restrict__ ti, const double *__restrict__ vals,
                                   const double *__restrict__ h0, const int64_t m, const int64_t n,
                                   double *__restrict__ hist, int32_t *__restrict__ is) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned i = ti[j];
        double v = MAX ? -Num<double>::inf() : Num<double>::inf();
        int64_t idx = n;
        if (i != 0xffffffffu) {
            idx = i;
            v = vals[idx];
        }
        if (h0) {
            const double a = h0[j];
            if (MAX ? (a >= v) : (a <= v)) {
                v = a;
                idx = n;
            }
        }
        hist[j] = v;
        is[j] = (int32_t)idx;
    }
}

// ===================================================================== MUL ==
template <typename T>
__global__ void k_mul_init(int32_t *__restrict__ n0, T *__restrict__ p, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        n0[j] = 0;
        p[j] = T(1);
    }
}

template <typename T>
__global__ void __launch_bounds__(1024)
k_hist_mul_smem(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                const int R, T *__restrict__ part_p, int32_t *__restrict__ part_z, unsigned *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    int32_t *sz = reinterpret_cast<int32_t *>(sp + (int64_t)m * R);
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) {
        sp[j] = T(1);
        sz[j] = 0;
    }
    __syncthreads();
    const int64_t off = (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (!in_range(k, m)) return;
        if (v == T(0)) atomicAdd(sz + off + k, 1);
        else atomic_mul(sp + off + k, v, err);
    });
    __syncthreads();
    // this block's partial table, combined across blocks by k_mul_reduce
    T *P = part_p + (int64_t)blockIdx.x * m;
    int32_t *Z = part_z + (int64_t)blockIdx.x * m;
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        T prod = T(1);
        int32_t z = 0;
        for (int r = 0; r < R; ++r) {
            prod *= sp[(int64_t)r * m + j];
            z += sz[(int64_t)r * m + j];
        }
        P[j] = prod;
        Z[j] = z;
    }
}

template <typename T>
__global__ void k_hist_mul_global(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n,
                                  const int64_t m, int32_t *__restrict__ n0, T *__restrict__ p,
                                  unsigned *__restrict__ err) {
    for_each_batch(keys, vals, n, [&](const int32_t (&kk)[8], const T (&vv)[8], const int64_t (&)[8], int cnt) {
        bool use[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = j < cnt && in_range(kk[j], m);
            if (ok && vv[j] == T(0)) atomicAdd(n0 + kk[j], 1);
            use[j] = ok && vv[j] != T(0);
        }
        mul_batch<T, 8>(p, kk, vv, use, err);
    });
}

// One block-wide shared table of products (up to ~200 KB); the rare zeros go
// straight to the global zero counts, the products to this block's partial row.
template <typename T>
__global__ void __launch_bounds__(1024)
k_hist_mul_smem_prod(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                     int32_t *__restrict__ n0, T *__restrict__ part_p, unsigned *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) sp[j] = T(1);
    __syncthreads();
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (!in_range(k, m)) return;
        if (v == T(0)) atomicAdd(n0 + k, 1);
        else atomic_mul(sp + k, v, err);
    });
    __syncthreads();
    T *P = part_p + (int64_t)blockIdx.x * m;  // combined across blocks by k_mul_reduce
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) P[j] = sp[j];
}

// ------------------------------------------------- per-thread private tables --
// For tiny m: every thread owns a column of a [bin][thread] shared table, so
// updates need no atomics and a warp's accesses hit 32 distinct banks whatever
// the keys.  The block then reduces each bin across its threads.
constexpr int kThrThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThrThreads)
k_hist_mul_thread(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                  T *__restrict__ part_p, int32_t *__restrict__ part_z, unsigned *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    int32_t *sz = reinterpret_cast<int32_t *>(sp + m * kThrThreads);
    for (int64_t j = threadIdx.x; j < m * kThrThreads; j += kThrThreads) {
        sp[j] = T(1);
        sz[j] = 0;
    }
    __syncthreads();
    const int t = threadIdx.x;
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (!in_range(k, m)) return;
        const int64_t o = (int64_t)k * kThrThreads + t;
        if (v == T(0)) sz[o] += 1;
        else sp[o] *= v;
    });
    __syncthreads();
    const int lane = t & 31, warp = t >> 5;
    for (int64_t j = warp; j < m; j += kThrThreads / kWarp) {
        T prod = T(1);
        int32_t z = 0;
        for (int u = lane; u < kThrThreads; u += kWarp) {
            prod *= sp[j * kThrThreads + u];
            z += sz[j * kThrThreads + u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            prod *= __shfl_xor_sync(0xffffffffu, prod, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            part_p[(int64_t)blockIdx.x * m + j] = prod;
            part_z[(int64_t)blockIdx.x * m + j] = z;
        }
    }
}

template <bool MAX>
__global__ void __launch_bounds__(kThrThreads)
k_hist_sel_thread(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                  unsigned long long *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *sh = reinterpret_cast<unsigned long long *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * kThrThreads; j += kThrThreads) sh[j] = Pack<MAX>::kEmpty;
    __syncthreads();
    const int t = threadIdx.x;
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t i) {
        if (!in_range(k, m)) return;
        const int64_t o = (int64_t)k * kThrThreads + t;
        const unsigned long long key = Pack<MAX>::key(v, i);
        if (Pack<MAX>::better(key, sh[o])) sh[o] = key;
    });
    __syncthreads();
    const int lane = t & 31, warp = t >> 5;
    for (int64_t j = warp; j < m; j += kThrThreads / kWarp) {
        unsigned long long b = Pack<MAX>::kEmpty;
        for (int u = lane; u < kThrThreads; u += kWarp) {
            const unsigned long long c = sh[j * kThrThreads + u];
            if (Pack<MAX>::better(c, b)) b = c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
            if (Pack<MAX>::better(c, b)) b = c;
        }
        if (lane == 0 && b != Pack<MAX>::kEmpty) Pack<MAX>::update(tab + j, b);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThrThreads)
k_hist_add_thread(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                  T *__restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sh = reinterpret_cast<T *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * kThrThreads; j += kThrThreads) sh[j] = T(0);
    __syncthreads();
    const int t = threadIdx.x;
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (in_range(k, m)) sh[(int64_t)k * kThrThreads + t] += v;
    });
    __syncthreads();
    const int lane = t & 31, warp = t >> 5;
    for (int64_t j = warp; j < m; j += kThrThreads / kWarp) {
        T s = T(0);
        for (int u = lane; u < kThrThreads; u += kWarp) s += sh[j * kThrThreads + u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && s != T(0)) atomicAdd(hist + j, s);
    }
}

template <typename T>
__global__ void k_hist_mul_final(const int32_t *__restrict__ n0, const T *__restrict__ p, const T *__restrict__ h0,
                                 const int64_t m, T *__restrict__ hist) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const T xs = n0[j] > 0 ? T(0) : p[j];
        hist[j] = h0 ? h0[j] * xs : xs;
    }
}

// The per-block partial tables of the shared-memory * strategies, combined
// per bin in block order (deterministic, no global compare-and-swap): P[g][j]
// products and, for the lifted form, Z[g][j] zero counts (or, when Z is null,
// the zero counts already accumulated in n0).  32 bins per block across the
// lanes (coalesced rows), the G partials split over the 32 warps, then the
// warps' results combined in warp order.  Writes n0, p and hist (lifted:
// hist = hist0 * (n0 ? 0 : p)), or hist = hist0 * product (original primal,
// n0 == p == null).
template <typename T>
__global__ void __launch_bounds__(1024)
k_mul_reduce(const T *__restrict__ P, const int32_t *__restrict__ Z, const int G, const int64_t m,
             int32_t *__restrict__ n0, T *__restrict__ p, const T *__restrict__ h0, T *__restrict__ hist) {
    __shared__ T s_p[32][33];
    __shared__ int32_t s_z[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    T prod = T(1);
    int32_t z = 0;
    if (j < m) {
        for (int g = w; g < G; g += 32) {
            prod *= P[(int64_t)g * m + j];
            if (Z) z += Z[(int64_t)g * m + j];
        }
    }
    s_p[w][lane] = prod;
    s_z[w][lane] = z;
    __syncthreads();
    if (w == 0 && j < m) {
        T q = T(1);
        int32_t zz = (Z == nullptr && n0 != nullptr) ? n0[j] : 0;
        for (int u = 0; u < 32; ++u) {
            q *= s_p[u][lane];
            zz += s_z[u][lane];
        }
        T xs = q;
        if (p != nullptr) {
            n0[j] = zz;
            p[j] = q;
            xs = zz > 0 ? T(0) : q;
        }
        hist[j] = h0 ? h0[j] * xs : xs;
    }
}

// =================================================== original primals ==
// The un-lifted primal of Sec. 4 (the program being differentiated): the
// plain product per bin (zeros included) and the plain min/max value.  Used
// to measure the AD overhead; it keeps no residuals.
template <typename T>
__global__ void __launch_bounds__(1024)
k_prim_mul_smem(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
                const int R, T *__restrict__ part_p, unsigned *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) sp[j] = T(1);
    __syncthreads();
    T *mine = sp + (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_elem(keys, vals, n, [&](int32_t k, T v, int64_t) {
        if (in_range(k, m)) atomic_mul(mine + k, v, err);
    });
    __syncthreads();
    T *P = part_p + (int64_t)blockIdx.x * m;  // combined across blocks by k_mul_reduce
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        T prod = T(1);
        for (int r = 0; r < R; ++r) prod *= sp[(int64_t)r * m + j];
        P[j] = prod;
    }
}

template <typename T>
__global__ void k_prim_mul_global(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n,
                                  const int64_t m, T *__restrict__ hist, unsigned *__restrict__ err) {
    for_each_batch(keys, vals, n, [&](const int32_t (&kk)[8], const T (&vv)[8], const int64_t (&)[8], int cnt) {
        bool use[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) use[j] = j < cnt && in_range(kk[j], m);
        mul_batch<T, 8>(hist, kk, vv, use, err);
    });
}

template <bool MAX>
__global__ void k_ord32_init(uint32_t *__restrict__ tab, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        tab[j] = Ord32<MAX>::kEmpty;
}

template <bool MAX>
__global__ void __launch_bounds__(1024)
k_prim_sel_smem(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                const int R, uint32_t *__restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw);
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) sh[j] = Ord32<MAX>::kEmpty;
    __syncthreads();
    uint32_t *mine = sh + (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_elem(keys, vals, n, [&](int32_t k, float v, int64_t) {
        if (in_range(k, m)) Ord32<MAX>::update(mine + k, ordered_key(v), true);
    });
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        uint32_t b = Ord32<MAX>::kEmpty;
        for (int r = 0; r < R; ++r) {
            const uint32_t c = sh[(int64_t)r * m + j];
            if (Ord32<MAX>::better(c, b)) b = c;
        }
        if (b != Ord32<MAX>::kEmpty) Ord32<MAX>::update(tab + j, b, false);
    }
}

template <bool MAX>
__global__ void k_prim_sel_global(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n,
                                  const int64_t m, uint32_t *__restrict__ tab) {
    for_each_batch(keys, vals, n, [&](const int32_t (&kk)[8], const float (&vv)[8], const int64_t (&)[8], int cnt) {
        uint32_t key[8], cur[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = j < cnt && in_range(kk[j], m);
            key[j] = ok ? ordered_key(vv[j]) : Ord32<MAX>::kEmpty;
            cur[j] = ok ? __ldcg(tab + kk[j]) : Ord32<MAX>::kEmpty;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (Ord32<MAX>::better(key[j], cur[j])) {
                if (MAX) atomicMax(tab + kk[j], key[j]);
                else atomicMin(tab + kk[j], key[j]);
            }
        }
    });
}

template <bool MAX, typename T, typename U>
__global__ void k_prim_sel_final(const U *__restrict__ tab, const T *__restrict__ h0, const int64_t m,
                                 T *__restrict__ hist, const U empty) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const U key = tab[j];
        T v = (key == empty) ? (MAX ? -Num<T>::inf() : Num<T>::inf()) : from_ordered(key);
        if (h0) v = MAX ? (h0[j] >= v ? h0[j] : v) : (h0[j] <= v ? h0[j] : v);
        hist[j] = v;
    }
}

// ==================================================================== VJPs ==
template <typename T>
__global__ void k_fill(T *__restrict__ a, const int64_t n) {
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = g; i < nv; i += stride) __stcs(reinterpret_cast<uint4 *>(a) + i, make_uint4(0, 0, 0, 0));
    for (int64_t i = nv * V + g; i < n; i += stride) a[i] = T(0);
}

// Sec. 4.2.1: valsbar_i (+)= histbar[k_i] (0 for out-of-range keys).
template <typename T>
__global__ void k_hist_add_vjp(const int32_t *__restrict__ keys, const T *__restrict__ hb, T *__restrict__ vb,
                               const int64_t n, const int64_t m, const int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nv = n / 4;
    for (int64_t v = g; v < nv; v += stride) {
        const int4 k = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        T o[4];
        if (accumulate) load_chunk(vb, v * 4, n, o, T(0));
        const int kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const T gv = in_range(kk[c], m) ? __ldg(hb + kk[c]) : T(0);
            o[c] = accumulate ? o[c] + gv : gv;
        }
        store_chunk(vb, v * 4, n, o);
    }
    for (int64_t i = nv * 4 + g; i < n; i += stride) {
        const int32_t k = keys[i];
        const T gv = in_range(k, m) ? hb[k] : T(0);
        vb[i] = accumulate ? vb[i] + gv : gv;
    }
}

// hist0bar (+)= histbar, masked per operator.
template <typename T>
__global__ void k_h0bar_add(const T *__restrict__ hb, T *__restrict__ h0b, const int64_t m, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        h0b[j] = accumulate ? h0b[j] + hb[j] : hb[j];
}

// Fig. 5 return sweep: valsbar[is[j]] += histbar[j]; hist0bar[j] gets histbar[j] where hist0 won.
template <typename T>
__global__ void k_hist_sel_vjp(const int32_t *__restrict__ is, const T *__restrict__ hb, T *__restrict__ vb,
                               T *__restrict__ h0b, const int64_t m, const int64_t n, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = is[j];
        if (i >= 0 && i < n) vb[i] += hb[j];
        if (h0b) {
            const T g = (i >= n) ? hb[j] : T(0);
            h0b[j] = accumulate ? h0b[j] + g : g;
        }
    }
}

// The same Fig. 5 return sweep as a gather, for large m (few values per bin):
// element i is the selected one of its bin iff is[k_i] == i.  One streaming
// pass over the keys replaces a zero-fill plus a scatter of partial sectors.
template <typename T>
__global__ void k_hist_sel_vjp_gather(const int32_t *__restrict__ keys, const int32_t *__restrict__ is,
                                      const T *__restrict__ hb, T *__restrict__ vb, const int64_t n, const int64_t m,
                                      const int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t keep = l2_evict_last_policy();  // is and histbar stay in L2; keys and valsbar stream
    const int64_t nv = n / 4;
    for (int64_t v = g; v < nv; v += stride) {
        const int4 k = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
        T o[4];
        if (accumulate) load_chunk(vb, v * 4, n, o, T(0));
        const int kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool sel = in_range(kk[c], m) && ld_keep(is + kk[c], keep) == (int32_t)(4 * v + c);
            const T gv = sel ? ld_keep(hb + kk[c], keep) : T(0);
            o[c] = accumulate ? o[c] + gv : gv;
        }
        store_chunk(vb, v * 4, n, o);
    }
    for (int64_t i = nv * 4 + g; i < n; i += stride) {
        const int32_t k = keys[i];
        const T gv = (in_range(k, m) && is[k] == (int32_t)i) ? hb[k] : T(0);
        vb[i] = accumulate ? vb[i] + gv : gv;
    }
}

// The same return sweep with a bitmap, for large m: one bit per element marks
// the selected ones (bit is[j] for every bin whose value came from an
// element), then one streaming pass writes vbar_i = histbar[k_i] where the bit
// is set and 0 elsewhere.  m coalesced reads and m random bit updates, and one
// gather per SELECTED element, replace a random gather of is[k_i] per element;
// the keys of a group of 4 elements are read only when one of them is set.
__global__ void k_sel_bits(const int32_t *__restrict__ is, uint32_t *__restrict__ bits, const int64_t m,
                           const int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = is[j];
        if (i >= 0 && i < n) atomicOr(bits + (i >> 5), 1u << (i & 31));
    }
}

template <typename T>
__global__ void k_hist_sel_vjp_bits(const int32_t *__restrict__ keys, const uint32_t *__restrict__ bits,
                                    const T *__restrict__ hb, T *__restrict__ vb, const int64_t n, const int64_t m,
                                    const int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nv = n / 4;
    for (int64_t v = g; v < nv; v += stride) {
        const uint32_t b4 = (__ldg(bits + ((4 * v) >> 5)) >> ((4 * v) & 31)) & 0xfu;  // the group's 4 bits
        T o[4];
        if (accumulate) load_chunk(vb, v * 4, n, o, T(0));
        if (b4) {
            const int4 k = __ldcs(reinterpret_cast<const int4 *>(keys) + v);
            const int kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const T gv = ((b4 >> c) & 1u) ? hb[kk[c]] : T(0);
                o[c] = accumulate ? o[c] + gv : gv;
            }
        } else if (!accumulate) {
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = T(0);
        }
        store_chunk(vb, v * 4, n, o);
    }
    for (int64_t i = nv * 4 + g; i < n; i += stride) {
        const T gv = ((__ldg(bits + (i >> 5)) >> (i & 31)) & 1u) ? hb[keys[i]] : T(0);
        vb[i] = accumulate ? vb[i] + gv : gv;
    }
}

template <typename T>
__global__ void k_h0bar_sel(const int32_t *__restrict__ is, const T *__restrict__ hb, T *__restrict__ h0b,
                            const int64_t m, const int64_t n, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const T g = (is[j] >= n) ? hb[j] : T(0);
        h0b[j] = accumulate ? h0b[j] + g : g;
    }
}

// Sec. 4.2.3 return sweep with the zero-count cases of Fig. 3, per bin.  Two
// per-bin coefficients are built first, with a = hist0[k] * p[k] * histbar[k]:
//   anz[k] = a if n0[k] == 0 else 0   -> vbar = anz[k] / v   for v != 0
//   az[k]  = a if n0[k] == 1 else 0   -> vbar = az[k]        for v == 0
// so the element pass gathers ONE word per non-zero value (and one from the
// second table for the rare zeros).
template <typename T>
__global__ void k_mul_vjp_prep(const int32_t *__restrict__ n0, const T *__restrict__ p, const T *__restrict__ h0,
                               const T *__restrict__ hb, T *__restrict__ anz, T *__restrict__ az, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t z = n0[j];
        const T a = p[j] * (h0 ? h0[j] * hb[j] : hb[j]);
        anz[j] = z == 0 ? a : T(0);
        az[j] = z == 1 ? a : T(0);
    }
}

template <typename T>
__global__ void k_hist_mul_vjp(const int32_t *__restrict__ keys, const T *__restrict__ vals,
                               const T *__restrict__ anz, const T *__restrict__ az, T *__restrict__ vb,
                               const int64_t n, const int64_t m, const int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t keep = l2_evict_last_policy();  // the coefficient tables stay in L2; keys and values stream
    auto grad = [&](int32_t k, T v) -> T {
        if (!in_range(k, m)) return T(0);
        return v != T(0) ? div_or_zero(ld_keep(anz + k, keep), v) : ld_keep(az + k, keep);
    };
    // two 4-element groups per thread and step: both groups' loads issued first
    const int64_t nv = n / 8;
    for (int64_t v = g; v < nv; v += stride) {
        const int4 k0 = __ldcs(reinterpret_cast<const int4 *>(keys) + 2 * v);
        const int4 k1 = __ldcs(reinterpret_cast<const int4 *>(keys) + 2 * v + 1);
        T a[8], o[8];
        load_chunk_cs(vals, v * 8, n, a, T(1));
        if (accumulate) load_chunk(vb, v * 8, n, o, T(0));
        const int kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T gv = grad(kk[c], a[c]);
            o[c] = accumulate ? o[c] + gv : gv;
        }
        store_chunk(vb, v * 8, n, o);
    }
    for (int64_t i = nv * 8 + g; i < n; i += stride) {
        const T gv = grad(keys[i], vals[i]);
        vb[i] = accumulate ? vb[i] + gv : gv;
    }
}

template <typename T>
__global__ void k_h0bar_mul(const int32_t *__restrict__ n0, const T *__restrict__ p, const T *__restrict__ hb,
                            T *__restrict__ h0b, const int64_t m, const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const T g = (n0[j] > 0 ? T(0) : p[j]) * hb[j];
        h0b[j] = accumulate ? h0b[j] + g : g;
    }
}

// ================================================================== host ==
static unsigned grid_for(int64_t work, int per_sm) {
    int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

static int g_force_strategy = -1;  // tests: force a strategy (-1: automatic)
static int g_sel_vjp_form = 0;     // min/max vjp: 0 automatic, 1 gather, 2 zero-fill + scatter

constexpr size_t kThrBudget = 64 * 1024;    // per-thread tables: 3 blocks of 256 threads per SM
constexpr size_t kWarpBudget = 48 * 1024;   // 8 per-warp copies, 4 blocks per SM
constexpr size_t kBlockBudget = 200 * 1024; // one copy per 1024-thread block

// Shared-memory bytes per bin and strategy.  MUL keeps its zero counts next to
// the products except in the block-wide table (zeros then go to global memory).
static size_t entry_bytes(adc_op op, size_t s, HistStrategy st) {
    switch (op) {
    case ADC_OP_ADD: return s;
    case ADC_OP_MUL: return st == kSmemBlock ? s : s + 4;
    case ADC_OP_MIN:
    case ADC_OP_MAX: return 8;
    default: return 0;
    }
}

static int part_mode(adc_op op, bool primal) {
    switch (op) {
    case ADC_OP_ADD: return kPAdd;
    case ADC_OP_MUL: return primal ? kPPrimMul : kPMul;
    case ADC_OP_MIN: return primal ? kPPrimMin : kPMin;
    case ADC_OP_MAX: return primal ? kPPrimMax : kPMax;
    default: return -1;
    }
}

// Below this many bins the bucketed tables get too small (heavy shared-memory
// contention) and the single-pass strategies win.
constexpr int64_t kPartMinBins = 1 << 18;

static bool fits(adc_op op, size_t s, HistStrategy st, int64_t m) {
    const size_t e = entry_bytes(op, s, st);
    switch (st) {
    case kPart: return part_applicable(part_mode(op, false), s, m);
    case kSmemThread: return (size_t)m * e * kThrThreads <= kThrBudget;
    case kSmemWarp: return (size_t)m * e * 8 <= kWarpBudget;
    case kSmemBlock: return (size_t)m * e <= kBlockBudget;
    case kSplit:
        return (op == ADC_OP_MIN || op == ADC_OP_MAX) && s == 4 && (size_t)m * 8 > kBlockBudget &&
               (size_t)m * 8 <= 4 * kBlockBudget;
    case kCluster:
        return (op == ADC_OP_MIN || op == ADC_OP_MAX) && s == 4 && (size_t)m * 8 > kBlockBudget &&
               (size_t)m * 8 <= (size_t)kMaxClusterBlocks * kBlockBudget;
    case kTwoPass:
    case kPairs:
        return (op == ADC_OP_MIN || op == ADC_OP_MAX) && s == 4 && (size_t)m * 8 > kBlockBudget &&
               (size_t)m * 4 <= kBlockBudget;
    default: return true;
    }
}

// Strategy for the lifted forward of op on a table of m bins.  fp64 min/max
// always uses the two global phases.
static HistStrategy pick(adc_op op, size_t s, int64_t m) {
    if ((op == ADC_OP_MIN || op == ADC_OP_MAX) && s == 8) return kGlobal;
    if (g_force_strategy >= 0 && g_force_strategy <= 8 && fits(op, s, (HistStrategy)g_force_strategy, m))
        return (HistStrategy)g_force_strategy;
    // min/max updates are rare after the first few values of a bin (a read
    // filters them), so per-warp copies beat per-thread tables there: the
    // latter's larger footprint costs occupancy.
    const bool select = op == ADC_OP_MIN || op == ADC_OP_MAX;
    // (SPLIT and CLUSTER are not chosen automatically: at m = 50,000 they
    // measured no faster than the filtered global atomics -- 0.40 ms for
    // CLUSTER against 0.28 ms.)
    for (HistStrategy st : {kSmemThread, kSmemWarp, kSmemBlock})
        if (!(select && st == kSmemThread) && fits(op, s, st, m)) return st;
    // packed table beyond one block but values within: two passes (at m = 50,000
    // 0.18 ms against 0.25 ms for the filtered global atomics and 0.31 ms for
    // PAIRS, which reads the input from DRAM once but stalls every SM's single
    // block at two barriers per round)
    if (fits(op, s, kTwoPass, m)) return kTwoPass;
    if (m >= kPartMinBins && fits(op, s, kPart, m)) return kPart;
    return kGlobal;
}

struct Launch {
    unsigned grid, block;
    size_t smem;
};

static Launch shape(adc_op op, size_t s, HistStrategy st, int64_t m, int64_t n) {
    const size_t e = entry_bytes(op, s, st);
    switch (st) {
    case kSmemThread: return {(unsigned)num_sms() * 3, (unsigned)kThrThreads, (size_t)m * e * kThrThreads};
    case kSmemWarp: return {(unsigned)num_sms() * 4, 256u, (size_t)m * e * 8};
    case kSmemBlock: return {(unsigned)num_sms(), 1024u, (size_t)m * e};
    default: return {grid_for(n / 4 + 1, 8), 256u, 0};
    }
}

template <typename K> static bool set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

static HistStrategy pick_entry(adc_op op, size_t s, size_t e, int64_t m, int *R);

// CLUSTER: blocks per cluster, bins per block, and the partial rows (at most
// one cluster per two SMs).
static int cluster_blocks(int64_t m) { return (int)(((size_t)m * 8 + kBlockBudget - 1) / kBlockBudget); }
static size_t cluster_rows_bytes(int64_t m) { return (size_t)(num_sms() / 2) * (size_t)m * 8; }
// TWOPASS: rows [SMs][m] of 32-bit keys, then best[m] and idx[m].
static size_t twopass_rows(int64_t m) { return align_up((size_t)num_sms() * (size_t)m * 4, 256); }
static size_t twopass_bytes(int64_t m) { return twopass_rows(m) + 2 * align_up((size_t)m * 4, 256); }
// PAIRS: one block per SM, so num_sms() / 2 pairs, each with a row of values
// and a row of indices; then best and idx as for TWOPASS.
static int pairs_count() { return num_sms() / 2 > 0 ? num_sms() / 2 : 1; }
static size_t pairs_rows(int64_t m) { return align_up((size_t)pairs_count() * (size_t)m * 4, 256); }
static size_t pairs_bytes(int64_t m) { return 2 * pairs_rows(m) + 2 * align_up((size_t)m * 4, 256); }

// Partial tables of the shared-memory * strategies (one row of m products, and
// for the lifted form m zero counts, per block), at the workspace's start: the
// lifted forward's strategy and the original primal's, whichever is larger.
static size_t mul_partial_p(size_t s, int64_t G, int64_t m) { return align_up((size_t)G * m * s, 256); }
static size_t mul_partial_bytes(size_t s, int64_t m) {
    size_t b = 0;
    const HistStrategy st = pick(ADC_OP_MUL, s, m);
    if (st == kSmemThread || st == kSmemWarp || st == kSmemBlock) {
        const int64_t G = shape(ADC_OP_MUL, s, st, m, 0).grid;
        b = mul_partial_p(s, G, m) + align_up((size_t)G * m * 4, 256);
    }
    int R;
    const HistStrategy sp = pick_entry(ADC_OP_MUL, s, s, m, &R);
    if (sp == kSmemWarp || sp == kSmemBlock) {
        const size_t c = mul_partial_p(s, sp == kSmemWarp ? (int64_t)num_sms() * 4 : (int64_t)num_sms(), m);
        b = c > b ? c : b;
    }
    return b;
}

// Workspace: the header, the operator's tables, then (where the partitioned
// strategy can run) its scratch at part_off().
static size_t base_ws(adc_op op, adc_dtype dt, int64_t m) {
    switch (op) {
    case ADC_OP_ADD: return kWsHeader;
    case ADC_OP_MUL: {
        const size_t vjp_tables = 2 * align_up((size_t)m * 8, 256);
        const size_t partials = mul_partial_bytes(dt == ADC_F64 ? 8 : 4, m);
        return kWsHeader + (vjp_tables > partials ? vjp_tables : partials);
    }
    case ADC_OP_MIN:
    case ADC_OP_MAX: {
        const size_t tab = (size_t)m * 8 + (dt == ADC_F64 ? (size_t)m * 4 + 256 : 0);
        // (CLUSTER is not chosen automatically: its rows only when it is forced)
        size_t rows =
            dt == ADC_F32 && g_force_strategy == kCluster && fits(op, 4, kCluster, m) ? cluster_rows_bytes(m) : 0;
        if (dt == ADC_F32 && fits(op, 4, kTwoPass, m)) {
            const size_t t = twopass_bytes(m) > pairs_bytes(m) ? twopass_bytes(m) : pairs_bytes(m);
            rows = t > rows ? t : rows;
        }
        return kWsHeader + (tab > rows ? tab : rows);
    }
    default: return 0;
    }
}
static size_t part_off(adc_op op, adc_dtype dt, int64_t m) { return align_up(base_ws(op, dt, m), 256); }

static size_t hist_ws_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    const size_t s = dt == ADC_F64 ? 8 : 4;
    // the partition scratch (about n * (2 + value bytes)) only where it can be chosen
    if (m < kPartMinBins && g_force_strategy != kPart) return base_ws(op, dt, m);
    const size_t a = part_ws_bytes(part_mode(op, false), s, n, m);
    const size_t b = part_ws_bytes(part_mode(op, true), s, n, m);
    return part_off(op, dt, m) + (a > b ? a : b);
}

size_t hist_ws_bytes(adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    if (op == ADC_OP_LIN) return histgen_ws_bytes(dt, n, m);
    if (op == ADC_OP_SOP) return kWsHeader;
    if (op != ADC_OP_ADD && op != ADC_OP_MUL && op != ADC_OP_MIN && op != ADC_OP_MAX) return 0;
    const size_t f = hist_ws_fwd(op, dt, n, m);
    if (op != ADC_OP_MIN && op != ADC_OP_MAX) return f;
    // the min/max vjp's bitmap form: one bit per element after the header
    const size_t bits = kWsHeader + align_up((size_t)((n + 31) / 32) * 4, 256);
    return f > bits ? f : bits;
}

size_t hist_saved_bytes(adc_op op, adc_dtype dt, int64_t n, int64_t m) {
    const size_t s = dt == ADC_F64 ? 8 : 4;
    switch (op) {
    case ADC_OP_ADD:
    case ADC_OP_SOP: return 16;
    case ADC_OP_MIN:
    case ADC_OP_MAX: return (size_t)m * 4;
    case ADC_OP_MUL: return align_up((size_t)m * 4, 16) + (size_t)m * s;
    case ADC_OP_LIN: return histgen_saved_bytes(dt, n, m);
    default: return 0;
    }
}

// Strategy for the un-lifted primal's table of `e`-byte entries (the same
// choices as the lifted forward's, so that the AD overhead compares like with
// like).
static HistStrategy pick_entry(adc_op op, size_t s, size_t e, int64_t m, int *R) {
    HistStrategy st;
    const bool part = part_applicable(part_mode(op, true), s, m);
    if (g_force_strategy == kPart && part) st = kPart;
    else if ((size_t)m * e * 8 <= kWarpBudget) st = kSmemWarp;
    else if ((size_t)m * e <= kBlockBudget) st = kSmemBlock;
    else if (m >= kPartMinBins && part) st = kPart;
    else st = kGlobal;
    *R = (st == kSmemWarp) ? 8 : 1;
    return st;
}

template <typename T>
static adc_status hist_primal_t(adc_op op, int64_t n, int64_t m, const int32_t *keys, const T *vals, const T *h0,
                                T *hist, void *ws, cudaStream_t s) {
    char *w = static_cast<char *>(ws);
    unsigned *err = reinterpret_cast<unsigned *>(w);
    const unsigned gm = grid_for(m, 4);
    const unsigned gglob = grid_for(n / 4 + 1, 8);
    int R;
    const adc_dtype dt = dt_of<T>();
    if (op == ADC_OP_MUL) {
        const HistStrategy st = pick_entry(op, sizeof(T), sizeof(T), m, &R);
        if (st == kPart && n > 0)
            return part_fwd(kPPrimMul, dt, n, m, keys, vals, h0, hist, nullptr, nullptr, nullptr, ws,
                            part_off(op, dt, m), s);
        if (n == 0 || st == kGlobal) {
            k_hist_init<T><<<gm, 256, 0, s>>>(hist, h0, m, T(1));
            if (n > 0) k_prim_mul_global<T><<<gglob, 256, 0, s>>>(keys, vals, n, m, hist, err);
            return check_launch();
        }
        // shared-memory strategies: per-block partial rows, combined by k_mul_reduce
        const size_t smem = (size_t)m * sizeof(T) * R;
        if (cudaFuncSetAttribute(k_prim_mul_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return ADC_ERR_CUDA;
        const int G = st == kSmemWarp ? num_sms() * 4 : num_sms();
        T *P = reinterpret_cast<T *>(w + kWsHeader);
        k_prim_mul_smem<T><<<G, st == kSmemWarp ? 256 : 1024, smem, s>>>(keys, vals, n, m, R, P, err);
        k_mul_reduce<T><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(P, nullptr, G, m, nullptr, nullptr, h0, hist);
        return check_launch();
    }
    const bool mx = op == ADC_OP_MAX;
    if (n > 0 && pick_entry(op, sizeof(T), sizeof(T), m, &R) == kPart)
        return part_fwd(mx ? kPPrimMax : kPPrimMin, dt, n, m, keys, vals, h0, hist, nullptr, nullptr, nullptr, ws,
                        part_off(op, dt, m), s);
    if constexpr (sizeof(T) == 4) {
        uint32_t *tab = reinterpret_cast<uint32_t *>(w + kWsHeader);
        const HistStrategy st = pick_entry(op, 4, 4, m, &R);
        if (mx) k_ord32_init<true><<<gm, 256, 0, s>>>(tab, m);
        else k_ord32_init<false><<<gm, 256, 0, s>>>(tab, m);
        if (n > 0) {
            if (st == kGlobal) {
                if (mx) k_prim_sel_global<true><<<gglob, 256, 0, s>>>(keys, vals, n, m, tab);
                else k_prim_sel_global<false><<<gglob, 256, 0, s>>>(keys, vals, n, m, tab);
            } else {
                auto kern = mx ? k_prim_sel_smem<true> : k_prim_sel_smem<false>;
                const size_t smem = (size_t)m * 4 * R;
                if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                    return ADC_ERR_CUDA;
                kern<<<st == kSmemWarp ? num_sms() * 4 : num_sms(), st == kSmemWarp ? 256 : 1024, smem, s>>>(
                    keys, vals, n, m, R, tab);
            }
        }
        if (mx) k_prim_sel_final<true, float, uint32_t><<<gm, 256, 0, s>>>(tab, h0, m, hist, 0u);
        else k_prim_sel_final<false, float, uint32_t><<<gm, 256, 0, s>>>(tab, h0, m, hist, 0xffffffffu);
    } else {
        unsigned long long *tab = reinterpret_cast<unsigned long long *>(w + kWsHeader);
        unsigned *ti = reinterpret_cast<unsigned *>(w + kWsHeader + align_up((size_t)m * 8, 256));
        const unsigned long long empty = mx ? 0ull : ~0ull;
        k_sel64_init<<<gm, 256, 0, s>>>(tab, ti, m, empty);
        if (n > 0) {
            if (mx) k_hist_sel64_value<true><<<gglob, 256, 0, s>>>(keys, vals, n, m, tab);
            else k_hist_sel64_value<false><<<gglob, 256, 0, s>>>(keys, vals, n, m, tab);
        }
        if (mx) k_prim_sel_final<true, double, unsigned long long><<<gm, 256, 0, s>>>(tab, h0, m, hist, empty);
        else k_prim_sel_final<false, double, unsigned long long><<<gm, 256, 0, s>>>(tab, h0, m, hist, empty);
    }
    return check_launch();
}

template <typename T>
static adc_status hist_fwd_t(adc_op op, int64_t n, int64_t m, const int32_t *keys, const T *vals, const T *h0,
                             T *hist, void *saved, void *ws, cudaStream_t s) {
    if (saved == nullptr && op != ADC_OP_ADD) return hist_primal_t<T>(op, n, m, keys, vals, h0, hist, ws, s);
    char *w = static_cast<char *>(ws);
    unsigned *err = reinterpret_cast<unsigned *>(w);
    const HistStrategy st = pick(op, sizeof(T), m);
    const Launch L = shape(op, sizeof(T), st, m, n);
    const unsigned gm = grid_for(m, 4);
    switch (op) {
    case ADC_OP_ADD: {
        if (st == kPart && n > 0)
            return part_fwd(kPAdd, dt_of<T>(), n, m, keys, vals, h0, hist, nullptr, nullptr, nullptr, ws,
                            part_off(op, dt_of<T>(), m), s);
        k_hist_init<T><<<gm, 256, 0, s>>>(hist, h0, m, T(0));
        if (n == 0) return check_launch();
        if (st == kGlobal) {
            k_hist_add_global<T><<<L.grid, L.block, 0, s>>>(keys, vals, n, m, hist);
        } else if (st == kSmemThread) {
            if (!set_smem(k_hist_add_thread<T>, L.smem)) return ADC_ERR_CUDA;
            k_hist_add_thread<T><<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, hist);
        } else {
            if (!set_smem(k_hist_add_smem<T>, L.smem)) return ADC_ERR_CUDA;
            k_hist_add_smem<T><<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, st == kSmemWarp ? 8 : 1, hist);
        }
        return check_launch();
    }
    case ADC_OP_MUL: {
        int32_t *n0 = static_cast<int32_t *>(saved);
        T *p = reinterpret_cast<T *>(static_cast<char *>(saved) + align_up((size_t)m * 4, 16));
        if (st == kPart && n > 0) {
            // the table blocks write n0, p and hist: no finaliser
            return part_fwd(kPMul, dt_of<T>(), n, m, keys, vals, h0, hist, n0, p, nullptr, ws,
                            part_off(op, dt_of<T>(), m), s);
        }
        // shared-memory strategies: per-block partial rows, combined by k_mul_reduce
        const bool partial = n > 0 && (st == kSmemThread || st == kSmemWarp || st == kSmemBlock);
        T *P = reinterpret_cast<T *>(w + kWsHeader);
        int32_t *Z = reinterpret_cast<int32_t *>(w + kWsHeader + mul_partial_p(sizeof(T), L.grid, m));
        if (!partial || st == kSmemBlock) k_mul_init<T><<<gm, 256, 0, s>>>(n0, p, m);
        if (n > 0) {
            if (st == kGlobal) {
                k_hist_mul_global<T><<<L.grid, L.block, 0, s>>>(keys, vals, n, m, n0, p, err);
            } else if (st == kSmemThread) {
                if (!set_smem(k_hist_mul_thread<T>, L.smem)) return ADC_ERR_CUDA;
                k_hist_mul_thread<T><<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, P, Z, err);
            } else if (st == kSmemBlock) {
                if (!set_smem(k_hist_mul_smem_prod<T>, L.smem)) return ADC_ERR_CUDA;
                k_hist_mul_smem_prod<T><<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, n0, P, err);
            } else {
                if (!set_smem(k_hist_mul_smem<T>, L.smem)) return ADC_ERR_CUDA;
                k_hist_mul_smem<T><<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, 8, P, Z, err);
            }
        }
        if (partial)
            k_mul_reduce<T><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(P, st == kSmemBlock ? nullptr : Z, (int)L.grid,
                                                                       m, n0, p, h0, hist);
        else
            k_hist_mul_final<T><<<gm, 256, 0, s>>>(n0, p, h0, m, hist);
        return check_launch();
    }
    case ADC_OP_MIN:
    case ADC_OP_MAX: {
        const bool mx = op == ADC_OP_MAX;
        unsigned long long *tab = reinterpret_cast<unsigned long long *>(w + kWsHeader);
        int32_t *is = static_cast<int32_t *>(saved);
        if constexpr (sizeof(T) == 4) {
            if (st == kPart && n > 0) {
                // the table blocks decode their bins into hist and is: no finaliser
                return part_fwd(mx ? kPMax : kPMin, ADC_F32, n, m, keys, vals, h0, hist, nullptr, nullptr, is, ws,
                                part_off(op, ADC_F32, m), s);
            } else if (!(n > 0 && (st == kTwoPass || st == kPairs || st == kCluster))) {  // those build their own tables
                if (mx) k_pack_init<true><<<gm, 256, 0, s>>>(tab, m);
                else k_pack_init<false><<<gm, 256, 0, s>>>(tab, m);
            }
            if (n > 0 && st != kPart) {
                if (st == kGlobal) {
                    if (mx) k_hist_sel_global<true><<<L.grid, L.block, 0, s>>>(keys, vals, n, m, tab, n >= 16 * m);
                    else k_hist_sel_global<false><<<L.grid, L.block, 0, s>>>(keys, vals, n, m, tab, n >= 16 * m);
                } else if (st == kPairs) {
                    const int P = pairs_count();
                    uint32_t *rows_val = reinterpret_cast<uint32_t *>(tab);  // the rows take the packed table's place
                    uint32_t *rows_idx = rows_val + pairs_rows(m) / 4;
                    uint32_t *best = rows_idx + pairs_rows(m) / 4;
                    uint32_t *idx = best + align_up((size_t)m * 4, 256) / 4;
                    const int64_t W = (m + 1) / 2;
                    const size_t smem = (size_t)W * 8;
                    auto p1 = mx ? k_sel_pairs<true> : k_sel_pairs<false>;
                    if (!set_smem(p1, smem)) return ADC_ERR_CUDA;
                    p1<<<2 * P, 1024, smem, s>>>(keys, vals, n, m, W, rows_val, rows_idx);
                    if (mx)
                        k_sel_pair_rows_reduce<true><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(rows_val, rows_idx, P,
                                                                                                 m, best, idx);
                    else
                        k_sel_pair_rows_reduce<false><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(rows_val, rows_idx, P,
                                                                                                  m, best, idx);
                    if (mx) k_sel_twopass_final<true><<<gm, 256, 0, s>>>(best, idx, vals, h0, m, n, hist, is);
                    else k_sel_twopass_final<false><<<gm, 256, 0, s>>>(best, idx, vals, h0, m, n, hist, is);
                    return check_launch();
                } else if (st == kTwoPass) {
                    const int G = num_sms();
                    uint32_t *rows = reinterpret_cast<uint32_t *>(tab);  // the rows take the packed table's place
                    uint32_t *best = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(tab) + twopass_rows(m));
                    uint32_t *idx = best + align_up((size_t)m * 4, 256) / 4;
                    const size_t smem = (size_t)m * 4;
                    auto p1 = mx ? k_sel_val_rows<true> : k_sel_val_rows<false>;
                    auto p2 = mx ? k_sel_index_pass<true> : k_sel_index_pass<false>;
                    if (!set_smem(p1, smem) || !set_smem(p2, smem)) return ADC_ERR_CUDA;
                    p1<<<G, 1024, smem, s>>>(keys, vals, n, m, rows);
                    if (mx) k_ord_rows_reduce<true><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(rows, G, m, best, idx);
                    else k_ord_rows_reduce<false><<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(rows, G, m, best, idx);
                    p2<<<G, 1024, smem, s>>>(keys, vals, n, m, best, idx);
                    if (mx) k_sel_twopass_final<true><<<gm, 256, 0, s>>>(best, idx, vals, h0, m, n, hist, is);
                    else k_sel_twopass_final<false><<<gm, 256, 0, s>>>(best, idx, vals, h0, m, n, hist, is);
                    return check_launch();
                } else if (st == kCluster) {
                    const int CS = cluster_blocks(m);
                    const int64_t H = (m + CS - 1) / CS;
                    const size_t smem = (size_t)H * 8;
                    auto kern = mx ? k_hist_sel_cluster<true> : k_hist_sel_cluster<false>;
                    if (!set_smem(kern, smem)) return ADC_ERR_CUDA;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeClusterDimension;
                    attr[0].val.clusterDim.x = (unsigned)CS;
                    attr[0].val.clusterDim.y = 1;
                    attr[0].val.clusterDim.z = 1;
                    cudaLaunchConfig_t cfg = {};
                    cfg.blockDim = dim3(1024);
                    cfg.dynamicSmemBytes = smem;
                    cfg.stream = s;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    cfg.gridDim = dim3((unsigned)((num_sms() / CS) * CS));
                    // one wave of clusters: as many as can be resident at once
                    int active = 0;
                    if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) != cudaSuccess || active < 1)
                        return ADC_ERR_CUDA;
                    const int C = active < num_sms() / CS ? active : num_sms() / CS;
                    cfg.gridDim = dim3((unsigned)(C * CS));
                    unsigned long long *rows = tab;  // the rows take the packed table's place
                    if (cudaLaunchKernelEx(&cfg, kern, keys, vals, n, m, CS, H, rows, err) != cudaSuccess)
                        return ADC_ERR_CUDA;
                    auto red = mx ? k_sel_reduce<true> : k_sel_reduce<false>;
                    red<<<(unsigned)((m + 31) / 32), 1024, 0, s>>>(rows, C, m, vals, h0, n, hist, is);
                    return check_launch();
                } else if (st == kSplit) {
                    const int S = (int)(((size_t)m * 8 + kBlockBudget - 1) / kBlockBudget);
                    const int64_t W = (m + S - 1) / S;
                    const size_t smem = (size_t)W * 8;
                    auto kern = mx ? k_hist_sel_split<true> : k_hist_sel_split<false>;
                    if (!set_smem(kern, smem)) return ADC_ERR_CUDA;
                    const int groups = num_sms() / S > 0 ? num_sms() / S : 1;
                    kern<<<(unsigned)(groups * S), 1024, smem, s>>>(keys, vals, n, m, S, W, tab);
                } else if (st == kSmemThread) {
                    auto kern = mx ? k_hist_sel_thread<true> : k_hist_sel_thread<false>;
                    if (!set_smem(kern, L.smem)) return ADC_ERR_CUDA;
                    kern<<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, tab);
                } else {
                    auto kern = mx ? k_hist_sel_smem<true> : k_hist_sel_smem<false>;
                    if (!set_smem(kern, L.smem)) return ADC_ERR_CUDA;
                    kern<<<L.grid, L.block, L.smem, s>>>(keys, vals, n, m, st == kSmemWarp ? 8 : 1, tab);
                }
            }
            if (mx) k_hist_sel_final<true><<<gm, 256, 0, s>>>(tab, vals, h0, m, n, hist, is);
            else k_hist_sel_final<false><<<gm, 256, 0, s>>>(tab, vals, h0, m, n, hist, is);
        } else {
            const unsigned gg = grid_for(n / 4 + 1, 8);
            unsigned *ti = reinterpret_cast<unsigned *>(w + kWsHeader + align_up((size_t)m * 8, 256));
            k_sel64_init<<<gm, 256, 0, s>>>(tab, ti, m, mx ? 0ull : ~0ull);
            if (n > 0) {
                if (mx) {
                    k_hist_sel64_value<true><<<gg, 256, 0, s>>>(keys, vals, n, m, tab);
                    k_hist_sel64_index<true><<<gg, 256, 0, s>>>(keys, vals, n, m, tab, ti);
                } else {
                    k_hist_sel64_value<false><<<gg, 256, 0, s>>>(keys, vals, n, m, tab);
                    k_hist_sel64_index<false><<<gg, 256, 0, s>>>(keys, vals, n, m, tab, ti);
                }
            }
            if (mx) k_hist_sel64_final<true><<<gm, 256, 0, s>>>(ti, vals, h0, m, n, hist, is);
            else k_hist_sel64_final<false><<<gm, 256, 0, s>>>(ti, vals, h0, m, n, hist, is);
        }
        return check_launch();
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status hist_fwd(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, void *hist, void *saved, void *ws, cudaStream_t s) {
    if (op == ADC_OP_LIN) return histgen_fwd(dt, n, m, keys, vals, hist0, hist, saved, ws, s);
    if (op == ADC_OP_SOP) return sop_hist_fwd(dt, n, m, keys, vals, hist0, hist, s);
    if (dt == ADC_F64)
        return hist_fwd_t<double>(op, n, m, keys, static_cast<const double *>(vals), static_cast<const double *>(hist0),
                                  static_cast<double *>(hist), saved, ws, s);
    return hist_fwd_t<float>(op, n, m, keys, static_cast<const float *>(vals), static_cast<const float *>(hist0),
                             static_cast<float *>(hist), saved, ws, s);
}

template <typename T>
static adc_status hist_vjp_t(adc_op op, int64_t n, int64_t m, const int32_t *keys, const T *vals, const T *h0,
                             const void *saved, const T *hb, T *vb, T *h0b, int acc, void *ws, cudaStream_t s) {
    const unsigned gm = grid_for(m, 4);
    const unsigned gn = grid_for(n / 4 + 1, 8);
    const unsigned gn8 = grid_for(n / 8 + 1, 8);  // the * vjp: 8 elements per step
    switch (op) {
    case ADC_OP_ADD:
        if (n > 0) k_hist_add_vjp<T><<<gn, 256, 0, s>>>(keys, hb, vb, n, m, acc);
        if (h0b) k_h0bar_add<T><<<gm, 256, 0, s>>>(hb, h0b, m, acc);
        return check_launch();
    case ADC_OP_MIN:
    case ADC_OP_MAX: {
        const int32_t *is = static_cast<const int32_t *>(saved);
        // few values per bin (8m > n): the bitmap of selected elements, then one
        // streaming pass (measured faster than the gather pass at m = 1e7,
        // n = 5e7: 0.147 against 0.239 ms); many values per bin: zero-fill and
        // scatter
        const bool sparse = m * 8 > n;
        if (g_sel_vjp_form == 3 || (g_sel_vjp_form == 0 && sparse)) {
            uint32_t *bits = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + kWsHeader);
            if (n > 0) {
                if (cudaMemsetAsync(bits, 0, (size_t)((n + 31) / 32) * 4, s) != cudaSuccess) return ADC_ERR_CUDA;
                k_sel_bits<<<gm, 256, 0, s>>>(is, bits, m, n);
                k_hist_sel_vjp_bits<T><<<gn, 256, 0, s>>>(keys, bits, hb, vb, n, m, acc);
            }
            if (h0b) k_h0bar_sel<T><<<gm, 256, 0, s>>>(is, hb, h0b, m, n, acc);
            return check_launch();
        }
        if (g_sel_vjp_form == 1) {  // one gather pass (is[k_i] == i)
            if (n > 0) k_hist_sel_vjp_gather<T><<<gn, 256, 0, s>>>(keys, is, hb, vb, n, m, acc);
            if (h0b) k_h0bar_sel<T><<<gm, 256, 0, s>>>(is, hb, h0b, m, n, acc);
        } else {          // many values per bin: zero-fill, then scatter m adjoints
            if (!acc && n > 0) k_fill<T><<<grid_for(n / 4 + 1, 8), 256, 0, s>>>(vb, n);
            k_hist_sel_vjp<T><<<gm, 256, 0, s>>>(is, hb, vb, h0b, m, n, acc);
        }
        return check_launch();
    }
    case ADC_OP_MUL: {
        const int32_t *n0 = static_cast<const int32_t *>(saved);
        const T *p = reinterpret_cast<const T *>(static_cast<const char *>(saved) + align_up((size_t)m * 4, 16));
        T *anz = reinterpret_cast<T *>(static_cast<char *>(ws) + kWsHeader);
        T *az = reinterpret_cast<T *>(static_cast<char *>(ws) + kWsHeader + align_up((size_t)m * sizeof(T), 256));
        if (n > 0) {
            k_mul_vjp_prep<T><<<gm, 256, 0, s>>>(n0, p, h0, hb, anz, az, m);
            k_hist_mul_vjp<T><<<gn8, 256, 0, s>>>(keys, vals, anz, az, vb, n, m, acc);
        }
        if (h0b) k_h0bar_mul<T><<<gm, 256, 0, s>>>(n0, p, hb, h0b, m, acc);
        return check_launch();
    }
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status hist_vjp(adc_op op, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, const void *hist, const void *saved, const void *histbar, void *valsbar,
                    void *hist0bar, int accumulate, void *ws, cudaStream_t s) {
    if (op == ADC_OP_LIN)
        return histgen_vjp(dt, n, m, keys, vals, hist0, hist, saved, histbar, valsbar, hist0bar, accumulate, ws, s);
    if (op == ADC_OP_SOP)
        return sop_hist_vjp(dt, n, m, keys, vals, hist0, hist, histbar, valsbar, hist0bar, accumulate, s);
    if (dt == ADC_F64)
        return hist_vjp_t<double>(op, n, m, keys, static_cast<const double *>(vals),
                                  static_cast<const double *>(hist0), saved, static_cast<const double *>(histbar),
                                  static_cast<double *>(valsbar), static_cast<double *>(hist0bar), accumulate, ws, s);
    return hist_vjp_t<float>(op, n, m, keys, static_cast<const float *>(vals), static_cast<const float *>(hist0), saved,
                             static_cast<const float *>(histbar), static_cast<float *>(valsbar),
                             static_cast<float *>(hist0bar), accumulate, ws, s);
}

}  // namespace adc

extern "C" void adc_debug_force_hist_strategy(int s) { adc::g_force_strategy = s; }
extern "C" void adc_debug_set_sel_vjp_form(int f) { adc::g_sel_vjp_form = (f >= 0 && f <= 3) ? f : 0; }
int adc::hist_forced_strategy() { return adc::g_force_strategy; }
