// reduce_by_index for tables far larger than shared memory, with the
// specialised operators of Sec. 4.2 (+, the lifted * with zero counting, the
// lifted min/max of Fig. 5) and the un-lifted primals.  Sec. 4.2.6's design
// space -- private sub-histograms in fast memory, merged afterwards -- carried
// to tables of millions of bins by partitioning the elements first.
//
// With m in the millions a direct global-atomic histogram makes every element
// a random L2 round trip (two for the compare-and-swap multiply) and waits on
// L2 latency with DRAM nearly idle.  Here the bins are split into B buckets of
// W consecutive bins, W chosen so that one bucket's table fills one block's
// shared memory, and the elements are moved by bucket into scratch:
//   1. count   per chunk of kPartChunk elements, how many fall in each bucket;
//   2. scan    exclusive +-scan of the bucket-major count matrix: where each
//              (bucket, chunk) run starts (the look-back scan engine);
//   3. scatter each chunk is counting-sorted by bucket in shared memory and
//              written out as contiguous runs of (bin within the bucket, 16
//              bits; payload), the payload being the value (+, *) or the packed
//              (value, index) key (lifted min/max); for fp32 a persistent block
//              per SM with the chunks staged by bulk (TMA) copies one ahead;
//   4. table   one block per bucket streams its run into a shared-memory table
//              of W bins and writes them out.  Every bin belongs to exactly one
//              bucket, so there are no global atomics at all.
// Traffic per element, fp32 *: 4 (count) + 8 + 6 (scatter) + 6 (table) bytes,
// all streaming.  The order in which a bin's values meet differs from the
// sequential loop only by the associativity and commutativity these operators
// have; min/max stay exact (the index travels with the value).
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"
#include "tile_io.cuh"
#include "tma.cuh"

namespace adc {

constexpr int kPartThreads = 512;                      // count and scatter blocks
constexpr int kPartItems = 16;                         // elements per thread per chunk
constexpr int kPartChunk = kPartThreads * kPartItems;  // 8192 elements
constexpr int kPartMaxBuckets = 2048;
constexpr int kPartTableThreads = 1024;
constexpr size_t kPartTableBudget = 200 * 1024;  // one table block per SM
constexpr int kPartSlot = 20;                    // workspace counter slot of the count scan

// k / W for in-range keys by a float reciprocal and one correction step: the
// quotients stay below 2^11, so the float estimate is off by at most one.
struct BucketDiv {
    uint32_t W;
    float inv;
    __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
        uint32_t b = __float2uint_rz(__uint2float_rz(k) * inv);
        if (b * W > k) --b;
        else if ((b + 1) * W <= k) ++b;
        return b;
    }
};

template <typename T> struct PartOut {
    T *hist;
    const T *h0;
    int32_t *n0;
    T *p;
    int32_t *is;     // lifted min/max: selected index per bin
    const T *vals;   // lifted min/max: the input values (a selected zero's sign)
    int64_t n;
};

// Order-preserving key type of a value type (un-lifted min/max).
template <typename T> struct OrdOf { using type = uint32_t; };
template <> struct OrdOf<double> { using type = unsigned long long; };

// ------------------------------------------------------------ per-mode ops --
// V: payload written by the scatter; kEntry: table bytes per bin; init /
// update / flush act on the shared-memory table of one bucket (W bins).
template <typename T, int MODE> struct PartTraits;

template <typename T> struct PartTraits<T, kPAdd> {
    using V = T;
    static constexpr size_t kEntry = sizeof(T);
    static __device__ __forceinline__ V enc(T v, int64_t) { return v; }
    static __device__ __forceinline__ void init(unsigned char *sm, int, int t) { reinterpret_cast<T *>(sm)[t] = T(0); }
    template <int U>
    static __device__ __forceinline__ void update(unsigned char *sm, int, const int32_t (&u)[U], const V (&v)[U],
                                                  const bool (&use)[U], unsigned *) {
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (use[j]) atomicAdd(reinterpret_cast<T *>(sm) + u[j], v[j]);
    }
    static __device__ __forceinline__ void flush(const unsigned char *sm, int, int t, int64_t j, const PartOut<T> &o) {
        const T a = reinterpret_cast<const T *>(sm)[t];
        o.hist[j] = o.h0 ? o.h0[j] + a : a;
    }
};

// Lifted * (Sec. 4.2.3): products of the non-zero values and zero counts.
template <typename T> struct PartTraits<T, kPMul> {
    using V = T;
    static constexpr size_t kEntry = sizeof(T) + 4;
    static __device__ __forceinline__ V enc(T v, int64_t) { return v; }
    static __device__ __forceinline__ void init(unsigned char *sm, int W, int t) {
        reinterpret_cast<T *>(sm)[t] = T(1);
        reinterpret_cast<int32_t *>(sm + (size_t)W * sizeof(T))[t] = 0;
    }
    template <int U>
    static __device__ __forceinline__ void update(unsigned char *sm, int W, const int32_t (&u)[U], const V (&v)[U],
                                                  const bool (&use)[U], unsigned *err) {
        // one compare-and-swap chain at a time: in shared memory the chains are
        // short and batching them only adds registers (measured slower)
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (!use[j]) continue;
            if (v[j] == T(0)) atomicAdd(reinterpret_cast<int32_t *>(sm + (size_t)W * sizeof(T)) + u[j], 1);
            else atomic_mul(reinterpret_cast<T *>(sm) + u[j], v[j], err);
        }
    }
    static __device__ __forceinline__ void flush(const unsigned char *sm, int W, int t, int64_t j, const PartOut<T> &o) {
        const T p = reinterpret_cast<const T *>(sm)[t];
        const int32_t z = reinterpret_cast<const int32_t *>(sm + (size_t)W * sizeof(T))[t];
        o.p[j] = p;
        o.n0[j] = z;
        const T xs = z > 0 ? T(0) : p;  // the bin's product (Fig. 3's lifted primal)
        o.hist[j] = o.h0 ? o.h0[j] * xs : xs;
    }
};

// Lifted min/max (Fig. 5), fp32: the packed (value, index) key.
template <bool MAX> struct PartSel {
    using V = unsigned long long;
    static constexpr size_t kEntry = 8;
    static __device__ __forceinline__ V enc(float v, int64_t i) { return Pack<MAX>::key(v, i); }
    static __device__ __forceinline__ void init(unsigned char *sm, int, int t) {
        reinterpret_cast<V *>(sm)[t] = Pack<MAX>::kEmpty;
    }
    // Few values per bin at the sizes this strategy serves: most updates win,
    // so the atomic is issued without a read filter.
    template <int U>
    static __device__ __forceinline__ void update(unsigned char *sm, int, const int32_t (&u)[U], const V (&v)[U],
                                                  const bool (&use)[U], unsigned *) {
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (!use[j]) continue;
            if (MAX) atomicMax(reinterpret_cast<V *>(sm) + u[j], v[j]);
            else atomicMin(reinterpret_cast<V *>(sm) + u[j], v[j]);
        }
    }
    // Decode the bin's key, fold hist0 in (it wins ties), write hist and is.
    static __device__ __forceinline__ void flush(const unsigned char *sm, int, int t, int64_t j,
                                                 const PartOut<float> &o) {
        const V key = reinterpret_cast<const V *>(sm)[t];
        float v = MAX ? -Num<float>::inf() : Num<float>::inf();
        int64_t idx = o.n;
        if (key != Pack<MAX>::kEmpty) {
            idx = Pack<MAX>::index(key);
            // the key holds the value; only a zero needs the stored element
            // (the key folds -0.0 onto +0.0)
            v = from_ordered((uint32_t)(key >> 32));
            if (v == 0.0f) v = o.vals[idx];
        }
        if (o.h0) {
            const float a = o.h0[j];
            if (MAX ? (a >= v) : (a <= v)) {
                v = a;
                idx = o.n;
            }
        }
        o.hist[j] = v;
        o.is[j] = (int32_t)idx;
    }
};
template <> struct PartTraits<float, kPMin> : PartSel<false> {};
template <> struct PartTraits<float, kPMax> : PartSel<true> {};

// Un-lifted * (the original program): the plain product, zeros included.
template <typename T> struct PartTraits<T, kPPrimMul> {
    using V = T;
    static constexpr size_t kEntry = sizeof(T);
    static __device__ __forceinline__ V enc(T v, int64_t) { return v; }
    static __device__ __forceinline__ void init(unsigned char *sm, int, int t) { reinterpret_cast<T *>(sm)[t] = T(1); }
    template <int U>
    static __device__ __forceinline__ void update(unsigned char *sm, int, const int32_t (&u)[U], const V (&v)[U],
                                                  const bool (&use)[U], unsigned *err) {
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (use[j]) atomic_mul(reinterpret_cast<T *>(sm) + u[j], v[j], err);
    }
    static __device__ __forceinline__ void flush(const unsigned char *sm, int, int t, int64_t j, const PartOut<T> &o) {
        const T a = reinterpret_cast<const T *>(sm)[t];
        o.hist[j] = o.h0 ? o.h0[j] * a : a;
    }
};

// Un-lifted min/max on order-preserving value keys.
template <typename T, bool MAX> struct PartPrimSel {
    using V = typename OrdOf<T>::type;
    static constexpr V kEmpty = MAX ? V(0) : ~V(0);
    static constexpr size_t kEntry = sizeof(V);
    static __device__ __forceinline__ V enc(T v, int64_t) { return (V)ordered_key(v); }
    static __device__ __forceinline__ void init(unsigned char *sm, int, int t) { reinterpret_cast<V *>(sm)[t] = kEmpty; }
    template <int U>
    static __device__ __forceinline__ void update(unsigned char *sm, int, const int32_t (&u)[U], const V (&v)[U],
                                                  const bool (&use)[U], unsigned *) {
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (!use[j]) continue;
            if (MAX) atomicMax(reinterpret_cast<V *>(sm) + u[j], v[j]);
            else atomicMin(reinterpret_cast<V *>(sm) + u[j], v[j]);
        }
    }
    static __device__ __forceinline__ void flush(const unsigned char *sm, int, int t, int64_t j, const PartOut<T> &o) {
        const V key = reinterpret_cast<const V *>(sm)[t];
        T v = (key == kEmpty) ? (MAX ? -Num<T>::inf() : Num<T>::inf()) : from_ordered(key);
        if (o.h0) v = MAX ? (o.h0[j] >= v ? o.h0[j] : v) : (o.h0[j] <= v ? o.h0[j] : v);
        o.hist[j] = v;
    }
};
template <typename T> struct PartTraits<T, kPPrimMin> : PartPrimSel<T, false> {};
template <typename T> struct PartTraits<T, kPPrimMax> : PartPrimSel<T, true> {};

// ----------------------------------------------------------------- kernels --
// The keys (and values) of one thread's k-th group of 4 in chunk `c`: 128-bit
// loads when the group is whole, element-wise at the ragged end (-1 = absent).
template <typename T>
__device__ __forceinline__ void load_group(const int32_t *__restrict__ keys, const T *__restrict__ vals, int64_t e,
                                           int64_t n, int32_t (&kk)[4], T (&vv)[4]) {
    if (e + 4 <= n) {
        const int4 k = __ldcs(reinterpret_cast<const int4 *>(keys + e));
        kk[0] = k.x;
        kk[1] = k.y;
        kk[2] = k.z;
        kk[3] = k.w;
        if (vals) load_chunk(vals, e, n, vv, T(0));
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            kk[c] = e + c < n ? keys[e + c] : -1;
            if (vals) vv[c] = e + c < n ? vals[e + c] : T(0);
        }
    }
}

// 1. counts[b * nchunks + chunk] = elements of the chunk in bucket b; row B is
// a zero row so that the scanned matrix also gives every bucket's end.
__global__ void __launch_bounds__(kPartThreads)
k_part_count(const int32_t *__restrict__ keys, const int64_t n, const int64_t m, const BucketDiv bdiv, const int B,
             const int64_t nchunks, int32_t *__restrict__ counts) {
    extern __shared__ int32_t s_cnt[];
    for (int b = threadIdx.x; b < B; b += kPartThreads) s_cnt[b] = 0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * kPartChunk;
#pragma unroll
    for (int r = 0; r < kPartItems / 4; ++r) {
        int32_t kk[4];
        float unused[4];
        load_group<float>(keys, nullptr, c0 + 4 * ((int64_t)r * kPartThreads + threadIdx.x), n, kk, unused);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (in_range(kk[c], m)) atomicAdd(&s_cnt[bdiv((uint32_t)kk[c])], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= B; b += kPartThreads)
        counts[(int64_t)b * nchunks + blockIdx.x] = b < B ? s_cnt[b] : 0;
}

// 3. Counting sort of one chunk by bucket in shared memory, then contiguous
// runs out: obin = bin - bucket * W, oval = payload, at offs[b][chunk] + rank.
// Register-lean so that two blocks fit an SM: a thread keeps only each
// element's (bucket, bin) word and its 16-bit rank, and reloads the values
// (just read, so L1/L2 hits) when it places the elements.
template <typename T, int MODE>
__global__ void __launch_bounds__(kPartThreads, 2)
k_part_scatter(const int32_t *__restrict__ keys, const T *__restrict__ vals, const int64_t n, const int64_t m,
               const BucketDiv bdiv, const int B, const int64_t nchunks, const int32_t *__restrict__ offs,
               uint16_t *__restrict__ obin, typename PartTraits<T, MODE>::V *__restrict__ oval) {
    using Tr = PartTraits<T, MODE>;
    using V = typename Tr::V;
    constexpr int NW = kPartThreads / kWarp;
    constexpr int PER = kPartMaxBuckets / kPartThreads;  // buckets per thread in the local scan
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s_v = reinterpret_cast<V *>(smem_raw);                          // [kPartChunk] payloads, bucket order
    uint32_t *s_k = reinterpret_cast<uint32_t *>(s_v + kPartChunk);    // [kPartChunk] bucket << 16 | bin
    int32_t *s_loc = reinterpret_cast<int32_t *>(s_k + kPartChunk);    // [B] counts, then local starts
    int32_t *s_dst = s_loc + B;                                        // [B] global start - local start
    __shared__ int32_t s_part[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < B; b += kPartThreads) s_loc[b] = 0;
    __syncthreads();

    const int64_t c = blockIdx.x;
    uint32_t bk[kPartItems];      // bucket << 16 | bin, or ~0u: not in range
    uint32_t rk2[kPartItems / 2]; // two 16-bit ranks per word
#pragma unroll
    for (int r = 0; r < kPartItems / 4; ++r) {
        const int64_t e = c * kPartChunk + 4 * ((int64_t)r * kPartThreads + tid);
        int32_t kk[4];
        T unused[4];
        load_group<T>(keys, nullptr, e, n, kk, unused);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * r + q;
            uint32_t rank = 0;
            bk[i] = 0xffffffffu;
            if (in_range(kk[q], m)) {
                const uint32_t b = bdiv((uint32_t)kk[q]);
                bk[i] = (b << 16) | ((uint32_t)kk[q] - b * bdiv.W);
                rank = (uint32_t)atomicAdd(&s_loc[b], 1);
            }
            if (i & 1) rk2[i >> 1] |= rank << 16;
            else rk2[i >> 1] = rank;
        }
    }
    __syncthreads();

    // exclusive scan of the B bucket counts (PER consecutive buckets per thread)
    int32_t own[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int b = tid * PER + j;
        own[j] = b < B ? s_loc[b] : 0;
        sum += own[j];
    }
    int32_t inc = sum;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == kWarp - 1) s_part[warp] = inc;
    __syncthreads();
    int32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int32_t x = s_part[w];
        if (w < warp) before += x;
        total += x;
    }
    int32_t run = before + inc - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int b = tid * PER + j;
        if (b < B) {
            s_loc[b] = run;
            s_dst[b] = offs[(int64_t)b * nchunks + c] - run;
            run += own[j];
        }
    }
    __syncthreads();

#pragma unroll
    for (int r = 0; r < kPartItems / 4; ++r) {
        const int64_t e = c * kPartChunk + 4 * ((int64_t)r * kPartThreads + tid);
        T xv[4];
        if (e + 4 <= n) {
            load_chunk(vals, e, n, xv, T(0));
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = e + q < n ? vals[e + q] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * r + q;
            if (bk[i] != 0xffffffffu) {
                const uint32_t rank = (i & 1) ? (rk2[i >> 1] >> 16) : (rk2[i >> 1] & 0xffffu);
                const int pos = s_loc[bk[i] >> 16] + (int)rank;
                s_k[pos] = bk[i];
                s_v[pos] = Tr::enc(xv[q], e + q);
            }
        }
    }
    __syncthreads();
    for (int pos = tid; pos < total; pos += kPartThreads) {
        const uint32_t x = s_k[pos];
        const int64_t g = (int64_t)s_dst[x >> 16] + pos;
        obin[g] = (uint16_t)(x & 0xffffu);
        oval[g] = s_v[pos];
    }
}

// 3 (fp32). The same counting sort as a persistent, double-buffered pipeline:
// block b owns chunks b, b + G, b + 2G, ... (G blocks, one per SM); each
// whole chunk's keys and values arrive in shared memory by two bulk copies
// issued one chunk ahead, so the DRAM reads of the next chunk overlap the
// ranking, the bucket scan and the writes of this one.  The chunk is ranked
// by bucket as above; a permutation of (bucket, element) words in bucket
// order takes the place of the sorted payload copy, and the readout gathers
// key and value from the staged chunk.  The ragged last chunk is loaded by plain loads.
constexpr int kScatThreads = 1024;
static_assert(kPartChunk == (1 << 13), "the permutation word keeps the element in its low 13 bits");
constexpr int kScatItems = kPartChunk / kScatThreads;  // 8 elements per thread

template <int MODE>
__global__ void __launch_bounds__(kScatThreads, 1)
k_part_scatter_tma(const int32_t *__restrict__ keys, const float *__restrict__ vals, const int64_t n, const int64_t m,
                   const BucketDiv bdiv, const int B, const int64_t nchunks, const int32_t *__restrict__ offs,
                   uint16_t *__restrict__ obin, typename PartTraits<float, MODE>::V *__restrict__ oval,
                   unsigned *__restrict__ err, const long long spin_limit) {
    using Tr = PartTraits<float, MODE>;
    constexpr int NW = kScatThreads / kWarp;
    constexpr int PER = kPartMaxBuckets / kScatThreads;  // buckets per thread in the local scan
    constexpr uint32_t kChunkBytes = kPartChunk * 4u;
    extern __shared__ __align__(16) unsigned char smem_raw[];  // bulk copies need 16-byte alignment
    int32_t *const s_key0 = reinterpret_cast<int32_t *>(smem_raw);        // [2][kPartChunk] keys
    float *const s_val0 = reinterpret_cast<float *>(s_key0 + 2 * kPartChunk);  // [2][kPartChunk] values
    uint32_t *const s_perm = reinterpret_cast<uint32_t *>(s_val0 + 2 * kPartChunk);  // [kPartChunk] b << 13 | i
    int32_t *const s_loc = reinterpret_cast<int32_t *>(s_perm + kPartChunk);        // [B]
    int32_t *const s_dst = s_loc + B;                                                // [B]
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int32_t s_part[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t G = gridDim.x;
    const auto whole = [&](int64_t c) { return (c + 1) * (int64_t)kPartChunk <= n; };
    // thread 0: keys and values of chunk c into buffer `buf`
    const auto issue = [&](int64_t c, int buf) {
        fence_proxy_async_smem();
        mbar_expect_tx(&s_bar[buf], 2u * kChunkBytes);
        bulk_g2s(s_key0 + buf * kPartChunk, keys + c * kPartChunk, kChunkBytes, &s_bar[buf]);
        bulk_g2s(s_val0 + buf * kPartChunk, vals + c * kPartChunk, kChunkBytes, &s_bar[buf]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
    }
    for (int b = tid; b < B; b += kScatThreads) s_loc[b] = 0;
    __syncthreads();
    if (tid == 0 && (int64_t)blockIdx.x < nchunks && whole(blockIdx.x)) issue(blockIdx.x, 0);
    uint32_t used0 = 0u, used1 = 0u;  // completed copy phases consumed, per buffer (same in every thread)
    int j = 0;
    for (int64_t c = blockIdx.x; c < nchunks; c += G, ++j) {
        const int buf = j & 1;
        const int64_t cn = c + G;
        const bool next_staged = cn < nchunks && whole(cn);
        if (tid == 0 && next_staged) issue(cn, buf ^ 1);  // that buffer's readers passed the last barrier
        int32_t *const sk = s_key0 + buf * kPartChunk;
        float *const sv = s_val0 + buf * kPartChunk;
        const int64_t e0 = c * kPartChunk;
        const int len = (int)((n - e0) < kPartChunk ? (n - e0) : kPartChunk);
        if (whole(c)) {
            const uint32_t mine = buf ? used1 : used0, other = buf ? used0 : used1;
            const bool ok = mbar_wait_bounded(&s_bar[buf], mine & 1u, spin_limit);
            if (buf) ++used1;
            else ++used0;
            if (!__syncthreads_and(ok)) {
                // give up: report, let the copy in flight into the other buffer land, leave
                if (tid == 0) {
                    set_error(err, kErrTimeout);
                    if (next_staged) mbar_wait_bounded(&s_bar[buf ^ 1], other & 1u, spin_limit);
                }
                return;
            }
        } else {
            for (int i = tid; i < len; i += kScatThreads) {
                sk[i] = keys[e0 + i];
                sv[i] = vals[e0 + i];
            }
            __syncthreads();
        }

        // this chunk's run starts of the thread's buckets in the scan below: loaded
        // now, so that their latency hides behind the ranking
        int32_t gofs[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = tid * PER + q;
            gofs[q] = b < B ? __ldg(offs + (int64_t)b * nchunks + c) : 0;
        }

        // rank every in-range element within its bucket
        uint32_t bk[kScatItems];       // bucket << 16 | bin, or ~0u: absent or out of range
        uint32_t rk2[kScatItems / 2];  // two 16-bit ranks per word
#pragma unroll
        for (int r = 0; r < kScatItems; ++r) {
            const int i = r * kScatThreads + tid;
            uint32_t rank = 0;
            bk[r] = 0xffffffffu;
            if (i < len) {
                const int32_t k = sk[i];
                if (in_range(k, m)) {
                    const uint32_t b = bdiv((uint32_t)k);
                    bk[r] = (b << 16) | ((uint32_t)k - b * bdiv.W);
                    rank = (uint32_t)atomicAdd(&s_loc[b], 1);
                }
            }
            if (r & 1) rk2[r >> 1] |= rank << 16;
            else rk2[r >> 1] = rank;
        }
        __syncthreads();

        // exclusive scan of the B bucket counts (PER consecutive buckets per thread)
        int32_t own[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = tid * PER + q;
            own[q] = b < B ? s_loc[b] : 0;
            sum += own[q];
        }
        int32_t inc = sum;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == kWarp - 1) s_part[warp] = inc;
        __syncthreads();
        int32_t before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int32_t x = s_part[w];
            if (w < warp) before += x;
            total += x;
        }
        int32_t run = before + inc - sum;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = tid * PER + q;
            if (b < B) {
                s_loc[b] = run;
                s_dst[b] = gofs[q] - run;
                run += own[q];
            }
        }
        __syncthreads();

        // the permutation: position in bucket order -> (bucket, element of the chunk)
#pragma unroll
        for (int r = 0; r < kScatItems; ++r) {
            if (bk[r] != 0xffffffffu) {
                const uint32_t rank = (r & 1) ? (rk2[r >> 1] >> 16) : (rk2[r >> 1] & 0xffffu);
                const uint32_t b = bk[r] >> 16;
                s_perm[s_loc[b] + (int)rank] = (b << 13) | (uint32_t)(r * kScatThreads + tid);
            }
        }
        __syncthreads();

        // contiguous runs out; the bucket counters are cleared for the next chunk
        for (int pos = tid; pos < total; pos += kScatThreads) {
            const uint32_t x = s_perm[pos];
            const int i = (int)(x & (kPartChunk - 1));
            const uint32_t b = x >> 13;
            const int32_t g = s_dst[b] + pos;  // < n < 2^31
            obin[g] = (uint16_t)((uint32_t)sk[i] - b * bdiv.W);
            oval[g] = Tr::enc(sv[i], e0 + i);
        }
        for (int b = tid; b < B; b += kScatThreads) s_loc[b] = 0;
        __syncthreads();
    }
}

// 4. One block per bucket: the bucket's W bins in shared memory, its run of
// (bin, payload) streamed in, the bins written out.
template <typename T, int MODE>
__global__ void __launch_bounds__(kPartTableThreads)
k_part_table(const uint16_t *__restrict__ obin, const typename PartTraits<T, MODE>::V *__restrict__ oval,
             const int32_t *__restrict__ offs, const int64_t nchunks, const int64_t m, const uint32_t W,
             const PartOut<T> out, unsigned *__restrict__ err) {
    using Tr = PartTraits<T, MODE>;
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t j0 = (int64_t)blockIdx.x * W;
    const int w = (int)((m - j0) < (int64_t)W ? (m - j0) : (int64_t)W);
    for (int t = threadIdx.x; t < w; t += kPartTableThreads) Tr::init(smem_raw, (int)W, t);
    __syncthreads();
    const int64_t start = offs[(int64_t)blockIdx.x * nchunks];
    const int64_t end = offs[(int64_t)(blockIdx.x + 1) * nchunks];
    constexpr int U = 8;
    for (int64_t g0 = start; g0 < end; g0 += (int64_t)U * kPartTableThreads) {
        int32_t u[U];
        V v[U];
        bool use[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t g = g0 + (int64_t)j * kPartTableThreads + threadIdx.x;
            use[j] = g < end;
            u[j] = use[j] ? (int32_t)__ldcs(obin + g) : 0;
            v[j] = use[j] ? __ldcs(oval + g) : V(0);
        }
        Tr::template update<U>(smem_raw, (int)W, u, v, use, err);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < w; t += kPartTableThreads) Tr::flush(smem_raw, (int)W, t, j0 + t, out);
}

// -------------------------------------------------------------------- host --
struct PartPlan {
    uint32_t W;
    float inv;
    int B;
    int64_t nchunks;
    bool ok;
};

// W bins per bucket: the largest that fits the table budget, lowered so that
// the bucket count is a whole number of waves of one block per SM.
static PartPlan part_plan(size_t entry, int64_t n, int64_t m) {
    PartPlan P{};
    P.inv = 0.0f;
    int64_t wmax = (int64_t)(kPartTableBudget / entry);
    if (wmax > 65536) wmax = 65536;
    const int64_t sms = num_sms();
    if (m <= 0 || sms <= 0) return P;
    const int64_t k = (m + wmax * sms - 1) / (wmax * sms);
    const int64_t W = (m + k * sms - 1) / (k * sms);
    const int64_t B = (m + W - 1) / W;
    P.W = (uint32_t)W;
    P.inv = (float)(1.0 / (double)W);
    P.B = (int)B;
    P.nchunks = n > 0 ? (n + kPartChunk - 1) / kPartChunk : 1;
    P.ok = B <= kPartMaxBuckets && W <= 65536;
    return P;
}

static size_t entry_of(int mode, size_t s) {
    switch (mode) {
    case kPAdd: return s;
    case kPMul: return s + 4;
    case kPMin:
    case kPMax: return 8;
    case kPPrimMul: return s;
    case kPPrimMin:
    case kPPrimMax: return s;
    default: return 0;
    }
}
static size_t payload_of(int mode, size_t s) { return (mode == kPMin || mode == kPMax) ? 8 : s; }

bool part_applicable(int mode, size_t s, int64_t m) {
    if ((mode == kPMin || mode == kPMax) && s != 4) return false;  // fp64 lifted min/max: two global phases
    return part_plan(entry_of(mode, s), 0, m).ok;
}

struct PartLayout {
    size_t counts, offs, scanreg, obin, oval, bytes;
};
static PartLayout part_layout(const PartPlan &P, size_t payload, int64_t n) {
    PartLayout L;
    const int64_t cells = (int64_t)(P.B + 1) * P.nchunks;
    size_t o = 0;
    L.counts = o;
    o = align_up(o + (size_t)cells * 4, 256);
    L.offs = o;
    o = align_up(o + (size_t)cells * 4, 256);
    L.scanreg = o;
    o = align_up(o + excl_scan_i32_region(cells), 256);
    L.obin = o;
    o = align_up(o + (size_t)n * 2, 256);
    L.oval = o;
    o = align_up(o + (size_t)n * payload, 256);
    L.bytes = o;
    return L;
}

size_t part_ws_bytes(int mode, size_t s, int64_t n, int64_t m) {
    if (!part_applicable(mode, s, m)) return 0;
    const PartPlan P = part_plan(entry_of(mode, s), n, m);
    return part_layout(P, payload_of(mode, s), n).bytes;
}

template <typename K> static bool smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

template <typename T, int MODE>
static adc_status part_run(int64_t n, int64_t m, const int32_t *keys, const T *vals, const PartOut<T> &out, void *ws,
                           size_t ws_off, cudaStream_t s) {
    using Tr = PartTraits<T, MODE>;
    using V = typename Tr::V;
    const PartPlan P = part_plan(Tr::kEntry, n, m);
    if (!P.ok) return ADC_ERR_UNSUPPORTED;
    const PartLayout L = part_layout(P, sizeof(V), n);
    char *w = static_cast<char *>(ws) + ws_off;
    int32_t *counts = reinterpret_cast<int32_t *>(w + L.counts);
    int32_t *offs = reinterpret_cast<int32_t *>(w + L.offs);
    uint16_t *obin = reinterpret_cast<uint16_t *>(w + L.obin);
    V *oval = reinterpret_cast<V *>(w + L.oval);
    unsigned *err = reinterpret_cast<unsigned *>(ws);
    const int64_t nc = P.nchunks;

    const BucketDiv bdiv{P.W, P.inv};
    k_part_count<<<(unsigned)nc, kPartThreads, (size_t)P.B * 4, s>>>(keys, n, m, bdiv, P.B, nc, counts);
    adc_status st = check_launch();
    if (st != ADC_OK) return st;
    st = excl_scan_i32(counts, offs, (int64_t)(P.B + 1) * nc, ws, kPartSlot, w + L.scanreg, s);
    if (st != ADC_OK) return st;
    if constexpr (sizeof(T) == 4) {
        // staged pipeline: 2 x (keys + values) + the permutation + the bucket arrays
        const size_t sm_tma = (size_t)kPartChunk * (4 * 4 + 4) + (size_t)P.B * 8;
        if (!smem_attr(k_part_scatter_tma<MODE>, sm_tma)) return ADC_ERR_CUDA;
        const int64_t grid = nc < num_sms() ? nc : num_sms();
        k_part_scatter_tma<MODE><<<(unsigned)grid, kScatThreads, sm_tma, s>>>(keys, vals, n, m, bdiv, P.B, nc, offs,
                                                                             obin, oval, err, spin_limit());
    } else {
        const size_t sm_scatter = (size_t)kPartChunk * (sizeof(V) + 4) + (size_t)P.B * 8;
        if (!smem_attr(k_part_scatter<T, MODE>, sm_scatter)) return ADC_ERR_CUDA;
        k_part_scatter<T, MODE><<<(unsigned)nc, kPartThreads, sm_scatter, s>>>(keys, vals, n, m, bdiv, P.B, nc, offs,
                                                                              obin, oval);
    }
    if ((st = check_launch()) != ADC_OK) return st;
    const size_t sm_table = (size_t)P.W * Tr::kEntry;
    if (!smem_attr(k_part_table<T, MODE>, sm_table)) return ADC_ERR_CUDA;
    k_part_table<T, MODE><<<(unsigned)P.B, kPartTableThreads, sm_table, s>>>(obin, oval, offs, nc, m, P.W, out, err);
    return check_launch();
}

template <typename T>
static adc_status part_fwd_t(int mode, int64_t n, int64_t m, const int32_t *keys, const T *vals, const T *h0, T *hist,
                             int32_t *n0, T *p, int32_t *is, void *ws, size_t ws_off, cudaStream_t s) {
    const PartOut<T> out{hist, h0, n0, p, is, vals, n};
    switch (mode) {
    case kPAdd: return part_run<T, kPAdd>(n, m, keys, vals, out, ws, ws_off, s);
    case kPMul: return part_run<T, kPMul>(n, m, keys, vals, out, ws, ws_off, s);
    case kPPrimMul: return part_run<T, kPPrimMul>(n, m, keys, vals, out, ws, ws_off, s);
    case kPPrimMin: return part_run<T, kPPrimMin>(n, m, keys, vals, out, ws, ws_off, s);
    case kPPrimMax: return part_run<T, kPPrimMax>(n, m, keys, vals, out, ws, ws_off, s);
    case kPMin:
    case kPMax:
        if constexpr (sizeof(T) == 4) {
            return mode == kPMin ? part_run<float, kPMin>(n, m, keys, vals, out, ws, ws_off, s)
                                 : part_run<float, kPMax>(n, m, keys, vals, out, ws, ws_off, s);
        }
        return ADC_ERR_UNSUPPORTED;
    default: return ADC_ERR_UNSUPPORTED;
    }
}

adc_status part_fwd(int mode, adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals,
                    const void *hist0, void *hist, int32_t *n0, void *p, int32_t *is, void *ws, size_t ws_off,
                    cudaStream_t s) {
    if (n <= 0) return ADC_ERR_INVALID_ARG;
    if (dt == ADC_F64)
        return part_fwd_t<double>(mode, n, m, keys, static_cast<const double *>(vals),
                                  static_cast<const double *>(hist0), static_cast<double *>(hist), n0,
                                  static_cast<double *>(p), is, ws, ws_off, s);
    return part_fwd_t<float>(mode, n, m, keys, static_cast<const float *>(vals), static_cast<const float *>(hist0),
                             static_cast<float *>(hist), n0, static_cast<float *>(p), is, ws, ws_off, s);
}

}  // namespace adc
