// reduce_by_index with sumOfProd, the associative, commutative and invertible
// operator of Sec. 3.3 on (p, s) pairs:
//   (p1, s1) . (p2, s2) = (p1 + p2 + s1*s2, s1 + s2),
// and its vjp by the invertible-operator rule (Sec. 3.3, applied per bin as in
// Sec. 4): for element i of bin k with result y = hist[k],
//   b_i = y (.)^-1 v_i,   vbar_i = d(b_i . v)/dv at v_i ^T histbar[k]
//                               = (hb.p, hb.p * (y.s - v_i.s) + hb.s),
// so the vjp needs the forward's output and nothing else.
//
// Forward without a pair-wide atomic: a bin's update (P, S) <- (P + p + S*s,
// S + s) is split into  s_old = atomicAdd(S, s);  atomicAdd(P, p + s_old*s).
// The first atomic puts the bin's updates in a total order and hands each one
// the S it follows, so P ends as the fold of the bin's pairs in that order --
// a valid order, the operator being commutative.  Tables: per-warp copies or
// one block copy in shared memory (flushed by the same pair of atomics), or
// the global histogram directly.
#include "common.cuh"
#include "hist_common.cuh"
#include "internal.h"
#include "tile_io.cuh"

namespace adc {

// (P, S) . (p, s) into a bin held as two scalars.
template <typename T> __device__ __forceinline__ void sop_update(T *P, T *S, T p, T s) {
    const T s_old = atomicAdd(S, s);
    atomicAdd(P, p + s_old * s);
}

template <typename T>
__global__ void k_sop_init(Pair<T> *__restrict__ h, const Pair<T> *__restrict__ h0, const int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        h[j] = h0 ? h0[j] : Pair<T>{T(0), T(0)};
}

// Elements as pairs, grid-stride over 16-byte words.
template <typename T, class F>
__device__ __forceinline__ void for_each_pair(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals,
                                              const int64_t n, F &&f) {
    constexpr int V = sizeof(Pair<T>) >= 16 ? 1 : 16 / (int)sizeof(Pair<T>);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c * V < n; c += stride) {
        Pair<T> v[V];
        int32_t k[V];
        load_chunk(vals, c * V, n, v, Pair<T>{T(0), T(0)});
        load_chunk(keys, c * V, n, k, (int32_t)-1);
#pragma unroll
        for (int j = 0; j < V; ++j)
            if (c * V + j < n) f(k[j], v[j]);
    }
}

// R private copies in shared memory (R = 8: one per warp; R = 1: one per block).
template <typename T>
__global__ void __launch_bounds__(1024)
k_sop_smem(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals, const int64_t n, const int64_t m,
           const int R, Pair<T> *__restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);  // [R][m] P, then [R][m] S
    T *ss = sp + (int64_t)R * m;
    for (int64_t j = threadIdx.x; j < m * R; j += blockDim.x) {
        sp[j] = T(0);
        ss[j] = T(0);
    }
    __syncthreads();
    const int64_t off = (int64_t)((threadIdx.x >> 5) % R) * m;
    for_each_pair(keys, vals, n, [&](int32_t k, const Pair<T> &v) {
        if (in_range(k, m)) sop_update(sp + off + k, ss + off + k, v.b, v.c);
    });
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        // fold the R copies in order, then into the global bin
        T P = T(0), S = T(0);
        for (int r = 0; r < R; ++r) {
            const T p2 = sp[(int64_t)r * m + j], s2 = ss[(int64_t)r * m + j];
            P = P + p2 + S * s2;
            S = S + s2;
        }
        if (P != T(0) || S != T(0)) sop_update(&hist[j].b, &hist[j].c, P, S);
    }
}

template <typename T>
__global__ void k_sop_global(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals, const int64_t n,
                             const int64_t m, Pair<T> *__restrict__ hist) {
    for_each_pair(keys, vals, n, [&](int32_t k, const Pair<T> &v) {
        if (in_range(k, m)) sop_update(&hist[k].b, &hist[k].c, v.b, v.c);
    });
}

template <typename T>
__global__ void k_sop_vjp(const int32_t *__restrict__ keys, const Pair<T> *__restrict__ vals,
                          const Pair<T> *__restrict__ hist, const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ vb,
                          const int64_t n, const int64_t m, const int accumulate) {
    constexpr int V = sizeof(Pair<T>) >= 16 ? 1 : 16 / (int)sizeof(Pair<T>);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c * V < n; c += stride) {
        Pair<T> v[V], o[V];
        int32_t k[V];
        load_chunk(vals, c * V, n, v, Pair<T>{T(0), T(0)});
        load_chunk(keys, c * V, n, k, (int32_t)-1);
        if (accumulate) load_chunk(vb, c * V, n, o, Pair<T>{T(0), T(0)});
#pragma unroll
        for (int j = 0; j < V; ++j) {
            Pair<T> g{T(0), T(0)};
            if (in_range(k[j], m)) {
                const Pair<T> y = hist[k[j]], b = hb[k[j]];
                g = Pair<T>{b.b, b.b * (y.c - v[j].c) + b.c};
            }
            o[j] = accumulate ? Pair<T>{o[j].b + g.b, o[j].c + g.c} : g;
        }
        store_chunk(vb, c * V, n, o);
    }
}

// hist0 is the first operand of every bin: the same rule with v = hist0.
template <typename T>
__global__ void k_sop_h0bar(const Pair<T> *__restrict__ h0, const Pair<T> *__restrict__ hist,
                            const Pair<T> *__restrict__ hb, Pair<T> *__restrict__ h0b, const int64_t m,
                            const int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const T s0 = h0 ? h0[j].c : T(0);
        const Pair<T> b = hb[j];
        const Pair<T> g{b.b, b.b * (hist[j].c - s0) + b.c};
        h0b[j] = accumulate ? Pair<T>{h0b[j].b + g.b, h0b[j].c + g.c} : g;
    }
}

static unsigned sop_grid(int64_t work, int per_sm) {
    int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename T>
static adc_status sop_fwd_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const Pair<T> *h0,
                            Pair<T> *hist, cudaStream_t s) {
    k_sop_init<T><<<sop_grid(m, 4), 256, 0, s>>>(hist, h0, m);
    if (n > 0) {
        const size_t bytes = (size_t)m * 2 * sizeof(T);  // P and S per copy
        int R = 0;
        if (bytes * 8 <= 48 * 1024) R = 8;
        else if (bytes <= 200 * 1024) R = 1;
        if (R) {
            const size_t smem = bytes * R;
            if (cudaFuncSetAttribute(k_sop_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return ADC_ERR_CUDA;
            const unsigned threads = R == 8 ? 256u : 1024u;
            const unsigned grid = (unsigned)num_sms() * (R == 8 ? 4 : 1);
            k_sop_smem<T><<<grid, threads, smem, s>>>(keys, vals, n, m, R, hist);
        } else {
            k_sop_global<T><<<sop_grid(n, 8), 256, 0, s>>>(keys, vals, n, m, hist);
        }
    }
    return check_launch();
}

template <typename T>
static adc_status sop_vjp_t(int64_t n, int64_t m, const int32_t *keys, const Pair<T> *vals, const Pair<T> *h0,
                            const Pair<T> *hist, const Pair<T> *hb, Pair<T> *vb, Pair<T> *h0b, int acc,
                            cudaStream_t s) {
    constexpr int V = sizeof(Pair<T>) >= 16 ? 1 : 16 / (int)sizeof(Pair<T>);
    if (n > 0) k_sop_vjp<T><<<sop_grid((n + V - 1) / V, 8), 256, 0, s>>>(keys, vals, hist, hb, vb, n, m, acc);
    if (h0b) k_sop_h0bar<T><<<sop_grid(m, 4), 256, 0, s>>>(h0, hist, hb, h0b, m, acc);
    return check_launch();
}

adc_status sop_hist_fwd(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                        void *hist, cudaStream_t s) {
    if (dt == ADC_F64)
        return sop_fwd_t<double>(n, m, keys, static_cast<const Pair<double> *>(vals),
                                 static_cast<const Pair<double> *>(hist0), static_cast<Pair<double> *>(hist), s);
    return sop_fwd_t<float>(n, m, keys, static_cast<const Pair<float> *>(vals), static_cast<const Pair<float> *>(hist0),
                            static_cast<Pair<float> *>(hist), s);
}

adc_status sop_hist_vjp(adc_dtype dt, int64_t n, int64_t m, const int32_t *keys, const void *vals, const void *hist0,
                        const void *hist, const void *histbar, void *valsbar, void *hist0bar, int accumulate,
                        cudaStream_t s) {
    if (dt == ADC_F64)
        return sop_vjp_t<double>(n, m, keys, static_cast<const Pair<double> *>(vals),
                                 static_cast<const Pair<double> *>(hist0), static_cast<const Pair<double> *>(hist),
                                 static_cast<const Pair<double> *>(histbar), static_cast<Pair<double> *>(valsbar),
                                 static_cast<Pair<double> *>(hist0bar), accumulate, s);
    return sop_vjp_t<float>(n, m, keys, static_cast<const Pair<float> *>(vals), static_cast<const Pair<float> *>(hist0),
                            static_cast<const Pair<float> *>(hist), static_cast<const Pair<float> *>(histbar),
                            static_cast<Pair<float> *>(valsbar), static_cast<Pair<float> *>(hist0bar), accumulate, s);
}

}  // namespace adc
