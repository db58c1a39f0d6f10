// Top-K truncation (Sec. I.A: an intermediate result keeps at most its K
// largest Pauli terms) on the device.
//
// The rule: rank the live strings by |c| descending, equal magnitudes by the
// string in export order (x words from the most significant, then z words)
// ascending, and keep the first K.  It is applied after every layer.
//
// Selection is a most-significant-digit radix select with 8-bit digits, never
// a sort: one histogram pass per digit over the strings whose higher digits
// match the prefix chosen so far, then one CTA picks the digit at which the
// running count from the top reaches the number still to keep.  The magnitude
// of a non-negative IEEE double (float) orders like its bit pattern as an
// unsigned integer, so the digits are the magnitude's bits.  If the K-th
// magnitude is shared by more strings than are still to keep, a second select
// over the key words (smallest first) picks which of them stay.  Dropped
// strings get coefficient 0, which every later kernel reads as "not live".
// All decisions stay on the device; the host only launches.
#pragma once

#include "pp_kernels.cuh"

namespace pp {

// Strings of a bucketed layout (regions [b*C, b*C + min(fill[b], C)) plus n_over
// grouped overflow strings) or, when fill is null, the compact array [0, n_over).
template <typename T>
struct Span {
    const uint64_t* x;
    const uint64_t* z;
    T* c;
    uint64_t cap;
    const uint32_t* fill;
    uint32_t B;
    uint64_t C;
    const uint64_t* ox;
    const uint64_t* oz;
    T* oc;
    uint64_t ocap;
    uint64_t n_over;
};

struct TopKState {
    unsigned long long k_left;     // strings still to keep at and below the prefix
    unsigned long long prefix;     // chosen magnitude digits (bits above `shift`)
    unsigned long long kprefix[2 * MAXW];   // chosen key digits, key word order x[W-1]..x[0], z[W-1]..z[0]
    int ties;                      // 1: the tie select runs (more strings at the K-th magnitude than to keep)
    int pad_;
    unsigned int hist[256];
};

template <typename T> struct MagBits;
template <> struct MagBits<double> {
    static constexpr int BITS = 64;
    __device__ static __forceinline__ unsigned long long of(double c) {
        return (unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffULL;
    }
};
template <> struct MagBits<float> {
    static constexpr int BITS = 32;
    __device__ static __forceinline__ unsigned long long of(float c) {
        return (unsigned long long)(__float_as_uint(c) & 0x7fffffffu);
    }
};

// Calls f(x words, z words, coefficient reference) for every string of a span.
template <int W, typename T, typename F>
__device__ __forceinline__ void for_each_string(const Span<T>& s, F&& f) {
    if (s.fill) {
        const int lane = threadIdx.x & 31;
        const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
        for (uint64_t b = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < s.B; b += warps) {
            const uint64_t nb = s.fill[b] < s.C ? s.fill[b] : s.C;
            for (uint64_t i = lane; i < nb; i += 32) f(s.x, s.z, s.cap, b * s.C + i, s.c);
        }
    }
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < s.n_over;
         k += (uint64_t)gridDim.x * blockDim.x)
        f(s.ox, s.oz, s.ocap, k, s.oc);
}

// Key word kw in significance order (0: most significant): x[W-1] .. x[0], z[W-1] .. z[0].
template <int W>
__device__ __forceinline__ uint64_t key_word(const uint64_t* x, const uint64_t* z, uint64_t cap, uint64_t i, int kw) {
    return kw < W ? x[(size_t)(W - 1 - kw) * cap + i] : z[(size_t)(2 * W - 1 - kw) * cap + i];
}

// Histogram of magnitude digit `shift` over live strings whose higher digits equal the prefix.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_topk_hist(Span<T> s, TopKState* st, int shift) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long hi_mask = shift + 8 >= 64 ? 0ull : ~0ull << (shift + 8);
    const unsigned long long pre = st->prefix & hi_mask;
    for_each_string<W, T>(s, [&](const uint64_t*, const uint64_t*, uint64_t, uint64_t i, T* c) {
        const T v = c[i];
        if (v == T(0)) return;
        const unsigned long long m = MagBits<T>::of(v);
        if ((m & hi_mask) != pre) return;
        atomicAdd(&h[(m >> shift) & 255u], 1u);
    });
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

// Picks the digit at which the count from the largest digit reaches k_left.
// One CTA of 256 threads.  last: this was the lowest digit; decide whether the
// tie select is needed.
__global__ void k_topk_pick(TopKState* st, int shift, int last) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = st->hist[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long above = 0;
        int d = 255;
        for (; d > 0; --d) {
            if (above + h[d] >= st->k_left) break;
            above += h[d];
        }
        st->k_left -= above;
        st->prefix |= (unsigned long long)d << shift;
        if (last) st->ties = (unsigned long long)h[d] > st->k_left ? 1 : 0;
    }
    __syncthreads();
    st->hist[threadIdx.x] = 0;
}

// Tie select: histogram of key digit (kw, shift) over strings at the K-th
// magnitude whose higher key digits equal the key prefix.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_topk_key_hist(Span<T> s, TopKState* st, int kw, int shift) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    if (st->ties) {
        const unsigned long long mk = st->prefix;
        const unsigned long long hi_mask = shift + 8 >= 64 ? 0ull : ~0ull << (shift + 8);
        for_each_string<W, T>(s, [&](const uint64_t* x, const uint64_t* z, uint64_t cap, uint64_t i, T* c) {
            const T v = c[i];
            if (v == T(0) || MagBits<T>::of(v) != mk) return;
            for (int j = 0; j < kw; ++j)
                if (key_word<W>(x, z, cap, i, j) != st->kprefix[j]) return;
            const uint64_t k = key_word<W>(x, z, cap, i, kw);
            if ((k & hi_mask) != (st->kprefix[kw] & hi_mask)) return;
            atomicAdd(&h[(k >> shift) & 255u], 1u);
        });
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

// Picks the key digit at which the count from the smallest digit reaches k_left.
__global__ void k_topk_key_pick(TopKState* st, int kw, int shift) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = st->hist[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0 && st->ties) {
        unsigned long long below = 0;
        int d = 0;
        for (; d < 255; ++d) {
            if (below + h[d] >= st->k_left) break;
            below += h[d];
        }
        st->k_left -= below;
        st->kprefix[kw] |= (unsigned long long)d << shift;
    }
    __syncthreads();
    st->hist[threadIdx.x] = 0;
}

// Drops every string ranked after the K-th.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_topk_mark(Span<T> s, const TopKState* st) {
    const unsigned long long mk = st->prefix;
    const int ties = st->ties;
    for_each_string<W, T>(s, [&](const uint64_t* x, const uint64_t* z, uint64_t cap, uint64_t i, T* c) {
        const T v = c[i];
        if (v == T(0)) return;
        const unsigned long long m = MagBits<T>::of(v);
        bool keep = m > mk;
        if (m == mk) {
            keep = true;
            if (ties) {
                // keep iff key <= the selected key (lexicographic over the words)
                for (int j = 0; j < 2 * W; ++j) {
                    const uint64_t k = key_word<W>(x, z, cap, i, j);
                    if (k != st->kprefix[j]) {
                        keep = k < st->kprefix[j];
                        break;
                    }
                }
            }
        }
        if (!keep) c[i] = T(0);
    });
}

__global__ void k_topk_init(TopKState* st, unsigned long long k) {
    st->k_left = k;
    st->prefix = 0;
    for (int j = 0; j < 2 * MAXW; ++j) st->kprefix[j] = 0;
    st->ties = 0;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->hist[i] = 0;
}

// Compacts the live strings of [0, n) of (x, z, c) into (dx, dz, dc); the
// count lands in *out_n.  Order is not kept (the export sorts).
template <int W, typename T>
__global__ void __launch_bounds__(256) k_compact(const uint64_t* x, const uint64_t* z, const T* c, uint64_t cap,
                                                 uint64_t n, uint64_t* dx, uint64_t* dz, T* dc, uint64_t dcap,
                                                 unsigned long long* out_n) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n;
         i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + lane;
        const bool lv = i < n && c[i] != T(0);
        const unsigned m = __ballot_sync(FULL, lv);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(out_n, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (lv) {
            const uint64_t q = base + __popc(m & ((1u << lane) - 1u));
            if (q < dcap) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    dx[(size_t)w * dcap + q] = x[(size_t)w * cap + i];
                    dz[(size_t)w * dcap + q] = z[(size_t)w * cap + i];
                }
                dc[q] = c[i];
            }
        }
    }
}

}  // namespace pp
