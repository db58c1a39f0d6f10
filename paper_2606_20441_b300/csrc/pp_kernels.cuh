// Kernels of libpp: bucket scatter, the fused sub-layer processor (shared-memory
// tiles, with a global-memory variant for oversized buckets), and the exact
// expectation reduction.
#pragma once

#include "pp_device.cuh"

namespace pp {

// Per-launch parameters of one sub-layer.  Term arrays are word-major:
// x[w * cap + i].  Bucket b of a layout owns indices [b*C, b*C + fill[b]).
struct StepParams {
    // source layout (this sub-layer's buckets)
    const uint64_t* sx;
    const uint64_t* sz;
    const void* sc;
    uint64_t scap;
    const uint32_t* sfill;        // strings routed to each bucket (may exceed sC)
    uint32_t sB;
    uint64_t sC;
    // source overflow: strings beyond a bucket's region, grouped by bucket
    const uint64_t* spx;
    const uint64_t* spz;
    const void* spc;
    uint64_t spcap;
    const uint64_t* soff;         // first overflow index of each bucket

    // destination layout (next sub-layer's buckets, or the compact result)
    uint64_t* dx;
    uint64_t* dz;
    void* dc;
    uint64_t dcap;
    uint32_t* dfill;
    uint32_t dB;
    uint64_t dC;
    // destination overflow, in arrival order: string, bucket, index past the region
    uint64_t* rpx;
    uint64_t* rpz;
    void* rpc;
    uint32_t* rpb;
    uint32_t* rps;
    uint64_t rpcap;

    const SubLayerDesc* desc;
    const SubLayerDesc* next;     // nullptr when desc is final
    NoiseDesc noise;
    int has_noise;
    double eps;
    float eps_f;                  // smallest float >= eps
    int w_max;

    unsigned long long* counters; // see CTR_* below
    long long* delta;             // [MAX_SITES] net change of live terms by listed gate
    const uint32_t* in_list;      // buckets to process (nullptr: all of 0..sB-1)
    uint32_t n_list;
    uint32_t* out_list;           // buckets this tier could not hold (nullptr: report failure)
    int work_ctr;                 // counter index of this launch's work queue
    int defer_ctr;                // counter index of out_list's length
    uint32_t max_load;            // buckets with more strings are passed on
};

enum {
    CTR_WORK = 0,        // work queues, one per tier
    CTR_WORK2 = 1,
    CTR_WORK3 = 2,
    CTR_OUT = 3,         // terms written (next layout or final)
    CTR_PROLOGUE = 4,    // live terms after the prologue (merge / noise)
    CTR_DEFER1 = 5,      // buckets passed from the main tier to the large tier
    CTR_DEFER2 = 6,      // buckets passed from the large tier to the global tier
    CTR_ERR_REGION = 7,  // strings dropped: overflow area or result full
    CTR_ERR_FALLBACK = 8,// buckets too large even for the global tier
    CTR_SPILL = 9,       // strings written to the destination overflow area
    CTR_LOADED = 12,     // strings loaded by completed buckets, per tier (12..14)
    CTR_EMITTED = 15,    // strings written by completed buckets, per tier (15..17)
    CTR_COUNT = 20
};

// Working set of one bucket.  Arrays live in shared memory (main kernel) or in a
// per-CTA global scratch slice (fallback kernel); both paths run the same code.
template <int W, typename T>
struct Tile {
    uint64_t* x;      // [W][cap]
    uint64_t* z;      // [W][cap]
    T* c;             // current coefficient, 0 = not live
    T* cn;            // coefficient after the current round
    int32_t* pj;      // partner index this round; -1 none; -2 inactive
    int16_t* ps;      // slot of this round's gate
    int8_t* ph;       // +1/-1: sign of the sin-branch contribution to the partner
    int8_t* rv;       // revived by a partner this round
    int32_t* hash;    // [hcap] entry index or -1
    int cap;
    int hcap;
    int* n;           // number of entries
    int* flag;        // capacity exceeded
    int* kmax;
    int* live;
};

template <int W, typename T>
__device__ __forceinline__ void tile_key(const Tile<W, T>& t, int i, uint64_t* x, uint64_t* z) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        x[w] = t.x[(size_t)w * t.cap + i];
        z[w] = t.z[(size_t)w * t.cap + i];
    }
}

template <int W, typename T>
__device__ __forceinline__ bool tile_key_eq(const Tile<W, T>& t, int i, const uint64_t* x,
                                            const uint64_t* z) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w)
        eq = eq && t.x[(size_t)w * t.cap + i] == x[w] && t.z[(size_t)w * t.cap + i] == z[w];
    return eq;
}

template <int W, typename T>
__device__ __forceinline__ int tile_lookup(const Tile<W, T>& t, const uint64_t* x, const uint64_t* z) {
    uint32_t h = (uint32_t)hash_key<W>(x, z) & (uint32_t)(t.hcap - 1);
    for (int probe = 0; probe < t.hcap; ++probe) {
        int s = t.hash[h];
        if (s < 0) return -1;
        if (tile_key_eq<W, T>(t, s, x, z)) return s;
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    return -1;
}

// Inserts entry idx (key already stored).  merge: if the key is present, add c
// into the existing entry instead and leave idx dead.
template <int W, typename T>
__device__ __forceinline__ void tile_insert(const Tile<W, T>& t, int idx, const uint64_t* x,
                                            const uint64_t* z, bool merge) {
    uint32_t h = (uint32_t)hash_key<W>(x, z) & (uint32_t)(t.hcap - 1);
    for (int probe = 0; probe < t.hcap; ++probe) {
        int prev = atomicCAS(&t.hash[h], -1, idx);
        if (prev < 0) return;
        if (merge && tile_key_eq<W, T>(t, prev, x, z)) {
            atomicAdd(&t.c[prev], t.c[idx]);
            t.c[idx] = T(0);
            return;
        }
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    atomicExch(t.flag, 1);
}

template <int W, typename T>
__device__ __forceinline__ T load_coef(const void* base, size_t i);
template <>
__device__ __forceinline__ double load_coef<1, double>(const void* base, size_t i) {
    return static_cast<const double*>(base)[i];
}
template <>
__device__ __forceinline__ double load_coef<2, double>(const void* base, size_t i) {
    return static_cast<const double*>(base)[i];
}
template <>
__device__ __forceinline__ float load_coef<1, float>(const void* base, size_t i) {
    return static_cast<const float*>(base)[i];
}
template <>
__device__ __forceinline__ float load_coef<2, float>(const void* base, size_t i) {
    return static_cast<const float*>(base)[i];
}

template <typename T>
__device__ __forceinline__ T eps_of(const StepParams& p);
template <>
__device__ __forceinline__ double eps_of<double>(const StepParams& p) { return p.eps; }
template <>
__device__ __forceinline__ float eps_of<float>(const StepParams& p) { return p.eps_f; }

// Appends a string to bucket nb of the destination layout: into the bucket's
// region while it has room, else into the overflow area.
template <int W, typename T>
__device__ __forceinline__ void emit(const StepParams& p, uint32_t nb, const uint64_t* x,
                                     const uint64_t* z, T c) {
    uint32_t slot = atomicAdd(&p.dfill[nb], 1u);
    if ((uint64_t)slot < p.dC) {
        size_t pos = (size_t)nb * p.dC + slot;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            p.dx[(size_t)w * p.dcap + pos] = x[w];
            p.dz[(size_t)w * p.dcap + pos] = z[w];
        }
        static_cast<T*>(p.dc)[pos] = c;
        return;
    }
    unsigned long long k = atomicAdd(&p.counters[CTR_SPILL], 1ull);
    if (k < p.rpcap) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            p.rpx[(size_t)w * p.rpcap + k] = x[w];
            p.rpz[(size_t)w * p.rpcap + k] = z[w];
        }
        static_cast<T*>(p.rpc)[k] = c;
        p.rpb[k] = nb;
        p.rps[k] = slot - (uint32_t)p.dC;
    } else {
        atomicAdd(&p.counters[CTR_ERR_REGION], 1ull);
    }
}

// Processes one bucket: load, prologue (merge/truncate the input observable,
// noise map), gate rounds, then writes the surviving strings into the next
// layout's buckets (or the compact final array).  Returns false, having
// written nothing, when the bucket does not fit the tile.
template <int W, typename T>
__device__ bool process_bucket(const Tile<W, T>& t, const StepParams& p, uint32_t b,
                               int* s_delta) {
    const SubLayerDesc& d = *p.desc;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T eps = eps_of<T>(p);
    const uint32_t n_in = p.sfill[b];

    for (int i = tid; i < t.hcap; i += nt) t.hash[i] = -1;
    for (int i = tid; i < MAX_SITES; i += nt) s_delta[i] = 0;
    if (tid == 0) {
        *t.n = (int)n_in;
        *t.flag = (n_in > p.max_load) ? 1 : 0;
        *t.kmax = 0;
        *t.live = 0;
    }
    __syncthreads();
    if (*t.flag) return false;

    // ---- load: the bucket's region, then its overflow strings
    const size_t base = (size_t)b * p.sC;
    const size_t obase = (n_in > p.sC) ? (size_t)p.soff[b] : 0;
    for (int i = tid; i < (int)n_in; i += nt) {
        uint64_t x[W], z[W];
        const bool reg = (uint64_t)i < p.sC;
        const size_t src = reg ? base + i : obase + (i - p.sC);
        const uint64_t* ax = reg ? p.sx : p.spx;
        const uint64_t* az = reg ? p.sz : p.spz;
        const size_t acap = reg ? p.scap : p.spcap;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            x[w] = ax[(size_t)w * acap + src];
            z[w] = az[(size_t)w * acap + src];
            t.x[(size_t)w * t.cap + i] = x[w];
            t.z[(size_t)w * t.cap + i] = z[w];
        }
        t.c[i] = load_coef<W, T>(reg ? p.sc : p.spc, src);
        t.rv[i] = 0;
        if (d.first) __threadfence_block();
        tile_insert<W, T>(t, i, x, z, d.first != 0);
    }
    __syncthreads();

    // ---- prologue: truncation of the merged input; noise map
    int my_live = 0, my_k = 0;
    for (int i = tid; i < (int)n_in; i += nt) {
        T c = t.c[i];
        uint64_t x[W], z[W];
        tile_key<W, T>(t, i, x, z);
        if (d.first && c != T(0)) {
            if (Coef<T>::small(c, eps) || (p.w_max >= 0 && weight_of<W>(x, z) > p.w_max)) c = T(0);
        }
        if (p.has_noise && c != T(0)) {
            double f = noise_factor(p.noise, noise_exponent<W>(p.noise, x, z));
            c = Coef<T>::mul(c, T(f));
            if (Coef<T>::small(c, eps)) c = T(0);
        }
        t.c[i] = c;
        if (c != T(0)) {
            ++my_live;
            uint64_t A[W], Mx[W], Mz[W];
            activity<W>(d, x, z, A, Mx, Mz);
            int k = count_active<W>(A);
            my_k = k > my_k ? k : my_k;
        }
    }
    if (my_live) atomicAdd(t.live, my_live);
    if (my_k) atomicMax(t.kmax, my_k);
    __syncthreads();
    const int kmax = *t.kmax;
    const int live0 = *t.live;

    // ---- gate rounds: round r applies each string's r-th acting gate
    for (int r = 0; r < kmax; ++r) {
        const int nr = *t.n;
        for (int i = tid; i < nr; i += nt) {
            int state = -2;
            T c = t.c[i];
            if (c != T(0)) {
                uint64_t x[W], z[W], A[W], Mx[W], Mz[W];
                tile_key<W, T>(t, i, x, z);
                activity<W>(d, x, z, A, Mx, Mz);
                if (count_active<W>(A) > r) {
                    int slot = select_slot<W>(d, A, r);
                    uint64_t rx[W], rz[W], qx[W], qz[W];
                    slot_generator<W>(d, slot, rx, rz);
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        qx[w] = x[w] ^ rx[w];
                        qz[w] = z[w] ^ rz[w];
                    }
                    state = tile_lookup<W, T>(t, qx, qz);
                    // i R P = i^{1+e} (R xor P): sign of P's sin-branch into its partner
                    int e = product_phase<W>(rx, rz, x, z);
                    t.ph[i] = ((1 + e) & 3) == 0 ? 1 : -1;
                    t.ps[i] = (int16_t)slot;
                }
            }
            t.pj[i] = state;
        }
        __syncthreads();
        for (int i = tid; i < nr; i += nt) {
            int j = t.pj[i];
            if (j == -2) continue;
            int slot = t.ps[i];
            T cs = T(d.cs[slot]), sn = T(d.sn[slot]);
            T c = t.c[i];
            int phi = t.ph[i];
            T c2 = (j >= 0) ? t.c[j] : T(0);
            if (j >= 0 && c2 != T(0)) {
                // partner P xor R is live: both members rotate; the partner's
                // contribution into P carries the opposite sign (i R Q = -phi P)
                t.cn[i] = Coef<T>::rot(cs, c, sn, c2, -phi);
            } else {
                t.cn[i] = Coef<T>::mul(cs, c);
                T v = Coef<T>::mul(sn, c);
                if (phi < 0) v = -v;
                if (!Coef<T>::small(v, eps)) {
                    uint64_t x[W], z[W], rx[W], rz[W];
                    tile_key<W, T>(t, i, x, z);
                    slot_generator<W>(d, slot, rx, rz);
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        x[w] ^= rx[w];
                        z[w] ^= rz[w];
                    }
                    if (p.w_max < 0 || weight_of<W>(x, z) <= p.w_max) {
                        atomicAdd(&s_delta[d.order[slot]], 1);
                        if (j >= 0) {
                            t.cn[j] = v;          // revive a string truncated earlier
                            t.rv[j] = 1;
                        } else {
                            int idx = atomicAdd(t.n, 1);
                            if (idx >= t.cap) {
                                atomicExch(t.flag, 1);
                            } else {
#pragma unroll
                                for (int w = 0; w < W; ++w) {
                                    t.x[(size_t)w * t.cap + idx] = x[w];
                                    t.z[(size_t)w * t.cap + idx] = z[w];
                                }
                                t.c[idx] = v;
                                t.pj[idx] = -2;
                                t.rv[idx] = 0;
                                tile_insert<W, T>(t, idx, x, z, false);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (*t.flag) return false;
        const int nn = *t.n;
        for (int i = tid; i < nr; i += nt) {
            if (t.pj[i] != -2) {
                T v = t.cn[i];
                if (Coef<T>::small(v, eps)) {
                    v = T(0);
                    atomicAdd(&s_delta[d.order[t.ps[i]]], -1);
                }
                t.c[i] = v;
            } else if (t.rv[i]) {
                t.c[i] = t.cn[i];
                t.rv[i] = 0;
            }
        }
        (void)nn;
        __syncthreads();
    }

    // ---- output
    if (d.final_) {
        __shared__ unsigned long long s_base;
        if (tid == 0) *t.live = 0;
        __syncthreads();
        const int nf = *t.n;
        int cnt = 0;
        for (int i = tid; i < nf; i += nt)
            if (t.c[i] != T(0)) ++cnt;
        int off = cnt ? atomicAdd(t.live, cnt) : 0;
        __syncthreads();
        if (tid == 0) {
            s_base = atomicAdd(&p.counters[CTR_OUT], (unsigned long long)*t.live);
            atomicAdd(&p.counters[CTR_EMITTED + (p.work_ctr - CTR_WORK)], (unsigned long long)*t.live);
        }
        __syncthreads();
        unsigned long long pos = s_base + off;
        for (int i = tid; i < nf; i += nt) {
            T c = t.c[i];
            if (c == T(0)) continue;
            if (pos < p.dcap) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    p.dx[(size_t)w * p.dcap + pos] = t.x[(size_t)w * t.cap + i];
                    p.dz[(size_t)w * p.dcap + pos] = t.z[(size_t)w * t.cap + i];
                }
                static_cast<T*>(p.dc)[pos] = c;
            } else {
                atomicAdd(&p.counters[CTR_ERR_REGION], 1ull);
            }
            ++pos;
        }
    } else {
        const SubLayerDesc& dn = *p.next;
        const uint32_t bmask = p.dB - 1;
        const int nf = *t.n;
        int cnt = 0;
        for (int i = tid; i < nf; i += nt) {
            T c = t.c[i];
            if (c == T(0)) continue;
            ++cnt;
            uint64_t x[W], z[W];
            tile_key<W, T>(t, i, x, z);
            uint32_t nb = bucket_of<W>(dn, x, z, bmask);
            emit<W, T>(p, nb, x, z, c);
        }
        if (cnt) {
            atomicAdd(&p.counters[CTR_OUT], (unsigned long long)cnt);
            atomicAdd(&p.counters[CTR_EMITTED + (p.work_ctr - CTR_WORK)], (unsigned long long)cnt);
        }
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&p.counters[CTR_PROLOGUE], (unsigned long long)live0);
        atomicAdd(&p.counters[CTR_LOADED + (p.work_ctr - CTR_WORK)], (unsigned long long)n_in);
    }
    for (int i = tid; i < MAX_SITES; i += nt)
        if (s_delta[i])
            atomicAdd(reinterpret_cast<unsigned long long*>(&p.delta[i]),
                      (unsigned long long)(long long)s_delta[i]);   // two's complement
    return true;
}

template <int W, typename T>
__host__ __device__ constexpr size_t tile_bytes_per_entry() {
    return 2 * W * sizeof(uint64_t) + 2 * sizeof(T) + sizeof(int32_t) + sizeof(int16_t) + 2 +
           2 * sizeof(int32_t);
}

template <int W, typename T>
__device__ __forceinline__ Tile<W, T> carve_tile(unsigned char* mem, int cap, int* ctl) {
    Tile<W, T> t;
    t.cap = cap;
    t.hcap = 2 * cap;
    unsigned char* q = mem;
    t.x = reinterpret_cast<uint64_t*>(q); q += sizeof(uint64_t) * W * cap;
    t.z = reinterpret_cast<uint64_t*>(q); q += sizeof(uint64_t) * W * cap;
    t.c = reinterpret_cast<T*>(q); q += sizeof(T) * cap;
    t.cn = reinterpret_cast<T*>(q); q += sizeof(T) * cap;
    t.hash = reinterpret_cast<int32_t*>(q); q += sizeof(int32_t) * 2 * cap;
    t.pj = reinterpret_cast<int32_t*>(q); q += sizeof(int32_t) * cap;
    t.ps = reinterpret_cast<int16_t*>(q); q += sizeof(int16_t) * cap;
    t.ph = reinterpret_cast<int8_t*>(q); q += cap;
    t.rv = reinterpret_cast<int8_t*>(q); q += cap;
    t.n = ctl + 0;
    t.flag = ctl + 1;
    t.kmax = ctl + 2;
    t.live = ctl + 3;
    return t;
}

// Shared-memory tiers: persistent CTAs take buckets from a work queue (all
// buckets, or the list a smaller tier passed on); a bucket that does not fit is
// passed to the next tier.
template <int W, typename T>
__global__ void k_process(StepParams p, int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ctl[4];
    __shared__ int s_delta[MAX_SITES];
    __shared__ uint32_t s_b;
    Tile<W, T> t = carve_tile<W, T>(smem, cap, ctl);
    const uint32_t n_items = p.in_list ? p.n_list : p.sB;
    for (;;) {
        if (threadIdx.x == 0) s_b = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        __syncthreads();
        const uint32_t k = s_b;
        if (k >= n_items) break;
        const uint32_t b = p.in_list ? p.in_list[k] : k;
        if (p.sfill[b] != 0) {
            bool ok = process_bucket<W, T>(t, p, b, s_delta);
            if (!ok && threadIdx.x == 0) {
                if (p.out_list) {
                    unsigned long long j = atomicAdd(&p.counters[p.defer_ctr], 1ull);
                    p.out_list[j] = b;
                } else {
                    atomicAdd(&p.counters[CTR_ERR_FALLBACK], 1ull);
                }
            }
        }
        __syncthreads();
    }
}

// Global tier for the largest buckets: the same processor with the tile in a
// per-CTA slice of global scratch memory.
template <int W, typename T>
__global__ void k_process_global(StepParams p, unsigned char* scratch, size_t slice_bytes, int cap) {
    __shared__ int ctl[4];
    __shared__ int s_delta[MAX_SITES];
    __shared__ uint32_t s_k;
    Tile<W, T> t = carve_tile<W, T>(scratch + slice_bytes * blockIdx.x, cap, ctl);
    for (;;) {
        if (threadIdx.x == 0) s_k = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        __syncthreads();
        const uint32_t k = s_k;
        if (k >= p.n_list) break;
        bool ok = process_bucket<W, T>(t, p, p.in_list[k], s_delta);
        if (!ok && threadIdx.x == 0) atomicAdd(&p.counters[CTR_ERR_FALLBACK], 1ull);
        __syncthreads();
    }
}

// Scatters the input observable into the first sub-layer's buckets (the
// destination layout of p).
template <int W, typename T>
__global__ void k_scatter_input(const uint64_t* ox, const uint64_t* oz, const double* oc, size_t n,
                                StepParams p) {
    const SubLayerDesc& d = *p.next;
    const uint32_t bmask = p.dB - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint64_t x[W], z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            x[w] = ox[i * W + w];
            z[w] = oz[i * W + w];
        }
        uint32_t b = bucket_of<W>(d, x, z, bmask);
        emit<W, T>(p, b, x, z, T(oc[i]));
    }
}

// Overflow bookkeeping: each bucket whose count exceeds its region gets a
// contiguous range of the grouped overflow area.
__global__ void k_spill_offsets(const uint32_t* fill, uint32_t nB, uint64_t C, uint64_t* soff,
                                unsigned long long* total) {
    __shared__ unsigned long long s_scan[1024];
    __shared__ unsigned long long s_base;
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long ex = 0;
    if (b < nB && (uint64_t)fill[b] > C) ex = (uint64_t)fill[b] - C;
    s_scan[threadIdx.x] = ex;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        unsigned long long v = (int)threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0ull;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (threadIdx.x == blockDim.x - 1) s_base = atomicAdd(total, s_scan[threadIdx.x]);
    __syncthreads();
    if (b < nB) soff[b] = s_base + s_scan[threadIdx.x] - ex;
}

template <int W, typename T>
__global__ void k_spill_move(const uint64_t* rx, const uint64_t* rz, const T* rc, const uint32_t* rb,
                             const uint32_t* rs, uint64_t rcap, uint64_t n, const uint64_t* soff,
                             uint64_t* ox, uint64_t* oz, T* oc, uint64_t ocap) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t dst = soff[rb[k]] + rs[k];
        if (dst >= ocap) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ox[(size_t)w * ocap + dst] = rx[(size_t)w * rcap + k];
            oz[(size_t)w * ocap + dst] = rz[(size_t)w * rcap + k];
        }
        oc[dst] = rc[k];
    }
}

// ----------------------------------------------------------------------------- expectation

// trunc(v * 2^80) as a 128-bit two's-complement integer (|v| < 2^46).
__device__ __forceinline__ __int128 to_fixed80(double v) {
    uint64_t bits = (uint64_t)__double_as_longlong(v);
    int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0) return 0;
    uint64_t m = (bits & 0xfffffffffffffULL) | (1ULL << 52);
    int sh = ex - 1075 + 80;
    __int128 mag;
    if (sh <= -64) mag = 0;
    else if (sh < 0) mag = (__int128)(m >> (-sh));
    else mag = ((__int128)m) << sh;
    return (bits >> 63) ? -mag : mag;
}

// Sum of c over strings with x == 0, in exact fixed point; one partial per CTA.
template <int W, typename T>
__global__ void k_expect(const uint64_t* x, const T* c, uint64_t cap, uint64_t n,
                         __int128* partial) {
    __shared__ __int128 s[256];
    __int128 acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        bool diag = true;
#pragma unroll
        for (int w = 0; w < W; ++w) diag = diag && x[(size_t)w * cap + i] == 0ull;
        if (diag) acc += to_fixed80((double)c[i]);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

}  // namespace pp
