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
    unsigned long long* spill_ctr;   // [NSPILL] fill of each shard of the overflow area

    const SubLayerDesc* desc;
    const SubLayerDesc* next;     // nullptr when desc is final
    NoiseDesc noise;
    int has_noise;
    double eps;
    float eps_f;                  // smallest float >= eps
    int w_max;

    unsigned long long* counters; // see CTR_* below
    const uint32_t* in_list;      // buckets to process (nullptr: all of 0..sB-1)
    uint32_t n_list;
    const unsigned long long* n_list_dev;   // when set, in_list's length is read here (the
                                            // previous tier's deferral counter) on the device
    uint32_t* out_list;           // buckets this tier could not hold (nullptr: report failure)
    int work_ctr;                 // counter index of this launch's work queue
    int defer_ctr;                // counter index of out_list's length
    uint32_t max_load;            // buckets with more strings are passed on
    int gcap;                     // global tier: strings per tile
    uint64_t gslice;              // global tier: bytes per CTA slice of its scratch
    unsigned long long* phase;    // [4] cycles spent in load, prologue, rounds, output (tier 0),
                                  // accumulated when tracing; nullptr otherwise
};

constexpr int N_TIERS = 5;   // warp tiles (two sizes), CTA tiles (two sizes), global-memory tile

enum {
    CTR_WORK = 0,        // work queues, one per tier (0..N_TIERS-1)
    CTR_OUT = N_TIERS,   // terms written (next layout or final)
    CTR_DEFER = CTR_OUT + 1,                // buckets passed from tier t to tier t+1 (N_TIERS - 1)
    CTR_ERR_REGION = CTR_DEFER + N_TIERS - 1,  // strings dropped: overflow area or result full
    CTR_ERR_FALLBACK,    // buckets too large even for the global tier
    CTR_SPILL,           // strings written to the destination overflow area
    CTR_LOADED,          // strings loaded by completed buckets, per tier (N_TIERS)
    CTR_EMITTED = CTR_LOADED + N_TIERS,     // strings written by completed buckets, per tier
    CTR_FAIL = CTR_EMITTED + N_TIERS,       // buckets passed on, by reason (4): load, entry pool, hash, list
    CTR_SPILL_TOTAL = CTR_FAIL + 4,         // scratch of the overflow grouping
    CTR_PHASE,           // warp-tier cycles per phase when tracing (4)
    CTR_PHASE_CTA = CTR_PHASE + 4,          // CTA-tier cycles per phase when tracing (4)
    CTR_UPDATES = CTR_PHASE_CTA + 4,        // canonical work count of the completed buckets (string lifetimes)
    CTR_STAT,            // tier-0 work statistics when tracing (8): buckets, rounds,
                         // list chunks, listed strings, live pairs, created, revived, 0
    CTR_DEBUG = CTR_STAT + 8,   // debug builds: the first failed bounds check (site number)
    CTR_COUNT
};

// Bounds checks of the debug build (compiled with PP_DEBUG).  PP_OOB(ok, site,
// counters) is true when the check fails: it records the first failing site in
// counters[CTR_DEBUG] and the caller skips the access (no trap, no fault); the
// host turns a recorded site into an error.  In other builds it is false and
// costs nothing.  Sites: 1 load source, 2 tile entry, 3 active list, 4 gate
// index, 5 destination region, 6 overflow area, 7 compact result, 8 bucket
// index, 9 global-tier slice.
#ifdef PP_DEBUG
__device__ __forceinline__ bool pp_oob(bool ok, int site, unsigned long long* counters) {
    if (!ok) atomicCAS(&counters[CTR_DEBUG], 0ull, (unsigned long long)site);
    return !ok;
}
#define PP_OOB(ok, site, counters) pp_oob((ok), (site), (counters))
#else
#define PP_OOB(ok, site, counters) false
#endif

// Number of work items (buckets) of a tier launch.
__device__ __forceinline__ uint32_t work_items(const StepParams& p) {
    if (!p.in_list) return p.sB;
    if (p.n_list_dev) return (uint32_t)*(volatile const unsigned long long*)p.n_list_dev;
    return p.n_list;
}

// A batched launch runs one instance per grid row: CTA row y takes the
// parameters ps[y] (each instance has its own layouts, counters and work
// queues); a plain launch passes ps = nullptr and its own parameters.  The
// CTA copies its parameters to shared memory once.  Returns, for the whole
// CTA, whether the launch's work queue still holds items (its claim counter
// only grows, so a CTA that finds it exhausted can leave before setting up).
__device__ __forceinline__ bool load_params(StepParams& dst, const StepParams& p, const StepParams* ps) {
    __shared__ int s_left;
    if (threadIdx.x == 0) {
        dst = ps ? ps[blockIdx.y] : p;
        s_left = *(volatile const unsigned long long*)&dst.counters[dst.work_ctr] < (unsigned long long)work_items(dst);
    }
    __syncthreads();
    return s_left != 0;
}

constexpr int NSPILL = 64;   // shards of the overflow area (one atomic counter each)

enum { FAIL_LOAD = 1, FAIL_POOL = 2, FAIL_HASH = 3, FAIL_CHUNK = 4 };

__device__ __forceinline__ int16_t atomic_cas_idx(int16_t* a, int16_t cmp, int16_t val) {
    return (int16_t)atomicCAS(reinterpret_cast<unsigned short*>(a), (unsigned short)cmp, (unsigned short)val);
}
__device__ __forceinline__ int32_t atomic_cas_idx(int32_t* a, int32_t cmp, int32_t val) {
    return atomicCAS(a, cmp, val);
}

// Working set of one bucket.  Arrays live in shared memory (the shared-memory
// tiers) or in a per-CTA slice of global scratch memory (the global tier); all
// tiers run the same code.  I is the entry-index type (int16_t in shared
// memory, int32_t in global memory).
template <int W, typename T, typename I>
struct Tile {
    uint64_t* x;      // [W][cap] string
    uint64_t* z;      // [W][cap]
    uint64_t* g;      // [W][cap] gates of the sub-layer still to apply (listed-order bits)
    T* c;             // coefficient buffer 0 (the loaded values), 0 = not live
    T* c1;            // coefficient buffer 1: round r reads buffer r & 1, writes the other
    uint8_t* sr;      // stamp of the last write of each string's coefficient: 0 at
                      // load, r + 1 in round r (the value sits in buffer stamp & 1)
    I* hash;          // [hcap] entry index or -1 (insert-only)
    I* act;           // [2][cap] strings with gates left: this round's list, the next one's
    int cap;
    int hcap;
    int hbits;
    int* n;           // entries used
    int* flag;        // nonzero (a FAIL_* reason): the bucket goes to the next tier
    int* live;
    int* nact;        // [3] lengths of the active lists (rotating counter slots)
    unsigned long long* ctr;   // the launch's counters (debug bounds checks)
    __device__ __forceinline__ T* cbuf(int k) const { return k ? c1 : c; }
};

// Current coefficient of entry i (after the rounds: its final one).
template <int W, typename T, typename I>
__device__ __forceinline__ T tile_coef(const Tile<W, T, I>& t, int i) {
    return t.cbuf(t.sr[i] & 1)[i];
}

constexpr int NWARPS = 16;    // warps per CTA of the global-memory tier (512 threads)

// Gates of the current sub-layer in listed order, staged in shared memory.
template <int W, typename T>
struct GateTab {
    uint64_t rx[64 * W][W];
    uint64_t rz[64 * W][W];
    T cs[64 * W];
    T sn[64 * W];
    uint8_t slot[64 * W];     // class sub-layers: first site of each gate
    int cls;
    int shift;
    uint32_t psign;           // SubLayerDesc::psign
};

// Slot of a tile's hash table for key (x, z): 32-bit multiply-add of the key's
// halves, then a multiply-xorshift finaliser.
template <int W>
__device__ __forceinline__ uint32_t tile_hash(const uint64_t* x, const uint64_t* z, int hbits) {
    uint32_t h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h += (uint32_t)x[w] * (0x9E3779B1u + 4u * w) + (uint32_t)(x[w] >> 32) * (0x85EBCA77u + 4u * w);
        h += (uint32_t)z[w] * (0xC2B2AE3Du + 4u * w) + (uint32_t)(z[w] >> 32) * (0x27D4EB2Fu + 4u * w);
    }
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 13;
    return h >> (32 - hbits);
}

// Letter code (x + 2z) of string (x, z) on qubit a.
template <int W>
__device__ __forceinline__ int letter_at(const uint64_t* x, const uint64_t* z, int a) {
    uint64_t xw = x[0], zw = z[0];
    if (W > 1 && a >= 64) {
        xw = x[W - 1];
        zw = z[W - 1];
    }
    const int b = a & 63;
    return (int)((xw >> b) & 1ull) | ((int)((zw >> b) & 1ull) << 1);
}

// Whether string (x, z), acted on by listed gate gg, sends its sin-branch into
// its partner with a negative sign: i R P = phi P' with phi = -1.  Class
// sub-layers read it from the letters on the gate's sites; generic ones take
// the product phase R P = i^e (R xor P).
template <int W, typename T>
__device__ __forceinline__ bool branch_negative(const GateTab<W, T>& tab, int gg, const uint64_t* x,
                                                const uint64_t* z) {
    if (tab.cls == CLS_GENERIC) {
        const int e = product_phase<W>(tab.rx[gg], tab.rz[gg], x, z);
        return ((1 + e) & 3) != 0;
    }
    const int a = tab.slot[gg];
    int code = letter_at<W>(x, z, a);
    if (tab.cls == CLS_LOCAL2) code |= letter_at<W>(x, z, a + tab.shift) << 2;
    return (tab.psign >> code) & 1u;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_coef(float* smem, const float* gmem) { cp_async4(smem, gmem); }
__device__ __forceinline__ void cp_async_coef(double* smem, const double* gmem) { cp_async8(smem, gmem); }

template <int W, typename T, typename I>
__device__ __forceinline__ void tile_key(const Tile<W, T, I>& t, int i, uint64_t* x, uint64_t* z) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        x[w] = t.x[(size_t)w * t.cap + i];
        z[w] = t.z[(size_t)w * t.cap + i];
    }
}

template <int W, typename T, typename I>
__device__ __forceinline__ bool tile_key_eq(const Tile<W, T, I>& t, int i, const uint64_t* x,
                                            const uint64_t* z) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w)
        eq = eq && t.x[(size_t)w * t.cap + i] == x[w] && t.z[(size_t)w * t.cap + i] == z[w];
    return eq;
}

// Entries are never removed from the table (a truncated string keeps its slot
// and may be revived), so a lookup of a key inserted earlier never meets an
// empty slot before it, whatever other warps insert meanwhile.
template <int W, typename T, typename I>
__device__ __forceinline__ int tile_lookup(const Tile<W, T, I>& t, const uint64_t* x, const uint64_t* z) {
    uint32_t h = tile_hash<W>(x, z, t.hbits);
    for (int probe = 0; probe < t.hcap; ++probe) {
        int s = (int)t.hash[h];
        if (s < 0) return -1;
        if (tile_key_eq<W, T, I>(t, s, x, z)) return s;
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    return -1;
}

// tile_lookup that also reports, for an absent key, the first empty slot on
// its probe path (where tile_insert_at starts).
template <int W, typename T, typename I>
__device__ __forceinline__ int tile_lookup_at(const Tile<W, T, I>& t, const uint64_t* x, const uint64_t* z,
                                              uint32_t* slot) {
    uint32_t h = tile_hash<W>(x, z, t.hbits);
    for (int probe = 0; probe < t.hcap; ++probe) {
        int s = (int)t.hash[h];
        if (s < 0) {
            *slot = h;
            return -1;
        }
        if (tile_key_eq<W, T, I>(t, s, x, z)) return s;
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    *slot = h;
    return -1;
}

// Inserts entry idx (no key of the table equals its key) probing from slot h
// on its probe path: slots taken meanwhile are skipped.
template <int W, typename T, typename I>
__device__ __forceinline__ void tile_insert_at(const Tile<W, T, I>& t, int idx, uint32_t h) {
    for (int probe = 0; probe < t.hcap; ++probe) {
        if ((int)atomic_cas_idx(&t.hash[h], (I)-1, (I)idx) < 0) return;
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    atomicExch(t.flag, (int)FAIL_HASH);
}

// Inserts entry idx (key and coefficient already stored).  merge: if the key is
// present, add the coefficient into the existing entry and leave idx dead.
template <int W, typename T, typename I>
__device__ __forceinline__ void tile_insert(const Tile<W, T, I>& t, int idx, const uint64_t* x,
                                            const uint64_t* z, bool merge) {
    uint32_t h = tile_hash<W>(x, z, t.hbits);
    for (int probe = 0; probe < t.hcap; ++probe) {
        int prev = (int)atomic_cas_idx(&t.hash[h], (I)-1, (I)idx);
        if (prev < 0) return;
        if (merge && tile_key_eq<W, T, I>(t, prev, x, z)) {
            atomicAdd(&t.c[prev], t.c[idx]);
            t.c[idx] = T(0);
            return;
        }
        h = (h + 1) & (uint32_t)(t.hcap - 1);
    }
    atomicExch(t.flag, (int)FAIL_HASH);
}

// Appends entry i to active list `which` (warp-aggregated; all lanes of the
// warp must call it together, `want` false for lanes that append nothing).
template <int W, typename T, typename I>
__device__ __forceinline__ void act_append(const Tile<W, T, I>& t, int which, int counter, bool want, int i) {
    const unsigned msk = __ballot_sync(0xffffffffu, want);
    if (!msk) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(msk) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&t.nact[counter], __popc(msk));
    base = __shfl_sync(0xffffffffu, base, leader);
    const int pos = base + __popc(msk & ((1u << lane) - 1u));
    if (want && !PP_OOB(pos < t.cap, 3, t.ctr)) t.act[(size_t)which * t.cap + pos] = (I)i;
}

template <typename T>
__device__ __forceinline__ T eps_of(const StepParams& p);
template <>
__device__ __forceinline__ double eps_of<double>(const StepParams& p) { return p.eps; }
template <>
__device__ __forceinline__ float eps_of<float>(const StepParams& p) { return p.eps_f; }

// Writes string (x, z, c) to slot `slot` of bucket nb of the destination
// layout (slot from the bucket's fill counter): into the bucket's region, or
// past it into the overflow area: the warp's own shard, or, when that one
// is full, the next shards in turn (a shard's counter may pass its capacity;
// readers clamp it).
template <int W, typename T>
__device__ __forceinline__ void emit_at(const StepParams& p, uint32_t nb, uint32_t slot, const uint64_t* x,
                                        const uint64_t* z, T c) {
    if (PP_OOB(nb < p.dB, 8, p.counters)) return;
    if ((uint64_t)slot < p.dC) {
        size_t pos = (size_t)nb * p.dC + slot;
        if (PP_OOB(pos < p.dcap, 5, p.counters)) return;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            p.dx[(size_t)w * p.dcap + pos] = x[w];
            p.dz[(size_t)w * p.dcap + pos] = z[w];
        }
        static_cast<T*>(p.dc)[pos] = c;
        return;
    }
    const uint64_t shard_cap = p.rpcap / NSPILL;
    int shard = (int)((blockIdx.x * 8 + (threadIdx.x >> 5)) % NSPILL);
    for (int tries = 0; tries < NSPILL; ++tries, shard = (shard + 1) % NSPILL) {
        unsigned long long k = atomicAdd(&p.spill_ctr[shard], 1ull);
        if (k >= shard_cap) continue;
        k += (unsigned long long)shard * shard_cap;
        if (PP_OOB(k < p.rpcap, 6, p.counters)) return;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            p.rpx[(size_t)w * p.rpcap + k] = x[w];
            p.rpz[(size_t)w * p.rpcap + k] = z[w];
        }
        static_cast<T*>(p.rpc)[k] = c;
        p.rpb[k] = nb;
        p.rps[k] = slot - (uint32_t)p.dC;
        return;
    }
    atomicAdd(&p.counters[CTR_ERR_REGION], 1ull);
}

// Appends a string to bucket nb of the destination layout (see emit_at).
template <int W, typename T>
__device__ __forceinline__ void emit(const StepParams& p, uint32_t nb, const uint64_t* x,
                                     const uint64_t* z, T c) {
    emit_at<W, T>(p, nb, atomicAdd(&p.dfill[nb], 1u), x, z, c);
}

// Scatters the live strings of a tile (entries i0, i0 + stride, ... below n)
// into the next layout's buckets.  The destination slots are taken
// EMIT_BATCH strings at a time, so that a thread has that many fill-counter
// atomics in flight before it writes (measured: 4 helps the CTA tiers, whose
// threads scatter many strings each; the warp tier is fastest with 1).
// Returns the number of strings written.
template <int EMIT_BATCH, int W, typename T, typename I, class D>
__device__ __forceinline__ int emit_tile(const Tile<W, T, I>& t, const D& adn, const StepParams& p, int i0,
                                         int stride, int n) {
    const uint32_t bmask = p.dB - 1;
    int cnt = 0;
    for (int ib = i0; ib < n; ib += EMIT_BATCH * stride) {
        uint32_t nb[EMIT_BATCH], slot[EMIT_BATCH];
        uint64_t x[EMIT_BATCH][W], z[EMIT_BATCH][W];
        T c[EMIT_BATCH];
#pragma unroll
        for (int j = 0; j < EMIT_BATCH; ++j) {
            const int i = ib + j * stride;
            c[j] = i < n ? tile_coef(t, i) : T(0);
            nb[j] = 0;
            if (c[j] != T(0)) {
                tile_key<W, T, I>(t, i, x[j], z[j]);
                nb[j] = bucket_of<W>(adn, x[j], z[j], bmask);
            }
        }
#pragma unroll
        for (int j = 0; j < EMIT_BATCH; ++j) slot[j] = c[j] != T(0) ? atomicAdd(&p.dfill[nb[j]], 1u) : 0u;
#pragma unroll
        for (int j = 0; j < EMIT_BATCH; ++j) {
            if (c[j] == T(0)) continue;
            emit_at<W, T>(p, nb[j], slot[j], x[j], z[j], c[j]);
            ++cnt;
        }
    }
    return cnt;
}

// Processes one bucket: load, prologue (merge/truncate the input observable,
// noise map), gate rounds, then writes the surviving strings into the next
// layout's buckets (or the compact final array).  Returns false, having
// written nothing, when the bucket does not fit the tile.
//
// The whole CTA works on one bucket; rounds are separated by CTA barriers.
// This serves the buckets too large for one warp (see k_process_warp).
template <int W, typename T, typename I>
__device__ bool process_bucket(const Tile<W, T, I>& t, const GateTab<W, T>& tab, const ActDesc& ad,
                               const ActDesc& adn, const StepParams& p, uint32_t b) {
    const SubLayerDesc& d = *p.desc;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31;
    const T eps = eps_of<T>(p);
    const uint32_t n_in = p.sfill[b];
    long long clk0 = p.phase ? clock64() : 0;
    auto phase_mark = [&](int ph) {
        if (p.phase && tid == 0) {
            long long clk1 = clock64();
            atomicAdd(&p.phase[4 + ph], (unsigned long long)(clk1 - clk0));
            clk0 = clk1;
        }
    };

    for (int i = tid; i < t.hcap; i += nt) t.hash[i] = (I)-1;
    // work count per lifetime (see pp_warp.cuh): births subtract g + 1, deaths
    // add g + 1, strings alive at the end add the sub-layer's gate count
    long long upd = 0;
    if (tid == 0) {
        *t.n = (int)n_in;
        *t.flag = (n_in > p.max_load) ? (int)FAIL_LOAD : 0;
        *t.live = 0;
        t.nact[0] = 0;
        t.nact[1] = 0;
        t.nact[2] = 0;
    }
    __syncthreads();
    if (*t.flag) return false;

    // ---- load: the bucket's region, then its overflow strings (shared-memory
    // tiles copy asynchronously, every thread's copies in flight at once), then
    // the hash table
    const size_t base = (size_t)b * p.sC;
    const size_t obase = (n_in > p.sC) ? (size_t)p.soff[b] : 0;
    constexpr bool kAsync = sizeof(I) == 2;   // the global tier's tile is in global memory
    for (int i = tid; i < (int)n_in; i += nt) {
        const bool reg = (uint64_t)i < p.sC;
        const size_t src = reg ? base + i : obase + (i - p.sC);
        const uint64_t* ax = reg ? p.sx : p.spx;
        const uint64_t* az = reg ? p.sz : p.spz;
        const size_t acap = reg ? p.scap : p.spcap;
        const T* ac = static_cast<const T*>(reg ? p.sc : p.spc);
        if (PP_OOB(src < acap && i < t.cap, 1, p.counters)) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (kAsync) {
                cp_async8(&t.x[(size_t)w * t.cap + i], &ax[(size_t)w * acap + src]);
                cp_async8(&t.z[(size_t)w * t.cap + i], &az[(size_t)w * acap + src]);
            } else {
                t.x[(size_t)w * t.cap + i] = ax[(size_t)w * acap + src];
                t.z[(size_t)w * t.cap + i] = az[(size_t)w * acap + src];
            }
        }
        if (kAsync) cp_async_coef(&t.c[i], ac + src);
        else t.c[i] = ac[src];
        t.sr[i] = 0;
    }
    if (kAsync) {
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    for (int i = tid; i < (int)n_in; i += nt) {
        uint64_t x[W], z[W];
        tile_key<W, T, I>(t, i, x, z);
        tile_insert<W, T, I>(t, i, x, z, d.first != 0);
    }
    __syncthreads();
    phase_mark(0);

    // ---- prologue: truncation of the merged input, noise map, and each live
    // string's gate mask (gates of the sub-layer that act on it, listed order)
    int my_live = 0;
    for (int i0 = 0; i0 < (int)n_in; i0 += nt) {
        const int i = i0 + tid;
        bool has_gates = false;
        if (i < (int)n_in) {
            T c = t.c[i];
            uint64_t x[W], z[W];
            tile_key<W, T, I>(t, i, x, z);
            if (d.first && c != T(0)) {
                if (Coef<T>::small(c, eps) || (p.w_max >= 0 && weight_of<W>(x, z) > p.w_max)) c = T(0);
            }
            if (p.has_noise && c != T(0)) {
                c = noise_scale<T>(p.noise, c, noise_exponent<W>(p.noise, x, z));
                if (Coef<T>::small(c, eps)) c = T(0);
            }
            t.c[i] = c;
            uint64_t gm[W];
#pragma unroll
            for (int w = 0; w < W; ++w) gm[w] = 0ull;
            if (c != T(0)) {
                ++my_live;
                uint64_t A[W], Mx[W], Mz[W];
                activity<W>(ad, x, z, A, Mx, Mz);
                if (ad.ident) {
#pragma unroll
                    for (int w = 0; w < W; ++w) gm[w] = A[w];
                } else {
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        uint64_t a = A[w];
                        while (a) {
                            int bpos = __ffsll((long long)a) - 1;
                            a &= a - 1;
                            int gidx = ad.order[64 * w + bpos];
                            gm[gidx >> 6] |= 1ull << (gidx & 63);
                        }
                    }
                }
#pragma unroll
                for (int w = 0; w < W; ++w) has_gates |= gm[w] != 0ull;
            }
#pragma unroll
            for (int w = 0; w < W; ++w) t.g[(size_t)w * t.cap + i] = gm[w];
        }
        act_append<W, T, I>(t, 0, 0, has_gates, i);
    }
    if (my_live) atomicAdd(t.live, my_live);
    __syncthreads();
    const int live0 = *t.live;
    phase_mark(1);

    // ---- gate rounds.  Round r: every listed string applies the next gate of
    // its mask (orbit members share the mask, so a string and its partner use
    // the same gate); the next round's list keeps the strings still live with
    // gates left, and new and revived strings join it.  A string's partner
    // under its round gate is unique to it, so lookup, rotation, truncation
    // and the next list share one pass: round r reads coefficients from
    // buffer r & 1 and writes the other, so both members of a pair read the
    // values from before the gate.  List counters rotate over three slots
    // (read in round r, appended in round r + 1, cleared meanwhile), so one
    // barrier per round suffices.  Counters are bumped once per warp (votes),
    // never once per thread: in a large orbit every string applies the same
    // gate in the same round.
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r <= 64 * W; ++r) {
        const int cur = r & 1, nxt = cur ^ 1;
        const int na = t.nact[r % 3];
        if (na == 0) break;
        if (tid == 0) t.nact[(r + 2) % 3] = 0;
        const I* L = t.act + (size_t)cur * t.cap;
        const T* ccur = t.cbuf(cur);
        T* cnxt = t.cbuf(nxt);
        const uint8_t stamp = (uint8_t)(r + 1);
        for (int k0 = 0; k0 < na; k0 += nt) {
            const int k = k0 + tid;
            bool create = false, revive = false, keep = false;
            int i = 0, j = -1, gg = -1;
            uint32_t hslot = 0;
            T v = T(0);
            uint64_t qx[W], qz[W], gm[W];
            if (k < na) {
                i = (int)L[k];
                uint64_t x[W], z[W];
                tile_key<W, T, I>(t, i, x, z);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    gm[w] = t.g[(size_t)w * t.cap + i];
                    if (gg < 0 && gm[w]) {
                        gg = 64 * w + __ffsll((long long)gm[w]) - 1;
                        gm[w] &= gm[w] - 1;
                    }
                }
                if (PP_OOB(gg >= 0, 4, t.ctr)) gg = 0;
                bool more = false;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    t.g[(size_t)w * t.cap + i] = gm[w];
                    more |= gm[w] != 0ull;
                    qx[w] = x[w] ^ tab.rx[gg][w];
                    qz[w] = z[w] ^ tab.rz[gg][w];
                }
                // a partner over the weight cap is never in the tile (every
                // string that enters it is within the cap, or is killed in the
                // prologue before any gate), and is never created
                const bool reach = p.w_max < 0 || weight_of<W>(qx, qz) <= p.w_max;
                if (reach) j = tile_lookup_at<W, T, I>(t, qx, qz, &hslot);
                if (PP_OOB(j < *t.n, 2, t.ctr)) j = -1;
                // i R P = phi Q: sign of P's sin-branch into its partner Q
                const int phi = branch_negative<W, T>(tab, gg, x, z) ? -1 : 1;
                const T cs = tab.cs[gg], sn = tab.sn[gg];
                const T c = ccur[i];
                T c2 = T(0);
                if (j >= 0) {
                    // the partner's value before this gate: it is live and in
                    // this round's list (stamp r, or r + 1 once its own thread
                    // has written), or dead
                    const uint8_t sj = t.sr[j];
                    if (sj == stamp || sj == (uint8_t)r) c2 = ccur[j];
                }
                T ci;
                if (c2 != T(0)) {
                    // both members of the pair rotate; the partner's contribution
                    // into P carries the opposite sign (i R Q = -phi P)
                    ci = Coef<T>::rot(cs, c, sn, c2, -phi);
                } else {
                    ci = Coef<T>::mul(cs, c);
                    v = Coef<T>::mul(sn, c);
                    if (phi < 0) v = -v;
                    if (reach && !Coef<T>::small(v, eps)) {
                        if (j >= 0) revive = true;
                        else create = true;
                    }
                }
                if (Coef<T>::small(ci, eps)) {
                    ci = T(0);
                    upd += gg + 1;
                }
                cnxt[i] = ci;
                t.sr[i] = stamp;
                keep = ci != T(0) && more;
            }
            // entry indices for new strings: one atomic per warp
            const unsigned cm = __ballot_sync(FULL, create);
            int nbase = 0;
            if (cm) {
                if (lane == __ffs(cm) - 1) nbase = atomicAdd(t.n, __popc(cm));
                nbase = __shfl_sync(FULL, nbase, __ffs(cm) - 1);
            }
            int idx = j;
            if (create) {
                idx = nbase + __popc(cm & lt);
                if (idx >= t.cap) {
                    atomicExch(t.flag, (int)FAIL_POOL);
                    create = false;
                }
            }
            if (create) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    t.x[(size_t)w * t.cap + idx] = qx[w];
                    t.z[(size_t)w * t.cap + idx] = qz[w];
                }
            }
            const bool born = create || revive;
            bool join = false;
            if (born) {
                // a new string, or one truncated earlier revived: it joins the
                // orbit with the gates the orbit has left
                cnxt[idx] = v;
                t.sr[idx] = stamp;
                bool more = false;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    t.g[(size_t)w * t.cap + idx] = gm[w];
                    more |= gm[w] != 0ull;
                }
                if (create) {
                    __threadfence_block();
                    tile_insert_at<W, T, I>(t, idx, hslot);
                }
                join = more;
                upd -= gg + 1;
            }
            act_append<W, T, I>(t, nxt, (r + 1) % 3, keep, i);
            act_append<W, T, I>(t, nxt, (r + 1) % 3, join, idx);
        }
        __syncthreads();
        if (*t.flag) return false;
    }
    phase_mark(2);

    // ---- output
    if (d.final_) {
        __shared__ unsigned long long s_base;
        if (tid == 0) *t.live = 0;
        __syncthreads();
        const int nf = *t.n;
        int cnt = 0;
        for (int i = tid; i < nf; i += nt)
            if (tile_coef(t, i) != T(0)) ++cnt;
        upd += (long long)cnt * d.n_gates;
        int off = cnt ? atomicAdd(t.live, cnt) : 0;
        __syncthreads();
        if (tid == 0) {
            s_base = atomicAdd(&p.counters[CTR_OUT], (unsigned long long)*t.live);
            atomicAdd(&p.counters[CTR_EMITTED + (p.work_ctr - CTR_WORK)], (unsigned long long)*t.live);
        }
        __syncthreads();
        unsigned long long pos = s_base + off;
        for (int i = tid; i < nf; i += nt) {
            const T c = tile_coef(t, i);
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
        const int cnt = emit_tile<4, W, T, I>(t, adn, p, tid, nt, *t.n);
        if (cnt) {
            atomicAdd(&p.counters[CTR_OUT], (unsigned long long)cnt);
            atomicAdd(&p.counters[CTR_EMITTED + (p.work_ctr - CTR_WORK)], (unsigned long long)cnt);
        }
        upd += (long long)cnt * d.n_gates;
    }
    __syncthreads();
    phase_mark(3);
    (void)live0;
    if (tid == 0) atomicAdd(&p.counters[CTR_LOADED + (p.work_ctr - CTR_WORK)], (unsigned long long)n_in);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) upd += __shfl_xor_sync(FULL, upd, o);
    if (lane == 0 && upd) atomicAdd(&p.counters[CTR_UPDATES], (unsigned long long)upd);
    return true;
}

// Hash slots of a tile: the power of two at least twice its entries.
__host__ __device__ constexpr size_t tile_hcap(size_t cap) {
    size_t h = 1;
    while (h < 2 * cap) h <<= 1;
    return h;
}

// Bytes carve_tile lays out for a tile of `cap` entries.
template <int W, typename T, typename I>
__host__ __device__ constexpr size_t tile_layout_bytes(size_t cap) {
    return sizeof(uint64_t) * W * cap * 3 + sizeof(T) * cap * 2 + sizeof(I) * tile_hcap(cap) +
           sizeof(I) * 2 * cap + cap;
}

template <int W, typename T, typename I>
__device__ __forceinline__ Tile<W, T, I> carve_tile(unsigned char* mem, int cap, int* ctl) {
    Tile<W, T, I> t;
    t.ctr = nullptr;
    t.cap = cap;
    t.hcap = (int)tile_hcap((size_t)cap);
    t.hbits = 31 - __clz(t.hcap);
    unsigned char* q = mem;
    t.x = reinterpret_cast<uint64_t*>(q); q += sizeof(uint64_t) * W * cap;
    t.z = reinterpret_cast<uint64_t*>(q); q += sizeof(uint64_t) * W * cap;
    t.g = reinterpret_cast<uint64_t*>(q); q += sizeof(uint64_t) * W * cap;
    t.c = reinterpret_cast<T*>(q); q += sizeof(T) * cap;
    t.c1 = reinterpret_cast<T*>(q); q += sizeof(T) * cap;
    t.hash = reinterpret_cast<I*>(q); q += sizeof(I) * t.hcap;
    t.act = reinterpret_cast<I*>(q); q += sizeof(I) * 2 * cap;
    t.sr = reinterpret_cast<uint8_t*>(q); q += cap;
    t.n = ctl + 0;
    t.flag = ctl + 1;
    t.live = ctl + 2;
    t.nact = ctl + 4;
    return t;
}

template <int W, typename T>
__device__ __forceinline__ void load_gate_table(GateTab<W, T>& tab, const SubLayerDesc& d) {
    if (threadIdx.x == 0) {
        tab.cls = d.cls;
        tab.shift = d.shift;
        tab.psign = d.psign;
    }
    for (int g = threadIdx.x; g < d.n_gates && g < 64 * W; g += blockDim.x) {
        int slot = d.cls == CLS_GENERIC ? g : d.slot_of[g];
        uint64_t rx[W], rz[W];
        slot_generator<W>(d, slot, rx, rz);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            tab.rx[g][w] = rx[w];
            tab.rz[g][w] = rz[w];
        }
        tab.cs[g] = T(d.cs[slot]);
        tab.sn[g] = T(d.sn[slot]);
        tab.slot[g] = (uint8_t)slot;
    }
}

// Shared-memory tiers: persistent CTAs take buckets from a work queue (all
// buckets, or the list a smaller tier passed on); a bucket that does not fit is
// passed to the next tier.
template <int W, typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 64 ? 4 : 1) k_process(const StepParams p0, const StepParams* ps, int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ctl[8];
    __shared__ uint32_t s_b;
    __shared__ GateTab<W, T> tab;
    __shared__ ActDesc s_ad, s_adn;
    __shared__ StepParams p;
    if (!load_params(p, p0, ps)) return;
    Tile<W, T, int16_t> t = carve_tile<W, T, int16_t>(smem, cap, ctl);
    t.ctr = p.counters;
    if (threadIdx.x == 0) make_act(*p.desc, s_ad);
    if (threadIdx.x == (NT > 32 ? 32 : 0) && p.next) make_act(*p.next, s_adn);
    load_gate_table<W, T>(tab, *p.desc);
    const uint32_t n_items = work_items(p);
    for (;;) {
        if (threadIdx.x == 0) s_b = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        __syncthreads();
        const uint32_t k = s_b;
        if (k >= n_items) break;
        const uint32_t b = p.in_list ? p.in_list[k] : k;
        if (p.sfill[b] != 0) {
            bool ok = process_bucket<W, T, int16_t>(t, tab, s_ad, s_adn, p, b);
            if (!ok && threadIdx.x == 0) {
                atomicAdd(&p.counters[CTR_FAIL + (*t.flag - 1)], 1ull);
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
__global__ void __launch_bounds__(NWARPS * 32) k_process_global(const StepParams p0, const StepParams* ps,
                                                                unsigned char* scratch, unsigned char* const* scratch_of,
                                                                size_t slice_bytes, int cap) {
    __shared__ int ctl[8];
    __shared__ uint32_t s_k;
    __shared__ GateTab<W, T> tab;
    __shared__ ActDesc s_ad, s_adn;
    __shared__ StepParams p;
    if (!load_params(p, p0, ps)) return;
    // the global-tier slices: the launch's own, or in a batched launch those of
    // instance y (scratch_of[y]), one per CTA column
    unsigned char* base = scratch_of ? scratch_of[blockIdx.y] : scratch;
    (void)slice_bytes;
    (void)cap;
    Tile<W, T, int32_t> t = carve_tile<W, T, int32_t>(base + p.gslice * blockIdx.x, p.gcap, ctl);
    t.ctr = p.counters;
    if (threadIdx.x == 0) make_act(*p.desc, s_ad);
    if (threadIdx.x == 32 && p.next) make_act(*p.next, s_adn);
    load_gate_table<W, T>(tab, *p.desc);
    const uint32_t n_items = work_items(p);
    for (;;) {
        if (threadIdx.x == 0) s_k = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        __syncthreads();
        const uint32_t k = s_k;
        if (k >= n_items) break;
        bool ok = process_bucket<W, T, int32_t>(t, tab, s_ad, s_adn, p, p.in_list[k]);
        if (!ok && threadIdx.x == 0) {
            atomicAdd(&p.counters[CTR_FAIL + (*t.flag - 1)], 1ull);
            atomicAdd(&p.counters[CTR_ERR_FALLBACK], 1ull);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- input merge

// The input observable's duplicate strings are summed before the first
// sub-layer, exactly and independently of their order: a hash table over the
// input keys (slot: owner = smallest input index with that key, count, and a
// 128-bit fixed-point accumulator) collects every duplicated string's
// coefficients as integers (trunc(c * 2^80)), and the owner carries the total,
// rounded once to the nearest double, into the first layout.  Strings without
// duplicates keep their coefficient untouched.
struct InputMerge {
    int* owner;                  // [H] smallest input index of the slot's key, -1: empty
    unsigned* count;             // [H] input strings with the slot's key
    unsigned long long* acc;     // [2H] 128-bit accumulator (low word, high word)
    uint32_t hmask;              // H - 1
};

template <int W>
__device__ __forceinline__ bool input_key_eq(const uint64_t* ox, const uint64_t* oz, size_t a, size_t b) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w) eq = eq && ox[a * W + w] == ox[b * W + w] && oz[a * W + w] == oz[b * W + w];
    return eq;
}

template <int W>
__device__ __forceinline__ uint32_t input_slot0(const uint64_t* ox, const uint64_t* oz, size_t i, uint32_t hmask) {
    return tile_hash<W>(ox + i * W, oz + i * W, 31) & hmask;
}

// Slot of input string i's key (after k_input_claim).
template <int W>
__device__ __forceinline__ uint32_t input_slot(const uint64_t* ox, const uint64_t* oz, size_t i, const InputMerge& m) {
    uint32_t h = input_slot0<W>(ox, oz, i, m.hmask);
    for (uint32_t probe = 0; probe <= m.hmask; ++probe) {
        const int o = m.owner[h];
        if (o < 0 || input_key_eq<W>(ox, oz, (size_t)o, i)) return h;
        h = (h + 1) & m.hmask;
    }
    return h;
}

template <int W>
__global__ void k_input_claim(const uint64_t* ox, const uint64_t* oz, size_t n, InputMerge m) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = input_slot0<W>(ox, oz, i, m.hmask);
        for (uint32_t probe = 0; probe <= m.hmask; ++probe) {
            const int prev = atomicCAS(&m.owner[h], -1, (int)i);
            // a slot's owner only ever moves to a smaller index of the same key
            if (prev < 0 || input_key_eq<W>(ox, oz, (size_t)prev, i)) {
                if (prev >= 0) atomicMin(&m.owner[h], (int)i);
                atomicAdd(&m.count[h], 1u);
                break;
            }
            h = (h + 1) & m.hmask;
        }
    }
}

template <int W>
__global__ void k_input_accumulate(const uint64_t* ox, const uint64_t* oz, const double* oc, size_t n,
                                   InputMerge m) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t h = input_slot<W>(ox, oz, i, m);
        if (m.count[h] < 2) continue;
        // two's-complement 128-bit addition, split into words with the carry
        const __int128 v = to_fixed80(oc[i]);
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
        const unsigned long long old = atomicAdd(&m.acc[2 * (size_t)h], lo);
        atomicAdd(&m.acc[2 * (size_t)h + 1], hi + (old + lo < old ? 1ull : 0ull));
    }
}

// Scatters the merged input observable into the first sub-layer's buckets
// (the destination layout of p): one string per key, from its owner.
template <int W, typename T>
__global__ void k_scatter_input(const uint64_t* ox, const uint64_t* oz, const double* oc, size_t n,
                                InputMerge m, StepParams p) {
    const SubLayerDesc& d = *p.next;
    const uint32_t bmask = p.dB - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t h = input_slot<W>(ox, oz, i, m);
        if (m.owner[h] != (int)i) continue;
        double c = oc[i];
        if (m.count[h] > 1) {
            const unsigned __int128 t = ((unsigned __int128)m.acc[2 * (size_t)h + 1] << 64) | m.acc[2 * (size_t)h];
            c = fixed80_to_double((__int128)t);
        }
        uint64_t x[W], z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            x[w] = ox[i * W + w];
            z[w] = oz[i * W + w];
        }
        uint32_t b = bucket_of<W>(d, x, z, bmask);
        emit<W, T>(p, b, x, z, T(c));
    }
}

// Whether a sub-layer's output outgrew its layout (strings lost to a full
// overflow area, or more strings than the capacity): the sub-layer then runs
// again from its input, whose grouped overflow strings share the grouped
// overflow area with the output's, so the output's must not be grouped.
__device__ __forceinline__ bool spill_outgrown(const unsigned long long* ctr, uint64_t dcap) {
    return ctr && (ctr[CTR_ERR_REGION] != 0 || ctr[CTR_OUT] > dcap);
}

// Arguments of the overflow grouping of one layout (batched launches take an
// array, one per grid row / slice).
struct SpillArgs {
    const uint32_t* fill;
    uint32_t nB;
    uint64_t C;
    uint64_t* soff;
    unsigned long long* total;
    const uint64_t* rx;
    const uint64_t* rz;
    const void* rc;
    const uint32_t* rb;
    const uint32_t* rs;
    uint64_t rcap;
    const unsigned long long* shard_fill;
    uint64_t* ox;
    uint64_t* oz;
    void* oc;
    uint64_t ocap;
    const unsigned long long* ctr;   // the sub-layer's counters (see spill_outgrown)
    uint64_t dcap;                   // capacity of the destination layout
    // zeroing at the start of a sub-layer (k_clear): the destination fill
    // counters [0, zero_n), the overflow shard counters, and the counters
    uint32_t* zero_fill;
    uint32_t zero_n;
    unsigned long long* zero_shards;
    unsigned long long* zero_ctr;
    int zero_ctr_n;
};

// Zeroes, for instance blockIdx.y, what a sub-layer starts from.
__global__ void k_clear(const SpillArgs* a) {
    const SpillArgs& s = a[blockIdx.y];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < s.zero_n; i += gridDim.x * blockDim.x)
        s.zero_fill[i] = 0u;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < NSPILL; i += blockDim.x) s.zero_shards[i] = 0ull;
        for (int i = threadIdx.x; i < s.zero_ctr_n; i += blockDim.x) s.zero_ctr[i] = 0ull;
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

// Grid (NSPILL, Y): blocks (s, y) move shard s's strings y*256 + t, stepping
// by Y*256, up to the shard's fill (nothing to do when nothing spilled).
// Batched k_spill_offsets: instance blockIdx.y (its `total` must start at 0).
__global__ void k_spill_offsets_batch(const SpillArgs* a) {
    __shared__ unsigned long long s_scan[1024];
    __shared__ unsigned long long s_base;
    const SpillArgs& s = a[blockIdx.y];
    for (uint32_t b0 = blockIdx.x * blockDim.x; b0 < s.nB; b0 += gridDim.x * blockDim.x) {
        const uint32_t b = b0 + threadIdx.x;
        unsigned long long ex = 0;
        if (b < s.nB && (uint64_t)s.fill[b] > s.C) ex = (uint64_t)s.fill[b] - s.C;
        s_scan[threadIdx.x] = ex;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            unsigned long long v = (int)threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0ull;
            __syncthreads();
            s_scan[threadIdx.x] += v;
            __syncthreads();
        }
        if (threadIdx.x == blockDim.x - 1) s_base = atomicAdd(s.total, s_scan[threadIdx.x]);
        __syncthreads();
        if (b < s.nB) s.soff[b] = s_base + s_scan[threadIdx.x] - ex;
        __syncthreads();
    }
}

// Batched k_spill_move: grid (NSPILL, Y, instances).
template <int W, typename T>
__global__ void k_spill_move_batch(const SpillArgs* a) {
    const SpillArgs& s = a[blockIdx.z];
    if (spill_outgrown(s.ctr, s.dcap)) return;
    const uint64_t shard_cap = s.rcap / NSPILL;
    const uint64_t sh = blockIdx.x;
    const uint64_t fill = s.shard_fill[sh] < shard_cap ? s.shard_fill[sh] : shard_cap;
    const T* rc = static_cast<const T*>(s.rc);
    T* oc = static_cast<T*>(s.oc);
    for (uint64_t j = blockIdx.y * (uint64_t)blockDim.x + threadIdx.x; j < fill; j += (uint64_t)gridDim.y * blockDim.x) {
        const uint64_t k = sh * shard_cap + j;
        const uint64_t dst = s.soff[s.rb[k]] + s.rs[k];
        if (dst >= s.ocap) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            s.ox[(size_t)w * s.ocap + dst] = s.rx[(size_t)w * s.rcap + k];
            s.oz[(size_t)w * s.ocap + dst] = s.rz[(size_t)w * s.rcap + k];
        }
        oc[dst] = rc[k];
    }
}

template <int W, typename T>
__global__ void k_spill_move(const uint64_t* rx, const uint64_t* rz, const T* rc, const uint32_t* rb,
                             const uint32_t* rs, uint64_t rcap, const unsigned long long* shard_fill,
                             const uint64_t* soff, uint64_t* ox, uint64_t* oz, T* oc, uint64_t ocap,
                             const unsigned long long* ctr, uint64_t dcap) {
    if (spill_outgrown(ctr, dcap)) return;
    const uint64_t shard_cap = rcap / NSPILL;
    const uint64_t s = blockIdx.x;
    const uint64_t fill = shard_fill[s] < shard_cap ? shard_fill[s] : shard_cap;
    for (uint64_t j = blockIdx.y * (uint64_t)blockDim.x + threadIdx.x; j < fill; j += (uint64_t)gridDim.y * blockDim.x) {
        const uint64_t k = s * shard_cap + j;
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

// ----------------------------------------------------------------------------- noise map

// Shared-memory copy of a noise map's tables (sizes fixed per map).
struct NoiseSmem {
    size_t grp, shift, xmask, pidx, c2, ftab;   // byte offsets
    size_t bytes;
};

// Shared-memory copy of a map's tables: the factor table of the coefficient
// type (FP64 entries, or float pairs: 16 KB either way), the group tables, the
// pair corrections and the cross-group pair index.
__host__ __device__ inline NoiseSmem noise_smem_layout(int n_sites, int n_groups, int n_shift, int n_pairs,
                                                       int W) {
    NoiseSmem L;
    size_t o = 0;
    L.ftab = o; o += sizeof(double) * 8 * 256;
    L.grp = o; o += sizeof(int64_t) * 256 * (size_t)n_groups;
    L.c2 = o; o += sizeof(int64_t) * 16 * (size_t)n_pairs;
    L.xmask = o; o += sizeof(uint64_t) * (size_t)n_shift * W;
    L.shift = o; o += sizeof(int32_t) * (size_t)n_shift;
    L.pidx = o; o += sizeof(int32_t) * (size_t)n_shift * n_sites;
    L.bytes = (o + 15) & ~(size_t)15;
    return L;
}

// Applies an inverse (or forward) Pauli-Lindblad map in place to every string
// of a bucketed layout: the buckets' regions, then the grouped overflow area.
// The map's tables are staged in shared memory; strings are streamed once.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_noise(const uint64_t* x, const uint64_t* z, T* c, uint64_t cap,
                                               const uint32_t* fill, uint32_t B, uint64_t C,
                                               const uint64_t* ox, const uint64_t* oz, T* oc, uint64_t ocap,
                                               uint64_t n_over, NoiseDesc nz, int n_pairs, double eps,
                                               float eps_f) {
    extern __shared__ __align__(16) unsigned char smem[];
    const NoiseSmem L = noise_smem_layout(nz.n_sites, nz.n_groups, nz.n_shift, n_pairs, W);
    {
        auto cp = [&](size_t off, const void* src, size_t bytes) {
            const uint32_t* s32 = static_cast<const uint32_t*>(src);
            uint32_t* d32 = reinterpret_cast<uint32_t*>(smem + off);
            for (size_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d32[i] = s32[i];
        };
        cp(L.ftab, sizeof(T) == 8 ? static_cast<const void*>(nz.etab) : static_cast<const void*>(nz.ftab),
           sizeof(double) * 8 * 256);
        cp(L.grp, nz.grp, sizeof(int64_t) * 256 * (size_t)nz.n_groups);
        cp(L.c2, nz.c2, sizeof(int64_t) * 16 * (size_t)n_pairs);
        cp(L.xmask, nz.xmask, sizeof(uint64_t) * (size_t)nz.n_shift * W);
        cp(L.shift, nz.shift, sizeof(int32_t) * (size_t)nz.n_shift);
        cp(L.pidx, nz.pidx, sizeof(int32_t) * (size_t)nz.n_shift * nz.n_sites);
    }
    __syncthreads();
    NoiseDesc sn = nz;
    sn.etab = reinterpret_cast<const double*>(smem + L.ftab);
    sn.ftab = reinterpret_cast<const float*>(smem + L.ftab);
    sn.grp = reinterpret_cast<const int64_t*>(smem + L.grp);
    sn.c2 = reinterpret_cast<const int64_t*>(smem + L.c2);
    sn.xmask = reinterpret_cast<const uint64_t*>(smem + L.xmask);
    sn.shift = reinterpret_cast<const int32_t*>(smem + L.shift);
    sn.pidx = reinterpret_cast<const int32_t*>(smem + L.pidx);
    const T e = sizeof(T) == 8 ? T(eps) : T(eps_f);

    auto apply = [&](const uint64_t* ax, const uint64_t* az, T* ac, uint64_t acap, uint64_t i) {
        T v = ac[i];
        if (v == T(0)) return;
        uint64_t xx[W], zz[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            xx[w] = ax[(size_t)w * acap + i];
            zz[w] = az[(size_t)w * acap + i];
        }
        v = noise_scale<T>(sn, v, noise_exponent<W>(sn, xx, zz));
        if (Coef<T>::small(v, e)) v = T(0);
        ac[i] = v;
    };
    // regions: one warp per bucket
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t b = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += warps) {
        const uint64_t f = fill[b] < C ? fill[b] : C;
        for (uint64_t i = lane; i < f; i += 32) apply(x, z, c, cap, b * C + i);
    }
    // grouped overflow strings
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_over;
         k += (uint64_t)gridDim.x * blockDim.x)
        apply(ox, oz, oc, ocap, k);
}

// ----------------------------------------------------------------------------- expectation

// Sum of c over strings with x == 0, in exact fixed point; one partial per CTA.
template <int W, typename T>
__global__ void k_expect(const uint64_t* x, const T* c, uint64_t cap, uint64_t n,
                         __int128* partial) {
    __shared__ __int128 s[256];
    __int128 acc = 0;
    bool bad = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        bool diag = true;
#pragma unroll
        for (int w = 0; w < W; ++w) diag = diag && x[(size_t)w * cap + i] == 0ull;
        if (diag) {
            const double v = (double)c[i];
            if (fix80_valid(v)) acc += to_fixed80(v);
            else bad = true;
        }
    }
    s[threadIdx.x] = acc;
    bad = __syncthreads_or(bad);
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = bad ? FIX80_INVALID : s[0];
}

}  // namespace pp
