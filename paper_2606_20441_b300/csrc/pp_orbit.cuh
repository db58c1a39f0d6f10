// Tier 0 for orbit sub-layers: one warp per bucket, strings grouped by orbit
// into dense per-orbit coefficient blocks.
//
// A sub-layer whose gates share one letter pattern, are listed in ascending
// slot order and have pairwise disjoint supports (an R_X layer; one colour of
// an R_ZZ layer) has a simple orbit structure.  If k of its gates act on a
// string P (anticommute with it; the same k gates act on every string P can
// become), the strings reachable from P are
//     P(u) = base * prod_{j: bit j of u set} R_{g_j},   u in [0, 2^k),
// where g_0 < g_1 < ... are the acting gates in listed order and `base` is the
// member whose "coordinate bits" are all 0.  The coordinate bit of gate g_j is
// one bit the gate flips on its first site (x if the gate has an X part there,
// else z); no other gate touches that site, so bit j of u reads it directly.
// Applying gate g_j pairs P(u) with P(u xor 2^j) and nothing else (Sec. I, Eq.
// evolve_gate: U^dag P U = cos(theta) P + i sin(theta) R P for anticommuting
// P), so gate-by-gate propagation with truncation after every gate (Sec. I.A)
// is, per orbit, a butterfly over the coordinate bits:
//
//   round r (the orbit's r-th acting gate): for every pair (u, u | 2^r),
//   rotate the two coefficients (an absent string has coefficient 0), then
//   truncate both.
//
// Each orbit of the bucket gets a dense block of 2^k coefficients.  Blocks are
// laid out by decreasing k, each aligned to its size, so the orbits that take
// part in round r (k > r) fill a prefix of the pool and pair j of round r is
// slots (s, s | 2^r) with s = j with a 0 bit inserted at position r, whatever
// orbit it falls in.  A round is one loop over that prefix: no lists, no
// allocation, no partner lookups.  Pairs with both coefficients 0 are skipped.
//
// The sign of a pair's sin-branches and the weight change of its members
// depend only on the letters the bit-0 member carries on the gate's sites,
// which are the base's (SubLayerDesc::ltab gives both); they are folded into
// per-orbit bit masks when the orbit is first seen.
//
// Work count (the canonical gate-by-gate number of live strings entering each
// gate) is kept per lifetime: a string live from listed gate b through listed
// gate d (inclusive) contributes d - b + 1, so each lane adds (g + 1) when a
// string dies at gate g, subtracts (g + 1) when one is born at gate g, and adds
// the sub-layer's gate count for every string alive at the end.
//
// A bucket's strings are staged in shared memory by asynchronous copies
// (cp.async) issued while the warp still works on the previous bucket.
// Buckets that do not fit the tile (too many strings, an orbit with more than
// ORB_KMAX acting gates, too many pool slots) are passed, untouched, to the
// sparse CTA tiers; nothing is written until a bucket is known to fit.
#pragma once

#include "pp_kernels.cuh"
#include "pp_warp.cuh"

namespace pp {

constexpr int ORB_WARPS = 4;            // warps per CTA; each owns its buckets
constexpr int ORB_KMAX = 12;            // largest orbit dimension this tier takes
constexpr int ORB_CLS = ORB_KMAX + 1;   // orbit size classes k = 0..ORB_KMAX
constexpr uint32_t ORB_EMPTY = 0xffffffffu;
constexpr uint8_t ORB_HOLE = 0xff;      // a string whose orbit another string of the bucket owns
constexpr uint32_t ORB_NONE = 0xffffffffu;

// Capacities of one warp's tile.
struct OrbCaps {
    int O;   // strings per bucket (the load limit); provisional orbit records
    int H;   // orbit hash slots (power of two, >= 2 O)
    int M;   // pool slots (sum of 2^k over the bucket's orbits)
    int S;   // round records (sum of k over the bucket's orbits)
};

// Byte offsets of a tile's arrays.
struct OrbLayout {
    size_t sx, sz, sc, rx, rz, om, pool, ou, oh, bo, pf, sb, rk, ri, cls, bytes;
};

template <int W, typename T>
__host__ __device__ constexpr OrbLayout orb_layout(OrbCaps k) {
    OrbLayout L{};
    size_t o = 0;
    auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    L.sx = o; o += a16(sizeof(uint64_t) * W * (size_t)k.O);
    L.sz = o; o += a16(sizeof(uint64_t) * W * (size_t)k.O);
    L.sc = o; o += a16(sizeof(T) * (size_t)k.O);
    L.rx = o; o += a16(sizeof(uint64_t) * W * (size_t)k.O);
    L.rz = o; o += a16(sizeof(uint64_t) * W * (size_t)k.O);
    L.om = o; o += a16(sizeof(uint64_t) * (size_t)k.O);
    L.pool = o; o += a16(sizeof(T) * (size_t)k.M);
    L.ou = o; o += a16(4 * (size_t)k.O);
    L.oh = o; o += a16(4 * (size_t)k.H);
    L.bo = o; o += a16(2 * (size_t)k.O);
    L.pf = o; o += a16(2 * (size_t)k.O);
    L.sb = o; o += a16(2 * (size_t)k.O);
    L.rk = o; o += a16((size_t)k.O);
    L.ri = o; o += a16((size_t)k.S);
    L.cls = o; o += a16(sizeof(int) * 4 * ORB_CLS);
    L.bytes = o;
    return L;
}

template <int W, typename T>
struct OrbTile {
    uint64_t* sx;      // [W][O] staged strings of the bucket (word-major)
    uint64_t* sz;
    T* sc;             // [O]
    uint64_t* rx;      // [W][O] orbit base, by provisional index (= the owner string's index)
    uint64_t* rz;
    uint64_t* om;      // [O] by final index: Pm | Nm << 16 | Sm << 32 | wb << 48 | k << 56
    T* pool;           // [M] dense coefficient blocks
    uint32_t* ou;      // [O] per staged string: provisional orbit index << 16 | u (ORB_EMPTY: dead)
    uint32_t* oh;      // [H] orbit hash: tag << 16 | provisional index
    uint16_t* bo;      // [O] final index -> provisional index
    uint16_t* pf;      // [O] provisional index -> final index
    uint16_t* sb;      // [O] final index -> first round record
    uint8_t* rk;       // [O] provisional index -> k (ORB_HOLE: not an orbit owner)
    uint8_t* ri;       // [S] slot of the r-th acting gate of each orbit
    int* cnt;          // [ORB_CLS] orbits per class, then their running rank
    int* start;        // [ORB_CLS] first pool slot of class k (classes by decreasing k)
    int* orb0;         // [ORB_CLS] first final index of class k
    int* ri0;          // [ORB_CLS] first round record of class k
};

template <int W, typename T>
__device__ __forceinline__ OrbTile<W, T> carve_orb(unsigned char* mem, OrbCaps k) {
    const OrbLayout L = orb_layout<W, T>(k);
    OrbTile<W, T> t;
    t.sx = reinterpret_cast<uint64_t*>(mem + L.sx);
    t.sz = reinterpret_cast<uint64_t*>(mem + L.sz);
    t.sc = reinterpret_cast<T*>(mem + L.sc);
    t.rx = reinterpret_cast<uint64_t*>(mem + L.rx);
    t.rz = reinterpret_cast<uint64_t*>(mem + L.rz);
    t.om = reinterpret_cast<uint64_t*>(mem + L.om);
    t.pool = reinterpret_cast<T*>(mem + L.pool);
    t.ou = reinterpret_cast<uint32_t*>(mem + L.ou);
    t.oh = reinterpret_cast<uint32_t*>(mem + L.oh);
    t.bo = reinterpret_cast<uint16_t*>(mem + L.bo);
    t.pf = reinterpret_cast<uint16_t*>(mem + L.pf);
    t.sb = reinterpret_cast<uint16_t*>(mem + L.sb);
    t.rk = mem + L.rk;
    t.ri = mem + L.ri;
    int* c = reinterpret_cast<int*>(mem + L.cls);
    t.cnt = c;
    t.start = c + ORB_CLS;
    t.orb0 = c + 2 * ORB_CLS;
    t.ri0 = c + 3 * ORB_CLS;
    return t;
}

// ----------------------------------------------------------------------------- async copies

// Starts copying bucket b's n_in strings (its region, then its grouped
// overflow strings) into the tile's staging arrays; n_in <= O.  The warp
// waits for them with cp_async_wait_all.
template <int W, typename T>
__device__ __forceinline__ void stage_bucket(const OrbTile<W, T>& t, const OrbCaps& K, const StepParams& p,
                                             uint32_t b, int n_in) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)b * p.sC;
    const size_t obase = ((uint64_t)n_in > p.sC) ? (size_t)p.soff[b] : 0;
    for (int i = lane; i < n_in; i += 32) {
        const bool reg = (uint64_t)i < p.sC;
        const size_t src = reg ? base + i : obase + (i - p.sC);
        const uint64_t* ax = reg ? p.sx : p.spx;
        const uint64_t* az = reg ? p.sz : p.spz;
        const size_t acap = reg ? p.scap : p.spcap;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            cp_async8(&t.sx[(size_t)w * K.O + i], &ax[(size_t)w * acap + src]);
            cp_async8(&t.sz[(size_t)w * K.O + i], &az[(size_t)w * acap + src]);
        }
        cp_async_coef(&t.sc[i], static_cast<const T*>(reg ? p.sc : p.spc) + src);
    }
    cp_async_commit();
}

// ----------------------------------------------------------------------------- helpers

// 32-bit hash of an orbit base for the tile's orbit table.
template <int W>
__device__ __forceinline__ uint32_t orb_hash(const uint64_t* x, const uint64_t* z) {
    uint64_t h = 0x243F6A8885A308D3ULL;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h ^= x[w] * (0x9E3779B97F4A7C15ULL + 2 * w);
        h ^= z[w] * (0xC2B2AE3D27D4EB4FULL + 2 * w);
        h ^= h >> 29;
    }
    h *= 0xD6E8FEB86659FD93ULL;
    return (uint32_t)(h >> 32);
}

// x, z ^= the generators of the gates at the slots set in C.
template <int W>
__device__ __forceinline__ void orb_flip(const ActDesc& d, const uint64_t* C, uint64_t* x, uint64_t* z) {
    uint64_t Cs[W];
    if (d.cls == CLS_LOCAL2) shl_words<W>(C, d.shift, Cs);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t cb = d.cls == CLS_LOCAL2 ? Cs[w] : 0ull;
        x[w] ^= (d.ax ? C[w] : 0ull) ^ (d.bx ? cb : 0ull);
        z[w] ^= (d.az ? C[w] : 0ull) ^ (d.bz ? cb : 0ull);
    }
}

// Size class of pool slot s, searching from class k_lo upward.  Classes are
// laid out by decreasing k (class k occupies [start[k], start[k - 1])), so s
// belongs to the smallest class k >= k_lo with start[k] <= s.
template <int W, typename T>
__device__ __forceinline__ int class_of(const OrbTile<W, T>& t, int s, int k_lo, int kmax) {
    int k = k_lo;
    while (k < kmax && s < t.start[k]) ++k;
    return k;
}

// Weight of orbit member u from the orbit's masks.
__device__ __forceinline__ int orb_weight(uint64_t om, uint32_t u) {
    const uint32_t pm = (uint32_t)(om & 0xffffu), nm = (uint32_t)((om >> 16) & 0xffffu);
    return (int)((om >> 48) & 0xffu) + __popc(u & pm) - __popc(u & nm);
}

// Processes one bucket whose n_in (<= O) strings are staged.  Once the staged
// strings are consumed it starts staging the next bucket (next_b, next_n) and
// sets *staged_next.  Returns false, having written nothing to global memory,
// when the bucket does not fit the tile.
template <int W, typename T>
__device__ bool orbit_bucket(const OrbTile<W, T>& t, const OrbCaps& K, const ActDesc& ad, const ActDesc& adn,
                             const uint8_t* ltab, const T* gcs, const T* gsn, const StepParams& p, int n_in,
                             uint32_t next_b, int next_n, bool* staged_next, WarpAcc& acc,
                             unsigned long long& upd_total) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const T eps = eps_of<T>(p);
    long long clk0 = p.phase ? clock64() : 0;
    auto phase_mark = [&](int ph) {
        if (p.phase) {
            const long long clk1 = clock64();
            if (lane == 0) atomicAdd(&p.phase[ph], (unsigned long long)(clk1 - clk0));
            clk0 = clk1;
        }
    };
    for (int i = lane; i < K.H; i += 32) t.oh[i] = ORB_EMPTY;
    if (lane < ORB_CLS) t.cnt[lane] = 0;
    __syncwarp();

    // ---- pass 1: each staged string's orbit (base, k, coordinate u)
    bool bad = false;
    int kmax = 0;
    for (int i0 = 0; i0 < n_in; i0 += 32) {
        const int i = i0 + lane;
        const bool have = i < n_in;
        uint64_t x[W], z[W];
        T c = T(0);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            x[w] = have ? t.sx[(size_t)w * K.O + i] : 0ull;
            z[w] = have ? t.sz[(size_t)w * K.O + i] : 0ull;
        }
        if (have) c = t.sc[i];
        const bool live = c != T(0);
        uint64_t A[W], Mx[W], Mz[W], C1[W], bx[W], bz[W];
        activity<W>(ad, x, z, A, Mx, Mz);
        int k = 0;
        uint32_t u = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            C1[w] = A[w] & (ad.ax ? x[w] : z[w]);
            bx[w] = x[w];
            bz[w] = z[w];
        }
        orb_flip<W>(ad, C1, bx, bz);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t m = live ? A[w] : 0ull;
            while (m) {
                const int bp = __ffsll((long long)m) - 1;
                m &= m - 1;
                if (k < 16 && ((C1[w] >> bp) & 1ull)) u |= 1u << k;
                ++k;
            }
        }
        if (k > ORB_KMAX) bad = true;
        // provisional record, at the string's own index
        if (live) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                t.rx[(size_t)w * K.O + i] = bx[w];
                t.rz[(size_t)w * K.O + i] = bz[w];
            }
        }
        __syncwarp();
        int o = i;
        bool owner = live;
        if (live && k > 0 && !bad) {
            const uint32_t h = orb_hash<W>(bx, bz);
            const uint32_t tag = h >> 16;
            uint32_t slot = h & (uint32_t)(K.H - 1);
            bool placed = false;
            for (int probe = 0; probe < K.H; ++probe) {
                const uint32_t v = atomicCAS(&t.oh[slot], ORB_EMPTY, (tag << 16) | (uint32_t)i);
                if (v == ORB_EMPTY) {
                    placed = true;
                    break;
                }
                if ((v >> 16) == tag) {
                    const int q = (int)(v & 0xffffu);
                    bool eq = true;
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        eq = eq && t.rx[(size_t)w * K.O + q] == bx[w] && t.rz[(size_t)w * K.O + q] == bz[w];
                    if (eq) {
                        o = q;
                        owner = false;
                        placed = true;
                        break;
                    }
                }
                slot = (slot + 1) & (uint32_t)(K.H - 1);
            }
            if (!placed) bad = true;
        }
        if (have) {
            t.rk[i] = (owner && !bad) ? (uint8_t)k : ORB_HOLE;
            t.ou[i] = live ? (((uint32_t)o << 16) | u) : ORB_EMPTY;
        }
        if (owner && !bad) atomicAdd(&t.cnt[k], 1);
        if (live && k > kmax) kmax = k;
    }
    if (__any_sync(FULL, bad)) return false;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, off));
    __syncwarp();

    // ---- class layout: pool blocks, final indices and round records by decreasing k
    int pool_n = 0, ri_n = 0;
    if (lane == 0) {
        int n_orb = 0;
        for (int k = kmax; k >= 0; --k) {
            t.start[k] = pool_n;
            t.orb0[k] = n_orb;
            t.ri0[k] = ri_n;
            pool_n += t.cnt[k] << k;
            ri_n += t.cnt[k] * k;
            n_orb += t.cnt[k];
            t.cnt[k] = 0;   // becomes the running rank
        }
    }
    pool_n = __shfl_sync(FULL, pool_n, 0);
    ri_n = __shfl_sync(FULL, ri_n, 0);
    if (pool_n > K.M || ri_n > K.S) return false;
    __syncwarp();

    // ---- pass 1.5: each orbit owner takes its rank; round records and masks
    for (int i = lane; i < n_in; i += 32) {
        const int k = t.rk[i];
        if (k == ORB_HOLE) continue;
        const int rank = atomicAdd(&t.cnt[k], 1);
        const int f = t.orb0[k] + rank;
        const int sbase = t.ri0[k] + rank * k;
        t.bo[f] = (uint16_t)i;
        t.pf[i] = (uint16_t)f;
        t.sb[f] = (uint16_t)sbase;
        uint64_t bx[W], bz[W], A[W], Mx[W], Mz[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            bx[w] = t.rx[(size_t)w * K.O + i];
            bz[w] = t.rz[(size_t)w * K.O + i];
        }
        activity<W>(ad, bx, bz, A, Mx, Mz);
        uint32_t pm = 0, nm = 0, sm = 0;
        int j = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t m = A[w];
            while (m && j < k) {
                const int bp = __ffsll((long long)m) - 1;
                m &= m - 1;
                const int slot = 64 * w + bp;
                int la = letter_at<W>(bx, bz, slot);
                if (ad.cls == CLS_LOCAL2) la += 4 * letter_at<W>(bx, bz, slot + ad.shift);
                const uint32_t le = ltab[la];
                const int dw = (int)((le >> 1) & 3u) - 1;
                if (le & 1u) sm |= 1u << j;
                if (dw > 0) pm |= 1u << j;
                if (dw < 0) nm |= 1u << j;
                t.ri[sbase + j] = (uint8_t)slot;
                ++j;
            }
        }
        const uint64_t wb = (uint64_t)weight_of<W>(bx, bz);
        t.om[f] = (uint64_t)pm | ((uint64_t)nm << 16) | ((uint64_t)sm << 32) | (wb << 48) | ((uint64_t)k << 56);
    }
    for (int s = lane; s < pool_n; s += 32) t.pool[s] = T(0);
    __syncwarp();

    // ---- pass 2: coefficients into their blocks
    for (int i = lane; i < n_in; i += 32) {
        const uint32_t ou = t.ou[i];
        if (ou == ORB_EMPTY) continue;
        const int o = (int)(ou >> 16);
        const int k = t.rk[o];
        const int f = t.pf[o];
        t.pool[t.start[k] + ((f - t.orb0[k]) << k) + (int)(ou & 0xffffu)] = t.sc[i];
    }
    __syncwarp();
    // the staged strings are consumed: start fetching the next bucket
    if (next_b != ORB_NONE && next_n > 0 && next_n <= K.O) {
        stage_bucket<W, T>(t, K, p, next_b, next_n);
        *staged_next = true;
    }
    phase_mark(0);

    // ---- rounds: butterflies over the pool prefix of the orbits with k > r
    long long upd = 0;          // this lane's share of the bucket's work count
    for (int r = 0; r < kmax; ++r) {
        const int npairs = t.start[r] >> 1;
        const int bit = 1 << r;
        for (int j = lane; j < npairs; j += 32) {
            const int s0 = ((j >> r) << (r + 1)) | (j & (bit - 1));
            const int s1 = s0 | bit;
            const T c0 = t.pool[s0], c1 = t.pool[s1];
            if (c0 == T(0) && c1 == T(0)) continue;
            const int k = class_of(t, s0, r + 1, kmax);
            const int off = s0 - t.start[k];
            const int f = t.orb0[k] + (off >> k);
            const uint32_t u0 = (uint32_t)(off & ((1 << k) - 1));
            const uint64_t om = t.om[f];
            const int slot = t.ri[t.sb[f] + r];
            const int g = ad.order[slot];
            const bool negphi = ((om >> (32 + r)) & 1ull) != 0;
            const T cs = gcs[slot], sn = gsn[slot];
            T n0, n1;
            if (c0 != T(0) && c1 != T(0)) {
                // each member keeps cos of itself plus the other's sin-branch; the
                // bit-1 member's branch into the bit-0 member has the opposite sign
                n0 = Coef<T>::rot(cs, c0, sn, c1, negphi ? 1 : -1);
                n1 = Coef<T>::rot(cs, c1, sn, c0, negphi ? -1 : 1);
            } else if (c0 != T(0)) {
                n0 = Coef<T>::mul(cs, c0);
                n1 = Coef<T>::mul(sn, c0);
                if (negphi) n1 = -n1;
            } else {
                n1 = Coef<T>::mul(cs, c1);
                n0 = Coef<T>::mul(sn, c1);
                if (!negphi) n0 = -n0;
            }
            if (Coef<T>::small(n0, eps)) n0 = T(0);
            if (Coef<T>::small(n1, eps)) n1 = T(0);
            if (p.w_max >= 0) {   // a string born here must respect the weight cap
                if (c0 == T(0) && n0 != T(0) && orb_weight(om, u0) > p.w_max) n0 = T(0);
                if (c1 == T(0) && n1 != T(0) && orb_weight(om, u0 | (uint32_t)bit) > p.w_max) n1 = T(0);
            }
            if (c0 != T(0) && n0 == T(0)) upd += g + 1;
            if (c0 == T(0) && n0 != T(0)) upd -= g + 1;
            if (c1 != T(0) && n1 == T(0)) upd += g + 1;
            if (c1 == T(0) && n1 != T(0)) upd -= g + 1;
            t.pool[s0] = n0;
            t.pool[s1] = n1;
        }
        __syncwarp();
    }
    phase_mark(2);

    // ---- output: rebuild each live string from its orbit base and coordinate
    const int G = ad.n_gates;
    unsigned long long emitted = 0;
    unsigned long long pos = 0;
    const bool fin = p.desc->final_ != 0;
    if (fin) {
        int cnt = 0;
        for (int s = lane; s < pool_n; s += 32) cnt += t.pool[s] != T(0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(FULL, cnt, off);
        if (lane == 0 && cnt) pos = atomicAdd(&p.counters[CTR_OUT], (unsigned long long)cnt);
        pos = __shfl_sync(FULL, pos, 0);
        emitted = (unsigned long long)cnt;
    }
    const uint32_t bmask = p.dB - 1;
    int cnt = 0;
    for (int s0 = 0; s0 < pool_n; s0 += 32) {
        const int s = s0 + lane;
        const T c = s < pool_n ? t.pool[s] : T(0);
        const bool lv = c != T(0);
        uint64_t x[W], z[W];
        if (lv) {
            const int k = class_of(t, s, 0, kmax);
            const int off = s - t.start[k];
            const int f = t.orb0[k] + (off >> k);
            uint32_t u = (uint32_t)(off & ((1 << k) - 1));
            const int o = t.bo[f];
            const int sbase = t.sb[f];
            uint64_t C[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                x[w] = t.rx[(size_t)w * K.O + o];
                z[w] = t.rz[(size_t)w * K.O + o];
                C[w] = 0ull;
            }
            while (u) {
                const int j = __ffs(u) - 1;
                u &= u - 1;
                const int slot = t.ri[sbase + j];
                C[slot >> 6] |= 1ull << (slot & 63);
            }
            orb_flip<W>(ad, C, x, z);
            upd += G;
        }
        if (fin) {
            const unsigned lm = __ballot_sync(FULL, lv);
            if (lv) {
                const unsigned long long q = pos + __popc(lm & lt);
                if (q < p.dcap) {
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        p.dx[(size_t)w * p.dcap + q] = x[w];
                        p.dz[(size_t)w * p.dcap + q] = z[w];
                    }
                    static_cast<T*>(p.dc)[q] = c;
                } else {
                    atomicAdd(&p.counters[CTR_ERR_REGION], 1ull);
                }
            }
            pos += __popc(lm);
        } else if (lv) {
            ++cnt;
            emit<W, T>(p, bucket_of<W>(adn, x, z, bmask), x, z, c);
        }
    }
    if (!fin) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(FULL, cnt, off);
        emitted = (unsigned long long)cnt;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) upd += __shfl_xor_sync(FULL, upd, off);
    phase_mark(3);
    upd_total += (unsigned long long)upd;
    acc.loaded += (unsigned long long)n_in;
    acc.emitted += emitted;
    return true;
}

template <int W, typename T>
__global__ void __launch_bounds__(32 * ORB_WARPS) k_process_orbit(const StepParams p0, const StepParams* ps, OrbCaps K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ T s_cs[64 * W], s_sn[64 * W];
    __shared__ uint8_t s_ltab[16];
    __shared__ unsigned long long s_acc[3];
    __shared__ ActDesc s_ad, s_adn;
    __shared__ StepParams p;
    if (!load_params(p, p0, ps)) return;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SubLayerDesc& d = *p.desc;
    if (threadIdx.x < 3) s_acc[threadIdx.x] = 0ull;
    if (threadIdx.x < 16) s_ltab[threadIdx.x] = d.ltab[threadIdx.x];
    for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) {
        s_cs[i] = T(d.cs[i]);
        s_sn[i] = T(d.sn[i]);
    }
    if (threadIdx.x == 0) make_act(d, s_ad);
    if (threadIdx.x == 32 && p.next) make_act(*p.next, s_adn);
    __syncthreads();

    const OrbTile<W, T> t = carve_orb<W, T>(smem + orb_layout<W, T>(K).bytes * wid, K);
    const int lim = (int)min((uint32_t)K.O, p.max_load);
    WarpAcc acc{0ull, 0ull, 0ull};
    unsigned long long upd = 0;
    const uint32_t n_items = work_items(p);
    // the next bucket of the warp's queue and its string count
    auto take = [&](uint32_t* b, int* n) {
        uint32_t k = 0;
        if (lane == 0) k = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        *b = k < n_items ? (p.in_list ? p.in_list[k] : k) : ORB_NONE;
        *n = *b != ORB_NONE ? (int)p.sfill[*b] : 0;
    };
    uint32_t b;
    int n;
    take(&b, &n);
    bool staged = false;
    if (b != ORB_NONE && n > 0 && n <= lim) {
        stage_bucket<W, T>(t, K, p, b, n);
        staged = true;
    }
    while (b != ORB_NONE) {
        uint32_t b2;
        int n2;
        take(&b2, &n2);
        if (n2 > lim) n2 = lim + 1;   // passed on unread
        bool staged2 = false;
        if (n > 0) {
            bool ok = false;
            int reason = FAIL_LOAD;
            if (n <= lim && staged) {
                cp_async_wait_all();
                __syncwarp();
                ok = orbit_bucket<W, T>(t, K, s_ad, s_adn, s_ltab, s_cs, s_sn, p, n, b2, n2 <= lim ? n2 : 0,
                                        &staged2, acc, upd);
                reason = FAIL_POOL;
            }
            if (!ok && lane == 0) {
                atomicAdd(&p.counters[CTR_FAIL + (reason - 1)], 1ull);
                const unsigned long long j = atomicAdd(&p.counters[p.defer_ctr], 1ull);
                p.out_list[j] = b;
            }
        }
        if (!staged2) {
            cp_async_wait_all();   // nothing of an abandoned bucket may still be landing
            __syncwarp();
            if (b2 != ORB_NONE && n2 > 0 && n2 <= lim) {
                stage_bucket<W, T>(t, K, p, b2, n2);
                staged2 = true;
            }
        }
        __syncwarp();
        b = b2;
        n = n2;
        staged = staged2;
    }
    cp_async_wait_all();
    if (lane == 0) {
        atomicAdd(&s_acc[0], upd);
        atomicAdd(&s_acc[1], acc.loaded);
        atomicAdd(&s_acc[2], acc.emitted);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int tier = p.work_ctr - CTR_WORK;
        if (s_acc[0]) atomicAdd(&p.counters[CTR_UPDATES], s_acc[0]);
        if (s_acc[1]) atomicAdd(&p.counters[CTR_LOADED + tier], s_acc[1]);
        if (s_acc[2]) {
            atomicAdd(&p.counters[CTR_EMITTED + tier], s_acc[2]);
            if (!d.final_) atomicAdd(&p.counters[CTR_OUT], s_acc[2]);
        }
    }
}

}  // namespace pp
