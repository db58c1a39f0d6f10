// Device-side core of libpp: sub-layer descriptors, per-string activity and
// orbit keys, Pauli-product phases, and the tile processor that applies every
// gate of one sub-layer to a bucket of strings held in shared memory.
//
// Method (Sec. I, Eq. evolve_gate / evolve_noise; App. G): backward propagation
// of a Pauli sum, one gate at a time, each gate followed by truncation.  The
// kernels reproduce that per-gate semantics exactly while reading and writing
// each string once per *sub-layer* (a run of commuting gates of one kind):
//
//   * A sub-layer's gates pairwise commute, so whether gate g acts on a string
//     (anticommutes with it) is the same for the string and for every string it
//     can be mapped to within the sub-layer.  The set of acting gates ("activity")
//     and the union of their supports are therefore invariant along the orbit.
//   * Masking the string with that union gives an orbit key: strings that can
//     ever meet (be each other's partner P xor R_g) share it.  Buckets are formed
//     by hashing the key, so every orbit lies inside one bucket.
//   * Inside a bucket the gates are applied in rounds: in round r each string
//     applies the r-th gate of its own activity set, in listed order.  Orbits are
//     independent, so this is the gate-by-gate result for every orbit at once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pp {

constexpr int MAXW = 2;          // up to 128 qubits
constexpr int MAX_SITES = 128;
constexpr int MAX_SEG = 4;
constexpr int MAX_GEN = 64;      // gates in a generic sub-layer
constexpr int FIX_SHIFT = 56;    // noise exponents in fixed point: value * 2^56

enum SubClass : int {
    CLS_NONE = 0,     // no gates (noise only, or the initial merge pass)
    CLS_LOCAL1 = 1,   // single-qubit rotations of one letter, e.g. R_X on sites
    CLS_LOCAL2 = 2,   // two-qubit rotations of one letter pair and one site shift, e.g. R_ZZ
    CLS_GENERIC = 3   // anything else: up to 64 explicit generators
};

// One fused sub-layer.  For class gates the "slot" of a gate is its first site a;
// the gate's generator is letter (ax,az) on a and, for LOCAL2, (bx,bz) on a+shift.
// The listed (backward-application) order is: segment 0's slots ascending, then
// segment 1's, ...  For generic sub-layers the slot is the gate index j.
struct SubLayerDesc {
    int cls;
    int ax, az, bx, bz;
    int shift;
    int nseg;
    int n_gates;
    int noise;                    // index of the noise map applied before the gates, or -1
    int first;                    // 1: input observable (merge duplicates, truncate)
    int final_;                   // 1: last sub-layer (outputs go to the compact result)
    int layer_end;                // 1: last sub-layer of a circuit layer (top-K applies after it)
    int ident;                    // 1: a gate's listed index equals its slot (one ascending
                                  //    segment starting at slot 0 with no gaps, or generic)
    uint16_t psign;               // class sub-layers: bit la + 4 lb set when a string with
                                  //    letters (la, lb) (code x + 2z) on a gate's sites
                                  //    (a, a + shift) sends its sin-branch into its partner
                                  //    with a negative sign (i R P = -P')
    int orb;                      // 1: one letter pattern, one ascending segment, disjoint
                                  //    supports: the orbit tier may process it (pp_orbit.cuh)
    // Orbit sub-layers: for the letters (la, lb) (code x + 2z) that the member
    // with coordinate bit 0 carries on a gate's sites (a, a + shift), entry
    // la + 4 lb holds bit 0: the sign of its sin-branch into its partner is
    // negative; bits 1-2: weight(partner) - weight(member) + 1 on those sites.
    // 0xff marks letter pairs that commute with the gate.
    uint8_t ltab[16];
    uint64_t seg[MAX_SEG][MAXW];
    uint64_t all[MAXW];           // union of segments
    double cs[MAX_SITES];         // cos(theta) by slot
    double sn[MAX_SITES];         // sin(theta) by slot
    int16_t order[MAX_SITES];     // listed index of the gate in each slot
    int16_t slot_of[MAX_SITES];   // slot of each listed gate
    uint64_t gx[MAX_GEN][MAXW];   // generic generators
    uint64_t gz[MAX_GEN][MAXW];
};

// The fields of a sub-layer that a string's activity, gate mask and orbit key
// need: small enough to stage in shared memory once per CTA.
struct ActDesc {
    int cls;
    int ax, az, bx, bz;
    int shift;
    int n_gates;
    int ident;                    // SubLayerDesc::ident
    uint64_t all[MAXW];
    int16_t order[MAX_SITES];
    const uint64_t* gx;           // generic generators [MAX_GEN][MAXW], in global memory
    const uint64_t* gz;
};

// Sparse Pauli-Lindblad map evaluated from tables.  Letter code l = x + 2z
// (I=0, X=1, Z=2, Y=3).  Exponents are 64-bit fixed point (2^-56 units), summed
// exactly, so any grouping of the terms gives the same exponent.
struct NoiseDesc {
    int mode;                     // 0: exp(+2s), 1: exp(-2s)
    int n_generic;
    int n_shift;                  // classes of 2-local generator supports (a, a + shift)
    int n_sites;
    int n_groups;                 // 4-site groups, (n_sites + 3) / 4
    const int64_t* grp;           // [n_groups][256] exponent part of group g (sites 4g..4g+3) by
                                  //   its letters, index (x nibble) | (z nibble) << 4: for each
                                  //   site, every 1- or 2-local generator touching it that
                                  //   anticommutes with its letter there (identity on the rest
                                  //   of its support), plus the correction of each pair inside
                                  //   the group
    const int32_t* shift;         // [n_shift] site distance of the class
    const uint64_t* xmask;        // [n_shift][W] first sites of the class's pairs that cross groups
    const int32_t* pidx;          // [n_shift][n] pair starting at site a in the class, or -1
    const int64_t* c2;            // [P][16] correction for pairs with both sites in the
                                  //         support: T2[la,lb] - T2[la,I] - T2[I,lb], index la + 4 lb
    const uint64_t* gen_x;        // [n_generic][W] heavier generators
    const uint64_t* gen_z;
    const int64_t* gen_lam;
    const double* etab;           // [8][256] exp(+-2 * b * 2^(8i - 56)): factor tables by
                                  //          byte i of the fixed-point exponent (FP64 form)
    const float* ftab;            // [8][256][2] the same factors as float pairs (head, tail),
                                  //          head + tail within 2^-48 of the factor (FP32 form)
};

// ----------------------------------------------------------------------------- bit helpers

__device__ __forceinline__ int popc64(uint64_t v) { return __popcll(v); }

// Leading zeros of a nonzero word, and a double from its bits, on host and device.
__host__ __device__ inline int clz64_hd(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
}
__host__ __device__ inline double __longlong_as_double_hd(long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double d;
    __builtin_memcpy(&d, &b, sizeof(d));
    return d;
#endif
}

template <int W>
__device__ __forceinline__ void shr_words(const uint64_t* v, int d, uint64_t* out) {
    // out = v >> d as a W-word little-endian integer (0 <= d < 64*W)
#pragma unroll
    for (int w = 0; w < W; ++w) {
        int src = w + d / 64;
        int sh = d % 64;
        uint64_t lo = (src < W) ? v[src] : 0ull;
        uint64_t hi = (src + 1 < W) ? v[src + 1] : 0ull;
        out[w] = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
    }
}

template <int W>
__device__ __forceinline__ void shl_words(const uint64_t* v, int d, uint64_t* out) {
#pragma unroll
    for (int w = W - 1; w >= 0; --w) {
        int src = w - d / 64;
        int sh = d % 64;
        uint64_t hi = (src >= 0) ? v[src] : 0ull;
        uint64_t lo = (src - 1 >= 0) ? v[src - 1] : 0ull;
        out[w] = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
    }
}

// Position of the r-th (0-based) set bit of v; v must have more than r set bits.
__device__ __forceinline__ int select64(uint64_t v, int r) {
    unsigned lo = (unsigned)v;
    int c = __popc(lo);
    if (r < c) return __fns(lo, 0, r + 1);
    return 32 + __fns((unsigned)(v >> 32), 0, r - c + 1);
}

// Power of i in R * S = i^e (R xor S) for Hermitian Pauli strings (Y = i X Z):
// per qubit e = r_x r_z + s_x s_z + 2 r_z s_x - (r_x^s_x)(r_z^s_z)  (mod 4).
template <int W>
__device__ __forceinline__ int product_phase(const uint64_t* rx, const uint64_t* rz,
                                             const uint64_t* sx, const uint64_t* sz) {
    int e = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        e += popc64(rx[w] & rz[w]) + popc64(sx[w] & sz[w]) + 2 * popc64(rz[w] & sx[w]) -
             popc64((rx[w] ^ sx[w]) & (rz[w] ^ sz[w]));
    }
    return e & 3;
}

template <int W>
__device__ __forceinline__ int anticommutes(const uint64_t* px, const uint64_t* pz,
                                            const uint64_t* rx, const uint64_t* rz) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += popc64((px[w] & rz[w]) ^ (pz[w] & rx[w]));
    return s & 1;
}

template <int W>
__device__ __forceinline__ int weight_of(const uint64_t* x, const uint64_t* z) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += popc64(x[w] | z[w]);
    return s;
}

__device__ __forceinline__ uint64_t fmix64(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdULL;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ULL;
    h ^= h >> 33;
    return h;
}

template <int W>
__device__ __forceinline__ uint64_t hash_key(const uint64_t* x, const uint64_t* z) {
    uint64_t h = 0x9e3779b97f4a7c15ULL;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h = fmix64(h ^ x[w]);
        h = fmix64(h ^ (z[w] + 0x632be59bd9b4e019ULL));
    }
    return h;
}

// ----------------------------------------------------------------------------- activity

// Row j of a generic-generator table, whether held as [MAX_GEN][MAXW] arrays
// (SubLayerDesc) or as a flat pointer (ActDesc).
__device__ __forceinline__ const uint64_t* gen_row(const uint64_t (*g)[MAXW], int j) { return g[j]; }
__device__ __forceinline__ const uint64_t* gen_row(const uint64_t* g, int j) { return g + (size_t)j * MAXW; }

__device__ __forceinline__ void make_act(const SubLayerDesc& s, ActDesc& d) {
    d.cls = s.cls;
    d.ax = s.ax; d.az = s.az; d.bx = s.bx; d.bz = s.bz;
    d.shift = s.shift;
    d.n_gates = s.n_gates;
    d.ident = s.ident;
    for (int w = 0; w < MAXW; ++w) d.all[w] = s.all[w];
    for (int i = 0; i < MAX_SITES; ++i) d.order[i] = s.order[i];
    d.gx = &s.gx[0][0];
    d.gz = &s.gz[0][0];
}

// Activity of string (x,z) in a sub-layer: bit per slot whose gate anticommutes
// with the string.  Also the union of the acting generators' supports (per
// letter bit), which masks the string into its orbit key.
template <int W, class D>
__device__ __forceinline__ void activity(const D& d, const uint64_t* x,
                                         const uint64_t* z, uint64_t* A, uint64_t* Mx,
                                         uint64_t* Mz) {
    if (d.cls == CLS_LOCAL1 || d.cls == CLS_LOCAL2) {
        uint64_t fa[W];
#pragma unroll
        for (int w = 0; w < W; ++w) fa[w] = (d.ax ? z[w] : 0ull) ^ (d.az ? x[w] : 0ull);
        if (d.cls == CLS_LOCAL1) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                A[w] = fa[w] & d.all[w];
                Mx[w] = d.ax ? A[w] : 0ull;
                Mz[w] = d.az ? A[w] : 0ull;
            }
        } else {
            uint64_t fb[W], fbs[W], As[W];
#pragma unroll
            for (int w = 0; w < W; ++w) fb[w] = (d.bx ? z[w] : 0ull) ^ (d.bz ? x[w] : 0ull);
            shr_words<W>(fb, d.shift, fbs);
#pragma unroll
            for (int w = 0; w < W; ++w) A[w] = (fa[w] ^ fbs[w]) & d.all[w];
            shl_words<W>(A, d.shift, As);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                Mx[w] = (d.ax ? A[w] : 0ull) | (d.bx ? As[w] : 0ull);
                Mz[w] = (d.az ? A[w] : 0ull) | (d.bz ? As[w] : 0ull);
            }
        }
    } else if (d.cls == CLS_GENERIC) {
        uint64_t a = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) Mx[w] = Mz[w] = 0ull;
        for (int j = 0; j < d.n_gates; ++j) {
            const uint64_t* gxj = gen_row(d.gx, j);
            const uint64_t* gzj = gen_row(d.gz, j);
            if (anticommutes<W>(x, z, gxj, gzj)) {
                a |= 1ull << j;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    Mx[w] |= gxj[w] | gzj[w];
                    Mz[w] |= gxj[w] | gzj[w];
                }
            }
        }
        A[0] = a;
#pragma unroll
        for (int w = 1; w < W; ++w) A[w] = 0ull;
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) A[w] = Mx[w] = Mz[w] = 0ull;
    }
}

template <int W>
__device__ __forceinline__ int count_active(const uint64_t* A) {
    int k = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) k += popc64(A[w]);
    return k;
}

// Slot of the r-th acting gate (listed order) for activity A.
template <int W>
__device__ __forceinline__ int select_slot(const SubLayerDesc& d, const uint64_t* A, int r) {
    if (d.cls == CLS_GENERIC) return select64(A[0], r);
    for (int s = 0; s < d.nseg; ++s) {
        uint64_t As[W];
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            As[w] = A[w] & d.seg[s][w];
            cnt += popc64(As[w]);
        }
        if (r < cnt) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int c = popc64(As[w]);
                if (r < c) return 64 * w + select64(As[w], r);
                r -= c;
            }
        }
        r -= cnt;
    }
    return -1;
}

// Generator (rx, rz) of the gate in `slot`.
template <int W>
__device__ __forceinline__ void slot_generator(const SubLayerDesc& d, int slot, uint64_t* rx,
                                               uint64_t* rz) {
    if (d.cls == CLS_GENERIC) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            rx[w] = d.gx[slot][w];
            rz[w] = d.gz[slot][w];
        }
        return;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) rx[w] = rz[w] = 0ull;
    int a = slot;
    uint64_t bit = 1ull << (a & 63);
    if (d.ax) rx[a >> 6] |= bit;
    if (d.az) rz[a >> 6] |= bit;
    if (d.cls == CLS_LOCAL2) {
        int b = a + d.shift;
        uint64_t bb = 1ull << (b & 63);
        if (d.bx) rx[b >> 6] |= bb;
        if (d.bz) rz[b >> 6] |= bb;
    }
}

// Multiply-xorshift hash of an orbit key for bucket selection.
template <int W>
__device__ __forceinline__ uint64_t bucket_hash(const uint64_t* kx, const uint64_t* kz) {
    uint64_t h = kx[0] * 0x9E3779B97F4A7C15ULL ^ (kz[0] + 0x632BE59BD9B4E019ULL) * 0xC2B2AE3D27D4EB4FULL;
#pragma unroll
    for (int w = 1; w < W; ++w)
        h ^= kx[w] * 0xD6E8FEB86659FD93ULL ^ (kz[w] + 0x85EBCA77C2B2AE63ULL) * 0xFF51AFD7ED558CCDULL;
    h ^= h >> 32;
    h *= 0xD6E8FEB86659FD93ULL;
    h ^= h >> 29;
    return h;
}

// Orbit key of a string for sub-layer d and its bucket among bmask + 1 buckets.
template <int W, class D>
__device__ __forceinline__ uint32_t bucket_of(const D& d, const uint64_t* x, const uint64_t* z,
                                              uint32_t bmask) {
    uint64_t A[W], Mx[W], Mz[W], kx[W], kz[W];
    activity<W>(d, x, z, A, Mx, Mz);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        kx[w] = x[w] & ~Mx[w];
        kz[w] = z[w] & ~Mz[w];
    }
    return (uint32_t)(bucket_hash<W>(kx, kz) >> 20) & bmask;
}

// ----------------------------------------------------------------------------- noise

// Exponent sum_{k: {P,E_k} = 0} lambda_k in 2^-56 fixed point: one table entry
// per 4-site group (the per-site terms, which already hold the one-sided part of
// every pair, and the pairs inside the group), plus a correction for each pair
// that crosses groups with both sites in supp(P), plus the heavier generators.
template <int W>
__device__ __forceinline__ int64_t noise_exponent(const NoiseDesc& nz, const uint64_t* x,
                                                  const uint64_t* z) {
    int64_t s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t xl = (uint32_t)x[w], xh = (uint32_t)(x[w] >> 32);
        const uint32_t zl = (uint32_t)z[w], zh = (uint32_t)(z[w] >> 32);
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const int G = 16 * w + g;
            if (G < nz.n_groups) {
                const uint32_t xv = g < 8 ? xl : xh, zv = g < 8 ? zl : zh;
                const int sh = 4 * (g & 7);
                const uint32_t idx = ((xv >> sh) & 15u) | (((zv >> sh) << 4) & 0xf0u);
                s += nz.grp[256 * G + idx];
            }
        }
    }
    if (nz.n_shift) {
        uint64_t sup[W];
#pragma unroll
        for (int w = 0; w < W; ++w) sup[w] = x[w] | z[w];
        for (int c = 0; c < nz.n_shift; ++c) {
            const int d = nz.shift[c];
            uint64_t sh[W];
            shr_words<W>(sup, d, sh);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t both = sup[w] & sh[w] & nz.xmask[(size_t)c * W + w];
                while (both) {
                    const int bpos = __ffsll((long long)both) - 1;
                    both &= both - 1;
                    const int a = 64 * w + bpos, bq = a + d;
                    const int la = (int)((x[w] >> bpos) & 1ull) + 2 * (int)((z[w] >> bpos) & 1ull);
                    const int lb = (int)((x[bq >> 6] >> (bq & 63)) & 1ull) + 2 * (int)((z[bq >> 6] >> (bq & 63)) & 1ull);
                    s += nz.c2[16 * nz.pidx[(size_t)c * nz.n_sites + a] + la + 4 * lb];
                }
            }
        }
    }
    for (int k = 0; k < nz.n_generic; ++k)
        if (anticommutes<W>(x, z, nz.gen_x + (size_t)k * W, nz.gen_z + (size_t)k * W))
            s += nz.gen_lam[k];
    return s;
}

// exp(+-2 s) for s = S * 2^-56 (S >= 0), as the product over the bytes of S of
// host-tabulated factors: exp(a + b) = exp(a) exp(b), so at most seven FP64
// multiplies instead of an FP64 exponential.  Each table entry is the exponential
// correctly rounded to double; the product carries at most a few ulp.
__device__ __forceinline__ double noise_factor(const NoiseDesc& nz, int64_t S) {
    uint64_t u = (uint64_t)S;
    double f = 1.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t byte = (uint32_t)(u >> (8 * i)) & 0xffu;
        if (byte) f = __dmul_rn(f, nz.etab[256 * i + byte]);
    }
    return f;
}

// The same product carried as an unevaluated float pair (head h, tail l), on the
// FP32 pipe (the FP64 pipe is narrow on this part).  Each step multiplies the
// pair by a table pair: the exact product of the heads (an FMA recovers its
// rounding error), the two cross terms folded into that error, and a Fast2Sum
// that renormalises; the tail-by-tail term (below 2^-48 relative) is dropped.
// Entry 0 of every byte table is (1, 0), so every byte takes the same path.  The
// pair stays within ~2^-44 of the factor (the product of eight steps).
__device__ __forceinline__ void noise_factor_pair(const NoiseDesc& nz, int64_t S, float& h, float& l) {
    const uint64_t u = (uint64_t)S;
    h = 1.0f;
    l = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t byte = (uint32_t)(u >> (8 * i)) & 0xffu;
        const float2 t = reinterpret_cast<const float2*>(nz.ftab)[256 * i + byte];
        const float p = __fmul_rn(h, t.x);
        float e = __fmaf_rn(h, t.x, -p);
        e = __fmaf_rn(h, t.y, e);
        e = __fmaf_rn(l, t.x, e);
        h = __fadd_rn(p, e);
        l = __fsub_rn(e, __fsub_rn(h, p));
    }
}

// ----------------------------------------------------------------------------- coefficient ops

template <typename T> struct Coef;

template <> struct Coef<double> {
    __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    // cs*c + phi*(sn*c2): exactly the oracle's two contributions, no fused multiply-add
    __device__ static __forceinline__ double rot(double cs, double c, double sn, double c2, int phi) {
        double t = __dmul_rn(sn, c2);
        return __dadd_rn(__dmul_rn(cs, c), phi > 0 ? t : -t);
    }
    __device__ static __forceinline__ bool small(double c, double eps) {
        // |c| < eps or c == 0 by the IEEE ordering of magnitudes
        uint64_t m = (uint64_t)__double_as_longlong(c) & 0x7fffffffffffffffULL;
        uint64_t e = (uint64_t)__double_as_longlong(eps) & 0x7fffffffffffffffULL;
        return m == 0 || m < e;
    }
};

template <> struct Coef<float> {
    __device__ static __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    // Compensated cs*c + phi*sn*c2: error-free products (FMA residuals) and an
    // error-free sum, folded into one final rounding (Ogita-Rump-Oishi Dot2).
    __device__ static __forceinline__ float rot(float cs, float c, float sn, float c2, int phi) {
        float p1 = __fmul_rn(cs, c);
        float e1 = __fmaf_rn(cs, c, -p1);
        float s2 = phi > 0 ? sn : -sn;
        float p2 = __fmul_rn(s2, c2);
        float e2 = __fmaf_rn(s2, c2, -p2);
        float s = __fadd_rn(p1, p2);
        float bp = __fsub_rn(s, p1);
        float e3 = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bp)), __fsub_rn(p2, bp));
        return __fadd_rn(s, __fadd_rn(e3, __fadd_rn(e1, e2)));
    }
    __device__ static __forceinline__ bool small(float c, float eps) {
        uint32_t m = (uint32_t)__float_as_uint(c) & 0x7fffffffu;
        uint32_t e = (uint32_t)__float_as_uint(eps) & 0x7fffffffu;
        return m == 0 || m < e;
    }
};

// c times the noise factor of exponent S.  FP64 form: the FP64 factor, one
// rounding.  FP32 form: c * (h + l) as one FMA over the float pair, c * l rounded
// first (its error is below 2^-48 of the result), so the coefficient is rounded
// once, to within ~2^-44 of c times the exact factor.
template <typename T> __device__ T noise_scale(const NoiseDesc& nz, T c, int64_t S);
template <> __device__ __forceinline__ double noise_scale<double>(const NoiseDesc& nz, double c, int64_t S) {
    return __dmul_rn(c, noise_factor(nz, S));
}
template <> __device__ __forceinline__ float noise_scale<float>(const NoiseDesc& nz, float c, int64_t S) {
    float h, l;
    noise_factor_pair(nz, S, h, l);
    return __fmaf_rn(c, h, __fmul_rn(c, l));
}

// The exact expectation sum: every diagonal coefficient becomes trunc(v * 2^80)
// as a 128-bit integer and the integers are added.  Coefficients must be finite
// with |v| < 2^32 (FIX80_LIMIT); a partial sum that met any other value is the
// sentinel FIX80_INVALID, and the result is then NaN.  With the sum of |v|
// below 2^46 no partial sum can reach the sentinel or wrap around.
constexpr double FIX80_LIMIT = 4294967296.0;
#define FIX80_INVALID ((__int128)(((unsigned __int128)1) << 127))

__host__ __device__ inline bool fix80_valid(double v) { return v > -FIX80_LIMIT && v < FIX80_LIMIT; }

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

// A 128-bit fixed-point total (units of 2^-80) rounded once to the nearest
// double (ties to even), in integer arithmetic; FIX80_INVALID gives NaN.  The
// host and the device use this one routine, so pp_expect and
// pp_expect_noalloc return the same bits.
__host__ __device__ inline double fixed80_to_double(__int128 tot) {
    if (tot == FIX80_INVALID) return __longlong_as_double_hd(0x7ff8000000000000LL);
    const bool neg = tot < 0;
    const unsigned __int128 mag = neg ? (unsigned __int128)0 - (unsigned __int128)tot : (unsigned __int128)tot;
    if (mag == 0) return 0.0;
    const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
    const int top = hi ? 127 - clz64_hd(hi) : 63 - clz64_hd(lo);   // highest set bit
    uint64_t m;
    int e = 0;   // the value is m * 2^(e - 80), m < 2^53
    if (top <= 52) {
        m = lo;
    } else {
        e = top - 52;
        m = (uint64_t)(mag >> e);
        const unsigned __int128 rem = mag & ((((unsigned __int128)1) << e) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (e - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m == (1ull << 53)) {
                m >>= 1;
                ++e;
            }
        }
    }
    // m < 2^53 is exact in a double; scaling by a power of two is exact
    const double v = ldexp((double)m, e - 80);
    return neg ? -v : v;
}

}  // namespace pp
