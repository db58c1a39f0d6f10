// Kernels on the propagation result: the last step of the exact expectation
// reduction, and the sort that orders O~'s strings by key for export.
//
// Export order (Sec. II, the observable is handed out as a list of strings):
// ascending by (x[W-1], ..., x[0], z[W-1], ..., z[0]) as unsigned words.  The
// sort is a least-significant-digit radix sort with 8-bit digits over the
// 2W key words, least significant first (z[0] ... z[W-1], then x[0] ...
// x[W-1]); each pass is stable, so the passes compose.  Digits that are equal
// in every key (high bits above the qubit count, constant Z words) are found in
// one pre-pass and skipped.  A pass is three steps: per-tile digit counts,
// an exclusive scan over (digit, tile), and a stable scatter in which each
// tile ranks its items by digit with warp match votes and per-warp counts.
#pragma once

#include "pp_device.cuh"

namespace pp {

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ROUNDS = 8;                             // items per thread per tile
constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;     // 2048 items per tile
constexpr int SORT_RADIX = 256;
constexpr int SCAN_CHUNK = SORT_THREADS * SORT_ROUNDS;    // elements per block of the scan
static_assert(SORT_THREADS == SORT_RADIX, "one thread per digit value in the histogram and scatter kernels");
static_assert(SORT_WARPS <= 32, "the warp offsets of a block scan fit one warp");

// One block folds the per-block partials of k_expect into partial[n].
__global__ void k_expect_final(__int128* partial, int n) {
    __shared__ __int128 s[256];
    __int128 acc = 0;
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const __int128 v = partial[i];
        if (v == FIX80_INVALID) bad = true;
        else acc += v;
    }
    s[threadIdx.x] = acc;
    bad = __syncthreads_or(bad);
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[n] = bad ? FIX80_INVALID : s[0];
}

// Key word kw in significance order: z[0..W-1], then x[0..W-1].
template <int W>
__device__ __forceinline__ uint64_t sort_word(const uint64_t* x, const uint64_t* z, uint64_t cap, uint64_t i,
                                              int kw) {
    return kw < W ? z[(size_t)kw * cap + i] : x[(size_t)(kw - W) * cap + i];
}

// varying[kw] |= word ^ word-of-item-0, over all items: the bits in which
// some key differs from the first.
template <int W>
__global__ void k_sort_varying(const uint64_t* x, const uint64_t* z, uint64_t cap, uint64_t n,
                               unsigned long long* varying) {
    uint64_t v[2 * W], k0[2 * W];
#pragma unroll
    for (int kw = 0; kw < 2 * W; ++kw) {
        v[kw] = 0ull;
        k0[kw] = sort_word<W>(x, z, cap, 0, kw);
    }
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int kw = 0; kw < 2 * W; ++kw) v[kw] |= sort_word<W>(x, z, cap, i, kw) ^ k0[kw];
    }
#pragma unroll
    for (int kw = 0; kw < 2 * W; ++kw) {
        uint64_t a = v[kw];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a |= __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0 && a) atomicOr(&varying[kw], (unsigned long long)a);
    }
}

// counts[d * n_tiles + tile] = items of the tile whose digit is d.
template <int W>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const uint64_t* x, const uint64_t* z, uint64_t cap,
                                                            uint64_t n, int kw, int shift, uint32_t* counts,
                                                            uint32_t n_tiles) {
    __shared__ uint32_t h[SORT_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const uint64_t i = t0 + (uint64_t)r * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(sort_word<W>(x, z, cap, i, kw) >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of one block's chunk of v (in place); the chunk total goes to
// sums[block].
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < SORT_WARPS ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SORT_WARPS) s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == SORT_WARPS - 1) *total = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[wid] + incl - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SORT_THREADS) k_scan_chunks(uint32_t* v, uint64_t len, uint32_t* sums) {
    __shared__ uint32_t s_warp[SORT_WARPS];
    __shared__ uint32_t s_total;
    // each thread owns SORT_ROUNDS consecutive elements
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK + (uint64_t)threadIdx.x * SORT_ROUNDS;
    uint32_t e[SORT_ROUNDS];
    uint32_t own = 0;
#pragma unroll
    for (int k = 0; k < SORT_ROUNDS; ++k) {
        e[k] = base + k < len ? v[base + k] : 0u;
        own += e[k];
    }
    uint32_t run = block_exclusive_scan(own, s_warp, &s_total);
#pragma unroll
    for (int k = 0; k < SORT_ROUNDS; ++k) {
        if (base + k < len) v[base + k] = run;
        run += e[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

// One block: exclusive scan of the chunk totals, in place.
__global__ void __launch_bounds__(SORT_THREADS) k_scan_sums(uint32_t* sums, uint32_t n) {
    __shared__ uint32_t s_warp[SORT_WARPS];
    __shared__ uint32_t s_total;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < n; c0 += SORT_THREADS) {
        const uint32_t i = c0 + threadIdx.x;
        const uint32_t x = i < n ? sums[i] : 0u;
        const uint32_t r = block_exclusive_scan(x, s_warp, &s_total);
        if (i < n) sums[i] = carry + r;
        carry += s_total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_scan_add(uint32_t* v, uint64_t len, const uint32_t* sums) {
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK + (uint64_t)threadIdx.x * SORT_ROUNDS;
    const uint32_t add = sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SORT_ROUNDS; ++k)
        if (base + k < len) v[base + k] += add;
}

// Stable scatter of one digit pass.  Round r of a tile takes items
// tile_start + r * SORT_THREADS + thread, so item order is (round, warp, lane);
// an item's place among its tile's items of the same digit is the count in
// earlier rounds, plus the count in lower warps of this round, plus the count
// in lower lanes of its own warp.
template <int W, typename T>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(
    const uint64_t* x, const uint64_t* z, const T* c, uint64_t cap_in, uint64_t n, int kw, int shift,
    const uint32_t* offs, uint32_t n_tiles, uint64_t* xo, uint64_t* zo, T* co, uint64_t cap_out) {
    __shared__ uint32_t s_base[SORT_RADIX];
    __shared__ uint32_t s_wcnt[SORT_WARPS][SORT_RADIX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    s_base[threadIdx.x] = offs[(size_t)threadIdx.x * n_tiles + blockIdx.x];
    for (int w = 0; w < SORT_WARPS; ++w) s_wcnt[w][threadIdx.x] = 0u;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const uint64_t i = t0 + (uint64_t)r * SORT_THREADS + threadIdx.x;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)(sort_word<W>(x, z, cap_in, i, kw) >> shift) & 0xffu : SORT_RADIX;
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const bool leader = lane == __ffs(same) - 1;
        if (valid && leader) s_wcnt[wid][d] = (uint32_t)__popc(same);
        __syncthreads();
        uint32_t pos = 0;
        if (valid) {
            pos = s_base[d] + (uint32_t)__popc(same & lt);
            for (int w = 0; w < wid; ++w) pos += s_wcnt[w][d];
        }
        uint32_t tot = 0;
        for (int w = 0; w < SORT_WARPS; ++w) tot += s_wcnt[w][threadIdx.x];
        __syncthreads();
        s_base[threadIdx.x] += tot;
        if (valid && leader) s_wcnt[wid][d] = 0u;
        if (valid) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                xo[(size_t)w * cap_out + pos] = x[(size_t)w * cap_in + i];
                zo[(size_t)w * cap_out + pos] = z[(size_t)w * cap_in + i];
            }
            co[pos] = c[i];
        }
        __syncthreads();
    }
}

}  // namespace pp
