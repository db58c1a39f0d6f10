// Tier 0 of the sub-layer processor: one warp per bucket.
//
// Most buckets hold a few dozen to a few hundred strings.  Giving each such
// bucket to one warp, with its own slice of shared memory, removes every
// CTA-wide barrier from the gate rounds: a round needs only __syncwarp, list
// appends and new-entry indices come from warp votes (no shared-memory
// atomics on counters), and the ~20 warps resident on an SM work on
// independent buckets, hiding each other's latencies.  The arithmetic and the
// per-gate semantics are those of process_bucket (pp_kernels.cuh); buckets that
// do not fit a warp tile are passed to the CTA tiers.
#pragma once

#include "pp_kernels.cuh"

namespace pp {

constexpr int WARP_TILE_WARPS = 4;   // warps per CTA; each owns its buckets

template <int W, typename T>
__host__ __device__ constexpr size_t warp_tile_bytes(size_t cap) {
    return (tile_layout_bytes<W, T, int16_t>(cap) + 15) & ~(size_t)15;
}

// Per-warp accumulators folded into the CTA's at the end of a bucket.
struct WarpAcc {
    unsigned long long prologue, loaded, emitted;
};

// Work count (the canonical gate-by-gate number of live strings entering each
// gate), kept per lifetime: a string live from listed gate b through listed
// gate d (inclusive) contributes d - b + 1.  A lane adds g + 1 when a string
// dies at gate g, subtracts g + 1 when one is born (created or revived) at
// gate g, and adds the sub-layer's gate count for every string alive at the
// end; strings of the input count from gate 0.

template <int W, typename T>
__device__ bool warp_bucket(const Tile<W, T, int16_t>& t, const GateTab<W, T>& tab, const ActDesc& ad,
                            const ActDesc& adn, const StepParams& p, uint32_t b, WarpAcc& acc,
                            unsigned long long& upd_total) {
    const SubLayerDesc& d = *p.desc;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const T eps = eps_of<T>(p);
    const int n_in = (int)p.sfill[b];
    if (n_in > (int)p.max_load) {
        if (lane == 0) *t.flag = (int)FAIL_LOAD;
        return false;
    }
    long long clk0 = p.phase ? clock64() : 0, clk1 = 0;
    auto phase_mark = [&](int ph) {
        if (p.phase) {
            clk1 = clock64();
            if (lane == 0) atomicAdd(&p.phase[ph], (unsigned long long)(clk1 - clk0));
            clk0 = clk1;
        }
    };
    for (int i = lane; i < t.hcap; i += 32) t.hash[i] = (int16_t)-1;
    if (lane == 0) *t.flag = 0;
    long long upd = 0;   // this lane's share of the bucket's work count
    __syncwarp();

    // ---- load: the bucket's region, then its overflow strings, copied into
    // the tile asynchronously (every lane's copies in flight at once), then
    // entered into the hash table
    const size_t base = (size_t)b * p.sC;
    const size_t obase = ((uint64_t)n_in > p.sC) ? (size_t)p.soff[b] : 0;
    for (int i = lane; i < n_in; i += 32) {
        const bool reg = (uint64_t)i < p.sC;
        const size_t src = reg ? base + i : obase + (i - p.sC);
        const uint64_t* ax = reg ? p.sx : p.spx;
        const uint64_t* az = reg ? p.sz : p.spz;
        const size_t acap = reg ? p.scap : p.spcap;
        if (PP_OOB(src < acap && i < t.cap, 1, p.counters)) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            cp_async8(&t.x[(size_t)w * t.cap + i], &ax[(size_t)w * acap + src]);
            cp_async8(&t.z[(size_t)w * t.cap + i], &az[(size_t)w * acap + src]);
        }
        cp_async_coef(&t.c[i], static_cast<const T*>(reg ? p.sc : p.spc) + src);
        t.sr[i] = 0;
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    for (int i = lane; i < n_in; i += 32) {
        uint64_t x[W], z[W];
        tile_key<W, T, int16_t>(t, i, x, z);
        tile_insert<W, T, int16_t>(t, i, x, z, d.first != 0);
    }
    __syncwarp();
    phase_mark(0);

    // ---- prologue: truncation of the merged input, noise map, gate masks
    int na = 0, live = 0;
    for (int i0 = 0; i0 < n_in; i0 += 32) {
        const int i = i0 + lane;
        bool alive = false, has_gates = false;
        if (i < n_in) {
            T c = t.c[i];
            uint64_t x[W], z[W];
            tile_key<W, T, int16_t>(t, i, x, z);
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
                alive = true;
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
        live += __popc(__ballot_sync(FULL, alive));
        const unsigned am = __ballot_sync(FULL, has_gates);
        if (has_gates && !PP_OOB(na + __popc(am & lt) < t.cap, 3, p.counters))
            t.act[na + __popc(am & lt)] = (int16_t)i;
        na += __popc(am);
    }
    __syncwarp();
    if (*(volatile int*)t.flag) return false;
    phase_mark(1);

    // ---- gate rounds (see process_bucket): one pass per round.  Round r reads
    // coefficients from buffer r & 1 and writes them to the other buffer, so a
    // string and its partner both read the pair's values from before the gate;
    // truncation, the work count and the next round's list are settled in the
    // same pass.  New-entry indices and list slots come from warp votes.
    int n = n_in;
    const bool tr = p.phase != nullptr;
    unsigned st_rounds = 0, st_chunks = 0, st_listed = 0, st_pairs = 0, st_new = 0, st_rev = 0;
    for (int r = 0; r <= 64 * W && na > 0; ++r) {
        if (tr) {
            ++st_rounds;
            st_chunks += (na + 31) >> 5;
            st_listed += na;
        }
        const int16_t* L = t.act + (size_t)(r & 1) * t.cap;
        int16_t* Ln = t.act + (size_t)((r & 1) ^ 1) * t.cap;
        const T* ccur = t.cbuf(r & 1);
        T* cnxt = t.cbuf((r & 1) ^ 1);
        const uint8_t stamp = (uint8_t)(r + 1);
        int nn = 0;
        bool over = false;
        for (int k0 = 0; k0 < na; k0 += 32) {
            const int k = k0 + lane;
            bool create = false, revive = false, keep = false;
            int i = 0, j = -1;
            uint32_t hslot = 0;
            T v = T(0);
            uint64_t qx[W], qz[W], gm[W];
            if (k < na) {
                i = (int)L[k];
                uint64_t x[W], z[W];
                tile_key<W, T, int16_t>(t, i, x, z);
                int gg = -1;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    gm[w] = t.g[(size_t)w * t.cap + i];
                    if (gg < 0 && gm[w]) {
                        gg = 64 * w + __ffsll((long long)gm[w]) - 1;
                        gm[w] &= gm[w] - 1;
                    }
                }
                if (PP_OOB(gg >= 0, 4, p.counters)) gg = 0;
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
                if (reach) j = tile_lookup_at<W, T, int16_t>(t, qx, qz, &hslot);
                if (PP_OOB(j < n, 2, p.counters)) j = -1;
                // i R P = phi Q: sign of P's sin-branch into its partner Q
                const int phi = branch_negative<W, T>(tab, gg, x, z) ? -1 : 1;
                const T cs = tab.cs[gg], sn = tab.sn[gg];
                const T c = ccur[i];
                T c2 = T(0);
                if (j >= 0) {
                    // the partner's value before this gate: it is live and in
                    // this round's list (stamp r, or r + 1 once its own lane has
                    // written), or dead
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
                if (create || revive) upd -= gg + 1;
                if (tr) {
                    st_pairs += c2 != T(0);
                    st_new += create;
                    st_rev += revive;
                }
            }
            const unsigned cm = __ballot_sync(FULL, create);
            int idx = j;
            if (create) {
                idx = n + __popc(cm & lt);
                if (idx >= t.cap) {
                    over = true;
                    create = false;
                }
            }
            n += __popc(cm);
            bool join = false;
            if (create || revive) {
                // a new string, or one truncated earlier revived: it joins the
                // orbit with the gates the orbit has left
                if (create) {
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        t.x[(size_t)w * t.cap + idx] = qx[w];
                        t.z[(size_t)w * t.cap + idx] = qz[w];
                    }
                }
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
                    tile_insert_at<W, T, int16_t>(t, idx, hslot);
                }
                join = more;
            }
            const unsigned km = __ballot_sync(FULL, keep);
            const unsigned jm = __ballot_sync(FULL, join);
            if (keep && !PP_OOB(nn + __popc(km & lt) < t.cap, 3, p.counters)) Ln[nn + __popc(km & lt)] = (int16_t)i;
            nn += __popc(km);
            if (join && !PP_OOB(nn + __popc(jm & lt) < t.cap, 3, p.counters)) Ln[nn + __popc(jm & lt)] = (int16_t)idx;
            nn += __popc(jm);
        }
        __syncwarp();
        const bool any_over = __any_sync(FULL, over);
        if (any_over || *(volatile int*)t.flag) {
            if (lane == 0) *t.flag = any_over ? (int)FAIL_POOL : (int)FAIL_HASH;
            return false;
        }
        na = nn;
    }

    phase_mark(2);
    if (p.phase) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_pairs += __shfl_xor_sync(FULL, st_pairs, o);
            st_new += __shfl_xor_sync(FULL, st_new, o);
            st_rev += __shfl_xor_sync(FULL, st_rev, o);
        }
        if (lane == 0) {
            unsigned long long* q = p.phase + (CTR_STAT - CTR_PHASE);
            atomicAdd(q + 0, 1ull);
            atomicAdd(q + 1, (unsigned long long)st_rounds);
            atomicAdd(q + 2, (unsigned long long)st_chunks);
            atomicAdd(q + 3, (unsigned long long)st_listed);
            atomicAdd(q + 4, (unsigned long long)st_pairs);
            atomicAdd(q + 5, (unsigned long long)st_new);
            atomicAdd(q + 6, (unsigned long long)st_rev);
        }
    }

    // ---- output
    unsigned long long emitted = 0;
    if (d.final_) {
        int cnt = 0;
        for (int i = lane; i < n; i += 32) cnt += tile_coef(t, i) != T(0);
        upd += (long long)cnt * d.n_gates;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
        unsigned long long pos = 0;
        if (lane == 0 && cnt) pos = atomicAdd(&p.counters[CTR_OUT], (unsigned long long)cnt);
        pos = __shfl_sync(FULL, pos, 0);
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const T ci = i < n ? tile_coef(t, i) : T(0);
            const bool lv = ci != T(0);
            const unsigned lm = __ballot_sync(FULL, lv);
            if (lv) {
                const unsigned long long q = pos + __popc(lm & lt);
                if (q < p.dcap) {
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        p.dx[(size_t)w * p.dcap + q] = t.x[(size_t)w * t.cap + i];
                        p.dz[(size_t)w * p.dcap + q] = t.z[(size_t)w * t.cap + i];
                    }
                    static_cast<T*>(p.dc)[q] = ci;
                } else {
                    atomicAdd(&p.counters[CTR_ERR_REGION], 1ull);
                }
            }
            pos += __popc(lm);
        }
        emitted = (unsigned long long)cnt;
    } else {
        int cnt = emit_tile<1, W, T, int16_t>(t, adn, p, lane, 32, n);
        upd += (long long)cnt * d.n_gates;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
        emitted = (unsigned long long)cnt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) upd += __shfl_xor_sync(FULL, upd, o);
    phase_mark(3);
    acc.prologue += (unsigned long long)live;
    acc.loaded += (unsigned long long)n_in;
    acc.emitted += emitted;
    upd_total += (unsigned long long)upd;
    return true;
}

#ifndef PP_WARP_MIN_BLOCKS
#define PP_WARP_MIN_BLOCKS 5   // resident CTAs per SM the register budget is sized for
#endif
template <int W, typename T, int NW>
__global__ void __launch_bounds__(32 * NW, PP_WARP_MIN_BLOCKS) k_process_warp(const StepParams p0, const StepParams* ps,
                                                                             int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GateTab<W, T> tab;
    __shared__ int s_ctl[NW][8];
    __shared__ unsigned long long s_acc[3];
    __shared__ ActDesc s_ad, s_adn;
    __shared__ StepParams p;
    if (!load_params(p, p0, ps)) return;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 3) s_acc[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) make_act(*p.desc, s_ad);
    if (threadIdx.x == (NW > 1 ? 32 : 0) && p.next) make_act(*p.next, s_adn);
    load_gate_table<W, T>(tab, *p.desc);
    __syncthreads();

    Tile<W, T, int16_t> t = carve_tile<W, T, int16_t>(smem + warp_tile_bytes<W, T>(cap) * wid, cap, s_ctl[wid]);
    t.ctr = p.counters;
    WarpAcc acc{0ull, 0ull, 0ull};
    unsigned long long upd = 0;
    const uint32_t n_items = work_items(p);
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = (uint32_t)atomicAdd(&p.counters[p.work_ctr], 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n_items) break;
        const uint32_t b = p.in_list ? p.in_list[k] : k;
        if (p.sfill[b] == 0) continue;
        if (!warp_bucket<W, T>(t, tab, s_ad, s_adn, p, b, acc, upd) && lane == 0) {
            atomicAdd(&p.counters[CTR_FAIL + (*t.flag - 1)], 1ull);
            unsigned long long j = atomicAdd(&p.counters[p.defer_ctr], 1ull);
            p.out_list[j] = b;
        }
        __syncwarp();
    }
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
            if (!p.desc->final_) atomicAdd(&p.counters[CTR_OUT], s_acc[2]);
        }
    }
}

}  // namespace pp
