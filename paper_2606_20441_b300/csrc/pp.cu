// libpp host side: the C ABI of include/pp.h, circuit planning into fused
// sub-layers, noise tables, the per-sub-layer launch sequence, capacity
// management, expectation and export.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <memory>
#include <tuple>
#include <thread>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pp.h"
#include "pp_kernels.cuh"
#include "pp_warp.cuh"
#include "pp_orbit.cuh"
#include "pp_topk.cuh"
#include "pp_result.cuh"

using namespace pp;

// NVTX ranges around each sub-layer's launches (visible in Nsight timelines).
#define PP_RANGE_PUSH(name) nvtxRangePushA(name)
#define PP_RANGE_POP() nvtxRangePop()

namespace {

// Processing tiers: a bucket goes to the first tier whose tile holds it.  Small
// CTAs first, many per SM, so that one CTA's per-round barriers overlap other
// CTAs' work; then larger shared-memory tiles; then a global-memory tile.
struct TierCfg {
    int threads;
    int cap1;     // tile entries for W = 1
    int cap2;     // tile entries for W = 2
    int load;     // largest bucket taken, in 1/100 of the tile: the rest of the tile
                  // holds the strings the gates create (a bucket that outgrows it
                  // anyway is passed on, its work lost)
};
#ifndef PP_CTA_TILE1_THREADS
#define PP_CTA_TILE1_THREADS 64
#endif
constexpr int WARP_TILE_WARPS2 = 2;   // warps per CTA of the second warp tier
#ifndef PP_CTA_TILE2_THREADS
#define PP_CTA_TILE2_THREADS 256
#endif
constexpr TierCfg kTiers[N_TIERS] = {
    {32 * WARP_TILE_WARPS, 248, 248, 60},   // one warp per bucket, 4 warps per CTA
    {32 * WARP_TILE_WARPS2, 512, 384, 60},  // one warp per bucket, larger tiles, 2 warps per CTA
    {PP_CTA_TILE1_THREADS, 1024, 1024, 75},     // CTA tiles: few warps, so that a round's
    {PP_CTA_TILE2_THREADS, 4096, 2048, 75},     // barriers wait on few warps
    {512, 1 << 20, 1 << 20, 75}};           // global-memory tile
constexpr int kGlobalTier = N_TIERS - 1;
constexpr int kFallbackCTAs = 16; // CTAs of the global tier
constexpr int kFallbackCap = 1 << 20;
constexpr size_t kMinCap = 4096;        // smallest capacity (terms per arena)
constexpr size_t kInitialCap = 1 << 16;  // first capacity of a handle without a fixed one

struct NoiseHost {
    int mode = 0;
    int n = 0;                        // sites
    std::vector<int64_t> grp;         // [(n+3)/4][256] group tables (NoiseDesc::grp)
    std::vector<int32_t> shift;       // [n_shift]
    std::vector<uint64_t> xmask;      // [n_shift][W] first sites of pairs that cross groups
    std::vector<int32_t> pidx;        // [n_shift][n]
    std::vector<int64_t> c2;          // [P][16]
    std::vector<uint64_t> gx, gz;
    std::vector<int64_t> glam;
    std::vector<double> etab;         // [8][256] exp(+-2 b 2^(8i-56))
    std::vector<float> ftab;          // [8][256][2] the same as float (head, tail) pairs
    // device copies
    double* d_etab = nullptr;
    float* d_ftab = nullptr;
    int64_t* d_grp = nullptr;
    int32_t* d_shift = nullptr;
    uint64_t* d_xmask = nullptr;
    int32_t* d_pidx = nullptr;
    int64_t* d_c2 = nullptr;
    uint64_t* d_gx = nullptr;
    uint64_t* d_gz = nullptr;
    int64_t* d_glam = nullptr;
};

struct Arena {
    uint64_t* x = nullptr;
    uint64_t* z = nullptr;
    void* c = nullptr;
};

}  // namespace

struct pp_handle {
    pp_options opt;
    pp_tuning tune{0, 0.0, 0, 0, {0, 0, 0, 0}};   // zeros select the library defaults
    int n = 0, W = 1;
    cudaStream_t st = nullptr;
    std::string err;
    int sm_count = 0;
    size_t smem_optin = 0;           // largest dynamic shared memory a CTA may opt into
    int device = 0;

    // circuit
    bool have_circuit = false;
    int n_layers = 0;
    std::vector<uint64_t> gx, gz;
    std::vector<double> theta;
    std::vector<int32_t> layer_of;
    std::map<int, NoiseHost> noise;
    std::vector<SubLayerDesc> subs;
    std::vector<int> sub_kind;     // growth-estimate class of each sub-layer
    SubLayerDesc* d_subs = nullptr;    // inside the table arena
    bool subs_dirty = true;
    unsigned char* tab_dev = nullptr;  // table arena: descriptors and noise tables
    size_t tab_cap = 0;
    std::vector<unsigned char> tab_host;

    // memory
    size_t cap = 0;                // terms per arena
    Arena arena[2];
    uint32_t* fill[2] = {nullptr, nullptr};
    uint32_t fill_cap = 0;
    unsigned long long* counters = nullptr;
    uint32_t* pass_list[N_TIERS - 1] = {};   // buckets passed tier t -> t+1
    size_t spill_cap = 0;          // overflow strings per layout
    Arena spill_raw, spill_grp;
    uint32_t* spill_b = nullptr;
    uint32_t* spill_s = nullptr;
    unsigned long long* spill_ctr = nullptr;   // [NSPILL]
    uint64_t* soff[2] = {nullptr, nullptr};
    unsigned char* fb_scratch = nullptr;   // global-tier tiles, allocated on first use
    size_t fb_slice = 0;
    int fb_cap = 0;                        // strings per global-tier tile
    uint64_t* stage = nullptr;     // input staging
    size_t stage_cap = 0;
    __int128* partial = nullptr;   // [4096] per-block partial sums, then the total
    unsigned char* sort_scratch = nullptr;   // export sort: digit counts and scan sums
    size_t sort_scratch_bytes = 0;
    std::vector<void*> owned;

    bool mem_ready = false;        // every work buffer below is allocated
    int growths = 0;               // capacity growths of the running propagation
    std::atomic<long long> run_gen{0};       // generation of the running (or last) propagation
    std::atomic<long long> cancel_gen{-1};   // generation pp_cancel asked to stop

    // per-tier device times (pp_options.timing): one event pair per tier,
    // reused every sub-layer
    bool timing = false;
    cudaEvent_t tier_ev[N_TIERS][2] = {};

    // top-K truncation (0: off) and its device state
    size_t top_k = 0;
    TopKState* topk_state = nullptr;

    // result
    bool have_result = false;
    int res_side = 0;
    size_t n_res = 0;
    pp_stats stats{};
};

namespace {

pp_status fail(pp_handle* h, pp_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, PP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

void* dev_alloc(pp_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->opt.alloc) {
        p = h->opt.alloc(bytes, h->opt.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->owned.push_back(p);
    return p;
}

void dev_free(pp_handle* h, void* p) {
    if (!p) return;
    auto it = std::find(h->owned.begin(), h->owned.end(), p);
    if (it != h->owned.end()) h->owned.erase(it);
    if (h->opt.free) h->opt.free(p, h->opt.alloc_ctx);
    else cudaFree(p);
}

inline int popc_words(const uint64_t* v, int W) {
    int s = 0;
    for (int w = 0; w < W; ++w) s += __builtin_popcountll(v[w]);
    return s;
}

inline int bit(const uint64_t* v, int q) { return (int)((v[q >> 6] >> (q & 63)) & 1ull); }

void trig(double theta, double* c, double* s) {
    *c = std::cos(theta);
    *s = std::sin(theta);
    if (std::fabs(*c) < 1e-15) { *c = 0.0; *s = (*s > 0) ? 1.0 : -1.0; }
    if (std::fabs(*s) < 1e-15) { *s = 0.0; *c = (*c > 0) ? 1.0 : -1.0; }
}

// Gate signature for grouping into sub-layers.
struct GateSig {
    int cls;      // CLS_LOCAL1 / CLS_LOCAL2 / CLS_GENERIC
    int ax, az, bx, bz, shift;
    int slot;     // first site
    bool same(const GateSig& o) const {
        return cls == o.cls && ax == o.ax && az == o.az && bx == o.bx && bz == o.bz && shift == o.shift;
    }
};

GateSig classify(const uint64_t* rx, const uint64_t* rz, int n, int W) {
    GateSig g{CLS_GENERIC, 0, 0, 0, 0, 0, -1};
    uint64_t sup[MAXW] = {0, 0};
    for (int w = 0; w < W; ++w) sup[w] = rx[w] | rz[w];
    int wt = popc_words(sup, W);
    std::vector<int> sites;
    for (int q = 0; q < n; ++q)
        if (bit(sup, q)) sites.push_back(q);
    if (wt == 1) {
        g.cls = CLS_LOCAL1;
        g.slot = sites[0];
        g.ax = bit(rx, sites[0]);
        g.az = bit(rz, sites[0]);
    } else if (wt == 2) {
        g.cls = CLS_LOCAL2;
        g.slot = sites[0];
        g.ax = bit(rx, sites[0]);
        g.az = bit(rz, sites[0]);
        g.bx = bit(rx, sites[1]);
        g.bz = bit(rz, sites[1]);
        g.shift = sites[1] - sites[0];
    }
    return g;
}

int sig_kind(const SubLayerDesc& d) {
    if (d.cls == CLS_LOCAL1) return 1 + 4 * (d.ax + 2 * d.az);
    if (d.cls == CLS_LOCAL2) return 2 + 4 * (d.ax + 2 * d.az + 4 * (d.bx + 2 * d.bz) + 16 * d.shift);
    return d.cls;
}

// Gates fused into one sub-layer.  An orbit of a sub-layer can hold up to
// 2^(acting gates) strings, so smaller sub-layers keep orbits small enough for
// the one-warp tiles at the price of more passes over the strings.
int max_fused_gates(const pp_handle* h) {
    // default: whole layers (up to 64 gates per mask word), the measured best on
    // the 7x8 TFIM workload (three passes per Trotter step instead of six)
    int m = h->tune.max_fused_gates > 0 ? h->tune.max_fused_gates : 64 * h->W;
    if (const char* e = getenv("PP_MAX_FUSED_GATES")) m = atoi(e);
    return std::max(1, std::min(m, 64 * h->W));
}

double bucket_headroom(const pp_handle* h) {
    return h->tune.bucket_headroom > 0.0 ? h->tune.bucket_headroom : 2.0;
}

// Marks class sub-layers as orbit sub-layers and fills their letter table:
// for the letters (la on a, lb on a + shift) of the orbit member whose
// coordinate bit is 0 (x on a if the gate has an X part there, else z), the
// sign of its sin-branch into its partner (i R P = phi P', Sec. I Eq.
// evolve_gate) and the change of Pauli weight on the gate's sites.
void set_orbit_table(SubLayerDesc& d) {
    d.orb = (d.cls == CLS_NONE) || ((d.cls == CLS_LOCAL1 || d.cls == CLS_LOCAL2) && d.nseg == 1);
    std::memset(d.ltab, 0xff, sizeof(d.ltab));
    // listed index == slot: generic sub-layers, and class sub-layers whose
    // slots form one ascending run 0, 1, ..., n_gates - 1
    d.ident = d.cls == CLS_GENERIC || d.cls == CLS_NONE;
    if ((d.cls == CLS_LOCAL1 || d.cls == CLS_LOCAL2) && d.nseg == 1) {
        bool ok = true;
        for (int g = 0; g < d.n_gates && ok; ++g) ok = d.slot_of[g] == g;
        d.ident = ok;
    }
    d.psign = 0;
    if (d.cls != CLS_LOCAL1 && d.cls != CLS_LOCAL2) return;
    const int two = d.cls == CLS_LOCAL2;
    const int ra = d.ax + 2 * d.az, rb = two ? d.bx + 2 * d.bz : 0;
    auto anti = [](int l, int r) { return ((l & 1) & (r >> 1)) ^ ((l >> 1) & (r & 1)); };
    auto wt = [](int l) { return l != 0 ? 1 : 0; };
    // power of i contributed by one qubit of R * S (letter codes x + 2z)
    auto ph = [](int r, int s) {
        const int rx = r & 1, rz = r >> 1, sx = s & 1, sz = s >> 1;
        return rx * rz + sx * sz + 2 * rz * sx - ((rx ^ sx) & (rz ^ sz));
    };
    // the sign of any acting string's sin-branch, by its letters on the sites
    for (int la = 0; la < 4; ++la)
        for (int lb = 0; lb < (two ? 4 : 1); ++lb) {
            if (!(anti(la, ra) ^ anti(lb, rb))) continue;
            const int e = (ph(ra, la) + (two ? ph(rb, lb) : 0)) & 3;
            if (((1 + e) & 3) != 0) d.psign |= (uint16_t)(1u << (la + 4 * lb));
        }
    for (int la = 0; la < 4; ++la)
        for (int lb = 0; lb < (two ? 4 : 1); ++lb) {
            const int cbit = d.ax ? (la & 1) : (la >> 1);
            if (cbit || !(anti(la, ra) ^ anti(lb, rb))) continue;
            const int e = (ph(ra, la) + (two ? ph(rb, lb) : 0)) & 3;
            const int negphi = ((1 + e) & 3) == 0 ? 0 : 1;
            const int dw = wt(la ^ ra) - wt(la) + (two ? wt(lb ^ rb) - wt(lb) : 0);
            d.ltab[la + 4 * lb] = (uint8_t)(negphi | ((dw + 1) << 1));
        }
}

// Splits a layer's gates (listed order) into fused sub-layers.
void plan_layer(pp_handle* h, const std::vector<int>& gates, int noise_idx, int layer) {
    const int W = h->W, n = h->n;
    const int max_gates = max_fused_gates(h);
    std::vector<SubLayerDesc> out;
    SubLayerDesc cur;
    bool open = false;
    GateSig cur_sig{};
    int last_slot = -1;
    std::vector<bool> used(MAX_SITES, false);        // sites touched by the open sub-layer's gates
    std::vector<bool> first_used(MAX_SITES, false);  // first sites (slots) of its gates
    auto close = [&]() {
        if (open) out.push_back(cur);
        open = false;
    };
    auto start = [&](const GateSig& s) {
        std::memset(&cur, 0, sizeof(cur));
        cur.cls = s.cls;
        cur.ax = s.ax; cur.az = s.az; cur.bx = s.bx; cur.bz = s.bz; cur.shift = s.shift;
        cur.noise = -1;
        cur.nseg = 0;
        open = true;
        cur_sig = s;
        last_slot = -1;
        std::fill(used.begin(), used.end(), false);
        std::fill(first_used.begin(), first_used.end(), false);
    };
    for (int g : gates) {
        const uint64_t* rx = &h->gx[(size_t)g * W];
        const uint64_t* rz = &h->gz[(size_t)g * W];
        GateSig s = classify(rx, rz, n, W);
        double cs, sn;
        trig(h->theta[g], &cs, &sn);
        if (s.cls == CLS_GENERIC) {
            if (!(open && cur.cls == CLS_GENERIC && cur.n_gates < std::min(MAX_GEN, max_gates))) {
                close();
                start(s);
            }
            int j = cur.n_gates++;
            for (int w = 0; w < W; ++w) {
                cur.gx[j][w] = rx[w];
                cur.gz[j][w] = rz[w];
            }
            cur.cs[j] = cs;
            cur.sn[j] = sn;
            cur.order[j] = (int16_t)j;
            cur.slot_of[j] = (int16_t)j;
            continue;
        }
        // With orbit tiles, a class sub-layer is one ascending run of slots
        // whose gates have pairwise disjoint supports: its orbits are then
        // hypercubes with one coordinate bit per acting gate (pp_orbit.cuh).
        // Otherwise runs of the same signature fuse across up to MAX_SEG
        // ascending segments (e.g. both colours of horizontal R_ZZ edges).
        bool fits;
        if (h->tune.orbit_tiles) {
            const bool disjoint = !used[s.slot] && (s.cls != CLS_LOCAL2 || !used[s.slot + s.shift]);
            fits = open && cur.cls != CLS_GENERIC && cur_sig.same(s) && s.slot > last_slot && disjoint &&
                   cur.n_gates < max_gates;
        } else {
            fits = open && cur.cls != CLS_GENERIC && cur_sig.same(s) && !first_used[s.slot] &&
                   (s.slot > last_slot || cur.nseg < MAX_SEG) && cur.n_gates < max_gates;
        }
        if (!fits) {
            close();
            start(s);
        }
        if (s.slot <= last_slot || cur.nseg == 0) cur.nseg++;
        int sg = cur.nseg - 1;
        cur.seg[sg][s.slot >> 6] |= 1ull << (s.slot & 63);
        cur.all[s.slot >> 6] |= 1ull << (s.slot & 63);
        cur.cs[s.slot] = cs;
        cur.sn[s.slot] = sn;
        cur.order[s.slot] = (int16_t)cur.n_gates;
        cur.slot_of[cur.n_gates] = (int16_t)s.slot;
        cur.n_gates++;
        used[s.slot] = true;
        first_used[s.slot] = true;
        if (s.cls == CLS_LOCAL2) used[s.slot + s.shift] = true;
        last_slot = s.slot;
    }
    close();
    for (auto& d : out) set_orbit_table(d);
    if (out.empty() && noise_idx >= 0) {
        SubLayerDesc d;
        std::memset(&d, 0, sizeof(d));
        d.cls = CLS_NONE;
        d.noise = -1;
        set_orbit_table(d);
        out.push_back(d);
    }
    if (!out.empty()) out[0].noise = noise_idx;
    for (auto& d : out) {
        h->subs.push_back(d);
        h->sub_kind.push_back(sig_kind(d));
    }
    (void)layer;
}

// Copies the sub-layer descriptors and every noise map's tables into the
// handle's table arena, one host-to-device copy.  The arena only grows, so
// loading circuits and noise allocates and frees nothing on the device in the
// steady state (a device free would synchronise every stream on the GPU).
pp_status upload_tables(pp_handle* h) {
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    std::vector<std::pair<const void*, size_t>> parts;
    size_t off = 0;
    std::vector<size_t> offs;
    auto add = [&](const void* p, size_t bytes) {
        offs.push_back(off);
        parts.push_back({p, bytes});
        off = align(off + std::max<size_t>(bytes, 16));
    };
    add(h->subs.data(), sizeof(SubLayerDesc) * h->subs.size());
    for (auto& kv : h->noise) {
        NoiseHost& nh = kv.second;
        add(nh.grp.data(), nh.grp.size() * 8);
        add(nh.shift.data(), nh.shift.size() * 4);
        add(nh.xmask.data(), nh.xmask.size() * 8);
        add(nh.pidx.data(), nh.pidx.size() * 4);
        add(nh.c2.data(), nh.c2.size() * 8);
        add(nh.etab.data(), nh.etab.size() * 8);
        add(nh.ftab.data(), nh.ftab.size() * 4);
        add(nh.gx.data(), nh.gx.size() * 8);
        add(nh.gz.data(), nh.gz.size() * 8);
        add(nh.glam.data(), nh.glam.size() * 8);
    }
    if (off > h->tab_cap) {
        if (h->tab_dev) {
            cudaStreamSynchronize(h->st);
            dev_free(h, h->tab_dev);
            h->tab_dev = nullptr;
        }
        h->tab_cap = align(off + off / 2);
        h->tab_dev = static_cast<unsigned char*>(dev_alloc(h, h->tab_cap));
        if (!h->tab_dev) {
            h->tab_cap = 0;
            return fail(h, PP_ERR_NOMEM, "table arena allocation failed");
        }
    }
    h->tab_host.assign(off, 0);
    for (size_t k = 0; k < parts.size(); ++k)
        if (parts[k].second) std::memcpy(h->tab_host.data() + offs[k], parts[k].first, parts[k].second);
    CK(cudaMemcpyAsync(h->tab_dev, h->tab_host.data(), off, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    size_t k = 0;
    h->d_subs = reinterpret_cast<SubLayerDesc*>(h->tab_dev + offs[k++]);
    for (auto& kv : h->noise) {
        NoiseHost& nh = kv.second;
        nh.d_grp = reinterpret_cast<int64_t*>(h->tab_dev + offs[k++]);
        nh.d_shift = reinterpret_cast<int32_t*>(h->tab_dev + offs[k++]);
        nh.d_xmask = reinterpret_cast<uint64_t*>(h->tab_dev + offs[k++]);
        nh.d_pidx = reinterpret_cast<int32_t*>(h->tab_dev + offs[k++]);
        nh.d_c2 = reinterpret_cast<int64_t*>(h->tab_dev + offs[k++]);
        nh.d_etab = reinterpret_cast<double*>(h->tab_dev + offs[k++]);
        nh.d_ftab = reinterpret_cast<float*>(h->tab_dev + offs[k++]);
        nh.d_gx = reinterpret_cast<uint64_t*>(h->tab_dev + offs[k++]);
        nh.d_gz = reinterpret_cast<uint64_t*>(h->tab_dev + offs[k++]);
        nh.d_glam = reinterpret_cast<int64_t*>(h->tab_dev + offs[k++]);
    }
    h->subs_dirty = false;
    return PP_OK;
}

pp_status build_plan(pp_handle* h) {
    h->subs.clear();
    h->sub_kind.clear();
    std::vector<std::vector<int>> by_layer(h->n_layers);
    for (size_t g = 0; g < h->theta.size(); ++g) by_layer[h->layer_of[g]].push_back((int)g);
    if (h->top_k > 0) {
        // the input observable gets its own pass (merge, truncation), so that
        // top-K can act on it before the first gate
        SubLayerDesc d;
        std::memset(&d, 0, sizeof(d));
        d.cls = CLS_NONE;
        d.noise = -1;
        d.layer_end = 1;
        set_orbit_table(d);
        h->subs.push_back(d);
        h->sub_kind.push_back(0);
    }
    for (int l = h->n_layers - 1; l >= 0; --l) {
        int nz = h->noise.count(l) ? l : -1;
        const size_t before = h->subs.size();
        plan_layer(h, by_layer[l], nz, l);
        if (h->subs.size() > before) h->subs.back().layer_end = 1;
    }
    if (h->subs.empty()) {
        SubLayerDesc d;
        std::memset(&d, 0, sizeof(d));
        d.cls = CLS_NONE;
        d.noise = -1;
        set_orbit_table(d);
        h->subs.push_back(d);
        h->sub_kind.push_back(0);
    }
    h->subs.front().first = 1;
    h->subs.back().final_ = 1;
    return upload_tables(h);
}

size_t term_bytes(const pp_handle* h) {
    return 2 * (size_t)h->W * 8 + (h->opt.precision == PP_PRECISION_FP32 ? 4 : 8);
}


// Bytes of one global-tier slice of `cap` strings (int32 indices).
size_t global_slice_bytes(const pp_handle* h, int cap) {
    size_t carved = h->opt.precision == PP_PRECISION_FP32
        ? (h->W == 1 ? tile_layout_bytes<1, float, int32_t>(cap) : tile_layout_bytes<2, float, int32_t>(cap))
        : (h->W == 1 ? tile_layout_bytes<1, double, int32_t>(cap) : tile_layout_bytes<2, double, int32_t>(cap));
    return (carved + 255) & ~(size_t)255;
}

pp_status alloc_arena(pp_handle* h, Arena* a, size_t cap) {
    a->x = static_cast<uint64_t*>(dev_alloc(h, cap * 8 * h->W));
    a->z = static_cast<uint64_t*>(dev_alloc(h, cap * 8 * h->W));
    a->c = dev_alloc(h, cap * (h->opt.precision == PP_PRECISION_FP32 ? 4 : 8));
    if (!a->x || !a->z || !a->c) return fail(h, PP_ERR_NOMEM, "term arena allocation (%zu terms) failed", cap);
    return PP_OK;
}

// The capacity-dependent work buffers: two term arenas, the raw and grouped
// overflow areas (a quarter of an arena each), bucket fill counters and
// overflow offsets, the tiers' work lists and the global tier's tiles.  They
// grow with the propagation (grow_capacity).  The other work buffers
// (counters, partial sums, top-K state) have fixed sizes.
struct CapMem {
    size_t cap = 0, spill_cap = 0;
    uint32_t fill_cap = 0;
    Arena arena[2], spill_raw, spill_grp;
    uint32_t* spill_b = nullptr;
    uint32_t* spill_s = nullptr;
    uint32_t* fill[2] = {nullptr, nullptr};
    uint64_t* soff[2] = {nullptr, nullptr};
    uint32_t* pass_list[N_TIERS - 1] = {};
    unsigned char* fb_scratch = nullptr;
    size_t fb_slice = 0;
    int fb_cap = 0;
};

void put_cap_memory(pp_handle* h, const CapMem& m) {
    h->cap = m.cap;
    h->spill_cap = m.spill_cap;
    h->fill_cap = m.fill_cap;
    for (int s = 0; s < 2; ++s) {
        h->arena[s] = m.arena[s];
        h->fill[s] = m.fill[s];
        h->soff[s] = m.soff[s];
    }
    h->spill_raw = m.spill_raw;
    h->spill_grp = m.spill_grp;
    h->spill_b = m.spill_b;
    h->spill_s = m.spill_s;
    for (int k = 0; k < N_TIERS - 1; ++k) h->pass_list[k] = m.pass_list[k];
    h->fb_scratch = m.fb_scratch;
    h->fb_slice = m.fb_slice;
    h->fb_cap = m.fb_cap;
}

// Moves the capacity-dependent buffers out of the handle, which then holds none.
CapMem take_cap_memory(pp_handle* h) {
    CapMem m;
    m.cap = h->cap;
    m.spill_cap = h->spill_cap;
    m.fill_cap = h->fill_cap;
    for (int s = 0; s < 2; ++s) {
        m.arena[s] = h->arena[s];
        m.fill[s] = h->fill[s];
        m.soff[s] = h->soff[s];
    }
    m.spill_raw = h->spill_raw;
    m.spill_grp = h->spill_grp;
    m.spill_b = h->spill_b;
    m.spill_s = h->spill_s;
    for (int k = 0; k < N_TIERS - 1; ++k) m.pass_list[k] = h->pass_list[k];
    m.fb_scratch = h->fb_scratch;
    m.fb_slice = h->fb_slice;
    m.fb_cap = h->fb_cap;
    put_cap_memory(h, CapMem());
    return m;
}

void free_cap_memory(pp_handle* h, CapMem& m) {
    for (Arena* a : {&m.arena[0], &m.arena[1], &m.spill_raw, &m.spill_grp})
        for (void* q : {(void*)a->x, (void*)a->z, a->c}) dev_free(h, q);
    for (void* q : {(void*)m.spill_b, (void*)m.spill_s, (void*)m.fill[0], (void*)m.fill[1], (void*)m.soff[0],
                    (void*)m.soff[1], (void*)m.fb_scratch})
        dev_free(h, q);
    for (uint32_t* q : m.pass_list) dev_free(h, q);
    m = CapMem();
}

// Allocates the capacity-dependent buffers for `cap` terms into the handle
// (which holds none).  On failure the caller releases what was made.
pp_status alloc_cap_memory(pp_handle* h, size_t cap) {
    h->cap = cap;
    pp_status st;
    for (int s = 0; s < 2; ++s)
        if ((st = alloc_arena(h, &h->arena[s], cap)) != PP_OK) return st;
    h->spill_cap = std::max<size_t>(cap / 4, 4096) / NSPILL * NSPILL;
    if ((st = alloc_arena(h, &h->spill_raw, h->spill_cap)) != PP_OK) return st;
    if ((st = alloc_arena(h, &h->spill_grp, h->spill_cap)) != PP_OK) return st;
    h->spill_b = static_cast<uint32_t*>(dev_alloc(h, sizeof(uint32_t) * h->spill_cap));
    h->spill_s = static_cast<uint32_t*>(dev_alloc(h, sizeof(uint32_t) * h->spill_cap));
    if (!h->spill_b || !h->spill_s) return fail(h, PP_ERR_NOMEM, "overflow index allocation failed");
    // up to one bucket per 16 terms of capacity
    h->fill_cap = (uint32_t)std::min<size_t>(std::max<size_t>(cap / 16, 1024), 1u << 28);
    for (int s = 0; s < 2; ++s) {
        h->fill[s] = static_cast<uint32_t*>(dev_alloc(h, sizeof(uint32_t) * h->fill_cap));
        h->soff[s] = static_cast<uint64_t*>(dev_alloc(h, sizeof(uint64_t) * h->fill_cap));
        if (!h->fill[s] || !h->soff[s]) return fail(h, PP_ERR_NOMEM, "bucket counters allocation failed");
    }
    for (int k = 0; k < N_TIERS - 1; ++k)
        if (!(h->pass_list[k] = static_cast<uint32_t*>(dev_alloc(h, sizeof(uint32_t) * h->fill_cap))))
            return fail(h, PP_ERR_NOMEM, "work lists allocation failed");
    // the global tier: kFallbackCTAs tiles of up to a quarter of the capacity
    // (at most kFallbackCap strings)
    h->fb_cap = (int)std::min<size_t>(kFallbackCap, std::max<size_t>(4096, cap / 4));
    h->fb_slice = global_slice_bytes(h, h->fb_cap);
    h->fb_scratch = static_cast<unsigned char*>(dev_alloc(h, h->fb_slice * kFallbackCTAs));
    if (!h->fb_scratch) return fail(h, PP_ERR_NOMEM, "global-tier scratch allocation failed");
    return PP_OK;
}

// Releases every work buffer of the handle (not its table arena) and resets
// the pointers, so that a failed set-up leaves the handle as it was created.
void release_work_memory(pp_handle* h) {
    CapMem m = take_cap_memory(h);
    free_cap_memory(h, m);
    auto rel = [&](auto*& ptr) {
        if (ptr) dev_free(h, (void*)ptr);
        ptr = nullptr;
    };
    rel(h->spill_ctr);
    rel(h->counters);
    rel(h->partial);
    rel(h->topk_state);
    rel(h->stage);
    rel(h->sort_scratch);
    h->stage_cap = 0;
    h->sort_scratch_bytes = 0;
    h->mem_ready = false;
}

// Largest capacity the handle may grow to: pp_options.max_terms, or, when
// that is 0, a quarter of the device memory that is free or already held by
// this handle's arenas per arena (two arenas and two quarter-arena overflow
// areas: ~62% of it).
size_t cap_limit(pp_handle* h) {
    if (h->opt.max_terms) return std::max<size_t>(h->opt.max_terms, kMinCap);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return std::max<size_t>(h->cap, kMinCap);
    }
    const double held = 2.5 * (double)h->cap * (double)term_bytes(h);
    return std::max<size_t>(kMinCap, (size_t)(0.25 * ((double)fr + held) / (double)term_bytes(h)));
}

// Work buffers, allocated at the first propagation with room for `want`
// terms (at most the capacity limit).  All or nothing: when an allocation
// fails, the ones made so far are released and PP_ERR_NOMEM is returned with
// the handle unchanged, so a later call can try again.
pp_status ensure_memory(pp_handle* h, size_t want) {
    if (h->mem_ready) return PP_OK;
    pp_status st = PP_OK;
    h->spill_ctr = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long) * NSPILL));
    h->counters = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long) * CTR_COUNT));
    h->partial = static_cast<__int128*>(dev_alloc(h, sizeof(__int128) * (4096 + 1)));
    h->topk_state = static_cast<TopKState*>(dev_alloc(h, sizeof(TopKState)));
    if (!h->spill_ctr || !h->counters || !h->partial || !h->topk_state)
        st = fail(h, PP_ERR_NOMEM, "work buffers allocation failed");
    if (st == PP_OK) st = alloc_cap_memory(h, std::max(kMinCap, std::min(want, cap_limit(h))));
    if (st != PP_OK) {
        cudaStreamSynchronize(h->st);
        std::string msg = h->err;
        release_work_memory(h);
        h->err = msg;
        return st;
    }
    h->mem_ready = true;
    return PP_OK;
}

// Grows the capacity to `want` terms (bounded by the limit; nothing happens
// when that is no gain), keeping the layout the next sub-layer reads: `B`
// bucket regions of `C` terms on arena `side`, their fill counters and
// overflow offsets, and `n_over` grouped overflow terms.  Word w of a term
// array starts at w * capacity, so each word's used prefix is copied to the
// same index in the larger array; the layout's region size stays C.  When
// the device cannot hold `want` terms next to the old buffers, smaller
// capacities down to `need` are tried (halving the step each time).  On
// PP_ERR_NOMEM the handle keeps its old buffers and layout.
pp_status grow_capacity(pp_handle* h, size_t want, int side, uint32_t B, uint64_t C, uint64_t n_over,
                        size_t need = 0) {
    size_t cap = std::min(want, cap_limit(h));
    if (cap <= h->cap) return PP_OK;
    // the new buffers are allocated while the old ones are still held: aim at
    // what fits next to them (two arenas, two quarter-arena overflow areas and
    // the per-bucket arrays: ~2.5 strings plus 4.5 bytes per term of
    // capacity, and a margin), but not below `need`
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        const double per = 2.5 * (double)term_bytes(h) + 4.5;
        const double fit = std::max(0.0, (double)fr - (double)(1ull << 30)) / per;
        if ((double)cap > fit) cap = std::max(need, (size_t)fit);
        if (cap <= h->cap) return PP_OK;
    } else {
        cudaGetLastError();
    }
    CapMem old = take_cap_memory(h);
    pp_status st = PP_OK;
    for (int attempt = 0;; ++attempt) {
        st = alloc_cap_memory(h, cap);
        if (st == PP_OK) break;
        std::string msg = h->err;
        CapMem part = take_cap_memory(h);
        free_cap_memory(h, part);
        const size_t smaller = std::max(need, old.cap + (cap - old.cap) / 2);
        if (attempt >= 4 || need == 0 || smaller >= cap || smaller <= old.cap) {
            put_cap_memory(h, old);
            h->err = msg;
            return st;
        }
        cap = smaller;
    }
    const size_t cb = h->opt.precision == PP_PRECISION_FP32 ? 4 : 8;
    const size_t n_reg = std::min<size_t>((size_t)B * C, old.cap);
    const size_t n_ov = std::min<size_t>(n_over, old.spill_cap);
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->st);
    };
    for (int w = 0; w < h->W; ++w) {
        cp(h->arena[side].x + (size_t)w * h->cap, old.arena[side].x + (size_t)w * old.cap, n_reg * 8);
        cp(h->arena[side].z + (size_t)w * h->cap, old.arena[side].z + (size_t)w * old.cap, n_reg * 8);
        cp(h->spill_grp.x + (size_t)w * h->spill_cap, old.spill_grp.x + (size_t)w * old.spill_cap, n_ov * 8);
        cp(h->spill_grp.z + (size_t)w * h->spill_cap, old.spill_grp.z + (size_t)w * old.spill_cap, n_ov * 8);
    }
    cp(h->arena[side].c, old.arena[side].c, n_reg * cb);
    cp(h->spill_grp.c, old.spill_grp.c, n_ov * cb);
    cp(h->fill[side], old.fill[side], sizeof(uint32_t) * B);
    cp(h->soff[side], old.soff[side], sizeof(uint64_t) * B);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    else cudaStreamSynchronize(h->st);
    free_cap_memory(h, old);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, PP_ERR_CUDA, "capacity growth copy failed: %s", cudaGetErrorString(e));
    }
    h->growths++;
    return PP_OK;
}

// Smallest power of two >= v, but at most the largest power of two <= cap.
uint32_t pow2_at_least(double v, uint32_t cap) {
    uint32_t b = 1;
    while ((double)b < v && 2ull * b <= cap) b <<= 1;
    return b;
}

// Per-device launch facts of one kernel: the dynamic shared-memory limit set
// on it and its resident CTAs per SM.  Both are properties of the device the
// handle runs on, so they are kept per device ordinal; the occupancy query is
// made once per device (it takes driver locks that concurrent handles share).
struct KernelFacts {
    static constexpr int kDevices = 64;
    std::atomic<size_t> attr[kDevices];
    std::atomic<unsigned long long> occ[kDevices];   // resident CTAs << 32 | dynamic smem they were counted for
    KernelFacts() {
        for (int i = 0; i < kDevices; ++i) {
            attr[i].store(0);
            occ[i].store(0);
        }
    }
};

// Raises the kernel's dynamic shared-memory limit on the handle's device to at
// least `smem`.  The limit only ever grows: handles that run concurrently with
// different tile or table sizes must not lower it under each other's launches.
template <typename K>
cudaError_t raise_smem_limit(const pp_handle* h, KernelFacts& f, K kernel, size_t smem) {
    const int dev = h->device;
    if (dev < 0 || dev >= KernelFacts::kDevices) return cudaErrorInvalidDevice;
    if (f.attr[dev].load() < smem) {
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        if (f.attr[dev].load() < smem) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            f.attr[dev].store(smem);
        }
    }
    return cudaSuccess;
}

template <typename K>
cudaError_t prepare_kernel(const pp_handle* h, KernelFacts& f, K kernel, int threads, size_t smem, int* per_sm) {
    const int dev = h->device;
    cudaError_t e0 = raise_smem_limit(h, f, kernel, smem);
    if (e0 != cudaSuccess) return e0;
    const unsigned long long o = f.occ[dev].load();
    int n = (int)(o >> 32);
    if (n == 0 || (o & 0xffffffffull) != (unsigned long long)smem) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
        if (e != cudaSuccess) return e;
        n = std::max(n, 1);
        f.occ[dev].store(((unsigned long long)n << 32) | (unsigned long long)(uint32_t)smem);
    }
    *per_sm = n;
    return cudaSuccess;
}

// A tier launch covers one instance (ps == nullptr: the parameters passed by
// value) or a batch: grid row y serves instance y with the parameters ps[y]
// (device memory) and, in the global tier, the scratch scratch_of[y].
struct LaunchRows {
    const StepParams* ps = nullptr;
    int n = 1;
    unsigned char* const* scratch_of = nullptr;
};

template <int W, typename T, int NT>
cudaError_t launch_smem_tier(pp_handle* h, const StepParams& p, int cap, uint32_t n_items, const LaunchRows& rows) {
    const size_t smem = tile_layout_bytes<W, T, int16_t>((size_t)cap);
    static KernelFacts facts;   // shared by the threads of pp_propagate_batch
    int per_sm = 1;
    cudaError_t e = prepare_kernel(h, facts, k_process<W, T, NT>, NT, smem, &per_sm);
    if (e != cudaSuccess) return e;
    uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(n_items, 1), (uint32_t)(per_sm * h->sm_count));
    k_process<W, T, NT><<<dim3(grid, rows.n), NT, smem, h->st>>>(p, rows.ps, cap);
    return cudaGetLastError();
}

// A tier whose tiles are processed one warp per bucket (pp_warp.cuh), NW
// warps per CTA.
template <int W, typename T, int NW>
cudaError_t launch_warp_tier(pp_handle* h, const StepParams& p, int cap, uint32_t n_items, const LaunchRows& rows) {
    const size_t smem = warp_tile_bytes<W, T>((size_t)cap) * NW;
    static KernelFacts facts;
    int per_sm = 1;
    cudaError_t e = prepare_kernel(h, facts, k_process_warp<W, T, NW>, 32 * NW, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const uint32_t want = n_items == UINT32_MAX ? UINT32_MAX : (n_items + NW - 1) / NW;
    uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(want, 1), (uint32_t)(per_sm * h->sm_count));
    k_process_warp<W, T, NW><<<dim3(grid, rows.n), 32 * NW, smem, h->st>>>(p, rows.ps, cap);
    return cudaGetLastError();
}

// Tile capacities of the orbit tier: strings per bucket, orbit hash slots,
// pool slots, round records.  PP_ORBIT_CAPS="O,H,M,S" overrides them for
// measurements.
template <int W, typename T>
OrbCaps orbit_caps() {
    OrbCaps k{128, 256, 1024, 512};
    if (const char* e = getenv("PP_ORBIT_CAPS")) {
        OrbCaps v{};
        if (sscanf(e, "%d,%d,%d,%d", &v.O, &v.H, &v.M, &v.S) == 4 && v.O > 0 && v.O <= 4096 && v.H >= 2 * v.O &&
            (v.H & (v.H - 1)) == 0 && v.M >= 64 && v.M <= 65536 && v.S > 0 && v.S <= 65535)
            k = v;
    }
    return k;
}

int tier_cap(const pp_handle* h, int tier);

template <int W, typename T>
cudaError_t launch_process(pp_handle* h, const StepParams& p, int tier, bool orbit, uint32_t n_items,
                           int* launches, const LaunchRows& rows) {
    ++*launches;
    const int cap = tier < kGlobalTier ? tier_cap(h, tier) : kTiers[tier].cap1;
    switch (tier) {
        case 0: {
            if (orbit) {
                const OrbCaps K = orbit_caps<W, T>();
                const size_t smem = orb_layout<W, T>(K).bytes * ORB_WARPS;
                static KernelFacts facts;
                int per_sm = 1;
                cudaError_t e = prepare_kernel(h, facts, k_process_orbit<W, T>, 32 * ORB_WARPS, smem, &per_sm);
                if (e != cudaSuccess) return e;
                uint32_t grid = std::min<uint32_t>(std::max<uint32_t>((n_items + ORB_WARPS - 1) / ORB_WARPS, 1),
                                                   (uint32_t)(per_sm * h->sm_count));
                k_process_orbit<W, T><<<dim3(grid, rows.n), 32 * ORB_WARPS, smem, h->st>>>(p, rows.ps, K);
                return cudaGetLastError();
            }
            return launch_warp_tier<W, T, WARP_TILE_WARPS>(h, p, cap, n_items, rows);
        }
        case 1: return launch_warp_tier<W, T, WARP_TILE_WARPS2>(h, p, cap, n_items, rows);
        case 2: return launch_smem_tier<W, T, kTiers[2].threads>(h, p, cap, n_items, rows);
        case 3: return launch_smem_tier<W, T, kTiers[3].threads>(h, p, cap, n_items, rows);
        default: {
            uint32_t grid = std::min<uint32_t>(n_items, (uint32_t)kFallbackCTAs);
            k_process_global<W, T><<<dim3(grid, rows.n), kTiers[kGlobalTier].threads, 0, h->st>>>(
                p, rows.ps, h->fb_scratch, rows.scratch_of, h->fb_slice,
                                                                                  h->fb_cap);
            return cudaGetLastError();
        }
    }
}

// Tile entries of a shared-memory tier; PP_TILE_CAPS="c0,c1,c2,c3" overrides
// the table for measurements.
int tier_cap(const pp_handle* h, int tier) {
    int c = h->W == 1 ? kTiers[tier].cap1 : kTiers[tier].cap2;
    if (tier < kGlobalTier && h->tune.tile_cap[tier] > 0) return h->tune.tile_cap[tier];
    if (tier < kGlobalTier) {
        if (const char* e = getenv("PP_TILE_CAPS")) {
            int v[4] = {0, 0, 0, 0};
            if (sscanf(e, "%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3]) == 4 && v[tier] >= 64 && v[tier] <= 8192)
                c = v[tier];
        }
    }
    return c;
}

// Dynamic shared memory of one CTA of shared-memory tier `tier` with tiles of
// `cap` strings, plus a margin for the kernels' static shared memory.
template <int W, typename T>
size_t tile_smem_bytes_t(int tier, int cap) {
    const size_t stat = 16384;
    if (tier == 0) return warp_tile_bytes<W, T>((size_t)cap) * WARP_TILE_WARPS + stat;
    if (tier == 1) return warp_tile_bytes<W, T>((size_t)cap) * WARP_TILE_WARPS2 + stat;
    return tile_layout_bytes<W, T, int16_t>((size_t)cap) + stat;
}
size_t tile_smem_bytes(const pp_handle* h, int tier, int cap) {
    const bool f32 = h->opt.precision == PP_PRECISION_FP32;
    if (h->W == 1) return f32 ? tile_smem_bytes_t<1, float>(tier, cap) : tile_smem_bytes_t<1, double>(tier, cap);
    return f32 ? tile_smem_bytes_t<2, float>(tier, cap) : tile_smem_bytes_t<2, double>(tier, cap);
}

cudaError_t dispatch_process(pp_handle* h, const StepParams& p, int tier, bool orbit, uint32_t n_items,
                             int* launches, const LaunchRows& rows = LaunchRows()) {
    bool f32 = h->opt.precision == PP_PRECISION_FP32;
    if (h->W == 1) return f32 ? launch_process<1, float>(h, p, tier, orbit, n_items, launches, rows)
                              : launch_process<1, double>(h, p, tier, orbit, n_items, launches, rows);
    return f32 ? launch_process<2, float>(h, p, tier, orbit, n_items, launches, rows)
               : launch_process<2, double>(h, p, tier, orbit, n_items, launches, rows);
}

// Load limit of a bucket of the orbit tier.
int orbit_load_cap(const pp_handle* h) {
    if (h->W == 1) return h->opt.precision == PP_PRECISION_FP32 ? orbit_caps<1, float>().O : orbit_caps<1, double>().O;
    return h->opt.precision == PP_PRECISION_FP32 ? orbit_caps<2, float>().O : orbit_caps<2, double>().O;
}

// Slots of the input-merge hash table for n input strings (load factor <= 1/2).
size_t input_merge_slots(size_t n) {
    size_t H = 64;
    while (H < 2 * n) H <<= 1;
    return H;
}

// Merges duplicate input strings (k_input_claim, k_input_accumulate) and
// scatters the merged observable into the first sub-layer's buckets.  `m`
// points at zeroed counts and accumulators and owners set to -1.
template <int W>
cudaError_t launch_input(pp_handle* h, const uint64_t* ox, const uint64_t* oz, const double* oc, size_t n,
                         const InputMerge& m, const StepParams& p) {
    const int grid = (int)std::max<size_t>(std::min<size_t>((n + 255) / 256, 4096), 1);
    k_input_claim<W><<<grid, 256, 0, h->st>>>(ox, oz, n, m);
    k_input_accumulate<W><<<grid, 256, 0, h->st>>>(ox, oz, oc, n, m);
    if (h->opt.precision == PP_PRECISION_FP32) k_scatter_input<W, float><<<grid, 256, 0, h->st>>>(ox, oz, oc, n, m, p);
    else k_scatter_input<W, double><<<grid, 256, 0, h->st>>>(ox, oz, oc, n, m, p);
    return cudaGetLastError();
}

cudaError_t dispatch_scatter(pp_handle* h, const uint64_t* ox, const uint64_t* oz, const double* oc,
                             size_t n, const InputMerge& m, const StepParams& p, int* launches) {
    *launches += 3;
    return h->W == 1 ? launch_input<1>(h, ox, oz, oc, n, m, p) : launch_input<2>(h, ox, oz, oc, n, m, p);
}

NoiseDesc noise_desc(const NoiseHost& nh) {
    NoiseDesc d;
    d.mode = nh.mode;
    d.n_generic = (int)nh.glam.size();
    d.n_shift = (int)nh.shift.size();
    d.n_sites = nh.n;
    d.n_groups = (nh.n + 3) / 4;
    d.grp = nh.d_grp;
    d.shift = nh.d_shift;
    d.xmask = nh.d_xmask;
    d.pidx = nh.d_pidx;
    d.c2 = nh.d_c2;
    d.etab = nh.d_etab;
    d.ftab = nh.d_ftab;
    d.gen_x = nh.d_gx;
    d.gen_z = nh.d_gz;
    d.gen_lam = nh.d_glam;
    return d;
}

// Applies noise map nh in place to layout `side` (B buckets of C, plus n_over
// grouped overflow strings).
cudaError_t apply_noise(pp_handle* h, const NoiseHost& nh, int side, uint32_t B, uint64_t C, uint64_t n_over,
                        double eps, float eps_f, int* launches) {
    NoiseDesc nz = noise_desc(nh);
    const int n_pairs = (int)(nh.c2.size() / 16);
    const NoiseSmem L = noise_smem_layout(nz.n_sites, nz.n_groups, nz.n_shift, n_pairs, h->W);
    const bool f32 = h->opt.precision == PP_PRECISION_FP32;
    const Arena& a = h->arena[side];
    const Arena& o = h->spill_grp;
    int per_sm = 1;
    cudaError_t e;
#define PP_NOISE_LAUNCH(WW, TT)                                                                         \
    {                                                                                                   \
        static KernelFacts facts;                                                                       \
        e = prepare_kernel(h, facts, k_noise<WW, TT>, 256, L.bytes, &per_sm);                           \
    }                                                                                                   \
    if (e != cudaSuccess) return e;                                                                     \
    k_noise<WW, TT><<<h->sm_count * std::min(per_sm, 8), 256, L.bytes, h->st>>>(a.x, a.z, (TT*)a.c, h->cap, h->fill[side], B, C, o.x, o.z, \
                                                 (TT*)o.c, h->spill_cap, n_over, nz, n_pairs, eps, eps_f)
    if (h->W == 1) {
        if (f32) { PP_NOISE_LAUNCH(1, float); } else { PP_NOISE_LAUNCH(1, double); }
    } else {
        if (f32) { PP_NOISE_LAUNCH(2, float); } else { PP_NOISE_LAUNCH(2, double); }
    }
#undef PP_NOISE_LAUNCH
    ++*launches;
    return cudaGetLastError();
}

// Groups the overflow strings of a freshly written layout by bucket.  Runs
// whether or not anything spilled (the kernels find out on the device); the
// number of grouped strings lands in counters[CTR_SPILL_TOTAL].  When the
// sub-layer's output outgrew its layout (it runs again from its input), the
// strings are not moved: the grouped overflow area still holds the input's.
cudaError_t group_spill(pp_handle* h, int side, uint32_t nB, uint64_t C, unsigned long long* counters,
                        int* launches) {
    cudaError_t e = cudaMemsetAsync(counters + CTR_SPILL_TOTAL, 0, sizeof(unsigned long long), h->st);
    if (e != cudaSuccess) return e;
    uint32_t grid = (nB + 1023) / 1024;
    k_spill_offsets<<<grid, 1024, 0, h->st>>>(h->fill[side], nB, C, h->soff[side], counters + CTR_SPILL_TOTAL);
    const dim3 g2(NSPILL, (unsigned)std::max(1, h->sm_count * 8 / NSPILL));
    const bool f32 = h->opt.precision == PP_PRECISION_FP32;
    const Arena& r = h->spill_raw;
    const Arena& o = h->spill_grp;
    if (h->W == 1) {
        if (f32) k_spill_move<1, float><<<g2, 256, 0, h->st>>>(r.x, r.z, (const float*)r.c, h->spill_b, h->spill_s, h->spill_cap, h->spill_ctr, h->soff[side], o.x, o.z, (float*)o.c, h->spill_cap, counters, h->cap);
        else k_spill_move<1, double><<<g2, 256, 0, h->st>>>(r.x, r.z, (const double*)r.c, h->spill_b, h->spill_s, h->spill_cap, h->spill_ctr, h->soff[side], o.x, o.z, (double*)o.c, h->spill_cap, counters, h->cap);
    } else {
        if (f32) k_spill_move<2, float><<<g2, 256, 0, h->st>>>(r.x, r.z, (const float*)r.c, h->spill_b, h->spill_s, h->spill_cap, h->spill_ctr, h->soff[side], o.x, o.z, (float*)o.c, h->spill_cap, counters, h->cap);
        else k_spill_move<2, double><<<g2, 256, 0, h->st>>>(r.x, r.z, (const double*)r.c, h->spill_b, h->spill_s, h->spill_cap, h->spill_ctr, h->soff[side], o.x, o.z, (double*)o.c, h->spill_cap, counters, h->cap);
    }
    *launches += 2;
    return cudaGetLastError();
}


float eps_float_ceil(double eps) {
    float f = (float)eps;
    if ((double)f < eps) f = std::nextafter(f, INFINITY);
    return f;
}

}  // namespace

namespace {

// Keeps the K largest live strings of a span (pp_topk.cuh); the rest get
// coefficient 0.  Every decision stays on the device.
template <int W, typename T>
cudaError_t top_k_span(pp_handle* h, const Span<T>& s, size_t K, int* launches) {
    TopKState* st = h->topk_state;
    const int grid = h->sm_count * 4;
    k_topk_init<<<1, 256, 0, h->st>>>(st, (unsigned long long)K);
    for (int shift = MagBits<T>::BITS - 8; shift >= 0; shift -= 8) {
        k_topk_hist<W, T><<<grid, 256, 0, h->st>>>(s, st, shift);
        k_topk_pick<<<1, 256, 0, h->st>>>(st, shift, shift == 0);
        *launches += 2;
    }
    for (int kw = 0; kw < 2 * W; ++kw)
        for (int shift = 56; shift >= 0; shift -= 8) {
            k_topk_key_hist<W, T><<<grid, 256, 0, h->st>>>(s, st, kw, shift);
            k_topk_key_pick<<<1, 256, 0, h->st>>>(st, kw, shift);
            *launches += 2;
        }
    k_topk_mark<W, T><<<grid, 256, 0, h->st>>>(s, st);
    *launches += 2;
    return cudaGetLastError();
}

// Top-K on layout `side` (B buckets of C, n_over grouped overflow strings), or
// on the compact result [0, n_over) of `side` when fill is false.
cudaError_t apply_top_k(pp_handle* h, int side, bool bucketed, uint32_t B, uint64_t C, uint64_t n_over,
                        int* launches) {
    const Arena& a = h->arena[side];
    const Arena& o = bucketed ? h->spill_grp : a;
    const uint64_t ocap = bucketed ? h->spill_cap : h->cap;
    const uint32_t* fill = bucketed ? h->fill[side] : nullptr;
#define PP_TOPK(WW, TT)                                                                                 \
    {                                                                                                   \
        Span<TT> s{a.x, a.z, (TT*)a.c, h->cap, fill, B, C, o.x, o.z, (TT*)o.c, ocap, n_over};         \
        return top_k_span<WW, TT>(h, s, h->top_k, launches);                                          \
    }
    const bool f32 = h->opt.precision == PP_PRECISION_FP32;
    if (h->W == 1) {
        if (f32) PP_TOPK(1, float) else PP_TOPK(1, double)
    } else {
        if (f32) PP_TOPK(2, float) else PP_TOPK(2, double)
    }
#undef PP_TOPK
}

// Compacts the live strings of the result [0, n) on `side` into the other arena.
cudaError_t compact_result(pp_handle* h, int side, uint64_t n, int* launches) {
    const Arena& a = h->arena[side];
    const Arena& d = h->arena[side ^ 1];
    unsigned long long* cnt = h->counters + CTR_SPILL_TOTAL;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->st);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(std::max<uint64_t>((n + 255) / 256, 1), (uint64_t)h->sm_count * 8);
    const bool f32 = h->opt.precision == PP_PRECISION_FP32;
    if (h->W == 1) {
        if (f32) k_compact<1, float><<<grid, 256, 0, h->st>>>(a.x, a.z, (const float*)a.c, h->cap, n, d.x, d.z, (float*)d.c, h->cap, cnt);
        else k_compact<1, double><<<grid, 256, 0, h->st>>>(a.x, a.z, (const double*)a.c, h->cap, n, d.x, d.z, (double*)d.c, h->cap, cnt);
    } else {
        if (f32) k_compact<2, float><<<grid, 256, 0, h->st>>>(a.x, a.z, (const float*)a.c, h->cap, n, d.x, d.z, (float*)d.c, h->cap, cnt);
        else k_compact<2, double><<<grid, 256, 0, h->st>>>(a.x, a.z, (const double*)a.c, h->cap, n, d.x, d.z, (double*)d.c, h->cap, cnt);
    }
    ++*launches;
    return cudaGetLastError();
}

// Orders the result's strings by key on the device (pp_result.cuh): radix
// passes ping-pong between the two term arenas; the sorted result stays the
// handle's result.
template <int W, typename T>
pp_status sort_result(pp_handle* h) {
    const size_t N = h->n_res;
    const uint32_t n_tiles = (uint32_t)((N + SORT_TILE - 1) / SORT_TILE);
    const size_t L = (size_t)SORT_RADIX * n_tiles;
    const size_t n_chunks = (L + SCAN_CHUNK - 1) / SCAN_CHUNK;
    const size_t bytes = 16 * 2 * W + 4 * (L + n_chunks);
    if (bytes > h->sort_scratch_bytes) {
        if (h->sort_scratch) {
            CK(cudaStreamSynchronize(h->st));
            dev_free(h, h->sort_scratch);
        }
        h->sort_scratch = static_cast<unsigned char*>(dev_alloc(h, bytes));
        h->sort_scratch_bytes = h->sort_scratch ? bytes : 0;
        if (!h->sort_scratch) return fail(h, PP_ERR_NOMEM, "export sort scratch allocation failed");
    }
    unsigned long long* varying = reinterpret_cast<unsigned long long*>(h->sort_scratch);
    uint32_t* counts = reinterpret_cast<uint32_t*>(h->sort_scratch + 16 * 2 * W);
    uint32_t* sums = counts + L;
    CK(cudaMemsetAsync(varying, 0, sizeof(unsigned long long) * 2 * W, h->st));
    int cur = h->res_side;
    {
        const Arena& a = h->arena[cur];
        const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)4 * h->sm_count);
        k_sort_varying<W><<<grid, 256, 0, h->st>>>(a.x, a.z, h->cap, N, varying);
        CK(cudaGetLastError());
    }
    unsigned long long vary[2 * W];
    CK(cudaMemcpyAsync(vary, varying, sizeof(vary), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int kw = 0; kw < 2 * W; ++kw)
        for (int shift = 0; shift < 64; shift += 8) {
            if (((vary[kw] >> shift) & 0xffull) == 0) continue;   // one digit value in every key
            const Arena& a = h->arena[cur];
            const Arena& b = h->arena[cur ^ 1];
            k_sort_hist<W><<<n_tiles, SORT_THREADS, 0, h->st>>>(a.x, a.z, h->cap, N, kw, shift, counts, n_tiles);
            k_scan_chunks<<<(unsigned)n_chunks, SORT_THREADS, 0, h->st>>>(counts, L, sums);
            k_scan_sums<<<1, SORT_THREADS, 0, h->st>>>(sums, (uint32_t)n_chunks);
            k_scan_add<<<(unsigned)n_chunks, SORT_THREADS, 0, h->st>>>(counts, L, sums);
            k_sort_scatter<W, T><<<n_tiles, SORT_THREADS, 0, h->st>>>(
                a.x, a.z, static_cast<const T*>(a.c), h->cap, N, kw, shift, counts, n_tiles, b.x, b.z,
                static_cast<T*>(b.c), h->cap);
            CK(cudaGetLastError());
            cur ^= 1;
        }
    h->res_side = cur;
    return PP_OK;
}

// ----------------------------------------------------------------------------- one propagation

// The state of one propagation, advanced one fused sub-layer at a time.  A
// single pp_propagate drives one; pp_propagate_batch drives many in lockstep,
// launching each kernel once for all of them.
struct Prop {
    pp_handle* h = nullptr;
    long long gen = 0;
    std::chrono::steady_clock::time_point t0;
    bool batch = false;              // part of a lockstep batch (no orbit tiles, no per-tier timing)
    int S = 0, s = 0, side = 0, attempt = 0;
    uint32_t B = 1, nB = 1;          // bucket counts of the source and destination layouts
    uint64_t C = 0, nC = 0;          // their region sizes
    size_t N = 0, peak = 0;
    double updates = 0.0;
    unsigned long long n_over_in = 0;   // grouped overflow strings of the source layout
    std::map<int, double> growth;    // observed output/input per sub-layer kind
    StepParams p;
    pp_stats stats{};
    int launches = 0;
    FILE* trace = nullptr;
    unsigned long long* ctr_dev = nullptr;   // the counters this propagation uses
    unsigned long long ctr[CTR_COUNT];
    float ms[N_TIERS] = {};
    bool finished = false;
    Prop() { std::memset(&p, 0, sizeof(p)); }
    ~Prop() {
        if (trace) fclose(trace);
    }
    Prop(const Prop&) = delete;
    Prop& operator=(const Prop&) = delete;

    double growth_of(int k) const {
        auto it = growth.find(h->sub_kind[k]);
        return it == growth.end() ? 3.0 : it->second;
    }
    // sub-layers processed by the orbit tiles first (the input observable,
    // which may hold duplicates, and sub-layers after a forced first tier go
    // to the sparse tiles)
    bool use_orbit(int k) const {
        const SubLayerDesc& d = h->subs[k];
        return !batch && d.orb && !d.first && h->tune.orbit_tiles && h->tune.first_tier == 0;
    }
    // buckets for sub-layer k holding about n strings: a sparse tile must also
    // hold the strings the sub-layer creates, so aim at cap / (headroom *
    // growth); an orbit tile holds only its input (at 3/4 of its limit)
    uint32_t buckets_for(int k, double n) const {
        const double g = bucket_headroom(h) * std::max(1.0, growth_of(k));
        double per = use_orbit(k) ? 0.75 * orbit_load_cap(h) : (double)tier_cap(h, 0) / g;
        per = std::max(per, 16.0);
        return pow2_at_least(n / per, h->fill_cap);
    }
};

#undef CK
#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, PP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

// The launch parameters that point into the capacity-dependent buffers
// (they move when the capacity grows).
void set_capacity_params(Prop& P) {
    pp_handle* h = P.h;
    StepParams& p = P.p;
    p.rpx = h->spill_raw.x;
    p.rpz = h->spill_raw.z;
    p.rpc = h->spill_raw.c;
    p.rpb = h->spill_b;
    p.rps = h->spill_s;
    p.rpcap = h->spill_cap;
    p.spx = h->spill_grp.x;
    p.spz = h->spill_grp.z;
    p.spc = h->spill_grp.c;
    p.spcap = h->spill_cap;
    p.gcap = h->fb_cap;
    p.gslice = h->fb_slice;
}

// Validates, plans, stages the observable and scatters it into the first
// sub-layer's buckets (one synchronisation).
pp_status prop_begin(Prop& P, pp_handle* h, size_t n_terms, const uint64_t* ox, const uint64_t* oz,
                     const double* oc, double eps, int w_max, unsigned long long* ctr_dev, bool batch) {
    P.h = h;
    P.batch = batch;
    P.ctr_dev = ctr_dev;
    h->err.clear();
    P.t0 = std::chrono::steady_clock::now();
    if (!h->have_circuit) return fail(h, PP_ERR_STATE, "no circuit loaded");
    if (n_terms && (!ox || !oz || !oc)) return fail(h, PP_ERR_ARG, "null observable arrays");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(h, PP_ERR_ARG, "eps must be finite and >= 0");
    h->have_result = false;
    P.gen = ++h->run_gen;
    pp_status st;
    if (h->subs_dirty && (st = build_plan(h)) != PP_OK) return st;
    h->growths = 0;
    const size_t want = std::max<size_t>(kInitialCap, 4 * n_terms);
    if ((st = ensure_memory(h, want)) != PP_OK) return st;
    if (2 * n_terms > h->cap && (st = grow_capacity(h, want, 0, 0, 0, 0)) != PP_OK) return st;
    if (!P.ctr_dev) P.ctr_dev = h->counters;
    const int W = h->W;

    // stage the observable, followed by the input-merge table
    if (n_terms > h->cap) return fail(h, PP_ERR_CAPACITY, "observable larger than capacity");
    if (n_terms > (size_t)INT32_MAX) return fail(h, PP_ERR_ARG, "more than 2^31 - 1 observable terms");
    for (size_t i = 0; i < n_terms; ++i)
        if (!(std::fabs(oc[i]) < 4294967296.0))
            return fail(h, PP_ERR_ARG, "observable coefficient %zu is not finite with magnitude below 2^32", i);
    const size_t H = input_merge_slots(n_terms);
    size_t need = std::max<size_t>(n_terms, 1) * (2 * W + 1) + 3 * H;
    if (need > h->stage_cap) {
        if (h->stage) dev_free(h, h->stage);
        h->stage = static_cast<uint64_t*>(dev_alloc(h, need * 8));
        if (!h->stage) {
            h->stage_cap = 0;
            return fail(h, PP_ERR_NOMEM, "staging allocation failed");
        }
        h->stage_cap = need;
    }
    uint64_t* sx = h->stage;
    uint64_t* sz = h->stage + n_terms * W;
    double* sc = reinterpret_cast<double*>(h->stage + 2 * n_terms * W);
    InputMerge im;
    unsigned char* mt = reinterpret_cast<unsigned char*>(h->stage + std::max<size_t>(n_terms, 1) * (2 * W + 1));
    im.owner = reinterpret_cast<int*>(mt);
    im.count = reinterpret_cast<unsigned*>(mt + 4 * H);
    im.acc = reinterpret_cast<unsigned long long*>(mt + 8 * H);
    im.hmask = (uint32_t)(H - 1);
    if (n_terms) {
        CK(cudaMemsetAsync(im.owner, 0xff, 4 * H, h->st));
        CK(cudaMemsetAsync(im.count, 0, 4 * H + 16 * H, h->st));
        CK(cudaMemcpyAsync(sx, ox, n_terms * W * 8, cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(sz, oz, n_terms * W * 8, cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(sc, oc, n_terms * 8, cudaMemcpyHostToDevice, h->st));
    }
    if (const char* tp = getenv("PP_TRACE")) P.trace = fopen(tp, "a");
    if (h->timing && !batch && !h->tier_ev[0][0])
        for (auto& pr : h->tier_ev)
            for (auto& e : pr) CK(cudaEventCreate(&e));

    StepParams& p = P.p;
    p.eps = eps;
    p.eps_f = eps_float_ceil(eps);
    p.w_max = w_max;
    p.counters = P.ctr_dev;
    p.spill_ctr = h->spill_ctr;
    p.phase = P.trace ? P.ctr_dev + CTR_PHASE : nullptr;
    set_capacity_params(P);

    // scatter the input into the first sub-layer's buckets
    P.side = 0;
    P.B = P.buckets_for(0, (double)n_terms);
    P.C = h->cap / P.B;
    CK(cudaMemsetAsync(h->fill[0], 0, sizeof(uint32_t) * P.B, h->st));
    CK(cudaMemsetAsync(P.ctr_dev, 0, sizeof(unsigned long long) * CTR_COUNT, h->st));
    CK(cudaMemsetAsync(h->spill_ctr, 0, sizeof(unsigned long long) * NSPILL, h->st));
    p.dx = h->arena[0].x;
    p.dz = h->arena[0].z;
    p.dc = h->arena[0].c;
    p.dcap = h->cap;
    p.dfill = h->fill[0];
    p.dB = P.B;
    p.dC = P.C;
    p.next = h->d_subs;
    if (n_terms) CK(dispatch_scatter(h, sx, sz, sc, n_terms, im, p, &P.launches));
    CK(group_spill(h, 0, P.B, P.C, P.ctr_dev, &P.launches));
    CK(cudaMemcpyAsync(P.ctr, P.ctr_dev, sizeof(P.ctr), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (P.ctr[CTR_DEBUG]) return fail(h, PP_ERR_CUDA, "device bounds check %llu failed", P.ctr[CTR_DEBUG]);
    if (P.ctr[CTR_ERR_REGION]) return fail(h, PP_ERR_CAPACITY, "input overflowed the overflow area");
    P.n_over_in = P.ctr[CTR_SPILL_TOTAL];
    P.N = P.peak = n_terms;
    P.S = (int)h->subs.size();
    P.s = 0;
    P.attempt = 0;
    return PP_OK;
}

// Plans sub-layer P.s: the destination buckets (unless a retry already sized
// them) and the launch parameters.
pp_status prop_setup(Prop& P) {
    pp_handle* h = P.h;
    const SubLayerDesc& d = h->subs[P.s];
    const bool fin = d.final_ != 0;
    if (P.attempt == 0) {
        const double out = (double)P.N * P.growth_of(P.s);   // expected output
        // grow first when the output would fill more than half the buffers
        if (2.0 * out > (double)h->cap) {
            pp_status st = grow_capacity(h, (size_t)(2.5 * out), P.side, P.B, P.C, P.n_over_in, (size_t)(1.25 * out));
            if (st != PP_OK) return st;
        }
        const double est = std::max(64.0, out * 1.3);
        P.nB = fin ? 1 : P.buckets_for(P.s + 1, est);
        P.nC = fin ? h->cap : h->cap / P.nB;
    }
    set_capacity_params(P);
    StepParams& p = P.p;
    p.sx = h->arena[P.side].x;
    p.sz = h->arena[P.side].z;
    p.sc = h->arena[P.side].c;
    p.scap = h->cap;
    p.sfill = h->fill[P.side];
    p.soff = h->soff[P.side];
    p.sB = P.B;
    p.sC = P.C;
    p.dx = h->arena[P.side ^ 1].x;
    p.dz = h->arena[P.side ^ 1].z;
    p.dc = h->arena[P.side ^ 1].c;
    p.dcap = h->cap;
    p.dfill = h->fill[P.side ^ 1];
    p.dB = P.nB;
    p.dC = P.nC;
    p.desc = h->d_subs + P.s;
    p.next = fin ? nullptr : h->d_subs + P.s + 1;
    // A noise map on the input observable itself stays in the processor's
    // prologue (after the merge and truncation of the input); any other is
    // applied by a streaming pass over the layout first (prop_noise).
    p.has_noise = d.noise >= 0 && d.first;
    if (p.has_noise) p.noise = noise_desc(h->noise[d.noise]);
    return PP_OK;
}

// The streaming noise pass of sub-layer P.s (not again on a retry: it acts in place).
pp_status prop_noise(Prop& P) {
    pp_handle* h = P.h;
    const SubLayerDesc& d = h->subs[P.s];
    if (d.noise >= 0 && !d.first && P.attempt == 0)
        CK(apply_noise(h, h->noise[d.noise], P.side, P.B, P.C, P.n_over_in, P.p.eps, P.p.eps_f, &P.launches));
    return PP_OK;
}

// Launch parameters of tier `tier` of sub-layer P.s; returns whether tier 0
// runs the orbit tiles, and the launch's work-item bound.
bool prop_tier(Prop& P, int tier, uint32_t* n_items) {
    pp_handle* h = P.h;
    StepParams& p = P.p;
    p.in_list = tier == 0 ? nullptr : h->pass_list[tier - 1];
    p.n_list = 0;
    p.n_list_dev = tier == 0 ? nullptr : P.ctr_dev + CTR_DEFER + tier - 1;
    *n_items = tier == 0 ? P.B : UINT32_MAX;   // the later tiers' counts are on the device
    p.out_list = tier < kGlobalTier ? h->pass_list[tier] : nullptr;
    p.work_ctr = CTR_WORK + tier;
    p.defer_ctr = CTR_DEFER + (tier < kGlobalTier ? tier : 0);
    const bool orbit = tier == 0 && P.use_orbit(P.s);
    p.max_load = (uint32_t)((size_t)(tier == kGlobalTier ? h->fb_cap : tier_cap(h, tier)) * kTiers[tier].load / 100);
    if (orbit) p.max_load = (uint32_t)orbit_load_cap(h);
    if (tier < h->tune.first_tier) p.max_load = 0;   // every bucket is passed on
    if (orbit) P.stats.orbit_launches++;
    P.stats.tier_launches[tier]++;
    return orbit;
}

// After the sub-layer's counters are back (P.ctr): statistics, errors, the
// retry decision, top-K, and the move to the next sub-layer.
pp_status prop_finish(Prop& P) {
    pp_handle* h = P.h;
    const int s = P.s;
    const SubLayerDesc& d = h->subs[s];
    const bool fin = d.final_ != 0;
    const unsigned long long* ctr = P.ctr;
    if (h->cancel_gen.load() == P.gen) return fail(h, PP_ERR_TIMEOUT, "cancelled after sub-layer %d", s);
    if (ctr[CTR_DEBUG])
        return fail(h, PP_ERR_CUDA, "sub-layer %d: device bounds check %llu failed", s, ctr[CTR_DEBUG]);
    for (int tier = 0; tier < N_TIERS; ++tier) {
        P.stats.tier_ms[tier] += P.ms[tier];
        P.stats.tier_strings[tier] += (double)ctr[CTR_LOADED + tier] + (double)ctr[CTR_EMITTED + tier];
    }
    unsigned long long passed[N_TIERS] = {};
    for (int tier = 0; tier + 1 < N_TIERS; ++tier) passed[tier] = ctr[CTR_DEFER + tier];
    P.stats.fallback_buckets += (int)passed[kGlobalTier - 1];
    if (ctr[CTR_ERR_FALLBACK])
        return fail(h, PP_ERR_CAPACITY, "sub-layer %d: a bucket exceeds the global tile (%d strings)", s, h->fb_cap);
    // A sub-layer whose output outgrew the planned buckets, the overflow area or
    // the capacity runs again (at most twice more), after the capacity has
    // grown to twice its true output, with buckets sized from that output: its
    // source layout is only read, and its noise map (applied in place) is not
    // applied again.
    const double out = (double)ctr[CTR_OUT];
    if ((ctr[CTR_ERR_REGION] || ctr[CTR_OUT] > h->cap) && P.attempt < 2) {
        P.growth[h->sub_kind[s]] = std::max(0.05, out / std::max<double>(1.0, (double)P.N));
        if (2.0 * out > (double)h->cap) {
            pp_status st = grow_capacity(h, (size_t)(2.0 * out), P.side, P.B, P.C, P.n_over_in, (size_t)(1.1 * out));
            if (st != PP_OK) return st;
        }
        if (out <= (double)h->cap) {
            P.nB = fin ? 1 : P.buckets_for(s + 1, std::max(64.0, 1.3 * out));
            P.nC = fin ? h->cap : h->cap / P.nB;
            P.stats.retries++;
            P.attempt++;
            return PP_OK;
        }
    }
    if (ctr[CTR_ERR_REGION] || ctr[CTR_OUT] > h->cap)
        return fail(h, PP_ERR_CAPACITY, "sub-layer %d: %llu live terms exceed the capacity (%zu terms, "
                    "%zu overflow; limit %zu); raise max_terms", s, (unsigned long long)ctr[CTR_OUT], h->cap,
                    h->spill_cap, cap_limit(h));
    const unsigned long long n_spill_out = fin ? 0ull : ctr[CTR_SPILL_TOTAL];
    // canonical gate-by-gate count (live terms entering each gate in listed
    // order), summed by the kernels over string lifetimes
    P.updates += (double)ctr[CTR_UPDATES];
    size_t Nout = (size_t)ctr[CTR_OUT];
    P.peak = std::max(P.peak, Nout);
    bool compacted = false;
    if (h->top_k > 0 && d.layer_end && Nout > h->top_k) {
        // keep the K largest strings of the layer's result (Sec. I.A)
        if (!fin) {
            CK(apply_top_k(h, P.side ^ 1, true, P.nB, P.nC, n_spill_out, &P.launches));
        } else {
            CK(apply_top_k(h, P.side ^ 1, false, 1, h->cap, Nout, &P.launches));
            CK(compact_result(h, P.side ^ 1, Nout, &P.launches));
            compacted = true;
        }
        Nout = h->top_k;
    }
    if (P.trace) {
        // one JSON line per sub-layer (PP_TRACE): sizes, per-tier figures, failures
        auto list = [](const unsigned long long* v, int n, int stride = 1) {
            std::string t = "[";
            for (int k = 0; k < n; ++k) t += (k ? ", " : "") + std::to_string(v[k * stride]);
            return t + "]";
        };
        std::string ms = "[", ts = "[";
        for (int tier = 0; tier < N_TIERS; ++tier) {
            char b[64];
            snprintf(b, sizeof(b), "%s%.4f", tier ? ", " : "", P.ms[tier]);
            ms += b;
            ts += (tier ? ", " : "") + std::to_string(ctr[CTR_LOADED + tier] + ctr[CTR_EMITTED + tier]);
        }
        ms += "]";
        ts += "]";
        fprintf(P.trace,
                "{\"sub\": %d, \"cls\": %d, \"gates\": %d, \"orbit\": %d, \"n_in\": %zu, \"n_out\": %zu, "
                "\"buckets_in\": %u, \"buckets_out\": %u, \"passed\": %s, \"spill\": %llu, \"ms\": %s, "
                "\"tier_strings\": %s, \"fail_load\": %llu, \"fail_pool\": %llu, \"fail_hash\": %llu, "
                "\"t0_cycles\": %s, \"cta_cycles\": %s, \"t0_stat\": %s}\n",
                s, d.cls, d.n_gates, (int)P.use_orbit(s), P.N, Nout, P.B, P.nB, list(passed, N_TIERS - 1).c_str(),
                n_spill_out, ms.c_str(), ts.c_str(), ctr[CTR_FAIL], ctr[CTR_FAIL + 1], ctr[CTR_FAIL + 2],
                list(ctr + CTR_PHASE, 4).c_str(), list(ctr + CTR_PHASE_CTA, 4).c_str(), list(ctr + CTR_STAT, 7).c_str());
    }
    if (P.N > 0) P.growth[h->sub_kind[s]] = std::max(0.05, (double)Nout / (double)P.N);
    P.N = Nout;
    P.n_over_in = n_spill_out;
    if (!compacted) P.side ^= 1;   // a compacted result went back to this sub-layer's source arena
    P.B = P.nB;
    P.C = P.nC;
    P.stats.n_sublayers++;
    for (float& m : P.ms) m = 0.f;
    P.s++;
    P.attempt = 0;
    return PP_OK;
}

void prop_end(Prop& P) {
    pp_handle* h = P.h;
    h->res_side = P.side;
    h->n_res = P.N;
    h->have_result = true;
    P.stats.n_terms = P.N;
    P.stats.peak_terms = P.peak;
    P.stats.updates = P.updates;
    P.stats.kernel_launches = P.launches;
    P.stats.bytes_per_string = (double)term_bytes(h);
    P.stats.growths = h->growths;
    P.stats.capacity = h->cap;
    P.stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - P.t0).count();
    h->stats = P.stats;
    P.finished = true;
}

// ----------------------------------------------------------------------------- lockstep batches

// Device buffers of one lockstep batch.
struct BatchBufs {
    pp_handle* h = nullptr;
    unsigned long long* ctr = nullptr;   // [n][CTR_COUNT]
    StepParams* ps = nullptr;            // [N_TIERS][n]
    SpillArgs* args = nullptr;           // [2][n]: clearing, overflow grouping
    unsigned char** scratch = nullptr;   // [n] global-tier scratch of each instance
    ~BatchBufs() {
        for (void* q : {(void*)ctr, (void*)ps, (void*)args, (void*)scratch})
            if (q) dev_free(h, q);
    }
};

template <int W, typename T>
void launch_spill_batch(pp_handle* h0, const SpillArgs* args, int rows) {
    k_spill_offsets_batch<<<dim3((unsigned)std::max(1, h0->sm_count), rows), 1024, 0, h0->st>>>(args);
    const dim3 g(NSPILL, (unsigned)std::max(1, h0->sm_count * 8 / NSPILL / std::max(1, rows)) + 1, rows);
    k_spill_move_batch<W, T><<<g, 256, 0, h0->st>>>(args);
}

// Runs the propagations of handles[idx[..]] (same device, mask width and
// precision) in lockstep on the first handle's stream: every lockstep step
// advances each unfinished propagation by one fused sub-layer, launching each
// kernel once for all of them (grid row = instance), and waits for the device
// once for the whole batch.  Each instance keeps its own plan, layouts and
// counters, so its result equals a pp_propagate of the same handle.
void run_lockstep(pp_handle* const* handles, const pp_batch_item* items, const std::vector<int>& idx,
                  std::vector<pp_status>& status) {
    const int n = (int)idx.size();
    pp_handle* h0 = handles[idx[0]];
    pp_handle* h = h0;   // for CK-style error reports on the batch's own buffers
    std::vector<cudaStream_t> saved(n);
    for (int k = 0; k < n; ++k) {
        saved[k] = handles[idx[k]]->st;
        handles[idx[k]]->st = h0->st;
    }
    auto finish_all = [&](pp_status st) {
        for (int k = 0; k < n; ++k)
            if (status[idx[k]] == PP_OK) status[idx[k]] = st;
    };
    BatchBufs bb;
    bb.h = h0;
    bb.ctr = static_cast<unsigned long long*>(dev_alloc(h0, sizeof(unsigned long long) * CTR_COUNT * n));
    bb.ps = static_cast<StepParams*>(dev_alloc(h0, sizeof(StepParams) * N_TIERS * n));
    bb.args = static_cast<SpillArgs*>(dev_alloc(h0, sizeof(SpillArgs) * 2 * n));
    bb.scratch = static_cast<unsigned char**>(dev_alloc(h0, sizeof(unsigned char*) * n));
    if (!bb.ctr || !bb.ps || !bb.args || !bb.scratch) {
        fail(h0, PP_ERR_NOMEM, "batch buffers allocation failed");
        finish_all(PP_ERR_NOMEM);
        for (int k = 0; k < n; ++k) handles[idx[k]]->st = saved[k];
        return;
    }
    std::vector<std::unique_ptr<Prop>> props(n);
    for (int k = 0; k < n; ++k) {
        props[k].reset(new Prop());
        const pp_batch_item& it = items[idx[k]];
        const pp_status st = prop_begin(*props[k], handles[idx[k]], it.n_terms, it.ox, it.oz, it.oc, it.eps,
                                        it.w_max, bb.ctr + (size_t)CTR_COUNT * k, true);
        if (st != PP_OK) {
            status[idx[k]] = st;
            props[k]->finished = true;
        } else if (props[k]->S == 0) {
            prop_end(*props[k]);
        }
    }
    const bool f32 = h0->opt.precision == PP_PRECISION_FP32;
    std::vector<StepParams> ps_host((size_t)N_TIERS * n);
    std::vector<SpillArgs> args_host((size_t)2 * n);
    std::vector<unsigned char*> scratch_host(n);
    std::vector<unsigned long long> ctr_host((size_t)CTR_COUNT * n);
    std::vector<int> act;
    for (;;) {
        act.clear();
        for (int k = 0; k < n; ++k)
            if (!props[k]->finished) act.push_back(k);
        if (act.empty()) break;
        const int m = (int)act.size();
        PP_RANGE_PUSH("pp lockstep step");
        pp_status bad = PP_OK;
        uint32_t max_zero = 1;
        for (int a = 0; a < m; ++a) {
            Prop& P = *props[act[a]];
            prop_setup(P);
            pp_handle* hk = P.h;
            const bool fin = hk->subs[P.s].final_ != 0;
            SpillArgs z{};
            z.zero_fill = fin ? nullptr : hk->fill[P.side ^ 1];
            z.zero_n = fin ? 0 : P.nB;
            z.zero_shards = hk->spill_ctr;
            z.zero_ctr = P.ctr_dev;
            z.zero_ctr_n = CTR_COUNT;
            args_host[a] = z;
            max_zero = std::max(max_zero, z.zero_n);
            SpillArgs g{};
            g.fill = hk->fill[P.side ^ 1];
            g.nB = fin ? 0 : P.nB;
            g.C = P.nC;
            g.soff = hk->soff[P.side ^ 1];
            g.total = P.ctr_dev + CTR_SPILL_TOTAL;
            g.ctr = P.ctr_dev;
            g.dcap = hk->cap;
            g.rx = hk->spill_raw.x;
            g.rz = hk->spill_raw.z;
            g.rc = hk->spill_raw.c;
            g.rb = hk->spill_b;
            g.rs = hk->spill_s;
            g.rcap = hk->spill_cap;
            g.shard_fill = hk->spill_ctr;
            g.ox = hk->spill_grp.x;
            g.oz = hk->spill_grp.z;
            g.oc = hk->spill_grp.c;
            g.ocap = hk->spill_cap;
            args_host[m + a] = g;
            scratch_host[a] = hk->fb_scratch;
        }
        cudaError_t e = cudaMemcpyAsync(bb.args, args_host.data(), sizeof(SpillArgs) * 2 * m,
                                        cudaMemcpyHostToDevice, h0->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bb.scratch, scratch_host.data(), sizeof(unsigned char*) * m, cudaMemcpyHostToDevice,
                                h0->st);
        if (e == cudaSuccess) {
            k_clear<<<dim3((unsigned)std::min<uint32_t>((max_zero + 255) / 256, 4u * h0->sm_count), m), 256, 0,
                      h0->st>>>(bb.args);
            e = cudaGetLastError();
        }
        for (int a = 0; a < m && e == cudaSuccess; ++a)
            if (prop_noise(*props[act[a]]) != PP_OK) e = cudaErrorUnknown;
        for (int tier = 0; tier < N_TIERS && e == cudaSuccess; ++tier) {
            uint32_t bound = 1;
            for (int a = 0; a < m; ++a) {
                uint32_t ni;
                prop_tier(*props[act[a]], tier, &ni);
                bound = std::max(bound, ni);
                ps_host[(size_t)tier * n + a] = props[act[a]]->p;
            }
            e = cudaMemcpyAsync(bb.ps + (size_t)tier * n, ps_host.data() + (size_t)tier * n, sizeof(StepParams) * m,
                                cudaMemcpyHostToDevice, h0->st);
            if (e != cudaSuccess) break;
            LaunchRows rows;
            rows.ps = bb.ps + (size_t)tier * n;
            rows.n = m;
            rows.scratch_of = bb.scratch;
            int dummy = 0;
            e = dispatch_process(h0, props[act[0]]->p, tier, false, bound, &dummy, rows);
        }
        if (e == cudaSuccess) {
            if (h0->W == 1) {
                if (f32) launch_spill_batch<1, float>(h0, bb.args + m, m);
                else launch_spill_batch<1, double>(h0, bb.args + m, m);
            } else {
                if (f32) launch_spill_batch<2, float>(h0, bb.args + m, m);
                else launch_spill_batch<2, double>(h0, bb.args + m, m);
            }
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            // the active instances' counters are scattered over the batch array
            e = cudaMemcpyAsync(ctr_host.data(), bb.ctr, sizeof(unsigned long long) * CTR_COUNT * n,
                                cudaMemcpyDeviceToHost, h0->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h0->st);
        PP_RANGE_POP();
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(h, PP_ERR_CUDA, "lockstep batch step failed: %s", cudaGetErrorString(e));
            bad = PP_ERR_CUDA;
        }
        for (int a = 0; a < m; ++a) {
            Prop& P = *props[act[a]];
            if (bad != PP_OK) {
                status[idx[act[a]]] = bad;
                P.finished = true;
                continue;
            }
            const size_t k = (size_t)act[a];
            std::memcpy(P.ctr, ctr_host.data() + (size_t)CTR_COUNT * k, sizeof(P.ctr));
            P.launches += 2 + N_TIERS;   // this instance's rows of the step's launches
            const pp_status st = prop_finish(P);
            if (st != PP_OK) {
                status[idx[act[a]]] = st;
                P.finished = true;
            } else if (P.s == P.S) {
                prop_end(P);
            }
        }
    }
    cudaStreamSynchronize(h0->st);
    for (int k = 0; k < n; ++k) handles[idx[k]]->st = saved[k];
}

}  // namespace

extern "C" {

void pp_default_options(pp_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = PP_PRECISION_FP64;
}

pp_status pp_create(const pp_options* opt, int n_qubits, pp_handle** out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > MAXW * 64) return PP_ERR_ARG;
    pp_handle* h = new pp_handle();
    if (opt) h->opt = *opt;
    else pp_default_options(&h->opt);
    if (h->opt.precision != PP_PRECISION_FP32) h->opt.precision = PP_PRECISION_FP64;
    h->n = n_qubits;
    h->W = (n_qubits + 63) / 64;
    h->timing = h->opt.timing != 0;
    h->st = static_cast<cudaStream_t>(h->opt.cuda_stream);
    h->device = 0;
    int dev = 0;
    int optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return PP_ERR_CUDA;
    }
    h->device = dev;
    h->smem_optin = (size_t)optin;
    *out = h;
    return PP_OK;
}

pp_status pp_destroy(pp_handle* h) {
    if (!h) return PP_OK;
    cudaStreamSynchronize(h->st);
    std::vector<void*> all = h->owned;
    for (void* p : all) dev_free(h, p);
    for (auto& pr : h->tier_ev)
        for (auto& e : pr)
            if (e) cudaEventDestroy(e);
    delete h;
    return PP_OK;
}

const char* pp_last_error(const pp_handle* h) { return h ? h->err.c_str() : "null handle"; }

pp_status pp_set_tuning(pp_handle* h, const pp_tuning* t) {
    if (!h || !t) return PP_ERR_ARG;
    h->err.clear();
    if (t->max_fused_gates < 0 || t->max_fused_gates > 64 * h->W)
        return fail(h, PP_ERR_ARG, "max_fused_gates must be 0 (default) or 1..64*W");
    if (t->bucket_headroom != 0.0 && !(t->bucket_headroom >= 1.0 && t->bucket_headroom <= 16.0))
        return fail(h, PP_ERR_ARG, "bucket_headroom must be 0 (default) or in [1, 16]");
    if (t->first_tier < 0 || t->first_tier >= N_TIERS) return fail(h, PP_ERR_ARG, "first_tier must be in 0..4");
    if (t->orbit_tiles != 0 && t->orbit_tiles != 1) return fail(h, PP_ERR_ARG, "orbit_tiles must be 0 or 1");
    for (int tier = 0; tier < kGlobalTier; ++tier) {
        const int c = t->tile_cap[tier];
        if (c == 0) continue;
        if (c < 64 || c > 8192) return fail(h, PP_ERR_ARG, "tile_cap[%d] must be 0 (default) or 64..8192", tier);
        const size_t need = tile_smem_bytes(h, tier, c);
        if (need > h->smem_optin)
            return fail(h, PP_ERR_ARG, "tile_cap[%d] = %d needs %zu bytes of shared memory per CTA (device: %zu)",
                        tier, c, need, h->smem_optin);
    }
    if (t->max_fused_gates != h->tune.max_fused_gates || t->orbit_tiles != h->tune.orbit_tiles) h->subs_dirty = true;
    h->tune = *t;
    return PP_OK;
}

pp_status pp_cancel(pp_handle* h) {
    if (!h) return PP_ERR_ARG;
    h->cancel_gen.store(h->run_gen.load());
    return PP_OK;
}

pp_status pp_set_top_k(pp_handle* h, size_t top_k) {
    if (!h) return PP_ERR_ARG;
    h->err.clear();
    if (top_k != h->top_k) h->subs_dirty = true;
    h->top_k = top_k;
    return PP_OK;
}

pp_status pp_get_tuning(const pp_handle* h, pp_tuning* t) {
    if (!h || !t) return PP_ERR_ARG;
    t->max_fused_gates = max_fused_gates(h);
    t->bucket_headroom = bucket_headroom(h);
    t->first_tier = h->tune.first_tier;
    t->orbit_tiles = h->tune.orbit_tiles;
    for (int tier = 0; tier < kGlobalTier; ++tier) t->tile_cap[tier] = tier_cap(h, tier);
    return PP_OK;
}

pp_status pp_load_circuit(pp_handle* h, size_t n_gates, const uint64_t* rx, const uint64_t* rz,
                          const double* theta, const int32_t* layer_of, int n_layers) {
    if (!h) return PP_ERR_ARG;
    h->err.clear();
    if (n_gates && (!rx || !rz || !theta || !layer_of)) return fail(h, PP_ERR_ARG, "null gate arrays");
    if (n_layers < 1) return fail(h, PP_ERR_ARG, "n_layers must be >= 1");
    const int W = h->W, n = h->n;
    for (size_t g = 0; g < n_gates; ++g) {
        if (layer_of[g] < 0 || layer_of[g] >= n_layers)
            return fail(h, PP_ERR_ARG, "gate %zu: layer %d out of [0,%d)", g, layer_of[g], n_layers);
        if (!std::isfinite(theta[g])) return fail(h, PP_ERR_ARG, "gate %zu: angle not finite", g);
        int wt = 0;
        for (int w = 0; w < W; ++w) {
            uint64_t sup = rx[g * W + w] | rz[g * W + w];
            if (w == W - 1 && (n % 64) && (sup >> (n % 64)))
                return fail(h, PP_ERR_ARG, "gate %zu acts beyond qubit %d", g, n - 1);
            wt += __builtin_popcountll(sup);
        }
        if (wt == 0) return fail(h, PP_ERR_ARG, "gate %zu: identity generator", g);
    }
    // gates of one layer must pairwise commute
    std::vector<std::vector<size_t>> by_layer(n_layers);
    for (size_t g = 0; g < n_gates; ++g) by_layer[layer_of[g]].push_back(g);
    for (int l = 0; l < n_layers; ++l) {
        const auto& gl = by_layer[l];
        for (size_t i = 0; i < gl.size(); ++i)
            for (size_t j = i + 1; j < gl.size(); ++j) {
                int s = 0;
                for (int w = 0; w < W; ++w)
                    s += __builtin_popcountll((rx[gl[i] * W + w] & rz[gl[j] * W + w]) ^
                                              (rz[gl[i] * W + w] & rx[gl[j] * W + w]));
                if (s & 1)
                    return fail(h, PP_ERR_ARG, "gates %zu and %zu of layer %d do not commute", gl[i], gl[j], l);
            }
    }
    h->gx.assign(rx, rx + n_gates * W);
    h->gz.assign(rz, rz + n_gates * W);
    h->theta.assign(theta, theta + n_gates);
    h->layer_of.assign(layer_of, layer_of + n_gates);
    h->n_layers = n_layers;
    h->noise.clear();
    h->have_circuit = true;
    h->have_result = false;
    h->subs_dirty = true;
    return PP_OK;
}

pp_status pp_load_noise(pp_handle* h, int layer, size_t n_gen, const uint64_t* ex, const uint64_t* ez,
                        const double* lambda, int mode) {
    if (!h) return PP_ERR_ARG;
    h->err.clear();
    if (!h->have_circuit) return fail(h, PP_ERR_STATE, "load the circuit before its noise");
    if (layer < 0 || layer >= h->n_layers) return fail(h, PP_ERR_ARG, "layer %d out of range", layer);
    if (mode != PP_NOISE_INVERSE && mode != PP_NOISE_FORWARD) return fail(h, PP_ERR_ARG, "bad noise mode");
    if (n_gen && (!ex || !ez || !lambda)) return fail(h, PP_ERR_ARG, "null generator arrays");
    const int W = h->W, n = h->n;
    NoiseHost nh;
    nh.mode = mode;
    nh.n = n;
    std::vector<int64_t> t1((size_t)n * 4, 0);   // [n][4] per-site sums, by letter on the site
    std::map<std::pair<int, int>, int> pid;
    std::vector<std::pair<int, int>> pairs;
    std::vector<int64_t> t2;            // [P][16] sum over 2-local generators on the pair
    double total = 0.0;
    // anticommutation of single-qubit letters (code x + 2z) by the symplectic form
    auto anti1 = [](int l, int e) { return ((l & 1) & (e >> 1)) ^ ((l >> 1) & (e & 1)); };
    for (size_t k = 0; k < n_gen; ++k) {
        const uint64_t* x = ex + k * W;
        const uint64_t* z = ez + k * W;
        if (!(lambda[k] >= 0.0) || !std::isfinite(lambda[k]))
            return fail(h, PP_ERR_ARG, "generator %zu: rate must be finite and >= 0", k);
        total += lambda[k];
        int64_t lf = (int64_t)std::llround(std::ldexp(lambda[k], FIX_SHIFT));
        std::vector<int> sites;
        for (int q = 0; q < n; ++q)
            if (bit(x, q) | bit(z, q)) sites.push_back(q);
        for (int w = 0; w < W; ++w) {
            uint64_t sup = x[w] | z[w];
            if (w == W - 1 && (n % 64) && (sup >> (n % 64)))
                return fail(h, PP_ERR_ARG, "generator %zu acts beyond qubit %d", k, n - 1);
        }
        if (sites.size() == 1) {
            int q = sites[0];
            int e = bit(x, q) + 2 * bit(z, q);
            for (int l = 1; l < 4; ++l)
                if (anti1(l, e)) t1[4 * q + l] += lf;
        } else if (sites.size() == 2) {
            int a = sites[0], b = sites[1];
            auto key = std::make_pair(a, b);
            int id;
            auto it = pid.find(key);
            if (it == pid.end()) {
                id = (int)pairs.size();
                pid[key] = id;
                pairs.push_back(key);
                t2.resize(t2.size() + 16, 0);
            } else {
                id = it->second;
            }
            int ea = bit(x, a) + 2 * bit(z, a), eb = bit(x, b) + 2 * bit(z, b);
            for (int la = 0; la < 4; ++la)
                for (int lb = 0; lb < 4; ++lb)
                    if (anti1(la, ea) ^ anti1(lb, eb)) t2[16 * id + la + 4 * lb] += lf;
        } else if (sites.size() > 2) {
            nh.gx.insert(nh.gx.end(), x, x + W);
            nh.gz.insert(nh.gz.end(), z, z + W);
            nh.glam.push_back(lf);
        }
    }
    if (total >= 60.0) return fail(h, PP_ERR_ARG, "sum of rates %.3g too large (must be < 60)", total);
    if (h->opt.precision == PP_PRECISION_FP32 && total >= 40.0)
        return fail(h, PP_ERR_ARG, "sum of rates %.3g too large for the FP32 form (must be < 40)", total);
    // Fold each pair's one-sided terms (the other site carries I) into the
    // per-site table; keep, per pair, the correction for strings that hold a
    // non-identity letter on both sites:
    //   T2[la,lb] = T2[la,I] + T2[I,lb] + C[la,lb]   (exact integers).
    std::vector<int64_t> corr(16 * pairs.size(), 0);
    for (size_t i = 0; i < pairs.size(); ++i) {
        const int a = pairs[i].first, b = pairs[i].second;
        const int64_t* T = &t2[16 * i];
        for (int l = 1; l < 4; ++l) {
            t1[4 * a + l] += T[l];          // (l, I)
            t1[4 * b + l] += T[4 * l];      // (I, l)
        }
        for (int la = 1; la < 4; ++la)
            for (int lb = 1; lb < 4; ++lb)
                corr[16 * i + la + 4 * lb] = T[la + 4 * lb] - T[la] - T[4 * lb];
    }
    // Group tables over sites 4g..4g+3, indexed by the group's x nibble | z
    // nibble << 4: the per-site terms of the four letters, plus the correction
    // of every pair inside the group.  The exponent is a sum of exact integers,
    // so this regrouping leaves it unchanged.
    const int ng = (n + 3) / 4;
    auto letter = [](int idx, int j) { return ((idx >> j) & 1) + 2 * ((idx >> (4 + j)) & 1); };
    nh.grp.assign((size_t)ng * 256, 0);
    for (int g = 0; g < ng; ++g)
        for (int idx = 0; idx < 256; ++idx) {
            int64_t v = 0;
            for (int j = 0; j < 4 && 4 * g + j < n; ++j) v += t1[4 * (4 * g + j) + letter(idx, j)];
            nh.grp[256 * (size_t)g + idx] = v;
        }
    // Pairs across groups keep their correction, reached through the shift
    // class of the pair and its first site.
    std::map<int, int> shift_class;
    for (size_t i = 0; i < pairs.size(); ++i) {
        const int a = pairs[i].first, b = pairs[i].second;
        if ((a >> 2) == (b >> 2)) {
            const int g = a >> 2;
            for (int idx = 0; idx < 256; ++idx)
                nh.grp[256 * (size_t)g + idx] += corr[16 * i + letter(idx, a & 3) + 4 * letter(idx, b & 3)];
            continue;
        }
        const int d = b - a;
        auto it = shift_class.find(d);
        int c;
        if (it == shift_class.end()) {
            c = (int)nh.shift.size();
            shift_class[d] = c;
            nh.shift.push_back(d);
            nh.xmask.resize(nh.xmask.size() + W, 0);
            nh.pidx.resize(nh.pidx.size() + n, -1);
        } else {
            c = it->second;
        }
        nh.xmask[(size_t)c * W + (a >> 6)] |= 1ull << (a & 63);
        nh.pidx[(size_t)c * n + a] = (int32_t)(nh.c2.size() / 16);
        nh.c2.insert(nh.c2.end(), corr.begin() + 16 * i, corr.begin() + 16 * (i + 1));
    }
    {
        // the streaming pass stages every table in one CTA's shared memory
        const size_t need = noise_smem_layout(n, ng, (int)nh.shift.size(), (int)(nh.c2.size() / 16), W).bytes;
        if (need > h->smem_optin)
            return fail(h, PP_ERR_ARG,
                        "noise map on layer %d: its tables need %zu bytes of shared memory (device: %zu); "
                        "%zu of its generator pairs cross 4-site groups",
                        layer, need, h->smem_optin, nh.c2.size() / 16);
    }
    h->noise.erase(layer);
    // factor tables: entry (i, b) = exp(+-2 * b * 2^(8i - 56)), evaluated in extended
    // precision and rounded once to double, and as a float (head, tail) pair: the
    // head rounded to float, the tail the rounded remainder.  Entries beyond the
    // float range (byte 7 above 44, unreachable under the rate limit of the FP32
    // form) saturate.
    nh.etab.assign(8 * 256, 1.0);
    nh.ftab.assign(8 * 256 * 2, 0.0f);
    for (int i = 0; i < 8; ++i)
        for (int b = 0; b < 256; ++b) {
            const long double e = std::ldexp((long double)b, 8 * i - FIX_SHIFT) * 2.0L;
            const long double v = std::exp(mode == PP_NOISE_INVERSE ? e : -e);
            nh.etab[256 * i + b] = (double)v;
            float hd = std::numeric_limits<float>::max(), tl = 0.0f;
            if (v < (long double)std::numeric_limits<float>::max()) {
                hd = (float)v;
                tl = (float)(v - (long double)hd);
            }
            nh.ftab[2 * (256 * i + b)] = hd;
            nh.ftab[2 * (256 * i + b) + 1] = tl;
        }
    h->noise[layer] = std::move(nh);
    h->have_result = false;
    h->subs_dirty = true;
    return PP_OK;
}

pp_status pp_propagate(pp_handle* h, size_t n_terms, const uint64_t* ox, const uint64_t* oz,
                       const double* oc, double eps, int w_max) {
    if (!h) return PP_ERR_ARG;
    Prop P;
    pp_status st = prop_begin(P, h, n_terms, ox, oz, oc, eps, w_max, h->counters, false);
    if (st != PP_OK) return st;
    // One host synchronisation per sub-layer: the tiers after the first read
    // their work counts from the device (the previous tier's deferral
    // counter), the overflow grouping always runs, and the counters come back
    // in one copy at the end.
    while (P.s < P.S) {
        if ((st = prop_setup(P)) != PP_OK) return st;
        PP_RANGE_PUSH("pp sub-layer");
        const bool fin = h->subs[P.s].final_ != 0;
        if (!fin) CK(cudaMemsetAsync(h->fill[P.side ^ 1], 0, sizeof(uint32_t) * P.nB, h->st));
        CK(cudaMemsetAsync(P.ctr_dev, 0, sizeof(unsigned long long) * CTR_COUNT, h->st));
        CK(cudaMemsetAsync(h->spill_ctr, 0, sizeof(unsigned long long) * NSPILL, h->st));
        if ((st = prop_noise(P)) != PP_OK) return st;
        for (int tier = 0; tier < N_TIERS; ++tier) {
            uint32_t n_items;
            const bool orbit = prop_tier(P, tier, &n_items);
            if (h->timing) CK(cudaEventRecord(h->tier_ev[tier][0], h->st));
            CK(dispatch_process(h, P.p, tier, orbit, n_items, &P.launches));
            if (h->timing) CK(cudaEventRecord(h->tier_ev[tier][1], h->st));
        }
        if (!fin) CK(group_spill(h, P.side ^ 1, P.nB, P.nC, P.ctr_dev, &P.launches));
        CK(cudaMemcpyAsync(P.ctr, P.ctr_dev, sizeof(P.ctr), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        PP_RANGE_POP();
        if (h->timing)
            for (int tier = 0; tier < N_TIERS; ++tier)
                CK(cudaEventElapsedTime(&P.ms[tier], h->tier_ev[tier][0], h->tier_ev[tier][1]));
        if ((st = prop_finish(P)) != PP_OK) return st;
    }
    prop_end(P);
    return PP_OK;
}

pp_status pp_expect(pp_handle* h, double* value) {
    if (!h || !value) return PP_ERR_ARG;
    h->err.clear();
    if (!h->have_result) return fail(h, PP_ERR_STATE, "no propagation result");
    const Arena& a = h->arena[h->res_side];
    int grid = (int)std::min<size_t>(std::max<size_t>((h->n_res + 255) / 256, 1), 4096);
    if (h->opt.precision == PP_PRECISION_FP32) {
        if (h->W == 1) k_expect<1, float><<<grid, 256, 0, h->st>>>(a.x, (const float*)a.c, h->cap, h->n_res, h->partial);
        else k_expect<2, float><<<grid, 256, 0, h->st>>>(a.x, (const float*)a.c, h->cap, h->n_res, h->partial);
    } else {
        if (h->W == 1) k_expect<1, double><<<grid, 256, 0, h->st>>>(a.x, (const double*)a.c, h->cap, h->n_res, h->partial);
        else k_expect<2, double><<<grid, 256, 0, h->st>>>(a.x, (const double*)a.c, h->cap, h->n_res, h->partial);
    }
    CK(cudaGetLastError());
    k_expect_final<<<1, 256, 0, h->st>>>(h->partial, grid);
    CK(cudaGetLastError());
    __int128 tot = 0;
    CK(cudaMemcpyAsync(&tot, h->partial + grid, sizeof(__int128), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    // the exact fixed-point total (units of 2^-80), rounded once to double
    *value = fixed80_to_double(tot);
    return PP_OK;
}

pp_status pp_export_terms(pp_handle* h, size_t cap, uint64_t* x, uint64_t* z, double* c, size_t* n_out) {
    if (!h || !n_out) return PP_ERR_ARG;
    h->err.clear();
    if (!h->have_result) return fail(h, PP_ERR_STATE, "no propagation result");
    *n_out = h->n_res;
    if (!x && !z && !c) return PP_OK;
    if (cap < h->n_res) return fail(h, PP_ERR_CAPACITY, "export buffer holds %zu < %zu terms", cap, h->n_res);
    const size_t N = h->n_res;
    const int W = h->W;
    if (N >= (1ull << 32)) return fail(h, PP_ERR_CAPACITY, "export of %zu terms: at most 2^32 - 1", N);
    if (N > 1) {
        const bool f32 = h->opt.precision == PP_PRECISION_FP32;
        pp_status st = W == 1 ? (f32 ? sort_result<1, float>(h) : sort_result<1, double>(h))
                              : (f32 ? sort_result<2, float>(h) : sort_result<2, double>(h));
        if (st != PP_OK) return st;
    }
    const Arena& a = h->arena[h->res_side];
    std::vector<uint64_t> hx(N * W), hz(N * W);
    std::vector<double> hc(N);
    for (int w = 0; w < W; ++w) {
        CK(cudaMemcpyAsync(hx.data() + w * N, a.x + (size_t)w * h->cap, N * 8, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(hz.data() + w * N, a.z + (size_t)w * h->cap, N * 8, cudaMemcpyDeviceToHost, h->st));
    }
    if (h->opt.precision == PP_PRECISION_FP32) {
        std::vector<float> hf(N);
        CK(cudaMemcpyAsync(hf.data(), a.c, N * 4, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        for (size_t i = 0; i < N; ++i) hc[i] = hf[i];
    } else {
        CK(cudaMemcpyAsync(hc.data(), a.c, N * 8, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
    }
    // word-major device layout to the caller's [N][W] rows
    for (size_t k = 0; k < N; ++k) {
        for (int w = 0; w < W; ++w) {
            if (x) x[k * W + w] = hx[w * N + k];
            if (z) z[k * W + w] = hz[w * N + k];
        }
        if (c) c[k] = hc[k];
    }
    return PP_OK;
}

pp_status pp_propagate_batch(int n, pp_handle* const* handles, const pp_batch_item* items, int max_threads,
                             pp_status* status_out) {
    if (n < 0 || (n > 0 && (!handles || !items))) return PP_ERR_ARG;
    bool bad = false;
    for (int i = 0; i < n; ++i)
        if (!handles[i]) bad = true;
    // a handle may appear once: its layouts hold one propagation
    std::vector<const pp_handle*> sorted(handles, handles + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) bad = true;
    if (bad) {
        if (status_out)
            for (int i = 0; i < n; ++i) status_out[i] = PP_ERR_ARG;
        return PP_ERR_ARG;
    }
    std::vector<pp_status> st(n, PP_OK);
    // Handles that share a device, a mask width and a precision run in lockstep
    // (run_lockstep); the groups run one after another.
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i)
        groups[std::make_tuple(handles[i]->device, handles[i]->W, handles[i]->opt.precision)].push_back(i);
    (void)max_threads;   // lockstep groups need no host threads
    for (auto& kv : groups) {
        if (cudaSetDevice(std::get<0>(kv.first)) != cudaSuccess) {
            cudaGetLastError();
            for (int i : kv.second) st[i] = PP_ERR_CUDA;
            continue;
        }
        run_lockstep(handles, items, kv.second, st);
    }
    pp_status first = PP_OK;
    for (int i = 0; i < n; ++i) {
        if (status_out) status_out[i] = st[i];
        if (first == PP_OK && st[i] != PP_OK) first = st[i];
    }
    return first;
}

pp_status pp_get_stats(const pp_handle* h, pp_stats* out) {
    if (!h || !out) return PP_ERR_ARG;
    *out = h->stats;
    return PP_OK;
}

}  // extern "C"
