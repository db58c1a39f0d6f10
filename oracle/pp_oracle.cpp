/*
 * CPU ORACLE for noisy-inverse Pauli propagation.  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Plain, slow, obviously correct FP64 reference.  The observable is a hash map
 * from a Pauli string (x words, z words) to a real coefficient; every step of the
 * backward (Heisenberg) propagation is applied one gate at a time:
 *
 *   for layer l = L-1 .. 0:
 *     - if a noise channel follows layer l in time: multiply every coefficient by
 *       exp(+2 * sum of lambda_k over generators E_k that anticommute with the
 *       string) (inverse map, Sec. I Eq. evolve_noise with 1-2q = e^{+2 lambda};
 *       App. G Eq. evolve_noise_fid), or by exp(-2 * ...) for the physical
 *       channel; then drop terms under the threshold;
 *     - for each gate of layer l in listed order, U = exp(-i theta R / 2): every
 *       string P that anticommutes with R contributes cos(theta) c to P and
 *       sin(theta) c phi to the string Q with i R P = phi Q (phi = +-1), the
 *       Heisenberg form U^dag P U = (cos theta + i sin theta R) P of Eq.
 *       evolve_gate (App. G); commuting strings pass unchanged; contributions are
 *       summed into a fresh map, which is then truncated.
 *   truncation (Sec. I.A): drop c == 0, |c| < eps, and Pauli weight > w_max.
 *   expectation on |0..0>: sum of c over strings with no X or Y letter.
 *
 * Paper readings it follows (silent points): truncation after every gate and
 * after every noise layer, on merged coefficients; strict |c| < eps; angles
 * whose cosine (sine) has magnitude below 1e-15 use exactly 0 and +-1.
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

const int MAXW = 2;   // up to 128 qubits

struct Key {
    uint64_t x[MAXW];
    uint64_t z[MAXW];
    bool operator==(const Key& o) const {
        for (int w = 0; w < MAXW; ++w)
            if (x[w] != o.x[w] || z[w] != o.z[w]) return false;
        return true;
    }
};

struct KeyHash {
    size_t operator()(const Key& k) const {
        uint64_t h = 0x12345678abcdefULL;
        for (int w = 0; w < MAXW; ++w) {
            h = (h ^ k.x[w]) * 0x100000001b3ULL;
            h ^= h >> 29;
            h = (h ^ k.z[w]) * 0x100000001b3ULL;
            h ^= h >> 31;
        }
        return (size_t)h;
    }
};

typedef std::unordered_map<Key, double, KeyHash> Sum;

// Single-qubit letters.
enum { LI = 0, LX = 1, LY = 2, LZ = 3 };

int letter(const Key& p, int q) {
    int bx = (int)((p.x[q / 64] >> (q % 64)) & 1ULL);
    int bz = (int)((p.z[q / 64] >> (q % 64)) & 1ULL);
    if (bx && !bz) return LX;
    if (bx && bz) return LY;
    if (!bx && bz) return LZ;
    return LI;
}

void set_letter(Key& p, int q, int L) {
    uint64_t bit = 1ULL << (q % 64);
    p.x[q / 64] &= ~bit;
    p.z[q / 64] &= ~bit;
    if (L == LX || L == LY) p.x[q / 64] |= bit;
    if (L == LZ || L == LY) p.z[q / 64] |= bit;
}

// Product of two single-qubit Paulis a*b = i^PHASE[a][b] * LETTER[a][b]:
// XY = iZ, YZ = iX, ZX = iY and the reversed orders with -i.
const int PROD_LETTER[4][4] = {
    /* I */ {LI, LX, LY, LZ},
    /* X */ {LX, LI, LZ, LY},
    /* Y */ {LY, LZ, LI, LX},
    /* Z */ {LZ, LY, LX, LI},
};
const int PROD_PHASE[4][4] = {
    /* I */ {0, 0, 0, 0},
    /* X */ {0, 0, 1, 3},   // XY = iZ, XZ = -iY
    /* Y */ {0, 3, 0, 1},   // YX = -iZ, YZ = iX
    /* Z */ {0, 1, 3, 0},   // ZX = iY, ZY = -iX
};

// Symplectic product <P,R>: 1 if the strings anticommute, counted qubit by qubit.
int anticommute(const Key& p, const Key& r, int n) {
    int cnt = 0;
    for (int q = 0; q < n; ++q) {
        int a = letter(p, q), b = letter(r, q);
        if (a != LI && b != LI && a != b) ++cnt;
    }
    return cnt & 1;
}

// Multiply r * p (r on the left): returns the string and the power of i.
Key multiply(const Key& r, const Key& p, int n, int* phase) {
    Key out;
    std::memset(&out, 0, sizeof(out));
    int ph = 0;
    for (int q = 0; q < n; ++q) {
        int a = letter(r, q), b = letter(p, q);
        ph += PROD_PHASE[a][b];
        set_letter(out, q, PROD_LETTER[a][b]);
    }
    *phase = ph % 4;
    return out;
}

int weight(const Key& p, int W) {
    int w = 0;
    for (int i = 0; i < W; ++i) w += __builtin_popcountll(p.x[i] | p.z[i]);
    return w;
}

bool supports_overlap(const Key& a, const Key& b, int W) {
    for (int i = 0; i < W; ++i)
        if ((a.x[i] | a.z[i]) & (b.x[i] | b.z[i])) return true;
    return false;
}

Key load_key(const uint64_t* xs, const uint64_t* zs, size_t idx, int W) {
    Key k;
    std::memset(&k, 0, sizeof(k));
    for (int w = 0; w < W; ++w) {
        k.x[w] = xs[idx * W + w];
        k.z[w] = zs[idx * W + w];
    }
    return k;
}

bool key_less(const Key& a, const Key& b) {
    for (int w = MAXW - 1; w >= 0; --w)
        if (a.x[w] != b.x[w]) return a.x[w] < b.x[w];
    for (int w = MAXW - 1; w >= 0; --w)
        if (a.z[w] != b.z[w]) return a.z[w] < b.z[w];
    return false;
}

}  // namespace

extern "C" {

typedef struct {
    int n_qubits;
    int n_layers;
    int64_t n_gates;
    const uint64_t* gx;
    const uint64_t* gz;
    const double* theta;
    const int32_t* layer_of;
    int n_noise;
    const int32_t* noise_layer;
    const int64_t* noise_off;   // n_noise + 1 offsets into ex/ez/lam
    const uint64_t* ex;
    const uint64_t* ez;
    const double* lam;
    const int32_t* noise_mode;  // per noise layer: 0 exp(+2 sum), 1 exp(-2 sum)
    int64_t n_obs;
    const uint64_t* ox;
    const uint64_t* oz;
    const double* oc;
    double eps;
    int w_max;                  // < 0: no cap
    int record;                 // record per-gate mass bookkeeping
    int64_t top_k;              // > 0: keep at most this many terms after each layer
} orc_problem;

typedef struct {
    std::vector<Key>* keys;
    std::vector<double>* coef;
    double expect;
    double updates;            // sum over gates of the live-term count entering the gate
    int64_t peak;
    std::vector<double>* records;   // per gate: [mass_in, mass_rotated, mass_kept, mass_dropped]
    int W;
    char err[128];
} orc_result;

static bool keep(double c, const Key& k, double eps, int w_max, int W) {
    if (c == 0.0) return false;
    if (std::fabs(c) < eps) return false;
    if (w_max >= 0 && weight(k, W) > w_max) return false;
    return true;
}

// Top-K truncation (Sec. I.A: keep at most the K largest Pauli terms of an
// intermediate result), applied to the input observable and after the gates
// of every layer.  Terms are ranked by |c| descending; equal magnitudes are
// ranked by the string, in the export order (x words from the most
// significant, then z words), smallest first; the first K are kept.
static void keep_top_k(Sum& cur, int64_t k) {
    if (k <= 0 || (int64_t)cur.size() <= k) return;
    std::vector<std::pair<Key, double>> all(cur.begin(), cur.end());
    std::sort(all.begin(), all.end(), [](const std::pair<Key, double>& a, const std::pair<Key, double>& b) {
        const double ma = std::fabs(a.second), mb = std::fabs(b.second);
        if (ma != mb) return ma > mb;
        return key_less(a.first, b.first);
    });
    cur.clear();
    for (int64_t i = 0; i < k; ++i) cur.insert(all[(size_t)i]);
}

static void trig(double theta, double* c, double* s) {
    *c = std::cos(theta);
    *s = std::sin(theta);
    if (std::fabs(*c) < 1e-15) { *c = 0.0; *s = (*s > 0) ? 1.0 : -1.0; }
    if (std::fabs(*s) < 1e-15) { *s = 0.0; *c = (*c > 0) ? 1.0 : -1.0; }
}

orc_result* orc_run(const orc_problem* pb) {
    orc_result* res = new orc_result();
    res->keys = new std::vector<Key>();
    res->coef = new std::vector<double>();
    res->records = new std::vector<double>();
    res->err[0] = 0;
    const int n = pb->n_qubits;
    const int W = (n + 63) / 64;
    res->W = W;
    if (n < 1 || W > MAXW) {
        std::snprintf(res->err, sizeof(res->err), "n_qubits out of range");
        return res;
    }

    Sum cur;
    for (int64_t t = 0; t < pb->n_obs; ++t) cur[load_key(pb->ox, pb->oz, t, W)] += pb->oc[t];
    for (auto it = cur.begin(); it != cur.end();) {
        if (!keep(it->second, it->first, pb->eps, pb->w_max, W)) it = cur.erase(it);
        else ++it;
    }
    keep_top_k(cur, pb->top_k);
    double updates = 0.0;
    int64_t peak = (int64_t)cur.size();

    for (int l = pb->n_layers - 1; l >= 0; --l) {
        // Noise channel that follows layer l in time: applied first going backwards.
        for (int m = 0; m < pb->n_noise; ++m) {
            if (pb->noise_layer[m] != l) continue;
            for (auto it = cur.begin(); it != cur.end();) {
                double s = 0.0;
                for (int64_t k = pb->noise_off[m]; k < pb->noise_off[m + 1]; ++k) {
                    Key e = load_key(pb->ex, pb->ez, k, W);
                    if (!supports_overlap(e, it->first, W)) continue;
                    if (anticommute(it->first, e, n)) s += pb->lam[k];
                }
                double f = pb->noise_mode[m] == 0 ? std::exp(2.0 * s) : std::exp(-2.0 * s);
                it->second = it->second * f;
                if (!keep(it->second, it->first, pb->eps, pb->w_max, W)) it = cur.erase(it);
                else ++it;
            }
        }
        // Gates of layer l, in listed order.
        for (int64_t g = 0; g < pb->n_gates; ++g) {
            if (pb->layer_of[g] != l) continue;
            Key r = load_key(pb->gx, pb->gz, g, W);
            double cs, sn;
            trig(pb->theta[g], &cs, &sn);
            updates += (double)cur.size();
            double m_in = 0.0, m_rot = 0.0, m_keep = 0.0, m_drop = 0.0;
            Sum nxt;
            nxt.reserve(cur.size() * 2);
            for (const auto& kv : cur) {
                const Key& p = kv.first;
                double c = kv.second;
                if (pb->record) m_in += c * c;
                if (anticommute(p, r, n)) {
                    int ph = 0;
                    Key q = multiply(r, p, n, &ph);
                    int total = (1 + ph) % 4;   // i * (r p) = i^(1+ph) q
                    double phi;
                    if (total == 0) phi = 1.0;
                    else if (total == 2) phi = -1.0;
                    else { std::snprintf(res->err, sizeof(res->err), "non-real phase"); return res; }
                    nxt[p] += cs * c;
                    nxt[q] += (sn * c) * phi;
                } else {
                    nxt[p] += c;
                }
            }
            cur.clear();
            for (const auto& kv : nxt) {
                if (pb->record) m_rot += kv.second * kv.second;
                if (keep(kv.second, kv.first, pb->eps, pb->w_max, W)) {
                    cur.insert(kv);
                    if (pb->record) m_keep += kv.second * kv.second;
                } else if (pb->record) {
                    m_drop += kv.second * kv.second;
                }
            }
            if ((int64_t)cur.size() > peak) peak = (int64_t)cur.size();
            if (pb->record) {
                res->records->push_back(m_in);
                res->records->push_back(m_rot);
                res->records->push_back(m_keep);
                res->records->push_back(m_drop);
            }
        }
        keep_top_k(cur, pb->top_k);
    }

    std::vector<std::pair<Key, double>> out(cur.begin(), cur.end());
    std::sort(out.begin(), out.end(),
              [](const std::pair<Key, double>& a, const std::pair<Key, double>& b) {
                  return key_less(a.first, b.first);
              });
    double e = 0.0;
    for (const auto& kv : out) {
        bool diag = true;
        for (int w = 0; w < W; ++w)
            if (kv.first.x[w]) diag = false;
        if (diag) e += kv.second;
        res->keys->push_back(kv.first);
        res->coef->push_back(kv.second);
    }
    res->expect = e;
    res->updates = updates;
    res->peak = peak;
    return res;
}

const char* orc_error(const orc_result* r) { return r->err; }
int64_t orc_n_terms(const orc_result* r) { return (int64_t)r->keys->size(); }
double orc_expect(const orc_result* r) { return r->expect; }
double orc_updates(const orc_result* r) { return r->updates; }
int64_t orc_peak(const orc_result* r) { return r->peak; }
int64_t orc_n_records(const orc_result* r) { return (int64_t)r->records->size() / 4; }

void orc_terms(const orc_result* r, uint64_t* x, uint64_t* z, double* c) {
    const int W = r->W;
    for (size_t i = 0; i < r->keys->size(); ++i) {
        for (int w = 0; w < W; ++w) {
            x[i * W + w] = (*r->keys)[i].x[w];
            z[i * W + w] = (*r->keys)[i].z[w];
        }
        c[i] = (*r->coef)[i];
    }
}

void orc_records(const orc_result* r, double* out) {
    std::memcpy(out, r->records->data(), r->records->size() * sizeof(double));
}

void orc_free(orc_result* r) {
    if (!r) return;
    delete r->keys;
    delete r->coef;
    delete r->records;
    delete r;
}

// Single-string primitives, exposed so tests can pin the product table against
// dense matrices.
int orc_anticommute(int n, const uint64_t* px, const uint64_t* pz, const uint64_t* rx,
                    const uint64_t* rz) {
    const int W = (n + 63) / 64;
    return anticommute(load_key(px, pz, 0, W), load_key(rx, rz, 0, W), n);
}

int orc_multiply(int n, const uint64_t* rx, const uint64_t* rz, const uint64_t* px,
                 const uint64_t* pz, uint64_t* qx, uint64_t* qz) {
    const int W = (n + 63) / 64;
    int ph = 0;
    Key q = multiply(load_key(rx, rz, 0, W), load_key(px, pz, 0, W), n, &ph);
    for (int w = 0; w < W; ++w) {
        qx[w] = q.x[w];
        qz[w] = q.z[w];
    }
    return ph;
}

}  // extern "C"
