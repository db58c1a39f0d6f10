/*
 * pp.h -- C ABI of libpp: noisy-inverse Pauli propagation on one B300 GPU.
 *
 * The library propagates an observable O, held as a sum of bit-packed Pauli
 * strings, backwards (Heisenberg picture) through a circuit of Pauli rotations
 * U = exp(-i theta R / 2) and sparse Pauli-Lindblad noise maps, giving the
 * noise-canceling observable O~ and its value <0..0|O~|0..0>.
 *
 *   gate rule (Sec. I, Eq. evolve_gate; Heisenberg form in App. G):
 *       U^dag P U = cos(theta) P + i sin(theta) R P      if P, R anticommute
 *                 = P                                   otherwise
 *   inverse-noise rule (Sec. I, Eq. evolve_noise, with q = (1 - e^{2 lambda})/2,
 *   so 1 - 2q = e^{+2 lambda}; App. G, Eq. evolve_noise_fid):
 *       Lambda^{-1}(P) = exp(+2 * sum_{k: {P,E_k} = 0} lambda_k) P
 *   truncation (Sec. I.A): after every gate and every noise map, a string is
 *       dropped when its coefficient is 0, |c| < eps, or its Pauli weight
 *       exceeds w_max.
 *
 * Conventions
 *   Qubits: n_qubits <= 128.  W = ceil(n_qubits / 64) uint64 words per mask.
 *   A Pauli string is (x[W], z[W]): bit q of word q/64 is qubit q; letter
 *   (x,z) = (0,0) I, (1,0) X, (1,1) Y, (0,1) Z.  Strings are Hermitian and every
 *   sign lives in the real coefficient.  Arrays of strings are row-major
 *   [count][W].
 *   Time order: layer 0 is applied to the state first.  A layer is a set of
 *   pairwise-commuting rotations; the backward pass applies a layer's gates in
 *   the order they are listed (the order only matters through truncation).
 *   A noise map attached to layer l acts after layer l's gates in time, so the
 *   backward pass applies it before them.
 *
 * Ownership and errors
 *   Every pointer argument is a HOST pointer unless its name ends in _dev.  The
 *   library copies all inputs; the caller keeps ownership of its buffers.  The
 *   handle owns its device memory, obtained through pp_options.alloc (or
 *   cudaMalloc when NULL) and released by pp_destroy.  Every call returns a
 *   pp_status; PP_OK is 0.  On any other status the handle stays valid and
 *   pp_last_error() describes the failure; results of a failed pp_propagate are
 *   discarded.  Calls on one handle must not overlap; distinct handles are
 *   independent.
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_handle pp_handle;

typedef enum {
    PP_OK = 0,
    PP_ERR_ARG = 1,       /* invalid argument (sizes, layer indices, non-commuting layer) */
    PP_ERR_STATE = 2,     /* call out of order (e.g. pp_expect before pp_propagate)       */
    PP_ERR_NOMEM = 3,     /* device allocation failed                                      */
    PP_ERR_CAPACITY = 4,  /* live terms exceeded the handle's capacity                     */
    PP_ERR_CUDA = 5,      /* a CUDA runtime call failed                                    */
    PP_ERR_TIMEOUT = 6    /* the propagation was cancelled (pp_cancel) before it finished  */
} pp_status;

enum { PP_PRECISION_FP64 = 64, PP_PRECISION_FP32 = 32 };
enum { PP_NOISE_INVERSE = 0, PP_NOISE_FORWARD = 1 };

typedef struct {
    int precision;                 /* PP_PRECISION_FP64 (default) or PP_PRECISION_FP32:
                                      storage and branching type of coefficients; noise
                                      exponents and the final sum are always exact or FP64 */
    size_t max_terms;              /* largest live-term capacity per buffer; 0 = a quarter of
                                      the free device memory (re-read at each growth).  The
                                      buffers start at 2^16 terms (or 4x the observable) and
                                      grow during a propagation when a sub-layer's planned
                                      output would need more (pp_stats.growths, .capacity) */
    void* (*alloc)(size_t bytes, void* ctx);   /* device allocator; NULL = cudaMalloc */
    void (*free)(void* ptr, void* ctx);        /* matching release; NULL = cudaFree   */
    void* alloc_ctx;
    void* cuda_stream;             /* cudaStream_t to run on; NULL = the legacy default stream */
    int timing;                    /* 1: record each processing tier's device time per
                                      sub-layer (pp_stats.tier_ms; one CUDA event pair per
                                      tier launch); 0 (default): tier_ms stays 0 */
} pp_options;

/* Fills *opt with defaults (FP64, automatic capacity, cudaMalloc, default stream). */
void pp_default_options(pp_options* opt);

/* Creates a handle for n_qubits (1..128).  opt may be NULL (defaults).
 * Errors: PP_ERR_ARG (n_qubits out of range, out NULL), PP_ERR_CUDA. */
pp_status pp_create(const pp_options* opt, int n_qubits, pp_handle** out);

/* Releases the handle and all its device memory.  NULL is a no-op. */
pp_status pp_destroy(pp_handle* h);

/* Loads the circuit (Sec. I: time-ordered Pauli rotations U_t = exp(-i R_t theta_t / 2)).
 *   rx, rz     [n_gates][W] generator R of each gate
 *   theta      [n_gates]    rotation angle
 *   layer_of   [n_gates]    layer index of each gate, in [0, n_layers); any order:
 *                           a layer's gates are applied in the order they are listed
 *                           (layers without gates are allowed and may carry noise)
 *   n_layers   number of layers (>= 1); lets trailing layers be empty
 * Gates of one layer must pairwise commute (else PP_ERR_ARG).  Clears any
 * previously loaded noise.  cos/sin of each angle are taken on the host; values
 * with magnitude below 1e-15 snap to exactly 0 (and the other to +-1). */
pp_status pp_load_circuit(pp_handle* h, size_t n_gates, const uint64_t* rx, const uint64_t* rz,
                          const double* theta, const int32_t* layer_of, int n_layers);

/* Attaches a sparse Pauli-Lindblad noise map after `layer` in time (Sec. I,
 * Lambda_t = composition of (1-p) . + p E . E with p = (1 - e^{-2 lambda})/2).
 *   ex, ez   [n_gen][W] generators E_k;  lambda [n_gen] rates, >= 0
 *   mode     PP_NOISE_INVERSE: coefficients scale by exp(+2 sum lambda) (antinoise);
 *            PP_NOISE_FORWARD: by exp(-2 sum lambda) (the physical channel)
 * The sum of the map's rates must be below 60 (below 40 on an FP32 handle, so
 * that every factor stays within float range), and its tables must fit one
 * CTA's shared memory: 16 KB, plus 2 KB per group of 4 sites, plus 128 B per
 * 2-site generator support whose sites lie in different groups, plus 4n + 8W B
 * per distinct distance between the two sites of such supports (a lattice's
 * nearest-neighbour pairs take a few KB), else PP_ERR_ARG.
 * Generators of weight 1 and 2 are evaluated from tables over groups of four
 * sites plus per-pair corrections (exact fixed-point sums, units of 2^-56); heavier
 * ones from a generic list.  The FP64 form multiplies by the factor in FP64; the
 * FP32 form by the factor carried as a float pair, rounding the coefficient once.
 * Replaces a map previously attached to the layer. */
pp_status pp_load_noise(pp_handle* h, int layer, size_t n_gen, const uint64_t* ex,
                        const uint64_t* ez, const double* lambda, int mode);

/* Propagates O = sum_t oc[t] P(ox[t], oz[t]) backwards through every layer.
 *   ox, oz [n_terms][W], oc [n_terms] (finite, |oc| < 2^32, else PP_ERR_ARG);
 *          duplicate strings are summed on the device exactly, independently of
 *          their order (128-bit fixed point, units of 2^-80, rounded once to the
 *          nearest double; a duplicated string's terms below 2^-80 are lost).
 *   eps    coefficient threshold (>= 0; 0 keeps every nonzero term)
 *   w_max  Pauli-weight cap (< 0: none)
 * The host waits for the device once per fused sub-layer (to size the next
 * sub-layer's buckets from the live-term count); the tiers of a sub-layer and
 * the overflow grouping run back to back on the device.  Before a sub-layer
 * whose planned output would fill more than half the buffers, and after one
 * whose output did not fit, the buffers grow (up to the capacity limit) and
 * the sub-layer runs (again) from its unchanged input.
 * Synchronises the handle's stream.  Errors: PP_ERR_STATE (no circuit),
 * PP_ERR_ARG, PP_ERR_NOMEM (a buffer, or a growth, could not be allocated; the
 * handle stays usable), PP_ERR_CAPACITY (more live terms than the capacity
 * limit; raise pp_options.max_terms), PP_ERR_TIMEOUT (pp_cancel), PP_ERR_CUDA. */
pp_status pp_propagate(pp_handle* h, size_t n_terms, const uint64_t* ox, const uint64_t* oz,
                       const double* oc, double eps, int w_max);

/* Asks the pp_propagate running on h (from another host thread) to stop.  It
 * returns PP_ERR_TIMEOUT after the fused sub-layer in flight completes (no
 * kernel is interrupted), the handle stays usable and holds no result.  A call
 * that arrives after the propagation finished has no effect on later ones.
 * This is the one call on a handle that may overlap another.  Errors:
 * PP_ERR_ARG (null handle). */
pp_status pp_cancel(pp_handle* h);

/* Top-K truncation for the following pp_propagate calls (Sec. I.A: each
 * intermediate result keeps at most its K largest Pauli terms).  After the
 * input observable is merged and truncated, and after the gates of every
 * layer, only the top_k strings of largest |c| survive; equal magnitudes are
 * ranked by the string in export order (x words from the most significant,
 * then z words), smallest first.  The threshold and weight rules still apply
 * after every gate.  0 (the default) turns it off.  Errors: PP_ERR_ARG (null
 * handle). */
pp_status pp_set_top_k(pp_handle* h, size_t top_k);

/* <0..0|O~|0..0> = sum of c over strings with no X or Y letter, of the last
 * successful pp_propagate (Sec. I.C: the noise-canceling observable's value
 * on the all-zero state).  Accumulated exactly in 128-bit fixed point (terms
 * below 2^-80 in magnitude are cut) and rounded once to the nearest double, so
 * the value does not depend on term order.  Diagonal coefficients must be
 * finite with |c| < 2^32 and sum in magnitude to less than 2^46; a value
 * outside that range makes the result NaN.  Synchronises.  Errors:
 * PP_ERR_STATE. */
pp_status pp_expect(pp_handle* h, double* value);

/* Copies O~ (Sec. I: the noise-canceling observable, a weighted sum of
 * Pauli strings) to caller-owned host buffers, sorted by (x, then z) as unsigned
 * integers (word W-1 most significant).  The sort runs on the device (a radix
 * sort of the result, which stays sorted in the handle); the host only copies.
 * x, z: [cap][W], c: [cap] (FP64 in both precisions).  *n_out = number of
 * terms; PP_ERR_CAPACITY if cap < *n_out or *n_out >= 2^32 (nothing copied);
 * PP_ERR_NOMEM if the sort's scratch (~N/2 bytes, kept by the handle) cannot be
 * allocated.  Any of x, z, c may be NULL to query *n_out only (no sort). */
pp_status pp_export_terms(pp_handle* h, size_t cap, uint64_t* x, uint64_t* z, double* c,
                          size_t* n_out);

/* One propagation of a batch: the arguments of pp_propagate. */
typedef struct {
    size_t n_terms;
    const uint64_t* ox;
    const uint64_t* oz;
    const double* oc;
    double eps;
    int w_max;
} pp_batch_item;

/* Runs pp_propagate(handles[i], items[i]) for i < n in lockstep: handles on
 * one device with the same mask width and precision form a group whose
 * propagations advance together, one fused sub-layer per lockstep step; each
 * step launches every kernel once for the whole group (grid row = instance,
 * each row reading its own launch parameters from device memory) and waits
 * for the device once, so a group of n instances costs one host
 * synchronisation per step instead of n.  The groups run one after another on
 * the stream of their first handle (the other handles' streams are not used;
 * the call returns after the device work is done).  Each instance keeps its
 * own plan, layouts, capacity, truncation (eps, w_max, top-K) and counters:
 * its result and statistics equal those of pp_propagate on the same handle,
 * except that the optional orbit tiles and per-tier timing are not used.  An
 * instance that fails (capacity, cancel) stops with its status; the others
 * go on.  Handles must be distinct (else every status is PP_ERR_ARG) and not
 * be used by other calls meanwhile.  max_threads is ignored (kept for
 * binary compatibility).  status_out (optional, [n]) receives each item's
 * status; the return value is PP_OK when all succeeded, else the first
 * failing item's status. */
pp_status pp_propagate_batch(int n, pp_handle* const* handles, const pp_batch_item* items,
                             int max_threads, pp_status* status_out);

typedef struct {
    size_t n_terms;          /* live terms of O~                                        */
    size_t peak_terms;       /* largest live-term count after any sub-layer             */
    double updates;          /* sum over gates of the live terms entering the gate
                                (canonical gate-by-gate count)                           */
    int n_sublayers;         /* fused sub-layers executed                               */
    int kernel_launches;     /* kernels this library launched in the last propagation  */
    int fallback_buckets;    /* buckets processed by the global-memory path            */
    double seconds;          /* wall time of the last pp_propagate (host clock)        */
    /* per processing tier (0, 1: one warp per bucket, tiles of 248 and 512 strings;
       2, 3: one CTA per bucket, tiles of 1024 and 4096 strings; 4: global-memory tile):
       launches, summed device time from CUDA events on the handle's stream, and strings
       read + written by completed buckets */
    int tier_launches[5];
    double tier_ms[5];
    double tier_strings[5];
    double bytes_per_string;  /* bytes of one stored string (x, z words and coefficient) */
    int orbit_launches;       /* tier-0 launches that used the orbit tiles (the rest of
                                 tier 0 used the sparse warp tiles)                      */
    int retries;              /* sub-layer runs repeated because their output outgrew
                                 the planned buckets, the overflow area or the capacity  */
    int growths;              /* capacity growths during the propagation                 */
    size_t capacity;          /* terms per arena at the end of the propagation           */
} pp_stats;

pp_status pp_get_stats(const pp_handle* h, pp_stats* out);

/* Description of the last failure on this handle ("" if none).  Valid until the next call. */
const char* pp_last_error(const pp_handle* h);

/* Plan tuning.  A propagation's result does not depend on it: every plan
 * reproduces gate-by-gate propagation with per-gate truncation exactly
 * (Sec. I, Eq. evolve_gate, truncation after every gate); only the run time
 * does.
 *   max_fused_gates  commuting gates fused into one sub-layer (one pass over
 *                    the strings), 1..64*W; 0 = library default (64*W: whole
 *                    layers).  More gates mean fewer passes but larger orbits
 *                    per bucket.
 *   bucket_headroom  buckets are sized so that a bucket's strings times the
 *                    sub-layer's observed growth, times this factor, fill one
 *                    warp tile; in [1, 16]; 0 = library default (2.0).  Larger
 *                    values mean more, emptier buckets.
 *   first_tier       0..4: buckets start at this processing tier (0: orbit or
 *                    sparse warp tiles, 1: larger warp tiles, 2 and 3: CTA
 *                    tiles in shared memory, 4: the global-memory tile); tiers
 *                    below it pass every bucket on.  0 (default) is the fastest; the others exist so that
 *                    tests can run every tier on small inputs.
 *   orbit_tiles      1: class sub-layers are planned as single runs of gates
 *                    with disjoint supports and tier 0 processes them with the
 *                    orbit tiles (strings grouped by orbit into dense
 *                    coefficient blocks); 0 (default): every sub-layer uses
 *                    the sparse (hashed) warp tiles and same-signature gates
 *                    fuse across up to four ascending segments.
 *   tile_cap         strings per tile of tiers 0..3 (the two warp tiers, the
 *                    two CTA tiers); 0 = library default (248, 512, 1024, 4096
 *                    for W = 1; 248, 384, 1024, 2048 for W = 2); else 64..8192,
 *                    and the tier's tiles must fit the device's shared memory
 *                    per CTA.  A bucket that outgrows a tile moves to the next
 *                    tier, so every choice gives the same result.
 * pp_set_tuning copies *t and takes effect at the next pp_propagate.
 * Errors: PP_ERR_ARG (NULL pointer, value out of range; the handle keeps its
 * previous tuning).  pp_get_tuning writes the values in effect (defaults
 * resolved). */
typedef struct {
    int max_fused_gates;
    double bucket_headroom;
    int first_tier;
    int orbit_tiles;
    int tile_cap[4];
} pp_tuning;

pp_status pp_set_tuning(pp_handle* h, const pp_tuning* t);
pp_status pp_get_tuning(const pp_handle* h, pp_tuning* t);

/* Largest term count pp_expect_noalloc accepts (2^27). */
#define PP_NOALLOC_MAX_TERMS ((size_t)134217728)

/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when they need <0..0|O~|0..0>: work recorded
 * while a stream is captured into a CUDA graph, applications whose own memory
 * pool owns the device and forbids other allocations, latency-critical paths
 * that must not enter the CUDA allocator.  It computes the same exact
 * fixed-point sum as pp_expect, rounded by the same routine (the same bits for
 * the same terms; NaN for a diagonal coefficient that is not finite or has
 * |c| >= 2^32), over terms in the caller's device buffers,
 * without a handle and without allocating: its scratch (one 128-bit partial
 * per 16384 terms, 128 KiB) is a fixed array in the library's device image,
 * present on every GPU that loads the library until the process exits.
 *   x_dev      [n_terms][W] X masks in device memory (only X decides diagonality)
 *   c_dev      [n_terms] FP64 coefficients in device memory
 *   value_dev  device pointer receiving the double result
 *   cuda_stream  stream to run on (NULL: legacy default stream); the call only
 *              enqueues work -- read value_dev after synchronising the stream
 * The first call on a device looks up the array's device address (set-up, with
 * that device current); make that first call before any stream capture begins.
 * Every call shares the one array, so calls that overlap on the GPU race and
 * must be serialised by the caller.
 * Errors: PP_ERR_ARG (n_qubits outside 1..128, null pointers), PP_ERR_CAPACITY
 * (n_terms above PP_NOALLOC_MAX_TERMS), PP_ERR_CUDA. */
pp_status pp_expect_noalloc(int n_qubits, size_t n_terms, const uint64_t* x_dev, const double* c_dev,
                            double* value_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
