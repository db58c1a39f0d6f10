"""CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs: bit-exact string sets (up to strings within 1e-12 relative of the
threshold), coefficients within 1e-12 relative in FP64, expectation within
1e-12 of the sum of |c| over diagonal strings, and the canonical gate-by-gate
update count."""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_2606_20441_b300 import inputs
from tests.parity import compare_terms, expect_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_20441_b300 import build, pp as ppmod
    build.build()
    return ppmod


def run_tuned(pp, inst, precision=64, **tuning):
    """One propagation with plan tuning; returns (x, z, c, expect, stats)."""
    h = pp.Handle(inst.n_qubits, precision=precision)
    try:
        h.load_instance(inst)
        h.pp_set_tuning(**tuning)
        h.run_instance(inst)
        e = h.pp_expect()
        x, z, c = h.pp_export_terms()
        return x, z, c, e, h.pp_get_stats()
    finally:
        h.close()


def check(pp, inst, precision=64, rel=1e-12, exp_rel=1e-12, max_terms=0, check_updates=True):
    ref = oracle.run(inst)
    got = pp.propagate(inst, precision=precision, max_terms=max_terms)
    info = compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), inst.eps, rel=rel)
    assert abs(got.expect - ref.expect) <= max(expect_tol((ref.x, ref.z, ref.c), exp_rel), 1e-300), \
        (got.expect, ref.expect)
    if check_updates and info["near_eps"] == 0 and precision == 64:
        assert got.stats.updates == ref.updates
    return ref, got, info


def test_appendix_d_example(pp):
    for lam1, lam2 in [(0.01, 0.02), (0.003, 0.0007)]:
        inst = inputs.one_qubit_appD(lam1, lam2)
        ref, got, _ = check(pp, inst)
        q1 = (1 - math.exp(2 * lam1)) / 2
        q2 = (1 - math.exp(2 * lam2)) / 2
        d = {(int(got.x[i, 0]), int(got.z[i, 0])): got.c[i] for i in range(len(got.c))}
        assert abs(d[(0, 1)] - (1 - q1)) < 1e-14
        assert abs(d[(1, 0)] + q1 * (1 - 2 * q2)) < 1e-14


def test_tfim_3x3_untruncated(pp):
    check(pp, inputs.workload_3x3())


@pytest.mark.parametrize("seed", range(16))
def test_random_generic_circuits(pp, seed):
    n = [3, 4, 5, 6, 9, 17, 70, 100][seed % 8]
    eps = [0.0, 1e-4, 1e-3, 1e-2][seed % 4]
    w_max = [-1, -1, 3, 5][(seed // 4) % 4]
    inst = inputs.random_circuit(seed, n, n_layers=8 if n < 20 else 12, eps=eps, w_max=w_max,
                                 max_gates=4, rate_hi=0.05)
    check(pp, inst)


@pytest.mark.parametrize("seed", range(4))
def test_heavy_noise_generators(pp, seed):
    """Generators of weight up to 4 (the generic noise path) next to 1- and 2-local ones."""
    inst = inputs.random_circuit(200 + seed, 12 + 30 * seed, n_layers=8, eps=1e-4, max_gates=4,
                                 rate_hi=0.05, n_gen=12, gen_weight=4)
    check(pp, inst)


@pytest.mark.parametrize("steps,eps", [(2, 1e-5), (3, 1e-5), (3, 1e-4)])
def test_tfim_6x6(pp, steps, eps):
    _, got, info = check(pp, inputs.workload_6x6(steps=steps, eps=eps))
    assert len(got.c) > 1000


def test_tfim_7x8_weight_cap(pp):
    check(pp, inputs.workload_7x8(eps=1e-4, w_max=10, steps=3))


def test_tfim_10x10_two_words(pp):
    rng = inputs.SplitMix64(99)
    inst = inputs.random_tfim(rng, "t10", 10, 10, 2, 2, 1e-4)
    check(pp, inst)


@pytest.mark.parametrize("mode", [inputs.NOISE_FORWARD, inputs.NOISE_INVERSE])
def test_noise_modes_with_truncation(pp, mode):
    inst = inputs.workload_6x6(steps=2, eps=1e-4).with_noise_mode(mode)
    check(pp, inst)


def test_clifford_angles(pp):
    rng = inputs.SplitMix64(5)
    n = 36
    tx = [[0.0, math.pi / 2, -math.pi / 2, math.pi][rng.randint(4)] for _ in range(n)]
    rates = inputs.draw_rates(rng, 4, inputs.n_lattice_generators(6, 6), 2e-3)
    inst = inputs.tfim_instance("cl", 6, 6, 4, math.pi / 2, tx, rates,
                                [({q: "Z"}, 1.0 / n) for q in range(n)])
    ref, got, _ = check(pp, inst)
    assert len(got.c) <= n


def test_small_capacity_uses_fallback_and_regrows(pp):
    """A tiny capacity forces bucket-region regrowth; results stay exact."""
    inst = inputs.workload_6x6(steps=3, eps=1e-5)
    check(pp, inst, max_terms=400_000)


def test_capacity_error_is_reported(pp):
    inst = inputs.workload_6x6(steps=3, eps=1e-5)
    with pytest.raises(pp.PPError) as ei:
        pp.propagate(inst, max_terms=5000)
    assert ei.value.status == pp.PP_ERR_CAPACITY


def test_handle_reusable_after_error(pp):
    inst = inputs.workload_6x6(steps=2, eps=1e-4)
    h = pp.Handle(inst.n_qubits, max_terms=4096)
    h.load_instance(inst)
    with pytest.raises(pp.PPError):
        h.run_instance(inst, eps=1e-7)
    h.run_instance(inst, eps=1e-3)
    ref = oracle.run(inst, eps=1e-3)
    assert abs(h.pp_expect() - ref.expect) <= 1e-12
    h.close()


def test_fp32_form_error_bound(pp):
    inst = inputs.workload_6x6(steps=3, eps=1e-5)
    ref = oracle.run(inst)
    got = pp.propagate(inst, precision=32)
    assert abs(got.expect - ref.expect) <= 1e-6


def test_empty_and_fully_truncated(pp):
    inst = inputs.workload_3x3(steps=1)
    got = pp.propagate(inst, eps=10.0)
    assert len(got.c) == 0 and got.expect == 0.0
    empty = inputs.Instance("e", 9, inst.gate_x, inst.gate_z, inst.theta, inst.layer_of,
                            inst.n_layers, inst.noise, np.zeros((0, 1), np.uint64),
                            np.zeros((0, 1), np.uint64), np.zeros(0))
    got = pp.propagate(empty)
    assert len(got.c) == 0 and got.expect == 0.0


def test_duplicate_input_strings_are_summed(pp):
    inst = inputs.workload_3x3(steps=1)
    dup = inputs.Instance("d", 9, inst.gate_x, inst.gate_z, inst.theta, inst.layer_of, inst.n_layers,
                          inst.noise, np.concatenate([inst.obs_x, inst.obs_x]),
                          np.concatenate([inst.obs_z, inst.obs_z]),
                          np.concatenate([inst.obs_c, inst.obs_c]))
    ref = oracle.run(dup)
    got = pp.propagate(dup)
    compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), 0.0)


@pytest.mark.parametrize("precision", [64, 32])
def test_duplicate_input_strings_sum_exactly_in_any_order(pp, precision):
    """Duplicates of one input string are summed exactly whatever their order:
    1 + 2^-40 - 1 + 2^-40 in any order gives 2^-39, also in the FP32 form,
    where a float sum in arrival order would lose the small terms.  The
    circuit is one R_X(0) gate (the identity) with no noise."""
    zx = np.zeros((1, 1), np.uint64)
    z0 = np.ones((1, 1), np.uint64)           # Z on qubit 0
    vals = np.array([1.0, 2.0 ** -40, -1.0, 2.0 ** -40])
    rng = np.random.default_rng(5)
    for perm in [np.arange(4), np.array([2, 1, 0, 3]), rng.permutation(4), rng.permutation(4)]:
        h = pp.Handle(2, precision=precision)
        h.pp_load_circuit(np.array([[1]], np.uint64), zx, np.array([0.0]), np.array([0], np.int32), 1)
        h.pp_propagate(np.repeat(zx, 4, 0), np.repeat(z0, 4, 0), vals[perm], 0.0, -1)
        assert h.pp_expect() == 2.0 ** -39
        x, z, c = h.pp_export_terms()
        assert len(c) == 1 and c[0] == 2.0 ** -39
        h.close()


def test_observable_coefficients_must_be_finite_and_below_2_32(pp):
    h = pp.Handle(2)
    zx = np.zeros((1, 1), np.uint64)
    h.pp_load_circuit(np.array([[1]], np.uint64), zx, np.array([0.3]), np.array([0], np.int32), 1)
    for bad in (np.nan, np.inf, 2.0 ** 32):
        with pytest.raises(pp.PPError):
            h.pp_propagate(zx, np.ones((1, 1), np.uint64), np.array([bad]), 0.0, -1)
    h.pp_propagate(zx, np.ones((1, 1), np.uint64), np.array([2.0 ** 31]), 0.0, -1)
    assert abs(h.pp_expect() - 2.0 ** 31 * np.cos(0.3)) <= 1e-6
    h.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("layer", [1, 0])
def test_noise_rate_limits_and_largest_factors(pp, precision, layer):
    """A map's rates must sum below 60 (below 40 in the FP32 form, whose
    factors must stay within float range); factors up to the limit are exact
    to the form's precision.  One qubit, two layers of one identity gate each,
    the map {X: a, Z: a} after layer 1 (the first sub-layer's prologue applies
    it) or after layer 0 (the streaming pass): X and Z anticommute with one
    generator each (factor e^{2a}), Y with both (e^{4a}); byte 7 of the
    fixed-point exponent carries the integer part."""
    zx = np.zeros((2, 1), np.uint64)
    one = np.ones((2, 1), np.uint64)
    h = pp.Handle(1, precision=precision)
    h.pp_load_circuit(one, zx, np.array([0.0, 0.0]), np.array([0, 1], np.int32), 2)
    gx, gz = np.array([[1], [0]], np.uint64), np.array([[0], [1]], np.uint64)
    limit = 60.0 if precision == 64 else 40.0
    with pytest.raises(pp.PPError):
        h.pp_load_noise(layer, gx, gz, np.array([limit / 2, limit / 2 + 0.5]))
    a = limit / 2 - 0.5
    h.pp_load_noise(layer, gx, gz, np.array([a, a]))
    tol = 1e-13 if precision == 64 else 2.0 ** -22
    for (ox, oz), k in (((1, 0), 1), ((0, 1), 1), ((1, 1), 2)):
        h.pp_propagate(np.array([[ox]], np.uint64), np.array([[oz]], np.uint64), np.array([1.0]), 0.0, -1)
        x, z, c = h.pp_export_terms()
        want = math.exp(2.0 * k * a)
        assert len(c) == 1 and int(x[0, 0]) == ox and int(z[0, 0]) == oz
        assert abs(c[0] - want) <= tol * want, (ox, oz, c[0], want)
    h.close()


def test_noise_tables_must_fit_shared_memory(pp):
    """The streaming noise pass stages a map's tables in one CTA's shared
    memory; a map whose 2-site generators cross 4-site groups in thousands of
    places (every ZZ pair among 80 of 128 qubits) is refused at load time with
    PP_ERR_ARG, and the handle keeps working (its nearest-neighbour subset
    loads and propagates)."""
    n, W = 128, 2
    h = pp.Handle(n)
    gx = np.zeros((1, W), np.uint64)
    gx[0, 0] = np.uint64(1)
    h.pp_load_circuit(gx, np.zeros((1, W), np.uint64), np.array([0.3]), np.array([0], np.int32), 1)
    pairs = [(a, b) for a in range(80) for b in range(a + 1, 80)]
    ex = np.zeros((len(pairs), W), np.uint64)
    ez = np.zeros((len(pairs), W), np.uint64)
    for k, (a, b) in enumerate(pairs):
        ez[k, a // 64] |= np.uint64(1 << (a % 64))
        ez[k, b // 64] |= np.uint64(1 << (b % 64))
    lam = np.full(len(pairs), 1e-5)
    with pytest.raises(pp.PPError) as err:
        h.pp_load_noise(0, ex, ez, lam)
    assert err.value.status == pp.PP_ERR_ARG and "shared memory" in str(err.value)
    near = [k for k, (a, b) in enumerate(pairs) if b == a + 1]
    h.pp_load_noise(0, ex[near], ez[near], lam[near])
    ox = np.zeros((1, W), np.uint64)
    ox[0, 0] = np.uint64(1)   # X on qubit 0: anticommutes with Z0Z1 only
    h.pp_propagate(ox, np.zeros((1, W), np.uint64), np.array([1.0]), 0.0, -1)
    x, z, c = h.pp_export_terms()
    assert len(c) == 1 and abs(c[0] - math.exp(2e-5)) <= 1e-13
    h.close()


# ----------------------------------------------------------------- every processing tier

TIER_CASES = {"6x6_s3": lambda: inputs.workload_6x6(steps=3, eps=1e-5),
              "7x8_s3": lambda: inputs.workload_7x8(eps=1e-4, steps=3)}


@pytest.fixture(scope="module")
def tier_refs():
    return {k: (f(), oracle.run(f())) for k, f in TIER_CASES.items()}


@pytest.mark.parametrize("case", sorted(TIER_CASES))
@pytest.mark.parametrize("first_tier", [1, 2, 3, 4])
def test_every_tier_against_oracle(pp, tier_refs, case, first_tier):
    """Buckets forced past the smaller tiers: the larger warp tiles (512
    strings), the CTA tiles (1024 and 4096 strings) and the global-memory tile
    each run whole propagations and match the oracle exactly (string sets,
    coefficients, update count)."""
    inst, ref = tier_refs[case]
    x, z, c, e, st = run_tuned(pp, inst, first_tier=first_tier)
    info = compare_terms((x, z, c), (ref.x, ref.z, ref.c), inst.eps)
    assert abs(e - ref.expect) <= expect_tol((ref.x, ref.z, ref.c))
    if info["near_eps"] == 0:
        assert st.updates == ref.updates
    assert st.tier_launches[first_tier] > 0 and st.tier_strings[first_tier] > 0
    for t in range(first_tier):
        assert st.tier_strings[t] == 0
    if first_tier == 4:
        assert st.fallback_buckets > 0


@pytest.mark.parametrize("case", sorted(TIER_CASES))
def test_orbit_tier_matches_sparse_tier(pp, tier_refs, case):
    """Tier 0 with the orbit tiles (single-run sub-layers, dense orbit blocks)
    and with the sparse hashed warp tiles (multi-segment sub-layers) give the
    same result bit for bit, and both match the oracle."""
    inst, ref = tier_refs[case]
    for prec in (64, 32):
        xo, zo, co, eo, so = run_tuned(pp, inst, precision=prec, orbit_tiles=1)
        xs, zs, cs, es, ss = run_tuned(pp, inst, precision=prec, orbit_tiles=0)
        assert so.orbit_launches > 0 and ss.orbit_launches == 0
        assert so.tier_strings[0] > 0
        # every plan reproduces gate-by-gate propagation, so the two agree bit for bit
        assert np.array_equal(xo, xs) and np.array_equal(zo, zs) and np.array_equal(co, cs)
        assert eo == es and so.updates == ss.updates
        if prec == 64:
            compare_terms((xo, zo, co), (ref.x, ref.z, ref.c), inst.eps)
            assert so.updates == ref.updates


# ----------------------------------------------------------------- the 7x8 workload deeper

def _digest_of(x, z):
    from tests.golden.make_oracle_digest import set_digest
    return set_digest(x, z)


def test_tfim_7x8_four_steps_golden(pp):
    """7x8, 4 Trotter steps, eps = 1e-5, w_max = 10 (3e6 strings): the oracle
    needs minutes, so its result is stored as a digest by
    tests/golden/make_oracle_digest.py: term count, set digest, expectation,
    update count and a sample of exact coefficients."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tfim7x8_s4_eps1e-5.json")))
    inst = inputs.workload_7x8(eps=1e-5, w_max=10, steps=4)
    got = pp.propagate(inst)
    assert g["near_eps"] == 0
    assert len(got.c) == g["n_terms"]
    assert _digest_of(got.x, got.z) == g["set_digest"]
    assert got.stats.updates == g["updates"]
    assert abs(got.expect - g["expect"]) <= 1e-12 * g["diag_abs_sum"]
    keys = np.concatenate([got.x, got.z], axis=1)
    sx = np.array(g["sample"]["x"], dtype=np.uint64)
    sz = np.array(g["sample"]["z"], dtype=np.uint64)
    sc = np.array([float.fromhex(v) for v in g["sample"]["c"]])
    want = np.concatenate([sx, sz], axis=1)
    kv = keys.view(np.dtype((np.void, keys.dtype.itemsize * keys.shape[1]))).ravel()
    wv = np.ascontiguousarray(want).view(np.dtype((np.void, want.dtype.itemsize * want.shape[1]))).ravel()
    common, ig, iw = np.intersect1d(kv, wv, return_indices=True)
    assert len(common) == len(wv)
    assert np.all(np.abs(got.c[ig] - sc[iw]) <= 1e-12 * np.abs(sc[iw]))


# ----------------------------------------------------------------- the benchmark configuration

def _bench_shaped(theta_zz, theta_x):
    """The 7x8 / 20-step / w_max 10 / eps 1e-6 benchmark circuit (same lattice,
    noise rates and observable) with other angles."""
    base = inputs.workload_7x8(eps=1e-6, w_max=10, steps=20)
    inst = inputs.tfim_instance("bench_shaped", 7, 8, 20, theta_zz, theta_x,
                                np.stack([m.lam for m in base.noise]),
                                [({a: "Z", b: "Z"}, 1.0 / 97) for (a, b) in base.meta["edges"]],
                                eps=1e-6, w_max=10)
    return inst


@pytest.mark.parametrize("precision", [64, 32])
def test_bench_configuration_clifford_angles(pp, precision):
    """The full benchmark configuration (7x8, 20 steps, the benchmark's noise
    and observable, eps 1e-6, w_max 10, default plan) at Clifford angles
    (R_ZZ(pi/2), per-site R_X in {0, pi/2, pi, -pi/2}): every string follows
    one path (App. A) until the weight cap ends it, computed independently by
    the symplectic tableau in oracle/clifford.py (79 of the 97 paths survive)."""
    from oracle import clifford
    rng = inputs.SplitMix64(3)
    tx = [[0.0, math.pi / 2, math.pi, -math.pi / 2][rng.randint(4)] for _ in range(56)]
    inst = _bench_shaped(math.pi / 2, tx)
    ref, ref_updates = clifford.propagate(inst, truncate=True, count_updates=True)
    got = pp.propagate(inst, precision=precision)
    assert len(ref) > 0 and len(got.c) == len(ref)
    tol = 1e-13 if precision == 64 else 2e-6
    for i in range(len(got.c)):
        key = (int(got.x[i, 0]), int(got.z[i, 0]))
        assert abs(got.c[i] - ref[key]) <= tol * abs(ref[key])
    assert got.stats.updates == ref_updates


def test_bench_configuration_theta_zero(pp):
    """The benchmark configuration with every angle 0: only the line diagram
    survives, O~ = O prod exp(2 sum lambda over anticommuting generators) (App.
    G, Eq. line-term)."""
    inst = _bench_shaped(0.0, 0.0)
    got = pp.propagate(inst)
    assert len(got.c) == len(inst.obs_c)
    for t in range(len(inst.obs_c)):
        s_tot = 0.0
        for m in inst.noise:
            anti = ((np.bitwise_and(m.ex[:, 0], inst.obs_z[t, 0]) ^ np.bitwise_and(m.ez[:, 0], inst.obs_x[t, 0])))
            par = np.array([bin(int(v)).count("1") & 1 for v in anti], dtype=bool)
            s_tot += float(np.sum(m.lam[par]))
        i = int(np.nonzero((got.x[:, 0] == inst.obs_x[t, 0]) & (got.z[:, 0] == inst.obs_z[t, 0]))[0][0])
        expected = float(inst.obs_c[t]) * math.exp(2.0 * s_tot)
        assert abs(got.c[i] - expected) <= 1e-13 * abs(expected)
    assert got.stats.updates == inst.n_gates * len(inst.obs_c)


def test_bench_configuration_theta_zero_fp32_rounds_once_per_map(pp):
    """The FP32 form of the zero-angle benchmark configuration: each noise map
    multiplies a coefficient by its exact factor exp(2 S 2^-56) (S the map's
    fixed-point exponent, an integer sum) and rounds once to float.  The factor
    is carried as a float pair; a pair that lost its tail (a plain float
    product) would be off by several ulp per map, twenty maps in a row."""
    from fractions import Fraction
    inst = _bench_shaped(0.0, 0.0)
    got = pp.propagate(inst, precision=32)
    assert len(got.c) == len(inst.obs_c)
    fix = [[int(Fraction(float(v)) * 2 ** 56 + Fraction(1, 2)) for v in m.lam] for m in inst.noise]
    exact = 0
    for t in range(len(inst.obs_c)):
        c = np.float32(inst.obs_c[t])
        for m, lf in sorted(zip(inst.noise, fix), key=lambda ml: -ml[0].layer):
            anti = np.bitwise_and(m.ex[:, 0], inst.obs_z[t, 0]) ^ np.bitwise_and(m.ez[:, 0], inst.obs_x[t, 0])
            S = sum(v for v, a in zip(lf, anti) if bin(int(a)).count("1") & 1)
            c = np.float32(float(c) * math.exp(2.0 * math.ldexp(S, -56)))
        i = int(np.nonzero((got.x[:, 0] == inst.obs_x[t, 0]) & (got.z[:, 0] == inst.obs_z[t, 0]))[0][0])
        g = np.float32(got.c[i])
        assert abs(float(g) - float(c)) <= 2 * float(np.spacing(c)), (t, g, c)
        exact += int(g == c)
    assert exact >= 0.95 * len(inst.obs_c)


# ----------------------------------------------------------------- top-K truncation

TOPK_CASES = {"6x6_s3": lambda: inputs.workload_6x6(steps=3, eps=1e-5),
              "7x8_s3": lambda: inputs.workload_7x8(eps=1e-4, steps=3)}


@pytest.mark.parametrize("case", sorted(TOPK_CASES))
@pytest.mark.parametrize("k", [100, 10_000, 1_000_000])
@pytest.mark.parametrize("precision", [64, 32])
def test_top_k_against_oracle(pp, case, k, precision):
    """Top-K after every layer (Sec. I.A), device radix select, against the
    oracle's sort: the same strings (FP64: the same coefficients too); K above
    the term count changes nothing."""
    import dataclasses
    inst = dataclasses.replace(TOPK_CASES[case](), top_k=k)
    ref = oracle.run(inst)
    got = pp.propagate(inst, precision=precision)
    assert len(got.c) <= k
    if precision == 64 or len(ref.c) == k:
        assert len(got.c) == len(ref.c)
    if precision == 64:
        compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), inst.eps)
        assert abs(got.expect - ref.expect) <= expect_tol((ref.x, ref.z, ref.c))
        assert got.stats.updates == ref.updates
    if k == 1_000_000:
        plain = oracle.run(dataclasses.replace(inst, top_k=0))
        assert len(plain.c) == len(ref.c)


def test_top_k_ties_on_the_input(pp):
    """The 97 equal coefficients of the 7x8 observable: K = 40 keeps the 40
    strings first in export order (the oracle's tie rule), then propagates."""
    import dataclasses
    inst = dataclasses.replace(inputs.workload_7x8(eps=1e-4, steps=2), top_k=40)
    ref = oracle.run(inst)
    got = pp.propagate(inst)
    compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), inst.eps)
    assert got.stats.updates == ref.updates


def test_expectation_is_the_correctly_rounded_exact_sum(pp):
    """<0|O~|0> is the exact sum of the diagonal coefficients rounded once
    (App. C's estimator is a plain sum; the library sums in 128-bit fixed
    point): 1 + 2^-53 + 2^-80 rounds to 1 + 2^-52, where adding in double
    precision would give 1."""
    from fractions import Fraction
    terms = [({0: "Z"}, 1.0), ({1: "Z"}, 2.0 ** -53), ({2: "Z"}, 2.0 ** -80), ({0: "X"}, 0.75)]
    ox, oz, oc = [], [], []
    for letters, c in terms:
        x, z = inputs.pauli_from_letters(letters, 1)
        ox.append(x); oz.append(z); oc.append(c)
    inst = inputs.Instance("exact", 3, np.zeros((0, 1), np.uint64), np.zeros((0, 1), np.uint64), np.zeros(0),
                           np.zeros(0, np.int32), 1, [], np.array(ox).reshape(-1, 1), np.array(oz).reshape(-1, 1),
                           np.array(oc))
    got = pp.propagate(inst)
    exact = float(sum(Fraction(c) for letters, c in terms if all(v == "Z" for v in letters.values())))
    assert exact == 1.0 + 2.0 ** -52
    assert got.expect == exact


def test_sub_layer_rerun_keeps_its_input(pp):
    """Early sub-layers of this 7x8 instance grow its strings ~10x, far past
    the planner's estimate: the sixth sub-layer outgrows the capacity and runs
    again from its input after the buffers grow, and that input has strings in
    the grouped overflow area, which the failed attempt must leave untouched.
    The result matches the oracle, twice in a row (runs are deterministic)."""
    import dataclasses
    inst = [i for i in inputs.workload_batch64(eps=1e-6) if i.name == "batch37"][0]
    cut = dataclasses.replace(inputs.layer_range(inst, inst.n_layers - 5, inst.n_layers), eps=1e-6, w_max=10)
    ref = oracle.run(cut)
    runs = [pp.propagate(cut) for _ in range(2)]
    for got in runs:
        assert got.stats.retries > 0
        compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), cut.eps)
        assert abs(got.expect - ref.expect) <= expect_tol((ref.x, ref.z, ref.c))
        assert got.stats.updates == ref.updates
    assert np.array_equal(runs[0].c, runs[1].c)


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_and_resume(pp, precision):
    """A propagation checkpointed after its later layers (the exported result)
    and resumed through the earlier layers, in a fresh handle, gives the same
    strings, coefficients and expectation as the uninterrupted propagation,
    bit for bit, and the update counts add up."""
    import dataclasses
    inst = inputs.workload_6x6(steps=4, eps=1e-5)
    k = inst.n_layers // 2
    whole = pp.propagate(inst, precision=precision)
    late = pp.propagate(inputs.layer_range(inst, k, inst.n_layers), precision=precision)
    early = dataclasses.replace(inputs.layer_range(inst, 0, k), obs_x=late.x, obs_z=late.z, obs_c=late.c)
    resumed = pp.propagate(early, precision=precision)
    assert np.array_equal(resumed.x, whole.x) and np.array_equal(resumed.z, whole.z)
    assert np.array_equal(resumed.c, whole.c)
    assert resumed.expect == whole.expect
    assert late.stats.updates + resumed.stats.updates == whole.stats.updates
