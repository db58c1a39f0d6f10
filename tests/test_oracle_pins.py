"""Pins for the CPU oracle: each test checks it against something other than
itself -- the paper's worked example, closed forms, dense matrix simulation,
brute force over all Paulis, an independent Clifford tableau, and invariants."""
import json
import math
import os

import numpy as np
import pytest

from oracle import clifford, dense, oracle
from paper_2606_20441_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def as_dict(res, n):
    """{(x int, z int): c} from an oracle result."""
    out = {}
    W = res.x.shape[1] if res.x.ndim == 2 else 1
    for i in range(len(res.c)):
        xi = sum(int(res.x[i, w]) << (64 * w) for w in range(W))
        zi = sum(int(res.z[i, w]) << (64 * w) for w in range(W))
        out[(xi, zi)] = float(res.c[i])
    return out


def symplectic_np(px, pz, ex, ez):
    """<P,E> for arrays of words, by the symplectic form x_p.z_e + z_p.x_e."""
    tot = 0
    for w in range(len(px)):
        tot += bin(int(px[w]) & int(ez[w])).count("1") + bin(int(pz[w]) & int(ex[w])).count("1")
    return tot & 1


# ----------------------------------------------------------------- Pauli algebra

@pytest.mark.parametrize("n", [1, 2, 3])
def test_signed_permutation_matches_kronecker(n):
    for xi in range(1 << n):
        for zi in range(1 << n):
            a = dense.pauli_dense_fast([xi], [zi], n)
            b = dense.pauli_dense_kron([xi], [zi], n)
            assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_product_table_against_matrices(n):
    """R * P = i^ph Q (oracle's table) against dense Kronecker products, for all pairs."""
    for rx in range(1 << n):
        for rz in range(1 << n):
            R = dense.pauli_dense_kron([rx], [rz], n)
            for px in range(1 << n):
                for pz in range(1 << n):
                    P = dense.pauli_dense_kron([px], [pz], n)
                    (qx, qz), ph = oracle.multiply(n, ([rx], [rz]), ([px], [pz]))
                    Q = dense.pauli_dense_kron(qx, qz, n)
                    assert np.allclose(R @ P, (1j ** ph) * Q, atol=0)
                    anti = oracle.anticommute(n, ([px], [pz]), ([rx], [rz]))
                    assert anti == int(np.allclose(R @ P + P @ R, 0))


def test_multiword_product_against_tableau_phase():
    """Words above 64 qubits: the table product against the g-function phase."""
    rng = inputs.SplitMix64(7)
    n = 100
    for _ in range(200):
        r = inputs.pauli_from_letters(inputs.random_pauli_letters(rng, [rng.randint(n) for _ in range(5)]), 2)
        p = inputs.pauli_from_letters(inputs.random_pauli_letters(rng, [rng.randint(n) for _ in range(8)]), 2)
        (qx, qz), ph = oracle.multiply(n, r, p)
        rxi, rzi = clifford._to_int(r[0]), clifford._to_int(r[1])
        pxi, pzi = clifford._to_int(p[0]), clifford._to_int(p[1])
        assert clifford._to_int(qx) == rxi ^ pxi and clifford._to_int(qz) == rzi ^ pzi
        assert ph == clifford.product_phase(rxi, rzi, pxi, pzi, n)
        assert oracle.anticommute(n, p, r) == clifford.symplectic(pxi, pzi, rxi, rzi)


# ----------------------------------------------------------------- worked example / closed forms

def test_appendix_d_worked_example():
    """App. D: O~ = (1 - q1) Z - q1 (1 - 2 q2) X with q = (1 - e^{2 lambda})/2."""
    with open(os.path.join(GOLDEN, "appD_one_qubit_example.json")) as f:
        fx = json.load(f)
    for lam1, lam2 in fx["lambdas"]:
        q1 = (1.0 - math.exp(2.0 * lam1)) / 2.0
        q2 = (1.0 - math.exp(2.0 * lam2)) / 2.0
        res = as_dict(oracle.run(inputs.one_qubit_appD(lam1, lam2)), 1)
        expect_z = 1.0 - q1
        expect_x = -q1 * (1.0 - 2.0 * q2)
        assert set(res) == {(0, 1), (1, 0)}
        assert abs(res[(0, 1)] - expect_z) <= 1e-14
        assert abs(res[(1, 0)] - expect_x) <= 1e-14


@pytest.mark.parametrize("theta", [0.1, 0.5, -1.3, 2.9])
def test_single_qubit_rx_closed_form(theta):
    """<0|R_X(theta)^dag Z R_X(theta)|0> = cos(theta); O~ = cos Z + sin Y."""
    x, z = inputs.pauli_from_letters({0: "X"}, 1)
    zx, zz = inputs.pauli_from_letters({0: "Z"}, 1)
    inst = inputs.Instance("rx", 1, x.reshape(1, 1), z.reshape(1, 1), np.array([theta]),
                           np.array([0], dtype=np.int32), 1, [], zx.reshape(1, 1),
                           zz.reshape(1, 1), np.array([1.0]))
    r = oracle.run(inst)
    d = as_dict(r, 1)
    assert abs(d[(0, 1)] - math.cos(theta)) < 1e-15
    assert abs(d[(1, 1)] - math.sin(theta)) < 1e-15
    assert abs(r.expect - math.cos(theta)) < 1e-15


@pytest.mark.parametrize("rows,cols,steps,after", [(3, 3, 4, "zz"), (6, 6, 3, "x"), (10, 10, 2, "zz")])
def test_theta_zero_line_diagram(rows, cols, steps, after):
    """All angles 0: only the line diagram survives (App. G, Eq. line-term with
    cos = 1): O~ = O * prod_layers exp(2 sum_{E_k anticommuting with O} lambda_k)."""
    rng = inputs.SplitMix64(11)
    n = rows * cols
    rates = inputs.draw_rates(rng, steps, inputs.n_lattice_generators(rows, cols), 2e-3)
    edges, _ = inputs.square_lattice(rows, cols)
    obs = [({0: "Z"}, 0.5), ({1: "X", 2: "Y"}, -0.25), ({edges[-1][0]: "Y", edges[-1][1]: "Z"}, 1.0)]
    inst = inputs.tfim_instance("zero", rows, cols, steps, 0.0, 0.0, rates, obs, noise_after=after)
    run = oracle.run(inst)
    res = as_dict(run, n)
    assert len(res) == len(obs)
    # nothing branches at theta = 0, so every gate sees exactly the |O| strings
    assert run.updates == inst.n_gates * len(obs)
    for t in range(len(obs)):
        s_tot = 0.0
        for m in inst.noise:
            for k in range(len(m.lam)):
                if symplectic_np(inst.obs_x[t], inst.obs_z[t], m.ex[k], m.ez[k]):
                    s_tot += float(m.lam[k])
        key = (clifford._to_int(inst.obs_x[t]), clifford._to_int(inst.obs_z[t]))
        expected = float(inst.obs_c[t]) * math.exp(2.0 * s_tot)
        assert abs(res[key] - expected) <= 1e-13 * abs(expected)


@pytest.mark.parametrize("rows,cols,steps", [(3, 3, 3), (6, 6, 4), (7, 8, 3), (10, 10, 2)])
def test_clifford_points_single_path(rows, cols, steps):
    """Clifford angles (Sec. III: no truncation error at theta = 0, pi/2): each
    string maps to one string; its coefficient is the product of gate signs and
    noise factors along the path (App. A), computed here by an independent
    symplectic tableau."""
    rng = inputs.SplitMix64(1000 + rows * cols)
    n = rows * cols
    choices = [0.0, math.pi / 2, -math.pi / 2, math.pi]
    tx = [choices[rng.randint(4)] for _ in range(n)]
    rates = inputs.draw_rates(rng, steps, inputs.n_lattice_generators(rows, cols), 2e-3)
    edges, _ = inputs.square_lattice(rows, cols)
    obs = [({q: "Z"}, 1.0 / n) for q in range(n)] + [({a: "Z", b: "Z"}, 0.3) for (a, b) in edges[:5]]
    inst = inputs.tfim_instance("cliff", rows, cols, steps, math.pi / 2, tx, rates, obs)
    ref = clifford.propagate(inst)
    ref = {k: v for k, v in ref.items() if v != 0.0}
    run = oracle.run(inst)
    got = as_dict(run, n)
    assert set(got) == set(ref)
    # one path per string: every gate sees exactly the |O| strings
    assert run.updates == inst.n_gates * len(obs)
    for k, v in ref.items():
        assert abs(got[k] - v) <= 1e-13 * abs(v)


def test_clifford_paths_with_truncation():
    """The 7x8 benchmark circuit at Clifford angles with its threshold and
    weight cap: single paths that end when the weight exceeds the cap (Sec.
    I.A, truncation after every gate), followed by the symplectic tableau,
    against the oracle's hash map: same strings, coefficients, update count."""
    base = inputs.workload_7x8(eps=1e-6, w_max=10, steps=20)
    rng = inputs.SplitMix64(3)
    tx = [[0.0, math.pi / 2, math.pi, -math.pi / 2][rng.randint(4)] for _ in range(56)]
    inst = inputs.tfim_instance("cliff78", 7, 8, 20, math.pi / 2, tx, np.stack([m.lam for m in base.noise]),
                                [({a: "Z", b: "Z"}, 1.0 / 97) for (a, b) in base.meta["edges"]],
                                eps=1e-6, w_max=10)
    ref, ref_updates = clifford.propagate(inst, truncate=True, count_updates=True)
    run = oracle.run(inst)
    got = as_dict(run, 56)
    assert 0 < len(ref) < len(inst.obs_c) and set(got) == set(ref)
    for k, v in ref.items():
        assert abs(got[k] - v) <= 1e-13 * abs(v)
    assert run.updates == ref_updates


# ----------------------------------------------------------------- dense simulation

@pytest.mark.slow
@pytest.mark.parametrize("after", ["zz", "x"])
def test_density_matrix_3x3(after):
    """The 3x3 workload against the 512x512 density matrix (Sec. II, Fig. 2:
    evaluation with respect to the exact density matrix), both noise placements,
    and every Pauli coefficient against the dense Heisenberg operator."""
    base = inputs.workload_3x3()
    if after == "x":
        for m in base.noise:
            m.layer += 1
    res = oracle.run(base)
    rho_val = dense.density_expect(base)
    assert abs(res.expect - rho_val) <= 1e-12 * max(1.0, abs(rho_val))
    coef = dense.heisenberg_coefficients(base)
    assert np.max(np.abs(coef.imag)) < 1e-12
    got = np.zeros_like(coef.real)
    for i in range(len(res.c)):
        got[int(res.x[i, 0]), int(res.z[i, 0])] = res.c[i]
    assert np.max(np.abs(got - coef.real)) <= 1e-12
    # every string the dense operator carries above rounding is present
    assert np.count_nonzero(np.abs(coef.real) > 1e-13) <= len(res.c)


@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_all_paulis_with_truncation(seed):
    """n <= 4, generic rotation axes, both noise directions, per-gate truncation
    by threshold and weight: oracle == dense conjugation over all 4^n Paulis."""
    n = 3 + seed % 2
    eps = [0.0, 1e-3, 3e-2, 0.1][seed % 4]
    w_max = [-1, -1, 2, 1][(seed // 2) % 4]
    inst = inputs.random_circuit(seed, n, n_layers=6, eps=eps, w_max=w_max, rate_hi=0.1)
    ref, ref_updates = dense.ptm_propagate(inst, count_updates=True)
    run = oracle.run(inst)
    got = as_dict(run, n)
    margin = 1e-9
    near = {k for k, v in list(ref.items()) + list(got.items())
            if eps > 0 and abs(abs(v) - eps) <= margin * eps}
    assert set(got) - near == set(ref) - near
    for k in set(got) & set(ref):
        assert abs(got[k] - ref[k]) <= 1e-12
    # the canonical work count (live strings entering each gate), counted on
    # the dense coefficient vector
    if not near:
        assert run.updates == ref_updates


@pytest.mark.parametrize("n,eps", [(6, 0.0), (9, 0.0), (8, 0.05), (10, 0.02)])
def test_update_count_closed_form(n, eps):
    """O = Z on n qubits, one layer of R_X(theta_j) on every site: gate j sees
    every product of the cos/sin factors of gates 0..j-1 whose magnitude is at
    least eps (each product is one string; truncation after every gate).  With
    eps = 0 that is 2^j strings, a total of 2^n - 1."""
    rng = inputs.SplitMix64(40 + n)
    theta = [rng.uniform(0.3, 1.2) * (1 if rng.uniform() < 0.5 else -1) for _ in range(n)]
    gx = np.zeros((n, 1), np.uint64)
    gz = np.zeros((n, 1), np.uint64)
    for q in range(n):
        gx[q, 0] = np.uint64(1) << np.uint64(q)
    ox, oz = inputs.pauli_from_letters({q: "Z" for q in range(n)}, 1)
    inst = inputs.Instance("cf", n, gx, gz, np.array(theta), np.zeros(n, np.int32), 1, [],
                           ox.reshape(1, 1), oz.reshape(1, 1), np.array([1.0]), eps=eps)
    expected = 0
    for j in range(n):
        # products of a cos-or-sin factor per gate 0..j-1, each kept at every
        # prefix (truncation after every gate drops a branch for good)
        live = [1.0]
        for t in range(j):
            live = [v * f for v in live for f in (math.cos(theta[t]), math.sin(theta[t]))
                    if abs(v * f) >= eps]
        expected += len(live)
    if eps == 0.0:
        assert expected == 2 ** n - 1
    run = oracle.run(inst)
    assert run.updates == expected


def test_dense_density_matches_small_random():
    for seed in range(4):
        inst = inputs.random_circuit(100 + seed, 4, n_layers=5, rate_hi=0.05)
        r = oracle.run(inst)
        assert abs(r.expect - dense.density_expect(inst)) <= 1e-12


# ----------------------------------------------------------------- invariants

def test_noise_then_inverse_is_identity():
    """Lambda^{-1} Lambda = identity (Sec. I: the inverse map negates lambda)."""
    base = inputs.workload_3x3()
    m = base.noise[0]
    fwd = inputs.NoiseLayer(1, m.ex, m.ez, m.lam, inputs.NOISE_FORWARD)
    inv = inputs.NoiseLayer(0, m.ex, m.ez, m.lam, inputs.NOISE_INVERSE)
    rng = inputs.SplitMix64(5)
    ox, oz, oc = [], [], []
    for _ in range(20):
        x, z = inputs.pauli_from_letters(inputs.random_pauli_letters(rng, [rng.randint(9), rng.randint(9)]), 1)
        ox.append(x); oz.append(z); oc.append(rng.uniform(-1, 1))
    inst = inputs.Instance("inv", 9, np.zeros((0, 1), np.uint64), np.zeros((0, 1), np.uint64),
                           np.zeros(0), np.zeros(0, np.int32), 2, [fwd, inv],
                           np.array(ox).reshape(-1, 1), np.array(oz).reshape(-1, 1), np.array(oc))
    no_noise = inputs.Instance("id", 9, inst.gate_x, inst.gate_z, inst.theta, inst.layer_of, 2, [],
                               inst.obs_x, inst.obs_z, inst.obs_c)
    a = as_dict(oracle.run(inst), 9)
    b = as_dict(oracle.run(no_noise), 9)
    assert set(a) == set(b)
    for k in a:
        assert abs(a[k] - b[k]) <= 1e-14 * abs(b[k])


@pytest.mark.parametrize("rows,cols,steps", [(3, 3, 2), (2, 5, 2)])
def test_mirror_circuit_returns_observable(rows, cols, steps):
    """Sec. II mirror circuits: forward then reversed evolution is the identity,
    so the propagated operator returns to O (no noise, no truncation)."""
    rng = inputs.SplitMix64(3)
    n = rows * cols
    tx = [rng.uniform(0.2, 0.9) for _ in range(n)]
    rates = np.zeros((steps, inputs.n_lattice_generators(rows, cols)))
    inst = inputs.tfim_instance("m", rows, cols, steps, 0.37, tx, rates,
                                [({0: "Z", n - 1: "Z"}, 1.0), ({n // 2: "X"}, 0.5)])
    res = as_dict(oracle.run(inputs.mirror_instance(inst)), n)
    big = {k: v for k, v in res.items() if abs(v) > 1e-12}
    assert len(big) == 2
    for t in range(2):
        key = (clifford._to_int(inst.obs_x[t]), clifford._to_int(inst.obs_z[t]))
        assert abs(big[key] - inst.obs_c[t]) <= 1e-12


def test_rotation_mass_bookkeeping():
    """Rotations are orthogonal on each (P, RP) pair: sum c^2 is preserved by
    every gate, and kept + truncated mass equals the rotated mass."""
    inst = inputs.workload_6x6(steps=2, eps=1e-4)
    rec = oracle.run(inst, record=True).records
    assert rec.shape[0] == 2 * (36 + 60)
    assert np.all(np.abs(rec[:, 1] - rec[:, 0]) <= 1e-12 * rec[:, 0])
    assert np.all(np.abs(rec[:, 2] + rec[:, 3] - rec[:, 1]) <= 1e-12 * rec[:, 1])
    assert np.sum(rec[:, 3]) > 0.0    # the threshold did act


# ----------------------------------------------------------------- top-K truncation

def _export_order_key(x_words, z_words):
    """Sort key of a string in export order: x words from the most significant,
    then z words."""
    return tuple(int(v) for v in x_words[::-1]) + tuple(int(v) for v in z_words[::-1])


def _obs_only(n, terms):
    """An instance with one empty layer: the observable itself."""
    W = inputs.n_words(n)
    ox, oz, oc = [], [], []
    for letters, c in terms:
        x, z = inputs.pauli_from_letters(letters, W)
        ox.append(x); oz.append(z); oc.append(c)
    return inputs.Instance("obs", n, np.zeros((0, W), np.uint64), np.zeros((0, W), np.uint64), np.zeros(0),
                           np.zeros(0, np.int32), 1, [], np.array(ox).reshape(-1, W),
                           np.array(oz).reshape(-1, W), np.array(oc))


def test_top_k_keeps_largest_magnitudes():
    """Sec. I.A keeps the K largest terms: on a sum with distinct magnitudes,
    exactly the K of largest |c| survive, with their coefficients."""
    rng = inputs.SplitMix64(77)
    terms = []
    seen = set()
    while len(terms) < 60:
        sites = sorted({rng.randint(70) for _ in range(1 + rng.randint(4))})
        letters = inputs.random_pauli_letters(rng, sites)
        key = tuple(sorted(letters.items()))
        if key in seen:
            continue
        seen.add(key)
        terms.append((letters, rng.uniform(-1, 1)))
    inst = _obs_only(70, terms)
    for k in (1, 10, 59):
        r = oracle.run(inst, top_k=k)
        want = sorted(np.abs(inst.obs_c), reverse=True)[:k]
        assert len(r.c) == k
        assert sorted(np.abs(r.c), reverse=True) == want
    # K >= N keeps everything
    assert len(oracle.run(inst, top_k=60).c) == 60 and len(oracle.run(inst, top_k=10**6).c) == 60


def test_top_k_ties_break_by_string_order():
    """Equal magnitudes: the strings that come first in export order are kept."""
    rng = inputs.SplitMix64(5)
    terms, seen = [], set()
    while len(terms) < 20:
        q = rng.randint(9)
        letters = {q: "XYZ"[rng.randint(3)], (q + 1 + rng.randint(8)) % 9: "XYZ"[rng.randint(3)]}
        key = tuple(sorted(letters.items()))
        if key in seen:
            continue
        seen.add(key)
        terms.append((letters, 0.5 if rng.uniform() < 0.5 else -0.5))
    inst = _obs_only(9, terms)
    r = oracle.run(inst, top_k=7)
    order = sorted(range(20), key=lambda t: _export_order_key(inst.obs_x[t], inst.obs_z[t]))[:7]
    want = {_export_order_key(inst.obs_x[t], inst.obs_z[t]) for t in order}
    got = {_export_order_key(r.x[i], r.z[i]) for i in range(len(r.c))}
    assert got == want


def test_top_k_after_a_layer_closed_form():
    """One R_X layer on Z^n (eps = 0): the layer produces every product of a
    cos-or-sin factor per site (the sin sites carry Y); top-K after the layer
    keeps the K products of largest magnitude (ties by string order)."""
    n, k = 9, 37
    rng = inputs.SplitMix64(123)
    theta = [rng.uniform(0.3, 1.2) for _ in range(n)]
    gx = np.array([[1 << q] for q in range(n)], dtype=np.uint64)
    gz = np.zeros((n, 1), np.uint64)
    ox, oz = inputs.pauli_from_letters({q: "Z" for q in range(n)}, 1)
    inst = inputs.Instance("tk", n, gx, gz, np.array(theta), np.zeros(n, np.int32), 1, [], ox.reshape(1, 1),
                           oz.reshape(1, 1), np.array([1.0]))
    prods = []
    for m in range(1 << n):
        v = 1.0
        for q in range(n):
            v = v * (math.sin(theta[q]) if (m >> q) & 1 else math.cos(theta[q]))
        prods.append((-abs(v), m))
    prods.sort()
    want = {m for _, m in prods[:k]}
    r = oracle.run(inst, top_k=k)
    assert {int(r.x[i, 0]) for i in range(len(r.c))} == want
    assert np.all(r.z[:, 0] == (1 << n) - 1)


def test_checkpoint_split_is_the_same_pass():
    """Propagating through the later layers, then from that result through the
    earlier ones, is the same backward pass (Sec. I: the Heisenberg image is
    taken gate by gate, truncation after every gate is idempotent on kept
    strings): the same strings, coefficients, expectation and update count."""
    import dataclasses
    inst = inputs.workload_6x6(steps=2, eps=1e-5)
    k = inst.n_layers // 2
    whole = oracle.run(inst)
    late = oracle.run(inputs.layer_range(inst, k, inst.n_layers))
    early = dataclasses.replace(inputs.layer_range(inst, 0, k), obs_x=late.x, obs_z=late.z, obs_c=late.c)
    resumed = oracle.run(early)
    key = lambda r: {(tuple(x), tuple(z)): c for x, z, c in zip(r.x, r.z, r.c)}
    assert key(resumed) == key(whole)
    assert resumed.expect == whole.expect
    assert late.updates + resumed.updates == whole.updates
