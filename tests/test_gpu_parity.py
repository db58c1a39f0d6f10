"""CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs: bit-exact string sets (up to strings within 1e-9 relative of the
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
