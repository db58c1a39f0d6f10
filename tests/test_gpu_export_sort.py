"""pp_export_terms orders O~ by key on the device: ascending by
(x[W-1], ..., x[0], z[W-1], ..., z[0]) as unsigned words.  The exported list
must be that order exactly (checked against numpy's lexsort of the same set),
for one and two mask words, both coefficient forms, results that need many
radix passes, and the trivial sizes; exporting twice gives the same list, and
the sort leaves the expectation unchanged."""
import numpy as np
import pytest

from paper_2606_20441_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_20441_b300 import build, pp as ppmod
    build.build()
    return ppmod


def key_order(x, z):
    W = x.shape[1]
    # np.lexsort: the last key is the primary one
    keys = tuple(z[:, w] for w in range(W)) + tuple(x[:, w] for w in range(W))
    return np.lexsort(keys)


def check_sorted_export(h):
    e0 = h.pp_expect()
    x, z, c = h.pp_export_terms()
    assert len(c) == h.pp_get_stats().n_terms
    o = key_order(x, z)
    assert np.array_equal(o, np.arange(len(c)))         # already in key order
    keys = np.concatenate([x, z], axis=1)
    if len(c) > 1:
        assert not np.any(np.all(keys[1:] == keys[:-1], axis=1))   # distinct strings
    x2, z2, c2 = h.pp_export_terms()
    assert np.array_equal(x, x2) and np.array_equal(z, z2) and np.array_equal(c, c2)
    assert h.pp_expect() == e0
    return x, z, c


@pytest.mark.parametrize("precision", [64, 32])
def test_sorted_export_one_word(pp, precision):
    inst = inputs.workload_6x6(steps=3, eps=1e-5)
    h = pp.Handle(inst.n_qubits, precision=precision, max_terms=20_000_000)
    h.load_instance(inst)
    h.run_instance(inst)
    x, z, c = check_sorted_export(h)
    assert len(c) > 10_000
    h.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_sorted_export_two_words(pp, precision):
    # a 9x10 lattice with observable terms on both sides of qubit 64, so the
    # keys differ in both mask words
    rng = inputs.SplitMix64(inputs.SEED_BASE + 77)
    rows, cols, steps = 9, 10, 3
    rates = inputs.draw_rates(rng, steps, inputs.n_lattice_generators(rows, cols), 2e-3)
    inst = inputs.tfim_instance("w2", rows, cols, steps, 0.3, 0.6, rates,
                                [({5: "Z"}, 0.5), ({75: "Z"}, 0.5)], eps=1e-4, w_max=8)
    assert inst.W == 2
    h = pp.Handle(inst.n_qubits, precision=precision, max_terms=40_000_000)
    h.load_instance(inst)
    h.run_instance(inst)
    x, z, c = check_sorted_export(h)
    assert len(c) > 1000
    # keys use bits of both words
    assert np.any(z[:, 1] != 0) and np.any(z[:, 0] != 0)
    h.close()


def test_sorted_export_small_sizes(pp):
    # 0 terms (everything truncated), 1 term, and a few terms
    inst = inputs.workload_3x3(steps=1)
    h = pp.Handle(inst.n_qubits, precision=64)
    h.load_instance(inst)
    for eps, lo, hi in [(10.0, 0, 0), (0.5, 0, 9), (0.0, 10, 10_000)]:
        h.run_instance(inst, eps=eps)
        x, z, c = check_sorted_export(h)
        assert lo <= len(c) <= hi
    h.close()
