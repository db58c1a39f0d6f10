"""Lockstep batches (pp_propagate_batch): handles on one device with the same
mask width and precision advance together, one fused sub-layer per lockstep
step, each kernel launched once for the whole batch.  Every instance of a
batch is checked against the oracle, and against the same instance run alone
(bit for bit: the batch changes the launch shape, not the arithmetic)."""
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


def small_batch(seed, count, eps=1e-3, w_max=6, lo=3, hi=5, steps=(2, 5)):
    """Batch-shaped instances (random TFIM lattices, depths, angles and
    observables) small enough for the oracle to finish in about a second."""
    rng = inputs.SplitMix64(inputs.SEED_BASE + seed)
    return [inputs.random_tfim(rng, "l%02d" % k, lo, hi, steps[0], steps[1], eps, w_max=w_max)
            for k in range(count)]


def run_batch(pp, insts, precision=64, top_k=None, max_terms=1 << 22):
    hs = [pp.Handle(i.n_qubits, precision=precision, max_terms=max_terms) for i in insts]
    for k, (h, i) in enumerate(zip(hs, insts)):
        h.load_instance(i)
        if top_k is not None:
            h.pp_set_top_k(top_k[k])
    st = pp.pp_propagate_batch(hs, insts)
    return hs, st


def alone(pp, inst, precision, top_k=0):
    h = pp.Handle(inst.n_qubits, precision=precision, max_terms=1 << 22)
    try:
        h.load_instance(inst)
        h.pp_set_top_k(top_k)
        h.run_instance(inst)
        x, z, c = h.pp_export_terms()
        return x, z, c, h.pp_expect(), h.pp_get_stats()
    finally:
        h.close()


def check_oracle(h, inst, top_k=None):
    ref = oracle.run(inst, top_k=top_k)
    x, z, c = h.pp_export_terms()
    info = compare_terms((x, z, c), (ref.x, ref.z, ref.c), inst.eps)
    e = h.pp_expect()
    assert abs(e - ref.expect) <= max(expect_tol((ref.x, ref.z, ref.c), 1e-12), 1e-300), (inst.name, e, ref.expect)
    if info["near_eps"] == 0:
        assert h.pp_get_stats().updates == ref.updates, inst.name
    return ref


def close_all(hs):
    for h in hs:
        h.close()


def test_lockstep_fp64_against_oracle(pp):
    """16 instances of different lattices and depths (so they finish at
    different lockstep steps) in FP64: each matches the oracle."""
    insts = small_batch(41, 16)
    assert len({len(i.obs_c) for i in insts}) >= 1 and len({i.n_qubits for i in insts}) > 2
    hs, st = run_batch(pp, insts, 64)
    try:
        assert all(s == pp.PP_OK for s in st), [(s, h.last_error()) for s, h in zip(st, hs)]
        for h, i in zip(hs, insts):
            check_oracle(h, i)
    finally:
        close_all(hs)


@pytest.mark.parametrize("precision", [64, 32])
def test_lockstep_equals_alone(pp, precision):
    """The same instances run alone give the same strings, coefficients,
    expectation and update count, bit for bit."""
    insts = small_batch(44, 12, eps=1e-4, w_max=8, lo=3, hi=4, steps=(2, 4))
    hs, st = run_batch(pp, insts, precision)
    try:
        assert all(s == pp.PP_OK for s in st), [(s, h.last_error()) for s, h in zip(st, hs)]
        for h, i in zip(hs, insts):
            x, z, c, e, stats = alone(pp, i, precision)
            bx, bz, bc = h.pp_export_terms()
            assert (bx == x).all() and (bz == z).all() and (bc == c).all(), i.name
            assert h.pp_expect() == e
            assert h.pp_get_stats().updates == stats.updates
            assert h.pp_get_stats().n_sublayers == stats.n_sublayers
    finally:
        close_all(hs)


def test_lockstep_mixed_widths_and_precisions(pp):
    """One call holding 64-bit and 128-bit masks, FP32 and FP64 handles: the
    call runs one lockstep group per (width, precision); every FP64 result
    matches the oracle and every FP32 result equals its run alone."""
    narrow = small_batch(45, 4)
    rng = inputs.SplitMix64(inputs.SEED_BASE + 43)
    wide = [inputs.random_tfim(rng, "w%02d" % k, 8, 10, 2, 4, 1e-3, w_max=6) for k in range(4)]
    wide = [w for w in wide if w.n_qubits > 64][:2] + [w for w in wide if w.n_qubits <= 64][:1]
    assert any(w.n_qubits > 64 for w in wide)
    insts = narrow + wide + narrow[:2] + wide[:1]
    precs = [64] * (len(narrow) + len(wide)) + [32] * 3
    hs = [pp.Handle(i.n_qubits, precision=p, max_terms=1 << 22) for i, p in zip(insts, precs)]
    try:
        for h, i in zip(hs, insts):
            h.load_instance(i)
        st = pp.pp_propagate_batch(hs, insts)
        assert all(s == pp.PP_OK for s in st), [(s, h.last_error()) for s, h in zip(st, hs)]
        for h, i, p in zip(hs, insts, precs):
            if p == 64:
                check_oracle(h, i)
            else:
                _, _, c, e, _ = alone(pp, i, 32)
                assert h.pp_expect() == e and len(h.pp_export_terms()[2]) == len(c)
    finally:
        close_all(hs)


def test_lockstep_top_k_against_oracle(pp):
    """Top-K truncation (Sec. I.A) per instance inside a batch: instances with
    different K (and none) side by side, each against the oracle's top-K."""
    insts = small_batch(46, 6)
    ks = [0, 1, 20, 100, 1000, 0]
    hs, st = run_batch(pp, insts, 64, top_k=ks)
    try:
        assert all(s == pp.PP_OK for s in st), [(s, h.last_error()) for s, h in zip(st, hs)]
        for h, i, k in zip(hs, insts, ks):
            ref = check_oracle(h, i, top_k=k or None)
            if k:
                assert len(ref.c) <= k
    finally:
        close_all(hs)


def test_lockstep_failure_is_isolated(pp):
    """An instance that outgrows its handle's capacity fails with
    PP_ERR_CAPACITY; the others of the batch finish and match the oracle."""
    insts = small_batch(47, 6)
    big = max(range(len(insts)), key=lambda k: len(oracle.run(insts[k]).c))
    hs = [pp.Handle(i.n_qubits, precision=64, max_terms=(64 if k == big else 1 << 22))
          for k, i in enumerate(insts)]
    try:
        for h, i in zip(hs, insts):
            h.load_instance(i)
        st = pp.pp_propagate_batch(hs, insts)
        assert st[big] == pp.PP_ERR_CAPACITY, (st, hs[big].last_error())
        for k, (h, i) in enumerate(zip(hs, insts)):
            if k != big:
                assert st[k] == pp.PP_OK, (k, h.last_error())
                check_oracle(h, i)
        with pytest.raises(pp.PPError):
            hs[big].pp_expect()
    finally:
        close_all(hs)


def test_lockstep_rejects_repeated_handles(pp):
    insts = small_batch(48, 2)
    h = pp.Handle(insts[0].n_qubits, precision=64)
    try:
        h.load_instance(insts[0])
        st = pp.pp_propagate_batch([h, h], [insts[0], insts[0]])
        assert st == [pp.PP_ERR_ARG, pp.PP_ERR_ARG]
    finally:
        h.close()


def test_lockstep_empty_and_single(pp):
    assert pp.pp_propagate_batch([], []) == []
    insts = small_batch(49, 1)
    hs, st = run_batch(pp, insts, 64)
    try:
        assert st == [pp.PP_OK]
        check_oracle(hs[0], insts[0])
    finally:
        close_all(hs)
