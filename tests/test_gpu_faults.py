"""Failure paths, made on the host (no GPU fault is ever provoked): an
allocator that refuses memory, and a propagation cancelled from another
thread.  Each time the call reports its status and the handle stays usable:
the next propagation matches the oracle."""
import threading
import time

import numpy as np
import pytest

from oracle import oracle
from paper_2606_20441_b300 import inputs
from tests.parity import compare_terms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_20441_b300 import build, pp as ppmod
    build.build()
    return ppmod


class RefusingAllocator:
    """Device memory from torch's caching allocator, refused once `budget`
    allocations have been made (the stand-in for an exhausted pool)."""

    def __init__(self, budget):
        import torch
        self.torch = torch
        self.budget = budget
        self.calls = 0
        self.refused = 0
        self.live = set()

    def alloc(self, nbytes):
        self.calls += 1
        if self.budget is not None and self.calls > self.budget:
            self.refused += 1
            return 0
        ptr = self.torch.cuda.caching_allocator_alloc(nbytes)
        self.live.add(ptr)
        return ptr

    def free(self, ptr):
        self.live.discard(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("budget", [0, 3, 12])
def test_refused_allocation_reports_nomem_and_recovers(pp, budget):
    inst = inputs.workload_6x6(steps=2, eps=1e-4)
    ref = oracle.run(inst)
    a = RefusingAllocator(budget)
    h = pp.Handle(inst.n_qubits, max_terms=1 << 20, allocator=(a.alloc, a.free))
    try:
        h.load_instance(inst)
        with pytest.raises(pp.PPError) as ei:
            h.run_instance(inst)
        assert ei.value.status == pp.PP_ERR_NOMEM and a.refused > 0
        # a failed set-up keeps nothing: every buffer made so far went back
        a.budget = None
        h.run_instance(inst)
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), inst.eps)
        assert abs(h.pp_expect() - ref.expect) <= 1e-12
    finally:
        h.close()
    assert not a.live


def test_cancel_mid_flight_then_reuse(pp):
    """pp_cancel from another thread stops a long propagation after its
    current sub-layer with PP_ERR_TIMEOUT; the handle then runs a new
    propagation correctly."""
    big = inputs.workload_7x8(eps=1e-6, w_max=10)   # several seconds
    h = pp.Handle(big.n_qubits)
    try:
        h.load_instance(big)
        box = {}

        def run():
            t = time.perf_counter()
            try:
                h.run_instance(big)
                box["status"] = pp.PP_OK
            except pp.PPError as ex:
                box["status"] = ex.status
            box["sec"] = time.perf_counter() - t

        th = threading.Thread(target=run)
        th.start()
        time.sleep(0.5)
        h.pp_cancel()
        th.join(timeout=60)
        assert not th.is_alive()
        assert box["status"] == pp.PP_ERR_TIMEOUT, box
        with pytest.raises(pp.PPError) as ei:
            h.pp_expect()                       # no result after a cancelled run
        assert ei.value.status == pp.PP_ERR_STATE
        small = inputs.workload_7x8(eps=1e-4, w_max=10, steps=3)
        ref = oracle.run(small)
        h.load_instance(small)
        h.run_instance(small)                   # a cancel of the earlier run does not carry over
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), small.eps)
    finally:
        h.close()


def test_cancel_after_finish_has_no_effect(pp):
    inst = inputs.workload_6x6(steps=2, eps=1e-4)
    h = pp.Handle(inst.n_qubits)
    try:
        h.load_instance(inst)
        h.run_instance(inst)
        e1 = h.pp_expect()
        h.pp_cancel()
        h.run_instance(inst)
        assert h.pp_expect() == e1
    finally:
        h.close()


def test_capacity_grows_during_a_propagation(pp):
    """A handle starts with small buffers and grows them when a sub-layer's
    output needs more; the result is the oracle's."""
    inst = inputs.workload_6x6(steps=4, eps=1e-4)      # peak 1.8e5 terms
    ref = oracle.run(inst)
    h = pp.Handle(inst.n_qubits)
    try:
        h.load_instance(inst)
        h.run_instance(inst)
        st = h.pp_get_stats()
        assert st.growths >= 1 and st.capacity >= st.peak_terms > (1 << 16)
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), inst.eps)
        assert abs(h.pp_expect() - ref.expect) <= 1e-12
        h.run_instance(inst)                    # already large enough: no growth
        assert h.pp_get_stats().growths == 0
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), inst.eps)
    finally:
        h.close()


def test_capacity_limit_reports_capacity(pp):
    inst = inputs.workload_6x6(steps=3, eps=1e-4)
    h = pp.Handle(inst.n_qubits, max_terms=10_000)     # the peak is 2.2e4 terms
    try:
        h.load_instance(inst)
        with pytest.raises(pp.PPError) as ei:
            h.run_instance(inst)
        assert ei.value.status == pp.PP_ERR_CAPACITY
        small = inputs.workload_6x6(steps=1, eps=1e-3)
        ref = oracle.run(small)
        h.load_instance(small)
        h.run_instance(small)
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), small.eps)
    finally:
        h.close()


def test_refused_growth_reports_nomem_and_recovers(pp):
    """The allocator refuses once the first propagation's buffers exist: the
    next propagation, which must grow them, ends with PP_ERR_NOMEM; the handle
    keeps its buffers and, once memory is given again, matches the oracle."""
    tiny = inputs.workload_6x6(steps=1, eps=1e-2)
    inst = inputs.workload_6x6(steps=4, eps=1e-4)
    ref = oracle.run(inst)
    a = RefusingAllocator(None)
    h = pp.Handle(inst.n_qubits, allocator=(a.alloc, a.free))
    try:
        h.load_instance(tiny)
        h.run_instance(tiny)
        assert h.pp_get_stats().growths == 0
        h.load_instance(inst)
        a.budget = a.calls + 1                   # e.g. the circuit tables, not a growth
        with pytest.raises(pp.PPError) as ei:
            h.run_instance(inst)
        assert ei.value.status == pp.PP_ERR_NOMEM and a.refused > 0
        a.budget = None
        h.run_instance(inst)
        assert h.pp_get_stats().growths >= 1
        compare_terms(h.pp_export_terms(), (ref.x, ref.z, ref.c), inst.eps)
    finally:
        h.close()
    assert not a.live
