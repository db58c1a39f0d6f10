"""pp_expect_noalloc: the expectation for callers that cannot allocate device
memory (stream capture, an application-owned memory pool).  It must return what
pp_expect returns for the same terms, call after call, although every call
reuses the library's one fixed scratch array."""
import numpy as np
import pytest

from paper_2606_20441_b300 import inputs
from tests.parity import expect_tol

pytestmark = pytest.mark.gpu


def _terms_and_value(pp, inst):
    h = pp.Handle(inst.n_qubits)
    try:
        h.load_instance(inst)
        h.run_instance(inst)
        value = h.pp_expect()
        x, z, c = h.pp_export_terms()
    finally:
        h.close()
    return x, z, c, value


def test_noalloc_expectation_matches_pp_expect_on_consecutive_calls():
    import torch
    from paper_2606_20441_b300 import build, pp
    assert torch.cuda.is_available()
    build.build()
    cases = [inputs.workload_6x6(steps=3, eps=1e-5),                      # W = 1, ~10 chunks
             inputs.random_tfim(inputs.SplitMix64(77), "w2", 9, 9, 3, 3, 1e-4)]   # W = 2
    stream = torch.cuda.current_stream().cuda_stream
    for inst in cases:
        x, z, c, ref = _terms_and_value(pp, inst)
        assert len(c) > 300
        x_dev = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
        c_dev = torch.from_numpy(np.ascontiguousarray(c)).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = pp.pp_expect_noalloc(inst.n_qubits, len(c), x_dev.data_ptr(), c_dev.data_ptr(),
                                  out.data_ptr(), stream)
        assert st == pp.PP_OK
        torch.cuda.synchronize()
        # both round the same exact 128-bit total with the same routine
        assert out.item() == ref, (out.item(), ref)
        assert abs(out.item() - ref) <= expect_tol((x, z, c))


def test_noalloc_rejects_more_terms_than_its_scratch_holds():
    import torch
    from paper_2606_20441_b300 import build, pp
    build.build()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pp.pp_expect_noalloc(36, pp.NOALLOC_MAX_TERMS + 1, 1, 1, out.data_ptr(), None)
    assert st == pp.PP_ERR_CAPACITY


def test_noalloc_out_of_range_coefficient_gives_nan():
    """A coefficient outside the exact sum's range (|c| >= 2^32, or not
    finite) makes the result NaN instead of a wrapped-around value."""
    import math
    import torch
    from paper_2606_20441_b300 import build, pp
    build.build()
    for bad in (2.0 ** 33, float("inf"), float("nan")):
        x_dev = torch.zeros(3, dtype=torch.int64, device="cuda")
        c_dev = torch.tensor([0.5, bad, 0.25], dtype=torch.float64, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert pp.pp_expect_noalloc(3, 3, x_dev.data_ptr(), c_dev.data_ptr(), out.data_ptr(), None) == pp.PP_OK
        torch.cuda.synchronize()
        assert math.isnan(out.item())
