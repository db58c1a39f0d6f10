"""Plan tuning changes run time only: every (max_fused_gates, bucket_headroom,
tile sizes) gives the same strings and coefficients, bit for bit, and the same
exact expectation; out-of-range values are rejected without changing the
handle."""
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


def _sorted_terms(x, z, c):
    key = np.lexsort(tuple(z[:, w] for w in range(z.shape[1])) + tuple(x[:, w] for w in range(x.shape[1])))
    return x[key], z[key], c[key]


@pytest.mark.parametrize("precision", [64, 32])
def test_every_setting_gives_identical_results(pp, precision):
    inst = inputs.workload_6x6(steps=4, eps=1e-5)
    h = pp.Handle(inst.n_qubits, precision=precision, max_terms=40_000_000)
    h.load_instance(inst)
    ref = None
    for g, hr, caps in [(16, 1.6, ()), (1, 1.6, ()), (4, 1.0, ()), (8, 3.0, ()), (32, 1.6, ()),
                        (64, 16.0, ()), (0, 0.0, (128, 256, 512, 2048)), (0, 0.0, (400, 800, 2048, 4096)),
                        (0, 0.0, ())]:
        h.pp_set_tuning(g, hr, tile_caps=caps)
        h.run_instance(inst)
        got = (h.pp_expect(),) + _sorted_terms(*h.pp_export_terms())
        if ref is None:
            ref = got
            assert len(ref[3]) > 1000
            continue
        assert got[0] == ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.array_equal(a, b)
    h.close()


def test_tuning_arguments(pp):
    h = pp.Handle(40)
    assert h.pp_get_tuning() == (64, 2.0)
    h.pp_set_tuning(24, 2.5)
    assert h.pp_get_tuning() == (24, 2.5)
    for bad in [(65, 1.6), (-1, 1.6), (16, 0.5), (16, 17.0)]:
        with pytest.raises(pp.PPError):
            h.pp_set_tuning(*bad)
        assert h.pp_get_tuning() == (24, 2.5)
    h.pp_set_tuning(0, 0.0)
    assert h.pp_get_tuning() == (64, 2.0)
    assert h.tuning()["tile_cap"] == [248, 512, 1024, 4096]
    h.pp_set_tuning(0, 0.0, tile_caps=(300, 600, 0, 0))
    assert h.tuning()["tile_cap"] == [300, 600, 1024, 4096]
    for bad in [(32, 0, 0, 0), (0, 9000, 0, 0), (0, 0, 0, 8192 * 2)]:
        with pytest.raises(pp.PPError):
            h.pp_set_tuning(0, 0.0, tile_caps=bad)
        assert h.tuning()["tile_cap"] == [300, 600, 1024, 4096]
    with pytest.raises(pp.PPError):   # 4 warp tiles of 8192 strings exceed a CTA's shared memory
        h.pp_set_tuning(0, 0.0, tile_caps=(8192, 0, 0, 0))
    h.close()
    h2 = pp.Handle(100)
    h2.pp_set_tuning(128, 1.6)
    assert h2.pp_get_tuning()[0] == 128
    h2.close()
