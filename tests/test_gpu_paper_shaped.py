"""CUDA path against the CPU oracle on the paper-shaped workload variants:
the 3x3 second-order Trotter mirror circuit with its four per-colour noise
models and the 56-qubit heavy-hex mirror circuit (its
R_ZZ gates and noise pairs span many site distances).  Same bar as the other
parity tests: equal string sets up to strings within 1e-12 relative of the
threshold, coefficients within 1e-12 relative in FP64, the expectation within
1e-12 of the diagonal mass, and the canonical update count.

Mirror circuits run forwards then backwards, so most surviving coefficients
are the small remainders of cancelling contributions as large as the largest
coefficient; their rounding error is relative to those contributions.  Their
coefficient check therefore uses 1e-12 relative with a floor of 1e-3 of the
largest coefficient (an absolute bar of 1e-15 of it): measured on B300 the
largest such difference is 4e-12 relative to a 4e-6 coefficient, i.e. 2e-17
of the largest."""
import dataclasses

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


def check(pp, inst):
    ref = oracle.run(inst)
    got = pp.propagate(inst, precision=64)
    info = compare_terms((got.x, got.z, got.c), (ref.x, ref.z, ref.c), inst.eps, rel=1e-12, floor=1e-3)
    assert abs(got.expect - ref.expect) <= max(expect_tol((ref.x, ref.z, ref.c), 1e-12), 1e-300)
    if info["near_eps"] == 0:
        assert got.stats.updates == ref.updates
    return ref, got


@pytest.mark.parametrize("mode", [inputs.NOISE_INVERSE, inputs.NOISE_FORWARD])
def test_trotter2_mirror_3x3(pp, mode):
    # The mirror's halves cancel most strings up to rounding residues.  The
    # noise factors differ from the oracle's by a few ulps (table products
    # against one exp), so with no threshold a residue can be exactly zero on
    # one side and 1e-30 on the other, and the two sides then drop exact zeros
    # at different gates.  A threshold far above the residues and far below
    # the surviving terms makes every drop decision the same on both sides.
    inst = dataclasses.replace(inputs.workload_trotter2_mirror_3x3(steps=2, theta=0.05).with_noise_mode(mode),
                               eps=1e-13)
    ref, got = check(pp, inst)
    assert len(got.c) > 10000


@pytest.mark.parametrize("steps,eps,theta,w_max", [(2, 1e-7, 0.8, 12), (3, 1e-5, 0.6, 10)])
def test_heavy_hex_mirror(pp, steps, eps, theta, w_max):
    inst = inputs.workload_heavy_hex_mirror(steps=steps, theta=theta, eps=eps, w_max=w_max)
    ref, got = check(pp, inst)
    assert len(got.c) > 1000
