"""Parity cases run against the debug build of the library (device bounds
checks on tile, list, gate, region and overflow indices; see PP_OOB in
pp_kernels.cuh).  Run as a script in its own process with PP_LIBRARY set to
the debug build: every case must match the oracle, and a failed bounds check
would surface as PP_ERR_CUDA from pp_propagate.  Prints one line per case and
exits non-zero on the first mismatch."""
import dataclasses
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2606_20441_b300 import inputs, pp  # noqa: E402
from tests.parity import compare_terms, expect_tol  # noqa: E402


def run(inst, precision=64, **tuning):
    h = pp.Handle(inst.n_qubits, precision=precision)
    try:
        h.load_instance(inst)
        if tuning:
            h.pp_set_tuning(**tuning)
        h.run_instance(inst)
        e = h.pp_expect()
        x, z, c = h.pp_export_terms()
        return x, z, c, e, h.pp_get_stats()
    finally:
        h.close()


def check(name, inst, precision=64, **tuning):
    ref = oracle.run(inst)
    x, z, c, e, st = run(inst, precision, **tuning)
    if precision == 64:
        compare_terms((x, z, c), (ref.x, ref.z, ref.c), inst.eps)
        assert abs(e - ref.expect) <= expect_tol((ref.x, ref.z, ref.c)), (e, ref.expect)
    else:
        assert abs(e - ref.expect) <= 1e-4, (e, ref.expect)
    print("ok %-28s terms %8d  tiers %s" % (name, len(c), list(st.tier_launches)), flush=True)


def main():
    assert pp.load_library()._name == os.environ.get("PP_LIBRARY", pp.LIB_PATH)
    check("6x6_s2_fp64", inputs.workload_6x6(steps=2, eps=1e-5))
    check("6x6_s2_fp32", inputs.workload_6x6(steps=2, eps=1e-5), precision=32)
    for t in range(5):
        check("7x8_s3_first_tier_%d" % t, inputs.workload_7x8(eps=1e-4, steps=3), first_tier=t)
    check("7x8_s3_orbit_tiles", inputs.workload_7x8(eps=1e-4, steps=3), orbit_tiles=1)
    check("7x8_s2_top_k", dataclasses.replace(inputs.workload_7x8(eps=1e-5, steps=2), top_k=2000))
    for seed in range(2):
        check("generic_%d" % seed, inputs.random_circuit(seed, n=10, n_layers=6))
    check("10x10_two_words", inputs.random_tfim(inputs.SplitMix64(99), "t10", 10, 10, 2, 2, 1e-4))
    check("3x3_exact", inputs.workload_3x3(steps=2))


if __name__ == "__main__":
    main()
