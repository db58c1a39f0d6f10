"""Command-line runner: one propagation of a named synthetic workload.

    python -m paper_2606_20441_b300 run --workload tfim7x8 --eps 1e-5 --precision 32

prints one JSON line with <0..0|O~|0..0>, the number of canonical updates, the
final and peak term counts and the per-tier launch/time/string counters of the
library's statistics.  This is the program the kernel profiles are taken on.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys

from . import inputs


def _instance(name: str, eps: float, steps: int, w_max: int) -> "inputs.Instance":
    if name == "tfim7x8":
        return inputs.workload_7x8(eps=eps, w_max=w_max, steps=steps or 20)
    if name == "tfim6x6":
        return inputs.workload_6x6(steps=steps or 10, eps=eps)
    if name == "tfim3x3":
        return inputs.workload_3x3(steps=steps or 4)
    if name == "heavyhex":
        return inputs.workload_heavy_hex_mirror(steps=steps or 4, eps=eps, w_max=w_max)
    if name == "mirror3x3":
        return inputs.workload_trotter2_mirror_3x3(steps=steps or 2, eps=eps)
    raise SystemExit("unknown workload %r (tfim7x8, tfim6x6, tfim3x3, heavyhex, mirror3x3)" % name)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2606_20441_b300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    r = sub.add_parser("run", help="propagate one workload on the current GPU")
    r.add_argument("--workload", default="tfim7x8")
    r.add_argument("--eps", type=float, default=1e-5)
    r.add_argument("--w-max", type=int, default=10)
    r.add_argument("--steps", type=int, default=0, help="Trotter steps (0: the workload's own)")
    r.add_argument("--precision", type=int, choices=[32, 64], default=32)
    r.add_argument("--max-terms", type=int, default=60_000_000)
    r.add_argument("--repeat", type=int, default=1)
    r.add_argument("--fused-gates", type=int, default=0, help="pp_set_tuning max_fused_gates (0: default)")
    r.add_argument("--headroom", type=float, default=0.0, help="pp_set_tuning bucket_headroom (0: default)")
    r.add_argument("--first-tier", type=int, default=0, help="pp_set_tuning first_tier (0: default)")
    r.add_argument("--orbit-tiles", action="store_true", help="pp_set_tuning orbit_tiles: orbit tiles in tier 0")
    r.add_argument("--tile-caps", default="0,0,0,0", help="pp_set_tuning tile_cap of tiers 0-3 (0: default)")
    r.add_argument("--top-k", type=int, default=0, help="keep the K largest terms after every layer (0: off)")
    a = ap.parse_args(argv)

    from . import pp
    inst = _instance(a.workload, a.eps, a.steps, a.w_max)
    if a.top_k > 0:
        inst = dataclasses.replace(inst, top_k=a.top_k)
    h = pp.Handle(inst.n_qubits, precision=a.precision, max_terms=a.max_terms, timing=True)
    h.load_instance(inst)
    h.pp_set_tuning(a.fused_gates, a.headroom, a.first_tier, int(a.orbit_tiles),
                    tile_caps=[int(v) for v in a.tile_caps.split(",")])
    for _ in range(a.repeat):
        h.run_instance(inst)
    e = h.pp_expect()
    s = h.pp_get_stats()
    print(json.dumps({"workload": inst.name, "eps": inst.eps, "w_max": inst.w_max, "precision": a.precision,
                      "expect": e, "updates": s.updates, "terms": s.n_terms, "peak_terms": s.peak_terms,
                      "tier_launches": list(s.tier_launches), "tier_ms": list(s.tier_ms),
                      "tier_strings": list(s.tier_strings), "bytes_per_string": s.bytes_per_string,
                      "kernel_launches": s.kernel_launches, "orbit_launches": s.orbit_launches,
                      "seconds": s.seconds,
                      "tuning": h.tuning()}), flush=True)
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
