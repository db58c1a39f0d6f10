"""Writes the oracle's result digest for a workload too slow to run in a test.

    python tests/golden/make_oracle_digest.py tfim7x8_s4_eps1e-5

Runs the CPU oracle (FP64, gate by gate) on the named seeded workload and
stores, in tests/golden/<name>.json: the term count, an order-independent
digest of the term set, <0..0|O~|0..0>, the sum of |c| over diagonal strings
(the scale of the expectation tolerance), the canonical update count, the
number of strings whose |c| lies within 1e-12 relative of the threshold, and a
sample of terms with their exact coefficients.  Only `oracle/` computes these
numbers; the GPU test recomputes the same digest from the library's export.
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_2606_20441_b300 import inputs  # noqa: E402

WORKLOADS = {
    "tfim7x8_s4_eps1e-5": lambda: inputs.workload_7x8(eps=1e-5, w_max=10, steps=4),
}
N_SAMPLE = 2000


def set_digest(x: np.ndarray, z: np.ndarray) -> str:
    """Sum over strings of a 64-bit mix of (x words, z words), modulo 2^64, as
    hex: independent of the order of the terms."""
    h = np.zeros(len(x), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for w in range(x.shape[1]):
            for part, k in ((x[:, w], 0x9E3779B97F4A7C15), (z[:, w], 0xC2B2AE3D27D4EB4F)):
                v = (part ^ np.uint64(k + 2 * w)) * np.uint64(0xFF51AFD7ED558CCD)
                v ^= v >> np.uint64(33)
                v *= np.uint64(0xC4CEB9FE1A85EC53)
                v ^= v >> np.uint64(29)
                h = h * np.uint64(0x100000001B3) + v
        return "%016x" % int(np.sum(h, dtype=np.uint64))


def main(name: str) -> None:
    inst = WORKLOADS[name]()
    t = time.time()
    r = oracle.run(inst)
    sec = time.time() - t
    diag = np.all(r.x == 0, axis=1)
    near = int(np.sum(np.abs(np.abs(r.c) - inst.eps) <= 1e-12 * inst.eps)) if inst.eps > 0 else 0
    idx = np.linspace(0, len(r.c) - 1, num=min(N_SAMPLE, len(r.c))).astype(np.int64)
    out = {
        "workload": name,
        "generator": "tests/golden/make_oracle_digest.py (oracle/ only)",
        "oracle_seconds": sec,
        "n_terms": int(len(r.c)),
        "set_digest": set_digest(r.x, r.z),
        "expect": float(r.expect),
        "diag_abs_sum": float(np.sum(np.abs(r.c[diag]))),
        "updates": float(r.updates),
        "peak": int(r.peak),
        "near_eps": near,
        "sample": {"x": [[int(v) for v in r.x[i]] for i in idx], "z": [[int(v) for v in r.z[i]] for i in idx],
                   "c": [float(r.c[i]).hex() for i in idx]},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json"), "w") as f:
        json.dump(out, f)
    print(name, out["n_terms"], out["expect"], "%.1f s" % sec)


if __name__ == "__main__":
    main(sys.argv[1])
