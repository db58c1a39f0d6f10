"""Autotuner for the sub-layer plan and the tile sizes (pp_set_tuning).

Three knobs shape a propagation's kernels: how many commuting gates are fused
into one sub-layer (fewer passes over the strings, but orbits of up to
2^gates strings per bucket, which push buckets into the slower tiers), the
bucket headroom (how full a warp tile a bucket is planned to be, i.e. how many
buckets a sub-layer's strings are hashed into), and the tile sizes of the two
warp tiers (larger tiles hold larger buckets but leave fewer warps resident).
The best setting depends on lattice size, depth, threshold and weight cap.

Every setting gives the same result, bit for bit: each plan reproduces
gate-by-gate propagation with truncation after every gate.  So tuning can run
on live traffic at no cost in accuracy: the tuner keys requests by workload
class, hands out each candidate in turn for the first requests of a class
(exploration), records the updates per second each one reached, and from then
on gives the class its fastest candidate.  `sweep` tunes one instance
explicitly by running it under every candidate.
"""
from __future__ import annotations

import json
import math
import threading
from typing import Dict, List, Optional, Sequence, Tuple

# (max_fused_gates, bucket_headroom) or (max_fused_gates, bucket_headroom,
# tier-0 tile, tier-1 tile); zeros select the library defaults
Setting = Tuple

# (0, 0.0) is the library default (whole layers, headroom 2.0, tiles 248 and 512)
CANDIDATES: List[Setting] = [(0, 0.0), (32, 2.4), (16, 1.6), (64, 1.6), (0, 0.0, 200, 448), (0, 0.0, 320, 640)]


def _setting(v) -> Setting:
    """A setting from its stored form (numbers or strings)."""
    return tuple([int(float(v[0])), float(v[1])] + [int(float(a)) for a in v[2:]])


def set_tuning(handle, setting: Setting):
    """Applies a setting to a handle (tile sizes 0 = library default)."""
    caps = tuple(setting[2:4]) + (0,) * (4 - len(setting[2:4]))
    handle.pp_set_tuning(setting[0], setting[1], tile_caps=caps)


def class_key(inst) -> str:
    """Workload class: mask words, lattice size band (16 qubits), depth band
    (5 layers), threshold and weight cap."""
    return "W%d_n%d_L%d_eps%g_w%d" % (inst.W, inst.n_qubits // 16, inst.n_layers // 5, inst.eps, inst.w_max)


class Tuner:
    def __init__(self, candidates: Sequence[Setting] = CANDIDATES, trials: int = 1):
        self.candidates = [tuple(c) for c in candidates]
        self.trials = trials
        self._lock = threading.Lock()
        # class -> candidate -> list of updates/s
        self.samples: Dict[str, Dict[Setting, List[float]]] = {}
        self.fixed: Dict[str, Setting] = {}
        self._handed: Dict[str, int] = {}

    # ------------------------------------------------------------ online use
    def choose(self, key: str) -> Setting:
        """The setting the next request of class `key` runs with."""
        with self._lock:
            if key in self.fixed:
                return self.fixed[key]
            k = self._handed.get(key, 0)
            self._handed[key] = k + 1
            if k < len(self.candidates) * self.trials:
                return self.candidates[k % len(self.candidates)]
            return self._best(key)

    def record(self, key: str, setting: Setting, updates_per_s: float):
        with self._lock:
            self.samples.setdefault(key, {}).setdefault(tuple(setting), []).append(float(updates_per_s))

    def _best(self, key: str) -> Setting:
        s = self.samples.get(key)
        if not s:
            return self.candidates[0]
        # median of each candidate's samples; untried candidates rank last
        def score(c):
            v = sorted(s.get(c, []))
            return v[len(v) // 2] if v else -math.inf
        return max(self.candidates, key=score)

    def best(self, key: str) -> Setting:
        with self._lock:
            return self.fixed.get(key) or self._best(key)

    def apply(self, handle, inst) -> Setting:
        """Sets the handle's tuning for this instance; returns the setting."""
        setting = self.choose(class_key(inst))
        set_tuning(handle, setting)
        return setting

    def observe(self, inst, setting: Setting, updates: float, seconds: float):
        if seconds > 0 and updates > 0:
            self.record(class_key(inst), setting, updates / seconds)

    # ------------------------------------------------------------ offline use
    def sweep(self, handle, inst, repeats: int = 1) -> Setting:
        """Runs `inst` under every candidate on `handle` and fixes its class's
        setting to the fastest."""
        key = class_key(inst)
        handle.load_instance(inst)
        for c in self.candidates:
            set_tuning(handle, c)
            for _ in range(repeats):
                handle.run_instance(inst)
                st = handle.pp_get_stats()
                self.record(key, c, st.updates / max(st.seconds, 1e-9))
        with self._lock:
            self.fixed[key] = self._best(key)
            return self.fixed[key]

    # ------------------------------------------------------------ persistence
    def to_json(self) -> str:
        with self._lock:
            return json.dumps({"fixed": {k: list(v) for k, v in self.fixed.items()},
                               "samples": {k: {",".join("%g" % a for a in c): v for c, v in d.items()}
                                           for k, d in self.samples.items()}})

    @classmethod
    def from_json(cls, text: str, candidates: Optional[Sequence[Setting]] = None) -> "Tuner":
        d = json.loads(text)
        t = cls(candidates or CANDIDATES)
        t.fixed = {k: _setting(v) for k, v in d.get("fixed", {}).items()}
        for k, m in d.get("samples", {}).items():
            for cs, v in m.items():
                t.samples.setdefault(k, {})[_setting(cs.split(","))] = list(v)
        for k, m in t.samples.items():
            if all(c in m for c in t.candidates):
                t._handed[k] = len(t.candidates) * t.trials
        return t
