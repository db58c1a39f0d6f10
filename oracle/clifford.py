"""Single-path propagation at Clifford angles (TEST INFRASTRUCTURE ONLY).

At theta in {0, pi/2, pi, -pi/2} every Pauli rotation is a Clifford gate, so a
Pauli string maps to exactly one string and there is no truncation error
(Sec. III: Clifford points).  Along that single path the coefficient picks up
sin/cos signs from the gates and the product of noise factors exp(+-2 sum
lambda) over generators anticommuting with the current string -- the
closed-form rescaling of App. A (the Clifford case O~ = O prod (1 - 2 q)).

This module follows each observable term independently with symplectic bit
arithmetic: anticommutation from the symplectic form x_p.z_r + z_p.x_r (mod 2),
and the phase of a Pauli product from the Aaronson-Gottesman g-function
(Phys. Rev. A 70, 052328, 2004), not from a single-qubit product table.  It
therefore checks the oracle's product table and noise scaling by a different
route, at any qubit count.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np


def _to_int(words) -> int:
    v = 0
    for w in range(len(words)):
        v |= int(words[w]) << (64 * w)
    return v


def symplectic(px: int, pz: int, rx: int, rz: int) -> int:
    return (bin(px & rz).count("1") + bin(pz & rx).count("1")) & 1


def _g(x1, z1, x2, z2) -> int:
    """Exponent of i contributed by one qubit of P1*P2 (Aaronson-Gottesman)."""
    if x1 == 0 and z1 == 0:
        return 0
    if x1 == 1 and z1 == 1:
        return z2 - x2
    if x1 == 1 and z1 == 0:
        return z2 * (2 * x2 - 1)
    return x2 * (1 - 2 * z2)


def product_phase(rx: int, rz: int, px: int, pz: int, n: int) -> int:
    """R * P = i^e * (R xor P); returns e mod 4."""
    e = 0
    for q in range(n):
        e += _g((rx >> q) & 1, (rz >> q) & 1, (px >> q) & 1, (pz >> q) & 1)
    return e % 4


def clifford_trig(theta: float) -> Tuple[int, int]:
    """(cos, sin) of a Clifford angle as exact integers."""
    k = theta / (math.pi / 2)
    kr = int(round(k))
    if abs(k - kr) > 1e-12:
        raise ValueError("not a Clifford angle: %r" % theta)
    return [(1, 0), (0, 1), (-1, 0), (0, -1)][kr % 4]


def propagate(inst, truncate: bool = False, count_updates: bool = False):
    """{(x int, z int): c} for an instance whose angles are all Clifford.

    With truncate, a path ends as soon as its string would be dropped after a
    gate or a noise map (Sec. I.A: |c| < eps or weight > w_max, checked after
    every gate and every noise map; the input observable is checked first).
    With count_updates, also returns the number of live strings entering each
    gate summed over gates (one per path per gate it is alive at), as
    (out, updates)."""
    eps = float(inst.eps) if truncate else 0.0
    w_max = int(inst.w_max) if truncate else -1

    def dropped(px, pz, c):
        if not truncate:
            return False
        return c == 0.0 or abs(c) < eps or (w_max >= 0 and bin(px | pz).count("1") > w_max)
    updates = 0
    n = inst.n_qubits
    gates = [(_to_int(inst.gate_x[g]), _to_int(inst.gate_z[g]), clifford_trig(float(inst.theta[g])),
              int(inst.layer_of[g])) for g in range(inst.n_gates)]
    noise_at: Dict[int, list] = {}
    for m in inst.noise:
        gens = [(_to_int(m.ex[k]), _to_int(m.ez[k]), float(m.lam[k])) for k in range(len(m.lam))]
        noise_at.setdefault(m.layer, []).append((gens, m.mode))
    out: Dict[Tuple[int, int], float] = {}
    for t in range(len(inst.obs_c)):
        px, pz = _to_int(inst.obs_x[t]), _to_int(inst.obs_z[t])
        c = float(inst.obs_c[t])
        alive = not dropped(px, pz, c)
        for l in range(inst.n_layers - 1, -1, -1):
            if not alive:
                break
            for gens, mode in noise_at.get(l, []):
                s = sum(lam for (ex, ez, lam) in gens if symplectic(px, pz, ex, ez))
                c *= math.exp(2.0 * s) if mode == 0 else math.exp(-2.0 * s)
                if dropped(px, pz, c):
                    alive = False
            for (rx, rz, (cs, sn), lay) in gates:
                if not alive or lay != l:
                    continue
                updates += 1
                if not symplectic(px, pz, rx, rz):
                    continue
                if sn == 0:
                    c *= cs
                else:
                    # U^dag P U = cos P + i sin R P, and i R P = i^{1+e} (R xor P)
                    e = product_phase(rx, rz, px, pz, n)
                    tot = (1 + e) % 4
                    assert tot in (0, 2)
                    c *= sn * (1 if tot == 0 else -1)
                    px, pz = px ^ rx, pz ^ rz
                if dropped(px, pz, c):
                    alive = False
        if alive:
            key = (px, pz)
            out[key] = out.get(key, 0.0) + c
    return (out, updates) if count_updates else out
