"""The paper-shaped workload variants: the 56-qubit heavy-hex mirror circuit
(Sec. III shape) and the 3x3 second-order Trotter mirror circuit (Sec. II,
Fig. 2a shape).  Their structure is checked directly; the oracle is checked on
them against the mirror identity (no noise: O comes back exactly) and, on
3x3, against the dense density-matrix simulation."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import dense, oracle
from paper_2606_20441_b300 import inputs


def test_heavy_hex_patch_structure():
    n, edges, colour = inputs.heavy_hex_56()
    assert n == 56 and len(edges) == 61 and len(set(edges)) == 61
    deg = np.zeros(n, dtype=int)
    for a, b in edges:
        assert 0 <= a < n and 0 <= b < n and a != b
        deg[a] += 1
        deg[b] += 1
    assert deg.max() == 3 and deg.min() >= 1
    # degree 3: the row qubits at a bridge end, except row ends (row 0 col 0, row 1 col 0)
    assert int((deg == 3).sum()) == 14
    # heavy-hex: every bridge qubit has degree 2 and joins two rows
    for b in list(range(16, 20)) + list(range(36, 40)):
        assert deg[b] == 2
    # each colour is a matching (a layer of commuting two-qubit gates)
    for col in range(3):
        seen = set()
        for (a, b), c in zip(edges, colour):
            if c == col:
                assert a not in seen and b not in seen
                seen |= {a, b}
    # bipartite (so 3 colours suffice)
    side = [-1] * n
    side[0] = 0
    todo = [0]
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    while todo:
        u = todo.pop()
        for v in adj[u]:
            if side[v] < 0:
                side[v] = 1 - side[u]
                todo.append(v)
            assert side[v] != side[u]


def test_heavy_hex_mirror_returns_observable_without_noise():
    inst = inputs.workload_heavy_hex_mirror(steps=1, theta=0.3, eps=0.0, w_max=-1)
    assert inst.n_qubits == 56 and inst.n_layers == 8 and len(inst.noise) == 6
    quiet = dataclasses.replace(inst, noise=[])
    # no truncation, so that the two halves cancel exactly up to rounding
    r = oracle.run(quiet, eps=0.0)
    k = int(np.argmax(np.abs(r.c)))
    assert np.array_equal(r.x[k], inst.obs_x[0]) and np.array_equal(r.z[k], inst.obs_z[0])
    assert abs(r.c[k] - 1.0) < 1e-12 and abs(r.expect - 1.0) < 1e-12
    assert np.abs(np.delete(r.c, k)).max(initial=0.0) < 1e-13


def test_heavy_hex_mirror_layers():
    inst = inputs.workload_heavy_hex_mirror(steps=4)
    # 4 forward steps of (R_X layer + 3 R_ZZ colour layers), mirrored
    assert inst.n_layers == 32 and len(inst.noise) == 24
    zz_layers = [m.layer for m in inst.noise]
    for l in zz_layers:
        g = np.nonzero(inst.layer_of == l)[0]
        assert all(bin(int(inst.gate_z[k, 0])).count("1") == 2 for k in g)
    # the backward half negates the angles of the forward half, layer by layer
    L = inst.n_layers
    for l in range(L // 2):
        f = np.sort(inst.theta[inst.layer_of == l])
        b = np.sort(-inst.theta[inst.layer_of == L - 1 - l])
        assert np.array_equal(f, b)


def test_trotter2_mirror_structure():
    inst = inputs.workload_trotter2_mirror_3x3(steps=2, theta=0.05)
    assert inst.n_qubits == 9
    # per step: R_X(theta/2), 4 R_ZZ colour layers, R_X(theta/2); mirrored
    assert inst.n_layers == 2 * 2 * 6 and len(inst.noise) == 2 * 2 * 4
    for l in range(inst.n_layers):
        th = inst.theta[inst.layer_of == l]
        assert np.allclose(np.abs(th), 0.025) or np.allclose(np.abs(th), 0.05)
    # four noise models, one per colour, reused by every layer of that colour
    models = {}
    for m in inst.noise:
        key = tuple(sorted(int(inst.gate_z[k, 0]) for k in np.nonzero(inst.layer_of == m.layer)[0]))
        models.setdefault(key, []).append(m.lam)
    assert len(models) == 4
    for lams in models.values():
        for lam in lams[1:]:
            assert np.array_equal(lam, lams[0])
    # the paper's generator set: X on every site, ZZ on every edge
    assert inst.noise[0].ex.shape[0] == 9 + 12


def test_trotter2_mirror_returns_observable_without_noise():
    inst = inputs.workload_trotter2_mirror_3x3(steps=2, theta=0.05)
    r = oracle.run(dataclasses.replace(inst, noise=[]), eps=0.0)
    k = int(np.argmax(np.abs(r.c)))
    assert abs(r.c[k] - 1.0) < 1e-12 and np.array_equal(r.z[k], inst.obs_z[0]) and not r.x[k].any()
    assert np.abs(np.delete(r.c, k)).max(initial=0.0) < 1e-13


@pytest.mark.parametrize("mode", [inputs.NOISE_FORWARD, inputs.NOISE_INVERSE])
def test_trotter2_mirror_oracle_matches_density_matrix(mode):
    inst = inputs.workload_trotter2_mirror_3x3(steps=1, theta=0.05, rate_hi=5e-3).with_noise_mode(mode)
    r = oracle.run(inst)
    d = dense.density_expect(inst)
    assert abs(r.expect - d) < 1e-12
    if mode == inputs.NOISE_FORWARD:
        assert r.expect < 1.0          # noise only damps <Z^9> on the mirror
    else:
        assert r.expect > 1.0          # the inverse map amplifies it
