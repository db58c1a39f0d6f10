"""Seeded synthetic workloads for noisy-inverse Pauli propagation.

The paper studies Trotterised 2D transverse-field-Ising circuits (Sec. II, Fig. 2:
3x3 lattice; Fig. 3: 4x5 lattice; Sec. III: 56 qubits) whose two-qubit layers are
each followed by a sparse Pauli-Lindblad noise channel (Sec. I, the Lambda_t
product form).  This module builds such circuits, with uniform random noise rates
standing in for a learned device noise model, as flat bit-packed arrays that both
the CUDA path and the CPU oracle consume.

It holds none of the method's arithmetic: no cosines, no exponentials, no
anticommutation tests.  It only lays out lattices, gate lists, rates and
observables, drawing every random number from SplitMix64 so that the CUDA path,
the oracle and the benchmarks see the same instance.

Bit layout of a Pauli string on n qubits: W = ceil(n/64) little-endian uint64
words for the X part and W for the Z part; bit q of word q//64 is qubit q.
Letter (x,z): (0,0)=I, (1,0)=X, (1,1)=Y, (0,1)=Z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1

NOISE_INVERSE = 0   # scale by exp(+2 * sum lambda)  (the antinoise map, Eq. evolve_noise)
NOISE_FORWARD = 1   # scale by exp(-2 * sum lambda)  (the physical channel)

LETTERS = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
PAIR_ORDER = [a + b for a in "XYZ" for b in "XYZ"]   # XX, XY, XZ, YX, ..., ZZ


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014); doubles are (u >> 11) * 2^-53."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, k: int) -> int:
        """Integer uniform in [0, k)."""
        return min(int(self.uniform() * k), k - 1)


def n_words(n_qubits: int) -> int:
    return max(1, (n_qubits + 63) // 64)


def mask_from_sites(sites: Sequence[int], W: int) -> np.ndarray:
    m = np.zeros(W, dtype=np.uint64)
    for q in sites:
        m[q // 64] |= np.uint64(1) << np.uint64(q % 64)
    return m


def pauli_from_letters(letters: dict, W: int) -> Tuple[np.ndarray, np.ndarray]:
    """{qubit: 'X'|'Y'|'Z'} -> (x words, z words)."""
    x = np.zeros(W, dtype=np.uint64)
    z = np.zeros(W, dtype=np.uint64)
    for q, L in letters.items():
        bx, bz = LETTERS[L]
        bit = np.uint64(1) << np.uint64(q % 64)
        if bx:
            x[q // 64] |= bit
        if bz:
            z[q // 64] |= bit
    return x, z


@dataclasses.dataclass
class NoiseLayer:
    """Sparse Pauli-Lindblad generators E_k with rates lambda_k >= 0 attached after `layer`."""
    layer: int
    ex: np.ndarray    # uint64 [K, W]
    ez: np.ndarray    # uint64 [K, W]
    lam: np.ndarray   # float64 [K]
    mode: int = NOISE_INVERSE


@dataclasses.dataclass
class Instance:
    """A circuit of Pauli rotations exp(-i theta R / 2) grouped into layers of
    pairwise-commuting gates (time order: layer 0 first), sparse Pauli-Lindblad
    noise after chosen layers, an observable, and truncation settings."""
    name: str
    n_qubits: int
    gate_x: np.ndarray       # uint64 [G, W]
    gate_z: np.ndarray       # uint64 [G, W]
    theta: np.ndarray        # float64 [G]
    layer_of: np.ndarray     # int32 [G], non-decreasing
    n_layers: int
    noise: List[NoiseLayer]
    obs_x: np.ndarray        # uint64 [T, W]
    obs_z: np.ndarray        # uint64 [T, W]
    obs_c: np.ndarray        # float64 [T]
    eps: float = 0.0
    w_max: int = -1
    meta: dict = dataclasses.field(default_factory=dict)
    top_k: int = 0           # > 0: keep at most this many terms after each layer

    @property
    def W(self) -> int:
        return n_words(self.n_qubits)

    @property
    def n_gates(self) -> int:
        return int(self.theta.shape[0])

    def with_truncation(self, eps: float, w_max: int = -1) -> "Instance":
        return dataclasses.replace(self, eps=float(eps), w_max=int(w_max))

    def with_noise_mode(self, mode: int) -> "Instance":
        return dataclasses.replace(self, noise=[dataclasses.replace(m, mode=int(mode))
                                                for m in self.noise])


# --------------------------------------------------------------------------- lattices

def square_lattice(rows: int, cols: int) -> Tuple[List[Tuple[int, int]], List[int]]:
    """Open-boundary square lattice, site index r*cols + c.

    Returns the edges in canonical order and each edge's colour.  The four
    colours are perfect-matching layers: horizontal edges starting at an even
    column, horizontal edges starting at an odd column, vertical edges starting
    at an even row, vertical edges starting at an odd row; each row-major.
    """
    edges, colour = [], []
    for par in (0, 1):
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                edges.append((r * cols + c, r * cols + c + 1))
                colour.append(par)
    for par in (0, 1):
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                edges.append((r * cols + c, (r + 1) * cols + c))
                colour.append(2 + par)
    return edges, colour


def lattice_generators(n: int, edges: Sequence[Tuple[int, int]], W: int):
    """Generator set of one noise layer: X, Y, Z on every site (site order), then
    the 9 two-qubit letter pairs XX, XY, ..., ZZ on every edge (edge order)."""
    ex, ez = [], []
    for q in range(n):
        for L in "XYZ":
            x, z = pauli_from_letters({q: L}, W)
            ex.append(x)
            ez.append(z)
    for (a, b) in edges:
        for P in PAIR_ORDER:
            x, z = pauli_from_letters({a: P[0], b: P[1]}, W)
            ex.append(x)
            ez.append(z)
    return np.array(ex, dtype=np.uint64).reshape(-1, W), np.array(ez, dtype=np.uint64).reshape(-1, W)


def tfim_instance(name: str, rows: int, cols: int, steps: int, theta_zz: float,
                  theta_x, rates: np.ndarray, obs: Sequence[Tuple[dict, float]],
                  eps: float = 0.0, w_max: int = -1, noise_after: str = "zz",
                  noise_mode: int = NOISE_INVERSE, meta: Optional[dict] = None) -> Instance:
    """First-order TFIM Trotter circuit on a rows x cols open square lattice.

    Time order of step s: layer 2s = R_ZZ(theta_zz) on every edge (canonical
    edge order); layer 2s+1 = R_X(theta_x[q]) on every site q (ascending).  The
    noise of step s (rates[s]) follows the R_ZZ layer (noise_after="zz", the
    paper's placement after each two-qubit layer, Fig. 2a) or the R_X layer
    (noise_after="x").  Gates in a layer are listed in the order the backward
    propagation applies them.
    """
    n = rows * cols
    W = n_words(n)
    edges, colour = square_lattice(rows, cols)
    tx = np.broadcast_to(np.asarray(theta_x, dtype=np.float64), (n,)).copy()
    gx, gz, th, lay = [], [], [], []
    for s in range(steps):
        for (a, b) in edges:
            x, z = pauli_from_letters({a: "Z", b: "Z"}, W)
            gx.append(x); gz.append(z); th.append(float(theta_zz)); lay.append(2 * s)
        for q in range(n):
            x, z = pauli_from_letters({q: "X"}, W)
            gx.append(x); gz.append(z); th.append(float(tx[q])); lay.append(2 * s + 1)
    ex, ez = lattice_generators(n, edges, W)
    rates = np.asarray(rates, dtype=np.float64).reshape(steps, ex.shape[0])
    noise = []
    for s in range(steps):
        layer = 2 * s if noise_after == "zz" else 2 * s + 1
        noise.append(NoiseLayer(layer, ex.copy(), ez.copy(), rates[s].copy(), noise_mode))
    ox, oz, oc = [], [], []
    for letters, c in obs:
        x, z = pauli_from_letters(letters, W)
        ox.append(x); oz.append(z); oc.append(float(c))
    m = dict(rows=rows, cols=cols, steps=steps, theta_zz=float(theta_zz),
             edges=edges, colour=colour, noise_after=noise_after)
    if meta:
        m.update(meta)
    return Instance(name=name, n_qubits=n,
                    gate_x=np.array(gx, dtype=np.uint64).reshape(-1, W),
                    gate_z=np.array(gz, dtype=np.uint64).reshape(-1, W),
                    theta=np.array(th, dtype=np.float64),
                    layer_of=np.array(lay, dtype=np.int32), n_layers=2 * steps,
                    noise=noise,
                    obs_x=np.array(ox, dtype=np.uint64).reshape(-1, W),
                    obs_z=np.array(oz, dtype=np.uint64).reshape(-1, W),
                    obs_c=np.array(oc, dtype=np.float64),
                    eps=float(eps), w_max=int(w_max), meta=m)


def draw_rates(rng: SplitMix64, steps: int, n_gen: int, hi: float) -> np.ndarray:
    """Rates uniform in [0, hi), drawn step-major then in generator order."""
    r = np.empty((steps, n_gen), dtype=np.float64)
    for s in range(steps):
        for k in range(n_gen):
            r[s, k] = rng.uniform(0.0, hi)
    return r


def n_lattice_generators(rows: int, cols: int) -> int:
    n = rows * cols
    return 3 * n + 9 * len(square_lattice(rows, cols)[0])


# --------------------------------------------------------------------------- workloads

SEED_BASE = 20441
EPS_SET = (1e-4, 1e-5, 1e-6, 1e-7)


def workload_3x3(steps: int = 4, seed: int = SEED_BASE + 1) -> Instance:
    """3x3, 4 steps, R_ZZ(0.2), R_X(0.5), O = (1/9) sum_i Z_i, rates U[0,1e-3), no truncation."""
    rng = SplitMix64(seed)
    rows = cols = 3
    rates = draw_rates(rng, steps, n_lattice_generators(rows, cols), 1e-3)
    obs = [({q: "Z"}, 1.0 / 9.0) for q in range(9)]
    return tfim_instance("tfim3x3_s%d" % steps, rows, cols, steps, 0.2, 0.5, rates, obs)


def workload_6x6(steps: int = 10, eps: float = 1e-5, seed: int = SEED_BASE + 2) -> Instance:
    """6x6, 10 steps, R_ZZ(0.3), per-site R_X U[0.2,0.8), O = Z_14 (site (2,2)),
    rates U[0,2e-3), eps = 1e-5, no weight cap.  Angles are drawn first (site
    order), then rates."""
    rng = SplitMix64(seed)
    rows = cols = 6
    tx = np.array([rng.uniform(0.2, 0.8) for _ in range(rows * cols)])
    rates = draw_rates(rng, steps, n_lattice_generators(rows, cols), 2e-3)
    centre = ((rows - 1) // 2) * cols + (cols - 1) // 2
    return tfim_instance("tfim6x6_s%d" % steps, rows, cols, steps, 0.3, tx, rates,
                         [({centre: "Z"}, 1.0)], eps=eps)


def workload_7x8(eps: float = 1e-5, w_max: int = 10, steps: int = 20,
                 seed: int = SEED_BASE + 3) -> Instance:
    """7x8, 20 steps, R_ZZ(0.3), R_X(0.6), O = mean of Z_a Z_b over the 97 edges,
    rates U[0,1e-3), threshold eps from {1e-4..1e-7}, weight cap 10."""
    rng = SplitMix64(seed)
    rows, cols = 7, 8
    edges, _ = square_lattice(rows, cols)
    rates = draw_rates(rng, steps, n_lattice_generators(rows, cols), 1e-3)
    obs = [({a: "Z", b: "Z"}, 1.0 / len(edges)) for (a, b) in edges]
    return tfim_instance("tfim7x8_s%d_eps%g" % (steps, eps), rows, cols, steps, 0.3, 0.6,
                         rates, obs, eps=eps, w_max=w_max)


def random_tfim(rng: SplitMix64, name: str, side_lo: int, side_hi: int, steps_lo: int,
                steps_hi: int, eps: float, rate_hi: float = 2e-3,
                zz_range=(0.1, 0.5), x_range=(0.2, 0.9), w_max: int = -1) -> Instance:
    """One random instance: rows, cols uniform in [side_lo, side_hi], steps
    uniform in [steps_lo, steps_hi], scalar angles, observable a random Z_i or a
    random edge Z_a Z_b.  Draw order: rows, cols, steps, theta_zz, theta_x,
    observable kind, observable site/edge, then rates."""
    rows = side_lo + rng.randint(side_hi - side_lo + 1)
    cols = side_lo + rng.randint(side_hi - side_lo + 1)
    steps = steps_lo + rng.randint(steps_hi - steps_lo + 1)
    tzz = rng.uniform(*zz_range)
    tx = rng.uniform(*x_range)
    edges, _ = square_lattice(rows, cols)
    if rng.uniform() < 0.5:
        obs = [({rng.randint(rows * cols): "Z"}, 1.0)]
    else:
        a, b = edges[rng.randint(len(edges))]
        obs = [({a: "Z", b: "Z"}, 1.0)]
    rates = draw_rates(rng, steps, n_lattice_generators(rows, cols), rate_hi)
    return tfim_instance(name, rows, cols, steps, tzz, tx, rates, obs, eps=eps, w_max=w_max)


def workload_batch64(count: int = 64, eps: float = 1e-6, seed: int = SEED_BASE + 4,
                     w_max: int = -1) -> List[Instance]:
    """64 independent instances: lattices 4x4..8x8, 5-25 steps, R_ZZ U[0.1,0.5),
    R_X U[0.2,0.9), random Z_i or Z_aZ_b, rates U[0,2e-3), eps = 1e-6 (the
    benchmark uses eps = 1e-4 and w_max = 8: at 1e-6, and at 1e-5 with w_max = 10,
    most instances outgrow a GPU)."""
    rng = SplitMix64(seed)
    return [random_tfim(rng, "batch%02d" % i, 4, 8, 5, 25, eps, w_max=w_max) for i in range(count)]


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    instance: Instance


def workload_serving(count: int = 2000, rate_hz: float = 200.0,
                     seed: int = SEED_BASE + 5, side_hi: int = 10,
                     steps_hi: int = 30, eps_set: Sequence[float] = EPS_SET,
                     w_max: int = -1) -> List[Request]:
    """Poisson stream: exponential inter-arrival times at rate_hz; lattices
    4x4..10x10 (up to 100 qubits, 2 words per mask), 5-30 steps, eps drawn from
    {1e-4, 1e-5, 1e-6, 1e-7}.  Draw order per request: inter-arrival time, eps
    index, then the instance draws of random_tfim."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        eps = eps_set[rng.randint(len(eps_set))]
        inst = random_tfim(rng, "req%04d" % i, 4, side_hi, 5, steps_hi, eps, w_max=w_max)
        out.append(Request(i, t, inst))
    return out


def layer_range(inst: Instance, lo: int, hi: int) -> Instance:
    """The instance restricted to its layers lo..hi-1 in time, renumbered from
    0, with the noise maps attached to them; observable and truncation
    unchanged.  Propagating through layers [k, L) and then, from the result,
    through [0, k) is the same backward pass as through [0, L): a checkpoint
    of a propagation is its exported result after the later layers."""
    keep = (inst.layer_of >= lo) & (inst.layer_of < hi)
    noise = [dataclasses.replace(m, layer=m.layer - lo) for m in inst.noise if lo <= m.layer < hi]
    return dataclasses.replace(inst, name="%s[%d:%d]" % (inst.name, lo, hi), gate_x=inst.gate_x[keep],
                               gate_z=inst.gate_z[keep], theta=inst.theta[keep],
                               layer_of=(inst.layer_of[keep] - lo).astype(np.int32), n_layers=hi - lo,
                               noise=noise)


def mirror_instance(inst: Instance) -> Instance:
    """The circuit followed by its exact inverse (gates reversed, angles negated,
    no noise): the Heisenberg image of any observable is the observable itself
    (the mirror construction of Sec. II, Fig. 2a)."""
    G = inst.n_gates
    L = inst.n_layers
    order = []
    for l in range(L):
        idx = np.nonzero(inst.layer_of == l)[0]
        order.append(idx)
    gx, gz, th, lay = [inst.gate_x], [inst.gate_z], [inst.theta], [inst.layer_of]
    for k, l in enumerate(range(L - 1, -1, -1)):
        idx = order[l][::-1]
        gx.append(inst.gate_x[idx]); gz.append(inst.gate_z[idx])
        th.append(-inst.theta[idx]); lay.append(np.full(len(idx), L + k, dtype=np.int32))
    return dataclasses.replace(inst, name=inst.name + "_mirror",
                               gate_x=np.concatenate(gx), gate_z=np.concatenate(gz),
                               theta=np.concatenate(th), layer_of=np.concatenate(lay),
                               n_layers=2 * L, noise=[])


# --------------------------------------------------------------------------- paper-shaped variants

def heavy_hex_56() -> Tuple[int, List[Tuple[int, int]], List[int]]:
    """A 56-qubit heavy-hex patch (the connectivity of the Sec. III device
    runs): three rows of 16 qubits, joined by 4 bridge qubits between rows 0
    and 1 (at columns 0, 4, 8, 12) and 4 between rows 1 and 2 (at columns 2, 6,
    10, 14).  Indices: row 0 = 0..15, bridges 16..19, row 1 = 20..35, bridges
    36..39, row 2 = 40..55.  Returns (n, edges, colour) with a proper 3-edge
    colouring (each colour a matching: one layer of two-qubit gates): rows 0
    and 2 alternate colours 0, 1 along the row, row 1 repeats 2, 0, 2, 1; the
    upper bridges take colours 2 (to row 0) and 0 (to row 1), the lower ones 1
    (to row 1) and 2 (to row 2), which are the colours free at their ends."""
    base = [0, 20, 40]
    row_pattern = [[0, 1, 0, 1], [2, 0, 2, 1], [0, 1, 0, 1]]
    edges, colour = [], []
    for r in range(3):
        for c in range(15):
            edges.append((base[r] + c, base[r] + c + 1))
            colour.append(row_pattern[r][c % 4])
    for k, c in enumerate((0, 4, 8, 12)):
        b = 16 + k
        edges += [(base[0] + c, b), (b, base[1] + c)]
        colour += [2, 0]
    for k, c in enumerate((2, 6, 10, 14)):
        b = 36 + k
        edges += [(base[1] + c, b), (b, base[2] + c)]
        colour += [1, 2]
    return 56, edges, colour


def layered_instance(name: str, n: int, layers: Sequence[Sequence[Tuple[dict, float]]],
                     noise_layers: Sequence[int], gens: Tuple[np.ndarray, np.ndarray],
                     rates: np.ndarray, obs: Sequence[Tuple[dict, float]], eps: float = 0.0,
                     w_max: int = -1, noise_mode: int = NOISE_INVERSE,
                     meta: Optional[dict] = None) -> Instance:
    """A circuit given as layers (time order) of commuting rotations, each a
    (Pauli letters, angle) pair; noise with generators `gens` and the rates of
    row k of `rates` follows layer noise_layers[k]."""
    W = n_words(n)
    gx, gz, th, lay = [], [], [], []
    for l, gates in enumerate(layers):
        for letters, theta in gates:
            x, z = pauli_from_letters(letters, W)
            gx.append(x); gz.append(z); th.append(float(theta)); lay.append(l)
    ex, ez = gens
    noise = [NoiseLayer(int(l), ex.copy(), ez.copy(), np.asarray(rates[k], dtype=np.float64).copy(), noise_mode)
             for k, l in enumerate(noise_layers)]
    ox, oz, oc = [], [], []
    for letters, c in obs:
        x, z = pauli_from_letters(letters, W)
        ox.append(x); oz.append(z); oc.append(float(c))
    return Instance(name=name, n_qubits=n,
                    gate_x=np.array(gx, dtype=np.uint64).reshape(-1, W),
                    gate_z=np.array(gz, dtype=np.uint64).reshape(-1, W),
                    theta=np.array(th, dtype=np.float64),
                    layer_of=np.array(lay, dtype=np.int32), n_layers=len(layers),
                    noise=noise,
                    obs_x=np.array(ox, dtype=np.uint64).reshape(-1, W),
                    obs_z=np.array(oz, dtype=np.uint64).reshape(-1, W),
                    obs_c=np.array(oc, dtype=np.float64),
                    eps=float(eps), w_max=int(w_max), meta=dict(meta or {}))


def _mirror_layers(forward: List[List[Tuple[dict, float]]]) -> List[List[Tuple[dict, float]]]:
    """The forward layers, then their inverses in reverse order (angles negated)."""
    back = [[(letters, -theta) for (letters, theta) in reversed(gates)] for gates in reversed(forward)]
    return forward + back


def workload_heavy_hex_mirror(steps: int = 4, theta: float = 0.3, rate_hi: float = 1e-3,
                              obs_edge: Tuple[int, int] = (21, 22), eps: float = 1e-5, w_max: int = 10,
                              seed: int = SEED_BASE + 6, noise_mode: int = NOISE_INVERSE) -> Instance:
    """Sec. III shape: a mirror circuit of first-order TFIM Trotter steps on the
    56-qubit heavy-hex patch.  Forward step: R_X(theta) on every site, then one
    R_ZZ(theta) layer per edge colour (3 layers); the backward half inverts
    the forward half.  Every R_ZZ layer (both halves) is followed by its own
    noise map: X, Y, Z on every site and the 9 letter pairs on every edge,
    rates uniform [0, rate_hi), drawn layer by layer.  With `steps` = 4 there
    are 24 R_ZZ layers (48 CZ layers once each R_ZZ is compiled to two).  The
    observable is Z_a Z_b on one edge (a weight-2 ZZ, as in the device runs)."""
    n, edges, colour = heavy_hex_56()
    fwd: List[List[Tuple[dict, float]]] = []
    for _ in range(steps):
        fwd.append([({q: "X"}, theta) for q in range(n)])
        for col in range(3):
            fwd.append([({a: "Z", b: "Z"}, theta) for (a, b), cc in zip(edges, colour) if cc == col])
    layers = _mirror_layers(fwd)
    zz = [l for l, gates in enumerate(layers) if len(next(iter(gates))[0]) == 2]
    gens = lattice_generators(n, edges, n_words(n))
    rng = SplitMix64(seed)
    rates = draw_rates(rng, len(zz), gens[0].shape[0], rate_hi)
    return layered_instance("heavyhex56_mirror_s%d" % steps, n, layers, zz, gens, rates,
                            [({obs_edge[0]: "Z", obs_edge[1]: "Z"}, 1.0)], eps=eps, w_max=w_max,
                            noise_mode=noise_mode, meta=dict(steps=steps, theta=theta, edges=edges,
                                                             colour=colour))


def workload_trotter2_mirror_3x3(steps: int = 2, theta: float = 0.05, rate_hi: float = 1e-3,
                                 seed: int = SEED_BASE + 7, eps: float = 0.0,
                                 noise_mode: int = NOISE_INVERSE) -> Instance:
    """Sec. II / Fig. 2a shape: the 3x3 lattice evolved forwards, then
    backwards, under second-order Trotter steps of the TFIM: R_X(theta/2),
    then the R_ZZ(theta) edge colours one layer each, then R_X(theta/2).  Each
    two-qubit layer is followed by the noise model of its colour: four models,
    one per colour, drawn once and reused; generators X on every site and ZZ on
    every edge (the paper's {X, ZZ} set), rates uniform [0, rate_hi).  The
    observable is Z on all nine qubits."""
    rows = cols = 3
    n = rows * cols
    edges, colour = square_lattice(rows, cols)
    half = [({q: "X"}, 0.5 * theta) for q in range(n)]
    fwd: List[List[Tuple[dict, float]]] = []
    for _ in range(steps):
        fwd.append(list(half))
        for col in range(4):
            fwd.append([({a: "Z", b: "Z"}, theta) for (a, b), cc in zip(edges, colour) if cc == col])
        fwd.append(list(half))
    layers = _mirror_layers(fwd)
    W = n_words(n)
    ex, ez = [], []
    for q in range(n):
        x, z = pauli_from_letters({q: "X"}, W); ex.append(x); ez.append(z)
    for (a, b) in edges:
        x, z = pauli_from_letters({a: "Z", b: "Z"}, W); ex.append(x); ez.append(z)
    gens = (np.array(ex, dtype=np.uint64).reshape(-1, W), np.array(ez, dtype=np.uint64).reshape(-1, W))
    rng = SplitMix64(seed)
    models = draw_rates(rng, 4, gens[0].shape[0], rate_hi)
    zz_layers, zz_models = [], []
    for l, gates in enumerate(layers):
        letters = gates[0][0]
        if len(letters) == 2:
            a, b = sorted(letters)
            zz_layers.append(l)
            zz_models.append(colour[edges.index((a, b))])
    rates = models[np.array(zz_models, dtype=np.int64)]
    return layered_instance("trotter2_mirror_3x3_s%d" % steps, n, layers, zz_layers, gens, rates,
                            [({q: "Z" for q in range(n)}, 1.0)], eps=eps, noise_mode=noise_mode,
                            meta=dict(steps=steps, theta=theta))


def random_pauli_letters(rng: SplitMix64, sites: Sequence[int]) -> dict:
    return {q: "XYZ"[rng.randint(3)] for q in sites}


def random_circuit(seed: int, n: int, n_layers: int, max_gates: int = 3, max_support: int = 3,
                   noise_prob: float = 0.6, n_gen: int = 4, rate_hi: float = 0.05,
                   n_obs: int = 3, eps: float = 0.0, w_max: int = -1,
                   modes: Sequence[int] = (NOISE_INVERSE, NOISE_FORWARD),
                   angles: Optional[Sequence[float]] = None, gen_weight: int = 2) -> Instance:
    """Random circuit of generic Pauli rotations (any axis, any weight up to
    max_support).  Gates inside a layer act on disjoint qubits, so they commute.
    Noise layers carry n_gen random generators of weight 1-2.  Angles are drawn
    uniformly from [-pi, pi) unless a list of allowed angles is given; noise
    generators have weight 1..gen_weight."""
    rng = SplitMix64(seed)
    W = n_words(n)
    gx, gz, th, lay, noise = [], [], [], [], []
    for l in range(n_layers):
        free = list(range(n))
        for _ in range(1 + rng.randint(max_gates)):
            if not free:
                break
            k = 1 + rng.randint(min(max_support, len(free)))
            sites = []
            for _ in range(k):
                sites.append(free.pop(rng.randint(len(free))))
            x, z = pauli_from_letters(random_pauli_letters(rng, sites), W)
            gx.append(x); gz.append(z); lay.append(l)
            if angles is None:
                th.append(rng.uniform(-math.pi, math.pi))
            else:
                th.append(float(angles[rng.randint(len(angles))]))
        if rng.uniform() < noise_prob:
            ex, ez, lam = [], [], []
            for _ in range(n_gen):
                k = 1 + rng.randint(min(gen_weight, n))
                sites = []
                pool = list(range(n))
                for _ in range(k):
                    sites.append(pool.pop(rng.randint(len(pool))))
                x, z = pauli_from_letters(random_pauli_letters(rng, sites), W)
                ex.append(x); ez.append(z); lam.append(rng.uniform(0.0, rate_hi))
            noise.append(NoiseLayer(l, np.array(ex, dtype=np.uint64).reshape(-1, W),
                                    np.array(ez, dtype=np.uint64).reshape(-1, W),
                                    np.array(lam), int(modes[rng.randint(len(modes))])))
    ox, oz, oc = [], [], []
    for _ in range(n_obs):
        k = 1 + rng.randint(n)
        pool = list(range(n))
        sites = [pool.pop(rng.randint(len(pool))) for _ in range(k)]
        x, z = pauli_from_letters(random_pauli_letters(rng, sites), W)
        ox.append(x); oz.append(z); oc.append(rng.uniform(-1.0, 1.0))
    return Instance(name="random_n%d_s%d" % (n, seed), n_qubits=n,
                    gate_x=np.array(gx, dtype=np.uint64).reshape(-1, W),
                    gate_z=np.array(gz, dtype=np.uint64).reshape(-1, W),
                    theta=np.array(th, dtype=np.float64),
                    layer_of=np.array(lay, dtype=np.int32), n_layers=n_layers, noise=noise,
                    obs_x=np.array(ox, dtype=np.uint64).reshape(-1, W),
                    obs_z=np.array(oz, dtype=np.uint64).reshape(-1, W),
                    obs_c=np.array(oc, dtype=np.float64), eps=eps, w_max=w_max)


def one_qubit_appD(lam1: float, lam2: float) -> Instance:
    """The one-qubit sequence of App. D in circuit form.  Heisenberg order on Z:
    U^dag . U with U = R_Y(pi/4); Lambda_X^{-1}; U = R_Y(-pi/4); Lambda_Z^{-1}.
    As layers in time order: layer 0 (no gates) then Lambda_Z; layer 1 =
    R_Y(-pi/4) then Lambda_X; layer 2 = R_Y(pi/4)."""
    W = 1
    y = pauli_from_letters({0: "Y"}, W)
    X = pauli_from_letters({0: "X"}, W)
    Z = pauli_from_letters({0: "Z"}, W)
    gx = np.array([y[0], y[0]], dtype=np.uint64).reshape(-1, 1)
    gz = np.array([y[1], y[1]], dtype=np.uint64).reshape(-1, 1)
    noise = [NoiseLayer(1, X[0].reshape(1, 1), X[1].reshape(1, 1), np.array([lam1])),
             NoiseLayer(0, Z[0].reshape(1, 1), Z[1].reshape(1, 1), np.array([lam2]))]
    return Instance(name="appD", n_qubits=1, gate_x=gx, gate_z=gz,
                    theta=np.array([-math.pi / 4, math.pi / 4]),
                    layer_of=np.array([1, 2], dtype=np.int32), n_layers=3, noise=noise,
                    obs_x=Z[0].reshape(1, 1), obs_z=Z[1].reshape(1, 1), obs_c=np.array([1.0]))
