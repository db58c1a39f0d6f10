"""Dense-matrix checkers for the oracle (TEST INFRASTRUCTURE ONLY).

These compute the same physics as the Pauli-propagation oracle by a different
route, straight from the paper's definitions, so the oracle can be pinned to
something other than itself:

* `density_expect`: the Schroedinger picture.  rho = |0..0><0..0| evolves forward
  through every gate U = expm(-i theta R / 2) (Sec. I, gate form U_t =
  exp(-i R_t theta_t / 2)) and every Pauli-Lindblad map, built generator by
  generator as (1-p) rho + p E rho E with p = (1 - e^{-2 lambda})/2, or, for the
  inverse map, lambda negated (Sec. I, definition of Lambda_t and q); the value
  is Tr[O rho_final] (Sec. II: evaluation against the exact density matrix).
* `heisenberg_coefficients`: the same maps applied to O as a matrix in reverse
  order, then every Pauli coefficient Tr[P O~] / 2^n.
* `ptm_propagate`: brute force for n <= 4 with the per-gate truncation rule: the
  observable as a vector over all 4^n Paulis, each gate/noise map applied as a
  dense matrix conjugation, entries dropped after each gate exactly as the
  oracle does.

Pauli matrices are built as Kronecker products of the textbook 2x2 matrices
(qubit 0 is the least significant bit of the basis index); `pauli_dense_fast`
is a signed-permutation shortcut that the tests check against the Kronecker
construction before it is used.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np
import scipy.linalg

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def _bits(words, n):
    out = []
    for q in range(n):
        out.append(int((int(words[q // 64]) >> (q % 64)) & 1))
    return out


def letters_of(x, z, n):
    xb, zb = _bits(x, n), _bits(z, n)
    return ["IXZY"[xb[q] + 2 * zb[q]] for q in range(n)]


def pauli_dense_kron(x, z, n) -> np.ndarray:
    mats = {"I": I2, "X": PX, "Y": PY, "Z": PZ}
    L = letters_of(x, z, n)
    M = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        M = np.kron(M, mats[L[q]])
    return M


def _int_mask(words, n):
    v = 0
    for q in range(n):
        v |= ((int(words[q // 64]) >> (q % 64)) & 1) << q
    return v


def pauli_perm(x, z, n) -> Tuple[np.ndarray, np.ndarray]:
    """Signed-permutation form: P[b, perm[b]] = val[b], all other entries 0."""
    xi, zi = _int_mask(x, n), _int_mask(z, n)
    dim = 1 << n
    b = np.arange(dim, dtype=np.int64)
    perm = b ^ xi
    # column c = b ^ x; X^x Z^z |c> = (-1)^{z.c} |c ^ x>, P = i^{|x&z|} X^x Z^z
    par = np.zeros(dim, dtype=np.int64)
    cz = perm & zi
    for q in range(n):
        par ^= (cz >> q) & 1
    val = (1j ** bin(xi & zi).count("1")) * np.where(par == 1, -1.0, 1.0)
    return perm, val.astype(np.complex128)


def pauli_dense_fast(x, z, n) -> np.ndarray:
    perm, val = pauli_perm(x, z, n)
    M = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    M[np.arange(1 << n), perm] = val
    return M


def _conj_pauli(P, M):
    """P M P for a Hermitian signed permutation P = (perm, val)."""
    perm, val = P
    return (val[:, None] * M[np.ix_(perm, perm)]) * np.conj(val)[None, :]


def _noise_p(lam: float, mode: int) -> float:
    # physical channel: p = (1 - e^{-2 lambda}) / 2; inverse map: lambda -> -lambda
    l = lam if mode == 1 else -lam
    return (1.0 - math.exp(-2.0 * l)) / 2.0


def _apply_noise(M, layer, n):
    for k in range(len(layer.lam)):
        p = _noise_p(float(layer.lam[k]), layer.mode)
        P = pauli_perm(layer.ex[k], layer.ez[k], n)
        M = (1.0 - p) * M + p * _conj_pauli(P, M)
    return M


def _gate_unitary(inst, g, n):
    R = pauli_dense_fast(inst.gate_x[g], inst.gate_z[g], n)
    return scipy.linalg.expm(-0.5j * float(inst.theta[g]) * R)


def observable_matrix(inst) -> np.ndarray:
    n = inst.n_qubits
    O = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in range(len(inst.obs_c)):
        O += inst.obs_c[t] * pauli_dense_fast(inst.obs_x[t], inst.obs_z[t], n)
    return O


def density_expect(inst) -> float:
    """Tr[O rho] with rho evolved forward in time through gates and noise maps."""
    n = inst.n_qubits
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1.0
    noise_at: Dict[int, list] = {}
    for m in inst.noise:
        noise_at.setdefault(m.layer, []).append(m)
    for l in range(inst.n_layers):
        for g in np.nonzero(inst.layer_of == l)[0]:
            U = _gate_unitary(inst, g, n)
            rho = U @ rho @ U.conj().T
        for m in noise_at.get(l, []):
            rho = _apply_noise(rho, m, n)
    return float(np.real(np.trace(observable_matrix(inst) @ rho)))


def heisenberg_matrix(inst) -> np.ndarray:
    """O~ as a dense matrix: adjoint maps applied to O from the last layer back."""
    n = inst.n_qubits
    O = observable_matrix(inst)
    noise_at: Dict[int, list] = {}
    for m in inst.noise:
        noise_at.setdefault(m.layer, []).append(m)
    for l in range(inst.n_layers - 1, -1, -1):
        for m in noise_at.get(l, []):
            O = _apply_noise(O, m, n)      # Pauli channels are self-adjoint
        for g in np.nonzero(inst.layer_of == l)[0]:
            U = _gate_unitary(inst, g, n)
            O = U.conj().T @ O @ U
    return O


def pauli_coefficients(O: np.ndarray, n: int) -> np.ndarray:
    """c[x, z] = Tr[P_{x,z} O] / 2^n for all 4^n Paulis (x, z as n-bit integers).

    Tr[X^x Z^z O] = sum_c (-1)^{z.c} O[c, c^x]: for each x a Walsh-Hadamard
    transform over c; P = i^{|x & z|} X^x Z^z."""
    dim = 1 << n
    idx = np.arange(dim)
    out = np.zeros((dim, dim), dtype=np.complex128)
    for x in range(dim):
        v = O[idx, idx ^ x].copy()
        h = 1
        while h < dim:
            v = v.reshape(-1, 2, h)
            a = v[:, 0, :].copy()
            b = v[:, 1, :].copy()
            v[:, 0, :] = a + b
            v[:, 1, :] = a - b
            v = v.reshape(dim)
            h *= 2
        # v[z] = sum_c (-1)^{popc(z & c)} O[c, c^x]
        ph = np.array([1j ** bin(x & zz).count("1") for zz in range(dim)])
        out[x, :] = ph * v / dim
    return out


def heisenberg_coefficients(inst) -> np.ndarray:
    return pauli_coefficients(heisenberg_matrix(inst), inst.n_qubits)


def ptm_propagate(inst, zero_tol: float = 1e-13, count_updates: bool = False):
    """Brute force over all 4^n Paulis (n <= 4) with truncation after every gate
    and every noise map.  Returns {(x, z): c} for the surviving strings.

    Dense traces leave rounding residue (~1e-17) on coefficients that are zero
    exactly; entries below `zero_tol` in magnitude count as exact zeros.

    With count_updates, also returns the canonical gate-by-gate work count:
    the number of surviving strings entering each gate, summed over gates
    (counted here on the dense coefficient vector, independently of any hash
    map), as (coef, updates)."""
    n = inst.n_qubits
    assert n <= 5
    dim = 1 << n
    basis = {}
    for xi in range(dim):
        for zi in range(dim):
            basis[(xi, zi)] = pauli_dense_fast([xi], [zi], n)

    def decompose(M):
        return {k: float(np.real(np.trace(P @ M))) / dim for k, P in basis.items()}

    def compose(coef):
        M = np.zeros((dim, dim), dtype=np.complex128)
        for k, c in coef.items():
            if c != 0.0:
                M += c * basis[k]
        return M

    def truncate(coef):
        out = {}
        for (xi, zi), c in coef.items():
            if abs(c) <= zero_tol or abs(c) < inst.eps:
                continue
            if inst.w_max >= 0 and bin(xi | zi).count("1") > inst.w_max:
                continue
            out[(xi, zi)] = c
        return out

    coef = {}
    for t in range(len(inst.obs_c)):
        k = (_int_mask(inst.obs_x[t], n), _int_mask(inst.obs_z[t], n))
        coef[k] = coef.get(k, 0.0) + float(inst.obs_c[t])
    coef = truncate(coef)
    updates = 0
    noise_at: Dict[int, list] = {}
    for m in inst.noise:
        noise_at.setdefault(m.layer, []).append(m)
    for l in range(inst.n_layers - 1, -1, -1):
        for m in noise_at.get(l, []):
            coef = truncate(decompose(_apply_noise(compose(coef), m, n)))
        for g in np.nonzero(inst.layer_of == l)[0]:
            updates += sum(1 for c in coef.values() if c != 0.0)
            U = _gate_unitary(inst, g, n)
            coef = truncate(decompose(U.conj().T @ compose(coef) @ U))
    return (coef, updates) if count_updates else coef
