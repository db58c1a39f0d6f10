"""Python front end of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Builds `liboracle.so` from `pp_oracle.cpp` with g++ (-O2 -ffp-contract=off, so
that no multiply-add is fused) and runs an `Instance` through it.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import this.
The CUDA library never does.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pp_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_qubits", ctypes.c_int),
        ("n_layers", ctypes.c_int),
        ("n_gates", ctypes.c_int64),
        ("gx", ctypes.c_void_p),
        ("gz", ctypes.c_void_p),
        ("theta", ctypes.c_void_p),
        ("layer_of", ctypes.c_void_p),
        ("n_noise", ctypes.c_int),
        ("noise_layer", ctypes.c_void_p),
        ("noise_off", ctypes.c_void_p),
        ("ex", ctypes.c_void_p),
        ("ez", ctypes.c_void_p),
        ("lam", ctypes.c_void_p),
        ("noise_mode", ctypes.c_void_p),
        ("n_obs", ctypes.c_int64),
        ("ox", ctypes.c_void_p),
        ("oz", ctypes.c_void_p),
        ("oc", ctypes.c_void_p),
        ("eps", ctypes.c_double),
        ("w_max", ctypes.c_int),
        ("record", ctypes.c_int),
        ("top_k", ctypes.c_int64),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_run.restype = ctypes.c_void_p
        _lib.orc_run.argtypes = [ctypes.POINTER(_Problem)]
        for name, rt in (("orc_n_terms", ctypes.c_int64), ("orc_expect", ctypes.c_double),
                         ("orc_updates", ctypes.c_double), ("orc_peak", ctypes.c_int64),
                         ("orc_n_records", ctypes.c_int64), ("orc_error", ctypes.c_char_p)):
            getattr(_lib, name).restype = rt
            getattr(_lib, name).argtypes = [ctypes.c_void_p]
        _lib.orc_terms.argtypes = [ctypes.c_void_p] * 4
        _lib.orc_records.argtypes = [ctypes.c_void_p] * 2
        _lib.orc_free.argtypes = [ctypes.c_void_p]
        _lib.orc_anticommute.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 4
        _lib.orc_multiply.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 6
    return _lib


@dataclasses.dataclass
class OracleResult:
    x: np.ndarray        # uint64 [N, W], sorted by (x as integer, then z)
    z: np.ndarray
    c: np.ndarray        # float64 [N]
    expect: float
    updates: float       # sum over gates of live terms entering the gate
    peak: int
    records: Optional[np.ndarray]   # [gates, 4]: mass in, rotated, kept, dropped


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def run(inst, record: bool = False, eps: Optional[float] = None,
        w_max: Optional[int] = None, top_k: Optional[int] = None) -> OracleResult:
    L = lib()
    W = inst.W
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    gx = arr(inst.gate_x.reshape(-1), np.uint64)
    gz = arr(inst.gate_z.reshape(-1), np.uint64)
    th = arr(inst.theta, np.float64)
    lay = arr(inst.layer_of, np.int32)
    nl = arr([m.layer for m in inst.noise] or [0], np.int32)
    nm = arr([m.mode for m in inst.noise] or [0], np.int32)
    off = [0]
    for m in inst.noise:
        off.append(off[-1] + len(m.lam))
    noff = arr(off, np.int64)
    if inst.noise:
        ex = arr(np.concatenate([m.ex.reshape(-1) for m in inst.noise]), np.uint64)
        ez = arr(np.concatenate([m.ez.reshape(-1) for m in inst.noise]), np.uint64)
        lam = arr(np.concatenate([m.lam for m in inst.noise]), np.float64)
    else:
        ex = arr([0] * W, np.uint64)
        ez = arr([0] * W, np.uint64)
        lam = arr([0.0], np.float64)
    ox = arr(inst.obs_x.reshape(-1), np.uint64)
    oz = arr(inst.obs_z.reshape(-1), np.uint64)
    oc = arr(inst.obs_c, np.float64)
    pb = _Problem(inst.n_qubits, inst.n_layers, inst.n_gates, _ptr(gx).value, _ptr(gz).value,
                  _ptr(th).value, _ptr(lay).value, len(inst.noise), _ptr(nl).value,
                  _ptr(noff).value, _ptr(ex).value, _ptr(ez).value, _ptr(lam).value,
                  _ptr(nm).value, len(oc), _ptr(ox).value, _ptr(oz).value,
                  _ptr(oc).value, float(inst.eps if eps is None else eps),
                  int(inst.w_max if w_max is None else w_max), int(record),
                  int(getattr(inst, "top_k", 0) if top_k is None else top_k))
    h = L.orc_run(ctypes.byref(pb))
    try:
        err = L.orc_error(h)
        if err:
            raise RuntimeError("oracle: " + err.decode())
        N = L.orc_n_terms(h)
        x = np.zeros((N, W), dtype=np.uint64)
        z = np.zeros((N, W), dtype=np.uint64)
        c = np.zeros(N, dtype=np.float64)
        if N:
            L.orc_terms(h, _ptr(x), _ptr(z), _ptr(c))
        rec = None
        if record:
            nr = L.orc_n_records(h)
            rec = np.zeros((nr, 4), dtype=np.float64)
            if nr:
                L.orc_records(h, _ptr(rec))
        return OracleResult(x, z, c, L.orc_expect(h), L.orc_updates(h), L.orc_peak(h), rec)
    finally:
        L.orc_free(h)


def anticommute(n: int, p, r) -> int:
    """p, r: (x words, z words) numpy uint64 arrays."""
    px, pz = [np.ascontiguousarray(a, dtype=np.uint64) for a in p]
    rx, rz = [np.ascontiguousarray(a, dtype=np.uint64) for a in r]
    return lib().orc_anticommute(n, _ptr(px), _ptr(pz), _ptr(rx), _ptr(rz))


def multiply(n: int, r, p):
    """r * p -> ((x, z), power of i)."""
    W = (n + 63) // 64
    rx, rz = [np.ascontiguousarray(a, dtype=np.uint64) for a in r]
    px, pz = [np.ascontiguousarray(a, dtype=np.uint64) for a in p]
    qx = np.zeros(W, dtype=np.uint64)
    qz = np.zeros(W, dtype=np.uint64)
    ph = lib().orc_multiply(n, _ptr(rx), _ptr(rz), _ptr(px), _ptr(pz), _ptr(qx), _ptr(qz))
    return (qx, qz), ph
