"""Thin ctypes binding of libpp (include/pp.h): the same entry points, argument
marshalling only.  Every step of the propagation runs in the library's CUDA
kernels; there is no CPU fallback: if libpp.so is missing or no GPU is
present, the calls raise.

PyTorch supplies device memory and streams: `Handle(..., torch_memory=True)`
routes the library's device allocations through torch's caching allocator and
runs on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpp.so")
N_TIERS = 5   # processing tiers (pp_stats.tier_*)

PP_OK, PP_ERR_ARG, PP_ERR_STATE, PP_ERR_NOMEM, PP_ERR_CAPACITY, PP_ERR_CUDA, PP_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "PP_OK", 1: "PP_ERR_ARG", 2: "PP_ERR_STATE", 3: "PP_ERR_NOMEM",
                4: "PP_ERR_CAPACITY", 5: "PP_ERR_CUDA", 6: "PP_ERR_TIMEOUT"}
PRECISION_FP64, PRECISION_FP32 = 64, 32
NOISE_INVERSE, NOISE_FORWARD = 0, 1

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class pp_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int),
                ("max_terms", ctypes.c_size_t),
                ("alloc", ALLOC_FN),
                ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p),
                ("cuda_stream", ctypes.c_void_p),
                ("timing", ctypes.c_int)]


class pp_stats(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_size_t),
                ("peak_terms", ctypes.c_size_t),
                ("updates", ctypes.c_double),
                ("n_sublayers", ctypes.c_int),
                ("kernel_launches", ctypes.c_int),
                ("fallback_buckets", ctypes.c_int),
                ("seconds", ctypes.c_double),
                ("tier_launches", ctypes.c_int * N_TIERS),
                ("tier_ms", ctypes.c_double * N_TIERS),
                ("tier_strings", ctypes.c_double * N_TIERS),
                ("bytes_per_string", ctypes.c_double),
                ("orbit_launches", ctypes.c_int),
                ("retries", ctypes.c_int),
                ("growths", ctypes.c_int),
                ("capacity", ctypes.c_size_t)]


class pp_batch_item(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_size_t),
                ("ox", ctypes.c_void_p),
                ("oz", ctypes.c_void_p),
                ("oc", ctypes.c_void_p),
                ("eps", ctypes.c_double),
                ("w_max", ctypes.c_int)]


class pp_tuning(ctypes.Structure):
    _fields_ = [("max_fused_gates", ctypes.c_int),
                ("bucket_headroom", ctypes.c_double),
                ("first_tier", ctypes.c_int),
                ("orbit_tiles", ctypes.c_int),
                ("tile_cap", ctypes.c_int * 4)]


class PPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


EXPORTED = ["pp_default_options", "pp_create", "pp_destroy", "pp_load_circuit", "pp_load_noise",
            "pp_propagate", "pp_expect", "pp_export_terms", "pp_get_stats", "pp_last_error",
            "pp_expect_noalloc", "pp_propagate_batch", "pp_set_tuning", "pp_get_tuning", "pp_set_top_k",
            "pp_cancel"]
NOALLOC_MAX_TERMS = 1 << 27

_lib = None


def _guarded_alloc(fn):
    """An allocation callback for the library: fn(nbytes) returns a device
    pointer.  Whatever fn raises (torch's OutOfMemoryError, say) becomes NULL,
    which the library reports as PP_ERR_NOMEM with the handle intact.  The
    guard is required: an exception escaping a ctypes callback leaves its
    return value unset, and the library would receive an arbitrary pointer."""
    def cb(nbytes, ctx):
        try:
            ptr = fn(int(nbytes))
            return int(ptr) if ptr else None
        except BaseException:   # nothing may propagate into C; NULL reports the failure
            return None
    return cb


def _guarded_free(fn):
    """A free callback for the library; an exception from fn(ptr) is dropped
    (it cannot propagate into C)."""
    def cb(ptr, ctx):
        try:
            fn(ptr)
        except BaseException:   # nothing may propagate into C
            pass
    return cb


def load_library(path: Optional[str] = None):
    """Loads libpp.so (raises OSError if it was not built).  The environment
    variable PP_LIBRARY selects another build of the library, e.g. the debug
    build (build.DEBUG_LIB) with device bounds checks."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PP_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise OSError("libpp.so not built at %s (run paper_2606_20441_b300.build.build())" % path)
    L = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    L.pp_default_options.argtypes = [ctypes.POINTER(pp_options)]
    L.pp_default_options.restype = None
    L.pp_create.argtypes = [ctypes.POINTER(pp_options), ctypes.c_int, ctypes.POINTER(vp)]
    L.pp_destroy.argtypes = [vp]
    L.pp_load_circuit.argtypes = [vp, sz, vp, vp, vp, vp, ctypes.c_int]
    L.pp_load_noise.argtypes = [vp, ctypes.c_int, sz, vp, vp, vp, ctypes.c_int]
    L.pp_propagate.argtypes = [vp, sz, vp, vp, vp, ctypes.c_double, ctypes.c_int]
    L.pp_expect.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.pp_export_terms.argtypes = [vp, sz, vp, vp, vp, ctypes.POINTER(sz)]
    L.pp_get_stats.argtypes = [vp, ctypes.POINTER(pp_stats)]
    L.pp_last_error.argtypes = [vp]
    L.pp_last_error.restype = ctypes.c_char_p
    L.pp_expect_noalloc.argtypes = [ctypes.c_int, sz, vp, vp, vp, vp]
    L.pp_propagate_batch.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(pp_batch_item),
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.pp_set_tuning.argtypes = [vp, ctypes.POINTER(pp_tuning)]
    L.pp_set_top_k.argtypes = [vp, sz]
    L.pp_cancel.argtypes = [vp]
    L.pp_get_tuning.argtypes = [vp, ctypes.POINTER(pp_tuning)]
    for f in EXPORTED:
        if f not in ("pp_default_options", "pp_last_error"):
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Handle:
    """One pp_handle: a circuit, its noise maps, and the last propagation."""

    def __init__(self, n_qubits: int, precision: int = PRECISION_FP64, max_terms: int = 0,
                 torch_memory: bool = False, stream: Optional[int] = None, timing: bool = False,
                 allocator=None):
        """stream: a cudaStream_t (as int) to run on; None = the legacy default stream.
        timing: record per-tier device times (pp_stats.tier_ms).
        allocator: optional (alloc(nbytes) -> device pointer or 0, free(ptr)) pair of
        Python callables used for every device allocation of the handle."""
        self.L = load_library()
        self.n_qubits = n_qubits
        self.W = inputs.n_words(n_qubits)
        opt = pp_options()
        self.L.pp_default_options(ctypes.byref(opt))
        opt.precision = precision
        opt.max_terms = max_terms
        opt.timing = int(bool(timing))
        self._cb = None
        if allocator is not None:
            a_fn, f_fn = allocator
            self._cb = (ALLOC_FN(_guarded_alloc(a_fn)), FREE_FN(_guarded_free(f_fn)))
            opt.alloc, opt.free = self._cb
            if stream is not None:
                opt.cuda_stream = stream
        elif torch_memory:
            import torch
            dev = torch.cuda.current_device()
            # blocks are cached per stream: allocate on the stream that uses them
            st = torch.cuda.current_stream().cuda_stream if stream is None else stream

            self._cb = (ALLOC_FN(_guarded_alloc(lambda n: torch.cuda.caching_allocator_alloc(n, dev, st))),
                        FREE_FN(_guarded_free(torch.cuda.caching_allocator_delete)))
            opt.alloc, opt.free = self._cb
            opt.cuda_stream = st
        elif stream is not None:
            opt.cuda_stream = stream
        h = ctypes.c_void_p()
        st_ = self.L.pp_create(ctypes.byref(opt), n_qubits, ctypes.byref(h))
        if st_ != PP_OK:
            raise PPError(st_, "pp_create failed")
        self.h = h

    def _check(self, status: int):
        if status != PP_OK:
            raise PPError(status, self.L.pp_last_error(self.h).decode())

    def last_error(self) -> str:
        return self.L.pp_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            self.L.pp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pp_load_circuit(self, rx: np.ndarray, rz: np.ndarray, theta: np.ndarray,
                        layer_of: np.ndarray, n_layers: int):
        rx = np.ascontiguousarray(rx, dtype=np.uint64)
        rz = np.ascontiguousarray(rz, dtype=np.uint64)
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        layer_of = np.ascontiguousarray(layer_of, dtype=np.int32)
        self._check(self.L.pp_load_circuit(self.h, len(theta), _p(rx), _p(rz), _p(theta),
                                           _p(layer_of), int(n_layers)))

    def pp_load_noise(self, layer: int, ex: np.ndarray, ez: np.ndarray, lam: np.ndarray,
                      mode: int = NOISE_INVERSE):
        ex = np.ascontiguousarray(ex, dtype=np.uint64)
        ez = np.ascontiguousarray(ez, dtype=np.uint64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._check(self.L.pp_load_noise(self.h, int(layer), len(lam), _p(ex), _p(ez), _p(lam),
                                         int(mode)))

    def pp_propagate(self, ox: np.ndarray, oz: np.ndarray, oc: np.ndarray, eps: float = 0.0,
                     w_max: int = -1):
        ox = np.ascontiguousarray(ox, dtype=np.uint64)
        oz = np.ascontiguousarray(oz, dtype=np.uint64)
        oc = np.ascontiguousarray(oc, dtype=np.float64)
        self._check(self.L.pp_propagate(self.h, len(oc), _p(ox), _p(oz), _p(oc), float(eps),
                                        int(w_max)))

    def pp_expect(self) -> float:
        v = ctypes.c_double()
        self._check(self.L.pp_expect(self.h, ctypes.byref(v)))
        return v.value

    def pp_export_terms(self):
        n = ctypes.c_size_t()
        self._check(self.L.pp_export_terms(self.h, 0, None, None, None, ctypes.byref(n)))
        N = n.value
        x = np.zeros((N, self.W), dtype=np.uint64)
        z = np.zeros((N, self.W), dtype=np.uint64)
        c = np.zeros(N, dtype=np.float64)
        self._check(self.L.pp_export_terms(self.h, N, _p(x), _p(z), _p(c), ctypes.byref(n)))
        return x, z, c

    def pp_cancel(self):
        """Stops the propagation running on this handle in another thread
        (it raises PPError with PP_ERR_TIMEOUT there)."""
        self._check(self.L.pp_cancel(self.h))

    def pp_set_top_k(self, top_k: int):
        self._check(self.L.pp_set_top_k(self.h, int(top_k)))

    def pp_get_stats(self) -> pp_stats:
        s = pp_stats()
        self._check(self.L.pp_get_stats(self.h, ctypes.byref(s)))
        return s

    def pp_set_tuning(self, max_fused_gates: int = 0, bucket_headroom: float = 0.0, first_tier: int = 0,
                      orbit_tiles: int = 0, tile_caps=(0, 0, 0, 0)):
        caps = (ctypes.c_int * 4)(*[int(c) for c in tuple(tile_caps) + (0,) * (4 - len(tile_caps))])
        t = pp_tuning(int(max_fused_gates), float(bucket_headroom), int(first_tier), int(orbit_tiles), caps)
        self._check(self.L.pp_set_tuning(self.h, ctypes.byref(t)))

    def pp_get_tuning(self):
        """(max_fused_gates, bucket_headroom) in effect."""
        t = pp_tuning()
        self._check(self.L.pp_get_tuning(self.h, ctypes.byref(t)))
        return t.max_fused_gates, t.bucket_headroom

    def tuning(self) -> dict:
        """Every tuning field in effect."""
        t = pp_tuning()
        self._check(self.L.pp_get_tuning(self.h, ctypes.byref(t)))
        d = {f: getattr(t, f) for f, _ in pp_tuning._fields_}
        d["tile_cap"] = list(d["tile_cap"])
        return d

    # convenience: a whole Instance
    def load_instance(self, inst: "inputs.Instance"):
        """A handle for n qubits runs any instance on at most n qubits with the
        same number of mask words."""
        if inst.n_qubits > self.n_qubits or inst.W != self.W:
            raise ValueError("instance on %d qubits does not fit a handle for %d" % (inst.n_qubits, self.n_qubits))
        self.pp_load_circuit(inst.gate_x, inst.gate_z, inst.theta, inst.layer_of, inst.n_layers)
        for m in inst.noise:
            self.pp_load_noise(m.layer, m.ex, m.ez, m.lam, m.mode)

    def run_instance(self, inst: "inputs.Instance", eps: Optional[float] = None,
                     w_max: Optional[int] = None):
        self.pp_set_top_k(getattr(inst, "top_k", 0))
        self.pp_propagate(inst.obs_x, inst.obs_z, inst.obs_c,
                          inst.eps if eps is None else eps,
                          inst.w_max if w_max is None else w_max)


def pp_propagate_batch(handles, instances, max_threads: int = 16, eps=None, w_max=None):
    """pp_propagate for many handles at once, in lockstep (handles of one
    device, mask width and precision advance one fused sub-layer per step, each
    kernel launched once per step for all of them); returns the per-item
    status list.  max_threads is ignored by the library."""
    L = load_library()
    n = len(handles)
    keep = []
    items = (pp_batch_item * max(n, 1))()
    for k, (h, inst) in enumerate(zip(handles, instances)):
        ox = np.ascontiguousarray(inst.obs_x, dtype=np.uint64)
        oz = np.ascontiguousarray(inst.obs_z, dtype=np.uint64)
        oc = np.ascontiguousarray(inst.obs_c, dtype=np.float64)
        keep += [ox, oz, oc]
        items[k] = pp_batch_item(len(oc), _p(ox).value, _p(oz).value, _p(oc).value,
                                 float(inst.eps if eps is None else eps),
                                 int(inst.w_max if w_max is None else w_max))
    hs = (ctypes.c_void_p * max(n, 1))(*[h.h.value for h in handles])
    st = (ctypes.c_int * max(n, 1))()
    L.pp_propagate_batch(n, hs, items, int(max_threads), st)
    return [st[k] for k in range(n)]


def pp_expect_noalloc(n_qubits: int, n_terms: int, x_dev: int, c_dev: int, value_dev: int,
                      stream: Optional[int] = None) -> int:
    """<0..0|O~|0..0> of terms in caller-owned device buffers (x masks row-major
    [n_terms][W], FP64 coefficients), written to the device double at value_dev,
    without any device allocation.  Returns the pp_status."""
    return load_library().pp_expect_noalloc(int(n_qubits), int(n_terms), x_dev, c_dev, value_dev, stream)


@dataclasses.dataclass
class Result:
    x: np.ndarray
    z: np.ndarray
    c: np.ndarray
    expect: float
    stats: pp_stats


def propagate(inst: "inputs.Instance", precision: int = PRECISION_FP64, max_terms: int = 0,
              export: bool = True, eps: Optional[float] = None,
              w_max: Optional[int] = None) -> Result:
    """One-shot: load, propagate, expectation (and the exported terms)."""
    h = Handle(inst.n_qubits, precision=precision, max_terms=max_terms)
    try:
        h.load_instance(inst)
        h.run_instance(inst, eps, w_max)
        e = h.pp_expect()
        if export:
            x, z, c = h.pp_export_terms()
        else:
            x = z = c = None
        return Result(x, z, c, e, h.pp_get_stats())
    finally:
        h.close()
