"""The binding's allocator callbacks (CPU, no GPU): an allocator that raises,
as torch's caching allocator does when the device is full, must reach the
library as NULL (which it reports as PP_ERR_NOMEM), never as an unset return
value; a free that raises must not escape into C."""
import ctypes

from paper_2606_20441_b300 import pp


def _call_alloc(fn, nbytes=4096):
    cb = pp.ALLOC_FN(pp._guarded_alloc(fn))
    # call through a C function pointer, as the library does
    ptr = ctypes.cast(cb, ctypes.c_void_p).value
    c_fn = pp.ALLOC_FN(ptr)
    return c_fn(nbytes, None), cb


def test_failing_allocator_returns_null():
    def full(n):
        raise MemoryError("device full")
    for _ in range(100):
        got, _cb = _call_alloc(full)
        assert got is None


def test_allocator_result_passes_through():
    seen = []

    def ok(n):
        seen.append(n)
        return 0x7F0000001000
    got, _cb = _call_alloc(ok, 123)
    assert got == 0x7F0000001000 and seen == [123]
    got, _cb = _call_alloc(lambda n: 0)
    assert got is None


def test_failing_free_does_not_escape():
    calls = []

    def bad_free(p):
        calls.append(p)
        raise RuntimeError("invalid device pointer")
    cb = pp.FREE_FN(pp._guarded_free(bad_free))
    c_fn = pp.FREE_FN(ctypes.cast(cb, ctypes.c_void_p).value)
    c_fn(0x1000, None)
    assert calls == [0x1000]
