"""Comparison helpers shared by the GPU parity tests."""
import numpy as np


def keys_of(x, z):
    """Rows of (x words, z words) as a structured void array for set operations."""
    k = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    return k.view(np.dtype((np.void, k.dtype.itemsize * k.shape[1]))).ravel()


def compare_terms(got, ref, eps, rel=1e-12, near=1e-12, floor=1e-6):
    """got/ref: (x, z, c).  Term sets must match except strings whose reference
    (or GPU) coefficient lies within `near` relative of eps; coefficients must
    agree within rel * max(|c|, floor * max|c_ref|).

    The floor only matters for coefficients more than 10^6 times smaller than
    the largest one, which arise by cancellation in untruncated runs (eps = 0):
    their rounding error is relative to the contributions that cancelled, not
    to the small remainder.  Returns a dict of counts."""
    gk, rk = keys_of(got[0], got[1]), keys_of(ref[0], ref[1])
    gi = np.argsort(gk, kind="stable")
    ri = np.argsort(rk, kind="stable")
    gk, gc = gk[gi], got[2][gi]
    rk, rc = rk[ri], ref[2][ri]
    common, ig, ir = np.intersect1d(gk, rk, assume_unique=True, return_indices=True)
    only_g = np.setdiff1d(np.arange(len(gk)), ig)
    only_r = np.setdiff1d(np.arange(len(rk)), ir)
    def near_eps(c):
        return eps > 0 and np.all(np.abs(np.abs(c) - eps) <= near * eps)
    bad_g = [i for i in only_g if not near_eps(gc[i])]
    bad_r = [i for i in only_r if not near_eps(rc[i])]
    assert not bad_g, "GPU has %d extra strings, e.g. c=%r" % (len(bad_g), gc[bad_g[:3]])
    assert not bad_r, "GPU misses %d strings, e.g. c=%r" % (len(bad_r), rc[bad_r[:3]])
    scale = np.max(np.abs(rc)) if len(rc) else 1.0
    d = np.abs(gc[ig] - rc[ir])
    tol = rel * np.maximum(np.abs(rc[ir]), floor * scale)
    worst = int(np.argmax(d - tol)) if len(d) else 0
    assert np.all(d <= tol), "coefficient mismatch: got %r ref %r" % (gc[ig][worst], rc[ir][worst])
    return {"common": len(common), "near_eps": len(only_g) + len(only_r),
            "max_rel": float(np.max(d / np.maximum(np.abs(rc[ir]), 1e-300))) if len(d) else 0.0}


def expect_tol(ref_terms, rel=1e-12):
    """Tolerance on <0|O~|0>: rel times the sum of |c| over diagonal strings."""
    x, c = ref_terms[0], ref_terms[2]
    diag = np.all(x == 0, axis=1)
    return rel * max(np.sum(np.abs(c[diag])), 1e-300)
