"""Parity tolerance for floating-point outputs.

Reading of "1e-5 relative, scaled by sqrt(n) * max|x|" (1e-12 for fp64):
output j passes when

    |gpu_j - oracle_j| <= rtol * max(|oracle_j|, sqrt(n_j) * M_j)

where n_j is the number of terms combined into output j (prefix length,
suffix length, bin population, or n for a whole-array reduction) and M_j the
largest magnitude among the partial results along that chain (for sums the
terms themselves; for products and linear recurrences the running partial
results).  Each test states its n_j and M_j.  Integer outputs (indices,
counts, permutations) and pure selections or copies are compared bit-exact
with ``np.array_equal`` instead.
"""
import numpy as np

RTOL = {np.dtype(np.float32): 1e-5, np.dtype(np.float64): 1e-12}


def rtol_for(dtype):
    return RTOL[np.dtype(dtype)]


def rowabs(a):
    a = np.abs(np.asarray(a, dtype=np.float64))
    if a.ndim > 1 and a.size == 0:
        return np.zeros(a.shape[0])
    return a.reshape(a.shape[0], -1).max(axis=1) if a.ndim > 1 else a


def prefix_max(a):
    r = rowabs(a)
    return np.maximum.accumulate(r) if r.size else r


def suffix_max(a):
    r = rowabs(a)
    return np.maximum.accumulate(r[::-1])[::-1] if r.size else r


def shift_prev(a, first):
    """a[j-1] with a[-1] := first (row-wise)."""
    a = np.asarray(a, dtype=np.float64)
    out = np.empty_like(a)
    if a.shape[0]:
        out[1:] = a[:-1]
        out[0] = first
    return out


def assert_tol(name, got, ref, nj, Mj, rtol):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, f"{name}: shape {got.shape} vs {ref.shape}"
    if ref.size == 0:
        return
    nj = np.broadcast_to(np.asarray(nj, dtype=np.float64), (ref.shape[0],))
    Mj = np.broadcast_to(np.asarray(Mj, dtype=np.float64), (ref.shape[0],))
    scale = np.sqrt(np.maximum(nj, 1.0)) * Mj
    if ref.ndim > 1:
        scale = scale.reshape(-1, *([1] * (ref.ndim - 1)))
    tol = rtol * np.maximum(np.abs(ref), scale)
    err = np.abs(got - ref)
    bad = ~(err <= tol)  # NaN counts as bad
    if bad.any():
        idx = np.argwhere(bad)[:5]
        ratio = np.nanmax(np.where(tol > 0, err / np.where(tol > 0, tol, 1), np.inf))
        raise AssertionError(
            f"{name}: {int(bad.sum())} of {ref.size} outside tolerance (worst err/tol {ratio:.3g}); "
            + "; ".join(f"{tuple(i)}: gpu={got[tuple(i)]!r} ref={ref[tuple(i)]!r} tol={tol[tuple(i)]:.3g}" for i in idx))


def max_ratio(got, ref, nj, Mj, rtol):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nj = np.broadcast_to(np.asarray(nj, dtype=np.float64), (ref.shape[0],))
    Mj = np.broadcast_to(np.asarray(Mj, dtype=np.float64), (ref.shape[0],))
    scale = np.sqrt(np.maximum(nj, 1.0)) * Mj
    if ref.ndim > 1:
        scale = scale.reshape(-1, *([1] * (ref.ndim - 1)))
    tol = rtol * np.maximum(np.abs(ref), scale)
    return float(np.max(np.abs(got - ref) / np.where(tol > 0, tol, np.inf))) if ref.size else 0.0
