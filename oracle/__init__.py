"""Sequential fp64 oracle (ctypes wrapper around ``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  Nothing in the
GPU library imports this package, and this package imports nothing from the
GPU library.

Every function takes numpy arrays, casts them to fp64 (keys to int64) and
returns fp64 numpy arrays.  Operators are named by strings:
``"add" "mul" "min" "max" "lin" "mm2" "mm3" "mm5" "sop"`` (Fig. 8 of the paper for the tuple
operators).  Tuple elements are arrays of shape ``[n, d]`` (d = 2 for lin as
``(b, c)`` and for sop as ``(p, s)``, d = 4 / 9 / 25 for the row-major 2x2 / 3x3 / 5x5
matrices).

Parity note: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, brute force, finite differences,
dot-product tests against the independent tangent code, textbook reductions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"add": 0, "mul": 1, "min": 2, "max": 3, "lin": 4, "mm2": 5, "sop": 6, "mm3": 7, "mm5": 8}
ARITY = {"add": 1, "mul": 1, "min": 1, "max": 1, "lin": 2, "mm2": 4, "sop": 2, "mm3": 9, "mm5": 25}


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C compiler (plain -O2, no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32 = ctypes.c_int64, ctypes.c_int
            p = ctypes.c_void_p
            sig = {
                "oracle_reduce_fwd": [i32, i64, p, p, p],
                "oracle_reduce_vjp": [i32, i64, p, p, p],
                "oracle_reduce_jvp": [i32, i64, p, p, p],
                "oracle_reduce_mul_lifted": [i64, p, p, p],
                "oracle_scan_fwd": [i32, i64, p, p],
                "oracle_scan_vjp": [i32, i64, p, p, p],
                "oracle_scan_vjp_rbar": [i32, i64, p, p, p, p],
                "oracle_scan_jvp": [i32, i64, p, p, p],
                "oracle_hist_fwd": [i32, i64, i64, p, p, p, p, p],
                "oracle_hist_vjp": [i32, i64, i64, p, p, p, p, p, p],
                "oracle_hist_jvp": [i32, i64, i64, p, p, p, p, p, p],
                "oracle_hist_mul_lifted": [i64, i64, p, p, p, p],
                "oracle_sort_perm": [i64, i64, p, p],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            _lib = lib
    return _lib


def _f64(a, d=1):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if d > 1:
        a = a.reshape(-1, d)
    else:
        a = a.reshape(-1)
    return a


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1))


def _p(a):
    return None if a is None else a.ctypes.data


def _shape(n, d):
    return (n,) if d == 1 else (n, d)


# ---------------------------------------------------------------- reduce ----
def reduce_fwd(op, x):
    """Returns y (scalar or [d]) and, for min/max, the selected index (n if none)."""
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    y = np.zeros(d)
    idx = np.zeros(1, dtype=np.int64)
    _load().oracle_reduce_fwd(OPS[op], n, _p(x), _p(y), _p(idx))
    y = y[0] if d == 1 else y
    if op in ("min", "max"):
        return y, int(idx[0])
    return y


def reduce_vjp(op, x, ybar):
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    yb = _f64(ybar)
    xb = np.zeros(_shape(n, d))
    _load().oracle_reduce_vjp(OPS[op], n, _p(x), _p(yb), _p(xb))
    return xb


def reduce_jvp(op, x, xdot):
    d = ARITY[op]
    x = _f64(x, d)
    xd = _f64(xdot, d)
    yd = np.zeros(d)
    _load().oracle_reduce_jvp(OPS[op], x.shape[0], _p(x), _p(xd), _p(yd))
    return yd[0] if d == 1 else yd


def reduce_mul_lifted(x):
    """Fig. 3's lifted primal: (number of zeros, product of non-zeros)."""
    x = _f64(x)
    nz = np.zeros(1, dtype=np.int64)
    p = np.zeros(1)
    _load().oracle_reduce_mul_lifted(x.shape[0], _p(x), _p(nz), _p(p))
    return int(nz[0]), float(p[0])


# ------------------------------------------------------------------ scan ----
def scan_fwd(op, x):
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    y = np.zeros(_shape(n, d))
    _load().oracle_scan_fwd(OPS[op], n, _p(x), _p(y))
    return y


def scan_vjp(op, x, ybar):
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    yb = _f64(ybar, d)
    xb = np.zeros(_shape(n, d))
    _load().oracle_scan_vjp(OPS[op], n, _p(x), _p(yb), _p(xb))
    return xb


def scan_vjp_rbar(op, x, ybar):
    """Returns (xbar, rbar): rbar[i] is the adjoint of the scan result y[i] (Sec. 5.1's rs-bar)."""
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    yb = _f64(ybar, d)
    xb = np.zeros(_shape(n, d))
    rb = np.zeros(_shape(n, d))
    _load().oracle_scan_vjp_rbar(OPS[op], n, _p(x), _p(yb), _p(xb), _p(rb))
    return xb, rb


def scan_jvp(op, x, xdot):
    d = ARITY[op]
    x = _f64(x, d)
    n = x.shape[0]
    xd = _f64(xdot, d)
    yd = np.zeros(_shape(n, d))
    _load().oracle_scan_jvp(OPS[op], n, _p(x), _p(xd), _p(yd))
    return yd


# -------------------------------------------------------- reduce_by_index ----
def hist_fwd(op, m, keys, vals, hist0=None):
    """Returns hist [m](,d) and, for min/max, the selected index per bin (n if none)."""
    d = ARITY[op]
    k = _i64(keys)
    v = _f64(vals, d)
    n = k.shape[0]
    assert v.shape[0] == n
    if op in ("min", "max"):
        assert not np.isnan(v).any(), "NaN inputs are undefined for min/max"
    h0 = None if hist0 is None else _f64(hist0, d)
    h = np.zeros(_shape(m, d))
    idx = np.zeros(max(m, 1), dtype=np.int64)
    _load().oracle_hist_fwd(OPS[op], n, m, _p(k), _p(v), _p(h0), _p(h), _p(idx))
    if op in ("min", "max"):
        return h, idx[:m]
    return h


def hist_vjp(op, m, keys, vals, histbar, hist0=None):
    """Returns (valsbar, hist0bar)."""
    d = ARITY[op]
    k = _i64(keys)
    v = _f64(vals, d)
    n = k.shape[0]
    h0 = None if hist0 is None else _f64(hist0, d)
    hb = _f64(histbar, d)
    vb = np.zeros(_shape(n, d))
    h0b = np.zeros(_shape(m, d))
    _load().oracle_hist_vjp(OPS[op], n, m, _p(k), _p(v), _p(h0), _p(hb), _p(vb), _p(h0b))
    return vb, h0b


def hist_jvp(op, m, keys, vals, valsdot, hist0=None, hist0dot=None):
    d = ARITY[op]
    k = _i64(keys)
    v = _f64(vals, d)
    n = k.shape[0]
    h0 = None if hist0 is None else _f64(hist0, d)
    vd = _f64(valsdot, d)
    h0d = None if hist0dot is None else _f64(hist0dot, d)
    hd = np.zeros(_shape(m, d))
    _load().oracle_hist_jvp(OPS[op], n, m, _p(k), _p(v), _p(h0), _p(vd), _p(h0d), _p(hd))
    return hd


def hist_mul_lifted(m, keys, vals):
    """Per-bin (zero count int64[m], product of non-zeros fp64[m])."""
    k = _i64(keys)
    v = _f64(vals)
    nz = np.zeros(max(m, 1), dtype=np.int64)
    p = np.zeros(max(m, 1))
    _load().oracle_hist_mul_lifted(k.shape[0], m, _p(k), _p(v), _p(nz), _p(p))
    return nz[:m], p[:m]


def sort_perm(m, keys):
    """Stable permutation sorting [0..n-1] by key; out-of-range keys last."""
    k = _i64(keys)
    perm = np.zeros(max(k.shape[0], 1), dtype=np.int64)
    _load().oracle_sort_perm(k.shape[0], m, _p(k), _p(perm))
    return perm[: k.shape[0]]


# ---------------------------------------------------- vectorised operators --
# reduce / scan / reduce_by_index with map2 (op) over rows of d elements: by
# definition each output column is the scalar combinator of the same input
# column (map2 never mixes columns), so the sequential definition is the scalar
# oracle applied column by column.

def vreduce_fwd(op, x):
    x = np.asarray(x, dtype=np.float64)
    return np.array([np.atleast_1d(reduce_fwd(op, x[:, c]))[0] for c in range(x.shape[1])])


def vreduce_vjp(op, x, ybar):
    x = np.asarray(x, dtype=np.float64)
    ybar = np.asarray(ybar, dtype=np.float64)
    return np.stack([reduce_vjp(op, x[:, c], ybar[c:c + 1]) for c in range(x.shape[1])], 1)


def vscan_fwd(op, x):
    x = np.asarray(x, dtype=np.float64)
    return np.stack([scan_fwd(op, x[:, c]) for c in range(x.shape[1])], 1)


def vscan_vjp(op, x, ybar):
    x = np.asarray(x, dtype=np.float64)
    ybar = np.asarray(ybar, dtype=np.float64)
    return np.stack([scan_vjp(op, x[:, c], ybar[:, c]) for c in range(x.shape[1])], 1)


def vhist_fwd(op, m, keys, vals, hist0=None):
    vals = np.asarray(vals, dtype=np.float64)
    cols = [hist_fwd(op, m, keys, vals[:, c], None if hist0 is None else np.asarray(hist0)[:, c])
            for c in range(vals.shape[1])]
    if op in ("min", "max"):
        return np.stack([c[0] for c in cols], 1), np.stack([c[1] for c in cols], 1)
    return np.stack(cols, 1)


def vhist_vjp(op, m, keys, vals, histbar, hist0=None):
    vals = np.asarray(vals, dtype=np.float64)
    histbar = np.asarray(histbar, dtype=np.float64)
    outs = [hist_vjp(op, m, keys, vals[:, c], histbar[:, c], None if hist0 is None else np.asarray(hist0)[:, c])
            for c in range(vals.shape[1])]
    return np.stack([o[0] for o in outs], 1), np.stack([o[1] for o in outs], 1)


# ------------------------------------------------------------- tuple scans --
# Scans whose element is a tuple of k blocks that combine independently:
# block c of a row is an element of operator ops[c] (arity a_c), the row is the
# blocks one after another (width D = sum a_c), and the tuple operator applies
# ops[c] to block c.  The Jacobian of every step is then block-diagonal with k
# blocks of a_c x a_c (Sec. 5.3.3).  By that definition block c of the scan
# (and of its vjp / jvp) is the scan of operator ops[c] over block c's columns.

def tuple_blocks(ops):
    """[(op, first column, arity)] for a list of operator names."""
    out, o = [], 0
    for op in ops:
        out.append((op, o, ARITY[op]))
        o += ARITY[op]
    return out


def _tuple_apply(ops, fn, *arrays):
    arrays = [np.asarray(a, dtype=np.float64) for a in arrays]
    n = arrays[0].shape[0]
    out = np.zeros((n, sum(ARITY[op] for op in ops)))
    for op, o, a in tuple_blocks(ops):
        cols = [arr[:, o:o + a] if a > 1 else arr[:, o] for arr in arrays]
        out[:, o:o + a] = np.asarray(fn(op, *cols)).reshape(n, a)
    return out


def tscan_fwd(ops, x):
    return _tuple_apply(ops, scan_fwd, x)


def tscan_vjp(ops, x, ybar):
    return _tuple_apply(ops, scan_vjp, x, ybar)


def tscan_jvp(ops, x, xdot):
    return _tuple_apply(ops, scan_jvp, x, xdot)
