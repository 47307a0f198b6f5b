"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 6.1.2).

This module only draws random numbers: it holds none of the method's
arithmetic, so both the CUDA path and the fp64 oracle can be fed from it.
Every array comes from ``numpy.random.default_rng(seed)`` on the host, in the
dtype the device will see, so both sides consume identical bits.

Workloads (the paper measures on "randomly generated arrays", fp32):
  * ``hist_add_small``   n = 100,000 values ~U(-1,1), keys uniform in [0, 1000),
                         hist0 ~U(-1,1), histogram adjoint ~N(0,1); the same
                         values also feed a +-reduce and a +-scan.
  * ``hist_spec``        n = 50M, m in {31, 401, 50,000, 10M}:  ``mul`` values
                         ~U(0.5,1.5) with 1% exact zeros; ``min``/``max``
                         values on 1024 exact levels (v = (k - 512)/64) so that
                         ties are common; ``mul_wc`` the well-conditioned
                         product variant with ln v ~U(-delta, delta),
                         delta = 10/sqrt(n/m).
  * ``scan_spec``        n = 100M fp32 / 10M fp64: ``add`` ~U(-1,1); ``mul``
                         ~U(0.9,1.1) with 0.1% exact zeros; ``lin`` pairs
                         (b, c) with c ~U(0.95,1.05), b ~N(0,1).
  * ``mm2``              n = 10M 2x2 matrices, entries ~U(-1,1)/sqrt(2); the
                         ``mm2_orth`` variant rho*R(theta), rho ~U(0.999,1.001).
  * ``hist_lin``         n = 10M (b, c) pairs as for ``scan_spec`` lin, keys
                         uniform in [0, 1000).
  * ``batched``          4096 instances, n_i log-uniform in [1e3, 1e6], m_i
                         log-uniform in [64, 65536], op + or max 50/50, values
                         ~U(-1,1).
"""
from __future__ import annotations

import numpy as np

HIST_SPEC_BINS = (31, 401, 50_000, 10_000_000)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform(g, n, lo, hi, dtype=np.float32):
    if dtype == np.float32:
        return (g.random(n, dtype=np.float32) * np.float32(hi - lo) + np.float32(lo)).astype(np.float32)
    return g.uniform(lo, hi, n).astype(dtype)


def normal(g, shape, dtype=np.float32):
    if dtype == np.float32:
        return g.standard_normal(shape, dtype=np.float32)
    return g.standard_normal(shape).astype(dtype)


def keys_uniform(g, n, m):
    return g.integers(0, m, n, dtype=np.int32)


def with_zeros(g, v, frac):
    mask = g.random(v.shape[0]) < frac
    v = v.copy()
    v[mask] = 0
    return v


# ------------------------------------------------------------- workloads ----
def hist_add_small(seed=0, n=100_000, m=1000, dtype=np.float32):
    g = rng(seed)
    vals = uniform(g, n, -1.0, 1.0, dtype)
    keys = keys_uniform(g, n, m)
    histbar = normal(g, m, dtype)
    ybar_reduce = normal(g, 1, dtype)
    ybar_scan = normal(g, n, dtype)
    hist0 = uniform(rng(seed + 1), m, -1.0, 1.0, dtype)
    return dict(n=n, m=m, keys=keys, vals=vals, hist0=hist0, histbar=histbar,
                ybar_reduce=ybar_reduce, ybar_scan=ybar_scan)


def hist_spec_values(g, op, n, m, dtype=np.float32):
    if op == "mul":
        return with_zeros(g, uniform(g, n, 0.5, 1.5, dtype), 0.01)
    if op == "mul_wc":
        delta = 10.0 / np.sqrt(max(n / m, 1.0))
        return np.exp(g.uniform(-delta, delta, n)).astype(dtype)
    if op in ("min", "max"):
        return ((g.integers(0, 1024, n) - 512) / 64.0).astype(dtype)
    if op == "add":
        return uniform(g, n, -1.0, 1.0, dtype)
    raise ValueError(op)


def hist_spec(op, m, seed=1, n=50_000_000, dtype=np.float32):
    g = rng(seed)
    keys = keys_uniform(g, n, m)
    vals = hist_spec_values(g, op, n, m, dtype)
    histbar = normal(g, m, dtype)
    return dict(n=n, m=m, keys=keys, vals=vals, histbar=histbar)


def scan_values(g, op, n, dtype=np.float32):
    if op == "add":
        return uniform(g, n, -1.0, 1.0, dtype)
    if op == "mul":
        return with_zeros(g, uniform(g, n, 0.9, 1.1, dtype), 0.001)
    if op == "lin":
        b = normal(g, n, dtype)
        c = uniform(g, n, 0.95, 1.05, dtype)
        return np.ascontiguousarray(np.stack([b, c], axis=1))
    if op == "sop":
        # sumOfProd pairs (p, s): both U(-1, 1)
        return np.ascontiguousarray(uniform(g, 2 * n, -1.0, 1.0, dtype).reshape(n, 2))
    if op == "mm2":
        return (uniform(g, 4 * n, -1.0, 1.0, dtype) / np.asarray(np.sqrt(2.0), dtype)).astype(dtype).reshape(n, 4)
    if op == "mm2_orth":
        rho = g.uniform(0.999, 1.001, n)
        th = g.uniform(0, 2 * np.pi, n)
        c, s = np.cos(th) * rho, np.sin(th) * rho
        return np.ascontiguousarray(np.stack([c, -s, s, c], axis=1).astype(dtype))
    if op in ("mm3", "mm5"):
        q = int(op[2])
        return (uniform(g, q * q * n, -1.0, 1.0, dtype) / np.asarray(np.sqrt(q), dtype)).astype(dtype).reshape(n, q * q)
    if op in ("mm3_orth", "mm5_orth"):
        # near-orthogonal q x q: Q of a Gaussian matrix's QR, times rho ~ U(0.999, 1.001)
        q = int(op[2])
        Q, _ = np.linalg.qr(g.standard_normal((n, q, q)))
        rho = g.uniform(0.999, 1.001, (n, 1, 1))
        return np.ascontiguousarray((Q * rho).reshape(n, q * q).astype(dtype))
    raise ValueError(op)


def scan_spec(op, seed=2, n=100_000_000, dtype=np.float32):
    g = rng(seed)
    x = scan_values(g, op, n, dtype)
    ybar = normal(g, x.shape, dtype)
    return dict(n=n, x=x, ybar=ybar)


def hist_lin(seed=3, n=10_000_000, m=1000, dtype=np.float32):
    g = rng(seed)
    keys = keys_uniform(g, n, m)
    vals = scan_values(g, "lin", n, dtype)
    histbar = normal(g, (m, 2), dtype)
    return dict(n=n, m=m, keys=keys, vals=vals, histbar=histbar)


def batched(seed=4, count=4096, n_lo=1e3, n_hi=1e6, m_lo=64, m_hi=65536):
    g = rng(seed)
    ns = np.round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi), count))).astype(np.int64)
    ms = np.round(np.exp(g.uniform(np.log(m_lo), np.log(m_hi), count))).astype(np.int64)
    ops = np.where(g.random(count) < 0.5, 0, 1).astype(np.int32)  # 0: add, 1: max
    total = int(ns.sum())
    keys = np.empty(total, dtype=np.int32)
    off = 0
    for i in range(count):
        keys[off:off + ns[i]] = g.integers(0, ms[i], ns[i], dtype=np.int32)
        off += int(ns[i])
    vals = uniform(g, total, -1.0, 1.0)
    return dict(count=count, ns=ns, ms=ms, ops=ops, keys=keys, vals=vals)
