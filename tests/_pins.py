"""Helpers for pinning the oracle: central finite differences and dot-product tests.

None of these helpers restate the oracle's arithmetic: finite differences only
call an oracle forward function at perturbed points.
"""
import numpy as np


def fd_vjp(f, x, ybar, h=1e-6):
    """Central finite-difference estimate of (df/dx)^T ybar for f: R^N -> R^M (fp64)."""
    x = np.asarray(x, dtype=np.float64)
    ybar = np.asarray(ybar, dtype=np.float64).reshape(-1)
    flat = x.reshape(-1)
    out = np.zeros_like(flat)
    for i in range(flat.size):
        xp = flat.copy()
        xm = flat.copy()
        xp[i] += h
        xm[i] -= h
        fp = np.asarray(f(xp.reshape(x.shape)), dtype=np.float64).reshape(-1)
        fm = np.asarray(f(xm.reshape(x.shape)), dtype=np.float64).reshape(-1)
        out[i] = np.dot((fp - fm) / (2 * h), ybar)
    return out.reshape(x.shape)


def assert_close(a, b, rtol=1e-6, atol=1e-8):
    np.testing.assert_allclose(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64),
                               rtol=rtol, atol=atol)
