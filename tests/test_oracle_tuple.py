"""Pins for the oracle's tuple scans (Sec. 5.3.3, block-diagonal Jacobians) -- CPU only.

The tuple operator is written out here once more, as plain numpy on a whole
row, so that the oracle's block-by-block evaluation is checked against the
unblocked definitions: the forward against per-block textbook formulas, the
vjp against the general rule of Fig. 7 run with the dense D x D step
Jacobians of that row operator (finite differences), whose off-block entries
must vanish.
"""
import numpy as np
import pytest

import oracle
from tests._pins import assert_close, fd_vjp

RNG = np.random.default_rng(4242)


def row_combine(ops, a, b):
    """(a . b) for one row of the tuple operator, each block by its Fig. 8 definition."""
    out = np.empty_like(a)
    for op, o, w in oracle.tuple_blocks(ops):
        x, y = a[o:o + w], b[o:o + w]
        if op == "add":
            r = x + y
        elif op == "mul":
            r = x * y
        elif op == "min":
            r = np.minimum(x, y)
        elif op == "max":
            r = np.maximum(x, y)
        elif op == "lin":  # x -> b + c x, applied left then right
            r = np.array([y[0] + y[1] * x[0], y[1] * x[1]])
        elif op == "sop":
            r = np.array([x[0] + y[0] + x[1] * y[1], x[1] + y[1]])
        else:
            q = int(round(np.sqrt(w)))
            r = (x.reshape(q, q) @ y.reshape(q, q)).reshape(-1)
        out[o:o + w] = r
    return out


def values(ops, n):
    cols = []
    for op in ops:
        w = oracle.ARITY[op]
        if op in ("min", "max"):
            cols.append(RNG.permutation(n)[:, None] / n + 0.1)  # distinct: differentiable
        elif op == "lin":
            cols.append(np.stack([RNG.standard_normal(n), RNG.uniform(0.9, 1.1, n)], 1))
        elif op in ("mm2", "mm3"):
            cols.append(RNG.uniform(-1, 1, (n, w)) / np.sqrt(w))
        else:
            cols.append(RNG.uniform(0.6, 1.3, (n, w)))
    return np.concatenate(cols, 1)


MIXES = [("add", "mul", "lin", "sop", "mm2", "min"), ("sop", "sop", "sop"), ("mm3", "max", "lin"), ("lin",)]


@pytest.mark.parametrize("ops", MIXES)
def test_tuple_scan_is_the_row_operator_scan(ops):
    # Sec. 5.1's loop with the row operator written out above
    n = 40
    x = values(ops, n)
    ref = np.empty_like(x)
    ref[0] = x[0]
    for i in range(1, n):
        ref[i] = row_combine(ops, ref[i - 1], x[i])
    assert_close(oracle.tscan_fwd(ops, x), ref, rtol=1e-12, atol=1e-12)


def test_tuple_scan_blocks_by_textbook_formulas():
    ops = ("add", "mul", "sop", "min")
    n = 100
    x = values(ops, n)
    y = oracle.tscan_fwd(ops, x)
    assert_close(y[:, 0], np.cumsum(x[:, 0]), rtol=1e-12, atol=1e-12)
    assert_close(y[:, 1], np.cumprod(x[:, 1]), rtol=1e-12, atol=0)
    S = np.cumsum(x[:, 3])
    assert_close(y[:, 3], S, rtol=1e-12, atol=1e-12)
    assert_close(y[:, 2], np.cumsum(x[:, 2]) + (S * S - np.cumsum(x[:, 3] ** 2)) / 2, rtol=1e-12, atol=1e-12)
    assert np.array_equal(y[:, 4], np.minimum.accumulate(x[:, 4]))


def step_jacobians(ops, a, b, h=1e-6):
    """d(a . b)/da and d(a . b)/db, dense D x D, by central differences."""
    D = a.size
    Ja, Jb = np.zeros((D, D)), np.zeros((D, D))
    for j in range(D):
        e = np.zeros(D)
        e[j] = h
        Ja[:, j] = (row_combine(ops, a + e, b) - row_combine(ops, a - e, b)) / (2 * h)
        Jb[:, j] = (row_combine(ops, a, b + e) - row_combine(ops, a, b - e)) / (2 * h)
    return Ja, Jb


@pytest.mark.parametrize("ops", MIXES)
def test_tuple_scan_vjp_is_the_dense_general_rule(ops):
    # Fig. 7 without any sparsity: lambda_{n-1} = ybar_{n-1},
    # lambda_i = ybar_i + J_{i+1}^T lambda_{i+1} with J_{i+1} = d(y_i . x_{i+1})/dy_i,
    # xbar_i = K_i^T lambda_i with K_i = d(y_{i-1} . x_i)/dx_i, xbar_0 = lambda_0.
    n = 25
    x = values(ops, n)
    yb = RNG.standard_normal(x.shape)
    y = oracle.tscan_fwd(ops, x)
    blocks = oracle.tuple_blocks(ops)
    lam = np.zeros_like(x)
    lam[n - 1] = yb[n - 1]
    xbar = np.zeros_like(x)
    for i in range(n - 1, 0, -1):
        Ja, Jb = step_jacobians(ops, y[i - 1], x[i])
        # block-diagonal sparsity (Sec. 5.3.3): nothing couples two blocks
        for _, o, w in blocks:
            mask = np.ones(Ja.shape, bool)
            mask[o:o + w, o:o + w] = False
            assert np.all(Ja[:, o:o + w][mask[:, o:o + w]] == 0) and np.all(Jb[:, o:o + w][mask[:, o:o + w]] == 0)
        xbar[i] = Jb.T @ lam[i]
        lam[i - 1] = yb[i - 1] + Ja.T @ lam[i]
    xbar[0] = lam[0]
    assert_close(oracle.tscan_vjp(ops, x, yb), xbar, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("ops", MIXES)
def test_tuple_scan_vjp_finite_differences_and_dot_product(ops):
    n = 12
    x = values(ops, n)
    yb = RNG.standard_normal(x.shape)
    assert_close(oracle.tscan_vjp(ops, x, yb), fd_vjp(lambda z: oracle.tscan_fwd(ops, z), x, yb),
                 rtol=1e-6, atol=1e-7)
    v = RNG.standard_normal(x.shape)
    assert_close(np.sum(oracle.tscan_jvp(ops, x, v) * yb), np.sum(v * oracle.tscan_vjp(ops, x, yb)),
                 rtol=1e-10, atol=1e-10)


def test_tuple_blocks_layout():
    assert oracle.tuple_blocks(("lin", "add", "mm3", "sop")) == [("lin", 0, 2), ("add", 2, 1), ("mm3", 3, 9),
                                                                 ("sop", 12, 2)]
