"""Pins for the oracle's reduce (Sec. 3) -- CPU only.

Each test checks the oracle against something other than itself: numpy's own
reductions, closed forms the paper states, brute force, finite differences, or
the dot-product identity <J v, u> = <v, J^T u> with the independent tangent
code.
"""
import functools

import numpy as np
import pytest

import oracle
from tests._pins import assert_close, fd_vjp

RNG = np.random.default_rng(12345)


def test_add_forward_and_broadcast_adjoint():
    # Sec. 3.2.1: the adjoint of y = reduce (+) 0 as is replicate n ybar.
    x = RNG.uniform(-1, 1, 1000)
    assert_close(oracle.reduce_fwd("add", x), np.sum(x), rtol=1e-12)
    xb = oracle.reduce_vjp("add", x, [0.37])
    assert np.all(xb == 0.37)


def test_empty_inputs_give_neutral_element():
    assert oracle.reduce_fwd("add", []) == 0.0
    assert oracle.reduce_fwd("mul", []) == 1.0
    y, k = oracle.reduce_fwd("min", [])
    assert y == np.inf and k == 0  # n = 0: sentinel index n
    y, k = oracle.reduce_fwd("max", [])
    assert y == -np.inf and k == 0
    assert_close(oracle.reduce_fwd("lin", np.zeros((0, 2))), [0.0, 1.0])
    assert_close(oracle.reduce_fwd("mm2", np.zeros((0, 4))), [1, 0, 0, 1])


@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_lowest_index_and_one_hot_adjoint(op):
    # Sec. 3.2.2: result and lowest index on ties; adjoint is ybar at k only.
    for trial in range(20):
        n = int(RNG.integers(1, 200))
        x = (RNG.integers(0, 8, n) - 4) / 2.0  # few levels -> many ties
        y, k = oracle.reduce_fwd(op, x)
        ref_k = int(np.argmin(x) if op == "min" else np.argmax(x))  # numpy: first occurrence
        assert k == ref_k and y == x[ref_k]
        xb = oracle.reduce_vjp(op, x, [1.5])
        expect = np.zeros(n)
        expect[ref_k] = 1.5
        assert np.array_equal(xb, expect)


def test_minmax_signed_zero_ties_return_stored_value():
    x = np.array([0.5, -0.0, 0.0, -0.0, 1.0])
    y, k = oracle.reduce_fwd("min", x)
    assert k == 1 and np.signbit(y)
    x = np.array([0.0, -0.0, -1.0])
    y, k = oracle.reduce_fwd("max", x)
    assert k == 0 and not np.signbit(y)


def brute_prod_except(x, i):
    return float(np.prod(np.delete(x, i)))


@pytest.mark.parametrize("nzeros", [0, 1, 2, 3])
def test_mul_adjoint_brute_force_and_zero_cases(nzeros):
    # Fig. 3: ab_i = l_i * r_i * ybar (= prod_{j != i} a_j * ybar), with the
    # three zero-count cases.
    n = 40
    x = RNG.uniform(0.5, 1.5, n) * RNG.choice([-1, 1], n)
    zero_at = RNG.choice(n, nzeros, replace=False)
    x[zero_at] = 0.0
    yb = 0.8
    xb = oracle.reduce_vjp("mul", x, [yb])
    brute = np.array([brute_prod_except(x, i) * yb for i in range(n)])
    assert_close(xb, brute, rtol=1e-12, atol=0)
    nz, p = oracle.reduce_mul_lifted(x)
    assert nz == nzeros
    assert_close(p, np.prod(x[x != 0]), rtol=1e-12)
    if nzeros == 0:
        # first case: (y / a) * ybar
        assert_close(xb, oracle.reduce_fwd("mul", x) / x * yb, rtol=1e-12)
    elif nzeros == 1:
        # second case: only the zero gets y^{>0} * ybar
        expect = np.zeros(n)
        expect[zero_at[0]] = p * yb
        assert_close(xb, expect, rtol=1e-12, atol=0)
    else:
        assert np.all(xb == 0)


def lin_textbook(bc):
    # x -> b + c*x composed left to right: Y_i = c_i Y_{i-1} + b_i, C_i = prod c.
    Y, C = 0.0, 1.0
    for b, c in bc:
        Y = c * Y + b
        C = c * C
    return np.array([Y, C])


def test_lin_forward_is_the_textbook_recurrence():
    bc = np.stack([RNG.standard_normal(300), RNG.uniform(0.9, 1.1, 300)], 1)
    assert_close(oracle.reduce_fwd("lin", bc), lin_textbook(bc), rtol=1e-12)


def test_mm2_forward_is_the_matrix_product():
    m = RNG.uniform(-1, 1, (50, 4))
    ref = functools.reduce(np.matmul, [a.reshape(2, 2) for a in m]).reshape(-1)
    assert_close(oracle.reduce_fwd("mm2", m), ref, rtol=1e-12, atol=1e-15)


def test_mm2_adjoint_matches_general_rule_with_numpy_products():
    # Eq. red-adj specialised to Z = L_i A_i R_i:  Abar_i = L_i^T Zbar R_i^T.
    n = 12
    m = RNG.uniform(-1, 1, (n, 4))
    mats = [a.reshape(2, 2) for a in m]
    zb = RNG.standard_normal(4)
    xb = oracle.reduce_vjp("mm2", m, zb)
    Zb = zb.reshape(2, 2)
    for i in range(n):
        L = functools.reduce(np.matmul, mats[:i], np.eye(2))
        R = functools.reduce(np.matmul, mats[i + 1:], np.eye(2))
        assert_close(xb[i].reshape(2, 2), L.T @ Zb @ R.T, rtol=1e-10, atol=1e-13)


def test_sop_forward_closed_form():
    # Sec. 3.3's sumOfProd on (p, s) pairs: the fold of (p_i, s_i) is
    # (sum p_i + sum_{i<j} s_i s_j, sum s_i); sum_{i<j} s_i s_j = ((sum s)^2 - sum s^2) / 2.
    # Small integers: every intermediate is exact in fp64.
    n = 57
    x = np.stack([RNG.integers(-9, 10, n), RNG.integers(-9, 10, n)], 1).astype(np.float64)
    p, s = x[:, 0], x[:, 1]
    y = oracle.reduce_fwd("sop", x)
    assert y[0] == p.sum() + (s.sum() ** 2 - (s ** 2).sum()) / 2
    assert y[1] == s.sum()
    # the paper's use: map (0, a_i), reduce, keep p  ->  sum over pairs i < j of a_i a_j
    a = np.array([1.0, 2.0, 3.0])
    assert oracle.reduce_fwd("sop", np.stack([np.zeros(3), a], 1))[0] == 1 * 2 + 1 * 3 + 2 * 3


def test_sop_adjoint_is_the_all_but_one_sum():
    # d/ds_i sum_{j<k} s_j s_k = sum_{j != i} s_j, and d/dp_i of the p-total is 1:
    # xbar_i = (ybar_p, ybar_p * (S - s_i) + ybar_s), S = sum s.
    n = 40
    x = RNG.uniform(-1, 1, (n, 2))
    yb = RNG.standard_normal(2)
    xb = oracle.reduce_vjp("sop", x, yb)
    S = x[:, 1].sum()
    assert_close(xb[:, 0], np.full(n, yb[0]), rtol=0, atol=1e-15)
    assert_close(xb[:, 1], yb[0] * (S - x[:, 1]) + yb[1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("q,op", [(3, "mm3"), (5, "mm5")])
def test_mmq_reduce_and_adjoint_match_numpy_products(q, op):
    # Eq. red-adj for Z = L_i A_i R_i:  Abar_i = L_i^T Zbar R_i^T, with numpy products.
    n = 10
    m = RNG.uniform(-1, 1, (n, q * q)) / np.sqrt(q)
    mats = [a.reshape(q, q) for a in m]
    assert_close(oracle.reduce_fwd(op, m).reshape(q, q), functools.reduce(np.matmul, mats, np.eye(q)),
                 rtol=1e-12, atol=1e-15)
    zb = RNG.standard_normal(q * q)
    xb = oracle.reduce_vjp(op, m, zb)
    Zb = zb.reshape(q, q)
    for i in range(n):
        L = functools.reduce(np.matmul, mats[:i], np.eye(q))
        R = functools.reduce(np.matmul, mats[i + 1:], np.eye(q))
        assert_close(xb[i].reshape(q, q), L.T @ Zb @ R.T, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("min", 1), ("max", 1), ("lin", 2), ("mm2", 4),
                                  ("sop", 2), ("mm3", 9)])
def test_vjp_finite_differences(op, d):
    n = 24
    shape = (n,) if d == 1 else (n, d)
    x = RNG.uniform(0.5, 1.5, shape)
    if op in ("min", "max"):
        x = RNG.permutation(n) / n + 0.1  # distinct values: differentiable point
    yb = RNG.standard_normal(d)

    def f(z):
        r = oracle.reduce_fwd(op, z)
        return r[0] if op in ("min", "max") else r

    assert_close(oracle.reduce_vjp(op, x, yb), fd_vjp(f, x, yb), rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("min", 1), ("max", 1), ("lin", 2), ("mm2", 4),
                                  ("sop", 2)])
def test_dot_product_vjp_vs_jvp(op, d):
    n = 64
    shape = (n,) if d == 1 else (n, d)
    x = RNG.uniform(-1.2, 1.2, shape)
    v = RNG.standard_normal(shape)
    u = RNG.standard_normal(d)
    jv = np.atleast_1d(oracle.reduce_jvp(op, x, v))
    jtu = oracle.reduce_vjp(op, x, u)
    assert_close(np.dot(jv, u), np.sum(v * jtu), rtol=1e-10, atol=1e-12)
