"""Pins for the oracle's scan (Sec. 5) -- CPU only."""
import functools

import numpy as np
import pytest

import oracle
from tests._pins import assert_close, fd_vjp

RNG = np.random.default_rng(777)


def test_add_scan_is_cumsum_and_adjoint_is_suffix_sum():
    # Sec. 5.3.1: the adjoint of a +-scan is the reversed +-scan of the reversed ybar.
    x = RNG.uniform(-1, 1, 500)
    yb = RNG.standard_normal(500)
    assert_close(oracle.scan_fwd("add", x), np.cumsum(x), rtol=1e-12, atol=1e-12)
    assert_close(oracle.scan_vjp("add", x, yb), np.cumsum(yb[::-1])[::-1], rtol=1e-12, atol=1e-12)
    # all-ones adjoint: n - i exactly
    n = 1000
    xb = oracle.scan_vjp("add", np.zeros(n), np.ones(n))
    assert np.array_equal(xb, n - np.arange(n, dtype=np.float64))


def test_mul_scan_is_cumprod():
    x = RNG.uniform(0.9, 1.1, 400)
    x[[17, 200]] = 0.0
    assert_close(oracle.scan_fwd("mul", x), np.cumprod(x), rtol=1e-12, atol=0)


def test_mul_scan_adjoint_brute_force():
    # xbar_i = sum_{k >= i} ybar_k * prod_{j <= k, j != i} x_j
    n = 30
    for zeros in ([], [5], [5, 9], [0], [n - 1]):
        x = RNG.uniform(0.5, 1.5, n)
        x[zeros] = 0.0
        yb = RNG.standard_normal(n)
        brute = np.zeros(n)
        for i in range(n):
            for k in range(i, n):
                brute[i] += yb[k] * np.prod(np.delete(x[:k + 1], i))
        assert_close(oracle.scan_vjp("mul", x, yb), brute, rtol=1e-11, atol=1e-13)


def lin_scan_textbook(bc):
    out = np.zeros_like(bc)
    Y, C = 0.0, 1.0
    for i, (b, c) in enumerate(bc):
        Y = c * Y + b
        C = c * C
        out[i] = (Y, C)
    return out


def test_lin_scan_is_the_textbook_recurrence():
    bc = np.stack([RNG.standard_normal(300), RNG.uniform(0.95, 1.05, 300)], 1)
    assert_close(oracle.scan_fwd("lin", bc), lin_scan_textbook(bc), rtol=1e-12, atol=1e-12)


def test_lin_with_unit_coefficients_is_a_plus_scan():
    b = RNG.standard_normal(200)
    bc = np.stack([b, np.ones(200)], 1)
    yb = np.stack([RNG.standard_normal(200), np.zeros(200)], 1)
    assert_close(oracle.scan_fwd("lin", bc)[:, 0], np.cumsum(b), rtol=1e-12, atol=1e-12)
    assert_close(oracle.scan_vjp("lin", bc, yb)[:, 0], oracle.scan_vjp("add", b, yb[:, 0]),
                 rtol=1e-12, atol=1e-12)


def test_lin_adjoint_textbook_recurrence():
    # Textbook adjoint of Y_i = c_i Y_{i-1} + b_i, C_i = c_i C_{i-1}:
    #   lam_i = ybar_i + c_{i+1} lam_{i+1}   (both components)
    #   bbar_i = lam_i.Y,  cbar_i = lam_i.Y * Y_{i-1} + lam_i.C * C_{i-1}, (Y_{-1}, C_{-1}) = (0, 1)
    n = 100
    bc = np.stack([RNG.standard_normal(n), RNG.uniform(0.9, 1.1, n)], 1)
    yb = RNG.standard_normal((n, 2))
    Ys = lin_scan_textbook(bc)
    lam = np.zeros((n, 2))
    for i in range(n - 1, -1, -1):
        lam[i] = yb[i] + (bc[i + 1, 1] * lam[i + 1] if i + 1 < n else 0)
    prev = np.vstack([[0.0, 1.0], Ys[:-1]])
    expect = np.stack([lam[:, 0], lam[:, 0] * prev[:, 0] + lam[:, 1] * prev[:, 1]], 1)
    assert_close(oracle.scan_vjp("lin", bc, yb), expect, rtol=1e-11, atol=1e-12)


def test_mm2_scan_is_the_running_matrix_product():
    m = RNG.uniform(-1, 1, (40, 4))
    acc = np.eye(2)
    ref = []
    for a in m:
        acc = acc @ a.reshape(2, 2)
        ref.append(acc.reshape(-1))
    assert_close(oracle.scan_fwd("mm2", m), np.array(ref), rtol=1e-12, atol=1e-15)


def lin_as_mm2(bc):
    # M_i = [[c_i, 0], [b_i, 1]]: P_i = M_0 ... M_i = [[C_i, 0], [Y_i, 1]]
    b, c = bc[:, 0], bc[:, 1]
    z, o = np.zeros_like(b), np.ones_like(b)
    return np.stack([c, z, b, o], 1)


def test_mm2_crosschecks_lin_forward_and_adjoint():
    n = 80
    bc = np.stack([RNG.standard_normal(n), RNG.uniform(0.9, 1.1, n)], 1)
    P = oracle.scan_fwd("mm2", lin_as_mm2(bc))
    L = oracle.scan_fwd("lin", bc)
    assert_close(P[:, 2], L[:, 0], rtol=1e-12, atol=1e-12)
    assert_close(P[:, 0], L[:, 1], rtol=1e-12, atol=1e-12)
    assert np.all(P[:, 1] == 0) and np.all(P[:, 3] == 1)
    # adjoint: lin outputs (Y, C) are P[1][0] and P[0][0]; lin inputs (b, c) are M[1][0] and M[0][0].
    yb = RNG.standard_normal((n, 2))
    Pb = np.zeros((n, 4))
    Pb[:, 2] = yb[:, 0]
    Pb[:, 0] = yb[:, 1]
    Mb = oracle.scan_vjp("mm2", lin_as_mm2(bc), Pb)
    Lb = oracle.scan_vjp("lin", bc, yb)
    assert_close(Mb[:, 2], Lb[:, 0], rtol=1e-11, atol=1e-12)
    assert_close(Mb[:, 0], Lb[:, 1], rtol=1e-11, atol=1e-12)


def test_mm2_diagonal_is_two_mul_scans():
    n = 60
    a, d = RNG.uniform(0.5, 1.5, n), RNG.uniform(0.5, 1.5, n)
    z = np.zeros(n)
    m = np.stack([a, z, z, d], 1)
    yb = RNG.standard_normal((n, 4))
    P = oracle.scan_fwd("mm2", m)
    assert_close(P[:, 0], np.cumprod(a), rtol=1e-12)
    assert_close(P[:, 3], np.cumprod(d), rtol=1e-12)
    Mb = oracle.scan_vjp("mm2", m, yb)
    assert_close(Mb[:, 0], oracle.scan_vjp("mul", a, yb[:, 0]), rtol=1e-11, atol=1e-12)
    assert_close(Mb[:, 3], oracle.scan_vjp("mul", d, yb[:, 3]), rtol=1e-11, atol=1e-12)


def test_mm2_scan_last_equals_reduce():
    m = RNG.uniform(-1, 1, (33, 4))
    assert_close(oracle.scan_fwd("mm2", m)[-1], oracle.reduce_fwd("mm2", m), rtol=0, atol=0)


@pytest.mark.parametrize("q,op", [(3, "mm3"), (5, "mm5")])
def test_mmq_scan_is_the_running_matrix_product(q, op):
    m = RNG.uniform(-1, 1, (30, q * q)) / np.sqrt(q)
    acc = np.eye(q)
    ref = []
    for a in m:
        acc = acc @ a.reshape(q, q)
        ref.append(acc.reshape(-1))
    assert_close(oracle.scan_fwd(op, m), np.array(ref), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("q,op", [(3, "mm3"), (5, "mm5")])
def test_mmq_scan_embeds_mm2_and_its_adjoint(q, op):
    # M -> blockdiag(M, I): the q x q running product is blockdiag(P, I), and the
    # adjoint restricted to the 2x2 block is the 2x2 adjoint.
    n = 25
    m2 = RNG.uniform(-1, 1, (n, 4))
    mq = np.zeros((n, q, q))
    mq[:, :2, :2] = m2.reshape(n, 2, 2)
    for k in range(2, q):
        mq[:, k, k] = 1.0
    P = oracle.scan_fwd(op, mq.reshape(n, -1)).reshape(n, q, q)
    assert_close(P[:, :2, :2].reshape(n, 4), oracle.scan_fwd("mm2", m2), rtol=1e-12, atol=1e-14)
    yb2 = RNG.standard_normal((n, 4))
    ybq = np.zeros((n, q, q))
    ybq[:, :2, :2] = yb2.reshape(n, 2, 2)
    Mb = oracle.scan_vjp(op, mq.reshape(n, -1), ybq.reshape(n, -1)).reshape(n, q, q)
    assert_close(Mb[:, :2, :2].reshape(n, 4), oracle.scan_vjp("mm2", m2, yb2), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_scan_is_the_running_extremum_with_one_hot_adjoints(op):
    # rs_i = min(as_0..as_i) (numpy's accumulate); with ties the earliest
    # index is selected, so the adjoint of rs_i goes to the first position
    # of the running extremum (brute force over every output).
    n = 300
    x = (RNG.integers(0, 20, n) - 10) / 4.0  # few levels: ties everywhere
    acc = np.minimum.accumulate if op == "min" else np.maximum.accumulate
    assert np.array_equal(oracle.scan_fwd(op, x), acc(x))
    yb = RNG.standard_normal(n)
    expect = np.zeros(n)
    for i in range(n):
        seg = x[: i + 1]
        j = int(np.argmin(seg) if op == "min" else np.argmax(seg))  # first occurrence
        expect[j] += yb[i]
    assert_close(oracle.scan_vjp(op, x, yb), expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_selections_can_be_read_off_y(op):
    # The reading the kernels use: x_i wins step i exactly when y_i differs
    # from y_{i-1} (a strict win changes the running extremum, a tie or a
    # loss keeps it), NaNs after position 0 never winning.  The adjoint built
    # from y alone -- lambda_i = ybar_i + [y_{i+1} == y_i] lambda_{i+1},
    # xbar_i = [i == 0 or y_i != y_{i-1}] lambda_i -- must equal the oracle's,
    # which compares x with y; integer ybar makes both sums exact.
    n = 2000
    x = (RNG.integers(0, 20, n) - 10) / 4.0
    x[RNG.random(n) < 0.05] = np.nan
    x[0] = 0.5
    y = oracle.scan_fwd(op, x)
    assert not np.isnan(y).any()
    yb = RNG.integers(-3, 4, n).astype(np.float64)
    lam = np.zeros(n)
    lam[n - 1] = yb[n - 1]
    for i in range(n - 2, -1, -1):
        lam[i] = yb[i] + (lam[i + 1] if y[i + 1] == y[i] else 0.0)
    sel = np.ones(n, bool)
    sel[1:] = y[1:] != y[:-1]
    assert np.array_equal(oracle.scan_vjp(op, x, yb), np.where(sel, lam, 0.0))


def test_sop_scan_closed_form():
    # sumOfProd (Fig. 8): scanning (p_i, s_i) gives S_k = sum_{j<=k} s_j and
    # P_k = sum_{j<=k} p_j + sum_{j<l<=k} s_j s_l = cumsum(p) + (S_k^2 - cumsum(s^2)) / 2.
    n = 300
    x = np.stack([RNG.standard_normal(n), RNG.uniform(-1, 1, n)], 1)
    S = np.cumsum(x[:, 1])
    P = np.cumsum(x[:, 0]) + (S * S - np.cumsum(x[:, 1] ** 2)) / 2
    assert_close(oracle.scan_fwd("sop", x), np.stack([P, S], 1), rtol=1e-12, atol=1e-12)
    # with elements (0, a_i) the last result is (sum_{i<j} a_i a_j, sum_i a_i), by brute force
    a = RNG.uniform(-1, 1, 12)
    brute = sum(a[i] * a[j] for i in range(12) for j in range(i + 1, 12))
    assert_close(oracle.scan_fwd("sop", np.stack([np.zeros(12), a], 1))[-1], [brute, a.sum()],
                 rtol=1e-13, atol=1e-13)


def test_sop_scan_adjoint_closed_form():
    # From the closed form: dP_k/dp_i = [i <= k], dS_k/ds_i = [i <= k],
    # dP_k/ds_i = [i <= k] (S_k - s_i), so
    #   pbar_i = sum_{k>=i} Pbar_k,   sbar_i = sum_{k>=i} (Sbar_k + Pbar_k (S_k - s_i)).
    n = 200
    x = np.stack([RNG.standard_normal(n), RNG.uniform(-1, 1, n)], 1)
    yb = RNG.standard_normal((n, 2))
    S = np.cumsum(x[:, 1])
    suf = lambda v: np.cumsum(v[::-1])[::-1]
    pbar = suf(yb[:, 0])
    sbar = suf(yb[:, 1]) + suf(yb[:, 0] * S) - x[:, 1] * suf(yb[:, 0])
    assert_close(oracle.scan_vjp("sop", x, yb), np.stack([pbar, sbar], 1), rtol=1e-11, atol=1e-11)


def test_sop_scan_jacobians_are_unit_upper_triangular():
    # The step y_i = y_{i-1} (.) x_i has dy_i/dy_{i-1} = [[1, s_i], [0, 1]]: the reverse
    # recurrence is lam_{i-1} = ybar_{i-1} + (lam_i.p, s_i lam_i.p + lam_i.s).
    n = 40
    x = np.stack([RNG.standard_normal(n), RNG.uniform(-1, 1, n)], 1)
    yb = RNG.standard_normal((n, 2))
    _, lam = oracle.scan_vjp_rbar("sop", x, yb)
    ref = np.zeros((n, 2))
    ref[n - 1] = yb[n - 1]
    for i in range(n - 1, 0, -1):
        ref[i - 1] = yb[i - 1] + [ref[i, 0], x[i, 1] * ref[i, 0] + ref[i, 1]]
    assert_close(lam, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("lin", 2), ("mm2", 4), ("mm3", 9), ("mm5", 25),
                                  ("min", 1), ("max", 1), ("sop", 2)])
def test_scan_vjp_finite_differences(op, d):
    n = 20
    shape = (n,) if d == 1 else (n, d)
    x = RNG.uniform(0.6, 1.3, shape)
    if op in ("mm3", "mm5"):
        x = x / np.sqrt(d)  # keep the running products O(1), so differences stay accurate
    if op in ("min", "max"):
        x = RNG.permutation(n) / n + 0.1  # distinct values: a differentiable point
    yb = RNG.standard_normal(shape)
    assert_close(oracle.scan_vjp(op, x, yb), fd_vjp(lambda z: oracle.scan_fwd(op, z), x, yb),
                 rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("lin", 2), ("mm2", 4), ("mm3", 9), ("mm5", 25),
                                  ("min", 1), ("max", 1), ("sop", 2)])
def test_scan_dot_product(op, d):
    n = 64
    shape = (n,) if d == 1 else (n, d)
    x = RNG.uniform(0.6, 1.3, shape)
    v = RNG.standard_normal(shape)
    u = RNG.standard_normal(shape)
    jv = oracle.scan_jvp(op, x, v)
    jtu = oracle.scan_vjp(op, x, u)
    assert_close(np.sum(jv * u), np.sum(v * jtu), rtol=1e-10, atol=1e-10)


def test_scan_empty_and_single():
    assert oracle.scan_fwd("add", []).shape == (0,)
    assert_close(oracle.scan_vjp("mul", [3.0], [2.0]), [2.0])
    assert_close(oracle.scan_vjp("mm2", np.ones((1, 4)), [[1, 2, 3, 4]]), [[1, 2, 3, 4]])


def test_scan_rbar_is_the_adjoint_of_the_scan_result():
    # rbar_i = d<ybar, y>/d y_i through the later outputs: for + it is the
    # suffix sum of ybar, for * the textbook recurrence lam_i = yb_i + x_{i+1} lam_{i+1}.
    n = 50
    x = RNG.uniform(0.8, 1.2, n)
    yb = RNG.standard_normal(n)
    xb, rb = oracle.scan_vjp_rbar("add", x, yb)
    assert_close(rb, np.cumsum(yb[::-1])[::-1], rtol=1e-12, atol=1e-12)
    xb, rb = oracle.scan_vjp_rbar("mul", x, yb)
    lam = np.zeros(n)
    for i in range(n - 1, -1, -1):
        lam[i] = yb[i] + (x[i + 1] * lam[i + 1] if i + 1 < n else 0.0)
    assert_close(rb, lam, rtol=1e-12, atol=1e-12)
    assert_close(xb, oracle.scan_vjp("mul", x, yb), rtol=0, atol=0)
