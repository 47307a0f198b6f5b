"""Pins for the oracle's reduce_by_index (Sec. 4) -- CPU only."""
import numpy as np
import pytest

import oracle
from tests._pins import assert_close, fd_vjp

RNG = np.random.default_rng(4242)


def keys_with_out_of_range(n, m):
    k = RNG.integers(-2, m + 2, n)
    return k


def test_add_matches_bincount_and_gather_adjoint():
    n, m = 2000, 37
    k = keys_with_out_of_range(n, m)
    v = RNG.uniform(-1, 1, n)
    h0 = RNG.uniform(-1, 1, m)
    inr = (k >= 0) & (k < m)
    ref = h0 + np.bincount(k[inr], weights=v[inr], minlength=m)
    assert_close(oracle.hist_fwd("add", m, k, v, h0), ref, rtol=1e-12, atol=1e-12)
    hb = RNG.standard_normal(m)
    vb, h0b = oracle.hist_vjp("add", m, k, v, hb, h0)
    # Sec. 4.2.1 (with the bounds reading 0 <= k < m): vb_i = hb[k_i], else 0.
    expect = np.where(inr, hb[np.clip(k, 0, m - 1)], 0.0)
    assert np.array_equal(vb, expect)
    assert np.array_equal(h0b, hb)


@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_brute_force_with_ties_and_hist0(op):
    n, m = 3000, 23
    k = keys_with_out_of_range(n, m)
    v = (RNG.integers(0, 16, n) - 8) / 4.0
    for h0 in (None, (RNG.integers(0, 16, m) - 8) / 4.0):
        h, idx = oracle.hist_fwd(op, m, k, v, h0)
        hb = RNG.standard_normal(m)
        vb, h0b = oracle.hist_vjp(op, m, k, v, hb, h0)
        vb_ref = np.zeros(n)
        for j in range(m):
            members = np.nonzero(k == j)[0]
            best = members[np.argmin(v[members]) if op == "min" else np.argmax(v[members])] if members.size else None
            neutral = np.inf if op == "min" else -np.inf
            bv = v[best] if best is not None else neutral
            h0wins = h0 is not None and (h0[j] <= bv if op == "min" else h0[j] >= bv)
            if h0wins:
                assert h[j] == h0[j] and idx[j] == n
                assert h0b[j] == hb[j]
            elif best is None:
                assert h[j] == neutral and idx[j] == n
                assert h0b[j] == (hb[j] if h0 is not None else h0b[j])
            else:
                assert h[j] == bv and idx[j] == best
                vb_ref[best] = hb[j]
                assert h0b[j] == 0.0
        assert np.array_equal(vb, vb_ref)


def test_mul_per_bin_brute_force_with_zero_counts():
    n, m = 400, 9
    k = keys_with_out_of_range(n, m)
    v = RNG.uniform(0.5, 1.5, n)
    # bin 0: no zero, bin 1: one zero, bin 2: two zeros
    for j, z in ((1, 1), (2, 2)):
        members = np.nonzero(k == j)[0]
        v[members[:z]] = 0.0
    h0 = RNG.uniform(0.5, 2, m)
    hb = RNG.standard_normal(m)
    h = oracle.hist_fwd("mul", m, k, v, h0)
    vb, h0b = oracle.hist_vjp("mul", m, k, v, hb, h0)
    nz, p = oracle.hist_mul_lifted(m, k, v)
    for j in range(m):
        members = np.nonzero(k == j)[0]
        assert_close(h[j], h0[j] * np.prod(v[members]), rtol=1e-12, atol=0)
        assert nz[j] == np.sum(v[members] == 0)
        assert_close(p[j], np.prod(v[members][v[members] != 0]), rtol=1e-12)
        assert_close(h0b[j], np.prod(v[members]) * hb[j], rtol=1e-12, atol=0)
        for t, i in enumerate(members):
            assert_close(vb[i], h0[j] * np.prod(np.delete(v[members], t)) * hb[j], rtol=1e-11, atol=0)
    out = (k < 0) | (k >= m)
    assert np.all(vb[out] == 0)


def test_lin_is_the_per_bin_sequential_fold_and_reduces_to_add():
    n, m = 500, 11
    k = keys_with_out_of_range(n, m)
    bc = np.stack([RNG.standard_normal(n), RNG.uniform(0.9, 1.1, n)], 1)
    h = oracle.hist_fwd("lin", m, k, bc)
    for j in range(m):
        Y, C = 0.0, 1.0
        for i in np.nonzero(k == j)[0]:  # increasing index order within the bin
            Y = bc[i, 1] * Y + bc[i, 0]
            C = bc[i, 1] * C
        assert_close(h[j], [Y, C], rtol=1e-12, atol=1e-12)
    # c == 1: the b component is a +-histogram and its adjoint the gather
    bc1 = bc.copy()
    bc1[:, 1] = 1.0
    hb = np.stack([RNG.standard_normal(m), np.zeros(m)], 1)
    assert_close(oracle.hist_fwd("lin", m, k, bc1)[:, 0], oracle.hist_fwd("add", m, k, bc1[:, 0]),
                 rtol=1e-12, atol=1e-12)
    vb, _ = oracle.hist_vjp("lin", m, k, bc1, hb)
    vb_add, _ = oracle.hist_vjp("add", m, k, bc1[:, 0], hb[:, 0])
    assert_close(vb[:, 0], vb_add, rtol=0, atol=0)


def test_sop_per_bin_closed_form_with_hist0():
    # per bin: hist0 (.) fold of the bin's pairs = (p0 + P + s0 * S, s0 + S) with
    # P = sum p_i + sum_{i<j} s_i s_j and S = sum s_i (sumOfProd, Sec. 3.3 / Sec. 4);
    # small integers keep every value exact.  Out-of-range keys are skipped.
    n, m = 300, 9
    k = keys_with_out_of_range(n, m)
    v = np.stack([RNG.integers(-5, 6, n), RNG.integers(-5, 6, n)], 1).astype(np.float64)
    h0 = np.stack([RNG.integers(-5, 6, m), RNG.integers(-5, 6, m)], 1).astype(np.float64)
    h = oracle.hist_fwd("sop", m, k, v, h0)
    for j in range(m):
        sel = v[k == j]
        P = sel[:, 0].sum() + (sel[:, 1].sum() ** 2 - (sel[:, 1] ** 2).sum()) / 2
        S = sel[:, 1].sum()
        assert h[j, 0] == h0[j, 0] + P + h0[j, 1] * S
        assert h[j, 1] == h0[j, 1] + S


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("min", 1), ("max", 1), ("lin", 2), ("sop", 2)])
def test_hist_vjp_finite_differences(op, d):
    n, m = 30, 5
    k = keys_with_out_of_range(n, m)
    shape = (n,) if d == 1 else (n, d)
    v = RNG.uniform(0.6, 1.4, shape)
    h0 = RNG.uniform(0.6, 1.4, (m,) if d == 1 else (m, d))
    if op in ("min", "max"):
        v = RNG.permutation(n) / n + 0.3
        h0 = RNG.permutation(m) / m + 0.31 + (0 if op == "min" else 0.6)
    hb = RNG.standard_normal((m,) if d == 1 else (m, d))

    def fv(z):
        r = oracle.hist_fwd(op, m, k, z, h0)
        return r[0] if op in ("min", "max") else r

    def fh(z):
        r = oracle.hist_fwd(op, m, k, v, z)
        return r[0] if op in ("min", "max") else r

    vb, h0b = oracle.hist_vjp(op, m, k, v, hb, h0)
    assert_close(vb, fd_vjp(fv, v, hb), rtol=1e-6, atol=1e-8)
    assert_close(h0b, fd_vjp(fh, h0, hb), rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("op,d", [("add", 1), ("mul", 1), ("min", 1), ("max", 1), ("lin", 2), ("sop", 2)])
def test_hist_dot_product(op, d):
    n, m = 200, 13
    k = keys_with_out_of_range(n, m)
    shape = (n,) if d == 1 else (n, d)
    hshape = (m,) if d == 1 else (m, d)
    v = RNG.uniform(0.6, 1.4, shape)
    h0 = RNG.uniform(0.6, 1.4, hshape)
    vd, h0d, u = RNG.standard_normal(shape), RNG.standard_normal(hshape), RNG.standard_normal(hshape)
    jv = oracle.hist_jvp(op, m, k, v, vd, h0, h0d)
    vb, h0b = oracle.hist_vjp(op, m, k, v, u, h0)
    assert_close(np.sum(jv * u), np.sum(vd * vb) + np.sum(h0d * h0b), rtol=1e-10, atol=1e-10)


def test_sort_perm_is_numpy_stable_argsort():
    n, m = 5000, 100
    k = keys_with_out_of_range(n, m)
    kk = np.where((k < 0) | (k >= m), m, k)
    assert np.array_equal(oracle.sort_perm(m, k), np.argsort(kk, kind="stable"))


def test_empty_histogram_inputs():
    h = oracle.hist_fwd("add", 4, np.zeros(0, np.int64), np.zeros(0))
    assert np.array_equal(h, np.zeros(4))
    h, idx = oracle.hist_fwd("max", 3, np.zeros(0, np.int64), np.zeros(0))
    assert np.all(h == -np.inf) and np.all(idx == 0)
