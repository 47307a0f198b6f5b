"""GPU parity: reduce forward and vjp (Sec. 3, Figs 2-3) against the fp64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, rowabs, rtol_for

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 31, 33, 1023, 1024, 1025, 4095, 4096, 4097, 3 * 4096 + 1, 100_003]


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def ybar_dev(g, d, dt):
    yb = synth.normal(g, d, dt)
    return yb, dev(yb)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_reduce_add(dt):
    g = np.random.default_rng(11)
    for n in SIZES:
        x = synth.uniform(g, n, -1, 1, dt)
        y, saved = adcomb.reduce_fwd("add", dev(x))
        assert_tol("reduce + fwd", host(y)[:1], [oracle.reduce_fwd("add", x)], n, np.abs(x).max() if n else 0,
                   rtol_for(dt))
        yb, ybd = ybar_dev(g, 1, dt)
        xb = adcomb.reduce_vjp("add", dev(x), y, saved, ybd)
        assert np.array_equal(host(xb), np.full(n, yb[0], dt))  # broadcast: bit-exact
        old = synth.normal(g, n, dt)
        xb = adcomb.reduce_vjp("add", dev(x), y, saved, ybd, xbar=dev(old), accumulate=True)
        assert np.array_equal(host(xb), old + yb[0])


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["min", "max"])
def test_reduce_minmax_ties_bit_exact(op, dt):
    g = np.random.default_rng(12)
    for n in SIZES:
        x = ((g.integers(0, 64, n) - 32) / 8.0).astype(dt)  # 64 levels: ties everywhere
        y, saved = adcomb.reduce_fwd(op, dev(x))
        yr, kr = oracle.reduce_fwd(op, x)
        k = int(host(saved.view(torch.int32))[0])
        assert k == kr
        hy = host(y)[0]
        assert (hy == yr) and (np.signbit(hy) == np.signbit(yr) if n else True)
        yb, ybd = ybar_dev(g, 1, dt)
        xb = adcomb.reduce_vjp(op, dev(x), y, saved, ybd)
        assert np.array_equal(host(xb), oracle.reduce_vjp(op, x, yb).astype(dt))
        if n:
            old = synth.normal(g, n, dt)
            xb = adcomb.reduce_vjp(op, dev(x), y, saved, ybd, xbar=dev(old), accumulate=True)
            expect = old.copy()
            expect[kr] = old[kr] + yb[0]
            assert np.array_equal(host(xb), expect)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("zeros", [0, 1, 2])
def test_reduce_mul_zero_counting(dt, zeros):
    g = np.random.default_rng(13 + zeros)
    for n in [z for z in SIZES if z >= zeros]:
        x = synth.uniform(g, n, 0.95, 1.05, dt)
        if zeros and n:
            x[g.choice(n, zeros, replace=False)] = 0
        y, saved = adcomb.reduce_fwd("mul", dev(x))
        rtol = rtol_for(dt)
        nz_r, p_r = oracle.reduce_mul_lifted(x)
        xs = x[x != 0].astype(np.float64)
        pmax = max(1.0, np.abs(np.cumprod(xs)).max()) if xs.size else 1.0
        sv = host(saved)
        assert int(sv[:4].view(np.int32)[0]) == nz_r
        p = sv[8:8 + np.dtype(dt).itemsize].view(dt)[0]
        assert_tol("reduce * y>0", [p], [p_r], n, pmax, rtol)
        assert_tol("reduce * y", host(y)[:1], [oracle.reduce_fwd("mul", x)], n, pmax, rtol)
        yb, ybd = ybar_dev(g, 1, dt)
        xb = adcomb.reduce_vjp("mul", dev(x), y, saved, ybd)
        ref = oracle.reduce_vjp("mul", x, yb)
        Mi = np.abs(yb[0]) * pmax / np.where(x != 0, np.minimum(np.abs(x.astype(np.float64)), 1.0), 1.0)
        assert_tol("reduce * vjp", host(xb), ref, n, Mi, rtol)
        torch.cuda.synchronize()


def suffix_partials(op, x):
    """max |R_i| over the suffix folds, via the oracle on the reversed, transposed sequence."""
    if op in ("mm2", "mm3", "mm5"):
        q = {"mm2": 2, "mm3": 3, "mm5": 5}[op]
        xt = x.reshape(-1, q, q).transpose(0, 2, 1).reshape(-1, q * q)[::-1]
        return rowabs(oracle.scan_fwd(op, xt)).max(initial=1.0)
    # lin as an exact 2x2 embedding M = [[c, 0], [b, 1]] (row-vector convention)
    m = np.stack([x[:, 1], np.zeros(len(x)), x[:, 0], np.ones(len(x))], 1)
    mt = m.reshape(-1, 2, 2).transpose(0, 2, 1).reshape(-1, 4)[::-1]
    return rowabs(oracle.scan_fwd("mm2", mt)).max(initial=1.0)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["lin", "mm2", "mm3", "mm5"])
def test_reduce_general(op, dt):
    g = np.random.default_rng(14)
    rtol = rtol_for(dt)
    d = {"lin": 2, "mm2": 4, "mm3": 9, "mm5": 25}[op]
    for n in SIZES:
        x = synth.scan_values(g, "lin" if op == "lin" else op + "_orth", n, dt).reshape(n, d)
        y, saved = adcomb.reduce_fwd(op, dev(x))
        yr = oracle.reduce_fwd(op, x)
        lmax = rowabs(oracle.scan_fwd(op, x)).max(initial=1.0)
        assert_tol(f"reduce {op} fwd", host(y)[None, :], yr[None, :], n, lmax, rtol)
        yb, ybd = ybar_dev(g, d, dt)
        for acc in (False, True):
            old = synth.normal(g, (n, d), dt)
            xb = adcomb.reduce_vjp(op, dev(x), y, saved, ybd, xbar=dev(old) if acc else None, accumulate=acc)
            ref = oracle.reduce_vjp(op, x, yb) + (old if acc else 0)
            M = max(d, 4) * lmax * suffix_partials(op, x) * np.abs(yb).max() + (rowabs(old) if acc else 0)
            assert_tol(f"reduce {op} vjp acc={acc}", host(xb), ref, n, M, rtol)


@pytest.mark.parametrize("op,x,k", [("min", [1.0, 0.0, -0.0, 2.0], 1), ("max", [-1.0, -0.0, 0.0, -0.0, -2.0], 1)])
def test_reduce_signed_zero_ties(op, x, k):
    # -0.0 == +0.0: the lowest index wins and its stored value is returned
    x = np.array(x, np.float32)
    y, saved = adcomb.reduce_fwd(op, dev(x))
    assert int(host(saved.view(torch.int32))[0]) == k
    assert np.signbit(host(y)[0]) == np.signbit(x[k])


def test_reduce_mm2_equals_last_scan_element():
    g = np.random.default_rng(15)
    x = synth.scan_values(g, "mm2_orth", 70_001, np.float32)
    y, _ = adcomb.reduce_fwd("mm2", dev(x))
    s = adcomb.scan_fwd("mm2", dev(x))
    ref = oracle.reduce_fwd("mm2", x)
    lmax = rowabs(oracle.scan_fwd("mm2", x)).max()
    assert_tol("reduce", host(y)[None], ref[None], 70_001, lmax, 1e-5)
    assert_tol("scan last", host(s)[-1][None], ref[None], 70_001, lmax, 1e-5)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_reduce_sop_invertible_rule(dt):
    """sumOfProd on (p, s) pairs (Sec. 3.3): forward against the oracle's left
    fold; vjp by the invertible-operator rule against the oracle's sequential
    chain rule.  M bounds every partial result of the fold: |p| <= sum|p_i| +
    (sum|s_i|)^2."""
    g = np.random.default_rng(14)
    rtol = rtol_for(dt)
    for n in SIZES:
        x = synth.uniform(g, (n, 2), -1, 1, dt)
        y, _ = adcomb.reduce_fwd("sop", dev(x))
        ref = oracle.reduce_fwd("sop", x)
        a = np.abs(x.astype(np.float64))
        M = a[:, 0].sum() + a[:, 1].sum() ** 2 if n else 0.0
        assert_tol("reduce sop fwd", host(y).reshape(1, 2), ref.reshape(1, 2), n, M, rtol)
        yb, ybd = ybar_dev(g, 2, dt)
        xb = adcomb.reduce_vjp("sop", dev(x), y, None, ybd)
        xr = oracle.reduce_vjp("sop", x, yb)
        if n:
            assert np.array_equal(host(xb)[:, 0], np.full(n, yb[0], dt))  # d/dp_i = 1: a broadcast
        Mv = abs(float(yb[0])) * (a[:, 1].sum() if n else 0.0) + abs(float(yb[1]))
        assert_tol("reduce sop vjp", host(xb).reshape(n, 2), xr.reshape(n, 2), n, Mv, rtol)
        if n:
            old = synth.normal(g, (n, 2), dt)
            xb = adcomb.reduce_vjp("sop", dev(x), y, None, ybd, xbar=dev(old), accumulate=True)
            assert_tol("reduce sop vjp acc", host(xb).reshape(n, 2), xr + old, n, Mv + rowabs(old), rtol)
