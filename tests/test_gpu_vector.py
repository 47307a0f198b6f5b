"""GPU parity: vectorised operators (map2 over rows of d; Irwim / Iswim and the
same interchange for reduce_by_index) against the oracle, column by column."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, rtol_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def values(g, op, n, d, dt):
    if op == "mul":
        x = synth.uniform(g, (n, d), 0.97, 1.03, dt)
        x[g.random((n, d)) < 0.002] = 0
        return x
    if op in ("min", "max"):
        return ((g.integers(0, 32, (n, d)) - 16) / 4.0).astype(dt)  # ties
    return synth.uniform(g, (n, d), -1, 1, dt)


def col_tol(name, got, ref, nj, M, rtol):
    """assert_tol column by column: nj per row, M per element (broadcast to the array)."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    M = np.broadcast_to(np.asarray(M, np.float64), ref.shape)
    for c in range(ref.shape[1]):
        assert_tol(f"{name} col {c}", got[:, c], ref[:, c], nj, M[:, c], rtol)


def colscale(x, op):
    """Per-column bound on the partial results: |x| sums (+), running |products| (*)."""
    a = np.abs(x.astype(np.float64))
    if op == "mul":
        b = np.where(a == 0, 1.0, a)
        return np.maximum(1.0, np.exp(np.maximum.accumulate(np.cumsum(np.log(b), 0), 0)[-1])) if len(a) else 1.0
    return a.max(0) if len(a) else 0.0


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("d", [1, 3, 16])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_vreduce(op, d, dt):
    g = np.random.default_rng(51 + d)
    rtol = rtol_for(dt)
    for n in [0, 1, 1000, 100_003]:
        x = values(g, op, n, d, dt)
        y, saved = adcomb.vreduce_fwd(op, dev(x))
        ref = oracle.vreduce_fwd(op, x)
        if op in ("min", "max"):
            assert np.array_equal(host(y), ref.astype(dt))
        else:
            assert_tol("vreduce fwd", host(y), ref, n, colscale(x, op), rtol)
        yb = synth.normal(g, d, dt)
        xb = adcomb.vreduce_vjp(op, dev(x), y, saved, dev(yb))
        xr = oracle.vreduce_vjp(op, x, yb)
        if op in ("add", "min", "max"):
            assert np.array_equal(host(xb), xr.astype(dt))  # broadcast / one-hot: exact
        else:
            M = colscale(x, op) * np.abs(yb) / np.where(x != 0, np.minimum(np.abs(x.astype(np.float64)), 1), 1)
            col_tol("vreduce * vjp", host(xb).reshape(n, d), xr.reshape(n, d), n, M, rtol)


def check_vscan(g, op, n, d, dt):
    rtol = rtol_for(dt)
    x = values(g, op, n, d, dt)
    y = adcomb.vscan_fwd(op, dev(x))
    ref = oracle.vscan_fwd(op, x)
    if op in ("min", "max"):
        assert np.array_equal(host(y), ref.astype(dt))
    else:
        col_tol("vscan fwd", host(y).reshape(n, d), ref.reshape(n, d), np.arange(1, n + 1), colscale(x, op), rtol)
    yb = synth.normal(g, (n, d), dt)
    for acc in (False, True):
        old = synth.normal(g, (n, d), dt)
        xb = adcomb.vscan_vjp(op, dev(x), y, dev(yb), xbar=dev(old) if acc else None, accumulate=acc)
        xr = oracle.vscan_vjp(op, x, yb) + (old if acc else 0)
        M = (np.abs(yb).max(0) if n else 0) * (colscale(x, op) if op == "mul" else 1.0) * 4 + \
            (np.abs(old) if acc else 0)
        col_tol(f"vscan {op} vjp", host(xb).reshape(n, d), xr.reshape(n, d), np.arange(n, 0, -1), M, rtol)


# d = 1 is the scalar scan; in the direct form d = 2, 3, 10, 16, 32 run warp
# units of 16, 10, 3, 2 and 1 parts (10: 2 idle lanes), d = 33 and 64 block
# units of 7 and 4 parts (33: 25 idle threads); n spans one partial tile
# (1000) to many units of one tile or less (100_003)
@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("d", [1, 2, 3, 10, 16, 32, 33, 64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_vscan(op, d, dt):
    g = np.random.default_rng(61 + d)
    for n in [0, 1, 1000, 100_003]:
        check_vscan(g, op, n, d, dt)


@pytest.mark.parametrize("d", [3, 16, 48])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_vscan_many_tiles_per_unit(op, d):
    """Enough rows that every unit of the direct form (warps for d = 3, 16,
    blocks for 48) rescans several tiles, carrying each column's prefix from
    tile to tile."""
    check_vscan(np.random.default_rng(90 + d), op, 2_000_003, d, np.float32)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("d", [3, 16, 48])
@pytest.mark.parametrize("op", ["min", "max"])
def test_vscan_minmax_nan_and_integer_adjoints(op, d, dt):
    """The min / max vjps read the selections off y (x_i wins step i exactly
    when y_i differs from y_{i-1}): with NaNs in x (never selected after row
    0) and integer ybar, every adjoint is an exact sum and equals the
    oracle's, which compares x with y.  Row 0 holds NaN in some columns: a
    NaN x_0 makes its whole column NaN (y_0 = x_0, and NaN never loses as the
    earlier operand) and sends the column's whole adjoint to x_0."""
    g = np.random.default_rng(95 + d)
    n = 100_003
    x = ((g.integers(0, 64, (n, d)) - 32) / 8.0).astype(dt)
    x[g.random((n, d)) < 0.05] = np.nan
    x[0] = 1.0
    x[0, ::2] = np.nan
    yb = g.integers(-3, 4, (n, d)).astype(dt)
    xd = dev(x)
    y = adcomb.vscan_fwd(op, xd)
    assert np.array_equal(host(y), oracle.vscan_fwd(op, x).astype(dt), equal_nan=True)
    xb = adcomb.vscan_vjp(op, xd, y, dev(yb))
    assert np.array_equal(host(xb), oracle.vscan_vjp(op, x, yb).astype(dt))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("d", [1, 4])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_vhist(op, d, dt):
    g = np.random.default_rng(71 + d)
    rtol = rtol_for(dt)
    for n, m in [(0, 5), (1000, 37), (100_003, 5000)]:
        k = g.integers(-2, m + 2, n).astype(np.int32)
        v = values(g, op, n, d, dt)
        h0 = values(g, op, m, d, dt)
        h, saved = adcomb.vhist_fwd(op, m, dev(k), dev(v), dev(h0))
        ref = oracle.vhist_fwd(op, m, k, v, h0)
        if op in ("min", "max"):
            assert np.array_equal(host(h), ref[0].astype(dt))
        else:
            col_tol("vhist fwd", host(h), ref, n + 1, max(colscale(v, op).max() if n else 1.0, 1.0) *
                    (np.abs(h0).max() if op == "mul" else 1.0) + np.abs(h0), rtol)
        hb = synth.normal(g, (m, d), dt)
        vb, h0b = adcomb.vhist_vjp(op, m, dev(k), dev(v), dev(h0), h, saved, dev(hb), want_hist0bar=True)
        vr, h0r = oracle.vhist_vjp(op, m, k, v, hb, h0)
        if op in ("add", "min", "max"):
            assert np.array_equal(host(vb), vr.astype(dt))
            assert np.array_equal(host(h0b), h0r.astype(dt))
        else:
            scale = 4 * np.abs(hb).max() * max(colscale(v, op).max() if n else 1.0, 1.0) * np.abs(h0).max()
            kc = np.clip(k, 0, m - 1)
            M = scale / np.where(v != 0, np.minimum(np.abs(v.astype(np.float64)), 1), 1)
            col_tol("vhist * vjp", host(vb).reshape(n, d), vr.reshape(n, d), n + 1, M, rtol)
            col_tol("vhist * hist0bar", host(h0b), h0r, n + 1, scale, rtol)


def test_transpose_roundtrip_bit_exact():
    g = np.random.default_rng(9)
    for shape in [(1, 1), (33, 65), (1000, 3), (3, 100_001)]:
        a = synth.normal(g, shape, np.float32)
        t = adcomb.transpose(dev(a))
        assert np.array_equal(host(t), a.T)
        assert np.array_equal(host(adcomb.transpose(t)), a)
