"""Pins for the oracle's vectorised operators (map2 over rows) -- CPU only:
numpy's own column-wise reductions, accumulations and scatter-adds."""
import numpy as np
import pytest

import oracle
from tests._pins import assert_close

RNG = np.random.default_rng(4242)


@pytest.mark.parametrize("op,ref,acc", [("add", np.sum, np.cumsum), ("mul", np.prod, np.cumprod),
                                        ("min", np.min, np.minimum.accumulate),
                                        ("max", np.max, np.maximum.accumulate)])
def test_vreduce_and_vscan_are_columnwise_numpy(op, ref, acc):
    x = RNG.uniform(0.5, 1.5, (200, 7))
    assert_close(oracle.vreduce_fwd(op, x), ref(x, axis=0), rtol=1e-12, atol=0)
    assert_close(oracle.vscan_fwd(op, x), acc(x, axis=0), rtol=1e-12, atol=0)


def test_vreduce_add_adjoint_broadcasts_each_column():
    x = RNG.standard_normal((50, 4))
    yb = RNG.standard_normal(4)
    assert_close(oracle.vreduce_vjp("add", x, yb), np.broadcast_to(yb, x.shape), rtol=0, atol=0)


def test_vscan_add_adjoint_is_columnwise_suffix_sum():
    x = RNG.standard_normal((60, 3))
    yb = RNG.standard_normal((60, 3))
    assert_close(oracle.vscan_vjp("add", x, yb), np.cumsum(yb[::-1], axis=0)[::-1], rtol=1e-12, atol=1e-12)


def test_vhist_add_is_columnwise_scatter_add_and_gather():
    n, m, d = 500, 13, 5
    k = RNG.integers(-2, m + 2, n)
    v = RNG.standard_normal((n, d))
    h = oracle.vhist_fwd("add", m, k, v)
    ref = np.zeros((m, d))
    ok = (k >= 0) & (k < m)
    np.add.at(ref, k[ok], v[ok])
    assert_close(h, ref, rtol=1e-12, atol=1e-12)
    hb = RNG.standard_normal((m, d))
    vb, _ = oracle.vhist_vjp("add", m, k, v, hb)
    expect = np.where(ok[:, None], hb[np.clip(k, 0, m - 1)], 0.0)
    assert_close(vb, expect, rtol=0, atol=0)
