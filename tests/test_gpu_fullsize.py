"""GPU parity at the sizes and launch shapes the benchmarks run, against the
fp64 oracle over the whole input (marked slow).

* the small reduce-by-index workload exactly as drawn (n = 100,000, m = 1000,
  hist0 ~ U(-1,1) with seed 1): the + histogram and its vjp, the + reduce and
  the inclusive + scan of the same values (Sec. 4.2.1, 3.2.1, 5.3.1);
* the general reduce (Sec. 3.1, Fig. 2) at sizes whose tile prefix / suffix
  scans span several scan tiles, so their look-back crosses tiles: 2x2
  matrices at n = 1e7 (both as drawn and near-orthogonal), linFnComp at 1e7,
  3x3 at 2.1e6 and 5x5 at 6e5;
* the specialised reduces (Sec. 3.2) at n = 1e8, where every block of the
  single-pass reduce folds many tiles and the last-block combine folds one
  partial per block;
* linFnComp reduce-by-index (Sec. 4.1, Fig. 4) at n = 1e7, m = 1000, with hist0,
  and with per-bin rows of chunk folds longer than one scan segment;
* the q x q matrix scans (Sec. 5.3.4) at the bench's sizes, 3x3 at n = 1e7 and
  5x5 at n = 4e6 (thousands of bulk-staged tiles, so the look-back runs over
  many steps), forward and vjp with accumulate.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, prefix_max, rowabs, rtol_for, suffix_max
from tests.test_gpu_hist import bin_stats, lin_bin_scales
from tests.test_gpu_reduce import suffix_partials
from tests.test_gpu_scan import check_scan

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()
    adcomb.debug_force_hist_strategy(-1)
    adcomb.debug_set_scan_engine(0)
    yield
    torch.cuda.empty_cache()


def test_small_workload_exactly_as_drawn():
    w = synth.hist_add_small()
    n, m, k, v, h0, hb = w["n"], w["m"], w["keys"], w["vals"], w["hist0"], w["histbar"]
    rtol = rtol_for(np.float32)
    # + reduce_by_index with hist0 (Sec. 4.2.1): bins of ~100 values, |v|, |hist0| <= 1
    h, saved = adcomb.hist_fwd("add", m, dev(k), dev(v), dev(h0))
    pop, _ = bin_stats(k, v, m)
    assert_tol("hist + fwd", host(h), oracle.hist_fwd("add", m, k, v, h0), pop + 1, 1.0, rtol)
    vb, h0b = adcomb.hist_vjp("add", m, dev(k), dev(v), dev(h0), h, saved, dev(hb), want_hist0bar=True)
    vr, h0r = oracle.hist_vjp("add", m, k, v, hb, h0)
    assert np.array_equal(host(vb), vr.astype(np.float32))   # a gather: bit-exact
    assert np.array_equal(host(h0b), h0r.astype(np.float32))
    # + reduce of the same values (Sec. 3.2.1): the adjoint is a broadcast
    y, sv = adcomb.reduce_fwd("add", dev(v))
    assert_tol("reduce + fwd", host(y)[:1], [oracle.reduce_fwd("add", v)], n, 1.0, rtol)
    xb = adcomb.reduce_vjp("add", dev(v), y, sv, dev(w["ybar_reduce"]))
    assert np.array_equal(host(xb), np.full(n, w["ybar_reduce"][0], np.float32))
    # inclusive + scan (Sec. 5.3.1): the adjoint is the suffix sum of ybar
    ys = adcomb.scan_fwd("add", dev(v))
    assert_tol("scan + fwd", host(ys), oracle.scan_fwd("add", v), np.arange(1, n + 1), 1.0, rtol)
    xs = adcomb.scan_vjp("add", dev(v), ys, dev(w["ybar_scan"]))
    assert_tol("scan + vjp", host(xs), oracle.scan_vjp("add", v, w["ybar_scan"]), n - np.arange(n),
               suffix_max(w["ybar_scan"]), rtol)


@pytest.mark.parametrize("op,variant,n", [("mm2", "mm2", 10_000_000), ("mm2", "mm2_orth", 10_000_000),
                                          ("lin", "lin", 10_000_000), ("mm3", "mm3_orth", 2_100_001),
                                          ("mm5", "mm5_orth", 600_001)])
def test_reduce_general_full(op, variant, n):
    """Forward, vjp and accumulate against the oracle's sequential chain rule;
    the tolerance bounds each adjoint by the largest prefix and suffix fold."""
    g = np.random.default_rng(140)
    rtol = rtol_for(np.float32)
    d = oracle.ARITY[op]
    x = synth.scan_values(g, variant, n).reshape(n, d)
    xd = dev(x)
    y, saved = adcomb.reduce_fwd(op, xd)
    lmax = rowabs(oracle.scan_fwd(op, x)).max(initial=1.0)
    assert_tol(f"reduce {op} fwd", host(y)[None, :], oracle.reduce_fwd(op, x)[None, :], n, lmax, rtol)
    yb = synth.normal(g, d)
    ref = oracle.reduce_vjp(op, x, yb)
    M = max(d, 4) * lmax * suffix_partials(op, x) * np.abs(yb).max()
    xb = adcomb.reduce_vjp(op, xd, y, saved, dev(yb))
    got = host(xb)
    assert np.isfinite(got).all()
    assert_tol(f"reduce {op} vjp", got, ref, n, M, rtol)
    old = synth.normal(g, (n, d))
    xb = adcomb.reduce_vjp(op, xd, y, saved, dev(yb), xbar=dev(old), accumulate=True)
    assert_tol(f"reduce {op} vjp acc", host(xb), ref + old, n, M + rowabs(old), rtol)


@pytest.mark.parametrize("case", ["add", "mul0", "mul1", "min", "max"])
def test_reduce_specialised_1e8(case):
    n = 100_000_000
    g = np.random.default_rng(150)
    rtol = rtol_for(np.float32)
    op = case[:3]
    if op == "add":
        x = synth.uniform(g, n, -1, 1)
        y, saved = adcomb.reduce_fwd("add", dev(x))
        assert_tol("reduce + fwd", host(y)[:1], [oracle.reduce_fwd("add", x)], n, 1.0, rtol)
        yb = synth.normal(g, 1)
        xb = adcomb.reduce_vjp("add", dev(x), y, saved, dev(yb))
        assert torch.equal(xb, torch.full_like(xb, float(yb[0])))
        return
    if op in ("min", "max"):
        x = synth.hist_spec_values(g, op, n, 1)  # 1024 levels: ~1e5 ties of the extremum
        y, saved = adcomb.reduce_fwd(op, dev(x))
        yr, kr = oracle.reduce_fwd(op, x)
        assert int(host(saved.view(torch.int32))[0]) == kr and host(y)[0] == yr
        yb = synth.normal(g, 1)
        xb = adcomb.reduce_vjp(op, dev(x), y, saved, dev(yb))
        expect = np.zeros(n, np.float32)
        expect[kr] = yb[0]
        assert torch.equal(xb, dev(expect))
        return
    # *: ln x ~ U(-d, d) with d = 10 / sqrt(n), so every partial product stays
    # within e^{+-10}; case mul1 plants one exact zero (the zero-count path)
    delta = 10.0 / np.sqrt(n)
    x = np.exp(g.uniform(-delta, delta, n)).astype(np.float32)
    zeros = int(case[3])
    if zeros:
        x[g.integers(0, n)] = 0
    y, saved = adcomb.reduce_fwd("mul", dev(x))
    nz_r, p_r = oracle.reduce_mul_lifted(x)
    xs = x[x != 0].astype(np.float64)
    pmax = max(1.0, float(np.exp(np.max(np.cumsum(np.log(xs))))))
    sv = host(saved)
    assert int(sv[:4].view(np.int32)[0]) == nz_r == zeros
    assert_tol("reduce * y>0", sv[8:12].view(np.float32), [p_r], n, pmax, rtol)
    assert_tol("reduce * y", host(y)[:1], [oracle.reduce_fwd("mul", x)], n, pmax, rtol)
    yb = synth.normal(g, 1)
    xb = adcomb.reduce_vjp("mul", dev(x), y, saved, dev(yb))
    ref = oracle.reduce_vjp("mul", x, yb)
    Mi = np.abs(yb[0]) * pmax / np.where(x != 0, np.minimum(np.abs(x.astype(np.float64)), 1.0), 1.0)
    assert_tol("reduce * vjp", host(xb), ref, n, Mi, rtol)


def test_hist_lin_full():
    """linFnComp reduce_by_index at n = 1e7, m = 1000 (about 1e4 values per bin,
    folded in index order after hist0) and its vjp w.r.t. values and hist0."""
    w = synth.hist_lin()
    n, m, k, v, hb = w["n"], w["m"], w["keys"], w["vals"], w["histbar"]
    g = np.random.default_rng(160)
    h0 = synth.scan_values(g, "lin", m)
    rtol = rtol_for(np.float32)
    h, saved = adcomb.hist_fwd("lin", m, dev(k), dev(v), dev(h0))
    ref = oracle.hist_fwd("lin", m, k, v, h0)
    pop, _ = bin_stats(k, v[:, 0], m)
    A, R = lin_bin_scales(k, v, m, h0)
    assert_tol("hist lin fwd", host(h), ref, pop + 1, A, rtol)
    vb, h0b = adcomb.hist_vjp("lin", m, dev(k), dev(v), dev(h0), h, saved, dev(hb), want_hist0bar=True)
    vr, h0r = oracle.hist_vjp("lin", m, k, v, hb, h0)
    assert_tol("hist lin vjp", host(vb), vr, pop[k] + 1, 3 * A[k] * R[k] * rowabs(hb)[k], rtol)
    assert_tol("hist lin hist0bar", host(h0b), h0r, pop + 1, 3 * A * R * rowabs(hb), rtol)


@pytest.mark.parametrize("dt,n", [(np.float32, 17_000_001), (np.float64, 5_000_003)])
def test_hist_lin_multi_segment_rows(dt, n):
    """linFnComp reduce_by_index with more chunk folds per bin than one
    shared-memory segment of the per-bin row scan holds (fp32: 4151 chunks of
    4096 elements against 4096 per segment; fp64: 2442 chunks of 2048 against
    2048), so the row scans carry across segments; m = 97, hist0."""
    g = np.random.default_rng(161)
    m = 97
    rtol = rtol_for(dt)
    k = g.integers(0, m, n).astype(np.int32)
    v = synth.scan_values(g, "lin", n, dt)
    h0 = synth.scan_values(g, "lin", m, dt)
    hb = synth.normal(g, (m, 2), dt)
    h, saved = adcomb.hist_fwd("lin", m, dev(k), dev(v), dev(h0))
    ref = oracle.hist_fwd("lin", m, k, v, h0)
    pop, _ = bin_stats(k, v[:, 0], m)
    A, R = lin_bin_scales(k, v, m, h0)
    assert_tol("hist lin fwd", host(h), ref, pop + 1, A, rtol)
    vb, h0b = adcomb.hist_vjp("lin", m, dev(k), dev(v), dev(h0), h, saved, dev(hb), want_hist0bar=True)
    vr, h0r = oracle.hist_vjp("lin", m, k, v, hb, h0)
    assert_tol("hist lin vjp", host(vb), vr, pop[k] + 1, 3 * A[k] * R[k] * rowabs(hb)[k], rtol)
    assert_tol("hist lin hist0bar", host(h0b), h0r, pop + 1, 3 * A * R * rowabs(hb), rtol)


@pytest.mark.parametrize("op,n", [("mm3", 10_000_000), ("mm5", 4_000_000)])
def test_mmq_scan_full(op, n):
    """Forward and vjp (with accumulate) against the oracle over the whole input,
    in the launch configuration the bench times (the automatic choice)."""
    g = np.random.default_rng(150 + len(op))
    x = synth.scan_values(g, op + "_orth", n)
    check_scan(op, x, synth.normal(g, x.shape, np.float32), np.float32, accumulate=True)
