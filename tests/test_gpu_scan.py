"""GPU parity: scan forward and vjp (Sec. 5, Fig. 7) against the fp64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, prefix_max, rowabs, rtol_for, shift_prev, suffix_max

pytestmark = pytest.mark.gpu

TILE = {("add", 4): 4096, ("mul", 4): 4096, ("lin", 4): 2048, ("mm2", 4): 1024, ("sop", 4): 2048,
        ("add", 8): 2048, ("mul", 8): 2048, ("lin", 8): 1024, ("mm2", 8): 512, ("sop", 8): 1024}
IDENT = {"add": [0.0], "mul": [1.0], "lin": [0.0, 1.0], "mm2": [1.0, 0.0, 0.0, 1.0], "sop": [0.0, 0.0],
         "mm3": list(np.eye(3).reshape(-1)), "mm5": list(np.eye(5).reshape(-1))}


def sizes(op, dt):
    t = TILE[(op, np.dtype(dt).itemsize)]
    return [0, 1, 2, 31, 32, 33, t - 1, t, t + 1, 3 * t + 1, 100_003]


def make_x(g, op, n, dt):
    if op in ("mm3", "mm5"):
        return synth.scan_values(g, op + "_orth" if n > 64 else op, n, dt)
    if op == "add":
        return synth.uniform(g, n, -1, 1, dt)
    if op == "mul":
        return synth.with_zeros(g, synth.uniform(g, n, 0.9, 1.1, dt), 0.001)
    if op in ("lin", "sop"):
        return synth.scan_values(g, op, n, dt)
    return synth.scan_values(g, "mm2_orth" if n > 64 else "mm2", n, dt)


def check_scan(op, x, ybar, dt, accumulate=False):
    rtol = rtol_for(dt)
    n = x.shape[0]
    xd, ybd = dev(x), dev(ybar)
    y = adcomb.scan_fwd(op, xd)
    yr = oracle.scan_fwd(op, x)
    nj_f = np.arange(1, n + 1)
    assert_tol(f"scan {op} fwd", host(y).reshape(yr.shape), yr, nj_f,
               prefix_max(np.maximum(rowabs(x), rowabs(yr))) if n else 0, rtol)
    old = None
    xbar = None
    if accumulate:
        old = synth.normal(np.random.default_rng(9), x.shape, dt)
        xbar = dev(old)
    xb = adcomb.scan_vjp(op, xd, y, ybd, xbar=xbar, accumulate=accumulate)
    xbr, lam = oracle.scan_vjp_rbar(op, x, ybar)
    if accumulate:
        xbr = xbr + old.astype(np.float64).reshape(xbr.shape)
    if op == "add":
        Mj = suffix_max(ybar)
        nj = n - np.arange(n)
    else:
        # xbar_j = D(y_{j-1}) lambda_j: both factors carry their chain's error
        yprev = shift_prev(yr, IDENT[op] if op != "mul" else 1.0)
        lam_scale = suffix_max(np.maximum(rowabs(lam), rowabs(ybar))) if n else 0
        Mj = np.maximum(1.0, rowabs(yprev)) * lam_scale + rowabs(lam) * np.maximum(1.0, prefix_max(yprev))
        nj = np.full(n, n)
    if accumulate:
        Mj = Mj + rowabs(old)
    assert_tol(f"scan {op} vjp", host(xb).reshape(xbr.shape), xbr, nj, Mj, rtol)


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()
    yield
    adcomb.debug_set_scan_engine(0)
    adcomb.debug_set_scan_range_tiles(0)


@pytest.fixture(params=[1, 2, 3, 4, 5], ids=["per-tile", "ranges", "staged", "tma", "ranges16"])
def engine(request):
    """All scan engines: per-tile look-back, range-partitioned,
    range-partitioned with TMA staging in shared memory (forced even for small
    n, where a range may be a single ragged tile), one tile per block staged
    in shared memory by TMA, and the range engine with 16 bytes per thread per
    tile."""
    adcomb.debug_set_scan_engine(request.param)
    yield request.param
    adcomb.debug_set_scan_engine(0)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "lin", "mm2", "sop"])
def test_scan_sizes(op, dt, engine):
    g = np.random.default_rng(1000 + len(op))
    for n in sizes(op, dt):
        x = make_x(g, op, n, dt)
        ybar = synth.normal(g, x.shape, dt)
        check_scan(op, x, ybar, dt)


@pytest.mark.parametrize("op", ["add", "mul", "lin", "mm2", "sop"])
def test_scan_accumulate(op, engine):
    g = np.random.default_rng(7)
    x = make_x(g, op, 9001, np.float32)
    check_scan(op, x, synth.normal(g, x.shape, np.float32), np.float32, accumulate=True)


@pytest.mark.parametrize("engine_id", [0, 3, 4, 5], ids=["auto", "staged", "tma", "ranges16"])
@pytest.mark.parametrize("range_tiles", [0, 3, 16])
@pytest.mark.parametrize("op", ["add", "lin", "mm2", "sop"])
def test_scan_ranges_engine_many_tiles(op, range_tiles, engine_id):
    """Large enough that the automatic choice is the range-partitioned engine
    (several tiles per range); also with more, smaller ranges than resident
    blocks (3 tiles: a ragged last range)."""
    g = np.random.default_rng(17)
    n = {"add": 12_000_003, "lin": 6_000_001, "mm2": 3_000_001, "sop": 6_000_001}[op]
    x = make_x(g, op, n, np.float32)
    try:
        adcomb.debug_set_scan_engine(engine_id)
        adcomb.debug_set_scan_range_tiles(range_tiles)
        check_scan(op, x, synth.normal(g, x.shape, np.float32), np.float32)
    finally:
        adcomb.debug_set_scan_range_tiles(0)
        adcomb.debug_set_scan_engine(0)


@pytest.mark.parametrize("range_tiles", [0, 8])
@pytest.mark.parametrize("op", ["add", "mul", "lin", "mm2", "min"])
def test_scan_ranges_with_l2_prefetch(op, range_tiles):
    """The range engine with every block's range prefetched into L2 (tuning
    hook): the same results as without."""
    g = np.random.default_rng(18)
    n = {"add": 12_000_003, "mul": 12_000_003, "lin": 6_000_001, "mm2": 3_000_001, "min": 12_000_003}[op]
    x = make_x(g, op, n, np.float32) if op != "min" else ((g.integers(0, 1024, n) - 512) / 64.0).astype(np.float32)
    try:
        adcomb.debug_set_scan_engine(2)
        adcomb.debug_set_scan_range_tiles(range_tiles)
        adcomb.debug_set_scan_prefetch(1)
        if op == "min":
            xd = dev(x)
            y = adcomb.scan_fwd(op, xd)
            assert np.array_equal(host(y), oracle.scan_fwd(op, x).astype(np.float32))
            yb = g.integers(-3, 4, n).astype(np.float32)
            assert np.array_equal(host(adcomb.scan_vjp(op, xd, y, dev(yb))), oracle.scan_vjp(op, x, yb).astype(np.float32))
        else:
            check_scan(op, x, synth.normal(g, x.shape, np.float32), np.float32)
    finally:
        adcomb.debug_set_scan_prefetch(0)
        adcomb.debug_set_scan_range_tiles(0)
        adcomb.debug_set_scan_engine(0)


def test_mul_scan_zero_paths_exact():
    # zeros cut the recurrence exactly: prefixes after a zero are 0 and the
    # adjoint of x_i stops at the next zero
    x = np.array([2.0, 0.5, 0.0, 3.0, 4.0, 0.0, 0.0, 5.0], np.float32)
    yb = np.array([1, 2, 3, 4, 5, 6, 7, 8], np.float32)
    y = adcomb.scan_fwd("mul", dev(x))
    assert np.array_equal(host(y), np.cumprod(x.astype(np.float64)).astype(np.float32))
    xb = adcomb.scan_vjp("mul", dev(x), y, dev(yb))
    np.testing.assert_allclose(host(xb), oracle.scan_vjp("mul", x, yb), rtol=1e-6, atol=0)


def test_plus_scan_all_ones_adjoint_is_exact():
    # Sec. 5.3.1 with ybar = 1: xbar_i = n - i, exact in fp32 for n < 2^24
    n = 1_000_003
    x = np.zeros(n, np.float32)
    xb = adcomb.scan_vjp("add", dev(x), dev(x), dev(np.ones(n, np.float32)))
    assert np.array_equal(host(xb), (n - np.arange(n)).astype(np.float32))


def test_mm2_scan_matches_lin_embedding():
    # M_i = [[c, 0], [b, 1]]: the mm2 scan carries the lin scan in column 0
    g = np.random.default_rng(3)
    bc = synth.scan_values(g, "lin", 50_001, np.float32)
    m = np.stack([bc[:, 1], np.zeros_like(bc[:, 0]), bc[:, 0], np.ones_like(bc[:, 0])], 1).astype(np.float32)
    P = host(adcomb.scan_fwd("mm2", dev(m)))
    L = host(adcomb.scan_fwd("lin", dev(bc)))
    ref = oracle.scan_fwd("lin", bc)
    Mj = prefix_max(ref)
    nj = np.arange(1, bc.shape[0] + 1)
    assert_tol("mm2 col (1,0)", P[:, 2], ref[:, 0], nj, Mj, 1e-5)
    assert_tol("lin Y", L[:, 0], ref[:, 0], nj, Mj, 1e-5)
    assert np.all(P[:, 1] == 0) and np.all(P[:, 3] == 1)


@pytest.mark.slow
@pytest.mark.parametrize("op,dt,n", [("add", np.float32, 100_000_000), ("mul", np.float32, 100_000_000),
                                     ("lin", np.float32, 100_000_000), ("add", np.float64, 10_000_000),
                                     ("mul", np.float64, 10_000_000), ("lin", np.float64, 10_000_000),
                                     ("sop", np.float32, 100_000_000)])
def test_scan_full_size(op, dt, n):
    """The scan workloads at their full sizes (1e8 fp32, 1e7 fp64), every element checked."""
    w = synth.scan_spec(op, n=n, dtype=dt)
    check_scan(op, w["x"], w["ybar"], dt)
    torch.cuda.empty_cache()


@pytest.mark.slow
@pytest.mark.parametrize("op", ["mm2", "mm2_orth"])
def test_mm2_scan_full_size(op):
    w = synth.scan_spec(op, n=10_000_000, dtype=np.float32)
    check_scan("mm2", w["x"], w["ybar"], np.float32)
    torch.cuda.empty_cache()


@pytest.mark.parametrize("engine_id", [0, 1, 2, 6], ids=["auto", "per-tile", "ranges", "bulk-staged"])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["mm3", "mm5"])
def test_mmq_scan(op, dt, engine_id):
    """q x q matrix-product scans (q = 3, 5): forward and the RBDS vjp with
    M_{i+1}^T, at sizes spanning several tiles and ragged tails.  Automatic
    and hook 6: the bulk-staged segment forms (runs of 7 / 5 matrices, tiles
    of 896 / 448 (3x3) and 640 / 320 / 160 (5x5) matrices); hooks 1 and 2:
    the register forms (3x3 forward tiles of 1024 / 512 matrices, segment
    runs of 8 in blocks of 256)."""
    g = np.random.default_rng(31 + len(op))
    try:
        adcomb.debug_set_scan_engine(engine_id)
        for n in [0, 1, 2, 7, 8, 9, 33, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 3 * 1024 + 1, 20_003,
                  100_003]:
            x = make_x(g, op, n, dt)
            check_scan(op, x, synth.normal(g, x.shape, dt), dt)
        x = make_x(g, op, 3001, dt)
        check_scan(op, x, synth.normal(g, x.shape, dt), dt, accumulate=True)
    finally:
        adcomb.debug_set_scan_engine(0)


@pytest.mark.parametrize("engine_id", [1, 2, 3, 4, 5], ids=["per-tile", "ranges", "staged", "tma", "ranges16"])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_scan(op, dt, engine_id):
    """Running min / max (the earlier element wins ties) and its vjp by the
    general arity-1 rule: forward and the selection are bit-exact; the adjoint
    sums ybar over the outputs each element is selected for (a subset of a
    suffix: nj = suffix length, M = largest |ybar| in it)."""
    g = np.random.default_rng(41 + len(op))
    rtol = rtol_for(dt)
    try:
        adcomb.debug_set_scan_engine(engine_id)
        for n in sizes("add", dt) + [1_000_003]:
            x = ((g.integers(0, 64, n) - 32) / 8.0).astype(dt)  # 64 levels: ties everywhere
            yb = synth.normal(g, n, dt)
            xd = dev(x)
            y = adcomb.scan_fwd(op, xd)
            assert np.array_equal(host(y), oracle.scan_fwd(op, x).astype(dt))
            for acc in (False, True):
                old = synth.normal(g, n, dt)
                xb = adcomb.scan_vjp(op, xd, y, dev(yb), xbar=dev(old) if acc else None, accumulate=acc)
                ref = oracle.scan_vjp(op, x, yb) + (old if acc else 0)
                assert_tol(f"scan {op} vjp", host(xb), ref, n - np.arange(n),
                           suffix_max(yb) + (np.abs(old) if acc else 0), rtol)
    finally:
        adcomb.debug_set_scan_engine(0)


@pytest.mark.parametrize("engine_id", [1, 2, 3, 4, 5], ids=["per-tile", "ranges", "staged", "tma", "ranges16"])
@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_scan_nan_and_integer_adjoints(op, engine_id):
    """NaN never wins a comparison, so a NaN x_i (i > 0) is never selected and
    leaves y unchanged.  The kernels read the selections off y (x_i wins step
    i exactly when y_i differs from y_{i-1}); with integer ybar every adjoint
    is an exact sum, so the vjp must equal the oracle's, which compares x with
    y.  A NaN x_0 makes every y_i NaN (y_0 = x_0, and NaN never loses as the
    earlier operand); all of the adjoint then goes to x_0."""
    g = np.random.default_rng(43)
    try:
        adcomb.debug_set_scan_engine(engine_id)
        for n, x0 in [(1000, 1.0), (100_003, 1.0), (1000, np.nan), (100_003, np.nan)]:
            x = ((g.integers(0, 64, n) - 32) / 8.0).astype(np.float32)
            x[g.random(n) < 0.05] = np.nan
            x[0] = x0
            yb = g.integers(-3, 4, n).astype(np.float32)
            xd = dev(x)
            y = adcomb.scan_fwd(op, xd)
            assert np.array_equal(host(y), oracle.scan_fwd(op, x).astype(np.float32), equal_nan=True)
            xb = adcomb.scan_vjp(op, xd, y, dev(yb))
            assert np.array_equal(host(xb), oracle.scan_vjp(op, x, yb).astype(np.float32))
    finally:
        adcomb.debug_set_scan_engine(0)
