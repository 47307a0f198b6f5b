"""GPU parity: tuple scans with block-diagonal Jacobians (Sec. 5.3.3) against
the fp64 oracle, in both layouts (rows [n][D] and one array per block)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, prefix_max, rowabs, rtol_for, shift_prev, suffix_max
from tests.test_gpu_scan import IDENT, make_x

pytestmark = pytest.mark.gpu

# uniform scalar rows (("add", "add"), ("add",) * 64, ("max",) * 5, ("mul",) * 3) and uniform lin /
# sumOfProd / 2x2 rows (("sop",) * 3, ("sop",) * 16, ("lin",) * 5, ("mm2",) * 3, and the widest rows
# the ABI takes, 64 values: ("lin",) * 32, ("mm2",) * 16) take the vectorised scan's direct form; the
# others split into planes
MIXES = [("add", "mul", "lin", "sop", "mm2", "min"), ("sop", "sop", "sop"), ("mm3", "max", "lin"), ("lin",),
         ("add", "add"), ("sop",) * 16, ("add",) * 64, ("mm5", "mm5"), ("mul", "mm3"), ("max",) * 5, ("mul",) * 3,
         ("min",) * 7, ("lin",) * 5, ("mm2",) * 3, ("lin",) * 32, ("mm2",) * 16]
SIZES = [0, 1, 2, 33, 1025, 4097, 100_003]


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def block_values(g, op, n, dt):
    if op in ("min", "max"):
        return ((g.integers(0, 64, n) - 32) / 8.0).astype(dt)  # ties everywhere
    return make_x(g, op, n, dt)


def make_rows(g, ops, n, dt):
    blocks = [block_values(g, op, n, dt).reshape(n, oracle.ARITY[op]) for op in ops]
    return np.ascontiguousarray(np.concatenate(blocks, 1))


def check_block(op, x, yb, y_gpu, xb_gpu, dt, old=None):
    """Block c's results against the oracle, with the scalar scan's tolerance."""
    rtol = rtol_for(dt)
    n = x.shape[0]
    x1 = x[:, 0] if x.shape[1] == 1 else x
    yb1 = yb[:, 0] if yb.shape[1] == 1 else yb
    w = x.shape[1]
    yr = oracle.scan_fwd(op, x1).reshape(n, w)
    if n:
        xbr, lam = oracle.scan_vjp_rbar(op, x1, yb1)
    else:
        xbr, lam = np.zeros((0, w)), np.zeros((0, w))
    xbr = xbr.reshape(n, w)
    lam = lam.reshape(n, w)
    if old is not None:
        xbr = xbr + old
    if op in ("min", "max"):
        assert np.array_equal(y_gpu, yr.astype(dt))
        assert_tol(f"tuple {op} vjp", xb_gpu, xbr, n - np.arange(n),
                   suffix_max(yb) + (rowabs(old) if old is not None else 0), rtol)
        return
    if n:
        assert_tol(f"tuple {op} fwd", y_gpu, yr, np.arange(1, n + 1), prefix_max(np.maximum(rowabs(x), rowabs(yr))),
                   rtol)
    if op == "add":
        Mj, nj = suffix_max(yb), n - np.arange(n)
    else:
        yprev = shift_prev(yr, IDENT[op])
        lam_scale = suffix_max(np.maximum(rowabs(lam), rowabs(yb))) if n else 0
        Mj = np.maximum(1.0, rowabs(yprev)) * lam_scale + rowabs(lam) * np.maximum(1.0, prefix_max(yprev))
        nj = np.full(n, n)
    if old is not None:
        Mj = Mj + rowabs(old)
    assert_tol(f"tuple {op} vjp", xb_gpu, xbr, nj, Mj, rtol)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("ops", MIXES, ids=lambda o: "-".join(o) if len(o) < 8 else f"{o[0]}x{len(o)}")
def test_tuple_scan_rows(ops, dt):
    g = np.random.default_rng(3000 + len(ops))
    blocks = oracle.tuple_blocks(ops)
    for n in SIZES:
        x = make_rows(g, ops, n, dt)
        yb = synth.normal(g, x.shape, dt)
        for acc in (False, True):
            old = synth.normal(g, x.shape, dt) if acc else None
            xd = dev(x)
            y = adcomb.tscan_fwd(ops, xd)
            all_add = all(op == "add" for op in ops)
            xb = adcomb.tscan_vjp(ops, None if all_add else xd, None if all_add else y, dev(yb),
                                  xbar=dev(old) if acc else None, accumulate=acc)
            yh, xbh = host(y), host(xb)
            for op, o, w in blocks:
                check_block(op, x[:, o:o + w], yb[:, o:o + w], yh[:, o:o + w], xbh[:, o:o + w], dt,
                            None if old is None else old[:, o:o + w].astype(np.float64))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("ops", MIXES[:4] + MIXES[4:5], ids=lambda o: "-".join(o))
def test_tuple_scan_blocks(ops, dt):
    g = np.random.default_rng(4000 + len(ops))
    for n in SIZES:
        xs = [block_values(g, op, n, dt).reshape(n, oracle.ARITY[op]) for op in ops]
        ybs = [synth.normal(g, x.shape, dt) for x in xs]
        xds = [dev(np.ascontiguousarray(x if x.shape[1] > 1 else x[:, 0])) for x in xs]
        ybds = [dev(np.ascontiguousarray(yb if yb.shape[1] > 1 else yb[:, 0])) for yb in ybs]
        ys = adcomb.tscan_fwd_blocks(ops, xds)
        # + blocks need neither x nor y: pass NULL entries for them
        xin = [None if op == "add" else t for op, t in zip(ops, xds)]
        yin = [None if op == "add" else t for op, t in zip(ops, ys)]
        for acc in (False, True):
            olds = [synth.normal(g, x.shape, dt) for x in xs] if acc else None
            xbars = [dev(np.ascontiguousarray(o if o.shape[1] > 1 else o[:, 0])) for o in olds] if acc else None
            xbs = adcomb.tscan_vjp_blocks(ops, xin, yin, ybds, xbars=xbars, accumulate=acc)
            for c, op in enumerate(ops):
                w = oracle.ARITY[op]
                check_block(op, xs[c], ybs[c], host(ys[c]).reshape(n, w), host(xbs[c]).reshape(n, w), dt,
                            None if not acc else olds[c].astype(np.float64))


def test_tuple_rows_equal_blocks_bit_for_bit():
    """The rows layout only moves data: on inputs where every partial result is
    an exact small integer (so the scans' combination order cannot change a
    bit), its results equal the blocks layout's exactly."""
    g = np.random.default_rng(77)
    ops = ("sop", "lin", "mm2", "add", "max")
    n = 50_001
    ints = lambda lo, hi, *shape: g.integers(lo, hi + 1, shape).astype(np.float32)
    perm = np.array([[1, 0, 0, 1], [0, 1, 1, 0], [-1, 0, 0, 1], [0, -1, 1, 0]], np.float32)
    x = np.concatenate([ints(-2, 2, n, 2),                                       # sop (p, s)
                        np.stack([ints(-3, 3, n), np.ones(n, np.float32)], 1),  # lin (b, c = 1)
                        perm[g.integers(0, 4, n)],                              # signed permutations
                        ints(-4, 4, n, 1), ints(-50, 50, n, 1)], 1)
    yb = ints(-3, 3, *x.shape)
    xd, ybd = dev(np.ascontiguousarray(x)), dev(yb)
    y = adcomb.tscan_fwd(ops, xd)
    xb = adcomb.tscan_vjp(ops, xd, y, ybd)
    blocks = oracle.tuple_blocks(ops)
    xs = [xd[:, o:o + w].contiguous() for _, o, w in blocks]
    ybs = [ybd[:, o:o + w].contiguous() for _, o, w in blocks]
    ys = adcomb.tscan_fwd_blocks(ops, xs)
    xbs = adcomb.tscan_vjp_blocks(ops, xs, ys, ybs)
    yr, xbr = oracle.tscan_fwd(ops, x), oracle.tscan_vjp(ops, x, yb)
    assert np.abs(yr).max() < 2 ** 23 and np.abs(xbr).max() < 2 ** 23
    assert np.array_equal(host(y), yr.astype(np.float32))
    assert np.array_equal(host(xb), xbr.astype(np.float32))
    for c, (_, o, w) in enumerate(blocks):
        assert torch.equal(y[:, o:o + w], ys[c])
        assert torch.equal(xb[:, o:o + w], xbs[c])


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("ops", [("min",) * 7, ("max",) * 3, ("min", "max", "add")], ids="-".join)
def test_tuple_minmax_ties_and_nans_exact(ops, dt):
    """Tied levels everywhere and NaNs (5% of the entries, and row 0 in some
    blocks) through the tuple entry points, with integer ybar: the selections
    and every adjoint (an exact sum) must equal the oracle's bit for bit.  A
    NaN never wins after row 0; a NaN in row 0 makes its whole block NaN and
    sends the block's whole adjoint to row 0."""
    g = np.random.default_rng(61 + len(ops))
    for n in (1000, 100_003):
        x = ((g.integers(0, 64, (n, len(ops))) - 32) / 8.0).astype(dt)
        x[g.random(x.shape) < 0.05] = np.nan
        x[0] = 1.0
        x[0, ::3] = np.nan
        yb = g.integers(-3, 4, x.shape).astype(dt)
        xd = dev(x)
        y = adcomb.tscan_fwd(ops, xd)
        xb = adcomb.tscan_vjp(ops, xd, y, dev(yb))
        assert np.array_equal(host(y), oracle.tscan_fwd(ops, x).astype(dt), equal_nan=True)
        assert np.array_equal(host(xb), oracle.tscan_vjp(ops, x, yb).astype(dt))


def test_tuple_single_block_equals_scalar_entry():
    """k = 1 scans the rows in place with the scalar entry's kernels (integer
    inputs: exact, so any combination order gives the same bits)."""
    g = np.random.default_rng(5)
    x = g.integers(-2, 3, (50_001, 2)).astype(np.float32)
    yb = g.integers(-3, 4, x.shape).astype(np.float32)
    xd, ybd = dev(x), dev(yb)
    y = adcomb.scan_fwd("sop", xd)
    assert np.array_equal(host(y), oracle.scan_fwd("sop", x).astype(np.float32))
    assert torch.equal(adcomb.tscan_fwd(("sop",), xd), y)
    xb = adcomb.scan_vjp("sop", xd, y, ybd)
    assert np.array_equal(host(xb), oracle.scan_vjp("sop", x, yb).astype(np.float32))
    assert torch.equal(adcomb.tscan_vjp(("sop",), xd, y, ybd), xb)


@pytest.mark.slow
def test_tuple_scan_rows_large():
    """16 sumOfProd blocks (D = 32) over 4M rows: several tiles per range in every block scan."""
    g = np.random.default_rng(9)
    ops = ("sop",) * 16
    n = 4_000_001
    x = make_rows(g, ops, n, np.float32)
    yb = synth.normal(g, x.shape, np.float32)
    xd = dev(x)
    y = adcomb.tscan_fwd(ops, xd)
    xb = adcomb.tscan_vjp(ops, xd, y, dev(yb))
    yh, xbh = host(y), host(xb)
    for op, o, w in oracle.tuple_blocks(ops)[:4]:
        check_block(op, x[:, o:o + w], yb[:, o:o + w], yh[:, o:o + w], xbh[:, o:o + w], np.float32)
    torch.cuda.empty_cache()
