"""GPU parity at the benchmark's full size: reduce_by_index with the lifted *,
min and max, fp32, n = 50M, m in {31, 401, 50,000, 10M} -- the inputs bench.py
draws (same generator, same seed) and the calls it times (one shared
workspace, preallocated residuals, default strategies) -- against the fp64
oracle over the whole input.  Indices, zero counts, min/max values and their
adjoints are compared bit-exact; * results within the product tolerance."""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_2310_03568_gb300 import adcomb
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, rtol_for

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def workload():
    ensure_lib()
    adcomb.debug_force_hist_strategy(-1)
    keys, vals, hbar = bench.make_inputs(bench.N)
    ws = adcomb.Workspace()
    ws.get(max(adcomb.workspace_bytes("hist", op, torch.float32, bench.N, m) for op in bench.OPS
               for m in bench.BINS), torch.device("cuda", 0))
    return keys, vals, hbar, ws


def bin_bounds(k, v, m):
    """Per bin: population, and the largest partial product of its non-zero
    values in index order (>= 1), from prefix sums of log|v| within each bin."""
    nz = v != 0
    kk = k[nz]
    lv = np.log(np.abs(v[nz].astype(np.float64)))
    order = np.argsort(kk, kind="stable")
    kk, lv = kk[order], lv[order]
    part = np.zeros(m)
    if kk.size:
        cs = np.cumsum(lv)
        first = np.r_[True, kk[1:] != kk[:-1]]
        base = np.maximum.accumulate(np.where(first, np.arange(kk.size), 0))
        within = cs - np.r_[0.0, cs][base]
        np.maximum.at(part, kk, within)
    return np.bincount(k, minlength=m).astype(np.float64), np.exp(part)


@pytest.mark.parametrize("m", bench.BINS)
@pytest.mark.parametrize("op", bench.OPS)
def test_bench_instance_full_size(workload, op, m):
    keys, vals, hbar, ws = workload
    k, v, hb = keys[m], vals[op], hbar[m]
    n = k.shape[0]
    kd, vd, hbd = dev(k), dev(v), dev(hb)
    hist = torch.empty(m, dtype=torch.float32, device="cuda")
    saved = torch.empty(max(adcomb.saved_bytes("hist", op, torch.float32, n, m), 16), dtype=torch.uint8,
                        device="cuda")
    vbar = torch.empty(n, dtype=torch.float32, device="cuda")
    adcomb.hist_fwd(op, m, kd, vd, None, hist, saved, ws=ws)
    adcomb.hist_vjp(op, m, kd, vd, None, hist, saved, hbd, valsbar=vbar, ws=ws)
    h, sv, vb = host(hist), host(saved), host(vbar)
    del kd, vd, saved, vbar
    if op in ("min", "max"):
        ref, idx = oracle.hist_fwd(op, m, k, v)
        assert np.array_equal(h, ref.astype(np.float32))
        assert np.array_equal(sv[: 4 * m].view(np.int32), idx.astype(np.int32))
        vr, _ = oracle.hist_vjp(op, m, k, v, hb)
        assert np.array_equal(vb, vr.astype(np.float32))
        return
    rtol = rtol_for(np.float32)
    nz_r, _ = oracle.hist_mul_lifted(m, k, v)
    assert np.array_equal(sv[: 4 * m].view(np.int32), nz_r.astype(np.int32))
    pop, pmax = bin_bounds(k, v, m)
    assert_tol("hist * fwd (50M)", h, oracle.hist_fwd(op, m, k, v), pop + 1, pmax, rtol)
    vr, _ = oracle.hist_vjp(op, m, k, v, hb)
    scale = pmax[k] * np.abs(hb[k]) / np.where(v != 0, np.minimum(np.abs(v.astype(np.float64)), 1), 1)
    assert_tol("hist * vjp (50M)", vb, vr, pop[k] + 1, scale, rtol)
