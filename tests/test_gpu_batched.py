"""GPU: batched hist -> +-scan -> sum over many instances, against the oracle,
the closed-form gradient, the per-instance launches and CUDA-graph replay."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import batched as B
from paper_2310_03568_gb300 import synth
from tests._gpu import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def small_workload(seed=31, count=48):
    """Log-uniform sizes like the full workload, scaled down; includes bins beyond
    the shared-memory table and instances with fewer values than bins."""
    w = synth.batched(seed=seed, count=count, n_lo=1e2, n_hi=2e5, m_lo=16, m_hi=65536)
    return w


def oracle_reference(desc, keys, vals):
    """Per instance: hist (zero initial histogram), scan, loss, selected indices
    and the value adjoint for a unit loss adjoint, all from the fp64 oracle."""
    out = []
    for d in desc:
        n, m, o = int(d["n"]), int(d["m"]), int(d["val_off"])
        op = "add" if d["op"] == B.OPCODE["add"] else "max"
        k, v = keys[o:o + n], vals[o:o + n]
        h0 = np.zeros(m)
        if op == "max":
            h, idx = oracle.hist_fwd("max", m, k, v, h0)
        else:
            h, idx = oracle.hist_fwd("add", m, k, v, h0), None
        s = oracle.scan_fwd("add", h)
        # loss_i = reduce (+) scan; the adjoint chain uses the oracle's own vjps
        sbar = oracle.reduce_vjp("add", s, [1.0])
        hbar = oracle.scan_vjp("add", h, sbar)
        vbar, _ = oracle.hist_vjp(op, m, k, v, hbar, h0)
        out.append(dict(h=h, idx=idx, s=s, loss=oracle.reduce_fwd("add", s), vbar=vbar, op=op))
    return out


def check_problem(p, desc, keys, vals, ref):
    hist, scan, is_ = p.hist.cpu().numpy(), p.scan.cpu().numpy(), p.is_.cpu().numpy()
    vb = p.valsbar.cpu().numpy()
    total_abs = 0.0
    for d, r in zip(desc, ref):
        n, m, o, b = int(d["n"]), int(d["m"]), int(d["val_off"]), int(d["bin_off"])
        if r["op"] == "max":
            assert np.array_equal(hist[b:b + m], r["h"].astype(np.float32))
            assert np.array_equal(is_[b:b + m], r["idx"].astype(np.int32))
        else:
            pop = np.bincount(keys[o:o + n], minlength=m)
            tol = 1e-5 * np.maximum(np.abs(r["h"]), np.sqrt(pop + 1) * 1.0)
            assert np.all(np.abs(hist[b:b + m] - r["h"]) <= tol)
        # gradients are exact integers (m - j), so the comparison is bit-exact
        assert np.array_equal(vb[o:o + n], r["vbar"].astype(np.float32))
        total_abs += np.abs(r["s"]).sum()
    loss_ref = sum(r["loss"] for r in ref)
    # a sum of fp32 scan values: bounded by rtol times the sum of magnitudes
    assert abs(float(p.loss.item()) - loss_ref) <= 1e-5 * total_abs


def test_batched_matches_oracle_and_closed_form():
    w = small_workload()
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, chunk=1 << 14)
    p.forward()
    p.backward()
    torch.cuda.synchronize()
    check_problem(p, desc, keys, vals, oracle_reference(desc, keys, vals))


@pytest.mark.parametrize("items", [1, 4, 8])
@pytest.mark.parametrize("chunk,smem_bins", [(1 << 10, 2048), (1 << 16, 8192), (1 << 20, 0), (333, 24000)])
def test_batched_tunings_agree(chunk, smem_bins, items):
    from paper_2310_03568_gb300 import adcomb
    w = small_workload(seed=32, count=24)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, chunk=chunk, smem_bins=smem_bins)
    try:
        adcomb.debug_set_batched_items(items)
        p.forward()
        p.backward()
        torch.cuda.synchronize()
    finally:
        adcomb.debug_set_batched_items(4)
    check_problem(p, desc, keys, vals, oracle_reference(desc, keys, vals))


def test_graph_replay_is_idempotent_and_equals_per_instance():
    w = small_workload(seed=33, count=40)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, chunk=1 << 15)
    runs = []
    for _ in range(3):
        p.replay_forward()
        p.replay_backward()
        torch.cuda.synchronize()
        runs.append((p.loss.item(), p.valsbar.cpu().numpy().copy(), p.is_.cpu().numpy().copy()))
    for r in runs[1:]:
        assert np.array_equal(r[1], runs[0][1]) and np.array_equal(r[2], runs[0][2])
        assert abs(r[0] - runs[0][0]) <= 1e-6 * abs(runs[0][0]) + 1e-3
    loss_pi, vb_pi = B.per_instance_loss(desc, p.keys, p.vals)
    torch.cuda.synchronize()
    vb = runs[0][1]
    vbp = vb_pi.cpu().numpy()
    for d in desc:
        o, n = int(d["val_off"]), int(d["n"])
        assert np.array_equal(vb[o:o + n], vbp[o:o + n])
    ref = oracle_reference(desc, keys, vals)
    total_abs = sum(np.abs(r["s"]).sum() for r in ref)
    assert abs(loss_pi.item() - runs[0][0]) <= 2e-5 * total_abs


def test_per_instance_graph_equals_batched():
    """The per-instance baseline captured as one CUDA graph (every buffer
    allocated before capture) gives the batched path's gradient bit for bit,
    on every replay."""
    w = small_workload(seed=35, count=40)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, chunk=1 << 15)
    p.forward()
    p.backward()
    torch.cuda.synchronize()
    vb = p.valsbar.cpu().numpy().copy()
    pig = B.PerInstanceGraph(desc, p.keys, p.vals)
    for _ in range(2):
        pig.replay()
        torch.cuda.synchronize()
        assert np.array_equal(pig.valsbar.cpu().numpy(), vb)
    ref = oracle_reference(desc, keys, vals)
    total_abs = sum(np.abs(r["s"]).sum() for r in ref)
    assert abs(pig.loss.item() - p.loss.item()) <= 2e-5 * total_abs


def test_batched_autograd():
    w = small_workload(seed=34, count=16)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, chunk=1 << 14)
    v = torch.tensor(vals, device="cuda", requires_grad=True)
    loss = B.batched_loss(v, p, use_graph=True)
    (2.0 * loss).backward()
    ref = oracle_reference(desc, keys, vals)
    g = v.grad.cpu().numpy()
    for d, r in zip(desc, ref):
        o, n = int(d["val_off"]), int(d["n"])
        assert np.array_equal(g[o:o + n], (2.0 * r["vbar"]).astype(np.float32))


@pytest.mark.slow
def test_batched_full_workload_gradient_closed_form():
    """The full workload (4096 instances, ~5.9e8 values): the value adjoint of a
    +-instance is m - k exactly, of a max-instance m - j at the selected index."""
    w = synth.batched()
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals)
    p.forward()
    p.backward()
    torch.cuda.synchronize()
    vb = p.valsbar.cpu().numpy()
    is_ = p.is_.cpu().numpy()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(desc), 64, replace=False):  # oracle on a sample of instances
        d = desc[i]
        n, m, o, b = int(d["n"]), int(d["m"]), int(d["val_off"]), int(d["bin_off"])
        k, v = keys[o:o + n], vals[o:o + n]
        if d["op"] == B.OPCODE["add"]:
            assert np.array_equal(vb[o:o + n], (m - k).astype(np.float32))
        else:
            _, idx = oracle.hist_fwd("max", m, k, v, np.zeros(m))
            assert np.array_equal(is_[b:b + m], idx.astype(np.int32))
            expect = np.zeros(n, np.float32)
            sel = idx < n
            expect[idx[sel]] = (m - np.arange(m))[sel]
            assert np.array_equal(vb[o:o + n], expect)


def test_autotuner_picks_a_configuration_and_caches_it(tmp_path, monkeypatch):
    from paper_2310_03568_gb300 import adcomb, autotune
    monkeypatch.setenv("ADC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    autotune._cache = None
    w = small_workload(seed=35, count=20)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals)
    entry = autotune.tune_batched(p)
    assert entry["chunk"] in autotune.BATCHED_CHUNKS and entry["smem_bins"] in autotune.BATCHED_SMEM_BINS
    assert entry["items"] in autotune.BATCHED_ITEMS
    assert len(entry["candidates"]) == (len(autotune.BATCHED_CHUNKS) * len(autotune.BATCHED_SMEM_BINS) *
                                        len(autotune.BATCHED_ITEMS))
    p.forward()
    p.backward()
    torch.cuda.synchronize()
    check_problem(p, desc, keys, vals, oracle_reference(desc, keys, vals))
    autotune._cache = None  # reload from the file: a cache hit, no re-measurement
    again = autotune.tune_batched(B.BatchedHistScan(desc, keys, vals))
    assert again["chunk"] == entry["chunk"] and again["smem_bins"] == entry["smem_bins"]
    assert again["items"] == entry["items"]
    # single-call histogram strategy
    n, m = 400_000, 401
    g = np.random.default_rng(36)
    k = g.integers(0, m, n).astype(np.int32)
    v = synth.hist_spec_values(g, "max", n, m)
    kd, vd = torch.tensor(k, device="cuda"), torch.tensor(v, device="cuda")
    try:
        e = autotune.tune_hist("max", m, kd, vd)
        assert e["strategy"] in autotune.HIST_STRATEGIES
        h, saved = adcomb.hist_fwd("max", m, kd, vd)
        ref, idx = oracle.hist_fwd("max", m, k, v)
        assert np.array_equal(h.cpu().numpy(), ref.astype(np.float32))
        assert np.array_equal(saved.view(torch.int32).cpu().numpy()[:m], idx.astype(np.int32))
        # single-call scan: items per thread and tile shape
        x = synth.scan_values(g, "lin", 3_000_001)
        xd = torch.tensor(x, device="cuda")
        e = autotune.tune_scan("lin", xd)
        assert (e["engine"], e["range_tiles"]) in autotune.SCAN_CANDIDATES
        assert len(e["candidates"]) == len(autotune.SCAN_CANDIDATES)
        y = adcomb.scan_fwd("lin", xd).cpu().numpy()
        yr = oracle.scan_fwd("lin", x)
        assert np.abs(y - yr).max() <= 1e-3 * np.abs(yr).max()
        autotune._cache = None  # a cache hit selects the same configuration again
        assert autotune.tune_scan("lin", xd)["engine"] == e["engine"]
    finally:
        autotune.apply_scan(None)
        adcomb.debug_force_hist_strategy(-1)
