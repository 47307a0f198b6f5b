"""GPU parity: reduce_by_index forward and vjp (Sec. 4) against the fp64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, rowabs, rtol_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()
    yield
    adcomb.debug_force_hist_strategy(-1)


def keys_oor(g, n, m, frac=0.02):
    """Uniform keys in [0, m) with a fraction replaced by out-of-range keys (negative or >= m)."""
    k = g.integers(0, m, n).astype(np.int32)
    bad = g.random(n) < frac
    k[bad] = np.where(g.random(int(bad.sum())) < 0.5, -1 - g.integers(0, 5, int(bad.sum())),
                      m + g.integers(0, 5, int(bad.sum()))).astype(np.int32)
    return k


def bin_stats(k, v, m):
    """Per-bin population and max |value|."""
    inr = (k >= 0) & (k < m)
    pop = np.bincount(k[inr], minlength=m)
    mx = np.zeros(m)
    np.maximum.at(mx, k[inr], np.abs(v[inr].astype(np.float64)))
    return pop, mx


def bin_partial_products(k, v, m):
    """Per-bin max |partial product| of the non-zero values (>= 1), from sorted log-sums."""
    inr = (k >= 0) & (k < m) & (v != 0)
    kk, lv = k[inr], np.log(np.abs(v[inr].astype(np.float64)))
    order = np.argsort(kk, kind="stable")
    kk, lv = kk[order], lv[order]
    cs = np.cumsum(lv)
    start = np.r_[0, np.nonzero(np.diff(kk))[0] + 1] if kk.size else np.zeros(0, int)
    seg_base = np.zeros_like(cs)
    if kk.size:
        base_vals = np.r_[0.0, cs][start]
        seg_id = np.cumsum(np.r_[0, np.diff(kk) != 0])
        seg_base = base_vals[seg_id]
    part = cs - seg_base
    out = np.zeros(m)
    if kk.size:
        np.maximum.at(out, kk, part)
    return np.exp(out)


STRATS = [-1, 0, 1, 2, 3, 4, 5, 6, 7, 8]  # auto, per-warp, per-block, global, per-thread, partitioned, split,
                                          # cluster, two passes, block pairs


def fits(op, dt, m, s):
    """Mirror of the library's shared-memory budgets: strategies that cannot hold
    the table are skipped (the library would fall back to its own choice)."""
    sz = np.dtype(dt).itemsize
    if op in ("min", "max") and dt == np.float64:
        return s in (-1, 2)
    if s == 4:
        return True
    if s == 5:  # lifted fp32 min/max whose packed table needs 2-4 block tables
        return op in ("min", "max") and sz == 4 and 200 * 1024 < m * 8 <= 4 * 200 * 1024
    if s == 6:  # the same spread over the blocks of a 2-8 block cluster
        return op in ("min", "max") and sz == 4 and 200 * 1024 < m * 8 <= 8 * 200 * 1024
    if s in (7, 8):  # value tables per block, then an index pass; block pairs with value and index tables
        return op in ("min", "max") and sz == 4 and m * 8 > 200 * 1024 and m * 4 <= 200 * 1024
    e = {"add": sz, "mul": sz + 4, "min": 8, "max": 8}[op]
    if s == 3:
        return m * e * 256 <= 64 * 1024
    if s == 0:
        return m * e * 8 <= 48 * 1024
    if s == 1:
        return m * (sz if op == "mul" else e) <= 200 * 1024
    return True


# the last case is large enough for the automatic choice to partition by bin range; m = 25,601 and
# 51,199 bound the range where lifted fp32 min/max tables need two blocks (odd halves), n = 5 the tail
CASES = [(0, 7), (1, 1), (33, 5), (4097, 31), (100_003, 401), (100_003, 5000), (300_001, 50_000),
         (5, 30_000), (100_001, 25_601), (400_003, 51_199), (3_000_001, 2_000_003)]


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("strategy", STRATS)
def test_hist_add(dt, strategy):
    g = np.random.default_rng(21)
    rtol = rtol_for(dt)
    for n, m in CASES:
        if not fits("add", dt, m, strategy):
            continue
        adcomb.debug_force_hist_strategy(strategy)
        k = keys_oor(g, n, m)
        v = synth.uniform(g, n, -1, 1, dt)
        h0 = synth.uniform(g, m, -1, 1, dt)
        for hist0 in (None, h0):
            h, saved = adcomb.hist_fwd("add", m, dev(k), dev(v), None if hist0 is None else dev(hist0))
            ref = oracle.hist_fwd("add", m, k, v, hist0)
            pop, mx = bin_stats(k, v, m)
            if hist0 is not None:
                mx = np.maximum(mx, np.abs(hist0))
            assert_tol("hist + fwd", host(h), ref, pop + 1, mx, rtol)
            hb = synth.normal(g, m, dt)
            vb, h0b = adcomb.hist_vjp("add", m, dev(k), dev(v), None, h, saved, dev(hb), want_hist0bar=True)
            vr, h0r = oracle.hist_vjp("add", m, k, v, hb, hist0)
            assert np.array_equal(host(vb), vr.astype(dt))   # a gather: bit-exact
            assert np.array_equal(host(h0b), h0r.astype(dt))
    adcomb.debug_force_hist_strategy(-1)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("op", ["min", "max"])
def test_hist_minmax_bit_exact(op, dt, strategy):
    g = np.random.default_rng(22)
    for n, m in CASES:
        if not fits(op, dt, m, strategy):
            continue
        adcomb.debug_force_hist_strategy(strategy)
        k = keys_oor(g, n, m)
        v = synth.hist_spec_values(g, op, n, m, dt)  # 1024 exact levels: ties in every bin
        h0 = ((g.integers(0, 1024, m) - 512) / 64.0).astype(dt)
        for hist0 in (None, h0):
            h, saved = adcomb.hist_fwd(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0))
            ref, idx = oracle.hist_fwd(op, m, k, v, hist0)
            assert np.array_equal(host(h), ref.astype(dt))
            assert np.array_equal(host(saved.view(torch.int32))[:m], idx.astype(np.int32))
            hb = synth.normal(g, m, dt)
            for acc in (False, True):
                old = synth.normal(g, n, dt)
                old_h0 = synth.normal(g, m, dt)
                vb, h0b = adcomb.hist_vjp(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                          dev(hb), valsbar=dev(old) if acc else None,
                                          hist0bar=dev(old_h0) if (acc and hist0 is not None) else None,
                                          want_hist0bar=hist0 is not None, accumulate=acc)
                vr, h0r = oracle.hist_vjp(op, m, k, v, hb, hist0)
                expect = (old.astype(np.float64) + vr).astype(dt) if acc else vr.astype(dt)
                assert np.array_equal(host(vb), expect)
                if hist0 is not None:
                    expect_h0 = (old_h0.astype(np.float64) + h0r).astype(dt) if acc else h0r.astype(dt)
                    assert np.array_equal(host(h0b), expect_h0)
    adcomb.debug_force_hist_strategy(-1)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("strategy", STRATS)
def test_hist_mul_zero_counting(dt, strategy):
    g = np.random.default_rng(23)
    rtol = rtol_for(dt)
    for n, m in CASES:
        if not fits("mul", dt, m, strategy):
            continue
        adcomb.debug_force_hist_strategy(strategy)
        k = keys_oor(g, n, m)
        # well-conditioned values so that bin products stay representable; 0, 1 or 2 zeros per bin
        v = np.exp(g.uniform(-1, 1, n) * 3.0 / np.sqrt(max(n / m, 1))).astype(dt)
        for j in range(min(m, 40)):
            members = np.nonzero(k == j)[0]
            v[members[: j % 3]] = 0
        h0 = synth.uniform(g, m, 0.5, 1.5, dt)
        for hist0 in (None, h0):
            h, saved = adcomb.hist_fwd("mul", m, dev(k), dev(v), None if hist0 is None else dev(hist0))
            ref = oracle.hist_fwd("mul", m, k, v, hist0)
            pop, _ = bin_stats(k, v, m)
            pmax = bin_partial_products(k, v, m) * (np.abs(hist0) if hist0 is not None else 1.0)
            assert_tol("hist * fwd", host(h), ref, pop + 1, pmax, rtol)
            sv = host(saved)
            nz_r, p_r = oracle.hist_mul_lifted(m, k, v)
            assert np.array_equal(sv[: 4 * m].view(np.int32), nz_r.astype(np.int32))
            off = ((4 * m + 15) // 16) * 16
            p = sv[off: off + m * np.dtype(dt).itemsize].view(dt)
            assert_tol("hist * p", p, p_r, pop, bin_partial_products(k, v, m), rtol)
            hb = synth.normal(g, m, dt)
            vb, h0b = adcomb.hist_vjp("mul", m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                      dev(hb), want_hist0bar=True)
            vr, h0r = oracle.hist_vjp("mul", m, k, v, hb, hist0)
            inr = (k >= 0) & (k < m)
            kc = np.clip(k, 0, m - 1)
            scale = pmax[kc] * np.abs(hb[kc]) / np.where(v != 0, np.minimum(np.abs(v.astype(np.float64)), 1), 1)
            assert_tol("hist * vjp", host(vb), vr, np.where(inr, pop[kc], 1), np.where(inr, scale, 0), rtol)
            assert_tol("hist * hist0bar", host(h0b), h0r, pop, bin_partial_products(k, v, m) * np.abs(hb), rtol)
    adcomb.debug_force_hist_strategy(-1)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("op", ["mul", "min", "max"])
def test_hist_original_primal(op, dt, strategy):
    """The un-lifted primal (saved = NULL: the program being differentiated,
    timed for the AD overhead) gives the same histogram as the lifted forward:
    min/max bit-exact; * within the product tolerance, exactly 0 where a bin
    holds a zero."""
    g = np.random.default_rng(24)
    rtol = rtol_for(dt)
    for n, m in CASES:
        if not fits(op, dt, m, strategy):
            continue
        adcomb.debug_force_hist_strategy(strategy)
        k = keys_oor(g, n, m)
        if op == "mul":
            v = np.exp(g.uniform(-1, 1, n) * 3.0 / np.sqrt(max(n / m, 1))).astype(dt)
            v[g.random(n) < 0.001] = 0
            h0 = synth.uniform(g, m, 0.5, 1.5, dt)
        else:
            v = synth.hist_spec_values(g, op, n, m, dt)
            h0 = ((g.integers(0, 1024, m) - 512) / 64.0).astype(dt)
        for hist0 in (None, h0):
            h = host(adcomb.hist_primal(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0)))
            ref = oracle.hist_fwd(op, m, k, v, hist0)
            if op == "mul":
                pop, _ = bin_stats(k, v, m)
                pmax = bin_partial_products(k, v, m) * (np.abs(hist0) if hist0 is not None else 1.0)
                assert_tol("hist * primal", h, ref, pop + 1, pmax, rtol)
                assert np.array_equal(h == 0, ref == 0)
            else:
                assert np.array_equal(h, ref[0].astype(dt))
    adcomb.debug_force_hist_strategy(-1)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_hist_sop_invertible_rule(dt):
    """sumOfProd reduce_by_index (Sec. 3.3 operator, Sec. 4 per bin): forward
    (atomics split into s_old = atomicAdd(S, s); atomicAdd(P, p + s_old*s)) and
    the invertible-operator vjp, against the oracle.  M_j bounds every partial
    result of bin j's fold: |p| <= sum|p| + (sum|s|)^2 over hist0 and the bin."""
    g = np.random.default_rng(25)
    rtol = rtol_for(dt)
    for n, m in CASES:
        k = keys_oor(g, n, m)
        v = synth.uniform(g, (n, 2), -1, 1, dt)
        h0 = synth.uniform(g, (m, 2), -1, 1, dt)
        for hist0 in (None, h0):
            h, saved = adcomb.hist_fwd("sop", m, dev(k), dev(v), None if hist0 is None else dev(hist0))
            ref = oracle.hist_fwd("sop", m, k, v, hist0)
            inr = (k >= 0) & (k < m)
            a = np.abs(v.astype(np.float64))
            sp = np.bincount(k[inr], weights=a[inr, 0], minlength=m)
            ss = np.bincount(k[inr], weights=a[inr, 1], minlength=m)
            if hist0 is not None:
                sp, ss = sp + np.abs(hist0[:, 0]), ss + np.abs(hist0[:, 1])
            pop, _ = bin_stats(k, v[:, 0] if n else np.zeros(0), m)
            assert_tol("hist sop fwd", host(h), ref, pop + 1, sp + ss ** 2, rtol)
            hb = synth.normal(g, (m, 2), dt)
            for acc in (False, True):
                old = synth.normal(g, (n, 2), dt)
                old_h0 = synth.normal(g, (m, 2), dt)
                vb, h0b = adcomb.hist_vjp("sop", m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                          dev(hb), valsbar=dev(old) if acc else None,
                                          hist0bar=dev(old_h0) if acc else None, want_hist0bar=True, accumulate=acc)
                vr, h0r = oracle.hist_vjp("sop", m, k, v, hb, hist0)
                kc = np.clip(k, 0, m - 1)
                Mv = np.abs(hb[:, 0]) * ss + np.abs(hb[:, 1])
                if acc:
                    vr, h0r = vr + old, h0r + old_h0
                assert_tol("hist sop vjp", host(vb), vr, np.where(inr, pop[kc] + 1, 1),
                           np.where(inr, Mv[kc], 0) + (rowabs(old) if acc else 0), rtol)
                assert_tol("hist sop hist0bar", host(h0b), h0r, pop + 1, Mv + (rowabs(old_h0) if acc else 0), rtol)


# ------------------------------------------------------- general (lin) ----
def lin_bin_scales(k, v, m, h0):
    """Per bin: max |partial fold| (hist0 first) and max suffix product of c, both >= 1."""
    A = np.ones(m) if h0 is None else np.maximum(1.0, rowabs(h0))
    R = np.ones(m)
    idx = np.nonzero((k >= 0) & (k < m))[0]
    order = idx[np.argsort(k[idx], kind="stable")]
    ks = k[order]
    if ks.size == 0:
        return A, R
    bounds = np.r_[0, np.nonzero(np.diff(ks))[0] + 1, ks.size]
    for a, b in zip(bounds[:-1], bounds[1:]):
        j = ks[a]
        members = order[a:b]
        seq = v[members].astype(np.float64)
        if h0 is not None:
            seq = np.vstack([h0[j:j + 1].astype(np.float64), seq])
        A[j] = max(1.0, rowabs(oracle.scan_fwd("lin", seq)).max())
        c = np.abs(v[members, 1].astype(np.float64))
        R[j] = max(1.0, float(np.exp(np.max(np.cumsum(np.log(c[::-1]))))))
    return A, R


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("path", ["auto", "sort"])
def test_hist_lin_general_sort_path(dt, path):
    """linFnComp reduce_by_index (not commutative: index order within a bin).
    'auto' takes the hierarchical path (chunk-local stable sort + column scans)
    for m <= 2047 (fp32) / 1023 (fp64) and the global stable radix sort above; 'sort' forces the
    global sort everywhere (strategy hook 2), whose permutation is checked
    bit-exact."""
    g = np.random.default_rng(24)
    rtol = rtol_for(dt)
    adcomb.debug_force_hist_strategy(2 if path == "sort" else -1)
    for n, m in [(0, 3), (1, 1), (33, 4), (5000, 7), (40_000, 1000), (70_001, 2047), (50_000, 3000), (20_000, 70_000),
                 (300_007, 1000)]:
        k = keys_oor(g, n, m)
        v = synth.scan_values(g, "lin", n, dt)
        h0 = synth.scan_values(g, "lin", m, dt)
        for hist0 in (None, h0):
            h, saved = adcomb.hist_fwd("lin", m, dev(k), dev(v), None if hist0 is None else dev(hist0))
            ref = oracle.hist_fwd("lin", m, k, v, hist0)
            pop, _ = bin_stats(k, v[:, 0] if n else np.zeros(0), m)
            A, R = lin_bin_scales(k, v, m, hist0)
            assert_tol("hist lin fwd", host(h), ref, pop + 1, A, rtol)
            if path == "sort" or m > (2047 if dt == np.float32 else 1023):
                # the sort permutation is unique (stable): bit-exact
                perm = host(saved[: 4 * n].view(torch.int32)) if n else np.zeros(0, np.int32)
                assert np.array_equal(perm, oracle.sort_perm(m, k).astype(np.int32))
            hb = synth.normal(g, (m, 2), dt)
            for acc in (False, True):
                old = synth.normal(g, (n, 2), dt)
                vb, h0b = adcomb.hist_vjp("lin", m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                          dev(hb), valsbar=dev(old) if acc else None, want_hist0bar=True,
                                          accumulate=acc)
                vr, h0r = oracle.hist_vjp("lin", m, k, v, hb, hist0)
                if acc:
                    vr = vr + old
                kc = np.clip(k, 0, m - 1)
                inr = (k >= 0) & (k < m)
                scale = np.where(inr, 3 * A[kc] * R[kc] * rowabs(hb)[kc], 0) + (rowabs(old) if acc else 0)
                assert_tol("hist lin vjp", host(vb), vr, np.where(inr, pop[kc] + 1, 1), scale, rtol)
                if not acc:
                    assert_tol("hist lin hist0bar", host(h0b), h0r, pop + 1, 3 * A * R * rowabs(hb), rtol)
    adcomb.debug_force_hist_strategy(-1)


def test_hist_unsupported_and_invalid():
    k = dev(np.zeros(4, np.int32))
    v = dev(np.zeros((4, 4), np.float32))
    with pytest.raises(adcomb.AdcError) as e:
        adcomb.hist_fwd("mm2", 3, k, v)
    assert e.value.code == 2
    with pytest.raises(adcomb.AdcError) as e:
        adcomb.hist_fwd("add", 0, k, dev(np.zeros(4, np.float32)))
    assert e.value.code == 1


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["min", "max"])
def test_hist_sel_vjp_forms(op, dt):
    """Every form of the min/max vjp (gather pass; zero-fill + scatter; bitmap
    of the selected elements + streaming pass), forced
    on both sides of the automatic threshold, equal the oracle bit-exactly
    (each adjoint is one histbar value or zero; with accumulate, one add)."""
    g = np.random.default_rng(61)
    try:
        for n, m in [(0, 5), (7, 3), (100_003, 31), (100_003, 50_000), (1_000_003, 400_000), (20_001, 200_000)]:
            k = keys_oor(g, n, m)
            v = ((g.integers(0, 64, n) - 32) / 8.0).astype(dt)
            hb = synth.normal(g, m, dt)
            h, saved = adcomb.hist_fwd(op, m, dev(k), dev(v))
            ref, _ = oracle.hist_vjp(op, m, k, v, hb)
            old = synth.normal(g, n, dt)
            for form in (0, 1, 2, 3):
                adcomb.debug_set_sel_vjp_form(form)
                vb, _ = adcomb.hist_vjp(op, m, dev(k), dev(v), None, h, saved, dev(hb))
                assert np.array_equal(host(vb), ref.astype(dt)), (n, m, form)
                vb2, _ = adcomb.hist_vjp(op, m, dev(k), dev(v), None, h, saved, dev(hb), valsbar=dev(old),
                                         accumulate=True)
                assert np.array_equal(host(vb2), (old + ref.astype(dt)).astype(dt)), (n, m, form)
    finally:
        adcomb.debug_set_sel_vjp_form(0)


@pytest.mark.parametrize("op", ["min", "max"])
def test_hist_sel_cluster_sizes(op):
    """Lifted fp32 min/max with the table spread over clusters of 2 to 8 blocks
    (distributed shared memory), forward and vjp bit-exact against the oracle,
    with and without hist0, with exact ties everywhere (64 value levels)."""
    g = np.random.default_rng(71)
    try:
        adcomb.debug_force_hist_strategy(6)
        for n, m in [(1, 25_601), (200_003, 30_000), (500_001, 50_000), (400_003, 120_007), (300_001, 204_800)]:
            k = keys_oor(g, n, m)
            v = ((g.integers(0, 64, n) - 32) / 8.0).astype(np.float32)
            h0 = ((g.integers(0, 64, m) - 40) / 8.0).astype(np.float32)
            hb = synth.normal(g, m, np.float32)
            for hist0 in (None, h0):
                h, saved = adcomb.hist_fwd(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0))
                ref, idx = oracle.hist_fwd(op, m, k, v, hist0)
                assert np.array_equal(host(h), ref.astype(np.float32)), (n, m)
                assert np.array_equal(host(saved.view(torch.int32))[:m], idx.astype(np.int32)), (n, m)
                vb, h0b = adcomb.hist_vjp(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                          dev(hb), want_hist0bar=True)
                vr, h0r = oracle.hist_vjp(op, m, k, v, hb, hist0)
                assert np.array_equal(host(vb), vr.astype(np.float32)), (n, m)
                assert np.array_equal(host(h0b), h0r.astype(np.float32)), (n, m)
    finally:
        adcomb.debug_force_hist_strategy(-1)


@pytest.mark.parametrize("op", ["min", "max"])
def test_hist_sel_twopass(op):
    """Lifted fp32 min/max by value tables per block plus an index pass, across
    its range of m, forward and vjp bit-exact (ties everywhere, signed zeros)."""
    g = np.random.default_rng(73)
    try:
        adcomb.debug_force_hist_strategy(7)
        for n, m in [(1, 25_601), (7, 30_000), (200_003, 30_000), (500_001, 50_000), (400_003, 51_200)]:
            k = keys_oor(g, n, m)
            v = ((g.integers(0, 64, n) - 32) / 8.0).astype(np.float32)
            v[g.random(n) < 0.05] = -0.0
            h0 = ((g.integers(0, 64, m) - 40) / 8.0).astype(np.float32)
            hb = synth.normal(g, m, np.float32)
            for hist0 in (None, h0):
                h, saved = adcomb.hist_fwd(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0))
                ref, idx = oracle.hist_fwd(op, m, k, v, hist0)
                assert np.array_equal(host(h).view(np.uint32), ref.astype(np.float32).view(np.uint32)), (n, m)
                assert np.array_equal(host(saved.view(torch.int32))[:m], idx.astype(np.int32)), (n, m)
                vb, h0b = adcomb.hist_vjp(op, m, dev(k), dev(v), None if hist0 is None else dev(hist0), h, saved,
                                          dev(hb), want_hist0bar=True)
                vr, h0r = oracle.hist_vjp(op, m, k, v, hb, hist0)
                assert np.array_equal(host(vb), vr.astype(np.float32)), (n, m)
                assert np.array_equal(host(h0b), h0r.astype(np.float32)), (n, m)
    finally:
        adcomb.debug_force_hist_strategy(-1)
