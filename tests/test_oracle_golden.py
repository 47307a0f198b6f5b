"""The oracle against small worked examples of the paper's rules (tests/golden/*.json)."""
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_reduce_mul_fig3():
    for c in load("reduce_mul_fig3.json")["cases"]:
        assert oracle.reduce_fwd("mul", c["as"]) == c["y"]
        assert oracle.reduce_mul_lifted(c["as"]) == (c["n0"], c["yp"])
        assert np.array_equal(oracle.reduce_vjp("mul", c["as"], [c["ybar"]]), c["abar"])


def test_reduce_minmax_sec322():
    for c in load("reduce_min_sec322.json")["cases"]:
        y, k = oracle.reduce_fwd(c["op"], c["as"])
        assert k == c["k"] and y == float(c["y"])
        assert np.array_equal(oracle.reduce_vjp(c["op"], c["as"], [c["ybar"]]), c["abar"])


def test_hist_min_fig5():
    g = load("hist_min_fig5.json")
    h, idx = oracle.hist_fwd(g["op"], g["w"], g["ks"], g["vs"])
    assert np.array_equal(h, g["hist"]) and np.array_equal(idx, g["is_min"])
    vb, _ = oracle.hist_vjp(g["op"], g["w"], g["ks"], g["vs"], g["xbar"])
    assert np.array_equal(vb, g["vbar"])


def test_scan_add_sec531():
    g = load("scan_add_sec531.json")
    assert np.array_equal(oracle.scan_fwd("add", g["as"]), g["ys"])
    assert np.array_equal(oracle.scan_vjp("add", g["as"], g["ybar"]), g["abar"])


def test_fig8_operators():
    g = load("fig8_operators.json")
    assert np.array_equal(oracle.scan_fwd("lin", g["lin_scan"]["as"]), g["lin_scan"]["ys"])
    assert np.array_equal(oracle.reduce_fwd("mm2", g["mm2_reduce"]["as"]), g["mm2_reduce"]["y"])
