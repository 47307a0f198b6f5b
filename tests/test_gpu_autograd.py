"""GPU: the torch.autograd.Function wrappers -- gradcheck in fp64, backward
against the oracle gradient, and identical results for save vs recompute."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import autograd as ag
from paper_2310_03568_gb300 import synth
from tests._gpu import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def t64(a, grad=True):
    return torch.tensor(np.asarray(a, np.float64), device="cuda", requires_grad=grad)


G = np.random.default_rng(99)


@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "lin", "mm2"])
def test_reduce_gradcheck(op):
    d = {"lin": 2, "mm2": 4}.get(op, 1)
    n = 37
    x = G.uniform(0.6, 1.4, (n, d) if d > 1 else n)
    if op in ("min", "max"):
        x = G.permutation(n) / n + 0.2
    if op == "mul":
        x[5] = 0.0  # exercises the one-zero case of Fig. 3
    xt = t64(x)
    assert torch.autograd.gradcheck(lambda z: ag.reduce(z, op), (xt,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("op", ["add", "mul", "lin", "mm2"])
@pytest.mark.parametrize("policy", ["save", "recompute"])
def test_scan_gradcheck(op, policy):
    d = {"lin": 2, "mm2": 4}.get(op, 1)
    n = 41
    x = G.uniform(0.6, 1.4, (n, d) if d > 1 else n)
    assert torch.autograd.gradcheck(lambda z: ag.scan(z, op, policy), (t64(x),), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "lin"])
def test_hist_gradcheck(op):
    d = 2 if op == "lin" else 1
    n, m = 60, 7
    k = torch.tensor(G.integers(-1, m + 1, n).astype(np.int32), device="cuda")
    v = G.uniform(0.6, 1.4, (n, d) if d > 1 else n)
    h0 = G.uniform(0.6, 1.4, (m, d) if d > 1 else m)
    if op in ("min", "max"):
        v = G.permutation(n) / n + 0.3
        h0 = G.permutation(m) / m + 0.31 + (0.0 if op == "min" else 0.6)
    f = lambda vv, hh: ag.reduce_by_index(vv, k, m, op, hist0=hh)  # noqa: E731
    assert torch.autograd.gradcheck(f, (t64(v), t64(h0)), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_backward_matches_oracle_and_policies_agree():
    n, m = 5000, 33
    k = G.integers(0, m, n).astype(np.int32)
    v = synth.scan_values(G, "lin", n, np.float32)
    hb = synth.normal(G, (m, 2), np.float32)
    grads = []
    for policy in ("save", "recompute"):
        vt = torch.tensor(v, device="cuda", requires_grad=True)
        h = ag.reduce_by_index(vt, torch.tensor(k, device="cuda"), m, "lin", policy=policy)
        h.backward(torch.tensor(hb, device="cuda"))
        grads.append(vt.grad.cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    ref, _ = oracle.hist_vjp("lin", m, k, v, hb)
    np.testing.assert_allclose(grads[0], ref, rtol=2e-3, atol=2e-3)
    x = synth.scan_values(G, "mm2_orth", n, np.float32)
    yb = synth.normal(G, x.shape, np.float32)
    sg = []
    for policy in ("save", "recompute"):
        xt = torch.tensor(x, device="cuda", requires_grad=True)
        ag.scan(xt, "mm2", policy).backward(torch.tensor(yb, device="cuda"))
        sg.append(xt.grad.cpu().numpy())
    assert np.array_equal(sg[0], sg[1])
    np.testing.assert_allclose(sg[0], oracle.scan_vjp("mm2", x, yb), rtol=2e-3, atol=2e-3)


def test_chained_hist_scan_sum_gradient_closed_form():
    # loss = sum_j scan(+)(hist)_j  =>  dloss/dhist_j = m - j, so a +-histogram's
    # value adjoint is m - k_i exactly (integers, exact in fp32 for m <= 2^24)
    n, m = 100_000, 1000
    k = torch.tensor(G.integers(0, m, n).astype(np.int32), device="cuda")
    v = torch.tensor(synth.uniform(G, n, -1, 1), device="cuda", requires_grad=True)
    loss = ag.reduce(ag.scan(ag.reduce_by_index(v, k, m, "add"), "add"), "add")
    loss.backward()
    assert torch.equal(v.grad, (m - k).to(torch.float32))
