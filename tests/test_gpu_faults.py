"""GPU: bounded device waits report an error status instead of hanging.

One scan tile is told (through the library's fault-injection hook) never to
publish its aggregate, so every tile that looks back across it waits on a flag
that nothing sets.  The waits are bounded: each waiter gives up after the spin
limit, marks its own tile as failed (so later tiles stop at once) and sets the
workspace error word; the host reads ADC_ERR_TIMEOUT.  Nothing traps, nothing
faults, and the context stays usable -- a normal scan right after is checked
against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()
    yield
    adcomb.debug_set_stall_tile(-1)
    adcomb.set_spin_limit(0)


@pytest.mark.parametrize("engine", [1, 2, 3, 4, 5], ids=["per-tile", "ranges", "staged", "tma", "ranges16"])
@pytest.mark.parametrize("op,stall", [("add", 3), ("lin", 0), ("mm2", 17)])
def test_stalled_tile_times_out_and_context_survives(op, stall, engine):
    g = np.random.default_rng(8)
    n = 200_000
    x = synth.scan_values(g, op, n) if op != "add" else synth.uniform(g, n, -1, 1)
    xd = dev(x)
    ws = adcomb.Workspace()
    try:
        adcomb.debug_set_scan_engine(engine)
        adcomb.set_spin_limit(2000)          # ~0.1-1 ms per wait
        adcomb.debug_set_stall_tile(stall)   # a tile (per-tile engines) or a range (range engines)
        adcomb.scan_fwd(op, xd, ws=ws)       # queues fine: the failure is on the device
        assert adcomb.check_device_error(ws) == 5  # ADC_ERR_TIMEOUT
    finally:
        adcomb.debug_set_stall_tile(-1)
        adcomb.set_spin_limit(0)
        adcomb.debug_set_scan_engine(0)
    # the context is intact and the same workspace works again
    y = adcomb.scan_fwd(op, xd, ws=ws)
    assert adcomb.check_device_error(ws) == 0
    ref = oracle.scan_fwd(op, x)
    np.testing.assert_allclose(host(y).reshape(ref.shape), ref, rtol=1e-3, atol=1e-2)


@pytest.mark.parametrize("op", ["mm3", "mm5"])
def test_bulk_staged_matrix_scan_stall_times_out(op):
    """The bulk-staged matrix segment scans (forward, and the vjp's reverse
    scan): the stalled tile's block still waits for its own bulk copies before
    it leaves, the tiles after it time out, and the context survives."""
    g = np.random.default_rng(10)
    n = 60_000
    x = synth.scan_values(g, op + "_orth", n)
    yb = synth.normal(g, x.shape)
    xd, ybd = dev(x), dev(yb)
    y = adcomb.scan_fwd(op, xd)
    ws = adcomb.Workspace()
    for call in (lambda: adcomb.scan_fwd(op, xd, ws=ws), lambda: adcomb.scan_vjp(op, xd, y, ybd, ws=ws)):
        try:
            adcomb.set_spin_limit(2000)
            adcomb.debug_set_stall_tile(3)
            call()
            assert adcomb.check_device_error(ws) == 5
        finally:
            adcomb.debug_set_stall_tile(-1)
            adcomb.set_spin_limit(0)
    xb = adcomb.scan_vjp(op, xd, y, ybd, ws=ws)
    assert adcomb.check_device_error(ws) == 0
    ref = oracle.scan_vjp(op, x, yb)
    np.testing.assert_allclose(host(xb).reshape(ref.shape), ref, rtol=1e-3, atol=1e-2)


def test_reverse_scan_stall_times_out():
    g = np.random.default_rng(9)
    n = 150_000
    x = synth.uniform(g, n, 0.9, 1.1)
    yb = synth.normal(g, n)
    xd, ybd = dev(x), dev(yb)
    y = adcomb.scan_fwd("mul", xd)
    ws = adcomb.Workspace()
    try:
        adcomb.set_spin_limit(2000)
        adcomb.debug_set_stall_tile(5)
        adcomb.scan_vjp("mul", xd, y, ybd, ws=ws)
        assert adcomb.check_device_error(ws) == 5
    finally:
        adcomb.debug_set_stall_tile(-1)
        adcomb.set_spin_limit(0)
    xb = adcomb.scan_vjp("mul", xd, y, ybd, ws=ws)
    assert adcomb.check_device_error(ws) == 0
    np.testing.assert_allclose(host(xb), oracle.scan_vjp("mul", x, yb), rtol=1e-3, atol=1e-2)


def test_host_side_errors_are_status_codes():
    x = dev(np.zeros(10, np.float32))
    with pytest.raises(adcomb.AdcError) as e:
        adcomb.vscan_fwd("lin", dev(np.zeros((10, 4), np.float32)))  # vectorised: scalar operators only
    assert e.value.code == 2
    small = adcomb.Workspace()
    small.buf = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(adcomb.AdcError) as e:
        adcomb.lib()  # the workspace query is honest: too small is reported, not overrun
        L = adcomb.lib()
        big = dev(np.zeros(10_000_000, np.float32))
        st = L.adc_scan_fwd(0, 0, big.shape[0], big.data_ptr(), big.data_ptr(), small.buf.data_ptr(), 256,
                            torch.cuda.current_stream().cuda_stream)
        adcomb._check("adc_scan_fwd", st)
    assert e.value.code == 3
