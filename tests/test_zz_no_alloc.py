"""GPU: adc_scan_fwd_noalloc, the scan forward for callers that cannot allocate.

Such callers (code inside an allocator or memory-pool callback, where
cudaMalloc would re-enter the allocator; plugins handed only fixed buffers)
pass inputs and outputs only; the scratch lives in the library's fixed device
array.  The entry point is called directly through the C ABI, twice in a row
(the second call must not be affected by what the first left in the shared
array), and compared with the regular adc_scan_fwd, which takes a caller
workspace, and with the fp64 oracle.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2310_03568_gb300 import adcomb, synth
from tests._gpu import dev, ensure_lib, host
from tests._tol import assert_tol, prefix_max, rowabs, rtol_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_lib()


def call_noalloc(op, x, y):
    L = adcomb.lib()
    st = L.adc_scan_fwd_noalloc(adcomb.OPS[op], adcomb.DTYPES[x.dtype], x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, adcomb.status_string(st)


def make_x(g, op, n, dt):
    if op == "mul":
        return synth.uniform(g, n, 0.9, 1.1, dt)
    if op in ("min", "max"):
        return ((g.integers(0, 1024, n) - 512) / 64.0).astype(dt)
    if op in ("mm2", "mm3", "mm5"):
        return synth.scan_values(g, op + "_orth", n, dt)
    return synth.scan_values(g, op, n, dt)


@pytest.mark.parametrize("op,dt,n", [("add", np.float32, 1_000_003), ("mul", np.float64, 70_001),
                                     ("lin", np.float32, 300_007), ("mm2", np.float32, 123_457),
                                     ("min", np.float32, 200_003), ("max", np.float64, 50_001),
                                     ("sop", np.float32, 100_003), ("mm3", np.float32, 30_011),
                                     ("mm5", np.float32, 9_001)])
def test_noalloc_matches_regular_scan_and_oracle_twice(op, dt, n):
    g = np.random.default_rng(5)
    for call in range(2):  # two calls in a row on the shared scratch array
        x = make_x(g, op, n, dt)
        xd = dev(x)
        y_ref = adcomb.scan_fwd(op, xd)
        y = torch.full_like(xd, float("nan"))
        call_noalloc(op, xd, y)
        ref = host(y_ref)
        got = host(y)
        if op in ("min", "max"):  # pure selection: bit-exact
            assert np.array_equal(got, ref), f"noalloc {op} call {call} vs adc_scan_fwd"
            assert np.array_equal(got.astype(np.float64), oracle.scan_fwd(op, x).reshape(got.shape))
            continue
        nj = np.arange(1, n + 1)
        yo = oracle.scan_fwd(op, x)
        Mj = prefix_max(np.maximum(rowabs(x), rowabs(yo)))
        assert_tol(f"noalloc {op} call {call} vs adc_scan_fwd", got.reshape(ref.shape), ref, nj, Mj, rtol_for(dt))
        assert_tol(f"noalloc {op} call {call} vs oracle", got.reshape(yo.shape), yo, nj, Mj, rtol_for(dt))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = adcomb.lib()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the checks come first
    assert L.adc_scan_fwd_noalloc(adcomb.OPS["mm2"], adcomb.DTYPES[torch.float64], 100_000_000, fake, fake,
                                  None) == 3
    assert L.adc_scan_fwd_noalloc(adcomb.OPS["mm5"], adcomb.DTYPES[torch.float32], 50_000_000, fake, fake,
                                  None) == 3
    assert L.adc_scan_fwd_noalloc(adcomb.OPS["min"], 0, 2_000_000_000, fake, fake, None) == 3
    assert L.adc_scan_fwd_noalloc(9, 0, 10, fake, fake, None) == 1  # no operator 9
