"""GPU: adc_scan_fwd_noalloc, the scan forward for callers that cannot allocate.

Such callers (allocator callbacks, plugins given only fixed buffers) pass
inputs and outputs only; the scratch lives in the library's fixed device
array.  The entry point is called directly through the C ABI, twice in a row
(the second call must not be affected by what the first left in the shared
array), and compared with the regular adc_scan_fwd, which takes a caller
workspace.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("op,dt,n", [("add", np.float32, 1_000_003), ("mul", np.float64, 70_001),
                                     ("lin", np.float32, 300_007), ("mm2", np.float32, 123_457)])
def test_noalloc_matches_regular_scan_twice(op, dt, n):
    g = np.random.default_rng(5)
    for call in range(2):  # two calls in a row on the shared scratch array
        x = synth.scan_values(g, "mm2_orth" if op == "mm2" else op, n, dt) if op != "mul" else \
            synth.uniform(g, n, 0.9, 1.1, dt)
        xd = dev(x)
        y_ref = adcomb.scan_fwd(op, xd)
        y = torch.full_like(xd, float("nan"))
        call_noalloc(op, xd, y)
        ref = host(y_ref)
        got = host(y)
        nj = np.arange(1, n + 1)
        assert_tol(f"noalloc {op} call {call}", got.reshape(ref.shape), ref, nj,
                   prefix_max(np.maximum(rowabs(x), rowabs(ref))), rtol_for(dt))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = adcomb.lib()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the size check comes first
    assert L.adc_scan_fwd_noalloc(adcomb.OPS["mm2"], adcomb.DTYPES[torch.float64], 100_000_000, fake, fake,
                                  None) == 3
    assert L.adc_scan_fwd_noalloc(adcomb.OPS["min"], 0, 10, fake, fake, None) == 2
