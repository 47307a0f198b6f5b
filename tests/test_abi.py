"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol include/adcomb.h declares, and rejects bad arguments on the host
before queueing any device work (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2310_03568_gb300 import adcomb
from paper_2310_03568_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adcomb.h")


@pytest.fixture(scope="module")
def L():
    build()
    return adcomb.lib()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 14
    raw = ctypes.CDLL(adcomb.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings(L):
    assert adcomb.status_string(0) == "ok"
    assert "timeout" in adcomb.status_string(5) or "expired" in adcomb.status_string(5)
    assert "sm_103a" in adcomb.version()


def test_size_queries(L):
    f32 = 0
    assert L.adc_workspace_bytes(1, 0, f32, 1000, 0) >= 256          # scan +
    assert L.adc_workspace_bytes(1, 2, f32, 1000, 0) >= 256          # scan min
    assert L.adc_workspace_bytes(2, 5, f32, 1000, 10) == 0           # hist mm2: unsupported
    assert L.adc_workspace_bytes(2, 0, f32, 1000, 0) == 0            # hist with m = 0
    assert L.adc_saved_bytes(2, 2, f32, 1000, 77) >= 77 * 4          # hist min: is[m]
    assert L.adc_saved_bytes(2, 1, f32, 1000, 77) >= 77 * 8          # hist *: n0[m], p[m]
    assert L.adc_saved_bytes(2, 4, f32, 1000, 77) >= 3 * 77 * 8       # hist lin, m <= 2047: L, R, A per bin
    assert L.adc_saved_bytes(2, 4, f32, 1000, 5000) >= 1000 * 16     # hist lin, larger m: perm, keys, values
    assert L.adc_saved_bytes(0, 5, f32, 10 ** 6, 0) > 0              # reduce mm2: tile prefixes
    assert L.adc_workspace_bytes(1, 6, f32, 1000, 0) >= 256          # scan sumOfProd
    assert L.adc_workspace_bytes(0, 6, f32, 1000, 0) >= 256          # reduce sumOfProd
    assert L.adc_workspace_bytes(2, 6, f32, 1000, 10) >= 256         # hist sumOfProd
    assert L.adc_workspace_bytes(0, 7, f32, 1000, 0) >= 256          # reduce 3x3 matrices
    assert L.adc_workspace_bytes(1, 8, f32, 1000, 0) >= 256          # scan 5x5 matrices
    assert L.adc_workspace_bytes(2, 7, f32, 1000, 10) == 0           # hist 3x3: unsupported
    assert L.adc_workspace_bytes(0, 9, f32, 1000, 0) == 0            # no operator 9


def test_tuple_size_queries(L):
    f32 = 0
    codes = lambda *c: (ctypes.c_int32 * len(c))(*c)
    assert L.adc_tscan_workspace_bytes(3, codes(6, 4, 0), f32, 1000, 1) >= 4 * 256   # rows: planes + 3 block ws
    assert L.adc_tscan_workspace_bytes(3, codes(6, 4, 0), f32, 1000, 0) >= 4 * 256   # blocks: 3 block ws
    assert L.adc_tscan_workspace_bytes(1, codes(6), f32, 1000, 1) == L.adc_workspace_bytes(1, 6, f32, 1000, 0)
    assert L.adc_tscan_workspace_bytes(3, codes(8, 8, 8), f32, 10, 1) == 0           # rows of 75 > 64 scalars
    assert L.adc_tscan_workspace_bytes(3, codes(8, 8, 8), f32, 10, 0) > 0            # as separate arrays: fine
    assert L.adc_tscan_workspace_bytes(0, codes(0), f32, 10, 1) == 0                  # no blocks
    assert L.adc_tscan_workspace_bytes(2, codes(0, 9), f32, 10, 1) == 0               # no operator 9
    assert L.adc_tscan_workspace_bytes(2, None, f32, 10, 1) == 0
    # rows of one scalar operator repeated k times are the vectorised scan of width k
    for op in (0, 1, 2, 3):
        for k in (2, 16, 64):
            assert L.adc_tscan_workspace_bytes(k, codes(*[op] * k), f32, 1000, 1) == \
                L.adc_vworkspace_bytes(1, op, f32, 1000, 0, k) > 0
    # rows of k equal lin (4) / 2x2 (5) / sumOfProd (6) blocks are scanned in place as element
    # columns: per-column states only, no planes, so the workspace does not grow with n
    for op, width in ((4, 2), (5, 4), (6, 2)):
        for k in (2, 16, 64 // width):
            for dt in (0, 1):
                small = L.adc_tscan_workspace_bytes(k, codes(*[op] * k), dt, 1000, 1)
                assert small > 0
                assert L.adc_tscan_workspace_bytes(k, codes(*[op] * k), dt, 10 ** 7, 1) == small
    # mixed rows split into planes: their workspace grows with n
    assert L.adc_tscan_workspace_bytes(2, codes(4, 6), f32, 10 ** 7, 1) > \
        L.adc_tscan_workspace_bytes(2, codes(4, 6), f32, 1000, 1)


def test_tuple_host_validation(L):
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation first
    codes = lambda *c: (ctypes.c_int32 * len(c))(*c)
    many = (ctypes.c_int32 * 65)(*([0] * 65))
    assert L.adc_tscan_fwd(65, many, 0, 10, fake, fake, fake, 1 << 20, None) == 1          # k > 64
    assert L.adc_tscan_fwd(2, codes(0, -1), 0, 10, fake, fake, fake, 1 << 20, None) == 1   # bad code
    assert L.adc_tscan_fwd(3, codes(8, 8, 8), 0, 10, fake, fake, fake, 1 << 20, None) == 1  # row width 75
    assert L.adc_tscan_fwd(2, codes(0, 6), 0, 10, None, fake, fake, 1 << 20, None) == 1    # null x
    assert L.adc_tscan_fwd(2, codes(0, 6), 0, 10, fake, fake, fake, 8, None) == 3          # workspace too small
    assert L.adc_tscan_fwd_blocks(2, codes(0, 6), 0, 10, None, None, fake, 1 << 20, None) == 1
    ptrs = (ctypes.c_void_p * 2)(1 << 20, (1 << 20) + 4)                                   # misaligned block
    assert L.adc_tscan_fwd_blocks(2, codes(0, 6), 0, 10, ptrs, ptrs, fake, 1 << 20, None) == 1


def test_host_validation_rejects_before_any_device_work(L):
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation first
    ws_small = 8
    # bad enums, negative sizes
    assert L.adc_scan_fwd(9, 0, 10, fake, fake, fake, 1 << 20, None) == 1
    assert L.adc_scan_fwd(9, 0, 10, fake, fake, fake, 1 << 20, None) == 1
    assert L.adc_scan_fwd(0, 7, 10, fake, fake, fake, 1 << 20, None) == 1
    assert L.adc_scan_fwd(0, 0, -1, fake, fake, fake, 1 << 20, None) == 1
    # unsupported operator / combinator pairs
    assert L.adc_hist_fwd(7, 0, 10, 4, fake, fake, None, fake, fake, fake, 1 << 20, None) == 2  # 3x3 hist
    assert L.adc_hist_fwd(5, 0, 10, 4, fake, fake, None, fake, fake, fake, 1 << 20, None) == 2
    # null / misaligned arrays
    assert L.adc_scan_fwd(0, 0, 10, None, fake, fake, 1 << 20, None) == 1
    assert L.adc_scan_fwd(0, 0, 10, ctypes.c_void_p((1 << 20) + 4), fake, fake, 1 << 20, None) == 1
    assert L.adc_reduce_fwd(2, 0, 10, fake, fake, None, fake, 1 << 20, None) == 1   # min needs `saved`
    # histogram bounds
    assert L.adc_hist_fwd(0, 0, 10, 0, fake, fake, None, fake, None, fake, 1 << 20, None) == 1
    assert L.adc_hist_fwd(0, 0, 1 << 31, 5, fake, fake, None, fake, None, fake, 1 << 40, None) == 1
    # workspace too small is reported, not overrun
    assert L.adc_scan_fwd(0, 0, 10 ** 6, fake, fake, fake, ws_small, None) == 3
    assert L.adc_hist_fwd(2, 0, 1000, 100, fake, fake, None, fake, fake, fake, ws_small, None) == 3
    # workspace must be 256-byte aligned
    assert L.adc_scan_fwd(0, 0, 10, fake, fake, ctypes.c_void_p((1 << 20) + 16), 1 << 20, None) == 1
