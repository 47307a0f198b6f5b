"""Thin ctypes binding of libadcomb (include/adcomb.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
torch supplies device memory and the current stream.  The library is loaded on
first use; if it is missing or cannot be loaded this module raises -- there is
no CPU fallback.

Names and argument order follow the C ABI: ``reduce_fwd``, ``reduce_vjp``,
``scan_fwd``, ``scan_vjp``, ``hist_fwd``, ``hist_vjp`` (plus workspace and
saved-buffer queries).  Tensors are CUDA tensors; tuple operators take
``[n, 2]`` (lin: ``(b, c)``) or ``[n, 4]`` (mm2: row-major 2x2) tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadcomb.so")

OPS = {"add": 0, "mul": 1, "min": 2, "max": 3, "lin": 4, "mm2": 5, "sop": 6, "mm3": 7, "mm5": 8}
ARITY = {"add": 1, "mul": 1, "min": 1, "max": 1, "lin": 2, "mm2": 4, "sop": 2, "mm3": 9, "mm5": 25}
DTYPES = {torch.float32: 0, torch.float64: 1}
KIND = {"reduce": 0, "scan": 1, "hist": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "workspace too small", 4: "CUDA error",
          5: "device wait expired"}


class AdcError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn}: status {code} ({STATUS.get(code, '?')})")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load libadcomb.so (build it first with paper_2310_03568_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libadcomb.so not found at {LIB_PATH}; run the build first")
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, sz, p = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
            sig = {
                "adc_workspace_bytes": ([i32, i32, i32, i64, i64], sz),
                "adc_saved_bytes": ([i32, i32, i32, i64, i64], sz),
                "adc_reduce_fwd": ([i32, i32, i64, p, p, p, p, sz, p], i32),
                "adc_reduce_vjp": ([i32, i32, i64, p, p, p, p, p, i32, p, sz, p], i32),
                "adc_scan_fwd": ([i32, i32, i64, p, p, p, sz, p], i32),
                "adc_scan_vjp": ([i32, i32, i64, p, p, p, p, i32, p, sz, p], i32),
                "adc_scan_fwd_noalloc": ([i32, i32, i64, p, p, p], i32),
                "adc_hist_fwd": ([i32, i32, i64, i64, p, p, p, p, p, p, sz, p], i32),
                "adc_hist_vjp": ([i32, i32, i64, i64, p, p, p, p, p, p, p, p, i32, p, sz, p], i32),
                "adc_check_device_error": ([p, sz, p], i32),
                "adc_transpose": ([i32, i64, i64, p, p, p], i32),
                "adc_vworkspace_bytes": ([i32, i32, i32, i64, i64, i64], sz),
                "adc_vsaved_bytes": ([i32, i32, i32, i64, i64, i64], sz),
                "adc_vreduce_fwd": ([i32, i32, i64, i64, p, p, p, p, sz, p], i32),
                "adc_vreduce_vjp": ([i32, i32, i64, i64, p, p, p, p, p, i32, p, sz, p], i32),
                "adc_vscan_fwd": ([i32, i32, i64, i64, p, p, p, sz, p], i32),
                "adc_vscan_vjp": ([i32, i32, i64, i64, p, p, p, p, i32, p, sz, p], i32),
                "adc_vhist_fwd": ([i32, i32, i64, i64, i64, p, p, p, p, p, p, sz, p], i32),
                "adc_vhist_vjp": ([i32, i32, i64, i64, i64, p, p, p, p, p, p, p, p, i32, p, sz, p], i32),
                "adc_tscan_workspace_bytes": ([i32, p, i32, i64, i32], sz),
                "adc_tscan_fwd": ([i32, p, i32, i64, p, p, p, sz, p], i32),
                "adc_tscan_vjp": ([i32, p, i32, i64, p, p, p, p, i32, p, sz, p], i32),
                "adc_tscan_fwd_blocks": ([i32, p, i32, i64, p, p, p, sz, p], i32),
                "adc_tscan_vjp_blocks": ([i32, p, i32, i64, p, p, p, p, i32, p, sz, p], i32),
                "adc_set_spin_limit": ([i64], None),
                "adc_debug_set_stall_tile": ([i64], None),
                "adc_debug_force_hist_strategy": ([i32], None),
                "adc_debug_set_sel_vjp_form": ([i32], None),
                "adc_debug_set_scan_engine": ([i32], None),
                "adc_debug_set_scan_range_tiles": ([i32], None),
                "adc_debug_set_scan_prefetch": ([i32], None),
                "adc_debug_set_batched_items": ([i32], None),
                "adc_status_string": ([i32], ctypes.c_char_p),
                "adc_version": ([], ctypes.c_char_p),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(fn, code):
    if code != 0:
        raise AdcError(fn, code)


def _dt(t):
    try:
        return DTYPES[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {t.dtype}") from None


class Workspace:
    """Caller-owned device scratch, grown on demand (torch allocation)."""

    def __init__(self, device=None):
        self.device = device
        self.buf = None

    def get(self, nbytes, device):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        return self.buf


_default_ws = {}


def default_workspace(device):
    key = (device.type, device.index)
    if key not in _default_ws:
        _default_ws[key] = Workspace()
    return _default_ws[key]


def workspace_bytes(kind, op, dtype, n, m=0):
    return int(lib().adc_workspace_bytes(KIND[kind], OPS[op], DTYPES[dtype], int(n), int(m)))


def saved_bytes(kind, op, dtype, n, m=0):
    return int(lib().adc_saved_bytes(KIND[kind], OPS[op], DTYPES[dtype], int(n), int(m)))


def _n(x, op):
    return x.shape[0] if x.dim() > 0 else 1


def _ws(kind, op, x, n, m, ws):
    need = workspace_bytes(kind, op, x.dtype, n, m)
    w = (ws or default_workspace(x.device)).get(need, x.device)
    return w, w.numel()


# ---------------------------------------------------------------- reduce ----
def reduce_fwd(op, x, y=None, saved=None, ws=None, stream=None):
    """Returns (y, saved).  y has shape [] (scalars) or [d]."""
    n = x.shape[0]
    d = ARITY[op]
    if y is None:
        y = torch.empty((d,) if d > 1 else (1,), dtype=x.dtype, device=x.device)
    if saved is None:
        saved = torch.empty(max(saved_bytes("reduce", op, x.dtype, n), 16), dtype=torch.uint8, device=x.device)
    w, wb = _ws("reduce", op, x, n, 0, ws)
    _check("adc_reduce_fwd", lib().adc_reduce_fwd(OPS[op], _dt(x), n, _ptr(x), _ptr(y), _ptr(saved), _ptr(w), wb,
                                                   _stream(stream)))
    return y, saved


def reduce_vjp(op, x, y, saved, ybar, xbar=None, accumulate=False, ws=None, stream=None):
    n = x.shape[0]
    if xbar is None:
        xbar = torch.empty_like(x)
    w, wb = _ws("reduce", op, x, n, 0, ws)
    _check("adc_reduce_vjp", lib().adc_reduce_vjp(OPS[op], _dt(x), n, _ptr(x), _ptr(y), _ptr(saved), _ptr(ybar),
                                                   _ptr(xbar), int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return xbar


# ------------------------------------------------------------------ scan ----
def scan_fwd(op, x, y=None, ws=None, stream=None):
    n = x.shape[0]
    if y is None:
        y = torch.empty_like(x)
    w, wb = _ws("scan", op, x, n, 0, ws)
    _check("adc_scan_fwd", lib().adc_scan_fwd(OPS[op], _dt(x), n, _ptr(x), _ptr(y), _ptr(w), wb, _stream(stream)))
    return y


def scan_fwd_noalloc(op, x, y=None, stream=None):
    """scan_fwd without caller scratch: for callers that cannot allocate (the
    library keeps the scratch in a fixed 4 MiB device array; see the header)."""
    n = x.shape[0]
    if y is None:
        y = torch.empty_like(x)
    _check("adc_scan_fwd_noalloc", lib().adc_scan_fwd_noalloc(OPS[op], _dt(x), n, _ptr(x), _ptr(y), _stream(stream)))
    return y


def scan_vjp(op, x, y, ybar, xbar=None, accumulate=False, ws=None, stream=None):
    n = ybar.shape[0]
    if xbar is None:
        xbar = torch.empty_like(ybar)
    w, wb = _ws("scan", op, ybar, n, 0, ws)
    _check("adc_scan_vjp", lib().adc_scan_vjp(OPS[op], _dt(ybar), n, _ptr(x), _ptr(y), _ptr(ybar), _ptr(xbar),
                                               int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return xbar


# ------------------------------------------------------- reduce_by_index ----
def hist_fwd(op, m, keys, vals, hist0=None, hist=None, saved=None, ws=None, stream=None):
    """Returns (hist, saved)."""
    n = keys.shape[0]
    d = ARITY[op]
    if hist is None:
        hist = torch.empty((m, d) if d > 1 else (m,), dtype=vals.dtype, device=vals.device)
    if saved is None:
        saved = torch.empty(max(saved_bytes("hist", op, vals.dtype, n, m), 16), dtype=torch.uint8,
                            device=vals.device)
    w, wb = _ws("hist", op, vals, n, m, ws)
    _check("adc_hist_fwd", lib().adc_hist_fwd(OPS[op], _dt(vals), n, int(m), _ptr(keys), _ptr(vals), _ptr(hist0),
                                               _ptr(hist), _ptr(saved), _ptr(w), wb, _stream(stream)))
    return hist, saved


def hist_primal(op, m, keys, vals, hist0=None, hist=None, ws=None, stream=None):
    """The original, un-lifted primal (no residuals): adc_hist_fwd with saved = NULL."""
    n = keys.shape[0]
    d = ARITY[op]
    if hist is None:
        hist = torch.empty((m, d) if d > 1 else (m,), dtype=vals.dtype, device=vals.device)
    w, wb = _ws("hist", op, vals, n, m, ws)
    _check("adc_hist_fwd", lib().adc_hist_fwd(OPS[op], _dt(vals), n, int(m), _ptr(keys), _ptr(vals), _ptr(hist0),
                                               _ptr(hist), None, _ptr(w), wb, _stream(stream)))
    return hist


def hist_vjp(op, m, keys, vals, hist0, hist, saved, histbar, valsbar=None, hist0bar=None, want_hist0bar=False,
             accumulate=False, ws=None, stream=None):
    """Returns (valsbar, hist0bar or None)."""
    n = keys.shape[0]
    if valsbar is None:
        valsbar = torch.empty_like(vals)
    if hist0bar is None and want_hist0bar:
        hist0bar = torch.empty_like(histbar)
    w, wb = _ws("hist", op, histbar, n, m, ws)
    _check("adc_hist_vjp", lib().adc_hist_vjp(OPS[op], _dt(histbar), n, int(m), _ptr(keys), _ptr(vals), _ptr(hist0),
                                               _ptr(hist), _ptr(saved), _ptr(histbar), _ptr(valsbar), _ptr(hist0bar),
                                               int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return valsbar, hist0bar


# -------------------------------------------------------------- controls ----
def check_device_error(ws, stream=None):
    w = ws.buf if isinstance(ws, Workspace) else ws
    return int(lib().adc_check_device_error(_ptr(w), w.numel(), _stream(stream)))


def set_spin_limit(iterations):
    lib().adc_set_spin_limit(int(iterations))


def debug_set_stall_tile(tile):
    lib().adc_debug_set_stall_tile(int(tile))


def debug_set_sel_vjp_form(form):
    """min/max reduce-by-index vjp: 0 automatic, 1 gather pass, 2 zero-fill + scatter."""
    lib().adc_debug_set_sel_vjp_form(int(form))


def debug_force_hist_strategy(strategy):
    """-1 automatic; 0 per-warp, 1 per-block, 3 per-thread shared-memory tables, 2 global atomics,
    4 partition by bin range, and for lifted fp32 min/max 5 split, 6 cluster, 7 two passes,
    8 block pairs (see adc_debug_force_hist_strategy)."""
    lib().adc_debug_force_hist_strategy(int(strategy))


def debug_set_scan_engine(engine):
    """0 automatic, 1 per-tile look-back only, 2 range-partitioned wherever it applies, 3 TMA-staged
    ranges, 4 TMA-staged tiles, 5 ranges with 16 bytes per thread per tile, 6 the bulk-staged matrix
    segment forms (see adc_debug_set_scan_engine)."""
    lib().adc_debug_set_scan_engine(int(engine))


def debug_set_scan_range_tiles(tiles):
    """Tiles per range of the range-partitioned scan engine; 0 lets the library choose."""
    lib().adc_debug_set_scan_range_tiles(int(tiles))


def debug_set_batched_items(items):
    """Elements per thread and step of the batched histogram launch (1, 4 or 8)."""
    lib().adc_debug_set_batched_items(int(items))


def debug_set_scan_prefetch(on):
    """1: each range of the range-partitioned scan engine is prefetched into L2 when its block starts."""
    lib().adc_debug_set_scan_prefetch(int(bool(on)))


# ------------------------------------------------- vectorised operators ----
# reduce / scan / reduce_by_index with the elementwise operator map2 (op) over
# rows of d elements (Irwim / Iswim rewrites: transpose + per-column scalar
# kernels, all in libadcomb).  x is [n][d].


def transpose(x, out=None, stream=None):
    """[rows][cols] -> [cols][rows]."""
    rows, cols = x.shape
    if out is None:
        out = torch.empty((cols, rows), dtype=x.dtype, device=x.device)
    _check("adc_transpose", lib().adc_transpose(_dt(x), rows, cols, _ptr(x), _ptr(out), _stream(stream)))
    return out


def _vws(kind, op, x, n, m, d, ws):
    need = int(lib().adc_vworkspace_bytes(KIND[kind], OPS[op], _dt(x), int(n), int(m), int(d)))
    w = (ws or default_workspace(x.device)).get(need, x.device)
    return w, w.numel()


def vsaved_bytes(kind, op, dtype, n, m, d):
    return int(lib().adc_vsaved_bytes(KIND[kind], OPS[op], DTYPES[dtype], int(n), int(m), int(d)))


def vreduce_fwd(op, x, y=None, saved=None, ws=None, stream=None):
    n, d = x.shape
    if y is None:
        y = torch.empty(d, dtype=x.dtype, device=x.device)
    if saved is None:
        saved = torch.empty(max(vsaved_bytes("reduce", op, x.dtype, n, 0, d), 16), dtype=torch.uint8,
                            device=x.device)
    w, wb = _vws("reduce", op, x, n, 0, d, ws)
    _check("adc_vreduce_fwd", lib().adc_vreduce_fwd(OPS[op], _dt(x), n, d, _ptr(x), _ptr(y), _ptr(saved), _ptr(w), wb,
                                                     _stream(stream)))
    return y, saved


def vreduce_vjp(op, x, y, saved, ybar, xbar=None, accumulate=False, ws=None, stream=None):
    n, d = x.shape
    if xbar is None:
        xbar = torch.empty_like(x)
    w, wb = _vws("reduce", op, x, n, 0, d, ws)
    _check("adc_vreduce_vjp", lib().adc_vreduce_vjp(OPS[op], _dt(x), n, d, _ptr(x), _ptr(y), _ptr(saved),
                                                     _ptr(ybar), _ptr(xbar), int(bool(accumulate)), _ptr(w), wb,
                                                     _stream(stream)))
    return xbar


def vscan_fwd(op, x, y=None, ws=None, stream=None):
    n, d = x.shape
    if y is None:
        y = torch.empty_like(x)
    w, wb = _vws("scan", op, x, n, 0, d, ws)
    _check("adc_vscan_fwd", lib().adc_vscan_fwd(OPS[op], _dt(x), n, d, _ptr(x), _ptr(y), _ptr(w), wb,
                                                 _stream(stream)))
    return y


def vscan_vjp(op, x, y, ybar, xbar=None, accumulate=False, ws=None, stream=None):
    n, d = ybar.shape
    if xbar is None:
        xbar = torch.empty_like(ybar)
    w, wb = _vws("scan", op, ybar, n, 0, d, ws)
    _check("adc_vscan_vjp", lib().adc_vscan_vjp(OPS[op], _dt(ybar), n, d, _ptr(x), _ptr(y), _ptr(ybar), _ptr(xbar),
                                                 int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return xbar


def vhist_fwd(op, m, keys, vals, hist0=None, hist=None, saved=None, primal=False, ws=None, stream=None):
    """Returns (hist [m][d], saved); primal=True runs the original program (no residuals)."""
    n, d = vals.shape
    if hist is None:
        hist = torch.empty((m, d), dtype=vals.dtype, device=vals.device)
    if saved is None and not primal:
        saved = torch.empty(max(vsaved_bytes("hist", op, vals.dtype, n, m, d), 16), dtype=torch.uint8,
                            device=vals.device)
    w, wb = _vws("hist", op, vals, n, m, d, ws)
    _check("adc_vhist_fwd", lib().adc_vhist_fwd(OPS[op], _dt(vals), n, int(m), d, _ptr(keys), _ptr(vals), _ptr(hist0),
                                                 _ptr(hist), None if primal else _ptr(saved), _ptr(w), wb,
                                                 _stream(stream)))
    return hist, saved


def vhist_vjp(op, m, keys, vals, hist0, hist, saved, histbar, valsbar=None, hist0bar=None, want_hist0bar=False,
              accumulate=False, ws=None, stream=None):
    n, d = vals.shape
    if valsbar is None:
        valsbar = torch.empty_like(vals)
    if hist0bar is None and want_hist0bar:
        hist0bar = torch.empty_like(histbar)
    w, wb = _vws("hist", op, vals, n, m, d, ws)
    _check("adc_vhist_vjp", lib().adc_vhist_vjp(OPS[op], _dt(vals), n, int(m), d, _ptr(keys), _ptr(vals), _ptr(hist0),
                                                 _ptr(hist), _ptr(saved), _ptr(histbar), _ptr(valsbar),
                                                 _ptr(hist0bar), int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return valsbar, hist0bar


def status_string(code):
    return lib().adc_status_string(int(code)).decode()


def version():
    return lib().adc_version().decode()


# ------------------------------------------------------------- tuple scans --
# Tuple operators whose blocks combine independently (block-diagonal
# Jacobians): ``ops`` names each block's operator; rows are [n][D] with the
# blocks side by side (D = sum of arities), or, for the *_blocks calls, one
# [n][a_c] tensor per block.

def _codes(ops):
    arr = (ctypes.c_int32 * len(ops))(*[OPS[o] for o in ops])
    return arr, ctypes.cast(arr, ctypes.c_void_p)


def _ptrs(ts):
    """Host array of device pointers (None entries stay NULL), or NULL for None."""
    if ts is None:
        return None, None
    arr = (ctypes.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])
    return arr, ctypes.cast(arr, ctypes.c_void_p)


def tscan_workspace_bytes(ops, dtype, n, rows=True):
    keep, codes = _codes(ops)
    return int(lib().adc_tscan_workspace_bytes(len(ops), codes, DTYPES[dtype], int(n), int(bool(rows))))


def _tws(ops, t, n, rows, ws):
    need = tscan_workspace_bytes(ops, t.dtype, n, rows)
    if need == 0:
        raise AdcError("adc_tscan_workspace_bytes", 1)
    w = (ws or default_workspace(t.device)).get(need, t.device)
    return w, w.numel()


def tscan_fwd(ops, x, y=None, ws=None, stream=None):
    n = x.shape[0]
    if y is None:
        y = torch.empty_like(x)
    w, wb = _tws(ops, x, n, True, ws)
    keep, codes = _codes(ops)
    _check("adc_tscan_fwd", lib().adc_tscan_fwd(len(ops), codes, _dt(x), n, _ptr(x), _ptr(y), _ptr(w), wb,
                                                 _stream(stream)))
    return y


def tscan_vjp(ops, x, y, ybar, xbar=None, accumulate=False, ws=None, stream=None):
    n = ybar.shape[0]
    if xbar is None:
        xbar = torch.empty_like(ybar)
    w, wb = _tws(ops, ybar, n, True, ws)
    keep, codes = _codes(ops)
    _check("adc_tscan_vjp", lib().adc_tscan_vjp(len(ops), codes, _dt(ybar), n, _ptr(x), _ptr(y), _ptr(ybar),
                                                 _ptr(xbar), int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return xbar


def tscan_fwd_blocks(ops, xs, ys=None, ws=None, stream=None):
    n = xs[0].shape[0]
    if ys is None:
        ys = [torch.empty_like(x) for x in xs]
    w, wb = _tws(ops, xs[0], n, False, ws)
    keep, codes = _codes(ops)
    kx, px = _ptrs(xs)
    ky, py = _ptrs(ys)
    _check("adc_tscan_fwd_blocks", lib().adc_tscan_fwd_blocks(len(ops), codes, _dt(xs[0]), n, px, py, _ptr(w), wb,
                                                               _stream(stream)))
    return ys


def tscan_vjp_blocks(ops, xs, ys, ybars, xbars=None, accumulate=False, ws=None, stream=None):
    n = ybars[0].shape[0]
    if xbars is None:
        xbars = [torch.empty_like(t) for t in ybars]
    w, wb = _tws(ops, ybars[0], n, False, ws)
    keep, codes = _codes(ops)
    kx, px = _ptrs(xs)
    ky, py = _ptrs(ys)
    kb, pb = _ptrs(ybars)
    kxb, pxb = _ptrs(xbars)
    _check("adc_tscan_vjp_blocks", lib().adc_tscan_vjp_blocks(len(ops), codes, _dt(ybars[0]), n, px, py, pb, pxb,
                                                               int(bool(accumulate)), _ptr(w), wb, _stream(stream)))
    return xbars
