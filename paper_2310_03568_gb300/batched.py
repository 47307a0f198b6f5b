"""Batched hist -> +-scan -> sum over many instances (adc_batched_* in libadcomb).

``BatchedHistScan`` holds one problem (instance table, work items, device
buffers) and runs its forward and vjp either as plain launches or replayed
from CUDA graphs captured once.  ``batched_loss`` is the autograd entry point.
``per_instance_loss`` is the baseline that issues the single-instance entry
points (reduce_by_index, scan, reduce and their vjps) once per instance.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import adcomb

INSTANCE = np.dtype([("n", "<i8"), ("m", "<i8"), ("val_off", "<i8"), ("bin_off", "<i8"), ("op", "<i4"),
                     ("pad", "<i4")])
WORK = np.dtype([("inst", "<i4"), ("pad", "<i4"), ("start", "<i8"), ("len", "<i8")])
OPCODE = {"add": adcomb.OPS["add"], "max": adcomb.OPS["max"]}

_sig_done = False


def _sigs():
    global _sig_done
    if _sig_done:
        return
    L = adcomb.lib()
    i32, i64, sz, p = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    L.adc_batched_plan.argtypes = [p, i32, i64, p, i64]
    L.adc_batched_plan.restype = i64
    L.adc_batched_workspace_bytes.argtypes = [i32, i64]
    L.adc_batched_workspace_bytes.restype = sz
    L.adc_batched_hist_scan_fwd.argtypes = [p, i32, p, i64, i64, p, p, p, p, p, p, p, i32, p, sz, p]
    L.adc_batched_hist_scan_fwd.restype = i32
    L.adc_batched_hist_scan_vjp.argtypes = [p, i32, p, i64, i64, p, p, p, p, p, p, sz, p]
    L.adc_batched_hist_scan_vjp.restype = i32
    _sig_done = True


def _aligned_offsets(sizes, align=4):
    padded = (np.asarray(sizes, dtype=np.int64) + align - 1) // align * align
    return np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64)


def make_table(ns, ms, ops):
    """Host instance table: values and bins concatenated in instance order, each
    instance starting on a 16-byte boundary (so that single-instance slices are
    valid arguments for the regular entry points)."""
    count = len(ns)
    desc = np.zeros(count, dtype=INSTANCE)
    desc["n"] = ns
    desc["m"] = ms
    desc["val_off"] = _aligned_offsets(ns)
    desc["bin_off"] = _aligned_offsets(ms)
    desc["op"] = [OPCODE[o] if isinstance(o, str) else (OPCODE["add"] if o == 0 else OPCODE["max"]) for o in ops]
    return desc


def layout(w):
    """From a synth.batched() workload (packed arrays) to (desc, keys, vals) in the
    padded layout; padding keys are out of range and never read."""
    desc = make_table(w["ns"], w["ms"], w["ops"])
    total = int((desc["val_off"] + desc["n"]).max())
    keys = np.full(total, -1, dtype=np.int32)
    vals = np.zeros(total, dtype=np.float32)
    src = np.concatenate([[0], np.cumsum(w["ns"])]).astype(np.int64)
    for i in range(len(desc)):
        o, n = int(desc["val_off"][i]), int(desc["n"][i])
        keys[o:o + n] = w["keys"][src[i]:src[i + 1]]
        vals[o:o + n] = w["vals"][src[i]:src[i + 1]]
    return desc, keys, vals


def plan(desc, chunk):
    _sigs()
    L = adcomb.lib()
    count = len(desc)
    k = L.adc_batched_plan(desc.ctypes.data, count, int(chunk), None, 0)
    if k < 0:
        raise ValueError("invalid instance table")
    items = np.zeros(max(k, 1), dtype=WORK)
    L.adc_batched_plan(desc.ctypes.data, count, int(chunk), items.ctypes.data, k)
    return items[:k]


class BatchedHistScan:
    """One batched problem resident on the device."""

    def __init__(self, desc, keys, vals, chunk=1 << 16, smem_bins=0, device="cuda"):
        _sigs()
        self.desc_h = desc
        self.count = len(desc)
        self.total_bins = int((desc["bin_off"] + desc["m"]).max())
        self.total_vals = int((desc["val_off"] + desc["n"]).max())
        self.chunk, self.smem_bins = int(chunk), int(smem_bins)
        dev = torch.device(device)
        self.dev = dev
        self.desc = torch.from_numpy(desc.view(np.uint8).copy()).to(dev)
        self.set_plan(chunk)
        self.keys = keys if isinstance(keys, torch.Tensor) else torch.from_numpy(keys).to(dev)
        self.vals = vals if isinstance(vals, torch.Tensor) else torch.from_numpy(vals).to(dev)
        f32 = dict(dtype=torch.float32, device=dev)
        self.hist = torch.empty(self.total_bins, **f32)
        self.scan = torch.empty(self.total_bins, **f32)
        self.is_ = torch.empty(self.total_bins, dtype=torch.int32, device=dev)
        self.loss_parts = torch.empty(self.count, **f32)
        self.loss = torch.empty(1, **f32)
        self.loss_bar = torch.ones(1, **f32)
        self.histbar = torch.empty(self.total_bins, **f32)
        self.valsbar = torch.zeros(self.total_vals, **f32)  # padding positions stay 0
        wsb = adcomb.lib().adc_batched_workspace_bytes(self.count, self.total_bins)
        self.ws = torch.empty(max(int(wsb), 256), dtype=torch.uint8, device=dev)
        self.graphs = None

    def set_plan(self, chunk):
        self.chunk = int(chunk)
        items = plan(self.desc_h, chunk)
        self.n_items = len(items)
        self.items = torch.from_numpy(items.view(np.uint8).copy()).to(self.dev)
        self.graphs = None

    def forward(self, stream=None):
        L = adcomb.lib()
        st = L.adc_batched_hist_scan_fwd(
            self.desc.data_ptr(), self.count, self.items.data_ptr(), self.n_items, self.total_bins,
            self.keys.data_ptr(), self.vals.data_ptr(), self.hist.data_ptr(), self.scan.data_ptr(),
            self.is_.data_ptr(), self.loss_parts.data_ptr(), self.loss.data_ptr(), self.smem_bins,
            self.ws.data_ptr(), self.ws.numel(), adcomb._stream(stream))
        adcomb._check("adc_batched_hist_scan_fwd", st)
        return self.loss

    def backward(self, stream=None):
        L = adcomb.lib()
        st = L.adc_batched_hist_scan_vjp(
            self.desc.data_ptr(), self.count, self.items.data_ptr(), self.n_items, self.total_bins,
            self.keys.data_ptr(), self.is_.data_ptr(), self.loss_bar.data_ptr(), self.histbar.data_ptr(),
            self.valsbar.data_ptr(), self.ws.data_ptr(), self.ws.numel(), adcomb._stream(stream))
        adcomb._check("adc_batched_hist_scan_vjp", st)
        return self.valsbar

    def capture(self):
        """Capture the forward and the vjp as two CUDA graphs (static buffers)."""
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up outside capture (sets kernel attributes)
            self.forward(s)
            self.backward(s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            self.forward()
        with torch.cuda.graph(gb):
            self.backward()
        self.graphs = (gf, gb)

    def replay_forward(self):
        if self.graphs is None:
            self.capture()
        self.graphs[0].replay()
        return self.loss

    def replay_backward(self):
        if self.graphs is None:
            self.capture()
        self.graphs[1].replay()
        return self.valsbar


class _BatchedFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, problem, use_graph):
        if vals.data_ptr() != problem.vals.data_ptr():
            problem.vals.copy_(vals)
        loss = problem.replay_forward() if use_graph else problem.forward()
        ctx.problem, ctx.use_graph = problem, use_graph
        return loss.clone().reshape(())

    @staticmethod
    def backward(ctx, lbar):
        p = ctx.problem
        p.loss_bar.copy_(lbar.reshape(1))
        vb = p.replay_backward() if ctx.use_graph else p.backward()
        return vb.clone(), None, None


def batched_loss(vals, problem, use_graph=True):
    """loss = sum over instances of sum_j scan(+)(reduce_by_index(...))_j, differentiable in vals."""
    return _BatchedFn.apply(vals, problem, use_graph)


# ------------------------------------------------------- per-instance baseline --
def per_instance_loss(desc, keys, vals, want_grad=True, loss_bar=1.0):
    """The same loss and gradient through the single-instance entry points,
    several launches per instance (the baseline the batched path is compared with)."""
    dev = keys.device
    count = len(desc)
    mmax = int(desc["m"].max())
    zeros = torch.zeros(mmax, dtype=torch.float32, device=dev)
    ws = adcomb.Workspace()
    losses = torch.empty(count, dtype=torch.float32, device=dev)
    saved_all = []
    for i in range(count):
        d = desc[i]
        n, m, vo = int(d["n"]), int(d["m"]), int(d["val_off"])
        op = "add" if d["op"] == OPCODE["add"] else "max"
        k, v = keys[vo:vo + n], vals[vo:vo + n]
        h, saved = adcomb.hist_fwd(op, m, k, v, zeros[:m], ws=ws)
        sc = adcomb.scan_fwd("add", h, ws=ws)
        y, _ = adcomb.reduce_fwd("add", sc, y=losses[i:i + 1], ws=ws)
        saved_all.append((op, m, k, v, h, saved, sc))
    loss = losses.sum()
    if not want_grad:
        return loss, None
    vbar = torch.zeros_like(vals)  # padding positions stay 0, as in the batched path
    lb = torch.full((1,), float(loss_bar), dtype=torch.float32, device=dev)
    for i, (op, m, k, v, h, saved, sc) in enumerate(saved_all):
        vo = int(desc[i]["val_off"])
        ybar = adcomb.reduce_vjp("add", sc, None, None, lb, ws=ws)
        hbar = adcomb.scan_vjp("add", None, None, ybar, ws=ws)
        adcomb.hist_vjp(op, m, k, v, zeros[:m], h, saved, hbar, valsbar=vbar[vo:vo + k.shape[0]], ws=ws)
    return loss, vbar


class PerInstanceGraph:
    """The per-instance baseline with every buffer allocated up front and the
    whole loop -- per instance reduce_by_index, +-scan and +-reduce forward,
    then their vjps, several launches per instance -- captured once as a CUDA
    graph.  Replaying it measures the per-instance launches themselves on the
    GPU, not Python or ctypes dispatch."""

    def __init__(self, desc, keys, vals, device="cuda"):
        dev = torch.device(device)
        self.desc, self.keys, self.vals, self.dev = desc, keys, vals, dev
        count = len(desc)
        f32 = dict(dtype=torch.float32, device=dev)
        total_bins = int((desc["bin_off"] + desc["m"]).max())
        self.h = torch.empty(total_bins, **f32)
        self.sc = torch.empty(total_bins, **f32)
        self.ybar = torch.empty(total_bins, **f32)
        self.hbar = torch.empty(total_bins, **f32)
        self.zeros = torch.zeros(int(desc["m"].max()), **f32)
        self.losses = torch.empty(count, **f32)
        self.loss = torch.empty(1, **f32)
        self.lb = torch.ones(1, **f32)
        self.rsaved = torch.empty(256, dtype=torch.uint8, device=dev)  # + reduce: no residuals
        self.valsbar = torch.zeros_like(vals)  # padding positions stay 0, as in the batched path
        ops = ["add" if d["op"] == OPCODE["add"] else "max" for d in desc]
        sb = [max(adcomb.saved_bytes("hist", op, torch.float32, int(d["n"]), int(d["m"])), 16)
              for op, d in zip(ops, desc)]
        soff = _aligned_offsets(sb, 256)
        self.saved = torch.empty(int(soff[-1] + sb[-1]), dtype=torch.uint8, device=dev)
        need = max(max(adcomb.workspace_bytes("hist", op, torch.float32, int(d["n"]), int(d["m"])),
                       adcomb.workspace_bytes("scan", "add", torch.float32, int(d["m"])),
                       adcomb.workspace_bytes("reduce", "add", torch.float32, int(d["m"])))
                   for op, d in zip(ops, desc))
        self.ws = adcomb.Workspace()
        self.ws.get(need, dev)
        self.inst = []
        for i, d in enumerate(desc):
            n, m, vo, bo = int(d["n"]), int(d["m"]), int(d["val_off"]), int(d["bin_off"])
            self.inst.append((ops[i], m, keys[vo:vo + n], vals[vo:vo + n], slice(bo, bo + m),
                              self.saved[int(soff[i]):int(soff[i]) + sb[i]], self.valsbar[vo:vo + n]))
        self.graph = None

    def forward(self):
        ws = self.ws
        for i, (op, m, k, v, b, sv, _) in enumerate(self.inst):
            adcomb.hist_fwd(op, m, k, v, self.zeros[:m], self.h[b], sv, ws=ws)
            adcomb.scan_fwd("add", self.h[b], self.sc[b], ws=ws)
            adcomb.reduce_fwd("add", self.sc[b], y=self.losses[i:i + 1], saved=self.rsaved, ws=ws)
        torch.sum(self.losses, dim=0, keepdim=True, out=self.loss)
        return self.loss

    def backward(self):
        ws = self.ws
        for op, m, k, v, b, sv, vb in self.inst:
            adcomb.reduce_vjp("add", self.sc[b], None, None, self.lb, xbar=self.ybar[b], ws=ws)
            adcomb.scan_vjp("add", None, None, self.ybar[b], xbar=self.hbar[b], ws=ws)
            adcomb.hist_vjp(op, m, k, v, self.zeros[:m], self.h[b], sv, self.hbar[b], valsbar=vb, ws=ws)
        return self.valsbar

    def capture(self):
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up outside capture (per-device caches, kernel attributes)
            self.forward()
            self.backward()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.forward()
            self.backward()
        self.graph = g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.loss, self.valsbar
