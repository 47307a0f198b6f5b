"""torch.autograd.Function wrappers over libadcomb.

Each Function's forward calls the library's *_fwd entry point and keeps only
what the paper's rule for that operator needs (Sec. 3-5); backward calls the
matching *_vjp entry point.  All compute runs in libadcomb's kernels.

Residual policy (``policy="save"`` or ``"recompute"``):
  reduce  +      : nothing (the adjoint is a broadcast, Sec. 3.2.1)
          min/max: the selected index only (Sec. 3.2.2)
          *      : x and (zero count, product of non-zeros) (Fig. 3)
          lin/mm2: x and the per-tile exclusive prefixes/suffixes (Fig. 2)
  scan    +      : nothing (reverse +-scan of ybar, Sec. 5.3.1)
          *, lin, mm2: x and y.  y is the forward's own output, so keeping it
                   costs no extra HBM traffic; "recompute" instead re-runs the
                   forward scan in backward and keeps only x (less memory, one
                   more pass).
  reduce_by_index +: keys; min/max: keys and is[m]; *: keys, values, (n0, p);
          lin    : m <= 2047: per (bin, input chunk) prefix and suffix tables
                   (about 16*m*n/4096 bytes; the chunk-local sort is redone in
                   backward anyway); larger m: the stable permutation with the
                   sorted keys and values (16 B/element).  "recompute" re-runs
                   the forward in backward instead.
"""
from __future__ import annotations

import torch

from . import adcomb

__all__ = ["reduce", "scan", "reduce_by_index", "ReduceFn", "ScanFn", "HistFn"]


def _flat(x, d):
    return x.contiguous() if d > 1 else x.contiguous().reshape(-1)


class ReduceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op, policy):
        d = adcomb.ARITY[op]
        x = _flat(x, d)
        y, saved = adcomb.reduce_fwd(op, x)
        ctx.op, ctx.n, ctx.d = op, x.shape[0], d
        if op == "add":
            ctx.save_for_backward()
        elif op in ("min", "max"):
            ctx.save_for_backward(saved)
        else:
            ctx.save_for_backward(x, y, saved)
        ctx.xshape, ctx.dtype, ctx.device = x.shape, x.dtype, x.device
        return y.reshape(()) if d == 1 else y

    @staticmethod
    def backward(ctx, ybar):
        op = ctx.op
        yb = ybar.contiguous().reshape(-1).to(ctx.dtype)
        if op in ("add", "min", "max"):
            # x is not read by these rules: the output buffer stands in for its shape
            saved = ctx.saved_tensors[0] if op != "add" else None
            xb = torch.empty(ctx.xshape, dtype=ctx.dtype, device=ctx.device)
            adcomb.reduce_vjp(op, xb, None, saved, yb, xbar=xb)
        else:
            x, y, saved = ctx.saved_tensors
            xb = adcomb.reduce_vjp(op, x, y, saved, yb)
        return xb, None, None


class ScanFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op, policy):
        d = adcomb.ARITY[op]
        x = _flat(x, d)
        y = adcomb.scan_fwd(op, x)
        ctx.op, ctx.policy = op, policy
        if op == "add":
            ctx.save_for_backward()
        elif policy == "recompute":
            ctx.save_for_backward(x)
        else:
            ctx.save_for_backward(x, y)
        ctx.yshape = y.shape
        return y

    @staticmethod
    def backward(ctx, ybar):
        op = ctx.op
        yb = ybar.contiguous()
        if op == "add":
            xb = adcomb.scan_vjp(op, None, None, yb)
        elif ctx.policy == "recompute":
            (x,) = ctx.saved_tensors
            y = adcomb.scan_fwd(op, x)
            xb = adcomb.scan_vjp(op, x, y, yb)
        else:
            x, y = ctx.saved_tensors
            xb = adcomb.scan_vjp(op, x, y, yb)
        return xb, None, None


class HistFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, hist0, keys, m, op, policy):
        d = adcomb.ARITY[op]
        vals = _flat(vals, d)
        keys = keys.contiguous()
        h0 = None if hist0 is None else _flat(hist0, d)
        hist, saved = adcomb.hist_fwd(op, m, keys, vals, h0)
        ctx.op, ctx.m, ctx.policy, ctx.has_h0 = op, m, policy, hist0 is not None
        if op == "lin" and policy == "recompute":
            saved = None  # re-sorted in backward
        ctx.save_for_backward(keys, vals, h0, hist, saved)
        return hist

    @staticmethod
    def backward(ctx, histbar):
        keys, vals, h0, hist, saved = ctx.saved_tensors
        op, m = ctx.op, ctx.m
        if saved is None:
            _, saved = adcomb.hist_fwd(op, m, keys, vals, h0)
        vb, h0b = adcomb.hist_vjp(op, m, keys, vals, h0, hist, saved, histbar.contiguous(),
                                  want_hist0bar=ctx.has_h0 and ctx.needs_input_grad[1])
        return vb, h0b, None, None, None, None


def reduce(x, op="add", policy="save"):
    """y = reduce (op) e x, differentiable in x."""
    return ReduceFn.apply(x, op, policy)


def scan(x, op="add", policy="save"):
    """Inclusive scan, differentiable in x."""
    return ScanFn.apply(x, op, policy)


def reduce_by_index(vals, keys, m, op="add", hist0=None, policy="save"):
    """hist = reduce_by_index hist0 (op) e keys vals, differentiable in vals and hist0."""
    return HistFn.apply(vals, hist0, keys, m, op, policy)
