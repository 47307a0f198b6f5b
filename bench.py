"""Benchmark: reverse-mode AD of reduce_by_index with the specialised operators.

Workload (the paper's reduce-by-index evaluation shape, Sec. 6.1.2, with the
histogram sizes 31 / 401 / 50,000 plus 10M): fp32, n = 50M values with
uniform int32 bin indices, for every m in {31, 401, 50000, 10M} and every
operator in {* (values ~U(0.5,1.5), 1% exact zeros), min, max (values on 1024
exact levels)}.  One step = the differentiated program for all twelve
(operator, m) instances: the lifted forward pass (histogram + residuals) and
the vjp w.r.t. the values given a histogram adjoint ~N(0,1).

Metric: vjp elements/s = (12 x 50M) / step time, whole job over all GPUs
(replicas: every rank runs the full workload on its own GPU).  Also reported:
the HBM roofline fraction of the dominant kernel, the AD overhead
(differentiated / original primal time) per instance, an end-to-end number
through the C ABI with host buffers, and the fp64 oracle timed on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 50_000_000
BINS = (31, 401, 50_000, 10_000_000)
OPS = ("mul", "min", "max")
METRIC = "vjp elements/s & % HBM roofline; AD overhead = vjp time / primal time"
WORKLOAD = ("reduce_by_index specialisations fp32: n=50M uniform int32 bins, m in {31,401,50000,10M}, "
            "ops * (1% zeros), min, max (1024 levels); lifted forward + vjp per (op, m)")
# DRAM bytes (read + write) per call measured by ncu on n = 20M, m = 10M and
# scaled to n by the parts that grow with n, plus the m-sized outputs (the
# partitioned-histogram kernels' capture): the roofline's `traffic` for the
# dominant call, when it is one of these.
TRAFFIC_PER_ELEM = {("fwd", "mul", 10_000_000): (22.1, 120e6), ("fwd", "min", 10_000_000): (29.7, 80e6),
                    ("fwd", "max", 10_000_000): (29.7, 80e6)}


def launches(phase, op, m, n):
    """Our kernels launched by one call (csrc/hist.cu, hist_part.cu): the lifted
    forward is init + table kernel + finaliser (for * with per-thread or
    per-warp tables: table kernel + cross-block reduce, which finalises; for
    min/max in two passes: value rows + row reduce + index pass + decode), or,
    partitioned by bin range (m >= 2^18), count + count scan + scatter +
    per-bucket tables (which also finalise);
    the * vjp is coefficient tables + gather; the min/max vjp is a zero-fill +
    scatter, or, when bins are sparse (8m > n), a bitmap of the selected
    elements + one streaming pass."""
    if phase == "fwd":
        if m >= (1 << 18):
            return 4
        # * with per-thread or per-warp tables: table kernel + cross-block reduce
        if op == "mul":
            return 2 if m * 8 * 8 <= 48 * 1024 else 3
        # min/max whose packed table exceeds a block but whose values fit:
        # value rows + row reduce + index pass + decode
        return 4 if m * 8 > 200 * 1024 and m * 4 <= 200 * 1024 else 3
    return 2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N, help="elements per instance (default: the full 50M)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-families", action="store_true")
    p.add_argument("--kernels", action="store_true",
                   help="instead of the bench line: per-kernel achieved bandwidth at full sizes (markdown)")
    p.add_argument("--only", default=None,
                   help="with --kernels: run only the families whose label contains this text, "
                        "e.g. 'scan add float32', 'reduce mul', 'hist add m=1000'")
    p.add_argument("--prefetch", action="store_true",
                   help="with --kernels: time the range-partitioned scans with L2 prefetch of each range")
    p.add_argument("--range-tiles", default="0",
                   help="with --kernels: comma list of tiles per range for the range-partitioned scan (0 = default)")
    return p.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_inputs(n, seed=1):
    """Keys per m and values per operator (numpy, host), drawn by the seeded generators."""
    from paper_2310_03568_gb300 import synth
    g = synth.rng(seed)
    keys = {m: synth.keys_uniform(g, n, m) for m in BINS}
    vals = {op: synth.hist_spec_values(g, op, n, 1, np.float32) for op in OPS}
    hbar = {m: synth.normal(g, m) for m in BINS}
    return keys, vals, hbar


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- our arm ----
def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2310_03568_gb300 import adcomb
    from paper_2310_03568_gb300.build import build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    adcomb.lib()
    n = args.n
    keys_h, vals_h, hbar_h = make_inputs(n)
    dev = torch.device("cuda", local)
    keys = {m: torch.from_numpy(keys_h[m]).to(dev) for m in BINS}
    vals = {op: torch.from_numpy(vals_h[op]).to(dev) for op in OPS}
    hbar = {m: torch.from_numpy(hbar_h[m]).to(dev) for m in BINS}
    hist = {m: torch.empty(m, dtype=torch.float32, device=dev) for m in BINS}
    saved = {(op, m): torch.empty(max(adcomb.saved_bytes("hist", op, torch.float32, n, m), 16), dtype=torch.uint8,
                                  device=dev) for op in OPS for m in BINS}
    vbar = torch.empty(n, dtype=torch.float32, device=dev)
    wsb = max(adcomb.workspace_bytes("hist", op, torch.float32, n, m) for op in OPS for m in BINS)
    ws = adcomb.Workspace()
    ws.get(wsb, dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        for m in BINS:
            for op in OPS:
                if ev is not None:
                    ev[(op, m, "fwd")][0].record(stream)
                adcomb.hist_fwd(op, m, keys[m], vals[op], None, hist[m], saved[(op, m)], ws=ws)
                if ev is not None:
                    ev[(op, m, "fwd")][1].record(stream)
                adcomb.hist_vjp(op, m, keys[m], vals[op], None, hist[m], saved[(op, m)], hbar[m], valsbar=vbar,
                                ws=ws)
                if ev is not None:
                    ev[(op, m, "vjp")][1].record(stream)

    def primal():
        """The original (non-lifted) primal of every instance, for the AD overhead."""
        out = {}
        for m in BINS:
            for op in OPS:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                adcomb.hist_primal(op, m, keys[m], vals[op], None, hist[m], ws=ws)
                b.record(stream)
                out[(op, m)] = (a, b)
        return out

    def new_events():
        ev = {}
        for op in OPS:
            for m in BINS:
                f0, f1, v1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                ev[(op, m, "fwd")] = (f0, f1)
                ev[(op, m, "vjp")] = (f1, v1)  # the vjp starts where the fwd ends
        return ev

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    events = [new_events() for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(events[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    per = {k: [ev[k][0].elapsed_time(ev[k][1]) for ev in events] for k in events[0]}
    step_ms = t0.elapsed_time(t1) / args.steps
    elapsed = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    step_ms = float(elapsed.item())

    # primal (original program) timing for the AD overhead
    for _ in range(2):
        primal()
    torch.cuda.synchronize()
    prim_ms = {k: [] for k in per if k[2] == "fwd"}
    for _ in range(3):
        ev = primal()
        torch.cuda.synchronize()
        for (op, m), (a, b) in ev.items():
            prim_ms[(op, m, "fwd")].append(a.elapsed_time(b))
    ad = {f"{op}/{m}": round((statistics.mean(per[(op, m, "fwd")]) + statistics.mean(per[(op, m, "vjp")])) /
                             statistics.mean(prim_ms[(op, m, "fwd")]), 2) for op in OPS for m in BINS}

    # dominant call and its roofline: algorithmic bytes per launch
    call_ms = {k: statistics.mean(v) for k, v in per.items()}
    dom = max(call_ms, key=call_ms.get)
    op_d, m_d, ph_d = dom
    alg = {"fwd": 8 * n, "vjp": {"mul": 12 * n, "min": 4 * n, "max": 4 * n}[op_d]}[ph_d]
    peak, peak_kind = read_peaks()
    achieved = alg / (call_ms[dom] * 1e-3) / 1e9
    tr = TRAFFIC_PER_ELEM.get((ph_d, op_d, m_d))
    traffic = tr[0] * n + tr[1] if tr else None
    total_elems = world * len(BINS) * len(OPS) * n
    value = total_elems / (step_ms * 1e-3)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, n, keys_h, vals_h, hbar_h, hist, saved, ws, dev, world)
    n_launch = args.steps * sum(launches("fwd", op, m, n) + launches("vjp", op, m, n) for op in OPS for m in BINS)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n, keys_h, vals_h, hbar_h)

    del keys, vals, vbar
    torch.cuda.empty_cache()
    families = None
    if not args.no_families:
        families = run_families(dev, peak)
    batched = None
    if not args.no_batched:
        batched = run_batched(dev, peak)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded numpy, shapes of the paper's Sec. 6.1.2)",
            "config": {"workload": WORKLOAD, "n": n, "bins": list(BINS), "ops": list(OPS),
                       "instances_per_step": len(BINS) * len(OPS), "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (200 MB keys + 200 MB values per instance); no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"hist_{ph_d} {op_d} m={m_d}", "algorithmic_bytes": alg,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "ad_overhead": ad,
            "per_call_ms": {f"{op}/{m}/{ph}": round(v, 4) for (op, m, ph), v in call_ms.items()},
            "primal_ms": {f"{op}/{m}": round(statistics.mean(v), 4) for (op, m, _), v in prim_ms.items()},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch, "clocks": clk,
            "batched": batched, "families": families,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(args, n, keys_h, vals_h, hbar_h, hist, saved, ws, dev, world):
    """Same metric through the C-ABI calls with host buffers: every step copies
    its inputs (4 key arrays, 3 value arrays, 4 histogram adjoints) from pinned
    host memory and reads every instance's results (histogram and value
    adjoint) back, inside the timed region.  Copies run on their own streams and
    overlap the compute of other instances (events order each buffer's use)."""
    import torch

    from paper_2310_03568_gb300 import adcomb
    pin_k = {m: torch.from_numpy(keys_h[m]).pin_memory() for m in BINS}
    pin_v = {op: torch.from_numpy(vals_h[op]).pin_memory() for op in OPS}
    pin_h = {m: torch.from_numpy(hbar_h[m]).pin_memory() for m in BINS}
    inst = [(op, m) for m in BINS for op in OPS]
    out_h = {i: torch.empty(i[1], dtype=torch.float32).pin_memory() for i in inst}
    out_v = {i: torch.empty(n, dtype=torch.float32).pin_memory() for i in inst}
    k_d = {m: torch.empty(n, dtype=torch.int32, device=dev) for m in BINS}
    v_d = {op: torch.empty(n, dtype=torch.float32, device=dev) for op in OPS}
    hb_d = {m: torch.empty(m, dtype=torch.float32, device=dev) for m in BINS}
    hist_d = {i: torch.empty(i[1], dtype=torch.float32, device=dev) for i in inst}
    vb_d = {i: torch.empty(n, dtype=torch.float32, device=dev) for i in inst}
    comp = torch.cuda.current_stream()
    # several copy streams per direction, so that the copy engines work in parallel
    s_ins = [torch.cuda.Stream(device=dev) for _ in range(2)]
    s_outs = [torch.cuda.Stream(device=dev) for _ in range(3)]
    ev = lambda: torch.cuda.Event()  # noqa: E731
    prev_done = None                      # compute of the previous step (inputs free)
    prev_read = {i: None for i in inst}   # D2H of the previous step (outputs free)
    h2d = d2h = 0

    def step():
        nonlocal prev_done, h2d, d2h
        h2d = d2h = 0
        ready_k, ready_v = {}, {}
        order = [("k", BINS[0])] + [("v", op) for op in OPS] + [("k", m) for m in BINS[1:]]
        for j, (kind, key) in enumerate(order):
            s_in = s_ins[j % len(s_ins)]
            with torch.cuda.stream(s_in):
                if prev_done is not None:
                    s_in.wait_event(prev_done)
                if kind == "k":
                    k_d[key].copy_(pin_k[key], non_blocking=True)
                    hb_d[key].copy_(pin_h[key], non_blocking=True)
                    h2d += 4 * n + 4 * key
                    ready_k[key] = ev()
                    ready_k[key].record(s_in)
                else:
                    v_d[key].copy_(pin_v[key], non_blocking=True)
                    h2d += 4 * n
                    ready_v[key] = ev()
                    ready_v[key].record(s_in)
        done = {}
        for op, m in inst:
            comp.wait_event(ready_k[m])
            comp.wait_event(ready_v[op])
            if prev_read[(op, m)] is not None:
                comp.wait_event(prev_read[(op, m)])
            adcomb.hist_fwd(op, m, k_d[m], v_d[op], None, hist_d[(op, m)], saved[(op, m)], ws=ws)
            adcomb.hist_vjp(op, m, k_d[m], v_d[op], None, hist_d[(op, m)], saved[(op, m)], hb_d[m],
                            valsbar=vb_d[(op, m)], ws=ws)
            done[(op, m)] = ev()
            done[(op, m)].record(comp)
        prev_done = done[inst[-1]]
        for j, i in enumerate(inst):
            s_out = s_outs[j % len(s_outs)]
            with torch.cuda.stream(s_out):
                s_out.wait_event(done[i])
                out_h[i].copy_(hist_d[i], non_blocking=True)
                out_v[i].copy_(vb_d[i], non_blocking=True)
                d2h += 4 * i[1] + 4 * n
                prev_read[i] = ev()
                prev_read[i].record(s_out)

    step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    for _ in range(steps):
        step()
    for so in s_outs:
        comp.wait_stream(so)
    b.record(comp)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"value": world * len(BINS) * len(OPS) * n / (ms * 1e-3), "unit": "elements/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms,
            "overlap": "H2D on 2 and D2H on 3 streams of their own, ordered by events against the compute stream"}


def run_batched(dev, peak, seed=4):
    """4096 hist -> +-scan -> sum instances (n_i, m_i log-uniform): forward + vjp
    as two replayed CUDA graphs of the batched entry points (work-item size and
    table size chosen by the autotuner), against the same work through the
    single-instance entry points (several launches per instance), both as one
    replayed CUDA graph of all instances (every buffer allocated before capture)
    and as eager launches from Python.  Reported beside the bench line; not
    part of its step."""
    import torch

    from paper_2310_03568_gb300 import autotune
    from paper_2310_03568_gb300 import batched as B
    from paper_2310_03568_gb300 import synth
    w = synth.batched(seed=seed)
    desc, keys, vals = B.layout(w)
    p = B.BatchedHistScan(desc, keys, vals, device=dev)
    tuned = autotune.tune_batched(p)
    p.graphs = None
    for _ in range(3):
        p.replay_forward()
        p.replay_backward()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record()
    for _ in range(reps):
        p.replay_forward()
        p.replay_backward()
    b.record()
    torch.cuda.synchronize()
    ms_batched = a.elapsed_time(b) / reps
    vb = p.valsbar.clone()
    # per-instance launches captured in one graph: the launches alone
    pig = B.PerInstanceGraph(desc, p.keys, p.vals, device=dev)
    pig.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(3):
        pig.replay()
    b.record()
    torch.cuda.synchronize()
    ms_graph = a.elapsed_time(b) / 3
    same_graph = bool(torch.equal(vb, pig.valsbar))
    # per-instance launches from Python (dispatch included)
    B.per_instance_loss(desc, p.keys, p.vals)  # warm-up
    torch.cuda.synchronize()
    a.record()
    loss_pi, vb_pi = B.per_instance_loss(desc, p.keys, p.vals)
    b.record()
    torch.cuda.synchronize()
    ms_pi = a.elapsed_time(b)
    same = bool(torch.equal(vb, vb_pi))
    total = int(desc["n"].sum())
    bins = int(desc["m"].sum())
    add = desc["op"] == B.OPCODE["add"]
    # forward: keys + values in, hist / scan / index words out; vjp: keys in (+ only), valsbar out
    alg = int(8 * total + (8 * desc["n"][add].sum() + 4 * desc["n"][~add].sum()) + 16 * bins)
    gbs = alg / (ms_batched * 1e-3) / 1e9
    return {"instances": int(len(desc)), "values": total, "bins": bins,
            "batched_graph_ms": ms_batched, "per_instance_graph_ms": ms_graph, "per_instance_ms": ms_pi,
            "speedup_vs_graph": ms_graph / ms_batched, "speedup": ms_pi / ms_batched,
            "batched_values_per_s": total / (ms_batched * 1e-3),
            "algorithmic_bytes": alg, "achieved_gbs": gbs, "frac": gbs / peak,
            "tuned": {"chunk": tuned["chunk"], "smem_bins": tuned["smem_bins"], "items": tuned["items"]},
            "gradients_bit_identical": same and same_graph,
            "loss_batched": float(p.loss.item()), "loss_per_instance": float(loss_pi.item()),
            "loss_per_instance_graph": float(pig.loss.item())}


# ------------------------------------------------------- other workloads ----
# Algorithmic bytes per element of each call (minimal reads + writes, fp32
# unless named): the roofline numerators of the families below.
SCAN_BYTES = {"add": (2, 2), "mul": (2, 4), "lin": (4, 8), "mm2": (8, 16)}  # scalars per element: fwd, vjp
REDUCE_BYTES = {"add": (1, 1), "mul": (1, 2), "min": (1, 1), "mm2": (4, 8), "lin": (2, 4)}


def cpu_info():
    """Host core count and CPU model (x86 'model name', else lscpu, else the Arm part ids)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for line in txt.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
        if model is None:
            r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
            for line in r.stdout.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        if model is None:
            ids = [ln.split(":", 1)[1].strip() for ln in txt.splitlines()
                   if ln.startswith(("CPU implementer", "CPU part"))][:2]
            model = "implementer/part " + "/".join(ids) if ids else None
    except Exception:
        pass
    return {"host_cpus": os.cpu_count(), "cpu_model": model}


class L2Flush:
    """Writes a buffer larger than L2 (256 MB) before each timed call."""

    def __init__(self, dev):
        import torch
        self.buf = torch.empty(64 << 20, dtype=torch.float32, device=dev)

    def __call__(self):
        self.buf.zero_()


def time_calls(fn, flush, reps=10, warm=3):
    """Mean device time of fn() in ms: CUDA events on the launching stream
    around each call, an L2 flush before each (outside the events)."""
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warm):
        flush()
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush()
        a.record(s)
        fn()
        b.record(s)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def family_entry(n, fwd_ms, vjp_ms, fwd_bytes, vjp_bytes, paper_bytes, peak, primal_ms=None):
    """One workload's numbers: device times, algorithmic GB/s and fraction of
    the measured copy bandwidth per call, AD overhead (fwd + vjp) / primal, and
    the paper's normalised GB/s (its Nbytes of the primal / primal time)."""
    primal_ms = fwd_ms if primal_ms is None else primal_ms
    gbs = lambda b, ms: b / (ms * 1e-3) / 1e9  # noqa: E731
    return {"n": n, "fwd_ms": round(fwd_ms, 5), "vjp_ms": round(vjp_ms, 5),
            "fwd_gbs": round(gbs(fwd_bytes, fwd_ms), 1), "vjp_gbs": round(gbs(vjp_bytes, vjp_ms), 1),
            "fwd_frac": round(gbs(fwd_bytes, fwd_ms) / peak, 3), "vjp_frac": round(gbs(vjp_bytes, vjp_ms) / peak, 3),
            "fwd_bytes": fwd_bytes, "vjp_bytes": vjp_bytes,
            "vjp_elements_per_s": n / (vjp_ms * 1e-3),
            "ad_overhead": round((fwd_ms + vjp_ms) / primal_ms, 2),
            "paper_gbs": round(gbs(paper_bytes, primal_ms), 1)}


def run_families(dev, peak):
    """The workloads beside the headline, each timed on its own at full size:
    the small reduce-by-index workload (n = 1e5), the scans (n = 1e8 fp32,
    1e7 fp64), the specialised reduces at 1e8, the 2x2 matrix scan and
    reduce at 1e7, the 3x3 (1e7) and 5x5 (4e6) matrix scans, linFnComp
    reduce-by-index at 1e7 / m = 1000, and tuple-scan rows of 16 sumOfProd
    blocks at 1e7.  Inputs are
    seeded and drawn on the device with the workloads' distributions."""
    import torch

    from paper_2310_03568_gb300 import adcomb
    flush = L2Flush(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    ws = adcomb.Workspace()
    out = {}

    def U(shape, lo, hi, dtype=torch.float32):
        return torch.rand(shape, generator=gen, device=dev, dtype=dtype) * (hi - lo) + lo

    def Nrm(shape, dtype=torch.float32):
        return torch.randn(shape, generator=gen, device=dev, dtype=dtype)

    def scan_x(op, n, dtype):
        if op == "add":
            return U(n, -1, 1, dtype)
        if op == "mul":
            x = U(n, 0.9, 1.1, dtype)
            x[torch.rand(n, generator=gen, device=dev) < 0.001] = 0
            return x
        if op == "lin":
            return torch.stack([Nrm(n, dtype), U(n, 0.95, 1.05, dtype)], 1).contiguous()
        return (U((n, 4), -1, 1, dtype) / np.sqrt(2.0)).contiguous()

    # small reduce-by-index workload: n = 1e5, m = 1000, hist0; + reduce and + scan of the same values
    n, m = 100_000, 1000
    k = torch.randint(0, m, (n,), generator=gen, device=dev, dtype=torch.int32)
    v, h0, hb = U(n, -1, 1), U(m, -1, 1), Nrm(m)
    h, sv = adcomb.hist_fwd("add", m, k, v, h0, ws=ws)
    vb, h0b = torch.empty_like(v), torch.empty_like(h0)
    f = time_calls(lambda: adcomb.hist_fwd("add", m, k, v, h0, h, sv, ws=ws), flush)
    b = time_calls(lambda: adcomb.hist_vjp("add", m, k, v, h0, h, sv, hb, valsbar=vb, hist0bar=h0b,
                                           want_hist0bar=True, ws=ws), flush)
    small = {"hist_add_m1000": family_entry(n, f, b, 8 * n + 8 * m, 8 * n + 8 * m, 12 * n + 8 * n, peak)}
    y, rs = adcomb.reduce_fwd("add", v, ws=ws)
    yb1, xb = Nrm(1), torch.empty_like(v)
    f = time_calls(lambda: adcomb.reduce_fwd("add", v, y, rs, ws=ws), flush)
    b = time_calls(lambda: adcomb.reduce_vjp("add", v, y, rs, yb1, xbar=xb, ws=ws), flush)
    small["reduce_add"] = family_entry(n, f, b, 4 * n, 4 * n, 4 * n, peak)
    ys, ybs = adcomb.scan_fwd("add", v, ws=ws), Nrm(n)
    f = time_calls(lambda: adcomb.scan_fwd("add", v, ys, ws=ws), flush)
    b = time_calls(lambda: adcomb.scan_vjp("add", v, ys, ybs, xbar=xb, ws=ws), flush)
    small["scan_add"] = family_entry(n, f, b, 8 * n, 8 * n, 8 * n, peak)
    out["small_n1e5_m1000"] = small
    del k, v, h0, hb, vb, xb

    # scans: n = 1e8 fp32 and 1e7 fp64 (+, * with 0.1% zeros, linFnComp)
    for dtype, n, label in [(torch.float32, 100_000_000, "scan_f32_n1e8"), (torch.float64, 10_000_000, "scan_f64_n1e7")]:
        es = 4 if dtype == torch.float32 else 8
        fam = {}
        for op in ("add", "mul", "lin"):
            x = scan_x(op, n, dtype)
            y = adcomb.scan_fwd(op, x, ws=ws)
            yb, xb = torch.randn(x.shape, generator=gen, device=dev, dtype=dtype), torch.empty_like(x)
            f = time_calls(lambda: adcomb.scan_fwd(op, x, y, ws=ws), flush)
            b = time_calls(lambda: adcomb.scan_vjp(op, x, y, yb, xbar=xb, ws=ws), flush)
            sf, sb = SCAN_BYTES[op]
            fam[op] = family_entry(n, f, b, sf * es * n, sb * es * n, sf * es * n, peak)
            del x, y, yb, xb
        out[label] = fam
    # specialised reduces at n = 1e8 fp32
    n = 100_000_000
    fam = {}
    for op in ("add", "mul", "min"):
        x = U(n, -1, 1) if op != "mul" else U(n, 0.999, 1.001)
        y, rs = adcomb.reduce_fwd(op, x, ws=ws)
        yb, xb = torch.ones_like(y), torch.empty_like(x)
        f = time_calls(lambda: adcomb.reduce_fwd(op, x, y, rs, ws=ws), flush)
        b = time_calls(lambda: adcomb.reduce_vjp(op, x, y, rs, yb, xbar=xb, ws=ws), flush)
        rf, rb = REDUCE_BYTES[op]
        fam[op] = family_entry(n, f, b, 4 * rf * n, 4 * rb * n, 4 * n, peak)
        del x, xb
    out["reduce_f32_n1e8"] = fam
    # general paths: 2x2 matrix scan and reduce at 1e7, linFnComp reduce-by-index at 1e7 / m = 1000
    n = 10_000_000
    x = scan_x("mm2", n, torch.float32)
    gen_fam = {}
    y = adcomb.scan_fwd("mm2", x, ws=ws)
    yb, xb = Nrm(x.shape), torch.empty_like(x)
    f = time_calls(lambda: adcomb.scan_fwd("mm2", x, y, ws=ws), flush)
    b = time_calls(lambda: adcomb.scan_vjp("mm2", x, y, yb, xbar=xb, ws=ws), flush)
    gen_fam["scan_mm2"] = family_entry(n, f, b, 32 * n, 64 * n, 32 * n, peak)
    yr, rs = adcomb.reduce_fwd("mm2", x, ws=ws)
    ybr = Nrm(4)
    f = time_calls(lambda: adcomb.reduce_fwd("mm2", x, yr, rs, ws=ws), flush)
    b = time_calls(lambda: adcomb.reduce_vjp("mm2", x, yr, rs, ybr, xbar=xb, ws=ws), flush)
    gen_fam["reduce_mm2"] = family_entry(n, f, b, 16 * n, 32 * n, 16 * n, peak)
    del x, y, yb, xb
    # q x q matrix scans (Sec. 5.3.4's q > 2 case): 3x3 at 1e7, 5x5 at 4e6, entries U(-1, 1) / sqrt(q)
    for op, nq, q in (("mm3", 10_000_000, 3), ("mm5", 4_000_000, 5)):
        x = (U((nq, q * q), -1, 1) / np.sqrt(q)).contiguous()
        y = adcomb.scan_fwd(op, x, ws=ws)
        yb, xb = Nrm(x.shape), torch.empty_like(x)
        f = time_calls(lambda: adcomb.scan_fwd(op, x, y, ws=ws), flush)
        b = time_calls(lambda: adcomb.scan_vjp(op, x, y, yb, xbar=xb, ws=ws), flush)
        es = 4 * q * q  # bytes per matrix
        gen_fam[f"scan_{op}"] = family_entry(nq, f, b, 2 * es * nq, 4 * es * nq, 2 * es * nq, peak)
        del x, y, yb, xb
    m = 1000
    k = torch.randint(0, m, (n,), generator=gen, device=dev, dtype=torch.int32)
    v = scan_x("lin", n, torch.float32)
    h, sv = adcomb.hist_fwd("lin", m, k, v, ws=ws)
    hb, vb = Nrm((m, 2)), torch.empty_like(v)
    f = time_calls(lambda: adcomb.hist_fwd("lin", m, k, v, None, h, sv, ws=ws), flush)
    b = time_calls(lambda: adcomb.hist_vjp("lin", m, k, v, None, h, sv, hb, valsbar=vb, ws=ws), flush)
    # keys + (b, c) in; the vjp reads keys and values and writes the adjoints
    gen_fam["hist_lin_m1000"] = family_entry(n, f, b, 12 * n, 20 * n, 3 * 8 * n + 8 * n, peak)
    out["general_n1e7"] = gen_fam
    del k, v, vb
    # tuple scan rows of 16 equal sumOfProd blocks (D = 32 values a row, U(-1, 1)), scanned in place;
    # a failure here is recorded in the line instead of ending the run
    try:
        n = 10_000_000
        ops16 = ("sop",) * 16
        x = U((n, 32), -1, 1).contiguous()
        y = adcomb.tscan_fwd(ops16, x, ws=ws)
        yb, xb = Nrm(tuple(x.shape)), torch.empty_like(x)
        f = time_calls(lambda: adcomb.tscan_fwd(ops16, x, y, ws=ws), flush)
        b = time_calls(lambda: adcomb.tscan_vjp(ops16, x, y, yb, xbar=xb, ws=ws), flush)
        out["tuple_rows_n1e7"] = {"sop_x16": family_entry(n, f, b, 2 * 32 * 4 * n, 4 * 32 * 4 * n,
                                                          2 * 32 * 4 * n, peak)}
        del x, y, yb, xb
    except Exception as e:  # noqa: BLE001
        out["tuple_rows_n1e7"] = {"error": f"{type(e).__name__}: {e}"}
    torch.cuda.empty_cache()
    out["timing"] = ("CUDA events on the launching stream around each call, mean of 10 after 3 warm-ups, "
                     "a 256 MB L2 flush before each call; frac of the measured copy bandwidth")
    return out


# --------------------------------------------------------- kernel rooflines ----
def run_kernels(args):
    """Achieved bandwidth of every kernel family at full size (CUDA events, inputs
    larger than L2, 3 warm-ups, mean of 10).  Prints a markdown table."""
    import torch

    from paper_2310_03568_gb300 import adcomb, synth
    from paper_2310_03568_gb300.build import build
    build()
    peak, kind = read_peaks()
    dev = torch.device("cuda", 0)
    g = np.random.default_rng(0)
    rows = []

    def timeit(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def row(name, n, nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        rows.append((name, n, nbytes, ms, gbs, gbs / peak))

    def want(label):
        return args.only is None or args.only in label

    rts = [int(t) for t in args.range_tiles.split(",")]

    ws = adcomb.Workspace()
    for op, dt, n in [("add", np.float32, 100_000_000), ("mul", np.float32, 100_000_000),
                      ("lin", np.float32, 100_000_000), ("mm2", np.float32, 10_000_000),
                      ("add", np.float64, 10_000_000), ("mul", np.float64, 10_000_000),
                      ("lin", np.float64, 10_000_000), ("mm3", np.float32, 10_000_000),
                      ("mm5", np.float32, 4_000_000), ("sop", np.float32, 100_000_000)]:
        if not want(f"scan {op} {np.dtype(dt).name}"):
            continue
        x = torch.from_numpy(synth.scan_values(g, op, n, dt)).to(dev)
        es = x.element_size() * (x.numel() // n)
        y = adcomb.scan_fwd(op, x, ws=ws)
        yb = torch.randn_like(x)
        xb = torch.empty_like(x)
        vb_bytes = (2 if op == "add" else 4) * n * es
        variants = ([(2, rt, "ranges" if rt == 0 else f"ranges rt={rt}") for rt in rts] +
                    [(3, rt, "staged" if rt == 0 else f"staged rt={rt}") for rt in rts] +
                    [(5, rt, "ranges16" if rt == 0 else f"ranges16 rt={rt}") for rt in rts] +
                    [(1, 0, "per-tile"), (4, 0, "tma")])
        if op in ("mm3", "mm5"):  # bulk-staged segment forms (automatic) and the register forms
            variants = [(0, 0, "bulk-staged"), (2, 0, "ranges"), (1, 0, "per-tile")]
        if args.prefetch:
            variants = [(2, rt, f"ranges rt={rt} prefetch") for rt in rts]
        adcomb.debug_set_scan_prefetch(1 if args.prefetch else 0)
        for eng, rt, label in variants:
            adcomb.debug_set_scan_engine(eng)
            adcomb.debug_set_scan_range_tiles(rt)
            row(f"scan {op} fwd {np.dtype(dt).name} [{label}]", n, 2 * n * es,
                timeit(lambda: adcomb.scan_fwd(op, x, y, ws=ws)))
            row(f"scan {op} vjp {np.dtype(dt).name} [{label}]", n, vb_bytes,
                timeit(lambda: adcomb.scan_vjp(op, x, y, yb, xbar=xb, ws=ws)))
        adcomb.debug_set_scan_engine(0)
        adcomb.debug_set_scan_range_tiles(0)
        adcomb.debug_set_scan_prefetch(0)
        del x, y, yb, xb
    # min / max scans (the general arity-1 rule), values on 1024 levels
    for op in ("min", "max"):
        if not want(f"scan {op} float32"):
            continue
        n = 100_000_000
        x = torch.from_numpy(((g.integers(0, 1024, n) - 512) / 64.0).astype(np.float32)).to(dev)
        y = adcomb.scan_fwd(op, x, ws=ws)
        yb = torch.randn_like(x)
        xb = torch.empty_like(x)
        for eng, label in [(0, "auto"), (4, "tma"), (5, "ranges16")]:
            adcomb.debug_set_scan_engine(eng)
            row(f"scan {op} fwd float32 [{label}]", n, 8 * n, timeit(lambda: adcomb.scan_fwd(op, x, y, ws=ws)))
            # the vjp reads y and ybar (the selections come from y), writes xbar
            row(f"scan {op} vjp float32 [{label}]", n, 12 * n,
                timeit(lambda: adcomb.scan_vjp(op, x, y, yb, xbar=xb, ws=ws)))
        adcomb.debug_set_scan_engine(0)
        del x, y, yb, xb
    # vectorised operators (Irwim / Iswim): the paper's [n][d] shapes, d = 16 (reduce, scan), 10 (hist)
    for fam, op, n, d in [("vscan", "add", 10_000_000, 16), ("vscan", "mul", 10_000_000, 16),
                          ("vscan", "max", 10_000_000, 16),
                          ("vreduce", "add", 10_000_000, 16), ("vreduce", "min", 10_000_000, 16),
                          ("vhist", "add", 10_000_000, 10), ("vhist", "max", 10_000_000, 10)]:
        if not want(f"{fam} {op}"):
            continue
        if op == "mul":
            x = (torch.rand(n, d, device=dev) * 0.2 + 0.9).contiguous()
        elif op in ("min", "max"):
            x = ((torch.randint(0, 1024, (n, d), device=dev) - 512) / 64.0).float().contiguous()
        else:
            x = (torch.rand(n, d, device=dev) * 2 - 1).contiguous()
        s = n * d * 4
        if fam == "vscan":
            y = adcomb.vscan_fwd(op, x, ws=ws)
            yb = torch.randn_like(x)
            xb = torch.empty_like(x)
            row(f"vscan {op} fwd d={d}", n, 2 * s, timeit(lambda: adcomb.vscan_fwd(op, x, y, ws=ws)))
            # vjp reads: ybar (+), x, y, ybar (*), y, ybar (min / max); writes xbar
            row(f"vscan {op} vjp d={d}", n, (2 if op == "add" else 3 if op in ("min", "max") else 4) * s,
                timeit(lambda: adcomb.vscan_vjp(op, x, y, yb, xbar=xb, ws=ws)))
        elif fam == "vreduce":
            y, sv = adcomb.vreduce_fwd(op, x, ws=ws)
            yb = torch.randn(d, device=dev)
            xb = torch.empty_like(x)
            row(f"vreduce {op} fwd d={d}", n, s, timeit(lambda: adcomb.vreduce_fwd(op, x, y, sv, ws=ws)))
            row(f"vreduce {op} vjp d={d}", n, s, timeit(lambda: adcomb.vreduce_vjp(op, x, y, sv, yb, xbar=xb, ws=ws)))
        else:
            m = 1000
            k = torch.randint(0, m, (n,), dtype=torch.int32, device=dev)
            h, sv = adcomb.vhist_fwd(op, m, k, x, ws=ws)
            hb = torch.randn(m, d, device=dev)
            vb = torch.empty_like(x)
            row(f"vhist {op} fwd d={d} m={m}", n, 4 * n + s, timeit(lambda: adcomb.vhist_fwd(op, m, k, x, None, h, sv, ws=ws)))
            row(f"vhist {op} vjp d={d} m={m}", n, 4 * n + s,
                timeit(lambda: adcomb.vhist_vjp(op, m, k, x, None, h, sv, hb, valsbar=vb, ws=ws)))
        del x
    # tuple scans (block-diagonal Jacobians): rows [n][D] and one array per block
    for ops, n in [(("sop",) * 16, 10_000_000), (("add", "mul", "lin", "sop", "mm2", "min"), 20_000_000)]:
        name = f"{ops[0]}x{len(ops)}" if len(set(ops)) == 1 else "-".join(ops)
        if not want(f"tscan {name}"):
            continue
        blocks = [torch.from_numpy(synth.scan_values(g, op, n) if op not in ("add", "min") else
                                   synth.uniform(g, n, -1, 1)).to(dev).reshape(n, -1) for op in ops]
        x = torch.cat(blocks, 1).contiguous()
        D = x.shape[1]
        y = adcomb.tscan_fwd(ops, x, ws=ws)
        yb = torch.randn_like(x)
        xb = torch.empty_like(x)
        row(f"tscan {name} fwd rows", n, 2 * n * D * 4, timeit(lambda: adcomb.tscan_fwd(ops, x, y, ws=ws)))
        row(f"tscan {name} vjp rows", n, 4 * n * D * 4, timeit(lambda: adcomb.tscan_vjp(ops, x, y, yb, xbar=xb, ws=ws)))
        xs = [b.contiguous().squeeze(1) if b.shape[1] == 1 else b.contiguous() for b in blocks]
        ys = adcomb.tscan_fwd_blocks(ops, xs, ws=ws)
        ybs = [torch.randn_like(t) for t in xs]
        xbs = [torch.empty_like(t) for t in xs]
        row(f"tscan {name} fwd blocks", n, 2 * n * D * 4, timeit(lambda: adcomb.tscan_fwd_blocks(ops, xs, ys, ws=ws)))
        row(f"tscan {name} vjp blocks", n, 4 * n * D * 4,
            timeit(lambda: adcomb.tscan_vjp_blocks(ops, xs, ys, ybs, xbars=xbs, ws=ws)))
        del x, y, yb, xb, xs, ys, ybs, xbs, blocks
    for op, n in [("add", 100_000_000), ("mul", 100_000_000), ("min", 100_000_000), ("mm2", 10_000_000),
                  ("sop", 50_000_000)]:
        if not want(f"reduce {op}"):
            continue
        if op == "sop":
            x = torch.from_numpy(synth.uniform(g, (n, 2), -1, 1)).to(dev)
        else:
            x = torch.from_numpy(synth.scan_values(g, "mm2_orth" if op == "mm2" else "add", n)).to(dev)
        if op == "mul":
            x = x * 0.05 + 1.0
        es = x.element_size() * (x.numel() // n)
        y, saved = adcomb.reduce_fwd(op, x, ws=ws)
        yb = torch.ones_like(y)
        xb = torch.empty_like(x)
        row(f"reduce {op} fwd", n, n * es, timeit(lambda: adcomb.reduce_fwd(op, x, y, saved, ws=ws)))
        vjp_bytes = {"add": n * es, "min": n * es, "mul": 2 * n * es, "mm2": 2 * n * es, "sop": 2 * n * es}[op]
        row(f"reduce {op} vjp", n, vjp_bytes, timeit(lambda: adcomb.reduce_vjp(op, x, y, saved, yb, xbar=xb, ws=ws)))
        del x, xb
    for op, n, m in [("add", 100_000_000, 1000), ("add", 50_000_000, 10_000_000), ("lin", 10_000_000, 1000),
                     ("sop", 50_000_000, 1000), ("sop", 50_000_000, 1_000_000)]:
        if not want(f"hist {op} m={m}"):
            continue
        k = torch.randint(0, m, (n,), dtype=torch.int32, device=dev)
        if op == "sop":
            v = torch.from_numpy(synth.uniform(g, (n, 2), -1, 1)).to(dev)
        else:
            v = torch.from_numpy(synth.scan_values(g, op, n)).to(dev)
        es = v.element_size() * (v.numel() // n)
        h, saved = adcomb.hist_fwd(op, m, k, v, ws=ws)
        hb = torch.randn_like(h)
        vb = torch.empty_like(v)
        row(f"hist {op} fwd m={m}", n, n * (4 + es), timeit(lambda: adcomb.hist_fwd(op, m, k, v, None, h, saved, ws=ws)))
        # vjp: keys in, valsbar out, and the values too where the rule reads them
        row(f"hist {op} vjp m={m}", n, n * (4 + (2 if op in ("lin", "sop") else 1) * es),
            timeit(lambda: adcomb.hist_vjp(op, m, k, v, None, h, saved, hb, valsbar=vb, ws=ws)))
        del k, v, vb
    # the benchmark's reduce-by-index instances (n = 50M fp32): lifted forward, and the
    # min/max vjp in both of its forms
    if args.only is not None and args.only.startswith("bench"):
        NB = args.n
        keys_h, vals_h, hbar_h = make_inputs(NB)
        for m in BINS:
            k = torch.from_numpy(keys_h[m]).to(dev)
            hb = torch.from_numpy(hbar_h[m]).to(dev)
            for op in OPS:
                if not want(f"bench {op} m={m}"):
                    continue
                v = torch.from_numpy(vals_h[op]).to(dev)
                h, saved = adcomb.hist_fwd(op, m, k, v, ws=ws)
                vb = torch.empty_like(v)
                row(f"bench {op} m={m} fwd", NB, 8 * NB,
                    timeit(lambda: adcomb.hist_fwd(op, m, k, v, None, h, saved, ws=ws)))
                if op != "mul" and 200 * 1024 < m * 8 <= 8 * 200 * 1024:
                    for strat, label in [(2, "global"), (6, "cluster"), (7, "two passes"), (8, "pairs")]:
                        adcomb.debug_force_hist_strategy(strat)
                        ws.get(adcomb.workspace_bytes("hist", op, torch.float32, NB, m), dev)
                        row(f"bench {op} m={m} fwd [{label}]", NB, 8 * NB,
                            timeit(lambda: adcomb.hist_fwd(op, m, k, v, None, h, saved, ws=ws)))
                    adcomb.debug_force_hist_strategy(-1)
                forms = [(1, "gather"), (2, "scatter"), (3, "bitmap")] if op != "mul" else [(0, "")]
                for f, label in forms:
                    adcomb.debug_set_sel_vjp_form(f)
                    row(f"bench {op} m={m} vjp {label}".strip(), NB, (12 if op == "mul" else 4) * NB,
                        timeit(lambda: adcomb.hist_vjp(op, m, k, v, None, h, saved, hb, valsbar=vb, ws=ws)))
                adcomb.debug_set_sel_vjp_form(0)
                del v, vb
            del k, hb
    print(f"| kernel | n | algorithmic bytes | ms | GB/s | frac of {kind} {peak:.0f} GB/s |")
    print("|---|---|---|---|---|---|")
    for name, n, nb, ms, gbs, fr in rows:
        print(f"| {name} | {n:.3g} | {nb / 1e6:.0f} MB | {ms:.4f} | {gbs:.0f} | {fr:.2f} |")


# ------------------------------------------------------------ cpu oracle ----
SAMPLE = 4_000_000


def cpu_baseline(n, keys_h, vals_h, hbar_h, sample=SAMPLE):
    """The fp64 oracle, as it stands, on the first `sample` elements of every
    instance (single-threaded by definition: sequential semantics)."""
    import oracle
    s = min(sample, n)
    t = time.perf_counter()
    for m in BINS:
        k = keys_h[m][:s]
        for op in OPS:
            v = vals_h[op][:s]
            oracle.hist_fwd(op, m, k, v)
            oracle.hist_vjp(op, m, k, v, hbar_h[m])
    dt = time.perf_counter() - t
    return {"value": len(BINS) * len(OPS) * s / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"first {s} of the {n} elements of each of the 12 (op, m) instances; forward + vjp, fp64",
            "seconds": dt, **cpu_info()}


def run_reference(args, world, rank):
    """The reference arm: the fp64 oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    n = args.n
    s = min(SAMPLE // 2, n)
    keys_h, vals_h, hbar_h = make_inputs(s)
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(s, keys_h, vals_h, hbar_h, sample=min(s, 200_000))
    times = []
    for _ in range(args.steps):
        r = cpu_baseline(s, keys_h, vals_h, hbar_h, sample=s)
        times.append(r["seconds"])
    ms = 1e3 * statistics.mean(times)
    value = len(BINS) * len(OPS) * s / (ms * 1e-3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "sample_per_instance": s},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": f"{s} elements of each of the 12 (op, m) instances per step; forward + vjp",
                         **cpu_info()},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.kernels:
        run_kernels(args)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
