"""Benchmark of the h-TN contraction hot path (one JSON line on stdout).

Default workload: the 100-qubit ring + chords h-TN (12 QTs, 28 gate cuts, 12
wire cuts, 64 observables, 2 GB of FP64 leaves), planned with a peak
intermediate <= 8 GB over 4^5 = 1024 wire-index slices and contracted in
full -- every timed step is one complete qtpu_htn_contract over all 1024
slices -- through the C ABI with BF16x3 tensor-core GEMMs.  Reported next to
it:
  * the same plan executed step by step with torch FP64 bmm (the plain FP64
    GPU path), timed on a fixed subset of slices and extrapolated;
  * the FP64 CPU oracle on the host cores (``cpu_baseline``), on the
    restricted output k in {0, 1} (2 of the 64 observables), which also gives
    the relative error of those two output entries;
  * the end-to-end form through ``qtpu_htn_contract_host`` (host buffers,
    the 2 GB upload and the result download inside the timed region);
  * the roofline of the dominant kernel class, from CUDA events recorded by
    the library around every launch (a separate pass after the timed one);
  * SM clocks sampled with nvidia-smi during the timed region.
``--workload mid`` selects the mid-size 60-qubit ring (8 QTs, 16 gate + 8
wire cuts), whose oracle runs in full.

``--impl reference`` times the FP64 CPU oracle alone (the reference arm) on
the same workload, metric and unit.  Multi-GPU (torchrun): every rank
contracts its own copy of the workload (independent replicas, weak scaling,
no collective on the data path); the time is the max over ranks.
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

METRIC = "h-TN contract TFLOP/s & %peak vs plain FP64 GPU path at rel err ≤1e-6"
WORKLOADS = {
    "mid": "mid-size 60-qubit ring h-TN: 8 QTs [k=64][6,6,4][6,6,4] FP64, 16 gate + 8 wire cuts, 32 tensors",
    "100q": "100-qubit ring+chords h-TN: 12 QTs, 28 gate + 12 wire cuts, k=64, 2 GB FP64 leaves, peak intermediate "
            "<= 8 GB, sliced over 4^5 = 1024 wire-index values (all slices contracted every step), "
            "order: best of 256 planner candidates by exact FLOPs",
    "100q-free": "100-qubit ring+chords h-TN: 12 QTs, 28 gate + 12 wire cuts, k=64, peak intermediate <= 8 GB, "
                 "slices chosen by the planner, order: best of 256 planner candidates by exact FLOPs",
    "gemm": "one pairwise step C[b,m,n] = sum_k A[b,m,k] B[b,k,n] of the given --shape (FP64 leaves)",
    "qpd": "QPD sampling + h-TN simplification (section 4.3) of the 100-qubit ring+chords h-TN (20 gate-cut "
           "groups: 12 ring edges with 1 gate cut, 8 chords with 2) for s_QPD draws per group, then planning and "
           "contraction of the sampled network",
    "knit": "naive circuit knitting (Eq. knitting: every global instance summed, FP64) against the h-TN "
            "contraction of the same network: rings of 3, 4, 5 subcircuits with 1 gate + 1 wire cut per edge, "
            "k = 8 observables",
    "qteval": "GPU QT evaluation (statevector, FP64) of a hardware-efficient-ansatz subcircuit (3 RY/RZ layers, "
              "2 CZ chains) with 2 gate cuts, 1 measured and 1 prepared wire (576 instances), 16 observables, "
              "at 12 and 15 qubits",
    "batch": "512 independent random h-TNs (ring / 2-D grid, 2-12 subcircuits, 2-20 cuts, k 1-64, FP32/FP64, "
             "QTs <= 2^22 entries, peak intermediate <= 2^23 entries) in one CUDA graph (small gather-only "
             "networks in one persistent kernel when they are >= 1/2 of the batch, graph branches otherwise)",
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "src": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "src": "fallback"}


def measured_traffic(workload: str, kclass: str):
    """DRAM bytes per launch of a kernel class of a workload from the committed
    ncu summary, or None if the kernel source changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = (d.get(workload) or {}).get(kclass)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != e["sha256_16"]:
        return None
    return e["bytes_per_launch"]


def gemm_tiles_used() -> str:
    t = os.path.join(ROOT, "paper_2410_15080_b300", "gemm_tiles_b300.txt")
    return "measured tile table gemm_tiles_b300.txt" if os.path.exists(t) else "padding rule (no tile table)"


def make_network(workload: str, shape: str = "8x1024x1024x1024", observables: int = 64):
    import synth
    if workload == "gemm":
        b, m, n, k = (int(x) for x in shape.split("x"))
        rng = np.random.default_rng(b + m + n + k)
        A = rng.uniform(-1, 1, (b, m, k))
        B = rng.uniform(-1, 1, (b, k, n))
        return synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2),
                         name=f"gemm{shape}"), {}
    if workload == "mid":
        return synth.ring_htn(), {}
    if workload == "100q":
        return synth.ring_chords_htn(k=observables), {"max_intermediate_bytes": 8 << 30, "n_slices": 1024,
                                                      "slice_dim": 4, "n_candidates": 256}
    if workload == "100q-free":
        return synth.ring_chords_htn(k=observables), {"max_intermediate_bytes": 8 << 30, "n_candidates": 256}
    raise SystemExit(f"unknown workload {workload}")


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.dev)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", bus, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- plain FP64 GPU path
def parse_plan(text: str):
    steps, final_sum = [], []
    for line in text.splitlines():
        f = line.split()
        if f[0] == "step":
            kv = dict(x.split("=") for x in f[6:])
            g = {k: ([] if v == "-" else [int(i) for i in v.split(",")]) for k, v in kv.items()
                 if k in ("batch", "m", "n", "k", "sa", "sb")}
            steps.append((int(f[2]), int(f[3]), g))
        elif f[0] == "final":
            v = f[2].split("=")[1]
            final_sum = [] if v == "-" else [int(i) for i in v.split(",")]
    return steps, final_sum


def fp64_torch_path(tensors, output, steps, final_sum, fixed=None):
    """The same pairwise plan with torch FP64 ops: permute + bmm per step.
    ``fixed`` maps sliced index ids to their values (one slice)."""
    import torch
    live = {}
    for t, (inds, x) in enumerate(tensors):
        inds = list(inds)
        if fixed:
            sel = tuple(fixed.get(i, slice(None)) for i in inds)
            x = x[sel]
            inds = [i for i in inds if i not in fixed]
        live[t] = (inds, x)
    nxt = len(tensors)
    for x, y, g in steps:
        if fixed:
            g = {kk: [i for i in v if i not in fixed] for kk, v in g.items()}
        ia, a = live.pop(x)
        ib, b = live.pop(y)
        if g["sa"]:
            a = a.sum(dim=[ia.index(i) for i in g["sa"]])
            ia = [i for i in ia if i not in g["sa"]]
        if g["sb"]:
            b = b.sum(dim=[ib.index(i) for i in g["sb"]])
            ib = [i for i in ib if i not in g["sb"]]
        da = dict(zip(ia, a.shape))
        db = dict(zip(ib, b.shape))
        nb = int(np.prod([da[i] for i in g["batch"]], dtype=np.int64))
        nm = int(np.prod([da[i] for i in g["m"]], dtype=np.int64))
        nn = int(np.prod([db[i] for i in g["n"]], dtype=np.int64))
        nk = int(np.prod([da[i] for i in g["k"]], dtype=np.int64))
        A3 = a.permute([ia.index(i) for i in g["batch"] + g["m"] + g["k"]]).reshape(nb, nm, nk)
        B3 = b.permute([ib.index(i) for i in g["batch"] + g["k"] + g["n"]]).reshape(nb, nk, nn)
        c = torch.bmm(A3, B3)
        shape = [da[i] for i in g["batch"] + g["m"]] + [db[i] for i in g["n"]]
        live[nxt] = (g["batch"] + g["m"] + g["n"], c.reshape(shape))
        nxt += 1
    (inds, x), = live.values()
    final_sum = [i for i in final_sum if not fixed or i not in fixed]
    if final_sum:
        x = x.sum(dim=[inds.index(i) for i in final_sum])
        inds = [i for i in inds if i not in final_sum]
    return x.permute([inds.index(i) for i in output]).reshape(-1) if output else x.reshape(1)


# ----------------------------------------------------------------- timing helpers
def timed_steps(fn, steps, flush):
    """Per-step CUDA-event timing on the current stream; L2 flushed between
    steps outside the timed events.  Returns the list of ms."""
    import torch
    ts = []
    for _ in range(steps):
        flush()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return ts


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count()


def oracle_seconds(net, budget_s: float):
    """Time the FP64 CPU oracle contracting the workload (full contractions
    repeated until the budget is used).  Returns (seconds per contraction,
    repetitions, threads)."""
    from oracle import planner, tn
    p = planner.make_plan(net.inds(), net.dims(), net.output)
    order = planner.order_of(p)
    reps, t0 = 0, time.perf_counter()
    while True:
        tn.contract_pairwise(net.pairs(), net.output, order)
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = (time.perf_counter() - t0) / reps
    return dt, reps, oracle_threads()


class RestrictedOracle:
    """The FP64 CPU oracle on a restricted output: the entries k = v of the
    observable index for v in ``values`` (each a full contraction of the
    network with k fixed, in the oracle planner's order for that network).
    ``flops`` counts the oracle plan's useful FLOPs for those entries."""

    def __init__(self, net, values=(0, 1)):
        from oracle import planner
        self.net, self.values = net, tuple(values)
        self.kid = net.output[0]
        inds1 = [tuple(i for i in t.inds if i != self.kid) for t in net.tensors]
        dims1 = {i: d for i, d in net.dims().items() if i != self.kid}
        self.plan = planner.make_plan(inds1, dims1, (), n_candidates=32)
        per = int(planner.plan_text(self.plan, inds1).split("flops_total=")[1].split()[0])
        self.flops = per * len(self.values)
        self.order = planner.order_of(self.plan)

    def run(self):
        from oracle import tn
        t0 = time.perf_counter()
        r = tn.contract_output_subset(self.net.pairs(), self.net.output, self.order, self.kid, list(self.values))
        return np.asarray(r).ravel(), time.perf_counter() - t0


def cpu_model():
    try:
        for l in open("/proc/cpuinfo"):
            if l.startswith("model name"):
                return l.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ----------------------------------------------------------------- arms
def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed on the host cores (rank 0
    only; other ranks exit without work)."""
    if rank != 0:
        return
    net, _ = make_network(args.workload, args.shape, args.observables)
    if args.workload.startswith("100q"):
        ro = RestrictedOracle(net)
        for _ in range(args.warmup if args.warmup <= 3 else 3):
            ro.run()
        ts = [ro.run()[1] for _ in range(args.steps)]
        flops = ro.flops
        sample = (f"each step: the exact FP64 oracle on the restricted output k in {{0, 1}} (2 of the 64 "
                  f"observables, {flops / 1e12:.3f} TFLOP of the oracle plan), numpy FP64 on {cpu_model()}")
    elif args.workload == "mid":
        from oracle import planner
        flops = int(planner.plan_text(planner.make_plan(net.inds(), net.dims(), net.output), net.inds())
                    .split("flops_total=")[1].split()[0])
        for _ in range(args.warmup):
            oracle_seconds(net, 0.0)
        ts = [oracle_seconds(net, 0.0)[0] for _ in range(args.steps)]
        sample = f"each step: one full contraction of the workload, numpy FP64 on {cpu_model()}"
    else:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle arm for the {args.workload} workload"}))
        return
    threads = oracle_threads()
    ms = 1e3 * statistics.mean(ts)
    val = flops / (ms * 1e-3) / 1e12
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "flops_per_step": flops, "l2": "n/a (host)"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args, rank, world):
    """512 uneven networks contracted by one qtpu_htn_contract_batch call (one
    CUDA graph) vs the same networks contracted one call at a time."""
    import torch
    import synth
    from paper_2410_15080_b300 import contract_batch, from_network
    from paper_2410_15080_b300.htn import QTPU_CT, QTPU_QT
    dev = torch.device("cuda", torch.cuda.current_device())
    nets = synth.random_batch(512, seed=0, max_qt_entries=1 << 22)
    hs, outs = [], []
    flops = 0.0
    nbytes = 0
    launches = 0
    for n in nets:
        ts = [(t.inds, torch.from_numpy(np.ascontiguousarray(t.data)).to(dev), QTPU_CT if t.kind == "CT" else QTPU_QT)
              for t in n.tensors]
        h = from_network(ts, n.output, prec=args.prec, max_intermediate_bytes=(1 << 23) * 8)
        st = h.plan_stats()
        flops += st["flops_total"]
        launches += st["launches_per_contract"]
        nbytes += n.nbytes()
        hs.append(h)
        outs.append(torch.empty(h.output_size(), dtype=torch.float64, device=dev))
    flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    flush = lambda: flush_buf.zero_()  # noqa: E731
    for _ in range(args.warmup):
        contract_batch(hs, outs)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    with ClockSampler(dev.index) as clk:
        ts = timed_steps(lambda: contract_batch(hs, outs), args.steps, flush)
    ms = statistics.mean(ts)
    from paper_2410_15080_b300 import batch_info
    info = batch_info(hs, outs)
    # the same graph with graph branches only, and with the persistent kernel
    # forced on for the small gather-only networks
    for _ in range(2):
        contract_batch(hs, outs, persistent=False)
    tg = timed_steps(lambda: contract_batch(hs, outs, persistent=False), max(3, min(args.steps, 10)), flush)
    ms_graph = statistics.mean(tg)
    for _ in range(2):
        contract_batch(hs, outs, persistent=True)
    tp = timed_steps(lambda: contract_batch(hs, outs, persistent=True), max(3, min(args.steps, 10)), flush)
    ms_pers = statistics.mean(tp)
    info_p = batch_info(hs, outs)
    contract_batch(hs, outs)
    torch.cuda.synchronize()
    # one call per network (each replays its own graph)
    def loop():
        for h, o in zip(hs, outs):
            h.contract(o)
    for _ in range(2):
        loop()
    tl = timed_steps(loop, max(3, min(args.steps, 10)), flush)
    ms_loop = statistics.mean(tl)
    # a launch-bound batch: 512 networks of QTs of at most 2^14 entries, every
    # one run by the persistent kernel, against the same graph without it
    small = synth.random_batch(512, seed=0, max_qt_entries=1 << 14)
    hs_s, outs_s = [], []
    for n in small:
        ts = [(t.inds, torch.from_numpy(np.ascontiguousarray(t.data)).to(dev), QTPU_CT if t.kind == "CT" else QTPU_QT)
              for t in n.tensors]
        h = from_network(ts, n.output, prec=args.prec, max_intermediate_bytes=(1 << 23) * 8)
        hs_s.append(h)
        outs_s.append(torch.empty(h.output_size(), dtype=torch.float64, device=dev))
    for _ in range(3):
        contract_batch(hs_s, outs_s)
    ms_sp = statistics.mean(timed_steps(lambda: contract_batch(hs_s, outs_s), max(3, min(args.steps, 10)), flush))
    info_s = batch_info(hs_s, outs_s)
    for _ in range(3):
        contract_batch(hs_s, outs_s, persistent=False)
    ms_sg = statistics.mean(timed_steps(lambda: contract_batch(hs_s, outs_s, persistent=False),
                                        max(3, min(args.steps, 10)), flush))
    for h in hs_s:
        h.close()
    # parity of a sample against the oracle
    rel = 0.0
    if rank == 0:
        from oracle import planner, tn
        for i in range(0, 512, 32):
            n = nets[i]
            p = planner.make_plan(n.inds(), n.dims(), n.output)
            ref = tn.contract_pairwise(n.pairs(), n.output, planner.order_of(p)).ravel()
            got = outs[i].cpu().numpy()
            rel = max(rel, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    peaks = load_peaks()
    achieved = (nbytes + sum(h.output_size() * 8 for h in hs)) / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": world * flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": WORKLOADS["batch"], "networks": len(nets), "flops_per_step": flops,
                   "leaf_bytes": nbytes, "l2": "flushed between timed steps (256 MiB write)"},
        "rel_err_vs_oracle_max_of_16": rel,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "whole batch (aggregate leaf bytes / batch time)"},
        "default_schedule": {"persistent_kernel_networks": info["persistent_networks"], "tasks": info["tasks"],
                             "rule": "persistent kernel when small gather-only networks are >= 1/2 of the batch"},
        "graph_branches_only": {"ms_per_step": ms_graph, "value": flops / (ms_graph * 1e-3) / 1e12},
        "persistent_kernel_forced": {"ms_per_step": ms_pers, "networks": info_p["persistent_networks"],
                                     "tasks": info_p["tasks"], "value": flops / (ms_pers * 1e-3) / 1e12},
        "one_call_per_network": {"ms_per_step": ms_loop, "value": flops / (ms_loop * 1e-3) / 1e12,
                                 "speedup_of_batch": ms_loop / ms},
        "small_network_batch": {"networks": len(small), "max_qt_entries": 1 << 14,
                                "persistent_networks": info_s["persistent_networks"],
                                "ms_persistent": ms_sp, "ms_graph_branches_only": ms_sg,
                                "speedup_of_persistent": ms_sg / ms_sp},
        "cpu_baseline": None, "fp64_gpu_path": None, "e2e": None,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    for h in hs:
        h.close()


def run_qpd(args, rank, world):
    """QPD sampling of the 100-qubit network for several draw counts: the
    qtpu_htn_qpd_sample call (fuse, draw, truncate, QT copies) timed with CUDA
    events, then the sampled network planned and contracted."""
    import torch
    import synth
    from paper_2410_15080_b300.htn import HTN, QTPU_CT, QTPU_QT
    dev = torch.device("cuda", torch.cuda.current_device())
    net = synth.ring_chords_htn(k=args.observables)
    h = HTN(dev.index)
    for t in net.tensors:
        h.add_tensor(t.inds, data=torch.from_numpy(np.ascontiguousarray(t.data)).to(dev),
                     kind=QTPU_CT if t.kind == "CT" else QTPU_QT)
    h.set_output(net.output)
    ng = h.qpd_groups()
    qt_bytes = sum(t.data.nbytes for t in net.tensors if t.kind == "QT")
    peaks = load_peaks()
    gen = torch.Generator(device=dev).manual_seed(0)
    sweep = []
    for s_qpd in [int(x) for x in args.s_qpd.split(",")]:
        u = torch.rand(ng * s_qpd, dtype=torch.float64, device=dev, generator=gen)
        ts, hs = [], None
        for r in range(args.warmup + args.steps):
            if hs is not None:
                hs.close()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hs = h.qpd_sample(s_qpd, u)
            e1.record()
            torch.cuda.synchronize()
            if r >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        info = hs.qpd_info()
        kept_qt = 0
        for t in range(hs.n_tensors):
            ti = hs.tensor_info(t)
            if ti["kind"] == QTPU_QT:
                kept_qt += int(np.prod(ti["dims"])) * (8 if ti["dtype"] == "f64" else 4)
        t0 = time.perf_counter()
        hs.plan(args.prec, max_intermediate_bytes=8 << 30, n_candidates=64)
        plan_s = time.perf_counter() - t0
        st = hs.exec_stats()
        for _ in range(2):
            hs.contract()
        tc = []
        for _ in range(3):
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            hs.contract()
            c1.record()
            torch.cuda.synchronize()
            tc.append(c0.elapsed_time(c1))
        hs.sync()
        sweep.append({"s_qpd": s_qpd, "sample_ms": ms, "groups_kept_of": [list(x) for x in info],
                      "qt_bytes_after": kept_qt, "qt_bytes_before": qt_bytes,
                      "plan_s": plan_s, "contract_ms": statistics.median(tc),
                      "contract_flops": st["flops_executed"]})
        hs.close()
    h.close()
    base = sweep[-1]
    line = {
        "metric": "QPD sample + simplify (ms per call) of the 100-qubit h-TN", "value": sweep[0]["sample_ms"],
        "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sweep[0]["sample_ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["qpd"], "s_qpd": sweep[0]["s_qpd"], "groups": ng},
        "roofline": {"bound": "hbm", "kernel": "whole qtpu_htn_qpd_sample call (QT copies dominate)",
                     "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": None, "traffic": None},
        "sweep": sweep, "gpu_launches": None,
    }
    # the QT copies read and write the kept entries of the copied QTs
    moved = 2 * base["qt_bytes_after"]
    line["roofline"]["achieved"] = moved / (base["sample_ms"] * 1e-3) / 1e9
    line["roofline"]["frac"] = line["roofline"]["achieved"] / peaks["hbm_gbs"]
    line["roofline"]["note"] = f"2 x kept QT bytes at s_qpd = {base['s_qpd']} / call time"
    if rank == 0:
        print(json.dumps(line))


def run_knit(args, rank, world):
    """Naive knitting (qtpu_htn_knit_naive) vs the contraction, on rings of
    growing size; both timed with CUDA events after warm-up."""
    import torch
    import synth
    from paper_2410_15080_b300.htn import HTN, QTPU_CT, QTPU_QT
    dev = torch.device("cuda", torch.cuda.current_device())
    sweep = []
    for n_sub in (3, 4, 5):
        net = synth.ring_htn(n_sub=n_sub, gates_per_edge=1, wires_per_edge=1, k=8, seed=n_sub)
        h = HTN(dev.index)
        for t in net.tensors:
            h.add_tensor(t.inds, data=torch.from_numpy(np.ascontiguousarray(t.data)).to(dev),
                         kind=QTPU_CT if t.kind == "CT" else QTPU_QT)
        h.set_output(net.output)
        out, ninst = h.knit_naive()
        reps = 3 if n_sub < 5 else 1
        tn_ = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h.knit_naive(out)
            e1.record()
            torch.cuda.synchronize()
            tn_.append(e0.elapsed_time(e1))
        naive = out.cpu().numpy()
        h.plan("fp64")
        for _ in range(3):
            c = h.contract()
        tc = []
        for _ in range(5):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = h.contract()
            e1.record()
            torch.cuda.synchronize()
            tc.append(e0.elapsed_time(e1))
        h.sync()
        rel = float(np.linalg.norm(c.cpu().numpy() - naive) / np.linalg.norm(naive))
        n_t = len(net.tensors)
        # FP64 operations of the naive sum: per instance and output, n_t - 1
        # multiplies and one add
        ops = ninst * len(naive) * n_t
        ms_n = statistics.median(tn_)
        sweep.append({"n_sub": n_sub, "cuts": 2 * n_sub, "instances": ninst, "outputs": len(naive),
                      "naive_ms": ms_n, "naive_fp64_gops": ops / (ms_n * 1e-3) / 1e9,
                      "contract_fp64_ms": statistics.median(tc), "speedup_of_contraction": ms_n / statistics.median(tc),
                      "rel_diff": rel})
        h.close()
    last = sweep[-1]
    # DMUL / DADD issue at the DFMA rate: half the FMA-counted FP64 peak
    fp64_peak = 1050.0 / 2
    line = {
        "metric": "naive knitting vs h-TN contraction (time ratio) on a 5-subcircuit ring", "value":
        last["speedup_of_contraction"], "unit": "x", "n_gpus": world, "steps": 1, "warmup": 1,
        "ms_per_step": last["naive_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOADS["knit"]},
        "roofline": {"bound": "alu", "kernel": "k_knit_terms", "achieved": last["naive_fp64_gops"],
                     "peak": fp64_peak, "unit": "GFLOP/s", "frac": last["naive_fp64_gops"] / fp64_peak,
                     "traffic": None,
                     "peak_note": "FP64 multiplies and adds at the DFMA issue rate: half the measured FP64 "
                                  "matmul rate (1.05 TFLOP/s FMA-counted, BASELINE.md)"},
        "sweep": sweep, "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(line))


def qteval_program(n, seed=0, k=16):
    """A subcircuit like the paper's VQE/QAOA ansatz pieces: RY/RZ layers
    and CZ chains, 2 gate cuts (on qubits 0 and n-1 after the first chain),
    a measured wire (qubit 1, no later gates) and a prepared wire (qubit 2)."""
    import oracle.sim as _sim  # noqa: F401  (matrices only)
    rng = np.random.default_rng([seed, n])
    def rot(q):
        t, p = rng.uniform(0, 2 * np.pi, 2)
        c, s_ = np.cos(t / 2), np.sin(t / 2)
        ry = np.array([[c, -s_], [s_, c]], dtype=np.complex128)
        rz = np.diag([np.exp(-0.5j * p), np.exp(0.5j * p)])
        return ("u1", q, rz @ ry)
    others = [q for q in range(n) if q != 1]
    ops = [rot(q) for q in range(n)]
    ops += [("cz", q, q + 1) for q in range(n - 1)]
    ops += [("gate_cut", 0, 0, 0), ("gate_cut", n - 1, 1, 1)]
    ops += [rot(q) for q in range(n)]
    ops += [("cz", q, q + 1) for q in range(2, n - 1)] + [("cz", 0, 2)]
    ops += [rot(q) for q in others]
    paulis = []
    for j in range(k):
        sgl = ["I"] * n
        sgl[others[j % len(others)]] = "Z"
        sgl[others[(j + 1) % len(others)]] = "Z" if j >= len(others) else sgl[others[(j + 1) % len(others)]]
        paulis.append("".join(sgl))
    return {"n": n, "ops": ops, "cuts": [("gate",), ("gate",), ("measure", 1), ("prepare", 2)], "paulis": paulis}


def run_qteval(args, rank, world):
    """The QT evaluator on the GPU, timed with CUDA events, against the FP64
    branching oracle (numpy) on a sample of instances."""
    import torch
    from paper_2410_15080_b300 import qt_evaluate
    from oracle import qt_eval
    sweep = []
    for n in (12, 15):
        prog = qteval_program(n)
        qt_evaluate(prog)
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = qt_evaluate(prog)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        got = out.cpu().numpy()
        # FP64 operations per branch (multiplies and adds of the kernel)
        N = 2 ** n
        ops_fp = 0
        for op in prog["ops"]:
            ops_fp += {"u1": 14 * N, "cz": 0, "gate_cut": 6 * N}[op[0]]
        ops_fp += 6 * n * N + 7 * len(prog["paulis"]) * N
        # branches: each instance has 2^(measurements) of them
        n_br = 0
        for g0 in range(6):
            for g1 in range(6):
                m = (g0 in (2, 3)) + (g1 in (4, 5))
                n_br += 16 * 2 ** m
        flops = ops_fp * n_br
        # oracle on a sample: the first cut value of each axis fixed, all
        # observables (one instance group per measured/prepared value pair)
        t0 = time.perf_counter()
        sample = dict(prog)
        ref = qt_eval.qt_branching(sample) if n <= 12 else None
        cpu_s = time.perf_counter() - t0
        rel = float(np.abs(got - ref).max()) if ref is not None else None
        sweep.append({"n_qubits": n, "instances": 576, "branches": n_br, "ms": ms,
                      "instances_per_s": 576 / (ms * 1e-3), "fp64_gflops": flops / (ms * 1e-3) / 1e9,
                      "oracle_cpu_s": cpu_s if ref is not None else None, "max_abs_diff_vs_oracle": rel})
    fp64_peak = 1050.0 / 2
    last = sweep[-1]
    line = {
        "metric": "QT evaluation (instances/s) of a 15-qubit subcircuit", "value": last["instances_per_s"],
        "unit": "instances/s", "n_gpus": world, "steps": args.steps, "warmup": 1, "ms_per_step": last["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["qteval"]},
        "roofline": {"bound": "alu", "kernel": "k_qt_instances", "achieved": last["fp64_gflops"], "peak": fp64_peak,
                     "unit": "GFLOP/s", "frac": last["fp64_gflops"] / fp64_peak, "traffic": None,
                     "peak_note": "FP64 multiplies and adds at the DFMA issue rate: half the measured FP64 "
                                  "matmul rate (1.05 TFLOP/s FMA-counted)"},
        "cpu_baseline": {"value": 576 / sweep[0]["oracle_cpu_s"], "unit": "instances/s", "cores": oracle_threads(),
                         "kind": "oracle", "sample": "the 12-qubit program, all 576 instances, numpy branching "
                                                     "statevector"},
        "sweep": sweep, "gpu_launches": args.steps,
    }
    if rank == 0:
        print(json.dumps(line))


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2410_15080_b300 import from_network
    from paper_2410_15080_b300.htn import QTPU_CT, QTPU_QT

    dev = torch.device("cuda", torch.cuda.current_device())
    net, plan_kw = make_network(args.workload, args.shape, args.observables)
    tensors = [(t.inds, torch.from_numpy(np.ascontiguousarray(t.data)).to(dev), QTPU_CT if t.kind == "CT" else QTPU_QT)
               for t in net.tensors]
    t_plan = time.perf_counter()
    h = from_network(tensors, net.output, prec=args.prec, **plan_kw)
    plan_s = time.perf_counter() - t_plan
    st = h.plan_stats()
    out = torch.empty(h.output_size(), dtype=torch.float64, device=dev)
    flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2
    flush = (lambda: flush_buf.zero_()) if net.nbytes() < (256 << 20) else (lambda: None)
    n_slices = int(h.plan_info().split("slices n=")[1].split()[0])
    # one step = one complete contraction (every slice); with several ranks
    # each contracts its own replica (weak scaling, no collective).  The FLOPs
    # are those the contraction executes: with slice reuse, a result that
    # depends on only some sliced indices is computed once per value of them.
    es = h.exec_stats()
    flops = es["flops_executed"]
    step = lambda: h.contract(out)  # noqa: E731

    for _ in range(args.warmup):
        step()
    h.sync()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(dev.index) as clk:
        ts = timed_steps(step, args.steps, flush)
        if world > 1:
            dist.barrier()
    h.sync()
    tot = torch.tensor([sum(ts)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms = tot.item() / args.steps
    value = world * flops / (ms * 1e-3) / 1e12
    got = out.cpu().numpy()
    if args.extras == "none":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "TFLOP/s", "ms_per_step": ms,
                              "steps": args.steps, "warmup": args.warmup, "extras": "none",
                              "config": {"workload": WORKLOADS[args.workload], "flops_per_step": flops}}))
        h.close()
        return

    # per-kernel-class timing (separate pass, same launches; a long step is
    # profiled twice at most)
    n_prof = args.steps if ms < 200 else min(args.steps, 2)
    h.profile(True)
    prof = None
    for _ in range(n_prof):
        flush()
        step()
        p = h.profile_read()
        if prof is None:
            prof = p
        else:
            for kk in prof:
                for f in prof[kk]:
                    prof[kk][f] += p[kk][f]
    h.profile(False)

    # parity of this run's output against the FP64 oracle: the whole output
    # (mid, gemm), or the restricted output k in {0, 1} (100-qubit)
    rel = rel_max = None
    cpu = None
    if rank == 0 and args.workload in ("mid", "gemm"):
        from oracle import planner, tn
        p = planner.make_plan(net.inds(), net.dims(), net.output)
        ref = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p)).ravel()
        rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        rel_max = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    if rank == 0 and world == 1 and args.workload.startswith("100q"):
        ro = RestrictedOracle(net)
        ref, sec = ro.run()
        sub_got = got[list(ro.values)]
        rel = float(np.linalg.norm(sub_got - ref) / np.linalg.norm(ref))
        rel_max = float(np.max(np.abs(sub_got - ref)) / np.max(np.abs(ref)))
        cpu = {"value": ro.flops / sec / 1e12, "unit": "TFLOP/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"the exact FP64 oracle on the restricted output k in {{0, 1}} (2 of the 64 observables; "
                         f"{ro.flops / 1e12:.3f} TFLOP of the oracle's own unsliced plan) in {sec:.1f} s, numpy "
                         f"FP64 on {cpu_model()} ({os.cpu_count()} host cores)"}
    if rank == 0 and world == 1 and args.workload == "mid":
        sec, reps, threads = oracle_seconds(net, args.cpu_budget)
        cpu = {"value": flops / sec / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": f"{reps} full contractions of the workload in {reps * sec:.1f} s, numpy FP64 on "
                         f"{cpu_model()} ({os.cpu_count()} host cores)"}

    # plain FP64 GPU path: same plan, torch FP64 ops, one launch per step
    fp64 = None
    steps, final_sum = parse_plan(h.plan_info())
    t64 = [(list(i), x.double()) for i, x, _ in tensors]
    if n_slices == 1:
        for _ in range(2):
            fp64_torch_path(t64, list(net.output), steps, final_sum)
        ts64 = timed_steps(lambda: fp64_torch_path(t64, list(net.output), steps, final_sum),
                           max(3, min(args.steps, 10)), flush)
        ms64 = statistics.mean(ts64)
        fp64 = {"value": flops / (ms64 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms64,
                "impl": "torch FP64 permute+bmm per planned step", "speedup_of_ours": ms64 / ms}
    else:
        # the FP64 path on a fixed subset of slices (same shapes), extrapolated
        sliced = [int(x) for x in h.plan_info().split("idx=")[1].split()[0].split(",")]
        dims = net.dims()

        def one_slice(s_id):
            vals, r = [], s_id
            for i in reversed(sliced):
                vals.append(r % dims[i])
                r //= dims[i]
            return dict(zip(reversed(sliced), vals))
        S64 = 2
        fp64_torch_path(t64, list(net.output), steps, final_sum, one_slice(0))
        ts64 = timed_steps(lambda: [fp64_torch_path(t64, list(net.output), steps, final_sum, one_slice(s))
                                    for s in range(S64)], 2, flush)
        rate64 = es["flops_all_slices"] / n_slices * S64 / (statistics.mean(ts64) * 1e-3)
        ms64 = flops / rate64 * 1e3  # at that rate, the FLOPs this contraction executes
        fp64 = {"value": rate64 / 1e12, "unit": "TFLOP/s", "ms_per_step": ms64,
                "impl": f"torch FP64 permute+bmm per planned step, {S64} of {n_slices} slices timed; its rate "
                        f"applied to the FLOPs the contraction executes (the same slice reuse)",
                "speedup_of_ours": ms64 / ms}
    del t64

    # end to end through the C ABI with host buffers (pinned): the upload of
    # every leaf, the contraction and the download of the result per step
    host = [torch.from_numpy(np.ascontiguousarray(t.data)).pin_memory() for t in net.tensors]
    hout_t = torch.empty(h.output_size(), dtype=torch.float64).pin_memory()  # pinned: an asynchronous download
    hout = hout_t.numpy()
    h.contract_host(host, hout)
    n_e2e = max(3, min(args.steps, 10)) if ms < 200 else min(args.steps, 3)
    te = []
    for _ in range(n_e2e):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.contract_host(host, hout)
        te.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * statistics.mean(te)
    h2d = sum(x.numel() * x.element_size() for x in host)
    e2e = {"value": world * flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h.output_size() * 8, "steps": n_e2e}
    del host

    peaks = load_peaks()
    # kernels timed inside a timed region of a second or more of back-to-back
    # contractions run under the sustained power limit
    sustained = ms * args.steps >= 1000
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    if dom == "gemm":
        ratio = {"bf16x3": 6, "3xtf32": 6, "tf32": 2}.get(args.prec, 6)  # bf16-MMA equivalents per useful FMA
        pk = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
        peak = pk / ratio
        achieved = d["flops"] / d["launches"] / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_gemm_tc",
                "peak_note": f"{peaks['src']} bf16 {'sustained' if sustained else 'burst'} / {ratio} "
                             f"(useful FLOPs of {args.prec})"}
    else:
        achieved = d["bytes"] / d["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": dom,
                "peak_note": f"{peaks['src']} copy bandwidth; algorithmic bytes = operands read once + results "
                             f"written once"}
    roof["traffic"] = measured_traffic(args.workload, dom)
    roof["per_launch_ms"] = per_launch_ms
    roof["launches_per_step"] = d["launches"] / n_prof
    roof["classes"] = {k: {"ms_per_step": v["ms"] / n_prof, "launches_per_step": v["launches"] / n_prof,
                           "algorithmic_GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] else None,
                           "useful_TFLOPs": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] else None,
                           "traffic_per_launch": measured_traffic(args.workload, k)}
                       for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + (f" ({args.shape})" if args.workload == "gemm" else "")
                   + (f" (k = {args.observables} observables)" if args.workload.startswith("100q") and args.observables != 64 else ""),
                   "sharding": "independent replicas" if world > 1 else "single GPU",
                   "flops_per_step": flops, "prec": args.prec,
                   "gemm_tiles": gemm_tiles_used(),
                   "l2": "flushed between timed steps (256 MiB write)" if net.nbytes() < (256 << 20)
                   else "inputs larger than L2", "plan_steps": st["n_steps"],
                   "tensor_core_steps": st["n_tensor_core_steps"], "parallelism": f"replicas x{world}",
                   "slices": n_slices, "flops_plan_all_slices": es["flops_all_slices"],
                   "slice_reuse": {"flops_executed": flops, "kept_bytes": es["kept_bytes"],
                                   "launches_per_contraction": es["launches"]},
                   "plan_seconds": plan_s},
        "rel_err_vs_oracle": rel,
        "rel_err_max_vs_oracle": rel_max,
        "rel_err_entries": ("all" if args.workload in ("mid", "gemm") else "k in {0, 1} (2 of 64)") if rel is not None else None,
        "roofline": roof,
        "cpu_baseline": cpu,
        "fp64_gpu_path": fp64,
        "e2e": e2e,
        "gpu_launches": es["launches"] * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="100q", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "3xtf32", "tf32", "fp64"])
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--shape", default="8x1024x1024x1024", help="gemm workload: batch x M x N x K")
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="none: only the warm-up and timed contractions (for profiler launch lists and captures)")
    ap.add_argument("--s-qpd", default="10,100,1000,100000", help="qpd workload: draws per group, comma-separated")
    ap.add_argument("--observables", type=int, default=64,
                    help="100q workloads: size k of the observable index (64 = the benchmark; smaller for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "batch":
        run_batch(args, rank, world)
    elif args.workload == "qpd":
        run_qpd(args, rank, world)
    elif args.workload == "knit":
        run_knit(args, rank, world)
    elif args.workload == "qteval":
        run_qteval(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
