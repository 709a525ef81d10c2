"""Learned cost model: rank candidate contraction plans by predicted time.

Section 6.1 step 3 chooses a contraction sequence before contracting; the
exact FLOP count is a proxy for time that ignores how each step maps onto
the hardware (tensor-core vs CUDA-core steps, padding of 128-row tiles,
memory-bound gathers, launch counts).  This module learns time from the
contractor's own measurements:

* ``candidates``  -- 64 plans per network: 16 orders (the greedy order and
  15 randomised greedy orders, ``seed`` of the plan options) x 4 slicing
  settings;
* ``plan_features`` -- a fixed-length vector computed from a plan's
  canonical text (FLOPs, sizes, slice count, the largest steps, how many
  steps reach the tensor cores);
* ``measure``     -- contracts a network with a given plan on the GPU and
  times it with CUDA events (median of replays);
* ``train``       -- fits the library's MLP (BF16 weights, FP32
  accumulation, Adam; forward and backward in the library's kernels) to
  log(time);
* ``choose``      -- the candidate with the smallest predicted time among
  those whose exact FLOP count is within a factor F of the fewest (the
  exact cost model bounds the model's error; F = 1 is the exact-cost choice
  itself, F = inf trusts the model alone); F is selected on held-out
  training networks.

The model only chooses among plans: every plan is contracted exactly as any
other, so results are unaffected by it.
"""
from __future__ import annotations

import json
import math
import statistics
import time

import numpy as np

from .htn import HTN, MLP, from_network, plan_text

N_FEATURES = 32
SLICINGS = [{}, {"n_slices": 4}, {"n_slices": 16}, {"n_slices": 64}]
N_ORDERS = 16


def _log2(x: float) -> float:
    return math.log2(x + 1.0)


def parse_plan(text: str):
    steps, n_slices, flops_total, peak, sliced = [], 1, 0, 0, set()
    for line in text.splitlines():
        f = line.split()
        if f[0] == "step":
            kv = dict(x.split("=") for x in f[6:])
            g = {k: ([] if v == "-" else [int(i) for i in v.split(",")]) for k, v in kv.items()
                 if k in ("batch", "m", "n", "k", "sa", "sb")}
            steps.append((g, int(kv["size"]), int(kv["flops"])))
        elif f[0] == "slices":
            n_slices = int(f[1].split("=")[1])
            sl = f[2].split("=")[1]
            sliced = set() if sl == "-" else {int(i) for i in sl.split(",")}
        elif f[0] == "cost":
            kv = dict(x.split("=") for x in f[1:])
            flops_total, peak = int(kv["flops_total"]), int(kv["peak"])
    return steps, n_slices, sliced, flops_total, peak


def plan_features(text: str, dims: dict, leaf_inds) -> np.ndarray:
    """Fixed-length description of a plan (FP32)."""
    steps, n_slices, sliced, flops_total, peak = parse_plan(text)
    d = lambda ix: math.prod(dims[i] for i in ix if i not in sliced)  # noqa: E731
    f = np.zeros(N_FEATURES, dtype=np.float64)
    per_slice = sum(s[2] for s in steps)
    tc_fl, other_fl, n_tc, sizes = 0, 0, 0, 0
    for g, size, fl in steps:
        nb, nm, nn, nk = d(g["batch"]), d(g["m"]), d(g["n"]), d(g["k"])
        gm, gn = (nn, nm) if nm < 64 <= nn else (nm, nn)
        tc = not g["sa"] and not g["sb"] and gm >= 64 and gn >= 32 and nk >= 32 and nb * nm * nn * nk >= 1 << 22
        n_tc += tc
        tc_fl += fl if tc else 0
        other_fl += 0 if tc else fl
        sizes += size
    f[0] = _log2(flops_total)
    f[1] = _log2(per_slice)
    f[2] = math.log2(n_slices)
    f[3] = _log2(peak)
    f[4] = len(steps) / 64.0
    f[5] = n_tc / 16.0
    f[6] = _log2(tc_fl)
    f[7] = _log2(other_fl)
    f[8] = _log2(sizes * n_slices)
    top = sorted(steps, key=lambda s: -s[2])[:8]
    for j, (g, size, fl) in enumerate(top):
        f[9 + 2 * j] = _log2(fl)
        f[10 + 2 * j] = _log2(size)
    f[25] = _log2(sum(1 for s in steps if s[2] > 1 << 20))
    f[26] = (top[0][2] / per_slice) if steps and per_slice else 0.0
    f[27] = math.log2(len(leaf_inds))
    f[28] = _log2(sum(math.prod(dims[i] for i in ix) for ix in leaf_inds))
    # launches the executor makes: steps that absorb a small leaf are folded
    # into their consumer, tensor-core steps launch 3 kernels, others 1
    n_leaves = len(leaf_inds)
    sizes_of = {t: math.prod(dims[i] for i in ix if i not in sliced) for t, ix in enumerate(leaf_inds)}
    launches, gathers = 1, 0
    for j, (g, size, fl) in enumerate(steps):
        xy = [int(v) for v in text.splitlines()[1 + j].split()[2:4]]
        small = [t < n_leaves and sizes_of[t] <= 256 for t in xy]
        nb, nm, nn, nk = d(g["batch"]), d(g["m"]), d(g["n"]), d(g["k"])
        gm, gn = (nn, nm) if nm < 64 <= nn else (nm, nn)
        tc = not g["sa"] and not g["sb"] and gm >= 64 and gn >= 32 and nk >= 32 and nb * nm * nn * nk >= 1 << 22
        if any(small) and j + 1 < len(steps):
            continue
        launches += (3 if tc else 1) * n_slices
        gathers += 0 if tc else n_slices
    f[29] = math.log2(launches)
    f[30] = _log2(gathers)
    f[31] = n_slices * len(steps) / 4096.0
    return f.astype(np.float32)


def candidates(net):
    """(plan kwargs, plan text) for 16 orders x 4 slicings."""
    out = []
    for seed in range(N_ORDERS):
        for s in SLICINGS:
            kw = dict(s, seed=seed)
            try:
                t = plan_text(net.inds(), net.dims(), net.output, **kw)
            except Exception:
                continue
            out.append((kw, t))
    return out


def measure(dev_tensors, output, kw, prec="bf16x3", reps=5):
    """Median device time (ms) of one contraction with the given plan."""
    import torch
    h = from_network(dev_tensors, output, prec=prec, **kw)
    out = torch.empty(h.output_size(), dtype=torch.float64, device=dev_tensors[0][1].device)
    h.contract(out)
    h.contract(out)
    ts = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        h.contract(out)
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    h.close()
    return statistics.median(ts), out


def to_device(net, device="cuda"):
    import torch
    return [(t.inds, torch.from_numpy(np.ascontiguousarray(t.data)).to(device), 1 if t.kind == "CT" else 0)
            for t in net.tensors]


def gen_dataset(nets, per_net=None, seed=0):
    """Features, measured log(ms), network ids and exact FLOPs of candidate
    plans of each network."""
    rng = np.random.default_rng(seed)
    X, y, groups, flops = [], [], [], []
    for gi, net in enumerate(nets):
        dev = to_device(net)
        cands = candidates(net)
        if per_net and len(cands) > per_net:
            cands = [cands[i] for i in rng.choice(len(cands), per_net, replace=False)]
        for kw, text in cands:
            ms, _ = measure(dev, net.output, kw)
            X.append(plan_features(text, net.dims(), net.inds()))
            y.append(math.log(ms))
            groups.append(gi)
            flops.append(float(parse_plan(text)[3]))
    return (np.array(X, dtype=np.float32), np.array(y, dtype=np.float32), np.array(groups),
            np.array(flops, dtype=np.float64))


class CostModel:
    """Standardised features -> MLP -> predicted log(ms)."""

    def __init__(self, hidden=256, seed=1):
        self.mlp = MLP(N_FEATURES, hidden, seed)
        self.mu = np.zeros(N_FEATURES, np.float32)
        self.sd = np.ones(N_FEATURES, np.float32)
        self.ymu = 0.0

    def _x(self, X):
        import torch
        return torch.from_numpy(((X - self.mu) / self.sd).astype(np.float32)).cuda()

    def train(self, X, y, epochs=200, batch=256, lr=2e-3, seed=0):
        import torch
        self.mu = X.mean(0)
        self.sd = X.std(0) + 1e-3
        self.ymu = float(y.mean())
        xt = self._x(X)
        yt = torch.from_numpy((y - self.ymu).astype(np.float32)).cuda()
        rng = np.random.default_rng(seed)
        losses = []
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(len(X))).cuda()
            tot = 0.0
            for i in range(0, len(X), batch):
                idx = perm[i:i + batch]
                tot += self.mlp.train_step(xt[idx].contiguous(), yt[idx].contiguous(), lr) * len(idx)
            losses.append(tot / len(X))
        return losses

    def predict(self, X):
        return self.mlp.forward(self._x(X)).cpu().numpy() + self.ymu


def pick(pred, flops, factor):
    """Index of the smallest prediction among candidates with at most
    factor x the fewest FLOPs (ties: fewer FLOPs, then lower index)."""
    flops = np.asarray(flops, dtype=np.float64)
    ok = flops <= factor * flops.min()
    idx = np.flatnonzero(ok)
    return int(min(idx, key=lambda i: (pred[i], flops[i], i)))


def select_factor(pred, y, flops, groups, factors=(1.0, 1.25, 1.5, 2.0, 3.0, 4.0, float("inf"))):
    """The factor whose choices have the smallest geometric-mean measured time."""
    best = None
    for f in factors:
        t = []
        for g in np.unique(groups):
            i = np.flatnonzero(groups == g)
            t.append(y[i][pick(pred[i], flops[i], f)])
        score = float(np.mean(t))
        if best is None or score < best[1] - 1e-12:
            best = (f, score)
    return best[0]


def choose(model, net, factor=float("inf")):
    """(model choice, exact-FLOP choice, candidates, predictions, flops)."""
    cands = candidates(net)
    X = np.stack([plan_features(t, net.dims(), net.inds()) for _, t in cands])
    pred = model.predict(X)
    flops = [float(parse_plan(t)[3]) for _, t in cands]
    return cands, pick(pred, flops, factor), int(np.argmin(flops)), pred


def evaluate(model, nets, factor):
    """Measured time of the model's choice (alone, and bounded by `factor`)
    and of the exact-cost choice, and ranking quality over all candidates."""
    from scipy.stats import spearmanr
    rows = []
    for net in nets:
        dev = to_device(net)
        cands, im, ie, pred = choose(model, net)
        flops = [float(parse_plan(t)[3]) for _, t in cands]
        ih = pick(pred, flops, factor)
        meas = [measure(dev, net.output, kw)[0] for kw, _ in cands]
        best = int(np.argmin(meas))
        rows.append({"n_tensors": len(net.tensors), "cands": len(cands), "ms_model_alone": meas[im],
                     "ms_model_bounded": meas[ih], "ms_exact": meas[ie], "ms_best": meas[best],
                     "spearman": float(spearmanr(pred, np.log(meas)).correlation)})
    return rows


def eval_networks(n, seed=1000):
    """Larger random networks (10-16 subcircuits, 30-50 cuts): the evaluation set."""
    import synth
    return [synth.random_htn(seed + i, n_sub_range=(10, 16), n_cuts_range=(30, 50), k_range=(8, 32),
                             max_qt_entries=1 << 20, max_cuts_per_pair=4, dtype=np.float64) for i in range(n)]


def train_networks(n, seed=0):
    """Training networks: the batched-workload generator, widened."""
    import synth
    return [synth.random_htn(seed + i, n_sub_range=(4, 14), n_cuts_range=(8, 44), k_range=(4, 32),
                             max_qt_entries=1 << 20, max_cuts_per_pair=4, dtype=np.float64) for i in range(n)]


def main():
    import argparse
    import os
    import torch
    ap = argparse.ArgumentParser(description="train the cost model on measured plans and compare its choices")
    ap.add_argument("--train-nets", type=int, default=64)
    ap.add_argument("--per-net", type=int, default=64)
    ap.add_argument("--eval-nets", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--data", default="", help="npz cache of the measured training set (read if present)")
    args = ap.parse_args()
    torch.cuda.init()
    t0 = time.time()
    if args.data and os.path.exists(args.data):
        z = np.load(args.data)
        X, y, groups, flops = z["X"], z["y"], z["groups"], z["flops"]
    else:
        X, y, groups, flops = gen_dataset(train_networks(args.train_nets), args.per_net)
        if args.data:
            np.savez(args.data, X=X, y=y, groups=groups, flops=flops)
    t_data = time.time() - t0
    # choose the FLOP bound on held-out training networks (last 20 %)
    ng = int(groups.max()) + 1
    hold = groups >= int(0.8 * ng)
    m0 = CostModel(seed=7)
    m0.train(X[~hold], y[~hold], epochs=args.epochs)
    factor = select_factor(m0.predict(X[hold]), y[hold], flops[hold], groups[hold])
    model = CostModel()
    t0 = time.time()
    losses = model.train(X, y, epochs=args.epochs)
    t_train = time.time() - t0
    rows = evaluate(model, eval_networks(args.eval_nets), factor)
    gm = lambda v: float(np.exp(np.mean(np.log(v))))  # noqa: E731
    summary = {
        "training_pairs": int(len(X)), "data_seconds": t_data, "train_seconds": t_train,
        "loss_first_last": [losses[0], losses[-1]], "flop_bound_factor": factor,
        "eval_networks": len(rows),
        "geomean_ms_model_alone": gm([r["ms_model_alone"] for r in rows]),
        "geomean_ms_model_bounded": gm([r["ms_model_bounded"] for r in rows]),
        "geomean_ms_exact_choice": gm([r["ms_exact"] for r in rows]),
        "geomean_ms_best_candidate": gm([r["ms_best"] for r in rows]),
        "mean_spearman": float(np.mean([r["spearman"] for r in rows])),
        "rows": rows,
    }
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
