"""Helpers for the GPU tests: move a synthetic network to the device and
contract it through the C ABI; compare with the oracle."""
import numpy as np

REL_TOL = 1e-6       # normwise relative error bound for the tensor-core forms
FP64_TOL = 1e-12     # all-FP64 path (only the summation order differs)


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def to_device(net, device="cuda:0"):
    import torch
    from paper_2410_15080_b300 import htn
    out = []
    for t in net.tensors:
        kind = htn.QTPU_CT if t.kind == "CT" else htn.QTPU_QT
        out.append((t.inds, torch.from_numpy(np.ascontiguousarray(t.data)).to(device), kind))
    return out


def contract_gpu(net, prec="bf16x3", **plan_kw):
    import torch
    from paper_2410_15080_b300 import from_network
    dev = to_device(net)
    h = from_network(dev, net.output, prec=prec, **plan_kw)
    out = h.contract()
    h.sync()
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    stats = h.plan_stats()
    h.close()
    return res, stats


def oracle_value(net):
    from oracle import planner, tn
    p = planner.make_plan(net.inds(), net.dims(), net.output)
    return tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p)).ravel()


def oracle_restricted(net, values=(0, 1)):
    """Exact FP64 oracle entries of the output with the (single) observable
    index fixed to each of ``values``: one full contraction of the network
    per value, in the oracle planner's best-of-32 order for the network
    without that index (cheap enough for the full-size 100-qubit network)."""
    from oracle import planner, tn
    kid = net.output[0]
    inds1 = [tuple(i for i in t.inds if i != kid) for t in net.tensors]
    dims1 = {i: d for i, d in net.dims().items() if i != kid}
    p = planner.make_plan(inds1, dims1, (), n_candidates=32)
    return np.asarray(tn.contract_output_subset(net.pairs(), net.output, planner.order_of(p), kid,
                                                list(values))).ravel()
