"""Batched contraction of many independent h-TNs of uneven size in one CUDA
graph (random ring / 2-D-grid networks, FP32 and FP64 leaves): the
persistent kernel that runs every gather-only network's launches as tasks,
and the graph branches of the others, against the FP64 oracle and against
one-by-one contraction; and the persistent kernel's bounded dependency wait."""
import numpy as np
import pytest

import synth
from tests.gpu_util import REL_TOL, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu

# the batched workload's caps: QTs of at most 2^22 entries, peak intermediate
# of at most 2^23 entries (8 bytes each)
QT_CAP = 1 << 22
PEAK_BYTES = (1 << 23) * 8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def _handles(nets):
    from paper_2410_15080_b300 import from_network
    return [from_network(to_device(n), n.output, prec="bf16x3", max_intermediate_bytes=PEAK_BYTES) for n in nets]


def test_batch_of_uneven_networks():
    import torch
    from paper_2410_15080_b300 import batch_info, contract_batch
    nets = synth.random_batch(40, seed=3, max_qt_entries=QT_CAP)
    assert len({n.meta["topology"] for n in nets}) == 2
    assert {t.data.dtype for n in nets for t in n.tensors} == {np.dtype(np.float32), np.dtype(np.float64)}
    hs = _handles(nets)
    one = [h.contract().cpu().numpy() for h in hs]
    torch.cuda.synchronize()
    outs = [torch.full((h.output_size(),), float("nan"), dtype=torch.float64, device="cuda") for h in hs]
    # graph branches only: the same kernels as one by one, the same bits
    contract_batch(hs, outs, persistent=False)
    torch.cuda.synchronize()
    for o, s in zip(outs, one):
        np.testing.assert_array_equal(o.cpu().numpy(), s)
    # the persistent kernel for the gather-only networks
    for o in outs:
        o.fill_(float("nan"))
    contract_batch(hs, outs, persistent=True)
    torch.cuda.synchronize()
    for h in hs:
        h.sync()
    info = batch_info(hs, outs)
    assert 0 < info["persistent_networks"] < len(nets) and info["tasks"] > info["persistent_networks"]
    first = [o.cpu().numpy() for o in outs]
    for n, got, s in zip(nets, first, one):
        assert rel_err(got, s) <= 2 * REL_TOL
        assert rel_err(got, oracle_value(n)) <= REL_TOL
    # replay of the cached graph: the same bits
    for o in outs:
        o.fill_(float("nan"))
    contract_batch(hs, outs, persistent=True)
    torch.cuda.synchronize()
    for o, s in zip(outs, first):
        np.testing.assert_array_equal(o.cpu().numpy(), s)
    for h in hs:
        h.close()


def test_batch_of_512_networks():
    """The batched workload at its full size: 512 random networks (2-12
    subcircuits, 2-20 cuts, k 1-64, FP32/FP64, QTs up to 2^22 entries) in one
    graph with the persistent kernel; every output matches the graph-branch
    schedule and a sample of 32 matches the FP64 oracle.  By default (more
    than half the networks small) the batch takes the persistent kernel; a
    batch of mostly larger networks runs as graph branches only."""
    import torch
    from paper_2410_15080_b300 import batch_info, contract_batch
    nets = synth.random_batch(512, seed=0, max_qt_entries=QT_CAP)
    hs = _handles(nets)
    outs = [torch.empty(h.output_size(), dtype=torch.float64, device="cuda") for h in hs]
    ref = [torch.empty_like(o) for o in outs]
    contract_batch(hs, ref, persistent=False)
    contract_batch(hs, outs, persistent=True)
    torch.cuda.synchronize()
    for h in hs:
        h.sync()
    info = batch_info(hs, outs)
    assert info["persistent_networks"] >= 200
    d = [torch.empty_like(o) for o in outs]
    contract_batch(hs, d)
    torch.cuda.synchronize()
    assert batch_info(hs, d)["persistent_networks"] == info["persistent_networks"]
    for o, p in zip(d, outs):
        assert torch.equal(o, p)
    # mostly networks with tensor-core steps: the default is graph branches
    big = [i for i, h in enumerate(hs) if h.plan_stats()["n_tensor_core_steps"] > 0]
    mixed = big + [i for i in range(512) if i not in big][: len(big) // 2]
    dm = [torch.empty_like(outs[i]) for i in mixed]
    contract_batch([hs[i] for i in mixed], dm)
    torch.cuda.synchronize()
    assert batch_info([hs[i] for i in mixed], dm)["persistent_networks"] == 0
    for o, i in zip(dm, mixed):
        assert torch.equal(o, ref[i])
    for o, r in zip(outs, ref):
        assert rel_err(o.cpu().numpy(), r.cpu().numpy()) <= 2 * REL_TOL
    for i in range(0, 512, 16):
        assert rel_err(outs[i].cpu().numpy(), oracle_value(nets[i])) <= REL_TOL
    for h in hs:
        h.close()


def test_persistent_wait_gives_up_and_reports_timeout():
    """A dependency that never completes (the test hook of the batch options)
    makes the persistent kernel's bounded wait give up after 50 ms: the
    stalled network reports QTPU_ETIMEOUT on sync, nothing faults, and the
    same handles then contract correctly."""
    import torch
    from paper_2410_15080_b300 import batch_info, contract_batch
    from paper_2410_15080_b300.htn import QTPU_ETIMEOUT, QtpuError
    nets = synth.random_batch(8, seed=5, max_qt_entries=1 << 12)
    hs = _handles(nets)
    outs = [torch.zeros(h.output_size(), dtype=torch.float64, device="cuda") for h in hs]
    contract_batch(hs, outs)
    torch.cuda.synchronize()
    info = batch_info(hs, outs)
    # small: every network is gather-only, so the default takes them all
    assert info["persistent_networks"] == len(nets)
    stalled = 3
    contract_batch(hs, outs, wait_limit_ns=50_000_000, test_stall_network=stalled)
    torch.cuda.synchronize()
    with pytest.raises(QtpuError) as ei:
        hs[stalled].sync()
    assert ei.value.status == QTPU_ETIMEOUT
    for h in hs:  # networks left incomplete by the abort report it too; clear them
        try:
            h.sync()
        except QtpuError as e:
            assert e.status == QTPU_ETIMEOUT
    contract_batch(hs, outs)
    torch.cuda.synchronize()
    for n, h, o in zip(nets, hs, outs):
        h.sync()
        assert rel_err(o.cpu().numpy(), oracle_value(n)) <= REL_TOL
    for h in hs:
        h.close()


def test_few_outputs_with_long_sums():
    """Networks of the batched workload whose last step sums 576-864 terms
    into 5-46 outputs (FP64): lanes share an output, each summing a
    contiguous run of the loop, in the typed fast kernel and in the generic
    one; each network matches the FP64 oracle."""
    import re
    from paper_2410_15080_b300.htn import lowering_text
    nets = synth.random_batch(512, seed=0, max_qt_entries=QT_CAP)
    pick = [nets[i] for i in (15, 148, 205, 339)]
    kinds = set()
    for n in pick:
        dts = ["f32" if t.data.dtype == np.float32 else "f64" for t in n.tensors]
        t = lowering_text(n.inds(), n.dims(), n.output, dtypes=dts, max_intermediate_bytes=PEAK_BYTES)
        last = next(l for l in t.splitlines() if l.startswith("launch ") and " dst=-1 " in l)
        out, loop = (int(re.search(k + r"=(\d+)", last).group(1)) for k in ("out", "loop"))
        assert out <= 64 and loop >= 512, last
        kinds.add(last.split()[3])
    assert kinds == {"fast", "generic"}
    for n, h in zip(pick, _handles(pick)):
        assert rel_err(h.contract().cpu().numpy(), oracle_value(n)) <= REL_TOL
        h.close()
