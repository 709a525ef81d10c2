"""Batched contraction of many independent h-TNs of uneven size in one CUDA
graph (random ring / 2-D-grid networks, FP32 and FP64 leaves) against the
FP64 oracle and against one-by-one contraction."""
import numpy as np
import pytest

import synth
from tests.gpu_util import REL_TOL, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def test_batch_of_uneven_networks():
    import torch
    from paper_2410_15080_b300 import contract_batch, from_network
    nets = synth.random_batch(40, seed=3)
    assert len({n.meta["topology"] for n in nets}) == 2
    assert {t.data.dtype for n in nets for t in n.tensors} == {np.dtype(np.float32), np.dtype(np.float64)}
    hs = [from_network(to_device(n), n.output, prec="bf16x3") for n in nets]
    outs = [torch.full((h.output_size(),), float("nan"), dtype=torch.float64, device="cuda") for h in hs]
    contract_batch(hs, outs)
    torch.cuda.synchronize()
    one = [h.contract().cpu().numpy() for h in hs]
    torch.cuda.synchronize()
    for n, o, s in zip(nets, outs, one):
        got = o.cpu().numpy()
        np.testing.assert_array_equal(got, s)  # same kernels, same order
        assert rel_err(got, oracle_value(n)) <= REL_TOL
    # replay of the cached graph
    for o in outs:
        o.fill_(float("nan"))
    contract_batch(hs, outs)
    torch.cuda.synchronize()
    for o, s in zip(outs, one):
        np.testing.assert_array_equal(o.cpu().numpy(), s)
    for h in hs:
        h.close()
