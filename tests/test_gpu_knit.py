"""Naive circuit knitting on the GPU (Eq. knitting, section 2.1): the sum
over every global instance against the oracle's brute force, the tiny
knitting circuit's exact expectation value, and the h-TN contraction."""
import numpy as np
import pytest

import synth
from oracle import knit, tn
from tests.gpu_util import FP64_TOL, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def _handle(net):
    from paper_2410_15080_b300.htn import HTN
    h = HTN(0)
    for inds, data, kind in to_device(net):
        h.add_tensor(inds, data=data, kind=kind)
    h.set_output(net.output)
    return h


@pytest.mark.parametrize("seed", [0, 3])
def test_tiny_circuit_knitting(seed):
    ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, size=48)
    TA, TB = knit.subcircuit_tensors(ang)
    net = synth.HTN([synth.Tensor("QT", (0, 1), TA), synth.Tensor("QT", (0, 2), TB),
                     synth.Tensor("CT", (0,), synth.GATE_CT.copy()),
                     synth.Tensor("CT", (1, 2), synth.WIRE_CT.copy())], ())
    h = _handle(net)
    out, ni = h.knit_naive()
    h.close()
    assert ni == 6 * 4 * 4
    got = float(out.cpu()[0])
    assert abs(got - knit.knit_brute_force(TA, TB, synth.GATE_CT, synth.WIRE_CT)) <= 1e-13
    assert abs(got - knit.uncut_expectation(ang)) <= 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_random_hyper_networks(seed):
    net = synth.tiny_random_htn(seed, n_tensors=3 + seed % 3, n_indices=6, n_output=seed % 3)
    h = _handle(net)
    out, _ = h.knit_naive()
    h.close()
    ref = tn.brute_force(net.pairs(), net.output).ravel()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_ring_equals_the_contraction(dtype):
    """A 3-subcircuit ring, 1 gate + 1 wire cut per edge, 4 observables:
    (6 * 16)^3 = 884,736 instances per output."""
    import torch
    net = synth.ring_htn(n_sub=3, gates_per_edge=1, wires_per_edge=1, k=4, seed=1, dtype=dtype)
    h = _handle(net)
    out, ni = h.knit_naive()
    assert ni == 96 ** 3
    naive = out.cpu().numpy()
    h.plan("fp64")
    c = h.contract()
    h.sync()
    torch.cuda.synchronize()
    h.close()
    ref = oracle_value(net)
    assert rel_err(naive, ref) <= FP64_TOL
    assert rel_err(c.cpu().numpy(), naive) <= FP64_TOL


def test_limits():
    from paper_2410_15080_b300.htn import QTPU_ENOTSUP, QtpuError
    net = synth.ring_htn(n_sub=8, gates_per_edge=2, wires_per_edge=1, k=2, seed=0)
    h = _handle(net)
    with pytest.raises(QtpuError) as e:
        h.knit_naive()  # 6^16 * 16^8 instances
    h.close()
    assert e.value.status == QTPU_ENOTSUP
