"""Failure detection without a GPU fault: a bounded device-side wait that
nothing satisfies gives up after its limit, the host reads QTPU_ETIMEOUT from
the status word, and the same handle keeps contracting correctly."""
import time

import pytest

import synth
from tests.gpu_util import REL_TOL, contract_gpu, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def test_bounded_wait_times_out_and_context_stays_usable():
    import torch
    from paper_2410_15080_b300 import from_network, htn
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=6)
    h = from_network(to_device(net), net.output, prec="bf16x3")
    h.contract()
    h.sync()
    t0 = time.perf_counter()
    h.selftest_timeout(50_000_000)  # 50 ms
    with pytest.raises(htn.QtpuError) as e:
        h.sync()
    dt = time.perf_counter() - t0
    assert e.value.status == htn.QTPU_ETIMEOUT
    assert 0.04 <= dt < 5.0
    h.sync()  # reported once
    out = h.contract()
    h.sync()
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), oracle_value(net)) <= REL_TOL
    h.close()


@pytest.mark.parametrize("pair", [0, 1], ids=["one-cta", "cta-pair"])
def test_gemm_waits_time_out_and_context_stays_usable(pair):
    """The tensor-core GEMM's own bounded waits: a launch whose producer
    issues no copies (the self-test flag) gives up in the MMA issuer and the
    epilogue after 50 ms, frees its TMEM (on a CTA pair, both CTAs' share)
    and returns; the host reads QTPU_ETIMEOUT, and the same handle then
    contracts correctly through the GEMM path."""
    import torch
    from paper_2410_15080_b300 import from_network, htn
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=6)
    h = from_network(to_device(net), net.output, prec="bf16x3")
    assert h.plan_stats()["n_tensor_core_steps"] > 0
    h.contract()
    h.sync()
    t0 = time.perf_counter()
    h.selftest_gemm_timeout(pair, 50_000_000)  # 50 ms
    with pytest.raises(htn.QtpuError) as e:
        h.sync()
    dt = time.perf_counter() - t0
    assert e.value.status == htn.QTPU_ETIMEOUT
    assert 0.04 <= dt < 5.0
    h.sync()  # reported once
    out = h.contract()
    h.sync()
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), oracle_value(net)) <= REL_TOL
    h.close()


def test_injected_workspace_allocation_failure_is_enomem(monkeypatch):
    from paper_2410_15080_b300 import from_network, htn
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=2, seed=1)
    monkeypatch.setenv("QTPU_TEST_FAIL_ALLOC", "1")
    with pytest.raises(htn.QtpuError) as e:
        from_network(to_device(net), net.output)
    assert e.value.status == htn.QTPU_ENOMEM
    monkeypatch.setenv("QTPU_TEST_FAIL_ALLOC", "0")
    got, _ = contract_gpu(net)
    assert rel_err(got, oracle_value(net)) <= REL_TOL
