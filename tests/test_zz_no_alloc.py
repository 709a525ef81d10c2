"""GPU test of qtpu_pairwise_contract_noalloc, the entry point for callers that
cannot allocate device memory at call time (a pre-sized memory pool owned by
someone else, a latency-critical loop where cudaMalloc would stall, a C
caller without an allocator).  It must give the same result as the regular
entry point (qtpu_htn_contract on the same two-tensor network), call after
call, while taking all its scratch from the library's fixed device array.

This file is collected last on purpose: a run that stops at the first
failure has run every other test before it."""
import numpy as np
import pytest

from tests.gpu_util import REL_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def _regular(A, B):
    """The same product through the planned-network entry point."""
    import torch
    from paper_2410_15080_b300 import from_network
    h = from_network([((0, 1, 3), A), ((0, 3, 2), B)], (0, 1, 2), prec="bf16x3")
    out = h.contract()
    h.sync()
    torch.cuda.synchronize()
    h.close()
    return out.reshape(A.shape[0], A.shape[1], B.shape[2])


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    import torch
    from paper_2410_15080_b300 import htn
    g = torch.Generator(device="cuda").manual_seed(7)
    # two calls in a row with different shapes: several tiles, ragged M/N/K
    for (b, m, n, k) in [(64, 144, 144, 144), (3, 300, 200, 333)]:
        A = torch.rand(b, m, k, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        B = torch.rand(b, k, n, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        C = torch.full((b, m, n), float("nan"), dtype=torch.float64, device="cuda")
        htn.pairwise_contract_noalloc(A, B, C)
        htn.noalloc_status()  # no device-side failure recorded
        torch.cuda.synchronize()
        ref = _regular(A, B)
        assert rel_err(C.cpu().numpy(), ref.cpu().numpy()) <= REL_TOL
        exact = torch.bmm(A, B)
        assert rel_err(C.cpu().numpy(), exact.cpu().numpy()) <= REL_TOL


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import ctypes as C
    import torch
    from paper_2410_15080_b300 import htn
    L = htn.lib()
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 8 * 1 * 4096 * 4096 bytes of product alone exceed 32 MiB
    st = L.qtpu_pairwise_contract_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()),
                                          C.c_void_p(A.data_ptr()), 1, 4096, 4096, 8, None)
    assert st == htn.QTPU_ELIMIT
    st = L.qtpu_pairwise_contract_noalloc(None, C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()),
                                          1, 4, 4, 4, None)
    assert st == htn.QTPU_EINVAL


def test_noalloc_scratch_boundary():
    """The largest call that fits the fixed scratch succeeds; one more row of A
    is refused with ELIMIT before anything is enqueued."""
    import ctypes as C
    import torch
    from paper_2410_15080_b300 import htn
    L = htn.lib()
    cap = 32 << 20
    # largest M (batch 1, N 8, K 8) that fits, found on the host only
    lo, hi = 1, 1 << 20
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if htn.noalloc_scratch_bytes(1, mid, 8, 8) <= cap:
            lo = mid
        else:
            hi = mid - 1
    m = lo
    assert htn.noalloc_scratch_bytes(1, m, 8, 8) <= cap < htn.noalloc_scratch_bytes(1, m + 1, 8, 8)
    # the header's stated bound holds for every size checked
    for (b, mm, n, k) in [(1, m, 8, 8), (3, 300, 200, 333), (64, 144, 144, 144), (1, 1, 1, 1)]:
        kp = (k + 7) // 8 * 8
        assert htn.noalloc_scratch_bytes(b, mm, n, k) <= 2304 + 6 * b * (mm + n) * kp + 8 * b * mm * n
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.rand(1, m, 8, dtype=torch.float64, device="cuda", generator=g) - 0.5
    B = torch.rand(1, 8, 8, dtype=torch.float64, device="cuda", generator=g) - 0.5
    Cm = torch.empty(1, m, 8, dtype=torch.float64, device="cuda")
    htn.pairwise_contract_noalloc(A, B, Cm)
    htn.noalloc_status()
    assert rel_err(Cm.cpu().numpy(), torch.bmm(A, B).cpu().numpy()) <= REL_TOL
    A2 = torch.zeros(1, m + 1, 8, dtype=torch.float64, device="cuda")
    C2 = torch.zeros(1, m + 1, 8, dtype=torch.float64, device="cuda")
    st = L.qtpu_pairwise_contract_noalloc(C.c_void_p(A2.data_ptr()), C.c_void_p(B.data_ptr()),
                                          C.c_void_p(C2.data_ptr()), 1, m + 1, 8, 8, None)
    assert st == htn.QTPU_ELIMIT
    assert b"scratch" in L.qtpu_last_error(None)


def test_noalloc_status_reports_a_timed_out_wait():
    """A bounded device wait that gives up is reported by qtpu_noalloc_status
    (once), and the entry point keeps working afterwards.  The wait is on a
    barrier nothing completes and ends by its own time limit: no fault."""
    import ctypes as C
    import torch
    from paper_2410_15080_b300 import htn
    L = htn.lib()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.qtpu_noalloc_selftest_timeout(50_000_000, C.c_void_p(stream)) == htn.QTPU_OK
    with pytest.raises(htn.QtpuError) as ei:
        htn.noalloc_status()
    assert ei.value.status == htn.QTPU_ETIMEOUT
    htn.noalloc_status()  # reported once
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.rand(2, 130, 70, dtype=torch.float64, device="cuda", generator=g) - 0.5
    B = torch.rand(2, 70, 90, dtype=torch.float64, device="cuda", generator=g) - 0.5
    Cm = torch.empty(2, 130, 90, dtype=torch.float64, device="cuda")
    htn.pairwise_contract_noalloc(A, B, Cm)
    htn.noalloc_status()
    assert rel_err(Cm.cpu().numpy(), torch.bmm(A, B).cpu().numpy()) <= REL_TOL
