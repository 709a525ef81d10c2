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
