"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: the all-FP64 path matches to 1e-12 (summation order only);
BF16x3 tensor-core steps to a normwise relative error of 1e-6; plain TF32
is reported, not required to meet 1e-6 (10-bit mantissa)."""
import numpy as np
import pytest

import synth
from oracle import knit, qpd, tn
from tests.gpu_util import FP64_TOL, REL_TOL, contract_gpu, oracle_value, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


@pytest.mark.parametrize("seed", [0, 3])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_tiny_knitting_equals_uncut_statevector(seed, prec):
    ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, size=48)
    exact = knit.uncut_expectation(ang)
    TA, TB = knit.subcircuit_tensors(ang)
    net = synth.HTN([synth.Tensor("QT", (0, 1), TA), synth.Tensor("QT", (0, 2), TB),
                     synth.Tensor("CT", (0,), synth.GATE_CT.copy()),
                     synth.Tensor("CT", (1, 2), synth.WIRE_CT.copy())], ())
    got, _ = contract_gpu(net, prec=prec)
    assert abs(got[0] - exact) <= 1e-12


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_hyper_networks(seed):
    net = synth.tiny_random_htn(seed, n_tensors=3 + seed % 4, n_indices=5 + seed % 4, n_output=seed % 3)
    ref = tn.brute_force(net.pairs(), net.output).ravel()
    got, _ = contract_gpu(net, prec="bf16x3")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


def test_single_tensor_and_disconnected():
    rng = np.random.default_rng(1)
    A = rng.uniform(-1, 1, (3, 4, 5))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 2), A)], (1,))
    got, _ = contract_gpu(net)
    np.testing.assert_allclose(got, A.sum(axis=(0, 2)), rtol=1e-13)
    B = rng.uniform(-1, 1, (6,))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 2), A), synth.Tensor("QT", (3,), B)], (3, 1))
    got, _ = contract_gpu(net)
    np.testing.assert_allclose(got.reshape(6, 4), np.outer(B, A.sum(axis=(0, 2))), rtol=1e-13)


GEMM_SHAPES = [(1, 128, 128, 128), (3, 300, 200, 333), (2, 64, 32, 32), (5, 144, 144, 144),
               (1, 513, 257, 1000), (7, 96, 40, 72), (4, 512, 512, 24), (2, 640, 384, 12), (9, 200, 20, 8)]


@pytest.mark.parametrize("shape", GEMM_SHAPES, ids=[str(s) for s in GEMM_SHAPES])
@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "tf32"])
def test_pairwise_gemm_shapes(shape, prec):
    """One pairwise step C[b,m,n] = sum_k A[b,m,k] B[b,k,n]: tiles, ragged
    M/N/K tails, several batches."""
    b, m, n, k = shape
    rng = np.random.default_rng(sum(shape))
    A = rng.uniform(-1, 1, (b, m, k))
    B = rng.uniform(-1, 1, (b, k, n))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2))
    got, st = contract_gpu(net, prec=prec)
    ref = np.matmul(A, B).ravel()
    err = rel_err(got, ref)
    tol = {"bf16x3": REL_TOL, "3xtf32": 1e-5, "tf32": 1e-2}[prec]
    assert err <= tol, (err, st)
    if m >= 64 and b * m * n * k >= 1 << 22:
        assert st["n_tensor_core_steps"] == 1


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_ring_small_with_tails(prec):
    # bond 144 (two gate cuts and a wire cut per edge): M, N and K are 144,
    # ragged against the 128-row tiles and 64-wide k-blocks
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=5)
    ref = oracle_value(net)
    got, st = contract_gpu(net, prec=prec)
    err = rel_err(got, ref)
    assert err <= (FP64_TOL if prec == "fp64" else REL_TOL), err
    if prec == "bf16x3":
        assert st["n_tensor_core_steps"] >= 1


def test_mid_ring_bf16x3():
    """The mid-size workload (8 QTs of [64][144][144], 16 gate + 8 wire cuts)."""
    net = synth.ring_htn()
    ref = oracle_value(net)
    got, st = contract_gpu(net, prec="bf16x3")
    err = rel_err(got, ref)
    print("mid ring bf16x3 rel err", err, st)
    assert err <= REL_TOL
    assert st["n_tensor_core_steps"] == 6


@pytest.mark.parametrize("prec", ["fp64", "tf32", "3xtf32"])
def test_mid_ring_other_precisions(prec):
    """The other precision forms on the mid-size ring, held to a few times
    their measured error on B300 (FP64 3.3e-16, 3xTF32 1.6e-6, TF32 6.3e-4):
    3xTF32 and TF32 do not meet 1e-6 and are reported, not claimed."""
    net = synth.ring_htn()
    ref = oracle_value(net)
    got, _ = contract_gpu(net, prec=prec)
    err = rel_err(got, ref)
    print(f"mid ring {prec} rel err", err)
    bound = {"fp64": FP64_TOL, "3xtf32": 5e-6, "tf32": 3e-3}[prec]
    assert err <= bound


@pytest.mark.parametrize("seed", [0, 1])
def test_signed_qpd_cts_rank1_qts_fp64_path(seed):
    """Rank-1 positive QTs contracted with the exact signed QPD coefficient
    tensors on the mid-size ring: every cut's sum cancels (the sum of
    magnitudes over the whole contraction is ~1e18 times the value), so the
    tensor-core forms lose accuracy in proportion; the FP64 path matches the
    closed form to 1e-9 (measured 1.5e-11 and 7.1e-12)."""
    from tests.test_oracle_tn import rank1_qts_closed_form
    net, fac = synth.rank1_qts_htn(synth.ring_htn(), seed=seed)
    want, mag = rank1_qts_closed_form(net, fac)
    assert np.max(mag.ravel() / np.abs(want.ravel())) > 1e15
    got, _ = contract_gpu(net, prec="fp64")
    assert rel_err(got, want.ravel()) <= 1e-9


def test_sliced_equals_unsliced():
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=5, seed=2)
    ref = oracle_value(net)
    got, st = contract_gpu(net, prec="bf16x3", n_slices=16, slice_dim=4)
    assert rel_err(got, ref) <= REL_TOL
    got64, _ = contract_gpu(net, prec="fp64", n_slices=64, slice_dim=6)
    assert rel_err(got64, ref) <= FP64_TOL


def test_fp32_leaves():
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=9, dtype=np.float32)
    ref = oracle_value(net)
    got, _ = contract_gpu(net, prec="bf16x3")
    assert rel_err(got, ref) <= REL_TOL


def test_contract_host_matches_device_path():
    import torch
    from paper_2410_15080_b300 import from_network
    from tests.gpu_util import to_device
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=4, seed=11)
    dev = to_device(net)
    h = from_network(dev, net.output, prec="bf16x3")
    d = h.contract().cpu().numpy()
    host = [torch.from_numpy(np.ascontiguousarray(t.data)).pin_memory() for t in net.tensors]
    for x in dev:  # clobber the device copies: contract_host must upload
        x[1].zero_()
    got = h.contract_host(host)
    h.close()
    np.testing.assert_array_equal(got, d)
    assert rel_err(got, oracle_value(net)) <= REL_TOL


def test_deterministic_repeat():
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=8, seed=4)
    a, _ = contract_gpu(net)
    b, _ = contract_gpu(net)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("fast", ["0", "1"])
@pytest.mark.parametrize("graph", ["0", "1"])
def test_generic_and_fast_gather_paths_agree(fast, graph, monkeypatch):
    """The typed fast gather kernels and the generic ones (and direct launches
    vs CUDA-graph replay) compute the same contraction."""
    monkeypatch.setenv("QTPU_NO_FAST", "0" if fast == "1" else "1")
    monkeypatch.setenv("QTPU_NO_GRAPH", "0" if graph == "1" else "1")
    net = synth.ring_htn(n_sub=5, gates_per_edge=2, wires_per_edge=1, k=3, seed=21)
    ref = oracle_value(net)
    got, _ = contract_gpu(net, prec="bf16x3")
    assert rel_err(got, ref) <= REL_TOL
    got64, _ = contract_gpu(net, prec="fp64")
    assert rel_err(got64, ref) <= FP64_TOL


def test_slice_ranges_sum_to_the_full_result():
    import torch
    from paper_2410_15080_b300 import from_network
    from tests.gpu_util import to_device
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=8)
    h = from_network(to_device(net), net.output, prec="bf16x3", n_slices=16, slice_dim=4)
    full = h.contract().clone()
    parts = [h.contract_slices(0, 5).clone(), h.contract_slices(5, 10).clone(), h.contract_slices(15, 1).clone()]
    h.sync()
    got = sum(p.cpu().numpy() for p in parts)
    assert rel_err(got, full.cpu().numpy()) <= 1e-12
    assert rel_err(got, oracle_value(net)) <= REL_TOL
    with pytest.raises(Exception):
        h.contract_slices(10, 7)
    h.close()


def test_skinny_m_runs_on_the_tensor_cores_with_swapped_operands():
    rng = np.random.default_rng(3)
    b, m, n, k = 4, 36, 1296, 576
    A = rng.uniform(-1, 1, (b, m, k))
    B = rng.uniform(-1, 1, (b, k, n))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2))
    got, st = contract_gpu(net, prec="bf16x3")
    assert st["n_tensor_core_steps"] == 1
    assert rel_err(got, np.matmul(A, B).ravel()) <= REL_TOL


def test_ring_with_chords_topology_sliced():
    """The 100-qubit topology (ring + chords (i, i+3)) with smaller bonds and a
    single observable, sliced over 4^3 wire values, against the oracle."""
    net = synth.ring_chords_htn(k=2, seed=4, gates_per_chord=1)
    ref = oracle_value(net)
    got, st = contract_gpu(net, prec="bf16x3", n_slices=64, slice_dim=4)
    assert rel_err(got, ref) <= REL_TOL, st


@pytest.mark.slow
def test_100q_rank1_closed_form_full_size():
    """Full-size 100-qubit network (28 gate + 12 wire cuts, k = 64, 2 GB of
    QTs, 1024 slices) with rank-1 tensors: the contraction factorises into a
    closed form computed on the CPU.  Positive factors keep the sum over
    slices well conditioned (with random signs the per-index sums cancel and
    the slice sum amplifies rounding by sum|slice| / |sum slice|)."""
    from tests.test_oracle_tn import rank1_closed_form
    base = synth.ring_chords_htn(materialize=False)
    net, fac = synth.rank1_htn(base, seed=5, signed=False)
    want = rank1_closed_form(net, fac).ravel()
    got, st = contract_gpu(net, prec="bf16x3", max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4)
    assert st["n_tensor_core_steps"] >= 5
    assert rel_err(got, want) <= REL_TOL, st


@pytest.mark.slow
@pytest.mark.parametrize("plan", ["1024 wire slices", "planner's own slices"])
def test_100q_full_size_random_signed_entries_vs_oracle(plan):
    """The full-size 100-qubit network (12 QTs, 28 gate + 12 wire cuts, k = 64,
    2 GB of QTs with signed entries ~U[-1, 1], contracted with the exact
    signed QPD coefficient tensors) against the exact FP64 oracle on the
    restricted output k in {0, 1}, element by element: the 1024-slice plan of
    the benchmark and the planner's own slicing under the 8 GB limit."""
    from tests.gpu_util import oracle_restricted
    net = synth.ring_chords_htn(seed=0)
    kw = dict(max_intermediate_bytes=8 << 30, n_candidates=256)
    if plan == "1024 wire slices":
        kw.update(n_slices=1024, slice_dim=4)
    got, st = contract_gpu(net, prec="bf16x3", **kw)
    ref = oracle_restricted(net, (0, 1))
    assert st["n_tensor_core_steps"] >= 5
    err = rel_err(got[:2], ref)
    assert err <= REL_TOL, (err, got[:2], ref, st)
    assert np.max(np.abs(got[:2] - ref)) / np.max(np.abs(ref)) <= REL_TOL


@pytest.mark.slow
def test_100q_full_size_slicing_invariance():
    """Full-size 100-qubit network with random entries: the result does not
    depend on how the contraction is sliced (1024 wire-index slices vs 256),
    which holds at any size."""
    net = synth.ring_chords_htn(seed=2)
    a, sa = contract_gpu(net, prec="bf16x3", max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4)
    b, sb = contract_gpu(net, prec="bf16x3", max_intermediate_bytes=16 << 30, n_slices=256, slice_dim=4)
    assert rel_err(a, b) <= 2 * REL_TOL, (sa, sb)


def _dot_nets():
    """Long sums over few outputs (the tiled dot kernel): operands transposed
    against each other, a tile that is not a multiple of the block, and two
    FP32-pair intermediates as operands."""
    rng = np.random.default_rng(17)
    A = rng.uniform(-1, 1, (5, 36, 6, 40))
    B = rng.uniform(-1, 1, (5, 40, 6, 36))
    yield synth.HTN([synth.Tensor("QT", (0, 1, 2, 3), A), synth.Tensor("QT", (0, 3, 2, 1), B)], (0,))
    A = rng.uniform(-1, 1, (3, 7, 13, 50))
    B = rng.uniform(-1, 1, (3, 50, 13, 7))
    yield synth.HTN([synth.Tensor("QT", (0, 1, 2, 3), A), synth.Tensor("QT", (0, 3, 2, 1), B)], (0,))
    A = rng.uniform(-1, 1, (2, 48, 32))
    B = rng.uniform(-1, 1, (32, 8, 64))
    C = rng.uniform(-1, 1, (2, 64, 8, 32))
    D = rng.uniform(-1, 1, (32, 48))
    yield synth.HTN([synth.Tensor("QT", (0, 1, 4), A), synth.Tensor("QT", (4, 2, 3), B),
                     synth.Tensor("QT", (0, 3, 2, 5), C), synth.Tensor("QT", (5, 1), D)], (0,))


@pytest.mark.parametrize("case", range(3))
def test_long_dot_reductions(case):
    net = list(_dot_nets())[case]
    ref = tn.brute_force(net.pairs(), net.output).ravel() if case < 2 else oracle_value(net)
    got, _ = contract_gpu(net, prec="bf16x3")
    assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("kc", ["1", "4", "16", "64"])
def test_bf16x3_with_magnitudes_varying_along_k_and_rows(kc, monkeypatch):
    """Entries whose magnitude changes by up to 2^24 along K and across rows,
    so neighbouring k-blocks sit on different piece grids, at several drain
    intervals (k-blocks per accumulator chunk)."""
    monkeypatch.setenv("QTPU_KC", kc)
    rng = np.random.default_rng(5)
    b, m, n, k = 2, 200, 150, 640
    sk = 2.0 ** rng.integers(-12, 13, k)
    A = rng.uniform(-1, 1, (b, m, k)) * 2.0 ** rng.integers(-12, 13, (1, m, 1)) * sk[None, None, :]
    B = rng.uniform(-1, 1, (b, k, n)) * 2.0 ** rng.integers(-12, 13, (1, 1, n)) * sk[None, ::-1, None]
    net = synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2))
    got, st = contract_gpu(net, prec="bf16x3")
    assert st["n_tensor_core_steps"] == 1
    assert rel_err(got, np.matmul(A, B).ravel()) <= REL_TOL


@pytest.mark.parametrize("mode", ["off", "k_along_columns", "k_along_rows"])
def test_epilogue_written_operand_pieces(mode, monkeypatch):
    """A GEMM whose result is the next GEMM's operand writes that operand's
    BF16x3 pieces from its epilogue, with the next K along the tile's columns
    (the layout the lowering prefers) or, with that preference off, along its
    rows; with the fusion switched off every operand goes through a split
    launch.  All match the oracle."""
    monkeypatch.setenv("QTPU_NO_FUSE", "1" if mode == "off" else "0")
    monkeypatch.setenv("QTPU_FUSE_KEEP_LAYOUT", "1" if mode == "k_along_rows" else "0")
    from paper_2410_15080_b300.htn import lowering_text
    seen = set()
    for net in (synth.ring_htn(n_sub=5, gates_per_edge=2, wires_per_edge=1, k=5, seed=23),
                synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=6),
                synth.ring_htn(seed=3)):
        t = lowering_text(net.inds(), net.dims(), net.output)
        summary = next(l for l in t.splitlines() if l.startswith("summary "))
        n_fused = int(summary.split("fused_splits=")[1].split()[0])
        assert (n_fused > 0) == (mode != "off"), summary
        seen |= {w for l in t.splitlines() for w in l.split() if w.startswith("k=")}
        got, _ = contract_gpu(net, prec="bf16x3")
        assert rel_err(got, oracle_value(net)) <= REL_TOL
    if mode == "k_along_columns":
        assert seen == {"k=N"}
    if mode == "k_along_rows":
        assert "k=M" in seen


def test_operand_split_with_a_summed_wire_index():
    """A QT with a wire CT folded in over a summed index (4 terms per operand
    entry, no fan-out) goes through the pipelined split with its loop table."""
    rng = np.random.default_rng(31)
    b, m, n, y = 8, 160, 144, 36
    A = rng.uniform(-1, 1, (b, m, 4, y))
    B = rng.uniform(-1, 1, (b, n, 4, y))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 4, 3), A), synth.Tensor("CT", (4, 5), synth.WIRE_CT.copy()),
                     synth.Tensor("QT", (0, 2, 5, 3), B)], (0, 1, 2))
    from paper_2410_15080_b300.htn import lowering_text
    t = lowering_text(net.inds(), net.dims(), net.output)
    assert any(" split " in l and " loop=4 " in l and " fan=1 " in l for l in t.splitlines()), t
    got, st = contract_gpu(net, prec="bf16x3")
    assert st["n_tensor_core_steps"] == 1
    ref = np.einsum("bmxy,xk,bnky->bmn", A, synth.WIRE_CT, B).ravel()
    assert rel_err(got, ref) <= REL_TOL


def _reuse_net():
    # ring + chords topology with smaller bonds, 16 observables: with 256 wire
    # slices 6 steps run on the tensor cores, most of them on only some of
    # the sliced indices
    return synth.ring_chords_htn(k=16, seed=9, gates_per_chord=1)


@pytest.mark.parametrize("reuse", ["all copies", "blocked", "off"])
def test_slice_reuse_matches_oracle(reuse, monkeypatch):
    """Slice reuse with every copy kept, with some sliced indices held fixed
    in an outer loop (a small budget), and off (one slice at a time): all
    give the oracle's value, and the same bits on a second call; with reuse
    the contraction executes fewer FLOPs than the plan's total.  (The blocked
    case sizes its budget from the workspace, so kept split results, which
    the workspace also holds, are off there.)"""
    from paper_2410_15080_b300.htn import HTN, lowering_text
    if reuse == "blocked":
        monkeypatch.setenv("QTPU_NO_KEPT_SPLITS", "1")
    net = _reuse_net()
    ref = oracle_value(net)
    kw = dict(n_slices=256, slice_dim=4)
    probe = HTN(device=-1)
    for t in net.tensors:
        probe.add_tensor(t.inds, list(t.data.shape))
    probe.set_output(net.output)
    probe.plan("bf16x3", **kw)
    full = probe.exec_stats()
    ws = probe.plan_stats()["workspace_bytes"]
    probe.close()
    assert full["kept_bytes"] > 0
    t = lowering_text(net.inds(), net.dims(), net.output, **kw)
    assert sum(" gemm " in l and " din=-" not in l for l in t.splitlines()) >= 3
    budget = {"all copies": 0, "blocked": ws - full["kept_bytes"] // 2, "off": 1}[reuse]
    import torch
    from paper_2410_15080_b300 import from_network
    from tests.gpu_util import to_device
    h = from_network(to_device(net), net.output, prec="bf16x3", reuse_bytes=budget, **kw)
    st = h.exec_stats()
    out = h.contract()
    h.sync()
    got = out.cpu().numpy()
    out2 = h.contract()
    h.sync()
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), got)
    h.close()
    assert rel_err(got, ref) <= REL_TOL, st
    if reuse == "off":
        assert st["kept_bytes"] == 0 and st["flops_executed"] == pytest.approx(st["flops_all_slices"])
    else:
        assert 0 < st["kept_bytes"] and st["flops_executed"] < st["flops_all_slices"]
    if reuse == "blocked":
        assert st["kept_bytes"] < full["kept_bytes"] and st["flops_executed"] > full["flops_executed"]


def test_slice_ranges_with_reuse_add_up():
    """Slice ranges (run as aligned blocks of the slice space) add up to the
    full contraction; both match the oracle (their sums over sliced indices
    are added in different orders, so they agree to rounding, not bits)."""
    import torch
    from paper_2410_15080_b300 import from_network
    from tests.gpu_util import to_device
    net = _reuse_net()
    h = from_network(to_device(net), net.output, prec="bf16x3", n_slices=256, slice_dim=4)
    full = h.contract().clone()
    parts = [h.contract_slices(a, b - a).clone() for a, b in [(0, 37), (37, 200), (200, 256)]]
    h.sync()
    torch.cuda.synchronize()
    tot = sum(p.cpu().numpy() for p in parts)
    h.close()
    ref = oracle_value(net)
    assert rel_err(tot, ref) <= REL_TOL
    assert rel_err(full.cpu().numpy(), ref) <= REL_TOL
    assert rel_err(tot, full.cpu().numpy()) <= 2 * REL_TOL


def test_sliced_mid_ring_with_reuse_and_epilogue_pieces():
    """The mid-size ring sliced over 4^2 wire values: under slice reuse three
    GEMM epilogues write the next operand's pieces in 4 copies (one per value
    of the sliced index they depend on), read through one tensor map per
    copy; the result matches the oracle."""
    from paper_2410_15080_b300.htn import lowering_text
    net = synth.ring_htn(seed=3)
    t = lowering_text(net.inds(), net.dims(), net.output, n_slices=16, slice_dim=4)
    assert sum("writes-pieces" in l and " din=-" not in l for l in t.splitlines()) >= 2
    got, st = contract_gpu(net, prec="bf16x3", n_slices=16, slice_dim=4)
    assert rel_err(got, oracle_value(net)) <= REL_TOL, st
