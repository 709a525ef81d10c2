"""C-ABI checks that need no GPU: the library loads, exports every entry
point the header declares, plans bit-exactly like the reference planner,
and reports argument and state errors as status codes."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import planner
from paper_2410_15080_b300 import build, htn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "qtpu_htn.h")).read()
    declared = set(re.findall(r"\b(qtpu_\w+)\s*\(", hdr))
    assert declared, "no declarations found"
    L = htn.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(htn.SYMBOLS)


def _ref_text(net_inds, dims, output, **kw):
    p = planner.make_plan(net_inds, dims, output, kw.get("max_intermediate_bytes", 0),
                          kw.get("n_slices", 0), kw.get("slice_dim", 0), kw.get("seed", 0),
                          kw.get("n_candidates", 0))
    return planner.plan_text(p, net_inds)


CASES = [
    ("ring8", lambda: synth.ring_htn(), {}),
    ("ring4_sliced", lambda: synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=8),
     {"n_slices": 16, "slice_dim": 4}),
    ("ring5_limit", lambda: synth.ring_htn(n_sub=5, gates_per_edge=1, wires_per_edge=2, k=3),
     {"max_intermediate_bytes": 20000}),
    ("chords100q", lambda: synth.ring_chords_htn(materialize=False), {}),
    ("chords100q_sliced", lambda: synth.ring_chords_htn(materialize=False),
     {"max_intermediate_bytes": 8 << 30, "n_slices": 1024, "slice_dim": 4}),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_planner_bit_exact(name, make, kw):
    net = make()
    got = htn.plan_text(net.inds(), net.dims(), net.output, **kw)
    assert got == _ref_text(net.inds(), net.dims(), net.output, **kw)


@pytest.mark.parametrize("seed", range(40))
def test_planner_bit_exact_random(seed):
    if seed < 20:
        net = synth.tiny_random_htn(seed, n_tensors=3 + seed % 5, n_indices=4 + seed % 6,
                                    n_output=seed % 3)
    else:
        net = synth.random_htn(seed)
    got = htn.plan_text(net.inds(), net.dims(), net.output)
    assert got == _ref_text(net.inds(), net.dims(), net.output)


def test_status_codes():
    h = htn.HTN(device=-1)
    with pytest.raises(htn.QtpuError) as e:
        h.plan()
    assert e.value.status == htn.QTPU_ESTATE
    h.add_tensor([0, 1], [2, 3])
    with pytest.raises(htn.QtpuError) as e:
        h.add_tensor([1], [4])  # dim mismatch for index 1
    assert e.value.status == htn.QTPU_EINVAL
    with pytest.raises(htn.QtpuError) as e:
        h.add_tensor([2, 2], [2, 2])  # repeated id
    assert e.value.status == htn.QTPU_EINVAL
    with pytest.raises(htn.QtpuError) as e:
        h.add_tensor([3], [0])
    assert e.value.status == htn.QTPU_EINVAL
    h.add_tensor([1, 2], [3, 5])
    h.set_output([7])
    with pytest.raises(htn.QtpuError) as e:
        h.plan()  # output index on no tensor
    assert e.value.status == htn.QTPU_EINVAL
    h.close()

    h = htn.HTN(device=-1)
    h.add_tensor([0, 1], [2, 3])
    h.add_tensor([1, 2], [3, 5])
    h.set_output([0])
    with pytest.raises(htn.QtpuError) as e:
        h.plan(max_intermediate_bytes=8)  # cannot slice below one entry per step
    assert e.value.status == htn.QTPU_ELIMIT
    h.close()

    h = htn.HTN(device=-1)
    h.add_tensor([0, 1], [2, 3])
    h.add_tensor([1, 2], [3, 5])
    h.set_output([0, 2])
    h.plan()
    assert h.output_size() == 10
    with pytest.raises(htn.QtpuError) as e:
        h.add_tensor([4], [2])
    assert e.value.status == htn.QTPU_ESTATE
    L = htn.lib()
    import ctypes as C
    st = L.qtpu_htn_contract(h._h, C.c_void_p(1))
    assert st == htn.QTPU_ENOTSUP
    # the failure-path self-tests need a device handle
    assert L.qtpu_htn_selftest_timeout(h._h, 1000) == htn.QTPU_ESTATE
    assert L.qtpu_htn_selftest_gemm_timeout(h._h, 0, 1000) == htn.QTPU_ESTATE
    h.close()


def test_overflow_is_enotsup():
    # four tensors of 15 open indices of dim 60000 each, all kept: the
    # result has 60000^60 entries, far beyond 2^255
    h = htn.HTN(device=-1)
    ids = list(range(60))
    for t in range(4):
        h.add_tensor(ids[15 * t:15 * t + 15] + [100], [60000] * 15 + [2])
    h.set_output(ids)
    with pytest.raises(htn.QtpuError) as e:
        h.plan()
    assert e.value.status == htn.QTPU_ENOTSUP


@pytest.mark.parametrize("seed", [1, 2, 3, 12345, 2 ** 63 + 5])
@pytest.mark.parametrize("net_id", ["ring8", "rand7", "chords"])
def test_randomised_planner_bit_exact(seed, net_id):
    net = {"ring8": lambda: synth.ring_htn(), "rand7": lambda: synth.random_htn(7),
           "chords": lambda: synth.ring_chords_htn(materialize=False)}[net_id]()
    kw = {"seed": seed, "n_slices": 16, "slice_dim": 4} if net_id == "chords" else {"seed": seed}
    got = htn.plan_text(net.inds(), net.dims(), net.output, **kw)
    assert got == _ref_text(net.inds(), net.dims(), net.output, **kw)


def test_splitmix64_reference_values():
    # the first outputs of the published SplitMix64 reference implementation
    # seeded with 1234567
    s, outs = 1234567, []
    for _ in range(3):
        s, r = planner.splitmix64(s)
        outs.append(r)
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423]


@pytest.mark.parametrize("net_id", ["ring8", "rand5", "chords"])
def test_best_of_candidates_planner_bit_exact(net_id):
    net = {"ring8": lambda: synth.ring_htn(), "rand5": lambda: synth.random_htn(5),
           "chords": lambda: synth.ring_chords_htn(materialize=False)}[net_id]()
    kw = {"n_candidates": 12, "seed": 0}
    if net_id == "chords":
        kw.update(max_intermediate_bytes=8 << 30)
    got = htn.plan_text(net.inds(), net.dims(), net.output, **kw)
    assert got == _ref_text(net.inds(), net.dims(), net.output, **kw)
    assert "search candidates=12" in got
    # never worse than the greedy plan under the same options
    kw0 = {k: v for k, v in kw.items() if k != "n_candidates"}
    g = htn.plan_text(net.inds(), net.dims(), net.output, **kw0)
    tot = lambda t: int(t.split("flops_total=")[1].split()[0])  # noqa: E731
    assert tot(got) <= tot(g)


def test_long_sum_over_few_outputs_lowers_to_the_tiled_dot():
    """A batched dot whose operands run along different unit-stride indices is
    tiled over both (36 x 40 entries here), one block range per output."""
    import synth
    from paper_2410_15080_b300.htn import lowering_text
    rng = np.random.default_rng(0)
    A = rng.uniform(-1, 1, (5, 36, 6, 40))
    B = rng.uniform(-1, 1, (5, 40, 6, 36))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 2, 3), A), synth.Tensor("QT", (0, 3, 2, 1), B)], (0,))
    t = lowering_text(net.inds(), net.dims(), net.output)
    line = [l for l in t.splitlines() if l.startswith("launch 0")][0]
    assert " dot tile=1440 outer=6 " in line


def test_mid_ring_lowering_writes_operands_from_gemm_epilogues():
    """On the 8-QT ring every GEMM result but the last feeds the next GEMM
    with K equal to one of its index groups: 5 operands are written in piece
    form by the producing epilogue, leaving 16 launches per slice."""
    import synth
    from paper_2410_15080_b300.htn import lowering_text
    net = synth.ring_htn()
    t = lowering_text(net.inds(), net.dims(), net.output)
    summary = next(l for l in t.splitlines() if l.startswith("summary "))
    assert "tensor_core_steps=6" in summary and "fused_splits=5" in summary, summary
    assert "launches_per_slice=16" in summary, summary
    # each producer stores the next step's K as its column (N) group
    assert sum("writes-pieces k=N" in l for l in t.splitlines()) == 5


def test_100q_absorptions_lower_to_the_typed_fast_path():
    """In the 100-qubit plan, a QT absorbs five small CTs whose joint index
    table would exceed the shared-memory limit; one CT is then read as a
    second large operand and the step takes the typed fast path (its W table
    is computed once per launch)."""
    import synth
    from paper_2410_15080_b300.htn import lowering_text
    net = synth.ring_chords_htn(materialize=False)
    t = lowering_text(net.inds(), net.dims(), net.output, max_intermediate_bytes=8 << 30, n_slices=1024,
                      slice_dim=4, n_candidates=256)
    lines = [l for l in t.splitlines() if l.startswith("launch") and " contract " in l and " ops=6 " in l]
    assert lines, t
    assert all(" fast " in l and " big=2 " in l for l in lines), lines
    assert all(" generic " not in l for l in t.splitlines())


def _host_handle(net, **plan_kw):
    from paper_2410_15080_b300.htn import HTN
    h = HTN(device=-1)
    for t in net.tensors:
        h.add_tensor(t.inds, list(t.data.shape))
    h.set_output(net.output)
    h.plan("bf16x3", **plan_kw)
    return h


def test_slice_reuse_executes_each_distinct_value_once():
    """Slice reuse on the 100-qubit 1024-slice plan.  A launch runs once per
    value of the sliced indices its inputs still depend on (a step that
    contracts a sliced index adds up over its values), so a contraction
    executes the FLOPs of the same contraction tree unsliced: the plan's
    per-slice FLOPs of each step times the values of the sliced indices among
    its operands' indices, far below the plan's total.  With reuse off every
    slice is computed in full."""
    import synth
    from oracle import planner
    net = synth.ring_chords_htn(materialize=False)
    kw = dict(max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4, n_candidates=256)
    h = _host_handle(net, **kw)
    st = h.exec_stats()
    plan_total = h.plan_stats()["flops_total"]
    t = h.lowering_info()
    ptext = h.plan_info()
    h.close()
    assert st["flops_all_slices"] == pytest.approx(plan_total, rel=1e-12)
    # the unsliced FLOPs of the plan's own tree, from the oracle planner's cost
    # rule (every index at its full dim)
    dims = net.dims()
    tensors = {i: tuple(x) for i, x in enumerate(net.inds())}
    unsliced = 0
    for l in ptext.splitlines():
        f = l.split()
        if f[0] != "step":
            continue
        x, y, o = int(f[2]), int(f[3]), int(f[5])
        g = {k: () if v == "-" else tuple(int(i) for i in v.split(",")) for k, v in
             (w.split("=") for w in f[6:12])}
        unsliced += planner.step_flops(dims, tensors[x], tensors[y], g["batch"], g["m"], g["n"], g["k"],
                                       g["sa"], g["sb"])
        tensors[o] = g["batch"] + g["m"] + g["n"]
    assert unsliced < plan_total / 25
    # the executor attributes absorbed CT steps to the launch that folds them
    # in, which may loop over more slice values: at most a sliver above
    assert unsliced <= st["flops_executed"] <= 1.001 * unsliced
    # the executed FLOPs recomputed from the launch list: FLOPs times runs; a
    # main launch runs once per value of its din, a split at least that often
    fe, n_launch = 0.0, 1
    for l in t.splitlines():
        if not l.startswith("launch "):
            continue
        f = dict(w.split("=", 1) for w in l.split() if "=" in w)
        runs = int(f["runs"])
        din = [] if f["din"] == "-" else f["din"].split(",")
        dout = [] if f["dout"] == "-" else f["dout"].split(",")
        if " split " in l:
            assert runs >= 4 ** len(din)
        else:
            assert runs == 4 ** len(din)
        if " gemm " in l:
            # one launch sums the values of the sliced indices it contracts
            assert int(f["launches"]) == runs // 4 ** (len(din) - len(dout))
        else:
            assert int(f["launches"]) == runs
        fe += int(f["flops"]) * runs
        n_launch += int(f["launches"])
    assert fe == pytest.approx(st["flops_executed"], rel=1e-12)
    assert n_launch == st["launches"]
    h2 = _host_handle(net, reuse_bytes=1, **kw)
    st2 = h2.exec_stats()
    h2.close()
    assert st2["flops_executed"] == pytest.approx(plan_total, rel=1e-12) and st2["kept_bytes"] == 0


def test_slice_reuse_budget_blocks_sliced_indices():
    """Under a budget below the all-copies layout, some sliced indices are
    held fixed in an outer loop: the workspace respects the budget and the
    executed FLOPs lie between the unlimited-reuse and no-reuse figures."""
    import synth
    net = synth.ring_chords_htn(materialize=False)
    kw = dict(max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4, n_candidates=256)
    full = _host_handle(net, **kw)
    sf = full.exec_stats()
    wf = full.plan_stats()["workspace_bytes"]
    full.close()
    budget = (wf - sf["kept_bytes"]) + sf["kept_bytes"] // 3
    h = _host_handle(net, reuse_bytes=budget, **kw)
    s = h.exec_stats()
    t = h.lowering_info()
    h.close()
    assert "reuse blocked=-" not in t
    assert s["kept_bytes"] < sf["kept_bytes"]
    assert sf["flops_executed"] < s["flops_executed"] < sf["flops_all_slices"]


def test_launch_features_of_the_lowered_launch_list():
    """One feature row per launch of the launch list (kind one-hot, work,
    shape, tile fill), with the kernel launches per contraction of each; the
    learned cost model needs a device handle."""
    import synth
    from paper_2410_15080_b300.htn import HTN, QtpuError, QTPU_ENOTSUP
    net = synth.ring_htn()
    h = _host_handle(net)
    f, n = h.launch_features()
    t = h.lowering_info()
    launches = [l for l in t.splitlines() if l.startswith("launch ")]
    assert f.shape == (len(launches), 32) and (n == 1).all()
    kinds = f[:, :6].argmax(1)
    assert (f[:, :6].sum(1) == 1).all() and (f[:, 31] == 1).all()
    for row, k, l in zip(f, kinds, launches):
        if " gemm " in l:
            assert k == 0 and 0 < row[18] <= 1 and 0 < row[20] <= 1
        elif " split " in l:
            assert k == 1
    assert sum(" gemm " in l for l in launches) == int((kinds == 0).sum()) == 6
    h.close()
    h2 = HTN(device=-1)
    for tt in net.tensors:
        h2.add_tensor(tt.inds, list(tt.data.shape))
    h2.set_output(net.output)
    with pytest.raises(QtpuError) as ei:
        h2.plan("bf16x3", cost_model=1)
    assert ei.value.status == QTPU_ENOTSUP
    h2.close()


def _gemm_launches(h):
    """batch, M, N, K and bn of every GEMM launch of the lowered plan"""
    out = []
    for line in h.lowering_info().splitlines():
        f = line.split()
        if len(f) > 2 and f[2] == "gemm":
            d = {k: int(v) for k, v in (w.split("=", 1) for w in f if "=" in w)
                 if k in ("batch", "M", "N", "K", "bn")}
            d["pair"] = int("pair" in f)
            out.append(d)
    return out


def _one_gemm_net(b=2, m=300, n=200, k=333):
    A = np.zeros((b, m, k))
    B = np.zeros((b, k, n))
    return synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2))


def test_tile_table_sets_orientation_and_n_tile(tmp_path):
    """A tile table entry (keyed either way round) decides the GEMM's
    orientation and N tile; without one the padding rule decides."""
    net = _one_gemm_net()
    for swap, bn in [(0, 48), (1, 80), (1, 128), (0, 112)]:
        path = tmp_path / "t.txt"
        path.write_text(f"# comment\n3 2 300 200 333 : {swap} {bn} 0.1 0.2\n3 2 200 300 333 : {1 - swap} {bn}\n")
        h = _host_handle(net, autotune_table=str(path))
        g = _gemm_launches(h)
        h.close()
        assert len(g) == 1 and g[0]["bn"] == bn and g[0]["M"] == (200 if swap else 300), g
    # padding rule: M = 300 -> 3 row tiles, N = 200 -> 2 tiles of 112
    # columns, 6 x (112 + 128); 128-column tiles weigh 6 x 256, and 300 along
    # the N tile takes 2 row tiles x 3 tiles of 112 (or 4 of 80)
    h = _host_handle(net, autotune_table="")
    g = _gemm_launches(h)
    h.close()
    assert g[0]["bn"] == 112 and g[0]["M"] == 300 and g[0]["pair"] == 0


def test_tile_table_sets_the_cta_pair_form(tmp_path):
    """The table's last field selects 256-row tiles on a pair of CTAs for a
    BF16x3 GEMM; an entry without it, and the padding rule, keep one CTA per
    tile."""
    net = _one_gemm_net()
    for pair in (0, 1):
        path = tmp_path / "t.txt"
        path.write_text(f"3 2 300 200 333 : 0 64 0.1 0.2 0.3 {pair}\n")
        h = _host_handle(net, autotune_table=str(path))
        g = _gemm_launches(h)
        h.close()
        assert len(g) == 1 and g[0]["bn"] == 64 and g[0]["M"] == 300 and g[0]["pair"] == pair, g


@pytest.mark.parametrize("bn", [160, 144])
def test_tile_table_takes_the_wide_one_cta_tiles(tmp_path, bn):
    """BF16x3 on one CTA also runs 160-column (the width of the fused-split
    producer) and 144-column tiles: a table entry selects one for a plain
    GEMM."""
    net = _one_gemm_net()
    path = tmp_path / f"t{bn}.txt"
    path.write_text(f"3 2 300 200 333 : 0 {bn} 0.1 0.2 0.3 0\n")
    h = _host_handle(net, autotune_table=str(path))
    g = _gemm_launches(h)
    h.close()
    assert len(g) == 1 and g[0]["bn"] == bn and g[0]["M"] == 300 and g[0]["pair"] == 0, g


def test_malformed_tile_table_is_rejected(tmp_path):
    net = _one_gemm_net()
    for text in ["3 2 300 200 333 : 1 100\n", "3 2 300 200 : 1 128\n", "3 2 300 200 333 : 2 128\n",
                 "3 2 300 200 333 : 0 128 1 1 1 2\n", "1 2 300 200 333 : 0 128 1 1 1 1\n",
                 "1 2 300 200 333 : 0 160 1 1 1 0\n", "3 2 300 200 333 : 0 160 1 1 1 1\n",
                 "2 2 300 200 333 : 0 144 1 1 1 0\n", "3 2 300 200 333 : 0 144 1 1 1 1\n"]:
        path = tmp_path / "bad.txt"
        path.write_text(text)
        with pytest.raises(htn.QtpuError) as e:
            _host_handle(net, autotune_table=str(path))
        assert e.value.status == htn.QTPU_EINVAL
    with pytest.raises(htn.QtpuError) as e:
        _host_handle(net, autotune_table=str(tmp_path / "missing.txt"))
    assert e.value.status == htn.QTPU_EINVAL


def test_autotune_needs_a_device_handle(tmp_path):
    h = _host_handle(_one_gemm_net())
    with pytest.raises(htn.QtpuError) as e:
        h.autotune(str(tmp_path / "t.txt"))
    h.close()
    assert e.value.status == htn.QTPU_ENOTSUP


def test_padding_rule_on_the_100_qubit_plan():
    """The 4-pair GEMMs of the 100-qubit plan (m = 216, n = 7776) run with
    the 7776 side along the 128-row tiles and 216 in two 112-column tiles;
    the 1296 x 1296 steps keep 128 columns (11 x 11 tiles of 256 against
    11 x 12 of 240), the 144 x 5184 steps take 80."""
    net = synth.ring_chords_htn(materialize=False)
    h = _host_handle(net, max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4, n_candidates=256,
                     autotune_table="")
    g = _gemm_launches(h)
    h.close()
    shapes = {(x["M"], x["N"], x["K"], x["bn"]) for x in g}
    assert (7776, 216, 216, 112) in shapes
    assert (1296, 1296, 576, 128) in shapes
    assert (5184, 144, 36, 80) in shapes


def test_exact_order_search_matches_the_oracle():
    """search = 2: the exact tree (absorption, subset DP, post order, slicing)
    has the oracle's plan text byte for byte."""
    import synth
    from oracle import order_search
    cases = [(synth.ring_htn(), {}),
             (synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=2), {"max_intermediate_bytes": 4096}),
             (synth.ring_chords_htn(materialize=False),
              {"max_intermediate_bytes": 8 << 30, "n_slices": 1024, "slice_dim": 4})]
    for net, kw in cases:
        h = _host_handle(net, search=2, **kw)
        txt = h.plan_info()
        h.close()
        op, _ = order_search.dp_plan(net.inds(), net.dims(), net.output, kw.get("max_intermediate_bytes", 0),
                                     kw.get("n_slices", 0), kw.get("slice_dim", 0))
        assert txt == planner.plan_text(op, net.inds())
        assert txt.rstrip().endswith("search exact tensors=%d" % op.search_dp)


def test_hyper_search_never_executes_more_than_its_candidates():
    """search = 1 keeps the candidate whose lowered launch list executes the
    fewest FLOPs: never more than the greedy best-of-n or the exact tree."""
    from paper_2410_15080_b300 import costmodel
    nets = costmodel.eval_networks(10)
    gains = []
    for net in (nets[0], nets[9]):
        g = _host_handle(net, n_candidates=16)
        fg = g.exec_stats()["flops_executed"]
        g.close()
        e = _host_handle(net, search=2)
        fe = e.exec_stats()["flops_executed"]
        e.close()
        hh = _host_handle(net, n_candidates=16, search=1)
        fh = hh.exec_stats()["flops_executed"]
        note = hh.plan_info().rstrip().splitlines()[-1]
        hh.close()
        assert note.startswith("search hyper candidates=17 chosen=")
        assert fh <= fg and fh <= fe
        gains.append(fg / fh)
    assert max(gains) > 1.1  # the exact tree wins on the second network


def test_search_option_errors():
    import synth
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=2)
    for kw in ({"search": 3}, {"search": 1, "cost_model": 1}):
        with pytest.raises(htn.QtpuError) as e:
            _host_handle(net, **kw)
        assert e.value.status in (htn.QTPU_EINVAL, htn.QTPU_ENOTSUP)
    big = synth.ring_htn(n_sub=17, gates_per_edge=1, wires_per_edge=1, k=2)
    with pytest.raises(htn.QtpuError) as e:
        _host_handle(big, search=2)
    assert e.value.status == htn.QTPU_ENOTSUP


def test_kept_split_results_remove_reruns(monkeypatch):
    """Slice reuse on the 100-qubit plan: an operand split whose own sliced
    positions vary inside an outer loop it does not depend on keeps one
    result per value of its positions, so every split runs once per distinct
    value (16 here) instead of once per visit (64)."""
    import synth
    net = synth.ring_chords_htn(materialize=False)
    kw = dict(max_intermediate_bytes=8 << 30, n_slices=1024, slice_dim=4, n_candidates=256)

    def runs(h):
        out = {}
        for line in h.lowering_info().splitlines():
            f = line.split()
            if len(f) > 3 and f[0] == "launch" and f[2] == "split":
                d = dict(w.split("=", 1) for w in f if "=" in w)
                out[int(f[1])] = (d["din"], int(d["runs"]))
        return out

    h = _host_handle(net, **kw)
    kept = runs(h)
    n_kept = h.exec_stats()["launches"]
    h.close()
    monkeypatch.setenv("QTPU_NO_KEPT_SPLITS", "1")
    h = _host_handle(net, **kw)
    plain = runs(h)
    n_plain = h.exec_stats()["launches"]
    h.close()
    for i, (din, r) in kept.items():
        distinct = 4 ** (0 if din == "-" else len(din.split(",")))
        assert r == distinct, (i, din, r)
    assert any(r > 4 ** len(d.split(",")) for d, r in plain.values() if d != "-")
    assert n_kept < n_plain


def test_greedy_tie_breaks_match_the_oracle():
    """The C++ planner resolves the greedy key's ties like the oracle (FLOPs,
    then x, then y): same plan text on networks built to tie each component."""
    from tests.test_oracle_planner import FLOP_TIE, ID_TIE_X, ID_TIE_Y, _tiny
    for case in (FLOP_TIE, ID_TIE_X, ID_TIE_Y):
        net = _tiny(*case)
        h = _host_handle(net)
        txt = h.plan_info()
        h.close()
        op = planner.make_plan(net.inds(), net.dims(), net.output)
        assert txt == planner.plan_text(op, net.inds())
