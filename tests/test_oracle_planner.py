"""Pins for the reference planner: its plans evaluate to the brute-force
value, its cost accounting matches the paper's worked example (section 4.2),
it never exceeds the naive knitting cost (section 2.1 / 4.2), and slicing
honours its targets."""
import itertools

import numpy as np
import pytest

import synth
from oracle import planner, qpd, tn


@pytest.mark.parametrize("seed", range(10))
def test_greedy_plan_evaluates_to_brute_force(seed):
    net = synth.tiny_random_htn(seed, n_tensors=5, n_indices=7, n_output=seed % 3)
    p = planner.make_plan(net.inds(), net.dims(), net.output)
    ref = tn.brute_force(net.pairs(), net.output)
    got = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_vector_matrix_vector_costs_20_multiplications(gold):
    # section 4.2: the last contraction (two 4-vectors and the 4x4 wire
    # tensor) costs 20 multiplications; the planner counts 2 per multiply-add
    net = [(1,), (1, 2), (2,)]
    p = planner.make_plan(net, {1: 4, 2: 4}, ())
    txt = planner.plan_text(p, net)
    total = int(txt.split("flops_total=")[1].split()[0])
    assert total == 2 * gold("htn_example_final_cost")


def _exhaustive_best(inds, dims, output):
    """Minimum 2*MNK cost over every pairwise sequence (tiny nets)."""
    n = len(inds)
    best = None

    def rec(live, cost):
        nonlocal best
        if len(live) == 1:
            best = cost if best is None else min(best, cost)
            return
        for a, b in itertools.combinations(sorted(live, key=lambda t: t[0]), 2):
            rest = [t for t in live if t is not a and t is not b]
            keep = set(output)
            for _, ix in rest:
                keep.update(ix)
            bt, m, nn, k, sa, sb = planner.classify(a[1], b[1], keep)
            f = planner.step_flops(dims, a[1], b[1], bt, m, nn, k, sa, sb)
            rec(rest + [(max(t[0] for t in live) + 1, bt + m + nn)], cost + f)
    rec([(i, tuple(x)) for i, x in enumerate(inds)], 0)
    return best


def test_greedy_never_worse_than_naive_and_report_gap():
    # the 5-cut example structure of section 2.1 / 4.2: 4 QTs, 4 gate cuts
    # (hyper-indices with a CT vector each) and one wire cut (4x4 CT)
    # QT1[g1,g2], QT2[g1,g2,a], QT3[b,g3,g4], QT4[g3,g4]
    inds = [(0, 1), (0, 1, 4), (5, 2, 3), (2, 3), (0,), (1,), (2,), (3,), (4, 5)]
    dims = {0: 6, 1: 6, 2: 6, 3: 6, 4: 4, 5: 4}
    p = planner.make_plan(inds, dims, ())
    total = int(planner.plan_text(p, inds).split("flops_total=")[1].split()[0])
    naive = qpd.naive_pp_flops(qpd.naive_instances(4, 1), 4, 5)
    assert total // 2 <= naive
    opt = _exhaustive_best(inds[:4] + inds[8:], dims, ())
    assert opt is not None


def test_plan_text_is_deterministic_and_complete():
    net = synth.ring_htn()
    p1 = planner.make_plan(net.inds(), net.dims(), net.output)
    p2 = planner.make_plan(net.inds(), net.dims(), net.output)
    t1, t2 = planner.plan_text(p1, net.inds()), planner.plan_text(p2, net.inds())
    assert t1 == t2
    assert t1.count("\nstep ") == len(net.tensors) - 1
    fl = int(t1.split("flops_total=")[1].split()[0])
    # 6 chain GEMMs of 2*64*144^3 plus the CT absorptions and the final trace
    assert 6 * 2 * 64 * 144 ** 3 < fl < 7 * 2 * 64 * 144 ** 3


def test_slicing_targets():
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=8)
    p = planner.make_plan(net.inds(), net.dims(), net.output, n_slices=16, slice_dim=4)
    assert p.n_slices == 16 and len(p.sliced) == 2
    assert all(net.dims()[i] == 4 for i in p.sliced)
    got = tn.contract_sliced(net.pairs(), net.output, planner.order_of(p), p.sliced)
    ref = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    p0 = planner.make_plan(net.inds(), net.dims(), net.output)
    peak0 = planner.slice_stats(p0, net.inds(), ())[0]
    lim = peak0 * 8 // 3
    p2 = planner.make_plan(net.inds(), net.dims(), net.output, max_bytes=lim)
    assert planner.slice_stats(p2, net.inds(), p2.sliced)[0] * 8 <= lim
    with pytest.raises(ValueError):
        planner.make_plan(net.inds(), net.dims(), net.output, max_bytes=8)
