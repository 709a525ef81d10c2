"""Pins for the exact order search (section 6.1 step 3; section 4.2 cost):
brute force over every pairwise order (of the whole network, and of the
tensors left after absorption), the emitted plan's step costs, the
contracted value."""
import itertools

import numpy as np
import pytest

import synth
from oracle import order_search, planner, tn


def _all_orders(n):
    def rec(live, nxt):
        if len(live) == 1:
            yield []
            return
        for a, b in itertools.combinations(sorted(live), 2):
            rest = [t for t in live if t not in (a, b)] + [nxt]
            for tail in rec(rest, nxt + 1):
                yield [(a, b)] + tail
    yield from rec(list(range(n)), n)


def _order_cost(tensors_inds, dims, output, order):
    """Plan cost of a given pairwise order, by the planner's step rule."""
    live = {t: tuple(x) for t, x in enumerate(tensors_inds)}
    count = {}
    for x in live.values():
        for i in set(x):
            count[i] = count.get(i, 0) + 1
    for i in output:
        count[i] = count.get(i, 0) + 1
    steps = []
    nxt = len(tensors_inds)
    total = 0
    for x, y in order:
        ia, ib = live[x], live[y]
        order_search._apply(live, count, steps, x, y, nxt, dims)
        st = steps[-1]
        total += planner.step_flops(dims, ia, ib, st.batch, st.m, st.n, st.k, st.sa, st.sb)
        nxt += 1
    return total


def _big_net(seed, n_tensors, n_indices=7):
    """Random hyper-networks whose leaves are all above the absorption size."""
    rng = np.random.default_rng([seed, 0xD9])
    dims = {i: int(rng.integers(2, 5)) for i in range(n_indices)}
    inds = []
    for _ in range(n_tensors):
        while True:
            r = int(rng.integers(4, 7))
            x = tuple(int(i) for i in rng.choice(n_indices, size=r, replace=False))
            if np.prod([dims[i] for i in x]) > order_search.SMALL:
                break
        inds.append(x)
    out = tuple(int(i) for i in rng.choice(n_indices, size=seed % 2, replace=False))
    return inds, dims, out


@pytest.mark.parametrize("seed", range(6))
def test_exact_cost_is_the_brute_force_minimum(seed):
    inds, dims, out = _big_net(seed, n_tensors=4 + seed % 2)
    best = min(_order_cost(inds, dims, out, o) for o in _all_orders(len(inds)))
    plan, cost = order_search.dp_plan(inds, dims, out)
    assert cost == best
    # the emitted plan's steps cost exactly that
    t = planner._tensor_inds(plan, inds)
    fl = sum(planner.step_flops(dims, t[st.x], t[st.y], st.batch, st.m, st.n, st.k, st.sa, st.sb)
             for st in plan.steps)
    assert fl == cost


def _orders_over(ids, nxt):
    """Every pairwise order over the given live ids (results numbered from nxt)."""
    def rec(live, n):
        if len(live) == 1:
            yield []
            return
        for a, b in itertools.combinations(sorted(live), 2):
            rest = [t for t in live if t not in (a, b)] + [n]
            for tail in rec(rest, n + 1):
                yield [(a, b)] + tail
    yield from rec(list(ids), nxt)


@pytest.mark.parametrize("seed", range(4))
def test_tree_after_absorption_is_the_brute_force_minimum(seed):
    """With coefficient tensors absorbed first, the exact tree over the
    remaining tensors costs the minimum over every pairwise order of them;
    the plan contracts to the greedy plan's value."""
    import copy
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=2, seed=seed)
    inds, dims = net.inds(), net.dims()
    live, count, steps, nxt = order_search.absorb(inds, dims, net.output)
    cost, split, ids = order_search.exact_tree(live, net.output, dims)
    best = None
    for order in _orders_over(ids, nxt):
        lv, ct, st = copy.deepcopy(live), dict(count), []
        tot, n = 0, nxt
        for x, y in order:
            ia, ib = lv[x], lv[y]
            order_search._apply(lv, ct, st, x, y, n, dims)
            s_ = st[-1]
            tot += planner.step_flops(dims, ia, ib, s_.batch, s_.m, s_.n, s_.k, s_.sa, s_.sb)
            n += 1
        best = tot if best is None else min(best, tot)
    assert cost[(1 << len(ids)) - 1] == best
    plan, _ = order_search.dp_plan(inds, dims, net.output)
    g = planner.make_plan(inds, dims, net.output)
    got = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(plan))
    ref = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(g))
    np.testing.assert_allclose(got, ref, rtol=1e-12)
    small = synth.tiny_random_htn(seed, n_tensors=4, n_indices=6, n_output=1)
    p2, _ = order_search.dp_plan(small.inds(), small.dims(), small.output)
    np.testing.assert_allclose(tn.contract_pairwise(small.pairs(), small.output, planner.order_of(p2)),
                               tn.brute_force(small.pairs(), small.output), rtol=1e-12, atol=1e-13)


def test_absorption_hosts():
    """Coefficient tensors go, in ascending id, into the lowest-id QT that
    carries one of their indices."""
    net = synth.ring_htn(n_sub=3, gates_per_edge=1, wires_per_edge=1, k=2, seed=0)
    inds = net.inds()
    n = len(inds)
    live, count, steps, nxt = order_search.absorb(inds, net.dims(), net.output)
    qts = [t for t, x in enumerate(net.tensors) if x.kind == "QT"]
    cts = [t for t, x in enumerate(net.tensors) if x.kind == "CT"]
    assert len(steps) == len(cts) and len(live) == len(qts)
    assert all(t in qts or t >= n for t in live)
    host_of = {q: q for q in qts}  # current id -> original QT
    for st, c in zip(steps, cts):
        assert c in (st.x, st.y)
        cur = st.y if st.x == c else st.x
        q = host_of[cur]
        assert q == min(t for t in qts if set(inds[t]) & set(inds[c]))
        host_of[st.out] = q
