"""Pins for the plain contraction (section 2.2 definition; section 4.2
order independence): brute force, every pairwise order, slicing, rank-1
closed form."""
import itertools

import numpy as np
import pytest

import synth
from oracle import planner, tn


def _all_orders(n):
    """Every pairwise contraction sequence of n leaves (as id pairs)."""
    def rec(live, nxt):
        if len(live) == 1:
            yield []
            return
        for a, b in itertools.combinations(sorted(live), 2):
            rest = [t for t in live if t not in (a, b)] + [nxt]
            for tail in rec(rest, nxt + 1):
                yield [(a, b)] + tail
    yield from rec(list(range(n)), n)


@pytest.mark.parametrize("seed", range(8))
def test_pairwise_equals_brute_force_every_order(seed):
    net = synth.tiny_random_htn(seed, n_tensors=4, n_indices=6, n_output=seed % 3)
    ref = tn.brute_force(net.pairs(), net.output)
    orders = list(_all_orders(4))
    assert len(orders) == 18  # 4 leaves: 6 * 3 sequences
    for order in orders:
        got = tn.contract_pairwise(net.pairs(), net.output, order)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_five_tensor_nets(seed):
    net = synth.tiny_random_htn(100 + seed, n_tensors=5, n_indices=7, n_output=2)
    ref = tn.brute_force(net.pairs(), net.output)
    rng = np.random.default_rng(seed)
    orders = list(_all_orders(5))
    for j in rng.choice(len(orders), size=20, replace=False):
        got = tn.contract_pairwise(net.pairs(), net.output, orders[j])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_brute_force_hand_example():
    # sum_{i,j} A[i] B[i,j] C[j] with a hyper-index kept in the output
    A = np.array([1.0, 2.0])
    B = np.array([[1.0, -1.0], [0.5, 3.0]])
    C = np.array([2.0, -2.0])
    # out[i] = A[i] * sum_j B[i,j] C[j]
    want = np.array([1.0 * (2 + 2), 2.0 * (1 - 6)])
    got = tn.brute_force([((0,), A), ((0, 1), B), ((1,), C)], (0,))
    np.testing.assert_allclose(got, want, rtol=0, atol=0)


def test_slicing_sums_to_unsliced():
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=3, seed=3)
    order = [(0, 4), (1, 5), (2, 6), (3, 7), (8, 9), (10, 11), (12, 13)]
    n = len(net.tensors)
    # absorb all CTs into QTs first, then the ring
    cts = list(range(4, n))
    order = []
    live_of = {0: 0, 1: 1, 2: 2, 3: 3}
    nxt = n
    for c in cts:
        ind = net.tensors[c].inds[0]
        host = next(q for q in range(4) if ind in net.tensors[q].inds)
        order.append((live_of[host], c))
        live_of[host] = nxt
        nxt += 1
    order.append((live_of[0], live_of[1]))
    a = nxt
    nxt += 1
    order.append((live_of[2], live_of[3]))
    b = nxt
    nxt += 1
    order.append((a, b))
    full = tn.contract_pairwise(net.pairs(), net.output, order)
    wire_ix = [t.inds[0] for t in net.tensors if t.kind == "CT" and len(t.inds) == 2]
    sl = tn.contract_sliced(net.pairs(), net.output, order, wire_ix[:2])
    np.testing.assert_allclose(sl, full, rtol=1e-12, atol=1e-13)
    sub = tn.contract_output_subset(net.pairs(), net.output, order, net.output[0], [2, 0])
    np.testing.assert_allclose(sub, full[[2, 0]], rtol=1e-12, atol=1e-13)


def rank1_closed_form(net, factors):
    """out[o] = prod over output indices of the product of their vectors,
    times, for every summed index, sum_x prod of the vectors on it."""
    dims = net.dims()
    carriers = {}
    for t, tens in enumerate(net.tensors):
        for ax, i in enumerate(tens.inds):
            carriers.setdefault(i, []).append(factors[t][ax])
    scal = 1.0
    for i in dims:
        if i in net.output:
            continue
        scal *= np.prod(np.stack(carriers[i]), axis=0).sum()
    out = np.ones(tuple(dims[o] for o in net.output))
    for p, o in enumerate(net.output):
        v = np.prod(np.stack(carriers[o]), axis=0)
        shape = [1] * len(net.output)
        shape[p] = dims[o]
        out = out * v.reshape(shape)
    return scal * out


def rank1_qts_closed_form(net, factors):
    """Closed form of a network of rank-1 QTs and CTs that share no index with
    each other: out[o] = prod of the QT vectors on the output indices, times,
    for every CT, the CT contracted with the product of the QT vectors on
    each of its indices, times, for every other summed index, sum_x prod of
    the QT vectors on it.  Also returns the same with |CT| entries (the sum
    of magnitudes of the terms), whose ratio to |out| bounds the cancellation."""
    dims = net.dims()
    carriers = {}
    for t, tens in enumerate(net.tensors):
        if tens.kind == "QT":
            for ax, i in enumerate(tens.inds):
                carriers.setdefault(i, []).append(factors[t][ax])
    vec = {i: np.prod(np.stack(c), axis=0) for i, c in carriers.items()}
    scal = mag = 1.0
    on_ct = set()
    for tens in net.tensors:
        if tens.kind != "CT":
            continue
        assert not (set(tens.inds) & on_ct), "CTs share an index"
        on_ct |= set(tens.inds)
        x, xa = tens.data, np.abs(tens.data)
        for ax, i in enumerate(tens.inds):
            shape = [1] * x.ndim
            shape[ax] = dims[i]
            x = x * vec[i].reshape(shape)
            xa = xa * np.abs(vec[i]).reshape(shape)
        scal *= x.sum()
        mag *= xa.sum()
    for i in dims:
        if i in net.output or i in on_ct:
            continue
        scal *= vec[i].sum()
        mag *= np.abs(vec[i]).sum()
    out = np.ones(tuple(dims[o] for o in net.output))
    for p, o in enumerate(net.output):
        shape = [1] * len(net.output)
        shape[p] = dims[o]
        out = out * vec[o].reshape(shape)
    return scal * out, mag * np.abs(out)


def test_rank1_qts_closed_form_with_signed_cts():
    """Rank-1 QTs with the exact signed QPD coefficient tensors: the closed
    form equals the plain pairwise contraction and the brute-force sum."""
    base = synth.ring_htn(n_sub=2, gates_per_edge=1, wires_per_edge=1, k=3, seed=2)
    net, fac = synth.rank1_qts_htn(base, seed=4)
    want, mag = rank1_qts_closed_form(net, fac)
    assert np.all(mag >= np.abs(want))
    got = tn.brute_force(net.pairs(), net.output)
    np.testing.assert_allclose(got, want, rtol=1e-12)
    p = planner.make_plan(net.inds(), net.dims(), net.output)
    got2 = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p))
    np.testing.assert_allclose(got2, want, rtol=1e-12)
    # a sign flip of one gate coefficient changes the value (the CT signs enter)
    bad = synth.HTN([synth.Tensor(t.kind, t.inds, t.data * np.where(np.arange(t.data.size) == 3, -1, 1)
                                  .reshape(t.data.shape) if t.kind == "CT" and len(t.inds) == 1 else t.data)
                     for t in net.tensors], net.output)
    assert not np.allclose(tn.brute_force(bad.pairs(), bad.output), want, rtol=1e-6)


def test_rank1_closed_form():
    base = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=5, seed=1)
    net, fac = synth.rank1_htn(base, seed=2)
    want = rank1_closed_form(net, fac)
    n = len(net.tensors)
    order = [(0, 1)] + [(n + i, 2 + i) for i in range(n - 2)]
    got = tn.contract_pairwise(net.pairs(), net.output, order)
    np.testing.assert_allclose(got, want, rtol=1e-12)
