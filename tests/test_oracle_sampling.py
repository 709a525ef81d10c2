"""Pins for the QPD-sampling oracle (section 4.3; Step 1 of section 6.1):
hand-computed fusion, value-preserving simplification, inverse-CDF draws,
truncation invariance and unbiasedness of the sampled estimate."""
import numpy as np
import pytest

import synth
from oracle import planner, sampling, tn


def _value(tensors, output):
    inds = [t[0] for t in tensors]
    dims = {}
    for i, a in tensors:
        for x, d in zip(i, np.shape(a)):
            dims[x] = d
    p = planner.make_plan(inds, dims, output)
    return tn.contract_pairwise(tensors, output, planner.order_of(p)).ravel()


def _net(n_sub=3, gates=2, wires=1, k=2, seed=0):
    net = synth.ring_htn(n_sub=n_sub, gates_per_edge=gates, wires_per_edge=wires, k=k, seed=seed)
    return net.pairs(), [t.kind for t in net.tensors], net.output


def test_fused_ct_hand_computed():
    got = sampling.fused_ct([[1.0, 2.0], [3.0, -1.0, 5.0]])
    np.testing.assert_array_equal(got, [3.0, -1.0, 5.0, 6.0, -2.0, 10.0])


def test_fuse_axes_by_loops():
    rng = np.random.default_rng(0)
    A = rng.uniform(-1, 1, (2, 3, 4, 5))
    # group (3, 1): index 3 (axis 3, dim 5) slowest, index 1 (axis 1, dim 3)
    # fastest; the fused axis sits where axis 1 was
    inds, B = sampling.fuse_axes((7, 1, 9, 3), A, [3, 1], 42)
    assert inds == (7, 42, 9) and B.shape == (2, 15, 4)
    for a in range(2):
        for i3 in range(5):
            for i1 in range(3):
                for c in range(4):
                    assert B[a, i3 * 3 + i1, c] == A[a, i1, c, i3]


def test_groups_skip_wire_and_output_cts():
    tensors, kinds, output = _net(n_sub=3, gates=2, wires=1)
    groups = sampling.gate_groups(tensors, kinds, output)
    assert [(a, b) for a, b, _, _ in groups] == [(0, 1), (0, 2), (1, 2)]
    assert all(len(c) == 2 for _, _, c, _ in groups)
    # a gate index kept in the output is not sampled
    gi = groups[0][3][0]
    g2 = sampling.gate_groups(tensors, kinds, output + (gi,))
    assert len(g2[0][2]) == 1


@pytest.mark.parametrize("seed", range(3))
def test_simplify_keeps_the_value(seed):
    tensors, kinds, output = _net(seed=seed)
    ref = _value(tensors, output)
    ft, fk, groups = sampling.simplify(tensors, kinds, output)
    assert len(ft) == len(tensors) - sum(len(g[2]) for g in groups) + len(groups)
    assert all(len(ft[len(ft) - len(groups) + x][1]) == 36 for x in range(len(groups)))
    np.testing.assert_allclose(_value(ft, output), ref, rtol=1e-12)


def test_simplify_brute_force_on_a_tiny_net():
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (2, 3, 2))     # (0, 1, 2)
    B = rng.uniform(-1, 1, (3, 2, 2))     # (1, 2, 3)
    c1 = np.array([0.5, -1.5, 0.25])
    c2 = np.array([2.0, -0.5])
    tensors = [((0, 1, 2), A), ((1, 2, 3), B), ((1,), c1), ((2,), c2)]
    kinds = ["QT", "QT", "CT", "CT"]
    ref = tn.brute_force(tensors, (0, 3))
    ft, fk, groups = sampling.simplify(tensors, kinds, (0, 3))
    assert groups == [(0, 1, [2, 3], [1, 2])]
    np.testing.assert_allclose(tn.brute_force(ft, (0, 3)), ref, rtol=1e-13)


def test_stratified_draws_are_within_one_of_the_mean():
    c = np.array([0.5, -0.25, 0.0, 1.0, -0.125, 0.125])
    s = 1000
    u = (np.arange(s) + 0.5) / s
    counts = sampling.draw_counts(c, s, u)
    p = np.abs(c) / np.abs(c).sum()
    assert counts.sum() == s and counts[2] == 0
    assert np.all(np.abs(counts - s * p) <= 1.0)


def test_a_single_nonzero_entry_takes_every_draw():
    c = np.array([0.0, 0.0, -0.7, 0.0])
    u = np.random.default_rng(1).uniform(0, 1, 50)
    counts = sampling.draw_counts(c, 50, u)
    np.testing.assert_array_equal(counts, [0, 0, 50, 0])
    np.testing.assert_array_equal(sampling.sampled_ct(c, counts, 50), [0.0, 0.0, -0.7, 0.0])
    # u close to 1 still lands on the last nonzero entry
    counts = sampling.draw_counts(np.array([0.3, 0.7, 0.0]), 1, np.array([1.0 - 2.0 ** -53]))
    np.testing.assert_array_equal(counts, [0, 1, 0])


def test_draws_match_a_linear_walk():
    rng = np.random.default_rng(7)
    for _ in range(20):
        D = int(rng.integers(1, 12))
        c = rng.uniform(-1, 1, D) * (rng.uniform(size=D) < 0.7)
        if not np.any(c):
            c[0] = 0.5
        s = int(rng.integers(1, 40))
        u = rng.uniform(0, 1, s)
        a = np.abs(c)
        P, acc = [], 0.0
        for x in a:
            acc += x
            P.append(acc)
        want = np.zeros(D, dtype=np.int64)
        for uj in u:
            t = uj * P[-1]
            i = next((i for i in range(D) if P[i] > t), None)
            want[i if i is not None else int(np.nonzero(a)[0][-1])] += 1
        np.testing.assert_array_equal(sampling.draw_counts(c, s, u), want)


def test_truncation_keeps_the_sampled_value():
    tensors, kinds, output = _net(seed=1)
    s = 12
    u = np.random.default_rng(2).uniform(0, 1, (3, s))
    tt, _, info = sampling.qpd_sample(tensors, kinds, output, s, u, truncate=True)
    tf, _, _ = sampling.qpd_sample(tensors, kinds, output, s, u, truncate=False)
    assert all(len(keep) <= s and len(keep) < d for d, keep in info)
    np.testing.assert_allclose(_value(tt, output), _value(tf, output), rtol=1e-12)


def test_sampled_estimate_is_unbiased():
    tensors, kinds, output = _net(n_sub=3, gates=1, wires=1, k=1, seed=4)
    exact = _value(tensors, output)[0]
    ft, fk, groups = sampling.simplify(tensors, kinds, output)
    s, n = 8, 600
    rng = np.random.default_rng(11)
    est = []
    for _ in range(n):
        u = rng.uniform(0, 1, (len(groups), s))
        tt, _, _ = sampling.qpd_sample(tensors, kinds, output, s, u)
        est.append(_value(tt, output)[0])
    est = np.array(est)
    se = est.std(ddof=1) / np.sqrt(n)
    assert se > 0
    assert abs(est.mean() - exact) <= 4 * se
