"""Contraction order by exact search over subsets (oracle; test infrastructure
only).

Section 6.1 step 3 computes the contraction order before the contraction,
and the paper hands it to a hyper-optimiser (section 6.1); section 4.2 makes
the cost of the post-processing the cost of that order.  Beyond the greedy
order (``oracle.planner``), the order here is the cheapest contraction tree
over the network's large tensors, found by dynamic programming over subsets:

1. Absorption.  Every small leaf (at most 256 entries: the coefficient
   tensors) that shares an index with a large leaf is contracted, in
   ascending leaf id, into the large leaf with the smallest id among those
   sharing one of its indices (each step (min id, max id) of the two current
   ids, classified by the planner's keep rule).
2. Exact tree.  Over the m live tensors left (ascending id; m <= 12), with
   K(S) the indices of a set S carried outside S or by the output, and the
   index tuple of S its tensor's for |S| = 1 and K(S) otherwise:
       cost(S) = min over A subset of S, A containing S's lowest member,
                 A != S, B = S \\ A, of  cost(A) + cost(B) + flops(A, B)
   with flops the planner's step cost (2 * batch * M * N * K, plus an
   operand's size when it has indices summed out first), keep = K(S).  Ties
   go to the smallest A (as a bit mask over the live tensors in ascending
   order).
3. The tree is emitted in post order (A's subtree, then B's, then the step
   joining them, operands as (min id, max id)), and the planner's slicer
   runs on it unchanged.

Pinned by tests/test_oracle_order_search.py: on tiny networks the exact cost
equals the minimum over every pairwise order enumerated by brute force (of
the whole network, and of the tensors left after absorption); the emitted
plan's own step costs add up to the DP cost; and the plan contracts to the
brute-force value.  (Absorbing every coefficient tensor first is a fixed
choice: on small networks a greedy order that absorbs later can be cheaper,
which is why the product ranks this plan among greedy candidates.)
"""
from __future__ import annotations

from math import prod

from . import planner

SMALL = 256
MAX_EXACT = 12


def _size(dims, inds):
    return prod(dims[i] for i in inds) if inds else 1


def _apply(live, count, steps, x, y, nxt, dims):
    """One pairwise step (x < y) with the planner's keep rule."""
    ia, ib = live[x], live[y]
    sx, sy = set(ia), set(ib)
    keep = {i for i in sx | sy if count.get(i, 0) - (i in sx) - (i in sy) > 0}
    batch, m, n, k, sa, sb = planner.classify(ia, ib, keep)
    for i in sx:
        count[i] -= 1
    for i in sy:
        count[i] -= 1
    del live[x], live[y]
    new = batch + m + n
    live[nxt] = new
    for i in set(new):
        count[i] = count.get(i, 0) + 1
    steps.append(planner.Step(x, y, nxt, batch, m, n, k, sa, sb))


def absorb(tensors_inds, dims, output):
    """Step 1: (live, count, steps, next id) after the absorption steps."""
    n = len(tensors_inds)
    live = {t: tuple(x) for t, x in enumerate(tensors_inds)}
    count = {}
    for x in live.values():
        for i in set(x):
            count[i] = count.get(i, 0) + 1
    for i in output:
        count[i] = count.get(i, 0) + 1
    small = [t for t in range(n) if _size(dims, tensors_inds[t]) <= SMALL]
    large = [t for t in range(n) if t not in small]
    cur = {t: t for t in large}
    steps = []
    nxt = n
    for t in small:
        hosts = [q for q in large if set(tensors_inds[q]) & set(tensors_inds[t])]
        if not hosts:
            continue
        h = min(hosts)
        x, y = sorted((cur[h], t))
        _apply(live, count, steps, x, y, nxt, dims)
        cur[h] = nxt
        nxt += 1
    return live, count, steps, nxt


def exact_tree(live, output, dims):
    """Step 2: (cost table, split table, ids) over the live tensors."""
    ids = sorted(live)
    m = len(ids)
    if m > MAX_EXACT:
        raise ValueError("too many tensors for the exact search")
    full = (1 << m) - 1
    outs = set(output)
    carried = [set(live[t]) for t in ids]

    def kept(mask):
        inside = set().union(*(carried[j] for j in range(m) if mask >> j & 1))
        outside = set().union(*[carried[j] for j in range(m) if not mask >> j & 1]) if mask != full else set()
        return {i for i in inside if i in outside or i in outs}

    tup = {}
    for mask in range(1, full + 1):
        if mask & (mask - 1) == 0:
            tup[mask] = live[ids[mask.bit_length() - 1]]
        else:
            K = kept(mask)
            tup[mask] = tuple(sorted(K))
    cost = {}
    split = {}
    for mask in range(1, full + 1):
        if mask & (mask - 1) == 0:
            cost[mask] = 0
            continue
        low = mask & -mask
        keep = kept(mask)
        best = None
        a = mask
        subs = []
        while a:
            a = (a - 1) & mask
            if a and a & low and a != mask:
                subs.append(a)
        for a in sorted(subs):
            b = mask ^ a
            ia, ib = tup[a], tup[b]
            batch, mm, nn, k, sa, sb = planner.classify(ia, ib, keep)
            f = planner.step_flops(dims, ia, ib, batch, mm, nn, k, sa, sb)
            c = cost[a] + cost[b] + f
            if best is None or c < best[0]:
                best = (c, a)
        cost[mask], split[mask] = best
    return cost, split, ids


def dp_plan(tensors_inds, dims, output, max_bytes=0, n_slices=0, slice_dim=0):
    """Steps 1-3: the plan (then sliced like the greedy plan)."""
    live, count, steps, nxt = absorb(tensors_inds, dims, output)
    cost, split, ids = exact_tree(live, output, dims)
    m = len(ids)
    state = {"nxt": nxt}

    def build(mask):
        if mask & (mask - 1) == 0:
            return ids[mask.bit_length() - 1]
        a = split[mask]
        xa = build(a)
        xb = build(mask ^ a)
        x, y = sorted((xa, xb))
        _apply(live, count, steps, x, y, state["nxt"], dims)
        state["nxt"] += 1
        return state["nxt"] - 1

    if m > 1:
        build((1 << m) - 1)
    plan = planner.Plan(n_leaves=len(tensors_inds), output=tuple(output), dims=dict(dims))
    plan.steps = steps
    (last,) = live.values()
    plan.final_inds = last
    plan.final_sum = tuple(i for i in last if i not in set(output))
    plan.search_dp = m
    plan = planner.slice_plan(plan, tensors_inds, max_bytes, n_slices, slice_dim)
    return plan, cost[(1 << m) - 1] if m > 1 else 0
