"""QPD sampling and h-TN simplification (oracle; test infrastructure only).

Section 4.3 and Step 1 of section 6.1: before contracting, the h-TN is
simplified and its coefficient tensors are sampled.

1. Simplification.  The gate-cut coefficient vectors between the same two
   QTs are fused: their tensor product becomes one CT over one fused index,
   and each of the two QTs has the corresponding cut axes merged into one
   axis.  The value of the contraction does not change.
2. Sampling.  Each fused CT c (length D) is sampled s times, entry i with
   probability |c_i| / gamma, gamma = sum_i |c_i|; the sampled CT is
   c'_i = gamma * sign(c_i) * count_i / s, so that E[c'_i] = c_i and, the CTs
   being sampled independently and the contraction linear in each, the
   contraction of the sampled network is an unbiased estimate of <O>.
3. Truncation.  Entries never drawn (count_i = 0) are dropped from the CT and
   the two QTs are restricted to the drawn values along the fused index.
The wire-cut tensor is not sampled (its instances are weighted equally).

Conventions this module fixes (the paper does not state them):

* A "gate-cut CT" is a rank-1 CT whose index is carried by exactly two QTs
  and by no other tensor, and is not an output index.  Rank-2 CTs (wire
  cuts) and everything else are left as they are.
* Groups: the gate-cut CTs between the same QT pair (a, b), a < b tensor ids,
  in ascending (a, b); within a group the CTs in ascending tensor id.  The
  fused value f enumerates the group's index values with the first CT's index
  slowest (C order).  Fused index ids are max(id) + 1 + x for group x.
* Fused CT entry f = c_1[i_1] * c_2[i_2] * ... in FP64, multiplied left to
  right.  A QT's fused axis sits at the position of the first of the group's
  axes in that QT; the other axes keep their order.
* Draw j of group x uses u[x, j] in [0, 1): t = u * gamma with
  P_i = |c_0| + ... + |c_i| accumulated left to right in FP64 and
  gamma = P_{D-1}; the draw is the first i with P_i > t, or, if there is none,
  the last i with c_i != 0.  (Floating point decides an integer here, so the
  CUDA path takes the same decision in the same precision and order.)
* c'_i = sign(c_i) * ((gamma * count_i) / s) in FP64; kept values ascending.

The random numbers are inputs (the caller's uniforms), so the oracle and the
CUDA path sample identically.

Pinned by tests/test_oracle_sampling.py: a hand-computed fused CT; fusing
leaves the brute-force value unchanged; stratified draws give every count
within 1 of s * p_i; a one-entry CT draws it s times; the truncated network's
value equals the untruncated network's with c' (zeros kept); the mean of the
sampled estimate over many seeds is within 4 standard errors of the exact
value; the draws match a linear walk over the prefix sums on small cases.
"""
from __future__ import annotations

import numpy as np


def gate_groups(tensors, kinds, output):
    """[(qa, qb, [ct tensor ids], [index ids])] per the conventions above.

    tensors: list of (inds, array); kinds: "QT" / "CT" per tensor."""
    carriers = {}
    for t, (inds, _) in enumerate(tensors):
        for i in inds:
            carriers.setdefault(i, []).append(t)
    groups = {}
    for t, (inds, arr) in enumerate(tensors):
        if kinds[t] != "CT" or len(inds) != 1:
            continue
        i = inds[0]
        if i in output:
            continue
        others = [u for u in carriers[i] if u != t]
        if len(others) != 2 or any(kinds[u] != "QT" for u in others):
            continue
        a, b = sorted(others)
        groups.setdefault((a, b), []).append((t, i))
    out = []
    for (a, b) in sorted(groups):
        cts = sorted(groups[(a, b)])
        out.append((a, b, [c for c, _ in cts], [i for _, i in cts]))
    return out


def fused_ct(vectors) -> np.ndarray:
    """Tensor product of the group's CT vectors, first vector slowest; each
    entry multiplied left to right in FP64."""
    vs = [np.asarray(v, dtype=np.float64) for v in vectors]
    dims = [len(v) for v in vs]
    D = int(np.prod(dims))
    out = np.empty(D)
    for f in range(D):
        r, digits = f, []
        for d in reversed(dims):
            digits.append(r % d)
            r //= d
        digits.reverse()
        p = vs[0][digits[0]]
        for v, i in zip(vs[1:], digits[1:]):
            p = p * v[i]
        out[f] = p
    return out


def fuse_axes(inds, arr, group_inds, fused_id):
    """Merge the axes `group_inds` (in that order, first slowest) of one QT
    into one axis `fused_id` at the position of the first of them."""
    pos = [inds.index(i) for i in group_inds]
    first = min(pos)
    rest = [a for a in range(len(inds)) if a not in pos]
    # axes before the first group axis, the group axes, then the rest
    before = [a for a in rest if a < first]
    after = [a for a in rest if a > first]
    perm = before + pos + after
    t = np.transpose(np.asarray(arr), perm)
    shape = ([arr.shape[a] for a in before] + [int(np.prod([arr.shape[a] for a in pos]))]
             + [arr.shape[a] for a in after])
    new_inds = tuple([inds[a] for a in before] + [fused_id] + [inds[a] for a in after])
    return new_inds, np.ascontiguousarray(t).reshape(shape)


def simplify(tensors, kinds, output):
    """Step 1: the fused network (tensors, kinds, groups).  The tensors that
    are not fused CTs keep their order; the fused CTs follow, group x at
    position len(tensors) - len(groups) + x, over index max(id) + 1 + x."""
    groups = gate_groups(tensors, kinds, output)
    max_id = max((i for inds, _ in tensors for i in inds), default=-1)
    qts = {t: (tuple(tensors[t][0]), np.asarray(tensors[t][1])) for t in range(len(tensors))}
    drop = set()
    fused_cts = []
    for x, (a, b, cts, inds) in enumerate(groups):
        fid = max_id + 1 + x
        for q in (a, b):
            qi, qa = qts[q]
            qts[q] = fuse_axes(qi, qa, inds, fid)
        fused_cts.append(((fid,), fused_ct([np.asarray(tensors[c][1]).ravel() for c in cts])))
        drop.update(cts)
    new_t, new_k = [], []
    for t in range(len(tensors)):
        if t in drop:
            continue
        new_t.append(qts[t])
        new_k.append(kinds[t])
    for ct in fused_cts:
        new_t.append(ct)
        new_k.append("CT")
    return new_t, new_k, groups


def draw_counts(c: np.ndarray, s: int, u: np.ndarray) -> np.ndarray:
    """Counts of s draws from |c| / gamma by inverse CDF on the uniforms u
    (length s), per the conventions above."""
    a = np.abs(np.asarray(c, dtype=np.float64))
    P = np.empty(len(a))
    acc = 0.0
    for i, x in enumerate(a):
        acc = acc + x
        P[i] = acc
    gamma = P[-1]
    nz = np.nonzero(a)[0]
    last = int(nz[-1]) if len(nz) else len(a) - 1
    t = np.asarray(u[:s], dtype=np.float64) * gamma
    idx = np.searchsorted(P, t, side="right")  # first i with P_i > t
    idx[idx >= len(a)] = last
    return np.bincount(idx, minlength=len(a)).astype(np.int64)


def sampled_ct(c: np.ndarray, counts: np.ndarray, s: int) -> np.ndarray:
    """c'_i = sign(c_i) * ((gamma * count_i) / s), gamma the left-to-right
    sum of |c|."""
    a = np.abs(np.asarray(c, dtype=np.float64))
    gamma = 0.0
    for x in a:
        gamma = gamma + x
    out = np.zeros(len(a))
    for i in range(len(a)):
        out[i] = np.sign(c[i]) * ((gamma * float(counts[i])) / float(s))
    return out


def qpd_sample(tensors, kinds, output, s: int, u: np.ndarray, truncate: bool = True):
    """Steps 1-3: the sampled, truncated network.  u: [n_groups, s] uniforms.

    Returns (tensors, kinds, info) with info[x] = (dim before, kept values)."""
    ft, fk, groups = simplify(tensors, kinds, output)
    n_g = len(groups)
    n_other = len(ft) - n_g
    max_id = max((i for inds, _ in tensors for i in inds), default=-1)
    info = []
    out_t = list(ft)
    for x in range(n_g):
        fid = max_id + 1 + x
        inds, c = ft[n_other + x]
        counts = draw_counts(c, s, u[x])
        cs = sampled_ct(c, counts, s)
        keep = np.nonzero(counts)[0] if truncate else np.arange(len(c))
        info.append((len(c), keep))
        out_t[n_other + x] = (inds, cs[keep])
        for t in range(n_other):
            ti, ta = out_t[t]
            if fid in ti:
                out_t[t] = (ti, np.take(ta, keep, axis=ti.index(fid)))
    return out_t, fk, info
