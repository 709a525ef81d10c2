"""Plain FP64 contraction of a tensor network with hyper-indices (oracle).

Section 2.2 defines the contraction: tensors are vertices, indices are edges,
an index shared by two or more tensors (a hyper-edge when more than two) is
summed over once, and indices named as output are kept.  Section 4.1 makes
circuit knitting exactly such a contraction (QTs evaluated to classical
tensors, joined to the coefficient tensors by hyper-indices), and section 4.2
states that the value does not depend on the pairwise order, only the cost.

A network here is ``(tensors, output)`` with ``tensors`` a list of
``(inds, array)`` pairs: ``inds`` a tuple of int index ids, one per array
axis, ``output`` a tuple of index ids (each must occur in some tensor).

Functions:

* ``brute_force``        -- the definition written out: for every assignment
  of every index, multiply one entry of every tensor and add it to the output
  entry (tiny networks only).
* ``contract_pairwise``  -- the same sum evaluated pairwise in a caller-given
  order; each pair is one ``numpy.matmul`` over [batch, M, K] x [batch, K, N]
  after classifying the pair's indices (kept-and-shared -> batch, shared-only
  -> summed, one side only -> kept M / N or summed away).
* ``contract_sliced``    -- fixes the given indices to each of their values,
  contracts every slice pairwise, and adds the slice results (slicing is how
  the peak intermediate is bounded; it does not change the value).
* ``contract_output_subset`` -- the contraction restricted to some values of
  one output index (used where the full contraction is too slow on a CPU).

Pinned by tests/test_oracle_tn.py: brute force equals pairwise contraction on
random tiny hyper-networks for every pairwise order, slicing sums to the
unsliced value, a rank-1 network matches its closed form, and the 4-tensor
knitting network of ``oracle.knit`` equals the uncut statevector value.
"""
from __future__ import annotations

import itertools
from typing import Sequence

import numpy as np


def _dims(tensors):
    d = {}
    for inds, arr in tensors:
        for ix, n in zip(inds, arr.shape):
            if ix in d and d[ix] != n:
                raise ValueError(f"index {ix}: dim {n} != {d[ix]}")
            d[ix] = n
    return d


def brute_force(tensors, output) -> np.ndarray:
    """out[o] = sum over all non-output index values of prod_t T_t[...]."""
    dims = _dims(tensors)
    allix = sorted(dims)
    out = np.zeros(tuple(dims[i] for i in output), dtype=np.float64)
    for vals in itertools.product(*[range(dims[i]) for i in allix]):
        a = dict(zip(allix, vals))
        p = 1.0
        for inds, arr in tensors:
            p *= float(arr[tuple(a[i] for i in inds)])
        out[tuple(a[i] for i in output)] += p
    return out


def contract_pair(A, B, keep: set):
    """Contract two tensors; ``keep`` = index ids still needed elsewhere
    (by another live tensor or by the output).

    Returns (inds, array) with inds ordered [batch..., M..., N...] where
    batch = in both and kept, M = only in A and kept, N = only in B and kept.
    Every other index of A or B is summed.
    """
    ia, a = A
    ib, b = B
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    sa, sb = set(ia), set(ib)
    batch = [i for i in ia if i in sb and i in keep]
    ksum = [i for i in ia if i in sb and i not in keep]
    m = [i for i in ia if i not in sb and i in keep]
    n = [i for i in ib if i not in sa and i in keep]
    # indices only on one side and not kept: sum them out first
    a_only = [i for i in ia if i not in sb and i not in keep]
    b_only = [i for i in ib if i not in sa and i not in keep]
    if a_only:
        a = a.sum(axis=tuple(ia.index(i) for i in a_only))
        ia = tuple(i for i in ia if i not in a_only)
    if b_only:
        b = b.sum(axis=tuple(ib.index(i) for i in b_only))
        ib = tuple(i for i in ib if i not in b_only)
    da = dict(zip(ia, a.shape))
    db = dict(zip(ib, b.shape))
    nb = int(np.prod([da[i] for i in batch], dtype=np.int64))
    nm = int(np.prod([da[i] for i in m], dtype=np.int64))
    nn = int(np.prod([db[i] for i in n], dtype=np.int64))
    nk = int(np.prod([da[i] for i in ksum], dtype=np.int64))
    A3 = np.transpose(a, [ia.index(i) for i in batch + m + ksum]).reshape(nb, nm, nk)
    B3 = np.transpose(b, [ib.index(i) for i in batch + ksum + n]).reshape(nb, nk, nn)
    C = np.matmul(A3, B3)
    shape = [da[i] for i in batch] + [da[i] for i in m] + [db[i] for i in n]
    return tuple(batch + m + n), C.reshape(shape)


def contract_pairwise(tensors, output, order: Sequence[tuple]) -> np.ndarray:
    """Contract in the given pairwise order.

    ``order`` is a list of (x, y) pairs of tensor ids: ids 0..n-1 are the
    input tensors, the result of step s gets id n + s.  After the last step
    the remaining tensor(s) are reduced to the output.
    """
    live = {t: (tuple(inds), np.asarray(arr, dtype=np.float64))
            for t, (inds, arr) in enumerate(tensors)}
    nxt = len(tensors)
    out_set = set(output)
    for x, y in order:
        A, B = live.pop(x), live.pop(y)
        keep = set(out_set)
        for inds, _ in live.values():
            keep.update(inds)
        live[nxt] = contract_pair(A, B, keep)
        nxt += 1
    # fold whatever is left (disconnected pieces) as outer products
    while len(live) > 1:
        ids = sorted(live)
        A, B = live.pop(ids[0]), live.pop(ids[1])
        keep = set(out_set)
        for inds, _ in live.values():
            keep.update(inds)
        live[nxt] = contract_pair(A, B, keep)
        nxt += 1
    (inds, arr), = live.values()
    # sum indices that are not output, then order as the output
    extra = [i for i in inds if i not in out_set]
    if extra:
        arr = arr.sum(axis=tuple(inds.index(i) for i in extra))
        inds = tuple(i for i in inds if i not in extra)
    return np.transpose(arr, [inds.index(i) for i in output]) if output else arr


def slice_network(tensors, fixed: dict):
    """Fix index values: every tensor carrying a fixed index loses that axis."""
    out = []
    for inds, arr in tensors:
        sl = tuple(fixed.get(i, slice(None)) for i in inds)
        out.append((tuple(i for i in inds if i not in fixed), np.asarray(arr)[sl]))
    return out


def contract_sliced(tensors, output, order, sliced: Sequence[int]) -> np.ndarray:
    """Sum over every assignment of the sliced indices of the pairwise
    contraction of that slice (same order for every slice)."""
    dims = _dims(tensors)
    total = None
    for vals in itertools.product(*[range(dims[i]) for i in sliced]):
        part = contract_pairwise(slice_network(tensors, dict(zip(sliced, vals))),
                                 output, order)
        total = part if total is None else total + part
    return total


def contract_output_subset(tensors, output, order, index: int, values):
    """Entries of the contraction with output index ``index`` fixed to each of
    ``values``; returns an array with that axis of length len(values)."""
    rest = tuple(i for i in output if i != index)
    parts = []
    for v in values:
        parts.append(contract_pairwise(slice_network(tensors, {index: v}), rest, order))
    res = np.stack(parts, axis=0)
    # move the fixed axis back to its place in ``output``
    return np.moveaxis(res, 0, list(output).index(index))
