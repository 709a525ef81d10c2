"""Reference contraction planner: greedy pairwise order plus slicing (oracle).

Section 4.2: the post-processing cost of an h-TN is the cost of contracting
its classical TN, which depends on the pairwise order; contracting pairwise
through the sparse structure is what makes it cheaper than knitting.  Section
6.1 (step 3) computes that order ahead of the contraction.  The paper hands
this to a hyper-optimiser; the build uses a greedy order with fully
specified tie-breaks, plus slicing over cut indices to bound the largest
intermediate (slicing is not in the paper; it is how a contraction with an
intermediate larger than device memory is made to fit).

Greedy rule (every quantity an exact Python int):
  candidates = live pairs (x < y) sharing an index (all pairs if none share);
  key(x, y)  = (size(out) - size(x) - size(y), flops(x, y), x, y), minimised;
  the result gets the next id.  An index of x or y is kept if the output or
  another live tensor carries it; kept indices in both -> batch, in x only ->
  M, in y only -> N; not kept and in both -> K (summed by the GEMM); not kept
  and on one side only -> summed out of that operand first.
  flops(x, y) = 2 * batch * M * N * K, plus size(x) if x has a pre-summed
  index, plus size(y) if y does.  The result's axes are [batch, M, N], each
  group in the order its indices have in x (batch, M) or y (N).
Slicing (fixed tree): while the peak intermediate exceeds the byte limit
  (8 bytes per entry) or the slice count is below the requested count, slice
  the non-output index (of dim ``slice_dim`` if nonzero) minimising
  (peak entries per slice, total flops over all slices, index id).

Randomised variant (seed != 0, the candidates a cost model ranks): at each
step the pair is drawn uniformly among the 3 smallest keys with the
SplitMix64 generator (Steele, Lea and Flood 2014; Vigna's reference
constants) seeded with ``seed`` and advanced once per step.

``plan_text`` is the canonical text the C++ planner must reproduce byte for
byte.  Sizes above 2**255 raise ``OverflowError`` (the C++ side returns
QTPU_ENOTSUP at the same point).

Pinned by tests/test_oracle_planner.py: a plan's cost never exceeds the naive
knitting cost (section 4.2, worst case equals naive), the paper's 432 and 20
FLOP components, the plan executes through ``oracle.tn`` to the brute-force
value, brute-force enumeration of orders on tiny nets, the slicer's choice
against peaks measured by a numpy contraction of one slice, and the greedy
key's tie-breaks on networks built to tie every earlier component.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import prod

LIMIT = 1 << 255


def _p(vals):
    r = prod(vals) if vals else 1
    if r >= LIMIT:
        raise OverflowError("size exceeds 2**255")
    return r


@dataclass
class Step:
    x: int
    y: int
    out: int
    batch: tuple
    m: tuple
    n: tuple
    k: tuple
    sa: tuple  # summed out of x first
    sb: tuple  # summed out of y first


@dataclass
class Plan:
    n_leaves: int
    output: tuple
    dims: dict
    steps: list = field(default_factory=list)
    final_inds: tuple = ()
    final_sum: tuple = ()
    sliced: tuple = ()
    n_slices: int = 1


def classify(ia, ib, keep):
    sa_, sb_ = set(ia), set(ib)
    batch = tuple(i for i in ia if i in sb_ and i in keep)
    k = tuple(i for i in ia if i in sb_ and i not in keep)
    m = tuple(i for i in ia if i not in sb_ and i in keep)
    n = tuple(i for i in ib if i not in sa_ and i in keep)
    sa = tuple(i for i in ia if i not in sb_ and i not in keep)
    sb = tuple(i for i in ib if i not in sa_ and i not in keep)
    return batch, m, n, k, sa, sb


def step_flops(dims, ia, ib, batch, m, n, k, sa, sb, sliced=()):
    d = lambda i: 1 if i in sliced else dims[i]  # noqa: E731
    f = 2 * _p([d(i) for i in batch + m + n + k])
    if sa:
        f += _p([d(i) for i in ia])
    if sb:
        f += _p([d(i) for i in ib])
    return f


M64 = (1 << 64) - 1
RAND_TOP = 3


def splitmix64(state):
    """One SplitMix64 step: returns (new state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def greedy(tensors_inds, dims, output, seed: int = 0) -> Plan:
    """Greedy pairwise order (see module header); seed != 0 randomises it."""
    n = len(tensors_inds)
    live = {t: tuple(inds) for t, inds in enumerate(tensors_inds)}
    count = {}
    for inds in live.values():
        for i in set(inds):
            count[i] = count.get(i, 0) + 1
    for i in output:
        count[i] = count.get(i, 0) + 1
    plan = Plan(n_leaves=n, output=tuple(output), dims=dict(dims))
    nxt = n
    rng = seed & M64
    while len(live) > 1:
        ids = sorted(live)
        pairs = [(x, y) for a, x in enumerate(ids) for y in ids[a + 1:]
                 if set(live[x]) & set(live[y])]
        if not pairs:
            pairs = [(x, y) for a, x in enumerate(ids) for y in ids[a + 1:]]
        best = None
        cands = []
        for x, y in pairs:
            ia, ib = live[x], live[y]
            sx, sy = set(ia), set(ib)
            keep = {i for i in sx | sy if count[i] - (i in sx) - (i in sy) > 0}
            batch, m, nn, k, sa, sb = classify(ia, ib, keep)
            size_out = _p([dims[i] for i in batch + m + nn])
            key = (size_out - _p([dims[i] for i in ia]) - _p([dims[i] for i in ib]),
                   step_flops(dims, ia, ib, batch, m, nn, k, sa, sb), x, y)
            cand = (key, Step(x, y, nxt, batch, m, nn, k, sa, sb))
            cands.append(cand)
            if best is None or key < best[0]:
                best = cand
        st = best[1]
        if seed:
            top = sorted(cands, key=lambda c: c[0])[:RAND_TOP]
            rng, r = splitmix64(rng)
            st = top[r % len(top)][1]
        for i in set(live[st.x]):
            count[i] -= 1
        for i in set(live[st.y]):
            count[i] -= 1
        del live[st.x], live[st.y]
        new = st.batch + st.m + st.n
        live[nxt] = new
        for i in set(new):
            count[i] = count.get(i, 0) + 1
        plan.steps.append(st)
        nxt += 1
    (last,) = live.values()
    plan.final_inds = last
    plan.final_sum = tuple(i for i in last if i not in set(output))
    return plan


def _tensor_inds(plan, tensors_inds):
    """Index tuple of every tensor id (leaves and step results)."""
    t = {i: tuple(x) for i, x in enumerate(tensors_inds)}
    for st in plan.steps:
        t[st.out] = st.batch + st.m + st.n
    return t


def slice_stats(plan, tensors_inds, sliced):
    """(peak entries per slice over step results, flops per slice)."""
    t = _tensor_inds(plan, tensors_inds)
    peak = 0
    fl = 0
    for st in plan.steps:
        sz = _p([1 if i in sliced else plan.dims[i] for i in t[st.out]])
        peak = max(peak, sz)
        fl += step_flops(plan.dims, t[st.x], t[st.y], st.batch, st.m, st.n,
                         st.k, st.sa, st.sb, sliced)
    return peak, fl


def slice_plan(plan, tensors_inds, max_bytes=0, n_slices=0, slice_dim=0):
    """Greedy slicing on the fixed tree (see module header)."""
    sliced = []
    nsl = 1
    all_ix = sorted(plan.dims)
    while True:
        peak, fl = slice_stats(plan, tensors_inds, sliced)
        if (max_bytes == 0 or peak * 8 <= max_bytes) and nsl >= n_slices:
            break
        cands = [i for i in all_ix if i not in plan.output and i not in sliced
                 and (slice_dim == 0 or plan.dims[i] == slice_dim)]
        if not cands:
            raise ValueError("peak limit cannot be met")  # QTPU_ELIMIT
        best = None
        for i in cands:
            p, f = slice_stats(plan, tensors_inds, sliced + [i])
            key = (p, _p([nsl, plan.dims[i], f]), i)
            if best is None or key < best:
                best = key
        sliced.append(best[2])
        nsl *= plan.dims[best[2]]
    plan.sliced = tuple(sliced)
    plan.n_slices = nsl
    return plan


def _l(v):
    return ",".join(str(i) for i in v) if v else "-"


def plan_text(plan, tensors_inds) -> str:
    """Canonical text (per-slice sizes and flops; totals over all slices)."""
    t = _tensor_inds(plan, tensors_inds)
    sl = set(plan.sliced)
    lines = [f"qtpu-plan 1 leaves={plan.n_leaves} output={_l(plan.output)}"]
    total = 0
    peak = 0
    for s, st in enumerate(plan.steps):
        size = _p([1 if i in sl else plan.dims[i] for i in t[st.out]])
        fl = step_flops(plan.dims, t[st.x], t[st.y], st.batch, st.m, st.n,
                        st.k, st.sa, st.sb, sl)
        total += fl
        peak = max(peak, size)
        lines.append(f"step {s} {st.x} {st.y} -> {st.out} batch={_l(st.batch)} "
                     f"m={_l(st.m)} n={_l(st.n)} k={_l(st.k)} sa={_l(st.sa)} "
                     f"sb={_l(st.sb)} size={size} flops={fl}")
    lines.append(f"final inds={_l(plan.final_inds)} sum={_l(plan.final_sum)}")
    lines.append(f"slices n={plan.n_slices} idx={_l(plan.sliced)}")
    lines.append(f"cost flops_per_slice={total} flops_total={total * plan.n_slices} "
                 f"peak={peak}")
    if getattr(plan, "search", None):
        lines.append(f"search candidates={plan.search[0]} seed={plan.search[1]}")
    if getattr(plan, "search_dp", None) is not None:
        lines.append(f"search exact tensors={plan.search_dp}")
    return "\n".join(lines) + "\n"


def make_plan(tensors_inds, dims, output, max_bytes=0, n_slices=0, slice_dim=0, seed=0, n_candidates=0):
    """One plan, or with n_candidates > 1 the plan with the fewest total flops
    among seeds seed .. seed+n-1 (ties: the lower seed; candidates that cannot
    meet the limit are skipped)."""
    if n_candidates > 1:
        best = None
        for s in range(seed, seed + n_candidates):
            try:
                p = make_plan(tensors_inds, dims, output, max_bytes, n_slices, slice_dim, s)
            except ValueError:
                continue
            tot = slice_stats(p, tensors_inds, p.sliced)[1] * p.n_slices
            if best is None or tot < best[0]:
                best = (tot, s, p)
        if best is None:
            raise ValueError("peak limit cannot be met")
        best[2].search = (n_candidates, best[1])
        return best[2]
    p = greedy(tensors_inds, dims, output, seed)
    return slice_plan(p, tensors_inds, max_bytes, n_slices, slice_dim)


def order_of(plan):
    """The pairwise order as (x, y) id pairs, for ``oracle.tn``."""
    return [(st.x, st.y) for st in plan.steps]
