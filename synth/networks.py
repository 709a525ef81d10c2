"""Synthetic h-TNs shaped like the paper's cut circuits (input data only).

Every entry is drawn from a seeded numpy Generator, so a network is a pure
function of its arguments.  Quantum tensors (QTs) stand for evaluated
subcircuit tensors: one 64-way observable batch index ``k`` (when ``k > 0``)
plus one index per cut touching the subcircuit, entries ~U[-1, 1].  Classical
tensors (CTs) carry the literal QPD coefficients a caller would pass:

* ``GATE_CT``: the six coefficients of the CZ gate QPD in the term order
  (I,I), (Z,Z), (M_Z,R_Z+), (M_Z,R_Z-), (R_Z+,M_Z), (R_Z-,M_Z); a gate cut's
  index (dim 6) is a hyper-index shared by both QTs and this vector;
* ``WIRE_CT``: the 4x4 wire-cut tensor of Eq. wire-tensor, rows = measured
  basis on the upstream QT's index ``a``, columns = prepared state on the
  downstream QT's index ``b``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GATE_CT = np.array([0.5, 0.5, 0.5, -0.5, 0.5, -0.5], dtype=np.float64)
WIRE_CT = 0.5 * np.array([[1, 1, 0, 0],
                          [1, -1, 0, 0],
                          [-1, -1, 2, 0],
                          [-1, -1, 0, 2]], dtype=np.float64)


@dataclass
class Tensor:
    kind: str           # "QT" or "CT"
    inds: tuple         # index ids, one per axis
    data: np.ndarray    # axes follow inds (C order)


@dataclass
class HTN:
    tensors: list
    output: tuple
    name: str = ""
    meta: dict = field(default_factory=dict)

    def dims(self) -> dict:
        d = {}
        for t in self.tensors:
            for i, n in zip(t.inds, t.data.shape):
                d[i] = n
        return d

    def inds(self):
        return [t.inds for t in self.tensors]

    def pairs(self):
        """(inds, array) list, the form ``oracle.tn`` takes."""
        return [(t.inds, t.data) for t in self.tensors]

    def nbytes(self) -> int:
        return sum(t.data.nbytes for t in self.tensors)


class _Ids:
    def __init__(self, start=0):
        self.n = start

    def __call__(self):
        self.n += 1
        return self.n - 1


def _qt(rng, inds, dims, dtype, materialize=True):
    shape = tuple(dims[i] for i in inds)
    if not materialize:  # structure only: a zero-stride view, no memory
        return Tensor("QT", tuple(inds), np.broadcast_to(np.zeros((), dtype=dtype), shape))
    return Tensor("QT", tuple(inds), rng.uniform(-1.0, 1.0, size=shape).astype(dtype))


def _edge_network(n_sub, edges, k, seed, dtype, name, materialize=True):
    """QTs joined by ``edges`` = list of (u, v, n_gate, n_wire); the wire
    index ``a`` sits on u (upstream), ``b`` on v (downstream)."""
    ids = _Ids()
    dims = {}
    kid = None
    if k > 0:
        kid = ids()
        dims[kid] = k
    qt_inds = [[kid] if kid is not None else [] for _ in range(n_sub)]
    cts = []
    for (u, v, ng, nw) in edges:
        for _ in range(ng):
            g = ids()
            dims[g] = 6
            qt_inds[u].append(g)
            qt_inds[v].append(g)
            cts.append(Tensor("CT", (g,), GATE_CT.astype(dtype)))
        for _ in range(nw):
            a, b = ids(), ids()
            dims[a] = dims[b] = 4
            qt_inds[u].append(a)
            qt_inds[v].append(b)
            cts.append(Tensor("CT", (a, b), WIRE_CT.astype(dtype)))
    tensors = []
    for j in range(n_sub):
        rng = np.random.default_rng([seed, j])
        tensors.append(_qt(rng, qt_inds[j], dims, dtype, materialize))
    tensors.extend(cts)
    out = (kid,) if kid is not None else ()
    return HTN(tensors, out, name=name,
               meta={"n_sub": n_sub, "edges": list(edges), "k": k, "seed": seed})


def ring_htn(n_sub=8, gates_per_edge=2, wires_per_edge=1, k=64, seed=0,
             dtype=np.float64) -> HTN:
    """QTs on a ring; each ring edge (j, j+1 mod n) carries the given cuts.

    The default is the mid-size workload: a 60-qubit QAOA-ring-like circuit
    cut into 8 subcircuits with 16 gate cuts and 8 wire cuts, 64 observables:
    every QT is [k=64] x (6,6,4) x (6,6,4) = 1,327,104 FP64 entries.
    Axis order of a QT: k, then the cuts of each incident edge in edge order
    (edge j joins QT_j and QT_j+1): gate indices, then the wire index (``a``
    on the upstream QT_j, ``b`` on QT_j+1).
    """
    edges = [(j, (j + 1) % n_sub, gates_per_edge, wires_per_edge) for j in range(n_sub)]
    if n_sub == 2:  # a 2-ring is a single doubled edge
        edges = [(0, 1, 2 * gates_per_edge, 2 * wires_per_edge)]
    return _edge_network(n_sub, edges, k, seed, dtype,
                         f"ring{n_sub}_g{gates_per_edge}_w{wires_per_edge}_k{k}")


def ring_chords_htn(k=64, seed=0, dtype=np.float64, n_sub=12, n_chords=8,
                    chord_step=3, materialize=True, gates_per_chord=2) -> HTN:
    """The 100-qubit workload: 12 QTs on a ring (1 gate + 1 wire cut per ring
    edge) plus chords (i, i+3 mod 12) for i < 8 with 2 gate cuts each, i.e.
    28 gate cuts and 12 wire cuts; five QTs carry 47.8 M entries."""
    edges = [(j, (j + 1) % n_sub, 1, 1) for j in range(n_sub)]
    edges += [(i, (i + chord_step) % n_sub, gates_per_chord, 0) for i in range(n_chords)]
    return _edge_network(n_sub, edges, k, seed, dtype,
                         f"ring{n_sub}_chords{n_chords}_k{k}", materialize)


def random_htn(seed: int, n_sub_range=(2, 12), n_cuts_range=(2, 20),
               k_range=(1, 64), max_qt_entries=1 << 18, max_cuts_per_pair=3,
               dtype=None) -> HTN:
    """One random network of the batched workload: ring or 2D-grid topology
    (half each), n_sub ~ U{2..12}, n_cuts ~ U{2..20} (each a gate cut with
    probability 2/3, else a wire cut), k ~ U{1..64}, FP32 or FP64 (half each).
    Cuts land on topology edges with at most ``max_cuts_per_pair`` per edge;
    the draw is repeated (same seed stream) until every QT has at most
    ``max_qt_entries`` entries."""
    rng = np.random.default_rng([seed, 0x5EED])
    for _ in range(1000):
        n_sub = int(rng.integers(n_sub_range[0], n_sub_range[1] + 1))
        n_cuts = int(rng.integers(n_cuts_range[0], n_cuts_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        dt = dtype or (np.float32 if rng.integers(0, 2) == 0 else np.float64)
        grid = bool(rng.integers(0, 2)) and n_sub >= 4
        if grid:
            w = int(np.floor(np.sqrt(n_sub)))
            topo = []
            for v in range(n_sub):
                r, c = divmod(v, w)
                if c + 1 < w and v + 1 < n_sub:
                    topo.append((v, v + 1))
                if v + w < n_sub:
                    topo.append((v, v + w))
        else:
            topo = [(j, (j + 1) % n_sub) for j in range(n_sub)] if n_sub > 2 else [(0, 1)]
        cap = max_cuts_per_pair * len(topo)
        n_cuts = min(n_cuts, cap)
        per = {e: [0, 0] for e in topo}
        # every topology edge gets at least one cut while cuts remain, so the
        # network stays connected
        order = list(topo) + [topo[int(i)] for i in rng.integers(0, len(topo), size=4 * cap)]
        placed = 0
        for e in order:
            if placed == n_cuts:
                break
            if sum(per[e]) >= max_cuts_per_pair:
                continue
            per[e][0 if rng.random() < 2 / 3 else 1] += 1
            placed += 1
        sizes = [k] * n_sub
        for (u, v), (ng, nw) in per.items():
            f = 6 ** ng * 4 ** nw
            sizes[u] *= f
            sizes[v] *= f
        if max(sizes) <= max_qt_entries:
            edges = [(u, v, ng, nw) for (u, v), (ng, nw) in per.items() if ng + nw > 0]
            net = _edge_network(n_sub, edges, k, int(rng.integers(0, 2 ** 31)), dt,
                                f"rand{seed}")
            net.meta["topology"] = "grid" if grid else "ring"
            return net
    raise RuntimeError("could not draw a network within the caps")


def random_batch(n: int, seed: int = 0, **kw):
    """``n`` independent random networks (the batched workload)."""
    return [random_htn(seed * 100003 + i, **kw) for i in range(n)]


def rank1_htn(net: HTN, seed: int = 0, signed: bool = True):
    """The same index structure with every tensor replaced by an outer product
    of seeded random vectors, one per axis (entries of magnitude in [0.5, 1.5],
    random signs unless ``signed`` is False).  Returns (network, factors) where
    factors[t][ax] is the vector of tensor t's axis ax."""
    rng = np.random.default_rng([seed, 0xA11])
    tensors, factors = [], []
    for t in net.tensors:
        vecs = [rng.uniform(0.5, 1.5, size=n) * (rng.choice([-1.0, 1.0], size=n) if signed else 1.0)
                for n in t.data.shape]
        arr = np.ones((), dtype=np.float64)
        for v in vecs:
            arr = np.multiply.outer(arr, v)
        tensors.append(Tensor(t.kind, t.inds, np.ascontiguousarray(arr).astype(t.data.dtype)))
        factors.append(vecs)
    return HTN(tensors, net.output, name=net.name + "_rank1", meta=dict(net.meta)), factors


def rank1_qts_htn(net: HTN, seed: int = 0, lo: float = 0.5, hi: float = 1.5):
    """The same network with every QT replaced by an outer product of seeded
    positive vectors (entries ~U[lo, hi]), one per axis, while the QPD
    coefficient tensors keep their exact signed entries.  Each cut's sum then
    factorises (sum_g u_g c_g v_g for a gate cut, u^T C v for a wire cut), so
    the contraction has a closed form, and the only signs are the QPD
    coefficients'.  Returns (network, factors) with factors[t][ax] the vector
    of QT t's axis ax (None for a CT)."""
    rng = np.random.default_rng([seed, 0xC7])
    tensors, factors = [], []
    for t in net.tensors:
        if t.kind == "CT":
            tensors.append(t)
            factors.append(None)
            continue
        vecs = [rng.uniform(lo, hi, size=n) for n in t.data.shape]
        arr = np.ones((), dtype=np.float64)
        for v in vecs:
            arr = np.multiply.outer(arr, v)
        tensors.append(Tensor(t.kind, t.inds, np.ascontiguousarray(arr).astype(t.data.dtype)))
        factors.append(vecs)
    return HTN(tensors, net.output, name=net.name + "_rank1qt", meta=dict(net.meta)), factors


def tiny_random_htn(seed: int, n_tensors=4, n_indices=6, max_dim=3,
                    n_output=1, max_rank=4) -> HTN:
    """A tiny random network with hyper-indices (an index on 1..3 tensors),
    small dims, for brute-force checks."""
    rng = np.random.default_rng([seed, 0x7177])
    dims = {i: int(rng.integers(1, max_dim + 1)) for i in range(n_indices)}
    inds = [[] for _ in range(n_tensors)]
    for i in range(n_indices):
        deg = int(rng.integers(1, 4))
        for t in rng.choice(n_tensors, size=min(deg, n_tensors), replace=False):
            if len(inds[t]) < max_rank:
                inds[int(t)].append(i)
    for t in range(n_tensors):
        if not inds[t]:
            inds[t].append(int(rng.integers(0, n_indices)))
    used = sorted({i for x in inds for i in x})
    out = tuple(int(i) for i in rng.choice(used, size=min(n_output, len(used)),
                                           replace=False)) if n_output else ()
    tensors = []
    for t in range(n_tensors):
        shape = tuple(dims[i] for i in inds[t])
        tensors.append(Tensor("QT", tuple(inds[t]), rng.uniform(-1, 1, size=shape)))
    return HTN(tensors, out, name=f"tiny{seed}")
