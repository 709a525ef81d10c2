"""The two subcircuits of the tiny cut circuit (``oracle.knit``) as QT
programs (``oracle.qt_eval`` format; test infrastructure only).  Their QTs
are T_A[g, a] and T_B[g, b] of ``oracle.knit`` with a leading observable axis
of size 1."""
from __future__ import annotations

import numpy as np

from . import sim


def _rot(angles, layer, q):
    t, p = angles[layer, q]
    return sim.rz(p) @ sim.ry(t)


def program_a(angles):
    """qubits 0, 1, 2 and the head of wire 3 (qubit 3)."""
    a = np.asarray(angles, dtype=np.float64).reshape(3, 8, 2)
    ops = [("u1", q, _rot(a, 0, q)) for q in range(4)]
    ops += [("cz", q, q + 1) for q in range(3)]
    ops += [("gate_cut", 3, 0, 0)]                       # CZ(3,4) of chain 1, first factor
    ops += [("u1", q, _rot(a, 1, q)) for q in range(4)]
    ops += [("cz", q, q + 1) for q in range(3)]          # chain 2 up to CZ(2,3)
    ops += [("u1", q, _rot(a, 2, q)) for q in range(3)]
    return {"n": 4, "ops": ops, "cuts": [("gate",), ("measure", 3)], "paulis": ["ZZZI"]}


def program_b(angles):
    """qubits 4..7 (local 0..3) and the tail of wire 3 (local 4)."""
    a = np.asarray(angles, dtype=np.float64).reshape(3, 8, 2)
    ops = [("u1", q - 4, _rot(a, 0, q)) for q in range(4, 8)]
    ops += [("gate_cut", 0, 0, 1)]                       # CZ(3,4) of chain 1, second factor
    ops += [("cz", q, q + 1) for q in range(3)]
    ops += [("u1", q - 4, _rot(a, 1, q)) for q in range(4, 8)]
    ops += [("cz", 4, 0)]                                # CZ(3,4) of chain 2 (tail, qubit 4)
    ops += [("cz", q, q + 1) for q in range(3)]
    ops += [("u1", 4, _rot(a, 2, 3))]
    ops += [("u1", q - 4, _rot(a, 2, q)) for q in range(4, 8)]
    return {"n": 5, "ops": ops, "cuts": [("gate",), ("prepare", 4)], "paulis": ["ZZZZZ"]}
