"""The tiny cut circuit, its subcircuit tensors, and brute-force knitting.

Circuit (an EfficientSU2-style hardware-efficient ansatz on 8 qubits):
three rotation layers [RY(theta), RZ(phi) on every qubit] separated by two
linear CZ chains (0,1),(1,2),...,(6,7); observable Z on every qubit.  The
final rotation layer matters: without it the last CZ chain commutes with
Z^(x)8 and the check would be vacuous.  48 angles, in (layer, qubit, RY then
RZ) order, are passed in by the caller (the test draws them from a seed).

Cuts (the reading of a '2 subcircuits, 1 gate cut + 1 wire cut' split):
* gate cut on CZ(3,4) of the first CZ chain, decomposed with the 6-term QPD
  of ``oracle.qpd`` (section 2.1);
* wire cut on qubit 3 right after CZ(2,3) of the second chain, decomposed with
  the 4x4 tensor of Eq. wire-tensor (section 4.1).
Subcircuit A = qubits 0,1,2 and the head of wire 3; it measures Z0 Z1 Z2 and
the wire-cut basis A_a on the head of wire 3, giving T_A[g, a].  Subcircuit B
= the tail of wire 3 (prepared in B_b) and qubits 4..7; it measures Z on all
five wires, giving T_B[g, b].  Then

    <O> = sum_{g,a,b} c_g[g] c_w[a,b] T_A[g,a] T_B[g,b]

which is the h-TN of four tensors with the 6-dim hyper-index g (section 4.1).
``knit_brute_force`` evaluates the same quantity as Eq. knitting (a sum over
the tensor product of the coefficient sets, one product of subcircuit values
per global instance).

Pinned by tests/test_oracle_knit.py: the knitted value equals the uncut
8-qubit statevector <Z^(x)8> to 1e-12, for several seeds.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import qpd, sim

N_QUBITS = 8


def _rot_layer(dev, angles, layer, qubits, qubit_map=None):
    for q in qubits:
        t, p = angles[layer, q]
        tgt = q if qubit_map is None else qubit_map[q]
        dev.unitary(sim.rz(p) @ sim.ry(t), [tgt])


def uncut_expectation(angles: np.ndarray) -> float:
    """<Z^(x)8> of the whole circuit, by statevector simulation."""
    angles = np.asarray(angles, dtype=np.float64).reshape(3, N_QUBITS, 2)
    sv = sim.StateVector(N_QUBITS)
    for layer in range(3):
        _rot_layer(sv, angles, layer, range(N_QUBITS))
        if layer < 2:
            for q in range(N_QUBITS - 1):
                sv.unitary(sim.CZ, [q, q + 1])
    val = sv.expectation({q: sim.Z for q in range(N_QUBITS)})
    return float(val.real)


def _subcircuit_a(angles, g_op, a_index):
    """T_A[g, a] for one (g, a): qubits 0,1,2 and the head of wire 3."""
    dm = sim.DensityMatrix(4)
    _rot_layer(dm, angles, 0, range(4))
    for q in range(3):
        dm.unitary(sim.CZ, [q, q + 1])  # CZ(0,1) CZ(1,2) CZ(2,3) of chain 1
    # CZ(3,4) of chain 1 is cut: the local op of this instance acts on qubit 3
    dm.rho = _apply_1q_map(dm, g_op, 3)
    _rot_layer(dm, angles, 1, range(4))
    for q in range(3):
        dm.unitary(sim.CZ, [q, q + 1])  # chain 2 up to CZ(2,3)
    # wire cut on qubit 3 here; the rest of wire 3 belongs to subcircuit B
    _rot_layer(dm, angles, 2, range(3))
    ops = {0: sim.Z, 1: sim.Z, 2: sim.Z, 3: qpd.WIRE_MEASURE[a_index]}
    return dm.expectation(ops).real


def _subcircuit_b(angles, g_op, b_index):
    """T_B[g, b] for one (g, b): qubits 4..7 (local 0..3) and the tail of wire 3
    (local 4, prepared in state B_b)."""
    qmap = {4: 0, 5: 1, 6: 2, 7: 3}
    dm = sim.DensityMatrix(4)
    _rot_layer(dm, angles, 0, range(4, 8), qmap)
    # chain 1: CZ(3,4) cut -> local op on qubit 4 first, then CZ(4,5)..(6,7)
    dm.rho = _apply_1q_map(dm, g_op, 0)
    for q in range(4, 7):
        dm.unitary(sim.CZ, [qmap[q], qmap[q + 1]])
    _rot_layer(dm, angles, 1, range(4, 8), qmap)
    t = dm.add_qubit(qpd.WIRE_PREPARE[b_index])  # tail of wire 3
    dm.unitary(sim.CZ, [t, qmap[4]])              # CZ(3,4) of chain 2
    for q in range(4, 7):
        dm.unitary(sim.CZ, [qmap[q], qmap[q + 1]])
    # final rotations on wire 3's tail and on qubits 4..7
    tt, pp = angles[2, 3]
    dm.unitary(sim.rz(pp) @ sim.ry(tt), [t])
    _rot_layer(dm, angles, 2, range(4, 8), qmap)
    return dm.expectation({q: sim.Z for q in range(5)}).real


def _apply_1q_map(dm, f, q):
    """Apply a linear map f (2x2 -> 2x2) to qubit q of the density matrix."""
    n = dm.n
    rho = np.moveaxis(dm.rho, [q, n + q], [0, 1])
    shp = rho.shape
    flat = rho.reshape(2, 2, -1)
    out = np.empty_like(flat)
    for j in range(flat.shape[2]):
        out[:, :, j] = f(flat[:, :, j])
    return np.moveaxis(out.reshape(shp), [0, 1], [q, n + q])


def subcircuit_tensors(angles: np.ndarray):
    """(T_A[6,4], T_B[6,4]) of the two subcircuits (FP64)."""
    angles = np.asarray(angles, dtype=np.float64).reshape(3, N_QUBITS, 2)
    terms = qpd.cz_qpd_terms()
    TA = np.zeros((6, 4))
    TB = np.zeros((6, 4))
    for g, (_, fa, fb) in enumerate(terms):
        for a in range(4):
            TA[g, a] = _subcircuit_a(angles, fa, a)
        for b in range(4):
            TB[g, b] = _subcircuit_b(angles, fb, b)
    return TA, TB


def knit_brute_force(TA, TB, cg, cw) -> float:
    """Eq. knitting: sum over every global instance (g, a, b) of its
    coefficient times the product of the two subcircuit results."""
    total = 0.0
    for g, a, b in itertools.product(range(6), range(4), range(4)):
        coeff = cg[g] * cw[a, b]
        total += coeff * TA[g, a] * TB[g, b]
    return float(total)
