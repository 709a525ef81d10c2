"""QT evaluation: the expectation values of a subcircuit's instances (oracle;
test infrastructure only).

Section 4.1 makes each subcircuit a quantum tensor (QT): one axis per cut
touching it plus the observable index, its entries the expectation values of
the subcircuit's instances.  Section 6.2 (Step 2) evaluates the QTs on QPUs
or simulators; here the evaluation is exact.

A program is the subcircuit: ``n`` qubits (qubit 0 the most significant bit,
as in ``oracle.sim``), a list of operations, a list of cuts and a list of
observables (Pauli strings over I, X, Y, Z, one character per qubit).
Operations:

* ``("u1", q, U)``: a 2 x 2 unitary on qubit q;
* ``("cz", q0, q1)``;
* ``("gate_cut", q, c, side)``: the local operation of gate cut c on qubit q
  for the cut's index value: term g of the CZ decomposition of
  ``oracle.qpd`` (section 2.1), its first factor (side 0) or its second
  (side 1), each followed by e^{-i pi/4 Z}.

Cuts (the QT's axes after the observable axis, in order): ``("gate",)``
(dim 6), ``("measure", q)`` (dim 4: the wire leaves the subcircuit at qubit
q; the instance measures A = I, Z, X, Y there, i.e. the observable carries A
on q) and ``("prepare", q)`` (dim 4: the wire enters at qubit q, prepared in
|0>, |1>, |+>, |i> before the first operation).  An observable must have I on
measured qubits.

QT[k, v_0, v_1, ...] = Re Tr(O_k' E_v(rho_0)), rho_0 the product of the
prepared states and |0> elsewhere, E_v the operations with cut values v, and
O_k' observable k with A_{v_c} on each measured qubit.

Two evaluators:

* ``qt_density``: the definition with density matrices and the maps of
  ``oracle.qpd`` (small n).
* ``qt_branching``: pure states; a signed measurement M_Z(rho) =
  P0 rho P0 - P1 rho P1 is carried as two branches, the projected
  (unnormalised) states P_s |psi>, whose expectation values are added with
  sign s.  This is what the CUDA evaluator computes; it scales to 15 qubits.

Pinned by tests/test_oracle_qt_eval.py: the two evaluators agree on random
programs; without cuts they reduce to ``sim.StateVector`` expectations and
closed forms; the two subcircuits of ``oracle.knit`` give its tensors, whose
knitting equals the uncut circuit's expectation value.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import qpd, sim

GATE_DIM, WIRE_DIM = 6, 4


def _dims(prog):
    return [GATE_DIM if c[0] == "gate" else WIRE_DIM for c in prog["cuts"]]


def _pauli(ch):
    return {"I": sim.I2, "X": sim.X, "Y": sim.Y, "Z": sim.Z}[ch]


def _apply_map(dm, f, q):
    """a linear map f on 2 x 2 operators applied to qubit q of dm.rho"""
    n = dm.n
    rho = np.moveaxis(dm.rho, [q, n + q], [0, 1])
    shp = rho.shape
    flat = rho.reshape(2, 2, -1)
    out = np.empty_like(flat)
    for j in range(flat.shape[2]):
        out[:, :, j] = f(flat[:, :, j])
    dm.rho = np.moveaxis(out.reshape(shp), [0, 1], [q, n + q])


def _initial_kets(prog, vals):
    kets = [sim.KET["0"]] * prog["n"]
    for c, cut in enumerate(prog["cuts"]):
        if cut[0] == "prepare":
            kets[cut[1]] = qpd.WIRE_PREPARE[vals[c]]
    return kets


def _observable(prog, k, vals):
    ops = {}
    for q, ch in enumerate(prog["paulis"][k]):
        if ch != "I":
            ops[q] = _pauli(ch)
    for c, cut in enumerate(prog["cuts"]):
        if cut[0] == "measure":
            assert prog["paulis"][k][cut[1]] == "I", "observable on a measured wire qubit"
            ops[cut[1]] = qpd.WIRE_MEASURE[vals[c]]
    return ops


def qt_density(prog) -> np.ndarray:
    """QT[k, v...] by density-matrix simulation (the definition)."""
    n, K = prog["n"], len(prog["paulis"])
    dims = _dims(prog)
    terms = qpd.cz_qpd_terms()
    out = np.zeros([K] + dims)
    for vals in itertools.product(*[range(d) for d in dims]):
        kets = _initial_kets(prog, vals)
        psi0 = kets[0]
        for k_ in kets[1:]:
            psi0 = np.kron(psi0, k_)
        dm = sim.DensityMatrix(n)
        dm.rho = np.outer(psi0, psi0.conj()).reshape((2,) * (2 * n))
        for op in prog["ops"]:
            if op[0] == "u1":
                dm.unitary(np.asarray(op[2], dtype=np.complex128), [op[1]])
            elif op[0] == "cz":
                dm.unitary(sim.CZ, [op[1], op[2]])
            else:
                _, q, c, side = op
                f = terms[vals[c]][1 + side]
                _apply_map(dm, f, q)
        for k in range(K):
            out[(k,) + vals] = dm.expectation(_observable(prog, k, vals)).real
    return out


# per term g of the CZ decomposition and side: the local operation as
# ("phase", d0, d1) (a diagonal unitary) or ("measure",), before the common
# e^{-i pi/4 Z}
def _local_ops():
    e = np.exp
    ident = ("phase", 1.0, 1.0)
    zz = ("phase", 1.0, -1.0)
    rp = ("phase", e(1j * np.pi / 4), e(-1j * np.pi / 4))   # e^{+i pi/4 Z}
    rm = ("phase", e(-1j * np.pi / 4), e(1j * np.pi / 4))   # e^{-i pi/4 Z}
    m = ("measure",)
    side0 = [ident, zz, m, m, rp, rm]
    side1 = [ident, zz, rp, rm, m, m]
    return side0, side1


POST = np.diag([np.exp(-1j * np.pi / 4), np.exp(1j * np.pi / 4)])  # e^{-i pi/4 Z}


def qt_branching(prog) -> np.ndarray:
    """QT[k, v...] with pure states; signed measurements as signed branches."""
    n, K = prog["n"], len(prog["paulis"])
    dims = _dims(prog)
    local = _local_ops()
    out = np.zeros([K] + dims)
    for vals in itertools.product(*[range(d) for d in dims]):
        kets = _initial_kets(prog, vals)
        psi0 = kets[0]
        for k_ in kets[1:]:
            psi0 = np.kron(psi0, k_)
        n_meas = sum(1 for op in prog["ops"] if op[0] == "gate_cut" and local[op[3]][vals[op[2]]][0] == "measure")
        acc = np.zeros(K)
        for bits in itertools.product((0, 1), repeat=n_meas):
            sv = sim.StateVector(n)
            sv.psi = psi0.reshape((2,) * n).copy()
            sign, j = 1.0, 0
            for op in prog["ops"]:
                if op[0] == "u1":
                    sv.unitary(np.asarray(op[2], dtype=np.complex128), [op[1]])
                elif op[0] == "cz":
                    sv.unitary(sim.CZ, [op[1], op[2]])
                else:
                    _, q, c, side = op
                    lo = local[side][vals[c]]
                    if lo[0] == "measure":
                        b = bits[j]
                        j += 1
                        sv.unitary(sim.P1 if b else sim.P0, [q])  # projection (not unitary)
                        sign *= -1.0 if b else 1.0
                    else:
                        sv.unitary(np.diag([lo[1], lo[2]]), [q])
                    sv.unitary(POST, [q])
            for k in range(K):
                acc[k] += sign * sv.expectation(_observable(prog, k, vals)).real
        out[(slice(None),) + vals] = acc
    return out
