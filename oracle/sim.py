"""Tiny FP64 density-matrix and statevector simulator (oracle, test-only).

Circuit knitting (section 2.1) reconstructs an expectation value <O> of a large
circuit from the expectation values <O_j^i> of its subcircuit instances.  To
check that reconstruction we need exact expectation values of small circuits,
including the non-unitary pieces the cuts insert: signed Z measurements and
state preparations (section 2.1, Fig. qpd; section 4.1 Eq. wire-tensor).

Conventions: qubit q is tensor axis q of a ``2**n``-dimensional vector in
big-endian order (qubit 0 is the most significant bit).  A density matrix is
kept as a ``(2,)*2n`` array, axes ``[k_0..k_{n-1}, b_0..b_{n-1}]``.

Pinned by tests/test_oracle_sim.py (closed forms, trace preservation,
density-matrix vs statevector agreement).
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)


def ry(theta: float) -> np.ndarray:
    """exp(-i theta Y / 2)."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    """exp(-i theta Z / 2)."""
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]],
                    dtype=np.complex128)


def expz(phi: float) -> np.ndarray:
    """exp(i phi Z)."""
    return np.array([[np.exp(1j * phi), 0], [0, np.exp(-1j * phi)]],
                    dtype=np.complex128)


CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)

# The four prepared states of the wire cut, in the order of Eq. wire-tensor:
# |0>, |1>, |+>, |i>.
KET = {
    "0": np.array([1, 0], dtype=np.complex128),
    "1": np.array([0, 1], dtype=np.complex128),
    "+": np.array([1, 1], dtype=np.complex128) / np.sqrt(2),
    "i": np.array([1, 1j], dtype=np.complex128) / np.sqrt(2),
}


class DensityMatrix:
    """rho on n qubits; every operation is an explicit linear map on rho."""

    def __init__(self, n: int):
        self.n = n
        rho = np.zeros((2,) * (2 * n), dtype=np.complex128)
        rho[(0,) * (2 * n)] = 1.0
        self.rho = rho

    def matrix(self) -> np.ndarray:
        d = 2 ** self.n
        return self.rho.reshape(d, d)

    def _apply_left_right(self, L: np.ndarray, R: np.ndarray, qubits) -> None:
        """rho -> L rho R on the given qubits (L, R act on len(qubits) qubits)."""
        k = len(qubits)
        n = self.n
        Lt = L.reshape((2,) * (2 * k))
        Rt = R.reshape((2,) * (2 * k))
        # left multiply: contract L's input axes with rho's ket axes
        rho = np.tensordot(Lt, self.rho, axes=(list(range(k, 2 * k)), list(qubits)))
        # tensordot put L's output axes first; move them back into place
        rho = np.moveaxis(rho, list(range(k)), list(qubits))
        # right multiply: contract rho's bra axes with R's output axes
        bra = [n + q for q in qubits]
        rho = np.tensordot(rho, Rt, axes=(bra, list(range(k))))
        rho = np.moveaxis(rho, list(range(2 * n - k, 2 * n)), bra)
        self.rho = rho

    def unitary(self, U: np.ndarray, qubits) -> None:
        self._apply_left_right(U, U.conj().T, qubits)

    def signed_measure_z(self, q: int) -> None:
        """rho -> P0 rho P0 - P1 rho P1 (measurement whose outcome sign weights
        the result); a linear, trace-annihilating-on-average map."""
        a = DensityMatrix.__new__(DensityMatrix)
        a.n, a.rho = self.n, self.rho.copy()
        a._apply_left_right(P0, P0, [q])
        self._apply_left_right(P1, P1, [q])
        self.rho = a.rho - self.rho

    def add_qubit(self, ket: np.ndarray) -> int:
        """Append a fresh qubit prepared in ``ket``; returns its index."""
        n = self.n
        r = self.rho.reshape((2 ** n, 2 ** n))
        s = np.outer(ket, ket.conj())
        new = np.kron(r, s)  # new qubit is least significant -> index n
        self.n = n + 1
        self.rho = new.reshape((2,) * (2 * self.n))
        return n

    def expectation(self, ops: dict) -> complex:
        """Tr(O rho) for O = tensor product of single-qubit ops (identity elsewhere)."""
        full = np.array([[1.0]], dtype=np.complex128)
        for q in range(self.n):
            full = np.kron(full, ops.get(q, I2))
        return complex(np.trace(full @ self.matrix()))

    def trace(self) -> complex:
        return complex(np.trace(self.matrix()))


class StateVector:
    def __init__(self, n: int):
        self.n = n
        psi = np.zeros((2,) * n, dtype=np.complex128)
        psi[(0,) * n] = 1.0
        self.psi = psi

    def unitary(self, U: np.ndarray, qubits) -> None:
        k = len(qubits)
        Ut = U.reshape((2,) * (2 * k))
        psi = np.tensordot(Ut, self.psi, axes=(list(range(k, 2 * k)), list(qubits)))
        self.psi = np.moveaxis(psi, list(range(k)), list(qubits))

    def expectation(self, ops: dict) -> complex:
        phi = self.psi
        for q, O in ops.items():
            phi = np.moveaxis(np.tensordot(O, phi, axes=([1], [q])), 0, q)
        return complex(np.vdot(self.psi, phi))
