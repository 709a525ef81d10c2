"""Quasiprobability decompositions (QPD) of a CZ gate and of a wire (oracle).

Section 2.1 writes a cut two-qubit gate as a weighted sum of six instances of
local operations, <O> = sum_i c_i <O_1^i><O_2^i>, but prints no coefficients.
The decomposition used here follows the construction the paper cites for gate
cutting (Mitarai and Fujii) and is derived, not copied:

* CZ = e^{i pi/4} (e^{-i pi/4 Z} (x) e^{-i pi/4 Z}) e^{i pi/4 Z(x)Z}.
* For U = e^{i theta A(x)B} with A^2 = B^2 = 1,
  U rho U^+ = cos^2 rho + sin^2 (A(x)B) rho (A(x)B) + cos sin i[A(x)B, rho],
  and i[A(x)B, rho] = M_A (x) (R_B(+pi/4) - R_B(-pi/4))
                    + (R_A(+pi/4) - R_A(-pi/4)) (x) M_B,
  with R_P(phi)(rho) = e^{i phi P} rho e^{-i phi P} and M_P the signed
  projective measurement sum_s s P_s rho P_s.
* At theta = pi/4 all weights are +-1/2, giving six terms (the paper's count
  of 6, with gamma = sum|c| = 3 so that the sampling overhead is 9^k).

The wire cut uses the 4x4 classical tensor of Eq. wire-tensor (section 4.1):
rows are the measured Pauli basis A = (I, Z, X, Y) on the upstream wire,
columns the prepared state B = (|0>, |1>, |+>, |i>) downstream.

Pinned by tests/test_oracle_qpd.py: the Choi matrix of the six-term sum equals
the Choi matrix of CZ (and of the identity channel for the wire tensor, which
fails for its transpose); sum|c_g| = 3; the naive PP cost formula reproduces
the paper's 10368 and 82944 (section 2.1) and the 432 / 20 components of the
884-FLOP example (section 4.2).
"""
from __future__ import annotations

import math

import numpy as np

from . import sim

# ---------------------------------------------------------------------------
# superoperators on one qubit as functions rho(2x2) -> 2x2 matrix


def _conj(U):
    return lambda r: U @ r @ U.conj().T


def _signed_measure_z(r):
    return sim.P0 @ r @ sim.P0 - sim.P1 @ r @ sim.P1


def _compose(f, g):
    """apply f, then g"""
    return lambda r: g(f(r))


_IDENT = lambda r: r  # noqa: E731


def cz_qpd_terms():
    """The six (c_i, A_i, B_i) of the CZ gate QPD, in the fixed term order

    (I,I), (Z,Z), (M_Z, R_Z(+pi/4)), (M_Z, R_Z(-pi/4)), (R_Z(+pi/4), M_Z),
    (R_Z(-pi/4), M_Z), each followed by e^{-i pi/4 Z} on both qubits.

    The coefficients come out of the derivation in the module header:
    cos^2(pi/4), sin^2(pi/4) and +-cos(pi/4) sin(pi/4).
    """
    th = math.pi / 4
    cc, ss, cs = math.cos(th) ** 2, math.sin(th) ** 2, math.cos(th) * math.sin(th)
    post = _conj(sim.expz(-math.pi / 4))  # e^{-i pi/4 Z} on each side
    Rp = _conj(sim.expz(+math.pi / 4))
    Rm = _conj(sim.expz(-math.pi / 4))
    Zc = _conj(sim.Z)
    M = _signed_measure_z
    raw = [
        (cc, _IDENT, _IDENT),
        (ss, Zc, Zc),
        (+cs, M, Rp),
        (-cs, M, Rm),
        (+cs, Rp, M),
        (-cs, Rm, M),
    ]
    return [(c, _compose(a, post), _compose(b, post)) for (c, a, b) in raw]


def cz_coefficients() -> np.ndarray:
    """c_g of the gate-cut classical tensor (a vector over the 6-term index)."""
    return np.array([c for c, _, _ in cz_qpd_terms()], dtype=np.float64)


def wire_coefficients() -> np.ndarray:
    """c_w of Eq. wire-tensor: c_w[a, b], a = measured (I,Z,X,Y), b = prepared
    (|0>,|1>,|+>,|i>)."""
    return 0.5 * np.array([[1, 1, 0, 0],
                           [1, -1, 0, 0],
                           [-1, -1, 2, 0],
                           [-1, -1, 0, 2]], dtype=np.float64)


WIRE_MEASURE = [sim.I2, sim.Z, sim.X, sim.Y]          # A = (I, Z, X, Y)
WIRE_PREPARE = [sim.KET[s] for s in ("0", "1", "+", "i")]  # B


# ---------------------------------------------------------------------------
# Choi matrices

def _basis(d, i, j):
    e = np.zeros((d, d), dtype=np.complex128)
    e[i, j] = 1.0
    return e


def choi_two_qubit(channel) -> np.ndarray:
    """Choi matrix sum_{ij} |i><j| (x) channel(|i><j|) of a map on 4x4 matrices."""
    out = np.zeros((16, 16), dtype=np.complex128)
    for i in range(4):
        for j in range(4):
            out += np.kron(_basis(4, i, j), channel(_basis(4, i, j)))
    return out


def choi_one_qubit(channel) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    for i in range(2):
        for j in range(2):
            out += np.kron(_basis(2, i, j), channel(_basis(2, i, j)))
    return out


def _local_pair(fa, fb):
    """(fa (x) fb) acting on a 4x4 two-qubit operator (qubit 0 = left factor)."""
    def ch(r):
        t = r.reshape(2, 2, 2, 2)  # [a, b, a', b']
        out = np.zeros_like(t)
        for b in range(2):
            for bp in range(2):
                out[:, b, :, bp] = fa(t[:, b, :, bp])
        res = np.zeros_like(out)
        for a in range(2):
            for ap in range(2):
                res[a, :, ap, :] = fb(out[a, :, ap, :])
        return res.reshape(4, 4)
    return ch


def cz_qpd_channel():
    """sum_i c_i (A_i (x) B_i) as a map on two-qubit operators."""
    terms = [(c, _local_pair(a, b)) for c, a, b in cz_qpd_terms()]
    return lambda r: sum(c * f(r) for c, f in terms)


def cz_channel():
    return lambda r: sim.CZ @ r @ sim.CZ.conj().T


def wire_channel(cw: np.ndarray):
    """rho -> sum_{a,b} cw[a,b] Tr(A_a rho) |b><b|  (measure upstream, prepare
    downstream, weighted by the wire tensor)."""
    preps = [np.outer(k, k.conj()) for k in WIRE_PREPARE]

    def ch(r):
        out = np.zeros((2, 2), dtype=np.complex128)
        for a in range(4):
            ta = np.trace(WIRE_MEASURE[a] @ r)
            for b in range(4):
                out += cw[a, b] * ta * preps[b]
        return out
    return ch


# ---------------------------------------------------------------------------
# naive knitting cost (section 2.1)

def naive_instances(n_gate_cuts: int, n_wire_cuts: int,
                    gate_terms: int = 6, wire_terms: int = 8) -> int:
    """|C| = prod of per-cut instance counts (C is the tensor product of all
    coefficient vectors; a wire counts 8 instances in section 2.1)."""
    return gate_terms ** n_gate_cuts * wire_terms ** n_wire_cuts


def naive_pp_flops(n_instances: int, s: int, n_g: int) -> int:
    """|C| (s + n_g - 1) multiplications (section 2.1)."""
    return n_instances * (s + n_g - 1)
