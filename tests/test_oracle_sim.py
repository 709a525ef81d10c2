"""Pins for the oracle's tiny simulator: closed forms and invariants."""
import numpy as np
import pytest

from oracle import sim


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, np.pi, 5.1])
def test_ry_closed_forms(theta):
    sv = sim.StateVector(1)
    sv.unitary(sim.ry(theta), [0])
    assert sv.expectation({0: sim.Z}).real == pytest.approx(np.cos(theta), abs=1e-14)
    assert sv.expectation({0: sim.X}).real == pytest.approx(np.sin(theta), abs=1e-14)
    dm = sim.DensityMatrix(1)
    dm.unitary(sim.ry(theta), [0])
    assert dm.expectation({0: sim.Z}).real == pytest.approx(np.cos(theta), abs=1e-14)


@pytest.mark.parametrize("theta,phi", [(0.4, 1.1), (2.0, -0.7)])
def test_rz_after_ry(theta, phi):
    # RZ(phi) rotates the Bloch vector about Z: <Y> = sin(theta) sin(phi)
    sv = sim.StateVector(1)
    sv.unitary(sim.rz(phi) @ sim.ry(theta), [0])
    assert sv.expectation({0: sim.Y}).real == pytest.approx(np.sin(theta) * np.sin(phi), abs=1e-14)
    assert sv.expectation({0: sim.X}).real == pytest.approx(np.sin(theta) * np.cos(phi), abs=1e-14)


def test_cz_on_plus_plus():
    # CZ|++> = (|0+> + |1->)/sqrt2: <X Z> = 1, <X X> = 0, <Z Z> = 0
    for cls in (sim.StateVector, sim.DensityMatrix):
        d = cls(2)
        h = sim.ry(np.pi / 2)
        d.unitary(h, [0])
        d.unitary(h, [1])
        d.unitary(sim.CZ, [0, 1])
        assert d.expectation({0: sim.X, 1: sim.Z}).real == pytest.approx(1.0, abs=1e-14)
        assert d.expectation({1: sim.X, 0: sim.Z}).real == pytest.approx(1.0, abs=1e-14)
        assert d.expectation({0: sim.X, 1: sim.X}).real == pytest.approx(0.0, abs=1e-14)


def test_density_matches_statevector_random_circuit():
    rng = np.random.default_rng(5)
    n = 4
    sv, dm = sim.StateVector(n), sim.DensityMatrix(n)
    for _ in range(12):
        q = int(rng.integers(0, n))
        U = sim.rz(rng.uniform(0, 6)) @ sim.ry(rng.uniform(0, 6))
        sv.unitary(U, [q])
        dm.unitary(U, [q])
        a = int(rng.integers(0, n - 1))
        sv.unitary(sim.CZ, [a, a + 1])
        dm.unitary(sim.CZ, [a, a + 1])
    for ops in ({0: sim.Z}, {1: sim.X, 3: sim.Y}, {q: sim.Z for q in range(n)}):
        assert dm.expectation(ops).real == pytest.approx(sv.expectation(ops).real, abs=1e-13)
    assert dm.trace().real == pytest.approx(1.0, abs=1e-14)


def test_signed_measurement_and_preparation():
    dm = sim.DensityMatrix(1)
    dm.unitary(sim.ry(0.9), [0])
    dm.signed_measure_z(0)
    # Tr(P0 rho) - Tr(P1 rho) = <Z>
    assert dm.trace().real == pytest.approx(np.cos(0.9), abs=1e-14)
    d2 = sim.DensityMatrix(1)
    q = d2.add_qubit(sim.KET["+"])
    assert q == 1
    assert d2.expectation({1: sim.X}).real == pytest.approx(1.0, abs=1e-14)
    assert d2.expectation({0: sim.Z}).real == pytest.approx(1.0, abs=1e-14)
    d3 = sim.DensityMatrix(1)
    d3.add_qubit(sim.KET["i"])
    assert d3.expectation({1: sim.Y}).real == pytest.approx(1.0, abs=1e-14)
