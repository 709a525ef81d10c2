"""Pins for the QT evaluator oracle (section 4.1 QTs; section 6.2 Step 2):
density matrices against signed branches, closed forms, the statevector
simulator, and the tiny knitting circuit."""
import numpy as np
import pytest

from oracle import knit, knit_programs, qpd, qt_eval, sim


def _rand_u(rng):
    a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_program(seed, n=None, n_ops=10, k=3):
    rng = np.random.default_rng([seed, 0x0E7A])
    n = n or int(rng.integers(2, 5))
    cuts, ops = [], []
    n_gate = int(rng.integers(0, 3))
    free = list(rng.permutation(n))
    prep = free.pop() if rng.uniform() < 0.5 and free else None
    meas = free.pop() if rng.uniform() < 0.5 and free else None
    for g in range(n_gate):
        cuts.append(("gate",))
    if prep is not None:
        cuts.append(("prepare", int(prep)))
    if meas is not None:
        cuts.append(("measure", int(meas)))
    gate_ops = [("gate_cut", int(rng.integers(0, n)), g, int(rng.integers(0, 2))) for g in range(n_gate)]
    for _ in range(n_ops):
        if rng.uniform() < 0.6:
            ops.append(("u1", int(rng.integers(0, n)), _rand_u(rng)))
        elif n > 1:
            a, b = rng.choice(n, 2, replace=False)
            ops.append(("cz", int(a), int(b)))
    for op in gate_ops:
        ops.insert(int(rng.integers(0, len(ops) + 1)), op)
    paulis = []
    for _ in range(k):
        s = [str(rng.choice(list("IXYZ"))) for _ in range(n)]
        if meas is not None:
            s[meas] = "I"
        paulis.append("".join(s))
    return {"n": n, "ops": ops, "cuts": cuts, "paulis": paulis}


@pytest.mark.parametrize("seed", range(12))
def test_branching_equals_density_matrix(seed):
    p = random_program(seed)
    np.testing.assert_allclose(qt_eval.qt_branching(p), qt_eval.qt_density(p), rtol=0, atol=1e-12)


def test_closed_form_without_cuts():
    th = 0.7
    p = {"n": 1, "ops": [("u1", 0, sim.ry(th))], "cuts": [], "paulis": ["Z", "X", "Y"]}
    got = qt_eval.qt_branching(p)
    np.testing.assert_allclose(got, [np.cos(th), np.sin(th), 0.0], atol=1e-15)


def test_statevector_agreement_without_cuts():
    p = random_program(3, n=4, n_ops=14, k=4)
    p["cuts"] = []
    p["ops"] = [op for op in p["ops"] if op[0] != "gate_cut"]
    p["paulis"] = [s.replace("I", "Z") for s in p["paulis"]]
    sv = sim.StateVector(4)
    for op in p["ops"]:
        sv.unitary(op[2] if op[0] == "u1" else sim.CZ, [op[1]] if op[0] == "u1" else [op[1], op[2]])
    want = [sv.expectation({q: {"X": sim.X, "Y": sim.Y, "Z": sim.Z}[c] for q, c in enumerate(s)}).real
            for s in p["paulis"]]
    np.testing.assert_allclose(qt_eval.qt_branching(p), want, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 3])
def test_tiny_knitting_circuit(seed):
    ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, size=48)
    TA, TB = knit.subcircuit_tensors(ang)
    qa = qt_eval.qt_branching(knit_programs.program_a(ang))[0]
    qb = qt_eval.qt_branching(knit_programs.program_b(ang))[0]
    np.testing.assert_allclose(qa, TA, atol=1e-12)
    np.testing.assert_allclose(qb, TB, atol=1e-12)
    val = knit.knit_brute_force(qa, qb, qpd.cz_coefficients(), qpd.wire_coefficients())
    assert abs(val - knit.uncut_expectation(ang)) <= 1e-12
