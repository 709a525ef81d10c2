"""The GPU QT evaluator (qtpu_qt_evaluate; sections 4.1 and 6.2) against the
oracle: random programs element by element, the tiny knitting circuit's
subcircuit tensors and its knitted value, and 13- and 15-qubit programs
(state in device memory) against the oracle's branching statevector."""
import numpy as np
import pytest

from oracle import knit, knit_programs, qpd, qt_eval
from tests.test_oracle_qt_eval import random_program

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


@pytest.mark.parametrize("seed", range(12))
def test_random_programs(seed):
    from paper_2410_15080_b300 import qt_evaluate
    p = random_program(seed, n_ops=14, k=4)
    got = qt_evaluate(p).cpu().numpy()
    np.testing.assert_allclose(got, qt_eval.qt_density(p), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 3])
def test_tiny_knitting_circuit(seed):
    from paper_2410_15080_b300 import qt_evaluate
    ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, size=48)
    TA, TB = knit.subcircuit_tensors(ang)
    qa = qt_evaluate(knit_programs.program_a(ang)).cpu().numpy()[0]
    qb = qt_evaluate(knit_programs.program_b(ang)).cpu().numpy()[0]
    np.testing.assert_allclose(qa, TA, atol=1e-12)
    np.testing.assert_allclose(qb, TB, atol=1e-12)
    val = knit.knit_brute_force(qa, qb, qpd.cz_coefficients(), qpd.wire_coefficients())
    assert abs(val - knit.uncut_expectation(ang)) <= 1e-12


@pytest.mark.parametrize("n", [12, 13, 15])
def test_larger_programs(n):
    """Shared-memory state at 12 qubits, device-memory state at 13 and 15."""
    from paper_2410_15080_b300 import qt_evaluate
    p = random_program(100 + n, n=n, n_ops=3 * n, k=3)
    # keep the branching oracle cheap: at most 2 cuts
    keep = [c for c in p["cuts"]][:2]
    p["cuts"] = keep
    gate_ids = [i for i, c in enumerate(keep) if c[0] == "gate"]
    ops = []
    for op in p["ops"]:
        if op[0] == "gate_cut":
            if op[2] in gate_ids:
                ops.append(op)
        else:
            ops.append(op)
    p["ops"] = ops
    got = qt_evaluate(p).cpu().numpy()
    np.testing.assert_allclose(got, qt_eval.qt_branching(p), rtol=0, atol=1e-12)


def test_malformed_programs_are_rejected():
    from paper_2410_15080_b300 import qt_evaluate
    from paper_2410_15080_b300.htn import QTPU_EINVAL, QtpuError
    bad = [
        {"n": 16, "ops": [], "cuts": [], "paulis": ["Z" * 16]},
        {"n": 2, "ops": [("cz", 0, 0)], "cuts": [], "paulis": ["ZZ"]},
        {"n": 2, "ops": [], "cuts": [("gate",)], "paulis": ["ZZ"]},          # gate cut without its operation
        {"n": 2, "ops": [], "cuts": [("measure", 1)], "paulis": ["ZZ"]},     # observable on a measured qubit
        {"n": 2, "ops": [], "cuts": [], "paulis": ["ZQ"]},
    ]
    for p in bad:
        with pytest.raises(QtpuError) as e:
            qt_evaluate(p)
        assert e.value.status == QTPU_EINVAL
