"""Pin: knitting the cut 8-qubit circuit reproduces the uncut statevector
value (section 2.1 Eq. knitting; section 4.1 h-TN of one gate and one wire
cut)."""
import numpy as np
import pytest

from oracle import knit, qpd, tn


def _angles(seed):
    return np.random.default_rng(seed).uniform(0, 2 * np.pi, size=48)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_knitted_equals_uncut(seed):
    ang = _angles(seed)
    exact = knit.uncut_expectation(ang)
    TA, TB = knit.subcircuit_tensors(ang)
    cg, cw = qpd.cz_coefficients(), qpd.wire_coefficients()
    brute = knit.knit_brute_force(TA, TB, cg, cw)
    assert brute == pytest.approx(exact, abs=1e-12)
    # the same value as a contraction of the 4-tensor h-TN (g = 0, a = 1, b = 2)
    net = [((0, 1), TA), ((0, 2), TB), ((0,), cg), ((1, 2), cw)]
    for order in ([(0, 2), (1, 3), (4, 5)], [(2, 3), (0, 4), (1, 5)], [(0, 1), (2, 3), (4, 5)]):
        v = tn.contract_pairwise(net, (), order)
        assert float(v) == pytest.approx(exact, abs=1e-12)
    # the final rotation layer makes the value depend on the angles
    assert abs(exact) > 1e-6 or seed != 0


def test_wrong_wire_orientation_breaks_knitting():
    ang = _angles(7)
    exact = knit.uncut_expectation(ang)
    TA, TB = knit.subcircuit_tensors(ang)
    bad = knit.knit_brute_force(TA, TB, qpd.cz_coefficients(), qpd.wire_coefficients().T)
    assert abs(bad - exact) > 1e-4
