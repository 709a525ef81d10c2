"""Pins for the QPD coefficient tensors and the cost formulas (section 2.1,
section 4.1 Eq. wire-tensor, section 4.2)."""
import numpy as np
import pytest

from oracle import qpd
import synth


def test_gate_qpd_choi_equals_cz():
    lhs = qpd.choi_two_qubit(qpd.cz_qpd_channel())
    rhs = qpd.choi_two_qubit(qpd.cz_channel())
    assert np.abs(lhs - rhs).max() < 1e-14


@pytest.mark.parametrize("i", range(6))
def test_gate_qpd_each_coefficient_matters(i):
    # flipping the sign of any one term breaks the identity
    terms = qpd.cz_qpd_terms()
    c = [t[0] for t in terms]
    c[i] = -c[i]
    chans = [qpd._local_pair(a, b) for _, a, b in terms]
    bad = qpd.choi_two_qubit(lambda r: sum(ci * f(r) for ci, f in zip(c, chans)))
    good = qpd.choi_two_qubit(qpd.cz_channel())
    assert np.abs(bad - good).max() > 0.1


def test_gate_qpd_counts(gold):
    c = qpd.cz_coefficients()
    assert len(c) == gold("gate_qpd_terms")
    # gamma = sum |c| = 3, so the sampling overhead base is gamma^2 = 9
    assert np.abs(c).sum() ** 2 == pytest.approx(gold("gate_sampling_base"), abs=1e-14)


def test_wire_tensor_matches_paper(gold):
    cw = qpd.wire_coefficients()
    for r, name in enumerate("IZXY"):
        assert tuple(cw[r]) == gold(f"wire_ct_row_{name}")


def test_wire_tensor_is_identity_channel_and_orientation_matters():
    ident = qpd.choi_one_qubit(lambda r: r)
    cw = qpd.wire_coefficients()
    good = qpd.choi_one_qubit(qpd.wire_channel(cw))
    assert np.abs(good - ident).max() < 1e-14
    bad = qpd.choi_one_qubit(qpd.wire_channel(cw.T))
    assert np.abs(bad - ident).max() > 0.1


def test_synth_coefficients_are_the_oracle_values():
    # the derivation evaluates cos^2(pi/4) etc. in floating point (one ulp)
    assert np.abs(synth.GATE_CT - qpd.cz_coefficients()).max() <= 2e-16
    assert np.array_equal(synth.WIRE_CT, qpd.wire_coefficients())


def test_naive_cost_formula_reproduces_paper(gold):
    n_c = qpd.naive_instances(4, 1)
    assert n_c == gold("naive_instances_5cut")
    assert qpd.naive_pp_flops(n_c, gold("naive_s"), gold("naive_n_g")) == gold("naive_pp_flops_5cut")
    # section 4.2: each QT pair (6x6 and 4x6x6 tensors joined by two gate
    # cuts, the wire index left open) costs |C_loc| (s + n_g - 1) with
    # |C_loc| = 6*6*4, s = 2, n_g = 2
    assert qpd.naive_pp_flops(qpd.naive_instances(2, 0) * 4, 2, 2) == gold("htn_example_pair_cost")
