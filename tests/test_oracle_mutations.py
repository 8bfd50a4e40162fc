"""Plants plausible mistakes in the oracle (CPU only) and checks that a pin catches
each one: the pins must fail for a dropped term, a swapped index, a transposed
operand or a wrong qubit-order convention."""
import numpy as np
import pytest

import oracle
from oracle import gates

import test_oracle_pins as P


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_swapped_two_qubit_operands(monkeypatch):
    orig = oracle.apply_2q
    monkeypatch.setattr(oracle, "apply_2q", lambda psi, a, b, U: orig(psi, b, a, U))
    _fails(P.test_2q_every_ordered_pair_vs_kron, 4)


def test_transposed_two_qubit_matrix(monkeypatch):
    orig = oracle.apply_2q
    monkeypatch.setattr(oracle, "apply_2q", lambda psi, a, b, U: orig(psi, a, b, np.asarray(U).T))
    _fails(P.test_2q_every_ordered_pair_vs_kron, 4)


def test_u3_phi_lambda_swapped(monkeypatch):
    orig = gates.u3
    monkeypatch.setattr(gates, "u3", lambda t, p, l: orig(t, l, p))
    _fails(P.test_u3_identities)


def test_control_and_target_swapped(monkeypatch):
    orig = oracle.apply_ctrl
    monkeypatch.setattr(oracle, "apply_ctrl",
                        lambda psi, c, s, t, U: orig(psi, [t] + list(c[1:]), s, c[0], U))
    _fails(P.test_paper_examples, "teleport.txt")


def test_control_states_ignored(monkeypatch):
    orig = oracle.apply_ctrl
    monkeypatch.setattr(oracle, "apply_ctrl", lambda psi, c, s, t, U: orig(psi, c, [1] * len(c), t, U))
    _fails(P.test_qec_final_state)


def test_reversed_qubit_order(monkeypatch):
    orig = oracle.apply_1q
    monkeypatch.setattr(oracle, "apply_1q",
                        lambda psi, q, U: orig(psi, int(psi.size).bit_length() - 2 - q, U))
    _fails(P.test_paper_examples, "teleport.txt")


def test_collapse_without_renormalisation(monkeypatch):
    orig = oracle.collapse
    monkeypatch.setattr(oracle, "collapse", lambda psi, q, o, Pr: orig(psi, q, o, 1.0))
    _fails(P.test_paper_examples, "bell.txt")


def test_probability_drops_imaginary_part(monkeypatch):
    monkeypatch.setattr(oracle, "probs", lambda psi: psi.real * psi.real)
    _fails(P.test_probs_definition)


def test_naive_cdf(monkeypatch):
    monkeypatch.setattr(oracle, "cdf", lambda p: np.cumsum(p))
    _fails(P.test_cdf_is_correctly_rounded_prefix)


def test_sampling_off_by_one(monkeypatch):
    orig = oracle.sample
    monkeypatch.setattr(oracle, "sample", lambda c, u: np.minimum(orig(c, u) + 1, c.size - 1).astype(np.uint64))
    _fails(P.test_sample_matches_linear_scan)


def test_qft_missing_swaps(monkeypatch):
    import workloads as W
    orig = W.qft
    monkeypatch.setattr(W, "qft", lambda n: [o for o in orig(n) if o.kind != "swap"])
    monkeypatch.setattr(P.W, "qft", W.qft)
    _fails(P.test_qft_is_scaled_inverse_fft, 3)


def test_wrong_rotation_sign(monkeypatch):
    monkeypatch.setattr(gates, "ry", lambda t: np.array([[np.cos(t / 2), np.sin(t / 2)],
                                                         [-np.sin(t / 2), np.cos(t / 2)]], dtype=complex))
    _fails(P.test_rotations_match_matrix_exponential)
