"""OpenQASM 2 front end (Sec. 4, toQASM): text in and out, no GPU.

The export is pinned to the text the paper prints for its Bell circuit
(tests/golden/bell_toqasm.qasm); the readings of u1/u2/open controls are pinned to the
gate matrices of the oracle; round trips keep every angle bit for bit."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates
from workloads import Op

import golden_io as G
from paper_2503_03016_gb300.qasm import from_qasm, to_qasm, _eval_angle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bell_toqasm.qasm")


def golden_lines():
    with open(GOLDEN) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("//")]


def fields(ops):
    return [(o.kind, tuple(o.qubits), tuple(float(p) for p in o.params),
             None if o.ctrl_states is None else tuple(o.ctrl_states)) for o in ops]


def test_export_matches_paper_bell_listing():
    ops = G.ops("h 0; cnot 0 1; measure 0; measure 1")
    assert to_qasm(2, ops).strip().split("\n") == golden_lines()


def test_import_of_paper_listing_gives_bell_circuit():
    with open(GOLDEN) as f:
        n, ops = from_qasm(f.read())
    assert n == 2
    assert fields(ops) == fields(G.ops("h 0; cnot 0 1; measure 0; measure 1"))
    res, pr, _ = oracle.simulate(n, ops, "00")
    assert res == ["00", "11"]
    np.testing.assert_allclose(pr, [0.5, 0.5], atol=1e-15)


@pytest.mark.parametrize("text,want", [
    ("pi", math.pi), ("pi/2", math.pi / 2), ("-pi/4", -math.pi / 4), ("2*pi/3", 2 * math.pi / 3),
    ("(1+2)*pi", 3 * math.pi), ("2^3", 8.0), ("2^3^2", 2.0 ** 9), ("-2^2", -4.0),
    ("1.5e-3", 1.5e-3), (".25", 0.25), ("3.", 3.0), ("pi - -pi", 2 * math.pi), ("1/4/2", 0.125),
])
def test_angle_expressions(text, want):
    assert _eval_angle(text) == want


@pytest.mark.parametrize("bad", ["", "pi pi", "(pi", "pi)", "2**3", "sin(pi)", "1+", "x"])
def test_bad_angle_expressions(bad):
    with pytest.raises(ValueError):
        _eval_angle(bad)


def test_header_comments_registers_and_broadcast():
    text = """OPENQASM 2.0;
include "qelib1.inc";  // standard library
qreg a[2];
qreg b[3];
creg c[5];
h a;               // both qubits of a
cx a[1], b[0];
barrier a, b;
cx a, b[1];        // a[0] -> b[1], a[1] -> b[1]
measure b[2] -> c[4];
reset a[0];
"""
    n, ops = from_qasm(text)
    assert n == 5
    assert fields(ops) == [
        ("h", (0,), (), None), ("h", (1,), (), None), ("cnot", (1, 2), (), None),
        ("cnot", (0, 3), (), None), ("cnot", (1, 3), (), None),
        ("measure", (4,), (), None), ("reset", (0,), (), None)]


def test_parametrised_gate_readings_match_oracle_matrices():
    _, ops = from_qasm("qreg q[1]; u1(0.3) q[0]; p(-1.1) q[0]; u2(0.2, 0.7) q[0]; U(1,2,3) q[0];")
    np.testing.assert_allclose(oracle.op_matrix(ops[0])[1], np.diag([1, np.exp(0.3j)]), atol=1e-16)
    np.testing.assert_allclose(oracle.op_matrix(ops[1])[1], np.diag([1, np.exp(-1.1j)]), atol=1e-16)
    # u2(phi, lambda) = (1/sqrt 2) [[1, -e^{i lambda}], [e^{i phi}, e^{i (phi + lambda)}]]
    u2 = np.array([[1, -np.exp(0.7j)], [np.exp(0.2j), np.exp(0.9j)]]) / np.sqrt(2)
    np.testing.assert_allclose(oracle.op_matrix(ops[2])[1], u2, atol=1e-15)
    np.testing.assert_allclose(oracle.op_matrix(ops[3])[1], gates.u3(1, 2, 3), atol=0)


def test_round_trip_every_kind_bit_exact():
    rng = np.random.default_rng(7)
    n = 5
    ops = []
    for k in ("h", "x", "y", "z", "s", "sdg", "t", "tdg"):
        ops.append(Op(k, (int(rng.integers(n)),)))
    for k in ("rx", "ry", "rz"):
        ops.append(Op(k, (int(rng.integers(n)),), (float(rng.uniform(-7, 7)),)))
    ops.append(Op("u3", (2,), tuple(float(x) for x in rng.uniform(0, 2 * np.pi, 3))))
    ops += [Op("cnot", (3, 1)), Op("cz", (0, 4)), Op("swap", (2, 0)),
            Op("cp", (1, 4), (float(rng.uniform(0, 7)),)), Op("mcx", (0, 2, 3), ctrl_states=(1, 1)),
            Op("measure", (2,)), Op("reset", (3,))]
    n2, back = from_qasm(to_qasm(n, ops, header=True))
    assert n2 == n
    assert fields(back) == fields(ops)


def test_parameter_indices_are_resolved():
    ops = W.ansatz(3, 1, ring=False)
    params = W.ansatz_params(3, 1, seed=9)
    _, back = from_qasm(to_qasm(3, ops, params=params))
    for o, b in zip(ops, back):
        if o.param_index is not None:
            assert b.params == (float(params[o.param_index]),)
    with pytest.raises(ValueError):
        to_qasm(3, ops)


def test_open_controls_and_basis_measurements_are_equivalent():
    """Exported open controls (X around ccx) and X/Y measurements (basis change
    around a Z measurement) give the same branches as the original ops."""
    v = W.random_state(3, seed=3)
    ops = [Op("h", (0,)), Op("mcx", (0, 1, 2), ctrl_states=(0, 1)), Op("ry", (1,), (0.4,)),
           Op("mcx", (2, 0), ctrl_states=(0,)), Op("measure_x", (1,)), Op("measure_y", (2,))]
    r0, p0, s0 = oracle.simulate(3, ops, v)
    _, back = from_qasm(to_qasm(3, ops))
    r1, p1, s1 = oracle.simulate(3, back, v)
    assert r0 == r1
    np.testing.assert_allclose(p0, p1, atol=1e-14)
    for a, b in zip(s0, s1):
        np.testing.assert_allclose(a, b, atol=1e-14)


@pytest.mark.parametrize("ops", [[Op("u1q", (0,), matrix=np.eye(2))], [Op("mcx", (0, 1, 2, 3))],
                                 [Op("ctrl", (0, 1), matrix=np.eye(2))], [Op("h", (7,))]])
def test_export_rejects_what_qelib1_cannot_say(ops):
    with pytest.raises(ValueError):
        to_qasm(4, ops)


@pytest.mark.parametrize("text", [
    "h q[0];",                                   # no register
    "qreg q[2]; h q[2];",                        # index out of range
    "qreg q[2]; gate foo a { h a; } foo q[0];",  # gate definitions
    "qreg q[2]; creg c[2]; if (c==1) x q[0];",   # classical condition
    "qreg q[2]; rx q[0];",                       # missing angle
    "qreg q[2]; cx q[0], q[0];",                 # repeated qubit
    "qreg q[2]; qreg r[3]; cx q, r;",            # register sizes differ
    "qreg q[2]; qreg q[2];",                     # declared twice
    "qreg q[2]; crz(0.1) q[0], q[1];",           # not in the subset
])
def test_import_errors(text):
    with pytest.raises(ValueError):
        from_qasm(text)
