"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test ties an oracle function to something other than itself: the paper's
printed worked examples (tests/golden), the literal Kronecker formula of Sec. 3.2,
closed forms (DFT, GHZ), library routines (scipy expm, math.fsum, numpy fft),
brute force on tiny inputs, and invariants (unitarity, circuit * inverse).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates, kron
from workloads import Op

import golden_io as G

RNG = np.random.default_rng(1234)


def rand_u(d, seed):
    return W.haar_unitaries(1, d, seed)[0]


# ---------------------------------------------------------------------------
# paper worked examples (Sec. 3.3, 5.1, 5.2, 5.3, 5.4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["bell.txt", "teleport.txt", "grover.txt", "qec.txt"])
def test_paper_examples(name):
    g = G.load(name)
    n = int(g["n"])
    tol = float(g["print_tol"])
    results, probs, states = oracle.simulate(n, G.ops(g["ops"]), G.init_state(g["init"], n))
    assert results == g["results"].split()
    np.testing.assert_allclose(probs, G.fvec(g["probabilities"]), atol=tol)
    for key, val in g.items():
        if key.startswith("state."):
            st = states[results.index(key.split(".")[1])]
            np.testing.assert_allclose(st, G.cvec(val), atol=tol)
        if key.startswith("reduced."):
            bits = key.split(".")[1]
            st = states[results.index(bits)]
            red = oracle.reduced_statevector(st, [0, 1], bits)
            np.testing.assert_allclose(red, G.cvec(val), atol=tol)


def test_teleport_every_outcome_recovers_v():
    """Sec. 5.1: every branch carries v on q2 (the paper prints branch '00')."""
    g = G.load("teleport.txt")
    results, probs, states = oracle.simulate(3, G.ops(g["ops"]), G.init_state(g["init"], 3))
    v = np.array([1, 1j]) / np.sqrt(2)
    for r, st in zip(results, states):
        np.testing.assert_allclose(oracle.reduced_statevector(st, [0, 1], r), v, atol=1e-15)


def test_qec_final_state():
    """Sec. 5.4: after correction the register holds v on q0..q2 encoded as
    a|000> + b|111> with ancillas '11': amplitudes at indices 0b00011 and 0b11111."""
    g = G.load("qec.txt")
    _, _, states = oracle.simulate(5, G.ops(g["ops"]), G.init_state(g["init"], 5))
    want = np.zeros(32, dtype=complex)
    want[3] = 1 / np.sqrt(2)
    want[31] = 1j / np.sqrt(2)
    np.testing.assert_allclose(states[0], want, atol=1e-15)


def test_tomography_exact_values():
    """Sec. 5.2: true P_x = (0.5, 0.5), S_2 = 1 for v = (1, i)/sqrt(2) (Y-basis
    measurement reading: S^dagger then H before the Z measurement), and rho_v."""
    g = G.load("tomography.txt")
    v = np.array([1, 1j]) / np.sqrt(2)
    for basis, want0 in (("x", float(g["px0"])), ("y", 0.5 * (1 + float(g["S2"])))):
        res, pr, _ = oracle.simulate(1, [Op("measure_" + basis, (0,))], v)
        d = dict(zip(res, pr))
        assert abs(d.get("0", 0.0) - want0) < 1e-15
    ex = oracle.expect_pauli(v.copy(), ["X", "Y", "Z"])
    np.testing.assert_allclose(ex, [0.0, 1.0, 0.0], atol=1e-15)
    rho = 0.5 * (np.eye(2) + ex[0] * gates.X + ex[1] * gates.Y + ex[2] * gates.Z)
    np.testing.assert_allclose(rho.ravel(), G.cvec(g["rho"]), atol=1e-15)


def test_reset_closed_forms():
    """Reset (Sec. 3.3; read as a Z measurement whose 1-branch is flipped by X):
    |1> -> |0> with certainty; on a Bell pair each branch keeps q1's value with q0 = 0;
    the branch keeps the collapsed state's phase."""
    res, pr, st = oracle.simulate(1, [Op("reset", (0,))], "1")
    assert res == ["1"] and pr == [1.0]
    np.testing.assert_array_equal(st[0], [1, 0])
    res, pr, st = oracle.simulate(2, [Op("h", (0,)), Op("cnot", (0, 1)), Op("reset", (0,))], "00")
    assert res == ["0", "1"]
    np.testing.assert_allclose(pr, [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(st[0], [1, 0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(st[1], [0, 1, 0, 0], atol=1e-15)
    v = np.kron(np.array([1, 1j]) / np.sqrt(2), np.array([0, 1]))  # (|0> + i|1>)/sqrt2 on q0, |1> on q1
    res, pr, st = oracle.simulate(2, [Op("reset", (0,))], v)
    np.testing.assert_allclose(st[0], [0, 1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(st[1], [0, 1j, 0, 0], atol=1e-15)


# ---------------------------------------------------------------------------
# gate matrices against library routines and identities
# ---------------------------------------------------------------------------

def test_rotations_match_matrix_exponential():
    from scipy.linalg import expm
    for t in RNG.uniform(0, 2 * np.pi, 5):
        np.testing.assert_allclose(gates.rx(t), expm(-0.5j * t * gates.X), atol=1e-14)
        np.testing.assert_allclose(gates.ry(t), expm(-0.5j * t * gates.Y), atol=1e-14)
        np.testing.assert_allclose(gates.rz(t), expm(-0.5j * t * gates.Z), atol=1e-14)


def test_u3_identities():
    np.testing.assert_allclose(gates.u3(np.pi / 2, 0, np.pi), gates.H, atol=1e-15)
    for th, ph, la in RNG.uniform(0, 2 * np.pi, (5, 3)):
        U = gates.u3(th, ph, la)
        np.testing.assert_allclose(U @ U.conj().T, np.eye(2), atol=1e-14)
        # OpenQASM: U3(theta, phi, lam) = e^{i(phi+lam)/2} RZ(phi) RY(theta) RZ(lam)
        W_ = np.exp(0.5j * (ph + la)) * gates.rz(ph) @ gates.ry(th) @ gates.rz(la)
        np.testing.assert_allclose(U, W_, atol=1e-14)
        np.testing.assert_allclose(gates.u3(th, 0, 0), gates.ry(th), atol=1e-15)


# ---------------------------------------------------------------------------
# loop form == the literal Kronecker formula of Sec. 3.2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 3, 6])
def test_1q_every_position_vs_kron(n):
    for q in range(n):
        U = rand_u(2, 10 + q)
        psi = W.random_state(n, q)
        want = kron.register_operator(n, U, [q]) @ psi
        oracle.apply_1q(psi, q, U)
        np.testing.assert_allclose(psi, want, atol=1e-14)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_2q_every_ordered_pair_vs_kron(n):
    for qa in range(n):
        for qb in range(n):
            if qa == qb:
                continue
            U = rand_u(4, 100 + 7 * qa + qb)
            psi = W.random_state(n, qa * n + qb)
            want = kron.register_operator(n, U, [qa, qb]) @ psi
            oracle.apply_2q(psi, qa, qb, U)
            np.testing.assert_allclose(psi, want, atol=1e-14)


def test_2q_adjacent_is_plain_kron():
    """For adjacent (q, q+1) the span operator is U itself: I_{2^q} (x) U (x) I."""
    n = 5
    U = rand_u(4, 7)
    for q in range(n - 1):
        full = np.kron(np.kron(np.eye(1 << q), U), np.eye(1 << (n - 2 - q)))
        psi = W.random_state(n, q)
        want = full @ psi
        oracle.apply_2q(psi, q, q + 1, U)
        np.testing.assert_allclose(psi, want, atol=1e-14)
    # and a product of independent single-qubit gates is their Kronecker product
    A, B = rand_u(2, 1), rand_u(2, 2)
    psi = W.random_state(2, 0)
    want = np.kron(A, B) @ psi
    oracle.apply_1q(psi, 0, A)
    oracle.apply_1q(psi, 1, B)
    np.testing.assert_allclose(psi, want, atol=1e-15)


@pytest.mark.parametrize("nctrl", [1, 2, 3])
def test_controlled_all_states_vs_kron(nctrl):
    n = 6
    rng = np.random.default_rng(nctrl)
    for trial in range(8):
        qs = rng.permutation(n)[: nctrl + 1]
        ctrls, tgt = [int(x) for x in qs[:-1]], int(qs[-1])
        states = [int(x) for x in rng.integers(0, 2, nctrl)]
        U = rand_u(2, 300 + trial)
        psi = W.random_state(n, trial)
        want = kron.register_operator(n, kron.controlled_operator(U, nctrl, states), ctrls + [tgt]) @ psi
        oracle.apply_ctrl(psi, ctrls, states, tgt, U)
        np.testing.assert_allclose(psi, want, atol=1e-14)


def test_kq_any_order_vs_kron():
    n = 6
    rng = np.random.default_rng(5)
    for k in (1, 2, 3, 4):
        for trial in range(4):
            qs = [int(x) for x in rng.permutation(n)[:k]]
            U = rand_u(1 << k, 50 + 10 * k + trial)
            psi = W.random_state(n, trial)
            want = kron.register_operator(n, U, qs) @ psi
            oracle.apply_kq(psi, qs, U)
            np.testing.assert_allclose(psi, want, atol=1e-14)


def test_u3_ladder_10q_vs_kron():
    """The 10-qubit U3 + CNOT-ladder workload, loop form against dense kron."""
    n = 10
    ops = W.u3_ladder(n, 20, 1)
    psi = oracle.basis_state(n, 0)
    oracle.run(psi, ops)
    want = kron.apply(oracle.basis_state(n, 0), n, ops)
    np.testing.assert_allclose(psi, want, atol=1e-13)


def test_circuit_unitary_small():
    n = 4
    ops = W.brickwork(n, 6, 9) + W.u3_ladder(n, 2, 3) + W.qft(n)
    M = kron.circuit_unitary(n, ops)
    np.testing.assert_allclose(M @ M.conj().T, np.eye(1 << n), atol=1e-13)
    for col in range(1 << n):
        psi = oracle.basis_state(n, col)
        oracle.run(psi, ops)
        np.testing.assert_allclose(psi, M[:, col], atol=1e-13)


# ---------------------------------------------------------------------------
# closed forms and invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_qft_is_scaled_inverse_fft(n):
    x = W.random_state(n, n)
    y = oracle.run(x.copy(), W.qft(n))
    np.testing.assert_allclose(y, np.sqrt(2.0 ** n) * np.fft.ifft(x), atol=1e-13)


def test_dft_samples_and_gaussian_generator():
    n = 10
    x = oracle.gaussian_state(n, 3)
    np.testing.assert_allclose(x, W.gaussian_state(n, 3), rtol=1e-14, atol=1e-16)
    y = np.sqrt(2.0 ** n) * np.fft.ifft(x)
    ks = [0, 1, 5, 511, 512, 1023]
    np.testing.assert_allclose(oracle.dft_gaussian_samples(n, 3, ks, False), y[ks], atol=1e-14)
    x32 = (x.real.astype(np.float32) + 1j * x.imag.astype(np.float32)).astype(np.complex128)
    y32 = np.sqrt(2.0 ** n) * np.fft.ifft(x32)
    np.testing.assert_allclose(oracle.dft_gaussian_samples(n, 3, ks, True), y32[ks], atol=1e-14)


def test_gaussian_generator_moments():
    g = W.gaussian_amplitudes(7, 0, 1 << 18)
    assert abs(g.real.mean()) < 0.01 and abs(g.imag.mean()) < 0.01
    assert abs(g.real.var() - 1) < 0.01 and abs(g.imag.var() - 1) < 0.01
    assert abs(np.mean(g.real * g.imag)) < 0.01


@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz_closed_forms(n):
    ops = [Op("h", (0,))] + [Op("cnot", (q, q + 1)) for q in range(n - 1)]
    psi = oracle.run(oracle.basis_state(n, 0), ops)
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / np.sqrt(2)
    np.testing.assert_allclose(psi, want, atol=1e-15)
    zz = W.zz_terms(n, ring=False)
    np.testing.assert_allclose(oracle.expect_pauli(psi, zz), np.ones(len(zz)), atol=1e-14)
    np.testing.assert_allclose(oracle.expect_pauli(psi, ["X" * n]), [1.0], atol=1e-14)


def test_pauli_expectation_product_state_closed_form():
    """RY(t_q) on qubit q of |0...0> (Sec. 2 gate definitions, qubit 0 the most
    significant): <Z_q> = cos t_q, <X_q> = sin t_q, <Y_q> = 0, and a string on several
    qubits is the product of its factors.  Distinct angles pin the character-to-qubit
    order and the signs independently of the dense Kronecker reference."""
    n = 6
    rng = np.random.default_rng(12)
    t = rng.uniform(0.2, 2.9, n)
    psi = oracle.run(oracle.basis_state(n, 0), [Op("ry", (q,), (float(t[q]),)) for q in range(n)])
    single = {"Z": np.cos, "X": np.sin, "Y": lambda a: 0.0 * a}
    strings, want = [], []
    for spec in [(("Z", 0),), (("Z", 5),), (("X", 2),), (("Y", 3),), (("Z", 0), ("Z", 1)),
                 (("X", 1), ("Z", 4)), (("Z", 0), ("X", 3), ("Z", 5)), (("X", 0), ("X", 5))]:
        s_ = ["I"] * n
        v = 1.0
        for c, q in spec:
            s_[q] = c
            v *= single[c](t[q])
        strings.append("".join(s_))
        want.append(v)
    np.testing.assert_allclose(oracle.expect_pauli(psi, strings), want, atol=1e-14)


def test_pauli_expectation_vs_dense():
    n = 5
    rng = np.random.default_rng(11)
    psi = W.random_state(n, 2)
    strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(20)]
    got = oracle.expect_pauli(psi, strings)
    want = [np.vdot(psi, kron.pauli_matrix(s) @ psi).real for s in strings]
    np.testing.assert_allclose(got, want, atol=1e-14)


def _masks_of(s: str):
    """(x, z) index-bit masks of a Pauli string (character j is qubit j, index bit
    n-1-j): X sets x, Z sets z, Y sets both."""
    n = len(s)
    x = z = 0
    for j, c in enumerate(s):
        b = 1 << (n - 1 - j)
        if c in "XY":
            x |= b
        if c in "ZY":
            z |= b
    return x, z


def test_pauli_mask_expectation_vs_dense_and_strings():
    """The (xmask, zmask) form of a Pauli term against the dense Kronecker Pauli matrix
    (n = 5, every string kind, coefficients) and against the string form (n = 9)."""
    n = 5
    rng = np.random.default_rng(21)
    psi = W.random_state(n, 3)
    strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(30)] + ["Y" * n, "I" * n, "XYZXY"]
    coeffs = rng.uniform(-2, 2, len(strings))
    terms = [_masks_of(s) + (c,) for s, c in zip(strings, coeffs)]
    got = oracle.expect_masks(psi, terms)
    want = [c * np.vdot(psi, kron.pauli_matrix(s) @ psi).real for s, c in zip(strings, coeffs)]
    np.testing.assert_allclose(got, want, atol=1e-14)
    n = 9
    psi = W.random_state(n, 4)
    strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(20)]
    terms = [_masks_of(s) + (1.0,) for s in strings]
    np.testing.assert_allclose(oracle.expect_masks(psi, terms), oracle.expect_pauli(psi, strings), atol=1e-14)


def test_pauli_mask_expectation_closed_forms():
    """RY product state: <Y_q> = 0, <X_q> = sin t_q, <Z_q> = cos t_q on index bit
    n-1-q; and <Y> = 1 on (|0> + i|1>)/sqrt(2) (Sec. 5.2's tomography vector), which
    fixes the sign of i^{|x & z|}."""
    n = 4
    t = np.array([0.4, 1.1, 2.0, 2.7])
    psi = oracle.run(oracle.basis_state(n, 0), [Op("ry", (q,), (float(t[q]),)) for q in range(n)])
    for q in range(n):
        b = 1 << (n - 1 - q)
        got = oracle.expect_masks(psi, [(b, 0, 1.0), (0, b, 1.0), (b, b, 1.0)])
        np.testing.assert_allclose(got, [np.sin(t[q]), np.cos(t[q]), 0.0], atol=1e-15)
    v = np.array([1.0, 1j]) / np.sqrt(2)
    np.testing.assert_allclose(oracle.expect_masks(v, [(1, 1, 1.0)]), [1.0], atol=1e-15)


def test_norm_and_inverse():
    n = 7
    ops = W.brickwork(n, 8, 4) + W.u3_ladder(n, 2, 4) + W.qft(n) + W.ansatz(n, 2, True)
    params = W.ansatz_params(n, 2, 1)
    x = W.random_state(n, 1)
    y = oracle.run(x.copy(), ops, params)
    assert abs(np.linalg.norm(y) - 1) < 1e-14
    z = oracle.run(y, W.circuit_inverse(ops), params)
    np.testing.assert_allclose(z, x, atol=1e-14)


def test_diagonal_gates_commute():
    n = 5
    a = [Op("cz", (0, 3)), Op("cp", (1, 4), (0.7,)), Op("rz", (2,), (1.3,)), Op("z", (4,))]
    x = W.random_state(n, 4)
    y1 = oracle.run(x.copy(), a)
    y2 = oracle.run(x.copy(), a[::-1])
    np.testing.assert_allclose(y1, y2, atol=1e-15)


# ---------------------------------------------------------------------------
# measurement, probabilities, CDF and sampling (Sec. 3.3; sampling reading)
# ---------------------------------------------------------------------------

def test_outcome_probs_and_collapse():
    n = 6
    psi = W.random_state(n, 8)
    p = np.abs(psi) ** 2
    for q in range(n):
        bit = (np.arange(1 << n) >> (n - 1 - q)) & 1
        P0 = oracle.outcome_prob(psi, q, 0)
        assert abs(P0 - p[bit == 0].sum()) < 1e-15
        for o in (0, 1):
            st = psi.copy()
            P = oracle.outcome_prob(st, q, o)
            oracle.collapse(st, q, o, P)
            assert abs(np.linalg.norm(st) - 1) < 1e-14
            np.testing.assert_array_equal(st[bit != o], 0)
            np.testing.assert_allclose(st[bit == o], psi[bit == o] / np.sqrt(P), atol=1e-15)


def test_probs_definition():
    psi = W.random_state(8, 1)
    p = oracle.probs(psi)
    # two rounded products, one rounded sum (numpy does not fuse)
    np.testing.assert_array_equal(p, psi.real * psi.real + psi.imag * psi.imag)
    assert abs(p.sum() - 1) < 1e-14


def test_cdf_is_correctly_rounded_prefix():
    rng = np.random.default_rng(3)
    p = rng.random(1500) ** 3
    p[::7] = 0.0
    c = oracle.cdf(p)
    want = np.array([math.fsum(p[: k + 1]) for k in range(p.size)])
    np.testing.assert_array_equal(c, want)


def test_sample_matches_linear_scan():
    rng = np.random.default_rng(4)
    p = rng.random(300)
    p[rng.integers(0, 300, 60)] = 0.0
    c = oracle.cdf(p)
    u = np.concatenate([[0.0, 1.0 - 2 ** -53], rng.random(5000), c[:50] / c[-1]])
    got = oracle.sample(c, u)
    T = c[-1]
    want = [next(k for k in range(p.size) if ui * T < c[k]) for ui in u]
    np.testing.assert_array_equal(got, want)
    assert np.all(p[got.astype(np.int64)] > 0)


def test_sampling_frequencies():
    psi = W.random_state(4, 9)
    p = oracle.probs(psi)
    u = W.uniforms(200000, 5)
    idx = oracle.sample(oracle.cdf(p), u)
    freq = np.bincount(idx.astype(np.int64), minlength=16) / u.size
    sigma = np.sqrt(p * (1 - p) / u.size)
    assert np.all(np.abs(freq - p) < 5 * sigma + 1e-12)


# ---------------------------------------------------------------------------
# gradients (reading: d<H>/dt = Im<lambda|G|psi>, checked via parameter shift)
# ---------------------------------------------------------------------------

def test_param_shift_closed_form():
    # <Z> after RY(t)|0> = cos t, d/dt = -sin t; <X> after RZ(s) RY(t)|0> = sin t cos s
    for t in (0.3, 1.9, 4.4):
        g = oracle.param_shift_grad(1, [Op("ry", (0,), param_index=0)], [t], ["Z"], [1.0])
        assert abs(g[0] + np.sin(t)) < 1e-14
    t, s = 0.8, 2.1
    ops = [Op("ry", (0,), param_index=0), Op("rz", (0,), param_index=1)]
    g = oracle.param_shift_grad(1, ops, [t, s], ["X"], [1.0])
    np.testing.assert_allclose(g, [np.cos(t) * np.cos(s), -np.sin(t) * np.sin(s)], atol=1e-14)


def test_param_shift_vs_central_difference():
    """Each parameter enters once with frequency 1, so f = A cos t + B sin t + C and a
    central difference with step h equals f'(t) sin(h)/h exactly."""
    n, L = 4, 2
    ops, params, terms, coeffs = W.adjoint_workload(n, L, 5)
    ps = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    h = 1e-3
    cd = oracle.central_diff_grad(n, ops, params, terms, coeffs, h, range(params.size))
    np.testing.assert_allclose(cd * h / np.sin(h), ps, atol=5e-11)


def test_param_shift_shared_parameter_vs_central_difference():
    """A parameter used by two gates: the per-occurrence shift rule (chain rule) agrees
    with a central difference (frequency <= 2, so FD error ~ h^2 f'''/6)."""
    n = 3
    ops = [Op("h", (0,)), Op("rx", (1,), param_index=0), Op("cnot", (0, 1)), Op("rx", (2,), param_index=0),
           Op("ry", (1,), param_index=1), Op("cz", (1, 2)), Op("rx", (1,), param_index=0)]
    params = np.array([0.7, -1.1])
    terms, coeffs = ["ZZI", "IXY", "YIZ"], [1.0, 0.5, -0.3]
    ps = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    h = 1e-4
    cd = oracle.central_diff_grad(n, ops, params, terms, coeffs, h, range(2))
    np.testing.assert_allclose(ps, cd, atol=1e-7)
