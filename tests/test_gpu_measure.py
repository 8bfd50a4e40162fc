"""GPU parity: measurement and collapse, probabilities, sampling and Pauli
expectations against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

import golden_io as G
from gpu_util import TOL, gpu_state, need_gpu, rel_l2

pytestmark = pytest.mark.gpu
DTYPES = ["c128", "c64"]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def gpu_simulate(n, ops, init, dtype):
    """The paper's branch semantics (Sec. 3.3) on the GPU: qc_state_copy +
    qc_collapse for each outcome with nonzero probability."""
    import paper_2503_03016_gb300 as P
    psi = oracle.basis_state(n, init) if isinstance(init, str) else np.asarray(init, dtype=np.complex128)
    branches = [("", 1.0, gpu_state(psi, dtype))]
    for op in ops:
        if op.kind.startswith("measure"):
            q = op.qubits[0]
            new = []
            for res, pr, st in branches:
                for o in (0, 1):
                    s2 = P.State(n, dtype)
                    P.qc_state_copy(s2.handle, st.handle)
                    try:
                        p = P.qc_collapse(s2.handle, q, o)
                    except P.QCError as e:
                        assert e.status == 5  # QC_ERR_ZERO_PROB
                        continue
                    new.append((res + str(o), pr * p, s2))
            branches = new
        else:
            for _, _, st in branches:
                st.run([op])
    return [b[0] for b in branches], [b[1] for b in branches], [b[2].numpy() for b in branches]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["bell.txt", "teleport.txt", "grover.txt", "qec.txt"])
def test_paper_examples_on_gpu(dtype, name):
    g = G.load(name)
    n = int(g["n"])
    res, probs, states = gpu_simulate(n, G.ops(g["ops"]), G.init_state(g["init"], n), dtype)
    wres, wprobs, wstates = oracle.simulate(n, G.ops(g["ops"]), G.init_state(g["init"], n))
    assert res == wres == g["results"].split()
    np.testing.assert_allclose(probs, wprobs, atol=1e-6 if dtype == "c64" else 1e-14)
    for a, b in zip(states, wstates):
        assert rel_l2(a, b) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_measure_and_collapse(dtype):
    import paper_2503_03016_gb300 as P
    n = 9
    psi = W.random_state(n, 3)
    for q in (0, 4, 8):
        for o in (0, 1):
            st = gpu_state(psi, dtype)
            P0 = P.qc_outcome_prob(st.handle, q, 0)
            assert abs(P0 - oracle.outcome_prob(psi, q, 0)) <= (1e-6 if dtype == "c64" else 1e-14)
            pr = P.qc_collapse(st.handle, q, o)
            want = psi.copy()
            Pw = oracle.outcome_prob(want, q, o)
            oracle.collapse(want, q, o, Pw)
            assert abs(pr - Pw) <= (1e-6 if dtype == "c64" else 1e-14)
            assert rel_l2(st.numpy(), want) <= TOL[dtype]
        # measure with a chosen u: outcome 1 iff u*T >= P(0)
        for u in (0.0, 0.3, 0.7, 0.999):
            st = gpu_state(psi, dtype)
            o, pr = P.qc_measure(st.handle, q, u)
            P0 = oracle.outcome_prob(psi, q, 0)
            assert o == (1 if u >= P0 else 0)


def test_collapse_zero_probability_is_rejected():
    import paper_2503_03016_gb300 as P
    st = P.State(3, "c128").init_basis(0)
    with pytest.raises(P.QCError) as e:
        P.qc_collapse(st.handle, 1, 1)
    assert e.value.status == 5
    np.testing.assert_array_equal(st.numpy(), oracle.basis_state(3, 0))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 6, 7, 13])
def test_probs_bit_exact(dtype, n):
    psi = W.random_state(n, n)
    st = gpu_state(psi, dtype)
    p = st.probs().cpu().numpy()
    amps = st.numpy().astype(np.complex128)  # the state's own amplitudes, widened exactly
    np.testing.assert_array_equal(p, oracle.probs(amps))


def test_probs_c64_special_values():
    """FP64 |a|^2 of complex64 amplitudes of every kind: zeros of both signs, subnormal
    and boundary floats, negative and large values, bit for bit against the oracle's
    rounded two-product form (the state is not normalised)."""
    f32 = np.float32
    vals = np.array([0.0, -0.0, 1e-40, -1e-45, 2.0 ** -126, -(2.0 ** -126) * (1 - 2.0 ** -23), 2.0 ** -149,
                     1.0, -1.0, 0.70710677, float(np.nextafter(f32(1), f32(2))), 1e-20, -3e19, 123.456,
                     1.8446743e19, -(2.0 ** -100)], dtype=np.float32)
    rng = np.random.default_rng(3)
    psi = (vals + 1j * vals[rng.permutation(vals.size)]).astype(np.complex64)
    for dt in ("c64", "c128"):
        st = gpu_state(psi, dt)
        p = st.probs().cpu().numpy()
        np.testing.assert_array_equal(p, oracle.probs(psi.astype(np.complex128)))


@pytest.mark.parametrize("n", [1, 2, 5, 6, 7, 12, 17])
def test_sampler_bit_exact_on_oracle_probabilities(n):
    """The GPU sampler fed the oracle's p gives the oracle's indices exactly."""
    import torch

    import paper_2503_03016_gb300 as P
    rng = np.random.default_rng(n)
    p = rng.random(1 << n) ** 4
    p[rng.integers(0, 1 << n, max(1, (1 << n) // 5))] = 0.0
    p /= p.sum()
    u = np.concatenate([[0.0, 1 - 2 ** -53], W.uniforms(20000, n)])
    want = oracle.sample(oracle.cdf(p), u)
    st = P.State(max(n, 1), "c64").init_basis(0)
    dp = torch.tensor(p, device="cuda")
    du = torch.tensor(u, device="cuda")
    out = torch.empty(u.size, dtype=torch.int64, device="cuda")
    P.qc_sample_probs(st.handle, dp, n, du, u.size, out)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("shots", [1, 3, 7, 1001])
def test_sampler_odd_shot_counts(shots):
    """A warp draws two shots; an odd count leaves the last warp's second half idle
    (it must write nothing).  The entries past `shots` keep their sentinel."""
    import torch

    import paper_2503_03016_gb300 as P
    n = 12
    rng = np.random.default_rng(shots)
    p = rng.random(1 << n) ** 2
    p /= p.sum()
    u = W.uniforms(shots, 40 + shots)
    want = oracle.sample(oracle.cdf(p), u)
    st = P.State(n, "c64").init_basis(0)
    out = torch.full((shots + 1,), -7, dtype=torch.int64, device="cuda")
    P.qc_sample_probs(st.handle, torch.tensor(p, device="cuda"), n, torch.tensor(u, device="cuda"), shots, out)
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[:shots].astype(np.uint64), want)
    assert got[shots] == -7


@pytest.mark.parametrize("n", [4, 10, 16])
def test_sample_state_c128_bit_exact(n):
    import torch
    psi = W.gaussian_state(n, 9)
    st = gpu_state(psi, "c128")
    u = W.uniforms(50000, 11)
    idx = st.sample(torch.tensor(u, device="cuda")).cpu().numpy().astype(np.uint64)
    want = oracle.sample(oracle.cdf(oracle.probs(st.numpy())), u)
    np.testing.assert_array_equal(idx, want)


def test_sample_c64_statistics():
    import torch
    n = 8
    psi = W.random_state(n, 4)
    st = gpu_state(psi, "c64")
    u = W.uniforms(400000, 12)
    idx = st.sample(torch.tensor(u, device="cuda")).cpu().numpy()
    p = oracle.probs(psi)
    freq = np.bincount(idx, minlength=1 << n) / u.size
    sigma = np.sqrt(p * (1 - p) / u.size)
    assert np.all(np.abs(freq - p) < 5 * sigma + 1e-6)
    # same p -> same indices as the oracle fed the state's own probabilities
    want = oracle.sample(oracle.cdf(oracle.probs(st.numpy().astype(np.complex128))), u)
    np.testing.assert_array_equal(idx.astype(np.uint64), want)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 8, 12])
def test_pauli_expectations(dtype, n):
    rng = np.random.default_rng(n)
    psi = W.random_state(n, 6)
    strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(40)]
    strings += W.zz_terms(n, ring=True) if n > 1 else []
    strings += W.x_terms(n)
    coeffs = rng.standard_normal(len(strings))
    st = gpu_state(psi, dtype)
    got = st.expect(strings, coeffs)
    want = oracle.expect_pauli(psi, strings, coeffs)
    tol = 1e-12 if dtype == "c128" else 2e-6
    np.testing.assert_allclose(got, want, atol=tol * (1 + np.abs(coeffs).max()))


@pytest.mark.parametrize("dtype", DTYPES)
def test_z_strings_24_qubits(dtype):
    """24 qubits (the Z-string kernel then gives each thread several chunks of 32
    amplitudes): strings on the highest index bits (qubits 0 and 1), on the chunk's own
    bits (< 5) and in between, plus the full ZZ ring, against the oracle."""
    n = 24
    psi = W.gaussian_state(n, 17)
    strings = W.zz_terms(n, ring=True)
    for qs in ((0,), (1,), (0, 1), (0, 23), (1, 20, 23), (2, 19), (0, 1, 2, 3, 21, 22, 23)):
        s = ["I"] * n
        for q in qs:
            s[q] = "Z"
        strings.append("".join(s))
    st = gpu_state(psi, dtype)
    got = st.expect(strings)
    want = oracle.expect_pauli(st.numpy().astype(np.complex128), strings)  # the stored amplitudes
    tol = 1e-12 if dtype == "c128" else 2e-6
    np.testing.assert_allclose(got, want, atol=tol)


def test_tomography_values_on_gpu():
    """Sec. 5.2: <X> = 0, <Y> = 1, <Z> = 0 for v = (1, i)/sqrt(2)."""
    st = gpu_state(np.array([1, 1j]) / np.sqrt(2), "c128")
    np.testing.assert_allclose(st.expect(["X", "Y", "Z"]), [0, 1, 0], atol=1e-15)
