"""Full-size checks in the benchmark's launch configuration (QC_RUN_FUSED):

* 32-qubit quantum Fourier transform (32 GiB complex64 / 64 GiB complex128): sampled
  outputs against the closed form y_k = N^{-1/2} sum_j x_j exp(2 pi i jk/N), computed
  one by one by the oracle (Gaussian start state) or in closed form (sparse start).
* 28-qubit brickwork output: probabilities and 1e6 inverse-CDF shots bit-exact
  against the oracle fed the same (widened) amplitudes.
"""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import need_gpu, record

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _free_gb():
    import torch
    free, _ = torch.cuda.mem_get_info()
    return free / 2 ** 30


@pytest.mark.parametrize("prec", ["native", "tf32x3"])
def test_qft32_c64_gaussian_sampled_outputs(prec):
    """The fused QFT-32 on the CUDA-core passes and on the tensor-core passes (deferred
    phase factors, relabeled SWAPs), sampled outputs against the DFT."""
    import torch

    import paper_2503_03016_gb300 as P
    n = 32
    if _free_gb() < 40:
        pytest.skip("needs ~34 GiB of device memory")
    st = P.State(n, "c64").init_gaussian(3)
    st.run(W.qft(n), mode=P.QC_RUN_FUSED, prec=P.QC_PREC_TF32X3 if prec == "tf32x3" else P.QC_PREC_NATIVE)
    assert P.qc_last_fused_path() == (2 if prec == "tf32x3" else 1)
    ks = [0, 0x9E3779B9, (1 << 32) - 1]
    got = np.array([complex(st.tensor[k].item()) for k in ks])
    want = oracle.dft_gaussian_samples(n, 3, ks, round_c64=True)
    # the complex64 target is 1e-5 relative L2, i.e. an RMS error of 1e-5 * 2^-16 per
    # output (outputs have RMS magnitude 2^-16); allow 3 sigma on a sampled output
    record("qft32_c64_gaussian_sampled", prec=prec, max_err_over_rms=float(np.abs(got - want).max() / 2.0 ** -16))
    assert np.abs(got - want).max() <= 3e-5 * 2.0 ** -16, (got, want)
    nrm = torch.linalg.vector_norm(st.tensor.to(torch.complex128)).item()
    assert abs(nrm - 1) < 1e-5
    st.free()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c64", "c128", "c64_tf32x3"])
def test_qft32_sparse_closed_form(dtype):
    import torch

    import paper_2503_03016_gb300 as P
    n = 32
    prec = P.QC_PREC_TF32X3 if dtype == "c64_tf32x3" else P.QC_PREC_NATIVE
    dtype = dtype[:3] if dtype == "c64_tf32x3" else dtype
    need = 34 if dtype == "c64" else 66
    if _free_gb() < need + 4:
        pytest.skip("needs %d GiB of device memory" % need)
    rng = np.random.default_rng(32)
    xs = [int(v) for v in rng.integers(0, 1 << n, 8)]
    cs = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    cs /= np.linalg.norm(cs)
    st = P.State(n, dtype)
    st.tensor.zero_()
    for x, c in zip(xs, cs):
        st.tensor[x] = complex(c)
    torch.cuda.synchronize()
    st.run(W.qft(n), mode=P.QC_RUN_FUSED, prec=prec)
    ks = [int(v) for v in rng.integers(0, 1 << n, 64)] + [0, 1, (1 << n) - 1]
    got = np.array([complex(st.tensor[k].item()) for k in ks])
    N = float(1 << n)
    want = np.array([sum(c * np.exp(2j * np.pi * (((x * k) % (1 << n)) / N)) for x, c in zip(xs, cs)) / np.sqrt(N)
                     for k in ks])
    # relative L2 targets (1e-12 / 1e-5) as an RMS error per output of RMS size 2^-16,
    # 3 sigma for a sampled output
    tol = 3 * (1e-12 if dtype == "c128" else 1e-5) * 2.0 ** -16
    record("qft32_fused_sparse", dtype=dtype, prec=int(prec), max_err_over_rms=float(np.abs(got - want).max() / 2.0 ** -16))
    assert np.abs(got - want).max() <= tol, np.abs(got - want).max()
    st.free()
    torch.cuda.empty_cache()


def test_brickwork28_probs_and_shots_bit_exact():
    import torch

    import paper_2503_03016_gb300 as P
    n = 28
    st = P.State(n, "c64").init_basis(0)
    st.run(W.brickwork(n, 40, 2), mode=P.QC_RUN_FUSED)
    p = st.probs().cpu().numpy()
    u = W.uniforms(1_000_000, 102)
    idx = st.sample(torch.tensor(u, device="cuda")).cpu().numpy().astype(np.uint64)
    amps = st.numpy().astype(np.complex128)  # exact widening of the complex64 amplitudes
    p_ref = oracle.probs(amps)
    np.testing.assert_array_equal(p, p_ref)
    np.testing.assert_array_equal(idx, oracle.sample(oracle.cdf(p_ref), u))
    st.free()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_z_strings_28_qubit_product_state(dtype):
    """<Z_S> on RY(t_0) x ... x RY(t_27)|0...0> is prod_{q in S} cos t_q (each factor
    is cos^2(t/2) - sin^2(t/2)).  28 qubits put strings on every part of the Z-string
    kernel's index split: the five transformed top bits (qubits 0..4), the Gray-code
    bits of the chunk number (qubits 5..7) and the per-thread low bits; the identity
    string checks that every chunk is counted once."""
    import paper_2503_03016_gb300 as P
    n = 28
    if _free_gb() < (2 if dtype == "c64" else 4) * 1.5:
        pytest.skip("not enough device memory")
    rng = np.random.default_rng(28)
    t = rng.uniform(0.2, 1.2, n)
    st = P.State(n, dtype).init_basis(0)
    for q in range(n):
        c, s = np.cos(t[q] / 2), np.sin(t[q] / 2)
        st.apply_1q(q, np.array([[c, -s], [s, c]]))
    sets = [(q, q + 1) for q in range(n - 1)]
    sets += [(), (0,), (4,), (5,), (6,), (7,), (0, 4), (3, 5), (5, 6, 7), (4, 8), (7, 27),
             (0, 1, 2, 3, 4), (2, 6, 13, 21, 27), (1, 5, 7, 20, 26)]
    strings = []
    for S in sets:
        s = ["I"] * n
        for q in S:
            s[q] = "Z"
        strings.append("".join(s))
    got = st.expect(strings)
    want = np.array([np.prod(np.cos(t[list(S)])) for S in sets])
    tol = 1e-12 if dtype == "c128" else 1e-5
    np.testing.assert_allclose(got, want, atol=tol)
    st.free()


def test_z_strings_26_qubit_gaussian_state():
    """A general 26-qubit state (the chunk number then has one Gray-code bit, index bit
    20 = qubit 5): Z strings across the kernel's index split against the oracle on the
    stored (widened) amplitudes."""
    import paper_2503_03016_gb300 as P
    n = 26
    st = P.State(n, "c64").init_gaussian(26)
    sets = [(5,), (0, 5, 25), (4, 5, 6), (1, 2, 3, 4, 5, 20), (0, 1)]
    strings = []
    for S in sets:
        s = ["I"] * n
        for q in S:
            s[q] = "Z"
        strings.append("".join(s))
    got = st.expect(strings)
    want = oracle.expect_pauli(st.numpy().astype(np.complex128), strings)
    np.testing.assert_allclose(got, want, atol=2e-6)
    st.free()
