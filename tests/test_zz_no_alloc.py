"""The allocation-free expectation entry point (qc_expect_pauli_noalloc) against
the regular one (qc_expect_pauli), called through the C ABI.

It exists for callers that cannot allocate device memory once they are running
(device memory wholly reserved by another allocator, or no tolerance for an
allocation failure or allocator synchronisation); its scratch is a fixed array in
the library's device image.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as W

from gpu_util import gpu_state, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
@pytest.mark.parametrize("n", [1, 6, 14])
def test_noalloc_matches_regular_entry_point(dtype, tol, n):
    import paper_2503_03016_gb300 as P
    rng = np.random.default_rng(100 + n)
    psi = W.random_state(n, 21)
    strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(37)]
    strings += W.x_terms(n)
    if n > 1:
        strings += W.zz_terms(n, ring=True)
    coeffs = rng.standard_normal(len(strings))
    st = gpu_state(psi, dtype)
    want = P.qc_expect_pauli(st.handle, strings, coeffs)
    scale = 1 + np.abs(coeffs).max()
    for _ in range(2):  # two calls in a row share (and overwrite) the fixed scratch
        got = P.qc_expect_pauli_noalloc(st.handle, strings, coeffs)
        np.testing.assert_allclose(got, want, atol=tol * scale, rtol=0)
    # a different state and term list right after: no stale contents leak through
    psi2 = W.random_state(n, 22)
    st2 = gpu_state(psi2, dtype)
    s2 = strings[::-1][:20]
    np.testing.assert_allclose(P.qc_expect_pauli_noalloc(st2.handle, s2), P.qc_expect_pauli(st2.handle, s2),
                               atol=tol * 2, rtol=0)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_noalloc_z_strings_against_oracle(dtype, tol):
    """More Z-only strings than one pass of the Z-string kernel takes (32), mixed with
    X/Y strings in the term list, against the oracle."""
    import oracle
    import paper_2503_03016_gb300 as P
    n = 12
    rng = np.random.default_rng(5)
    psi = W.random_state(n, 23)
    strings = ["".join(rng.choice(list("IZ"), n)) for _ in range(45)] + ["I" * n]
    strings += ["".join(rng.choice(list("IXYZ"), n)) for _ in range(10)]
    strings = [strings[i] for i in rng.permutation(len(strings))]
    st = gpu_state(psi, dtype)
    got = P.qc_expect_pauli_noalloc(st.handle, strings)
    np.testing.assert_allclose(got, oracle.expect_pauli(psi, strings), atol=tol, rtol=0)


def test_noalloc_rejects_too_many_terms():
    import paper_2503_03016_gb300 as P
    st = gpu_state(W.random_state(3, 1), "c64")
    with pytest.raises(P.QCError) as e:
        P.qc_expect_pauli_noalloc(st.handle, ["ZZZ"] * 257)
    assert e.value.status == 1 and "256" in str(e.value)


def test_noalloc_grid_caps_at_22_qubits():
    """At 22 qubits (32 MiB, complex64) both grid caps of the fixed array are reached:
    the X/Y reduction's 1216 blocks and the Z-string kernel's 608 blocks of 32 partial
    sums, which fill the partial-sum region up to the term values.  More than 32 Z-only
    strings (two passes of the Z-string kernel) mixed with X/Y strings, twice in a row,
    against the regular entry point."""
    import paper_2503_03016_gb300 as P
    n = 22
    rng = np.random.default_rng(22)
    strings = ["".join(rng.choice(list("IZ"), n)) for _ in range(40)]
    strings += ["".join(rng.choice(list("IXYZ"), n)) for _ in range(24)] + W.x_terms(n)[:6]
    strings = [strings[i] for i in rng.permutation(len(strings))]
    coeffs = rng.standard_normal(len(strings))
    st = P.State(n, "c64").init_gaussian(22)
    want = P.qc_expect_pauli(st.handle, strings, coeffs)
    for _ in range(2):
        got = P.qc_expect_pauli_noalloc(st.handle, strings, coeffs)
        np.testing.assert_allclose(got, want, atol=2e-6 * (1 + np.abs(coeffs).max()), rtol=0)
