"""The paper's simulate / reducedStatevector / counts on the GPU (measurement
branching, subsystem gathers, marginal distributions) against the oracle and the
printed worked examples."""
import numpy as np
import pytest

import oracle
import workloads as W

import golden_io as G
from gpu_util import TOL, gpu_state, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("name", ["bell.txt", "teleport.txt", "grover.txt", "qec.txt"])
def test_simulate_paper_examples(dtype, name):
    import paper_2503_03016_gb300 as P
    g = G.load(name)
    n = int(g["n"])
    res, probs, states = P.simulate(n, G.ops(g["ops"]), G.init_state(g["init"], n), dtype=dtype)
    assert res == g["results"].split()
    np.testing.assert_allclose(probs, G.fvec(g["probabilities"]), atol=float(g["print_tol"]))
    wres, wprobs, wstates = oracle.simulate(n, G.ops(g["ops"]), G.init_state(g["init"], n))
    for st, w in zip(states, wstates):
        assert rel_l2(st.numpy(), w) <= TOL[dtype]
    for key, val in g.items():
        if key.startswith("reduced."):
            bits = key.split(".")[1]
            red = P.reduced_statevector(states[res.index(bits)], [0, 1], bits).cpu().numpy()
            np.testing.assert_allclose(red, G.cvec(val), atol=float(g["print_tol"]))


def test_simulate_x_and_y_basis():
    """Sec. 5.2: v = (1, i)/sqrt(2) measured in X gives 0.5/0.5, in Y outcome 0 with
    probability 1."""
    import paper_2503_03016_gb300 as P
    from workloads import Op
    v = np.array([1, 1j]) / np.sqrt(2)
    res, pr, _ = P.simulate(1, [Op("measure_x", (0,))], v)
    assert res == ["0", "1"]
    np.testing.assert_allclose(pr, [0.5, 0.5], atol=1e-15)
    res, pr, st = P.simulate(1, [Op("measure_y", (0,))], v)
    assert res == ["0"] and abs(pr[0] - 1) < 1e-15
    np.testing.assert_allclose(st[0].numpy(), v, atol=1e-15)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_simulate_mid_circuit_reset(dtype):
    """Reset (Z measurement, then X on the 1-branch) in the middle of a circuit, with
    gates after it, against the oracle branch by branch."""
    import paper_2503_03016_gb300 as P
    from workloads import Op
    n = 4
    v = W.random_state(n, seed=21)
    ops = [Op("h", (0,)), Op("cnot", (0, 2)), Op("reset", (2,)), Op("ry", (2,), (0.7,)),
           Op("cz", (2, 3)), Op("reset", (0,)), Op("measure_x", (3,))]
    res, pr, st = P.simulate(n, ops, v, dtype=dtype)
    wres, wpr, wst = oracle.simulate(n, ops, v)
    assert res == wres
    np.testing.assert_allclose(pr, wpr, rtol=TOL[dtype])
    for a, b in zip(st, wst):
        assert rel_l2(a.numpy(), b) <= TOL[dtype]


@pytest.mark.parametrize("name", ["teleport.txt", "qec.txt"])
def test_qasm_front_end_paper_examples(name):
    """The teleportation and error-correction circuits written out as OpenQASM
    (Sec. 4), read back and simulated on the GPU, against the oracle on the original
    ops (open controls become X around ccx in the text)."""
    import paper_2503_03016_gb300 as P
    g = G.load(name)
    n = int(g["n"])
    ops = G.ops(g["ops"])
    n2, back = P.from_qasm(P.to_qasm(n, ops, header=True))
    assert n2 == n
    res, pr, st = P.simulate(n, back, G.init_state(g["init"], n), dtype="c128")
    wres, wpr, wst = oracle.simulate(n, ops, G.init_state(g["init"], n))
    assert res == wres == g["results"].split()
    np.testing.assert_allclose(pr, wpr, atol=1e-14)
    for a, b in zip(st, wst):
        assert rel_l2(a.numpy(), b) <= TOL["c128"]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_reduced_state_gather(dtype):
    import torch

    import paper_2503_03016_gb300 as P
    n = 9
    psi = W.random_state(n, 3)
    st = gpu_state(psi, dtype)
    rng = np.random.default_rng(2)
    for m in (1, 3, 5, 8):
        known = [int(x) for x in rng.permutation(n)[:m]]
        bits = "".join(str(int(b)) for b in rng.integers(0, 2, m))
        got = P.reduced_statevector(st, known, bits).cpu().numpy()
        want = oracle.reduced_statevector(st.numpy().astype(np.complex128), known, bits)
        np.testing.assert_array_equal(got.astype(np.complex128), want)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_marginal_probs_and_counts(dtype):
    import torch

    import paper_2503_03016_gb300 as P
    n = 11
    psi = W.random_state(n, 5)
    st = gpu_state(psi, dtype)
    p = oracle.probs(st.numpy().astype(np.complex128)).reshape([2] * n)
    for qubits in ([3], [0, 10], [7, 2, 5], list(range(n))):
        marg = torch.empty(1 << len(qubits), dtype=torch.float64, device="cuda")
        P.qc_marginal_probs(st.handle, qubits, marg)
        others = tuple(q for q in range(n) if q not in qubits)
        want = np.transpose(p.sum(axis=others) if others else p,
                            np.argsort(np.argsort(qubits))).reshape(-1)
        np.testing.assert_allclose(marg.cpu().numpy(), want, atol=1e-15, rtol=1e-12)
    u = torch.tensor(W.uniforms(200000, 8), device="cuda")
    qubits = [4, 1, 9]
    cnt = P.counts(st, qubits, u)
    marg = torch.empty(8, dtype=torch.float64, device="cuda")
    P.qc_marginal_probs(st.handle, qubits, marg)
    pm = marg.cpu().numpy()
    # the sampler is exact given the marginal it was fed
    idx = oracle.sample(oracle.cdf(pm), u.cpu().numpy())
    np.testing.assert_array_equal(cnt, np.bincount(idx.astype(np.int64), minlength=8))
    sigma = np.sqrt(pm * (1 - pm) / u.numel())
    assert np.all(np.abs(cnt / u.numel() - pm) < 5 * sigma + 1e-9)
