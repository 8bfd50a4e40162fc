"""GPU adjoint gradients against the oracle's exact parameter-shift gradient and
against central differences (reading: each parameter enters once with frequency 1,
so a central difference with step h equals f'(t) sin(h)/h exactly)."""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def gpu_energy(n, ops, params, terms, coeffs, dtype):
    import paper_2503_03016_gb300 as P
    st = P.State(n, dtype).init_basis(0)
    st.run(ops, params, mode=P.QC_RUN_FUSED)
    return float(np.sum(st.expect(terms, coeffs)))


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-5)])
@pytest.mark.parametrize("n,layers", [(4, 2), (10, 3)])
def test_adjoint_vs_parameter_shift(dtype, tol, n, layers):
    import paper_2503_03016_gb300 as P
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 5)
    circ = P.Circuit(n, ops)
    e, g = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128 if dtype == "c128" else P.QC_C64)
    e_ref = oracle.energy(n, ops, params, terms, coeffs)
    g_ref = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    scale = np.abs(g_ref).max() + 1
    assert abs(e - e_ref) <= tol * scale
    np.testing.assert_allclose(g, g_ref, atol=tol * scale, rtol=0)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-5)])
def test_adjoint_mixed_generators_and_shared_parameters(dtype, tol):
    """RX/RY/RZ rotations, a parameter used by two gates, non-rotation gates between
    them and a Hamiltonian with X, Y and Z strings (several X masks, one H psi launch)."""
    import paper_2503_03016_gb300 as P
    from workloads import Op
    n = 5
    ops = [Op("h", (0,)), Op("rx", (1,), param_index=0), Op("cnot", (1, 2)), Op("ry", (2,), param_index=1),
           Op("rz", (3,), param_index=2), Op("cz", (0, 3)), Op("rx", (4,), param_index=0), Op("swap", (1, 4)),
           Op("ry", (0,), param_index=3), Op("cp", (2, 3), (0.4,)), Op("rz", (2,), param_index=1)]
    params = np.array([0.3, 1.2, -0.7, 2.2])
    terms = ["XYZII", "ZZIII", "IIYIX", "YIIIZ", "IXXXI"]
    coeffs = np.array([0.5, -1.0, 0.7, 0.2, 1.3])
    circ = P.Circuit(n, ops)
    e, g = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128 if dtype == "c128" else P.QC_C64)
    assert abs(e - oracle.energy(n, ops, params, terms, coeffs)) < tol
    np.testing.assert_allclose(g, oracle.param_shift_grad(n, ops, params, terms, coeffs), atol=tol)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-5)])
def test_fused_sweep_vs_parameter_shift(dtype, tol):
    """Registers of 12 qubits and more take the fused reverse sweep (tile passes over
    psi and lambda together): 13 qubits, 2 layers, ring ZZ + sum X."""
    import paper_2503_03016_gb300 as P
    n, layers = 13, 2
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 6)
    circ = P.Circuit(n, ops)
    e, g = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128 if dtype == "c128" else P.QC_C64)
    e_ref = oracle.energy(n, ops, params, terms, coeffs)
    g_ref = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    scale = np.abs(g_ref).max() + 1
    assert abs(e - e_ref) <= tol * scale
    np.testing.assert_allclose(g, g_ref, atol=tol * scale, rtol=0)
    # fixed-order sums: a second call gives the same bits
    e2, g2 = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128 if dtype == "c128" else P.QC_C64)
    assert e2 == e
    np.testing.assert_array_equal(g2, g)


def test_fused_sweep_mixed_gates():
    """The fused sweep with RX/RY/RZ on every kind of bit position (low bits, tile bits,
    bits left to the tile number), shared parameters, dense two-qubit gates, controlled
    and diagonal gates between the rotations, and X/Y/Z Hamiltonian strings."""
    import paper_2503_03016_gb300 as P
    from workloads import Op
    n = 14
    rng = np.random.default_rng(8)
    U = W.haar_unitaries(2, 4, 9)
    ops = []
    k = 0
    for layer in range(2):
        for q in range(n):
            kind = ("rx", "ry", "rz")[(q + layer) % 3]
            ops.append(Op(kind, (q,), param_index=k % 20))  # parameters shared between gates
            k += 1
        ops += [Op("cnot", (0, 13)), Op("u2q", (3, 11), matrix=U[layer]), Op("cp", (5, 12), (0.7,)),
                Op("swap", (2, 9)), Op("h", (7,)), Op("mcx", (1, 6, 10), ctrl_states=(1, 0)), Op("cz", (4, 8))]
    params = rng.uniform(0, 2 * np.pi, 20)
    terms = ["X" + "I" * 12 + "Z", "I" * 5 + "YY" + "I" * 7, "Z" * n, "I" * 12 + "XY", "IZIXIIIIIIYIII"]
    coeffs = np.array([0.8, -0.4, 0.3, 1.1, -0.6])
    circ = P.Circuit(n, ops)
    e, g = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128)
    assert abs(e - oracle.energy(n, ops, params, terms, coeffs)) < 1e-11
    np.testing.assert_allclose(g, oracle.param_shift_grad(n, ops, params, terms, coeffs), atol=1e-11)


def test_autograd_function():
    import torch

    import paper_2503_03016_gb300 as P
    n, layers = 6, 2
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 7)
    circ = P.Circuit(n, ops)
    theta = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    e = P.AdjointExpectation.apply(theta, circ, terms, coeffs, P.QC_C128)
    (3.0 * e).backward()
    g_ref = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * g_ref, atol=1e-11)


@pytest.mark.slow
def test_adjoint_24q_central_differences():
    """Full size: 24 qubits, 10 layers, 480 parameters, H = ring ZZ + sum X.  The
    complex128 adjoint gradient against central differences of the GPU complex128
    energy (step 1e-3, corrected by h/sin h) on 12 seeded parameters; complex64
    against complex128."""
    import paper_2503_03016_gb300 as P
    n, layers = 24, 10
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 5)
    circ = P.Circuit(n, ops)
    e128, g128 = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C128)
    e64, g64 = P.qc_adjoint_grad(circ, params, terms, coeffs, P.QC_C64)
    assert g128.size == 480
    assert abs(e128 - gpu_energy(n, ops, params, terms, coeffs, "c128")) < 1e-10
    h = 1e-3
    idx = np.random.default_rng(5).choice(480, 12, replace=False)
    for p in idx:
        a = params.copy()
        a[p] += h
        b = params.copy()
        b[p] -= h
        fd = (gpu_energy(n, ops, a, terms, coeffs, "c128") - gpu_energy(n, ops, b, terms, coeffs, "c128")) / (2 * h)
        assert abs(fd * h / np.sin(h) - g128[p]) < 1e-8, (p, fd, g128[p])
    assert abs(e64 - e128) < 1e-4 * (1 + abs(e128))
    assert np.abs(g64 - g128).max() < 1e-4 * (1 + np.abs(g128).max())


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-5)])
def test_adjoint_device_form_matches_host_form(dtype, tol):
    """qc_adjoint_grad_dev (device angles, mask-form H, device outputs on the stream)
    gives the host form's values bit for bit, and both match the oracle's parameter
    shift; two calls in a row on another stream leave the same outputs."""
    import torch

    import paper_2503_03016_gb300 as P
    n, layers = 13, 2
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 11)
    circ = P.Circuit(n, ops)
    code = P.QC_C128 if dtype == "c128" else P.QC_C64
    e_host, g_host = P.qc_adjoint_grad(circ, params, terms, coeffs, code)
    ham = P.Hamiltonian.from_strings(terms, coeffs)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(params.size, dtype=torch.float64, device="cuda")
    P.qc_adjoint_grad_dev(circ, dp, ham, code, e, g)
    torch.cuda.synchronize()
    assert e.item() == e_host
    np.testing.assert_array_equal(g.cpu().numpy(), g_host)
    side = torch.cuda.Stream()
    e2 = torch.empty_like(e)
    g2 = torch.empty_like(g)
    with torch.cuda.stream(side):
        P.qc_adjoint_grad_dev(circ, dp, ham, code, e2, g2)
        P.qc_adjoint_grad_dev(circ, dp, ham, code, e2, g2)
    side.synchronize()
    assert e2.item() == e_host
    np.testing.assert_array_equal(g2.cpu().numpy(), g_host)
    g_ref = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    scale = np.abs(g_ref).max() + 1
    np.testing.assert_allclose(g_host, g_ref, atol=tol * scale, rtol=0)


def test_autograd_function_on_device():
    """The autograd function with CUDA parameters: the gradient stays on the device."""
    import torch

    import paper_2503_03016_gb300 as P
    n, layers = 6, 2
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 8)
    circ = P.Circuit(n, ops)
    theta = torch.tensor(params, dtype=torch.float64, device="cuda", requires_grad=True)
    e = P.AdjointExpectation.apply(theta, circ, terms, coeffs, P.QC_C128)
    assert e.device.type == "cuda"
    (2.0 * e).backward()
    assert theta.grad.device.type == "cuda"
    g_ref = oracle.param_shift_grad(n, ops, params, terms, coeffs)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), 2.0 * g_ref, atol=1e-11)
    assert abs(e.item() - oracle.energy(n, ops, params, terms, coeffs)) < 1e-12
