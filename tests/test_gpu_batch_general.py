"""The general batch entry point (qc_run_batch): independent circuits of any gate kinds
and uneven qubit counts in one launch, each with its own Pauli-sum observable, against
the oracle circuit by circuit (final states element by element, values against the
oracle's expectation of the same terms)."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

from gpu_util import TOL, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _strings_terms(n, strings, coeffs):
    out = []
    for s, c in zip(strings, coeffs):
        x = z = 0
        for j, ch in enumerate(s):
            b = 1 << (n - 1 - j)
            x |= b if ch in "XY" else 0
            z |= b if ch in "ZY" else 0
        out.append((x, z, float(c)))
    return out


def mixed_family():
    """QFTs, Haar brickworks, parameterised ansatz circuits (ring), U3 ladders with
    CNOTs, controlled gates with open controls and swaps, on 1 to 16 qubits (both sides
    of the 13-qubit shared-memory limit)."""
    rng = np.random.default_rng(77)
    fam = []
    params = []

    def add(ops, n, p=None):
        off = sum(len(q) for q in params)
        if p is not None:
            params.append(np.asarray(p, dtype=np.float64))
        fam.append((n, ops, off if p is not None else 0, p))

    for n in (3, 9, 12, 14):
        add(W.qft(n), n)
    for i, n in enumerate((2, 6, 11, 13, 16)):
        add(W.brickwork(n, 6, 40 + i), n)
    for i, n in enumerate((6, 10, 15)):
        add(W.ansatz(n, 3, ring=True), n, W.ansatz_params(n, 3, 50 + i))
    add(W.u3_ladder(8, 3, 9), 8)
    ops = []
    n = 10
    U = W.haar_unitaries(3, 4, 12)
    for k in range(30):
        a, b, c = (int(x) for x in rng.permutation(n)[:3])
        ops += [Op("mcx", (a, b, c), ctrl_states=(int(k % 2), 1)), Op("swap", (a, c)),
                Op("u2q", (b, a), matrix=U[k % 3]), Op("cp", (c, b), (0.3 * k,)), Op("t", (a,)),
                Op("ctrl", (c, a), matrix=W.haar_unitaries(1, 2, 100 + k)[0], ctrl_states=(0,))]
    add(ops, n)
    # parameterised U3 and CP with an adjoint op, and a one-qubit circuit
    p = rng.uniform(0, 2 * np.pi, 8)
    add([Op("h", (0,)), Op("u3", (1,), param_index=0), Op("cp", (0, 2), param_index=3),
         Op("rx_dag", (2,), param_index=4), Op("ry", (3,), param_index=5), Op("cnot", (3, 0)),
         Op("rz", (1,), param_index=6)], 4, p)
    add([Op("h", (0,)), Op("rz", (0,), param_index=0), Op("ry", (0,), param_index=1)], 1, rng.uniform(0, 6, 2))
    flat = np.concatenate(params) if params else np.zeros(1)
    return fam, flat


def test_general_batch_mixed_family_against_oracle():
    import torch

    import paper_2503_03016_gb300 as P
    fam, flat = mixed_family()
    rng = np.random.default_rng(5)
    circs, hams, want_vals, want_states, states = [], [], [], [], []
    for n, ops, off, p in fam:
        circs.append(P.Circuit(n, ops))
        strings = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(6)] + (W.zz_terms(n, True) if n > 1 else [])
        coeffs = rng.uniform(-1, 1, len(strings))
        terms = _strings_terms(n, strings, coeffs)
        hams.append(P.Hamiltonian(terms))
        psi = oracle.run(oracle.basis_state(n, 0), ops, None if p is None else p)
        want_states.append(psi)
        want_vals.append(float(np.sum(oracle.expect_masks(psi, terms))))
        states.append(torch.empty(1 << n, dtype=torch.complex64, device="cuda"))
    dparams = torch.tensor(flat, dtype=torch.float64, device="cuda")
    offs = [off for _, _, off, _ in fam]
    out = torch.full((len(fam),), float("nan"), dtype=torch.float64, device="cuda")
    P.qc_run_batch(circs, hams, dparams, offs, states, out)
    torch.cuda.synchronize()
    assert P.qc_last_batch_path() == 0
    got = out.cpu().numpy()
    errs, verrs = [], []
    for i, (n, ops, _, _) in enumerate(fam):
        e = rel_l2(states[i].cpu().numpy(), want_states[i])
        scale = float(np.sum(np.abs([t[2] for t in hams[i].terms])))
        ve = abs(got[i] - want_vals[i]) / scale
        errs.append(e)
        verrs.append(ve)
        assert e <= TOL["c64"], (i, n, e)
        assert ve <= TOL["c64"], (i, n, got[i], want_vals[i])
    record("general_batch_mixed", circuits=len(fam), max_state_rel_l2=max(errs), max_value_err_over_scale=max(verrs))
    # the same batch without state outputs and with one shared observable on same-size
    # circuits gives the same values (tables re-uploaded, workspace path for n > 13)
    out2 = torch.empty(len(fam), dtype=torch.float64, device="cuda")
    P.qc_run_batch(circs, hams, dparams, offs, None, out2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out2.cpu().numpy(), got)


def test_general_batch_ansatz_fast_path():
    """Circuits that are all the layered RY.RZ + CZ-chain ansatz with the ZZ-chain
    observable run on the ansatz kernel (angles rounded to FP32); the same circuits with
    state outputs run on the general kernel; both against the oracle."""
    import torch

    import paper_2503_03016_gb300 as P
    layers = 4
    ns = [6, 9, 12, 14, 17, 13, 8]
    params = [W.ansatz_params(n, layers, 60 + i) for i, n in enumerate(ns)]
    offs = np.cumsum([0] + [p.size for p in params[:-1]])
    flat = np.concatenate(params)
    circs = [P.Circuit(n, W.ansatz(n, layers, ring=False)) for n in ns]
    hams = [P.Hamiltonian.from_strings(W.zz_terms(n, ring=False)) for n in ns]
    dparams = torch.tensor(flat, dtype=torch.float64, device="cuda")
    out = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    P.qc_run_batch(circs, hams, dparams, offs, None, out)
    torch.cuda.synchronize()
    assert P.qc_last_batch_path() == 1
    fast = out.cpu().numpy()
    states = [torch.empty(1 << n, dtype=torch.complex64, device="cuda") for n in ns]
    P.qc_run_batch(circs, hams, dparams, offs, states, out)
    torch.cuda.synchronize()
    assert P.qc_last_batch_path() == 0
    gen = out.cpu().numpy()
    errs = []
    for i, n in enumerate(ns):
        ops = W.ansatz(n, layers, ring=False)
        want = oracle.energy(n, ops, params[i], W.zz_terms(n, False), np.ones(n - 1))
        errs += [abs(fast[i] - want) / (n - 1), abs(gen[i] - want) / (n - 1)]
        assert abs(fast[i] - want) <= 1e-5 * (n - 1), (n, fast[i], want)
        assert abs(gen[i] - want) <= 1e-5 * (n - 1), (n, gen[i], want)
    record("general_batch_ansatz_paths", max_value_err_over_scale=max(errs))


def test_general_batch_errors():
    import torch

    import paper_2503_03016_gb300 as P
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.QCError) as e:
        P.qc_run_batch([P.Circuit(21, [Op("h", (0,))])], [P.Hamiltonian([(0, 1, 1.0)])], None, None, None, out)
    assert e.value.status == 4
    with pytest.raises(P.QCError) as e:  # the angle lies outside dev_params
        dp = torch.zeros(2, dtype=torch.float64, device="cuda")
        P.qc_run_batch([P.Circuit(3, [Op("ry", (0,), param_index=5)])], None, dp, None, None, None)
    assert e.value.status == 1
    with pytest.raises(P.QCError) as e:  # a term on a qubit the circuit does not have
        P.qc_run_batch([P.Circuit(3, [Op("h", (0,))])], [P.Hamiltonian([(0, 1 << 3, 1.0)])], None, None, None, out)
    assert e.value.status == 1
