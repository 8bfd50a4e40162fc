"""The sharded state vector (top index bits over processes) on CPU ranks: 2 and 4
gloo processes, each shard held by an oracle-backed engine written here (the product
engine keeps its shard on a GPU); the placement logic, the pairwise half-shard
exchanges, the rank-resolved controls and diagonal gates, and the cross-process sums
are the product's own code.  Checked against the oracle on the full vector."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

pytestmark = pytest.mark.timeout(300) if hasattr(pytest.mark, "timeout") else []


class OracleShard:
    """A shard held on the host, every gate and readout by the oracle."""

    def __init__(self, nl):
        self.nl = nl
        self.dtype = "c128"
        self.psi = np.zeros(1 << nl, dtype=np.complex128)

    def amplitudes(self):
        import torch
        return torch.from_numpy(self.psi)

    def init_basis(self, index):
        self.psi[:] = 0
        if index is not None:
            self.psi[index] = 1.0

    def load(self, amps):
        self.psi[:] = amps

    def run(self, ops, params=None):
        oracle.run(self.psi, ops, params)

    def probs(self):
        return oracle.probs(self.psi)

    def expect(self, strings, coeffs):
        return oracle.expect_pauli(self.psi, strings, coeffs)

    def outcome_prob(self, q, outcome):
        return oracle.outcome_prob(self.psi, q, outcome)

    def scratch_amplitudes(self):
        import torch
        if not hasattr(self, "scr"):
            self.scr = np.zeros(1 << self.nl, dtype=np.complex128)
        return torch.from_numpy(self.scr)

    def scratch_run(self, ops):
        oracle.run(self.scr, ops)

    def inner_scratch(self):
        return oracle.inner(self.psi, self.scr)

    def collapse_norm(self, q, outcome, p):
        if q < 0:
            self.psi[:] = self.psi / np.sqrt(p) if p > 0 else 0.0
        else:
            oracle.collapse(self.psi, q, outcome, p)


def circuit(n, seed):
    """Every gate kind on every qubit, global ones included."""
    rng = np.random.default_rng(seed)
    ops = []
    U = W.haar_unitaries(4, 4, seed)
    k1 = ["h", "x", "y", "z", "s", "sdg", "t", "tdg", "t_dag", "s_dag"]
    for i in range(70):
        c = i % 12
        qs = [int(x) for x in rng.permutation(n)[:3]]
        if c == 0:
            ops.append(Op(k1[rng.integers(0, len(k1))], (qs[0],)))
        elif c == 1:
            ops.append(Op(["rx", "ry", "rz"][i % 3], (qs[0],), (float(rng.uniform(0, 6)),)))
        elif c == 2:
            ops.append(Op("u3", (qs[0],), tuple(float(a) for a in rng.uniform(0, 6, 3))))
        elif c == 3:
            ops.append(Op("cnot", (qs[0], qs[1])))
        elif c == 4:
            ops.append(Op("cz", (qs[0], qs[1])))
        elif c == 5:
            ops.append(Op("cp", (qs[0], qs[1]), (float(rng.uniform(0, 6)),)))
        elif c == 6:
            ops.append(Op("swap", (qs[0], qs[1])))
        elif c == 7:
            ops.append(Op("u2q", (qs[0], qs[1]), matrix=U[i % 4]))
        elif c == 8:
            ops.append(Op("mcx", tuple(qs), ctrl_states=(int(rng.integers(0, 2)), int(rng.integers(0, 2)))))
        elif c == 9:
            ops.append(Op("ctrl", (qs[0], qs[1]), matrix=W.haar_unitaries(1, 2, 900 + i)[0], ctrl_states=(0,)))
        elif c == 10:
            ops.append(Op("ry", (qs[0],), param_index=i % 5))
        else:
            ops.append(Op("cp_dag", (qs[0], qs[1]), param_index=(i + 1) % 5))
    return ops


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, outdir):
    import torch.distributed as dist

    from paper_2503_03016_gb300.sharded import ShardedState
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    g = world.bit_length() - 1
    res = {}
    params = np.random.default_rng(3).uniform(0, 6, 5)
    ops = circuit(n, 10 + world)
    st = ShardedState(n, OracleShard(n - g))
    st.init_basis(0b101 % (1 << n))
    st.run(ops, params)
    res["mixed"] = st.gather()
    res["exchanges"] = np.array([st.exchanges])
    # QFT of a random state, then the readouts
    x = W.random_state(n, 7)
    st.init_vector(x)
    st.run(W.qft(n))
    st.run(W.brickwork(n, 4, 3))
    strings = ["X" * n, "Y" + "I" * (n - 2) + "Z", "ZZ" + "I" * (n - 2), "I" * (n - 1) + "X", "XYZ" + "I" * (n - 3)]
    res["expect"] = st.expect(strings, np.arange(1, len(strings) + 1, dtype=float))
    res["p_q0"] = np.array([st.outcome_prob(0, 0), st.outcome_prob(0, 1), st.outcome_prob(n - 1, 1)])
    res["state2"] = st.gather()
    res["probs"] = np.asarray(st.probs())
    res["collapse_p"] = np.array([st.collapse(0, 1), st.collapse(n - 2, 0)])
    res["state3"] = st.gather()
    np.savez(os.path.join(outdir, "r%d.npz" % rank), **res)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_state_against_oracle(world):
    import torch.multiprocessing as mp
    n = 6
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), n, d), nprocs=world, start_method="spawn")
        rs = [np.load(os.path.join(d, "r%d.npz" % r)) for r in range(world)]
        params = np.random.default_rng(3).uniform(0, 6, 5)
        want = oracle.run(oracle.basis_state(n, 0b101 % (1 << n)), circuit(n, 10 + world), params)
        for r in rs:
            np.testing.assert_allclose(r["mixed"], want, atol=1e-12)
        assert rs[0]["exchanges"][0] > 0  # the gates on global qubits moved data
        psi = oracle.run(W.random_state(n, 7), W.qft(n) + W.brickwork(n, 4, 3))
        strings = ["X" * n, "Y" + "I" * (n - 2) + "Z", "ZZ" + "I" * (n - 2), "I" * (n - 1) + "X",
                   "XYZ" + "I" * (n - 3)]
        ev = oracle.expect_pauli(psi, strings, np.arange(1, len(strings) + 1, dtype=float))
        p_want = [oracle.outcome_prob(psi, 0, 0), oracle.outcome_prob(psi, 0, 1), oracle.outcome_prob(psi, n - 1, 1)]
        L = (1 << n) // world
        probs = oracle.probs(psi)
        for rank, r in enumerate(rs):
            np.testing.assert_allclose(r["expect"], ev, atol=1e-12)
            np.testing.assert_allclose(r["p_q0"], p_want, atol=1e-13)
            np.testing.assert_allclose(r["state2"], psi, atol=1e-12)
            np.testing.assert_allclose(r["probs"], probs[rank * L:(rank + 1) * L], atol=1e-13)
        c = psi.copy()
        P1 = oracle.outcome_prob(c, 0, 1)
        oracle.collapse(c, 0, 1, P1)
        P2 = oracle.outcome_prob(c, n - 2, 0)
        oracle.collapse(c, n - 2, 0, P2)
        for r in rs:
            np.testing.assert_allclose(r["collapse_p"], [P1, P2], atol=1e-13)
            np.testing.assert_allclose(r["state3"], c, atol=1e-12)
