"""A state vector split over processes by its top index bits: the full state vector of
QCLAB Sec. 3 held by W = 2^g processes (one GPU each), 2^(n-g) amplitudes per process.

Physical positions.  The register's n qubits sit at physical positions 0..n-1 (position
p is index bit n-1-p, so position 0 is the most significant bit).  Positions 0..g-1 are
*global*: they are the bits of the process rank (position p is rank bit g-1-p).
Positions g..n-1 are *local*: position p is qubit p-g of the process's own shard
register.  ``pos[q]`` is the position of logical qubit q; a SWAP of two qubits only
exchanges their positions (no data moves).

Gates (Sec. 3.2 applied to the distributed register):

* every target local: the gate runs on the shard (the library's fused tile passes), its
  controls on global positions resolved from the rank: a control whose rank bit does not
  read its required value makes the gate the identity on this process, one that does is
  dropped;
* CZ and CP with one qubit global: they are symmetric, so the global qubit is taken as
  the control;
* Z, S, S^dagger, T, T^dagger (diag(1, d)) on a global position, and CZ / CP with both
  qubits global: no communication; a process whose bits read 1 multiplies its whole
  shard by d, applied on its local qubit 0 as G X G X = diag(d, d);
* any other gate with a global target: the target is first brought to a local position
  by a pairwise exchange: the global position p and the top local position g swap
  their qubits, which moves the half of each shard whose top local bit differs from the
  rank bit to the partner process (rank with bit g-1-p flipped) -- one contiguous half
  each way (torch.distributed send/recv; NCCL between GPUs), received into a staging
  buffer and copied into place.  The qubit evicted from the local positions is the one
  used least recently; a local SWAP first moves it to the top local position.

Every placement decision depends only on the gate sequence, never on the rank, so all
processes take the same exchanges in the same order and every send meets its receive.

Readouts: probabilities after restoring the identity placement (each process holds its
slice of the vector, index offset rank * 2^(n-g)); Pauli expectations: Z factors on
global positions become the rank's sign (the library multiplies by it as the term's
coefficient); a string with X or Y factors on global positions pairs each process with
the partner its X part maps it to, which sends its whole shard (the library applies
the local factors to the copy and forms the inner product); the shares are summed over
the processes (all-reduce); outcome probabilities and collapse (Sec. 3.3) with the outcome
probability summed over the processes and the shards renormalised by it
(qc_collapse_norm).  All arithmetic runs in the library's kernels; this module moves
data between processes and keeps the placement.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import _binding as B

_SELF_DIAG_1Q = ("z", "s", "sdg", "t", "tdg")  # diag(1, d): identity where the bit reads 0
_ONE_Q = ("h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "u3", "u1q")
_CTRL = ("cnot", "cz", "cp", "mcx", "ctrl")


@dataclass(frozen=True)
class ShardOp:
    """A gate on the shard register (same fields as the circuit descriptions
    :class:`Circuit` accepts)."""
    kind: str
    qubits: tuple
    params: tuple = ()
    matrix: Optional[np.ndarray] = None
    ctrl_states: Optional[tuple] = None
    param_index: Optional[int] = None


class CudaShard:
    """The local engine of a process: its shard as a complex64/complex128 state on the
    process's GPU, every gate and readout in the library."""

    def __init__(self, n_local: int, dtype: str = "c64", stream=None):
        from .state import State
        self.nl = n_local
        self.dtype = dtype
        self.st = State(n_local, dtype, stream)

    def amplitudes(self):
        return self.st.tensor

    def init_basis(self, index: Optional[int]) -> None:
        B.qc_state_init_basis(self.st.handle, 0 if index is None else index)
        if index is None:  # this process holds none of the amplitude: all zero
            B.qc_collapse_norm(self.st.handle, -1, 0, 0.0)

    def load(self, amps) -> None:
        self.st.init_vector(amps)

    def run(self, ops: Sequence[ShardOp], params=None) -> None:
        if ops:
            self.st.run(B.Circuit(self.nl, list(ops)), params, mode=B.QC_RUN_FUSED)

    def probs(self):
        return self.st.probs()

    def expect(self, strings, coeffs) -> np.ndarray:
        return B.qc_expect_pauli(self.st.handle, strings, coeffs)

    def outcome_prob(self, q: int, outcome: int) -> float:
        return B.qc_outcome_prob(self.st.handle, q, outcome)

    def collapse_norm(self, q: int, outcome: int, p: float) -> None:
        B.qc_collapse_norm(self.st.handle, q, outcome, p)

    def download(self) -> np.ndarray:
        return self.st.numpy()

    # a second shard-sized buffer (a partner's shard for cross-process expectations)
    def scratch_amplitudes(self):
        if getattr(self, "scr", None) is None:
            from .state import State
            self.scr = State(self.nl, self.dtype, None)
        return self.scr.tensor

    def scratch_run(self, ops) -> None:
        if ops:
            self.scr.run(B.Circuit(self.nl, list(ops)), None, mode=B.QC_RUN_PER_GATE)

    def inner_scratch(self) -> complex:
        """<own shard | scratch>."""
        return B.qc_inner(self.st.handle, self.scr.handle)


class ShardedState:
    """An n-qubit register over the processes of ``group`` (a power of two of them),
    each holding its shard in ``engine`` (a :class:`CudaShard` on its GPU)."""

    def __init__(self, n: int, engine, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        world = dist.get_world_size(group)
        g = world.bit_length() - 1
        if 1 << g != world:
            raise ValueError("the number of processes must be a power of two, got %d" % world)
        if engine.nl != n - g or n - g < 1:
            raise ValueError("a shard must hold n - log2(processes) >= 1 qubits")
        self.n, self.g, self.world = n, g, world
        self.rank = dist.get_rank(group)
        self.eng = engine
        self.pos = list(range(n))  # physical position of each logical qubit
        self.at = list(range(n))  # logical qubit at each physical position
        self.last_use = [0] * n
        self.clock = 0
        self.pending: List[ShardOp] = []
        self.params = None
        self.exchanges = 0
        self._stage = None

    # placement ---------------------------------------------------------------
    def _global(self, q: int) -> bool:
        return self.pos[q] < self.g

    def _bit(self, q: int) -> int:
        return (self.rank >> (self.g - 1 - self.pos[q])) & 1

    def _local(self, q: int) -> int:
        return self.pos[q] - self.g

    def _relabel(self, x: int, y: int) -> None:
        qx, qy = self.at[x], self.at[y]
        self.at[x], self.at[y] = qy, qx
        self.pos[qx], self.pos[qy] = y, x

    # shard work ----------------------------------------------------------------
    def _emit(self, op: ShardOp) -> None:
        self.pending.append(op)

    def _flush(self) -> None:
        if self.pending:
            self.eng.run(self.pending, self.params)
            self.pending = []

    def _swap_local_positions(self, x: int, y: int) -> None:
        """Swaps the qubits at local positions x and y (a SWAP on the shard)."""
        self._emit(ShardOp("swap", (x - self.g, y - self.g)))
        self._relabel(x, y)

    def _exchange_top(self, p: int) -> None:
        """Swaps the qubits at global position p and the top local position g: the half
        of the shard whose top local bit differs from rank bit g-1-p goes to the partner,
        whose matching half comes back into the same place."""
        import torch
        self._flush()
        a = (self.rank >> (self.g - 1 - p)) & 1
        partner = self.rank ^ (1 << (self.g - 1 - p))
        t = self.eng.amplitudes()
        half = t.numel() // 2
        send = t[(1 - a) * half:(2 - a) * half]
        if self._stage is None or self._stage.numel() != half or self._stage.dtype != t.dtype:
            self._stage = torch.empty(half, dtype=t.dtype, device=t.device)
        sr, rr = torch.view_as_real(send), torch.view_as_real(self._stage)
        ops = [self.dist.P2POp(self.dist.isend, sr, partner, self.group),
               self.dist.P2POp(self.dist.irecv, rr, partner, self.group)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()
        send.copy_(self._stage)
        self._relabel(p, self.g)
        self.exchanges += 1

    def _swap_positions(self, x: int, y: int) -> None:
        """Exchanges the qubits at any two physical positions."""
        if x == y:
            return
        if x > y:
            x, y = y, x
        g = self.g
        if x >= g:
            self._swap_local_positions(x, y)
        elif y >= g:
            if y == g:
                self._exchange_top(x)
            else:
                self._swap_local_positions(y, g)
                self._exchange_top(x)
                self._swap_local_positions(y, g)
        else:  # both global: (x g)(y g)(x g) = (x y)
            self._swap_positions(x, g)
            self._swap_positions(y, g)
            self._swap_positions(x, g)

    def _swap_in(self, qubits: Sequence[int]) -> None:
        """Brings every qubit of `qubits` to a local position, evicting the local qubits
        used least recently (never one of `qubits`)."""
        keep = set(qubits)
        for q in qubits:
            if not self._global(q):
                continue
            cands = [p for p in range(self.g, self.n) if self.at[p] not in keep]
            if not cands:
                raise ValueError("a gate needs more qubits local than a shard holds")
            victim = min(cands, key=lambda p: (self.last_use[self.at[p]], -p))
            if victim != self.g:
                self._swap_local_positions(victim, self.g)
            self._exchange_top(self.pos[q])

    def normalize(self) -> None:
        """Restores the identity placement (logical qubit q at position q)."""
        for p in range(self.n):
            if self.at[p] != p:
                self._swap_positions(p, self.pos[p])
        self._flush()

    # initialisation ----------------------------------------------------------
    def init_basis(self, index: int) -> "ShardedState":
        self.pos = list(range(self.n))
        self.at = list(range(self.n))
        self.pending = []
        L = self.n - self.g
        owner = index >> L
        self.eng.init_basis(index & ((1 << L) - 1) if owner == self.rank else None)
        return self

    def init_vector(self, full) -> "ShardedState":
        """Loads this process's slice of a full host vector (identity placement)."""
        self.pos = list(range(self.n))
        self.at = list(range(self.n))
        self.pending = []
        L = 1 << (self.n - self.g)
        self.eng.load(np.ascontiguousarray(full[self.rank * L:(self.rank + 1) * L]))
        return self

    # gates ---------------------------------------------------------------------
    def run(self, ops, params=None) -> "ShardedState":
        """Applies the circuit description ``ops`` (the kinds :class:`Circuit` accepts)
        in order; ``params`` supplies angles of ops with a parameter index."""
        self.params = None if params is None else np.asarray(params, dtype=np.float64)
        for op in ops:
            self.clock += 1
            for q in op.qubits:
                self.last_use[q] = self.clock
            self._gate(op)
        self._flush()
        return self

    def _shard_scalar(self, gate: str, params=(), param_index=None) -> None:
        """The whole shard times d for the diagonal gate diag(1, d) named `gate`:
        G X G X = diag(d, d) on local qubit 0."""
        for k in (gate, "x", gate, "x"):
            self._emit(ShardOp(k, (0,), params if k == gate else (), None, None,
                               param_index if k == gate else None))

    def _gate(self, op) -> None:
        kind = op.kind
        dag = kind.endswith("_dag")
        base = kind[:-4] if dag else kind
        sfx = "_dag" if dag else ""
        qs = list(op.qubits)
        if base == "swap":
            self._relabel(self.pos[qs[0]], self.pos[qs[1]])
            return
        if base in _CTRL:
            ctrls, tgt = qs[:-1], qs[-1]
            states = list(op.ctrl_states) if op.ctrl_states is not None else [1] * len(ctrls)
            if base in ("cz", "cp") and self._global(tgt) and not self._global(ctrls[0]):
                ctrls, tgt = [tgt], ctrls[0]
            if self._global(tgt) and base not in ("cz", "cp"):
                # placement changes are taken by every process alike (before the rank
                # decides whether the gate acts on it), so exchanges always pair up
                self._swap_in([tgt] + [c for c in ctrls if not self._global(c)])
            keep_c, keep_s = [], []
            for c, s in zip(ctrls, states):
                if self._global(c):
                    if self._bit(c) != int(s):
                        return  # the identity on this process
                else:
                    keep_c.append(c)
                    keep_s.append(int(s))
            if self._global(tgt):  # CZ / CP with both qubits global, the control reads 1
                if self._bit(tgt) == 1:
                    if base == "cz":
                        self._shard_scalar("z")
                    else:
                        self._shard_scalar("u3" + sfx, (0.0, 0.0, self._angle(op)))
                return
            self._emit_ctrl(base, sfx, op, keep_c, keep_s, tgt)
            return
        if base in _ONE_Q:
            q = qs[0]
            if self._global(q):
                if base in _SELF_DIAG_1Q:
                    if self._bit(q) == 1:
                        self._shard_scalar(kind)
                    return
                self._swap_in([q])
            self._emit(ShardOp(kind, (self._local(q),), tuple(op.params), op.matrix, None, op.param_index))
            return
        # dense multi-qubit gates
        self._swap_in(qs)
        self._emit(ShardOp(kind, tuple(self._local(q) for q in qs), tuple(op.params), op.matrix, op.ctrl_states,
                           op.param_index))

    def _angle(self, op) -> float:
        if op.param_index is not None:
            return float(self.params[op.param_index])
        return float(op.params[0])

    def _emit_ctrl(self, base, sfx, op, keep_c, keep_s, tgt) -> None:
        lc = tuple(self._local(c) for c in keep_c)
        lt = self._local(tgt)
        if not lc:
            if base in ("cnot", "mcx"):
                self._emit(ShardOp("x", (lt,)))
            elif base == "cz":
                self._emit(ShardOp("z", (lt,)))
            elif base == "cp":
                self._emit(ShardOp("u3" + sfx, (lt,), (0.0, 0.0, self._angle(op))))
            else:
                self._emit(ShardOp("u1q" + sfx, (lt,), (), op.matrix))
            return
        if base in ("cnot", "cz", "cp"):
            self._emit(ShardOp(base + sfx, lc + (lt,), tuple(op.params), None, None, op.param_index))
        elif base == "mcx":
            self._emit(ShardOp("mcx", lc + (lt,), (), None, tuple(keep_s)))
        else:
            self._emit(ShardOp("ctrl" + sfx, lc + (lt,), (), op.matrix, tuple(keep_s)))

    # readout -------------------------------------------------------------------
    def _sum(self, v: np.ndarray) -> np.ndarray:
        import torch
        t = torch.tensor(np.asarray(v, dtype=np.float64))
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def probs(self):
        """This process's slice of the probability vector (index offset
        rank * 2^(n-g)), after restoring the identity placement."""
        self.normalize()
        return self.eng.probs()

    def gather(self) -> np.ndarray:
        """The full state vector on every process (identity placement); for checks."""
        import torch
        self.normalize()
        t = self.eng.amplitudes()
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather([torch.view_as_real(p) for p in parts], torch.view_as_real(t.contiguous()),
                             group=self.group)
        return np.concatenate([p.cpu().numpy() for p in parts])

    def expect(self, strings: Sequence[str], coeffs=None) -> np.ndarray:
        """coeffs[t] <psi| P_t |psi> over the whole register (strings of I/X/Y/Z,
        character j on qubit j)."""
        out = np.zeros(len(strings))
        plain, plain_idx = [], []
        for t, s in enumerate(strings):
            if any(c in "XYxy" and self._global(q) for q, c in enumerate(s)):
                out[t] = self._cross_expect(s)
            else:
                plain.append(s)
                plain_idx.append(t)
        if plain:
            vals = self._local_expect(plain, plain_idx)
            for t, v in zip(plain_idx, vals):
                out[t] = v
        if coeffs is not None:
            out = out * np.asarray(coeffs, dtype=np.float64)
        return self._sum(out)

    def _cross_expect(self, s: str) -> float:
        """This process's share of <psi|P|psi> when P has X or Y factors on global
        positions.  With P|j> = i^{ny} (-1)^{|j & z|} |j ^ x>, the share of process r is
        i^{ny} (-1)^{|(r ^ xg) & zg|} <psi_r| X^{xl} Z^{zl} psi_{r ^ xg}>: the partner
        r ^ xg (global part xg of x) sends its whole shard, Z then X act on the local
        factors of the received copy, and the library forms the inner product."""
        import torch
        self._flush()
        xg = zg = 0
        ny = 0
        zops, xops = [], []
        for q, c in enumerate(s.upper()):
            if c == "I":
                continue
            ny += c == "Y"
            if self._global(q):
                b = 1 << (self.g - 1 - self.pos[q])
                xg |= b if c in "XY" else 0
                zg |= b if c in "ZY" else 0
            else:
                if c in "ZY":
                    zops.append(ShardOp("z", (self._local(q),)))
                if c in "XY":
                    xops.append(ShardOp("x", (self._local(q),)))
        partner = self.rank ^ xg
        own = self.eng.amplitudes()
        other = self.eng.scratch_amplitudes()
        ops = [self.dist.P2POp(self.dist.isend, torch.view_as_real(own), partner, self.group),
               self.dist.P2POp(self.dist.irecv, torch.view_as_real(other), partner, self.group)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()
        self.exchanges += 1
        self.eng.scratch_run(zops + xops)
        v = self.eng.inner_scratch()
        sign = -1.0 if bin(partner & zg).count("1") & 1 else 1.0
        return float((v * (1j ** ny) * sign).real)

    def _local_expect(self, strings, idx) -> np.ndarray:
        self._flush()
        nl = self.n - self.g
        loc, sign = [], []
        for s in strings:
            ls = ["I"] * nl
            sg = 1.0
            for q, c in enumerate(s):
                c = c.upper()
                if c == "I":
                    continue
                if self._global(q):  # only Z factors remain on global positions
                    if self._bit(q):
                        sg = -sg
                else:
                    ls[self._local(q)] = c
            loc.append("".join(ls))
            sign.append(sg)
        return self.eng.expect(loc, np.array(sign))

    def outcome_prob(self, q: int, outcome: int) -> float:
        """P(outcome) of qubit q summed over the processes (Sec. 3.3)."""
        self._flush()
        if self._global(q):
            v = self.eng.expect(["I" * (self.n - self.g)], np.ones(1))[0] if self._bit(q) == outcome else 0.0
        else:
            v = self.eng.outcome_prob(self._local(q), outcome)
        return float(self._sum(np.array([v]))[0])

    def collapse(self, q: int, outcome: int, zero_prob: Optional[float] = None) -> float:
        """Collapses qubit q onto `outcome` and renormalises every shard by the total
        outcome probability; returns it (QCError-free: raises ValueError when it is
        below the branch threshold)."""
        P = self.outcome_prob(q, outcome)
        thr = zero_prob if zero_prob is not None else (1e-6 if self.eng.dtype == "c64" else 1e-12)
        if P <= thr:
            raise ValueError("outcome %d of qubit %d has probability %.3g" % (outcome, q, P))
        if self._global(q):
            self.eng.collapse_norm(-1, 0, P if self._bit(q) == outcome else 0.0)
        else:
            self.eng.collapse_norm(self._local(q), outcome, P)
        return P
