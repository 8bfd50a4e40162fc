"""OpenQASM 2 text for circuits (Sec. 4: QCLAB writes a circuit as OpenQASM with
``toQASM`` so that it can be run elsewhere).

``to_qasm(n, ops)`` writes one statement per operation in the form the paper prints
for its Bell circuit -- ``qreg q[n];`` then ``h q[0];``, ``cx q[0], q[1];``,
``measure q[0];`` -- optionally preceded by the standard ``OPENQASM 2.0;`` /
``include "qelib1.inc";`` header.  ``from_qasm(text)`` reads that subset of OpenQASM 2
back into operation records that ``State.run``, ``Circuit`` and ``simulate`` accept.

Host-side text handling only: no amplitude is touched here.

Gate names (qelib1): ``h x y z s sdg t tdg``, ``rx ry rz`` (one angle), ``u3``/``u``/``U``
(theta, phi, lambda), ``u1``/``p`` (lambda, read as u3(0, 0, lambda) = diag(1, e^{i lambda})),
``u2`` (phi, lambda, read as u3(pi/2, phi, lambda)), ``cx``/``CX``, ``cz``, ``cp``/``cu1``,
``swap``, ``ccx``; ``measure``, ``reset``; ``barrier``, ``creg`` and the header are
accepted and ignored.  Angles are expressions of numbers and ``pi`` with ``+ - * /``,
``^``, unary minus and parentheses.  A statement naming a whole register (``h q;``)
applies to each of its qubits.  Several ``qreg`` declarations are laid out in the
order they are declared (the first register's qubit 0 is qubit 0 of the circuit).
"""
from __future__ import annotations

import math
import re
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class GateOp:
    """One circuit operation (the fields ``Circuit`` reads)."""

    kind: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = None
    ctrl_states: Optional[Tuple[int, ...]] = None
    param_index: Optional[int] = None


_FIXED_1Q = ("h", "x", "y", "z", "s", "sdg", "t", "tdg")
_ROT_1Q = ("rx", "ry", "rz")


# ---------------------------------------------------------------------------
# export
# ---------------------------------------------------------------------------

def _fmt(x: float) -> str:
    return repr(float(x))  # shortest decimal that reads back to the same double


def _angles(op, params) -> Tuple[float, ...]:
    if op.param_index is not None:
        if params is None:
            raise ValueError("op %s takes parameter %d: pass params" % (op.kind, op.param_index))
        cnt = 3 if op.kind == "u3" else 1
        return tuple(float(params[op.param_index + j]) for j in range(cnt))
    return tuple(float(p) for p in op.params)


def to_qasm(n: int, ops: Sequence, params=None, header: bool = False) -> str:
    """OpenQASM 2 text of ``ops`` on ``n`` qubits.  Ops with a caller-supplied matrix
    (``u1q``/``u2q``/``ukq``/``ctrl``) and controlled X with more than two controls have
    no qelib1 form and raise ValueError.  X- and Y-basis measurements are written as
    their basis change around a Z measurement (H .. H; S^dagger H .. H S)."""
    if n < 1:
        raise ValueError("n must be positive")
    lines = []
    if header:
        lines += ["OPENQASM 2.0;", 'include "qelib1.inc";']
    lines.append("qreg q[%d];" % n)

    def q(i):
        if not 0 <= i < n:
            raise ValueError("qubit %d out of range" % i)
        return "q[%d]" % i

    for op in ops:
        k, qs = op.kind, tuple(int(x) for x in op.qubits)
        if k in _FIXED_1Q:
            lines.append("%s %s;" % (k, q(qs[0])))
        elif k in _ROT_1Q:
            (a,) = _angles(op, params)
            lines.append("%s(%s) %s;" % (k, _fmt(a), q(qs[0])))
        elif k == "u3":
            a = _angles(op, params)
            lines.append("u3(%s,%s,%s) %s;" % (_fmt(a[0]), _fmt(a[1]), _fmt(a[2]), q(qs[0])))
        elif k in ("cnot", "cz", "swap"):
            name = {"cnot": "cx", "cz": "cz", "swap": "swap"}[k]
            lines.append("%s %s, %s;" % (name, q(qs[0]), q(qs[1])))
        elif k == "cp":
            (a,) = _angles(op, params)
            lines.append("cp(%s) %s, %s;" % (_fmt(a), q(qs[0]), q(qs[1])))
        elif k == "mcx":
            ctrls, tgt = qs[:-1], qs[-1]
            states = op.ctrl_states if op.ctrl_states is not None else (1,) * len(ctrls)
            if len(ctrls) > 2:
                raise ValueError("controlled X with %d controls has no qelib1 gate" % len(ctrls))
            opened = [c for c, s in zip(ctrls, states) if not s]
            lines += ["x %s;" % q(c) for c in opened]  # an open control is X . control . X
            name = "cx" if len(ctrls) == 1 else "ccx"
            lines.append("%s %s;" % (name, ", ".join(q(c) for c in ctrls + (tgt,))))
            lines += ["x %s;" % q(c) for c in opened]
        elif k in ("measure", "measure_z"):
            lines.append("measure %s;" % q(qs[0]))
        elif k == "measure_x":
            lines += ["h %s;" % q(qs[0]), "measure %s;" % q(qs[0]), "h %s;" % q(qs[0])]
        elif k == "measure_y":
            lines += ["sdg %s;" % q(qs[0]), "h %s;" % q(qs[0]), "measure %s;" % q(qs[0]),
                      "h %s;" % q(qs[0]), "s %s;" % q(qs[0])]
        elif k == "reset":
            lines.append("reset %s;" % q(qs[0]))
        else:
            raise ValueError("op kind %r has no OpenQASM 2 (qelib1) form" % k)
    return "\n".join(lines) + "\n"


# ---------------------------------------------------------------------------
# import
# ---------------------------------------------------------------------------

_TOKEN = re.compile(r"\s*(?:(\d+\.\d*(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?)|(pi)|([-+*/^()]))")


def _eval_angle(s: str) -> float:
    """Value of an angle expression: numbers, pi, + - * / ^, unary minus, parentheses
    (recursive descent; ^ binds tightest and is right-associative)."""
    toks = []
    pos = 0
    s = s.strip()
    while pos < len(s):
        m = _TOKEN.match(s, pos)
        if not m or m.end() == pos:
            raise ValueError("bad angle expression %r" % s)
        toks.append(m.group(1) or m.group(2) or m.group(3))
        pos = m.end()
        while pos < len(s) and s[pos].isspace():
            pos += 1
    i = 0

    def peek():
        return toks[i] if i < len(toks) else None

    def take():
        nonlocal i
        i += 1
        return toks[i - 1]

    def atom():
        t = take() if peek() is not None else None
        if t is None:
            raise ValueError("bad angle expression %r" % s)
        if t == "(":
            v = expr()
            if peek() != ")":
                raise ValueError("unbalanced parentheses in %r" % s)
            take()
            return v
        if t == "pi":
            return math.pi
        if t == "-":
            return -power()
        if t == "+":
            return power()
        try:
            return float(t)
        except ValueError:
            raise ValueError("bad angle expression %r" % s) from None

    def power():
        b = atom()
        if peek() == "^":
            take()
            return b ** power()
        return b

    def term():
        v = power()
        while peek() in ("*", "/"):
            if take() == "*":
                v *= power()
            else:
                v /= power()
        return v

    def expr():
        v = term()
        while peek() in ("+", "-"):
            if take() == "+":
                v += term()
            else:
                v -= term()
        return v

    v = expr()
    if i != len(toks):
        raise ValueError("bad angle expression %r" % s)
    return v


_STMT = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)\s*(?:\((.*)\))?\s*(.*)$", re.S)
_ARG = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)\s*(?:\[\s*(\d+)\s*\])?$")


def _split_args(s: str) -> List[str]:
    out, depth, cur = [], 0, ""
    for ch in s:
        if ch == "(":
            depth += 1
        elif ch == ")":
            depth -= 1
        if ch == "," and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    if cur.strip():
        out.append(cur)
    return [a.strip() for a in out]


def from_qasm(text: str) -> Tuple[int, List[GateOp]]:
    """(n, ops) of an OpenQASM 2 program in the subset described in the module
    docstring.  Anything else (gate definitions, classical conditions, opaque
    gates, unknown gate names) raises ValueError naming the statement."""
    text = re.sub(r"//[^\n]*", "", text)
    regs = {}  # name -> (offset, size)
    n = 0
    ops: List[GateOp] = []
    for raw in text.split(";"):
        st = " ".join(raw.split())
        if not st:
            continue
        if st.startswith("OPENQASM") or st.startswith("include"):
            continue
        if st.startswith("gate ") or st.startswith("opaque ") or st.startswith("if"):
            raise ValueError("unsupported statement: %r" % st)
        m = _STMT.match(st)
        if not m:
            raise ValueError("cannot parse statement %r" % st)
        name, pargs, rest = m.group(1), m.group(2), m.group(3).strip()
        if name in ("qreg", "creg"):
            a = _ARG.match(rest)
            if not a or a.group(2) is None:
                raise ValueError("bad register declaration %r" % st)
            if name == "qreg":
                if a.group(1) in regs:
                    raise ValueError("register %s declared twice" % a.group(1))
                regs[a.group(1)] = (n, int(a.group(2)))
                n += int(a.group(2))
            continue
        if name == "barrier":
            continue
        if name == "measure":
            rest = rest.split("->")[0].strip()
        angles = tuple(_eval_angle(p) for p in _split_args(pargs)) if pargs else ()
        targets = []
        for a in _split_args(rest):
            am = _ARG.match(a)
            if not am or am.group(1) not in regs:
                raise ValueError("unknown qubit argument %r in %r" % (a, st))
            off, size = regs[am.group(1)]
            if am.group(2) is None:
                targets.append([off + j for j in range(size)])
            else:
                j = int(am.group(2))
                if j >= size:
                    raise ValueError("index %d out of range for %s in %r" % (j, am.group(1), st))
                targets.append([off + j])
        widths = {len(t) for t in targets if len(t) > 1}
        if len(widths) > 1:
            raise ValueError("register arguments of different sizes in %r" % st)
        reps = widths.pop() if widths else 1
        for r in range(reps):
            qs = tuple(t[r] if len(t) > 1 else t[0] for t in targets)
            ops.append(_gate(name, angles, qs, st))
    if n == 0:
        raise ValueError("no qreg declared")
    return n, ops


def _gate(name: str, a: Tuple[float, ...], qs: Tuple[int, ...], st: str) -> GateOp:
    def need(na, nq):
        if len(a) != na or len(qs) != nq:
            raise ValueError("%s takes %d angle(s) and %d qubit(s): %r" % (name, na, nq, st))
        if len(set(qs)) != len(qs):
            raise ValueError("repeated qubit in %r" % st)

    if name in _FIXED_1Q:
        need(0, 1)
        return GateOp(name, qs)
    if name in _ROT_1Q:
        need(1, 1)
        return GateOp(name, qs, a)
    if name in ("u3", "u", "U"):
        need(3, 1)
        return GateOp("u3", qs, a)
    if name in ("u1", "p"):
        need(1, 1)
        return GateOp("u3", qs, (0.0, 0.0, a[0]))
    if name == "u2":
        need(2, 1)
        return GateOp("u3", qs, (math.pi / 2, a[0], a[1]))
    if name in ("cx", "CX"):
        need(0, 2)
        return GateOp("cnot", qs)
    if name in ("cz", "swap"):
        need(0, 2)
        return GateOp(name, qs)
    if name in ("cp", "cu1"):
        need(1, 2)
        return GateOp("cp", qs, a)
    if name == "ccx":
        need(0, 3)
        return GateOp("mcx", qs, ctrl_states=(1, 1))
    if name in ("measure", "reset"):
        need(0, 1)
        return GateOp(name, qs)
    raise ValueError("unsupported gate %r in %r" % (name, st))
