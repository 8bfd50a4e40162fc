"""ctypes binding of the C ABI in include/qc.h (argument marshalling only).

Every function keeps the C name.  Device buffers are passed as torch CUDA tensors
(or raw integer addresses); streams default to torch's current stream.  A non-zero
status raises :class:`QCError` carrying ``qc_last_error()``.  There is no CPU
fallback: if the CUDA library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqcgb.so")

QC_C64, QC_C128 = 0, 1
QC_PREC_NATIVE, QC_PREC_TF32X3, QC_PREC_BF16X3, QC_PREC_AUTO = 0, 1, 2, 3
QC_RUN_PER_GATE, QC_RUN_FUSED = 0, 1
STATUS = {0: "QC_OK", 1: "QC_ERR_INVALID_ARG", 2: "QC_ERR_OOM", 3: "QC_ERR_CUDA", 4: "QC_ERR_UNSUPPORTED",
          5: "QC_ERR_ZERO_PROB", 6: "QC_ERR_TIMEOUT"}

GATE = {"u1q": 0, "u2q": 1, "h": 2, "x": 3, "y": 4, "z": 5, "s": 6, "sdg": 7, "t": 8, "tdg": 9, "rx": 10,
        "ry": 11, "rz": 12, "u3": 13, "cnot": 14, "cz": 15, "cp": 16, "swap": 17, "mcx": 18, "ctrl": 19}
MAX_OP_QUBITS = 8


class QCError(RuntimeError):
    def __init__(self, func: str, status: int, msg: str):
        super().__init__("%s failed: %s (%s)" % (func, STATUS.get(status, status), msg))
        self.status = status


class qc_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nq", ctypes.c_int32), ("qubits", ctypes.c_int32 * MAX_OP_QUBITS),
                ("ctrl_states", ctypes.c_uint32), ("param", ctypes.c_int32), ("adjoint", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("angle", ctypes.c_double * 3), ("matrix", ctypes.c_int64)]


class qc_circuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nops", ctypes.c_int32), ("ops", ctypes.POINTER(qc_op)),
                ("pool", ctypes.POINTER(ctypes.c_double)), ("pool_len", ctypes.c_int64)]


class qc_ansatz_batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("layers", ctypes.c_int32), ("n", ctypes.POINTER(ctypes.c_int32)),
                ("param_offset", ctypes.POINTER(ctypes.c_int64)), ("dev_params", ctypes.c_void_p),
                ("nparams", ctypes.c_int64)]


class qc_pauli_term(ctypes.Structure):
    _fields_ = [("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64), ("coeff", ctypes.c_double)]


class qc_hamiltonian(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int32), ("reserved", ctypes.c_int32), ("terms", ctypes.POINTER(qc_pauli_term))]


class qc_batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("shared_observable", ctypes.c_int32),
                ("circuits", ctypes.POINTER(qc_circuit)), ("param_offset", ctypes.POINTER(ctypes.c_int64)),
                ("dev_params", ctypes.c_void_p), ("nparams", ctypes.c_int64),
                ("observables", ctypes.POINTER(qc_hamiltonian)), ("dev_states", ctypes.POINTER(ctypes.c_void_p))]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "qc_last_error": (ctypes.c_char_p, []),
    "qc_abi_version": (ctypes.c_int, []),
    "qc_launch_count": (ctypes.c_uint64, []),
    "qc_status_of_device_word": (ctypes.c_int, [ctypes.c_int]),
    "qc_last_pass_count": (ctypes.c_int, []),
    "qc_last_fused_path": (ctypes.c_int, []),
    "qc_last_stage_count": (ctypes.c_int, []),
    "qc_plan_info": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, _I, _I, _I]),
    "qc_tc_box_plan": (ctypes.c_int, [ctypes.c_int, _I, _I, _I, _I]),
    "qc_tc_block_plan": (ctypes.c_int, [ctypes.c_int, _I, ctypes.c_int, _I, _I, _I]),
    "qc_tc_emulate": (ctypes.c_int, [ctypes.c_void_p, _D, _D]),
    "qc_tc_plan_info": (ctypes.c_int, [ctypes.c_void_p, _D, _I, _I, _I, _I]),
    "qc_tile_emulate": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, _D]),
    "qc_adjoint_emulate": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, _D, _D, _D, ctypes.c_int]),
    "qc_state_alloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "qc_state_wrap": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(_P)]),
    "qc_state_free": (ctypes.c_int, [_P]),
    "qc_state_info": (ctypes.c_int, [_P, _I, _I, ctypes.POINTER(_P)]),
    "qc_state_set_stream": (ctypes.c_int, [_P, _P]),
    "qc_state_init_basis": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "qc_state_init_vector": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
    "qc_state_init_gaussian": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "qc_state_copy": (ctypes.c_int, [_P, _P]),
    "qc_state_download": (ctypes.c_int, [_P, _P]),
    "qc_apply_1q": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "qc_apply_2q": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
    "qc_apply_ctrl": (ctypes.c_int, [_P, _I, _I, ctypes.c_int, ctypes.c_int, _D]),
    "qc_apply_fused_k": (ctypes.c_int, [_P, _I, ctypes.c_int, _D, ctypes.c_int]),
    "qc_measure": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _I, _D]),
    "qc_collapse": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
    "qc_outcome_prob": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
    "qc_collapse_norm": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "qc_inner": (ctypes.c_int, [_P, _P, _D]),
    "qc_probs": (ctypes.c_int, [_P, _P]),
    "qc_sample": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "qc_sample_probs": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int64, _P]),
    "qc_expect_pauli": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_char_p), _D, ctypes.c_int, _D]),
    "qc_reduced_state": (ctypes.c_int, [_P, _I, _I, ctypes.c_int, _P]),
    "qc_marginal_probs": (ctypes.c_int, [_P, _I, ctypes.c_int, _P]),
    "qc_expect_pauli_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_char_p), _D, ctypes.c_int, _D]),
    "qc_run_circuit": (ctypes.c_int, [_P, ctypes.POINTER(qc_circuit), _D, ctypes.c_int, ctypes.c_int]),
    "qc_adjoint_grad": (ctypes.c_int, [ctypes.POINTER(qc_circuit), _D, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_char_p), _D, ctypes.c_int, ctypes.c_int, _P, _D,
                                       _D]),
    "qc_adjoint_grad_dev": (ctypes.c_int, [ctypes.POINTER(qc_circuit), _P, ctypes.c_int, ctypes.POINTER(qc_hamiltonian),
                                           ctypes.c_int, _P, _P, _P]),
    "qc_run_ansatz_batch": (ctypes.c_int, [ctypes.POINTER(qc_ansatz_batch), _P, _P]),
    "qc_run_batch": (ctypes.c_int, [ctypes.POINTER(qc_batch), _P, _P]),
    "qc_last_batch_path": (ctypes.c_int, []),
    "qc_batch_fusion_width": (ctypes.c_int, []),
}

_lib = None


def lib():
    """The loaded CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() (no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(name: str, st: int):
    if st != 0:
        msg = lib().qc_last_error().decode(errors="replace")
        raise QCError(name, st, msg)


def _call(name: str, *args):
    _check(name, getattr(lib(), name)(*args))


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError("expected a tensor, ndarray or address, got %r" % type(x))


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream) or None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None


def _mat(U, dim: int):
    a = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(dim, dim)).view(np.float64).ravel()
    return a, a.ctypes.data_as(_D)


def qc_launch_count() -> int:
    return int(lib().qc_launch_count())


def qc_last_pass_count() -> int:
    return int(lib().qc_last_pass_count())


def qc_last_fused_path() -> int:
    """0 per gate, 1 CUDA-core tile passes, 2 tile passes with tensor-core stages."""
    return int(lib().qc_last_fused_path())


def qc_last_stage_count() -> int:
    """Register stages (or tensor-core stage blocks) of the most recent fused circuit."""
    return int(lib().qc_last_stage_count())


# ---------------------------------------------------------------------------
# state handles
# ---------------------------------------------------------------------------

def qc_state_alloc(n: int, dtype: int = QC_C64, stream=None) -> int:
    h = _P()
    _call("qc_state_alloc", n, dtype, _stream(stream), ctypes.byref(h))
    return h.value


def qc_state_wrap(n: int, dtype: int, amps, stream=None) -> int:
    h = _P()
    _call("qc_state_wrap", n, dtype, _ptr(amps), _stream(stream), ctypes.byref(h))
    return h.value


def qc_state_free(h: int) -> None:
    _call("qc_state_free", h)


def qc_state_info(h: int):
    n, dt, p = ctypes.c_int(), ctypes.c_int(), _P()
    _call("qc_state_info", h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p))
    return n.value, dt.value, p.value


def qc_state_set_stream(h: int, stream) -> None:
    _call("qc_state_set_stream", h, _stream(stream))


def qc_state_init_basis(h: int, index: int) -> None:
    _call("qc_state_init_basis", h, ctypes.c_uint64(int(index)))


def qc_state_init_vector(h: int, amps, src_dtype: int, on_host: bool) -> None:
    _call("qc_state_init_vector", h, _ptr(amps), src_dtype, 1 if on_host else 0)


def qc_state_init_gaussian(h: int, seed: int) -> None:
    _call("qc_state_init_gaussian", h, ctypes.c_uint64(int(seed)))


def qc_state_copy(dst: int, src: int) -> None:
    _call("qc_state_copy", dst, src)


def qc_state_download(h: int) -> np.ndarray:
    n, dt, _ = qc_state_info(h)
    out = np.empty(1 << n, dtype=np.complex64 if dt == QC_C64 else np.complex128)
    _call("qc_state_download", h, out.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# gates
# ---------------------------------------------------------------------------

def qc_apply_1q(h: int, q: int, U) -> None:
    a, p = _mat(U, 2)
    _call("qc_apply_1q", h, q, p)


def qc_apply_2q(h: int, qa: int, qb: int, U) -> None:
    a, p = _mat(U, 4)
    _call("qc_apply_2q", h, qa, qb, p)


def qc_apply_ctrl(h: int, ctrls: Sequence[int], ctrl_states: Optional[Sequence[int]], target: int, U) -> None:
    a, p = _mat(U, 2)
    c = (ctypes.c_int * max(1, len(ctrls)))(*ctrls)
    s = None if ctrl_states is None else (ctypes.c_int * max(1, len(ctrls)))(*ctrl_states)
    _call("qc_apply_ctrl", h, c, s, len(ctrls), target, p)


def qc_apply_fused_k(h: int, qubits: Sequence[int], U, prec: int = QC_PREC_NATIVE) -> None:
    k = len(qubits)
    a, p = _mat(U, 1 << k)
    q = (ctypes.c_int * k)(*qubits)
    _call("qc_apply_fused_k", h, q, k, p, prec)


# ---------------------------------------------------------------------------
# measurement, probabilities, sampling, expectations
# ---------------------------------------------------------------------------

def qc_measure(h: int, q: int, u: float):
    o, p = ctypes.c_int(), ctypes.c_double()
    _call("qc_measure", h, q, float(u), ctypes.byref(o), ctypes.byref(p))
    return o.value, p.value


def qc_collapse(h: int, q: int, outcome: int) -> float:
    p = ctypes.c_double()
    _call("qc_collapse", h, q, outcome, ctypes.byref(p))
    return p.value


def qc_inner(a: int, b: int) -> complex:
    out = np.zeros(2)
    _call("qc_inner", a, b, out.ctypes.data_as(_D))
    return complex(out[0], out[1])


def qc_collapse_norm(h: int, q: int, outcome: int, p: float) -> None:
    _call("qc_collapse_norm", h, q, outcome, float(p))


def qc_outcome_prob(h: int, q: int, outcome: int) -> float:
    p = ctypes.c_double()
    _call("qc_outcome_prob", h, q, outcome, ctypes.byref(p))
    return p.value


def qc_probs(h: int, out) -> None:
    _call("qc_probs", h, _ptr(out))


def qc_sample(h: int, u, shots: int, out) -> None:
    _call("qc_sample", h, _ptr(u), int(shots), _ptr(out))


def qc_sample_probs(h: int, p, n: int, u, shots: int, out) -> None:
    _call("qc_sample_probs", h, _ptr(p), n, _ptr(u), int(shots), _ptr(out))


def qc_reduced_state(h: int, known: Sequence[int], bits: Sequence[int], out) -> None:
    m = len(known)
    k = (ctypes.c_int * max(1, m))(*known)
    v = (ctypes.c_int * max(1, m))(*[int(x) for x in bits])
    _call("qc_reduced_state", h, k, v, m, _ptr(out))


def qc_marginal_probs(h: int, qubits: Sequence[int], out) -> None:
    q = (ctypes.c_int * len(qubits))(*qubits)
    _call("qc_marginal_probs", h, q, len(qubits), _ptr(out))


def _strings(strings: Sequence[str]):
    enc = [s.encode() for s in strings]
    arr = (ctypes.c_char_p * max(1, len(enc)))(*enc)
    return enc, arr


def qc_expect_pauli(h: int, strings: Sequence[str], coeffs=None) -> np.ndarray:
    enc, arr = _strings(strings)
    out = np.zeros(len(strings))
    c = None
    if coeffs is not None:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
    _call("qc_expect_pauli", h, arr, None if c is None else c.ctypes.data_as(_D), len(strings),
          out.ctypes.data_as(_D))
    return out


def qc_expect_pauli_noalloc(h: int, strings: Sequence[str], coeffs=None) -> np.ndarray:
    """qc_expect_pauli without device allocation (fixed library-resident scratch;
    at most 256 terms; concurrent calls race)."""
    enc, arr = _strings(strings)
    out = np.zeros(len(strings))
    c = None
    if coeffs is not None:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
    _call("qc_expect_pauli_noalloc", h, arr, None if c is None else c.ctypes.data_as(_D), len(strings),
          out.ctypes.data_as(_D))
    return out


# ---------------------------------------------------------------------------
# circuits
# ---------------------------------------------------------------------------

class Circuit:
    """A qc_circuit built from workload descriptions (kind names as in
    ``workloads.Op``); matrices of 'u1q' / 'u2q' / 'ctrl' ops go to the FP64 pool.
    Holds the ctypes arrays alive."""

    def __init__(self, n: int, ops):
        self.n = n
        pool = []
        arr = (qc_op * max(1, len(ops)))()
        for i, o in enumerate(ops):
            kind = o.kind
            adj = kind.endswith("_dag")
            if adj:
                kind = kind[:-4]
            if kind not in GATE:
                raise ValueError("gate kind %r has no C-ABI code" % kind)
            r = arr[i]
            r.kind = GATE[kind]
            r.nq = len(o.qubits)
            if r.nq > MAX_OP_QUBITS:
                raise ValueError("too many qubits in op %d" % i)
            for j, q in enumerate(o.qubits):
                r.qubits[j] = int(q)
            st = 0
            if o.ctrl_states is not None:
                for j, b in enumerate(o.ctrl_states):
                    st |= (int(b) & 1) << j
            elif kind in ("mcx", "ctrl"):
                st = (1 << (r.nq - 1)) - 1
            r.ctrl_states = st
            r.adjoint = 1 if adj else 0
            r.param = -1 if o.param_index is None else int(o.param_index)
            for j, a in enumerate(o.params[:3]):
                r.angle[j] = float(a)
            r.matrix = -1
            if o.matrix is not None:
                r.matrix = len(pool)
                pool.extend(np.ascontiguousarray(o.matrix, dtype=np.complex128).view(np.float64).ravel().tolist())
        self._ops = arr
        self._pool = np.ascontiguousarray(pool if pool else [0.0], dtype=np.float64)
        self.c = qc_circuit(n, len(ops), arr, self._pool.ctypes.data_as(_D), len(pool))


def qc_plan_info(circuit: Circuit, params=None, dtype: int = QC_C64):
    """(passes, stages, ops) the fused planner produces; host only."""
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
        p = params.ctypes.data_as(_D)
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _call("qc_plan_info", ctypes.addressof(circuit.c), p, dtype, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def _box_plan_result(local, dims, coords):
    return ([int(v) for v in local], [tuple(int(v) for v in dims[3 * d:3 * d + 3]) for d in range(5)],
            [(int(coords[1 + 2 * q]), int(coords[2 + 2 * q])) for q in range(int(coords[0]))])


def qc_tc_box_plan(n: int, tile_bits):
    """(local bits, [(first bit, bits, whole)] x 5, [(dimension, bit)] per coordinate bit)
    of the tensor-core passes' box plan for a tile; host only."""
    tb = np.ascontiguousarray(tile_bits, dtype=np.int32)
    local, dims, coords = (np.zeros(k, dtype=np.int32) for k in (12, 15, 5))
    _call("qc_tc_box_plan", int(n), tb.ctypes.data_as(_I), local.ctypes.data_as(_I), dims.ctypes.data_as(_I),
          coords.ctypes.data_as(_I))
    return _box_plan_result(local, dims, coords)


def qc_tc_block_plan(n: int, qubits):
    """The one-stage tensor-core block pass's tile and box plan for a block on `qubits`
    (as :func:`qc_tc_box_plan`); host only."""
    qs = np.ascontiguousarray(qubits, dtype=np.int32)
    local, dims, coords = (np.zeros(k, dtype=np.int32) for k in (12, 15, 5))
    _call("qc_tc_block_plan", int(n), qs.ctypes.data_as(_I), len(qs), local.ctypes.data_as(_I),
          dims.ctypes.data_as(_I), coords.ctypes.data_as(_I))
    return _box_plan_result(local, dims, coords)


def qc_tc_emulate(circuit: Circuit, state, params=None) -> np.ndarray:
    """The tensor-core passes' plan applied on the host to a copy of `state` (complex128,
    2^n values); host only."""
    out = np.ascontiguousarray(state, dtype=np.complex128).copy()
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
        p = params.ctypes.data_as(_D)
    _call("qc_tc_emulate", ctypes.addressof(circuit.c), p, out.ctypes.data_as(_D))
    return out


def qc_tile_emulate(circuit: Circuit, state, params=None, dtype: int = QC_C64) -> np.ndarray:
    """The CUDA-core tile-pass plan for a state of `dtype` applied on the host, in FP64, to
    a copy of `state` (complex128, 2^n values); host only."""
    out = np.ascontiguousarray(state, dtype=np.complex128).copy()
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
        p = params.ctypes.data_as(_D)
    _call("qc_tile_emulate", ctypes.addressof(circuit.c), p, int(dtype), out.ctypes.data_as(_D))
    return out


def qc_adjoint_emulate(circuit: Circuit, params, psi, lam, dtype: int = QC_C64) -> np.ndarray:
    """The records (Im <lambda|G|psi> per rotation, circuit order) of the fused reverse
    sweep's plan applied on the host to copies of psi and lam = H psi; host only."""
    ps = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    ls = np.ascontiguousarray(lam, dtype=np.complex128).copy()
    params = np.ascontiguousarray(params, dtype=np.float64)
    nrot = sum(1 for i in range(circuit.c.nops) if circuit._ops[i].param >= 0)
    rec = np.zeros(max(1, nrot))
    _call("qc_adjoint_emulate", ctypes.addressof(circuit.c), params.ctypes.data_as(_D), int(dtype),
          ps.ctypes.data_as(_D), ls.ctypes.data_as(_D), rec.ctypes.data_as(_D), len(rec))
    return rec[:nrot]


def qc_tc_plan_info(circuit: Circuit, params=None):
    """(passes, stage blocks, deferred factors, relabeling-only passes) of the
    tensor-core plan; host only."""
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
        p = params.ctypes.data_as(_D)
    v = [ctypes.c_int() for _ in range(4)]
    _call("qc_tc_plan_info", ctypes.addressof(circuit.c), p, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def qc_run_circuit(h: int, circuit: Circuit, params=None, mode: int = QC_RUN_PER_GATE,
                   prec: int = QC_PREC_NATIVE) -> None:
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float64)
        p = params.ctypes.data_as(_D)
    _call("qc_run_circuit", h, ctypes.byref(circuit.c), p, mode, prec)


def qc_adjoint_grad(circuit: Circuit, params, strings: Sequence[str], coeffs, dtype: int, stream=None):
    params = np.ascontiguousarray(params, dtype=np.float64)
    enc, arr = _strings(strings)
    c = np.ascontiguousarray(coeffs if coeffs is not None else np.ones(len(strings)), dtype=np.float64)
    e = ctypes.c_double()
    g = np.zeros(params.size)
    _call("qc_adjoint_grad", ctypes.byref(circuit.c), params.ctypes.data_as(_D), params.size, arr,
          c.ctypes.data_as(_D), len(strings), dtype, _stream(stream), ctypes.byref(e), g.ctypes.data_as(_D))
    return e.value, g


def qc_adjoint_grad_dev(circuit: "Circuit", dev_params, hamiltonian: "Hamiltonian", dtype: int, dev_energy,
                        dev_grad, stream=None) -> None:
    """Device-pointer adjoint gradient: dev_params (device FP64, contiguous), outputs
    dev_energy (one FP64) and dev_grad (device FP64, len = params) on the stream."""
    n = int(dev_params.numel()) if hasattr(dev_params, "numel") else 0
    _call("qc_adjoint_grad_dev", ctypes.byref(circuit.c), _ptr(dev_params), n, ctypes.byref(hamiltonian.h), dtype,
          _stream(stream), _ptr(dev_energy), _ptr(dev_grad))


def qc_run_ansatz_batch(ns, layers: int, param_offsets, dev_params, nparams: int, out, stream=None) -> None:
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    offs = np.ascontiguousarray(param_offsets, dtype=np.int64)
    b = qc_ansatz_batch(len(ns), layers, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(dev_params), int(nparams))
    _call("qc_run_ansatz_batch", ctypes.byref(b), _stream(stream), _ptr(out))


class Hamiltonian:
    """A Pauli sum as qc_pauli_term records (xmask, zmask, coeff) on index bits; holds
    the ctypes array alive.  ``from_strings`` converts strings of I/X/Y/Z (character j
    acts on qubit j, i.e. index bit n-1-j) to masks."""

    def __init__(self, terms):
        terms = list(terms)
        self.arr = (qc_pauli_term * max(1, len(terms)))()
        for i, (x, z, c) in enumerate(terms):
            self.arr[i] = qc_pauli_term(int(x), int(z), float(c))
        self.h = qc_hamiltonian(len(terms), 0, self.arr)
        self.terms = terms

    @classmethod
    def from_strings(cls, strings, coeffs=None):
        out = []
        for t, s in enumerate(strings):
            n = len(s)
            x = z = 0
            for j, ch in enumerate(s.upper()):
                b = 1 << (n - 1 - j)
                if ch in "XY":
                    x |= b
                if ch in "ZY":
                    z |= b
                if ch not in "IXYZ":
                    raise ValueError("invalid Pauli character %r" % ch)
            out.append((x, z, 1.0 if coeffs is None else float(coeffs[t])))
        return cls(out)


def qc_run_batch(circuits, observables=None, dev_params=None, param_offsets=None, dev_states=None, out=None,
                 stream=None, shared_observable: bool = False, nparams: Optional[int] = None) -> None:
    """One launch over independent circuits (list of :class:`Circuit`).  observables:
    one :class:`Hamiltonian` per circuit (or one with shared_observable); out: device
    FP64 tensor of len(circuits); dev_params: device FP64 tensor; dev_states: list of
    device complex64 tensors (or None entries) receiving the final states."""
    cnt = len(circuits)
    carr = (qc_circuit * max(1, cnt))(*[c.c for c in circuits])
    offs = None
    if param_offsets is not None:
        offs = np.ascontiguousarray(param_offsets, dtype=np.int64)
    harr = None
    if observables is not None:
        hs = observables if isinstance(observables, (list, tuple)) else [observables]
        harr = (qc_hamiltonian * max(1, len(hs)))(*[h.h for h in hs])
    sarr = None
    if dev_states is not None:
        sarr = (ctypes.c_void_p * max(1, cnt))(*[(_ptr(t) if t is not None else None) for t in dev_states])
    if nparams is None:
        nparams = int(dev_params.numel()) if dev_params is not None and hasattr(dev_params, "numel") else 0
    b = qc_batch(cnt, 1 if shared_observable else 0, carr,
                 None if offs is None else offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                 _ptr(dev_params), int(nparams), harr, sarr)
    _call("qc_run_batch", ctypes.byref(b), _stream(stream), _ptr(out))


def qc_last_batch_path() -> int:
    """0 general batch kernel, 1 ansatz kernel (most recent qc_run_batch of this thread)."""
    return int(lib().qc_last_batch_path())


def qc_batch_fusion_width() -> int:
    return int(lib().qc_batch_fusion_width())
