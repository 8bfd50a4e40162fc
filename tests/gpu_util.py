"""Helpers for the GPU parity tests (call the CUDA path through the C ABI)."""
import numpy as np
import pytest

TOL = {"c128": 1e-12, "c64": 1e-5}


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.complex128)
    want = np.asarray(want, dtype=np.complex128)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))


def gpu_state(psi, dtype):
    import paper_2503_03016_gb300 as P
    n = int(psi.size).bit_length() - 1
    st = P.State(n, dtype)
    st.init_vector(psi.astype(np.complex64) if dtype == "c64" else psi)
    return st


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def record(name: str, **vals) -> None:
    """Appends the achieved error of a parity check to the JSON-lines file named by
    QC_PARITY_LOG (if set), so that the errors behind each tolerance can be reported."""
    import json
    import os
    path = os.environ.get("QC_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps(dict(test=name, **{k: (float(v) if isinstance(v, (np.floating, float)) else v)
                                              for k, v in vals.items()})) + "\n")
