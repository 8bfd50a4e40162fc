"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares; the oracle is not reachable from the product package."""
import glob
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s+(qc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2503_03016_gb300 import build as B
    lib = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (qc_\w+)", out))
    decl = declared_functions()
    assert len(decl) >= 25
    missing = decl - exported
    assert not missing, missing


def test_library_loads_on_cpu():
    import paper_2503_03016_gb300 as P
    L = P.lib()
    assert L.qc_abi_version() == 2
    assert L.qc_last_error() == b""


def test_invalid_arguments_rejected_before_any_launch():
    import ctypes
    import paper_2503_03016_gb300 as P
    h = ctypes.c_void_p()
    assert P.lib().qc_state_alloc(0, 0, None, ctypes.byref(h)) == 1
    assert b"invalid" in P.lib().qc_last_error()
    assert P.lib().qc_state_free(None) == 0


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2503_03016_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(path).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
            assert "qc_oracle" not in src and "libqcoracle" not in src, path


def test_device_status_word_mapping():
    """The status the tensor-core entry points return for their kernels' status word
    (host only, no kernel: a timed-out wait is never provoked on a GPU)."""
    import ctypes

    import paper_2503_03016_gb300 as P
    L = P.lib()
    assert L.qc_status_of_device_word(0) == 0
    assert L.qc_status_of_device_word(1) == 6  # QC_ERR_TIMEOUT
    msg = L.qc_last_error().decode()
    assert "undefined" in msg and "bounded wait" in msg
    assert L.qc_status_of_device_word(7) == 3  # QC_ERR_CUDA
    assert "7" in L.qc_last_error().decode()
