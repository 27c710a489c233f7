"""The C-ABI library loads and exports every symbol include/sem.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_symbols():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = re.sub(r"//[^\n]*", "", text)
            for m in re.finditer(r"\b(sem_[a-z0-9_]+)\s*\(", text):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2107_01243_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2107_01243_gb300 import build
        build.build()
    return _lib.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("sem_setup", "sem_ax", "sem_dssum", "sem_cg_solve", "sem_helmholtz_grad",
                     "sem_destroy", "sem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert declared_symbols() <= exported


def test_binding_covers_every_declared_symbol():
    from paper_2107_01243_gb300 import _lib
    assert declared_symbols() == set(_lib.SIGNATURES)


def test_binding_loads_without_gpu(lib_path):
    from paper_2107_01243_gb300 import _lib
    lib = _lib.load()
    assert lib.sem_last_error() == b""


def test_user_coordinates_of_the_wrong_size_are_refused_before_the_call(lib_path):
    """sem_setup reads exactly 3 n_L host coordinates from xyz_gll; the binding
    refuses any other size before the library could read past the array."""
    import numpy as np
    import paper_2107_01243_gb300 as sem
    with pytest.raises(sem.SemError, match="3 x n_L = 192"):
        sem.sem_setup((2, 2, 2), 1, xyz=np.zeros(10))
