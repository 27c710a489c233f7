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


def _header_text():
    text = open(os.path.join(HEADER_DIR, "sem.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def test_binding_constants_equal_the_header_enums():
    from paper_2107_01243_gb300 import _lib
    names = re.findall(r"\b(SEM_[A-Z0-9_]+)\s*=\s*(\d+)", _header_text())
    assert len(names) > 40
    for name, value in names:
        assert getattr(_lib, name) == int(value), name


def test_binding_structs_match_the_c_layout(tmp_path):
    """Offsets and sizes of every struct of the boundary, as gcc lays them
    out from include/sem.h, equal those of the ctypes mirrors."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2107_01243_gb300 import _lib
    structs = {"sem_mesh_desc": _lib.MeshDesc, "sem_solve_opts": _lib.SolveOpts,
               "sem_solve_info": _lib.SolveInfo, "sem_tuning": _lib.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sem.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = 0
    for line in out.splitlines():
        cname, field, value = line.split()
        cls = structs[cname]
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (cname, field, got, value)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_binding_signatures_have_the_header_arity():
    """Every function the binding declares takes as many arguments as its
    prototype in include/sem.h, with the same pointer / integer / floating
    kind at each position."""
    from paper_2107_01243_gb300 import _lib
    protos = {}
    for m in re.finditer(r"\b(?:sem_status|void|const char\*)\s+(sem_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                         _header_text()):
        params = [p.strip() for p in m.group(2).split(",")]
        protos[m.group(1)] = [] if params == ["void"] else params
    assert set(_lib.SIGNATURES) == set(protos)          # the binding covers the whole ABI

    def kind_c(p):
        if "*" in p:
            return "ptr"
        return "float" if p.split()[0] in ("double", "float") else "int"

    def kind_ct(t):
        if t in (ctypes.c_double, ctypes.c_float):
            return "float"
        if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32):
            return "int"
        return "ptr"

    for name, (_, args) in _lib.SIGNATURES.items():
        assert len(args) == len(protos[name]), name
        assert [kind_ct(t) for t in args] == [kind_c(p) for p in protos[name]], name


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built library the first call raises."""
    from paper_2107_01243_gb300 import _lib
    import paper_2107_01243_gb300 as sem
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libsem_gb300.so"))
    with pytest.raises(sem.SemError, match="CUDA library not built"):
        sem.sem_setup((1, 1, 1), 2)


def test_plain_c_client_links_and_calls_host_entry_points(tmp_path, lib_path):
    """The library is usable from C alone (no Python, no torch): a C program
    compiled against include/sem.h links libsem_gb300.so, reads the solver
    defaults and gets SEM_ERR_ARG with a message for a null mesh (both host
    paths: no GPU needed)."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "client.c"
    src.write_text(r'''
#include <stdio.h>
#include "sem.h"
int main(void) {
  sem_solve_opts o;
  sem_solve_opts_default(&o);
  printf("%g %d %d %d %d %g %d\n", o.tol, o.maxit, o.check_every, o.use_graph, o.x0_is_zero,
         o.inner_tol, o.max_outer);
  sem_handle* h = (sem_handle*)1;
  sem_status st = sem_setup(NULL, 7, SEM_PREC_F64, NULL, &h);
  printf("%d %d [%s]\n", (int)st, h == (sem_handle*)1, sem_last_error());
  return 0;
}
''')
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c11", "-I", HEADER_DIR, str(src), "-L", libdir, "-lsem_gb300",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    tol, maxit, every, graph, x0z, itol, mouter = out[0].split()
    assert (float(tol), int(maxit), int(every), int(graph), int(x0z)) == (1e-8, 20000, 16, 1, 1)
    assert (float(itol), int(mouter)) == (1e-4, 30)
    st, untouched, msg = out[1].split(" ", 2)
    assert int(st) == 1 and "null mesh" in msg          # SEM_ERR_ARG, out not written


def test_setup_arguments_are_checked_before_any_cuda_call(lib_path):
    """sem_setup validates its arguments before it touches the device, so the
    error codes of the boundary are checked here without a GPU; a valid call
    on a machine without one fails loudly (no CPU fallback)."""
    import torch
    import paper_2107_01243_gb300 as sem
    bad = [dict(nel=(2, 2, 2), N=11), dict(nel=(2, 2, 2), N=0), dict(nel=(0, 1, 1), N=3),
           dict(nel=(1, 1, 1), N=3, length=(1.0, 0.0, 1.0)),
           dict(nel=(1, 1, 1), N=3, precision=0), dict(nel=(1000, 1000, 1000), N=7)]
    for kw in bad:
        nel, N = kw.pop("nel"), kw.pop("N")
        with pytest.raises(sem.SemError) as e:
            sem.sem_setup(nel, N, stream=0, **kw)       # stream 0: no torch.cuda call
        assert e.value.status == 1, (nel, N, kw, str(e.value))
    if not torch.cuda.is_available():
        with pytest.raises(sem.SemError) as e:
            sem.sem_setup((1, 1, 1), 3, stream=0)
        assert e.value.status == 2                   # SEM_ERR_CUDA: no device, no fallback


NULL_PROBE = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_2107_01243_gb300 import _lib
lib = _lib.load()
for name, (res, args) in _lib.SIGNATURES.items():
    if name == "sem_last_error":
        continue
    vals = [1.0 if t in (ctypes.c_double, ctypes.c_float) else
            1 if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32) else None for t in args]
    print(name, getattr(lib, name)(*vals), flush=True)
"""


def test_every_entry_point_rejects_null_pointers(lib_path):
    """Every call, given null pointers (and unit scalars), returns an error
    status without touching the device or crashing; the destroy calls accept
    NULL as a no-op."""
    import sys
    out = subprocess.run([sys.executable, "-c", NULL_PROBE, ROOT], capture_output=True,
                         text=True, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    seen = {}
    for line in out.stdout.splitlines():
        name, st = line.split()
        seen[name] = st
    from paper_2107_01243_gb300 import _lib
    assert set(seen) == set(_lib.SIGNATURES) - {"sem_last_error"}
    for name, st in seen.items():
        if name.endswith("_destroy"):
            assert st == "0", name
        elif name == "sem_solve_opts_default":
            assert st == "None"
        else:
            assert st == "1", (name, st)                 # SEM_ERR_ARG
