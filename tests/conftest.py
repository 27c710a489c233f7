import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# tests/mutation_sweep.py: with SEM_ORACLE_MUTATION = {"module", "old", "new"}
# (JSON) the named oracle module is imported with its first occurrence of
# "old" replaced by "new", so that the pins can be checked against a planted
# mistake without touching the file on disk (and without bytecode caching)
_MUTATION = os.environ.get("SEM_ORACLE_MUTATION")
if _MUTATION:
    import importlib.abc
    import importlib.util
    import json

    _mut = json.loads(_MUTATION)

    class _MutatedSource(importlib.abc.SourceLoader):
        def __init__(self, path):
            self.path = path

        def get_filename(self, fullname):
            return self.path

        def get_data(self, path):
            with open(path, encoding="utf-8") as f:
                src = f.read()
            if _mut["old"] not in src:
                raise RuntimeError(f"mutation text not found in {path}")
            return src.replace(_mut["old"], _mut["new"], 1).encode("utf-8")

    class _MutationFinder(importlib.abc.MetaPathFinder):
        def find_spec(self, fullname, path, target=None):
            if fullname != _mut["module"]:
                return None
            fn = os.path.join(ROOT, *fullname.split(".")) + ".py"
            return importlib.util.spec_from_file_location(fullname, fn,
                                                          loader=_MutatedSource(fn))

    sys.meta_path.insert(0, _MutationFinder())


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")
