"""The mutation sweep (tests/mutation_sweep.py) stays runnable: every planted
fragment still occurs in its oracle module, and the import hook really plants
the mistake (one mutation run against the pin that must catch it)."""
import json
import os
import subprocess
import sys

from tests import mutation_sweep as ms


def test_every_fragment_occurs_in_its_module():
    for module, name, old, new in ms.MUTATIONS:
        path = os.path.join(ms.ROOT, *module.split(".")) + ".py"
        with open(path, encoding="utf-8") as f:
            assert old in f.read(), name
        assert old != new, name


def test_planted_mistake_fails_its_pin_and_the_file_is_untouched():
    module, name, old, new = next(m for m in ms.MUTATIONS if m[1] == "deform_y")
    path = os.path.join(ms.ROOT, "oracle", "mesh.py")
    with open(path, encoding="utf-8") as f:
        before = f.read()
    cmd = [sys.executable, "-m", "pytest", "tests/test_oracle_operator.py", "-q", "-x",
           "-k", "deformation_structure"]
    base = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    base.pop("SEM_ORACLE_MUTATION", None)
    ok = subprocess.run(cmd, cwd=ms.ROOT, env=base, capture_output=True, text=True, timeout=300)
    assert ok.returncode == 0, ok.stdout[-1000:]
    env = dict(base, SEM_ORACLE_MUTATION=json.dumps({"module": module, "old": old, "new": new}))
    bad = subprocess.run(cmd, cwd=ms.ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert bad.returncode == 1, bad.stdout[-1000:]
    with open(path, encoding="utf-8") as f:
        assert f.read() == before
