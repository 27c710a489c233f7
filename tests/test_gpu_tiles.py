"""Every Ax tile the autotuner can choose gives the oracle's result, and the
autotuner's choice is applied and cached."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TILES32 = [("global-load", 2, 1), ("bulk-copy", 1, 1), ("bulk-copy", 2, 1), ("bulk-copy", 3, 1),
           ("bulk-copy", 1, 2), ("bulk-copy", 2, 2)]


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((3, 2, 3), 5), ((3, 3, 1), 9), ((3, 1, 2), 3)])
@pytest.mark.parametrize("h2", [0.0, 1.5])
def test_every_tile_matches_oracle(nel, N, h2):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    u = si.uniform(o.shape, 70)
    ref32 = o.ax(u.astype(np.float32).astype(np.float64), 1.0, h2)
    ref64 = o.ax(u, 1.0, h2)
    u32 = torch.from_numpy(u).to(DEV, torch.float32).view(-1)
    u64 = torch.from_numpy(u).to(DEV).view(-1)
    outs = []
    for kind, stages, elems in TILES32:
        for f64_stages in (1, 2):
            sem.sem_set_tuning(h, kind, stages, elems, f64_stages)
            w32 = torch.empty_like(u32)
            sem.sem_ax(h, u32, w32, 1.0, h2)
            w64 = torch.empty_like(u64)
            sem.sem_ax(h, u64, w64, 1.0, h2)
            sem.sem_sync(h)
            assert rel_inf(w32.double().cpu().numpy().reshape(o.shape), ref32) < 2e-5
            assert rel_inf(w64.cpu().numpy().reshape(o.shape), ref64) < 1e-12
            if kind == "bulk-copy":
                outs.append(w32.cpu())
    # the bulk-copy tiles only reorder work across CTAs: results are bitwise equal
    for w in outs[1:]:
        assert torch.equal(w, outs[0])


def test_autotune_choice_is_applied_and_cached():
    h = sem.sem_setup((6, 4, 4), 7, length=(TWO_PI,) * 3, deform=0.1)
    t = sem.sem_autotune(h)
    assert t["ax32_stages"] in (1, 2, 3) and t["ax32_elems_per_cta"] in (1, 2)
    assert t["f64_stages"] in (1, 2) and t["ax32_ms"] > 0 and t["ax64_ms"] > 0
    h2 = sem.sem_setup((6, 4, 4), 7, length=(TWO_PI,) * 3, deform=0.1)
    t2 = sem.sem_autotune(h2)
    assert t2["from_cache"] and {k: t2[k] for k in ("ax32_kernel", "ax32_stages",
                                                     "ax32_elems_per_cta", "f64_stages")} == \
        {k: t[k] for k in ("ax32_kernel", "ax32_stages", "ax32_elems_per_cta", "f64_stages")}
