"""sem_dot_noalloc, the entry point for callers that cannot allocate device
memory at the call site (stream capture, fixed memory budgets): called through
the C ABI twice in a row, it must give the same inner product as sem_dot.
Collected last on purpose: it uses the library's static scratch array."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL64 = 1e-12


def _vec(shape, seed):
    return torch.from_numpy(si.uniform(shape, seed)).to(DEV).view(-1)


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((8, 8, 4), 9)])
def test_noalloc_dot_matches_sem_dot_twice(nel, N):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    shape = h.shape
    ref = torch.empty(1, dtype=torch.float64, device=DEV)
    got = torch.empty(1, dtype=torch.float64, device=DEV)
    for call, (sa, sb) in enumerate(((60, 61), (62, 63))):
        a, b = _vec(shape, sa), _vec(shape, sb)
        sem.sem_dot(h, a, b, ref)
        sem.sem_dot_noalloc(h, a, b, got)
        torch.cuda.synchronize()
        scale = float((a * b).abs().sum())
        assert abs(float(got) - float(ref)) <= TOL64 * scale, (call, float(got), float(ref))
    # the same inputs again give the same bits (the static scratch is reused)
    first = float(got)
    sem.sem_dot_noalloc(h, a, b, got)
    assert float(got) == first
