"""sem_dot_noalloc, the entry point for callers that cannot allocate device
memory at the call site (stream capture, fixed memory budgets): called through
the C ABI twice in a row, it must give the oracle's unique-dof inner product
sum_L a b / mult and the same value as sem_dot.
Collected last on purpose: it uses the library's static scratch array."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh, operator
from tests.helpers import TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL64 = 1e-12


def _vec(shape, seed):
    return torch.from_numpy(si.uniform(shape, seed)).to(DEV).view(-1)


POINTS_PER_BLOCK = 4096      # local points summed by one block of the kernel


# (3, 3, 1) at N = 7 and (513, 1, 1) at N = 1 end just above a multiple of the
# block's 4096 points, so the last block is mostly empty
@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((8, 8, 4), 9), ((3, 3, 1), 7),
                                   ((513, 1, 1), 1)])
def test_noalloc_dot_matches_sem_dot_twice(nel, N):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    shape = h.shape
    if nel in ((3, 3, 1), (513, 1, 1)):
        tail = h.n_local % POINTS_PER_BLOCK
        assert h.n_local > POINTS_PER_BLOCK and 0 < tail <= 512, (h.n_local, tail)
    mult = mesh.multiplicity(mesh.global_ids(*nel, N))
    ref = torch.empty(1, dtype=torch.float64, device=DEV)
    got = torch.empty(1, dtype=torch.float64, device=DEV)
    for call, (sa, sb) in enumerate(((60, 61), (62, 63))):
        an, bn = si.uniform(shape, sa), si.uniform(shape, sb)
        a, b = _vec(shape, sa), _vec(shape, sb)
        sem.sem_dot(h, a, b, ref)
        sem.sem_dot_noalloc(h, a, b, got)
        torch.cuda.synchronize()
        want = operator.weighted_dot(an, bn, mult)
        scale = float(np.sum(np.abs(an * bn) / mult))
        assert abs(float(got) - want) <= TOL64 * scale, (call, float(got), want)
        assert abs(float(got) - float(ref)) <= TOL64 * scale, (call, float(got), float(ref))
    # the same inputs again give the same bits (the static scratch is reused)
    first = float(got)
    sem.sem_dot_noalloc(h, a, b, got)
    assert float(got) == first


def test_noalloc_dot_refuses_more_points_than_its_array_holds():
    """A mesh one block beyond SEM_NOALLOC_MAX_POINTS (N = 1, 8 points per
    element): the call returns SEM_ERR_ARG naming the limit and launches
    nothing; sem_dot still works on the same vectors."""
    nel = (2049, 64, 64)                      # 67,141,632 local points
    h = sem.sem_setup(nel, 1, length=(1.0, 1.0, 1.0), precision=sem.SEM_PREC_F64)
    assert sem.SEM_NOALLOC_MAX_POINTS < h.n_local <= sem.SEM_NOALLOC_MAX_POINTS + 65536
    a = torch.ones(h.n_local, dtype=torch.float64, device=DEV)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=DEV)
    with pytest.raises(sem.SemError) as exc:
        sem.sem_dot_noalloc(h, a, a, out)
    assert exc.value.status == sem.SEM_ERR_ARG
    assert str(sem.SEM_NOALLOC_MAX_POINTS) in str(exc.value)
    torch.cuda.synchronize()
    assert float(out) == -1.0
    sem.sem_dot(h, a, a, out)
    # <1, 1> over unique points = the number of global points
    assert float(out) == pytest.approx((2049 + 1) * (64 + 1) * (64 + 1), rel=1e-12)
    del a
    sem.sem_destroy(h)
