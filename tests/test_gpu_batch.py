"""Batched solves through the C ABI: problems of different element counts,
orders and Helmholtz coefficients solved together, each judged by the
oracle's FP64 residual and against its own single solve; the inner solves
run on global vectors (the default) or on L-vectors."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# on L-vectors, with orders N = 1, 3 the batch runs the element kernel and the
# gather-scatter kernel; with N in {5, 7, 9} only, the fused operator (segments
# of four elements, split gather-scatter): partial segments, single-element
# rows and meshes one element thick are included.  On global vectors every
# order runs the gathering element kernel.
PROBLEMS = [((3, 2, 2), 5, 0.7), ((2, 2, 2), 7, 3.1), ((4, 3, 2), 3, 0.1), ((1, 1, 2), 9, 9.5),
            ((3, 3, 3), 7, 1.7), ((3, 3, 2), 1, 2.0)]
PROBLEMS_FUSED = [((3, 2, 2), 5, 0.7), ((2, 2, 2), 7, 3.1), ((1, 1, 2), 9, 9.5),
                  ((3, 3, 3), 7, 1.7), ((5, 1, 3), 5, 0.4), ((7, 3, 1), 7, 2.2),
                  ((6, 5, 4), 9, 0.9)]


def _setup(problems):
    hs, oracles, bs = [], [], []
    for q, (nel, N, lam) in enumerate(problems):
        h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
        o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
        f = si.eval_fourier(si.fourier_modes(2000 + q), o.x, o.y, o.z)
        b_ref = o.rhs(f)
        hs.append(h)
        oracles.append(o)
        bs.append((b_ref, torch.from_numpy(b_ref).to(DEV).view(-1)))
    return hs, oracles, bs


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("problems", [PROBLEMS, PROBLEMS_FUSED], ids=["unfused", "fused"])
@pytest.mark.parametrize("inner", [sem.SEM_INNER_AUTO, sem.SEM_INNER_LOCAL],
                         ids=["global-vectors", "local-vectors"])
def test_batch_matches_oracle_and_single_solves(use_graph, problems, inner):
    hs, oracles, bs = _setup(problems)
    for h in hs:
        sem.sem_set_inner_vectors(h, inner)
    batch = sem.sem_batch_create(hs)
    xs = [torch.empty_like(b) for _, b in bs]
    lams = [lam for _, _, lam in problems]
    infos = sem.sem_batch_solve(batch, [b for _, b in bs], xs, [1.0] * len(hs), lams, tol=1e-8,
                                check_every=5, use_graph=use_graph)
    for q, (h, o, (b_ref, b), x, info) in enumerate(zip(hs, oracles, bs, xs, infos)):
        assert info["status"] == "SEM_OK", (q, info)
        xg = x.cpu().numpy().reshape(o.shape)
        res = o.residual(xg, b_ref, h1=1.0, h2=lams[q])
        assert res <= 1.05e-8, (q, res)
        assert abs(res - info["rel_res"]) < 1e-12
        single = torch.empty_like(b)
        sem.sem_cg_solve(h, b, single, h1=1.0, h2=lams[q], tol=1e-8,
                         precision=sem.SEM_SOLVE_MIXED)
        # both solve to 1e-8; the solutions agree to the conditioning of the problem
        assert rel_inf(xg, single.cpu().numpy().reshape(o.shape)) < 1e-5


def test_batch_rejects_even_order():
    h = sem.sem_setup((2, 2, 2), 4)
    with pytest.raises(sem.SemError):
        sem.sem_batch_create([h])
