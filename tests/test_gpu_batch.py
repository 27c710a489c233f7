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


@pytest.mark.parametrize("concurrent", [True, False], ids=["branches", "serial"])
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("problems", [PROBLEMS, PROBLEMS_FUSED], ids=["unfused", "fused"])
@pytest.mark.parametrize("inner", [sem.SEM_INNER_AUTO, sem.SEM_INNER_LOCAL],
                         ids=["global-vectors", "local-vectors"])
def test_batch_matches_oracle_and_single_solves(use_graph, problems, inner, concurrent):
    """The order classes' element launches one after another (the default)
    or as concurrent branches (parallel paths of the iteration graph)."""
    hs, oracles, bs = _setup(problems)
    for h in hs:
        sem.sem_set_inner_vectors(h, inner)
    batch = sem.sem_batch_create(hs)
    sem.sem_batch_set_concurrency(batch, concurrent)
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


# Problems large enough that every persistent grid of the batched inner solve
# on global vectors walks its work more than once and crosses from one problem
# to the next inside a CTA: per order class more elements than 2 x 8 CTAs per
# SM x the device's SMs, and more global-vector work items (16,384 values each)
# than the 8 blocks per SM of the vector kernels.
PROBLEMS_LARGE = [((16, 16, 16), 9, 0.7), ((16, 16, 15), 9, 3.1), ((14, 14, 14), 7, 1.7),
                  ((16, 16, 16), 9, 9.5), ((12, 12, 12), 5, 0.4), ((16, 15, 16), 9, 2.2),
                  ((16, 16, 16), 7, 5.0), ((15, 16, 16), 9, 0.9), ((16, 16, 16), 9, 4.4),
                  ((13, 13, 12), 5, 7.3), ((16, 16, 14), 9, 1.1), ((16, 14, 16), 9, 6.6)]
GCHUNK = 16384


def test_batch_large_grids_walk_across_problems():
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    per_order = {}
    items = 0
    for nel, N, _ in PROBLEMS_LARGE:
        E = nel[0] * nel[1] * nel[2]
        per_order[N] = per_order.get(N, 0) + E
        ng = (N * nel[0] + 1) * (N * nel[1] + 1) * (N * nel[2] + 1)
        ngp = (ng + 3) // 4 * 4
        items += (ngp + GCHUNK - 1) // GCHUNK
    assert all(E > 2 * 8 * nsm for E in per_order.values()), per_order
    assert items > 8 * nsm, items

    hs, bs, refs, oracles = [], [], [], []
    for q, (nel, N, lam) in enumerate(PROBLEMS_LARGE):
        h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
        o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
        b_ref = o.rhs(si.eval_fourier(si.fourier_modes(3000 + q), o.x, o.y, o.z))
        del o.x, o.y, o.z, o.detJ                  # keep what the residual needs
        hs.append(h)
        oracles.append(o)
        refs.append(b_ref)
        bs.append(torch.from_numpy(b_ref).to(DEV).view(-1))
    lams = [lam for _, _, lam in PROBLEMS_LARGE]
    batch = sem.sem_batch_create(hs)
    runs = {}
    for use_graph, concurrent in ((True, False), (False, False), (True, True)):
        sem.sem_batch_set_concurrency(batch, concurrent)
        xs = [torch.empty_like(b) for b in bs]
        infos = sem.sem_batch_solve(batch, bs, xs, [1.0] * len(hs), lams, tol=1e-8,
                                    check_every=8, use_graph=use_graph)
        assert all(i["status"] == "SEM_OK" for i in infos), infos
        runs[(use_graph, concurrent)] = (xs, infos)
    sem.sem_batch_destroy(batch)
    for q, ((nel, N, lam), h, b, b_ref, o) in enumerate(zip(PROBLEMS_LARGE, hs, bs, refs,
                                                              oracles)):
        single = torch.empty_like(b)
        sem.sem_cg_solve(h, b, single, h1=1.0, h2=lam, tol=1e-8, precision=sem.SEM_SOLVE_MIXED)
        xsingle = single.cpu().numpy().reshape(o.shape)
        for use_graph, (xs, infos) in runs.items():
            xg = xs[q].cpu().numpy().reshape(o.shape)
            res = o.residual(xg, b_ref, h1=1.0, h2=lam)
            assert res <= 1.05e-8, (q, use_graph, res)
            assert abs(res - infos[q]["rel_res"]) < 1e-11, (q, res, infos[q])
            assert rel_inf(xg, xsingle) < 1e-5, q
