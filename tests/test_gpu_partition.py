"""Element partition across ranks (paper §3.2, Algorithm 1) on the GPU.

The device side of the partition (sem_gather, sem_scatter_add,
sem_set_multiplicity, sem_jacobi_diag / sem_jacobi_invert, sem_cg_update,
sem_cg_direction) against plain tensor arithmetic, then the partitioned
operator and PCG of the package on 2 and 4 ranks: separate processes that
share this GPU (their kernels never wait on one another; the interface
buffers go through host memory over gloo), each on its sub-box handle,
against the single-domain oracle."""
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import paper_2107_01243_gb300 as sem
from paper_2107_01243_gb300 import partition as part
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gather_scatter_and_cg_kernels():
    h = sem.sem_setup((3, 2, 2), 5, length=(TWO_PI,) * 3, deform=0.1)
    n = h.n_local
    g = torch.Generator().manual_seed(5)
    v = torch.rand(n, dtype=torch.float64, generator=g).to(DEV)
    idx = torch.randperm(n, generator=g)[:500].to(DEV)
    buf = torch.empty(500, dtype=torch.float64, device=DEV)
    sem.sem_gather(h, v, idx, buf)
    assert torch.equal(buf, v[idx])
    src = torch.rand(700, dtype=torch.float64, generator=g).to(DEV)
    pos = torch.randint(0, 700, (500,), generator=g).to(DEV)
    ref = v.clone()
    ref[idx] += src[pos]
    sem.sem_scatter_add(h, v, idx, pos, src)
    sem.sem_sync(h)
    assert torch.equal(v, ref)
    # an index outside the vector is skipped and reported by sem_sync
    bad = idx.clone()
    bad[7] = n + 3
    before = v.clone()
    sem.sem_scatter_add(h, v, bad, pos, src)
    with pytest.raises(sem.SemError) as exc:
        sem.sem_sync(h)
    assert exc.value.status == sem.SEM_ERR_ARG
    expect = before.clone()
    keep = torch.arange(500, device=DEV) != 7
    expect[idx[keep]] += src[pos[keep]]
    assert torch.equal(v, expect)
    sem.sem_sync(h)                           # the record was cleared
    # Jacobi diagonal and inverse against the solver's own (FP64 PCG)
    b = torch.rand(n, dtype=torch.float64, generator=g).to(DEV)
    sem.sem_dssum(h, b)
    x = torch.empty_like(b)
    sem.sem_cg_solve(h, b, x, 1.0, 0.7, tol=1e-6)
    dinv_ref = torch.empty_like(b)
    sem.sem_get_field(h, sem.SEM_FIELD_DINV, dinv_ref)
    d = torch.empty_like(b)
    dinv = torch.empty_like(b)
    sem.sem_jacobi_diag(h, d, 1.0, 0.7)
    sem.sem_jacobi_invert(h, d, dinv)
    assert rel_inf(dinv.cpu().numpy(), dinv_ref.cpu().numpy()) < 1e-14
    # CG vector step and direction against tensor arithmetic, unique-dof dots
    mult = torch.empty_like(b)
    sem.sem_get_field(h, sem.SEM_FIELD_MULT, mult)
    p, w, xx, r, z = (torch.rand(n, dtype=torch.float64, generator=g).to(DEV) for _ in range(5))
    xr, rr_ = xx + 0.3 * p, r - 0.3 * w
    zr = dinv * rr_
    dots = torch.empty(2, dtype=torch.float64, device=DEV)
    sem.sem_cg_update(h, 0.3, p, w, xx, r, dinv, z, dots)
    assert torch.allclose(xx, xr, rtol=0, atol=1e-15) and torch.allclose(r, rr_, rtol=0, atol=1e-15)
    # the kernel forms r - alpha w with one rounding (FMA), the tensor
    # arithmetic above with two; z is dinv times the r the kernel returned
    assert torch.equal(z, dinv * r)
    for got, want in zip(dots.cpu().tolist(), [(rr_ * zr / mult).sum().item(),
                                               (rr_ * rr_ / mult).sum().item()]):
        assert abs(got - want) <= 1e-13 * abs(want)
    sem.sem_cg_direction(h, 0.25, z, p)
    # multiplicities replaced: the dot follows them
    m2 = mult * 2.0
    sem.sem_set_multiplicity(h, m2)
    out = torch.empty(1, dtype=torch.float64, device=DEV)
    sem.sem_dot(h, r, r, out)
    assert abs(float(out) - (r * r / m2).sum().item()) <= 1e-13 * (r * r / m2).sum().item()


def _global_elements(sub):
    nx, ny, _ = sub.nel_global
    e = np.arange(np.prod(sub.count))
    ex = e % sub.count[0] + sub.offset[0]
    ey = (e // sub.count[0]) % sub.count[1] + sub.offset[1]
    ez = e // (sub.count[0] * sub.count[1]) + sub.offset[2]
    return ex + nx * (ey + ny * ez)


def _rank_main(rank, world, port, nel, N, out_dir):
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        sub, h, be, op = part.setup_rank(nel, N, world, rank, length=(TWO_PI,) * 3,
                                         deform=0.1, host_staged=True)
        ge = _global_elements(sub)
        u = si.uniform((int(np.prod(nel)),) + (N + 1,) * 3, 92)[ge]
        w = be.zeros()
        op.apply(torch.from_numpy(u.ravel().copy()).to(DEV), w, 1.0, 0.3)
        xs = [torch.empty(h.n_local, dtype=torch.float64, device=DEV) for _ in range(3)]
        for t, f in zip(xs, (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z)):
            sem.sem_get_field(h, f, t)
        X, Y, Z = (t.cpu().numpy() for t in xs)
        f = torch.from_numpy(si.eval_fourier(si.fourier_modes(93), X, Y, Z)).to(DEV)
        b = be.zeros()
        sem.sem_rhs(h, f, b)
        op.exchange(b)
        x = be.zeros()
        its, rel, status = part.partitioned_pcg(op, b, x, 1.0, 0.3, tol=1e-10)
        sem.sem_sync(h)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), w=w.cpu().numpy(),
                 x=x.cpu().numpy(), b=b.cpu().numpy(), ge=ge)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"iters": its, "rel": rel, "status": status}, fh)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nel,world,N", [((6, 4, 3), 2, 7), ((5, 4, 3), 4, 5)])
def test_partitioned_operator_and_pcg_two_and_four_ranks(tmp_path, nel, world, N):
    mp.spawn(_rank_main, args=(world, _free_port(), nel, N, str(tmp_path)), nprocs=world,
             join=True)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    w_ref = o.matvec(si.uniform(o.shape, 92), 1.0, 0.3)
    b_ref = o.rhs(si.eval_fourier(si.fourier_modes(93), o.x, o.y, o.z))
    ref = o.pcg(b_ref, h1=1.0, h2=0.3, tol=1e-10)
    xs = np.zeros_like(b_ref)
    for r in range(world):
        z = np.load(tmp_path / f"rank{r}.npz")
        meta = json.loads((tmp_path / f"rank{r}.json").read_text())
        ge = z["ge"]
        shp = (len(ge),) + o.shape[1:]
        assert np.abs(z["w"].reshape(shp) - w_ref[ge]).max() / np.abs(w_ref).max() < 1e-12, r
        assert rel_inf(z["b"].reshape(shp), b_ref[ge]) < 1e-12, r
        assert meta["status"] == "ok" and abs(meta["iters"] - ref.iters) <= 1, (meta, ref.iters)
        xs[ge] = z["x"].reshape(shp)
    assert rel_inf(xs, ref.x) < 1e-8
    assert o.residual(xs, b_ref, 1.0, 0.3) <= 1.05e-10
