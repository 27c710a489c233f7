"""Element partition across ranks (paper §3.2, Algorithm 1) on the CPU.

The package's partition, interface index lists, interface exchange (x, then
y, then z faces over torch.distributed) and partitioned PCG run on 2, 4 and 8
gloo ranks; each rank's compute is the oracle's (tests/partition_oracle.py).
The partitioned operator must equal the single-domain oracle operator on
every rank's elements to 1e-12, and the partitioned PCG must take the
single-domain oracle PCG's iterations (+-1) and reach its solution."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2107_01243_gb300 import partition as part
from tests.helpers import OracleProblem, rel_inf, TWO_PI
import seeded_inputs as si

FACES = 63


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("nel,world", [((4, 3, 2), 2), ((4, 3, 2), 4), ((5, 4, 3), 8),
                                       ((7, 1, 1), 3), ((2, 2, 2), 8), ((9, 5, 6), 12)])
def test_split_covers_every_element_once(nel, world):
    owner = -np.ones(nel, dtype=int)
    subs = [part.split_box(nel, world, r) for r in range(world)]
    assert np.prod(subs[0].dims) == world
    for s in subs:
        sl = tuple(slice(s.offset[d], s.offset[d] + s.count[d]) for d in range(3))
        assert (owner[sl] == -1).all()
        owner[sl] = s.rank
    assert (owner >= 0).all()
    for s in subs:
        for f, nb in enumerate(s.neighbours):
            if nb is None:
                continue
            t = subs[nb]
            assert t.neighbours[f ^ 1] == s.rank              # the opposite face
            d = f // 2
            for a in range(3):
                if a != d:
                    assert (s.offset[a], s.count[a]) == (t.offset[a], t.count[a])
            # adjacent along d
            lo, hi = (s, t) if f % 2 else (t, s)
            assert lo.offset[d] + lo.count[d] == hi.offset[d]


def test_grid_dims_prefers_the_least_interface():
    assert part.grid_dims((16, 16, 16), 8) == (2, 2, 2)
    assert part.grid_dims((64, 4, 4), 4) == (4, 1, 1)
    assert part.grid_dims((3, 1, 1), 3) == (3, 1, 1)
    with pytest.raises(ValueError):
        part.grid_dims((1, 1, 1), 2)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_face_lists_follow_the_mesh_numbering(N):
    """Every local point on a face plane, and only those, is listed; copies of
    one global point get one face point; the packed copy is a copy of it; and
    the face points of two ranks that share the face sit at the same physical
    coordinates (so both number the plane alike)."""
    from oracle import mesh
    nel, world = (4, 3, 2), 4
    subs = [part.split_box(nel, world, r) for r in range(world)]
    L = (TWO_PI,) * 3
    coords = {}
    for s in subs:
        gid = mesh.global_ids(*s.count, N)
        P = N + 1
        x0, ln = s.local_mesh((0.0, 0.0, 0.0), L)
        X = mesh.box_coords(*s.count, N, x0, ln, 0.1)
        coords[s.rank] = X
        for f in range(6):
            pack, add_idx, add_pos = part.face_lists(s.count, N, f)
            d, side = divmod(f, 2)
            lattice = [None, None, None]
            # lattice coordinate of every local point along each direction
            e = np.arange(gid.shape[0])
            ex, ey, ez = e % s.count[0], (e // s.count[0]) % s.count[1], e // (s.count[0] * s.count[1])
            kk, jj, ii = np.meshgrid(np.arange(P), np.arange(P), np.arange(P), indexing="ij")
            lattice[0] = (N * ex[:, None, None, None] + ii[None]).ravel()
            lattice[1] = (N * ey[:, None, None, None] + jj[None]).ravel()
            lattice[2] = (N * ez[:, None, None, None] + kk[None]).ravel()
            want = lattice[d] == (N * s.count[d] if side else 0)
            assert set(add_idx.tolist()) == set(np.flatnonzero(want).tolist())
            g = gid.ravel()
            # one face point per global point, the same for all its copies
            by_gid = {}
            for q, m in zip(add_idx, add_pos):
                by_gid.setdefault(g[q], set()).add(int(m))
            assert all(len(v) == 1 for v in by_gid.values())
            assert len(by_gid) == len(pack)
            assert all(g[pack[m]] == g[q] for q, m in zip(add_idx, add_pos))
    for s in subs:
        for f, nb in enumerate(s.neighbours):
            if nb is None:
                continue
            mine = part.face_lists(s.count, N, f)[0]
            theirs = part.face_lists(subs[nb].count, N, f ^ 1)[0]
            assert len(mine) == len(theirs)
            for a in range(3):
                np.testing.assert_allclose(coords[s.rank][a].ravel()[mine],
                                           coords[nb][a].ravel()[theirs], rtol=0, atol=1e-12)


def _global_elements(sub):
    """Global element index of each of the sub-box's elements, in its order."""
    nx, ny, _ = sub.nel_global
    e = np.arange(np.prod(sub.count))
    ex = e % sub.count[0] + sub.offset[0]
    ey = (e // sub.count[0]) % sub.count[1] + sub.offset[1]
    ez = e // (sub.count[0] * sub.count[1]) + sub.offset[2]
    return ex + nx * (ey + ny * ez)


def _rank_main(rank, world, port, nel, N, out_dir):
    import torch
    import torch.distributed as dist
    from tests.partition_oracle import OracleBackend
    torch.set_num_threads(1)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        L = (TWO_PI,) * 3
        sub = part.split_box(nel, world, rank)
        x0, ln = sub.local_mesh((0.0, 0.0, 0.0), L)
        be = OracleBackend(sub.count, N, x0, ln, 0.1, sub.local_faces(FACES))
        op = part.PartitionedOperator(be, sub, N)
        ge = _global_elements(sub)
        u = si.uniform((int(np.prod(nel)),) + (N + 1,) * 3, 90)[ge]
        w = be.zeros()
        op.apply(torch.from_numpy(u.ravel().copy()), w, 1.0, 0.3)
        # right-hand side: the single-domain b restricted to the rank (continuous)
        o = be.o
        b = o.rhs(si.eval_fourier(si.fourier_modes(91), o.x, o.y, o.z))
        bt = torch.from_numpy(b.ravel().copy())
        op.exchange(bt)                          # mask o QQ^T (B f) over all ranks
        x = be.zeros()
        its, rel, status = part.partitioned_pcg(op, bt, x, 1.0, 0.3, tol=1e-10)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), w=w.numpy(), x=x.numpy(),
                 b=bt.numpy(), ge=ge)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"iters": its, "rel": rel, "status": status,
                       "dot_bb": op.dot(bt, bt)}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nel,world,N", [((4, 3, 2), 2, 5), ((4, 3, 2), 4, 3), ((4, 4, 4), 8, 3)])
def test_partitioned_operator_and_pcg_on_gloo_ranks(tmp_path, nel, world, N):
    mp.spawn(_rank_main, args=(world, _free_port(), nel, N, str(tmp_path)), nprocs=world,
             join=True)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=FACES)
    u = si.uniform(o.shape, 90)
    w_ref = o.matvec(u, 1.0, 0.3)
    b_ref = o.rhs(si.eval_fourier(si.fourier_modes(91), o.x, o.y, o.z))
    ref = o.pcg(b_ref, h1=1.0, h2=0.3, tol=1e-10)
    scale = np.abs(w_ref).max()
    xs = np.zeros_like(b_ref)
    for r in range(world):
        z = np.load(tmp_path / f"rank{r}.npz")
        meta = json.loads((tmp_path / f"rank{r}.json").read_text())
        ge = z["ge"]
        shp = (len(ge),) + o.shape[1:]
        assert np.abs(z["w"].reshape(shp) - w_ref[ge]).max() / scale < 1e-12, r
        # the exchanged right-hand side is the single-domain one
        assert rel_inf(z["b"].reshape(shp), b_ref[ge]) < 1e-12, r
        assert meta["status"] == "ok" and abs(meta["iters"] - ref.iters) <= 1, (meta, ref.iters)
        assert abs(meta["dot_bb"] - float(np.sum(b_ref * b_ref / o.mult))) <= \
            1e-12 * float(np.sum(b_ref * b_ref / o.mult))
        xs[ge] = z["x"].reshape(shp)
    assert rel_inf(xs, ref.x) < 1e-8
    assert o.residual(xs, b_ref, 1.0, 0.3) <= 1.05e-10
