"""Work captured into CUDA graphs as the first library call of a process.

The library's once-per-process setup (constant tables of the double-float
kernels, kernel attributes, the address of sem_dot_noalloc's static array)
runs in sem_setup, outside any stream capture.  So a solve whose iterations
are captured into a CUDA graph, or a sem_dot_noalloc captured with
torch.cuda.graph, works as the very first call after sem_setup.  Each case
runs in a fresh interpreter: inside one pytest process an earlier test would
have made the first use."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, math, sys
import torch
sys.path.insert(0, sys.argv[1])
import paper_2107_01243_gb300 as sem
import seeded_inputs as si

case, N = sys.argv[2], int(sys.argv[3])
dev = "cuda:0"
h = sem.sem_setup((4, 3, 3), N, length=(2 * math.pi,) * 3, deform=0.1)
n = h.n_local
vec = lambda seed: torch.from_numpy(si.uniform(n, seed)).to(dev)
if case == "noalloc":
    a, b = vec(11), vec(12)
    got = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sem.sem_dot_noalloc(h, a, b, got)
    g.replay()
    torch.cuda.synchronize()
    ref = torch.zeros_like(got)
    sem.sem_dot(h, a, b, ref)
    torch.cuda.synchronize()
    print(json.dumps(dict(got=float(got), ref=float(ref), scale=float((a * b).abs().sum()))))
else:
    b = torch.empty(n, dtype=torch.float64, device=dev)
    sem.sem_rhs(h, vec(13), b)
    x = torch.empty_like(b)
    if case == "pipelined":
        sem.sem_set_cg_variant(h, sem.SEM_CG_PIPELINED)
    prec = sem.SEM_SOLVE_MIXED if case == "mixed" else sem.SEM_SOLVE_F64
    info = sem.sem_cg_solve(h, b, x, tol=1e-8, precision=prec, use_graph=True)
    w = torch.empty_like(b)
    sem.sem_apply(h, x, w)
    r = b - w
    rr = torch.zeros(1, dtype=torch.float64, device=dev)
    bb = torch.zeros_like(rr)
    sem.sem_dot(h, r, r, rr)
    sem.sem_dot(h, b, b, bb)
    torch.cuda.synchronize()
    print(json.dumps(dict(status=info["status"], rel_res=info["rel_res"],
                          check=math.sqrt(float(rr) / float(bb)))))
"""


def run_child(case, N):
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT, case, str(N)], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("case,N", [("f64", 7), ("f64", 5), ("f64", 9), ("mixed", 7),
                                    ("pipelined", 7)])
def test_graph_captured_solve_as_first_call(case, N):
    res = run_child(case, N)
    assert res["status"] == "SEM_OK", res
    assert res["rel_res"] <= 1e-8 and res["check"] <= 1.0001e-8, res
    assert abs(res["check"] - res["rel_res"]) <= 1e-12, res


def test_noalloc_dot_captured_as_first_call():
    res = run_child("noalloc", 7)
    assert abs(res["got"] - res["ref"]) <= 1e-12 * res["scale"], res
