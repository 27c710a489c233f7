"""The seeded input recipe: the named workloads have the sizes the bench and
the parity tests quote, the generators are deterministic per seed, and the
batched workload spans the stated ranges (CPU only)."""
import math

import numpy as np

import seeded_inputs as si


def test_named_workloads():
    assert si.THROUGHPUT["nel"] == (32, 32, 32) and si.THROUGHPUT["N"] == 7
    assert si.THROUGHPUT["deform"] == 0.1 and si.THROUGHPUT["seed"] == 42
    assert math.prod(si.THROUGHPUT["nel"]) * 8 ** 3 == 16_777_216
    assert si.SOLVE["nel"] == (48, 48, 48) and si.SOLVE["tol"] == 1e-8
    assert math.prod(si.SOLVE["nel"]) * 8 ** 3 == 56_623_104
    assert si.MANUFACTURED["nel"] == (4, 4, 4) and si.MANUFACTURED["deform"] == 0.0
    assert si.ADJOINT["nel"] == (16, 16, 16)
    for w in (si.THROUGHPUT, si.SOLVE, si.ADJOINT):
        assert w["length"] == (si.TWO_PI,) * 3


def test_generators_are_deterministic_per_seed():
    a, b, c = si.uniform(1000, 5), si.uniform(1000, 5), si.uniform(1000, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= -1.0 and a.max() < 1.0
    m1, m2 = si.fourier_modes(9), si.fourier_modes(9)
    for p, q in zip(m1, m2):
        assert np.array_equal(p, q)
    amp, k, phi = m1
    assert amp.shape == (8,) and k.shape == (8, 3) and phi.shape == (8,)
    assert k.min() >= 1 and k.max() <= 4 and phi.min() >= 0.0 and phi.max() < si.TWO_PI
    # a drift of zero steps is the field itself
    for p, q in zip(si.drifting_modes(9, 0), m1):
        assert np.array_equal(p, q)


def test_batched_workload_ranges():
    probs = si.batch_problems()
    assert len(probs) == 64 and [p["seed"] for p in probs] == list(range(1000, 1064))
    for p in probs:
        nx, ny, nz = p["nel"]
        assert 512 <= p["E_target"] <= 32768
        assert nx <= ny <= nz <= 2 * nx                 # near-cubic box
        assert abs(nx * ny * nz - p["E_target"]) <= 0.05 * p["E_target"]
        assert p["N"] in (5, 7, 9) and 0.1 <= p["lam"] <= 10.0
    assert {p["N"] for p in probs} == {5, 7, 9}


def test_manufactured_source_is_minus_laplacian():
    """f = -lap u for u = sin(pi x) sin(pi y) sin(pi z), by central
    differences at a few interior points."""
    h = 1e-4
    for x, y, z in ((0.3, 0.4, 0.6), (0.7, 0.2, 0.5)):
        lap = 0.0
        for d in range(3):
            e = [0.0, 0.0, 0.0]
            e[d] = h
            up = si.manufactured_u(x + e[0], y + e[1], z + e[2])
            dn = si.manufactured_u(x - e[0], y - e[1], z - e[2])
            lap += (up - 2 * si.manufactured_u(x, y, z) + dn) / h ** 2
        assert abs(si.manufactured_f(x, y, z) + lap) < 1e-5 * si.manufactured_f(x, y, z)
