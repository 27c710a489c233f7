"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds random draws and workload definitions only -- none of the
SEM arithmetic.  The CUDA path and the oracle each build their own mesh,
coordinates and operators; both receive the arrays made here.

Workloads (hexahedral deformed boxes with 8-10 GLL points per direction stand
in for the paper's meshes, which are not available):

* ``manufactured_*``  -- Poisson on the unit cube, u = sin(pi x) sin(pi y) sin(pi z)
* ``uniform``         -- local fields u ~ U(-1, 1) (operator throughput inputs)
* ``fourier_modes``   -- smooth fields sum_m a_m sin(k_m . x + phi_m), 8 modes,
                         a_m ~ N(0,1), k_m in {1..4}^3, phi_m ~ U(0, 2 pi)
* ``batch_problems``  -- independent Helmholtz problems with E in [512, 32768]
                         (nearest near-cubic box), N in {5,7,9},
                         lambda ~ U(0.1, 10); problem p uses seed 1000 + p
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def uniform(shape, seed, lo=-1.0, hi=1.0, dtype=np.float64):
    """Seeded U(lo, hi) array (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(dtype, copy=False)


def fourier_modes(seed, n_modes=8, kmax=4):
    """(a, k, phi) of a seeded smooth field; k has shape (n_modes, 3)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_modes)
    k = rng.integers(1, kmax + 1, size=(n_modes, 3))
    phi = rng.uniform(0.0, TWO_PI, size=n_modes)
    return a, k, phi


def eval_fourier(modes, x, y, z):
    """sum_m a_m sin(k_m . (x,y,z) + phi_m) at the given points."""
    a, k, phi = modes
    f = np.zeros_like(x, dtype=np.float64)
    for m in range(len(a)):
        f += a[m] * np.sin(k[m, 0] * x + k[m, 1] * y + k[m, 2] * z + phi[m])
    return f


def drifting_modes(seed, step, rate=0.05, n_modes=8, kmax=4):
    """The modes of fourier_modes(seed) with every phase advanced by
    step * rate * omega_m (omega_m ~ U(0.5, 1.5), seeded): a sequence of
    slowly varying right-hand sides, as successive time steps produce."""
    a, k, phi = fourier_modes(seed, n_modes, kmax)
    omega = np.random.default_rng(seed + 7919).uniform(0.5, 1.5, size=n_modes)
    return a, k, phi + step * rate * omega


def manufactured_u(x, y, z):
    return np.sin(math.pi * x) * np.sin(math.pi * y) * np.sin(math.pi * z)


def manufactured_f(x, y, z):
    """-lap u for u = sin(pi x) sin(pi y) sin(pi z)."""
    return 3.0 * math.pi ** 2 * manufactured_u(x, y, z)


def near_cubic_box(E_target, max_side=64):
    """(nelx, nely, nelz) with nelx <= nely <= nelz <= 2 nelx minimising
    |nelx nely nelz - E_target| (ties: the most cubic)."""
    best = None
    for a in range(1, max_side + 1):
        for b in range(a, min(2 * a, max_side) + 1):
            c_lo = max(b, 1)
            c_hi = min(2 * a, max_side)
            if c_hi < c_lo:
                continue
            c = int(round(E_target / (a * b)))
            for cc in (c - 1, c, c + 1):
                if c_lo <= cc <= c_hi:
                    key = (abs(a * b * cc - E_target), cc - a)
                    if best is None or key < best[0]:
                        best = (key, (a, b, cc))
    return best[1]


def batch_problems(n_problems=64, seed_base=1000, e_lo=512, e_hi=32768,
                   orders=(5, 7, 9), lam_lo=0.1, lam_hi=10.0):
    """List of dicts (seed, nel, N, lam, rhs_modes) for the batched workload."""
    out = []
    for p in range(n_problems):
        seed = seed_base + p
        rng = np.random.default_rng(seed)
        E = int(rng.integers(e_lo, e_hi + 1))
        N = int(orders[int(rng.integers(0, len(orders)))])
        lam = float(rng.uniform(lam_lo, lam_hi))
        out.append(dict(seed=seed, nel=near_cubic_box(E), E_target=E, N=N, lam=lam,
                        rhs_modes=fourier_modes(seed + 100000)))
    return out


def smooth_coefficient(x, y, z, seed=77):
    """h1 = 1 + 0.5 tanh(g) for a seeded Fourier field g."""
    return 1.0 + 0.5 * np.tanh(eval_fourier(fourier_modes(seed), x, y, z))


# Named workloads (sizes of the paper-derived configurations)
MANUFACTURED = dict(nel=(4, 4, 4), N=7, x0=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0),
                    deform=0.0, tol=1e-10)
THROUGHPUT = dict(nel=(32, 32, 32), N=7, x0=(0.0, 0.0, 0.0),
                  length=(TWO_PI, TWO_PI, TWO_PI), deform=0.1, seed=42)
SOLVE = dict(nel=(48, 48, 48), N=7, x0=(0.0, 0.0, 0.0),
             length=(TWO_PI, TWO_PI, TWO_PI), deform=0.1, seed=1234, tol=1e-8)
ADJOINT = dict(nel=(16, 16, 16), N=7, x0=(0.0, 0.0, 0.0),
               length=(TWO_PI, TWO_PI, TWO_PI), deform=0.1,
               h1_seed=77, target_seed=78, rhs_seed=79)
