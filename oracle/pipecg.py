"""Pipelined Jacobi-preconditioned CG (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's outlook (§10) names non-blocking or pipelined Krylov solvers as
the way around the global reductions that bound strong scaling.  Reading:
the pipelined PCG of Ghysels and Vanroose (2014), which needs one reduction
per iteration for both inner products, computed from vectors that are all
updated by recurrences, so that the reduction can overlap the operator:

    r = b - H x, u = M r, w = H u
    repeat: gamma = <r, u>, delta = <w, u>, ||r||^2;  stop if ||r|| <= tol ||b||
            m = M w, n = H m
            beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
            (first iteration: beta = 0, alpha = gamma / delta)
            z = n + beta z,  q = m + beta q,  s = w + beta s,  p = u + beta p
            x += alpha p,  r -= alpha s,  u -= alpha q,  w -= alpha z

with M = dinv (point Jacobi) and the unique-dof inner product of the CG
solver.  In exact arithmetic the iterates equal those of standard PCG.  The
residual r is a recurrence; when it reaches the tolerance the true residual
b - H x is checked and the iteration restarts from it if it has not.
"""
import numpy as np

from .operator import weighted_dot


class PipeResult:
    def __init__(self, x, iters, rel_res, status, restarts):
        self.x, self.iters, self.rel_res, self.status, self.restarts = (x, iters, rel_res,
                                                                       status, restarts)


def pipecg(b, matvec, dinv, mult, tol=1e-8, maxit=20000, max_restarts=5, history=None):
    """Solve H x = b from x = 0; matvec(v) = H v.  history: optional list that
    receives x after every iteration."""
    dot = lambda a, c: weighted_dot(a, c, mult)
    x = np.zeros_like(b)
    bnorm = np.sqrt(dot(b, b))
    if bnorm == 0.0:
        return PipeResult(x, 0, 0.0, "ok", 0)
    it = 0
    restarts = 0
    while True:
        r = b - matvec(x)
        u = dinv * r
        w = matvec(u)
        z = np.zeros_like(b)
        q = np.zeros_like(b)
        s = np.zeros_like(b)
        p = np.zeros_like(b)
        gamma_old = alpha_old = None
        while True:
            gamma, delta, rr = dot(r, u), dot(w, u), dot(r, r)
            if np.sqrt(rr) <= tol * bnorm or it >= maxit:
                break
            m = dinv * w
            n = matvec(m)
            if gamma_old is None:
                beta, alpha = 0.0, gamma / delta
            else:
                beta = gamma / gamma_old
                alpha = gamma / (delta - beta * gamma / alpha_old)
            z = n + beta * z
            q = m + beta * q
            s = w + beta * s
            p = u + beta * p
            x = x + alpha * p
            r = r - alpha * s
            u = u - alpha * q
            w = w - alpha * z
            gamma_old, alpha_old = gamma, alpha
            it += 1
            if history is not None:
                history.append(x.copy())
        rt = b - matvec(x)
        rel = np.sqrt(dot(rt, rt)) / bnorm
        if rel <= tol:
            return PipeResult(x, it, rel, "ok", restarts)
        if it >= maxit or restarts >= max_restarts:
            return PipeResult(x, it, rel, "noconv", restarts)
        restarts += 1
