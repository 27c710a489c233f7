"""Flexible GMRES(m) with right preconditioning (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§4 and Table 2: Neko solves the pressure Poisson equation by preconditioned
GMRES, the preconditioner being the two-level Schwarz method whose coarse
level is solved only approximately (a few CG iterations), so the
preconditioner changes from one application to the next.  Reading: the
flexible variant (Saad 1993) with restarts, which keeps the preconditioned
directions z_j and forms x from them:

* x = x0, r = b - H x, beta = ||r||, v_1 = r / beta, g = beta e_1;
* for j = 1 .. m: z_j = M^-1 v_j, w = H z_j; h_ij = <v_i, w> and
  w -= sum_i h_ij v_i, done twice (classical Gram-Schmidt, repeated);
  h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; the Givens rotations of the
  earlier columns are applied to column j, a new rotation zeroes h_{j+1,j}
  and updates g; |g_{j+1}| is the residual norm of the least-squares
  solution; stop the cycle when it is <= tol ||b||;
* x += Z y with y the solution of the triangular system; restart (from the
  true residual) until ||b - H x|| <= tol ||b|| or maxit iterations;
* <a, b> = sum_L a b / mult, the unique-dof inner product of the CG solver.
"""
import numpy as np

from .operator import weighted_dot


class GMRESResult:
    def __init__(self, x, iters, rel_res, status, history):
        self.x, self.iters, self.rel_res, self.status, self.history = (x, iters, rel_res,
                                                                       status, history)


def givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def fgmres(b, matvec, precond, mult, tol=1e-8, m=30, maxit=1000, x0=None, basis=None):
    """Solve H x = b; matvec(v) = H v, precond(v) = M^-1 v (L-vectors).
    basis: optional list that receives the Arnoldi vectors V of every cycle."""
    dot = lambda a, c: weighted_dot(a, c, mult)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.sqrt(dot(b, b))
    if bnorm == 0.0:
        return GMRESResult(np.zeros_like(b), 0, 0.0, "ok", [])
    history = []
    total = 0
    while True:
        r = b - matvec(x)
        beta = np.sqrt(dot(r, r))
        history.append(beta / bnorm)
        if beta <= tol * bnorm:
            return GMRESResult(x, total, beta / bnorm, "ok", history)
        if total >= maxit:
            return GMRESResult(x, total, beta / bnorm, "noconv", history)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            Z.append(precond(V[j]))
            w = matvec(Z[j])
            for _ in range(2):
                h = np.array([dot(V[i], w) for i in range(j + 1)])
                for i in range(j + 1):
                    w = w - h[i] * V[i]
                H[:j + 1, j] += h
            H[j + 1, j] = np.sqrt(dot(w, w))
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            hn = H[j + 1, j]
            cs[j], sn[j] = givens(H[j, j], hn)
            H[j, j] = cs[j] * H[j, j] + sn[j] * hn
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            total += 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or total >= maxit or hn == 0.0:
                break
            V.append(w / hn)
        if basis is not None:
            basis.append(list(V))
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
