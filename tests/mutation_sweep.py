"""Plants single-line mistakes in the oracle, one at a time, and checks that
the CPU pins catch every one.

    python tests/mutation_sweep.py [name ...]

Each mutation replaces one fragment of one oracle module (a dropped term, a
wrong sign, index or operand, a transposed contraction) at import time,
through the hook in tests/conftest.py: the files on disk are never written.
For each, the oracle pin tests run in a fresh interpreter and must fail.
Exit status 1 if a mutation survives or the unmutated pins fail.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_gll.py", "tests/test_oracle_operator.py",
        "tests/test_oracle_solve.py", "tests/test_oracle_adjoint.py",
        "tests/test_oracle_projection.py", "tests/test_oracle_pipecg.py",
        "tests/test_oracle_schwarz.py"]

# (module, name, fragment, replacement)
MUTATIONS = [
    ("oracle.gll", "weight_denominator", "w = 2.0 / (N * (N + 1) * legendre(N, xi) ** 2)",
     "w = 2.0 / (N * (N + 2) * legendre(N, xi) ** 2)"),
    ("oracle.gll", "D00_sign", "D[0, 0] = -N * (N + 1) / 4.0", "D[0, 0] = N * (N + 1) / 4.0"),
    ("oracle.gll", "D_offdiagonal_swapped", "D[i, j] = LN[i] / (LN[j] * (xi[i] - xi[j]))",
     "D[i, j] = LN[j] / (LN[i] * (xi[i] - xi[j]))"),
    ("oracle.geometry", "ds_transposed", "fs = np.einsum('jl,ekli->ekji', D, f)",
     "fs = np.einsum('lj,ekli->ekji', D, f)"),
    ("oracle.geometry", "G12_G13_swapped", "scale * M[..., 0, 1], scale * M[..., 0, 2]",
     "scale * M[..., 0, 2], scale * M[..., 0, 1]"),
    ("oracle.geometry", "quadrature_weight", "w[None, None, :, None] * w[None, None, None, :]",
     "w[None, None, :, None] * w[None, None, :, None]"),
    ("oracle.geometry", "metric_transposed", "np.einsum('...ba,...ca->...bc', Jinv, Jinv)",
     "np.einsum('...ab,...ac->...bc', Jinv, Jinv)"),
    ("oracle.operator", "wr_G_swapped", "wr = c * (G11 * ur + G12 * us + G13 * ut)",
     "wr = c * (G11 * ur + G13 * us + G12 * ut)"),
    ("oracle.operator", "s_contraction_not_transposed", "+ np.einsum('lj,ekli->ekji', D, ws)",
     "+ np.einsum('jl,ekli->ekji', D, ws)"),
    ("oracle.operator", "mass_term_drops_u", "w = w + h2 * B * u", "w = w + h2 * B"),
    ("oracle.operator", "dssum_of_magnitudes", "weights=w.ravel())",
     "weights=np.abs(w.ravel()))"),
    ("oracle.operator", "dot_without_multiplicity", "return float(np.sum(a * b / mult))",
     "return float(np.sum(a * b))"),
    ("oracle.operator", "h1_field_ignored", "c = h1 if h1_field is None else h1_field", "c = h1"),
    ("oracle.mesh", "iy_along_k", "iy = N * ey[:, None, None, None] + i[None, None, :, None]",
     "iy = N * ey[:, None, None, None] + i[None, :, None, None]"),
    ("oracle.mesh", "deform_x", "xd = x + a * np.sin(y) * np.sin(z)",
     "xd = x + a * np.sin(y) * np.sin(y)"),
    ("oracle.mesh", "deform_y", "yd = y + a * np.sin(z) * np.sin(x)",
     "yd = y + a * np.sin(z) * np.sin(y)"),
    ("oracle.mesh", "deform_z", "zd = z + a * np.sin(x) * np.sin(y)",
     "zd = z + a * np.sin(x) * np.sin(z)"),
    ("oracle.mesh", "global_id_stride", "return (ix + gx * (iy + gy * iz)).astype(np.int64)",
     "return (ix + gx * (iy + gx * iz)).astype(np.int64)"),
    ("oracle.mesh", "mask_xmax_off_by_one", "m[ix == N * nelx] = 0.0",
     "m[ix == N * nelx - 1] = 0.0"),
    ("oracle.mesh", "mask_zmin_on_y", "m[iz == 0] = 0.0", "m[iy == 0] = 0.0"),
    ("oracle.mesh", "element_y_index", "    ey = (e // nelx) % nely\n    ez = e // (nelx * nely)\n    hx",
     "    ey = (e // nely) % nely\n    ez = e // (nelx * nely)\n    hx"),
    ("oracle.mesh", "y_spacing", "length[1] / nely", "length[1] / nelx"),
    ("oracle.solve", "diagonal_cross_factor", "d = d + 2.0 * (di * dj * G12",
     "d = d + 1.0 * (di * dj * G12"),
    ("oracle.solve", "diagonal_G22_transposed", "+ np.einsum('lj,ekli->ekji', D2, G22)",
     "+ np.einsum('jl,ekli->ekji', D2, G22)"),
    ("oracle.solve", "diagonal_without_mass", "d = d + h2 * B", "d = d + 0.0 * B"),
    ("oracle.solve", "rhs_without_mass", "return apply_dirichlet(dssum(B * f, gid), mask)",
     "return apply_dirichlet(dssum(f, gid), mask)"),
    ("oracle.solve", "beta_inverted", "beta = rz_new / rz", "beta = rz / rz_new"),
    ("oracle.solve", "x_update_along_z", "x = x + alpha * p", "x = x + alpha * z"),
    ("oracle.solve", "stopping_test_loose", "if rel <= tol:", "if rel <= 10.0 * tol:"),
    ("oracle.adjoint", "gradient_sign", "return -(lr * gu_r + ls * gu_s + lt * gu_t)",
     "return (lr * gu_r + ls * gu_s + lt * gu_t)"),
    ("oracle.adjoint", "gradient_G13_for_G23", "gu_s = G12 * ur + G22 * us + G23 * ut",
     "gu_s = G12 * ur + G22 * us + G13 * ut"),
    ("oracle.adjoint", "loss_gradient_without_multiplicity", "return 2.0 * (u - u_target) / mult",
     "return 2.0 * (u - u_target)"),
    ("oracle.gmres", "givens_sign", "H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]",
     "H[i + 1, j] = sn[i] * H[i, j] + cs[i] * H[i + 1, j]"),
    ("oracle.gmres", "one_gram_schmidt_pass", "for _ in range(2):\n                h = np.array",
     "for _ in range(1):\n                h = np.array"),
    ("oracle.gmres", "gram_schmidt_unweighted",
     "h = np.array([dot(V[i], w) for i in range(j + 1)])",
     "h = np.array([float(np.sum(V[i] * w)) for i in range(j + 1)])"),
    ("oracle.gmres", "residual_rotation_sign", "g[j + 1] = -sn[j] * g[j]", "g[j + 1] = sn[j] * g[j]"),
    ("oracle.gmres", "solution_from_V", "x = x + y[i] * Z[i]", "x = x + y[i] * V[i]"),
    ("oracle.gmres", "back_substitution_sign",
     "y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]",
     "y[i] = (g[i] + H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]"),
    ("oracle.projection", "projected_residual_sign", "r = r - a * w", "r = r + a * w"),
    ("oracle.projection", "space_not_normalised", "s = 1.0 / np.sqrt(nrm2)", "s = 1.0"),
    ("oracle.projection", "H_x_without_projection", "hx = b - r + hd", "hx = b + hd"),
    ("oracle.pipecg", "u_recurrence", "u = u - alpha * q", "u = u - alpha * s"),
    ("oracle.pipecg", "z_recurrence", "z = n + beta * z", "z = m + beta * z"),
    ("oracle.pipecg", "alpha_sign", "alpha = gamma / (delta - beta * gamma / alpha_old)",
     "alpha = gamma / (delta + beta * gamma / alpha_old)"),
    ("oracle.dense", "barycentric_ratio_inverted", "D[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])",
     "D[i, j] = (lam[i] / lam[j]) / (xi[i] - xi[j])"),
    ("oracle.dense", "kronecker_axes_swapped", "Dr = np.kron(I, np.kron(I, D1))",
     "Dr = np.kron(I, np.kron(D1, I))"),
    ("oracle.dense", "inverse_jacobian_not_transposed", "JinvT = np.linalg.inv(J).T",
     "JinvT = np.linalg.inv(J)"),
    ("oracle.dense", "mass_without_detJ", "M[e, q] = W[q] * detJ", "M[e, q] = W[q]"),
    ("oracle.schwarz", "grown_points_reversed", "    idx = np.arange(N - 1, 2 * N + 2)",
     "    idx = np.arange(N - 1, 2 * N + 2)[::-1]"),
    ("oracle.schwarz", "dirichlet_point_kept", "            keep[1] = False", "            pass"),
    ("oracle.schwarz", "left_neighbour_ignored",
     "        if (m == 0 and lo != NEIGHBOUR) or (m == 2 and hi != NEIGHBOUR):",
     "        if m == 0 or (m == 2 and hi != NEIGHBOUR):"),
    ("oracle.schwarz", "restriction_without_multiplicity", "        rm = r / self.mult",
     "        rm = r"),
    ("oracle.schwarz", "fdm_mass_sign",
     "    t = t / (h1 * (lx[None, None, :] + ly[None, :, None] + lz[:, None, None]) + h2)",
     "    t = t / (h1 * (lx[None, None, :] + ly[None, :, None] + lz[:, None, None]) - h2)"),
    ("oracle.schwarz", "1d_mass_scale", "    be = (L / 2.0) * w", "    be = L * w"),
]


def run_pins(mutation=None):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("SEM_ORACLE_MUTATION", None)
    if mutation is not None:
        env["SEM_ORACLE_MUTATION"] = json.dumps(mutation)
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-q", "-x", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    last = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr.strip()[-200:]
    return r.returncode, last


def main(names):
    for module, name, old, _ in MUTATIONS:
        path = os.path.join(ROOT, *module.split(".")) + ".py"
        with open(path, encoding="utf-8") as f:
            assert old in f.read(), f"{name}: fragment not found in {module}"
    rc, last = run_pins()
    print(f"{'unmutated':40s} {'pass' if rc == 0 else 'FAIL'}  {last}", flush=True)
    if rc != 0:
        return 1
    survived = []
    for module, name, old, new in MUTATIONS:
        if names and name not in names:
            continue
        rc, last = run_pins({"module": module, "old": old, "new": new})
        caught = rc == 1                      # a failed pin (not a crash or a collection error)
        print(f"{module + ':' + name:40s} {'caught' if caught else 'SURVIVED'}  {last}",
              flush=True)
        if not caught:
            survived.append(name)
    print("survived:", survived)
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
