"""Writes df_tables.cuh: the derivative-matrix tables of the double-float
element kernel (ax_df.cu) as compile-time constants.

The kernel's line tasks use the even-odd halves of D (or D^T) on the
Gauss-Lobatto-Legendre nodes (arXiv 2107.01243 §2: D is the derivative matrix
of the Lagrange basis on the N + 1 GLL points).  With the tables known at
compile time every coefficient is an immediate operand of its instruction,
so the kernel issues no constant-memory loads for them.

Everything is computed here in 60-digit decimal arithmetic, so each float
pair (high part = the value rounded to float, low part = the remainder
rounded to float) is the correctly rounded split of the exact entry:

* nodes: -1, 1 and the roots of L_N' (Newton from the Chebyshev-Lobatto
  points, with L_N'' from the Legendre equation);
* D_ij = L_N(x_i) / (L_N(x_j) (x_i - x_j)) for i != j, D_00 = -N(N+1)/4,
  D_NN = N(N+1)/4, other diagonal entries 0;
* for M = D (forward) and M = D^T (transposed), with H = P/2:
  A_il = (M_il - M_{i,N-l}) / 2 and S_il = (M_il + M_{i,N-l}) / 2, i, l < H;
* bounds of the extraction dots: (1 + 2^-18) sum_l |high part of A_il| (and
  of S_il), and the entries (1 + 2^-18) |high part| themselves, for M = D^T.

Run: python gen_df_tables.py  (rewrites df_tables.cuh beside this file)
"""
import decimal
import math
import os
import struct

decimal.getcontext().prec = 60
Dec = decimal.Decimal
ORDERS = (6, 8, 10)                  # P = N + 1 of the double-float kernel


def legendre(N, x):
    """L_N(x) and L_{N-1}(x) by the three-term recurrence (N >= 1)."""
    p0, p1 = Dec(1), x
    for n in range(2, N + 1):
        p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
    return p1, p0


def gll_nodes(N):
    x = [Dec(-1)] + [Dec(0)] * (N - 1) + [Dec(1)]
    for j in range(1, N):
        xj = Dec(-math.cos(math.pi * j / N))
        for _ in range(200):
            L, Lm = legendre(N, xj)
            dL = N * (xj * L - Lm) / (xj * xj - 1)     # (x^2 - 1) L_N' = N (x L_N - L_{N-1})
            d2L = (2 * xj * dL - N * (N + 1) * L) / (1 - xj * xj)
            step = dL / d2L
            xj -= step
            if abs(step) < Dec("1e-55"):
                break
        x[j] = xj
    return x


def deriv_matrix(N):
    x = gll_nodes(N)
    L = [legendre(N, xi)[0] for xi in x]
    P = N + 1
    D = [[Dec(0)] * P for _ in range(P)]
    for i in range(P):
        for j in range(P):
            if i != j:
                D[i][j] = L[i] / (L[j] * (x[i] - x[j]))
    D[0][0] = Dec(-N * (N + 1)) / 4
    D[N][N] = Dec(N * (N + 1)) / 4
    return D


def f32(v):
    """v rounded to the nearest float.  The decimal goes through the nearest
    double first; a double rounding is resolved by comparing the candidate's
    two float neighbours with the exact value."""
    c = struct.unpack("f", struct.pack("f", float(v)))[0]
    bits = struct.unpack("I", struct.pack("f", c))[0]
    best = c
    for nb in (bits - 1, bits + 1):
        if 0 <= nb < 0x7F800000 or 0x80000000 <= nb < 0xFF800000:
            nb32 = struct.unpack("f", struct.pack("I", nb))[0]
            if abs(Dec(nb32) - v) < abs(Dec(best) - v):
                best = nb32
    return best


def split(v):
    hi = f32(v)
    lo = f32(v - Dec(hi))
    return hi, lo


def lit(v):
    """C++ hexadecimal float literal (exact)."""
    return "0.0f" if v == 0.0 else float.hex(v) + "f"


def tables(P):
    N, H = P - 1, P // 2
    D = deriv_matrix(N)
    eo = [[[[0.0] * (H * H) for _ in range(2)] for _ in range(2)] for _ in range(2)]
    for t in range(2):
        M = (lambda i, l: D[l][i]) if t else (lambda i, l: D[i][l])
        for i in range(H):
            for l in range(H):
                a = (M(i, l) - M(i, N - l)) / 2
                s = (M(i, l) + M(i, N - l)) / 2
                eo[t][0][0][i * H + l], eo[t][0][1][i * H + l] = split(a)
                eo[t][1][0][i * H + l], eo[t][1][1][i * H + l] = split(s)
    grow = Dec(1) + Dec(2) ** -18
    rb = [[f32(sum(abs(Dec(eo[1][a][0][i * H + l])) for l in range(H)) * grow)
           for i in range(H)] for a in range(2)]
    ab = [[f32(abs(Dec(eo[1][a][0][q])) * grow) for q in range(H * H)] for a in range(2)]
    return eo, rb, ab


def render():
    out = ["// Generated by gen_df_tables.py (run it to rewrite this file): the",
           "// even-odd tables of the GLL derivative matrix for the double-float",
           "// element kernel, as float pairs of the exact entries, and the bounds",
           "// of its extraction dot products.  See gen_df_tables.py for the",
           "// definitions.",
           "#pragma once", "", "namespace sem {", "",
           "// DFTab<P>::eo(t, a, hl, q): t = 0 D, 1 D^T; a = 0 A (odd half), 1 S (even",
           "// half); hl = 0 high, 1 low part; q = i (P/2) + l.  rb(a, i): row bounds,",
           "// ab(a, q): entry bounds, both of D^T.  Called with indices that are",
           "// compile-time constants after unrolling, so every value folds into an",
           "// immediate operand.",
           "template <int P>", "struct DFTab;", ""]
    for P in ORDERS:
        H = P // 2
        eo, rb, ab = tables(P)
        flat = [eo[t][a][hl][q] for t in range(2) for a in range(2) for hl in range(2)
                for q in range(H * H)]
        out.append("template <>")
        out.append(f"struct DFTab<{P}> {{")
        out.append("  __host__ __device__ static constexpr float eo(int t, int a, int hl, int q) {")
        out.append(f"    constexpr float v[{len(flat)}] = {{")
        for k in range(0, len(flat), 4):
            out.append("        " + ", ".join(lit(x) for x in flat[k:k + 4]) + ",")
        out.append("    };")
        out.append(f"    return v[((t * 2 + a) * 2 + hl) * {H * H} + q];")
        out.append("  }")
        fr = [rb[a][i] for a in range(2) for i in range(H)]
        out.append("  __host__ __device__ static constexpr float rb(int a, int i) {")
        out.append(f"    constexpr float v[{len(fr)}] = {{" + ", ".join(lit(x) for x in fr) + "};")
        out.append(f"    return v[a * {H} + i];")
        out.append("  }")
        fa = [ab[a][q] for a in range(2) for q in range(H * H)]
        out.append("  __host__ __device__ static constexpr float ab(int a, int q) {")
        out.append(f"    constexpr float v[{len(fa)}] = {{")
        for k in range(0, len(fa), 4):
            out.append("        " + ", ".join(lit(x) for x in fa[k:k + 4]) + ",")
        out.append("    };")
        out.append(f"    return v[a * {H * H} + q];")
        out.append("  }")
        out.append("};")
        out.append("")
    out.append("}  // namespace sem")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "df_tables.cuh")
    with open(path, "w", encoding="utf-8") as fh:
        fh.write(render())
    print(path)
