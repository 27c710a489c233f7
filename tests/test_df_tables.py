"""The compile-time derivative tables of the double-float element kernel
(paper_2107_01243_gb300/csrc/df_tables.cuh, written by gen_df_tables.py).

Checked on the CPU against the oracle's GLL derivative matrix (§2: D is the
derivative matrix of the Lagrange basis on the GLL points) and against the
two properties the kernel relies on: the rows of the forward even half S sum
to zero (D annihilates constants, so the kernel drops one term of every
even-half dot), and the extraction bounds cover the entries they bound.
"""
import importlib.util
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.gll import deriv_matrix

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_01243_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_df_tables",
                                                  os.path.join(CSRC, "gen_df_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


GEN = _gen()


def test_header_is_the_generators_output():
    with open(os.path.join(CSRC, "df_tables.cuh"), encoding="utf-8") as fh:
        assert fh.read() == GEN.render()


def _halves(M, H):
    N = M.shape[0] - 1
    A = 0.5 * (M[:H, :H] - M[:H, ::-1][:, :H])
    S = 0.5 * (M[:H, :H] + M[:H, ::-1][:, :H])
    return A, S


@pytest.mark.parametrize("P", [6, 8, 10])
def test_pairs_are_the_oracle_matrix(P):
    """hi + lo of every entry equals the oracle's D (and D^T) halves to the
    oracle's own FP64 accuracy, and lo is below half an ulp of hi (a
    correctly rounded split)."""
    H = P // 2
    eo, _, _ = GEN.tables(P)
    D = deriv_matrix(P - 1)
    for t, M in ((0, D), (1, D.T)):
        for a, ref in enumerate(_halves(M, H)):
            hi = np.array(eo[t][a][0], dtype=np.float32).reshape(H, H)
            lo = np.array(eo[t][a][1], dtype=np.float32).reshape(H, H)
            got = hi.astype(np.float64) + lo.astype(np.float64)
            assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max(), (t, a)
            ulp = np.spacing(np.abs(hi)).astype(np.float64)
            assert np.all(np.abs(lo.astype(np.float64)) <= 0.5 * ulp)


@pytest.mark.parametrize("P", [6, 8, 10])
def test_forward_even_rows_sum_to_zero(P):
    """sum_l S_il = (1/2) sum_l D_il = 0: the kernel replaces S e by
    sum_{l >= 1} S_il (e_l - e_0).  The stored pairs keep the sum below
    2^-46 of the row's absolute sum."""
    H = P // 2
    eo, _, _ = GEN.tables(P)
    for i in range(H):
        tot = sum(Fraction(eo[0][1][0][i * H + l]) + Fraction(eo[0][1][1][i * H + l])
                  for l in range(H))
        absum = sum(abs(Fraction(eo[0][1][0][i * H + l])) for l in range(H))
        assert abs(tot) <= Fraction(1, 2 ** 46) * absum, i


@pytest.mark.parametrize("P", [6, 8, 10])
def test_extraction_bounds_cover_the_entries(P):
    """rb(a, i) >= (1 + 2^-19) sum_l |hi A_il| and ab(a, q) >= (1 + 2^-19)
    |hi| for the transposed halves, so a bound formed in float arithmetic from
    them stays above the exact sum of |c z| (the extraction needs sigma >=
    that sum times 1 + 2^-20)."""
    H = P // 2
    eo, rb, ab = GEN.tables(P)
    grow = 1 + Fraction(1, 2 ** 19)
    for a in range(2):
        for i in range(H):
            row = sum(abs(Fraction(eo[1][a][0][i * H + l])) for l in range(H))
            assert Fraction(rb[a][i]) >= row * grow
        for q in range(H * H):
            assert Fraction(ab[a][q]) >= abs(Fraction(eo[1][a][0][q])) * grow
