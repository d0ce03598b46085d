"""Pins for the oracle's GLL constants (Table 1).

Each check is fixed by the paper or by the mathematics, not by the oracle:
the N=2 values printed in Sec. 2.1, the textbook closed forms for N=3 and
N=4, exactness of the quadrature, exact differentiation of polynomials of
degree <= N, and the symmetries of the nodes and of Dhat.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                vals[k] = [float(Fraction(x)) for x in v]
    return vals


def test_n2_matches_printed_example(orc):
    g = _read_golden("gll_n2.txt")
    xi, w, D = orc.gll(2)
    np.testing.assert_allclose(xi, g["xi"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, g["w"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(D.reshape(-1), g["D"], rtol=0, atol=1e-14)


def test_n3_n4_closed_forms(orc):
    # N=3: nodes +-1, +-1/sqrt(5); weights 1/6, 5/6.
    xi, w, _ = orc.gll(3)
    np.testing.assert_allclose(xi, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    # N=4: nodes +-1, +-sqrt(3/7), 0; weights 1/10, 49/90, 32/45.
    xi, w, _ = orc.gll(4)
    np.testing.assert_allclose(xi, [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 11, 15])
def test_quadrature_exact_to_degree_2n_minus_1(orc, N):
    xi, w, _ = orc.gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(0, 2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, xi ** p) - exact) < 1e-13, p
    if N >= 1:
        # GLL is NOT exact for degree 2N (this separates it from Gauss-Legendre)
        p = 2 * N
        assert abs(np.dot(w, xi ** p) - 2.0 / (p + 1)) > 1e-10


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 11, 15])
def test_differentiation_exact_for_polynomials(orc, N):
    xi, _, D = orc.gll(N)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0.0, atol=1e-12)
    for p in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** p, p * xi ** (p - 1), atol=2e-12 * N * N)


@pytest.mark.parametrize("N", [2, 3, 5, 7, 15])
def test_symmetries(orc, N):
    xi, w, D = orc.gll(N)
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)
    # centro-antisymmetry of Dhat: D[N-i][N-j] = -D[i][j]
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-12)
    # nodes are the interior zeros of L_N' (checked with numpy's Legendre class)
    dL = np.polynomial.legendre.Legendre.basis(N).deriv()
    np.testing.assert_allclose(dL(xi[1:-1]), 0.0, atol=1e-10)
    # weights from the formula printed in Table 1, with numpy's L_N
    LN = np.polynomial.legendre.Legendre.basis(N)(xi)
    np.testing.assert_allclose(w, 2.0 / (N * (N + 1) * LN ** 2), rtol=1e-13)


@pytest.mark.parametrize("N", [2, 4, 7])
def test_dhat_is_lagrange_derivative(orc, N):
    # D[i][j] = pi_j'(xi_i): build pi_j with numpy polyfit-free Lagrange products
    xi, _, D = orc.gll(N)
    for j in range(N + 1):
        others = np.delete(xi, j)
        num = np.poly1d(others, r=True)
        pj = num / np.prod(xi[j] - others)
        np.testing.assert_allclose(pj.deriv()(xi), D[:, j], atol=1e-11)
