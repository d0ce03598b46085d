"""Pins for the oracle's AxLocal (Algorithm 1, Poisson case of Eq. 3).

What fixes the answer independently of the oracle:
* brute force: the dense element matrix D^T blkdiag(G) D built with numpy
  Kronecker products (Table 1) for N <= 4;
* A 1 = 0, symmetry, positive semidefiniteness with a one-dimensional kernel;
* exact energy on affine elements: for polynomials u, v of total degree <= N,
  v^T A u equals the integral of grad u . grad v over the element, computed
  here by tensor Gauss-Legendre quadrature (numpy) of the analytic gradients;
* linear u on a trilinear element (N >= 2): u^T A u = |a|^2 vol(element),
  with the volume from the divergence theorem over the six bilinear faces.
A dropped term, a sign, a transposed Dhat or a swapped index fails at least
one of these.
"""
import itertools

import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs


def _trilinear_elements(E=3, seed=20):
    V = inputs.box_vertices(E, 1, 1, perturb=0.0)
    rng = np.random.default_rng(seed)
    return V + rng.uniform(-0.03, 0.03, size=V.shape)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_matches_dense_element_matrix(orc, N):
    V = _trilinear_elements()
    G, bad = orc.factors(V, N)
    assert bad == 0
    X = inputs.element_vectors(V.shape[0], N, seed=21)
    Y = orc.axlocal(G, X, N)
    for e in range(V.shape[0]):
        A = orc.dense_element_matrix(G[e], N)
        ref = A @ X[e]
        assert np.max(np.abs(Y[e] - ref)) <= 1e-13 * np.max(np.abs(ref)) * (N + 1) ** 2


@pytest.mark.parametrize("N", [2, 3, 4])
def test_dense_matrix_is_spsd_with_constant_kernel(orc, N):
    V = _trilinear_elements(E=2)
    G, _ = orc.factors(V, N)
    for e in range(2):
        A = orc.dense_element_matrix(G[e], N)
        np.testing.assert_allclose(A, A.T, atol=1e-14 * np.abs(A).max())
        lam = np.linalg.eigvalsh(A)
        assert lam[0] > -1e-12 * lam[-1]
        assert lam[1] > 1e-6 * lam[-1]  # one zero eigenvalue only
        np.testing.assert_allclose(A @ np.ones(A.shape[0]), 0.0, atol=1e-12 * lam[-1])


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_constant_kernel_and_symmetry_matrix_free(orc, N):
    V = inputs.box_vertices(2, 2, 1, perturb=0.1, seed=0)
    E = V.shape[0]
    G, _ = orc.factors(V, N)
    ones = np.ones((E, (N + 1) ** 3))
    Y1 = orc.axlocal(G, ones, N)
    X = inputs.element_vectors(E, N, seed=1)
    Z = inputs.element_vectors(E, N, seed=2)
    AX, AZ = orc.axlocal(G, X, N), orc.axlocal(G, Z, N)
    scale = np.abs(AX).max()
    assert np.abs(Y1).max() < 1e-13 * scale
    lhs, rhs = np.einsum("ij,ij->i", Z, AX), np.einsum("ij,ij->i", X, AZ)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.abs(lhs).max()


def _monomials(p):
    return [(a, b, c) for a in range(p + 1) for b in range(p + 1 - a) for c in range(p + 1 - a - b)]


def _poly_and_grad(coef, exps, x):
    """u(x) and grad u(x) for u = sum coef * x^a y^b z^c; x is [..., 3]."""
    u = np.zeros(x.shape[:-1])
    g = np.zeros(x.shape)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    for c, (a, b, d) in zip(coef, exps):
        u += c * X ** a * Y ** b * Z ** d
        if a:
            g[..., 0] += c * a * X ** (a - 1) * Y ** b * Z ** d
        if b:
            g[..., 1] += c * b * X ** a * Y ** (b - 1) * Z ** d
        if d:
            g[..., 2] += c * d * X ** a * Y ** b * Z ** (d - 1)
    return u, g


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_exact_energy_on_parallelepipeds(orc, N):
    V = inputs.parallelepiped_vertices(2, 1, 1)
    E = V.shape[0]
    G, bad = orc.factors(V, N)
    assert bad == 0
    XYZ = orc.nodal_coords(V, N).transpose(0, 2, 1)  # [E][n3][3]
    exps = _monomials(N)
    rng = np.random.default_rng(30 + N)
    cu, cv = rng.uniform(-1, 1, len(exps)), rng.uniform(-1, 1, len(exps))
    # Gauss-Legendre (not GLL) on the reference cube, exact to degree 2N+3
    gq, gw = np.polynomial.legendre.leggauss(N + 2)
    R = np.stack(np.meshgrid(gq, gq, gq, indexing="ij"), axis=-1).reshape(-1, 3)
    Wq = np.einsum("i,j,k->ijk", gw, gw, gw).reshape(-1)
    for e in range(E):
        c0 = V[e].mean(axis=0)
        B = np.column_stack([V[e][1] - V[e][0], V[e][2] - V[e][0], V[e][4] - V[e][0]]) / 2.0
        u, _ = _poly_and_grad(cu, exps, XYZ[e] - c0)
        v, _ = _poly_and_grad(cv, exps, XYZ[e] - c0)
        Au = orc.axlocal(G[e:e + 1], u[None], N)[0]
        xq = R @ B.T
        _, gu = _poly_and_grad(cu, exps, xq)
        _, gv = _poly_and_grad(cv, exps, xq)
        exact = np.sum(Wq * np.einsum("qc,qc->q", gu, gv)) * abs(np.linalg.det(B))
        scale = np.sqrt(np.sum(Wq * np.einsum("qc,qc->q", gu, gu)) * np.sum(Wq * np.einsum("qc,qc->q", gv, gv)))
        scale *= abs(np.linalg.det(B))
        assert abs(v @ Au - exact) < 1e-11 * scale


def _hex_volume_divergence(Ve):
    """Volume of a trilinear hex: (1/3) sum over the six bilinear faces of the
    integral of x . (dP/da x dP/db), orientation from the reference frame."""
    gq, gw = np.polynomial.legendre.leggauss(3)
    corners = {v: Ve[v] for v in range(8)}

    def patch(P00, P10, P01, P11):
        tot = 0.0
        for a, wa in zip(gq, gw):
            for b, wb in zip(gq, gw):
                P = ((1 - a) * (1 - b) * P00 + (1 + a) * (1 - b) * P10 + (1 - a) * (1 + b) * P01 + (1 + a) * (1 + b) * P11) / 4
                Pa = ((1 - b) * (P10 - P00) + (1 + b) * (P11 - P01)) / 4
                Pb = ((1 - a) * (P01 - P00) + (1 + a) * (P11 - P10)) / 4
                tot += wa * wb * P @ np.cross(Pa, Pb)
        return tot

    def v(a, b, c):
        return corners[a + 2 * b + 4 * c]

    flux = 0.0
    for side, sgn in ((0, -1.0), (1, 1.0)):
        # r = +-1, parameters (s, t); s = +-1, parameters (t, r); t = +-1, parameters (r, s)
        flux += sgn * patch(v(side, 0, 0), v(side, 1, 0), v(side, 0, 1), v(side, 1, 1))
        flux += sgn * patch(v(0, side, 0), v(0, side, 1), v(1, side, 0), v(1, side, 1))
        flux += sgn * patch(v(0, 0, side), v(1, 0, side), v(0, 1, side), v(1, 1, side))
    return flux / 3.0


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_linear_energy_on_trilinear_elements(orc, N):
    V = inputs.box_vertices(2, 2, 2, perturb=0.1, seed=0)
    G, _ = orc.factors(V, N)
    XYZ = orc.nodal_coords(V, N)  # [E][3][n3]
    a = np.array([0.3, -1.1, 0.7])
    u = np.einsum("c,ecn->en", a, XYZ) + 0.25
    Au = orc.axlocal(G, u, N)
    for e in range(V.shape[0]):
        vol = _hex_volume_divergence(V[e])
        assert abs(u[e] @ Au[e] - (a @ a) * vol) < 1e-13 * (a @ a) * vol * (N + 1) ** 2


def test_cube_volume_sanity():
    V = inputs.box_vertices(1, 1, 1, perturb=0.0)[0] * 0.5
    assert abs(_hex_volume_divergence(V) - 0.125) < 1e-15


def test_axlocal_vertices_equals_two_step(orc):
    N = 5
    V = inputs.box_vertices(3, 2, 2, perturb=0.1, seed=0)
    X = inputs.element_vectors(V.shape[0], N, seed=1)
    G, _ = orc.factors(V, N)
    Y1 = orc.axlocal(G, X, N)
    Y2, bad = orc.axlocal_vertices(V, X, N)
    assert bad == 0
    np.testing.assert_array_equal(Y1, Y2)
