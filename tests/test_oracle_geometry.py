"""Pins for the oracle's trilinear map (Eq. 8), Jacobian (Eq. 9) and
geometric factors (Eq. 7).

Fixed independently of the oracle by: corner reproduction of the map,
central finite differences of the map, the constant Jacobian of an affine
element (edge vectors / 2), the closed form of G for a cube, the algebraic
identity G (J^T J) = W det(J) I, and the standard discrete Jacobian of
Sec. 3.2 (a second route inside the oracle, exact for trilinear maps).
"""
import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs


def _rand_hex(rng, amp=0.15):
    base = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=float)
    return base + rng.uniform(-amp, amp, size=(8, 3))


def test_map_reproduces_vertices(orc):
    rng = np.random.default_rng(10)
    V = _rand_hex(rng)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        X = orc.trilinear_map(V, 2 * a - 1, 2 * b - 1, 2 * c - 1)
        np.testing.assert_allclose(X, V[v], atol=1e-15)
    # centre is the vertex mean
    np.testing.assert_allclose(orc.trilinear_map(V, 0, 0, 0), V.mean(axis=0), atol=1e-15)


def test_jacobian_matches_finite_differences(orc):
    rng = np.random.default_rng(11)
    V = _rand_hex(rng, 0.2)
    h = 1e-5
    for _ in range(20):
        p = rng.uniform(-1, 1, size=3)
        J = orc.jacobian(V, *p)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fd = (orc.trilinear_map(V, *(p + e)) - orc.trilinear_map(V, *(p - e))) / (2 * h)
            np.testing.assert_allclose(J[:, d], fd, atol=1e-9)


def test_affine_element_has_constant_jacobian(orc):
    V = inputs.parallelepiped_vertices(1, 1, 1)[0]
    J0 = np.column_stack([V[1] - V[0], V[2] - V[0], V[4] - V[0]]) / 2.0
    rng = np.random.default_rng(12)
    for _ in range(10):
        np.testing.assert_allclose(orc.jacobian(V, *rng.uniform(-1, 1, 3)), J0, atol=1e-15)


def test_cube_factors_closed_form(orc):
    # cube of side h: J = (h/2) I, |J| = h^3/8, G = W (h/2) I, gwj = W h^3/8
    h, N = 0.25, 3
    V = inputs.box_vertices(1, 1, 1, perturb=0.0)[0] * (h / 1.0)
    G, bad = orc.factors(V[None], N)
    assert bad == 0
    xi, w, _ = orc.gll(N)
    W = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    np.testing.assert_allclose(G[0, 0], W * h / 2, rtol=1e-14)
    np.testing.assert_allclose(G[0, 3], W * h / 2, rtol=1e-14)
    np.testing.assert_allclose(G[0, 5], W * h / 2, rtol=1e-14)
    for q in (1, 2, 4):
        np.testing.assert_allclose(G[0, q], 0.0, atol=1e-16)
    np.testing.assert_allclose(G[0, 6], W * h ** 3 / 8, rtol=1e-14)


def test_factor_identity(orc):
    rng = np.random.default_rng(13)
    for _ in range(20):
        J = np.eye(3) + 0.3 * rng.uniform(-1, 1, (3, 3))
        W = rng.uniform(0.1, 1.0)
        g, det = orc.factors_from_jacobian(J, W)
        assert abs(det - np.linalg.det(J)) < 1e-14
        G = np.array([[g[0], g[1], g[2]], [g[1], g[3], g[4]], [g[2], g[4], g[5]]])
        np.testing.assert_allclose(G @ (J.T @ J), W * det * np.eye(3), atol=1e-13)
        assert abs(g[6] - W * det) < 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_discrete_jacobian_route_agrees(orc, N):
    V = inputs.box_vertices(2, 2, 2, perturb=0.1, seed=0)
    Ga, bad_a = orc.factors(V, N, "eq9")
    Gb, bad_b = orc.factors(V, N, "discrete")
    assert bad_a == 0 and bad_b == 0
    # relative to the size of the 3x3 factor matrix (off-diagonal entries are
    # small on a near-cubic mesh); the discrete derivative costs ~N^2 eps
    scale = np.abs(Ga[:, :6]).max()
    assert np.max(np.abs(Ga[:, :6] - Gb[:, :6])) / scale < 1e-13
    assert np.max(np.abs(Ga[:, 6] - Gb[:, 6])) / np.abs(Ga[:, 6]).max() < 1e-13


def test_inverted_element_is_counted(orc):
    V = inputs.box_vertices(1, 1, 1, perturb=0.0)
    V = V[:, [1, 0, 3, 2, 5, 4, 7, 6], :]  # mirror in r: det J < 0 everywhere
    _, bad = orc.factors(V, 3)
    assert bad == 4 ** 3


def test_nodal_coords_interpolate_linear_fields(orc):
    # the GLL nodes of the reference cube map to Phi(xi_i, xi_j, xi_k)
    N = 4
    V = inputs.box_vertices(1, 1, 1, perturb=0.0)
    XYZ = orc.nodal_coords(V, N)
    xi, _, _ = orc.gll(N)
    r = np.tile(xi, (N + 1) ** 2)
    np.testing.assert_allclose(XYZ[0, 0], (r + 1) / 2, atol=1e-15)
