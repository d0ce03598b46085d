"""Pins for the oracle's element diagonals and (P)CG on the assembled,
Dirichlet-masked Poisson system (Eq. 1).

Fixed independently of the oracle by:
* the diagonal of the dense element matrix (numpy Kronecker products);
* numpy.linalg.solve on the dense assembled matrix restricted to the
  unmasked nodes;
* spectral convergence of the discrete solution of -lap u = 3 pi^2 u,
  u = sin(pi x) sin(pi y) sin(pi z), on the unit cube as N grows;
* the Jacobi and plain CG solutions agreeing.
"""
import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs


def _problem(orc, ex, ey, ez, N, perturb=0.1):
    V = inputs.box_vertices(ex, ey, ez, perturb=perturb, seed=0)
    G, bad = orc.factors(V, N)
    assert bad == 0
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    return V, G, gid, ng, mask


def _rhs(orc, V, G, gid, ng, N):
    XYZ = orc.nodal_coords(V, N)
    u = np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
    f = 3 * np.pi ** 2 * u
    b = orc.gather(G[:, 6, :] * f, gid, ng)  # Q^T (w|J| f): GLL-lumped mass times f
    u_g = np.zeros(ng)
    u_g[gid.reshape(-1)] = u.reshape(-1)
    return b, u_g


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_element_diagonals_match_dense(orc, N):
    V, G, *_ = _problem(orc, 2, 1, 1, N)
    d = orc.element_diagonals(G, N)
    for e in range(V.shape[0]):
        A = orc.dense_element_matrix(G[e], N)
        np.testing.assert_allclose(d[e], np.diag(A), rtol=1e-13, atol=1e-15 * np.abs(A).max())


def test_pcg_matches_dense_solve(orc):
    N = 3
    V, G, gid, ng, mask = _problem(orc, 2, 2, 2, N)
    A = np.zeros((ng, ng))
    for e in range(V.shape[0]):
        Ae = orc.dense_element_matrix(G[e], N)
        A[np.ix_(gid[e], gid[e])] += Ae
    free = np.where(mask == 0)[0]
    rng = np.random.default_rng(50)
    b = rng.uniform(-1, 1, ng)
    x_ref = np.zeros(ng)
    x_ref[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    for diag in (None, orc.gather(orc.element_diagonals(G, N), gid, ng)):
        x, it, rr, ok = orc.pcg(G, gid, ng, mask, b, N, diag_global=diag, rtol=1e-14, maxit=1000)
        assert ok and rr <= 1e-14
        assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
        assert np.all(x[mask == 1] == 0.0)


def test_spectral_convergence_manufactured_solution(orc):
    errs = []
    for N in (2, 4, 6):
        V, G, gid, ng, mask = _problem(orc, 2, 2, 2, N)
        b, u = _rhs(orc, V, G, gid, ng, N)
        x, it, rr, ok = orc.pcg(G, gid, ng, mask, b, N, rtol=1e-13, maxit=5000)
        assert ok
        errs.append(np.max(np.abs(x - u)))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


def test_jacobi_and_plain_cg_agree(orc):
    N = 5
    V, G, gid, ng, mask = _problem(orc, 3, 2, 2, N)
    b, _ = _rhs(orc, V, G, gid, ng, N)
    x1, it1, _, ok1 = orc.pcg(G, gid, ng, mask, b, N, rtol=1e-12, maxit=5000)
    dg = orc.gather(orc.element_diagonals(G, N), gid, ng)
    x2, it2, _, ok2 = orc.pcg(G, gid, ng, mask, b, N, diag_global=dg, rtol=1e-12, maxit=5000)
    assert ok1 and ok2
    assert np.max(np.abs(x1 - x2)) <= 1e-9 * np.max(np.abs(x1))
    assert it2 <= it1
