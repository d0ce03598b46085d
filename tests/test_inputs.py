"""The seeded synthetic workloads follow their stated recipes (the inputs module
is shared by the CUDA path and the oracle, so a recipe error would go unseen
by the parity tests): mesh geometry and vertex order, perturbation bounds,
parallelepiped affinity, sweep sizes, the uneven batch, global numbering."""
import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs


def test_box_vertex_order_and_perturbation():
    ex, ey, ez = 4, 3, 2
    h = 1.0 / ex
    V0 = inputs.box_vertices(ex, ey, ez, perturb=0.0)
    V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    assert V.shape == (ex * ey * ez, 8, 3)
    # element e = ix + ex (iy + ey iz); vertex a + 2b + 4c at corner (ix + a, iy + b, iz + c)
    for e in range(V0.shape[0]):
        ix, iy, iz = e % ex, (e // ex) % ey, e // (ex * ey)
        for v in range(8):
            a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
            np.testing.assert_allclose(V0[e, v], [(ix + a) * h, (iy + b) * h, (iz + c) * h], atol=1e-15)
    d = V - V0
    assert np.abs(d).max() <= 0.1 * h + 1e-15 and np.abs(d).max() > 0.05 * h
    on_boundary = np.isclose(V0[..., 0], 0) | np.isclose(V0[..., 0], ex * h) | np.isclose(V0[..., 1], 0) | \
        np.isclose(V0[..., 1], ey * h) | np.isclose(V0[..., 2], 0) | np.isclose(V0[..., 2], ez * h)
    assert np.all(d[on_boundary] == 0.0)
    # shared grid points move together (a conforming mesh)
    np.testing.assert_array_equal(V[0, 1], V[1, 0])
    np.testing.assert_array_equal(V[0, 7], V[ex * ey + ex + 1, 0])
    np.testing.assert_array_equal(V, inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0))


def test_parallelepiped_elements_are_affine_and_distinct():
    V = inputs.parallelepiped_vertices(3, 3, 2)
    x0 = V[:, 0]
    e1, e2, e3 = V[:, 1] - x0, V[:, 2] - x0, V[:, 4] - x0
    np.testing.assert_allclose(V[:, 3] - x0, e1 + e2, atol=1e-14)
    np.testing.assert_allclose(V[:, 5] - x0, e1 + e3, atol=1e-14)
    np.testing.assert_allclose(V[:, 6] - x0, e2 + e3, atol=1e-14)
    np.testing.assert_allclose(V[:, 7] - x0, e1 + e2 + e3, atol=1e-14)
    det = np.einsum("ei,ei->e", e1, np.cross(e2, e3))
    assert np.all(det > 0)
    J = np.stack([e1, e2, e3], axis=-1)
    assert len({tuple(np.round(j.ravel(), 12)) for j in J}) == J.shape[0]


@pytest.mark.parametrize("N", [3, 5, 7, 9, 11, 15])
def test_sweep_sizes(N):
    ex, ey, ez = inputs.sweep_box(N)
    dofs = ex * ey * ez * (N + 1) ** 3
    assert abs(dofs - 64 * 2 ** 20) <= 0.02 * 64 * 2 ** 20


def test_uneven_batch():
    spec = inputs.batch_meshes()
    assert len(spec) == 64 and spec == inputs.batch_meshes()
    E = np.array([ex * ey * ez for ex, ey, ez, _ in spec])
    Ns = {N for *_, N in spec}
    assert Ns <= {3, 5, 7, 9} and len(Ns) == 4
    assert E.min() >= 64 * 0.95 and E.max() <= 4096 * 1.05
    assert E.max() / E.min() > 16  # uneven


def test_global_numbering_and_mask():
    ex, ey, ez, N = 3, 2, 2, 3
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    assert ng == (ex * N + 1) * (ey * N + 1) * (ez * N + 1)
    assert np.array_equal(np.unique(gid), np.arange(ng))
    N1 = N + 1
    g = gid.reshape(-1, N1, N1, N1)  # [e][k][j][i]
    # the face i = N of element 0 is the face i = 0 of element 1
    np.testing.assert_array_equal(g[0, :, :, N], g[1, :, :, 0])
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    assert int(mask.sum()) == ng - (ex * N - 1) * (ey * N - 1) * (ez * N - 1)
