"""Pins for the oracle's gather-scatter (Eq. 1: Q^T and Q) and the structured
box numbering that feeds it.

Fixed by: the (E, N, unique nodes) = (3, 4, 325) example of Fig. 1; node
multiplicities of a structured box (1 inside an element, 2 on faces, 4 on
edges, 8 at corners); adjointness <Q^T y, u> = <y, Q u>.
"""
import os

import numpy as np

from paper_2504_07042_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fig1_node_count():
    vals = {}
    for line in open(os.path.join(GOLDEN, "gs_count.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = int(v)
    gid, n_global = inputs.box_global_ids(vals["E"], 1, 1, vals["N"])
    assert n_global == vals["n_global"]
    assert len(np.unique(gid)) == vals["n_global"]


def test_multiplicities(orc):
    N = 3
    gid, ng = inputs.box_global_ids(2, 2, 2, N)
    mult = orc.gs(np.ones(gid.shape), gid, ng)
    counts = np.bincount(mult.reshape(-1).astype(int))
    n3 = (N + 1) ** 3
    # centre lattice point shared by all 8 elements: 8 local copies carry 8
    assert counts[8] == 8
    # every local node's multiplicity equals the number of elements touching it
    assert set(np.unique(mult)) == {1.0, 2.0, 4.0, 8.0}
    assert mult.size == 8 * n3


def test_adjoint_and_idempotence(orc):
    N = 4
    gid, ng = inputs.box_global_ids(3, 2, 1, N)
    rng = np.random.default_rng(40)
    Yl = rng.standard_normal(gid.shape)
    ug = rng.standard_normal(ng)
    lhs = orc.gather(Yl, gid, ng) @ ug
    rhs = np.sum(Yl * orc.scatter(ug, gid))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # Q Q^T y equals scatter(gather(y))
    np.testing.assert_allclose(orc.gs(Yl, gid, ng), orc.scatter(orc.gather(Yl, gid, ng), gid), rtol=1e-15)


def test_local_node_coordinates_agree_across_elements(orc):
    # nodes with the same global id have the same physical coordinates
    N = 3
    V = inputs.box_vertices(3, 2, 2, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(3, 2, 2, N)
    XYZ = orc.nodal_coords(V, N)
    for c in range(3):
        xc = XYZ[:, c, :]
        mult = orc.gs(np.ones(gid.shape), gid, ng)
        avg = orc.gs(xc, gid, ng) / mult
        assert np.max(np.abs(avg - xc)) < 1e-14
