"""Batched AxLocal and batched independent PCG solves over meshes of uneven
size and order, against the FP64 oracle mesh by mesh (AxLocal by Eq. 9,
Eq. 7 and Algorithm 1; PCG by the oracle's textbook Jacobi-PCG) and against
the per-mesh paths of the C ABI."""
import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ax():
    from paper_2504_07042_gb300 import build

    build.build()
    from paper_2504_07042_gb300 import ax as _ax

    return _ax


def _meshes():
    # uneven batch: orders and sizes mixed, orders repeated and out of order
    spec = [(3, 2, 2, 3), (2, 2, 1, 5), (4, 3, 2, 1), (2, 2, 2, 7), (1, 1, 1, 3), (3, 1, 1, 9), (2, 1, 1, 5)]
    out = []
    for s, (ex, ey, ez, N) in enumerate(spec):
        V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=s)
        gid, ng = inputs.box_global_ids(ex, ey, ez, N)
        mask = inputs.box_boundary_mask(ex, ey, ez, N)
        out.append((V, N, gid, ng, mask))
    return out


def _dev(meshes):
    return [(torch.from_numpy(V).to(DEV), N, torch.from_numpy(g).to(DEV), ng, torch.from_numpy(m).to(DEV))
            for V, N, g, ng, m in meshes]


# parity tolerances of each precision (relative max-norm against the FP64 oracle)
TOL = {"fp64": 1e-12, "f64dw": 1e-12, "fp32": 2e-5, "tf32": 4 * 2.0 ** -11, "fp16": 4 * 2.0 ** -11,
       "bf16": 4 * 2.0 ** -8}


@pytest.mark.parametrize("prec", ["fp32", "fp64", "f64dw", "tf32", "bf16", "fp16"])
def test_batch_local_matches_oracle(ax, orc, prec):
    meshes = _meshes()
    bt = ax.AxBatch(_dev(meshes), "trilinear", prec)
    Xh = np.random.default_rng(71).uniform(-1, 1, bt.n_local)
    X = torch.from_numpy(Xh).to(DEV, bt.dtype)
    Xh = X.double().cpu().numpy()  # the values the kernel sees
    for tuned in (False, True):
        if tuned:
            bt.ax_batch_tune()
        Y = torch.full_like(X, float("nan"))
        bt.ax_batch_local(X, Y)
        Yh = Y.double().cpu().numpy()
        for m, (V, N, gid, ng, mask) in enumerate(meshes):
            n3 = (N + 1) ** 3
            lo = bt.local_offsets[m]
            Xm = Xh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3)
            Yref, bad = orc.axlocal_vertices(V, Xm, N)
            assert bad == 0
            Ym = Yh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3)
            err = np.max(np.abs(Ym - Yref)) / np.max(np.abs(Yref))
            assert err <= TOL[prec], (m, N, tuned, err)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "f64dw", "tf32", "bf16"])
def test_batch_local_equals_per_mesh(ax, prec):
    meshes = _meshes()
    bt = ax.AxBatch(_dev(meshes), "trilinear", prec)
    X = torch.from_numpy(np.random.default_rng(70).uniform(-1, 1, bt.n_local)).to(DEV, bt.dtype)
    Y = torch.full_like(X, float("nan"))
    bt.ax_batch_local(X, Y)
    for tuned in (False, True):
        if tuned:
            choice = bt.ax_batch_tune()
            assert set(choice) == set(m[1] for m in meshes)
            Y = torch.full_like(X, float("nan"))
            bt.ax_batch_local(X, Y)
        for m, (V, N, gid, ng, mask) in enumerate(meshes):
            n = V.shape[0] * (N + 1) ** 3
            lo = bt.local_offsets[m]
            op = ax.Ax(torch.from_numpy(V).to(DEV), N, "trilinear", prec)
            Ym = torch.empty(n, dtype=bt.dtype, device=DEV)
            op.ax_local(X[lo:lo + n], Ym)
            assert torch.equal(Ym, Y[lo:lo + n]), (m, tuned)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("fp64", 1e-9)])
def test_batch_pcg_graph_vs_per_mesh(ax, orc, prec, tol):
    meshes = _meshes()
    bt = ax.AxBatch(_dev(meshes), "trilinear", prec)
    bt.ax_batch_tune()
    # right-hand sides: b = Q^T (w|J| f) per mesh, f = 3 pi^2 sin sin sin (oracle mass and gather)
    bvec = np.zeros(bt.n_global)
    for m, (V, N, gid, ng, mask) in enumerate(meshes):
        G, _ = orc.factors(V, N)
        XYZ = orc.nodal_coords(V, N)
        f = 3 * np.pi ** 2 * np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
        bvec[bt.global_offsets[m]:bt.global_offsets[m + 1]] = orc.gather(G[:, 6, :] * f + 0.1, gid, ng)
    bd = torch.from_numpy(bvec).to(DEV, bt.dtype)
    rtol = 1e-5 if prec == "fp32" else 1e-10
    x1 = torch.zeros_like(bd)
    it1, rr1, st1 = bt.ax_batch_pcg(bd, x1, rtol=rtol, maxit=5000, graph=1)
    x0 = torch.zeros_like(bd)
    it0, rr0, st0 = bt.ax_batch_pcg(bd, x0, rtol=rtol, maxit=5000, graph=0)
    assert st1 == ax.AX_OK and st0 == ax.AX_OK
    assert all(r <= rtol for r in rr1)
    for m in range(bt.B):
        a, b = bt.global_offsets[m], bt.global_offsets[m + 1]
        d = float((x1[a:b] - x0[a:b]).abs().max()) / float(x0[a:b].abs().max())
        assert d <= tol, (m, d)
        assert abs(it1[m] - it0[m]) <= 2, (m, it1[m], it0[m])


@pytest.mark.parametrize("prec,rtol,tol", [("fp32", 1e-5, 1e-4), ("fp64", 1e-10, 1e-8), ("f64dw", 1e-10, 1e-8)])
def test_batch_pcg_matches_oracle(ax, orc, prec, rtol, tol):
    # each mesh's solution against the oracle's Jacobi-PCG of the same mesh and
    # right-hand side (built by the oracle), solved to 1e-13; the tolerance is
    # what stopping at rtol leaves (the oracle itself, stopped at 1e-5 and
    # 1e-10 on these meshes, is 1e-6 to 5e-6 and 1e-11 to 2e-11 away)
    meshes = _meshes()
    bt = ax.AxBatch(_dev(meshes), "trilinear", prec)
    bvec = np.zeros(bt.n_global)
    xref = []
    for m, (V, N, gid, ng, mask) in enumerate(meshes):
        G, _ = orc.factors(V, N)
        XYZ = orc.nodal_coords(V, N)
        f = 3 * np.pi ** 2 * np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
        b = orc.gather(G[:, 6, :] * f + 0.1, gid, ng)
        bvec[bt.global_offsets[m]:bt.global_offsets[m + 1]] = b
        x, it, rr, ok = orc.pcg(G, gid, ng, mask, b, N, rtol=1e-13, maxit=5000)
        assert ok
        xref.append(x)
    bd = torch.from_numpy(bvec).to(DEV, bt.dtype)
    x = torch.zeros_like(bd)
    it, rr, st = bt.ax_batch_pcg(bd, x, rtol=rtol, maxit=5000, graph=1)
    assert st == ax.AX_OK and all(r <= rtol for r in rr)
    xh = x.double().cpu().numpy()
    for m in range(bt.B):
        a, b = bt.global_offsets[m], bt.global_offsets[m + 1]
        d = np.max(np.abs(xh[a:b] - xref[m])) / np.max(np.abs(xref[m]))
        assert d <= tol, (m, d)


def _c4_like():
    # orders 3, 5, 7, 9 interleaved, sizes uneven (the persistent kernel's case)
    spec = [(3, 3, 2, 5), (2, 2, 2, 9), (4, 4, 4, 3), (1, 2, 3, 7), (2, 3, 3, 5), (5, 4, 3, 3), (2, 2, 1, 9),
            (3, 3, 3, 7)]
    out = []
    for s, (ex, ey, ez, N) in enumerate(spec):
        V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=10 + s)
        gid, ng = inputs.box_global_ids(ex, ey, ez, N)
        mask = inputs.box_boundary_mask(ex, ey, ez, N)
        out.append((V, N, gid, ng, mask))
    return out


@pytest.mark.parametrize("kind", ["trilinear", "stored", "parallelepiped", "partial"])
def test_persistent_local_one_launch(ax, orc, kind):
    # FP32 batch of orders 3..9: AxLocal is one launch; it equals the launch-per-order
    # path bit for bit (same per-element arithmetic) and the oracle per mesh
    meshes = _c4_like()
    if kind == "parallelepiped":  # affine elements: the sheared parallelepiped boxes
        meshes = []
        for ex, ey, ez, N in [(3, 3, 2, 5), (2, 2, 2, 9), (4, 4, 4, 3), (1, 2, 3, 7)]:
            V = inputs.parallelepiped_vertices(ex, ey, ez)
            gid, ng = inputs.box_global_ids(ex, ey, ez, N)
            meshes.append((V, N, gid, ng, inputs.box_boundary_mask(ex, ey, ez, N)))
    bt = ax.AxBatch(_dev(meshes), kind, "fp32")
    info = bt.ax_batch_info()
    assert info == {"persistent": 1, "local_launches": 1, "iteration_launches": 1}
    X = torch.from_numpy(np.random.default_rng(72).uniform(-1, 1, bt.n_local)).to(DEV, torch.float32)
    Yp = torch.full_like(X, float("nan"))
    bt.ax_batch_local(X, Yp)
    bt.ax_batch_tune()
    Yt = torch.full_like(X, float("nan"))
    bt.ax_batch_local(X, Yt)
    bt.ax_batch_set_persistent(False)
    assert bt.ax_batch_info()["local_launches"] == len(set(m[1] for m in meshes))
    Yg = torch.full_like(X, float("nan"))
    bt.ax_batch_local(X, Yg)
    assert torch.equal(Yp, Yg) and torch.equal(Yt, Yg)
    Xh, Yh = X.double().cpu().numpy(), Yp.double().cpu().numpy()
    for m, (V, N, gid, ng, mask) in enumerate(meshes):
        n3 = (N + 1) ** 3
        lo = bt.local_offsets[m]
        Yref, _ = orc.axlocal_vertices(V, Xh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3), N)
        err = np.max(np.abs(Yh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3) - Yref)) / np.max(np.abs(Yref))
        assert err <= TOL["fp32"], (m, err)


def _c4_rhs(orc, bt, meshes):
    bvec = np.zeros(bt.n_global)
    xref = []
    for m, (V, N, gid, ng, mask) in enumerate(meshes):
        G, _ = orc.factors(V, N)
        XYZ = orc.nodal_coords(V, N)
        f = 3 * np.pi ** 2 * np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
        b = orc.gather(G[:, 6, :] * f + 0.1, gid, ng)
        bvec[bt.global_offsets[m]:bt.global_offsets[m + 1]] = b
        x, it, rr, ok = orc.pcg(G, gid, ng, mask, b, N, rtol=1e-13, maxit=5000)
        assert ok
        xref.append(x)
    return bvec, xref


def test_persistent_pcg_matches_oracle(ax, orc):
    # one persistent launch per CG iteration (scatter fused into the AxLocal
    # load, per-mesh bounded waits between the phases): every mesh's solution
    # against the oracle's solve
    meshes = _c4_like()
    bt = ax.AxBatch(_dev(meshes), "trilinear", "fp32")
    bt.ax_batch_tune()
    bvec, xref = _c4_rhs(orc, bt, meshes)
    bd = torch.from_numpy(bvec).to(DEV, torch.float32)
    x = torch.zeros_like(bd)
    it, rr, st = bt.ax_batch_pcg(bd, x, rtol=1e-5, maxit=5000, graph=1)
    assert st == ax.AX_OK and all(r <= 1e-5 for r in rr)
    xh = x.double().cpu().numpy()
    for m in range(bt.B):
        a, b = bt.global_offsets[m], bt.global_offsets[m + 1]
        d = np.max(np.abs(xh[a:b] - xref[m])) / np.max(np.abs(xref[m]))
        assert d <= 1e-4, (m, d)
    # the grouped launches take the same iterations within a couple
    bt.ax_batch_set_persistent(False)
    x2 = torch.zeros_like(bd)
    it2, rr2, st2 = bt.ax_batch_pcg(bd, x2, rtol=1e-5, maxit=5000, graph=1)
    assert st2 == ax.AX_OK and all(abs(a - b) <= 2 for a, b in zip(it, it2))


def test_persistent_wait_times_out(ax, orc):
    # a dependency nothing completes (the test hook) with a 1 ms budget: the
    # solve stops with AX_ETIMEOUT instead of hanging; afterwards the batch
    # solves normally
    meshes = _c4_like()
    bt = ax.AxBatch(_dev(meshes), "trilinear", "fp32")
    bvec, xref = _c4_rhs(orc, bt, meshes)
    bd = torch.from_numpy(bvec).to(DEV, torch.float32)
    bt.ax_batch_set_wait(1_000_000, stuck_mesh=2)
    x = torch.zeros_like(bd)
    it, rr, st = bt.ax_batch_pcg(bd, x, rtol=1e-5, maxit=200, graph=1, check=False)
    assert st == ax.AX_ETIMEOUT
    bt.ax_batch_set_wait(2_000_000_000, stuck_mesh=-1)
    x = torch.zeros_like(bd)
    it, rr, st = bt.ax_batch_pcg(bd, x, rtol=1e-5, maxit=5000, graph=1)
    assert st == ax.AX_OK
    xh = x.double().cpu().numpy()
    for m in range(bt.B):
        a, b = bt.global_offsets[m], bt.global_offsets[m + 1]
        assert np.max(np.abs(xh[a:b] - xref[m])) <= 1e-4 * np.max(np.abs(xref[m]))
    with pytest.raises(ax.AxError) as ei:
        bt.ax_batch_set_wait(0)
    assert ei.value.status == ax.AX_EINVAL


def test_persistent_unsupported(ax):
    meshes = _c4_like()
    bt = ax.AxBatch(_dev(meshes), "trilinear", "f64dw")
    assert bt.ax_batch_info()["persistent"] == 0
    with pytest.raises(ax.AxError) as ei:
        bt.ax_batch_set_persistent(True)
    assert ei.value.status == ax.AX_EUNSUPPORTED


@pytest.mark.parametrize("kind", ["trilinear", "partial"])
def test_persistent_every_order(ax, orc, kind):
    # one batch with every order the persistent kernel carries (N = 1..9,
    # N1 = 2..10: the CTA's idle threads and each order's shape), one launch
    spec = [(2, 2, 2, N) for N in (9, 1, 8, 2, 7, 3, 6, 4, 5)] + [(2, 2, 3, 9), (3, 2, 2, 2)]
    meshes = []
    for s, (ex, ey, ez, N) in enumerate(spec):
        V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=40 + s)
        gid, ng = inputs.box_global_ids(ex, ey, ez, N)
        meshes.append((V, N, gid, ng, inputs.box_boundary_mask(ex, ey, ez, N)))
    bt = ax.AxBatch(_dev(meshes), kind, "fp32")
    assert bt.ax_batch_info()["local_launches"] == 1
    X = torch.from_numpy(np.random.default_rng(73).uniform(-1, 1, bt.n_local)).to(DEV, torch.float32)
    Y = torch.full_like(X, float("nan"))
    bt.ax_batch_local(X, Y)
    Xh, Yh = X.double().cpu().numpy(), Y.double().cpu().numpy()
    for m, (V, N, gid, ng, mask) in enumerate(meshes):
        n3 = (N + 1) ** 3
        lo = bt.local_offsets[m]
        Yref, _ = orc.axlocal_vertices(V, Xh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3), N)
        err = np.max(np.abs(Yh[lo:lo + V.shape[0] * n3].reshape(V.shape[0], n3) - Yref)) / np.max(np.abs(Yref))
        assert err <= TOL["fp32"], (m, N, err)
    bvec, xref = _c4_rhs(orc, bt, meshes)
    bd = torch.from_numpy(bvec).to(DEV, torch.float32)
    x = torch.zeros_like(bd)
    it, rr, st = bt.ax_batch_pcg(bd, x, rtol=1e-5, maxit=5000, graph=1)
    assert st == ax.AX_OK
    xh = x.double().cpu().numpy()
    for m in range(bt.B):
        a, b = bt.global_offsets[m], bt.global_offsets[m + 1]
        assert np.max(np.abs(xh[a:b] - xref[m])) <= 1e-4 * np.max(np.abs(xref[m])), m
