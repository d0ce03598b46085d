"""GPU parity of gather-scatter (Eq. 1), the lumped mass, element diagonals
and (P)CG against the CPU oracle, through the C ABI."""
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


def _ctx(ax, V, N, kind, prec, gid=None, ng=None, mask=None):
    op = ax.Ax(torch.from_numpy(V).to(DEV), N, kind, prec)
    if gid is not None:
        m = None if mask is None else torch.from_numpy(mask).to(DEV)
        op.gs_setup(torch.from_numpy(gid).to(DEV), ng, m)
    return op


def _manufactured(orc, V, G, gid, ng, N):
    XYZ = orc.nodal_coords(V, N)
    u = np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
    f = 3 * np.pi ** 2 * u
    u_g = np.zeros(ng)
    u_g[gid.reshape(-1)] = u.reshape(-1)
    return f, u_g


@pytest.mark.parametrize("prec", ["fp64", "f64dw", "fp32"])
def test_gs_assemble_gather_scatter(ax, orc, prec):
    N = 4
    ex, ey, ez = 3, 2, 2
    V = inputs.box_vertices(ex, ey, ez)
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    op = _ctx(ax, V, N, "trilinear", prec, gid, ng, mask)
    dt = op.dtype
    rng = np.random.default_rng(60)
    Y = rng.standard_normal(gid.shape)
    u = rng.standard_normal(ng)
    Yd = torch.from_numpy(Y).to(DEV, dt)
    tol = 0.0 if dt == torch.float64 else 1e-6
    # Q Q^T Y
    Ya = op.gs_assemble(Yd.clone()).double().cpu().numpy()
    ref = orc.gs(Y.astype(np.float32).astype(np.float64) if tol else Y, gid, ng)
    assert np.max(np.abs(Ya - ref)) <= tol * np.abs(ref).max()
    # Q^T Y, masked
    yg = op.gs_gather(Yd, torch.empty(ng, dtype=dt, device=DEV)).double().cpu().numpy()
    refg = orc.gather(Y.astype(np.float32).astype(np.float64) if tol else Y, gid, ng)
    refg[mask == 1] = 0.0
    assert np.max(np.abs(yg - refg)) <= tol * np.abs(refg).max()
    # Q u
    U = op.gs_scatter(torch.from_numpy(u).to(DEV, dt), torch.empty(gid.shape, dtype=dt, device=DEV))
    refU = orc.scatter(u, gid)
    assert np.max(np.abs(U.double().cpu().numpy() - refU)) <= tol * np.abs(refU).max()


@pytest.mark.parametrize("kind", ["stored", "trilinear", "parallelepiped"])
def test_mass_and_diagonal(ax, orc, kind):
    N = 4
    V = inputs.parallelepiped_vertices(3, 2, 1) if kind == "parallelepiped" else inputs.box_vertices(3, 2, 1)
    G, _ = orc.factors(V, N)
    op = _ctx(ax, V, N, kind, "fp64")
    F = inputs.element_vectors(V.shape[0], N, seed=61)
    M = op.ax_mass(torch.from_numpy(F).to(DEV), torch.empty(F.shape, dtype=torch.float64, device=DEV)).cpu().numpy()
    ref = G[:, 6, :] * F
    assert np.max(np.abs(M - ref)) <= 1e-14 * np.abs(ref).max()
    d = op.ax_diag(torch.empty(F.shape, dtype=torch.float64, device=DEV)).cpu().numpy()
    dref = orc.element_diagonals(G, N)
    assert np.max(np.abs(d - dref)) <= 1e-13 * np.abs(dref).max()


@pytest.mark.parametrize("prec", ["fp64", "f64dw"])
@pytest.mark.parametrize("kind", ["stored", "trilinear", "partial"])
def test_pcg_matches_oracle(ax, orc, kind, prec):
    N = 5
    ex, ey, ez = 3, 3, 3
    V = inputs.box_vertices(ex, ey, ez)
    G, _ = orc.factors(V, N)
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    f, u = _manufactured(orc, V, G, gid, ng, N)
    b = orc.gather(G[:, 6, :] * f, gid, ng)
    dg = orc.gather(orc.element_diagonals(G, N), gid, ng)
    x_ref, it_ref, _, ok = orc.pcg(G, gid, ng, mask, b, N, diag_global=dg, rtol=1e-12, maxit=2000)
    assert ok
    op = _ctx(ax, V, N, kind, prec, gid, ng, mask)
    # the right-hand side is built on the GPU too: b = Q^T (w|J| f)
    Fd = torch.from_numpy(f).to(DEV)
    bl = op.ax_mass(Fd, torch.empty_like(Fd))
    bd = op.gs_gather(bl, torch.empty(ng, dtype=torch.float64, device=DEV))
    assert np.max(np.abs(bd.cpu().numpy() - np.where(mask == 1, 0.0, b))) <= 1e-13 * np.abs(b).max()
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    it, rr, st = op.pcg_solve(bd, x, rtol=1e-12, maxit=2000, precond=1)
    assert st == ax.AX_OK and rr <= 1e-12
    x = x.cpu().numpy()
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.abs(x_ref).max()
    assert abs(it - it_ref) <= 2
    assert np.max(np.abs(x - u)) < 1e-3  # the discretisation error of this coarse mesh


def test_pcg_statuses(ax, orc):
    N = 3
    ex, ey, ez = 2, 2, 2
    V = inputs.box_vertices(ex, ey, ez)
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    op = _ctx(ax, V, N, "trilinear", "fp64", gid, ng, mask)
    b = torch.from_numpy(np.random.default_rng(62).uniform(-1, 1, ng)).to(DEV)
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    it, rr, st = op.pcg_solve(b, x, rtol=1e-14, maxit=1, precond=1)
    assert st == ax.AX_ENOTCONV and it == 1
    x.zero_()
    it, rr, st = op.pcg_solve(torch.zeros_like(b), x, rtol=1e-10, maxit=10)
    assert st == ax.AX_OK and it == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(ax.AxError) as ei:  # the learned preconditioner has its own entry point
        op.pcg_solve(b, x, rtol=1e-8, maxit=10, precond=2)
    assert ei.value.status == ax.AX_EINVAL and "pcg_solve_learned" in str(ei.value)
    with pytest.raises(ax.AxError) as ei:
        op.pcg_solve(b, x, rtol=1e-8, maxit=10, precond=3)
    assert ei.value.status == ax.AX_EUNSUPPORTED
    with pytest.raises(ax.AxError) as ei:
        op.gs_setup(torch.from_numpy(gid + ng).to(DEV), ng)
    assert ei.value.status == ax.AX_EINVAL


def test_c3_poisson_to_1e8(ax, orc):
    # 16^3 perturbed trilinear elements at N = 7 (2.1M local, 1.37M unknowns)
    N, n = 7, 16
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    op = _ctx(ax, V, N, "trilinear", "f64dw", gid, ng, mask)
    XYZ = torch.empty((V.shape[0], 3, (N + 1) ** 3), dtype=torch.float64, device=DEV)
    op.ax_node_coords(XYZ)
    u = torch.sin(np.pi * XYZ[:, 0]) * torch.sin(np.pi * XYZ[:, 1]) * torch.sin(np.pi * XYZ[:, 2])
    bl = op.ax_mass(3 * np.pi ** 2 * u, torch.empty_like(u))
    b = op.gs_gather(bl, torch.empty(ng, dtype=torch.float64, device=DEV))
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    it, rr, st = op.pcg_solve(b, x, rtol=1e-8, maxit=5000, precond=1)
    assert st == ax.AX_OK and rr <= 1e-8
    ug = torch.zeros(ng, dtype=torch.float64, device=DEV)
    ug[torch.from_numpy(gid.reshape(-1)).to(DEV)] = u.reshape(-1)
    assert float((x - ug).abs().max()) < 1e-6
