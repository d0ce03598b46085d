"""Mixed-precision solve (FP64 iterative refinement around a float32 inner
Jacobi-PCG) against the FP64 oracle PCG and the FP64 GPU PCG."""
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


def _pair(ax, V, N, kind, hi_prec, gid, ng, mask, lo_prec="fp32"):
    Vd = torch.from_numpy(V).to(DEV)
    hi = ax.Ax(Vd, N, kind, hi_prec)
    hi.gs_setup(torch.from_numpy(gid).to(DEV), ng, torch.from_numpy(mask).to(DEV))
    lo = ax.Ax(Vd, N, kind, lo_prec)
    return hi, lo


def _rhs_gpu(op, V, N, ng):
    XYZ = torch.empty((V.shape[0], 3, (N + 1) ** 3), dtype=torch.float64, device=DEV)
    op.ax_node_coords(XYZ)
    u = torch.sin(np.pi * XYZ[:, 0]) * torch.sin(np.pi * XYZ[:, 1]) * torch.sin(np.pi * XYZ[:, 2])
    bl = op.ax_mass(3 * np.pi ** 2 * u, torch.empty_like(u))
    return op.gs_gather(bl, torch.empty(ng, dtype=torch.float64, device=DEV)), u


@pytest.mark.parametrize("hi_prec", ["fp64", "f64dw"])
@pytest.mark.parametrize("kind", ["stored", "trilinear"])
def test_mixed_matches_oracle(ax, orc, kind, hi_prec):
    N, n = 5, 3
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    G, _ = orc.factors(V, N)
    hi, lo = _pair(ax, V, N, kind, hi_prec, gid, ng, mask)
    b, _ = _rhs_gpu(hi, V, N, ng)
    x_ref, _, _, ok = orc.pcg(G, gid, ng, mask, b.cpu().numpy(), N, rtol=1e-13, maxit=5000)
    assert ok
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    outer, inner, rr, st = hi.pcg_solve_mixed(lo, b, x, rtol=1e-12, inner_rtol=1e-3)
    assert st == ax.AX_OK and rr <= 1e-12
    assert outer >= 2  # float32 alone cannot reach 1e-12: refinement steps were needed
    x = x.cpu().numpy()
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.abs(x_ref).max()


def test_mixed_c3_to_1e10(ax):
    # 16^3 perturbed trilinear elements at N = 7: refinement to 1e-10, against FP64 PCG to 1e-10
    N, n = 7, 16
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    hi, lo = _pair(ax, V, N, "trilinear", "f64dw", gid, ng, mask)
    b, u = _rhs_gpu(hi, V, N, ng)
    x64 = torch.zeros(ng, dtype=torch.float64, device=DEV)
    it, rr64, st = hi.pcg_solve(b, x64, rtol=1e-10, maxit=10000, precond=1)
    assert st == ax.AX_OK
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    outer, inner, rr, st = hi.pcg_solve_mixed(lo, b, x, rtol=1e-10, inner_rtol=1e-3)
    assert st == ax.AX_OK and rr <= 1e-10
    diff = float((x - x64).abs().max()) / float(x64.abs().max())
    assert diff < 1e-8


@pytest.mark.parametrize("lo_prec", ["tf32", "bf16", "fp16"])
def test_mixed_tensor_core_inner_c3(ax, lo_prec):
    # inner CG with tensor-core contractions (FP32 accumulation), FP64 refinement to 1e-10:
    # the refinement removes the inner operator's error; the answer matches FP64 PCG
    N, n = 7, 16
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    hi, lo = _pair(ax, V, N, "trilinear", "f64dw", gid, ng, mask, lo_prec)
    b, u = _rhs_gpu(hi, V, N, ng)
    x64 = torch.zeros(ng, dtype=torch.float64, device=DEV)
    it, rr64, st = hi.pcg_solve(b, x64, rtol=1e-10, maxit=10000, precond=1)
    assert st == ax.AX_OK
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    outer, inner, rr, st = hi.pcg_solve_mixed(lo, b, x, rtol=1e-10, inner_rtol=1e-2, max_outer=100)
    print("%s: outer %d inner %d relres %.2e" % (lo_prec, outer, inner, rr))
    assert st == ax.AX_OK and rr <= 1e-10
    diff = float((x - x64).abs().max()) / float(x64.abs().max())
    assert diff < 1e-8


def test_mixed_rejects_bad_pairs(ax):
    N, n = 3, 2
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    hi, lo = _pair(ax, V, N, "trilinear", "fp64", gid, ng, mask)
    b = torch.ones(ng, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    with pytest.raises(ax.AxError) as ei:
        lo.pcg_solve_mixed(hi, b, x)  # roles swapped
    assert ei.value.status == ax.AX_EINVAL
    o, i, rr, st = hi.pcg_solve_mixed(lo, b, x, rtol=1e-14, inner_rtol=1e-1, max_outer=1)
    assert st == ax.AX_ENOTCONV and o == 1
