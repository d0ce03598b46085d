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


_SOLVES = {}


def _oracle_solution(orc, V, N, gid, ng, mask, rtol=1e-13):
    """The oracle's own solve of -lap u = 3 pi^2 sin sin sin: its factors
    (Eq. 7), nodal coordinates, GLL-collocated mass and gather build b.
    Cached per mesh (the C3 solve takes tens of seconds on the host)."""
    key = (V.shape[0], N, rtol, float(V.sum()))
    if key in _SOLVES:
        return _SOLVES[key]
    G, _ = orc.factors(V, N)
    XYZ = orc.nodal_coords(V, N)
    f = 3 * np.pi ** 2 * np.sin(np.pi * XYZ[:, 0]) * np.sin(np.pi * XYZ[:, 1]) * np.sin(np.pi * XYZ[:, 2])
    b = orc.gather(G[:, 6, :] * f, gid, ng)
    x, it, rr, ok = orc.pcg(G, gid, ng, mask, b, N, rtol=rtol, maxit=5000)
    assert ok
    _SOLVES[key] = x
    return x


@pytest.mark.parametrize("lo_prec", ["fp32", "tf32", "bf16", "fp16"])
@pytest.mark.parametrize("hi_prec", ["fp64", "f64dw"])
@pytest.mark.parametrize("kind", ["stored", "trilinear"])
def test_mixed_matches_oracle(ax, orc, kind, hi_prec, lo_prec):
    # FP64 refinement around an inner CG whose AxLocal contracts in FP32 or on
    # the tensor cores (TF32/BF16/FP16 operands, FP32 accumulation): the
    # refined solution matches the oracle's FP64 solve
    N, n = 5, 3
    V = inputs.box_vertices(n, n, n)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    x_ref = _oracle_solution(orc, V, N, gid, ng, mask)
    hi, lo = _pair(ax, V, N, kind, hi_prec, gid, ng, mask, lo_prec)
    b, _ = _rhs_gpu(hi, V, N, ng)
    x = torch.zeros(ng, dtype=torch.float64, device=DEV)
    inner_rtol = 1e-3 if lo_prec == "fp32" else 1e-2
    outer, inner, rr, st = hi.pcg_solve_mixed(lo, b, x, rtol=1e-12, inner_rtol=inner_rtol, max_outer=100)
    assert st == ax.AX_OK and rr <= 1e-12
    assert outer >= 2  # the inner precision alone cannot reach 1e-12: refinement steps were needed
    x = x.cpu().numpy()
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.abs(x_ref).max()


def test_mixed_c3_to_1e10(ax, orc):
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
    # both against the oracle's FP64 solve of the C3 problem (to 1e-12)
    x_ref = torch.from_numpy(_oracle_solution(orc, V, N, gid, ng, mask, rtol=1e-12)).to(DEV)
    nrm = float(x_ref.abs().max())
    e64 = float((x64 - x_ref).abs().max()) / nrm
    emx = float((x - x_ref).abs().max()) / nrm
    print("C3 error vs oracle solve: FP64 PCG %.2e, mixed (FP32 inner) %.2e" % (e64, emx))
    assert e64 < 1e-8 and emx < 1e-8


@pytest.mark.parametrize("lo_prec", ["tf32", "bf16", "fp16"])
def test_mixed_tensor_core_inner_c3(ax, orc, lo_prec):
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
    # the C3 error against the oracle's FP64 solve
    x_ref = torch.from_numpy(_oracle_solution(orc, V, N, gid, ng, mask, rtol=1e-12)).to(DEV)
    err = float((x - x_ref).abs().max()) / float(x_ref.abs().max())
    print("%s inner: C3 error vs oracle solve %.2e" % (lo_prec, err))
    assert err < 1e-8


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
