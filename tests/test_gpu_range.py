"""Number range of the FP64-accurate double-word AxLocal (float64 in HBM,
float32 pairs in the arithmetic): X anywhere in float64's range and meshes
scaled far from unit size, against the FP64 oracle (Eq. 9, Eq. 7,
Algorithm 1) at the 1e-12 tolerance; element sizes outside what the float32
pairs carry are refused at setup with AX_ERANGE."""
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


def _run(ax, V, X, N, kind, prec):
    op = ax.Ax(torch.from_numpy(V).to(DEV), N, kind, prec)
    Xd = torch.from_numpy(X).to(DEV)
    Yd = torch.full_like(Xd, float("nan"))
    op.ax_local(Xd, Yd)
    torch.cuda.synchronize()
    op.ax_destroy()
    return Yd.cpu().numpy()


def _mesh(kind, n=3, scale=1.0):
    V = inputs.parallelepiped_vertices(n, n, n) if kind == "parallelepiped" else inputs.box_vertices(n, n, n, 0.1, 0)
    return V * scale


@pytest.mark.parametrize("xscale", [1e30, 1e-30, 1e300, 1e-300, 2.0 ** 61, 2.0 ** -61])
@pytest.mark.parametrize("kind", ["stored", "trilinear", "parallelepiped", "partial"])
@pytest.mark.parametrize("prec", ["f64dw", "fp64"])
def test_x_scaled(ax, orc, kind, prec, xscale):
    # every element's X far outside float32's range: the double-word kernel
    # scales each element by a power of two on the way in and back on the way out
    N = 5
    V = _mesh(kind)
    X = inputs.element_vectors(V.shape[0], N, seed=1) * xscale
    Y = _run(ax, V, X, N, kind, prec)
    Yref, bad = orc.axlocal_vertices(V, X, N)
    assert bad == 0
    assert np.isfinite(Y).all()
    assert np.max(np.abs(Y - Yref)) <= 1e-12 * np.max(np.abs(Yref))


@pytest.mark.parametrize("kind", ["trilinear", "stored"])
def test_x_mixed_scales_per_element(ax, orc, kind):
    # elements of very different magnitude in one launch (some 1e-200, some
    # 1e200, one all zero, one with a few tiny entries): each element's Y holds
    # 1e-12 relative to its own largest value
    N = 7
    V = _mesh(kind, n=4)
    E = V.shape[0]
    X = inputs.element_vectors(E, N, seed=2)
    s = 10.0 ** np.random.default_rng(3).integers(-200, 200, E)
    X *= s[:, None]
    X[5] = 0.0
    X[6, :7] *= 1e-250
    Y = _run(ax, V, X, N, kind, "f64dw")
    Yref, _ = orc.axlocal_vertices(V, X, N)
    for e in range(E):
        m = np.max(np.abs(Yref[e]))
        if m == 0.0:
            assert np.all(Y[e] == 0.0)
        else:
            assert np.max(np.abs(Y[e] - Yref[e])) <= 1e-12 * m, e


@pytest.mark.parametrize("N", [5, 7, 15])
def test_x_entries_below_direct_conversion(ax, orc, N):
    # elements of magnitude 2^-58 with single entries near 2^-76 and 2^-72:
    # the main kernel converts X to float pairs by integer instructions down
    # to 2^-74 only; an entry below that sends its block through the scaled
    # pass (were it flushed to zero, Y would be off by about 2^-18 relative)
    V = _mesh("trilinear", n=3)
    E = V.shape[0]
    X = inputs.element_vectors(E, N, seed=4) * 2.0 ** -58
    rng = np.random.default_rng(5)
    for e in range(E):
        idx = rng.choice(X.shape[1], 6, replace=False)
        X[e, idx] = 2.0 ** rng.choice([-76.0, -72.0], 6) * rng.uniform(1.0, 2.0, 6) * rng.choice([-1.0, 1.0], 6)
    Y = _run(ax, V, X, N, "trilinear", "f64dw")
    Yref, _ = orc.axlocal_vertices(V, X, N)
    for e in range(E):
        assert np.max(np.abs(Y[e] - Yref[e])) <= 1e-12 * np.max(np.abs(Yref[e])), e


@pytest.mark.parametrize("mscale", [1e-4, 1e-5, 1e7])
@pytest.mark.parametrize("kind", ["stored", "trilinear", "parallelepiped", "partial"])
@pytest.mark.parametrize("N", [3, 7])
def test_mesh_scaled(ax, orc, kind, N, mscale):
    # element extents from about 3e-6 to 3e6 (inside [2^-20, 2^24])
    V = _mesh(kind, scale=mscale)
    X = inputs.element_vectors(V.shape[0], N, seed=1)
    Y = _run(ax, V, X, N, kind, "f64dw")
    Yref, bad = orc.axlocal_vertices(V, X, N)
    assert bad == 0
    assert np.max(np.abs(Y - Yref)) <= 1e-12 * np.max(np.abs(Yref))


@pytest.mark.parametrize("mscale", [1e-7, 1e9])
@pytest.mark.parametrize("prec", ["f64dw", "fp32", "tf32"])
def test_mesh_out_of_range_refused(ax, orc, prec, mscale):
    # element extents of about 3e-8 and 3e8: refused for the FP32-based
    # precisions; native FP64 takes them and still matches the oracle
    N = 3
    V = _mesh("trilinear", scale=mscale)
    with pytest.raises(ax.AxError) as ei:
        ax.Ax(torch.from_numpy(V).to(DEV), N, "trilinear", prec)
    assert ei.value.status == ax.AX_ERANGE
    X = inputs.element_vectors(V.shape[0], N, seed=1)
    Y = _run(ax, V, X, N, "trilinear", "fp64")
    Yref, _ = orc.axlocal_vertices(V, X, N)
    assert np.max(np.abs(Y - Yref)) <= 1e-12 * np.max(np.abs(Yref))
