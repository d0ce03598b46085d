"""The learned preconditioner on the GPU: forward and gradients of the BF16
tensor-core MLP against the FP64 CPU oracle (oracle/mlp.py), training, and
the flexible PCG that uses the trained network against Jacobi-PCG."""
import numpy as np
import pytest

from paper_2504_07042_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
I, IP, H, O = 536, 544, 512, 512


@pytest.fixture(scope="module")
def ax():
    from paper_2504_07042_gb300 import build

    build.build()
    from paper_2504_07042_gb300 import ax as _ax

    return _ax


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _split(flat):
    o, out = 0, []
    for shape in ((H, IP), (H,), (H, H), (H,), (O, H), (O,)):
        n = int(np.prod(shape))
        out.append(flat[o:o + n].reshape(shape))
        o += n
    return out


def _setup(ax, seed=3, M=256):
    rng = np.random.default_rng(seed)
    mlp = ax.AxMLP(seed=11)
    p = mlp.ax_mlp_get_params()
    P = _split(p.astype(np.float64))
    # biases nonzero so every path is exercised
    P[1][:] = 0.1 * rng.standard_normal(H)
    P[3][:] = 0.1 * rng.standard_normal(H)
    P[5][:] = 0.1 * rng.standard_normal(O)
    flat = np.concatenate([q.reshape(-1) for q in P]).astype(np.float32)
    mlp.ax_mlp_set_params(flat)
    X = np.zeros((M, IP), dtype=np.float32)
    X[:, :I] = rng.uniform(-1, 1, (M, I))
    T = rng.standard_normal((M, O)).astype(np.float32)
    Xd = torch.from_numpy(X).to(DEV).to(torch.bfloat16)
    Td = torch.from_numpy(T).to(DEV)
    # what the oracle sees: bf16-rounded weights and inputs, float64 arithmetic
    Pq = [_bf16(P[0][:, :I]), P[1], _bf16(P[2]), P[3], _bf16(P[4]), P[5]]
    return mlp, Xd, Td, _bf16(X[:, :I]), T.astype(np.float64), Pq


U_BF16 = 2.0 ** -8  # unit roundoff of bfloat16 (8 significand bits)
GELU_LIP = 1.13  # max |gelu'|: a bound on how much gelu magnifies an error in its argument


def _rss(A, B):
    """Entry (i, j): sqrt(sum_m (A[m, i] B[m, j])^2), the root-sum-square size
    of the terms of (A^T B)[i, j].  Independent roundings of the terms leave
    an error of about u times this, while a wrong index, sign or dropped term
    moves the entry by about this much."""
    return np.sqrt((A * A).T @ (B * B))


def _scales(Pq, X, T):
    """Per-entry error scales of the forward output and the six gradients.
    Forward: each layer's pre-activation scale is the root-sum-square of its
    terms (plus the bias and what the layer's input already carries), and
    gelu magnifies it by at most GELU_LIP.  Backward: dY is at most
    (|Y| + |T|) / (M O) in size, and each back-propagated quantity gets the
    root-sum-square of its terms (times GELU_LIP through gelu'), so that an
    entry's scale is the size its terms give it, not a worst-case sum."""
    W1, b1, W2, b2, W3, b3 = Pq
    M, O = T.shape
    Z1 = np.sqrt((X * X) @ (W1 * W1).T) + np.abs(b1)
    H1 = GELU_LIP * Z1
    Z2 = np.sqrt((H1 * H1) @ (W2 * W2).T) + np.abs(b2)
    H2 = GELU_LIP * Z2
    Y = np.sqrt((H2 * H2) @ (W3 * W3).T) + np.abs(b3)
    dY = (Y + np.abs(T)) / (M * O)
    dZ2 = np.sqrt((dY * dY) @ (W3 * W3)) * GELU_LIP
    dZ1 = np.sqrt((dZ2 * dZ2) @ (W2 * W2)) * GELU_LIP
    return Y, [_rss(dZ1, X), np.sqrt((dZ1 * dZ1).sum(0)), _rss(dZ2, H1), np.sqrt((dZ2 * dZ2).sum(0)),
               _rss(dY, H2), np.sqrt((dY * dY).sum(0))]


def test_forward_matches_oracle(ax):
    from oracle import mlp as om

    mlp, Xd, Td, Xq, T, Pq = _setup(ax)
    Y = torch.empty((Xd.shape[0], O), dtype=torch.float32, device=DEV)
    mlp.ax_mlp_forward(Xd, Y)
    Yref, _ = om.forward(Pq, Xq)
    err = np.max(np.abs(Y.cpu().numpy() - Yref)) / np.max(np.abs(Yref))
    assert err < 2e-2  # bf16 hidden activations: ~2^-9 relative per rounding
    # element by element: every output within a few bf16 roundings of its own scale
    Ys, _ = _scales(Pq, Xq, np.zeros_like(Yref))
    ratio = np.abs(Y.cpu().numpy() - Yref) / (U_BF16 * Ys)
    print("forward: max |err| / (u * scale) = %.3f" % ratio.max())
    assert ratio.max() < 8.0


def test_gradients_match_oracle(ax):
    from oracle import mlp as om

    mlp, Xd, Td, Xq, T, Pq = _setup(ax, seed=5, M=256)
    loss, g = mlp.ax_mlp_grad(Xd, Td)
    Lref, gref = om.grads(Pq, Xq, T)
    assert abs(loss - Lref) / Lref < 1e-2
    G = _split(g.astype(np.float64))
    G[0] = G[0][:, :I]
    _, scales = _scales(Pq, Xq, T)
    for name, a, b, sc in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), G, gref, scales):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel < 5e-2 and cos > 0.998, (name, rel, cos)
        # element by element, against each entry's own error scale: a wrong row,
        # column or sign moves an entry by about its scale, bf16 roundings by ~u of it
        ratio = np.abs(a - b) / (U_BF16 * sc)
        print("%s: max |err| / (u * scale) = %.3f at %s" % (name, ratio.max(), np.unravel_index(ratio.argmax(), ratio.shape)))
        assert ratio.max() < 8.0, (name, ratio.max())
    # the padded input columns never receive gradient
    assert np.all(_split(g)[0][:, I:] == 0.0)


def test_training_reduces_loss(ax):
    rng = np.random.default_rng(8)
    mlp = ax.AxMLP(seed=1)
    n = 8192
    X = np.zeros((n, IP), dtype=np.float32)
    X[:, :I] = rng.uniform(-1, 1, (n, I))
    T = np.tanh(X[:, :O] * 1.5) * 0.5  # a smooth elementwise map the network can learn
    hist = mlp.ax_mlp_train(torch.from_numpy(X).to(DEV).to(torch.bfloat16), torch.from_numpy(T).to(DEV),
                            epochs=8, batch=512, lr=2e-3, seed=3)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.5 * hist[0], hist


def test_learned_pcg(ax, orc):
    from paper_2504_07042_gb300 import learned

    N, n = 7, 6
    V = inputs.box_vertices(n, n, n, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    Vd = torch.from_numpy(V).to(DEV)
    op = ax.Ax(Vd, N, "trilinear", "f64dw")
    op.gs_setup(torch.from_numpy(gid).to(DEV), ng, torch.from_numpy(mask).to(DEV))
    F, T = learned.collect_pairs(op, ng, seeds=range(100, 112), per_snapshot=n ** 3)
    assert F.shape[0] == 12 * 4 * n ** 3 and torch.isfinite(T).all()
    mlp = ax.AxMLP(seed=2)
    hist = mlp.ax_mlp_train(F, T, epochs=30, batch=512, lr=1e-3, seed=4)
    assert hist[-1] < 0.5 * hist[0]
    XYZ = learned.node_coords(op).cpu().numpy()
    f = torch.from_numpy(inputs.smooth_rhs(XYZ, 300)).to(DEV)
    b = learned.rhs_from_f(op, f, ng)
    xj = torch.zeros(ng, dtype=torch.float64, device=DEV)
    itj, rrj, stj = op.pcg_solve(b, xj, rtol=1e-8, maxit=5000, precond=1)
    xl = torch.zeros_like(xj)
    itl, rrl, stl, fb = ax.pcg_solve_learned(op, mlp, b, xl, rtol=1e-8, maxit=5000, omega=0.5)
    assert stj == ax.AX_OK and stl == ax.AX_OK and rrl <= 1e-8 and fb == 0
    d = float((xl - xj).abs().max()) / float(xj.abs().max())
    assert d < 1e-6
    print("learned flexible PCG: %d iterations, Jacobi-PCG: %d" % (itl, itj))
    assert itl < 0.9 * itj  # what the trained network gains over the method without it
    # an untrained network (zero output layer) is the Jacobi step: same iterations as Jacobi-PCG
    p = mlp.ax_mlp_get_params()
    p[512 * 544 + 512 + 512 * 512 + 512:] = 0.0
    mlp.ax_mlp_set_params(p)
    x0 = torch.zeros_like(xj)
    it0, _, st0, _ = ax.pcg_solve_learned(op, mlp, b, x0, rtol=1e-8, maxit=5000, omega=0.5)
    assert st0 == ax.AX_OK and abs(it0 - itj) <= 2
