"""Launch one AxLocal case a few times (for ncu captures and quick timing).

  python -m paper_2504_07042_gb300.profile --N 7 --kind trilinear --prec f64dw \
      --box 32 32 32 --launches 3

Builds the perturbed-box mesh (or the parallelepiped box with --mesh
parallelepiped), sets up the context, runs `--launches` AxLocal calls on the
current stream and prints the CUDA-event time of each.

Other modes (same box options):
  --pcg K            K Jacobi-PCG iterations (--mixed: one outer step of the
                     mixed solver with K inner iterations)
  --learned K        K flexible-PCG iterations with the learned preconditioner
                     (untrained network; N = 7, double-word context)
  --mlp M            `--launches` MLP forward passes on M rows (tcgen05 GEMMs)
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from paper_2504_07042_gb300 import ax, inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--kind", default="trilinear", choices=sorted(ax.KINDS))
    ap.add_argument("--prec", default="f64dw", choices=sorted(ax.PRECS))
    ap.add_argument("--mesh", default="trilinear", choices=["trilinear", "parallelepiped"])
    ap.add_argument("--box", type=int, nargs=3, default=[32, 32, 32])
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--pcg", type=int, default=0, help="instead: run this many Jacobi-PCG iterations on the box")
    ap.add_argument("--mixed", action="store_true", help="with --pcg: the mixed-precision solver (float32 inner)")
    ap.add_argument("--learned", type=int, default=0, help="instead: this many learned flexible-PCG iterations")
    ap.add_argument("--mlp", type=int, default=0, help="instead: MLP forward passes on this many rows")
    a = ap.parse_args()
    if a.pcg:
        return run_pcg(a)
    if a.learned:
        return run_learned(a)
    if a.mlp:
        return run_mlp(a)
    ex, ey, ez = a.box
    V = inputs.parallelepiped_vertices(ex, ey, ez) if a.mesh == "parallelepiped" else \
        inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    dev = torch.device("cuda:0")
    op = ax.Ax(torch.from_numpy(V).to(dev), a.N, a.kind, a.prec)
    X = torch.from_numpy(inputs.element_vectors(V.shape[0], a.N, seed=1)).to(dev, op.dtype)
    Y = torch.empty_like(X)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(a.launches):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        op.ax_local(X, Y, s)
        t1.record(s)
        torch.cuda.synchronize()
        times.append(t0.elapsed_time(t1))
    info = op.ax_query()
    print(json.dumps({"E": op.E, "N": a.N, "kind": a.kind, "prec": a.prec, "ms": times,
                      "gdofs": [op.E * op.n3 / (t * 1e-3) / 1e9 for t in times], "info": info}))


def run_pcg(a):
    """-lap u = 3 pi^2 u on the box mesh, homogeneous Dirichlet, --pcg iterations."""
    import time

    import torch

    from paper_2504_07042_gb300 import ax, inputs

    ex, ey, ez = a.box
    N = a.N
    V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    dev = torch.device("cuda:0")
    Vd = torch.from_numpy(V).to(dev)
    op = ax.Ax(Vd, N, a.kind, a.prec)
    op.gs_setup(torch.from_numpy(gid).to(dev), ng, torch.from_numpy(mask).to(dev))
    XYZ = torch.empty((V.shape[0], 3, (N + 1) ** 3), dtype=torch.float64, device=dev)
    op.ax_node_coords(XYZ)
    u = torch.sin(torch.pi * XYZ[:, 0]) * torch.sin(torch.pi * XYZ[:, 1]) * torch.sin(torch.pi * XYZ[:, 2])
    f = (3 * torch.pi ** 2 * u).to(op.dtype)
    b = op.gs_gather(op.ax_mass(f, torch.empty_like(f)), torch.empty(ng, dtype=op.dtype, device=dev))
    x = torch.zeros(ng, dtype=op.dtype, device=dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    if a.mixed:
        lo = ax.Ax(Vd, N, a.kind, "fp32")
        res = op.pcg_solve_mixed(lo, b, x, rtol=1e-30, inner_rtol=1e-3, max_outer=1, max_inner=a.pcg)
    else:
        res = op.pcg_solve(b, x, rtol=1e-30, maxit=a.pcg, precond=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    print(json.dumps({"E": op.E, "N": N, "n_global": ng, "result": list(res), "seconds": dt}))


def run_learned(a):
    """--learned K flexible-PCG iterations (rtol 0) on the box, N = 7, double-word."""
    import time

    import torch

    from paper_2504_07042_gb300 import ax, inputs, learned

    ex, ey, ez = a.box
    N = 7
    V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(ex, ey, ez, N)
    mask = inputs.box_boundary_mask(ex, ey, ez, N)
    dev = torch.device("cuda:0")
    op = ax.Ax(torch.from_numpy(V).to(dev), N, "trilinear", "f64dw")
    op.gs_setup(torch.from_numpy(gid).to(dev), ng, torch.from_numpy(mask).to(dev))
    XYZ = learned.node_coords(op).cpu().numpy()
    b = learned.rhs_from_f(op, torch.from_numpy(inputs.smooth_rhs(XYZ, 300)).to(dev), ng)
    mlp = ax.AxMLP(seed=2)
    x = torch.zeros(ng, dtype=torch.float64, device=dev)
    ax.pcg_solve_learned(op, mlp, b, x, rtol=0.0, maxit=16, omega=0.5, check=False)  # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    res = ax.pcg_solve_learned(op, mlp, b, x.zero_(), rtol=0.0, maxit=a.learned, omega=0.5, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"E": op.E, "n_global": ng, "result": list(res), "seconds": time.perf_counter() - t}))


def run_mlp(a):
    """--launches forward passes of the MLP on --mlp rows of random bf16 inputs."""
    import torch

    from paper_2504_07042_gb300 import ax

    dev = torch.device("cuda:0")
    mlp = ax.AxMLP(seed=2)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    X = torch.rand((a.mlp, ax.AxMLP.IN_PAD), generator=g, device=dev).to(torch.bfloat16)
    Y = torch.empty((a.mlp, ax.AxMLP.OUT), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(a.launches):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        mlp.ax_mlp_forward(X, Y, s)
        t1.record(s)
        torch.cuda.synchronize()
        times.append(t0.elapsed_time(t1))
    flops = 2.0 * a.mlp * (ax.AxMLP.IN_PAD * 512 + 512 * 512 + 512 * 512)
    print(json.dumps({"rows": a.mlp, "ms": times, "tflops": [flops / (t * 1e-3) / 1e12 for t in times]}))


if __name__ == "__main__":
    main()
