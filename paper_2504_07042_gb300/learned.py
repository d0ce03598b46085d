"""Training pipeline of the learned preconditioner (orchestration of C-ABI calls).

Every computation runs in libax kernels: the solves (pcg_solve,
pcg_solve_mixed), the residual/error pairs (ax_mlp_pairs), the training
(ax_mlp_train) and the preconditioned solve (pcg_solve_learned).  This module
only sequences the calls and draws the seeded inputs.
"""
from __future__ import annotations

import numpy as np


def rhs_from_f(op, f_local, ng):
    """b = Q^T (w|J| f) on the device, through the library."""
    import torch
    bl = op.ax_mass(f_local, torch.empty_like(f_local))
    return op.gs_gather(bl, torch.empty(ng, dtype=f_local.dtype, device=f_local.device))


def node_coords(op):
    import torch
    XYZ = torch.empty((op.E, 3, op.n3), dtype=torch.float64, device="cuda")
    op.ax_node_coords(XYZ)
    return XYZ


def collect_pairs(op, lo, ng, seeds, snapshots=(0, 2, 8, 32), per_snapshot=1024, sample_seed=7, noise=0.1):
    """Residual/error pairs from solves with random smooth sources (one per seed).

    Each solve of A x = b starts from x0 = x* + eta (eta ~ U(-1,1) noise times
    `noise` max|x*|, zero on Dirichlet nodes), so the errors e_k = x* - x_k of
    its first Jacobi-PCG iterates are dominated by element-scale components:
    those a per-element network can predict from the local residual (the
    smooth remainder is CG's job).  op: FP64-accurate context with gs_setup;
    lo: its float32 twin (mixed solver for x*).
    Returns (F bf16 [n][544], T float32 [n][512]) on the device."""
    import torch
    from paper_2504_07042_gb300 import ax, inputs
    XYZ = node_coords(op).cpu().numpy()
    rng = np.random.default_rng(sample_seed)
    Fs, Ts = [], []
    for sd in seeds:
        f = torch.from_numpy(inputs.smooth_rhs(XYZ, sd)).to("cuda")
        b = rhs_from_f(op, f, ng)
        xs = torch.zeros(ng, dtype=torch.float64, device="cuda")
        op.pcg_solve_mixed(lo, b, xs, rtol=1e-11, inner_rtol=1e-3)
        amp = noise * float(xs.abs().max())
        eta = torch.from_numpy(rng.uniform(-amp, amp, ng)).to("cuda")
        for k in snapshots:
            xk = xs + eta
            if k > 0:
                op.pcg_solve(b, xk, rtol=0.0, maxit=k, precond=1, check=False)
            el = torch.from_numpy(rng.choice(op.E, size=min(per_snapshot, op.E), replace=False).astype(np.int64)).cuda()
            F = torch.empty((el.numel(), ax.AxMLP.IN_PAD), dtype=torch.bfloat16, device="cuda")
            T = torch.empty((el.numel(), ax.AxMLP.OUT), dtype=torch.float32, device="cuda")
            ax.ax_mlp_pairs(op, b, xs, xk, el, F, T)
            Fs.append(F)
            Ts.append(T)
    return torch.cat(Fs), torch.cat(Ts)
