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


def collect_pairs(op, ng, seeds, snapshots=(0, 2, 8, 32), per_snapshot=1024, sample_seed=7, noise=0.1):
    """Residual/error pairs from solves with random smooth data (one per seed).

    Each seed's smooth field u (the sine series of inputs.smooth_rhs at the
    nodes; it vanishes on the unit cube's faces) is the exact solution of
    A x = b with b = A u, the source it defines.  Each solve starts from
    x0 = u + eta (eta ~ U(-1,1) times `noise` max|u|, zero on Dirichlet
    nodes) and runs k Jacobi-PCG iterations; the pairs are (local residual
    b - A x_k, local error u - x_k) on sampled elements.  The errors of these
    early iterates are dominated by element-scale components: those a
    per-element network can predict from the local residual (the smooth
    remainder is CG's job).  op: FP64-accurate context with gs_setup.
    Returns (F bf16 [n][544], T float32 [n][512]) on the device."""
    import torch
    from paper_2504_07042_gb300 import ax, inputs
    XYZ = node_coords(op)
    # the sine factors of the seeded smooth fields, evaluated once on the device
    order = 3
    S = [torch.stack([torch.sin(a * np.pi * XYZ[:, d]) for a in range(1, order + 1)]) for d in range(3)]
    U = torch.empty((op.E, op.n3), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(U)
    mult = op.gs_gather(torch.ones_like(U), torch.empty(ng, dtype=torch.float64, device="cuda"))
    mult = torch.where(mult > 0, mult, torch.ones_like(mult))
    rng = np.random.default_rng(sample_seed)
    Fs, Ts = [], []
    for sd in seeds:
        C = torch.from_numpy(inputs.smooth_rhs_coeffs(sd, order)).to("cuda")
        u_local = torch.einsum("abc,aen,ben,cen->en", C, S[0], S[1], S[2]).contiguous()
        xs = op.gs_gather(u_local, torch.empty(ng, dtype=torch.float64, device="cuda")) / mult  # masked: 0 on faces
        op.gs_scatter(xs, U)
        op.ax_local(U, Y)
        b = op.gs_gather(Y, torch.empty(ng, dtype=torch.float64, device="cuda"))
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


def train_select(mlp, F, T, op_val, b_val, chunks=(3, 3, 3, 3, 4, 4), omegas=(0.5, 0.75, 1.0), batch=4096, lr=1e-3,
                 seed=4, maxit=20000):
    """Train in chunks of epochs and keep the checkpoint and damping omega that
    solve a held-out validation problem (op_val, b_val: another source on a
    mesh with gs_setup) in the fewest flexible-PCG iterations, without the
    Jacobi fallback.  The solver the network serves is what decides: a
    lower training loss does not by itself mean fewer iterations.
    Returns (omega, validation iterations, loss history, trace of (epochs, omega, iterations))."""
    import torch
    from paper_2504_07042_gb300 import ax
    best = (None, None, 1 << 30)
    hist, trace, done = [], [], 0
    ng = b_val.numel()
    for ch in chunks:
        hist += list(mlp.ax_mlp_train(F, T, epochs=ch, batch=batch, lr=lr, seed=seed + done))
        done += ch
        for om in omegas:
            x = torch.zeros(ng, dtype=torch.float64, device=b_val.device)
            it, rr, st, fb = ax.pcg_solve_learned(op_val, mlp, b_val, x, rtol=1e-8, maxit=maxit, omega=om, check=False)
            trace.append((done, om, it if st == ax.AX_OK else None, fb))
            if st == ax.AX_OK and not fb and it < best[2]:
                best = (mlp.ax_mlp_get_params(), om, it)
    if best[0] is not None:
        mlp.ax_mlp_set_params(best[0])
    return best[1], best[2], hist, trace
