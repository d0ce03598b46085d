"""Seeded synthetic inputs: meshes, element vectors and global numberings.

This module is the one place the CUDA path and the CPU oracle share.  It holds
none of the method's arithmetic (no GLL constants, no Jacobians, no operator):
only numpy random draws and integer bookkeeping that build the inputs both
sides consume.

Meshes are structured boxes of ``ex * ey * ez`` hexahedra, element
``e = ix + ex * (iy + ey * iz)``.  Vertex arrays are ``[E][8][3]`` float64 in
the Kronecker order of the paper's trilinear map (Eq. 8): vertex
``v = a + 2 b + 4 c`` sits at grid corner ``(ix + a, iy + b, iz + c)``.

Recipes (the paper's own benchmark meshes are synthetic boxes, Sec. 5.1):

* ``box_vertices``: uniform grid of spacing ``h = 1/ex`` in every direction
  (so the box is ``[0,1] x [0, ey/ex] x [0, ez/ex]``); every grid point not on
  the boundary is moved by ``U(-a h, a h)`` per coordinate (``a = 0.1``),
  drawn with ``numpy.random.default_rng(seed)`` for all grid points in
  C order of ``(ix, iy, iz, coord)`` and then zeroed on the boundary.
* ``parallelepiped_vertices``: a tensor grid whose spacings per axis are
  ``U(0.8, 1.2) h`` (rng ``seed_spacing``), mapped by ``x -> M x`` with
  ``M = I + 0.2 U(-1,1)^{3x3}`` (rng ``seed_map``); every element is then a
  distinct parallelepiped.
* ``element_vectors``: ``U(-1, 1)`` float64 of shape ``[E][(N+1)^3]``.
"""
from __future__ import annotations

import math

import numpy as np


def _grid_to_elements(P: np.ndarray) -> np.ndarray:
    """Grid points P[ix][iy][iz][3] -> element vertices [E][8][3]."""
    ex, ey, ez = (s - 1 for s in P.shape[:3])
    V = np.empty((ez, ey, ex, 8, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                sub = P[a:a + ex, b:b + ey, c:c + ez]  # [ex][ey][ez][3]
                V[:, :, :, a + 2 * b + 4 * c, :] = sub.transpose(2, 1, 0, 3)
    return np.ascontiguousarray(V.reshape(ex * ey * ez, 8, 3))


def box_grid(ex: int, ey: int, ez: int, perturb: float = 0.1, seed: int = 0) -> np.ndarray:
    h = 1.0 / ex
    gx, gy, gz = np.meshgrid(np.arange(ex + 1) * h, np.arange(ey + 1) * h, np.arange(ez + 1) * h, indexing="ij")
    P = np.stack([gx, gy, gz], axis=-1)
    if perturb:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-perturb * h, perturb * h, size=P.shape)
        interior = np.zeros(P.shape[:3], dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        P = P + d * interior[..., None]
    return P


def box_vertices(ex: int, ey: int, ez: int, perturb: float = 0.1, seed: int = 0) -> np.ndarray:
    """Perturbed trilinear box mesh, vertices [E][8][3]."""
    return _grid_to_elements(box_grid(ex, ey, ez, perturb, seed))


def parallelepiped_vertices(ex: int, ey: int, ez: int, seed_spacing: int = 2, seed_map: int = 3) -> np.ndarray:
    """Box of distinct parallelepipeds: non-uniform tensor grid, then x -> M x."""
    h = 1.0 / ex
    rs = np.random.default_rng(seed_spacing)
    coords = []
    for n in (ex, ey, ez):
        sp = rs.uniform(0.8, 1.2, size=n) * h
        coords.append(np.concatenate([[0.0], np.cumsum(sp)]))
    gx, gy, gz = np.meshgrid(*coords, indexing="ij")
    P = np.stack([gx, gy, gz], axis=-1)
    rm = np.random.default_rng(seed_map)
    while True:
        M = np.eye(3) + 0.2 * rm.uniform(-1.0, 1.0, size=(3, 3))
        if np.linalg.det(M) > 0.2:
            break
    return _grid_to_elements(P @ M.T)


def element_vectors(E: int, N: int, seed: int = 1, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(E, (N + 1) ** 3)).astype(dtype)


def box_global_ids(ex: int, ey: int, ez: int, N: int):
    """Global node numbering of a structured box (the binary Q of Eq. 1).

    Local node [i,j,k] of element (ix,iy,iz) is global lattice point
    (ix*N + i, iy*N + j, iz*N + k) of the (ex*N+1) x (ey*N+1) x (ez*N+1) lattice,
    numbered x-fastest.  Returns (gid [E][(N+1)^3] int64, n_global)."""
    N1 = N + 1
    gx, gy, gz = ex * N + 1, ey * N + 1, ez * N + 1
    i = np.arange(N1)
    li, lj, lk = np.meshgrid(i, i, i, indexing="ij")  # li[i][j][k]
    # local index l = i + j N1 + k N1^2  ->  order arrays as [k][j][i]
    li, lj, lk = (a.transpose(2, 1, 0).reshape(-1) for a in (li, lj, lk))
    ix, iy, iz = np.meshgrid(np.arange(ex), np.arange(ey), np.arange(ez), indexing="ij")
    ix, iy, iz = (a.transpose(2, 1, 0).reshape(-1) for a in (ix, iy, iz))  # element order e = ix + ex(iy + ey iz)
    X = ix[:, None] * N + li[None, :]
    Y = iy[:, None] * N + lj[None, :]
    Z = iz[:, None] * N + lk[None, :]
    gid = (X + gx * (Y + gy * Z)).astype(np.int64)
    return np.ascontiguousarray(gid), gx * gy * gz


def box_boundary_mask(ex: int, ey: int, ez: int, N: int) -> np.ndarray:
    """uint8 [n_global]: 1 on lattice points of the box boundary (Dirichlet)."""
    gx, gy, gz = ex * N + 1, ey * N + 1, ez * N + 1
    m = np.zeros((gz, gy, gx), dtype=np.uint8)
    m[0, :, :] = m[-1, :, :] = 1
    m[:, 0, :] = m[:, -1, :] = 1
    m[:, :, 0] = m[:, :, -1] = 1
    return m.reshape(-1)


def near_cubic_box(E_target: int):
    """(ex, ey, ez), ex >= ey >= ez, with ex*ey*ez within 5% of E_target (or the
    closest product found) and the smallest aspect ratio ex/ez among those."""
    cands = []
    for ez in range(1, int(round(E_target ** (1.0 / 3.0))) + 2):
        for ey in range(ez, int(math.isqrt(max(1, E_target // ez))) + 2):
            ex = max(ey, int(round(E_target / (ey * ez))))
            cands.append((abs(ex * ey * ez - E_target) / E_target, ex / ez, (ex, ey, ez)))
    good = [c for c in cands if c[0] <= 0.05]
    if good:
        return min(good, key=lambda c: (c[1], c[0]))[2]
    return min(cands, key=lambda c: (c[0], c[1]))[2]


def sweep_box(N: int):
    """Box dimensions giving about 64M local nodes at order N (the order sweep)."""
    table = {3: (128, 128, 64), 5: (68, 68, 67), 7: (64, 64, 32), 9: (41, 41, 40),
             11: (34, 34, 34), 15: (32, 32, 16)}
    if N in table:
        return table[N]
    return near_cubic_box(int(round(64 * 2 ** 20 / (N + 1) ** 3)))


def batch_meshes(n_meshes: int = 64, seed_e: int = 4, seed_n: int = 5):
    """Uneven batch: E log-uniform on [64, 4096] (rounded to a near-cubic box),
    N uniform on {3,5,7,9}.  Returns a list of (ex, ey, ez, N)."""
    re, rn = np.random.default_rng(seed_e), np.random.default_rng(seed_n)
    Es = np.exp(re.uniform(math.log(64), math.log(4096), size=n_meshes))
    Ns = rn.choice([3, 5, 7, 9], size=n_meshes)
    out = []
    for E, N in zip(Es, Ns):
        out.append(near_cubic_box(int(round(E))) + (int(N),))
    return out


def smooth_rhs(XYZ: np.ndarray, seed: int, order: int = 3) -> np.ndarray:
    """Random smooth source f(x) = sum_{a,b,c=1..order} c_abc sin(a pi x) sin(b pi y) sin(c pi z),
    c_abc ~ N(0,1) / (a^2 + b^2 + c^2), evaluated at node coordinates XYZ [E][3][n3]
    (rng seed `seed`; the training solves use seeds 100..299)."""
    C = smooth_rhs_coeffs(seed, order)
    f = np.zeros(XYZ[:, 0].shape)
    sx = [np.sin(a * np.pi * XYZ[:, 0]) for a in range(1, order + 1)]
    sy = [np.sin(b * np.pi * XYZ[:, 1]) for b in range(1, order + 1)]
    sz = [np.sin(c * np.pi * XYZ[:, 2]) for c in range(1, order + 1)]
    for a in range(order):
        for b in range(order):
            for c in range(order):
                f += C[a, b, c] * sx[a] * sy[b] * sz[c]
    return f


def smooth_rhs_coeffs(seed: int, order: int = 3) -> np.ndarray:
    """The coefficients c_abc of smooth_rhs (same draw order: a, then b, then c)."""
    rng = np.random.default_rng(seed)
    C = np.empty((order, order, order))
    for a in range(order):
        for b in range(order):
            for c in range(order):
                C[a, b, c] = rng.standard_normal() / ((a + 1) ** 2 + (b + 1) ** 2 + (c + 1) ** 2)
    return C
