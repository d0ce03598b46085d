"""Python face of the FP64 CPU oracle (``oracle.c``) plus the dense tiny-N path.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  It shares no
code with the CUDA library; the two meet only through the seeded input
generators in ``paper_2504_07042_gb300.inputs``.

The C oracle is compiled with plain gcc (``build()``), loaded with ctypes and
called on numpy arrays.  The dense path builds the element matrix of Eq. 3
from Kronecker products (Table 1) with numpy and is used only for N <= 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O3, OpenMP).  No
    -march=native: the same source builds on x86-64 and Arm hosts, and the
    compiler may not reassociate (no -ffast-math), so -O3 keeps the order of
    every floating-point operation as written."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB lets the mutation tests point the pins at a deliberately
        # broken copy of the oracle; normal runs build and load _build/liboracle.so
        path = os.environ.get("ORACLE_LIB")
        if not path:
            path = build()
        L = ctypes.CDLL(path)
        i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_num_threads.restype = c_int
        L.orc_set_num_threads.argtypes = [c_int]
        L.orc_gll.argtypes = [c_int, _dp, _dp, _dp]
        L.orc_gll.restype = c_int
        L.orc_trilinear_map.argtypes = [_dp, c_double, c_double, c_double, _dp]
        L.orc_jacobian_trilinear.argtypes = [_dp, c_double, c_double, c_double, _dp]
        L.orc_factors_from_jacobian.argtypes = [_dp, c_double, _dp]
        L.orc_factors_from_jacobian.restype = c_double
        L.orc_factors_eq9.argtypes = [i64, c_int, _dp, _dp]
        L.orc_factors_eq9.restype = i64
        L.orc_factors_discrete.argtypes = [i64, c_int, _dp, _dp]
        L.orc_factors_discrete.restype = i64
        L.orc_nodal_coords.argtypes = [i64, c_int, _dp, _dp]
        L.orc_nodal_coords.restype = c_int
        L.orc_axlocal.argtypes = [i64, c_int, _dp, _dp, _dp]
        L.orc_axlocal.restype = c_int
        L.orc_axlocal_vertices.argtypes = [i64, c_int, _dp, _dp, _dp]
        L.orc_axlocal_vertices.restype = i64
        L.orc_gs.argtypes = [i64, _ip, i64, _dp]
        L.orc_gs.restype = c_int
        L.orc_gather.argtypes = [i64, _ip, i64, _dp, _dp]
        L.orc_gather.restype = c_int
        L.orc_scatter.argtypes = [i64, _ip, i64, _dp, _dp]
        L.orc_scatter.restype = c_int
        L.orc_diag.argtypes = [i64, c_int, _dp, _dp]
        L.orc_diag.restype = c_int
        _u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        L.orc_pcg.argtypes = [i64, c_int, _dp, _ip, i64, ctypes.c_void_p, _dp, _dp, ctypes.c_void_p, c_double,
                              c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]
        L.orc_pcg.restype = c_int
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def gll(N: int):
    """(xi, w, D) of Table 1: GLL points, weights and differentiation matrix."""
    N1 = N + 1
    xi, w, D = np.zeros(N1), np.zeros(N1), np.zeros(N1 * N1)
    if lib().orc_gll(int(N), xi, w, D):
        raise ValueError("unsupported N=%d" % N)
    return xi, w, D.reshape(N1, N1)


def trilinear_map(V, r, s, t):
    out = np.zeros(3)
    lib().orc_trilinear_map(_f64(V).reshape(24), float(r), float(s), float(t), out)
    return out


def jacobian(V, r, s, t):
    """J[c][d] = d x_c / d ref_d at (r,s,t) from Eq. 9."""
    J = np.zeros(9)
    lib().orc_jacobian_trilinear(_f64(V).reshape(24), float(r), float(s), float(t), J)
    return J.reshape(3, 3)


def factors_from_jacobian(J, W):
    g = np.zeros(7)
    det = lib().orc_factors_from_jacobian(_f64(J).reshape(9), float(W), g)
    return g, det


def factors(V, N: int, route: str = "eq9"):
    """Geometric factors [E][7][n3] (g00 g01 g02 g11 g12 g22 gwj) and the
    number of nodes with det J <= 0.  route: "eq9" (analytic Jacobian) or
    "discrete" (discrete gradient of the nodal coordinates, Sec. 3.2)."""
    V = _f64(V)
    E = V.shape[0]
    n3 = (N + 1) ** 3
    G = np.zeros((E, 7, n3))
    fn = lib().orc_factors_eq9 if route == "eq9" else lib().orc_factors_discrete
    bad = fn(E, int(N), V.reshape(-1), G.reshape(-1))
    if bad < 0:
        raise ValueError("oracle factors failed")
    return G, int(bad)


def nodal_coords(V, N: int):
    V = _f64(V)
    E = V.shape[0]
    out = np.zeros((E, 3, (N + 1) ** 3))
    if lib().orc_nodal_coords(E, int(N), V.reshape(-1), out.reshape(-1)):
        raise ValueError("oracle nodal_coords failed")
    return out


def axlocal(G, X, N: int):
    """Algorithm 1 (Poisson) for every element: Y[e] = A^(e) X[e]."""
    G, X = _f64(G), _f64(X)
    E = X.shape[0]
    Y = np.zeros_like(X)
    if lib().orc_axlocal(E, int(N), G.reshape(-1), X.reshape(-1), Y.reshape(-1)):
        raise MemoryError("oracle axlocal failed")
    return Y


def axlocal_vertices(V, X, N: int):
    """Eq. 9 + Eq. 7 + Algorithm 1 per element, straight from the vertices."""
    V, X = _f64(V), _f64(X)
    E = X.shape[0]
    Y = np.zeros_like(X)
    bad = lib().orc_axlocal_vertices(E, int(N), V.reshape(-1), X.reshape(-1), Y.reshape(-1))
    if bad < 0:
        raise MemoryError("oracle axlocal_vertices failed")
    return Y, int(bad)


def gs(Y, gid, n_global: int):
    """Y <- Q Q^T Y (Eq. 1)."""
    Y = _f64(Y).copy()
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    if lib().orc_gs(Y.size, gid.reshape(-1), int(n_global), Y.reshape(-1)):
        raise ValueError("bad global id")
    return Y


def gather(Yl, gid, n_global: int):
    """Q^T Y: sum the local copies into the global vector."""
    Yl = _f64(Yl)
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    yg = np.zeros(int(n_global))
    if lib().orc_gather(Yl.size, gid.reshape(-1), int(n_global), Yl.reshape(-1), yg):
        raise ValueError("bad global id")
    return yg


def scatter(ug, gid):
    """Q u: copy the global vector to its local copies."""
    ug = _f64(ug)
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    Ul = np.zeros(gid.shape)
    if lib().orc_scatter(gid.size, gid.reshape(-1), ug.size, ug, Ul.reshape(-1)):
        raise ValueError("bad global id")
    return Ul


# ---------------------------------------------------------------------------
# Dense tiny-N path: A^(e) = D^T blkdiag(G) D as an explicit n3 x n3 matrix
# (Eq. 3, Poisson), with D = [I(x)I(x)Dhat ; I(x)Dhat(x)I ; Dhat(x)I(x)I]
# (Table 1).  np.kron is the library primitive; nothing else is fused.
# ---------------------------------------------------------------------------
def dense_element_matrix(Ge, N: int):
    """Dense A^(e) from one element's factors Ge [7][n3] (only N <= 4)."""
    if N > 4:
        raise ValueError("dense path is for tiny N only")
    _, _, Dh = gll(N)
    I = np.eye(N + 1)
    Dr = np.kron(I, np.kron(I, Dh))
    Ds = np.kron(I, np.kron(Dh, I))
    Dt = np.kron(Dh, np.kron(I, I))
    Dfull = np.vstack([Dr, Ds, Dt])
    g00, g01, g02, g11, g12, g22 = (np.diag(Ge[q]) for q in range(6))
    Gblk = np.block([[g00, g01, g02], [g01, g11, g12], [g02, g12, g22]])
    return Dfull.T @ Gblk @ Dfull


def element_diagonals(G, N: int):
    """diag[e][l] = e_l^T A^(e) e_l by Algorithm 1 on unit vectors (small meshes)."""
    G = _f64(G)
    E = G.shape[0]
    d = np.zeros((E, (N + 1) ** 3))
    if lib().orc_diag(E, int(N), G.reshape(-1), d.reshape(-1)):
        raise MemoryError("oracle diag failed")
    return d


def pcg(G, gid, n_global: int, mask, b, N: int, x0=None, diag_global=None, rtol=1e-10, maxit=10000):
    """Textbook (P)CG on the assembled, Dirichlet-masked system (Eq. 1).
    Returns (x, iterations, relative residual, converged)."""
    G = _f64(G)
    E = G.shape[0]
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    b = _f64(b)
    x = np.zeros(int(n_global)) if x0 is None else _f64(x0).copy()
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    dg = None if diag_global is None else _f64(diag_global)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    st = lib().orc_pcg(E, int(N), G.reshape(-1), gid.reshape(-1), int(n_global),
                       None if m is None else m.ctypes.data, b, x, None if dg is None else dg.ctypes.data,
                       float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rr))
    if st < 0:
        raise MemoryError("oracle pcg failed")
    return x, it.value, rr.value, st == 0
