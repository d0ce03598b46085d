"""Thin ctypes binding of libax (include/ax.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors (device memory and streams are the
only things PyTorch provides); host buffers for ``ax_local_host`` are numpy
arrays or CPU tensors.  If libax.so has not been built, importing this module
raises ``ImportError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libax.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libax.so is not built (run paper_2504_07042_gb300.build.build()); no fallback exists")

_lib = ctypes.CDLL(LIB_PATH)

# enums (mirror include/ax.h)
AX_OK, AX_EINVAL, AX_ENOMEM, AX_ECUDA, AX_EINVERTED, AX_ENOTPARALLELEPIPED, AX_ENOTCONV, AX_ETIMEOUT, \
    AX_EUNSUPPORTED, AX_ERANGE = range(10)
AX_GEOM_STORED, AX_GEOM_TRILINEAR, AX_GEOM_PARALLELEPIPED, AX_GEOM_TRILINEAR_PARTIAL = range(4)
AX_FP64, AX_FP32, AX_TF32, AX_BF16, AX_FP16, AX_F64DW = range(6)

KINDS = {"stored": AX_GEOM_STORED, "trilinear": AX_GEOM_TRILINEAR, "parallelepiped": AX_GEOM_PARALLELEPIPED,
         "partial": AX_GEOM_TRILINEAR_PARTIAL}
PRECS = {"fp64": AX_FP64, "fp32": AX_FP32, "tf32": AX_TF32, "bf16": AX_BF16, "fp16": AX_FP16, "f64dw": AX_F64DW}


class ax_info(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int64), ("N", ctypes.c_int), ("kind", ctypes.c_int), ("prec", ctypes.c_int),
                ("bytes_per_element", ctypes.c_double), ("flops_ax_per_element", ctypes.c_double),
                ("pipe_ops_per_element", ctypes.c_double), ("pipe", ctypes.c_int)]


_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_lib.ax_setup.argtypes = [ctypes.POINTER(_vp), _i64, _int, _vp, _int, _int, _vp]
_lib.ax_setup.restype = _int
_lib.ax_local.argtypes = [_vp, _vp, _vp, _vp]
_lib.ax_local.restype = _int
_lib.ax_local_host.argtypes = [_vp, _vp, _vp, _vp]
_lib.ax_local_host.restype = _int
_lib.ax_local_host_static.argtypes = [_vp, _vp, _vp, _vp]
_lib.ax_local_host_static.restype = _int
_lib.ax_factors.argtypes = [_vp, _vp, _vp]
_lib.ax_factors.restype = _int
_lib.ax_node_coords.argtypes = [_vp, _vp, _vp]
_lib.ax_node_coords.restype = _int
_lib.gs_setup.argtypes = [_vp, _vp, _i64, _vp, _vp]
_lib.gs_setup.restype = _int
for _n in ("gs_gather", "gs_scatter", "ax_mass"):
    getattr(_lib, _n).argtypes = [_vp, _vp, _vp, _vp]
    getattr(_lib, _n).restype = _int
for _n in ("gs_assemble", "ax_diag"):
    getattr(_lib, _n).argtypes = [_vp, _vp, _vp]
    getattr(_lib, _n).restype = _int
_lib.pcg_solve.argtypes = [_vp, _vp, _vp, _dbl, _int, _int, ctypes.POINTER(_int), ctypes.POINTER(_dbl), _vp]
_lib.pcg_solve.restype = _int
_lib.pcg_solve_mixed.argtypes = [_vp, _vp, _vp, _vp, _dbl, _dbl, _int, _int, ctypes.POINTER(_int),
                                  ctypes.POINTER(_int), ctypes.POINTER(_dbl), _vp]
_lib.pcg_solve_mixed.restype = _int
_lib.ax_batch_setup.argtypes = [ctypes.POINTER(_vp), _int, ctypes.POINTER(_i64), ctypes.POINTER(_int),
                                ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_vp),
                                _int, _int, _vp]
_lib.ax_batch_setup.restype = _int
_lib.ax_batch_sizes.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64)]
_lib.ax_batch_sizes.restype = _int
_lib.ax_batch_local.argtypes = [_vp, _vp, _vp, _vp]
_lib.ax_batch_local.restype = _int
_lib.ax_batch_tune.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_i64), _vp]
_lib.ax_batch_tune.restype = _int
_lib.ax_batch_pcg.argtypes = [_vp, _vp, _vp, _dbl, _int, _int, ctypes.POINTER(_int), ctypes.POINTER(_dbl), _vp]
_lib.ax_batch_pcg.restype = _int
_lib.ax_check.argtypes = [_vp, _vp]
_lib.ax_check.restype = _int
_lib.ax_batch_set_persistent.argtypes = [_vp, _int]
_lib.ax_batch_set_persistent.restype = _int
_lib.ax_batch_info.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]
_lib.ax_batch_info.restype = _int
_lib.ax_batch_set_wait.argtypes = [_vp, _i64, _int]
_lib.ax_batch_set_wait.restype = _int
_lib.ax_batch_last_error.argtypes = [_vp]
_lib.ax_batch_last_error.restype = ctypes.c_char_p
_lib.ax_batch_destroy.argtypes = [_vp]
_lib.ax_batch_destroy.restype = None
_lib.ax_mlp_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_uint64, _vp]
_lib.ax_mlp_create.restype = _int
_lib.ax_mlp_num_params.argtypes = [_vp]
_lib.ax_mlp_num_params.restype = _i64
for _n in ("ax_mlp_get_params", "ax_mlp_set_params"):
    getattr(_lib, _n).argtypes = [_vp, _vp, _vp]
    getattr(_lib, _n).restype = _int
_lib.ax_mlp_forward.argtypes = [_vp, _vp, _vp, _i64, _vp]
_lib.ax_mlp_forward.restype = _int
_lib.ax_mlp_grad.argtypes = [_vp, _vp, _vp, _i64, ctypes.POINTER(ctypes.c_float), _vp, _vp]
_lib.ax_mlp_grad.restype = _int
_lib.ax_mlp_train.argtypes = [_vp, _vp, _vp, _i64, _int, _int, ctypes.c_float, ctypes.c_uint64, _vp, _vp]
_lib.ax_mlp_train.restype = _int
_lib.ax_mlp_pairs.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]
_lib.ax_mlp_pairs.restype = _int
_lib.pcg_solve_learned.argtypes = [_vp, _vp, _vp, _vp, _dbl, _int, _dbl, ctypes.POINTER(_int), ctypes.POINTER(_dbl),
                                   ctypes.POINTER(_int), _vp]
_lib.pcg_solve_learned.restype = _int
_lib.ax_mlp_last_error.argtypes = [_vp]
_lib.ax_mlp_last_error.restype = ctypes.c_char_p
_lib.ax_mlp_destroy.argtypes = [_vp]
_lib.ax_mlp_destroy.restype = None
_lib.ax_query.argtypes = [_vp, ctypes.POINTER(ax_info)]
_lib.ax_query.restype = _int
_lib.ax_last_error.argtypes = [_vp]
_lib.ax_last_error.restype = ctypes.c_char_p
_lib.ax_status_string.argtypes = [_int]
_lib.ax_status_string.restype = ctypes.c_char_p
_lib.ax_destroy.argtypes = [_vp]
_lib.ax_destroy.restype = None

EXPORTS = ("ax_setup", "ax_local", "ax_local_host", "ax_local_host_static", "ax_factors", "ax_node_coords", "ax_query",
           "gs_setup", "gs_assemble", "gs_gather", "gs_scatter", "ax_mass", "ax_diag", "pcg_solve", "pcg_solve_mixed",
           "ax_batch_setup", "ax_batch_sizes", "ax_batch_local", "ax_batch_tune", "ax_batch_pcg",
           "ax_batch_last_error", "ax_batch_destroy",
           "ax_mlp_create", "ax_mlp_num_params", "ax_mlp_get_params", "ax_mlp_set_params", "ax_mlp_forward",
           "ax_mlp_grad", "ax_mlp_train", "ax_mlp_pairs", "pcg_solve_learned", "ax_mlp_last_error", "ax_mlp_destroy",
           "ax_last_error", "ax_status_string", "ax_destroy")


class AxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_lib.ax_status_string(status).decode(), msg))
        self.status = status


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy
        return t.ctypes.data
    return int(t)


def _check(st: int, ctx=None):
    if st != AX_OK:
        raise AxError(st, _lib.ax_last_error(ctx).decode())


class Ax:
    """Owns an ax_ctx.  Method names follow the C ABI."""

    def __init__(self, vertices, N: int, kind="trilinear", prec="fp64", stream=None):
        import torch
        kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        prec = PRECS[prec] if isinstance(prec, str) else int(prec)
        if not (isinstance(vertices, torch.Tensor) and vertices.is_cuda and vertices.dtype == torch.float64):
            raise TypeError("vertices must be a float64 CUDA tensor [E][8][3]")
        vertices = vertices.contiguous()
        self.E = int(vertices.shape[0])
        self.N = int(N)
        self.kind, self.prec = kind, prec
        self.ctx = _vp()
        _check(_lib.ax_setup(ctypes.byref(self.ctx), self.E, self.N, _ptr(vertices), kind, prec, _stream(stream)))
        self.n3 = (self.N + 1) ** 3
        self.dtype = torch.float64 if prec in (AX_FP64, AX_F64DW) else torch.float32

    def ax_local(self, X, Y, stream=None):
        _check(_lib.ax_local(self.ctx, _ptr(X), _ptr(Y), _stream(stream)), self.ctx)
        return Y

    def _host_io(self, name, X_host, Y_host):
        """Host buffers for the host entry points: C-contiguous, the context's
        value type, at least E * (N+1)^3 values each (the C side copies that
        many bytes from X and to Y)."""
        import numpy as np
        import torch
        want = self.E * self.n3
        for tag, a in (("X_host", X_host), ("Y_host", Y_host)):
            if isinstance(a, torch.Tensor):
                ok = a.device.type == "cpu" and a.is_contiguous() and a.dtype == self.dtype and a.numel() >= want
            elif isinstance(a, np.ndarray):
                npdt = np.float64 if self.dtype == torch.float64 else np.float32
                ok = a.flags["C_CONTIGUOUS"] and a.dtype == npdt and a.size >= want
            else:
                ok = False
            if not ok:
                raise TypeError("%s: %s must be a C-contiguous host array of %s with at least %d values"
                                % (name, tag, self.dtype, want))

    def ax_local_host(self, X_host, Y_host, stream=None):
        self._host_io("ax_local_host", X_host, Y_host)
        _check(_lib.ax_local_host(self.ctx, _ptr(X_host), _ptr(Y_host), _stream(stream)), self.ctx)
        return Y_host

    def ax_local_host_static(self, X_host, Y_host, stream=None):
        """ax_local_host without device allocation (fixed 16 MiB per vector)."""
        self._host_io("ax_local_host_static", X_host, Y_host)
        _check(_lib.ax_local_host_static(self.ctx, _ptr(X_host), _ptr(Y_host), _stream(stream)), self.ctx)
        return Y_host

    def ax_factors(self, G_out, stream=None):
        _check(_lib.ax_factors(self.ctx, _ptr(G_out), _stream(stream)), self.ctx)
        return G_out

    def ax_node_coords(self, XYZ_out, stream=None):
        _check(_lib.ax_node_coords(self.ctx, _ptr(XYZ_out), _stream(stream)), self.ctx)
        return XYZ_out

    def gs_setup(self, global_id, n_global: int, dirichlet_mask=None, stream=None):
        _check(_lib.gs_setup(self.ctx, _ptr(global_id), int(n_global), _ptr(dirichlet_mask), _stream(stream)),
               self.ctx)
        self.n_global = int(n_global)

    def gs_assemble(self, Y_local, stream=None):
        _check(_lib.gs_assemble(self.ctx, _ptr(Y_local), _stream(stream)), self.ctx)
        return Y_local

    def gs_gather(self, Y_local, y_global, stream=None):
        _check(_lib.gs_gather(self.ctx, _ptr(Y_local), _ptr(y_global), _stream(stream)), self.ctx)
        return y_global

    def gs_scatter(self, u_global, U_local, stream=None):
        _check(_lib.gs_scatter(self.ctx, _ptr(u_global), _ptr(U_local), _stream(stream)), self.ctx)
        return U_local

    def ax_mass(self, F_local, Y_local, stream=None):
        _check(_lib.ax_mass(self.ctx, _ptr(F_local), _ptr(Y_local), _stream(stream)), self.ctx)
        return Y_local

    def ax_diag(self, diag_local, stream=None):
        _check(_lib.ax_diag(self.ctx, _ptr(diag_local), _stream(stream)), self.ctx)
        return diag_local

    def pcg_solve(self, b_global, x_global, rtol=1e-8, maxit=10000, precond=1, stream=None, check=True):
        """Returns (iterations, relative residual, status)."""
        it, rr = _int(0), _dbl(0.0)
        st = _lib.pcg_solve(self.ctx, _ptr(b_global), _ptr(x_global), float(rtol), int(maxit), int(precond),
                            ctypes.byref(it), ctypes.byref(rr), _stream(stream))
        if check and st not in (AX_OK, AX_ENOTCONV):
            _check(st, self.ctx)
        return it.value, rr.value, st

    def pcg_solve_mixed(self, lo: "Ax", b_global, x_global, rtol=1e-8, inner_rtol=1e-3, max_outer=50,
                        max_inner=5000, stream=None, check=True):
        """FP64 refinement (this context) around a float32 inner PCG (lo).
        Returns (outer iterations, total inner iterations, relative residual, status)."""
        o, i, rr = _int(0), _int(0), _dbl(0.0)
        st = _lib.pcg_solve_mixed(self.ctx, lo.ctx, _ptr(b_global), _ptr(x_global), float(rtol), float(inner_rtol),
                                  int(max_outer), int(max_inner), ctypes.byref(o), ctypes.byref(i), ctypes.byref(rr),
                                  _stream(stream))
        if check and st not in (AX_OK, AX_ENOTCONV):
            _check(st, self.ctx)
        return o.value, i.value, rr.value, st

    def ax_check(self, stream=None):
        """Synchronise and report a bounded wait that ran out (AxError AX_ETIMEOUT)."""
        _check(_lib.ax_check(self.ctx, _stream(stream)), self.ctx)

    def ax_query(self) -> dict:
        info = ax_info()
        _check(_lib.ax_query(self.ctx, ctypes.byref(info)), self.ctx)
        return {k: getattr(info, k) for k, _ in ax_info._fields_}

    def ax_destroy(self):
        if self.ctx:
            _lib.ax_destroy(self.ctx)
            self.ctx = _vp()

    def __del__(self):
        try:
            self.ax_destroy()
        except Exception:
            pass


def ax_setup(vertices, N, kind="trilinear", prec="fp64", stream=None) -> Ax:
    return Ax(vertices, N, kind, prec, stream)


def _bcheck(st: int, b=None):
    if st != AX_OK:
        raise AxError(st, _lib.ax_batch_last_error(b).decode())


class AxBatch:
    """Owns an ax_batch: many meshes of uneven size and order.  Method names follow the C ABI."""

    def __init__(self, meshes, kind="trilinear", prec="fp32", stream=None):
        """meshes: list of (vertices [E][8][3] float64 CUDA tensor, N, global_id [E][n3] int64 CUDA
        tensor, n_global, mask uint8 CUDA tensor or None)."""
        kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        prec = PRECS[prec] if isinstance(prec, str) else int(prec)
        B = len(meshes)
        self._keep = [m for m in meshes]  # keep the tensors alive during setup
        E = (_i64 * B)(*[int(m[0].shape[0]) for m in meshes])
        Ns = (_int * B)(*[int(m[1]) for m in meshes])
        V = (_vp * B)(*[_ptr(m[0].contiguous()) for m in meshes])
        G = (_vp * B)(*[_ptr(m[2].contiguous()) for m in meshes])
        NG = (_i64 * B)(*[int(m[3]) for m in meshes])
        M = (_vp * B)(*[_ptr(m[4]) if m[4] is not None else None for m in meshes])
        self.b = _vp()
        _bcheck(_lib.ax_batch_setup(ctypes.byref(self.b), B, E, Ns, V, G, NG, M, kind, prec, _stream(stream)))
        self.B, self.prec = B, prec
        nl, ng = _i64(0), _i64(0)
        lo, go = (_i64 * B)(), (_i64 * (B + 1))()
        _bcheck(_lib.ax_batch_sizes(self.b, ctypes.byref(nl), ctypes.byref(ng), lo, go), self.b)
        self.n_local, self.n_global = nl.value, ng.value
        self.local_offsets, self.global_offsets = list(lo), list(go)
        import torch
        self.dtype = torch.float64 if prec in (AX_FP64, AX_F64DW) else torch.float32
        self.groups = sorted(set(int(m[1]) for m in meshes), key=[int(m[1]) for m in meshes].index)
        self._keep = None

    def ax_batch_local(self, X, Y, stream=None):
        _bcheck(_lib.ax_batch_local(self.b, _ptr(X), _ptr(Y), _stream(stream)), self.b)
        return Y

    def ax_batch_tune(self, stream=None):
        n = len(self.groups)
        tiles, grids = (_int * n)(), (_i64 * n)()
        _bcheck(_lib.ax_batch_tune(self.b, tiles, grids, _stream(stream)), self.b)
        return {N: (tiles[i], grids[i]) for i, N in enumerate(self.groups)}

    def ax_batch_pcg(self, b_global, x_global, rtol=1e-8, maxit=10000, graph=1, stream=None, check=True):
        it, rr = (_int * self.B)(), (_dbl * self.B)()
        st = _lib.ax_batch_pcg(self.b, _ptr(b_global), _ptr(x_global), float(rtol), int(maxit), int(graph), it, rr,
                               _stream(stream))
        if check and st not in (AX_OK, AX_ENOTCONV):
            _bcheck(st, self.b)
        return list(it), list(rr), st

    def ax_batch_set_persistent(self, on: bool):
        _bcheck(_lib.ax_batch_set_persistent(self.b, int(bool(on))), self.b)

    def ax_batch_info(self) -> dict:
        """{"persistent": 0/1, "local_launches": L, "iteration_launches": I}."""
        p, l, i = _int(0), _int(0), _int(0)
        _bcheck(_lib.ax_batch_info(self.b, ctypes.byref(p), ctypes.byref(l), ctypes.byref(i)), self.b)
        return {"persistent": p.value, "local_launches": l.value, "iteration_launches": i.value}

    def ax_batch_set_wait(self, budget_ns: int, stuck_mesh: int = -1):
        _bcheck(_lib.ax_batch_set_wait(self.b, int(budget_ns), int(stuck_mesh)), self.b)

    def ax_batch_destroy(self):
        if self.b:
            _lib.ax_batch_destroy(self.b)
            self.b = _vp()

    def __del__(self):
        try:
            self.ax_batch_destroy()
        except Exception:
            pass


def _mcheck(st: int, m=None):
    if st != AX_OK:
        raise AxError(st, _lib.ax_mlp_last_error(m).decode())


class AxMLP:
    """Owns an ax_mlp (the learned preconditioner's network).  Names follow the C ABI."""

    IN, IN_PAD, HID, OUT = 536, 544, 512, 512

    def __init__(self, seed: int = 0, stream=None):
        self.m = _vp()
        _mcheck(_lib.ax_mlp_create(ctypes.byref(self.m), int(seed), _stream(stream)))
        self.num_params = int(_lib.ax_mlp_num_params(self.m))

    def ax_mlp_get_params(self, out=None, stream=None):
        import numpy as np
        out = np.empty(self.num_params, dtype=np.float32) if out is None else out
        _mcheck(_lib.ax_mlp_get_params(self.m, _ptr(out), _stream(stream)), self.m)
        return out

    def ax_mlp_set_params(self, params, stream=None):
        _mcheck(_lib.ax_mlp_set_params(self.m, _ptr(params), _stream(stream)), self.m)

    def ax_mlp_forward(self, X_bf16, Y, stream=None):
        _mcheck(_lib.ax_mlp_forward(self.m, _ptr(X_bf16), _ptr(Y), int(X_bf16.shape[0]), _stream(stream)), self.m)
        return Y

    def ax_mlp_grad(self, X_bf16, T, grads=None, stream=None):
        import numpy as np
        grads = np.empty(self.num_params, dtype=np.float32) if grads is None else grads
        loss = ctypes.c_float(0.0)
        _mcheck(_lib.ax_mlp_grad(self.m, _ptr(X_bf16), _ptr(T), int(X_bf16.shape[0]), ctypes.byref(loss), _ptr(grads),
                                 _stream(stream)), self.m)
        return loss.value, grads

    def ax_mlp_train(self, X_bf16, T, epochs=4, batch=4096, lr=1e-3, seed=0, stream=None):
        import numpy as np
        hist = np.zeros(int(epochs), dtype=np.float32)
        _mcheck(_lib.ax_mlp_train(self.m, _ptr(X_bf16), _ptr(T), int(X_bf16.shape[0]), int(epochs), int(batch),
                                  float(lr), int(seed), _ptr(hist), _stream(stream)), self.m)
        return hist

    def ax_mlp_destroy(self):
        if self.m:
            _lib.ax_mlp_destroy(self.m)
            self.m = _vp()

    def __del__(self):
        try:
            self.ax_mlp_destroy()
        except Exception:
            pass


def ax_mlp_pairs(op: "Ax", b_global, x_star, x_k, elements, F_bf16, T, stream=None):
    _mcheck(_lib.ax_mlp_pairs(op.ctx, _ptr(b_global), _ptr(x_star), _ptr(x_k), _ptr(elements), int(elements.numel()),
                              _ptr(F_bf16), _ptr(T), _stream(stream)))
    return F_bf16, T


def pcg_solve_learned(op: "Ax", mlp: AxMLP, b_global, x_global, rtol=1e-8, maxit=10000, omega=0.5, stream=None,
                      check=True):
    """Returns (iterations, relative residual, status, fell_back)."""
    it, rr, fb = _int(0), _dbl(0.0), _int(0)
    st = _lib.pcg_solve_learned(op.ctx, mlp.m, _ptr(b_global), _ptr(x_global), float(rtol), int(maxit), float(omega),
                                ctypes.byref(it), ctypes.byref(rr), ctypes.byref(fb), _stream(stream))
    if check and st not in (AX_OK, AX_ENOTCONV):
        _mcheck(st, mlp.m)
    return it.value, rr.value, st, fb.value
