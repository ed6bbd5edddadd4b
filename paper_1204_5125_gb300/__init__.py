"""Python binding of the GB300 Ginzburg-Landau Jacobian-solve library.

Thin ctypes marshalling over the C ABI in ``include/gl.h``: every function
below has the name of the C entry point it calls, takes torch tensors (CUDA,
complex128, contiguous) for device buffers and numpy arrays for host outputs,
and raises :class:`GLError` on a non-GL_OK status.  All arithmetic happens in
the CUDA library ``_build/libgl_gb300.so``; nothing here falls back to the CPU.
If the library cannot be loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB, build as _build

__all__ = [
    "GLError", "Options", "SolveInfo", "GL_FP64", "GL_MIXED", "GL_MIXED_PRECOND", "library", "options",
    "gl_options_default", "gl_mesh_create", "gl_mesh_destroy", "gl_mesh_info", "gl_mesh_nedges", "gl_mesh_edges",
    "gl_mesh_khat", "gl_residual", "gl_jacobian_apply", "gl_precond_setup", "gl_precond_apply",
    "gl_precond_destroy", "gl_precond_levels", "gl_precond_level_info", "gl_precond_level_aggregates",
    "gl_precond_level_colors", "gl_precond_level_matrix", "gl_precond_level_P", "gl_jacobian_solve",
    "gl_newton_step", "gl_batch_solve", "gl_batch_create", "gl_batch_run", "gl_batch_destroy",
    "gl_profile_begin", "gl_profile_end", "gl_jacobian_apply_noalloc", "gl_precond_cost",
    "gl_warmstart_create", "gl_warmstart_destroy", "gl_warmstart_get_params", "gl_warmstart_set_params",
    "gl_warmstart_predict", "gl_warmstart_grad", "gl_warmstart_train", "gl_warmstart_adam_step", "GL_WS_NPARAM",
    "gl_last_error", "EXPORTED", "GL_CYCLES_INF", "ContOptions", "ContPoint", "gl_mesh_create_edge",
    "gl_mesh_set_mu", "gl_residual_dmu", "gl_energy", "cont_options", "gl_continuation", "gl_precond_setup_like",
    "GL_COLOR_SL", "GL_COLOR_JP", "GL_COLOR_PSL", "gl_mesh_create_dipole", "gl_mesh_create_simplicial", "gl_precond_apply_precision", "gl_precond_debug",
    "GL_DEBUG_STALL_SWEEPS", "GL_DEBUG_NEGATE_COARSEST", "gl_precond_level_sweep", "gl_measure_fma_peak",
    "gl_measure_sync_latency", "GL_APPLY_FP64_TABLES",
    "gl_profile_flops",
]

GL_FP64, GL_MIXED, GL_MIXED_PRECOND = 0, 1, 2
GL_APPLY_FP64_TABLES = 3  # gl_jacobian_apply: the FP64 apply from the lattice stencil's FP64 tables
GL_CYCLES_INF = -1  # options.cycles: R_inf, the V-cycle repeated until the 1e-12 residual test
GL_COLOR_SL, GL_COLOR_JP, GL_COLOR_PSL = 0, 1, 2  # options.coloring of the coarse levels
GL_DEBUG_STALL_SWEEPS, GL_DEBUG_NEGATE_COARSEST = 1, 2  # gl_precond_debug actions (fault injection for tests)
STATUS = {0: "GL_OK", 1: "GL_ERR_ARG", 2: "GL_ERR_CUDA", 3: "GL_ERR_OOM", 4: "GL_ERR_NOT_CONVERGED",
          5: "GL_ERR_BREAKDOWN", 6: "GL_ERR_NAN", 7: "GL_ERR_TIMEOUT", 8: "GL_ERR_CAPACITY"}

# every entry point declared in include/gl.h
EXPORTED = [
    "gl_options_default", "gl_mesh_create", "gl_mesh_destroy", "gl_mesh_info", "gl_residual", "gl_jacobian_apply",
    "gl_precond_setup", "gl_precond_apply", "gl_precond_destroy", "gl_precond_levels", "gl_precond_level_info",
    "gl_precond_level_aggregates", "gl_precond_level_colors", "gl_precond_level_matrix", "gl_precond_level_P",
    "gl_mesh_nedges", "gl_mesh_edges", "gl_mesh_khat", "gl_jacobian_solve", "gl_newton_step", "gl_batch_solve",
    "gl_profile_begin", "gl_profile_end", "gl_jacobian_apply_noalloc", "gl_batch_create", "gl_batch_run",
    "gl_batch_destroy", "gl_precond_cost", "gl_warmstart_create", "gl_warmstart_destroy", "gl_warmstart_get_params",
    "gl_warmstart_set_params", "gl_warmstart_predict", "gl_warmstart_grad", "gl_warmstart_train",
    "gl_warmstart_adam_step", "gl_last_error", "gl_mesh_create_edge", "gl_mesh_set_mu", "gl_residual_dmu",
    "gl_energy", "gl_cont_options_default", "gl_continuation", "gl_precond_setup_like", "gl_mesh_create_dipole",
    "gl_mesh_create_simplicial",
    "gl_precond_apply_precision", "gl_precond_debug", "gl_precond_level_sweep", "gl_measure_fma_peak",
    "gl_measure_sync_latency",
    "gl_profile_flops",
]

GL_WS_NPARAM = 4 * 64 * 128 + 2 * 64


class GLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("maxit", C.c_int), ("cycles", C.c_int), ("max_coarse", C.c_int),
        ("max_levels", C.c_int), ("power_its", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double),
        ("max_outer", C.c_int), ("check_every", C.c_int), ("autotune", C.c_int), ("lattice", C.c_int),
        ("cluster_sweeps", C.c_int),
        ("warmstart", C.c_void_p), ("coloring", C.c_int), ("sweep_sync", C.c_int), ("coarse_df", C.c_int),
        ("device_loop", C.c_int), ("warmstart_hint", C.c_void_p),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("outer_iters", C.c_int), ("converged", C.c_int), ("true_relres", C.c_double),
        ("est_relres", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
        ("warmstart_used", C.c_int), ("lattice_stencil", C.c_int), ("df_jacobian", C.c_int),
        ("stall_restarts", C.c_int), ("matvec_equiv", C.c_double), ("cycles_per_apply", C.c_double),
        ("jacobian_tables", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ContOptions(C.Structure):
    _fields_ = [
        ("ds", C.c_double), ("ds_min", C.c_double), ("ds_max", C.c_double), ("mu_max", C.c_double),
        ("max_steps", C.c_int), ("newton_tol", C.c_double), ("newton_maxit", C.c_int), ("solver", Options),
    ]


class ContPoint(C.Structure):
    _fields_ = [
        ("mu", C.c_double), ("energy", C.c_double), ("gl_norm", C.c_double), ("ds", C.c_double),
        ("newton_steps", C.c_int), ("iters_last", C.c_int), ("iters_total", C.c_int), ("retries", C.c_int),
        ("setup_ms", C.c_double), ("solve_ms", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None
vp = C.c_void_p
i64p = C.POINTER(C.c_int64)


def library(build_if_missing: bool = True):
    """Loads (building first if needed) the CUDA library and declares signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build() if build_if_missing else LIB
        if not os.path.exists(path):
            raise OSError(f"CUDA library not built: {path}")
        L = C.CDLL(path)
        sig = {
            "gl_options_default": [C.POINTER(Options)],
            "gl_mesh_create": [C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), vp, C.POINTER(vp)],
            "gl_mesh_destroy": [vp],
            "gl_mesh_info": [vp, i64p, i64p, vp],
            "gl_mesh_nedges": [vp, i64p],
            "gl_mesh_edges": [vp, vp, vp, vp, vp],
            "gl_mesh_khat": [vp, vp, vp, vp],
            "gl_residual": [vp, vp, vp, vp],
            "gl_jacobian_apply": [vp, vp, vp, vp, C.c_int, vp],
            "gl_precond_setup": [vp, vp, C.POINTER(Options), vp, C.POINTER(vp)],
            "gl_precond_apply": [vp, vp, vp, vp],
            "gl_precond_apply_precision": [vp, vp, vp, C.c_int, vp],
            "gl_precond_debug": [vp, C.c_int],
            "gl_measure_fma_peak": [C.c_int, C.POINTER(C.c_double), vp],
            "gl_measure_sync_latency": [C.POINTER(C.c_double), vp],
            "gl_profile_flops": [C.POINTER(C.c_double)],
            "gl_precond_level_sweep": [vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)],
            "gl_precond_destroy": [vp],
            "gl_precond_levels": [vp, C.POINTER(C.c_int)],
            "gl_precond_level_info": [vp, C.c_int, i64p, i64p, C.POINTER(C.c_int32), i64p, C.POINTER(C.c_double)],
            "gl_precond_level_aggregates": [vp, C.c_int, vp],
            "gl_precond_level_colors": [vp, C.c_int, vp],
            "gl_precond_level_matrix": [vp, C.c_int, vp, vp, vp],
            "gl_precond_level_P": [vp, C.c_int, vp, vp, vp],
            "gl_jacobian_solve": [vp, vp, vp, vp, vp, C.POINTER(Options), C.POINTER(SolveInfo), vp],
            "gl_newton_step": [vp, vp, C.POINTER(Options), C.POINTER(SolveInfo), C.POINTER(C.c_double), vp],
            "gl_batch_solve": [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                               C.POINTER(Options), C.POINTER(SolveInfo), vp],
            "gl_profile_begin": [C.c_char_p, C.c_int],
            "gl_jacobian_apply_noalloc": [vp, vp, vp, vp, vp],
            "gl_batch_create": [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(Options), vp, C.POINTER(vp)],
            "gl_batch_run": [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveInfo), vp],
            "gl_batch_destroy": [vp],
            "gl_profile_end": [i64p, i64p, C.POINTER(C.c_double), C.POINTER(C.c_double)],
            "gl_precond_cost": [vp, C.c_int, C.POINTER(C.c_double)],
            "gl_warmstart_create": [vp, C.POINTER(vp)],
            "gl_warmstart_destroy": [vp],
            "gl_warmstart_get_params": [vp, vp],
            "gl_warmstart_set_params": [vp, vp],
            "gl_warmstart_predict": [vp, vp, vp, vp, vp, vp, vp],
            "gl_warmstart_grad": [vp, vp, vp, vp, vp, vp, C.POINTER(C.c_double), vp],
            "gl_warmstart_train": [vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.c_int,
                                   C.c_int, C.c_float, vp, vp],
            "gl_warmstart_adam_step": [vp, vp, C.c_float],
            "gl_mesh_create_edge": [C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double), vp,
                                    C.POINTER(vp)],
            "gl_mesh_set_mu": [vp, C.c_double, vp],
            "gl_mesh_create_simplicial": [C.c_int, C.c_int64, vp, C.c_int64, vp, C.c_double, vp, vp, vp, vp,
                                          C.POINTER(vp)],
            "gl_mesh_create_dipole": [C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), vp, C.POINTER(vp)],
            "gl_precond_setup_like": [vp, vp, C.POINTER(Options), vp, vp, C.POINTER(vp)],
            "gl_residual_dmu": [vp, vp, vp, vp],
            "gl_energy": [vp, vp, C.POINTER(C.c_double), vp],
            "gl_cont_options_default": [C.POINTER(ContOptions)],
            "gl_continuation": [vp, vp, C.POINTER(ContOptions), C.POINTER(ContPoint), C.c_int, C.POINTER(C.c_int),
                                C.POINTER(vp), vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.gl_last_error.restype = C.c_char_p
        L.gl_last_error.argtypes = []
        _lib = L
        return L


def gl_last_error() -> str:
    return library().gl_last_error().decode()


def _check(st: int):
    if st != 0:
        raise GLError(st, gl_last_error())


def _ptr(t):
    """Device pointer of a contiguous complex128/float64 CUDA tensor."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def gl_options_default() -> Options:
    o = Options()
    _check(library().gl_options_default(C.byref(o)))
    return o


def options(**kw) -> Options:
    o = gl_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def gl_mesh_create(dim: int, n_per_side: int, mu: float, bhat=(0.0, 0.0, 1.0), stream=None, edge: float = 1.0):
    b = (C.c_double * 3)(*bhat)
    out = C.c_void_p()
    if edge == 1.0:
        _check(library().gl_mesh_create(dim, n_per_side, float(mu), b, _stream(stream), C.byref(out)))
    else:
        _check(library().gl_mesh_create_edge(dim, n_per_side, float(edge), float(mu), b, _stream(stream),
                                             C.byref(out)))
    return out


def gl_mesh_create_edge(dim: int, n_per_side: int, edge: float, mu: float, bhat=(0.0, 0.0, 1.0), stream=None):
    b = (C.c_double * 3)(*bhat)
    out = C.c_void_p()
    _check(library().gl_mesh_create_edge(dim, n_per_side, float(edge), float(mu), b, _stream(stream), C.byref(out)))
    return out


def gl_mesh_create_dipole(dim: int, n_per_side: int, edge: float, mu: float, x0=(0.0, 0.0, 6.0),
                          mom=(0.0, 0.0, 1.0), stream=None):
    """Mesh in mu A_d, the field of a dipole of moment `mom` at `x0`."""
    a = (C.c_double * 3)(*x0)
    b = (C.c_double * 3)(*mom)
    out = C.c_void_p()
    _check(library().gl_mesh_create_dipole(dim, n_per_side, float(edge), float(mu), a, b, _stream(stream),
                                           C.byref(out)))
    return out


def gl_mesh_create_simplicial(dim: int, x, simplices, mu: float, bhat=None, dipole=None, stream=None):
    """A general simplicial mesh: x (n x 3, or n x dim), simplices (m x (dim + 1)) node
    ids (host arrays); A = (mu/2) bhat x x, or mu A_d with dipole=(x0, m)."""
    x = np.asarray(x, dtype=np.float64)
    if x.shape[1] == 2:
        x = np.hstack([x, np.zeros((x.shape[0], 1))])
    x = np.ascontiguousarray(x)
    sp = np.ascontiguousarray(simplices, dtype=np.int32)
    b = None if bhat is None else (C.c_double * 3)(*bhat)
    xd = md = None
    if dipole is not None:
        xd = (C.c_double * 3)(*dipole[0])
        md = (C.c_double * 3)(*dipole[1])
    out = C.c_void_p()
    _check(library().gl_mesh_create_simplicial(dim, x.shape[0], x.ctypes.data, sp.shape[0], sp.ctypes.data,
                                               float(mu), b, xd, md, _stream(stream), C.byref(out)))
    return out


def gl_mesh_set_mu(mesh, mu: float, stream=None):
    _check(library().gl_mesh_set_mu(mesh, float(mu), _stream(stream)))


def gl_residual_dmu(mesh, psi, out, stream=None):
    _check(library().gl_residual_dmu(mesh, _ptr(psi), _ptr(out), _stream(stream)))


def gl_energy(mesh, psi, stream=None) -> float:
    F = C.c_double()
    _check(library().gl_energy(mesh, _ptr(psi), C.byref(F), _stream(stream)))
    return F.value


def cont_options(**kw) -> ContOptions:
    """gl_cont_options_default() with fields overridden; solver=dict(...) overrides solver fields."""
    o = ContOptions()
    _check(library().gl_cont_options_default(C.byref(o)))
    for k, v in kw.items():
        if k == "solver":
            for sk, sv in v.items():
                setattr(o.solver, sk, sv)
        else:
            setattr(o, k, v)
    return o


def gl_continuation(mesh, psi, opts: ContOptions | None = None, max_points: int = 256, states=None, stream=None,
                    raise_on_fail: bool = True):
    """Runs the pseudo-arclength continuation; returns (status, list of point dicts)."""
    if opts is None:
        opts = cont_options()
    pts = (ContPoint * max_points)()
    npts = C.c_int()
    st_arr = None
    if states is not None:
        st_arr = (vp * max_points)(*[_ptr(t).value for t in states] + [None] * (max_points - len(states)))
    st = library().gl_continuation(mesh, _ptr(psi), C.byref(opts), pts, int(max_points), C.byref(npts), st_arr,
                                   _stream(stream))
    if st != 0 and (raise_on_fail or st != 4):
        _check(st)
    return st, [pts[i].as_dict() for i in range(npts.value)]


def gl_mesh_destroy(mesh):
    _check(library().gl_mesh_destroy(mesh))


def gl_mesh_info(mesh, volumes=None):
    n, nnz = C.c_int64(), C.c_int64()
    _check(library().gl_mesh_info(mesh, C.byref(n), C.byref(nnz), _ptr(volumes) if volumes is not None else None))
    return n.value, nnz.value


def gl_mesh_nedges(mesh) -> int:
    ne = C.c_int64()
    _check(library().gl_mesh_nedges(mesh, C.byref(ne)))
    return ne.value


def gl_mesh_edges(mesh):
    ne = gl_mesh_nedges(mesh)
    ej, ek = np.zeros(ne, np.int32), np.zeros(ne, np.int32)
    al, th = np.zeros(ne), np.zeros(ne)
    _check(library().gl_mesh_edges(mesh, ej.ctypes.data, ek.ctypes.data, al.ctypes.data, th.ctypes.data))
    return ej, ek, al, th


def gl_mesh_khat(mesh):
    n, nnz = gl_mesh_info(mesh)
    rp, ci, v = np.zeros(n + 1, np.int64), np.zeros(nnz, np.int32), np.zeros(nnz, np.complex128)
    _check(library().gl_mesh_khat(mesh, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    return rp, ci, v


def gl_residual(mesh, psi, r, stream=None):
    _check(library().gl_residual(mesh, _ptr(psi), _ptr(r), _stream(stream)))


def gl_jacobian_apply(mesh, psi, phi, y, precision=GL_FP64, stream=None):
    _check(library().gl_jacobian_apply(mesh, _ptr(psi), _ptr(phi), _ptr(y), int(precision), _stream(stream)))


def gl_jacobian_apply_noalloc(mesh, psi, phi, y, stream=None):
    """FP64 Jacobian apply that allocates no device memory (static scratch; see gl.h)."""
    _check(library().gl_jacobian_apply_noalloc(mesh, _ptr(psi), _ptr(phi), _ptr(y), _stream(stream)))


def gl_precond_setup(mesh, psi, opts: Options | None = None, stream=None):
    out = C.c_void_p()
    o = opts if opts is not None else gl_options_default()
    _check(library().gl_precond_setup(mesh, _ptr(psi), C.byref(o), _stream(stream), C.byref(out)))
    return out


def gl_precond_setup_like(mesh, psi, like, opts: Options | None = None, stream=None):
    """Setup for a new psi / mu taking over `like`'s aggregates, colours and kernel choices."""
    out = C.c_void_p()
    o = opts if opts is not None else gl_options_default()
    _check(library().gl_precond_setup_like(mesh, _ptr(psi), C.byref(o), like, _stream(stream), C.byref(out)))
    return out


def gl_precond_apply(prec, x, z, stream=None):
    _check(library().gl_precond_apply(prec, _ptr(x), _ptr(z), _stream(stream)))


def gl_precond_apply_precision(prec, x, z, precision=GL_FP64, stream=None):
    _check(library().gl_precond_apply_precision(prec, _ptr(x), _ptr(z), precision, _stream(stream)))


def gl_precond_debug(prec, action: int):
    _check(library().gl_precond_debug(prec, action))


def gl_precond_level_sweep(prec, level: int, precision=GL_FP64) -> dict:
    """How a level's Gauss-Seidel steps run: lanes per row, sync (0 grid barrier,
    1 neighbour flags, 3 cluster, -1 none) and CTAs."""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(library().gl_precond_level_sweep(prec, level, precision, C.byref(a), C.byref(b), C.byref(c)))
    return dict(lanes=a.value, sync=b.value, ctas=c.value)


def gl_measure_fma_peak(precision=GL_FP64, stream=None) -> float:
    """Measured FMA rate of the GPU in GFLOP/s (GL_FP64 or GL_MIXED for FP32)."""
    g = C.c_double()
    _check(library().gl_measure_fma_peak(precision, C.byref(g), _stream(stream)))
    return g.value


def gl_measure_sync_latency(stream=None) -> dict:
    """Hand-off (median, max), dependent L2 load and store + fence latencies in ns."""
    out = (C.c_double * 4)()
    _check(library().gl_measure_sync_latency(out, _stream(stream)))
    return dict(handoff_ns=out[0], handoff_max_ns=out[1], l2_load_ns=out[2], fence_ns=out[3])


def gl_precond_destroy(prec):
    _check(library().gl_precond_destroy(prec))


def gl_precond_levels(prec) -> int:
    n = C.c_int()
    _check(library().gl_precond_levels(prec, C.byref(n)))
    return n.value


def gl_precond_level_info(prec, level: int) -> dict:
    n, nnz, pnnz = C.c_int64(), C.c_int64(), C.c_int64()
    nc = C.c_int32()
    om = C.c_double()
    _check(library().gl_precond_level_info(prec, level, C.byref(n), C.byref(nnz), C.byref(nc), C.byref(pnnz),
                                           C.byref(om)))
    return dict(n=n.value, nnz=nnz.value, ncolors=nc.value, p_nnz=pnnz.value, omega=om.value)


def gl_precond_level_aggregates(prec, level: int):
    a = np.zeros(gl_precond_level_info(prec, level)["n"], np.int32)
    _check(library().gl_precond_level_aggregates(prec, level, a.ctypes.data))
    return a


def gl_precond_level_colors(prec, level: int):
    a = np.zeros(gl_precond_level_info(prec, level)["n"], np.int32)
    _check(library().gl_precond_level_colors(prec, level, a.ctypes.data))
    return a


def gl_precond_level_matrix(prec, level: int):
    info = gl_precond_level_info(prec, level)
    rp, ci, v = np.zeros(info["n"] + 1, np.int64), np.zeros(info["nnz"], np.int32), np.zeros(info["nnz"], complex)
    _check(library().gl_precond_level_matrix(prec, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    return rp, ci, v


def gl_precond_level_P(prec, level: int):
    info = gl_precond_level_info(prec, level)
    rp, ci, v = np.zeros(info["n"] + 1, np.int64), np.zeros(info["p_nnz"], np.int32), np.zeros(info["p_nnz"], complex)
    _check(library().gl_precond_level_P(prec, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    return rp, ci, v


def gl_jacobian_solve(mesh, psi, prec, b, x, opts: Options | None = None, stream=None, raise_on_fail=True):
    """Solves J(psi) x = b in place (x holds the initial guess). Returns (status, SolveInfo)."""
    o = opts if opts is not None else gl_options_default()
    info = SolveInfo()
    st = library().gl_jacobian_solve(mesh, _ptr(psi), prec if prec is not None else None, _ptr(b), _ptr(x),
                                     C.byref(o), C.byref(info), _stream(stream))
    if raise_on_fail and st not in (0, 4):
        _check(st)
    return st, info


def gl_newton_step(mesh, psi, opts: Options | None = None, stream=None):
    o = opts if opts is not None else gl_options_default()
    info = SolveInfo()
    gn = C.c_double()
    st = library().gl_newton_step(mesh, _ptr(psi), C.byref(o), C.byref(info), C.byref(gn), _stream(stream))
    if st not in (0, 4):
        _check(st)
    return st, info, gn.value


def _vparr(xs_):
    return (vp * len(xs_))(*[x.value if isinstance(x, C.c_void_p) else _ptr(x).value for x in xs_])


def gl_batch_create(meshes, psis, opts: Options | None = None, stream=None):
    o = opts if opts is not None else gl_options_default()
    out = C.c_void_p()
    _check(library().gl_batch_create(len(meshes), _vparr(meshes), _vparr(psis), C.byref(o), _stream(stream),
                                     C.byref(out)))
    return out


def gl_batch_run(batch, bs, xs, stream=None):
    infos = (SolveInfo * len(bs))()
    st = library().gl_batch_run(batch, _vparr(bs), _vparr(xs), infos, _stream(stream))
    if st not in (0, 4):
        _check(st)
    return st, list(infos)


def gl_batch_destroy(batch):
    _check(library().gl_batch_destroy(batch))


def gl_batch_solve(meshes, psis, bs, xs, opts: Options | None = None, stream=None):
    k = len(meshes)
    o = opts if opts is not None else gl_options_default()
    arr = lambda xs_: (vp * k)(*[x.value if isinstance(x, C.c_void_p) else _ptr(x).value for x in xs_])
    infos = (SolveInfo * k)()
    st = library().gl_batch_solve(k, arr(meshes), arr(psis), arr(bs), arr(xs), C.byref(o), infos, _stream(stream))
    if st not in (0, 4):
        _check(st)
    return st, list(infos)


def gl_profile_begin(kernel_class: str | None = None, max_launches: int = 0):
    _check(library().gl_profile_begin(kernel_class.encode() if kernel_class else None, int(max_launches)))


def gl_profile_end() -> dict:
    la, ti = C.c_int64(), C.c_int64()
    ms, by = C.c_double(), C.c_double()
    _check(library().gl_profile_end(C.byref(la), C.byref(ti), C.byref(ms), C.byref(by)))
    fl = C.c_double()
    _check(library().gl_profile_flops(C.byref(fl)))
    return dict(launches=la.value, timed=ti.value, ms=ms.value, bytes=by.value, flops=fl.value)


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != GL_WS_NPARAM:
        raise ValueError(f"expected {GL_WS_NPARAM} parameters, got {a.size}")
    return a


def gl_warmstart_create(params=None):
    """New warm-start network (params: GL_WS_NPARAM floats, None = zeros)."""
    out = C.c_void_p()
    p = None if params is None else _f32(params)
    _check(library().gl_warmstart_create(None if p is None else p.ctypes.data_as(vp), C.byref(out)))
    return out


def gl_warmstart_destroy(ws):
    _check(library().gl_warmstart_destroy(ws))


def gl_warmstart_get_params(ws) -> np.ndarray:
    out = np.zeros(GL_WS_NPARAM, np.float32)
    _check(library().gl_warmstart_get_params(ws, out.ctypes.data_as(vp)))
    return out


def gl_warmstart_set_params(ws, params):
    p = _f32(params)
    _check(library().gl_warmstart_set_params(ws, p.ctypes.data_as(vp)))


def _optptr(t):
    return _ptr(t) if t is not None else None


def gl_warmstart_predict(ws, mesh, psi, b, x0, stream=None, hint=None):
    """x0 = the network's guess; hint (nullable): a vector the solution should resemble."""
    _check(library().gl_warmstart_predict(ws, mesh, _ptr(psi), _ptr(b), _optptr(hint), _ptr(x0), _stream(stream)))


def gl_warmstart_grad(ws, mesh, psi, b, stream=None, hint=None):
    """(loss, gradient as GL_WS_NPARAM float32) of one sample."""
    g = np.zeros(GL_WS_NPARAM, np.float32)
    L = C.c_double()
    _check(library().gl_warmstart_grad(ws, mesh, _ptr(psi), _ptr(b), _optptr(hint), g.ctypes.data_as(vp), C.byref(L),
                                       _stream(stream)))
    return L.value, g


def gl_warmstart_train(ws, meshes, psis, bs, steps: int, batch: int = 1, lr: float = 1e-3, stream=None,
                       hints=None):
    """Adam training on samples (meshes[k], psis[k], bs[k][, hints[k]]); returns the mean
    loss of every step.  hints: None, or one tensor or None per sample."""
    losses = np.zeros(max(steps, 1), np.float64)
    harr = None
    if hints is not None:
        harr = (vp * len(hints))(*[_ptr(h).value if h is not None else None for h in hints])
    _check(library().gl_warmstart_train(ws, len(meshes), _vparr(meshes), _vparr(psis), _vparr(bs), harr,
                                        int(steps), int(batch), float(lr), losses.ctypes.data_as(vp),
                                        _stream(stream)))
    return losses[:steps]


def gl_warmstart_adam_step(ws, grad, lr: float):
    g = _f32(grad)
    _check(library().gl_warmstart_adam_step(ws, g.ctypes.data_as(vp), float(lr)))


def gl_precond_cost(prec, cycles: int = 1) -> float:
    """Cost of R_k in matrix-vector-product equivalents (Fig. 1)."""
    c = C.c_double()
    _check(library().gl_precond_cost(prec, int(cycles), C.byref(c)))
    return c.value
