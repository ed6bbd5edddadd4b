"""Python access to the CPU oracle (``oracle/glref.c``) through ctypes.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports this package, and this package never imports the CUDA library.

All complex arrays are numpy complex128 (interleaved re/im doubles).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

CYCLES_INF = -1        # options(cycles=CYCLES_INF): R_inf, the V-cycle repeated to high accuracy
RINF_TOL = 1e-12       # ... until ||D^-1 (D v - P-hat z)||_D <= RINF_TOL ||v||_D
RINF_MAXCYC = 200      # ... or this many cycles

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libglref.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile glref.c into a shared library with gcc (plain C11, -O2, OpenMP for the
    optional multi-threaded row loops)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_c128p = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class Options(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("maxit", C.c_int),
        ("cycles", C.c_int),
        ("max_coarse", C.c_int),
        ("max_levels", C.c_int),
        ("power_its", C.c_int),
        ("coloring", C.c_int),
    ]


class Info(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("converged", C.c_int),
        ("true_relres", C.c_double),
        ("est_relres", C.c_double),
    ]


def set_threads(n: int) -> int:
    """Host threads for the oracle's row loops (results do not depend on it); 0 or
    less: every processor.  Returns the count now in use."""
    L = lib()
    L.glref_set_threads(int(n) if n > 0 else L.glref_max_threads())
    return L.glref_get_threads()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.glref_mesh_create.restype = vp
            L.glref_mesh_create.argtypes = [C.c_int, C.c_int, C.c_double, _f64p, _f64p]
            L.glref_mesh_create_edge.restype = vp
            L.glref_mesh_create_edge.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _f64p, _f64p]
            L.glref_mesh_create_dipole.restype = vp
            L.glref_mesh_create_dipole.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _f64p, _f64p]
            L.glref_mesh_create_simplicial.restype = vp
            L.glref_mesh_create_simplicial.argtypes = [C.c_int, C.c_int64, _f64p, C.c_int64,
                                                       np.ctypeslib.ndpointer(np.int32, flags="C"), C.c_double,
                                                       vp, vp, vp]
            L.glref_set_threads.argtypes = [C.c_int]
            L.glref_get_threads.restype = C.c_int
            L.glref_max_threads.restype = C.c_int
            L.glref_edge_integral1.restype = C.c_double
            L.glref_edge_integral1.argtypes = [vp, _f64p, _f64p]
            L.glref_residual_dmu.argtypes = [vp, _c128p, _c128p]
            L.glref_mesh_destroy.argtypes = [vp]
            for f in ("glref_mesh_n", "glref_mesh_nedges", "glref_mesh_nnz"):
                getattr(L, f).restype = C.c_int64
                getattr(L, f).argtypes = [vp]
            L.glref_mesh_nodes.argtypes = [vp, _f64p]
            L.glref_mesh_volumes.argtypes = [vp, _f64p]
            L.glref_mesh_edges.argtypes = [vp, _i32p, _i32p, _f64p, _f64p]
            L.glref_mesh_khat.argtypes = [vp, _i64p, _i32p, _c128p]
            L.glref_kinetic_apply.argtypes = [vp, _c128p, _c128p]
            L.glref_residual.argtypes = [vp, _c128p, _c128p]
            L.glref_jacobian_apply.argtypes = [vp, _c128p, _c128p, _c128p]
            L.glref_energy.restype = C.c_double
            L.glref_energy.argtypes = [vp, _c128p]
            L.glref_inner_r.restype = C.c_double
            L.glref_inner_r.argtypes = [vp, _c128p, _c128p]
            L.glref_simplex_alpha_linsys.restype = C.c_int
            L.glref_simplex_alpha_linsys.argtypes = [C.c_int, _f64p, _f64p]
            L.glref_simplex_alpha_dihedral.restype = C.c_int
            L.glref_simplex_alpha_dihedral.argtypes = [_f64p, _f64p]
            L.glref_simplex_alpha_cot.restype = C.c_int
            L.glref_simplex_alpha_cot.argtypes = [_f64p, _f64p]
            L.glref_hash32.restype = C.c_uint32
            L.glref_hash32.argtypes = [C.c_uint32]
            L.glref_aggregate.restype = C.c_int64
            L.glref_aggregate.argtypes = [C.c_int64, _i64p, _i32p, _i32p]
            L.glref_color_jp.restype = C.c_int32
            L.glref_color_jp.argtypes = [C.c_int64, _i64p, _i32p, _i32p]
            L.glref_color_psl.restype = C.c_int32
            L.glref_color_psl.argtypes = [C.c_int64, _i64p, _i32p, _i32p, _i32p]
            L.glref_color_sl.restype = C.c_int32
            L.glref_color_sl.argtypes = [C.c_int64, _i64p, _i32p, _i32p, _i32p]
            L.glref_precond_setup.restype = vp
            L.glref_precond_setup.argtypes = [vp, _c128p, C.POINTER(Options)]
            L.glref_precond_destroy.argtypes = [vp]
            L.glref_prec_nlevels.restype = C.c_int
            L.glref_prec_nlevels.argtypes = [vp]
            L.glref_prec_level_info.argtypes = [
                vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                C.POINTER(C.c_int64), C.POINTER(C.c_double),
            ]
            L.glref_prec_level_matrix.argtypes = [vp, C.c_int, _i64p, _i32p, _c128p]
            L.glref_prec_level_P.argtypes = [vp, C.c_int, _i64p, _i32p, _c128p]
            L.glref_prec_level_aggregates.argtypes = [vp, C.c_int, _i32p]
            L.glref_prec_level_colors.argtypes = [vp, C.c_int, _i32p]
            L.glref_precond_apply.argtypes = [vp, _c128p, _c128p]
            L.glref_precond_apply_count.restype = C.c_int
            L.glref_precond_apply_count.argtypes = [vp, _c128p, _c128p]
            L.glref_vcycle.argtypes = [vp, C.c_int, _c128p, _c128p]
            L.glref_minres.restype = C.c_int
            L.glref_minres.argtypes = [vp, _c128p, vp, _c128p, _c128p, C.POINTER(Options), C.POINTER(Info)]
            L.glref_jacobian_solve.restype = C.c_int
            L.glref_jacobian_solve.argtypes = [vp, _c128p, _c128p, _c128p, C.POINTER(Options), C.POINTER(Info)]
            L.glref_newton_step.restype = C.c_int
            L.glref_newton_step.argtypes = [vp, _c128p, C.POINTER(Options), C.POINTER(Info), C.POINTER(C.c_double)]
            L.glref_jacobian_dense_real.argtypes = [vp, _c128p, _f64p]
            L.glref_lu_solve.restype = C.c_int
            L.glref_lu_solve.argtypes = [C.c_int64, _f64p, _f64p]
            L.glref_dense_solve.restype = C.c_int
            L.glref_dense_solve.argtypes = [vp, _c128p, _c128p, _c128p]
            L.glref_spectral_radius.restype = C.c_double
            _lib = L
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


# coarse-level colourings: smallest-last greedy, Jones-Plassmann, smallest-last in rounds (default)
COLOR_SL, COLOR_JP, COLOR_PSL = 0, 1, 2
PSL_SLACK = 4  # degree slack of one removal round of COLOR_PSL


def options(tol=1e-10, maxit=500, cycles=1, max_coarse=512, max_levels=10, power_its=20,
            coloring=COLOR_PSL) -> Options:
    return Options(tol, maxit, cycles, max_coarse, max_levels, power_its, coloring)


@dataclass
class SolveInfo:
    status: int
    iters: int
    converged: bool
    true_relres: float
    est_relres: float


class Mesh:
    """Structured square (dim=2) or cube (dim=3) mesh of N nodes per side on the
    square/cube of side `edge` centred at the origin, with A(x) = (mu/2) bhat x x + a0."""

    def __init__(self, dim: int, N: int, mu: float, bhat=(0.0, 0.0, 1.0), a0=(0.0, 0.0, 0.0), edge: float = 1.0,
                 dipole=None, _ptr=None):
        """dipole=(x0, m): A = mu A_d, the field of a dipole of moment m at x0 (bhat, a0 unused)."""
        self._lib = lib()
        if _ptr is not None:  # made by from_simplices
            self.ptr = _ptr
            self.dim, self.N, self.mu, self.edge = dim, 0, float(mu), 0.0
            self.bhat, self.a0 = tuple(float(c) for c in bhat), (0.0, 0.0, 0.0)
            self.n = self._lib.glref_mesh_n(self.ptr)
            self.nedges = self._lib.glref_mesh_nedges(self.ptr)
            self.nnz = self._lib.glref_mesh_nnz(self.ptr)
            return
        b = np.ascontiguousarray(bhat, dtype=np.float64)
        a = np.ascontiguousarray(a0, dtype=np.float64)
        if dipole is None:
            self.ptr = self._lib.glref_mesh_create_edge(dim, N, float(edge), float(mu), b, a)
        else:
            xd = np.ascontiguousarray(dipole[0], dtype=np.float64)
            md = np.ascontiguousarray(dipole[1], dtype=np.float64)
            self.ptr = self._lib.glref_mesh_create_dipole(dim, N, float(edge), float(mu), xd, md)
        if not self.ptr:
            raise ValueError("glref_mesh_create failed")
        self.dim, self.N, self.mu, self.edge = dim, N, float(mu), float(edge)
        self.bhat, self.a0 = tuple(float(c) for c in bhat), tuple(float(c) for c in a0)
        self.n = self._lib.glref_mesh_n(self.ptr)
        self.nedges = self._lib.glref_mesh_nedges(self.ptr)
        self.nnz = self._lib.glref_mesh_nnz(self.ptr)

    @classmethod
    def from_simplices(cls, dim: int, x, simplices, mu: float, bhat=(0.0, 0.0, 1.0), dipole=None):
        """A general simplicial mesh: x (n x 3, or n x dim), simplices (m x (dim + 1))
        node ids; A = (mu/2) bhat x x, or mu A_d with dipole=(x0, m)."""
        L = lib()
        x = np.asarray(x, dtype=np.float64)
        if x.shape[1] == 2:
            x = np.hstack([x, np.zeros((x.shape[0], 1))])
        x = np.ascontiguousarray(x)
        sp = np.ascontiguousarray(simplices, dtype=np.int32)
        b = np.ascontiguousarray(bhat, dtype=np.float64)
        xd = md = None
        if dipole is not None:
            xd = np.ascontiguousarray(dipole[0], dtype=np.float64)
            md = np.ascontiguousarray(dipole[1], dtype=np.float64)
        ptr = L.glref_mesh_create_simplicial(dim, x.shape[0], x.ravel(), sp.shape[0], sp.ravel(), float(mu),
                                             b.ctypes.data, xd.ctypes.data if xd is not None else None,
                                             md.ctypes.data if md is not None else None)
        if not ptr:
            raise ValueError("glref_mesh_create_simplicial failed")
        return cls(dim, 0, mu, bhat=bhat, _ptr=ptr)

    def __del__(self):
        p = getattr(self, "ptr", None)
        if p:
            self._lib.glref_mesh_destroy(p)
            self.ptr = None

    def nodes(self) -> np.ndarray:
        x = np.zeros(3 * self.n)
        self._lib.glref_mesh_nodes(self.ptr, x)
        return x.reshape(self.n, 3)

    def volumes(self) -> np.ndarray:
        v = np.zeros(self.n)
        self._lib.glref_mesh_volumes(self.ptr, v)
        return v

    def edges(self):
        ne = self.nedges
        ej, ek = np.zeros(ne, np.int32), np.zeros(ne, np.int32)
        al, th = np.zeros(ne), np.zeros(ne)
        self._lib.glref_mesh_edges(self.ptr, ej, ek, al, th)
        return ej, ek, al, th

    def khat_csr(self):
        rp = np.zeros(self.n + 1, np.int64)
        ci = np.zeros(self.nnz, np.int32)
        v = np.zeros(self.nnz, np.complex128)
        self._lib.glref_mesh_khat(self.ptr, rp, ci, v)
        return rp, ci, v

    def khat_dense(self) -> np.ndarray:
        rp, ci, v = self.khat_csr()
        K = np.zeros((self.n, self.n), np.complex128)
        for i in range(self.n):
            K[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        return K

    def kinetic(self, psi):
        y = np.zeros(self.n, np.complex128)
        self._lib.glref_kinetic_apply(self.ptr, _c128(psi), y)
        return y

    def residual(self, psi):
        r = np.zeros(self.n, np.complex128)
        self._lib.glref_residual(self.ptr, _c128(psi), r)
        return r

    def jacobian(self, psi, phi):
        y = np.zeros(self.n, np.complex128)
        self._lib.glref_jacobian_apply(self.ptr, _c128(psi), _c128(phi), y)
        return y

    def edge_integral1(self, xa, xb) -> float:
        """Integral of the mesh's potential per unit mu along the segment xa -> xb."""
        return self._lib.glref_edge_integral1(self.ptr, np.ascontiguousarray(xa, dtype=np.float64),
                                              np.ascontiguousarray(xb, dtype=np.float64))

    def residual_dmu(self, psi):
        """d GL / d mu at fixed psi."""
        out = np.zeros(self.n, np.complex128)
        self._lib.glref_residual_dmu(self.ptr, _c128(psi), out)
        return out

    def energy(self, psi) -> float:
        return self._lib.glref_energy(self.ptr, _c128(psi))

    def inner_r(self, x, y) -> float:
        return self._lib.glref_inner_r(self.ptr, _c128(x), _c128(y))

    def jacobian_dense_real(self, psi) -> np.ndarray:
        J = np.zeros((2 * self.n, 2 * self.n))
        self._lib.glref_jacobian_dense_real(self.ptr, _c128(psi), J)
        return J

    def dense_solve(self, psi, b):
        x = np.zeros(self.n, np.complex128)
        rc = self._lib.glref_dense_solve(self.ptr, _c128(psi), _c128(b), x)
        if rc:
            raise np.linalg.LinAlgError("singular realified Jacobian")
        return x

    def solve(self, psi, b, x0=None, **opts):
        """R_1-preconditioned MINRES (setup included). Returns (x, SolveInfo)."""
        o = options(**opts)
        x = np.zeros(self.n, np.complex128) if x0 is None else _c128(x0).copy()
        info = Info()
        rc = self._lib.glref_jacobian_solve(self.ptr, _c128(psi), _c128(b), x, C.byref(o), C.byref(info))
        return x, SolveInfo(rc, info.iters, bool(info.converged), info.true_relres, info.est_relres)

    def newton_step(self, psi, **opts):
        """One Newton step in place on a copy; returns (psi_new, ||GL(psi)||_R, SolveInfo)."""
        o = options(**opts)
        p = _c128(psi).copy()
        info = Info()
        gn = C.c_double()
        rc = self._lib.glref_newton_step(self.ptr, p, C.byref(o), C.byref(info), C.byref(gn))
        return p, gn.value, SolveInfo(rc, info.iters, bool(info.converged), info.true_relres, info.est_relres)


class Precond:
    """R_k(psi) = AMG_k(K-hat + 2 D |psi|^2, D .) (Eq. prec2)."""

    def __init__(self, mesh: Mesh, psi, **opts):
        self._lib = lib()
        self.mesh = mesh
        self.psi = _c128(psi).copy()
        self.opts = options(**opts)
        self.ptr = self._lib.glref_precond_setup(mesh.ptr, self.psi, C.byref(self.opts))
        if not self.ptr:
            raise RuntimeError("glref_precond_setup failed (coarsest operator not HPD?)")
        self.nlevels = self._lib.glref_prec_nlevels(self.ptr)

    def __del__(self):
        p = getattr(self, "ptr", None)
        if p:
            self._lib.glref_precond_destroy(p)
            self.ptr = None

    def level_info(self, l: int):
        n, nnz, pnnz = C.c_int64(), C.c_int64(), C.c_int64()
        nc = C.c_int32()
        om = C.c_double()
        self._lib.glref_prec_level_info(self.ptr, l, C.byref(n), C.byref(nnz), C.byref(nc), C.byref(pnnz), C.byref(om))
        return dict(n=n.value, nnz=nnz.value, ncolors=nc.value, p_nnz=pnnz.value, omega=om.value)

    def level_matrix(self, l: int):
        info = self.level_info(l)
        rp = np.zeros(info["n"] + 1, np.int64)
        ci = np.zeros(info["nnz"], np.int32)
        v = np.zeros(info["nnz"], np.complex128)
        self._lib.glref_prec_level_matrix(self.ptr, l, rp, ci, v)
        return rp, ci, v

    def level_P(self, l: int):
        info = self.level_info(l)
        rp = np.zeros(info["n"] + 1, np.int64)
        ci = np.zeros(info["p_nnz"], np.int32)
        v = np.zeros(info["p_nnz"], np.complex128)
        self._lib.glref_prec_level_P(self.ptr, l, rp, ci, v)
        return rp, ci, v

    def aggregates(self, l: int):
        a = np.zeros(self.level_info(l)["n"], np.int32)
        self._lib.glref_prec_level_aggregates(self.ptr, l, a)
        return a

    def colors(self, l: int):
        c = np.zeros(self.level_info(l)["n"], np.int32)
        self._lib.glref_prec_level_colors(self.ptr, l, c)
        return c

    def apply(self, v):
        z = np.zeros(self.mesh.n, np.complex128)
        self._lib.glref_precond_apply(self.ptr, _c128(v), z)
        return z

    def apply_count(self, v):
        """(R v, number of V-cycles applied); with cycles=CYCLES_INF, R_inf."""
        z = np.zeros(self.mesh.n, np.complex128)
        k = self._lib.glref_precond_apply_count(self.ptr, _c128(v), z)
        return z, k

    def vcycle(self, l: int, b):
        x = np.zeros(self.level_info(l)["n"], np.complex128)
        self._lib.glref_vcycle(self.ptr, l, _c128(b), x)
        return x

    def vcycle_cost(self) -> tuple[float, float]:
        """(entries visited by one V-cycle, entries of the finest operator K-hat).

        Per level above the coarsest: the pre-smoothing symmetric Gauss-Seidel
        step from x = 0 (the first colour reads only its diagonals), the
        post-smoothing step (every colour), where a colour visit reads its rows'
        off-diagonals and diagonals and the backward pass starts one colour before
        the last; the residual (every entry); restriction and prolongation
        (nnz(P) each).  The coarsest level: n_c^2 entries of the dense inverse.
        This counts the GPU's sweep order (the backward pass skips the repeated
        last colour); the oracle's own sweeps repeat it."""
        E = 0.0
        L = self.nlevels
        for lvl in range(L - 1):
            info = self.level_info(lvl)
            rp, _, _ = self.level_matrix(lvl)
            col = self.colors(lvl)
            rowlen = np.diff(rp)  # off-diagonals + diagonal
            nc = info["ncolors"]
            visit = np.array([rowlen[col == c].sum() for c in range(nc)], dtype=float)
            rows0 = float(np.sum(col == 0))
            allv = visit.sum()
            back = allv - visit[nc - 1]
            E += (allv - visit[0] + rows0) + back
            E += allv + back
            E += allv
            E += 2.0 * info["p_nnz"]
        nc_rows = self.level_info(L - 1)["n"]
        E += float(nc_rows) ** 2
        return E, float(self.mesh.nnz)

    def cost(self, k: int) -> float:
        """R_k in matrix-vector-product equivalents (Fig. 1): k V-cycles and k - 1
        finest residuals, over the entries of K-hat."""
        E, fine = self.vcycle_cost()
        return (k * E + (k - 1) * fine) / fine

    def cost_inf(self, k: int) -> float:
        """One R_inf apply that took k cycles, in matvec equivalents: k V-cycles
        and the k residuals that decide whether to stop."""
        E, fine = self.vcycle_cost()
        return k * (E + fine) / fine

    def minres(self, b, x0=None):
        x = np.zeros(self.mesh.n, np.complex128) if x0 is None else _c128(x0).copy()
        info = Info()
        rc = self._lib.glref_minres(self.mesh.ptr, self.psi, self.ptr, _c128(b), x, C.byref(self.opts), C.byref(info))
        return x, SolveInfo(rc, info.iters, bool(info.converged), info.true_relres, info.est_relres)


def aggregate(rp, ci):
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    agg = np.zeros(n, np.int32)
    nagg = lib().glref_aggregate(n, rp, ci, agg)
    return nagg, agg


def color_jp(rp, ci):
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    col = np.zeros(n, np.int32)
    nc = lib().glref_color_jp(n, rp, ci, col)
    return nc, col


def color_psl(rp, ci):
    """(ncolors, colours, levels): smallest-last colouring in removal rounds."""
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    col = np.zeros(n, np.int32)
    level = np.zeros(n, np.int32)
    nc = lib().glref_color_psl(n, rp, ci, col, level)
    return nc, col, level


def color_sl(rp, ci):
    """(ncolors, colours, order): smallest-last greedy colouring and its colouring order."""
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    col = np.zeros(n, np.int32)
    order = np.zeros(n, np.int32)
    nc = lib().glref_color_sl(n, rp, ci, col, order)
    return nc, col, order


def simplex_alpha(dim: int, verts, method: str = "linsys"):
    p = np.zeros(12)
    v = np.asarray(verts, dtype=np.float64)
    p[: 3 * (dim + 1)].reshape(dim + 1, 3)[:, : v.shape[1]] = v
    ne = dim * (dim + 1) // 2
    a = np.zeros(6)
    if method == "cot":
        assert dim == 2
        rc = lib().glref_simplex_alpha_cot(p, a)
    elif method == "dihedral":
        assert dim == 3
        rc = lib().glref_simplex_alpha_dihedral(p, a)
    else:
        rc = lib().glref_simplex_alpha_linsys(dim, p, a)
    if rc:
        raise ValueError("degenerate simplex")
    return a[:ne]


def hash32(i: int) -> int:
    return lib().glref_hash32(i)
