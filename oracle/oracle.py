"""ctypes front end of the FP64 CPU oracle (``swe_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py``.  Nothing in the
product package imports this module, and this module imports nothing from the
product package.

The oracle follows Sect. 2 (Eqs. 1-12, the Lax-Friedrichs flux and Eq. 10) and
Sect. 3 (Eq. 13, the base/correction split and the truncated system uH = q) of
Faghih-Naini et al. (2023) step by step in plain FP64 C; see the header of
``swe_oracle.c`` for the passage each part follows and for the readings taken
where the paper is silent.

State layout everywhere: ``c[3][15][ne]`` (field xi, U, V; modal index; element),
rows at or above K(p_e) are zero.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

KMAX = 15
K_OF_P = (1, 3, 6, 10, 15)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")

_lib = None
_lib_omp = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, FMA contraction off so
    that every product is rounded as written).  openmp=True builds the same
    source with -fopenmp into a second library whose element loops run on all
    host cores (bitwise the same results; see the header of swe_oracle.c)."""
    out = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class _Params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("h_min", C.c_double), ("rk_order", C.c_int),
                ("tide_amp", C.c_double), ("tide_period", C.c_double), ("tide_phase", C.c_double),
                ("fric_lin", C.c_double), ("fric_quad", C.c_double), ("f_c", C.c_double)]


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if openmp and _lib_omp is not None:
        return _lib_omp
    if not openmp and _lib is not None:
        return _lib
    lib = C.CDLL(build(openmp=openmp))
    P = C.c_void_p
    d = C.c_double
    i64 = C.c_int64
    lib.or_mesh_new.restype = P
    lib.or_mesh_new.argtypes = [i64, P, P, i64, P, P, P, C.POINTER(C.c_int)]
    lib.or_mesh_free.argtypes = [P]
    lib.or_set_orders.argtypes = [P, P]
    lib.or_mesh_geometry.argtypes = [P, P, P, P, P]
    lib.or_mesh_neighbours.argtypes = [P, P, P, P, P]
    lib.or_p1_modes.argtypes = [P, P, P]
    lib.or_tri_rule.argtypes = [C.c_int, P, P, P]
    lib.or_proj_points.argtypes = [P, C.c_int, P]
    lib.or_project.argtypes = [P, C.c_int, P, P]
    lib.or_usolve.argtypes = [P, P, P, P]
    lib.or_usolve.restype = C.c_int
    lib.or_rhs.argtypes = [P, P, P, d, P, C.c_int, P]
    lib.or_rhs.restype = C.c_int
    lib.or_dt.argtypes = [P, P, P, P]
    lib.or_dt.restype = d
    lib.or_step.argtypes = [P, P, P, P, d, P]
    lib.or_step.restype = C.c_int
    lib.or_run.argtypes = [P, P, P, P, i64, d]
    lib.or_run.restype = C.c_int
    lib.or_mass.argtypes = [P, P]
    lib.or_mass.restype = d
    lib.or_energy.argtypes = [P, P, P, C.POINTER(C.c_int)]
    lib.or_energy.restype = d
    lib.or_indicator.argtypes = [P, P, d, d, C.c_int, C.c_int, P, P]
    lib.or_indicator.restype = i64
    lib.or_Ktr.argtypes = [C.c_int, C.c_int]
    lib.or_Ktr.restype = C.c_int
    lib.or_poly_grid.restype = C.c_int
    for n in ("D", "G", "T", "S2", "S3", "X2", "X3", "M", "L"):
        getattr(lib, "or_tensor_" + n).argtypes = [P]
    lib.or_basis_monomials.argtypes = [P]
    lib.or_degrees.argtypes = [P]
    lib.or_set_threads.argtypes = [C.c_int]
    lib.or_max_threads.restype = C.c_int
    if openmp:
        _lib_omp = lib
    else:
        _lib = lib
    return lib


def threaded(threads: int = 0):
    """the threaded oracle library with `threads` OpenMP threads (0: every
    host core); returns the number of threads it will use"""
    lib = _load(openmp=True)
    lib.or_set_threads(int(threads) if threads > 0 else (os.cpu_count() or 1))
    return lib.or_max_threads()


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def tensors() -> dict:
    """Reference-element tensors (exact monomial integration).

    D[k,q,i]      = int phi_i d_k phi_q
    G[k,q,i,j]    = int phi_i phi_j d_k phi_q
    T[n,i,j]      = int phi_n phi_i phi_j
    S2[k,q,i]     = int_0^1 phi_q phi_i (gamma_k(s)) ds
    S3[k,q,i,j]   = int_0^1 phi_q phi_i phi_j (gamma_k(s)) ds
    X2[k,k',q,i]  = int_0^1 phi_q(gamma_k(s)) phi_i(gamma_k'(1-s)) ds
    X3[k,k',q,i,j]
    M[i,j]        = int phi_i phi_j
    L[v,i]        = int lambda_v phi_i   (P1 hat functions)
    """
    lib = _load()
    shapes = {"D": (2, KMAX, KMAX), "G": (2, KMAX, KMAX, KMAX), "T": (KMAX,) * 3, "S2": (3, KMAX, KMAX),
              "S3": (3, KMAX, KMAX, KMAX), "X2": (3, 3, KMAX, KMAX), "X3": (3, 3, KMAX, KMAX, KMAX),
              "M": (KMAX, KMAX), "L": (3, KMAX)}
    out = {}
    for n, sh in shapes.items():
        a = np.zeros(sh)
        getattr(lib, "or_tensor_" + n)(_ptr(a))
        out[n] = a
    return out


def basis_monomials() -> np.ndarray:
    """[15, PD, PD] monomial coefficients: phi_i = sum c[i,a,b] x^a y^b."""
    lib = _load()
    pd = lib.or_poly_grid()
    a = np.zeros((KMAX, pd, pd))
    lib.or_basis_monomials(_ptr(a))
    return a


def degrees() -> np.ndarray:
    lib = _load()
    a = np.zeros(KMAX, dtype=np.int32)
    lib.or_degrees(_ptr(a))
    return a


def Ktr(i: int, j: int) -> int:
    return _load().or_Ktr(i, j)


def tri_rule(n: int):
    lib = _load()
    x = np.zeros(n * n); y = np.zeros(n * n); w = np.zeros(n * n)
    lib.or_tri_rule(n, _ptr(x), _ptr(y), _ptr(w))
    return x, y, w


class Params:
    def __init__(self, g=9.81, cfl=0.1, h_min=1e-8, rk_order=2, tide_amp=0.0, tide_period=0.0, tide_phase=0.0,
                 fric_lin=0.0, fric_quad=0.0, f_c=0.0):
        """fric_lin, fric_quad: bottom friction tau_bf = fric_lin H + fric_quad |u| from the
        element means (Sect. 3; the paper's setups use 1e-4 H and 0.009 |u|); f_c: Coriolis."""
        self.s = _Params(g, cfl, h_min, rk_order, tide_amp, tide_period, tide_phase, fric_lin, fric_quad, f_c)

    @property
    def g(self):
        return self.s.g


class Mesh:
    """Oracle mesh: vertices [nv,2], triangles [ne,3], vertex depths, optional
    boundary tags [ne,3] (edge k opposite vertex k; 0 interior/land, 1 land,
    2 open sea) and orders [ne]."""

    def __init__(self, xy, tri, hv, orders=None, bc_tag=None, threads: int = 1):
        """threads > 1 (or 0: every host core) runs the element loops of this
        mesh's calls on the threaded build of the same source"""
        lib = _load(openmp=threads != 1)
        if threads != 1:
            threaded(threads)
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.hv = np.ascontiguousarray(hv, dtype=np.float64)
        self.nv = self.xy.shape[0]
        self.ne = self.tri.shape[0]
        self.orders = np.ascontiguousarray(orders if orders is not None else np.ones(self.ne), dtype=np.int8)
        self.bc_tag = None if bc_tag is None else np.ascontiguousarray(bc_tag, dtype=np.int8)
        err = C.c_int(0)
        h = lib.or_mesh_new(self.nv, _ptr(self.xy), _ptr(self.hv), self.ne, _ptr(self.tri), _ptr(self.bc_tag),
                            _ptr(self.orders), C.byref(err))
        if not h:
            raise ValueError(f"oracle rejected the mesh (status {err.value})")
        self.h = C.c_void_p(h)
        self._lib = lib

    def __del__(self):
        if getattr(self, "h", None) is not None and self._lib is not None:
            self._lib.or_mesh_free(self.h)
            self.h = None

    def set_orders(self, orders):
        self.orders = np.ascontiguousarray(orders, dtype=np.int8)
        self._lib.or_set_orders(self.h, _ptr(self.orders))

    def geometry(self):
        ne = self.ne
        area = np.zeros(ne); s = np.zeros(ne); hb = np.zeros((ne, 3)); dhb = np.zeros((ne, 2))
        self._lib.or_mesh_geometry(self.h, _ptr(area), _ptr(s), _ptr(hb), _ptr(dhb))
        return dict(area=area, s=s, hb=hb, dhb=dhb)

    def neighbours(self):
        ne = self.ne
        nb = np.zeros((ne, 3), np.int64); nbk = np.zeros((ne, 3), np.int8)
        bc = np.zeros((ne, 3), np.int8); tri = np.zeros((ne, 3), np.int32)
        self._lib.or_mesh_neighbours(self.h, _ptr(nb), _ptr(nbk), _ptr(bc), _ptr(tri))
        return dict(nb=nb, nbk=nbk, bc=bc, tri=tri)

    def p1_modes(self, vertex_values) -> np.ndarray:
        v = np.ascontiguousarray(vertex_values, dtype=np.float64)
        out = np.zeros((3, self.ne))
        self._lib.or_p1_modes(self.h, _ptr(v), _ptr(out))
        return out

    def proj_points(self, n: int) -> np.ndarray:
        out = np.zeros((self.ne, n * n, 2))
        self._lib.or_proj_points(self.h, n, _ptr(out))
        return out

    def project(self, n: int, values) -> np.ndarray:
        """L2 projection of point values (from ``proj_points(n)``) -> [15, ne]."""
        v = np.ascontiguousarray(values, dtype=np.float64).reshape(self.ne, n * n)
        out = np.zeros((KMAX, self.ne))
        self._lib.or_project(self.h, n, _ptr(v), _ptr(out))
        return out

    def project_state(self, fn, n: int = 8) -> np.ndarray:
        """fn(x, y) -> (xi, U, V) arrays; returns c[3,15,ne]."""
        pts = self.proj_points(n)
        xi, U, V = fn(pts[..., 0], pts[..., 1])
        c = np.zeros((3, KMAX, self.ne))
        for f, val in enumerate((xi, U, V)):
            c[f] = self.project(n, np.broadcast_to(val, pts.shape[:2]))
        return c

    # ---- the scheme -------------------------------------------------
    def usolve(self, P: Params, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        u = np.zeros((2, KMAX, self.ne))
        st = self._lib.or_usolve(self.h, C.byref(P.s), _ptr(c), _ptr(u))
        return u, st

    def rhs(self, P: Params, c, t: float = 0.0, part: int = 0, with_u: bool = False):
        """part 0: whole scheme, 1: base (all indices <= 3), 2: correction."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        r = np.zeros((3, KMAX, self.ne))
        u = np.zeros((2, KMAX, self.ne))
        st = self._lib.or_rhs(self.h, C.byref(P.s), _ptr(c), float(t), _ptr(r), int(part), _ptr(u))
        if st != 0:
            raise FloatingPointError(f"oracle rhs status {st}")
        return (r, u) if with_u else r

    def dt(self, P: Params, c) -> float:
        c = np.ascontiguousarray(c, dtype=np.float64)
        u, st = self.usolve(P, c)
        return self._lib.or_dt(self.h, C.byref(P.s), _ptr(c), _ptr(u))

    def step(self, P: Params, c, t: float, dt: float = 0.0):
        """One SSP-RK step (dt <= 0: CFL step).  Returns (c_new, t_new, dt_used)."""
        c = np.array(c, dtype=np.float64, order="C", copy=True)
        tt = C.c_double(t); du = C.c_double(0.0)
        st = self._lib.or_step(self.h, C.byref(P.s), _ptr(c), C.byref(tt), float(dt), C.byref(du))
        if st != 0:
            raise FloatingPointError(f"oracle step status {st}")
        return c, tt.value, du.value

    def run(self, P: Params, c, t: float, nsteps: int, dt: float = 0.0):
        c = np.array(c, dtype=np.float64, order="C", copy=True)
        tt = C.c_double(t)
        st = self._lib.or_run(self.h, C.byref(P.s), _ptr(c), C.byref(tt), int(nsteps), float(dt))
        if st != 0:
            raise FloatingPointError(f"oracle run status {st}")
        return c, tt.value

    def indicator(self, c, theta_up, theta_down, p_min, p_max):
        """Modal-decay adaptivity indicator (module docstring of swe_oracle.c):
        returns (new orders [ne] int8, s [ne], number changed)."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        po = np.zeros(self.ne, np.int8)
        so = np.zeros(self.ne)
        n = self._lib.or_indicator(self.h, _ptr(c), float(theta_up), float(theta_down), int(p_min), int(p_max),
                                   _ptr(po), _ptr(so))
        return po, so, int(n)

    def adapt_state(self, c, new_orders):
        """Hierarchical order change: modes beyond K(p_new) dropped, new modes zero."""
        c = np.array(c, dtype=np.float64, copy=True)
        K = np.array(K_OF_P)[np.asarray(new_orders, dtype=np.int64)]
        c[:, np.arange(KMAX)[:, None] >= K[None, :]] = 0.0
        self.set_orders(new_orders)
        return c

    def mass(self, c) -> float:
        c = np.ascontiguousarray(c, dtype=np.float64)
        return self._lib.or_mass(self.h, _ptr(c))

    def energy(self, P: Params, c) -> float:
        c = np.ascontiguousarray(c, dtype=np.float64)
        st = C.c_int(0)
        e = self._lib.or_energy(self.h, C.byref(P.s), _ptr(c), C.byref(st))
        return e
