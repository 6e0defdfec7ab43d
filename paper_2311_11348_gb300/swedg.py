"""Thin ctypes binding of libswedg (include/swedg.h): argument marshalling only.

Every call lands in the CUDA library; there is no Python or CPU fallback.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they must be
C-contiguous float64 (int32/int8 for the mesh arrays).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KMAX = 15
PREC_FP64 = 0
PREC_MIXED_FP32 = 1
PREC_MIXED_TF32 = 2
STATUS_DEPTH = 1
STATUS_NONFINITE = 2

_ERRORS = {-1: "invalid argument", -2: "bad mesh", -3: "depth <= h_min", -4: "non-finite state",
           -5: "CUDA error", -6: "device wait timeout"}


class SweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libswedg error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("h_min", C.c_double), ("rk_order", C.c_int),
                ("precision", C.c_int), ("tide_amp", C.c_double), ("tide_period", C.c_double),
                ("tide_phase", C.c_double), ("cuda_stream", C.c_void_p), ("fric_lin", C.c_double),
                ("fric_quad", C.c_double), ("f_c", C.c_double)]


_lib = None

# every symbol include/swedg.h declares
SYMBOLS = ("swe_default_params", "swe_create", "swe_destroy", "swe_last_error", "swe_set_mesh",
           "swe_set_bathymetry", "swe_set_orders", "swe_set_state", "swe_get_state", "swe_p1_modes", "swe_rhs",
           "swe_rhs_parts", "swe_rk_step", "swe_run", "swe_mass", "swe_energy", "swe_reference_tensors",
           "swe_edge_table", "swe_profile", "swe_profile_read", "swe_rhs_p1_noalloc", "swe_adapt",
           "swe_run_adaptive", "swe_set_members", "swe_set_member_times", "swe_get_member_times",
           "swe_memory_bytes", "swe_tc_operand_image", "swe_get_launch_shape", "swe_set_launch_shape",
           "swe_autotune", "swe_selftest_wait", "swe_packed_size", "swe_set_state_packed",
           "swe_get_state_packed", "swe_set_state_packed_async", "swe_run_async", "swe_get_state_packed_async",
           "swe_sync", "swe_member_status", "swe_mesh_adjacency")


def library_path() -> str:
    return _build.LIB


def load():
    """Load the in-tree libswedg.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libswedg is not built ({path}); run `python -m paper_2311_11348_gb300.build`")
    lib = C.CDLL(path)
    P = C.c_void_p
    i64 = C.c_int64
    d = C.c_double
    lib.swe_default_params.argtypes = [C.POINTER(Params)]
    lib.swe_create.argtypes = [C.POINTER(P), C.POINTER(Params)]
    lib.swe_destroy.argtypes = [P]
    lib.swe_last_error.argtypes = [P]
    lib.swe_last_error.restype = C.c_char_p
    lib.swe_set_mesh.argtypes = [P, i64, P, i64, P, P]
    lib.swe_mesh_adjacency.argtypes = [i64, P, i64, P, P, P]
    lib.swe_set_bathymetry.argtypes = [P, P]
    lib.swe_set_orders.argtypes = [P, P]
    lib.swe_set_state.argtypes = [P, P, d]
    lib.swe_get_state.argtypes = [P, P, C.POINTER(d)]
    lib.swe_packed_size.argtypes = [P]
    lib.swe_set_state_packed.argtypes = [P, P, d]
    lib.swe_get_state_packed.argtypes = [P, P, C.POINTER(d)]
    lib.swe_set_state_packed_async.argtypes = [P, P, d]
    lib.swe_run_async.argtypes = [P, i64, d]
    lib.swe_get_state_packed_async.argtypes = [P, P]
    lib.swe_sync.argtypes = [P]
    lib.swe_p1_modes.argtypes = [P, P, P]
    lib.swe_rhs.argtypes = [P, P, P]
    lib.swe_rhs_parts.argtypes = [P, P, P, P]
    lib.swe_rk_step.argtypes = [P, d, C.POINTER(d)]
    lib.swe_run.argtypes = [P, i64, d, C.POINTER(d)]
    lib.swe_mass.argtypes = [P, C.POINTER(d)]
    lib.swe_energy.argtypes = [P, C.POINTER(d)]
    lib.swe_reference_tensors.argtypes = [P, P, P]
    lib.swe_edge_table.argtypes = [C.c_int, P, P, P]
    lib.swe_profile.argtypes = [P, C.c_int]
    lib.swe_profile_read.argtypes = [P, C.c_int, C.POINTER(C.c_char_p), C.POINTER(d), C.POINTER(i64)]
    lib.swe_rhs_p1_noalloc.argtypes = [i64, P, P, i64, P, P, P, d, P, P]
    lib.swe_adapt.argtypes = [P, d, d, C.c_int, C.c_int, C.POINTER(i64), P]
    lib.swe_run_adaptive.argtypes = [P, i64, i64, d, d, d, C.c_int, C.c_int, C.POINTER(d)]
    lib.swe_set_members.argtypes = [P, C.c_int32, P]
    lib.swe_set_member_times.argtypes = [P, P]
    lib.swe_get_member_times.argtypes = [P, P, P]
    lib.swe_memory_bytes.argtypes = [P, C.POINTER(i64)]
    lib.swe_member_status.argtypes = [P, P]
    for s in SYMBOLS:
        if s not in ("swe_destroy", "swe_default_params", "swe_last_error"):
            getattr(lib, s).restype = C.c_int
    lib.swe_tc_operand_image.restype = C.c_int64
    lib.swe_packed_size.restype = C.c_int64
    _lib = lib
    return lib


def _ptr(a, dtype=np.float64):
    """(pointer, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), arr


def reference_tensors():
    lib = load()
    D = np.zeros((2, KMAX, KMAX)); G = np.zeros((2, KMAX, KMAX, KMAX)); T = np.zeros((KMAX,) * 3)
    lib.swe_reference_tensors(D.ctypes.data_as(C.c_void_p), G.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p))
    return D, G, T


def tc_operand_image(K: int):
    """the shared-memory image of the tensor-core B operands for K modes (host only)"""
    lib = load()
    n = lib.swe_tc_operand_image(int(K), None, C.c_int64(0))
    if n < 0:
        raise SweError(int(n), "swe_tc_operand_image")
    out = np.zeros(n, np.float32)
    lib.swe_tc_operand_image(int(K), out.ctypes.data_as(C.c_void_p), C.c_int64(n))
    return out


def mesh_adjacency(xy, tri):
    """(nbr [ne,3] int32, nbk [ne,3] int8) of the library's adjacency build
    (host only, no device): the triangle across the edge opposite vertex k and
    its local index of that edge, -1 on the boundary"""
    lib = load()
    pxy, kx = _ptr(xy)
    pt, kt = _ptr(tri, np.int32)
    ne = int(np.shape(tri)[0])
    nbr = np.zeros((ne, 3), np.int32)
    nbk = np.zeros((ne, 3), np.int8)
    rc = lib.swe_mesh_adjacency(int(np.shape(xy)[0]), pxy, ne, pt, nbr.ctypes.data_as(C.c_void_p),
                                nbk.ctypes.data_as(C.c_void_p))
    if rc:
        raise SweError(rc, lib.swe_last_error(None).decode())
    return nbr, nbk


def edge_table(npts: int):
    lib = load()
    s = np.zeros(npts); w = np.zeros(npts); B = np.zeros((3, KMAX, npts))
    rc = lib.swe_edge_table(npts, s.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p), B.ctypes.data_as(C.c_void_p))
    if rc:
        raise SweError(rc, "swe_edge_table")
    return s, w, B


NOALLOC_MAX_ELEMENTS = 65536


def _check_device_tensor(name, a, dtype, shape):
    """a must be a contiguous CUDA tensor of the current device with this dtype
    and shape (the entry point reads and writes exactly these extents)"""
    import torch
    if not isinstance(a, torch.Tensor):
        raise ValueError(f"{name}: a torch CUDA tensor is required, got {type(a).__name__}")
    if a.dtype != dtype:
        raise ValueError(f"{name}: dtype {a.dtype}, expected {dtype}")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {tuple(shape)}")
    if not a.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if not a.is_cuda:
        raise ValueError(f"{name}: must be on a CUDA device, not {a.device}")
    if a.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {a.device}, but the current device is cuda:{torch.cuda.current_device()}")


def rhs_p1_noalloc(xy, hv, tri, nbr, c, g, out, stream=None):
    """swe_rhs_p1_noalloc on caller-owned device tensors (see include/swedg.h):
    xy [nv,2] float64, hv [nv] float64, tri [ne,3] int32, nbr [ne,3] int32,
    c [3,3,ne] float64, out [3,3,ne] float64, all contiguous on the current
    CUDA device; anything else raises ValueError before the call."""
    import torch
    if not hasattr(xy, "shape") or len(xy.shape) != 2 or not hasattr(tri, "shape") or len(tri.shape) != 2:
        raise ValueError("xy must be [nv, 2] and tri [ne, 3]")
    nv, ne = int(xy.shape[0]), int(tri.shape[0])
    for name, a, dt, sh in (("xy", xy, torch.float64, (nv, 2)), ("hv", hv, torch.float64, (nv,)),
                            ("tri", tri, torch.int32, (ne, 3)), ("nbr", nbr, torch.int32, (ne, 3)),
                            ("c", c, torch.float64, (3, 3, ne)), ("out", out, torch.float64, (3, 3, ne))):
        _check_device_tensor(name, a, dt, sh)
    lib = load()
    args = [_ptr(a) for a in (xy, hv, tri, nbr, c, out)]
    rc = lib.swe_rhs_p1_noalloc(nv, args[0][0], args[1][0], ne, args[2][0], args[3][0], args[4][0], float(g),
                                args[5][0], stream)
    if rc:
        raise SweError(rc, "swe_rhs_p1_noalloc")
    return out


class Solver:
    """One libswedg context (one mesh, one device state)."""

    def __init__(self, g=9.81, cfl=0.1, h_min=1e-8, rk_order=2, precision=PREC_FP64, tide=(0.0, 0.0, 0.0),
                 friction=(0.0, 0.0), f_c=0.0,
                 stream=None):
        self._lib = load()
        p = Params()
        self._lib.swe_default_params(C.byref(p))
        p.g, p.cfl, p.h_min, p.rk_order, p.precision = g, cfl, h_min, rk_order, precision
        p.tide_amp, p.tide_period, p.tide_phase = tide
        p.fric_lin, p.fric_quad = friction
        p.f_c = f_c
        p.cuda_stream = stream
        h = C.c_void_p()
        rc = self._lib.swe_create(C.byref(h), C.byref(p))
        if rc:
            raise SweError(rc, self._lib.swe_last_error(None).decode())
        self.h = h
        self.ne = 0
        self.nv = 0

    def close(self):
        if getattr(self, "h", None):
            self._lib.swe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc:
            raise SweError(rc, self._lib.swe_last_error(self.h).decode())

    def set_mesh(self, xy, tri, bc_tag=None):
        pxy, kx = _ptr(xy)
        pt, kt = _ptr(tri, np.int32)
        pb, kb = _ptr(bc_tag, np.int8)
        nv, ne = int(xy.shape[0]), int(tri.shape[0])
        self._ck(self._lib.swe_set_mesh(self.h, nv, pxy, ne, pt, pb))
        self.nv, self.ne = nv, ne

    def set_bathymetry(self, hv):
        p, k = _ptr(hv)
        self._ck(self._lib.swe_set_bathymetry(self.h, p))

    def set_orders(self, orders):
        p, k = _ptr(orders, np.int8)
        self._ck(self._lib.swe_set_orders(self.h, p))

    def set_state(self, c, t=0.0):
        p, k = _ptr(c)
        self._ck(self._lib.swe_set_state(self.h, p, float(t)))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((3, KMAX, self.ne))
        p, k = _ptr(out)
        t = C.c_double(0.0)
        self._ck(self._lib.swe_get_state(self.h, p, C.byref(t)))
        return out, t.value

    def packed_size(self):
        """doubles in the packed state layout (sum over elements of 3 K(p))"""
        n = self._lib.swe_packed_size(self.h)
        if n < 0:
            self._ck(int(n))
        return int(n)

    def set_state_packed(self, c, t=0.0):
        """state in the packed layout: element by element, 3 K(p) values (xi, U, V modes)"""
        n = c.numel() if hasattr(c, "numel") else np.size(c)
        if n != self.packed_size():
            raise ValueError(f"packed state has {n} values, the orders need {self.packed_size()}")
        p, k = _ptr(c)
        self._ck(self._lib.swe_set_state_packed(self.h, p, float(t)))

    def get_state_packed(self, out=None):
        if out is None:
            out = np.zeros(self.packed_size())
        n = out.numel() if hasattr(out, "numel") else np.size(out)
        if n != self.packed_size():
            raise ValueError(f"packed state buffer has {n} values, the orders need {self.packed_size()}")
        p, k = _ptr(out)
        t = C.c_double(0.0)
        self._ck(self._lib.swe_get_state_packed(self.h, p, C.byref(t)))
        return out, t.value

    # asynchronous variants: enqueue and return; sync() waits and reports errors.
    # The caller keeps the buffers alive and untouched until sync() returns.
    def set_state_packed_async(self, c, t=0.0):
        n = c.numel() if hasattr(c, "numel") else np.size(c)
        if n != self.packed_size():
            raise ValueError(f"packed state has {n} values, the orders need {self.packed_size()}")
        if not hasattr(c, "data_ptr"):
            raise ValueError("asynchronous calls take torch tensors (pinned host or CUDA), which the caller keeps alive")
        p, _ = _ptr(c)
        self._ck(self._lib.swe_set_state_packed_async(self.h, p, float(t)))

    def run_async(self, nsteps, dt_fixed=0.0):
        self._ck(self._lib.swe_run_async(self.h, int(nsteps), float(dt_fixed)))

    def get_state_packed_async(self, out):
        n = out.numel() if hasattr(out, "numel") else np.size(out)
        if n != self.packed_size():
            raise ValueError(f"packed state buffer has {n} values, the orders need {self.packed_size()}")
        if not hasattr(out, "data_ptr"):
            raise ValueError("asynchronous calls take torch tensors (pinned host or CUDA), which the caller keeps alive")
        p, _ = _ptr(out)
        self._ck(self._lib.swe_get_state_packed_async(self.h, p))

    def sync(self):
        self._ck(self._lib.swe_sync(self.h))

    def p1_modes(self, vals, out=None):
        if out is None:
            out = np.zeros((3, self.ne))
        pv, kv = _ptr(vals)
        po, ko = _ptr(out)
        self._ck(self._lib.swe_p1_modes(self.h, pv, po))
        return out

    def rhs(self, c, out=None):
        if out is None:
            out = np.zeros((3, KMAX, self.ne))
        pc, kc = _ptr(c)
        po, ko = _ptr(out)
        self._ck(self._lib.swe_rhs(self.h, pc, po))
        return out

    def rhs_parts(self, c):
        b = np.zeros((3, KMAX, self.ne)); r = np.zeros((3, KMAX, self.ne))
        pc, kc = _ptr(c)
        self._ck(self._lib.swe_rhs_parts(self.h, pc, _ptr(b)[0], _ptr(r)[0]))
        return b, r

    def rk_step(self, dt=0.0):
        du = C.c_double(0.0)
        self._ck(self._lib.swe_rk_step(self.h, float(dt), C.byref(du)))
        return du.value

    def run(self, nsteps, dt_fixed=0.0):
        t = C.c_double(0.0)
        self._ck(self._lib.swe_run(self.h, int(nsteps), float(dt_fixed), C.byref(t)))
        return t.value

    def adapt(self, theta_up, theta_down, p_min=1, p_max=4):
        """one indicator pass; returns (new orders, number changed)"""
        n = C.c_int64(0)
        out = np.zeros(self.ne, np.int8)
        self._ck(self._lib.swe_adapt(self.h, float(theta_up), float(theta_down), int(p_min), int(p_max), C.byref(n),
                                     out.ctypes.data_as(C.c_void_p)))
        return out, n.value

    def run_adaptive(self, nsteps, every, theta_up, theta_down, p_min=1, p_max=4, dt_fixed=0.0):
        t = C.c_double(0.0)
        self._ck(self._lib.swe_run_adaptive(self.h, int(nsteps), int(every), float(dt_fixed), float(theta_up),
                                            float(theta_down), int(p_min), int(p_max), C.byref(t)))
        return t.value

    def set_members(self, nmembers, member=None):
        pm, km = _ptr(member, np.int32)
        self._ck(self._lib.swe_set_members(self.h, int(nmembers), pm))
        self.nmembers = int(nmembers)

    def member_times(self):
        n = getattr(self, "nmembers", 1)
        t = np.zeros(n); dt = np.zeros(n)
        self._ck(self._lib.swe_get_member_times(self.h, t.ctypes.data_as(C.c_void_p), dt.ctypes.data_as(C.c_void_p)))
        return t, dt

    def set_member_times(self, t):
        t = np.ascontiguousarray(t, dtype=np.float64)
        self._ck(self._lib.swe_set_member_times(self.h, t.ctypes.data_as(C.c_void_p)))

    def launch_shape(self):
        """(base blocks per SM, base threads, u-solve threads, correction threads, schedule, base tiles)"""
        v = np.zeros(6, np.int32)
        self._ck(self._lib.swe_get_launch_shape(self.h, v.ctypes.data_as(C.c_void_p)))
        return tuple(int(x) for x in v)

    def set_launch_shape(self, shape):
        v = np.ascontiguousarray(shape, dtype=np.int32)
        if v.shape != (6,):
            raise ValueError("a launch shape has 6 entries")
        self._ck(self._lib.swe_set_launch_shape(self.h, v.ctypes.data_as(C.c_void_p)))

    def autotune(self, steps=5):
        """choose the launch shape by timing trial steps; returns (shape, ms per step)"""
        v = np.zeros(6, np.int32)
        ms = C.c_double(0.0)
        self._ck(self._lib.swe_autotune(self.h, int(steps), v.ctypes.data_as(C.c_void_p), C.byref(ms)))
        return tuple(int(x) for x in v), ms.value

    def selftest_wait(self, spins=1000):
        """run the bounded-wait self-test (raises SweError SWE_ETIMEOUT by design)"""
        self._ck(self._lib.swe_selftest_wait(self.h, C.c_int64(int(spins))))

    def member_status(self):
        """per ensemble member: STATUS_DEPTH | STATUS_NONFINITE bits set since the last call (cleared)"""
        n = getattr(self, "nmembers", 1)
        out = np.zeros(n, np.uint32)
        self._ck(self._lib.swe_member_status(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def memory_bytes(self):
        b = C.c_int64(0)
        self._ck(self._lib.swe_memory_bytes(self.h, C.byref(b)))
        return b.value

    def mass(self):
        m = C.c_double(0.0)
        self._ck(self._lib.swe_mass(self.h, C.byref(m)))
        return m.value

    def energy(self):
        e = C.c_double(0.0)
        self._ck(self._lib.swe_energy(self.h, C.byref(e)))
        return e.value

    def profile(self, enable=True):
        self._ck(self._lib.swe_profile(self.h, int(enable)))

    def profile_read(self):
        n = 16
        names = (C.c_char_p * n)()
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        k = self._lib.swe_profile_read(self.h, n, names, ms, cnt)
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k)}
