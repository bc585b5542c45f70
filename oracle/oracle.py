"""ctypes wrapper of the plain FP64 CPU oracle (``swdg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never does.  The
oracle shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "swdg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_c_int, _c_double, _c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE, no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class OraConfig(ctypes.Structure):
    _fields_ = [("degree", _c_int), ("subgrid_mode", _c_int), ("tableau", _c_int),
                ("g", _c_double), ("eps_vel", _c_double), ("h_lim", _c_double),
                ("eps0", _c_double), ("cfl", _c_double), ("newton_max", _c_int),
                ("newton_tol", _c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.ora_create.restype = _P
        L.ora_create.argtypes = [ctypes.POINTER(OraConfig), _c_i64, _P, _P, _P, _P, _c_i64, _c_i64,
                                 _c_double, _c_double, _c_double, _c_double]
        L.ora_destroy.argtypes = [_P]
        L.ora_error.restype = ctypes.c_char_p
        L.ora_set_boundary.argtypes = [_P, _c_int, _c_int, _c_double, _c_double, _c_double]
        L.ora_set_manning.argtypes = [_P, _P]
        L.ora_set_state.argtypes = [_P, _P, _P, _P, _P]
        L.ora_get_state.argtypes = [_P, _P, _P, _P, _P]
        L.ora_get_flags.argtypes = [_P, _P]
        L.ora_residual.argtypes = [_P, _c_double, _c_i64, _P, _P, _P, _P, _P, _P, _P]
        L.ora_cfl_dt.argtypes = [_P, _c_double, _P]
        L.ora_degree_switch.argtypes = [_P]
        L.ora_step.argtypes = [_P, _c_int, _c_double, _P]
        L.ora_diagnostics.argtypes = [_P, _P]
        L.ora_gauges.argtypes = [_P, _c_int, _P, _P]
        L.ora_lake_at_rest.argtypes = [_P, _c_double, _P]
        L.ora_cell_mass.argtypes = [_P, _P]
        L.ora_rule.argtypes = [_c_int, _c_int, _P, _P]
        L.ora_subgrid_rect.argtypes = [_P, _c_double, _c_double, _c_double, _c_double, _c_double,
                                       _P, _P]
        L.ora_subgrid_point.argtypes = [_P, _c_i64, _c_int, _c_int, _c_double, _P, _P]
        L.ora_zb_point.restype = _c_double
        L.ora_zb_point.argtypes = [_P, _c_double, _c_double]
        L.ora_face_flux_p.argtypes = [_P, _P, _P]
        L.ora_tableau.argtypes = [_c_int, _P, _P, _P, _P, _P, _P]
        L.ora_set_tracer_diffusivity.argtypes = [_P, _P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def rule(kind: int, n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().ora_rule(kind, n, _ptr(x), _ptr(w)):
        raise ValueError(lib().ora_error().decode())
    return x, w


def tableau(t: int):
    s = ctypes.c_int(0)
    a, at = np.zeros(16), np.zeros(16)
    b, bt, c = np.zeros(4), np.zeros(4), np.zeros(4)
    lib().ora_tableau(t, ctypes.byref(s), _ptr(a), _ptr(at), _ptr(b), _ptr(bt), _ptr(c))
    n = s.value
    return dict(s=n, a=a.reshape(4, 4)[:n, :n], at=at.reshape(4, 4)[:n, :n], b=b[:n], bt=bt[:n],
                c=c[:n])


class Oracle:
    """One oracle instance over a mesh and raster (copied)."""

    def __init__(self, mesh, raster, degree=1, subgrid_mode=0, tableau=0, g=9.81, eps_vel=0.01,
                 h_lim=0.01, eps0=1e-6, cfl=0.1, newton_max=20, newton_tol=1e-12):
        L = lib()
        self.cfg = OraConfig(degree, subgrid_mode, tableau, g, eps_vel, h_lim, eps0, cfl,
                             newton_max, newton_tol)
        self.n = int(mesh.n)
        self.nd = (degree + 1) ** 2
        x0y0 = np.ascontiguousarray(mesh.x0y0, dtype=np.float64)
        hxhy = np.ascontiguousarray(mesh.hxhy, dtype=np.float64)
        nbr = np.ascontiguousarray(mesh.nbr, dtype=np.int32)
        z = np.ascontiguousarray(raster.z, dtype=np.float64)
        ny, nx = z.shape
        h = L.ora_create(ctypes.byref(self.cfg), self.n, _ptr(x0y0), _ptr(hxhy), _ptr(nbr), _ptr(z),
                         nx, ny, raster.xo, raster.yo, raster.dx, raster.dy)
        if not h:
            raise ValueError(L.ora_error().decode())
        self.h = ctypes.c_void_p(h)

    @classmethod
    def from_workload(cls, wl, **over):
        o = cls(wl.mesh, wl.raster, **wl.config(**over))
        for (tag, kind, amp, per, ph) in wl.boundaries:
            o.set_boundary(tag, kind, amp, per, ph)
        if wl.manning is not None:
            o.set_manning(wl.manning)
        if getattr(wl, "tracer_diffusivity", None) is not None:
            o.set_tracer_diffusivity(wl.tracer_diffusivity)
        o.set_state(*wl.state())
        return o

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.ora_destroy(self.h)
            self.h = None

    def set_boundary(self, tag, kind, amp=0.0, period=1.0, phase=0.0):
        if lib().ora_set_boundary(self.h, tag, kind, amp, period, phase):
            raise ValueError(lib().ora_error().decode())

    def set_tracer_diffusivity(self, nu):
        if nu is None:
            lib().ora_set_tracer_diffusivity(self.h, None)
            return
        a = np.ascontiguousarray(nu, dtype=np.float64)
        lib().ora_set_tracer_diffusivity(self.h, _ptr(a))

    def set_manning(self, n):
        a = np.ascontiguousarray(n, dtype=np.float64)
        lib().ora_set_manning(self.h, _ptr(a))

    def set_state(self, zeta, qx, qy, c):
        arr = [np.ascontiguousarray(v, dtype=np.float64).reshape(self.n, self.nd)
               for v in (zeta, qx, qy, c)]
        lib().ora_set_state(self.h, *[_ptr(a) for a in arr])

    def get_state(self):
        out = [np.zeros((self.n, self.nd)) for _ in range(4)]
        lib().ora_get_state(self.h, *[_ptr(a) for a in out])
        return out

    def flags(self):
        f = np.zeros(self.n, dtype=np.uint8)
        lib().ora_get_flags(self.h, _ptr(f))
        return f

    def residual(self, t=0.0, cells=None):
        if cells is None:
            m = self.n
            cp = None
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            m = len(cells)
            cp = _ptr(cells)
        out = [np.zeros((m, self.nd)) for _ in range(6)]
        lib().ora_residual(self.h, t, m, cp, *[_ptr(a) for a in out])
        return dict(zip(("F", "Gx", "Gy", "R", "Lx", "Ly"), out))

    def cfl_dt(self, t=0.0):
        d = ctypes.c_double(0.0)
        lib().ora_cfl_dt(self.h, t, ctypes.byref(d))
        return d.value

    def degree_switch(self):
        lib().ora_degree_switch(self.h)

    def step(self, n=1, dt=-1.0, t=None):
        tt = ctypes.c_double(0.0 if t is None else t)
        lib().ora_step(self.h, n, dt, ctypes.byref(tt) if t is not None else None)
        return tt.value if t is not None else self.diagnostics()["t"]

    def diagnostics(self):
        d = np.zeros(8)
        lib().ora_diagnostics(self.h, _ptr(d))
        keys = ("mass", "tracer_mass", "min_h", "r_cells", "newton_max", "positivity_violations",
                "dt", "t")
        return dict(zip(keys, d.tolist()))

    def gauges(self, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        out = np.zeros(len(xy))
        lib().ora_gauges(self.h, len(xy), _ptr(xy), _ptr(out))
        return out

    def lake_at_rest(self, zeta0=0.0):
        out = np.zeros((self.n, self.nd))
        lib().ora_lake_at_rest(self.h, zeta0, _ptr(out))
        return out

    def cell_mass(self):
        out = np.zeros(self.n)
        lib().ora_cell_mass(self.h, _ptr(out))
        return out

    def subgrid_rect(self, X0, X1, Y0, Y1, eta):
        V, A = ctypes.c_double(), ctypes.c_double()
        lib().ora_subgrid_rect(self.h, X0, X1, Y0, Y1, eta, ctypes.byref(V), ctypes.byref(A))
        return V.value, A.value

    def subgrid_point(self, K, pset, p, eta):
        V, A = ctypes.c_double(), ctypes.c_double()
        if lib().ora_subgrid_point(self.h, K, pset, p, eta, ctypes.byref(V), ctypes.byref(A)):
            raise ValueError(lib().ora_error().decode())
        return V.value, A.value

    def zb_point(self, x, y):
        return lib().ora_zb_point(self.h, x, y)

    def face_flux_p(self, zm, qxm, qym, cm, zbm, zp, qxp, qyp, cp, zbp, nx, ny):
        inp = np.array([zm, qxm, qym, cm, zbm, zp, qxp, qyp, cp, zbp, nx, ny], dtype=np.float64)
        out = np.zeros(7)
        lib().ora_face_flux_p(self.h, _ptr(inp), _ptr(out))
        return dict(zip(("F", "Gx", "Gy", "R", "lam", "hsm", "hsp"), out.tolist()))
