"""Thin ctypes binding of the C-ABI in ``include/swdg.h``.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libswdg.so``.  NumPy arrays are passed as host buffers, torch
CUDA tensors as device buffers on the current torch stream.  There is no CPU
fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libswdg.so")

SWDG_OK = 0
SWDG_EINVAL = -1
SWDG_ECUDA = -2
SWDG_ENEWTON = -3
SWDG_EPOSITIVITY = -4
SWDG_ENAN = -5
SWDG_ESTATE = -6
SWDG_HOST = 0
SWDG_DEVICE = 1
SWDG_BC_WALL = 0
SWDG_BC_TIDE = 1
SWDG_PIX_F32 = 0
SWDG_PIX_F64 = 1
SWDG_KIND_BEGIN = 0
SWDG_KIND_RESIDUAL = 1
SWDG_KIND_STAGE = 2
SWDG_KIND_AUX = 3

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64


class swdg_config(ctypes.Structure):
    _fields_ = [("degree", _I), ("precision", _I), ("subgrid_mode", _I), ("tableau", _I),
                ("g", _D), ("eps_vel", _D), ("h_lim", _D), ("eps0", _D), ("cfl", _D),
                ("newton_max", _I), ("newton_tol", _D), ("stream", _P)]


class swdg_forest(ctypes.Structure):
    _fields_ = [("nx0", _I), ("ny0", _I), ("x0", _D), ("y0", _D), ("hx0", _D), ("hy0", _D),
                ("max_level", _I), ("h_min", _D), ("tags", _I * 4), ("periodic", _I * 2)]


def make_forest(nx0, ny0, x0, y0, hx0, hy0, max_level, h_min=0.0, tags=(0, 0, 0, 0),
                periodic=(False, False)):
    return swdg_forest(nx0, ny0, x0, y0, hx0, hy0, max_level, h_min, (_I * 4)(*tags),
                       (_I * 2)(*[int(p) for p in periodic]))


class SwdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swdg error {code}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes), mirroring include/swdg.h
SIGNATURES = {
    "swdg_create": (_I, [ctypes.POINTER(swdg_config), ctypes.POINTER(_P)]),
    "swdg_upload_mesh": (_I, [_P, _I64, _P, _P, _P]),
    "swdg_upload_bathymetry": (_I, [_P, _P, _I, _I64, _I64, _D, _D, _D, _D]),
    "swdg_set_boundary": (_I, [_P, _I, _I, _D, _D, _D]),
    "swdg_set_manning": (_I, [_P, _P, _I]),
    "swdg_set_tracer_diffusivity": (_I, [_P, _P, _I]),
    "swdg_set_state": (_I, [_P, _P, _P, _P, _P, _I]),
    "swdg_get_state": (_I, [_P, _P, _P, _P, _P, _I]),
    "swdg_residual": (_I, [_P, _D, _P, _P, _P, _P, _P, _P, _I]),
    "swdg_cfl_dt": (_I, [_P, _D, ctypes.POINTER(_D)]),
    "swdg_step": (_I, [_P, _I, _D, ctypes.POINTER(_D)]),
    "swdg_step_profile": (_I, [_P, _I, _D, ctypes.POINTER(_D), _P]),
    "swdg_degree_switch": (_I, [_P, _P]),
    "swdg_gather_gauges": (_I, [_P, _I, _P, _P]),
    "swdg_gauges_vjp": (_I, [_P, _I, _P, _P, _P, _I]),
    "swdg_diagnostics": (_I, [_P, _P]),
    "swdg_residual_noalloc": (_I, [ctypes.POINTER(swdg_config), _I64, _P, _P, _P, _I, _I, _P, _P,
                                   _P, _P, _P, _P, _D, _P, _P, ctypes.c_char_p, _I]),
    "swdg_residual_vjp": (_I, [_P, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I]),
    "swdg_step_record": (_I, [_P, _D, ctypes.POINTER(_D)]),
    "swdg_step_vjp": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I]),
    "swdg_set_bathymetry_offset": (_I, [_P, _P, _I]),
    "swdg_adjoint_slots": (_I, [_P, _I]),
    "swdg_step_record_slot": (_I, [_P, _I, _D, ctypes.POINTER(_D)]),
    "swdg_step_vjp_slot": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I]),
    "swdg_forest_flags": (_I, [ctypes.POINTER(swdg_forest), _I64, _P, _P, _D, _D, _P]),
    "swdg_forest_adapt": (_I, [ctypes.POINTER(swdg_forest), _I64, _P, _P, _I64, _P,
                               ctypes.POINTER(_I64)]),
    "swdg_forest_mesh": (_I, [ctypes.POINTER(swdg_forest), _I64, _P, _P, _P, _P]),
    "swdg_amr_setup": (_I, [_P, ctypes.POINTER(swdg_forest)]),
    "swdg_amr_indicator": (_I, [_P, _I, _P]),
    "swdg_amr_adapt": (_I, [_P, _P, _I, _D, _D, _P]),
    "swdg_amr_leaves": (_I, [_P, _P]),
    "swdg_set_members": (_I, [_P, _I, _P]),
    "swdg_upload_bathymetry_members": (_I, [_P, _P, _I, _P, _P]),
    "swdg_set_boundary_member": (_I, [_P, _I, _I, _I, _D, _D, _D]),
    "swdg_member_times": (_I, [_P, _P, _P, _I]),
    "swdg_member_diagnostics": (_I, [_P, _P]),
    "swdg_gather_gauges_member": (_I, [_P, _I, _I, _P, _P]),
    "swdg_set_shape": (_I, [_P, _I, _I, _I]),
    "swdg_get_shapes": (_I, [_P, _P]),
    "swdg_autotune": (_I, [_P, _I, _P]),
    "swdg_probe_fma": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "swdg_probe_roots": (_I, [_P, _I64, _P, _P]),
    "swdg_last_error": (ctypes.c_char_p, [_P]),
    "swdg_destroy": (None, [_P]),
}


def load():
    """Load the in-tree library (build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build the CUDA extension first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _buf(a, dtype):
    """(pointer, where, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, SWDG_HOST, None
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: t.float64, np.float32: t.float32, np.int32: t.int32,
                np.uint8: t.uint8}[dtype]
        if a.dtype != want:
            raise TypeError(f"tensor dtype {a.dtype}, expected {want}")
        return ctypes.c_void_p(a.data_ptr()), (SWDG_DEVICE if a.is_cuda else SWDG_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), SWDG_HOST, arr


def forest_flags(forest, lij, eta, theta_r, theta_c):
    """refine (1) / coarsen (-1) / keep (0) flags of Sec. 3.4 (host)"""
    lij = np.ascontiguousarray(lij, dtype=np.int32)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    out = np.zeros(len(lij), dtype=np.int8)
    rc = load().swdg_forest_flags(ctypes.byref(forest), len(lij), lij.ctypes.data_as(_P),
                                  eta.ctypes.data_as(_P), theta_r, theta_c, out.ctypes.data_as(_P))
    if rc:
        raise SwdgError(rc, "swdg_forest_flags failed")
    return out


def forest_adapt(forest, lij, flags):
    """the adapted, 2:1-balanced, Morton-ordered leaf set (host)"""
    lij = np.ascontiguousarray(lij, dtype=np.int32)
    flags = np.ascontiguousarray(flags, dtype=np.int8)
    nout = _I64(0)
    cap = 4 * len(lij) + 64
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        rc = load().swdg_forest_adapt(ctypes.byref(forest), len(lij), lij.ctypes.data_as(_P),
                                      flags.ctypes.data_as(_P), cap, out.ctypes.data_as(_P),
                                      ctypes.byref(nout))
        if rc == 0:
            return out[:nout.value]
        if nout.value <= cap:
            raise SwdgError(rc, "swdg_forest_adapt failed")
        cap = nout.value


def probe_fma(dtype):
    """Measured FMA-chain peak of the current device for SWDG_PIX_F64 or
    SWDG_PIX_F32: (TFLOP/s, ms of the best launch)."""
    tf, ms = _D(0.0), _D(0.0)
    rc = load().swdg_probe_fma(dtype, ctypes.byref(tf), ctypes.byref(ms))
    if rc:
        raise SwdgError(rc, "swdg_probe_fma failed")
    return tf.value, ms.value


def probe_roots(h):
    """the kernels' z = h^(-1/3) and z^3 for host values h > 0: (z, z^3)"""
    h = np.ascontiguousarray(h, dtype=np.float64)
    z, r = np.empty_like(h), np.empty_like(h)
    rc = load().swdg_probe_roots(h.ctypes.data_as(_P), h.size, z.ctypes.data_as(_P),
                                 r.ctypes.data_as(_P))
    if rc:
        raise SwdgError(rc, "swdg_probe_roots failed")
    return z, r


def forest_mesh(forest, lij):
    """x0y0 [n, 2], hxhy [n, 2], nbr [n, 4, 2] of an ordered leaf set (host)"""
    lij = np.ascontiguousarray(lij, dtype=np.int32)
    n = len(lij)
    x0y0, hxhy = np.zeros((n, 2)), np.zeros((n, 2))
    nbr = np.zeros((n, 4, 2), dtype=np.int32)
    rc = load().swdg_forest_mesh(ctypes.byref(forest), n, lij.ctypes.data_as(_P),
                                 x0y0.ctypes.data_as(_P), hxhy.ctypes.data_as(_P),
                                 nbr.ctypes.data_as(_P))
    if rc:
        raise SwdgError(rc, "swdg_forest_mesh failed")
    return x0y0, hxhy, nbr


def residual_noalloc(cfg, n_cells, hxhy, nbr, tiles, pixels_per_side, pix_dtype, manning, state,
                     t, residual, dt_out=None, bc=None):
    """Allocation-free residual (see swdg_residual_noalloc in include/swdg.h).
    Every array argument is a contiguous CUDA tensor; ``cfg`` a swdg_config;
    ``bc`` an optional list of (tag, kind, amp, period, phase)."""
    kind = (ctypes.c_int32 * 16)(*([SWDG_BC_WALL] * 16))
    amp = (_D * 16)(*([0.0] * 16))
    per = (_D * 16)(*([1.0] * 16))
    ph = (_D * 16)(*([0.0] * 16))
    for (tag, k, a, p, f) in (bc or []):
        kind[tag], amp[tag], per[tag], ph[tag] = k, a, p, f
    err = ctypes.create_string_buffer(256)

    def ptr(x):
        return ctypes.c_void_p(x.data_ptr()) if x is not None else None

    rc = load().swdg_residual_noalloc(
        ctypes.byref(cfg), n_cells, ptr(hxhy), ptr(nbr), ptr(tiles), pixels_per_side, pix_dtype,
        ptr(manning), ctypes.cast(kind, _P), ctypes.cast(amp, _P), ctypes.cast(per, _P),
        ctypes.cast(ph, _P), ptr(state), t, ptr(residual), ptr(dt_out), err, 256)
    if rc:
        raise SwdgError(rc, err.value.decode())
    return rc


class Context:
    """One swdg context (owns its device memory).  Methods mirror the C-ABI."""

    def __init__(self, degree=1, subgrid_mode=0, tableau=0, g=9.81, eps_vel=0.01, h_lim=0.01,
                 eps0=1e-6, cfl=0.1, newton_max=20, newton_tol=1e-12, stream=None, precision=0):
        L = load()
        if stream is None:
            t = _torch()
            if t is not None and t.cuda.is_available():
                stream = t.cuda.current_stream().cuda_stream
        self.cfg = swdg_config(degree, precision, subgrid_mode, tableau, g, eps_vel, h_lim, eps0,
                               cfl, newton_max, newton_tol, ctypes.c_void_p(stream or 0))
        h = ctypes.c_void_p()
        rc = L.swdg_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if rc:
            raise SwdgError(rc, "swdg_create failed")
        self.h = h
        self.degree = degree
        self.nd = (degree + 1) ** 2
        self.n = 0

    def _ck(self, rc):
        if rc:
            raise SwdgError(rc, load().swdg_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.swdg_destroy(self.h)
            self.h = None

    __del__ = close

    def upload_mesh(self, x0y0, hxhy, nbr):
        a, _, ka = _buf(x0y0, np.float64)
        b, _, kb = _buf(hxhy, np.float64)
        c, _, kc = _buf(nbr, np.int32)
        n = int(np.asarray(ka.shape[0] if hasattr(ka, "shape") else len(x0y0)))
        self._ck(load().swdg_upload_mesh(self.h, n, a, b, c))
        self.n = n

    def upload_bathymetry(self, z, xo, yo, dx, dy):
        z = np.ascontiguousarray(z)
        dtype = SWDG_PIX_F32 if z.dtype == np.float32 else SWDG_PIX_F64
        if dtype == SWDG_PIX_F64:
            z = np.ascontiguousarray(z, dtype=np.float64)
        ny, nx = z.shape
        self._ck(load().swdg_upload_bathymetry(self.h, z.ctypes.data_as(_P), dtype, nx, ny, xo, yo,
                                               dx, dy))

    def set_boundary(self, tag, kind, amp=0.0, period=1.0, phase=0.0):
        self._ck(load().swdg_set_boundary(self.h, tag, kind, amp, period, phase))

    def set_manning(self, n):
        p, where, keep = _buf(n, np.float64)
        self._ck(load().swdg_set_manning(self.h, p, where))

    def set_tracer_diffusivity(self, nu):
        """tracer numerical diffusivity nu_c per cell (Eq. numdiff); None: off"""
        p, where, keep = _buf(nu, np.float64)
        self._ck(load().swdg_set_tracer_diffusivity(self.h, p, where))

    def set_state(self, zeta, qx, qy, c):
        bufs = [_buf(v, np.float64) for v in (zeta, qx, qy, c)]
        where = bufs[0][1]
        self._ck(load().swdg_set_state(self.h, *[b[0] for b in bufs], where))

    def get_state(self, out=None):
        if out is None:
            out = [np.empty((self.n, self.nd)) for _ in range(4)]
        bufs = [_buf(v, np.float64) for v in out]
        self._ck(load().swdg_get_state(self.h, *[b[0] for b in bufs], bufs[0][1]))
        return out

    def residual(self, t=0.0, out=None):
        if out is None:
            out = [np.empty((self.n, self.nd)) for _ in range(6)]
        bufs = [_buf(v, np.float64) for v in out]
        self._ck(load().swdg_residual(self.h, t, *[b[0] for b in bufs], bufs[0][1]))
        return dict(zip(("F", "Gx", "Gy", "R", "Lx", "Ly"), out))

    def residual_vjp(self, cot, t=0.0):
        """discrete adjoint of the residual: cotangents of (F, Gx, Gy, R, Lx, Ly)
        (host arrays [n, nd], None = 0) to those of (zeta, qx, qy, c) [n, nd],
        the Manning coefficients [n] and per-cell bathymetry offsets [n]"""
        ins = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in cot]
        outs = [np.empty((self.n, self.nd)) for _ in range(4)] + [np.empty(self.n), np.empty(self.n)]
        ptr = [None if a is None else a.ctypes.data_as(_P) for a in ins]
        self._ck(load().swdg_residual_vjp(self.h, t, *ptr, *[o.ctypes.data_as(_P) for o in outs],
                                          SWDG_HOST))
        return dict(zip(("zeta", "qx", "qy", "c", "manning", "delta"), outs))

    def clock(self):
        """(t, last dt) of the context (member 0 of an ensemble)"""
        m = max(getattr(self, "m", 1), 1)
        t, dt = np.empty(m), np.empty(m)
        self._ck(load().swdg_member_times(self.h, t.ctypes.data_as(_P), dt.ctypes.data_as(_P), 0))
        return float(t[0]), float(dt[0])

    def set_bathymetry_offset(self, delta):
        """every depth of cell K deepened by delta[K] (absolute, None = 0)"""
        p, where, keep = _buf(delta, np.float64)
        self._ck(load().swdg_set_bathymetry_offset(self.h, p, where))

    # dynamic h-adaptation
    def amr_setup(self, forest):
        self.forest = forest
        self._ck(load().swdg_amr_setup(self.h, ctypes.byref(forest)))

    def amr_indicator(self, kind):
        eta = np.empty(self.n)
        self._ck(load().swdg_amr_indicator(self.h, kind, eta.ctypes.data_as(_P)))
        return eta

    def amr_adapt(self, theta_r, theta_c, eta=None, kind=0):
        """adapt the mesh (Sec. 3.4); returns the report of swdg_amr_adapt"""
        e = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        rep = np.zeros(9)
        self._ck(load().swdg_amr_adapt(self.h, None if e is None else e.ctypes.data_as(_P), kind,
                                       theta_r, theta_c, rep.ctypes.data_as(_P)))
        self.n = int(rep[1])
        return dict(zip(("cells_before", "cells_after", "refined", "coarsened", "Q", "tracer_Q",
                         "indicator_ms", "forest_ms", "rebuild_ms"), rep.tolist()))

    def amr_leaves(self):
        out = np.zeros((self.n, 3), dtype=np.int32)
        self._ck(load().swdg_amr_leaves(self.h, out.ctypes.data_as(_P)))
        return out

    def adjoint_slots(self, n):
        """reserve n step records (see swdg_adjoint_slots)"""
        self._ck(load().swdg_adjoint_slots(self.h, n))

    def step_record(self, dt, t=None, slot=None):
        """one fixed step of size dt, recorded for step_vjp; returns the end time"""
        tt = _D(0.0 if t is None else t)
        pt = ctypes.byref(tt) if t is not None else None
        if slot is None:
            self._ck(load().swdg_step_record(self.h, dt, pt))
        else:
            self._ck(load().swdg_step_record_slot(self.h, slot, dt, pt))
        return tt.value if t is not None else None

    def step_vjp(self, cot, slot=None):
        """adjoint of the recorded step: cotangent of the state after it (4 arrays
        [n, nd], host numpy or CUDA tensors) -> that of the state before it, the
        Manning coefficients [n] and the bathymetry offsets [n]"""
        dev = _torch() is not None and isinstance(cot[0], _torch().Tensor) and cot[0].is_cuda
        if dev:
            t = _torch()
            outs = [t.empty_like(cot[0]) for _ in range(4)] + \
                [t.empty(self.n, dtype=t.float64, device=cot[0].device) for _ in range(2)]
            keep = [a.contiguous() for a in cot]
            ptrs = [ctypes.c_void_p(a.data_ptr()) for a in keep] + \
                [ctypes.c_void_p(o.data_ptr()) for o in outs]
            where = SWDG_DEVICE
        else:
            keep = [np.ascontiguousarray(a, dtype=np.float64) for a in cot]
            outs = [np.empty((self.n, self.nd)) for _ in range(4)] + [np.empty(self.n),
                                                                        np.empty(self.n)]
            ptrs = [a.ctypes.data_as(_P) for a in keep] + [o.ctypes.data_as(_P) for o in outs]
            where = SWDG_HOST
        if slot is None:
            self._ck(load().swdg_step_vjp(self.h, *ptrs, where))
        else:
            self._ck(load().swdg_step_vjp_slot(self.h, slot, *ptrs, where))
        return dict(zip(("zeta", "qx", "qy", "c", "manning", "delta"), outs))

    def cfl_dt(self, t=0.0):
        d = _D(0.0)
        self._ck(load().swdg_cfl_dt(self.h, t, ctypes.byref(d)))
        return d.value

    def step(self, n=1, dt=-1.0, t=None):
        tt = _D(0.0 if t is None else t)
        self._ck(load().swdg_step(self.h, n, dt, ctypes.byref(tt) if t is not None else None))
        return tt.value if t is not None else None

    def step_profile(self, n=1, dt=-1.0, t=None):
        """per-kernel-slot milliseconds (CUDA events) summed over n eager steps"""
        tt = _D(0.0 if t is None else t)
        ms = np.zeros(13)
        self._ck(load().swdg_step_profile(self.h, n, dt, ctypes.byref(tt) if t is not None else None,
                                          ms.ctypes.data_as(_P)))
        return ms, (tt.value if t is not None else None)

    def degree_switch(self):
        f = np.empty(self.n, dtype=np.uint8)
        self._ck(load().swdg_degree_switch(self.h, f.ctypes.data_as(_P)))
        return f

    def gather_gauges(self, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        out = np.empty(len(xy))
        self._ck(load().swdg_gather_gauges(self.h, len(xy), xy.ctypes.data_as(_P),
                                           out.ctypes.data_as(_P)))
        return out

    def gauges_vjp(self, xy, gbar, zeta_b):
        """zeta_b (host array or CUDA tensor [n, nd], updated in place) += the
        transpose of the gauge interpolation at xy [ng, 2] applied to gbar [ng]"""
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        g = np.ascontiguousarray(gbar, dtype=np.float64)
        if g.shape != (len(xy),):
            raise ValueError("gbar must have one value per gauge")
        p, where, keep = _buf(zeta_b, np.float64)
        if keep is not zeta_b:
            raise ValueError("zeta_b must be a contiguous float64 array or tensor")
        self._ck(load().swdg_gauges_vjp(self.h, len(xy), xy.ctypes.data_as(_P),
                                        g.ctypes.data_as(_P), p, where))

    DIAG_KEYS = ("mass", "tracer_mass", "min_h", "r_cells", "newton_max",
                 "positivity_violations", "dt", "t")

    def diagnostics(self):
        d = np.empty(8)
        self._ck(load().swdg_diagnostics(self.h, d.ctypes.data_as(_P)))
        return dict(zip(self.DIAG_KEYS, d.tolist()))

    # launch shapes and the autotuner
    def set_shape(self, kind, grid, warps_per_block):
        self._ck(load().swdg_set_shape(self.h, kind, grid, warps_per_block))

    def shapes(self):
        out = np.zeros(8, dtype=np.int32)
        self._ck(load().swdg_get_shapes(self.h, out.ctypes.data_as(_P)))
        return {k: (int(out[2 * i]), int(out[2 * i + 1]))
                for i, k in enumerate(("begin", "residual", "stage", "aux"))}

    def autotune(self, repeats=2):
        """pick the fastest launch shape per kernel kind on this context's own
        mesh and state; returns {kind: (grid, warps per block, ms per step)}"""
        rep = np.zeros(9)
        self._ck(load().swdg_autotune(self.h, repeats, rep.ctypes.data_as(_P)))
        return {k: (int(rep[3 * i]), int(rep[3 * i + 1]), float(rep[3 * i + 2]))
                for i, k in enumerate(("begin", "residual", "stage"))}

    @classmethod
    def from_workload(cls, wl, stream=None, **over):
        cfg = wl.config(**over)
        ctx = cls(stream=stream, **cfg)
        ctx.upload_mesh(wl.mesh.x0y0, wl.mesh.hxhy, wl.mesh.nbr)
        r = wl.raster
        ctx.upload_bathymetry(r.z, r.xo, r.yo, r.dx, r.dy)
        for (tag, kind, amp, per, ph) in wl.boundaries:
            ctx.set_boundary(tag, kind, amp, per, ph)
        if wl.manning is not None:
            ctx.set_manning(wl.manning)
        if getattr(wl, "tracer_diffusivity", None) is not None:
            ctx.set_tracer_diffusivity(wl.tracer_diffusivity)
        ctx.set_state(*wl.state())
        return ctx


class Ensemble(Context):
    """Independent members (one Workload each) advanced by the same launches:
    the context's mesh is the disjoint union of the members' meshes, every
    member keeps its own CFL step, clock, tide and bathymetry raster."""

    def set_members(self, first_cell):
        first = np.ascontiguousarray(first_cell, dtype=np.int64)
        self._ck(load().swdg_set_members(self.h, len(first) - 1, first.ctypes.data_as(_P)))
        self.first = first
        self.m = len(first) - 1

    def upload_bathymetry_members(self, rasters):
        """rasters: list of workloads.Raster, one per member"""
        zs = [np.ascontiguousarray(r.z) for r in rasters]
        f32 = all(z.dtype == np.float32 for z in zs)
        dtype = SWDG_PIX_F32 if f32 else SWDG_PIX_F64
        zs = [np.ascontiguousarray(z, dtype=np.float32 if f32 else np.float64) for z in zs]
        ptrs = (_P * len(zs))(*[z.ctypes.data for z in zs])
        nxny = np.array([[z.shape[1], z.shape[0]] for z in zs], dtype=np.int64)
        geo = np.array([[r.xo, r.yo, r.dx, r.dy] for r in rasters], dtype=np.float64)
        self._ck(load().swdg_upload_bathymetry_members(self.h, ctypes.cast(ptrs, _P), dtype,
                                                       nxny.ctypes.data_as(_P),
                                                       geo.ctypes.data_as(_P)))

    def set_boundary_member(self, member, tag, kind, amp=0.0, period=1.0, phase=0.0):
        self._ck(load().swdg_set_boundary_member(self.h, member, tag, kind, amp, period, phase))

    def times(self):
        t = np.empty(self.m)
        dt = np.empty(self.m)
        self._ck(load().swdg_member_times(self.h, t.ctypes.data_as(_P), dt.ctypes.data_as(_P), 0))
        return t, dt

    def set_times(self, t):
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), (self.m,)))
        self._ck(load().swdg_member_times(self.h, t.ctypes.data_as(_P), None, 1))

    def step(self, n=1, dt=-1.0, t=None):
        if t is not None:
            raise ValueError("an ensemble keeps one clock per member: use set_times/times")
        self._ck(load().swdg_step(self.h, n, dt, None))

    def member_diagnostics(self):
        d = np.empty((self.m, 8))
        self._ck(load().swdg_member_diagnostics(self.h, d.ctypes.data_as(_P)))
        return [dict(zip(self.DIAG_KEYS, row.tolist())) for row in d]

    def member_slice(self, m):
        return slice(int(self.first[m]), int(self.first[m + 1]))

    def member_state(self, m):
        return [a[self.member_slice(m)] for a in self.get_state()]

    def gather_gauges_member(self, member, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        out = np.empty(len(xy))
        self._ck(load().swdg_gather_gauges_member(self.h, member, len(xy), xy.ctypes.data_as(_P),
                                                  out.ctypes.data_as(_P)))
        return out

    @classmethod
    def from_workloads(cls, wls, stream=None, **over):
        """one member per workload; the solver settings (degree, tableau, cfl,
        eps, ...) must agree across the workloads and are taken from the first"""
        from .workloads import union_mesh
        cfg = wls[0].config(**over)
        for w in wls[1:]:
            if w.config(**over) != cfg:
                raise ValueError(f"member {w.name}: solver settings differ from {wls[0].name}")
        ctx = cls(stream=stream, **cfg)
        x0y0, hxhy, nbr, first = union_mesh([w.mesh for w in wls])
        ctx.upload_mesh(x0y0, hxhy, nbr)
        ctx.set_members(first)
        ctx.upload_bathymetry_members([w.raster for w in wls])
        for m, w in enumerate(wls):
            for (tag, kind, amp, per, ph) in w.boundaries:
                ctx.set_boundary_member(m, tag, kind, amp, per, ph)
        man = np.concatenate([w.manning if w.manning is not None else np.zeros(w.mesh.n)
                              for w in wls])
        ctx.set_manning(man)
        if any(getattr(w, "tracer_diffusivity", None) is not None for w in wls):
            ctx.set_tracer_diffusivity(np.concatenate(
                [w.tracer_diffusivity if w.tracer_diffusivity is not None else np.zeros(w.mesh.n)
                 for w in wls]))
        st = [np.concatenate(parts) for parts in zip(*[w.state() for w in wls])]
        ctx.set_state(*st)
        return ctx
