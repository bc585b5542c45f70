"""Shared test helpers: golden-file reader, closed-form solutions written from
the paper, and error norms evaluated with library quadrature (numpy)."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def golden_dict(name):
    return {r[0]: float(r[1]) for r in golden_rows(name)}


# ---------------------------------------------------------------------------
# travelling vortex (Sec. 4.4): h(R) = h0 - 4/g (4 Gamma r0/pi)^2 (H(pi/2) - H(rho/2)),
# rho = pi R / r0, omega = 4 Gamma cos^4(rho/2), u = u_inf - (y-y0) omega,
# v = (x-x0) omega; Gamma fixed by h(0) = h_min
# ---------------------------------------------------------------------------
def vortex_H(x):
    c, s = np.cos(x), np.sin(x)
    return (35 * np.cos(2 * x) / 384 + 35 * x * np.sin(2 * x) / 192 + c ** 6 * (c ** 2 / 64 + 7 / 288)
            + 35 * np.cos(2 * x) ** 2 / 3072 + 35 * x ** 2 / 256
            + 35 * x * np.cos(2 * x) * np.sin(2 * x) / 768 + x * c ** 5 * s * (c ** 2 + 7 / 6) / 8)


class Vortex:
    def __init__(self, g=9.81):
        p = golden_dict("vortex_parameters.txt")
        self.g = g
        self.h0, self.hmin, self.uinf, self.r0 = p["h0"], p["hmin"], p["uinf"], p["r0"]
        self.xc, self.yc, self.T = p["x0"], p["y0"], p["T"]
        self.Lx, self.Ly = p["Lx"], p["Ly"]
        dH = vortex_H(np.pi / 2) - vortex_H(0.0)
        self.Gam = (np.pi / (4 * self.r0)) * np.sqrt(g * (self.h0 - self.hmin) / (4 * dH))

    def __call__(self, X, Y, t):
        dx = X - (self.xc + self.uinf * t)
        dy = Y - self.yc
        R = np.sqrt(dx * dx + dy * dy)
        rho = np.pi * R / self.r0
        inside = rho < np.pi
        om = np.where(inside, 4 * self.Gam * np.cos(rho / 2) ** 4, 0.0)
        k = (4 / self.g) * (4 * self.Gam * self.r0 / np.pi) ** 2
        h = self.h0 - np.where(inside, k * (vortex_H(np.pi / 2) - vortex_H(np.minimum(rho, np.pi) / 2)), 0.0)
        return h, self.uinf - dy * om, dx * om


def cell_quadrature(mesh, n=6):
    """Points and weights of an n x n Gauss-Legendre rule on every cell."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (1 + x)
    w = 0.5 * w
    A, B = np.meshgrid(x, x)
    WA, WB = np.meshgrid(w, w)
    px = (mesh.x0y0[:, 0:1] + mesh.hxhy[:, 0:1] * A.ravel()[None, :]).ravel()
    py = (mesh.x0y0[:, 1:2] + mesh.hxhy[:, 1:2] * B.ravel()[None, :]).ravel()
    wt = (mesh.hxhy[:, 0:1] * mesh.hxhy[:, 1:2] * (WA * WB).ravel()[None, :]).ravel()
    return px, py, wt


def rel_inf(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(float(np.abs(b).max()) if b.size else 0.0, floor)
    if den == 0.0:
        return float(np.abs(a - b).max()) if a.size else 0.0
    return float(np.abs(a - b).max()) / den


FIELDS = ("F", "Gx", "Gy", "R", "Lx", "Ly")


def residual_errors(got, ref, floor_frac=1e-3):
    """Per-field relative errors of a residual against the oracle's: for each
    field f, max|got_f - ref_f| / max(max|ref_f|, floor_frac * max|ref_f|), the
    floor taken from the same field only, so a small field (F or L next to
    the g h grad zeta term of G) is held to its own scale.  ``got`` and ``ref``
    map field names to arrays; a field that is zero in the oracle is compared
    absolutely."""
    out = {}
    for k in ref:
        r = np.asarray(ref[k], dtype=np.float64)
        g = np.asarray(got[k], dtype=np.float64)
        own = float(np.abs(r).max()) if r.size else 0.0
        out[k] = rel_inf(g, r, floor=floor_frac * own)
    return out


# ---------------------------------------------------------------------------
# Thacker's oscillating paraboloid (Sec. 4.3).  The free surface is taken with
# a plus sign, zeta = h0 (s - 1 - R^2/a^2 (s^2 - 1)), s = sqrt(1 - A^2) /
# (1 - A cos(omega t)): with the depth z_b = h0 (1 - R^2/a^2) this gives
# h = zeta + z_b = h0 s (1 - s R^2/a^2), which solves the equations with the
# printed velocity (checked in the tests); the leading minus sign of the
# printed formula does not.
# ---------------------------------------------------------------------------
class Thacker:
    def __init__(self, g=9.81, sign=1.0):
        p = golden_dict("thacker_parameters.txt")
        self.g, self.sign = g, sign
        self.h0, self.L, self.a, self.r0 = p["h0"], p["L"], p["a"], p["r0"]
        self.h_lim, self.eps400, self.periods = p["h_lim"], p["eps_at_400"], int(p["periods"])
        self.omega = np.sqrt(8 * g * self.h0) / self.a
        self.A = (self.a ** 2 - self.r0 ** 2) / (self.a ** 2 + self.r0 ** 2)
        self.T = 2 * np.pi / self.omega

    def zb(self, X, Y):
        R2 = (X - self.L / 2) ** 2 + (Y - self.L / 2) ** 2
        return self.h0 * (1 - R2 / self.a ** 2)

    def __call__(self, X, Y, t):
        """free surface (of the paraboloid, also where it lies below the
        ground) and velocity"""
        R2 = (X - self.L / 2) ** 2 + (Y - self.L / 2) ** 2
        den = 1 - self.A * np.cos(self.omega * t)
        s = np.sqrt(1 - self.A ** 2) / den
        zeta = self.sign * self.h0 * (s - 1 - R2 / self.a ** 2 * (s * s - 1))
        f = self.A * self.omega * np.sin(self.omega * t) / (2 * den)
        return zeta, f * (X - self.L / 2), f * (Y - self.L / 2)
