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
