"""Pins of the oracle's sub-grid operators (Sec. 3.3) against brute-force
supersampling, calculus identities and special cases."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def one_cell(z, degree=1, mode=0, L=1.0):
    ny, nx = z.shape
    mesh = W.uniform_mesh(1, 1, L, L)
    ras = W.Raster(np.asarray(z, dtype=np.float64), 0.0, 0.0, L / nx, L / ny)
    return Oracle(mesh, ras, degree=degree, subgrid_mode=mode), ras


def brute(z, X0, X1, Y0, Y1, eta, m):
    """midpoint supersampling with m x m samples inside the rectangle"""
    ny, nx = z.shape
    xs = X0 + (np.arange(m) + 0.5) * (X1 - X0) / m
    ys = Y0 + (np.arange(m) + 0.5) * (Y1 - Y0) / m
    Xs, Ys = np.meshgrid(xs, ys)
    zz = z[np.minimum((Ys * ny).astype(int), ny - 1), np.minimum((Xs * nx).astype(int), nx - 1)]
    d = eta + zz
    return np.mean(np.maximum(d, 0.0)), np.mean(d > 0)


def test_rect_equals_brute_force_on_dyadic_rectangles():
    rng = np.random.default_rng(1)
    z = rng.uniform(-1.0, 1.0, size=(4, 4))
    o, _ = one_cell(z)
    for _ in range(40):
        e = rng.integers(0, 65, size=4) / 64.0
        X0, X1 = sorted(e[:2])
        Y0, Y1 = sorted(e[2:])
        if X1 - X0 < 1 / 64 or Y1 - Y0 < 1 / 64:
            continue
        eta = rng.uniform(-1, 1)
        V, A = o.subgrid_rect(X0, X1, Y0, Y1, eta)
        # 1/64 grid aligned samples resolve the pixel (1/4) and rectangle edges exactly
        m = int(round((X1 - X0) * 64)) * 8, int(round((Y1 - Y0) * 64)) * 8
        xs = X0 + (np.arange(m[0]) + 0.5) * (X1 - X0) / m[0]
        ys = Y0 + (np.arange(m[1]) + 0.5) * (Y1 - Y0) / m[1]
        Xs, Ys = np.meshgrid(xs, ys)
        zz = z[(Ys * 4).astype(int), (Xs * 4).astype(int)]
        d = eta + zz
        assert abs(V - np.mean(np.maximum(d, 0))) < 1e-14
        assert abs(A - np.mean(d > 0)) < 1e-14


def test_rect_brute_force_general_rectangle():
    rng = np.random.default_rng(2)
    z = rng.uniform(-2.0, 2.0, size=(3, 5))
    o, _ = one_cell(z)
    for _ in range(5):
        X0, X1 = np.sort(rng.uniform(0, 1, 2))
        Y0, Y1 = np.sort(rng.uniform(0, 1, 2))
        eta = rng.uniform(-1, 1)
        V, A = o.subgrid_rect(X0, X1, Y0, Y1, eta)
        Vb, Ab = brute(z, X0, X1, Y0, Y1, eta, 1500)
        assert abs(V - Vb) < 5e-3 and abs(A - Ab) < 5e-3


def test_area_is_derivative_of_volume_and_volume_is_convex():
    rng = np.random.default_rng(3)
    z = rng.uniform(-1.0, 1.0, size=(4, 4))
    o, _ = one_cell(z, degree=3)
    etas = np.linspace(-1.2, 1.2, 241)
    for p in range(25):
        V = np.array([o.subgrid_point(0, 1, p, e)[0] for e in etas])
        d2 = V[2:] - 2 * V[1:-1] + V[:-2]
        assert d2.min() > -1e-13            # convex
        assert np.all(np.diff(V) >= -1e-15)  # monotone
        for e in rng.uniform(-1, 1, 5):
            if np.min(np.abs(e + z)) < 1e-4:
                continue
            h = 1e-7
            fd = (o.subgrid_point(0, 1, p, e + h)[0] - o.subgrid_point(0, 1, p, e - h)[0]) / (2 * h)
            assert abs(fd - o.subgrid_point(0, 1, p, e)[1]) < 1e-7


@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("pset", [0, 1, 2])
def test_sub_cells_partition_the_cell(degree, pset):
    """sum_p w_p V_p(eta) = (1/|K|) int_K max(eta + z_b, 0): the sub-cells of a
    rule tile the cell with areas equal to the weights (mass exactness of R1)."""
    rng = np.random.default_rng(4)
    z = rng.uniform(-1.0, 1.0, size=(16, 16))
    o, _ = one_cell(z, degree=degree)
    n = {0: (3 * degree) // 2 + 1, 1: degree + 2, 2: degree + 1}[pset]
    kind = {0: 0, 1: 1, 2: 0}[pset]
    x, w = __import__("oracle.oracle", fromlist=["rule"]).rule(kind, n)
    for eta in (-0.5, 0.0, 0.3):
        s = sum(w[p % n] * w[p // n] * o.subgrid_point(0, pset, p, eta)[0] for p in range(n * n))
        Vc, _ = o.subgrid_rect(0, 1, 0, 1, eta)
        assert abs(s - Vc) < 1e-14
        assert abs(Vc - np.mean(np.maximum(eta + z, 0))) < 1e-14


def test_constant_raster_reduces_to_pointwise_max():
    o, _ = one_cell(np.full((8, 8), 0.7), degree=2)
    for eta in (-1.0, -0.7, -0.2, 0.5):
        for p in range(16):
            V, A = o.subgrid_point(0, 1, p, eta)
            assert abs(V - max(eta + 0.7, 0.0)) < 1e-15
            assert abs(A - (1.0 if eta + 0.7 > 0 else 0.0)) < 1e-15


def test_mode_p_bilinear_is_exact_on_linear_raster():
    nx, ny = 8, 6
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc)
    z = 0.3 + 1.7 * X - 0.9 * Y
    o, _ = one_cell(z, mode=1)
    rng = np.random.default_rng(5)
    for _ in range(50):
        x = rng.uniform(xc[0], xc[-1])
        y = rng.uniform(yc[0], yc[-1])
        assert abs(o.zb_point(x, y) - (0.3 + 1.7 * x - 0.9 * y)) < 1e-14
    # clamped outside the pixel centres
    assert abs(o.zb_point(0.0, yc[2]) - z[2, 0]) < 1e-14


def test_mode_p_point_operator():
    rng = np.random.default_rng(6)
    z = rng.uniform(-1.0, 1.0, size=(8, 8))
    o, _ = one_cell(z, mode=1, degree=2)
    xm, _ = __import__("oracle.oracle", fromlist=["rule"]).rule(1, 4)
    for p in range(16):
        zb = o.zb_point(xm[p % 4], xm[p // 4])
        for eta in (-0.3, 0.2):
            V, A = o.subgrid_point(0, 1, p, eta)
            assert V == max(eta + zb, 0.0) and A == float(eta + zb > 0)
