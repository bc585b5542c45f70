"""Pins of the adaptation reference (oracle/amr.py): the adapted leaf sets
tile the domain and are 2:1 balanced with mutual neighbours, the criteria of
Sec. 3.4 are honoured, the mesh of a static forest agrees with the
independent input generator, prolongation is exact and restriction after it
the identity, restriction conserves every field's integral, and the
indicators of Sec. 4.4 and Sec. 5 reproduce closed forms."""
import numpy as np
import pytest

from oracle.amr import Forest, indicator, remap
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def forest(periodic=(False, False), max_level=3):
    return Forest(6, 4, 0.0, 0.0, 100.0, 100.0, max_level, 0.0, (1, 0, 2, 0), periodic)


def check_balanced(F, leaves):
    x0y0, hxhy, nbr = F.mesh(leaves)
    area = (hxhy[:, 0] * hxhy[:, 1]).sum()
    assert abs(area - 6 * 4 * 100.0 * 100.0) < 1e-6
    lev = {k: c[0] for k, c in enumerate(leaves)}
    for k in range(len(leaves)):
        for f in range(4):
            s0, s1 = nbr[k, f]
            if s0 < 0:
                continue
            for nb in ([s0, s1] if s1 >= 0 else [s0]):
                assert abs(lev[nb] - lev[k]) <= 1
                assert k in nbr[nb, f ^ 1]
    assert len(set(leaves)) == len(leaves)


@pytest.mark.parametrize("periodic", [(False, False), (True, True)])
def test_adapt_is_balanced_and_honours_the_criteria(periodic):
    F = forest(periodic)
    leaves = F.order({(0, i, j) for i in range(6) for j in range(4)})
    rng = np.random.default_rng(3)
    for it in range(5):
        eta = rng.uniform(0.0, 1.0, len(leaves))
        eta[rng.integers(len(leaves))] = 5.0
        flags = F.flags(leaves, eta, 0.3, 0.1)
        new = F.adapt(leaves, flags)
        check_balanced(F, new)
        S = set(new)
        for c, fl in zip(leaves, flags):
            if fl == 1:  # refined: the cell is no leaf any more
                assert c not in S
        for c in S:
            if c not in set(leaves) and F.covering(set(leaves), *c) is None:
                # a new coarse leaf: all four children were leaves marked for coarsening
                l, i, j = c
                kids = [(l + 1, 2 * i + a, 2 * j + b) for a in (0, 1) for b in (0, 1)]
                idx = {x: k for k, x in enumerate(leaves)}
                assert all(x in idx and flags[idx[x]] == -1 for x in kids)
        leaves = new
    assert max(c[0] for c in leaves) >= 2


def test_mesh_of_a_static_forest_matches_the_input_generator():
    refine = lambda l, x, y, hx, hy: (np.abs(x - 250.0) < 120.0) & (y < 250.0)
    mesh, level = W.forest_mesh(6, 4, 600.0, 400.0, 3, refine, tags=(1, 0, 2, 0))
    F = Forest(6, 4, 0.0, 0.0, 100.0, 100.0, int(level.max()), 0.0, (1, 0, 2, 0))
    leaves = F.order(F.leaves_of_mesh(mesh))
    x0y0, hxhy, nbr = F.mesh(leaves)
    np.testing.assert_array_equal(x0y0, mesh.x0y0)
    np.testing.assert_array_equal(hxhy, mesh.hxhy)
    np.testing.assert_array_equal(nbr, mesh.nbr)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_remap_prolongation_exact_restriction_conservative(degree):
    F = forest()
    leaves = F.order({(0, i, j) for i in range(6) for j in range(4)})
    nd = (degree + 1) ** 2
    rng = np.random.default_rng(7)
    u = [rng.standard_normal((len(leaves), nd)) for _ in range(2)]
    flags = [1 if k % 3 == 0 else 0 for k in range(len(leaves))]
    fine = F.adapt(leaves, flags)
    up = remap(F, leaves, u, fine, degree)
    # the fine fields integrate like the coarse ones
    from oracle.oracle import rule
    xs, _ = rule(1, degree + 1)
    xg, wg = rule(0, degree + 1)
    from oracle.amr import _lagrange

    def integrals(lv, fld):
        out = 0.0
        for c, val in zip(lv, fld):
            hx, hy = F.size(c[0])
            for qb, wb in zip(xg, wg):
                for qa, wa in zip(xg, wg):
                    out += hx * hy * wa * wb * np.outer(_lagrange(xs, qb), _lagrange(xs, qa)).ravel() @ val
        return out

    for a, b in zip(u, up):
        assert abs(integrals(leaves, a) - integrals(fine, b)) <= 1e-9 * np.abs(a).sum()
    # restriction of the prolonged field gives back the coarse nodal values
    back = remap(F, fine, up, leaves, degree)
    for a, b in zip(u, back):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-11)
    # restriction of an arbitrary fine field conserves its integral
    v = [rng.standard_normal((len(fine), nd))]
    coarse = remap(F, fine, v, leaves, degree)
    assert abs(integrals(fine, v[0]) - integrals(leaves, coarse[0])) <= 1e-9 * np.abs(v[0]).sum()


@pytest.mark.parametrize("degree", [1, 2])
def test_indicators_closed_forms(degree):
    mesh, ras = W.flat_periodic(4, 3, 400.0, 300.0, 5.0, degree, pix=2)
    Xn, Yn = W.nodal_coordinates(mesh, degree)
    om, a, b = 1e-3, 0.002, -0.001
    h0 = 5.0
    zeta = np.zeros_like(Xn)
    qx, qy = -h0 * om * Yn, h0 * om * Xn  # solid-body rotation on a flat bottom: curl u = 2 om
    c = a * Xn + b * Yn
    o = Oracle(mesh, ras, degree=degree)
    o.set_state(zeta, qx, qy, c)
    e0 = indicator(o, mesh, (zeta, qx, qy, c), degree, 0, 0.01)
    e1 = indicator(o, mesh, (zeta, qx, qy, c), degree, 1, 0.01)
    np.testing.assert_allclose(e0, 2 * om, rtol=1e-11)
    np.testing.assert_allclose(e1, np.hypot(a, b), rtol=1e-11)
