"""Pins of the oracle's quadrature rules and time integrators against closed
forms, library routines and the numbers the paper prints."""
import numpy as np
import pytest

from helpers import golden_rows
from oracle import oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exactness_and_library(n):
    x, w = O.rule(0, n)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * n):  # exact up to degree 2n-1
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    xl, wl = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (1 + xl), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wl, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gauss_lobatto_exactness_and_endpoints(n):
    x, w = O.rule(1, n)
    assert x[0] == 0.0 and x[-1] == 1.0
    for k in range(2 * n - 2):  # exact up to degree 2n-3
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    # not exact one degree higher (the rule is not a Gauss rule)
    assert abs(np.dot(w, x ** (2 * n - 2)) - 1.0 / (2 * n - 1)) > 1e-6
    # end-point weight of the n-point rule on [0, 1]: 1 / (n (n - 1))
    assert abs(w[0] - 1.0 / (n * (n - 1))) < 1e-15


def test_gll_closed_forms():
    x, w = O.rule(1, 3)
    np.testing.assert_allclose(x, [0, 0.5, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    x, w = O.rule(1, 5)
    np.testing.assert_allclose(w, [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20], atol=1e-15)
    np.testing.assert_allclose(x, 0.5 * (1 + np.array([-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1])),
                               atol=1e-15)


def test_cfl_table_matches_paper():
    """Table tab:cfl: CFL = w_1 / a_21 with w_1 the end weight of the (r+2)-point
    GLL rule and a_21 = 2 chi of RK32; printed 0.28 / 0.14 / 0.085."""
    tab = O.tableau(0)
    a21 = tab["a"][1, 0]
    rows = [r for r in golden_rows("cfl_table.txt") if r[0] != "inv_a21"]
    for r, printed, linear in rows:
        r = int(r)
        x, w = O.rule(1, r + 2)
        cfl = w[0] / a21
        assert round(cfl, 2 if r < 3 else 3) == float(printed)
        assert abs(1.0 / (2 * r + 1) - float(linear)) < 1e-9
    inv = [r for r in golden_rows("cfl_table.txt") if r[0] == "inv_a21"][0]
    assert abs(1.0 / a21 - float(inv[1])) < 0.01


def test_rk32_imex_order_and_coupling_conditions():
    """Appendix A: sum b = sum b~ = 1; sum b c = sum b~ c~ = sum b c~ = sum b~ c = 1/2;
    row sums of A and A~ equal c; b = b~ (linear invariants); a_32 = 1/2."""
    t = O.tableau(0)
    a, at, b, bt, c = t["a"], t["at"], t["b"], t["bt"], t["c"]
    chi = 1 - np.sqrt(2) / 2
    assert abs(a[1, 0] - 2 * chi) < 1e-15 and a[2, 1] == 0.5
    np.testing.assert_allclose(a.sum(1), c, atol=1e-15)
    np.testing.assert_allclose(at.sum(1), c, atol=1e-15)
    np.testing.assert_allclose(b, bt, atol=0)
    for x in (b, bt):
        assert abs(x.sum() - 1) < 1e-15
        assert abs(np.dot(x, c) - 0.5) < 1e-15
    # DIRK: a~_lm = 0 for l < m; L-stable TR-BDF2 last row = b~ (stiffly accurate)
    assert np.all(np.triu(at, 1) == 0)
    np.testing.assert_allclose(at[2], bt, atol=0)
    assert np.all(np.triu(a) == 0)


def test_ssp33_and_rk44_order_conditions():
    t = O.tableau(1)
    a, b, c = t["a"], t["b"], t["c"]
    assert abs(b.sum() - 1) < 1e-15 and abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15 and abs(b @ a @ c - 1 / 6) < 1e-15
    t = O.tableau(2)
    a, b, c = t["a"], t["b"], t["c"]
    conds = [(b.sum(), 1), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ a @ c, 1 / 6),
             (b @ c ** 3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ a @ c ** 2, 1 / 12),
             (b @ a @ a @ c, 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < 1e-15
