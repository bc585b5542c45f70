"""The library's host-side forest (swdg_forest_flags / _adapt / _mesh; no
GPU) against the adaptation reference in oracle/amr.py: identical flags,
leaf sets (in Morton order) and meshes over random adaptation sequences,
with and without periodicity."""
import numpy as np
import pytest

from oracle.amr import Forest
from paper_2505_18743_gb300 import swdg


@pytest.mark.parametrize("periodic", [(False, False), (True, False), (True, True)])
def test_forest_functions_match_the_reference(periodic):
    args = (5, 3, 10.0, -20.0, 80.0, 60.0, 4, 6.0, (1, 2, 3, 4), periodic)
    ref = Forest(*args)
    lib = swdg.make_forest(*args)
    leaves = ref.order({(0, i, j) for i in range(5) for j in range(3)})
    rng = np.random.default_rng(11)
    for it in range(8):
        eta = rng.uniform(0.0, 1.0, len(leaves)) ** 3
        eta[rng.integers(len(leaves), size=2)] = 2.0
        lij = np.array(leaves, dtype=np.int32)
        f_ref = np.array(ref.flags(leaves, eta, 0.2, 0.05), dtype=np.int8)
        f_lib = swdg.forest_flags(lib, lij, eta, 0.2, 0.05)
        np.testing.assert_array_equal(f_lib, f_ref)
        new_ref = ref.adapt(leaves, f_ref)
        new_lib = swdg.forest_adapt(lib, lij, f_lib)
        np.testing.assert_array_equal(new_lib, np.array(new_ref, dtype=np.int32))
        m_ref = ref.mesh(new_ref)
        m_lib = swdg.forest_mesh(lib, new_lib)
        for a, b in zip(m_lib, m_ref):
            np.testing.assert_array_equal(a, b)
        leaves = new_ref
    assert max(c[0] for c in leaves) >= 3 and len(leaves) > 15


def test_forest_rejects_bad_input():
    lib = swdg.make_forest(2, 2, 0.0, 0.0, 1.0, 1.0, 2)
    with pytest.raises(swdg.SwdgError):
        swdg.forest_adapt(lib, np.array([[3, 0, 0]], dtype=np.int32), np.zeros(1, np.int8))
    # a leaf set that is not 2:1 balanced has no mesh
    bad = np.array([[0, 0, 0], [0, 0, 1], [0, 1, 1]] +
                   [[2, 4 + a, b] for a in range(4) for b in range(4)], dtype=np.int32)
    with pytest.raises(swdg.SwdgError):
        swdg.forest_mesh(lib, bad)
