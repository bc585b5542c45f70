"""Host-side ensemble inputs: the disjoint union of member meshes and the
seeded member draws (no GPU)."""
import numpy as np

from paper_2505_18743_gb300 import workloads as W


def test_union_mesh_shifts_neighbours_and_keeps_tags():
    a = W.uniform_mesh(3, 2, 30.0, 20.0, tags=(1, 0, 0, 0))
    b, _ = W.forest_mesh(2, 2, 20.0, 20.0, 2, lambda l, x, y, hx, hy: x < 10.0)
    c = W.uniform_mesh(2, 2, 20.0, 20.0, periodic=(True, True))
    x0y0, hxhy, nbr, first = W.union_mesh([a, b, c])
    assert list(first) == [0, a.n, a.n + b.n, a.n + b.n + c.n]
    assert x0y0.shape == (first[-1], 2) and hxhy.shape == (first[-1], 2)
    for m, mesh in enumerate((a, b, c)):
        sl = slice(first[m], first[m + 1])
        np.testing.assert_array_equal(x0y0[sl], mesh.x0y0)
        own = nbr[sl]
        inner = mesh.nbr >= 0
        np.testing.assert_array_equal(own[inner], mesh.nbr[inner] + first[m])
        np.testing.assert_array_equal(own[~inner], mesh.nbr[~inner])  # tags and empty slots
        # no neighbour outside the member
        assert np.all((own < 0) | ((own >= first[m]) & (own < first[m + 1])))


def test_beach_ensemble_draws_are_seeded_and_in_range():
    e1 = W.beach_ensemble(members=6, sizes=(4, 6, 8), pix=4)
    e2 = W.beach_ensemble(members=6, sizes=(4, 6, 8), pix=4)
    for w1, w2 in zip(e1, e2):
        assert w1.mesh.n == w2.mesh.n and w1.boundaries == w2.boundaries
        np.testing.assert_array_equal(w1.raster.z, w2.raster.z)
    for w in e1:
        amp = w.boundaries[0][2]
        assert 0.2 <= amp <= 1.5 and w.boundaries[0][0] == 1
        assert np.all((w.manning >= 0.01) & (w.manning <= 0.04))
        n = int(round(np.sqrt(w.mesh.n)))
        assert n in (4, 6, 8) and w.raster.z.shape == (4 * n, 4 * n)
        assert w.raster.dx * 4 * n == 20000.0
    assert len({w.boundaries[0][2] for w in e1}) == len(e1)
