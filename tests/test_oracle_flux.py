"""Pins of the oracle's face flux: hydrostatic reconstruction (Eqs. hydro_rec,
hydro_rec_vars), Rusanov parameter (Eq. lxf_parameter), desingularised velocity
(Eq. velocity), consistency with the physical flux and the non-conservative
pressure term (Eq. pressure_tumolo)."""
import numpy as np

from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W

G = 9.81


def make(eps=1e-3):
    mesh = W.uniform_mesh(1, 1, 1.0, 1.0)
    ras = W.Raster(np.zeros((2, 2)), 0.0, 0.0, 0.5, 0.5)
    return Oracle(mesh, ras, degree=1, subgrid_mode=1, eps_vel=eps)


def rand_side(rng, wet=True):
    zb = rng.uniform(0.5, 3.0)
    z = rng.uniform(-0.5, 0.5) if wet else -zb - rng.uniform(0.0, 1.0)
    return z, rng.normal(0, 1), rng.normal(0, 1), rng.uniform(0, 1), zb


def test_reconstruction_identities():
    o = make()
    rng = np.random.default_rng(7)
    for _ in range(200):
        m = rand_side(rng, rng.uniform() < 0.8)
        p = rand_side(rng, rng.uniform() < 0.8)
        n = [(1, 0), (-1, 0), (0, 1), (0, -1)][rng.integers(4)]
        f = o.face_flux_p(*m, *p, *n)
        zs = min(m[4], p[4])  # z_b* = min(z_b-, z_b+)
        assert f["hsm"] == max(m[0] + zs, 0.0)
        assert f["hsp"] == max(p[0] + zs, 0.0)
        assert f["hsm"] <= max(m[0] + m[4], 0.0) and f["hsp"] <= max(p[0] + p[4], 0.0)


def test_lake_at_rest_faces_carry_no_flux():
    """Proposition 3.1 at a face: equal elevations (wet-wet), dry-dry at the
    Def. 3.1 level, and wet-dry with the wet level below the dry bank."""
    o = make()
    cases = [
        ((0.2, 0, 0, 1, 3.0), (0.2, 0, 0, 1, 0.4)),    # wet-wet, discontinuous bed
        ((-1.0, 0, 0, 1, 1.0), (-2.0, 0, 0, 1, 2.0)),  # dry-dry at -max z_b
        ((0.0, 0, 0, 1, 2.0), (1.0, 0, 0, 1, -1.0)),   # wet-dry, bank 1 m above datum
    ]
    for m, p in cases:
        for n in [(1, 0), (0, -1)]:
            f = o.face_flux_p(*m, *p, *n)
            assert f["F"] == 0.0 and f["Gx"] == 0.0 and f["Gy"] == 0.0 and f["R"] == 0.0


def test_consistency_with_physical_flux():
    """Identical states and bed on both sides: the Rusanov flux reduces to the
    physical flux and lambda to |u.n| + sqrt(g h)."""
    o = make()
    rng = np.random.default_rng(8)
    for _ in range(50):
        z, qx, qy, c, zb = rand_side(rng)
        h = z + zb
        n = np.array([(1, 0), (-1, 0), (0, 1), (0, -1)][rng.integers(4)], dtype=float)
        f = o.face_flux_p(z, qx, qy, c, zb, z, qx, qy, c, zb, *n)
        u = np.array([qx, qy]) / h  # h > eps: desingularisation inactive
        q = np.array([qx, qy])
        assert abs(f["F"] - q @ n) < 1e-13
        assert abs(f["Gx"] - qx * (u @ n)) < 1e-13 and abs(f["Gy"] - qy * (u @ n)) < 1e-13
        assert abs(f["R"] - c * (q @ n)) < 1e-13
        assert abs(f["lam"] - (abs(u @ n) + np.sqrt(G * h))) < 1e-13


def test_conservative_antisymmetry_and_pressure_term():
    """F and R are antisymmetric under exchange of the sides; the momentum flux
    is antisymmetric up to the non-conservative term g {{h*}} {{phi}} [[zeta*]],
    which both sides receive with the same sign (Eq. pressure_tumolo)."""
    o = make()
    rng = np.random.default_rng(9)
    for _ in range(100):
        m = rand_side(rng, rng.uniform() < 0.8)
        p = rand_side(rng, rng.uniform() < 0.8)
        n = np.array([(1, 0), (0, 1)][rng.integers(2)], dtype=float)
        a = o.face_flux_p(*m, *p, *n)
        b = o.face_flux_p(*p, *m, *(-n))
        assert a["F"] == -b["F"] and a["R"] == -b["R"] and a["lam"] == b["lam"]
        pres = G * 0.25 * (a["hsm"] + a["hsp"]) * (a["hsm"] - a["hsp"])
        assert abs(a["Gx"] + b["Gx"] + 2 * pres * n[0]) < 1e-12
        assert abs(a["Gy"] + b["Gy"] + 2 * pres * n[1]) < 1e-12


def test_desingularised_velocity_limits():
    """Eq. velocity: u = sqrt(2) h q / sqrt(max(h^4, eps^4) + h^4) is q/h for
    h >= eps and vanishes with h; the fluxes use q* = h* u (Eq. hydro_rec_vars)."""
    eps = 0.05
    o = make(eps)
    for h in (1e-9, 1e-4, 0.01, 0.05, 0.2):
        z, zb = h - 1.0, 1.0
        f = o.face_flux_p(z, 0.3, 0.0, 1.0, zb, z, 0.3, 0.0, 1.0, zb, 1.0, 0.0)
        ux = np.sqrt(2) * h * 0.3 / np.sqrt(max(h ** 4, eps ** 4) + h ** 4)
        # reconstructed discharge q* = h* u with h* = h on a continuous bed
        assert abs(f["F"] - h * ux) < 1e-15 * max(1, abs(h * ux))
        assert abs(f["Gx"] - h * ux * ux) < 1e-15 * max(1, abs(h * ux * ux))
        if h >= eps:
            assert abs(ux - 0.3 / h) < 1e-12 * (0.3 / h)
