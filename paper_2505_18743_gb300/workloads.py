"""Seeded synthetic workloads: meshes, bathymetry rasters and initial states.

This module only *generates inputs*.  It holds none of the method's
arithmetic (no quadrature, no sub-grid integral, no flux), so both the CUDA
path and the CPU oracle can take their inputs from it.  Every generator is
seeded with ``numpy.random.default_rng``.

Conventions (the C-ABI's):
  * cell K = [x0, x0+hx] x [y0, y0+hy]; ``x0y0``/``hxhy`` are ``[n, 2]`` float64;
  * ``nbr`` is ``[n, 4, 2]`` int32, faces W, E, S, N; slot 0 is the neighbour,
    or ``-1 - tag`` on a boundary face; slot 1 is the second fine neighbour of
    a 2:1 hanging face, else -1;
  * nodal DoFs sit on the (r+1) x (r+1) Gauss-Lobatto support points of each
    cell, index ``a + (r+1) b`` with x fastest;
  * the raster is row-major ``[ny, nx]``; its value is the bathymetry depth
    z_b (positive down), so the water depth is max(zeta + z_b, 0).

The synthetic coastal workloads stand in for the paper's Venice Lagoon
bathymetry (Sec. 5), which is not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 20250524

BC_WALL = 0
BC_TIDE = 1


@dataclass
class Mesh:
    x0y0: np.ndarray
    hxhy: np.ndarray
    nbr: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x0y0.shape[0])


@dataclass
class Raster:
    z: np.ndarray  # [ny, nx], float32 or float64, depth positive down
    xo: float
    yo: float
    dx: float
    dy: float


@dataclass
class Workload:
    name: str
    degree: int
    mesh: Mesh
    raster: Raster
    zeta: np.ndarray
    qx: np.ndarray
    qy: np.ndarray
    c: np.ndarray
    tableau: int = 0  # 0 RK32-IMEX, 1 SSP33, 2 RK44, 3 forward Euler
    cfl: float = 0.1
    eps_vel: float = 0.01
    h_lim: float = 0.01
    eps0: float = 1e-6
    g: float = 9.81
    subgrid_mode: int = 0  # 0 S, 1 P
    boundaries: list = field(default_factory=list)  # (tag, kind, amp, period, phase)
    manning: np.ndarray | None = None
    tracer_diffusivity: np.ndarray | None = None  # nu_c per cell (Eq. numdiff), None: none
    steps: int = 100

    def config(self, **over):
        d = dict(degree=self.degree, subgrid_mode=self.subgrid_mode, tableau=self.tableau,
                 g=self.g, eps_vel=self.eps_vel, h_lim=self.h_lim, eps0=self.eps0,
                 cfl=self.cfl, newton_max=20, newton_tol=1e-12)
        d.update(over)
        return d

    def state(self):
        return self.zeta, self.qx, self.qy, self.c


# ----------------------------------------------------------------------------
# DoF locations: the Gauss-Lobatto support points of the nodal basis (the
# input convention of set_state), from numpy's Legendre series.
# ----------------------------------------------------------------------------
def support_points(degree: int) -> np.ndarray:
    n = degree + 1
    if n == 2:
        return np.array([0.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots()
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (1.0 + x)


def nodal_coordinates(mesh: Mesh, degree: int):
    """Physical coordinates of every DoF, [n, (r+1)^2] arrays X, Y."""
    s = support_points(degree)
    a = np.tile(s, degree + 1)
    b = np.repeat(s, degree + 1)
    X = mesh.x0y0[:, 0:1] + mesh.hxhy[:, 0:1] * a[None, :]
    Y = mesh.x0y0[:, 1:2] + mesh.hxhy[:, 1:2] * b[None, :]
    return X, Y


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def uniform_mesh(nx: int, ny: int, Lx: float, Ly: float, x0: float = 0.0, y0: float = 0.0,
                 tags=(0, 0, 0, 0), periodic=(False, False)) -> Mesh:
    """nx x ny uniform cells, row-major (x fastest); boundary faces carry
    tags (W, E, S, N); periodic wraps replace them by neighbours."""
    hx, hy = Lx / nx, Ly / ny
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    i = i.ravel()
    j = j.ravel()
    n = nx * ny
    x0y0 = np.stack([x0 + i * hx, y0 + j * hy], axis=1).astype(np.float64)
    hxhy = np.tile(np.array([[hx, hy]]), (n, 1))
    nbr = np.full((n, 4, 2), -1, dtype=np.int32)
    k = i + nx * j

    def put(face, cond, other, tag, wrap):
        nb = np.where(cond, other, wrap if wrap is not None else -1 - tag)
        nbr[k, face, 0] = nb

    put(0, i > 0, k - 1, tags[0], (k + nx - 1) if periodic[0] else None)
    put(1, i < nx - 1, k + 1, tags[1], (k - nx + 1) if periodic[0] else None)
    put(2, j > 0, k - nx, tags[2], (k + nx * (ny - 1)) if periodic[1] else None)
    put(3, j < ny - 1, k + nx, tags[3], (k - nx * (ny - 1)) if periodic[1] else None)
    return Mesh(x0y0, hxhy, nbr)


def crop_mesh(nx_full: int, i0: int, j0: int, w: int, h: int, hx: float, hy: float,
              tags=(0, 0, 0, 0)) -> Mesh:
    """The w x h window (i0, j0) of an nx_full-wide uniform mesh, as a stand-alone
    uniform mesh (boundaries as given)."""
    return uniform_mesh(w, h, w * hx, h * hy, x0=i0 * hx, y0=j0 * hy, tags=tags)


def union_mesh(meshes):
    """Disjoint union of meshes (one ensemble member each): cells of mesh m
    follow those of meshes 0..m-1, neighbour indices are shifted by the same
    offset and boundary tags are kept.  Returns x0y0, hxhy, nbr and
    ``first`` [M + 1], member m owning cells first[m] .. first[m+1] - 1."""
    first = np.zeros(len(meshes) + 1, dtype=np.int64)
    nbrs = []
    for m, mesh in enumerate(meshes):
        first[m + 1] = first[m] + mesh.n
        nb = mesh.nbr.astype(np.int64)
        nbrs.append(np.where(nb >= 0, nb + first[m], nb).astype(np.int32))
    x0y0 = np.concatenate([m.x0y0 for m in meshes])
    hxhy = np.concatenate([m.hxhy for m in meshes])
    return x0y0, hxhy, np.concatenate(nbrs), first


# ----------------------------------------------------------------------------
# noise helpers
# ----------------------------------------------------------------------------
def fractal_noise(rng, ny: int, nx: int, rms: float) -> np.ndarray:
    """White noise filtered to amplitude |k|^-1 (power spectral slope -2),
    rescaled to the given rms."""
    w = rng.standard_normal((ny, nx))
    W = np.fft.rfft2(w)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    amp = np.zeros_like(k)
    amp[k > 0] = 1.0 / k[k > 0]
    f = np.fft.irfft2(W * amp, s=(ny, nx))
    f -= f.mean()
    return f * (rms / np.sqrt(np.mean(f * f)))


def smooth_field(rng, X, Y, L, modes=32, kmax=3):
    """Sum of low-wavenumber Fourier modes, min-max scaled to [0, 1]."""
    f = np.zeros_like(X)
    for _ in range(modes):
        kx, ky = rng.integers(0, kmax + 1, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.standard_normal()
        f += a * np.cos(2 * np.pi * (kx * X + ky * Y) / L + ph)
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


# ----------------------------------------------------------------------------
# configuration 1: degree 1, 16 x 16 cells, 1 km closed basin, 8 x 8 pixels/cell
# ----------------------------------------------------------------------------
def closed_basin(seed: int = DEFAULT_SEED, n: int = 16, pix: int = 8, degree: int = 1,
                 L: float = 1000.0) -> Workload:
    rng = np.random.default_rng(seed)
    npx = n * pix
    dx = L / npx
    xc = (np.arange(npx) + 0.5) * dx
    Xc, Yc = np.meshgrid(xc, xc)
    cx = cy = 0.5 * L
    z = 10.0 - 6.0 * np.exp(-((Xc - cx) ** 2 + (Yc - cy) ** 2) / 150.0 ** 2)
    for _ in range(20):
        x0, y0 = rng.uniform(0, L, size=2)
        w, h = rng.uniform(50, 300, size=2)
        sgn = rng.choice([-1.0, 1.0])
        m = (Xc >= x0) & (Xc < x0 + w) & (Yc >= y0) & (Yc < y0 + h)
        z[m] += 2.0 * sgn
    mesh = uniform_mesh(n, n, L, L)
    X, Y = nodal_coordinates(mesh, degree)
    zeta = 0.1 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / 100.0 ** 2)
    c = (((X - cx) ** 2 + (Y - cy) ** 2) < 200.0 ** 2).astype(np.float64)
    zero = np.zeros_like(zeta)
    return Workload("closed-basin-16x16-r1", degree, mesh, Raster(z.astype(np.float64), 0.0, 0.0,
                    dx, dx), zeta, zero.copy(), zero.copy(), c, tableau=1, cfl=0.1,
                    eps_vel=0.01, h_lim=0.01, steps=100)


# ----------------------------------------------------------------------------
# configuration 2: degree 3, 256 x 256 cells, 20 km tidal beach, 16 x 16 px/cell
# ----------------------------------------------------------------------------
def beach_raster(rng, npx: int, L: float, deep: float = 30.0, top: float = -5.0,
                 beach_start: float = 0.75, rms: float = 1.5, channels: int = 8):
    dx = L / npx
    xc = (np.arange(npx) + 0.5) * dx
    base = np.where(xc < beach_start * L, deep,
                    deep + (top - deep) * (xc - beach_start * L) / ((1 - beach_start) * L))
    z = np.repeat(base[None, :], npx, axis=0)
    z = z + fractal_noise(rng, npx, npx, rms)
    i_start = int(beach_start * npx)
    for _ in range(channels):
        yc = rng.uniform(0.1, 0.9) * npx
        width = rng.integers(3, 6)
        for i in range(i_start, npx):
            yc = min(max(yc + rng.normal(0.0, 1.0), 0.0), npx - 1.0)
            j0 = int(yc - width / 2)
            z[max(j0, 0):min(j0 + width, npx), i] += 3.0
    return z, dx


def tidal_beach(seed: int = DEFAULT_SEED, n: int = 256, pix: int = 16, degree: int = 3,
                L: float = 20000.0, dtype=np.float32, window=None) -> Workload:
    """The 20 km tidal beach.  ``window=(i0, j0, w, h)`` crops a w x h block of
    cells (and its pixels) out of the full n x n case; faces cut by the crop
    become walls except the west edge of the domain, which keeps the tide."""
    rng = np.random.default_rng(seed)
    z, dx = beach_raster(rng, n * pix, L)
    hcell = L / n
    if window is None:
        i0, j0, w, h = 0, 0, n, n
    else:
        i0, j0, w, h = window
    tags = (1 if i0 == 0 else 0, 0, 0, 0)
    mesh = uniform_mesh(w, h, w * hcell, h * hcell, x0=i0 * hcell, y0=j0 * hcell, tags=tags)
    zc = np.ascontiguousarray(z[j0 * pix:(j0 + h) * pix, i0 * pix:(i0 + w) * pix]).astype(dtype)
    X, Y = nodal_coordinates(mesh, degree)
    rng_c = np.random.default_rng(seed + 1)
    c = smooth_field(rng_c, X, Y, L)
    zero = np.zeros_like(X)
    man = np.full(mesh.n, 0.02)
    name = f"tidal-beach-{n}x{n}-r{degree}" if window is None else \
        f"tidal-beach-{n}x{n}-r{degree}-crop{w}x{h}@{i0},{j0}"
    return Workload(name, degree, mesh, Raster(zc, i0 * hcell, j0 * hcell, dx, dx),
                    zero.copy(), zero.copy(), zero.copy(), c, tableau=0, cfl=0.08,
                    eps_vel=0.1, h_lim=0.1, boundaries=[(1, BC_TIDE, 1.0, 44712.0, 0.0)],
                    manning=man, steps=1000)


def gauge_misfit_case(seed: int = DEFAULT_SEED, ngauges: int = 50, window=(128, 64, 128, 128),
                      pix: int = 16, dtype=np.float64):
    """The adjoint case: a 128 x 128-cell, r = 2 crop of the beach (16 x 16 px
    per cell, cells 128..255 x 64..191, the shoreline band included) flooded
    0.3 m with a 0.2 m hump offshore, ``ngauges`` seeded gauges in wet cells
    (offshore of x = 18.5 km, one per cell, at uniform offsets within the
    cell's middle 80 %), and a truth Manning field 0.02 (1 + 0.3 (2 s - 1))
    with s a smooth field in [0, 1] (a +-30 % perturbation).  The pixel depths
    are the beach's float32 values held as float64, so that a per-cell
    bathymetry offset moves them without rounding.
    Returns (workload, gauge xy [ngauges, 2], truth Manning [n])."""
    wl = tidal_beach(seed, window=window, degree=2, pix=pix, dtype=dtype)
    Xn, Yn = nodal_coordinates(wl.mesh, wl.degree)
    wl.zeta = 0.3 + 0.2 * np.exp(-((Xn - 16000.0) ** 2 + (Yn - 7000.0) ** 2) / 1500.0 ** 2)
    rng = np.random.default_rng(seed + 5)
    xc = wl.mesh.x0y0 + 0.5 * wl.mesh.hxhy
    wet = np.nonzero(xc[:, 0] < 18500.0)[0]
    cells = rng.choice(wet, ngauges, replace=False)
    xy = wl.mesh.x0y0[cells] + rng.uniform(0.1, 0.9, (ngauges, 2)) * wl.mesh.hxhy[cells]
    pert = smooth_field(np.random.default_rng(seed + 6), xc[:, 0], xc[:, 1], 20000.0)
    return wl, xy, wl.manning * (1.0 + 0.3 * (2.0 * pert - 1.0))


def beach_ensemble(seed: int = DEFAULT_SEED, members: int = 64, sizes=(32, 64, 128, 256),
                   pix: int = 8, degree: int = 2, L: float = 20000.0, dtype=np.float32):
    """Ensemble of independent tidal beaches (a parameter sweep): member m,
    seeded with seed + m, draws its mesh size N x N from ``sizes``, its tide
    amplitude from U[0.2, 1.5] m and its Manning coefficient from U[0.01,
    0.04], and builds the beach of ``tidal_beach`` on the same 20 km domain
    with ``pix`` x ``pix`` pixels per cell (so the rasters differ in
    resolution).  CFL number 0.12 for r = 2 (0.08 for r = 3)."""
    wls = []
    for m in range(members):
        rng = np.random.default_rng(seed + m)
        n = int(rng.choice(np.asarray(sizes)))
        amp = float(rng.uniform(0.2, 1.5))
        man = float(rng.uniform(0.01, 0.04))
        wl = tidal_beach(seed=seed + m, n=n, pix=pix, degree=degree, L=L, dtype=dtype)
        wl.name = f"beach-member{m}-{n}x{n}-r{degree}-p{pix}"
        wl.boundaries = [(1, BC_TIDE, amp, 44712.0, 0.0)]
        wl.manning = np.full(wl.mesh.n, man)
        wl.cfl = {1: 0.2, 2: 0.12, 3: 0.08}[degree]
        wls.append(wl)
    return wls


# ----------------------------------------------------------------------------
# paper test geometries
# ----------------------------------------------------------------------------
def lake_at_rest_bump(n: int = 20, pix: int = 4, degree: int = 1, submerged: bool = True) -> Workload:
    """The lake-at-rest basin of Sec. 4.1: 2 m x 1 m, free surface at 1 m
    (taken as the datum here, so zeta = 0 and z_b = 1 - bump height), mesh
    2n x n; the submerged bump has a jump on the block (0.9,1.1)x(0.3,0.7)."""
    L, H = 2.0, 1.0
    nxp, nyp = 2 * n * pix, n * pix
    dx = L / nxp
    xc = (np.arange(nxp) + 0.5) * dx
    yc = (np.arange(nyp) + 0.5) * dx
    X, Y = np.meshgrid(xc, yc)
    if submerged:
        z0 = 0.65
        inside = (X > 0.9) & (X < 1.1) & (Y > 0.3) & (Y < 0.7)
        psi = np.where(inside, np.sqrt((X - 0.9) ** 2 + (Y - 0.5) ** 2),
                       -5 * (X - 0.9) ** 2 - 50 * (Y - 0.5) ** 2)
    else:
        z0 = 1.3
        psi = -5 * (X - 0.9) ** 2 - 50 * (Y - 0.5) ** 2
    bump = z0 * np.exp(psi)  # bottom height above the basin floor
    z = 1.0 - bump           # depth below the still surface zeta = 0
    mesh = uniform_mesh(2 * n, n, L, H)
    nd = (degree + 1) ** 2
    zero = np.zeros((mesh.n, nd))
    return Workload(f"lake-at-rest-{'sub' if submerged else 'emerged'}-{2*n}x{n}-r{degree}", degree,
                    mesh, Raster(z, 0.0, 0.0, dx, dx), zero.copy(), zero.copy(), zero.copy(),
                    np.ones((mesh.n, nd)), tableau=0, cfl=0.9 * {1: 0.28, 2: 0.14, 3: 0.085}[degree],
                    eps_vel=1e-3, h_lim=1e-3, steps=200)


def flat_periodic(nx: int, ny: int, Lx: float, Ly: float, depth: float, degree: int, pix: int = 1,
                  periodic=(True, True)) -> tuple[Mesh, Raster]:
    mesh = uniform_mesh(nx, ny, Lx, Ly, periodic=periodic)
    dx = Lx / (nx * pix)
    dy = Ly / (ny * pix)
    z = np.full((ny * pix, nx * pix), depth)
    return mesh, Raster(z, 0.0, 0.0, dx, dy)


# ----------------------------------------------------------------------------
# 2:1-balanced quadtree forests (non-conforming meshes with hanging faces)
# ----------------------------------------------------------------------------
def forest_mesh(nx0: int, ny0: int, Lx: float, Ly: float, levels: int, refine,
                x0: float = 0.0, y0: float = 0.0, tags=(0, 0, 0, 0),
                periodic=(False, False)) -> tuple[Mesh, np.ndarray]:
    """Leaves of a forest of nx0 x ny0 quadtrees over [x0, x0+Lx] x [y0, y0+Ly],
    refined while ``refine(level, xc, yc, hx, hy)`` (vectorised over cells)
    says so, up to ``levels`` levels, then 2:1 balanced across faces.
    Returns the mesh (neighbour slots as in the module docstring) and the level
    of each leaf.  Leaves are sorted along a Morton curve."""
    leaves = {(0, i, j) for i in range(nx0) for j in range(ny0)}

    def geom(l, i, j):
        hx, hy = Lx / (nx0 << l), Ly / (ny0 << l)
        return x0 + i * hx, y0 + j * hy, hx, hy

    for lev in range(levels - 1):
        cur = [c for c in leaves if c[0] == lev]
        if not cur:
            break
        arr = np.array(cur)
        hx, hy = Lx / (nx0 << lev), Ly / (ny0 << lev)
        xc = x0 + (arr[:, 1] + 0.5) * hx
        yc = y0 + (arr[:, 2] + 0.5) * hy
        mask = np.asarray(refine(lev, xc, yc, hx, hy), dtype=bool)
        for (l, i, j), m in zip(cur, mask):
            if m:
                leaves.remove((l, i, j))
                leaves.update({(l + 1, 2 * i + a, 2 * j + b) for a in (0, 1) for b in (0, 1)})

    def covering(l, i, j):
        """the leaf covering cell (l, i, j) if it is this cell or an ancestor"""
        while l >= 0:
            if (l, i, j) in leaves:
                return (l, i, j)
            l, i, j = l - 1, i // 2, j // 2
        return None

    # 2:1 balance: a leaf whose face neighbour region is covered by a leaf two
    # or more levels coarser forces that coarse leaf to split
    changed = True
    while changed:
        changed = False
        for (l, i, j) in list(leaves):
            if (l, i, j) not in leaves:
                continue
            nxl, nyl = nx0 << l, ny0 << l
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if periodic[0]:
                    ii %= nxl
                if periodic[1]:
                    jj %= nyl
                if not (0 <= ii < nxl and 0 <= jj < nyl):
                    continue
                c = covering(l, ii, jj)
                if c is not None and c[0] < l - 1:
                    leaves.remove(c)
                    cl, ci, cj = c
                    leaves.update({(cl + 1, 2 * ci + a, 2 * cj + b) for a in (0, 1) for b in (0, 1)})
                    changed = True

    # Morton order on the finest grid of the leaf's lower-left corner
    L = max(c[0] for c in leaves)

    def morton(c):
        l, i, j = c
        x, y = i << (L - l), j << (L - l)
        key = 0
        for bit in range(24):
            key |= ((x >> bit) & 1) << (2 * bit) | ((y >> bit) & 1) << (2 * bit + 1)
        return key

    order = sorted(leaves, key=morton)
    index = {c: k for k, c in enumerate(order)}
    n = len(order)
    x0y0 = np.zeros((n, 2))
    hxhy = np.zeros((n, 2))
    nbr = np.full((n, 4, 2), -1, dtype=np.int32)
    level = np.zeros(n, dtype=np.int32)
    for k, (l, i, j) in enumerate(order):
        gx, gy, hx, hy = geom(l, i, j)
        x0y0[k] = (gx, gy)
        hxhy[k] = (hx, hy)
        level[k] = l
        nxl, nyl = nx0 << l, ny0 << l
        for f, (di, dj) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
            ii, jj = i + di, j + dj
            if periodic[0]:
                ii %= nxl
            if periodic[1]:
                jj %= nyl
            if not (0 <= ii < nxl and 0 <= jj < nyl):
                nbr[k, f, 0] = -1 - tags[f]
                continue
            if (l, ii, jj) in leaves:
                nbr[k, f, 0] = index[(l, ii, jj)]
            elif l > 0 and (l - 1, ii // 2, jj // 2) in leaves:
                nbr[k, f, 0] = index[(l - 1, ii // 2, jj // 2)]
            else:
                # two finer leaves along the face, by increasing tangential coordinate
                if di != 0:
                    a = 0 if di > 0 else 1
                    kids = [(l + 1, 2 * ii + a, 2 * jj + b) for b in (0, 1)]
                else:
                    b = 0 if dj > 0 else 1
                    kids = [(l + 1, 2 * ii + a, 2 * jj + b) for a in (0, 1)]
                nbr[k, f, 0] = index[kids[0]]  # ii, jj are already wrapped
                nbr[k, f, 1] = index[kids[1]]
    return Mesh(x0y0, hxhy, nbr), level


def fractal_curve(rng, n: int, amp: float, rough: float = 0.55) -> np.ndarray:
    """1D midpoint-displacement curve with n + 1 samples (n a power of two)"""
    y = np.zeros(n + 1)
    step, a = n, amp
    while step > 1:
        half = step // 2
        y[half::step] = 0.5 * (y[:-1:step] + y[step::step]) + rng.normal(0.0, a, size=len(y[half::step]))
        step, a = half, a * rough
    return y


# ----------------------------------------------------------------------------
# configuration 3: degree 2 on a 3-level 2:1 forest over a 50 km x 30 km lagoon
# ----------------------------------------------------------------------------
def lagoon(seed: int = DEFAULT_SEED, nx0: int = 256, ny0: int = 128, levels: int = 3,
           degree: int = 2, Lx: float = 50000.0, Ly: float = 30000.0, pix0: int = 32,
           band=(8000.0, 4200.0), window=None) -> Workload:
    """Barrier-island lagoon: open sea to the south (tide on the south
    boundary), a barrier along a seeded fractal coastline cut by two 15 m
    inlets, a 0.5-3 m lagoon with tidal flats at datum +-0.3 m to the north.
    Cells are refined toward the coastline (levels 1..3: 32, 16, 8 pixels per
    side) and 2:1 balanced.  ``window=(x0, y0, Lx, Ly, nx0, ny0)`` builds the
    same construction over a sub-rectangle (a small case for parity tests)."""
    rng = np.random.default_rng(seed)
    npx, npy = nx0 * pix0, ny0 * pix0
    dx, dy = Lx / npx, Ly / npy
    coast = 12000.0 + fractal_curve(rng, 1 << 12, 1500.0)
    xs = np.linspace(0.0, Lx, len(coast))
    xc = (np.arange(npx) + 0.5) * dx
    yc = (np.arange(npy) + 0.5) * dy
    cy = np.interp(xc, xs, coast)
    X, Y = np.meshgrid(xc, yc)
    d = Y - cy[None, :]                      # signed distance north of the coast (in y)
    sea = 3.0 + 12.0 * np.clip(-d / 8000.0, 0.0, 1.0)
    lag = 0.5 + 2.5 * (0.5 + 0.5 * np.sin(X / 2300.0 + 1.3) * np.cos(Y / 1700.0))
    flats = fractal_noise(rng, npy, npx, 1.0)
    lag = np.where(flats > 0.9, 0.3 * np.tanh(flats - 1.2), lag)   # tidal flats around datum
    z = np.where(d < -300.0, sea, np.where(d > 300.0, lag, -2.0))   # barrier 2 m above datum
    for xi in (0.3 * Lx, 0.68 * Lx):                                # two inlets, 15 m deep
        m = (np.abs(X - xi) < 250.0) & (np.abs(d) < 900.0)
        z[m] = 15.0 - 10.0 * np.abs(d[m]) / 900.0
    z = z.astype(np.float32)

    def refine(lev, xcc, ycc, hx, hy):
        yy = np.interp(xcc, xs, coast)
        return np.abs(ycc - yy) < band[lev] + 0.5 * hy

    if window is None:
        wx0, wy0, wLx, wLy, wnx, wny = 0.0, 0.0, Lx, Ly, nx0, ny0
    else:
        wx0, wy0, wLx, wLy, wnx, wny = window
    tags = (0, 0, 1 if wy0 == 0.0 else 0, 0)
    mesh, level = forest_mesh(wnx, wny, wLx, wLy, levels, refine, x0=wx0, y0=wy0, tags=tags)
    i0, j0 = int(round(wx0 / dx)), int(round(wy0 / dy))
    ni, nj = int(round(wLx / dx)), int(round(wLy / dy))
    zc = np.ascontiguousarray(z[j0:j0 + nj, i0:i0 + ni])
    Xn, Yn = nodal_coordinates(mesh, degree)
    rng_c = np.random.default_rng(seed + 2)
    c = smooth_field(rng_c, Xn, Yn, Lx)
    zero = np.zeros_like(Xn)
    name = f"lagoon-forest-{mesh.n}cells-r{degree}" + ("" if window is None else "-window")
    wl = Workload(name, degree, mesh, Raster(zc, wx0, wy0, dx, dy), zero.copy(), zero.copy(),
                  zero.copy(), c, tableau=0, cfl=0.8 * {1: 0.28, 2: 0.14, 3: 0.085}[degree],
                  eps_vel=0.1, h_lim=0.1, boundaries=[(1, BC_TIDE, 1.0, 44712.0, 0.0)],
                  manning=np.full(mesh.n, 0.02), steps=1000)
    wl.level = level
    return wl
