"""The synthetic inputs follow their stated recipe (the generators'
docstrings in workloads.py): the tidal
beach's depth profile, its |k|^-1 fractal noise of rms 1.5 m, eight channels
3-5 pixels wide and 3 m deeper across the beach, the boundary, friction and
tracer data, seeded and reproducible.  CPU only."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2505_18743_gb300 import workloads as W  # noqa: E402

N, PIX, L = 32, 16, 20000.0  # a 512^2 raster: the recipe does not depend on resolution


def _parts(seed):
    """The beach raster split into its profile, noise and channels, the noise
    regenerated from the same seeded stream the raster draws it from."""
    wl = W.tidal_beach(seed, n=N, pix=PIX, dtype=np.float64)
    npx = N * PIX
    dx = L / npx
    xc = (np.arange(npx) + 0.5) * dx
    base = np.where(xc < 0.75 * L, 30.0, 30.0 - 35.0 * (xc - 0.75 * L) / (0.25 * L))
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((npx, npx))
    noise = W.fractal_noise(np.random.default_rng(seed), npx, npx, 1.5)
    chan = wl.raster.z - base[None, :] - noise
    return wl, xc, white, noise, chan


def test_beach_profile_noise_and_channels():
    wl, xc, white, noise, chan = _parts(W.DEFAULT_SEED)
    assert wl.raster.z.shape == (N * PIX, N * PIX)
    # the noise: zero mean, rms 1.5 m, amplitude spectrum |k|^-1 times the white noise's
    assert abs(noise.mean()) < 1e-12 and abs(np.sqrt(np.mean(noise ** 2)) - 1.5) < 1e-12
    k = np.hypot(np.fft.fftfreq(N * PIX)[:, None], np.fft.rfftfreq(N * PIX)[None, :])
    ratio = np.abs(np.fft.rfft2(noise)) / np.maximum(np.abs(np.fft.rfft2(white)), 1e-300)
    sel = (k > 0) & (np.abs(np.fft.rfft2(white)) > 1e-6)
    kr = ratio[sel] * k[sel]
    assert np.allclose(kr, kr[0], rtol=1e-8)
    # channels: whole multiples of 3 m, none offshore of 15 km, between 3 and 40
    # deepened pixels in every column of the beach (8 channels, 3-5 px, may overlap)
    steps = chan / 3.0
    assert np.allclose(steps, np.round(steps), atol=1e-9)
    beach = xc >= 0.75 * L
    assert np.all(np.abs(chan[:, ~beach]) < 1e-9)
    per_col = (np.round(steps[:, beach]) > 0).sum(axis=0)
    assert per_col.min() >= 3 and per_col.max() <= 40


def test_beach_data_and_seeding():
    wl = W.tidal_beach(W.DEFAULT_SEED, n=N, pix=PIX)
    assert wl.raster.z.dtype == np.float32 and wl.degree == 3 and wl.mesh.n == N * N
    assert wl.boundaries == [(1, W.BC_TIDE, 1.0, 44712.0, 0.0)] and wl.cfl == 0.08
    assert np.all(wl.manning == 0.02)
    assert np.all(wl.zeta == 0.0) and np.all(wl.qx == 0.0) and np.all(wl.qy == 0.0)
    assert wl.c.min() == 0.0 and wl.c.max() == 1.0
    again = W.tidal_beach(W.DEFAULT_SEED, n=N, pix=PIX)
    assert np.array_equal(again.raster.z, wl.raster.z) and np.array_equal(again.c, wl.c)
    other = W.tidal_beach(W.DEFAULT_SEED + 1, n=N, pix=PIX)
    assert not np.array_equal(other.raster.z, wl.raster.z)
    # a crop holds the same pixels as the full raster's block
    crop = W.tidal_beach(W.DEFAULT_SEED, n=N, pix=PIX, window=(8, 4, 6, 5))
    assert crop.mesh.n == 30
    assert np.array_equal(crop.raster.z, wl.raster.z[4 * PIX:9 * PIX, 8 * PIX:14 * PIX])
