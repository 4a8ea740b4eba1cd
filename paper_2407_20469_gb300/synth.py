"""Seeded synthetic inputs shaped like the paper's 10x / 0.25 NA workload.

This module holds input recipes only (illumination layouts, random sample
transmissions, random aberration coefficients); it contains none of the
reconstruction's arithmetic and is the one module both the CUDA path's tests
and the float64 checker draw their inputs from.

Physical defaults (Sec. 3): 0.25 NA objective, 3.45 um camera pixels at 10x
magnification (0.345 um in the sample plane), green light. The wavelength of
the synthetic workloads is 0.52 um; the paper quotes 522-523 nm.

Sample recipe: amplitude in [0.8, 1.0] and phase in [0, pi], each a white
Gaussian field smoothed by a Gaussian of standard deviation ``sigma_px``
(upsampled-grid pixels) and min-max scaled into its range.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NA = np.float32(0.25)
WAVELENGTH_UM = np.float32(0.52)
PIXEL_UM = np.float32(0.345)
UPSAMPLE = 2
PHOTONS = 1.0e4            # photons per pixel at unit intensity


@dataclass(frozen=True)
class Illumination:
    """Transverse wave-vectors (cycles/um, float32) of the LEDs of one set-up."""

    kx: np.ndarray
    ky: np.ndarray
    n_bf: int

    @property
    def n_df(self) -> int:
        return len(self.kx) - self.n_bf


def ring(na_ill: float, count: int, offset_deg: float, wavelength_um=WAVELENGTH_UM):
    """``count`` LEDs evenly spaced on a ring of illumination NA ``na_ill``."""
    ang = np.deg2rad(offset_deg + 360.0 * np.arange(count) / count)
    r = float(na_ill) / float(wavelength_um)
    return r * np.cos(ang), r * np.sin(ang)


def illumination(n_bf: int = 8, df_rings=((0.30, 8, 0.0), (0.38, 8, 22.5)),
                 na=NA, wavelength_um=WAVELENGTH_UM) -> Illumination:
    """NA-matching ring (illumination NA = objective NA) plus darkfield rings.

    Default: 8 NA-matching LEDs at 45 degree steps and 16 darkfield LEDs on two
    rings (NA 0.30, and NA 0.38 turned by 22.5 degrees), inside the 0.27-0.40
    illumination-NA range of the 8 + 16 workload.
    """
    kx = [ring(na, n_bf, 0.0, wavelength_um)[0]]
    ky = [ring(na, n_bf, 0.0, wavelength_um)[1]]
    for na_ill, count, off in df_rings:
        x, y = ring(na_ill, count, off, wavelength_um)
        kx.append(x)
        ky.append(y)
    return Illumination(kx=np.concatenate(kx).astype(np.float32),
                        ky=np.concatenate(ky).astype(np.float32), n_bf=n_bf)


def illumination_8_24() -> Illumination:
    """8 NA-matching + 24 darkfield LEDs on rings at NA 0.29, 0.34 and 0.40."""
    return illumination(8, ((0.29, 8, 0.0), (0.34, 8, 22.5), (0.40, 8, 11.25)))


def illumination_12_22() -> Illumination:
    """The paper's set-up size (Sec. 3): 12 NA-matching LEDs and 22 darkfield LEDs up
    to illumination NA 0.44, here on rings at NA 0.31 (6), 0.375 (8) and 0.44 (8);
    the exact positions are not printed, so the rings are this recipe's choice."""
    return illumination(12, ((0.31, 6, 0.0), (0.375, 8, 22.5), (0.44, 8, 0.0)))


def _smooth_noise(rng: np.random.Generator, H: int, W: int, sigma_px: float) -> np.ndarray:
    z = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    g = np.exp(-2.0 * (math.pi * sigma_px) ** 2 * (fx * fx + fy * fy))
    return np.real(np.fft.ifft2(np.fft.fft2(z) * g))


def _scale(a: np.ndarray, lo: float, hi: float) -> np.ndarray:
    a = a - a.min()
    top = a.max()
    return lo + (hi - lo) * (a / top if top > 0 else a)


def sample_object(rng: np.random.Generator, H: int, W: int, sigma_px: float = 4.0,
                  amp=(0.8, 1.0), phase=(0.0, math.pi)) -> np.ndarray:
    """Complex transmission on the upsampled H x W grid (complex128)."""
    a = _scale(_smooth_noise(rng, H, W, sigma_px), *amp)
    p = _scale(_smooth_noise(rng, H, W, sigma_px), *phase)
    return a * np.exp(1j * p)


def zernike_coefficients(rng: np.random.Generator, scale: float = 1.0) -> np.ndarray:
    """15 Noll coefficients (rad): j = 4..15 uniform in [-scale, scale], j = 1..3 zero."""
    c = np.zeros(15)
    c[3:] = rng.uniform(-scale, scale, 12)
    return c


def quadratic_field(rng: np.random.Generator, scale: float = 1.0) -> np.ndarray:
    """Field-dependent aberrations: c_j(u, v) = sum of the 6 quadratic monomials.

    Returns a [6, 15] coefficient table for the monomials (1, u, v, u^2, uv,
    v^2) with u, v in [-1, 1]; every c_j stays within [-scale, scale].
    """
    t = rng.uniform(-1.0, 1.0, (6, 15))
    t[:, :3] = 0.0
    t *= scale / np.abs(t).sum(axis=0).clip(min=1.0)
    return t


def coefficients_at(table: np.ndarray, u: float, v: float) -> np.ndarray:
    """Evaluate a ``quadratic_field`` table at tile coordinates (u, v)."""
    mono = np.array([1.0, u, v, u * u, u * v, v * v])
    return mono @ table


def tile_grid_uv(rows: int, cols: int) -> np.ndarray:
    """Tile-centre coordinates in [-1, 1]^2 for a rows x cols grid, [rows*cols, 2] (u, v)."""
    v, u = np.meshgrid(np.linspace(-1, 1, rows), np.linspace(-1, 1, cols), indexing="ij")
    return np.stack([u.ravel(), v.ravel()], axis=1).astype(np.float32)


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea and Flood, 2014) on uint64 arrays."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_uniform(seed: int, shape, stream: int = 0) -> np.ndarray:
    """Uniform numbers in (0, 1), one per element, from a counter-based generator:
    element i is mix64(key + (i + 1) * golden) with key = mix64(seed, stream), so it
    depends on (seed, stream, i) only and uses integer arithmetic alone (the same
    bits on every platform)."""
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed & 0xFFFFFFFF) | ((stream & 0xFFFFFFFF) << 32)], dtype=np.uint64))[0]
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = _mix64(key + i * _GOLDEN)
    return (((z >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53).reshape(shape)


def poisson_counts(lam: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """Poisson(lam) photon counts by inversion of the Poisson distribution function
    at one counter-based uniform per element (``counter_uniform``). Each count
    depends only on its own uniform and mean, so inputs regenerated on another
    platform agree element by element (a count can differ only where its uniform
    falls within rounding of a distribution-function step)."""
    from scipy import stats
    lam = np.asarray(lam, dtype=np.float64)
    u = counter_uniform(seed, lam.shape, stream)
    out = np.zeros(lam.shape, dtype=np.float64)
    m = lam > 0
    out[m] = stats.poisson.ppf(u[m], lam[m])
    return out


def noisy_stack(I: np.ndarray, photons: float, seed: int, stream: int = 0) -> np.ndarray:
    """Shot-noise version of a noise-free intensity stack: poisson_counts(photons I) / photons."""
    return poisson_counts(np.asarray(I, np.float64) * photons, seed, stream) / photons
