"""The APIC forward model, Eq. 1-2, in float64.

Test infrastructure only (see the package docstring).

Eq. 1: the camera-plane spectrum under LED i is the object spectrum shifted by
the illumination wave-vector, cut by the pupil and multiplied by the
aberration phase: S_i(k) = O(k - k_i) Circ_NA(k) exp(j phi(k)).
Eq. 2: the camera records I_i = |IDFT(S_i)|^2.

The object is a complex transmission sampled on the upsampled grid (pitch
dx/u); its Fourier-series coefficients O(K) share the frequency step of the
camera grid, so O(k - k_i) is read by index. Pinned by Eq. 3 (the intensity is
unchanged when the spectrum is re-centred), by a single plane wave (uniform
intensity |O(0)|^2) and by Parseval.
"""
from __future__ import annotations

import numpy as np

from . import grid, zernike


def object_spectrum(obj: np.ndarray) -> np.ndarray:
    """Fourier-series coefficients of the object on the upsampled grid."""
    return grid.spectrum(obj.astype(np.complex128))


def camera_spectrum(O_hat: np.ndarray, geom: grid.Geometry, k_led, c15) -> np.ndarray:
    """S_i(k) of Eq. 1 on the h x w camera grid (DFT index order)."""
    H, W = O_hat.shape
    S = np.zeros((geom.h, geom.w), dtype=np.complex128)
    k = grid.pupil_points(geom)                       # camera frequencies in the pupil
    K = k - np.asarray(k_led, dtype=np.int64)[None, :]  # object frequency k - k_i
    if np.any(np.abs(K[:, 0]) >= W // 2) or np.any(np.abs(K[:, 1]) >= H // 2):
        raise ValueError("illumination reaches beyond the object grid")
    px, py = geom.pupil_coords(k[:, 0], k[:, 1])
    phi = zernike.phase(c15, px, py)
    S[k[:, 1] % geom.h, k[:, 0] % geom.w] = O_hat[K[:, 1] % H, K[:, 0] % W] * np.exp(1j * phi)
    return S


def intensity(O_hat: np.ndarray, geom: grid.Geometry, k_led, c15) -> np.ndarray:
    """I_i(x) = |IDFT(S_i)|^2 of Eq. 2 (float64, h x w)."""
    s = grid.synthesize(camera_spectrum(O_hat, geom, k_led, c15))
    return (s.real ** 2 + s.imag ** 2)


def intensity_stack(obj: np.ndarray, geom: grid.Geometry, k_leds, c15,
                    photons: float | None = None, rng: np.random.Generator | None = None) -> np.ndarray:
    """All images of one tile, optionally with Poisson shot noise.

    ``photons`` is the photon count of unit intensity; the noisy image is
    Poisson(photons * I) / photons, drawn from ``rng``.
    """
    O_hat = object_spectrum(obj)
    out = np.stack([intensity(O_hat, geom, k, c15) for k in k_leds])
    if photons is not None:
        if rng is None:
            raise ValueError("noise needs a generator")
        out = rng.poisson(out * photons) / photons
    return out
