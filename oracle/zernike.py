"""Noll-ordered, RMS-normalised Zernike polynomials: the aberration basis.

Test infrastructure only (see the package docstring).

The paper models the pupil phase phi of Eq. 1 and solves Eq. 10 for it in
terms of "aberration functions" (Sec. 2.3) without naming a basis; its pupil
figures (Fig. 4b, 5b) are Zernike-type maps. This oracle's reading: phi is a
sum of Noll-ordered Zernike polynomials, normalised to unit RMS over the unit
disc, evaluated at unit-pupil coordinates (kx/Rx, ky/Ry). Radial orders 2-4
(Noll j = 4..15) are solved; piston and tilts (j = 1..3) lie in the null space
of the difference operator D of Eq. 10 and are reported as zero.

Written from the general definition (radial polynomial as a finite factorial
sum, times cos or sin of m*theta) rather than from expanded Cartesian forms.
Pinned by orthonormality over the unit disc and by closed-form values.
"""
from __future__ import annotations

from math import factorial, sqrt

import numpy as np

N_ZERNIKE = 15          # Noll j = 1..15 (radial orders 0..4)
FIRST_SOLVED = 4        # j = 4..15 are estimated


def noll_to_nm(j: int) -> tuple[int, int]:
    """Noll index j >= 1 -> (radial order n, signed azimuthal frequency m).

    m > 0 denotes a cos(m theta) term (even j), m < 0 a sin(|m| theta) term
    (odd j); |m| rises through the order as 0, 2, 2, 4, 4, ... (n even) or
    1, 1, 3, 3, ... (n odd).
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    p = j - n * (n + 1) // 2 - 1
    if n % 2 == 0:
        am = 2 * ((p + 1) // 2)
    else:
        am = 2 * (p // 2) + 1
    if am == 0:
        return n, 0
    return n, (am if j % 2 == 0 else -am)


def radial(n: int, am: int, rho: np.ndarray) -> np.ndarray:
    """Zernike radial polynomial R_n^{|m|}(rho) by its finite-sum definition."""
    out = np.zeros_like(rho, dtype=np.float64)
    for s in range((n - am) // 2 + 1):
        coef = ((-1) ** s * factorial(n - s)
                / (factorial(s) * factorial((n + am) // 2 - s) * factorial((n - am) // 2 - s)))
        out = out + coef * rho ** (n - 2 * s)
    return out


def zernike(j: int, x, y) -> np.ndarray:
    """Z_j at unit-pupil Cartesian coordinates (x, y), RMS-normalised over the disc."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, m = noll_to_nm(j)
    rho = np.hypot(x, y)
    theta = np.arctan2(y, x)
    if m == 0:
        return sqrt(n + 1) * radial(n, 0, rho)
    norm = sqrt(2 * (n + 1))
    if m > 0:
        return norm * radial(n, m, rho) * np.cos(m * theta)
    return norm * radial(n, -m, rho) * np.sin(-m * theta)


def basis(x, y, js=range(1, N_ZERNIKE + 1)) -> np.ndarray:
    """Stack of Z_j(x, y) for the given Noll indices along a new last axis."""
    return np.stack([zernike(j, x, y) for j in js], axis=-1)


def phase(c15, x, y) -> np.ndarray:
    """phi(x, y) = sum_j c_j Z_j(x, y) for a 15-vector of Noll coefficients (rad)."""
    c15 = np.asarray(c15, dtype=np.float64)
    return basis(x, y) @ c15
