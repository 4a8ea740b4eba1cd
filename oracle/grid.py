"""Grid conventions, pupil geometry and index sets for the APIC oracle.

Test infrastructure only (see the package docstring).

Conventions (readings of the paper, Sec. 2.2-2.3):

* A tile is h x w low-resolution camera pixels of pitch ``dx`` (sample plane).
  The frequency step is 1/(w dx) along x and 1/(h dx) along y, and the same
  step is kept on the upsampled u*h x u*w grid, so the object spectrum embeds
  into the high-resolution grid by index.
* Spectra are Fourier-series coefficients: S_hat = DFT(S) / (h w), and
  S = IDFT(S_hat) * (h w). A unit plane wave has S_hat(0) = 1.
* Integer frequencies are signed: index i of an n-point axis holds the
  frequency i for i < n/2 and i - n otherwise (the Nyquist bin is -n/2).
* The pupil (Circ_NA of Eq. 1) is the ellipse, in index units,
  (kx/Rx)^2 + (ky/Ry)^2 <= 1 + 1e-9 with Rx = NA w dx / lambda and
  Ry = NA h dx / lambda (a circle of radius R = NA n dx / lambda for square
  tiles).
* Illumination wave-vectors are snapped to the integer frequency grid (the tile
  is periodic, Eq. 3 needs an integer shift); see ``snap_leds``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PUPIL_TOL = 1e-9          # inclusion tolerance of the pupil boundary
UNKNOWN_FRACTION_MAX = 0.42  # largest unknown share of a darkfield disc (Sec. 4)


def signed_freqs(n: int) -> np.ndarray:
    """Signed integer frequency of each DFT index 0..n-1 (Nyquist -> -n/2)."""
    i = np.arange(n, dtype=np.int64)
    return np.where(i < (n + 1) // 2, i, i - n)


def spectrum(f: np.ndarray) -> np.ndarray:
    """Fourier-series coefficients of a sampled field: DFT(f) / (number of samples)."""
    return np.fft.fft2(f) / f.size


def synthesize(F: np.ndarray) -> np.ndarray:
    """Sampled field from its Fourier-series coefficients: IDFT(F) * size."""
    return np.fft.ifft2(F) * F.size


@dataclass
class Geometry:
    """Optical and sampling geometry of one tile-size class (Sec. 2.2, Sec. 3).

    ``na``, ``wavelength_um`` and ``pixel_um`` are taken as given (callers pass
    float32-representable values, the precision of the library's C interface).
    """

    h: int
    w: int
    na: float
    wavelength_um: float
    pixel_um: float
    upsample: int = 2

    @property
    def Rx(self) -> float:
        return (self.na * self.w * self.pixel_um) / self.wavelength_um

    @property
    def Ry(self) -> float:
        return (self.na * self.h * self.pixel_um) / self.wavelength_um

    @property
    def H(self) -> int:
        return self.upsample * self.h

    @property
    def W(self) -> int:
        return self.upsample * self.w

    def in_pupil(self, kx, ky):
        """Circ_NA of Eq. 1 on integer frequencies (array or scalar)."""
        kx = np.asarray(kx, dtype=np.float64)
        ky = np.asarray(ky, dtype=np.float64)
        Rx, Ry = self.Rx, self.Ry
        return (kx * kx) / (Rx * Rx) + (ky * ky) / (Ry * Ry) <= 1.0 + PUPIL_TOL

    def pupil_coords(self, kx, ky):
        """Unit-pupil coordinates (kx/Rx, ky/Ry) at which the aberration is evaluated."""
        return np.asarray(kx, np.float64) / self.Rx, np.asarray(ky, np.float64) / self.Ry


def kk_edge_clean(geom: Geometry, kx: int, ky: int) -> bool:
    """True if the pupil shifted by -k holds no grid point K != 0 with K . k >= 0.

    Eq. 5 assumes the shifted spectrum of an NA-matching image lies in the
    half-plane K . k_i < 0 with the DC term on the edge of its support (Sec. 2.3).
    On the integer grid that holds when every point of the shifted pupil other
    than K = 0 has a negative (physical) dot product with k_i. Such a point
    would satisfy ||K||^2 <= 1 + tol - ||k||^2 in the pupil-normalised norm, so
    only that small box is searched.
    """
    h, w = geom.h, geom.w
    Rx, Ry = geom.Rx, geom.Ry
    slack = 1.0 + PUPIL_TOL - ((kx * kx) / (Rx * Rx) + (ky * ky) / (Ry * Ry))
    if slack < 0:
        return False
    ax = int(math.floor(Rx * math.sqrt(slack))) + 1
    ay = int(math.floor(Ry * math.sqrt(slack))) + 1
    for qy in range(-ay, ay + 1):
        for qx in range(-ax, ax + 1):
            if qx == 0 and qy == 0:
                continue
            if qx * kx * h * h + qy * ky * w * w < 0:
                continue
            if geom.in_pupil(qx + kx, qy + ky):
                return False
    return True


def snap_leds(kx_phys, ky_phys, n_bf: int, geom: Geometry) -> np.ndarray:
    """Snap illumination wave-vectors (cycles/um) to integer grid frequencies.

    The first ``n_bf`` entries are NA-matching LEDs, the rest darkfield LEDs.
    An NA-matching LED goes to the grid point nearest its ideal position
    p = (kx w dx, ky h dx), among the points of the window
    |c - floor(p)| <= 2 + floor(0.2 max(Rx, Ry)) per axis that lie inside the
    pupil and keep the DC term on the edge of the shifted support
    (``kk_edge_clean``); ties go to the smaller ky, then the smaller kx. A
    darkfield LED goes to (floor(px + 0.5), floor(py + 0.5)).
    Returns int64 array [n, 2] of (kx, ky) in index units.
    """
    out = []
    win = 2 + int(math.floor(0.2 * max(geom.Rx, geom.Ry)))
    for idx, (kxp, kyp) in enumerate(zip(kx_phys, ky_phys)):
        px = float(kxp) * float(geom.w) * float(geom.pixel_um)
        py = float(kyp) * float(geom.h) * float(geom.pixel_um)
        if idx < n_bf:
            best = None
            fx, fy = math.floor(px), math.floor(py)
            for cy in range(fy - win, fy + win + 1):
                for cx in range(fx - win, fx + win + 1):
                    if not geom.in_pupil(cx, cy):
                        continue
                    d2 = (cx - px) * (cx - px) + (cy - py) * (cy - py)
                    key = (d2, cy, cx)
                    if best is not None and key >= best:
                        continue
                    if not kk_edge_clean(geom, cx, cy):
                        continue
                    best = key
            if best is None:
                raise ValueError(f"NA-matching LED {idx} has no admissible grid point")
            out.append((best[2], best[1]))
        else:
            out.append((math.floor(px + 0.5), math.floor(py + 0.5)))
    return np.asarray(out, dtype=np.int64)


def grid_points(h: int, w: int):
    """All signed integer frequencies of an h x w grid as flat (kx, ky) arrays."""
    ky, kx = np.meshgrid(signed_freqs(h), signed_freqs(w), indexing="ij")
    return kx.ravel(), ky.ravel()


def pupil_points(geom: Geometry) -> np.ndarray:
    """Camera-plane frequencies k with Circ_NA(k) != 0, int64 [N, 2] (kx, ky).

    Ordered by ky ascending, then kx ascending.
    """
    ax = int(math.ceil(geom.Rx)) + 1
    ay = int(math.ceil(geom.Ry)) + 1
    ky, kx = np.meshgrid(np.arange(-ay, ay + 1), np.arange(-ax, ax + 1), indexing="ij")
    kx, ky = kx.ravel(), ky.ravel()
    m = geom.in_pupil(kx, ky)
    return np.stack([kx[m], ky[m]], axis=1).astype(np.int64)


def disc_points(geom: Geometry, k_led) -> np.ndarray:
    """Object frequencies K with Circ_NA(K + k_i) != 0 (the support in Eq. 7).

    int64 [N, 2] (Kx, Ky); K = k - k_i for the pupil points k, in their order.
    """
    return pupil_points(geom) - np.asarray(k_led, dtype=np.int64)[None, :]


def overlap_points(geom: Geometry, k_i, k_l) -> np.ndarray:
    """The overlap set S_il of Eq. 8 as int64 [N, 2] object frequencies."""
    D = disc_points(geom, k_i)
    m = geom.in_pupil(D[:, 0] + k_l[0], D[:, 1] + k_l[1])
    return D[m]


def darkfield_order(k_df: np.ndarray) -> np.ndarray:
    """Processing order of darkfield images: increasing |k_j|, then angle.

    The paper extends the spectrum "across all darkfield measurements" without
    an order (Sec. 2.3); this reading takes them from the inside out.
    """
    r2 = k_df[:, 0] ** 2 + k_df[:, 1] ** 2
    ang = np.arctan2(k_df[:, 1].astype(np.float64), k_df[:, 0].astype(np.float64))
    return np.lexsort((np.arange(len(k_df)), ang, r2))


def minkowski_difference(A: np.ndarray, B: np.ndarray, half: int) -> np.ndarray:
    """Indicator of {a - b : a in A, b in B} on the lag grid [-half, half]^2.

    Returns a boolean array L with L[y + half, x + half] True iff (x, y) = a - b
    for some a in A, b in B. ``half`` must bound every |coordinate| of a - b.
    """
    size = 2 * half + 1
    out = np.zeros((size, size), dtype=bool)
    if len(A) == 0 or len(B) == 0:
        return out
    if len(A) < len(B):       # loop over the shorter list
        for a in A:
            d = a - B
            out[d[:, 1] + half, d[:, 0] + half] = True
    else:
        for b in B:
            d = A - b
            out[d[:, 1] + half, d[:, 0] + half] = True
    return out


@dataclass
class DarkfieldSets:
    """Index sets of one darkfield image (Eq. 11-13), object-frequency coordinates."""

    j: int                      # index of the LED in the darkfield list
    k: tuple                    # snapped wave-vector
    D: np.ndarray               # disc points, [.., 2]
    U: np.ndarray               # unknown points (D minus known), N = len(U)
    P: np.ndarray               # known points (D and known)
    Q: np.ndarray               # equation lags, M = len(Q), sorted (ky, kx)
    used: bool                  # False when the image is skipped (see below)


def darkfield_sets(D: np.ndarray, known: set, j: int, k) -> DarkfieldSets:
    """Split a darkfield disc into unknown U / known P and find the lag region Q.

    Eq. 12: F(I) = U*U + U*P + P*U + P*P (correlations). With the reading
    UP(k) = sum_q U(q) conj(P(q - k)), the U*P term is supported on U - P, the
    mirrored cross term on P - U and the unknown autocorrelation on U - U; Q is
    the part of U - P that neither other term reaches, so Eq. 13 holds there
    exactly. The image is used only when M >= N and N <= 0.42 |D| (Sec. 4);
    otherwise it is skipped and its unknown points stay unknown.
    """
    isknown = np.array([tuple(p) in known for p in D.tolist()], dtype=bool)
    U = D[~isknown]
    P = D[isknown]
    half = int(2 * np.abs(D).max()) + 1 if len(D) else 1
    up = minkowski_difference(U, P, half)
    pu = minkowski_difference(P, U, half)
    uu = minkowski_difference(U, U, half)
    qy, qx = np.nonzero(up & ~pu & ~uu)          # row-major: ky ascending, then kx
    Q = np.stack([qx - half, qy - half], axis=1).astype(np.int64)
    used = len(U) > 0 and len(Q) >= len(U) and len(U) <= UNKNOWN_FRACTION_MAX * len(D)
    return DarkfieldSets(j=j, k=tuple(int(v) for v in k), D=D, U=U, P=P, Q=Q, used=used)
