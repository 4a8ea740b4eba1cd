"""Per-tile APIC reconstruction in float64 (Sec. 2.3, Eq. 3-13).

Test infrastructure only (see the package docstring).

Steps, in the paper's order:

1. Kramers-Kronig field recovery from each NA-matching image (Eq. 4-6) and
   its spectrum (Eq. 7).
2. Phase differences on the overlap of every pair of recovered spectra
   (Eq. 8-9) and the least-squares aberration solve D phi = beta (Eq. 10), with
   phi in the Zernike basis of ``zernike``.
3. Aberration correction of each recovered spectrum and stitching of the
   corrected spectra (end of the brightfield part of Sec. 2.3).
4. Darkfield extension, one image at a time (Eq. 11-13): split the disc into
   known P and unknown U, form b = F(I) - P*P on the region Q, build the
   block-Toeplitz matrix C of the correlation P*U restricted to Q x U, solve
   C U = b in the least-squares sense and add the corrected U to the spectrum.
5. Inverse transform of the stitched spectrum on the upsampled grid.

Readings where the paper is silent or garbled are stated at each function.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import grid, zernike

SOLVED = list(range(zernike.FIRST_SOLVED, zernike.N_ZERNIKE + 1))   # Noll 4..15
# Value-refinement passes of the phase-difference solve; see ``aberration_solve``.
DEFAULT_PASSES = 2
LOG_FLOOR = 1e-6          # log(max(I, LOG_FLOOR * mean(I))) in Eq. 5


def wrap(a):
    """Wrap angles into (-pi, pi]."""
    return np.pi - np.mod(np.pi - np.asarray(a, dtype=np.float64), 2 * np.pi)


# ----------------------------------------------------------------------------
# 0. Background test (Sec. 3.2)
# ----------------------------------------------------------------------------

def background_contrast2(I_bf: np.ndarray) -> float:
    """Squared RMS contrast of a tile: the mean over its NA-matching images of
    var(I) / mean(I)^2 (population variance over the pixels).

    Sec. 3.2 skips patches without sample by a threshold on their variation;
    the statistic is read as this normalised variance, compared with the square
    of the contrast threshold (2 %).
    """
    I = np.asarray(I_bf, dtype=np.float64)
    out = 0.0
    for img in I:
        mu = img.mean()
        out += ((img - mu) ** 2).mean() / mu ** 2 if mu > 0 else 0.0
    return float(out / len(I))


# ----------------------------------------------------------------------------
# 1. Kramers-Kronig recovery (Eq. 4-7)
# ----------------------------------------------------------------------------

def kk_field(I: np.ndarray, k_led, geom: grid.Geometry) -> np.ndarray:
    """S'_i(x) exp(-j theta_i) from one NA-matching image, Eq. 5-6.

    Eq. 5 keeps F(log I) on the half-plane k . k_i < 0, halves it on the line
    k . k_i = 0 and zeroes the rest; Eq. 6 exponentiates the inverse transform.
    Readings: Eq. 4's "arg[S' - theta]" is read as arg[S'] - theta; F(log I) is
    used unscaled as printed (the one-sided spectrum then carries both the real
    and the imaginary part of the auxiliary function); the dot product is the
    physical one, k_x k_ix / w^2 + k_y k_iy / h^2, evaluated exactly on
    integers; the Nyquist bins take their signed value -n/2; log(0) is avoided
    with a floor of 1e-6 times the mean intensity.
    """
    h, w = I.shape
    L = np.log(np.maximum(I, LOG_FLOOR * I.mean()))
    G = np.fft.fft2(L)
    ky = grid.signed_freqs(h)[:, None]
    kx = grid.signed_freqs(w)[None, :]
    dot = kx * int(k_led[0]) * h * h + ky * int(k_led[1]) * w * w
    mask = np.where(dot < 0, 1.0, np.where(dot == 0, 0.5, 0.0))
    return np.exp(np.fft.ifft2(G * mask))


def kk_spectrum(I: np.ndarray, k_led, geom: grid.Geometry) -> np.ndarray:
    """Recovered spectrum S'_i(k) exp(-j theta_i) of Eq. 7 (series coefficients, DFT order)."""
    return grid.spectrum(kk_field(I, k_led, geom))


def sample(spec: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Values of a DFT-ordered spectrum at signed integer frequencies K [N, 2]."""
    h, w = spec.shape
    return spec[K[:, 1] % h, K[:, 0] % w]


# ----------------------------------------------------------------------------
# 2. Aberration solve (Eq. 8-10)
# ----------------------------------------------------------------------------

@dataclass
class OverlapRows:
    """Rows of the linear system D phi = beta of Eq. 10 in the Zernike basis."""

    pair: np.ndarray        # [rows, 2] image indices (i, l), i < l
    K: np.ndarray           # [rows, 2] object frequency in S_il
    A: np.ndarray           # [rows, 12] D applied to Z_4..Z_15
    nbr: np.ndarray         # [rows, 2] row index of K + (1, 0) and K + (0, 1) in the
                            # same overlap set, or -1


def overlap_rows(geom: grid.Geometry, k_bf: np.ndarray) -> OverlapRows:
    """Enumerate S_il (Eq. 8) for all pairs and evaluate the rows of D (Eq. 10).

    Row at K in S_il: Z(K + k_i) - Z(K + k_l) - Z(k_i) + Z(k_l) for each basis
    function Z (the printed subscript D0_ij is read as D0_il). Pairs are taken
    once (i < l); the reversed pair repeats the same equation with both sides
    negated.
    """
    pairs, Ks, As = [], [], []
    for i in range(len(k_bf)):
        for l in range(i + 1, len(k_bf)):
            K = grid.overlap_points(geom, k_bf[i], k_bf[l])
            if len(K) == 0:
                continue
            xi, yi = geom.pupil_coords(K[:, 0] + k_bf[i, 0], K[:, 1] + k_bf[i, 1])
            xl, yl = geom.pupil_coords(K[:, 0] + k_bf[l, 0], K[:, 1] + k_bf[l, 1])
            ci = zernike.basis(*geom.pupil_coords(k_bf[i, 0], k_bf[i, 1]), js=SOLVED)
            cl = zernike.basis(*geom.pupil_coords(k_bf[l, 0], k_bf[l, 1]), js=SOLVED)
            A = zernike.basis(xi, yi, js=SOLVED) - zernike.basis(xl, yl, js=SOLVED) - ci + cl
            pairs.append(np.tile([i, l], (len(K), 1)))
            Ks.append(K)
            As.append(A)
    pair = np.concatenate(pairs)
    K = np.concatenate(Ks)
    where = {(int(p0), int(p1), int(kx), int(ky)): r
             for r, (p0, p1, kx, ky) in enumerate(np.concatenate([pair, K], axis=1).tolist())}
    nbr = np.full((len(K), 2), -1, dtype=np.int64)
    for r, (p0, p1, kx, ky) in enumerate(np.concatenate([pair, K], axis=1).tolist()):
        nbr[r, 0] = where.get((p0, p1, kx + 1, ky), -1)
        nbr[r, 1] = where.get((p0, p1, kx, ky + 1), -1)
    return OverlapRows(pair=pair, K=K, A=np.concatenate(As), nbr=nbr)


def phase_differences(X: list, rows: OverlapRows) -> np.ndarray:
    """beta_Delta of Eq. 9-10: arg X_i(K) - arg X_l(K), wrapped into (-pi, pi]."""
    out = np.empty(len(rows.K))
    for i in range(len(X)):
        for l in range(i + 1, len(X)):
            m = (rows.pair[:, 0] == i) & (rows.pair[:, 1] == l)
            if not np.any(m):
                continue
            K = rows.K[m]
            out[m] = wrap(np.angle(sample(X[i], K)) - np.angle(sample(X[l], K)))
    return out


def _normal_solve(A: np.ndarray, y: np.ndarray) -> np.ndarray:
    """argmin ||A x - y|| through the normal equations and a Cholesky factor."""
    L = np.linalg.cholesky(A.T @ A)
    return np.linalg.solve(L.T, np.linalg.solve(L, A.T @ y))


def aberration_solve(beta: np.ndarray, rows: OverlapRows,
                     passes=DEFAULT_PASSES) -> np.ndarray:
    """Least-squares solution of Eq. 10 for the Noll coefficients 4..15.

    The paper solves D phi = beta_Delta by least squares (Eq. 10). Measured
    phase differences are known only modulo 2 pi and, for aberrations of a
    radian or more, most of them wrap; the paper does not say how this is
    handled. This reading resolves the wraps in two stages:

    1. Differences of neighbouring rows: for K and K + e (e a unit grid step)
       in the same overlap set, wrap(beta(K + e) - beta(K)) equals the true
       change whenever the phase difference moves by less than pi per grid
       step, so the least-squares fit of those changes by the matching
       differences of the rows of D gives a first estimate c0 with no
       unwrapping.
    2. ``passes`` refinements on the rows of Eq. 10 themselves:
       c <- c + argmin || D dc - wrap(beta - D c) ||. Once every residual is
       below pi, one pass gives exactly the least-squares solution of Eq. 10
       on the unwrapped differences; further passes leave it unchanged.

    Returns the 15-vector of Noll coefficients with j = 1..3 set to zero.
    """
    pairs = [(r, rows.nbr[r, a]) for a in (0, 1) for r in range(len(rows.K)) if rows.nbr[r, a] >= 0]
    r0 = np.array([p[0] for p in pairs], dtype=np.int64)
    r1 = np.array([p[1] for p in pairs], dtype=np.int64)
    c = _normal_solve(rows.A[r1] - rows.A[r0], wrap(beta[r1] - beta[r0]))
    for _ in range(passes):
        c = c + _normal_solve(rows.A, wrap(beta - rows.A @ c))
    out = np.zeros(zernike.N_ZERNIKE)
    out[zernike.FIRST_SOLVED - 1:] = c
    return out


def pupil_phase(geom: grid.Geometry, c15, kx, ky) -> np.ndarray:
    """phi at camera-plane integer frequencies (kx, ky)."""
    x, y = geom.pupil_coords(kx, ky)
    return zernike.phase(c15, x, y)


# ----------------------------------------------------------------------------
# 3. Correction and brightfield stitching
# ----------------------------------------------------------------------------

class Spectrum:
    """The object spectrum being assembled on the upsampled H x W grid."""

    def __init__(self, geom: grid.Geometry):
        self.geom = geom
        self.values = np.zeros((geom.H, geom.W), dtype=np.complex128)
        self.known = np.zeros((geom.H, geom.W), dtype=bool)

    def _idx(self, K):
        H, W = self.geom.H, self.geom.W
        if np.any(np.abs(K[:, 0]) >= W // 2) or np.any(np.abs(K[:, 1]) >= H // 2):
            raise ValueError("spectrum support exceeds the upsampled grid")
        return K[:, 1] % H, K[:, 0] % W

    def get(self, K):
        return self.values[self._idx(K)]

    def is_known(self, K):
        return self.known[self._idx(K)]

    def put(self, K, v):
        iy, ix = self._idx(K)
        self.values[iy, ix] = v
        self.known[iy, ix] = True

    def known_set(self) -> set:
        H, W = self.geom.H, self.geom.W
        iy, ix = np.nonzero(self.known)
        ky = np.where(iy < H // 2, iy, iy - H)
        kx = np.where(ix < W // 2, ix, ix - W)
        return set(zip(kx.tolist(), ky.tolist()))


def stitch_brightfield(X: list, geom: grid.Geometry, k_bf: np.ndarray, c15) -> Spectrum:
    """Correct each recovered spectrum and stitch them (Sec. 2.3, after Eq. 10).

    Eq. 7 gives X_i(K) = O(K) exp(j[phi(K + k_i) - phi(k_i)]) on the disc of
    image i, so the corrected spectrum is X_i(K) exp(-j[phi(K + k_i) - phi(k_i)]).
    The paper "assembles" the corrected spectra; this reading takes the
    arithmetic mean of all corrected spectra that cover K.
    """
    acc = np.zeros((geom.H, geom.W), dtype=np.complex128)
    cnt = np.zeros((geom.H, geom.W), dtype=np.int64)
    spec = Spectrum(geom)
    for i, k in enumerate(k_bf):
        K = grid.disc_points(geom, k)
        corr = (pupil_phase(geom, c15, K[:, 0] + k[0], K[:, 1] + k[1])
                - pupil_phase(geom, c15, np.array([k[0]]), np.array([k[1]]))[0])
        v = sample(X[i], K) * np.exp(-1j * corr)
        iy, ix = spec._idx(K)
        np.add.at(acc, (iy, ix), v)
        np.add.at(cnt, (iy, ix), 1)
    m = cnt > 0
    spec.values[m] = acc[m] / cnt[m]
    spec.known[m] = True
    return spec


# ----------------------------------------------------------------------------
# 4. Darkfield extension (Eq. 11-13)
# ----------------------------------------------------------------------------

def _lookup_grid(points: np.ndarray, values: np.ndarray, half: int):
    """Dense table of values at integer points on [-half, half]^2 (zero elsewhere)."""
    size = 2 * half + 1
    t = np.zeros((size, size), dtype=np.complex128)
    t[points[:, 1] + half, points[:, 0] + half] = values
    return t


def darkfield_system(sets: grid.DarkfieldSets, I: np.ndarray, spec: Spectrum,
                     geom: grid.Geometry, c15):
    """Matrix C, right-hand side b and known spectrum P of Eq. 13.

    P(K) = O_known(K) exp(j phi(K + k_j)) is the known part of the shifted
    camera spectrum (Eq. 11 with Eq. 1). With the reading
    (P*U)(k) = sum_q U(q) conj(P(q - k)), Eq. 13 on Q is C U = b with
    C[k, q] = conj(P(q - k)) (zero when q - k is not in P) and
    b(k) = F(I)(k) - (P*P)(k), F(I) the series coefficients of the image. This
    conjugate form equals the printed P*U by the Hermitian symmetry of F(I)
    (I is real), with Q mirrored.
    """
    kj = np.asarray(sets.k, dtype=np.int64)
    P, U, Q = sets.P, sets.U, sets.Q
    phiP = pupil_phase(geom, c15, P[:, 0] + kj[0], P[:, 1] + kj[1])
    Pv = spec.get(P) * np.exp(1j * phiP)
    half = int(np.abs(sets.D).max() + np.abs(Q).max()) + 2 if len(Q) else 2
    tab = _lookup_grid(P, Pv, half)
    # C[m, n] = conj(P(U_n - Q_m))
    dx = U[None, :, 0] - Q[:, None, 0]
    dy = U[None, :, 1] - Q[:, None, 1]
    C = np.conj(tab[dy + half, dx + half])
    # (P*P)(Q_m) = sum_p P(p) conj(P(p - Q_m))
    PP = np.empty(len(Q), dtype=np.complex128)
    chunk = max(1, 4_000_000 // max(1, len(P)))
    for s in range(0, len(Q), chunk):
        q = Q[s:s + chunk]
        ex = P[None, :, 0] - q[:, None, 0]
        ey = P[None, :, 1] - q[:, None, 1]
        PP[s:s + chunk] = np.conj(tab[ey + half, ex + half]) @ Pv
    Ihat = grid.spectrum(I)
    h, w = I.shape
    if np.any(np.abs(Q[:, 0]) >= w // 2) or np.any(np.abs(Q[:, 1]) >= h // 2):
        raise ValueError("darkfield lags exceed the camera grid")
    b = Ihat[Q[:, 1] % h, Q[:, 0] % w] - PP
    return C, b, Pv


def lstsq_normal(C: np.ndarray, b: np.ndarray) -> np.ndarray:
    """min ||C x - b|| through the normal equations and a Cholesky factor.

    If the Gram matrix is not numerically positive definite, a diagonal of
    1e-12 trace / N is added once (the paper states the system "can be
    solved" and gives no regularisation).
    """
    G = C.conj().T @ C
    r = C.conj().T @ b
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        G = G + np.eye(len(G)) * (1e-12 * np.trace(G).real / len(G))
        L = np.linalg.cholesky(G)
    y = np.linalg.solve(L, r)
    return np.linalg.solve(L.conj().T, y)


def darkfield_extend(spec: Spectrum, I_df: np.ndarray, geom: grid.Geometry,
                     k_df: np.ndarray, c15, solver=lstsq_normal) -> list:
    """Extend the spectrum with every darkfield image, inside-out (Eq. 11-13).

    The solved unknown spectrum is the camera-plane spectrum, so the object
    spectrum is U(q) exp(-j phi(q + k_j)). Returns the per-image index sets.
    """
    log = []
    for j in grid.darkfield_order(k_df):
        D = grid.disc_points(geom, k_df[j])
        sets = grid.darkfield_sets(D, spec.known_set(), int(j), k_df[j])
        log.append(sets)
        if not sets.used:
            continue
        C, b, _ = darkfield_system(sets, I_df[j], spec, geom, c15)
        x = solver(C, b)
        U = sets.U
        phiU = pupil_phase(geom, c15, U[:, 0] + k_df[j, 0], U[:, 1] + k_df[j, 1])
        spec.put(U, x * np.exp(-1j * phiU))
    return log


# ----------------------------------------------------------------------------
# 5. Whole tile
# ----------------------------------------------------------------------------

def pupil_function(geom: grid.Geometry, c15) -> np.ndarray:
    """Circ_NA(k) exp(j phi(k)) on the camera grid (DFT order), as in Eq. 1."""
    P = np.zeros((geom.h, geom.w), dtype=np.complex128)
    k = grid.pupil_points(geom)
    P[k[:, 1] % geom.h, k[:, 0] % geom.w] = np.exp(1j * pupil_phase(geom, c15, k[:, 0], k[:, 1]))
    return P


@dataclass
class TileResult:
    field: np.ndarray            # complex high-resolution field, H x W
    c15: np.ndarray              # Noll coefficients (rad), j = 1..3 zero
    pupil: np.ndarray            # Circ exp(j phi), h x w, DFT order
    spectrum: Spectrum
    df_sets: list = field(default_factory=list)


def reconstruct_tile(I: np.ndarray, geom: grid.Geometry, k_leds: np.ndarray, n_bf: int,
                     passes=DEFAULT_PASSES, c15_given=None,
                     solver=lstsq_normal, darkfield: bool = True) -> TileResult:
    """Full APIC reconstruction of one tile from its intensity stack.

    ``I`` is [n_img, h, w] (NA-matching images first), ``k_leds`` the snapped
    integer wave-vectors. ``c15_given`` bypasses the aberration solve.
    """
    k_bf = k_leds[:n_bf]
    k_df = k_leds[n_bf:]
    X = [kk_spectrum(I[i], k_bf[i], geom) for i in range(n_bf)]
    if c15_given is None:
        rows = overlap_rows(geom, k_bf)
        c15 = aberration_solve(phase_differences(X, rows), rows, passes)
    else:
        c15 = np.asarray(c15_given, dtype=np.float64)
    spec = stitch_brightfield(X, geom, k_bf, c15)
    log = []
    if darkfield and len(k_df):
        log = darkfield_extend(spec, I[n_bf:], geom, k_df, c15, solver)
    field_hr = grid.synthesize(spec.values)
    return TileResult(field=field_hr, c15=c15, pupil=pupil_function(geom, c15),
                      spectrum=spec, df_sets=log)
