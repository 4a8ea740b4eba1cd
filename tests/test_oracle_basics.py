"""Pins of the oracle's conventions, basis and geometry against independent facts.

Each test checks the float64 oracle against something other than itself:
a brute-force DFT, quadrature, closed-form values, exhaustive enumeration.
"""
import math

import numpy as np
import pytest

from oracle import grid, zernike
from paper_2407_20469_gb300 import synth


def brute_dft2(f):
    """O(N^4) DFT by its definition, sum_x f(x) exp(-2 pi i k.x / n)."""
    h, w = f.shape
    out = np.zeros((h, w), dtype=np.complex128)
    for ky in range(h):
        for kx in range(w):
            acc = 0j
            for y in range(h):
                for x in range(w):
                    acc += f[y, x] * complex(math.cos(-2 * math.pi * (ky * y / h + kx * x / w)),
                                             math.sin(-2 * math.pi * (ky * y / h + kx * x / w)))
            out[ky, kx] = acc
    return out


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (5, 5)])
def test_spectrum_matches_brute_force_dft(shape):
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = brute_dft2(f) / f.size
    assert np.max(np.abs(grid.spectrum(f) - ref)) < 1e-13


def test_series_roundtrip_parseval_and_plane_wave():
    rng = np.random.default_rng(4)
    f = rng.standard_normal((16, 12)) + 1j * rng.standard_normal((16, 12))
    F = grid.spectrum(f)
    assert np.max(np.abs(grid.synthesize(F) - f)) < 1e-12
    # Parseval for series coefficients: mean |f|^2 = sum |F|^2
    assert abs(np.mean(np.abs(f) ** 2) - np.sum(np.abs(F) ** 2)) < 1e-12
    # a unit plane wave exp(2 pi i (3 x / 12 - 2 y / 16)) has F(3, -2) = 1
    y, x = np.mgrid[0:16, 0:12]
    pw = np.exp(2j * np.pi * (3 * x / 12 - 2 * y / 16))
    P = grid.spectrum(pw)
    assert abs(P[(-2) % 16, 3] - 1) < 1e-13
    assert np.sum(np.abs(P)) - 1 < 1e-12


def test_signed_freqs_nyquist():
    assert grid.signed_freqs(8).tolist() == [0, 1, 2, 3, -4, -3, -2, -1]
    assert grid.signed_freqs(5).tolist() == [0, 1, 2, -2, -1]


# ----------------------------------------------------------------- Zernike

NOLL_TABLE = [(0, 0), (1, 1), (1, -1), (2, 0), (2, -2), (2, 2), (3, -1), (3, 1), (3, -3),
              (3, 3), (4, 0), (4, 2), (4, -2), (4, 4), (4, -4)]
# Noll (1976), Table 1: j -> (n, m); m < 0 marks the sin terms (odd j).


def test_noll_index_table():
    assert [zernike.noll_to_nm(j) for j in range(1, 16)] == NOLL_TABLE


def test_zernike_orthonormal_on_unit_disc():
    # Gauss-Legendre in r (weight r dr) x uniform theta: exact for these polynomials
    nr, nt = 24, 64
    xr, wr = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * (xr + 1)
    wr = 0.5 * wr * r
    th = 2 * np.pi * np.arange(nt) / nt
    R, T = np.meshgrid(r, th, indexing="ij")
    W = np.outer(wr, np.full(nt, 2 * np.pi / nt))
    Z = zernike.basis(R * np.cos(T), R * np.sin(T))
    G = np.einsum("ab,abi,abj->ij", W, Z, Z) / np.pi
    assert np.max(np.abs(G - np.eye(15))) < 1e-12


def test_zernike_closed_form_values():
    s3, s5, s6, s8, s10 = map(math.sqrt, (3, 5, 6, 8, 10))
    assert abs(zernike.zernike(4, 0.0, 0.0) + s3) < 1e-14          # sqrt3 (2 rho^2 - 1)
    assert abs(zernike.zernike(4, 1.0, 0.0) - s3) < 1e-14
    assert abs(zernike.zernike(11, 0.0, 0.0) - s5) < 1e-14         # sqrt5 (6r^4 - 6r^2 + 1)
    assert abs(zernike.zernike(11, 0.0, 1.0) - s5) < 1e-14
    c = math.sqrt(0.5)
    assert abs(zernike.zernike(5, c, c) - s6) < 1e-14              # sqrt6 r^2 sin 2t
    assert abs(zernike.zernike(6, 1.0, 0.0) - s6) < 1e-14          # sqrt6 r^2 cos 2t
    assert abs(zernike.zernike(8, 1.0, 0.0) - s8) < 1e-14          # sqrt8 (3r^3-2r) cos t
    assert abs(zernike.zernike(10, -1.0, 0.0) + s8) < 1e-14        # sqrt8 r^3 cos 3t
    assert abs(zernike.zernike(14, 0.0, 1.0) - s10) < 1e-14        # sqrt10 r^4 cos 4t
    x, y = 0.3, -0.4
    assert abs(zernike.zernike(13, x, y) - s10 * (4 * 0.25 - 3) * 0.25 * math.sin(2 * math.atan2(y, x))) < 1e-14


# ----------------------------------------------------------------- geometry

def geom(n, up=2):
    return grid.Geometry(n, n, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), up)


def test_pupil_point_count_near_area():
    for n in (64, 128, 256):
        g = geom(n)
        N = len(grid.pupil_points(g))
        # lattice points in a circle: |N - pi R^2| is bounded by a multiple of the perimeter
        assert abs(N - math.pi * g.Rx ** 2) < 2 * math.pi * g.Rx


def _edge_clean_exhaustive(g, kx, ky):
    k = grid.pupil_points(g) - np.array([kx, ky])          # the shifted pupil, all of it
    dot = k[:, 0] * kx * g.h * g.h + k[:, 1] * ky * g.w * g.w
    other = ~((k[:, 0] == 0) & (k[:, 1] == 0))
    return not np.any(other & (dot >= 0))


def test_edge_clean_matches_exhaustive_search():
    g = geom(64)
    for kx in range(-12, 13):
        for ky in range(-12, 13):
            if not g.in_pupil(kx, ky) or (kx == 0 and ky == 0):
                continue
            assert grid.kk_edge_clean(g, kx, ky) == _edge_clean_exhaustive(g, kx, ky), (kx, ky)


@pytest.mark.parametrize("n", [64, 128, 256, 512, 320, 375])
def test_snapped_na_matching_leds_are_admissible(n):
    g = geom(n)
    ill = synth.illumination()
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    for kx, ky in k[:ill.n_bf]:
        assert g.in_pupil(kx, ky)
        assert _edge_clean_exhaustive(g, kx, ky)
        # within 20% of the pupil radius of the ideal ring position, and on the ring
        assert abs(math.hypot(kx, ky) - g.Rx) < 0.02 * g.Rx + 1.0
    for (kx, ky), px, py in zip(k[ill.n_bf:], ill.kx[ill.n_bf:], ill.ky[ill.n_bf:]):
        assert abs(kx - float(px) * n * float(synth.PIXEL_UM)) <= 0.5
        assert abs(ky - float(py) * n * float(synth.PIXEL_UM)) <= 0.5


def test_minkowski_difference_matches_set_arithmetic():
    rng = np.random.default_rng(9)
    A = rng.integers(-5, 6, (17, 2))
    B = rng.integers(-5, 6, (11, 2))
    L = grid.minkowski_difference(A, B, 10)
    brute = {(a[0] - b[0], a[1] - b[1]) for a in A.tolist() for b in B.tolist()}
    ys, xs = np.nonzero(L)
    assert set(zip((xs - 10).tolist(), (ys - 10).tolist())) == brute


def test_darkfield_sets_partition_and_exclusions():
    g = geom(64)
    ill = synth.illumination()
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    known = set()
    for kb in k[:ill.n_bf]:
        known.update(map(tuple, grid.disc_points(g, kb).tolist()))
    for j in range(ill.n_bf, len(k)):
        D = grid.disc_points(g, k[j])
        s = grid.darkfield_sets(D, known, j, k[j])
        U = set(map(tuple, s.U.tolist()))
        P = set(map(tuple, s.P.tolist()))
        assert U | P == set(map(tuple, D.tolist())) and not (U & P)
        Q = set(map(tuple, s.Q.tolist()))
        up = {(a[0] - b[0], a[1] - b[1]) for a in U for b in P}
        pu = {(b[0] - a[0], b[1] - a[1]) for a in U for b in P}
        uu = {(a[0] - b[0], a[1] - b[1]) for a in U for b in U}
        assert Q == up - pu - uu


def _corr_brute(pts, vals):
    """(s * s)(k) = sum_q s(q) conj(s(q - k)), pair by pair: the image spectrum of Eq. 12."""
    out = {}
    for q, a in zip(pts, vals):
        for q2, b in zip(pts, vals):
            k = (q[0] - q2[0], q[1] - q2[1])
            out[k] = out.get(k, 0) + a * np.conj(b)
    return out


def test_eq13_holds_exactly_on_q_and_nowhere_else_in_u_minus_p():
    # sets where the mirrored cross term reaches lags of U - P that U * U does not
    U = [(0, 1), (-1, -2), (0, 3), (-1, 0), (1, 1), (-1, 2), (3, -1), (2, -1)]
    P = [(1, 0), (-1, 3)]
    rng = np.random.default_rng(12)
    u = rng.standard_normal(len(U)) + 1j * rng.standard_normal(len(U))
    p = rng.standard_normal(len(P)) + 1j * rng.standard_normal(len(P))
    full = _corr_brute(U + P, np.concatenate([u, p]))
    PP = _corr_brute(P, p)
    s = grid.darkfield_sets(np.array(U + P), set(P), 0, (0, 0))
    assert set(map(tuple, s.U.tolist())) == set(U)
    Q = set(map(tuple, s.Q.tolist()))
    up = {(a[0] - b[0], a[1] - b[1]) for a in U for b in P}
    assert Q <= up and len(up - Q) >= 3
    for k in up:
        cross = sum(u[i] * np.conj(p[m]) for i, a in enumerate(U) for m, b in enumerate(P)
                    if (a[0] - b[0], a[1] - b[1]) == k)
        exact = abs(full[k] - PP.get(k, 0) - cross) < 1e-12
        assert exact == (k in Q)          # F(I) - P*P = C U holds on Q, and only there


def test_darkfield_solvability_rules():
    # one unknown point between two known ones: U - P is symmetric, the mirrored term
    # covers all of it, no equation is left
    D = np.array([[0, 0], [1, 0], [-1, 0]])
    s = grid.darkfield_sets(D, {(1, 0), (-1, 0)}, 0, (0, 0))
    assert len(s.U) == 1 and len(s.Q) == 0 and not s.used
    # Sec. 4 bounds the unknown share of a darkfield disc by 42 %
    g = geom(64)
    k = (30, 0)
    D = grid.disc_points(g, k)
    order = np.argsort(D[:, 0], kind="stable")             # unknown = the cap of largest Kx
    for frac, ok in ((0.41, True), (0.43, False)):
        nu = int(round(frac * len(D)))
        s = grid.darkfield_sets(D, set(map(tuple, D[order[:len(D) - nu]].tolist())), 0, k)
        assert len(s.U) == nu and len(s.Q) >= nu
        assert s.used == ok


def test_darkfield_order_inside_out():
    k = np.array([[5, 0], [0, 3], [3, 0], [-3, 0], [0, -3]])
    order = grid.darkfield_order(k)
    # |k|=3 first, by angle from -pi: (0,-3) -pi/2, (3,0) 0, (0,3) pi/2, (-3,0) pi
    assert order.tolist() == [4, 2, 1, 3, 0]
