"""Pins of the oracle's reconstruction steps (Eq. 1-13) against facts that fix them.

* Forward model: Eq. 3 (re-centring leaves the intensity unchanged), a plane
  wave, Parseval.
* Kramers-Kronig: an exact closed-form construction where Eq. 5-6 must return
  the field to round-off, and consistency with the forward model on a
  weak-phase object.
* Aberration solve: exact recovery from forward-model spectra, including
  wrapped differences; the null space of D.
* Darkfield: exact recovery of the unknown spectrum given the true known part;
  the block-Toeplitz matrix against an FFT correlation and a loop.
* End to end: recovery of a known object and pupil on noise-free tiles.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import apic, forward, grid, zernike
from paper_2407_20469_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def geom(n, up=2):
    return grid.Geometry(n, n, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), up)


def leds(g, ill=None):
    ill = ill or synth.illumination()
    return grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g), ill.n_bf


def align(est, ref):
    """Remove the global phase of est relative to ref."""
    z = np.vdot(est, ref)
    return est * (z / abs(z)) if abs(z) > 0 else est


def rel_l2(est, ref):
    return np.linalg.norm(align(est, ref) - ref) / np.linalg.norm(ref)


# ----------------------------------------------------------- forward model

def test_forward_eq3_recentring_and_parseval():
    g = geom(32)
    rng = np.random.default_rng(1)
    obj = synth.sample_object(rng, g.H, g.W, 2.0)
    c = synth.zernike_coefficients(rng, 0.5)
    O = forward.object_spectrum(obj)
    k = np.array([5, -3])
    S = forward.camera_spectrum(O, g, k, c)
    I = forward.intensity(O, g, k, c)
    # Eq. 3: shifting the spectrum by +k_i multiplies the field by a phase ramp only
    Sp = np.roll(S, shift=(-k[1], -k[0]), axis=(0, 1))
    Ip = np.abs(grid.synthesize(Sp)) ** 2
    assert np.max(np.abs(I - Ip)) < 1e-12
    # Parseval: mean intensity equals the energy of the camera spectrum
    assert abs(I.mean() - np.sum(np.abs(S) ** 2)) < 1e-12


def test_forward_shot_noise_statistics():
    """Poisson(photons I) / photons: mean I and variance I / photons (uniform I = 1 under a plane wave)."""
    g = geom(64)
    k, _ = leds(g)
    obj = np.ones((g.H, g.W), dtype=np.complex128)
    I = forward.intensity_stack(obj, g, k[:8], np.zeros(15), photons=1e4, rng=np.random.default_rng(5))
    assert abs(I.mean() - 1.0) < 2e-4
    assert abs(I.var() / 1e-4 - 1.0) < 0.05


def test_forward_plane_wave_object():
    g = geom(32)
    y, x = np.mgrid[0:g.H, 0:g.W]
    obj = 0.7 * np.exp(2j * np.pi * (2 * x / g.W + 1 * y / g.H))     # O(2, 1) = 0.7
    c = np.zeros(15)
    for k, inside in (([0, 0], True), ([-2, -1], True), ([8, 0], False)):
        # the wave reaches the camera at k = (2, 1) + k_led; inside the pupil -> |O|^2
        kk = np.array(k)
        I = forward.intensity(forward.object_spectrum(obj), g, kk, c)
        assert bool(g.in_pupil(2 + kk[0], 1 + kk[1])) == inside
        expect = 0.49 if inside else 0.0
        assert np.max(np.abs(I - expect)) < 1e-12


# ----------------------------------------------------------- Kramers-Kronig

def _halfplane_field(n, k_led, rng, amp=0.3):
    """S = exp(IDFT(L)) with L supported strictly in k . k_i < 0 plus a real DC."""
    f = grid.signed_freqs(n)
    ky, kx = np.meshgrid(f, f, indexing="ij")
    dot = kx * k_led[0] + ky * k_led[1]
    band = (np.abs(kx) < n // 2 - 2) & (np.abs(ky) < n // 2 - 2) & (np.hypot(kx, ky) < n / 5)
    L = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * amp / n
    L = np.where((dot < 0) & band, L, 0)
    L[0, 0] = 0.4                                           # real DC: log|S| mean
    return np.exp(grid.synthesize(L))


@pytest.mark.parametrize("k_led", [(7, 0), (5, 5), (0, -6), (-4, 3)])
def test_kk_exact_on_halfplane_field(k_led):
    n = 32
    rng = np.random.default_rng(11)
    S = _halfplane_field(n, k_led, rng)
    I = np.abs(S) ** 2
    rec = apic.kk_field(I, k_led, geom(n))
    assert np.max(np.abs(rec - S)) / np.max(np.abs(S)) < 1e-12


def test_kk_catches_wrong_scaling_and_side():
    # the exact construction separates Eq. 5 as printed from plausible misreadings
    n, k_led = 32, (5, 5)
    S = _halfplane_field(n, k_led, np.random.default_rng(12))
    I = np.abs(S) ** 2
    L = np.log(I)
    f = grid.signed_freqs(n)
    ky, kx = np.meshgrid(f, f, indexing="ij")
    dot = kx * k_led[0] + ky * k_led[1]
    for mask_of_dot, scale in (((dot < 0) * 1.0 + (dot == 0) * 0.5, 0.5),   # 1/2 log I
                               ((dot > 0) * 1.0 + (dot == 0) * 0.5, 1.0)):  # wrong side
        wrong = np.exp(np.fft.ifft2(np.fft.fft2(scale * L) * mask_of_dot))
        assert np.max(np.abs(wrong - S)) > 1e-3


def test_kk_consistency_at_na_matching_weak_phase():
    """Eq. 7 on a weak-phase object: recovered spectra match the forward model."""
    g = geom(128)
    k, n_bf = leds(g)
    rng = np.random.default_rng(21)
    obj = synth.sample_object(rng, g.H, g.W, 4.0, phase=(0.0, 0.3))
    c = synth.zernike_coefficients(rng, 0.5)
    O = forward.object_spectrum(obj)
    g0 = np.angle(O[0, 0])
    for i in range(n_bf):
        I = forward.intensity(O, g, k[i], c)
        X = apic.kk_spectrum(I, k[i], g)
        K = grid.disc_points(g, k[i])
        phi = (apic.pupil_phase(g, c, K[:, 0] + k[i, 0], K[:, 1] + k[i, 1])
               - apic.pupil_phase(g, c, np.array([k[i, 0]]), np.array([k[i, 1]]))[0])
        truth = O[K[:, 1] % g.H, K[:, 0] % g.W] * np.exp(1j * (phi - g0))
        assert np.linalg.norm(apic.sample(X, K) - truth) / np.linalg.norm(truth) < 2e-3


# ----------------------------------------------------------- aberration solve

def test_difference_operator_annihilates_piston_and_tilt():
    g = geom(64)
    k, n_bf = leds(g)
    kb = k[:n_bf]
    for i in range(n_bf):
        for l in range(i + 1, n_bf):
            K = grid.overlap_points(g, kb[i], kb[l])
            if len(K) == 0:
                continue
            for j in (1, 2, 3):
                f = lambda kk: zernike.zernike(j, *g.pupil_coords(kk[:, 0], kk[:, 1]))
                row = f(K + kb[i]) - f(K + kb[l]) - f(kb[i][None]) + f(kb[l][None])
                assert np.max(np.abs(row)) < 1e-12


def _exact_spectra(g, k_bf, c, rng):
    obj = synth.sample_object(rng, g.H, g.W, 4.0)
    O = forward.object_spectrum(obj)
    X = []
    for kb in k_bf:
        K = grid.disc_points(g, kb)
        phi = apic.pupil_phase(g, c, K[:, 0] + kb[0], K[:, 1] + kb[1]) - apic.pupil_phase(
            g, c, np.array([kb[0]]), np.array([kb[1]]))[0]
        Xi = np.zeros((g.h, g.w), dtype=np.complex128)
        Xi[K[:, 1] % g.h, K[:, 0] % g.w] = O[K[:, 1] % g.H, K[:, 0] % g.W] * np.exp(1j * phi) * np.exp(-0.7j)
        X.append(Xi)
    return X


@pytest.mark.parametrize("n,scale,seeds", [(128, 0.3, range(3)), (256, 1.0, range(3))])
def test_aberration_solve_exact_on_forward_spectra(n, scale, seeds):
    g = geom(n)
    k, n_bf = leds(g)
    rows = apic.overlap_rows(g, k[:n_bf])
    for s in seeds:
        rng = np.random.default_rng(100 + s)
        c = synth.zernike_coefficients(rng, scale)
        X = _exact_spectra(g, k[:n_bf], c, rng)
        beta = apic.phase_differences(X, rows)
        if scale >= 1.0:
            assert np.mean(np.abs(rows.A @ c[3:]) > np.pi) > 0.2       # really wrapped
        est = apic.aberration_solve(beta, rows)
        assert np.max(np.abs(est - c)) < 1e-9


# ----------------------------------------------------------- darkfield

def test_darkfield_matrix_equals_fft_correlation_and_loops():
    g = geom(32)
    k, n_bf = leds(g)
    rng = np.random.default_rng(5)
    spec = apic.Spectrum(g)
    for kb in k[:n_bf]:
        K = grid.disc_points(g, kb)
        spec.put(K, rng.standard_normal(len(K)) + 1j * rng.standard_normal(len(K)))
    j = n_bf + 9
    D = grid.disc_points(g, k[j])
    sets = grid.darkfield_sets(D, spec.known_set(), j, k[j])
    assert sets.used
    I = rng.random((g.h, g.w))
    c = synth.zernike_coefficients(rng, 0.5)
    C, b, Pv = apic.darkfield_system(sets, I, spec, g, c)
    x = rng.standard_normal(len(sets.U)) + 1j * rng.standard_normal(len(sets.U))
    # loop form of the correlation sum_q U(q) conj P(q - k)
    Pd = {tuple(p): v for p, v in zip(sets.P.tolist(), Pv)}
    loop = np.array([sum(xq * np.conj(Pd.get((q[0] - kk[0], q[1] - kk[1]), 0))
                         for q, xq in zip(sets.U.tolist(), x)) for kk in sets.Q.tolist()])
    assert np.max(np.abs(C @ x - loop)) < 1e-12
    # FFT form: series coefficients of u(x) conj(p(x)) on a grid larger than the lags
    m = 64
    uf = np.zeros((m, m), complex)
    pf = np.zeros((m, m), complex)
    uf[sets.U[:, 1] % m, sets.U[:, 0] % m] = x
    pf[sets.P[:, 1] % m, sets.P[:, 0] % m] = Pv
    prod = grid.spectrum(grid.synthesize(uf) * np.conj(grid.synthesize(pf)))
    assert np.max(np.abs(C @ x - prod[sets.Q[:, 1] % m, sets.Q[:, 0] % m])) < 1e-11


def test_normal_equation_solver_matches_qr():
    rng = np.random.default_rng(6)
    C = rng.standard_normal((200, 40)) + 1j * rng.standard_normal((200, 40))
    b = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    ref = np.linalg.lstsq(C, b, rcond=None)[0]
    assert np.max(np.abs(apic.lstsq_normal(C, b) - ref)) < 1e-12


def test_darkfield_exact_with_true_known_spectrum():
    """Eq. 13 with the true P and pupil returns the true unknown spectrum."""
    g = geom(64)
    k, n_bf = leds(g)
    rng = np.random.default_rng(31)
    obj = synth.sample_object(rng, g.H, g.W, 2.0)
    c = synth.zernike_coefficients(rng, 0.5)
    O = forward.object_spectrum(obj)
    spec = apic.Spectrum(g)
    for kb in k[:n_bf]:
        K = grid.disc_points(g, kb)
        spec.put(K, O[K[:, 1] % g.H, K[:, 0] % g.W])
    I_df = np.stack([forward.intensity(O, g, kk, c) for kk in k[n_bf:]])
    log = apic.darkfield_extend(spec, I_df, g, k[n_bf:], c)
    used = [s for s in log if s.used]
    assert len(used) == len(k) - n_bf
    for s in used:
        got = spec.get(s.U)
        ref = O[s.U[:, 1] % g.H, s.U[:, 0] % g.W]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9


# ----------------------------------------------------------- end to end

def _truth(O, spec):
    t = np.where(spec.known, O, 0)
    return grid.synthesize(t)


@pytest.mark.parametrize("phase_hi,scale,tol", [(0.3, 0.5, 1e-2), (math.pi, 1.0, 5e-3)])
def test_end_to_end_recovers_field_and_pupil(phase_hi, scale, tol):
    g = geom(128)
    k, n_bf = leds(g)
    rng = np.random.default_rng(41)
    obj = synth.sample_object(rng, g.H, g.W, 4.0, phase=(0.0, phase_hi))
    c = synth.zernike_coefficients(rng, scale)
    I = forward.intensity_stack(obj, g, k, c)
    res = apic.reconstruct_tile(I, g, k, n_bf)
    O = forward.object_spectrum(obj)
    assert rel_l2(res.field, _truth(O, res.spectrum)) < tol
    # pupil phase RMS over the disc (orthonormal basis: RMS = |dc| for j >= 4)
    assert np.sqrt(np.sum((res.c15 - c) ** 2)) < 0.05
    assert np.all(res.c15[:3] == 0)
    # the pupil out is the forward model's transfer function of Eq. 1 (a flat object
    # spectrum seen under normal incidence: Circ exp(+j phi) on the camera grid)
    assert rel_l2(res.pupil, forward.camera_spectrum(np.ones((g.H, g.W)), g, (0, 0), c)) < 1e-2


def test_synthetic_aperture_resolution_matches_paper_formula():
    """Sec. 3.1: resolution lambda / (NA + NA_illum) from the final aperture."""
    with open(os.path.join(GOLDEN, "paper_resolution.json")) as f:
        paper = json.load(f)
    na, na_ill, lam = paper["na"], paper["na_illum"], paper["wavelength_um"]
    n = 128
    g = grid.Geometry(n, n, na, lam, 0.345, 3)
    ill = synth.illumination(12, ((0.36, 10, 0.0), (na_ill, 12, 15.0)), na=na, wavelength_um=lam)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    spec = apic.Spectrum(g)
    for kb in k[:ill.n_bf]:
        spec.put(grid.disc_points(g, kb), 1.0)
    for j in range(ill.n_bf, len(k)):
        spec.put(grid.disc_points(g, k[j]), 1.0)     # full discs: the synthetic aperture
    H, W = g.H, g.W
    iy, ix = np.nonzero(spec.known)
    kx = np.where(ix < W // 2, ix, ix - W) / (n * 0.345)
    ky = np.where(iy < H // 2, iy, iy - H) / (n * 0.345)
    kmax = np.max(np.hypot(kx, ky))                   # cycles/um
    res_um = 1.0 / kmax
    theory = lam / (na + na_ill)
    assert abs(res_um - theory) / theory < 0.02
    # the paper prints 761 nm for 522 nm / (0.44 + 0.25); the ratio itself is 756.5 nm
    assert abs(theory * 1000 - paper["printed_theory_nm"]) / paper["printed_theory_nm"] < 0.01


def test_background_contrast_closed_forms():
    """var / mean^2 of I = m (1 + a cos(2 pi k x / n)) over whole periods is a^2 / 2;
    a constant image has 0; the statistic is scale invariant and averages images."""
    from oracle import apic as oapic
    n = 32
    x = np.arange(n)
    a = 0.3
    I1 = 5.0 * (1.0 + a * np.cos(2 * np.pi * 3 * x / n))[None, :] * np.ones((n, 1))
    I2 = np.full((n, n), 2.0)
    assert abs(oapic.background_contrast2(I1[None]) - a * a / 2) < 1e-15
    assert oapic.background_contrast2(I2[None]) == 0.0
    assert abs(oapic.background_contrast2(np.stack([I1, I2])) - a * a / 4) < 1e-15
    assert abs(oapic.background_contrast2((7 * I1)[None]) - a * a / 2) < 1e-14
