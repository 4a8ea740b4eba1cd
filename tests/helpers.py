"""Shared helpers of the test suite: seeded tiles, oracle runs, comparisons.

Inputs come from the seeded recipes in paper_2407_20469_gb300.synth and the
float64 forward model of the checker; expected values come only from the
checker (oracle/).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import apic as oapic
from oracle import forward, grid
from paper_2407_20469_gb300 import synth


def geometry(n, up=2):
    return grid.Geometry(n, n, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), up)


def make_tiles(n, count, seed, ill=None, phase_hi=math.pi, scale=1.0, photons=None, sigma=4.0):
    """(intensity float32 [count, n_img, n, n], zernike [count, 15], objects) from the oracle."""
    ill = ill or synth.illumination()
    g = geometry(n)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    rng = np.random.default_rng(seed)
    Is, cs, objs = [], [], []
    for _ in range(count):
        obj = synth.sample_object(rng, g.H, g.W, sigma, phase=(0.0, phase_hi))
        c = synth.zernike_coefficients(rng, scale)
        I = forward.intensity_stack(obj, g, k, c, photons=photons, rng=rng if photons else None)
        Is.append(I.astype(np.float32))
        cs.append(c)
        objs.append(obj)
    return np.stack(Is), np.stack(cs), objs


def oracle_tile(I32, n, ill=None, **kw):
    """Checker reconstruction of one tile from the float32 stack the GPU also sees."""
    ill = ill or synth.illumination()
    g = geometry(n)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    return oapic.reconstruct_tile(I32.astype(np.float64), g, k, ill.n_bf, **kw)


def align(est, ref):
    z = np.vdot(est, ref)
    return est * (z / abs(z)) if abs(z) > 0 else est


def rel_l2(est, ref):
    """Relative L2 error after removing the global phase of est."""
    return float(np.linalg.norm(align(est, ref) - ref) / np.linalg.norm(ref))


def pupil_rms(c_est, c_ref):
    """RMS pupil-phase difference over the disc (orthonormal Noll basis, j >= 4)."""
    d = np.asarray(c_est, np.float64)[3:] - np.asarray(c_ref, np.float64)[3:]
    return float(np.sqrt(np.sum(d * d)))


def as_complex(t):
    """torch float tensor [..., 2k] interleaved -> complex128 numpy [..., k]."""
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0::2] + 1j * a[..., 1::2]


def to_interleaved(z):
    z = np.asarray(z)
    out = np.empty(z.shape[:-1] + (2 * z.shape[-1],), dtype=np.float32)
    out[..., 0::2] = z.real
    out[..., 1::2] = z.imag
    return out


GOLDEN_512_SEED = 3


def golden_512_inputs(seed=GOLDEN_512_SEED):
    """The seeded 512 x 512 tile with 8 + 24 images of the mixed-precision workload:
    amplitude 0.8-1.0, phase 0-pi, Noll 4..15 uniform in +-1 rad, shot noise at 1e4
    photons per unit intensity (counter-based, so the same on every platform).
    Returns (intensity float32 [32, 512, 512], c15, geometry, snapped LEDs, illumination)."""
    n, ill = 512, synth.illumination_8_24()
    g = geometry(n)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    rng = np.random.default_rng(seed)
    obj = synth.sample_object(rng, g.H, g.W, 4.0)
    c = synth.zernike_coefficients(rng, 1.0)
    I = forward.intensity_stack(obj, g, k, c)
    I = synth.noisy_stack(I, synth.PHOTONS, seed).astype(np.float32)
    return I, c, g, k, ill


def unpack_mask(bits, shape):
    return np.unpackbits(bits, count=int(np.prod(shape))).reshape(shape).astype(bool)
