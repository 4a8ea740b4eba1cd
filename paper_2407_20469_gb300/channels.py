"""Multi-wavelength (e.g. RGB) batches: one plan per wavelength, made once and reused.

Each colour channel is the same per-tile reconstruction with that wavelength's
geometry: the pupil radius NA / lambda (Eq. 1) in frequency units, the LEDs'
transverse wave-vectors sin(theta) / lambda for the same LED positions, and its
own aberration, estimated per channel by that channel's aberration solve
(Eq. 8-10), so chromatic pupils come out per channel. This module only keeps
the plans and loops over channels; every step is a library call.
"""
from __future__ import annotations

from . import apic, synth


class ChannelPlans:
    """Plans for one tile size and LED layout at several wavelengths (um)."""

    def __init__(self, tile: int, wavelengths_um, n_bf: int = 8, df_rings=((0.30, 8, 0.0), (0.38, 8, 22.5)),
                 na: float = float(synth.NA), **plan_kw):
        self.tile = tile
        self.wavelengths = [float(w) for w in wavelengths_um]
        self.illuminations = {}
        self.plans = {}
        for w in self.wavelengths:
            ill = synth.illumination(n_bf, df_rings, na=na, wavelength_um=w)
            self.illuminations[w] = ill
            self.plans[w] = apic.Plan.from_illumination(tile, ill, na=na, wavelength_um=w, **plan_kw)

    def plan(self, wavelength_um: float) -> apic.Plan:
        return self.plans[float(wavelength_um)]

    def reconstruct(self, n_tiles, intensity, field, zernike, tile_status=None, stream=None):
        """intensity [C][n_tiles][n_img][h][w], field [C][n_tiles][u h][2 u w], zernike
        [C][n_tiles][15], tile_status [C][n_tiles] or None (device tensors; channel c is
        wavelengths_um[c]), all channels on one stream."""
        for c, w in enumerate(self.wavelengths):
            self.plans[w].reconstruct_batch(n_tiles, intensity[c], field[c], zernike[c], None,
                                            None if tile_status is None else tile_status[c], stream)

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans = {}
