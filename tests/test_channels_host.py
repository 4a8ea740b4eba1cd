"""Multi-wavelength plans (host-only): each channel's geometry is that
wavelength's - pupil radius NA n dx / lambda (Eq. 1) and the snapped LED
wave-vectors sin(theta) / lambda of the same LED rings - set by set equal to the
float64 checker's at that wavelength."""
import numpy as np
import pytest

from oracle import grid
from paper_2407_20469_gb300 import apic, channels, synth

RGB = (0.47, 0.52, 0.63)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()


@pytest.mark.parametrize("n", [128, 256])
def test_channel_plans_take_each_wavelengths_geometry(n):
    cp = channels.ChannelPlans(n, RGB, flags=apic.APIC_HOST_ONLY)
    radii = []
    for w in RGB:
        plan, ill = cp.plan(w), cp.illuminations[w]
        w32 = float(np.float32(w))                   # the plan's parameters are float32
        g = grid.Geometry(n, n, float(synth.NA), w32, float(synth.PIXEL_UM), 2)
        assert abs(plan.info.pupil_rx / (float(synth.NA) * n * float(synth.PIXEL_UM) / w) - 1) < 1e-6
        assert abs(plan.info.pupil_rx - g.Rx) < 1e-12
        k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
        assert np.array_equal(plan.table(apic.APIC_TABLE_LEDS), k)
        assert np.array_equal(plan.table(apic.APIC_TABLE_PUPIL), grid.pupil_points(g))
        radii.append(plan.info.pupil_rx)
    assert radii[0] > radii[1] > radii[2]           # shorter wavelength, larger pupil in frequency steps
    cp.close()
