"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-side geometry (C++) equals the float64 checker's, set by set.

The geometry is integer index work, so the bar is bit-exact equality.
"""
import re
import os

import numpy as np
import pytest

from oracle import apic as oapic
from oracle import grid
from paper_2407_20469_gb300 import apic, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "apic.h")).read()
    declared = set(re.findall(r"^(?:apic_status|const char\*|size_t)\s+(apic_\w+)\(", header, re.M))
    assert declared == set(apic.EXPORTS)
    lib = apic.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.apic_status_string(apic.APIC_EINVAL).startswith(b"APIC_EINVAL")


def _geom(n):
    return grid.Geometry(n, n, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), 2)


@pytest.mark.parametrize("n,ill", [(64, synth.illumination()), (128, synth.illumination()),
                                   (128, synth.illumination_8_24()), (256, synth.illumination()),
                                   (128, synth.illumination_12_22())])
def test_host_geometry_matches_oracle(n, ill):
    plan = apic.Plan.from_illumination(n, ill, flags=apic.APIC_HOST_ONLY)
    assert plan.info.df_wave == 0                  # no device: no darkfield grid
    g = _geom(n)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    assert np.array_equal(plan.table(apic.APIC_TABLE_LEDS), k)
    assert np.array_equal(plan.table(apic.APIC_TABLE_PUPIL), grid.pupil_points(g))
    assert abs(plan.info.pupil_rx - g.Rx) < 1e-12
    rows = oapic.overlap_rows(g, k[:ill.n_bf])
    assert plan.info.n_rows == len(rows.K)
    # darkfield sets, image by image, in processing order
    spec = oapic.Spectrum(g)
    for kb in k[:ill.n_bf]:
        spec.put(grid.disc_points(g, kb), 1.0)
    order = grid.darkfield_order(k[ill.n_bf:])
    used = 0
    for idx, j in enumerate(order):
        D = grid.disc_points(g, k[ill.n_bf + j])
        s = grid.darkfield_sets(D, spec.known_set(), int(j), k[ill.n_bf + j])
        kj = np.asarray(s.k)
        U, meta = plan.df_set(idx, 0)
        P, _ = plan.df_set(idx, 1)
        Q, _ = plan.df_set(idx, 2)
        assert meta[0] == ill.n_bf + j and bool(meta[1]) == s.used
        assert np.array_equal(U, s.U + kj) and np.array_equal(P, s.P + kj) and np.array_equal(Q, s.Q)
        if s.used:
            used += 1
            spec.put(s.U, 1.0)
    assert plan.info.n_df_used == used
    ap = plan.table(apic.APIC_TABLE_APERTURE)
    iy, ix = np.nonzero(spec.known)
    ky = np.where(iy < g.H // 2, iy, iy - g.H)
    kx = np.where(ix < g.W // 2, ix, ix - g.W)
    ref = sorted(zip(ky.tolist(), kx.tolist()))
    assert [(y, x) for x, y in ap.tolist()] == ref


def test_plan_rejects_bad_arguments():
    ill = synth.illumination()
    with pytest.raises(apic.ApicError) as e:
        apic.Plan.from_illumination(100, ill, flags=apic.APIC_HOST_ONLY)      # not a power of two
    assert e.value.code == apic.APIC_EINVAL
    with pytest.raises(apic.ApicError) as e:
        apic.Plan.from_illumination(128, ill, na=0.0, flags=apic.APIC_HOST_ONLY)
    assert e.value.code == apic.APIC_EINVAL
    # an illumination ring far outside the pupil leaves no admissible NA-matching point
    bad = synth.illumination(8, (), na=0.5)
    with pytest.raises(apic.ApicError) as e:
        apic.Plan(128, bad.kx, bad.ky, 8, na=0.25, flags=apic.APIC_HOST_ONLY)
    assert e.value.code == apic.APIC_EGEOMETRY


def test_host_only_plan_refuses_device_calls():
    plan = apic.Plan.from_illumination(64, synth.illumination(), flags=apic.APIC_HOST_ONLY)
    with pytest.raises(apic.ApicError) as e:
        plan.reconstruct_batch(1, 0, 0, 0, stream=0)
    assert e.value.code == apic.APIC_EINVAL


def test_binding_refuses_buffers_the_callee_cannot_reach():
    torch = pytest.importorskip("torch")
    assert apic._ptr(None) is None and apic._ptr(1234) == 1234
    with pytest.raises(ValueError, match="contiguous"):
        apic._ptr(torch.zeros(4, 4).t())
    with pytest.raises(ValueError, match="device buffer"):
        apic._ptr(torch.zeros(4))                            # pageable host memory for a device argument
    t = torch.zeros(4)
    assert apic._ptr(t, host=True) == t.data_ptr()
    plan = apic.Plan.from_illumination(64, synth.illumination(), flags=apic.APIC_HOST_ONLY)
    with pytest.raises(ValueError):
        plan.background(1, torch.zeros(24, 64, 64), torch.zeros(1), torch.zeros(1, dtype=torch.int32))


def test_upsampling_3_plans_and_refusals():
    """The output side may be 2^k or 3 * 2^k (upsampling 3 for the paper's set-up size): the
    host aperture at 3x equals the checker's synthetic aperture on the 3n grid; other
    factors that break both forms are refused."""
    ill = synth.illumination_12_22()
    plan = apic.Plan.from_illumination(128, ill, upsample=3, flags=apic.APIC_HOST_ONLY)
    assert (plan.info.out_h, plan.info.out_w) == (384, 384)
    g = grid.Geometry(128, 128, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), 3)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    spec = oapic.Spectrum(g)
    for kb in k[:ill.n_bf]:
        spec.put(grid.disc_points(g, kb), 1.0)
    for j in grid.darkfield_order(k[ill.n_bf:]):
        s = grid.darkfield_sets(grid.disc_points(g, k[ill.n_bf + j]), spec.known_set(), int(j), k[ill.n_bf + j])
        if s.used:
            spec.put(s.U, 1.0)
    assert plan.info.n_aperture == int(spec.known.sum())
    for u in (5, 7):
        with pytest.raises(apic.ApicError) as e:
            apic.Plan.from_illumination(128, ill, upsample=u, flags=apic.APIC_HOST_ONLY)
        assert e.value.code == apic.APIC_EINVAL
