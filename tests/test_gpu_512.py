"""512 x 512 tiles with 8 + 24 images (the mixed-precision workload, the paper's
patch size): the GPU path against the float64 checker's stored reconstruction of
one seeded tile (tests/golden/apic_512_8x24.npz, written by
tests/golden/make_apic_512.py from oracle/ alone), element by element, for the
register kernels (wide darkfield kernel, 512-point Kramers-Kronig) and the
shared-memory Stockham kernels.

Bars (the workload's): field <= 1e-3 relative L2 after global-phase alignment,
the darkfield-only part of the spectrum <= 1e-3, pupil <= 0.05 rad RMS.
"""
import os

import numpy as np
import pytest

from helpers import as_complex, golden_512_inputs, pupil_rms, rel_l2, unpack_mask
from oracle import grid
from paper_2407_20469_gb300 import apic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "apic_512_8x24.npz")
FIELD_TOL = 1e-3
DARK_TOL = 1e-3
PUPIL_TOL = 0.05


@pytest.fixture(scope="module")
def case():
    from paper_2407_20469_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    gz = np.load(GOLDEN)
    I, c_true, g, k, ill = golden_512_inputs(int(gz["seed"]))
    sums = I.astype(np.float64).sum(axis=(1, 2))
    assert np.allclose(sums, gz["input_sums"], rtol=1e-6, atol=0), "the input recipe no longer gives the golden tile"
    shape = tuple(int(s) for s in gz["shape"])
    known = unpack_mask(gz["known"], shape)
    bf = unpack_mask(gz["bf_known"], shape)
    spec = np.zeros(shape, np.complex128)
    spec[known] = gz["values"].astype(np.complex128)
    return dict(I=I, ill=ill, g=g, known=known, dark=known & ~bf, spec=spec, c15=gz["c15"],
                field=grid.synthesize(spec))


def run(case, flags=0, grids=None):
    ill = case["ill"]
    plan = apic.Plan.from_illumination(512, ill, max_tiles=1, flags=flags)
    for idx, (mx, my) in (grids or {}).items():
        plan.set_df_grid(idx, mx, my)
    H = plan.info.out_h
    field = torch.zeros((1, H, 2 * H), dtype=torch.float32, device="cuda")
    z = torch.zeros((1, 15), dtype=torch.float32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    plan.reconstruct_batch(1, torch.from_numpy(case["I"])[None].cuda(), field, z, None, st)
    torch.cuda.synchronize()
    info = plan.info
    plan.close()
    return as_complex(field)[0], z[0].cpu().numpy(), int(st.item()), info


def spectrum_of(field):
    """Fourier-series coefficients of an output field (the checker's convention)."""
    return np.fft.fft2(field) / field.size


def check(case, flags=0):
    f, z, st, info = run(case, flags)
    assert st == 0
    assert rel_l2(f, case["field"]) < FIELD_TOL
    S = spectrum_of(f)
    d = case["dark"]
    assert rel_l2(S[d], case["spec"][d]) < DARK_TOL
    assert pupil_rms(z, case["c15"]) < PUPIL_TOL
    return f, info


def test_register_kernels_match_golden(case):
    check(case)


def test_stockham_kernels_match_golden(case):
    check(case, flags=apic.APIC_LEGACY_KERNELS)


def test_every_wide_grid_gives_the_same_solution(case):
    """All supported grids that are exact for an image give the same least-squares
    solution (up to rounding): force the longest grid (320 x 320) on every image."""
    f0, _, _, _ = run(case)
    ill = case["ill"]
    f1, _, st, _ = run(case, grids={i: (320, 320) for i in range(ill.n_df)})
    assert st == 0
    assert rel_l2(f1, f0) < 2e-4
    S0, S1 = spectrum_of(f0), spectrum_of(f1)
    d = case["dark"]
    assert rel_l2(S1[d], S0[d]) < 5e-4
