"""Upsampling 3 (the paper's set-up size, Sec. 3: 12 NA-matching + 22 darkfield LEDs up to
illumination NA 0.44, an output about three times the camera sampling): the output
transform has 3 * 2^k points (a radix-3 Stockham step before the radix-4 / 2 steps).
The synthesis and the simulator's object transform against numpy's DFT through the
checker, and the whole reconstruction against the float64 checker at the same
geometry (field <= 1e-3 relative L2, pupil <= 0.05 rad)."""
import numpy as np
import pytest

from helpers import as_complex, geometry, make_tiles, pupil_rms, rel_l2, to_interleaved
from oracle import apic as oapic
from oracle import forward, grid
from paper_2407_20469_gb300 import apic, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [64, 128, 256])
def test_synthesis_on_a_3n_grid_matches_the_dft(n):
    ill = synth.illumination_12_22()
    plan = apic.Plan.from_illumination(n, ill, max_tiles=2, upsample=3)
    H = plan.info.out_h
    assert H == 3 * n
    ap = plan.table(apic.APIC_TABLE_APERTURE)
    rng = np.random.default_rng(n)
    vals = rng.standard_normal((2, len(ap))) + 1j * rng.standard_normal((2, len(ap)))
    field = torch.zeros((2, H, 2 * H), dtype=torch.float32, device="cuda")
    plan.synthesize(2, dev(to_interleaved(vals)), field)
    torch.cuda.synchronize()
    got = as_complex(field)
    for t in range(2):
        F = np.zeros((H, H), np.complex128)
        F[ap[:, 1] % H, ap[:, 0] % H] = vals[t]
        ref = grid.synthesize(F)
        assert np.linalg.norm(got[t] - ref) / np.linalg.norm(ref) < 1e-5


def test_simulator_object_transform_on_a_3n_grid():
    n, ill = 64, synth.illumination_12_22()
    g = geometry(n, 3)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    rng = np.random.default_rng(4)
    obj = synth.sample_object(rng, g.H, g.W, 3.0)
    c = synth.zernike_coefficients(rng, 0.5)
    plan = apic.Plan.from_illumination(n, ill, max_tiles=1, upsample=3)
    I_d = torch.zeros((1, len(k), n, n), dtype=torch.float32, device="cuda")
    plan.simulate(1, dev(to_interleaved(obj[None])), dev(c[None].astype(np.float32)), 0.0, 0, I_d)
    torch.cuda.synchronize()
    ref = forward.intensity_stack(obj, g, k, c)
    assert np.max(np.abs(I_d[0].cpu().numpy() - ref)) / np.max(ref) < 2e-5


@pytest.mark.parametrize("n,count", [(128, 2), (256, 1)])
def test_12_22_upsampling_3_matches_oracle(n, count):
    ill = synth.illumination_12_22()
    I, _, _ = make_tiles(n, count, seed=300 + n, ill=ill)
    plan = apic.Plan.from_illumination(n, ill, max_tiles=count, upsample=3)
    H = plan.info.out_h
    field = torch.zeros((count, H, 2 * H), dtype=torch.float32, device="cuda")
    z = torch.zeros((count, 15), dtype=torch.float32, device="cuda")
    st = torch.full((count,), -1, dtype=torch.int32, device="cuda")
    plan.reconstruct_batch(count, dev(I), field, z, None, st)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    g = geometry(n, 3)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    f = as_complex(field)
    for t in range(count):
        res = oapic.reconstruct_tile(I[t].astype(np.float64), g, k, ill.n_bf)
        assert res.field.shape == (3 * n, 3 * n)
        assert rel_l2(f[t], res.field) < 1e-3
        assert pupil_rms(z[t].cpu().numpy(), res.c15) < 0.05
