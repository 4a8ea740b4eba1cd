"""Multi-wavelength batch (channels.ChannelPlans) vs the float64 checker run at
each channel's wavelength on identical seeded inputs: field <= 1e-3 relative L2,
pupil <= 0.05 rad RMS, per channel and tile."""
import math

import numpy as np
import pytest

from helpers import as_complex, pupil_rms, rel_l2
from oracle import apic as oapic
from oracle import forward, grid
from paper_2407_20469_gb300 import channels, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RGB = (0.47, 0.52, 0.63)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def test_rgb_batch_matches_oracle_per_channel():
    n, T = 128, 2
    cp = channels.ChannelPlans(n, RGB, max_tiles=T)
    rng = np.random.default_rng(31)
    geoms, ks, stacks = [], [], []
    for w in RGB:
        g = grid.Geometry(n, n, float(synth.NA), float(np.float32(w)), float(synth.PIXEL_UM), 2)
        ill = cp.illuminations[w]
        k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
        tiles = []
        for _ in range(T):
            obj = synth.sample_object(rng, g.H, g.W, 4.0, phase=(0.0, math.pi))
            c = synth.zernike_coefficients(rng, 1.0)
            tiles.append(forward.intensity_stack(obj, g, k, c).astype(np.float32))
        geoms.append(g)
        ks.append(k)
        stacks.append(np.stack(tiles))
    I = torch.from_numpy(np.ascontiguousarray(np.stack(stacks))).cuda()
    H = cp.plan(RGB[0]).info.out_h
    C = len(RGB)
    field = torch.zeros((C, T, H, 2 * H), dtype=torch.float32, device="cuda")
    zern = torch.zeros((C, T, 15), dtype=torch.float32, device="cuda")
    st = torch.full((C, T), -1, dtype=torch.int32, device="cuda")
    cp.reconstruct(T, I, field, zern, st)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    zz = zern.cpu().numpy()
    for c in range(C):
        f = as_complex(field[c])
        for t in range(T):
            res = oapic.reconstruct_tile(stacks[c][t].astype(np.float64), geoms[c], ks[c], 8)
            assert rel_l2(f[t], res.field) < 1e-3, (RGB[c], t)
            assert pupil_rms(zz[c, t], res.c15) < 0.05, (RGB[c], t)
    cp.close()
