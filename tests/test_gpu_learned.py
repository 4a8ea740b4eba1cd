"""What the trained network gains over the closed-form aberration solve.

The network is trained on the GPU (own forward/backward/AdamW kernels) on
simulated tiles whose coefficients follow a fixed field-dependent table plus
a per-tile defocus offset, 30 % of them near-blank. On fresh tiles from the
same slide model the closed-form-only reconstruction is compared with the
learned one (warm start on solved tiles, replacement on low-contrast tiles),
both compared with the true coefficients.
"""
import time

import numpy as np
import pytest

from paper_2407_20469_gb300 import apic, learn, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 128


@pytest.fixture(scope="module")
def trained():
    from paper_2407_20469_gb300 import build
    build.build()
    ill = synth.illumination()
    table = learn.field_table()
    bf = apic.Plan(N, ill.kx[:8], ill.ky[:8], 8, max_tiles=256)
    t0 = time.perf_counter()
    feat, uv, zern, _ = learn.dataset(bf, 8192, 11, table, blank_frac=0.3)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = apic.Net(256)
    net.set_params(learn.init_params(1))
    hist = learn.train(net, feat, uv, zern, epochs=8, batch=64, lr=3e-3, log=print)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(f"dataset {t1 - t0:.1f} s, training {t2 - t1:.1f} s, losses {[round(h, 5) for h in hist]}")
    del feat, uv, zern
    return ill, table, net, hist


def test_training_converges(trained):
    hist = trained[3]
    assert hist[-1] < 0.2 * hist[0]
    assert all(np.isfinite(hist))


def test_learned_reconstruction_beats_closed_form_on_background(trained):
    ill, table, net, _ = trained
    T = 512
    plan = apic.Plan.from_illumination(N, ill, max_tiles=T, bg_contrast=0.02)
    uv, zern, blank = learn.draw_tiles(T, 99, table, 0.3)
    I = learn.simulate(plan, zern, blank, 99)
    H = plan.info.out_h
    field = torch.empty((T, H, 2 * H), dtype=torch.float32, device="cuda")
    z_cf = torch.empty((T, 15), dtype=torch.float32, device="cuda")
    z_l = torch.empty_like(z_cf)
    st_cf = torch.empty(T, dtype=torch.int32, device="cuda")
    st_l = torch.empty_like(st_cf)
    plan.reconstruct_batch(T, I, field, z_cf, tile_status=st_cf)          # closed form on every tile
    uv_d = torch.as_tensor(uv, device="cuda")
    plan.reconstruct_learned(net, apic.APIC_NET_WARM | apic.APIC_NET_REPLACE, T, I, uv_d, field, z_l,
                             tile_status=st_l)
    feat = torch.empty((T, 64, 64, 8), dtype=torch.float32, device="cuda")
    plan.features(T, I, feat)
    z_net = learn.predict(net, feat, uv_d).cpu().numpy()
    torch.cuda.synchronize()
    z_cf, z_l, st_l = z_cf.cpu().numpy(), z_l.cpu().numpy(), st_l.cpu().numpy()

    def err(z):
        d = z[:, 3:].astype(np.float64) - zern[:, 3:]
        return np.sqrt((d * d).sum(axis=1))

    e_cf, e_l, e_net = err(z_cf), err(z_l), err(z_net)
    learned = (st_l & apic.APIC_TILE_LEARNED) != 0
    warm = (st_l & apic.APIC_TILE_WARM) != 0
    fg = ~blank
    print(f"blank tiles {blank.sum()}: median pupil error closed form {np.median(e_cf[blank]):.3f} rad, "
          f"learned {np.median(e_l[blank]):.3f} rad")
    print(f"other tiles {fg.sum()}: closed form {np.median(e_cf[fg]):.4f}, learned {np.median(e_l[fg]):.4f}, "
          f"network alone {np.median(e_net[fg]):.4f}; warm start kept on {warm[fg].sum()}")
    print(f"flagged learned: {learned[blank].mean():.3f} of blank, {learned[fg].mean():.3f} of others")
    # the contrast test routes the near-blank tiles, and only those, to the network
    assert learned[blank].mean() > 0.9
    assert not learned[fg].any()
    # replacement: much better than the ill-conditioned closed form on background tiles
    assert np.median(e_l[blank]) < 0.5 * np.median(e_cf[blank])
    assert np.median(e_l[blank]) < 0.25
    # warm start: the residual comparison keeps the closed-form quality elsewhere
    assert np.median(e_l[fg]) <= np.median(e_cf[fg]) + 0.01
    assert np.all(np.isfinite(z_l))
