"""Whole-slide tiling on the GPU: cutting and pasting are exact copies, and a
slide laid out from independently simulated tiles reconstructs exactly as the
tiles do in one batch, through uneven batches."""
import numpy as np
import pytest

from paper_2407_20469_gb300 import apic, learn, slide, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def plan():
    from paper_2407_20469_gb300 import build
    build.build()
    return apic.Plan.from_illumination(64, synth.illumination(), max_tiles=8)


def test_cut_tiles_is_exact_and_rejects_windows_outside(plan):
    rng = np.random.default_rng(3)
    Hs, Ws, n_img = 150, 211, 24
    s = rng.random((n_img, Hs, Ws), dtype=np.float32)
    win = apic.slide_windows(Hs, Ws, 64, 48)
    bad = win[:1].copy()
    bad[0, 1] = Ws - 63                                   # one column beyond the slide
    allw = np.concatenate([win, bad])
    out = torch.empty((len(allw), n_img, 64, 64), dtype=torch.float32, device="cuda")
    plan.cut_tiles(len(allw), torch.as_tensor(s, device="cuda"), Hs, Ws, torch.as_tensor(allw, device="cuda"), out)
    got = out.cpu().numpy()
    for k, r in enumerate(win):
        assert np.array_equal(got[k], s[:, r[0]:r[0] + 64, r[1]:r[1] + 64])
    assert np.all(np.isnan(got[-1]))


def test_paste_fields_writes_owned_parts_exactly(plan):
    rng = np.random.default_rng(4)
    Hs, Ws = 150, 211
    win = apic.slide_windows(Hs, Ws, 64, 40)
    f = rng.standard_normal((len(win), 128, 256)).astype(np.float32)
    out = torch.full((2 * Hs, 4 * Ws), 7.0, dtype=torch.float32, device="cuda")
    plan.paste_fields(len(win), torch.as_tensor(f, device="cuda"), torch.as_tensor(win, device="cuda"), Hs, Ws, out)
    exp = np.full((2 * Hs, 4 * Ws), 7.0, dtype=np.float32)
    for k, (y0, x0, oy0, ox0, oy1, ox1) in enumerate(win):
        tile = f[k].reshape(128, 128, 2)
        exp.reshape(2 * Hs, 2 * Ws, 2)[2 * oy0:2 * oy1, 2 * ox0:2 * ox1] = \
            tile[2 * (oy0 - y0):2 * (oy1 - y0), 2 * (ox0 - x0):2 * (ox1 - x0)]
    got = out.cpu().numpy()
    assert np.array_equal(got, exp)                       # owned parts cover everything once


def test_slide_of_tiles_matches_the_batch(plan):
    rows, cols, n = 2, 3, 64
    uv, zern, blank = learn.draw_tiles(rows * cols, 8, learn.field_table())
    I = learn.simulate(plan, zern, blank, 8)                         # [6, 24, 64, 64]
    s = I.reshape(rows, cols, 24, n, n).permute(2, 0, 3, 1, 4).reshape(24, rows * n, cols * n).contiguous()
    out, z, st, win = slide.reconstruct_slide(plan, s, rows * n, cols * n, stride=n, batch=4)
    H = plan.info.out_h
    f_ref = torch.empty((rows * cols, H, 2 * H), dtype=torch.float32, device="cuda")
    z_ref = torch.empty((rows * cols, 15), dtype=torch.float32, device="cuda")
    plan.reconstruct_batch(rows * cols, I, f_ref, z_ref)
    torch.cuda.synchronize()
    assert np.array_equal(win[:, :2], np.array([[r * n, c * n] for r in range(rows) for c in range(cols)]))
    assert np.all(st.cpu().numpy() == 0)
    assert torch.equal(z, z_ref)
    exp = f_ref.reshape(rows, cols, H, H, 2).permute(0, 2, 1, 3, 4).reshape(rows * H, cols * H * 2)
    assert torch.equal(out, exp)


def test_ragged_slide_through_the_learned_path(plan):
    rng = np.random.default_rng(5)
    Hs, Ws = 100, 150                                      # not multiples of the tile
    s = torch.as_tensor(rng.random((24, Hs, Ws), dtype=np.float32) + 0.5, device="cuda")
    net = apic.Net(8)
    net.set_params(learn.init_params(2))
    out, z, st, win = slide.reconstruct_slide(plan, s, Hs, Ws, stride=56, batch=3, net=net,
                                              mode=apic.APIC_NET_WARM | apic.APIC_NET_REPLACE)
    torch.cuda.synchronize()
    assert len(win) == 6                                   # 2 x 3 windows, the last of each axis moved inward
    assert torch.isfinite(out).all() and torch.isfinite(z).all()
    assert not np.any(st.cpu().numpy() & apic.APIC_TILE_BADINPUT)


def _blend_case(plan, Hs, Ws, stride, fields_np):
    win = apic.slide_windows(Hs, Ws, 64, stride)
    f = torch.as_tensor(np.ascontiguousarray(np.stack([fields_np.real, fields_np.imag], -1).astype(np.float32))
                        .reshape(len(win), 128, 256), device="cuda")
    out, corr, phase = slide.blend_slide(plan, f, win, Hs, Ws)
    torch.cuda.synchronize()
    c = corr.cpu().numpy().astype(np.float64)
    z = phase.cpu().numpy().astype(np.float64)
    o = out.cpu().numpy().astype(np.float64).reshape(2 * Hs, 2 * Ws, 2)
    return win, c[:, 0::2] + 1j * c[:, 1::2], z[:, 0] + 1j * z[:, 1], o[..., 0] + 1j * o[..., 1]


def test_blend_matches_the_oracle_on_unrelated_fields(plan):
    from oracle import blend
    rng = np.random.default_rng(6)
    Hs, Ws, stride = 150, 211, 48                          # ragged: the last window of each axis moved inward
    n = len(apic.slide_windows(Hs, Ws, 64, stride))
    fields = (rng.standard_normal((n, 128, 128)) + 1j * rng.standard_normal((n, 128, 128))).astype(np.complex64)
    win, c, z, o = _blend_case(plan, Hs, Ws, stride, fields)
    f64 = fields.astype(np.complex128)
    rows, cols = blend.grid_shape(win)
    c_ref = blend.correlations(f64, win, 2)
    scale = blend.correlations(np.abs(f64), win, 2).real   # sum over each overlap of |f_t| |f_s|
    assert np.all(np.abs(c - c_ref) <= 1e-6 * scale)       # FP32 products and partial sums
    assert np.all(c[0] == 0) and np.all(c[cols:, 1] != 0) and np.all(c[:cols, 1] == 0)
    z_own = blend.phases(c, rows, cols)                    # the chain of the kernel's own correlations
    assert np.max(np.abs(z - z_own)) < 1e-5
    o_ref = blend.blend(f64, win, z, Hs, Ws, 2)
    assert np.linalg.norm(o - o_ref) / np.linalg.norm(o_ref) < 2e-6


@pytest.mark.parametrize("stride", [40, 12])       # 12: six windows cover a pixel, the per-pixel rule
def test_phase_shifted_crops_reassemble_on_the_gpu(plan, stride):
    rng = np.random.default_rng(7)
    Hs, Ws = 150, 211
    win = apic.slide_windows(Hs, Ws, 64, stride)
    G = rng.standard_normal((2 * Hs, 2 * Ws)) + 1j * rng.standard_normal((2 * Hs, 2 * Ws))
    theta = rng.uniform(-np.pi, np.pi, len(win))
    fields = np.stack([np.exp(1j * theta[k]) * G[2 * y:2 * y + 128, 2 * x:2 * x + 128]
                       for k, (y, x) in enumerate(win[:, :2])])
    _, _, z, o = _blend_case(plan, Hs, Ws, stride, fields)
    assert np.max(np.abs(z * np.exp(1j * theta) - np.exp(1j * theta[0]))) < 1e-5
    assert np.max(np.abs(o - np.exp(1j * theta[0]) * G)) < 1e-4


def test_blend_without_overlap_equals_paste(plan):
    rows, cols, n = 2, 3, 64
    uv, zern, blank = learn.draw_tiles(rows * cols, 8, learn.field_table())
    I = learn.simulate(plan, zern, blank, 8)
    s = I.reshape(rows, cols, 24, n, n).permute(2, 0, 3, 1, 4).reshape(24, rows * n, cols * n).contiguous()
    a, za, _, _ = slide.reconstruct_slide(plan, s, rows * n, cols * n, stride=n, batch=4)
    b, zb, _, _ = slide.reconstruct_slide(plan, s, rows * n, cols * n, stride=n, batch=4, blend=True)
    torch.cuda.synchronize()
    assert torch.equal(za, zb)
    assert torch.equal(a, b)                               # no overlap: zero correlations, unit phases and weights


def test_blended_reconstruction_of_an_overlapping_slide(plan):
    rng = np.random.default_rng(8)
    Hs, Ws = 100, 150
    s = torch.as_tensor(rng.random((24, Hs, Ws), dtype=np.float32) + 0.5, device="cuda")
    out, z, st, win = slide.reconstruct_slide(plan, s, Hs, Ws, stride=40, batch=3, blend=True)
    torch.cuda.synchronize()
    assert out.shape == (2 * Hs, 4 * Ws)
    assert torch.isfinite(out).all()


def test_unaligned_buffers_take_the_per_pixel_rule(plan):
    """Field and output 8 bytes off a 16-byte boundary: the per-pixel kernel, same result."""
    rng = np.random.default_rng(9)
    Hs, Ws, stride = 150, 211, 44
    win = apic.slide_windows(Hs, Ws, 64, stride)
    n = len(win)
    f = torch.as_tensor(rng.standard_normal((n, 128, 256)).astype(np.float32), device="cuda")
    rows, cols = slide.grid_shape(win)
    w_d = torch.as_tensor(win, device="cuda")
    ref, _, _ = slide.blend_slide(plan, f, win, Hs, Ws)
    fb = torch.empty(n * 128 * 256 + 2, dtype=torch.float32, device="cuda")
    fu = fb[2:].view(n, 128, 256)                           # 8 bytes past the allocation's alignment
    fu.copy_(f)
    ob = torch.empty(2 * Hs * 4 * Ws + 2, dtype=torch.float32, device="cuda")
    ou = ob[2:].view(2 * Hs, 4 * Ws)
    corr = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ph = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    assert fu.data_ptr() % 16 == 8 and ou.data_ptr() % 16 == 8
    plan.blend_fields(n, fu, w_d, rows, cols, Hs, Ws, corr, ph, ou)
    torch.cuda.synchronize()
    d = (ou - ref).abs().max().item()
    assert d <= 1e-6 * ref.abs().max().item()


@pytest.mark.parametrize("n", [64, 512])
def test_skipped_background_tiles_leave_the_others_bit_exact(n):
    """Uneven work: with APIC_SKIP_BACKGROUND the near-blank tiles of a mixed batch are
    skipped (status BACKGROUND, zero outputs) and the darkfield blocks take the remaining
    tiles from a shared counter; each sample tile's result is bit for bit that of a batch
    holding the sample tiles alone."""
    from paper_2407_20469_gb300 import learn
    ill = synth.illumination() if n == 64 else synth.illumination_8_24()
    T = 40 if n == 64 else 6
    blank = np.zeros(T, dtype=bool)
    blank[1::3] = True
    blank[-1] = True
    zern = learn.coefficients(learn.field_table(), np.zeros((T, 2), np.float32))
    plan = apic.Plan.from_illumination(n, ill, max_tiles=T, bg_contrast=0.02, flags=apic.APIC_SKIP_BACKGROUND)
    I = learn.simulate(plan, zern, blank, 5)
    H = plan.info.out_h
    f_mix = torch.full((T, H, 2 * H), 7.0, dtype=torch.float32, device="cuda")
    z_mix = torch.zeros((T, 15), dtype=torch.float32, device="cuda")
    s_mix = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    plan.reconstruct_batch(T, I, f_mix, z_mix, None, s_mix)
    keep = np.nonzero(~blank)[0]
    k = len(keep)
    idx = torch.as_tensor(keep, device="cuda")
    f_s = torch.zeros((k, H, 2 * H), dtype=torch.float32, device="cuda")
    z_s = torch.zeros((k, 15), dtype=torch.float32, device="cuda")
    s_s = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    plan.reconstruct_batch(k, I[idx].contiguous(), f_s, z_s, None, s_s)
    torch.cuda.synchronize()
    st = s_mix.cpu().numpy()
    assert np.all((st[blank] & apic.APIC_TILE_BACKGROUND) != 0) and np.all(st[~blank] == 0)
    assert torch.count_nonzero(f_mix[torch.as_tensor(np.nonzero(blank)[0], device="cuda")]) == 0
    assert torch.equal(f_mix[idx], f_s) and torch.equal(z_mix[idx], z_s)
