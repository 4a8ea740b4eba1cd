"""Host-side parts of bench.py: the blend call's algorithmic byte count against a
brute-force count of covered pixels, the illumination sets behind --images,
the default options of the timing contract, and the reference arm's JSON line
(the float64 checker on one small tile, no GPU)."""
import json
import subprocess
import sys

import numpy as np
import pytest

import bench
from paper_2407_20469_gb300 import apic


@pytest.mark.parametrize("h,w,tile,stride", [(150, 211, 64, 48), (100, 150, 64, 20), (300, 420, 64, 60)])
def test_blend_bytes_count_fields_output_and_overlap_strips(h, w, tile, stride):
    win = apic.slide_windows(h, w, tile, stride)
    u, L = 2, 2 * tile
    rows = len(np.unique(win[:, 0]))
    cols = len(win) // rows
    strips = 0
    for k in range(len(win)):
        for nb in ((k - 1) if k % cols else -1, (k - cols) if k >= cols else -1):
            if nb < 0:
                continue
            a = np.zeros((u * h, u * w), dtype=bool)       # pixels of window k ...
            a[u * win[k, 0]:u * win[k, 0] + L, u * win[k, 1]:u * win[k, 1] + L] = True
            b = np.zeros_like(a)                           # ... that window nb covers too
            b[u * win[nb, 0]:u * win[nb, 0] + L, u * win[nb, 1]:u * win[nb, 1] + L] = True
            strips += 2 * int(np.count_nonzero(a & b))
    assert bench.blend_bytes(win, u, L, u * u * h * w) == 8 * (len(win) * L * L + u * u * h * w + strips)


def test_image_sets_behind_the_images_option():
    for name, (n_bf, n_df) in {"8+16": (8, 16), "8+24": (8, 24), "12+22": (12, 22)}.items():
        ill = bench.illumination_for(name)
        assert (ill.n_bf, len(ill.kx) - ill.n_bf) == (n_bf, n_df)


def test_default_options_keep_the_timing_contract(monkeypatch):
    """The default line is the largest single-GPU workload: 2048 tiles of 512 x 512
    with 8 + 24 images; --workload cfg2 is 512 tiles of 256 x 256 with 8 + 16."""
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl, a.workload, a.images, a.tiles, a.tile) == (1, "apic", "cfg3", "8+24", 2048, 512)
    assert a.zgrid == (32, 64) and a.warmup >= 3 and a.steps >= 1 and a.e2e_steps >= 10
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "cfg2"])
    a = bench.parse()
    assert (a.images, a.tiles, a.tile, a.zgrid) == ("8+16", 512, 256, (16, 32))


def test_oracle_tile_pieces_reproduce_the_checker_and_its_sets():
    """bench.OracleTile runs the checker's functions in the checker's order: on a small
    tile its spectrum equals oracle reconstruct_tile's and its geometry-only set sizes
    equal the sets the checker used; the per-tile estimate with every solve measured is
    the plain sum."""
    from oracle import apic as oapic
    I, g, k, ill = bench.oracle_tile_sample(64, "8+16", 5)
    ot = bench.OracleTile(I, g, k, ill.n_bf)
    t_bf = ot.brightfield()
    meas = [ot.darkfield_next() for _ in range(len(ot.order))]
    ref = oapic.reconstruct_tile(I.astype(np.float64), g, k, ill.n_bf)
    assert np.array_equal(ot.spec.values, ref.spectrum.values)
    assert ot.sizes == [(len(s.U), len(s.Q)) if s.used else (0, 0) for s in ref.df_sets]
    assert ot.tile_seconds(t_bf, meas) == pytest.approx(t_bf + sum(b + s for b, s, _ in meas))


def test_reference_arm_prints_one_line_on_the_host():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--tile", "64", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [x for x in out.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mpx/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
