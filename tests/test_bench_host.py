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
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl, a.workload, a.images, a.tiles, a.tile) == (1, "apic", "tiles", "8+16", 512, 256)
    assert a.warmup >= 3 and a.steps >= 1


def test_reference_arm_prints_one_line_on_the_host():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--tile", "64", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [x for x in out.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mpx/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
