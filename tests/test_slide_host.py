"""CPU checks of the whole-slide windows (host-only C entry point)."""
import numpy as np
import pytest

from paper_2407_20469_gb300 import apic


@pytest.mark.parametrize("h,w,tile,stride", [(700, 1000, 256, 256), (700, 1000, 256, 224), (256, 256, 256, 128),
                                             (300, 257, 128, 1), (513, 640, 128, 100), (128, 384, 128, 128)])
def test_windows_cover_the_slide_once(h, w, tile, stride):
    win = apic.slide_windows(h, w, tile, stride)
    y0, x0, oy0, ox0, oy1, ox1 = win.T
    # every window is a full tile inside the slide
    assert np.all(y0 >= 0) and np.all(x0 >= 0) and np.all(y0 + tile <= h) and np.all(x0 + tile <= w)
    # owned rectangles lie inside their windows and partition the slide
    assert np.all(oy0 >= y0) and np.all(oy1 <= y0 + tile) and np.all(ox0 >= x0) and np.all(ox1 <= x0 + tile)
    count = np.zeros((h, w), dtype=np.int32)
    for r in win:
        count[r[2]:r[4], r[3]:r[5]] += 1
    assert np.all(count == 1)
    # interior steps equal the stride; only the last window of a row or column moves inward
    ys = np.unique(y0)
    steps = np.diff(ys)
    assert np.all(steps[:-1] == stride) and (len(steps) == 0 or 0 < steps[-1] <= stride)
    assert ys[-1] == h - tile


def test_windows_reject_bad_arguments():
    with pytest.raises(apic.ApicError):
        apic.slide_windows(100, 300, 128, 64)          # shorter than a tile
    with pytest.raises(apic.ApicError):
        apic.slide_windows(300, 300, 128, 0)
    with pytest.raises(apic.ApicError):
        apic.slide_windows(300, 300, 128, 129)
