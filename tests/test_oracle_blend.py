"""Pins of the float64 blending checker (oracle/blend.py) against what the
definition fixes: crops of one field given arbitrary global phases blend back
to that field exactly (up to one global phase); the ramps of two overlapping
windows sum to one and are one outside overlaps and at the slide's edges; across
a seam between two constant fields the blend is the linear interpolation."""
import numpy as np
import pytest

from oracle import blend


def windows_for(h, w, tile, stride):
    """Row-major windows: starts 0, stride, ... while the window fits, then the last
    one moved inward to end at the edge (own bounds unused here)."""
    def starts(L):
        s = list(range(0, L - tile, stride)) + [L - tile]
        return sorted(set(s))
    ys, xs = starts(h), starts(w)
    return np.array([[y, x, 0, 0, 0, 0] for y in ys for x in xs], dtype=np.int64)


# stride < tile / 2: three or more windows cover a pixel and the weights no longer sum to one
@pytest.mark.parametrize("h,w,tile,stride,u", [(64, 96, 32, 24, 2), (40, 40, 16, 12, 1), (50, 70, 32, 20, 2),
                                               (40, 40, 16, 6, 1), (64, 96, 32, 10, 2)])
def test_crops_with_random_phases_blend_back_to_the_field(h, w, tile, stride, u):
    rng = np.random.default_rng(h + w)
    win = windows_for(h, w, tile, stride)
    H, W, L = u * h, u * w, u * tile
    G = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    theta = rng.uniform(-np.pi, np.pi, len(win))
    fields = np.stack([np.exp(1j * theta[k]) * G[u * y:u * y + L, u * x:u * x + L]
                       for k, (y, x) in enumerate(win[:, :2])])
    rows, cols = blend.grid_shape(win)
    assert rows * cols == len(win)
    c = blend.correlations(fields, win, u)
    z = blend.phases(c, rows, cols)
    assert np.allclose(np.abs(z), 1.0)
    assert np.allclose(z * np.exp(1j * theta), np.exp(1j * theta[0]))        # phi_t - phi_0 = theta_t - theta_0
    out = blend.blend(fields, win, z, h, w, u)
    assert np.max(np.abs(out - np.exp(1j * theta[0]) * G)) < 1e-12


def test_ramps_are_a_partition_of_unity_across_each_overlap():
    starts = np.array([0, 24, 48, 64])           # last window moved inward: overlaps 8, 8, 16
    L = 32
    for p in range(0, 96):
        cover = [j for j in range(len(starts)) if starts[j] <= p < starts[j] + L]
        ws = [blend.ramp(starts, j, p, L) for j in cover]
        assert all(0.0 < x <= 1.0 for x in ws)
        if len(cover) == 1:
            assert ws[0] == 1.0                      # outside overlaps and at the edges
        elif len(cover) == 2:
            assert abs(sum(ws) - 1.0) < 1e-12


def test_seam_between_two_constant_fields_is_a_linear_interpolation():
    win = windows_for(16, 40, 16, 12, )            # x starts 0, 12, 24: overlaps of 4 pixels
    L = 16
    vals = np.array([1.0, 3.0, 3.0])
    fields = np.stack([np.full((L, L), v, dtype=np.complex128) for v in vals])
    out = blend.blend(fields, win, np.ones(len(win)), 16, 40, 1)
    row = out[5].real
    assert np.all(row[:12] == 1.0) and np.all(row[16:] == 3.0)
    expect = [1.0 + 2.0 * (p - 12 + 0.5) / 4 for p in range(12, 16)]
    assert np.allclose(row[12:16], expect)
