"""Whole-slide reconstruction driver: windows, uneven batches, paste.

The slide's raw stack [n_img][slide_h][slide_w] (device) is cut into windows of
the plan's tile size (apic_slide_windows: edge windows move inward, so no tile
is ragged), reconstructed in batches of up to `batch` windows (the last batch
uneven), optionally with the aberration network, and each window's owned part
of the field is pasted into one slide-sized field. Every step is a library
call; this module only loops and holds buffers.
"""
from __future__ import annotations

import numpy as np

from . import apic


def window_positions(windows: np.ndarray, slide_h: int, slide_w: int, tile: int) -> np.ndarray:
    """Window centres scaled to [-1, 1]^2 as (u, v) = (x, y), the network's position input."""
    cy = windows[:, 0].astype(np.float64) + tile / 2.0
    cx = windows[:, 1].astype(np.float64) + tile / 2.0
    u = 2.0 * cx / slide_w - 1.0
    v = 2.0 * cy / slide_h - 1.0
    return np.stack([u, v], axis=1).astype(np.float32)


def reconstruct_slide(plan: apic.Plan, slide, slide_h: int, slide_w: int, stride: int, batch: int | None = None,
                      net: apic.Net | None = None, mode: int = 0, stream=None):
    """(field [u slide_h][2 u slide_w] float32 interleaved complex, zernike [n][15], status [n], windows [n][6])."""
    import torch
    tile = plan.info.tile_h
    windows = apic.slide_windows(slide_h, slide_w, tile, stride)
    n = len(windows)
    batch = min(batch or plan.params.max_tiles, plan.params.max_tiles)
    dev = slide.device
    n_img = plan.info.n_bf + plan.info.n_df
    H = plan.info.out_h
    win_d = torch.as_tensor(windows, device=dev)
    uv_d = torch.as_tensor(window_positions(windows, slide_h, slide_w, tile), device=dev)
    I = torch.empty((batch, n_img, tile, tile), dtype=torch.float32, device=dev)
    field = torch.empty((batch, H, 2 * H), dtype=torch.float32, device=dev)
    zern = torch.empty((n, 15), dtype=torch.float32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    out = torch.zeros((plan.info.out_h // tile * slide_h, 2 * (plan.info.out_w // tile) * slide_w),
                      dtype=torch.float32, device=dev)
    for t0 in range(0, n, batch):
        c = min(batch, n - t0)
        plan.cut_tiles(c, slide, slide_h, slide_w, win_d[t0:t0 + c], I, stream)
        if net is None:
            plan.reconstruct_batch(c, I, field, zern[t0:t0 + c], None, status[t0:t0 + c], stream)
        else:
            plan.reconstruct_learned(net, mode, c, I, uv_d[t0:t0 + c], field, zern[t0:t0 + c], None,
                                     status[t0:t0 + c], stream)
        plan.paste_fields(c, field, win_d[t0:t0 + c], slide_h, slide_w, out, stream)
    return out, zern, status, windows
