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


def _release(stream):
    """Temporaries of these helpers are torch allocations on the current stream, safe to free
    while work queued on that stream still uses them; with another stream the helper waits
    for the device before returning them."""
    if stream is not None:
        import torch
        torch.cuda.synchronize()


def grid_shape(windows: np.ndarray):
    """(rows, cols) of a row-major window list from apic_slide_windows."""
    cols = int(np.sum(windows[:, 0] == windows[0, 0]))
    return len(windows) // cols, cols


def blend_slide(plan: apic.Plan, fields, windows: np.ndarray, slide_h: int, slide_w: int, stream=None):
    """Blend the fields [n][u h][2 u w] of a slide's whole window grid where windows overlap
    (apic_blend_fields): (slide field [u slide_h][2 u slide_w], correlations [n][4], phases [n][2])."""
    import torch
    rows, cols = grid_shape(windows)
    n = len(windows)
    dev = fields.device
    u = plan.info.out_h // plan.info.tile_h
    corr = torch.empty((n, 4), dtype=torch.float32, device=dev)
    phase = torch.empty((n, 2), dtype=torch.float32, device=dev)
    out = torch.empty((u * slide_h, 2 * u * slide_w), dtype=torch.float32, device=dev)
    win_d = torch.as_tensor(windows, device=dev)
    plan.blend_fields(n, fields, win_d, rows, cols, slide_h, slide_w, corr, phase, out, stream)
    _release(stream)
    return out, corr, phase


def reconstruct_slide(plan: apic.Plan, slide, slide_h: int, slide_w: int, stride: int, batch: int | None = None,
                      net: apic.Net | None = None, mode: int = 0, stream=None, blend: bool = False):
    """(field [u slide_h][2 u slide_w] float32 interleaved complex, zernike [n][15], status [n], windows [n][6]).

    blend=False pastes each window's owned part (each tile keeps its own global phase);
    blend=True keeps every window's field and blends the overlaps (blend_slide)."""
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
    kept = torch.empty((n, H, 2 * H), dtype=torch.float32, device=dev) if blend else None
    for t0 in range(0, n, batch):
        c = min(batch, n - t0)
        fc = kept[t0:t0 + c] if blend else field
        plan.cut_tiles(c, slide, slide_h, slide_w, win_d[t0:t0 + c], I, stream)
        if net is None:
            plan.reconstruct_batch(c, I, fc, zern[t0:t0 + c], None, status[t0:t0 + c], stream)
        else:
            plan.reconstruct_learned(net, mode, c, I, uv_d[t0:t0 + c], fc, zern[t0:t0 + c], None,
                                     status[t0:t0 + c], stream)
        if not blend:
            plan.paste_fields(c, field, win_d[t0:t0 + c], slide_h, slide_w, out, stream)
    if blend:
        out = blend_slide(plan, kept, windows, slide_h, slide_w, stream)[0]
    _release(stream)
    return out, zern, status, windows
