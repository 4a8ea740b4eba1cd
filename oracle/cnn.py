"""Float64 reference of the Zernike-predicting network and its gradients.

Test infrastructure only (see the package docstring).

The network maps the intensity-spectrum magnitudes of the 8 NA-matching images
of a tile (a 64 x 64 low-frequency crop each) plus the tile's position (u, v)
on the slide to the Noll coefficients 4..15 of the pupil phase (the basis of
``zernike``). Its input feature, per image, is
    f(ky, kx) = log(|F(I)(kx, ky)| / |F(I)(0, 0)| + 1e-4),  kx, ky in [-32, 32),
stored at [ky + 32, kx + 32]. Layers (NCHW here):
    conv 3x3 (pad 1) 8 -> 32, ReLU, max-pool 2     -> 32 x 32 x 32
    conv 3x3 32 -> 64, ReLU, max-pool 2             -> 64 x 16 x 16
    conv 3x3 64 -> 128, ReLU, max-pool 2            -> 128 x 8 x 8
    conv 3x3 128 -> 256, ReLU, global mean          -> 256
    concat (u, v), dense 258 -> 256, ReLU, dense 256 -> 12
Loss: mean squared error over the batch and the 12 outputs.
Backward passes are written analytically; pinned by central finite differences.
"""
from __future__ import annotations

import numpy as np

CROP = 64
CHANNELS = (8, 32, 64, 128, 256)
HIDDEN = 256
OUTPUTS = 12
FEATURE_FLOOR = 1e-4


def features(I: np.ndarray) -> np.ndarray:
    """[n_bf, h, w] intensities -> [n_bf, 64, 64] log spectrum-magnitude crops."""
    out = np.empty((I.shape[0], CROP, CROP))
    half = CROP // 2
    for i in range(I.shape[0]):
        F = np.abs(np.fft.fft2(I[i].astype(np.float64)))
        F = F / F[0, 0]
        ky = np.arange(-half, half)
        crop = F[np.ix_(ky % I.shape[1], ky % I.shape[2])]
        out[i] = np.log(crop + FEATURE_FLOOR)
    return out


def init_params(rng: np.random.Generator) -> dict:
    """He-normal convolution and dense weights, zero biases."""
    p = {}
    for l in range(4):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        p[f"w{l}"] = rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (cin * 9))
        p[f"b{l}"] = np.zeros(cout)
    p["w4"] = rng.standard_normal((HIDDEN, CHANNELS[4] + 2)) * np.sqrt(2.0 / (CHANNELS[4] + 2))
    p["b4"] = np.zeros(HIDDEN)
    p["w5"] = rng.standard_normal((OUTPUTS, HIDDEN)) * np.sqrt(1.0 / HIDDEN)
    p["b5"] = np.zeros(OUTPUTS)
    return p


def _conv(x, w, b):
    """3x3 convolution, zero padding 1: y[n, co, i, j] = b + sum w[co, ci, dy, dx] x[n, ci, i+dy-1, j+dx-1]."""
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((n, w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nchw,oc->nohw", xp[:, :, dy:dy + h, dx:dx + wd], w[:, :, dy, dx])
    return y + b[None, :, None, None]


def _conv_backward(x, w, gy):
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("nohw,nchw->oc", gy, xp[:, :, dy:dy + h, dx:dx + wd])
            gxp[:, :, dy:dy + h, dx:dx + wd] += np.einsum("nohw,oc->nchw", gy, w[:, :, dy, dx])
    return gxp[:, :, 1:-1, 1:-1], gw, gy.sum(axis=(0, 2, 3))


def _pool(x):
    n, c, h, w = x.shape
    r = x.reshape(n, c, h // 2, 2, w // 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, h // 2, w // 2, 4)
    arg = np.argmax(r, axis=-1)                      # first maximum in (dy, dx) order
    return np.take_along_axis(r, arg[..., None], -1)[..., 0], arg


def _pool_backward(gy, arg, shape):
    n, c, h, w = shape
    g = np.zeros((n, c, h // 2, w // 2, 4))
    np.put_along_axis(g, arg[..., None], gy[..., None], -1)
    return g.reshape(n, c, h // 2, w // 2, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(shape)


def forward(p: dict, x: np.ndarray, uv: np.ndarray):
    """x [B, 8, 64, 64], uv [B, 2] -> (out [B, 12], cache)."""
    cache = []
    a = x
    for l in range(4):
        z = _conv(a, p[f"w{l}"], p[f"b{l}"])
        r = np.maximum(z, 0.0)
        if l < 3:
            pooled, arg = _pool(r)
            cache.append((a, z, r.shape, arg))
            a = pooled
        else:
            cache.append((a, z, r.shape, None))
            a = r.mean(axis=(2, 3))
    h_in = np.concatenate([a, uv], axis=1)
    z4 = h_in @ p["w4"].T + p["b4"]
    h4 = np.maximum(z4, 0.0)
    out = h4 @ p["w5"].T + p["b5"]
    return out, (cache, h_in, z4, h4)


def loss_and_grads(p: dict, x: np.ndarray, uv: np.ndarray, target: np.ndarray):
    """Mean squared error and its gradient with respect to every parameter."""
    out, (cache, h_in, z4, h4) = forward(p, x, uv)
    B = x.shape[0]
    diff = out - target
    loss = float(np.mean(diff ** 2))
    g_out = 2.0 * diff / diff.size
    g = {}
    g["w5"] = g_out.T @ h4
    g["b5"] = g_out.sum(axis=0)
    g_h4 = g_out @ p["w5"]
    g_z4 = g_h4 * (z4 > 0)
    g["w4"] = g_z4.T @ h_in
    g["b4"] = g_z4.sum(axis=0)
    g_hin = g_z4 @ p["w4"]
    g_a = g_hin[:, :CHANNELS[4]]
    for l in range(3, -1, -1):
        a_in, z, rshape, arg = cache[l]
        if l == 3:
            g_r = np.broadcast_to(g_a[:, :, None, None] / (rshape[2] * rshape[3]), rshape).copy()
        else:
            g_r = _pool_backward(g_a, arg, rshape)
        g_z = g_r * (z > 0)
        g_a, g[f"w{l}"], g[f"b{l}"] = _conv_backward(a_in, p[f"w{l}"], g_z)
    return loss, g


def param_count(p: dict) -> int:
    return int(sum(v.size for v in p.values()))
