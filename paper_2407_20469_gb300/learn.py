"""Training data and training loop of the aberration network (apic_net_*).

The network learns a microscope's field-dependent aberrations: per-tile Noll
coefficients that follow a smooth quadratic table over the slide position
(u, v) in [-1, 1]^2, plus a per-tile defocus offset (tile-to-tile focus
variation, the part that must be read from the spectra). Training tiles are
simulated on the device by the library's forward model (Eq. 1-2, Poisson
noise) from smooth random objects; a fraction can be near-blank background
(contrast below 2 %). Features, forward, backward and AdamW all run in the
library's kernels; torch only holds device memory and draws the objects.
"""
from __future__ import annotations

import math

import numpy as np

from . import apic, synth

BLANK_AMP, BLANK_PHASE = 0.01, 0.02        # near-blank objects: 1 % amplitude, 0.02 rad phase
DEFOCUS_JITTER = 0.2                      # per-tile offset of Noll 4 (rad), uniform +-


def device_objects(T: int, H: int, seed: int, device, blank=None, sigma: float = 4.0, scale=None):
    """Smooth random transmissions, interleaved complex64 [T, H, 2H].

    Amplitude 0.8 + 0.2 s0 and phase pi s1 from min-max normalised smoothed
    noise s0, s1; tiles with blank[t] get amplitude 0.99 + 0.01 s0 and phase
    0.02 s1 instead. scale[t] (faint tissue) multiplies a sample tile's
    amplitude range 0.2 and phase range pi.
    """
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    f = torch.fft.fftfreq(H, device=device)
    gauss = torch.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    out = torch.empty((T, H, 2 * H), dtype=torch.float32, device=device)
    a = torch.full((T,), 0.2, device=device)
    p = torch.full((T,), math.pi, device=device)
    if scale is not None:
        f = torch.as_tensor(np.asarray(scale, dtype=np.float32), device=device)
        a *= f
        p *= f
    if blank is not None:
        b = torch.as_tensor(np.asarray(blank, dtype=bool), device=device)
        a[b] = BLANK_AMP
        p[b] = BLANK_PHASE
    for t0 in range(0, T, 64):
        t1 = min(T, t0 + 64)
        z = torch.randn((2, t1 - t0, H, H), device=device, generator=g)
        s = torch.fft.ifft2(torch.fft.fft2(z) * gauss).real
        lo = s.amin(dim=(-2, -1), keepdim=True)
        hi = s.amax(dim=(-2, -1), keepdim=True)
        s = (s - lo) / (hi - lo)
        aa, pp = a[t0:t1, None, None], p[t0:t1, None, None]
        amp = 1.0 - aa + aa * s[0]
        ph = pp * s[1]
        out[t0:t1] = torch.view_as_real(torch.polar(amp, ph)).reshape(t1 - t0, H, 2 * H)
    return out


def field_table(seed: int = 2407, scale: float = 1.0) -> np.ndarray:
    """The microscope's quadratic aberration table [6, 15] (see synth.quadratic_field)."""
    return synth.quadratic_field(np.random.default_rng(seed), scale)


def coefficients(table: np.ndarray, uv: np.ndarray, defocus: np.ndarray | None = None) -> np.ndarray:
    """Noll coefficients [T, 15] at positions uv [T, 2], plus a Noll-4 offset."""
    u, v = uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64)
    mono = np.stack([np.ones_like(u), u, v, u * u, u * v, v * v], axis=1)
    c = mono @ table
    if defocus is not None:
        c[:, 3] += defocus
    return c.astype(np.float32)


def tile_positions(rows: int, cols: int) -> np.ndarray:
    """Tile-centre positions [rows * cols, 2] (u, v) of a rows x cols slide grid in [-1, 1]^2."""
    return synth.tile_grid_uv(rows, cols)


def draw_tiles(n: int, seed: int, table: np.ndarray, blank_frac: float = 0.0, uv: np.ndarray | None = None):
    """Positions, coefficients and background mask of n tiles (host arrays)."""
    rng = np.random.default_rng(seed)
    if uv is None:
        uv = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32)
    defocus = rng.uniform(-DEFOCUS_JITTER, DEFOCUS_JITTER, n)
    blank = rng.random(n) < blank_frac
    return uv.astype(np.float32), coefficients(table, uv, defocus), blank


def simulate(plan: apic.Plan, zern, blank, seed: int, photons: float = 1e4, start: int = 0, count: int | None = None,
             scale=None):
    """Intensity stacks [count, n_img, h, w] (device) of tiles start..start+count (scale: see device_objects)."""
    import torch
    n = plan.info.tile_h
    H = plan.info.out_h
    count = len(zern) - start if count is None else count
    obj = device_objects(count, H, seed * 7919 + start, "cuda", blank[start:start + count],
                         scale=None if scale is None else scale[start:start + count])
    z = torch.as_tensor(np.ascontiguousarray(zern[start:start + count]), device="cuda")
    I = torch.empty((count, plan.info.n_bf + plan.info.n_df, n, n), dtype=torch.float32, device="cuda")
    plan.simulate(count, obj, z, photons, seed * 104729 + start, I)
    return I


def dataset(plan: apic.Plan, n: int, seed: int, table: np.ndarray, blank_frac: float = 0.0, chunk: int = 256,
            photons: float = 1e4):
    """(features [n, 64, 64, 8], uv [n, 2], zern [n, 15]) device tensors and the host blank mask."""
    import torch
    uv, zern, blank = draw_tiles(n, seed, table, blank_frac)
    feat = torch.empty((n, apic.CROP, apic.CROP, 8), dtype=torch.float32, device="cuda")
    for t0 in range(0, n, chunk):
        c = min(chunk, n - t0)
        I = simulate(plan, zern, blank, seed, photons, t0, c)
        plan.features(c, I, feat[t0:t0 + c])
        del I
    return feat, torch.as_tensor(uv, device="cuda"), torch.as_tensor(zern, device="cuda"), blank


def init_params(seed: int, out_gain: float = 1.0) -> np.ndarray:
    """He-normal weights (fan-in scaled), zero biases, in the library's flat layout; out_gain scales
    the output layer's weights (small: the first outputs stay near zero)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in apic.param_shapes():
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:]))
            gain = 1.0 if name == "w5" else 2.0
            p[name] = rng.standard_normal(shape) * math.sqrt(gain / fan_in) * (out_gain if name == "w5" else 1.0)
    return apic.pack_params(p)


PARAMS_TAG = b"APICNET1"


def save_params(path: str, flat, meta: dict | None = None):
    """Network parameters (the flat float32 layout of apic_net_get_params) to a file: the tag
    PARAMS_TAG, one JSON header line (count, layer shapes, caller's meta), then the values as
    little-endian float32. Weights only: training resumes with fresh optimizer moments."""
    import json
    v = np.ascontiguousarray(flat, dtype="<f4").ravel()
    head = {"count": int(v.size), "layers": [[n, list(sh)] for n, sh in apic.param_shapes()], "meta": meta or {}}
    with open(path, "wb") as fh:
        fh.write(PARAMS_TAG)
        fh.write(json.dumps(head).encode() + b"\n")
        fh.write(v.tobytes())


BLOB_MAGIC = b"APICNB16"


def bf16_bits(flat) -> np.ndarray:
    """float32 -> BF16 bit patterns (uint16), rounded to nearest, ties to even."""
    u = np.ascontiguousarray(flat, dtype="<f4").ravel().view("<u4").astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype("<u2")


def bf16_values(flat) -> np.ndarray:
    """The float32 values a BF16 checkpoint of `flat` holds (what apic_net_load restores)."""
    return (bf16_bits(flat).astype("<u4") << 16).view("<f4").astype(np.float32)


def bf16_blob(flat, meta: dict | None = None) -> bytes:
    """A BF16 checkpoint of the network parameters in the layout apic_net_load reads: BLOB_MAGIC,
    the little-endian uint32 length of a JSON header (format, count, layer shapes, caller's meta),
    the header, then the values as little-endian BF16."""
    import json
    v = bf16_bits(flat)
    head = json.dumps({"format": "apic-net-bf16", "count": int(v.size),
                       "layers": [[n, list(sh)] for n, sh in apic.param_shapes()], "meta": meta or {}}).encode()
    return BLOB_MAGIC + np.uint32(len(head)).astype("<u4").tobytes() + head + v.tobytes()


def save_params_bf16(path: str, flat, meta: dict | None = None):
    """bf16_blob to a file (half the size of save_params; values rounded to BF16)."""
    with open(path, "wb") as fh:
        fh.write(bf16_blob(flat, meta))


def load_params(path: str):
    """(flat float32 parameters, meta) from save_params; ValueError if the file is not such a file,
    is truncated, or holds another layout than this library's network."""
    import json
    with open(path, "rb") as fh:
        if fh.read(len(PARAMS_TAG)) != PARAMS_TAG:
            raise ValueError(f"{path}: not a network parameter file")
        head = json.loads(fh.readline().decode())
        body = fh.read()
    want = [[n, list(sh)] for n, sh in apic.param_shapes()]
    total = sum(int(np.prod(sh)) for _, sh in apic.param_shapes())
    if head.get("layers") != want or head.get("count") != total:
        raise ValueError(f"{path}: layer shapes differ from this library's network")
    if len(body) != 4 * total:
        raise ValueError(f"{path}: expected {total} values, found {len(body) // 4}")
    return np.frombuffer(body, dtype="<f4").astype(np.float32), head.get("meta", {})


def train(net: apic.Net, feat, uv, zern, epochs: int = 4, batch: int = 64, lr: float = 1e-3,
          weight_decay: float = 1e-4, seed: int = 0, log=None):
    """AdamW on mean squared coefficient error; returns the mean loss of each epoch."""
    import torch
    n = feat.shape[0]
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    g = torch.Generator(device="cuda").manual_seed(int(seed))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    fb = torch.empty((batch,) + tuple(feat.shape[1:]), dtype=torch.float32, device="cuda")
    ub = torch.empty((batch, 2), dtype=torch.float32, device="cuda")
    zb = torch.empty((batch, 15), dtype=torch.float32, device="cuda")
    history = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            torch.index_select(feat, 0, idx, out=fb)
            torch.index_select(uv, 0, idx, out=ub)
            torch.index_select(zern, 0, idx, out=zb)
            step += 1
            # cosine decay to 5 % of the initial rate
            rate = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / max(1, total))))
            net.forward(batch, fb, ub)
            net.backward(zb, loss)
            net.adamw(rate, step, weight_decay=weight_decay)
            acc += loss
        history.append(float(acc.item()) / max(1, steps_per_epoch))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {history[-1]:.5f}")
    return history


def predict(net: apic.Net, feat, uv, batch: int | None = None):
    """Network coefficients [n, 15] (device)."""
    import torch
    n = feat.shape[0]
    batch = batch or net.max_batch
    out = torch.empty((n, 15), dtype=torch.float32, device="cuda")
    for t0 in range(0, n, batch):
        c = min(batch, n - t0)
        net.forward(c, feat[t0:t0 + c], uv[t0:t0 + c], out[t0:t0 + c])
    return out
