"""Thin Python binding of the C interface in include/apic.h (ctypes).

Argument marshalling only: every computation runs in libapic.so's kernels.
Device buffers are passed as torch CUDA tensors (their data_ptr()) or raw
integer addresses; streams default to torch's current stream. Loading fails
loudly when the shared object is missing - there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapic.so")

APIC_OK, APIC_EINVAL, APIC_ENOMEM, APIC_ECUDA, APIC_EGEOMETRY, APIC_EINTERNAL, APIC_ENOTCONV = range(7)
APIC_TILE_OK, APIC_TILE_BACKGROUND, APIC_TILE_NOTCONV, APIC_TILE_BADINPUT = 0, 1, 2, 4
APIC_TILE_LEARNED, APIC_TILE_WARM = 8, 16
APIC_NET_WARM, APIC_NET_REPLACE = 1, 2
APIC_SKIP_BACKGROUND = 1
APIC_HOST_ONLY = 2
APIC_LEGACY_KERNELS = 4
APIC_N_ZERNIKE = 15
APIC_TABLE_LEDS, APIC_TABLE_PUPIL, APIC_TABLE_APERTURE = 0, 1, 2

# Every symbol include/apic.h declares (checked by the CPU test suite).
EXPORTS = [
    "apic_status_string", "apic_last_error", "apic_plan_create", "apic_plan_destroy",
    "apic_plan_query", "apic_plan_table", "apic_plan_df_set", "apic_plan_df_grid", "apic_plan_set_df_grid",
    "apic_plan_counters", "apic_plan_timing",
    "apic_plan_stage_ms", "apic_reconstruct_batch", "apic_reconstruct_host", "apic_background",
    "apic_kk_spectra", "apic_kk_spectra_noalloc", "apic_aberration", "apic_stitch", "apic_darkfield", "apic_synthesize",
    "apic_pupil", "apic_simulate", "apic_net_param_count", "apic_net_feature_count", "apic_net_create",
    "apic_net_destroy", "apic_net_set_params", "apic_net_get_params", "apic_net_get_grads", "apic_net_forward",
    "apic_net_backward", "apic_net_adamw", "apic_net_activation", "apic_features", "apic_reconstruct_learned",
    "apic_slide_windows", "apic_cut_tiles", "apic_paste_fields", "apic_blend_fields", "apic_plan_autotune",
    "apic_measure_fma_rate", "apic_net_load",
]


class apic_params(C.Structure):
    _fields_ = [
        ("tile_h", C.c_int), ("tile_w", C.c_int), ("n_bf", C.c_int), ("n_df", C.c_int),
        ("h_kx", C.POINTER(C.c_float)), ("h_ky", C.POINTER(C.c_float)),
        ("na", C.c_float), ("wavelength_um", C.c_float), ("pixel_um", C.c_float),
        ("upsample", C.c_int), ("max_tiles", C.c_int), ("df_iters", C.c_int), ("df_tol", C.c_float),
        ("ab_passes", C.c_int), ("bg_contrast", C.c_float), ("flags", C.c_int),
    ]


class apic_plan_info(C.Structure):
    _fields_ = [
        ("tile_h", C.c_int), ("tile_w", C.c_int), ("out_h", C.c_int), ("out_w", C.c_int),
        ("n_bf", C.c_int), ("n_df", C.c_int), ("n_pupil", C.c_int), ("n_aperture", C.c_int),
        ("n_rows", C.c_int), ("n_df_used", C.c_int), ("fft_m", C.c_int),
        ("pupil_rx", C.c_double), ("pupil_ry", C.c_double), ("df_wave", C.c_int),
    ]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libapic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2407_20469_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, f32, sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
    sig = {
        "apic_status_string": (C.c_char_p, [i32]),
        "apic_last_error": (C.c_char_p, []),
        "apic_plan_create": (i32, [C.POINTER(apic_params), C.POINTER(vp)]),
        "apic_measure_fma_rate": (i32, [i32, C.POINTER(C.c_double)]),
        "apic_net_load": (i32, [vp, C.c_char_p, sz]),
        "apic_plan_destroy": (i32, [vp]),
        "apic_plan_query": (i32, [vp, C.POINTER(apic_plan_info)]),
        "apic_plan_table": (i32, [vp, i32, C.POINTER(C.c_int32), sz]),
        "apic_plan_df_set": (i32, [vp, i32, i32, C.POINTER(C.c_int32), sz, C.POINTER(C.c_int32)]),
        "apic_plan_df_grid": (i32, [vp, i32, C.POINTER(C.c_int32)]),
        "apic_plan_set_df_grid": (i32, [vp, i32, i32, i32]),
        "apic_plan_counters": (i32, [vp, C.POINTER(C.c_int64), i32, i32]),
        "apic_plan_timing": (i32, [vp, i32]),
        "apic_plan_stage_ms": (i32, [vp, C.POINTER(C.c_double), i32, C.POINTER(C.c_int32), i32]),
        "apic_reconstruct_batch": (i32, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "apic_reconstruct_host": (i32, [vp, i32, vp, vp, vp, vp]),
        "apic_background": (i32, [vp, i32, vp, vp, vp, vp]),
        "apic_kk_spectra": (i32, [vp, i32, vp, vp, vp]),
        "apic_kk_spectra_noalloc": (i32, [vp, i32, vp, vp, vp]),
        "apic_aberration": (i32, [vp, i32, vp, vp, vp]),
        "apic_stitch": (i32, [vp, i32, vp, vp, vp, vp]),
        "apic_darkfield": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "apic_synthesize": (i32, [vp, i32, vp, vp, vp]),
        "apic_pupil": (i32, [vp, i32, vp, vp, vp]),
        "apic_simulate": (i32, [vp, i32, vp, vp, f32, C.c_uint64, vp, vp]),
        "apic_net_param_count": (sz, []),
        "apic_net_feature_count": (sz, []),
        "apic_net_create": (i32, [i32, C.POINTER(vp)]),
        "apic_net_destroy": (i32, [vp]),
        "apic_net_set_params": (i32, [vp, C.POINTER(C.c_float), sz]),
        "apic_net_get_params": (i32, [vp, C.POINTER(C.c_float), sz]),
        "apic_net_get_grads": (i32, [vp, C.POINTER(C.c_float), sz]),
        "apic_net_forward": (i32, [vp, i32, vp, vp, vp, vp]),
        "apic_net_backward": (i32, [vp, vp, vp, vp]),
        "apic_net_adamw": (i32, [vp, f32, f32, f32, f32, f32, i32, vp]),
        "apic_net_activation": (i32, [vp, i32, C.POINTER(C.c_float), sz]),
        "apic_features": (i32, [vp, i32, vp, vp, vp]),
        "apic_reconstruct_learned": (i32, [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
        "apic_plan_autotune": (i32, [vp, i32, vp, C.POINTER(C.c_double), i32]),
        "apic_slide_windows": (i32, [i32, i32, i32, i32, C.POINTER(C.c_int32), i32, C.POINTER(C.c_int)]),
        "apic_cut_tiles": (i32, [vp, i32, vp, i32, i32, vp, vp, vp]),
        "apic_paste_fields": (i32, [vp, i32, vp, vp, i32, i32, vp, vp]),
        "apic_blend_fields": (i32, [vp, i32, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ApicError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.apic_last_error().decode()
        super().__init__(f"{where}: {lib.apic_status_string(code).decode()} ({msg})")
        self.code = code


def _check(code: int, where: str):
    if code != APIC_OK:
        raise ApicError(code, where)


def _ptr(x, host: bool = False) -> int | None:
    """Address of a buffer for the C ABI: None, a raw address, or a contiguous tensor that the
    callee can reach - device memory or pinned host memory for device arguments, CPU memory for
    host arguments (host=True). Anything else raises ValueError here instead of reaching a kernel."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_contiguous():
        raise ValueError("buffers passed to the library must be contiguous")
    if host:
        if x.device.type != "cpu":
            raise ValueError(f"expected a host (CPU) buffer, got one on {x.device}")
    elif x.device.type != "cuda" and not x.is_pinned():
        raise ValueError(f"expected a device buffer (CUDA or pinned host memory), got pageable memory on {x.device}")
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def validate_net_blob(blob: bytes):
    """Checks a BF16 network checkpoint blob without a network (apic_net_load with NULL); raises
    ApicError (APIC_EINVAL) with the library's reason if it is malformed."""
    _check(load().apic_net_load(None, bytes(blob), len(blob)), "apic_net_load")


def measure_fma_rate(precision: int = 32) -> float:
    """Measured FMA throughput (flop/s) of the current device's CUDA cores, FP32 or FP64."""
    out = C.c_double()
    _check(load().apic_measure_fma_rate(int(precision), C.byref(out)), "apic_measure_fma_rate")
    return float(out.value)


def slide_windows(slide_h: int, slide_w: int, tile: int, stride: int) -> np.ndarray:
    """Windows [n, 6] int32 (y0, x0, oy0, ox0, oy1, ox1) covering a slide (apic_slide_windows)."""
    lib = load()
    n = C.c_int(0)
    _check(lib.apic_slide_windows(slide_h, slide_w, tile, stride, None, 0, C.byref(n)), "apic_slide_windows")
    out = np.zeros((n.value, 6), dtype=np.int32)
    _check(lib.apic_slide_windows(slide_h, slide_w, tile, stride, out.ctypes.data_as(C.POINTER(C.c_int32)),
                                  n.value, C.byref(n)), "apic_slide_windows")
    return out


class Plan:
    """An apic_plan: geometry of one tile-size class plus its device workspace."""

    def __init__(self, tile: int, kx, ky, n_bf: int, na=0.25, wavelength_um=0.52, pixel_um=0.345,
                 upsample: int = 2, max_tiles: int = 64, df_iters: int = 0, df_tol: float = 0.0,
                 ab_passes: int = -1, bg_contrast: float = 0.02, flags: int = 0):
        lib = load()
        self._kx = np.ascontiguousarray(kx, dtype=np.float32)
        self._ky = np.ascontiguousarray(ky, dtype=np.float32)
        p = apic_params()
        p.tile_h = p.tile_w = tile
        p.n_bf = n_bf
        p.n_df = len(self._kx) - n_bf
        p.h_kx = self._kx.ctypes.data_as(C.POINTER(C.c_float))
        p.h_ky = self._ky.ctypes.data_as(C.POINTER(C.c_float))
        p.na, p.wavelength_um, p.pixel_um = float(na), float(wavelength_um), float(pixel_um)
        p.upsample, p.max_tiles, p.df_iters, p.df_tol = upsample, max_tiles, df_iters, df_tol
        p.ab_passes, p.bg_contrast, p.flags = ab_passes, bg_contrast, flags
        h = C.c_void_p()
        _check(lib.apic_plan_create(C.byref(p), C.byref(h)), "apic_plan_create")
        self.handle = h
        self.params = p
        info = apic_plan_info()
        _check(lib.apic_plan_query(h, C.byref(info)), "apic_plan_query")
        self.info = info

    @classmethod
    def from_illumination(cls, tile: int, ill, **kw) -> "Plan":
        return cls(tile, ill.kx, ill.ky, ill.n_bf, **kw)

    def close(self):
        if getattr(self, "handle", None):
            load().apic_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def table(self, which: int) -> np.ndarray:
        n = {APIC_TABLE_LEDS: self.info.n_bf + self.info.n_df, APIC_TABLE_PUPIL: self.info.n_pupil,
             APIC_TABLE_APERTURE: self.info.n_aperture}[which]
        out = np.zeros((n, 2), dtype=np.int32)
        _check(load().apic_plan_table(self.handle, which, out.ctypes.data_as(C.POINTER(C.c_int32)), out.size),
               "apic_plan_table")
        return out

    def df_set(self, index: int, which: int):
        """(points [k, 2] int32, meta {led, used, nU, nP, nQ}) of darkfield image `index`."""
        meta = np.zeros(5, dtype=np.int32)
        lib = load()
        P32 = C.POINTER(C.c_int32)
        _check(lib.apic_plan_df_set(self.handle, index, which, None, 0, meta.ctypes.data_as(P32)), "apic_plan_df_set")
        out = np.zeros((int(meta[2 + which]), 2), dtype=np.int32)
        _check(lib.apic_plan_df_set(self.handle, index, which, out.ctypes.data_as(P32), out.size,
                                    meta.ctypes.data_as(P32)), "apic_plan_df_set")
        return out, meta

    def df_grid(self, index: int):
        """(solved with x and y swapped, row grid points, column grid points) of darkfield image `index`."""
        g = np.zeros(3, dtype=np.int32)
        _check(load().apic_plan_df_grid(self.handle, index, g.ctypes.data_as(C.POINTER(C.c_int32))),
               "apic_plan_df_grid")
        return int(g[0]), int(g[1]), int(g[2])

    def set_df_grid(self, index: int, mx: int, my: int):
        """Use the mx x my register grid for darkfield image `index` (a supported, exact pair)."""
        _check(load().apic_plan_set_df_grid(self.handle, index, mx, my), "apic_plan_set_df_grid")

    def counters(self, reset: bool = False) -> dict:
        """Work counters: kernel launches, CGLS iterations, darkfield solves, and the CGLS
        iterations of each used darkfield image (synchronises)."""
        k = 3 + min(self.info.n_df_used, 256)
        out = np.zeros(k, dtype=np.int64)
        _check(load().apic_plan_counters(self.handle, out.ctypes.data_as(C.POINTER(C.c_int64)), k, int(reset)),
               "apic_plan_counters")
        return {"launches": int(out[0]), "cg_iterations": int(out[1]), "df_solves": int(out[2]),
                "cg_iterations_per_image": [int(v) for v in out[3:]]}

    STAGES = ("background", "kk", "aberration", "stitch", "darkfield", "synthesize", "pupil")

    def timing(self, enable: bool = True):
        _check(load().apic_plan_timing(self.handle, int(enable)), "apic_plan_timing")

    def stage_ms(self, reset: bool = False):
        """({stage: summed ms}, calls) over the timed reconstruct_batch calls (synchronises)."""
        ms = np.zeros(7, dtype=np.float64)
        calls = C.c_int32(0)
        _check(load().apic_plan_stage_ms(self.handle, ms.ctypes.data_as(C.POINTER(C.c_double)), 7, C.byref(calls),
                                         int(reset)), "apic_plan_stage_ms")
        return dict(zip(self.STAGES, ms.tolist())), int(calls.value)

    # -- entry points (same names as the C interface, without the prefix)
    def reconstruct_batch(self, n_tiles, intensity, field, zernike, pupil=None, tile_status=None, stream=None):
        _check(load().apic_reconstruct_batch(self.handle, n_tiles, _ptr(intensity), _ptr(field), _ptr(zernike),
                                             _ptr(pupil), _ptr(tile_status), _stream(stream)),
               "apic_reconstruct_batch")

    def reconstruct_host(self, n_tiles, intensity, field, zernike, tile_status=None) -> int:
        """Host-memory reconstruction, pipelined in chunks (pass pinned CPU tensors for overlap).
        Returns APIC_OK, or APIC_ENOTCONV when every output was written but some tile's darkfield
        solve stopped above its tolerance (reported only with tile_status); raises otherwise."""
        code = load().apic_reconstruct_host(self.handle, n_tiles, _ptr(intensity, True), _ptr(field, True),
                                            _ptr(zernike, True), _ptr(tile_status, True))
        if code != APIC_ENOTCONV:
            _check(code, "apic_reconstruct_host")
        return code

    def background(self, n_tiles, intensity, contrast2, tile_status, stream=None):
        _check(load().apic_background(self.handle, n_tiles, _ptr(intensity), _ptr(contrast2), _ptr(tile_status),
                                      _stream(stream)), "apic_background")

    def kk_spectra(self, n_tiles, intensity, xdisc, stream=None):
        _check(load().apic_kk_spectra(self.handle, n_tiles, _ptr(intensity), _ptr(xdisc), _stream(stream)),
               "apic_kk_spectra")

    def kk_spectra_noalloc(self, n_tiles, intensity, xdisc, stream=None):
        """apic_kk_spectra without any allocation: scratch from the library's fixed device array.

        n_tiles is not bounded by the plan's max_tiles, so tensors are checked to hold
        n_tiles tiles (float32) before the call."""
        info = self.info
        for name, t, per_tile in (("intensity", intensity, (info.n_bf + info.n_df) * info.tile_h * info.tile_w),
                                  ("xdisc", xdisc, info.n_bf * 2 * info.n_pupil)):
            if hasattr(t, "numel"):
                if str(t.dtype) != "torch.float32":
                    raise ValueError(f"{name} must be float32")
                if t.numel() < n_tiles * per_tile:
                    raise ValueError(f"{name} holds {t.numel()} values; {n_tiles} tiles need {n_tiles * per_tile}")
        _check(load().apic_kk_spectra_noalloc(self.handle, n_tiles, _ptr(intensity), _ptr(xdisc), _stream(stream)),
               "apic_kk_spectra_noalloc")

    def aberration(self, n_tiles, xdisc, zernike, stream=None):
        _check(load().apic_aberration(self.handle, n_tiles, _ptr(xdisc), _ptr(zernike), _stream(stream)),
               "apic_aberration")

    def stitch(self, n_tiles, xdisc, zernike, spec, stream=None):
        _check(load().apic_stitch(self.handle, n_tiles, _ptr(xdisc), _ptr(zernike), _ptr(spec), _stream(stream)),
               "apic_stitch")

    def darkfield(self, n_tiles, intensity, zernike, spec, tile_status=None, stream=None):
        _check(load().apic_darkfield(self.handle, n_tiles, _ptr(intensity), _ptr(zernike), _ptr(spec),
                                     _ptr(tile_status), _stream(stream)), "apic_darkfield")

    def synthesize(self, n_tiles, spec, field, stream=None):
        _check(load().apic_synthesize(self.handle, n_tiles, _ptr(spec), _ptr(field), _stream(stream)),
               "apic_synthesize")

    def pupil(self, n_tiles, zernike, pupil, stream=None):
        _check(load().apic_pupil(self.handle, n_tiles, _ptr(zernike), _ptr(pupil), _stream(stream)), "apic_pupil")

    def simulate(self, n_tiles, obj, zernike, photons, seed, intensity, stream=None):
        _check(load().apic_simulate(self.handle, n_tiles, _ptr(obj), _ptr(zernike), float(photons), int(seed),
                                    _ptr(intensity), _stream(stream)), "apic_simulate")

    def autotune(self, n_tiles, intensity) -> dict:
        """Times the register and Stockham variants of the transform stages (and, for 512-pixel
        tiles, the darkfield kernel with 1, 2, 4 blocks per tile) on a sample; keeps the fastest."""
        ms = np.full(7, -1.0)
        _check(load().apic_plan_autotune(self.handle, n_tiles, _ptr(intensity),
                                         ms.ctypes.data_as(C.POINTER(C.c_double)), 7), "apic_plan_autotune")
        return {"kk_register": ms[0], "kk_stockham": ms[1], "darkfield_register": ms[2],
                "darkfield_stockham": ms[3], "darkfield_wide_1": ms[4], "darkfield_wide_2": ms[5],
                "darkfield_wide_4": ms[6]}

    def cut_tiles(self, n_tiles, slide, slide_h, slide_w, windows, intensity, stream=None):
        _check(load().apic_cut_tiles(self.handle, n_tiles, _ptr(slide), slide_h, slide_w, _ptr(windows),
                                     _ptr(intensity), _stream(stream)), "apic_cut_tiles")

    def paste_fields(self, n_tiles, field, windows, slide_h, slide_w, slide_field, stream=None):
        _check(load().apic_paste_fields(self.handle, n_tiles, _ptr(field), _ptr(windows), slide_h, slide_w,
                                        _ptr(slide_field), _stream(stream)), "apic_paste_fields")

    def blend_fields(self, n_tiles, field, windows, n_rows, n_cols, slide_h, slide_w, corr, phase, slide_field,
                     stream=None):
        _check(load().apic_blend_fields(self.handle, n_tiles, _ptr(field), _ptr(windows), n_rows, n_cols, slide_h,
                                        slide_w, _ptr(corr), _ptr(phase), _ptr(slide_field), _stream(stream)),
               "apic_blend_fields")

    def features(self, n_tiles, intensity, feat, stream=None):
        """Network input features [n_tiles][64][64][8] of the first 8 images of each stack."""
        _check(load().apic_features(self.handle, n_tiles, _ptr(intensity), _ptr(feat), _stream(stream)),
               "apic_features")

    def reconstruct_learned(self, net: "Net", mode, n_tiles, intensity, uv, field, zernike, pupil=None,
                            tile_status=None, stream=None):
        _check(load().apic_reconstruct_learned(self.handle, net.handle, int(mode), n_tiles, _ptr(intensity), _ptr(uv),
                                               _ptr(field), _ptr(zernike), _ptr(pupil), _ptr(tile_status),
                                               _stream(stream)), "apic_reconstruct_learned")


# ----------------------------------------------------------------------------- network

CONV_CHANNELS = (8, 32, 64, 128, 256)
HIDDEN, OUTPUTS = 256, 12
CROP = 64


def param_shapes():
    """Per-layer (name, shape) in the oracle's convention: conv w [co, ci, 3, 3], dense w [out, in]."""
    shapes = []
    for l in range(4):
        ci, co = CONV_CHANNELS[l], CONV_CHANNELS[l + 1]
        shapes += [(f"w{l}", (co, ci, 3, 3)), (f"b{l}", (co,))]
    shapes += [("w4", (HIDDEN, CONV_CHANNELS[4] + 2)), ("b4", (HIDDEN,)), ("w5", (OUTPUTS, HIDDEN)), ("b5", (OUTPUTS,))]
    return shapes


def pack_params(p: dict) -> np.ndarray:
    """Per-layer arrays -> the library's flat vector (W_l [out][taps + 1], taps (dy, dx, ci), bias last)."""
    out = []
    for l in range(6):
        w, b = np.asarray(p[f"w{l}"], dtype=np.float64), np.asarray(p[f"b{l}"], dtype=np.float64)
        if l < 4:
            w = w.transpose(0, 2, 3, 1).reshape(w.shape[0], -1)
        out.append(np.concatenate([w, b[:, None]], axis=1).ravel())
    return np.concatenate(out).astype(np.float32)


def unpack_params(v: np.ndarray) -> dict:
    """Inverse of pack_params (float64 arrays)."""
    v = np.asarray(v, dtype=np.float64)
    p, o = {}, 0
    shapes = dict(param_shapes())
    for l in range(6):
        ws = shapes[f"w{l}"]
        rows = ws[0]
        taps = int(np.prod(ws[1:]))
        m = v[o:o + rows * (taps + 1)].reshape(rows, taps + 1)
        o += rows * (taps + 1)
        w = m[:, :taps]
        if l < 4:
            w = w.reshape(rows, 3, 3, ws[1]).transpose(0, 3, 1, 2)
        p[f"w{l}"] = np.ascontiguousarray(w)
        p[f"b{l}"] = m[:, taps].copy()
    return p


class Net:
    """An apic_net: the aberration network with workspace for batches up to max_batch."""

    def __init__(self, max_batch: int):
        lib = load()
        h = C.c_void_p()
        _check(lib.apic_net_create(int(max_batch), C.byref(h)), "apic_net_create")
        self.handle = h
        self.max_batch = int(max_batch)
        self.n_params = int(lib.apic_net_param_count())

    def close(self):
        if getattr(self, "handle", None):
            load().apic_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_blob(self, blob: bytes):
        """Parameters from a BF16 checkpoint blob (apic_net_load; learn.bf16_blob writes one)."""
        _check(load().apic_net_load(self.handle, bytes(blob), len(blob)), "apic_net_load")

    def set_params(self, flat: np.ndarray):
        v = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load().apic_net_set_params(self.handle, v.ctypes.data_as(C.POINTER(C.c_float)), v.size),
               "apic_net_set_params")

    def get_params(self) -> np.ndarray:
        v = np.zeros(self.n_params, dtype=np.float32)
        _check(load().apic_net_get_params(self.handle, v.ctypes.data_as(C.POINTER(C.c_float)), v.size),
               "apic_net_get_params")
        return v

    def get_grads(self) -> np.ndarray:
        v = np.zeros(self.n_params, dtype=np.float32)
        _check(load().apic_net_get_grads(self.handle, v.ctypes.data_as(C.POINTER(C.c_float)), v.size),
               "apic_net_get_grads")
        return v

    def forward(self, batch, feat, uv, out=None, stream=None):
        _check(load().apic_net_forward(self.handle, int(batch), _ptr(feat), _ptr(uv), _ptr(out), _stream(stream)),
               "apic_net_forward")

    def backward(self, target, loss=None, stream=None):
        _check(load().apic_net_backward(self.handle, _ptr(target), _ptr(loss), _stream(stream)), "apic_net_backward")

    def adamw(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(load().apic_net_adamw(self.handle, float(lr), float(beta1), float(beta2), float(eps),
                                     float(weight_decay), int(step), _stream(stream)), "apic_net_adamw")

    def activation(self, which: int, batch: int) -> np.ndarray:
        shapes = {0: (64, 64, 32), 1: (32, 32, 64), 2: (16, 16, 128), 3: (8, 8, 256), 4: (258,), 5: (256,),
                  6: (12,)}
        out = np.zeros((batch,) + shapes[which], dtype=np.float32)
        _check(load().apic_net_activation(self.handle, int(which), out.ctypes.data_as(C.POINTER(C.c_float)),
                                          out.size), "apic_net_activation")
        return out
