#!/usr/bin/env python3
"""Throughput benchmark of the GB300 APIC library (one JSON line on stdout).

Default workload (one step, the mixed-precision configuration): 2048 tiles of
512 x 512 low-resolution pixels (the paper's patch size), 8 NA-matching + 24
darkfield images each (illumination NA 0.29 / 0.34 / 0.40), 0.25 NA, 0.52 um,
0.345 um pixels, 2x upsampling to 1024 x 1024, per-tile Zernike coefficients
varying as a 2-D quadratic across a 32 x 64 tile grid, Poisson noise at 1e4
photons per pixel; the sample is a smoothed random transmission (amplitude
0.8-1.0, phase 0-pi). Inputs are synthesised on the device before timing and
are far larger than L2 (68.7 GB of intensities per step).
--workload cfg2: 512 tiles of 256 x 256 with 8 + 16 images (NA 0.30 / 0.38).

value: output Mpx/s = tiles * 1024^2 * steps / timed seconds, all ranks.
e2e:   the same through host buffers (apic_reconstruct_host: pinned H2D of the
       intensities and D2H of the fields inside the timed region).
roofline: the darkfield kernel (the dominant one) against the measured FP32
       FMA rate of this GPU (apic_measure_fma_rate); hbm_frac: the step's
       algorithmic bytes (inputs + fields) over the step time against the
       measured HBM copy rate.
cpu_baseline: the float64 checker on a bounded sample of one tile of the same
       workload, on the host cores.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload cfg2|rgb|blend]
Multi-GPU (torchrun): each rank reconstructs its own tiles (weak scaling, no
collective on the data path); barrier + max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "APIC output Mpx/s at <=1e-3 rel L2 vs FP64 oracle; % of HBM roofline"
WORKLOADS = {
    # name: (tile, tiles, images, zernike grid rows x cols)
    "cfg3": (512, 2048, "8+24", (32, 64)),
    "cfg2": (256, 512, "8+16", (16, 32)),
}
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILES = os.path.join(ROOT, "profiles")
DEFAULT_DF_TOL = 3e-4          # the library's darkfield CG tolerance (apic_params.df_tol <= 0)
DF_SOURCES = {256: ["kernels_dfr.cu", "regfft.cuh", "common.cuh", "internal.cuh"],
              512: ["kernels_dfw.cu", "regfft.cuh", "t4grid.cuh", "common.cuh", "internal.cuh"]}
DF_KERNEL = {256: "k_darkfield_reg", 512: "k_darkfield_wide"}
HOST_E2E_RAM_FRAC = 0.45       # pinned host buffers of the end-to-end leg: at most this share of host RAM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["apic", "reference"], default="apic")
    ap.add_argument("--tiles", type=int, default=None, help="tiles per step (default: the workload's)")
    ap.add_argument("--tile", type=int, default=None, help="tile side (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-host-tiles", type=int, default=0,
                    help="tiles the end-to-end leg's pinned host buffers hold (0: the whole step if host RAM allows)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-assisted timing")
    ap.add_argument("--per-tile", type=int, default=32,
                    help="tiles timed one call at a time for the unbatched comparison (0: skip)")
    ap.add_argument("--images", choices=["8+16", "8+24", "12+22"], default=None,
                    help="illumination set (8+24: rings at NA 0.29 / 0.34 / 0.40; 12+22: the paper's set-up size, "
                         "darkfield rings at NA 0.31 / 0.375 / 0.44)")
    ap.add_argument("--workload", choices=["cfg3", "cfg2", "rgb", "blend", "learned", "slide"], default="cfg3",
                    help="cfg3: 2048 tiles of 512 x 512 with 8 + 24 images (default line); cfg2: 512 tiles of "
                         "256 x 256 with 8 + 16 images; rgb: the cfg2 batch at three wavelengths, one plan each; "
                         "blend: overlap blending of a 16 x 32 window grid with 6 %% overlap; learned: the network "
                         "trained on 20,000 tiles and evaluated on 4096 (30 %% near-blank); slide: a strip of the "
                         "whole-slide stream (512-pixel windows, 40 %% background)")
    ap.add_argument("--slide-rows", type=int, default=32)
    ap.add_argument("--slide-cols", type=int, default=64)
    ap.add_argument("--slide-overlap", type=float, default=0.0, help="window overlap fraction of the slide line")
    ap.add_argument("--slide-net", choices=["warm", "closed_form"], default="warm",
                    help="slide line: aberration network warm start (trained first) or the closed-form solve alone")
    ap.add_argument("--slide-train", type=int, default=20000, help="simulated 512-pixel tiles the slide network trains on")
    ap.add_argument("--seed", type=int, default=2407)
    ap.add_argument("--df-tol", type=float, default=0.0, help="CGLS tolerance (0: library default)")
    ap.add_argument("--df-iters", type=int, default=0, help="CGLS iteration cap (0: library default)")
    a = ap.parse_args()
    tile, tiles, images, grid = WORKLOADS["cfg2" if a.workload in ("cfg2", "rgb", "blend", "learned") else "cfg3"]
    a.tile = a.tile or tile
    a.tiles = a.tiles or tiles
    a.images = a.images or images
    a.zgrid = grid if a.tile == tile and a.tiles == tiles else (16, 32)
    return a


# ----------------------------------------------------------------------------- inputs

def field_zernike(rows=16, cols=32, seed=2407):
    """Per-tile Noll coefficients from a 2-D quadratic field over the tile grid."""
    from paper_2407_20469_gb300 import synth
    rng = np.random.default_rng(seed)
    table = synth.quadratic_field(rng, 1.0)
    uv = synth.tile_grid_uv(rows, cols)
    return np.stack([synth.coefficients_at(table, u, v) for u, v in uv]).astype(np.float32)


def device_objects(T, H, seed, device, sigma=4.0):
    """Smoothed random transmissions (amplitude 0.8-1.0, phase 0-pi), interleaved complex64."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    f = torch.fft.fftfreq(H, device=device)
    gauss = torch.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    out = torch.empty((T, H, 2 * H), dtype=torch.float32, device=device)
    for t0 in range(0, T, 64):
        t1 = min(T, t0 + 64)
        z = torch.randn((2, t1 - t0, H, H), device=device, generator=g)
        s = torch.fft.ifft2(torch.fft.fft2(z) * gauss).real
        lo = s.amin(dim=(-2, -1), keepdim=True)
        hi = s.amax(dim=(-2, -1), keepdim=True)
        s = (s - lo) / (hi - lo)
        amp = 0.8 + 0.2 * s[0]
        ph = math.pi * s[1]
        out[t0:t1] = torch.view_as_real(torch.polar(amp, ph)).reshape(t1 - t0, H, 2 * H)
    return out


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": min(sm),
                "power_w_median": statistics.median(pw) if pw else None}


# ----------------------------------------------------------------------------- reference arm

def oracle_tile_sample(n, images, seed, zgrid=(16, 32)):
    """One tile of the workload from the checker's forward model (float64 on the host)."""
    from oracle import forward, grid
    from paper_2407_20469_gb300 import synth
    ill = illumination_for(images)
    g = grid.Geometry(n, n, float(synth.NA), float(synth.WAVELENGTH_UM), float(synth.PIXEL_UM), 2)
    k = grid.snap_leds(ill.kx, ill.ky, ill.n_bf, g)
    rng = np.random.default_rng(seed)
    obj = synth.sample_object(rng, g.H, g.W, 4.0)
    c = field_zernike(*zgrid)[0].astype(np.float64)
    I = forward.intensity_stack(obj, g, k, c, photons=synth.PHOTONS, rng=rng).astype(np.float32)
    return I, g, k, ill


class OracleTile:
    """The float64 checker run on one tile in the paper's order, one piece at a time:
    the brightfield stages (Kramers-Kronig, aberration solve, stitch), then the
    darkfield solves one image at a time (each on the spectrum the previous ones
    left). Only oracle/ functions compute; this class times them."""

    def __init__(self, I, g, k, n_bf):
        from oracle import grid
        self.I, self.g, self.k, self.n_bf = I.astype(np.float64), g, k, n_bf
        self.order = [int(j) for j in grid.darkfield_order(k[n_bf:])]
        self.next = 0
        self.spec = None
        self.sizes = self._sizes()

    def _sizes(self):
        """(|U|, |Q|) of every darkfield image in order (geometry only: the known set
        grows by each used image's U)."""
        from oracle import grid
        from oracle import apic as oapic
        spec = oapic.Spectrum(self.g)
        for kb in self.k[:self.n_bf]:
            spec.put(grid.disc_points(self.g, kb), 1.0)
        out = []
        for j in self.order:
            kj = self.k[self.n_bf + j]
            sets = grid.darkfield_sets(grid.disc_points(self.g, kj), spec.known_set(), j, kj)
            out.append((len(sets.U), len(sets.Q)) if sets.used else (0, 0))
            if sets.used:
                spec.put(sets.U, 1.0)
        return out

    def brightfield(self):
        from oracle import apic as oapic
        t0 = time.perf_counter()
        g, k, nb = self.g, self.k, self.n_bf
        X = [oapic.kk_spectrum(self.I[i], k[i], g) for i in range(nb)]
        rows = oapic.overlap_rows(g, k[:nb])
        self.c15 = oapic.aberration_solve(oapic.phase_differences(X, rows), rows)
        self.spec = oapic.stitch_brightfield(X, g, k[:nb], self.c15)
        self.next = 0
        return time.perf_counter() - t0

    def darkfield_next(self):
        """Solves the next darkfield image; returns (build seconds, solve seconds, index in order)."""
        from oracle import apic as oapic
        from oracle import grid
        if self.spec is None or self.next >= len(self.order):
            self.brightfield()
        idx = self.next
        j = self.order[idx]
        self.next += 1
        kj = self.k[self.n_bf + j]
        t0 = time.perf_counter()
        sets = grid.darkfield_sets(grid.disc_points(self.g, kj), self.spec.known_set(), j, kj)
        if not sets.used:
            return time.perf_counter() - t0, 0.0, idx
        C, b, _ = oapic.darkfield_system(sets, self.I[self.n_bf + j], self.spec, self.g, self.c15)
        t1 = time.perf_counter()
        x = oapic.lstsq_normal(C, b)
        U = sets.U
        phiU = oapic.pupil_phase(self.g, self.c15, U[:, 0] + kj[0], U[:, 1] + kj[1])
        self.spec.put(U, x * np.exp(-1j * phiU))
        return t1 - t0, time.perf_counter() - t1, idx

    def tile_seconds(self, t_bf, measured):
        """Per-tile time: the brightfield stages plus every darkfield solve, measured ones
        as measured and the others estimated from them (the dense system build taken as
        constant per image - its cost is |Q| |P|, nearly the same for every image - and
        the normal-equation solve scaled by |U|^2 |Q|)."""
        builds = [b for b, _, _ in measured]
        rate = sum(s for _, s, _ in measured) / max(1e-300, sum(self.sizes[i][0] ** 2 * self.sizes[i][1]
                                                                for _, _, i in measured))
        done = {i: b + s for b, s, i in measured}
        total = t_bf
        for i, (N, M) in enumerate(self.sizes):
            if N == 0:
                continue
            total += done[i] if i in done else statistics.mean(builds) + rate * N * N * M
        return total


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_baseline(n, images, seed, zgrid, df_solves):
    """cpu_baseline dict: the checker on one tile of the workload, the brightfield stages
    and the first `df_solves` darkfield solves timed (all of them if df_solves <= 0)."""
    I, g, k, ill = oracle_tile_sample(n, images, seed, zgrid)
    ot = OracleTile(I, g, k, ill.n_bf)
    t_bf = ot.brightfield()
    count = len(ot.order) if df_solves <= 0 else min(df_solves, len(ot.order))
    measured = [ot.darkfield_next() for _ in range(count)]
    secs = ot.tile_seconds(t_bf, measured)
    work = t_bf + sum(b + s for b, s, _ in measured)
    est = "" if count == len(ot.order) else (f"; the other {len(ot.order) - count} solves estimated from the "
                                             f"measured one(s) (build time per image, solve time scaled by |U|^2 |Q|)")
    return {"value": (2 * n) ** 2 / secs / 1e6, "unit": "Mpx/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"1 tile of {n}x{n} ({images} images), numpy float64: brightfield stages and "
                      f"{count} of {len(ot.order)} darkfield solves timed ({work:.1f} s of CPU work){est}; "
                      f"tile time {secs:.1f} s",
            "tile_seconds": secs}


def reference_arm(args):
    """The float64 checker on the host cores. 256-pixel tiles: one whole tile per step.
    512-pixel tiles: one darkfield solve per step, in order on one tile (the brightfield
    stages of the tile run, timed, before the first step); value from the per-tile time
    of OracleTile.tile_seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.tile
    I, g, k, ill = oracle_tile_sample(n, args.images, args.seed, args.zgrid)
    ot = OracleTile(I, g, k, ill.n_bf)
    if n <= 256:
        def step():
            t0 = time.perf_counter()
            t_bf = ot.brightfield()
            meas = [ot.darkfield_next() for _ in range(len(ot.order))]
            return time.perf_counter() - t0, t_bf, meas
        for _ in range(args.warmup):
            step()
        runs = [step() for _ in range(args.steps)]
        times = [r[0] for r in runs]
        tile_s = statistics.mean(times)
        sample = f"1 whole tile of {n}x{n} ({args.images} images) per step"
    else:
        t_bf = ot.brightfield()
        for _ in range(args.warmup):
            ot.darkfield_next()
        meas, times = [], []
        for _ in range(args.steps):
            if ot.next >= len(ot.order):
                t_bf = ot.brightfield()
            t0 = time.perf_counter()
            meas.append(ot.darkfield_next())
            times.append(time.perf_counter() - t0)
        tile_s = ot.tile_seconds(t_bf, meas)
        sample = (f"one darkfield solve per step, in order on one {n}x{n} tile ({args.images} images); "
                  f"per-tile time {tile_s:.1f} s = brightfield stages {t_bf:.1f} s + the {len(ot.order)} solves "
                  f"(measured or estimated from the measured ones)")
    value = (2 * n) ** 2 / tile_s / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpx/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.tiles, n, 2 * n, args.images, args.zgrid), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Mpx/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def fft2_flops(a, b):
    """Algorithmic flops of one complex a x b 2-D FFT: 5 N log2 N, N = a b."""
    N = a * b
    return 5.0 * N * math.log2(N)


def df_flops(plan, n):
    """Per used darkfield image: (setup flops per solve, flops per CG iteration), dense-grid counts.

    Setup: for 512-pixel tiles the known field's inverse and the forward transform of
    I - |p|^2 on the camera grid (two); otherwise the image's n x n transform and P * P
    (two transforms on the register grid); then the known field and C^H b on the
    image's grid (three). Per CG iteration C d and C^H r (four transforms on the
    image's grid)."""
    m = plan.info.fft_m
    out = []
    for i in range(plan.info.n_df):
        _, meta = plan.df_set(i, 0)
        if not meta[1]:
            continue
        _, mx, my = plan.df_grid(i)
        mx, my = (mx or m), (my or m)
        rhs = 2 * fft2_flops(n, n) if n == 512 else fft2_flops(n, n) + 2 * fft2_flops(m, m)
        out.append((rhs + 3 * fft2_flops(mx, my), 4 * fft2_flops(mx, my)))
    return out


def source_sha(n):
    """Hash of the darkfield kernel's code (comments and whitespace left out, so that
    only a code change invalidates the recorded counters)."""
    h = hashlib.sha256()
    for f in DF_SOURCES[512 if n == 512 else 256]:
        with open(os.path.join(ROOT, "paper_2407_20469_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_counters(n, T, images, tol, iters):
    """ncu figures of the darkfield kernel recorded under profiles/ for this workload and
    this kernel source, or {}: DRAM bytes per launch (scaled to the bench's launch) and
    the FMA-pipe share (executed work)."""
    path = os.path.join(PROFILES, f"darkfield_counters_{n}.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        tr = json.load(fh)
    if (tr.get("source_sha") != source_sha(n) or tr.get("tile") != n or tr.get("images") != images
            or abs(tr.get("df_tol", 0) - tol) > 1e-12 or iters):
        return {}
    out = {}
    if tr.get("dram_bytes_per_tile"):
        out["traffic"] = tr["dram_bytes_per_tile"] * T
    if tr.get("fma_pipe_frac") is not None:
        out["frac_executed"] = tr["fma_pipe_frac"]
    return out


def workload_name(T, n, H, images, zgrid):
    na = {"8+16": "NA 0.30/0.38", "8+24": "NA 0.29/0.34/0.40", "12+22": "NA 0.31/0.375/0.44"}[images]
    return (f"{T} tiles x {n}x{n} low-res ({H}x{H} output), {images} images (darkfield {na}), quadratic "
            f"field-dependent Zernike over a {zgrid[0]}x{zgrid[1]} tile grid, Poisson 1e4 photons/px")


def measured_peaks():
    """(HBM GB/s, kind) from MEASURED_PEAKS.json, else the recipe's fallback."""
    if os.path.exists(PEAKS):
        with open(PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    return 6800.0, "fallback"


def learned_timing(args, plan, ill, T, n, H, I, field, zern, status, device):
    """Mpx/s of apic_reconstruct_learned (APIC_NET_WARM) with a briefly trained network."""
    import torch
    from paper_2407_20469_gb300 import apic, learn
    bf = apic.Plan(n, ill.kx[:ill.n_bf], ill.ky[:ill.n_bf], ill.n_bf, max_tiles=256)
    t0 = time.perf_counter()
    feat, uv, zt, _ = learn.dataset(bf, 4096, args.seed, learn.field_table(), blank_frac=0.3)
    net = apic.Net(T)
    net.set_params(learn.init_params(args.seed))
    hist = learn.train(net, feat, uv, zt, epochs=4, batch=64, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del feat, uv, zt
    bf.close()
    uv = torch.as_tensor(np.resize(learn.tile_positions(16, 32), (T, 2)), device=device)
    for _ in range(args.warmup):
        plan.reconstruct_learned(net, apic.APIC_NET_WARM, T, I, uv, field, zern, None, status)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.reconstruct_learned(net, apic.APIC_NET_WARM, T, I, uv, field, zern, None, status)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = status.cpu().numpy()
    net.close()
    return {"value": T * H * H * args.steps / (ms / 1e3) / 1e6, "unit": "Mpx/s", "mode": "APIC_NET_WARM",
            "ms_per_step": ms / args.steps, "train_s": train_s, "train_tiles": 4096, "train_epochs": 4,
            "final_loss": hist[-1], "warm_kept_tiles": int(np.count_nonzero(st & apic.APIC_TILE_WARM))}


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    from paper_2407_20469_gb300 import apic, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        if rank == 0:
            build.build()
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
    else:
        build.build()
    device = torch.device("cuda", torch.cuda.current_device())

    n, T = args.tile, args.tiles
    ill = illumination_for(args.images)
    plan = apic.Plan.from_illumination(n, ill, max_tiles=T, df_tol=args.df_tol, df_iters=args.df_iters)
    info = plan.info
    H = info.out_h
    n_img = info.n_bf + info.n_df

    # ---- inputs (device), outside the timed region
    zern_true = torch.from_numpy(np.resize(field_zernike(*args.zgrid), (T, 15))).to(device)
    I = torch.empty((T, n_img, n, n), dtype=torch.float32, device=device)
    for t0 in range(0, T, 256):         # objects in slices: (2n)^2 complex values per tile
        t1 = min(T, t0 + 256)
        obj = device_objects(t1 - t0, H, args.seed + 7919 * rank + t0, device)
        plan.simulate(t1 - t0, obj, zern_true[t0:t1], synth.PHOTONS, args.seed + rank + t0, I[t0:t1])
        del obj
    field = torch.empty((T, H, 2 * H), dtype=torch.float32, device=device)
    zern = torch.empty((T, 15), dtype=torch.float32, device=device)
    status = torch.empty((T,), dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    # roofline denominators measured on this GPU (before the timed region)
    fp32_peak = apic.measure_fma_rate(32) / 1e12
    fp64_peak = apic.measure_fma_rate(64) / 1e12
    sms = torch.cuda.get_device_properties(device).multi_processor_count

    for _ in range(args.warmup):
        plan.reconstruct_batch(T, I, field, zern, None, status)
    torch.cuda.synchronize()
    plan.timing(True)
    plan.stage_ms(reset=True)
    plan.counters(reset=True)

    clocks = ClockSampler(clock_id(device))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.5)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.reconstruct_batch(T, I, field, zern, None, status)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stage, calls = plan.stage_ms(reset=True)
    cnt = plan.counters(reset=True)
    plan.timing(False)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    status_np = status.cpu().numpy()

    # ---- the same library called one tile at a time (no batching, no persistence
    # across tiles): what the batched launch buys on this workload
    per_tile = None
    if args.per_tile > 0:
        k = min(args.per_tile, T)
        plan.reconstruct_batch(1, I[0:1], field[0:1], zern[0:1], None, status[0:1])
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for t in range(k):
            plan.reconstruct_batch(1, I[t:t + 1], field[t:t + 1], zern[t:t + 1], None, status[t:t + 1])
        c1.record(stream)
        torch.cuda.synchronize()
        pt_ms = c0.elapsed_time(c1)
        pt_value = k * H * H / (pt_ms / 1e3) / 1e6
        per_tile = {"value": pt_value, "unit": "Mpx/s", "tiles": k, "ms_per_tile": pt_ms / k,
                    "batched_over_per_tile": None}

    # ---- learned-assisted reconstruction on the same inputs, for tiles of up to 256 pixels
    # (the slide line trains and times its own 512-pixel network): a network trained here
    # for a few seconds on simulated tiles, warm-starting the aberration solve (features +
    # network forward + second refinement inside the timing)
    learned = None
    if not args.no_learned and n <= 256:
        learned = learned_timing(args, plan, ill, T, n, H, I, field, zern, status, device)

    # ---- end to end through host buffers: apic_reconstruct_host pipelines the pinned
    # host->device copies, the reconstruction and the device->host copies. The pinned
    # buffers hold the whole step when that fits HOST_E2E_RAM_FRAC of the host's RAM
    # (86 GB for 2048 512-pixel tiles); otherwise a step is several calls over
    # consecutive tile ranges, each copying its inputs in and its fields out.
    e2e = None
    if args.e2e_steps > 0:
        per_tile_bytes = n_img * n * n * 4 + H * H * 8
        try:
            ram = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        except (ValueError, OSError, AttributeError):
            ram = 0
        Th = max(1, min(T, int(HOST_E2E_RAM_FRAC * ram // per_tile_bytes))) if ram else min(T, 512)
        if args.e2e_host_tiles > 0:
            Th = min(Th, args.e2e_host_tiles)
        while True:          # a pinned allocation the host refuses: halve the buffers
            try:
                I_host = torch.empty((Th,) + tuple(I.shape[1:]), dtype=torch.float32, pin_memory=True)
                f_host = torch.empty((Th,) + tuple(field.shape[1:]), dtype=torch.float32, pin_memory=True)
                break
            except RuntimeError:
                I_host = f_host = None
                if Th == 1:
                    raise
                Th = max(1, Th // 2)
        I_host.copy_(I[:Th])
        z_host = torch.empty((Th, 15), dtype=torch.float32, pin_memory=True)
        s_host = torch.empty((Th,), dtype=torch.int32, pin_memory=True)
        del I
        torch.cuda.synchronize()
        chunks = [(a, min(T, a + Th)) for a in range(0, T, Th)]
        plan.reconstruct_host(Th, I_host, f_host, z_host, s_host)      # first call sets up the pipeline
        # host link bandwidth for context: one pinned host->device copy of the inputs
        probe = torch.empty(I_host.shape, dtype=torch.float32, device=device)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record()
        probe.copy_(I_host, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        h2d_gbs = I_host.numel() * 4 / (c0.elapsed_time(c1) / 1e3) / 1e9
        c0.record()
        f_host.copy_(probe.view(-1)[:f_host.numel()].view(f_host.shape), non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        d2h_gbs = f_host.numel() * 4 / (c0.elapsed_time(c1) / 1e3) / 1e9
        del probe
        if world > 1:
            dist.barrier()
        step_ms = []
        e2e_clocks = ClockSampler(clock_id(device))
        e2e_clocks.start()
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            for a, b in chunks:
                plan.reconstruct_host(b - a, I_host, f_host, z_host, s_host)
            step_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_clk = e2e_clocks.stop()
        ems = sum(step_ms)
        if world > 1:
            t = torch.tensor([ems], dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        per_tile_in = I_host[0].numel() * 4
        per_tile_out = f_host[0].numel() * 4 + 15 * 4 + 4
        e2e = {"value": world * T * H * H * args.e2e_steps / (ems / 1e3) / 1e6, "unit": "Mpx/s",
               "h2d_bytes_per_step": int(T * per_tile_in), "d2h_bytes_per_step": int(T * per_tile_out),
               "steps": args.e2e_steps,
               "api": f"apic_reconstruct_host (pinned host buffers of {Th} tiles, {len(chunks)} call(s) per step)",
               "h2d_gbs_measured": h2d_gbs, "d2h_gbs_measured": d2h_gbs,
               "step_ms": [round(v, 2) for v in step_ms], "step_ms_median": statistics.median(step_ms),
               "clocks": e2e_clk}
        del I_host, f_host, z_host, s_host

    # ---- roofline of the darkfield kernel: dense-grid algorithmic flops of its launches
    # (per image: setup per solve + CG iterations x per-iteration flops) over their live
    # event time, against the measured FP32 FMA rate
    df_ms = stage["darkfield"] / max(calls, 1)
    per_img = df_flops(plan, n)
    iters_img = cnt["cg_iterations_per_image"]
    solves_per_img = cnt["df_solves"] / max(1, len(per_img))
    flops = sum(solves_per_img * s + it * p for (s, p), it in zip(per_img, iters_img)) / max(calls, 1)
    achieved = flops / (df_ms / 1e3) / 1e12
    tol = args.df_tol if args.df_tol > 0 else DEFAULT_DF_TOL
    rec = recorded_counters(n, T, args.images, tol, args.df_iters)
    hbm_gbs, hbm_kind = measured_peaks()
    bytes_per_step = T * (n_img * n * n * 4 + H * H * 8)
    roofline = {"bound": "alu", "kernel": DF_KERNEL[512 if n == 512 else 256], "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": rec.get("traffic"),
                "peak_kind": f"measured FP32 FMA rate of this GPU (apic_measure_fma_rate; {sms} SMs)",
                "flops_kind": "dense-grid count: 5 N log2 N per 2-D transform of each image's own grid; the kernel "
                              "transforms only band rows, so it executes fewer",
                "frac_executed": rec.get("frac_executed"),
                "fp64_peak_tflops": fp64_peak,
                "launch_ms": df_ms, "cg_iterations_per_launch": cnt["cg_iterations"] / max(calls, 1),
                "solves_per_launch": cnt["df_solves"] / max(calls, 1),
                "stage_ms_per_step": {k: v / max(calls, 1) for k, v in stage.items()},
                "hbm_frac": bytes_per_step / (ms / args.steps / 1e3) / (hbm_gbs * 1e9),
                "hbm_frac_kind": f"algorithmic bytes per step (intensities in + fields out, "
                                 f"{bytes_per_step / 1e9:.1f} GB) / step time / {hbm_gbs:.0f} GB/s {hbm_kind}"}

    value = world * T * H * H * args.steps / (ms / 1e3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mpx/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(T, n, H, args.images, args.zgrid), "tiles_per_gpu": T, "tile": n,
                   "output": H, "images": n_img,
                   "l2": f"inputs_larger_than_l2 ({T * n_img * n * n * 4 / 1e9:.1f} GB intensities per step)",
                   "launch": "direct C-ABI calls", "tiles_per_s": world * T * args.steps / (ms / 1e3),
                   "df_tol": args.df_tol or "library default", "fft_m": info.fft_m,
                   "precision": "FFTs, elementwise math and CG vectors FP32; aberration normal equations and "
                                "darkfield CG step lengths / cross-warp sums FP64",
                   "tiles_status_nonzero": int(np.count_nonzero(status_np))},
        "roofline": roofline, "e2e": e2e, "gpu_launches": cnt["launches"], "clocks": clk,
    }
    if learned is not None:
        line["learned"] = learned
    if per_tile is not None:
        per_tile["batched_over_per_tile"] = value / per_tile["value"]
        line["per_tile_calls"] = per_tile
    plan.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(n, args.images, args.seed, args.zgrid, 1 if n > 256 else 0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def illumination_for(images):
    from paper_2407_20469_gb300 import synth
    return {"8+16": synth.illumination, "8+24": synth.illumination_8_24,
            "12+22": synth.illumination_12_22}[images]()


def clock_id(device):
    import torch
    props = torch.cuda.get_device_properties(device)
    uuid = str(getattr(props, "uuid", ""))
    return ("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or str(device.index))


def timed(fn, steps, device):
    """(ms over `steps` calls of fn on the current stream, clock record), after a synchronize."""
    import torch
    clocks = ClockSampler(clock_id(device))
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.5)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), clocks.stop()


RGB_UM = (0.47, 0.52, 0.63)


def rgb_arm(args):
    """The batch workload at three wavelengths (one plan per colour, kept): one step reconstructs
    every tile in every channel. Darkfield roofline summed over the channels' launches."""
    import torch
    from paper_2407_20469_gb300 import apic, build, channels, synth
    build.build()
    device = torch.device("cuda", torch.cuda.current_device())
    n, T = args.tile, args.tiles
    cp = channels.ChannelPlans(n, RGB_UM, max_tiles=T)
    C = len(RGB_UM)
    info = cp.plan(RGB_UM[0]).info
    H = info.out_h
    zern_true = torch.from_numpy(np.resize(field_zernike(*args.zgrid), (T, 15))).to(device)
    I, F, Z, S = [], [], [], []
    for c, w in enumerate(RGB_UM):
        p = cp.plan(w)
        obj = device_objects(T, H, args.seed + 7919 * c, device)
        x = torch.empty((T, p.info.n_bf + p.info.n_df, n, n), dtype=torch.float32, device=device)
        p.simulate(T, obj, zern_true, synth.PHOTONS, args.seed + c, x)
        del obj
        I.append(x)
        F.append(torch.empty((T, H, 2 * H), dtype=torch.float32, device=device))
        Z.append(torch.empty((T, 15), dtype=torch.float32, device=device))
        S.append(torch.empty((T,), dtype=torch.int32, device=device))
    step = lambda: cp.reconstruct(T, I, F, Z, S)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for w in RGB_UM:
        cp.plan(w).timing(True)
        cp.plan(w).stage_ms(reset=True)
        cp.plan(w).counters(reset=True)
    fp32_peak = apic.measure_fma_rate(32) / 1e12
    ms, clk = timed(step, args.steps, device)
    df_ms = flops = launches = 0.0
    per_channel = {}
    for w in RGB_UM:
        p = cp.plan(w)
        stage, calls = p.stage_ms(reset=True)
        cnt = p.counters(reset=True)
        p.timing(False)
        per_img = df_flops(p, n)
        spi = cnt["df_solves"] / max(1, len(per_img))
        f = sum(spi * a + it * b for (a, b), it in zip(per_img, cnt["cg_iterations_per_image"])) / max(calls, 1)
        d = stage["darkfield"] / max(calls, 1)
        df_ms += d
        flops += f
        launches += cnt["launches"]
        per_channel[str(w)] = {"darkfield_ms_per_step": d, "cg_iterations_per_step": cnt["cg_iterations"] / max(calls, 1),
                               "fft_m": p.info.fft_m, "n_df_used": p.info.n_df_used}
    achieved = flops / (df_ms / 1e3) / 1e12
    st = np.concatenate([s.cpu().numpy() for s in S])
    value = C * T * H * H * args.steps / (ms / 1e3) / 1e6
    line = {
        "metric": "APIC output Mpx/s over all colour channels", "value": value, "unit": "Mpx/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{T} tiles x {n}x{n} low-res ({H}x{H} output) at {C} wavelengths "
                               f"{list(RGB_UM)} um, 8+16 images each, one plan per wavelength",
                   "channels": C, "tiles_per_channel": T, "l2": "inputs_larger_than_l2",
                   "tiles_status_nonzero": int(np.count_nonzero(st)), "per_channel": per_channel},
        "roofline": {"bound": "alu", "kernel": "k_darkfield_reg", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_kind": "measured FP32 FMA rate of this GPU (apic_measure_fma_rate)",
                     "launch_ms": df_ms},
        "e2e": None, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    cp.close()


def blend_bytes(windows, u, L, out_px):
    """Algorithmic bytes of one apic_blend_fields call: every window's field read once, the slide
    field (out_px pixels) written once, and the overlap strips with the left / upper neighbour read
    (both sides) by the correlation pass, complex64."""
    rows = int(np.sum(windows[:, 1] == windows[0, 1]))
    cols = len(windows) // rows
    ov = 0
    for k in range(len(windows)):
        for nb in ((k - 1) if k % cols else -1, (k - cols) if k >= cols else -1):
            if nb < 0:
                continue
            dy = L - abs(u * int(windows[k, 0]) - u * int(windows[nb, 0]))
            dx = L - abs(u * int(windows[k, 1]) - u * int(windows[nb, 1]))
            if dy > 0 and dx > 0:
                ov += 2 * dy * dx
    return 8 * (len(windows) * L * L + out_px + ov)


def blend_arm(args):
    """Overlap blending of a 16 x 32 grid of windows with 6 % overlap (the paper's scan overlap):
    correlations, phase chain and the weighted sum, one apic_blend_fields call per step."""
    import torch
    from paper_2407_20469_gb300 import apic, build, slide, synth
    build.build()
    device = torch.device("cuda", torch.cuda.current_device())
    n = args.tile
    rows, cols = 16, 32
    stride = n - int(round(0.06 * n))
    Hs, Ws = (rows - 1) * stride + n, (cols - 1) * stride + n
    plan = apic.Plan.from_illumination(n, synth.illumination(), max_tiles=1)
    u = plan.info.out_h // n
    L = u * n
    win = apic.slide_windows(Hs, Ws, n, stride)
    assert len(win) == rows * cols
    g = torch.Generator(device=device).manual_seed(args.seed)
    fields = torch.randn((len(win), L, 2 * L), device=device, generator=g)
    out, corr, phase = slide.blend_slide(plan, fields, win, Hs, Ws)      # buffers, and the first call
    win_d = torch.as_tensor(win, device=device)
    step = lambda: plan.blend_fields(len(win), fields, win_d, rows, cols, Hs, Ws, corr, phase, out)
    for _ in range(args.warmup):
        step()
    ms, clk = timed(step, args.steps, device)
    nbytes = blend_bytes(win, u, L, u * u * Hs * Ws)
    achieved = nbytes / (ms / args.steps / 1e3) / 1e9
    peak, kind = 6800.0, "fallback"
    if os.path.exists(PEAKS):
        with open(PEAKS) as fh:
            peak, kind = float(json.load(fh)["hbm_gbs"]), "measured"
    value = u * u * Hs * Ws * args.steps / (ms / 1e3) / 1e6
    line = {
        "metric": "blended slide output Mpx/s", "value": value, "unit": "Mpx/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{rows}x{cols} windows of {n}x{n} ({L}x{L} output fields), stride {stride} "
                               f"(6 % overlap), slide {Hs}x{Ws} low-res",
                   "l2": f"inputs_larger_than_l2 ({len(win) * L * L * 8 / 1e9:.2f} GB of fields)",
                   "finite": bool(torch.isfinite(out).all().item())},
        "roofline": {"bound": "hbm", "kernel": "apic_blend_fields (k_blend_corr + k_blend_phases + k_blend_pairs)",
                     "achieved": achieved, "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "algorithmic_bytes_per_call": nbytes},
        "e2e": None, "gpu_launches": 3 * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def learned_arm(args):
    """The learned-aberration configuration: the network trained on 20,000 simulated tiles of
    256 x 256 (30 % near-blank), then 4096 fresh tiles (30 % near-blank) reconstructed with the
    closed-form aberration solve, with the network's warm start, and with warm start plus
    replacement on low-contrast tiles; the pupil error of each against the true coefficients,
    per class, and the output rate of each."""
    import torch
    from paper_2407_20469_gb300 import apic, build, learn, synth
    build.build()
    device = torch.device("cuda", torch.cuda.current_device())
    n, n_train, n_eval, blank_frac = 256, 20000, 4096, 0.3
    ill = synth.illumination()
    table = learn.field_table(args.seed)
    bf = apic.Plan(n, ill.kx[:ill.n_bf], ill.ky[:ill.n_bf], ill.n_bf, max_tiles=256)
    t0 = time.perf_counter()
    feat, uv, zt, _ = learn.dataset(bf, n_train, args.seed, table, blank_frac=blank_frac)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = apic.Net(256)
    net.set_params(learn.init_params(args.seed))
    hist = learn.train(net, feat, uv, zt, epochs=8, batch=64, lr=3e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del feat, uv, zt
    bf.close()
    plan = apic.Plan.from_illumination(n, ill, max_tiles=n_eval, bg_contrast=0.02)
    H = plan.info.out_h
    uv_e, z_true, blank = learn.draw_tiles(n_eval, args.seed + 1, table, blank_frac)
    I = learn.simulate(plan, z_true, blank, args.seed + 1)
    uv_d = torch.as_tensor(uv_e, device=device)
    field = torch.empty((n_eval, H, 2 * H), dtype=torch.float32, device=device)
    zern = torch.empty((n_eval, 15), dtype=torch.float32, device=device)
    status = torch.empty((n_eval,), dtype=torch.int32, device=device)
    modes = {"closed_form": None, "warm": apic.APIC_NET_WARM,
             "warm_and_replace": apic.APIC_NET_WARM | apic.APIC_NET_REPLACE}
    out, clk = {}, None
    for name, mode in modes.items():
        if mode is None:
            step = lambda: plan.reconstruct_batch(n_eval, I, field, zern, None, status)
        else:
            step = lambda m=mode: plan.reconstruct_learned(net, m, n_eval, I, uv_d, field, zern, None, status)
        for _ in range(args.warmup):
            step()
        plan.counters(reset=True)
        ms, clk = timed(step, args.steps, device)
        cnt = plan.counters(reset=True)
        z = zern.cpu().numpy().astype(np.float64)
        st = status.cpu().numpy()
        d = z[:, 3:] - z_true[:, 3:].astype(np.float64)
        err = np.sqrt((d * d).sum(axis=1))
        out[name] = {"Mpx_s": n_eval * H * H * args.steps / (ms / 1e3) / 1e6, "ms_per_step": ms / args.steps,
                     "pupil_rms_median_rad": {"background": float(np.median(err[blank])),
                                              "sample": float(np.median(err[~blank]))},
                     "pupil_rms_p90_rad": {"background": float(np.percentile(err[blank], 90)),
                                           "sample": float(np.percentile(err[~blank], 90))},
                     "cg_iterations_per_solve": cnt["cg_iterations"] / max(1, cnt["df_solves"]),
                     "tiles_notconv": int(np.count_nonzero(st & apic.APIC_TILE_NOTCONV)),
                     "tiles_learned": int(np.count_nonzero(st & apic.APIC_TILE_LEARNED)),
                     "tiles_warm_kept": int(np.count_nonzero(st & apic.APIC_TILE_WARM))}
    best = out["warm_and_replace"]
    line = {
        "metric": "APIC output Mpx/s with the learned aberration network (warm start + replacement on low-contrast "
                  "tiles); pupil error vs the true coefficients per class",
        "value": best["Mpx_s"], "unit": "Mpx/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": best["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (network bf16, FP32 accumulate)", "data": "synthetic",
        "config": {"workload": f"network trained on {n_train} simulated tiles of {n}x{n} ({int(100 * blank_frac)} % "
                               f"near-blank, contrast < 2 %), evaluated on {n_eval} fresh tiles of {n}x{n} "
                               f"(8 + 16 images, {int(blank.sum())} near-blank); field-dependent quadratic Zernike "
                               f"table plus per-tile defocus jitter",
                   "train": {"tiles": n_train, "epochs": 8, "batch": 64, "dataset_s": t1 - t0, "train_s": t2 - t1,
                             "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]},
                   "modes": out, "l2": "inputs_larger_than_l2"},
        "roofline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    net.close()
    plan.close()


def slide_arm(args):
    """Whole-slide stream: a contiguous strip of a 76.2 x 25.4 mm slide at 10x / 0.25 NA
    (0.345 um pixels: the slide is 220,870 x 73,623 low-res pixels, about 20,000 windows of 512),
    cut into 512-pixel windows, 40 % of them background (blob-shaped tissue mask over the window
    grid), 8 + 24 images; one step = cut, reconstruct (background windows skipped by the contrast
    test) and paste the whole strip. The strip's stacks are simulated window by window (each on
    its own periodic grid), so windows that overlap would see their neighbours' simulations at
    their edges; by default the windows therefore tile the strip without overlap
    (--slide-overlap gives the overlap fraction; overlap blending has its own line). With the
    learned warm start (default) the aberration network is first trained on --slide-train
    simulated 512-pixel tiles (random positions, 40 % near-blank), outside the timed region."""
    import torch
    from paper_2407_20469_gb300 import apic, build, learn, slide, synth
    build.build()
    device = torch.device("cuda", torch.cuda.current_device())
    n, rows, cols = 512, args.slide_rows, args.slide_cols
    stride = n - int(round(args.slide_overlap * n))
    Hs, Ws = (rows - 1) * stride + n, (cols - 1) * stride + n
    ill = illumination_for("8+24")
    batch = 1024
    plan = apic.Plan.from_illumination(n, ill, max_tiles=batch, bg_contrast=0.02, flags=apic.APIC_SKIP_BACKGROUND)
    info = plan.info
    H = info.out_h
    n_img = info.n_bf + info.n_df
    win = apic.slide_windows(Hs, Ws, n, stride)
    assert len(win) == rows * cols
    # tissue mask over the window grid: a smooth random field, its lowest 40 % background
    rng = np.random.default_rng(args.seed)
    f = np.fft.fftfreq(rows)[:, None] ** 2 + np.fft.fftfreq(cols)[None, :] ** 2
    fld = np.real(np.fft.ifft2(np.fft.fft2(rng.standard_normal((rows, cols))) * np.exp(-f * 60.0)))
    blank = (fld <= np.quantile(fld, 0.4)).ravel()
    table = learn.field_table(args.seed)
    uv = slide.window_positions(win, Hs, Ws, n)
    zern = learn.coefficients(table, uv)
    I_slide = torch.zeros((n_img, Hs, Ws), dtype=torch.float32, device=device)
    for t0 in range(0, len(win), 152):
        t1 = min(len(win), t0 + 152)
        I = learn.simulate(plan, zern, blank, args.seed, start=t0, count=t1 - t0)
        for k in range(t1 - t0):
            y0, x0 = int(win[t0 + k, 0]), int(win[t0 + k, 1])
            I_slide[:, y0:y0 + n, x0:x0 + n] = I[k]
        del I
    torch.cuda.synchronize()
    net, train_s = None, None
    if args.slide_net == "warm":
        t0 = time.perf_counter()
        bf = apic.Plan(n, ill.kx[:ill.n_bf], ill.ky[:ill.n_bf], ill.n_bf, max_tiles=256)
        feat, uv_t, z_t, _ = learn.dataset(bf, args.slide_train, args.seed + 2, table, blank_frac=0.4)
        bf.close()
        net = apic.Net(256)
        net.set_params(learn.init_params(args.seed))
        learn.train(net, feat, uv_t, z_t, epochs=8, batch=64, lr=3e-3)
        del feat, uv_t, z_t
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
    step = lambda m=apic.APIC_NET_WARM: slide.reconstruct_slide(plan, I_slide, Hs, Ws, stride, batch=batch,
                                                                net=net, mode=m)
    for _ in range(args.warmup):
        res = step()
    plan.counters(reset=True)
    plan.timing(True)
    plan.stage_ms(reset=True)
    ms, clk = timed(step, args.steps, device)
    cnt = plan.counters(reset=True)
    stage, calls = plan.stage_ms(reset=True)
    plan.timing(False)
    out_f, z, st, _ = step()
    st = st.cpu().numpy()
    skipped = int(np.count_nonzero(st & apic.APIC_TILE_BACKGROUND))
    solved = (st & apic.APIC_TILE_BACKGROUND) == 0

    def pupil_err(zz):
        d = zz.cpu().numpy().astype(np.float64)[:, 3:] - zern[:, 3:].astype(np.float64)
        e = np.sqrt((d * d).sum(axis=1))[solved]
        return {"median": float(np.median(e)), "p90": float(np.percentile(e, 90))} if e.size else None

    pupil = {"this_run": pupil_err(z)}
    if net is not None:
        pupil["closed_form_alone"] = pupil_err(slide.reconstruct_slide(plan, I_slide, Hs, Ws, stride, batch=batch)[1])
        pupil["warm_kept"] = int(np.count_nonzero(st & apic.APIC_TILE_WARM))
    sec = ms / args.steps / 1e3
    slide_px = 4.0 * Hs * Ws
    line = {
        "metric": "whole-slide APIC output Mpx/s (slide area, background windows skipped)",
        "value": slide_px / sec / 1e6, "unit": "Mpx/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"strip of {rows} x {cols} windows of {n}x{n} (stride {stride}, "
                               f"{100 * args.slide_overlap:.0f} % overlap; "
                               f"{Hs} x {Ws} low-res px = {Hs * 0.345e-3:.2f} x {Ws * 0.345e-3:.2f} mm of the "
                               f"76.2 x 25.4 mm slide, {100.0 * rows * cols / 20000:.0f} % of its ~20,000 windows), "
                               f"8 + 24 images, {int(blank.sum())} background windows ({100 * blank.mean():.0f} %), "
                               f"paste of each window's owned part",
                   "windows": rows * cols, "windows_per_s": rows * cols / sec,
                   "reconstructed_windows": rows * cols - skipped, "skipped_background": skipped,
                   "reconstructed_tiles_per_s": (rows * cols - skipped) / sec,
                   "reconstructed_output_Mpx_s": (rows * cols - skipped) * H * H / sec / 1e6,
                   "batch": batch, "l2": f"inputs_larger_than_l2 ({n_img * Hs * Ws * 4 / 1e9:.1f} GB slide stack)",
                   "cg_iterations_per_solve": cnt["cg_iterations"] / max(1, cnt["df_solves"]),
                   "tiles_notconv": int(np.count_nonzero(st & apic.APIC_TILE_NOTCONV)),
                   "stage_ms_per_step": {k: v / max(1, args.steps) for k, v in stage.items()},
                   "output_finite": bool(torch.isfinite(out_f).all().item()),
                   "learned_warm_start": (f"network trained on {args.slide_train} simulated 512-pixel tiles in "
                                          f"{train_s:.1f} s (outside the timed region)" if net is not None
                                          else "not used (--slide-net closed_form)"),
                   "pupil_rms_rad_reconstructed_windows": pupil},
        "roofline": None, "e2e": None, "gpu_launches": cnt["launches"] // max(1, args.steps), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "rgb":
        rgb_arm(args)
    elif args.workload == "blend":
        blend_arm(args)
    elif args.workload == "learned":
        learned_arm(args)
    elif args.workload == "slide":
        slide_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
