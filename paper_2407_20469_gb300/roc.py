"""Calibration of the background skip (Sec. 3.2) against a CNN classifier.

Sec. 3.2 skips a patch as background when the variation of its low-resolution
images falls below a threshold, and gives no value for that threshold. The
library's statistic (apic_background) is the mean over the NA-matching images
of var(I) / mean(I)^2, and a tile is background below bg_contrast^2. This
module measures how well the statistic separates near-blank tiles (contrast
below 2 %) from sample tiles, next to a classifier with the aberration
network's architecture and input features (apic_net_*), trained to put 1 on
background and 0 on sample in its first output (the Noll 4 slot). For each it
reports the ROC, the area under it, and the operating point under a bound on
the fraction of sample tiles skipped (the costly error: lost tissue).

Background is the positive class: "false positive rate" = sample tiles
skipped, "true positive rate" = background tiles skipped (work saved). Every
per-tile number comes from the library's kernels (simulation, statistic,
features, network); this module draws the tiles and sorts scores.

    python -m paper_2407_20469_gb300.roc [--tile 256 --train 20000 --eval 4096]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import apic, learn, synth

FAINT_RANGE = (0.03, 1.0)          # faint tissue: contrast factor log-uniform in this range


def roc(score, positive):
    """ROC of the rule 'positive when score >= t' over every threshold t.

    Returns (fpr, tpr, thresholds), thresholds descending from +inf (the point
    (0, 0)); tiles with equal scores change class together. Raises ValueError
    without both classes."""
    s = np.asarray(score, dtype=np.float64).ravel()
    y = np.asarray(positive, dtype=bool).ravel()
    n_pos, n_neg = int(y.sum()), int((~y).sum())
    if n_pos == 0 or n_neg == 0:
        raise ValueError("an ROC needs tiles of both classes")
    if not np.all(np.isfinite(s)):
        raise ValueError("scores must be finite")
    order = np.argsort(-s, kind="mergesort")
    s, y = s[order], y[order]
    last = np.r_[np.nonzero(np.diff(s))[0], len(s) - 1]       # last tile of each run of equal scores
    tp = np.cumsum(y)[last]
    fp = np.cumsum(~y)[last]
    return (np.r_[0.0, fp / n_neg], np.r_[0.0, tp / n_pos], np.r_[np.inf, s[last]])


def auc(fpr, tpr) -> float:
    """Area under a piecewise-linear ROC (trapezoids)."""
    fpr, tpr = np.asarray(fpr, np.float64), np.asarray(tpr, np.float64)
    return float(np.sum(np.diff(fpr) * (tpr[1:] + tpr[:-1]) * 0.5))


def operating_point(score, positive, max_fpr: float):
    """(threshold, tpr, fpr) of the ROC point with the largest tpr whose fpr <= max_fpr."""
    fpr, tpr, thr = roc(score, positive)
    ok = np.nonzero(fpr <= max_fpr)[0]
    i = ok[np.argmax(tpr[ok])]
    return float(thr[i]), float(tpr[i]), float(fpr[i])


def contrast_threshold(contrast2, background, max_false_skip: float):
    """The RMS-contrast threshold (for bg_contrast) that skips the most background tiles while
    skipping at most max_false_skip of the sample tiles, set halfway (in contrast^2) between the
    last statistic it skips and the next one: (bg_contrast, tpr, fpr)."""
    c2 = np.asarray(contrast2, np.float64)
    t, tpr, fpr = operating_point(-c2, background, max_false_skip)
    if not np.isfinite(t):
        return 0.0, tpr, fpr
    above = c2[c2 > -t]
    nxt = float(above.min()) if len(above) else -t * 2.0
    return math.sqrt(0.5 * (-t + nxt)), tpr, fpr


def classifier_targets(background) -> np.ndarray:
    """Training targets [n, 15] of the classifier: 1 in the first network output (Noll 4) on background."""
    b = np.asarray(background, dtype=bool)
    t = np.zeros((len(b), 15), dtype=np.float32)
    t[:, 3] = b
    return t


def draw(n: int, seed: int, blank_frac: float = 0.3, faint_frac: float = 0.0, table=None):
    """Tiles of the learned configuration: (uv, zernike, blank, scale); a faint_frac share of the
    sample tiles gets a contrast factor log-uniform in FAINT_RANGE."""
    table = learn.field_table() if table is None else table
    uv, zern, blank = learn.draw_tiles(n, seed, table, blank_frac)
    rng = np.random.default_rng(seed + 7)
    faint = (rng.random(n) < faint_frac) & ~blank
    lo, hi = np.log(FAINT_RANGE[0]), np.log(FAINT_RANGE[1])
    scale = np.where(faint, np.exp(rng.uniform(lo, hi, n)), 1.0).astype(np.float32)
    return uv, zern, blank, scale


def measure(plan: apic.Plan, tiles, seed: int, net: apic.Net | None = None, chunk: int = 256,
            photons: float = 1e4):
    """Per tile on the GPU: (contrast2 [n], library background flag [n], network score [n] or None,
    features [n, 64, 64, 8] device tensor, uv device tensor)."""
    import torch
    uv, zern, blank, scale = tiles
    n = len(zern)
    c2 = torch.empty(n, dtype=torch.float32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    feat = torch.empty((n, apic.CROP, apic.CROP, 8), dtype=torch.float32, device="cuda")
    for t0 in range(0, n, chunk):
        c = min(chunk, n - t0)
        I = learn.simulate(plan, zern, blank, seed, photons, t0, c, scale=scale)
        plan.background(c, I, c2[t0:t0 + c], st[t0:t0 + c])
        plan.features(c, I, feat[t0:t0 + c])
        del I
    uv_d = torch.as_tensor(uv, device="cuda")
    score = None
    if net is not None:
        score = learn.predict(net, feat, uv_d)[:, 3].cpu().numpy()
    bg = (st.cpu().numpy() & apic.APIC_TILE_BACKGROUND) != 0
    return c2.cpu().numpy(), bg, score, feat, uv_d


def train_classifier(plan: apic.Plan, n: int, seed: int, epochs: int = 6, faint_frac: float = 0.5,
                     lr: float = 1e-3, batch: int = 64, out_gain: float = 0.01, log=None):
    """The network trained as a background classifier on n fresh tiles: (net, loss history)."""
    import torch
    tiles = draw(n, seed, faint_frac=faint_frac)
    _, _, _, feat, uv = measure(plan, tiles, seed)
    target = torch.as_tensor(classifier_targets(tiles[2]), device="cuda")
    net = apic.Net(256)
    net.set_params(learn.init_params(seed, out_gain))
    hist = learn.train(net, feat, uv, target, epochs=epochs, batch=batch, lr=lr, seed=seed, log=log)
    del feat
    return net, hist


def evaluate(plan: apic.Plan, net: apic.Net, n: int, seed: int, faint_frac: float, max_false_skip: float):
    """ROC summary of the variance statistic and the classifier on n fresh tiles; the library's own
    flags are those of the plan's bg_contrast."""
    bg_contrast = round(float(plan.params.bg_contrast), 6)          # the float32 field, as set
    tiles = draw(n, seed, faint_frac=faint_frac)
    blank = tiles[2]
    c2, flag, score, _, _ = measure(plan, tiles, seed, net)
    out = {"tiles": n, "background": int(blank.sum()), "faint_share_of_samples": faint_frac}
    fpr, tpr, _ = roc(-c2.astype(np.float64), blank)
    thr, v_tpr, v_fpr = contrast_threshold(c2, blank, max_false_skip)
    out["variance"] = {
        "auc": auc(fpr, tpr),
        "at_bg_contrast": {"bg_contrast": bg_contrast, "skipped_background": float(flag[blank].mean()),
                           "skipped_sample": float(flag[~blank].mean())},
        "calibrated": {"bg_contrast": thr, "skipped_background": v_tpr, "skipped_sample": v_fpr},
        "contrast_rms": {"background_max": float(np.sqrt(c2[blank].max())),
                         "sample_min": float(np.sqrt(c2[~blank].min()))},
    }
    fpr, tpr, _ = roc(score, blank)
    t, c_tpr, c_fpr = operating_point(score, blank, max_false_skip)
    out["cnn"] = {"auc": auc(fpr, tpr),
                  "calibrated": {"score_threshold": t, "skipped_background": c_tpr, "skipped_sample": c_fpr}}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="ROC of the background skip against a CNN classifier")
    ap.add_argument("--tile", type=int, default=256)
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--eval", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--max-false-skip", type=float, default=1e-3)
    ap.add_argument("--bg-contrast", type=float, default=0.02)
    ap.add_argument("--seed", type=int, default=20469)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    ill = synth.illumination()
    plan = apic.Plan(a.tile, ill.kx[:8], ill.ky[:8], 8, max_tiles=256, bg_contrast=a.bg_contrast)
    t0 = time.perf_counter()
    net, hist = train_classifier(plan, a.train, a.seed, a.epochs)
    t1 = time.perf_counter()
    res = {"tile": a.tile, "train_tiles": a.train, "epochs": a.epochs, "train_loss": [round(h, 6) for h in hist],
           "train_seconds": round(t1 - t0, 1), "max_false_skip": a.max_false_skip}
    for name, ff, s in (("standard", 0.0, a.seed + 1), ("faint", 1.0, a.seed + 2)):
        res[name] = evaluate(plan, net, a.eval, s, ff, a.max_false_skip)
    print(json.dumps(res))
    net.close()
    plan.close()


if __name__ == "__main__":
    main()
