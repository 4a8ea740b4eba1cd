"""The ROC bookkeeping of the background-skip calibration, pinned by what
defines it: the area under the ROC equals the probability that a random
positive outscores a random negative (ties counting one half, the
Mann-Whitney statistic, counted here pair by pair), each ROC point is the
rule 'score >= t' applied by brute force, and the calibrated contrast
threshold, applied with the library's strict comparison, skips exactly the
tiles its operating point counts."""
import numpy as np
import pytest

from paper_2407_20469_gb300 import roc


def pair_auc(score, pos):
    s_p, s_n = score[pos], score[~pos]
    d = s_p[:, None] - s_n[None, :]
    return (np.sum(d > 0) + 0.5 * np.sum(d == 0)) / d.size


@pytest.mark.parametrize("seed,ties", [(0, False), (1, True), (2, True)])
def test_auc_is_the_mann_whitney_statistic(seed, ties):
    rng = np.random.default_rng(seed)
    n = 300
    pos = rng.random(n) < 0.3
    s = rng.standard_normal(n) + 1.2 * pos
    if ties:
        s = np.round(s * 2) / 2                        # many equal scores across classes
    fpr, tpr, thr = roc.roc(s, pos)
    assert abs(roc.auc(fpr, tpr) - pair_auc(s, pos)) < 1e-12


def test_each_point_is_the_threshold_rule():
    rng = np.random.default_rng(3)
    pos = rng.random(200) < 0.4
    s = np.round(rng.standard_normal(200), 1)
    fpr, tpr, thr = roc.roc(s, pos)
    assert fpr[0] == 0 and tpr[0] == 0 and thr[0] == np.inf
    assert fpr[-1] == 1 and tpr[-1] == 1
    assert np.all(np.diff(thr) < 0)
    for f, t, th in zip(fpr, tpr, thr):
        called = s >= th
        assert f == np.mean(called[~pos]) and t == np.mean(called[pos])


def test_extreme_and_degenerate_cases():
    pos = np.array([True, True, False, False])
    assert roc.auc(*roc.roc(np.array([4.0, 3.0, 2.0, 1.0]), pos)[:2]) == 1.0
    assert roc.auc(*roc.roc(np.array([1.0, 2.0, 3.0, 4.0]), pos)[:2]) == 0.0
    assert roc.auc(*roc.roc(np.zeros(4), pos)[:2]) == 0.5
    with pytest.raises(ValueError):
        roc.roc(np.zeros(3), np.array([True, True, True]))
    with pytest.raises(ValueError):
        roc.roc(np.array([0.0, np.nan]), np.array([True, False]))


def test_operating_point_is_the_best_admissible_threshold():
    rng = np.random.default_rng(4)
    pos = rng.random(500) < 0.3
    s = rng.standard_normal(500) + 2.0 * pos
    for max_fpr in (0.0, 0.01, 0.1, 0.5):
        t, tp, fp = roc.operating_point(s, pos, max_fpr)
        best = 0.0
        for th in np.r_[np.inf, np.unique(s)]:        # brute force over every threshold
            c = s >= th
            if np.mean(c[~pos]) <= max_fpr:
                best = max(best, np.mean(c[pos]))
        assert tp == best and fp <= max_fpr


def test_calibrated_contrast_threshold_applies_with_the_strict_rule():
    rng = np.random.default_rng(5)
    blank = rng.random(400) < 0.3
    c2 = np.where(blank, rng.uniform(1e-5, 4e-4, 400), rng.uniform(2e-4, 5e-2, 400))   # overlapping classes
    for max_fs in (0.0, 0.02, 0.2):
        bg, tp, fp = roc.contrast_threshold(c2, blank, max_fs)
        skipped = c2 < bg * bg                          # apic_background: background below bg_contrast^2
        assert np.mean(skipped[blank]) == pytest.approx(tp, abs=1e-12)
        assert np.mean(skipped[~blank]) == pytest.approx(fp, abs=1e-12)
        assert fp <= max_fs


def test_classifier_targets_put_the_label_in_the_first_output():
    t = roc.classifier_targets(np.array([True, False, True]))
    assert t.shape == (3, 15) and t.dtype == np.float32
    assert np.array_equal(t[:, 3], [1, 0, 1]) and np.count_nonzero(t) == 2


def test_faint_draw_only_scales_sample_tiles():
    uv, z, blank, scale = roc.draw(2000, 9, blank_frac=0.3, faint_frac=0.5)
    assert np.all(scale[blank] == 1.0)
    f = scale[~blank]
    faint = f < 1.0
    assert 0.4 < faint.mean() < 0.6
    assert f[faint].min() >= roc.FAINT_RANGE[0] * (1 - 1e-6)
