"""Background-skip calibration on the GPU (small case): the library's flags are
its statistic against bg_contrast^2; on tiles of the learned configuration
(30 % near-blank) the variance statistic separates background from sample and
the trained classifier ranks them well; the stress set with faint tissue
gives a valid ROC summary whose calibrated point keeps its bound."""
import numpy as np
import pytest

from paper_2407_20469_gb300 import apic, roc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_2407_20469_gb300 import build
    build.build()
    ill = synth.illumination()
    plan = apic.Plan(64, ill.kx[:8], ill.ky[:8], 8, max_tiles=256, bg_contrast=0.02)
    net, hist = roc.train_classifier(plan, 2048, 31, epochs=4)
    return plan, net, hist


def test_flags_are_the_statistic_below_the_threshold(setup):
    plan = setup[0]
    tiles = roc.draw(512, 32, faint_frac=0.5)
    c2, flag, _, _, _ = roc.measure(plan, tiles, 32)
    assert np.array_equal(flag, c2 < np.float32(0.02) * np.float32(0.02))
    assert np.all(np.isfinite(c2)) and np.all(c2 >= 0)


def test_standard_tiles_separate(setup):
    plan, net, hist = setup
    assert hist[-1] < hist[0]
    r = roc.evaluate(plan, net, 1024, 33, 0.0, 1e-3)
    v = r["variance"]
    assert v["auc"] > 0.999
    assert v["at_bg_contrast"]["skipped_sample"] == 0.0
    assert v["at_bg_contrast"]["skipped_background"] > 0.95
    assert v["calibrated"]["skipped_sample"] <= 1e-3
    assert r["cnn"]["auc"] > 0.95


def test_faint_tissue_roc_is_valid(setup):
    plan, net, _ = setup
    r = roc.evaluate(plan, net, 1024, 34, 1.0, 1e-2)
    for k in ("variance", "cnn"):
        assert 0.5 < r[k]["auc"] <= 1.0
        assert r[k]["calibrated"]["skipped_sample"] <= 1e-2
