"""CNR (Eq. 10), SNR (Eq. 11) and the phantom ROIs used for them."""
import math

import numpy as np

from paper_1009_1351_gb300 import quality, synth


def test_cnr_closed_form():
    rng = np.random.default_rng(0)
    img = 1.0 + 0.1 * rng.standard_normal((64, 64))
    roi = np.zeros_like(img, dtype=bool)
    roi[10:20, 10:20] = True
    img[roi] = 2.0
    bg = ~roi
    ref = abs(2.0 - img[bg].mean()) / img[bg].std()
    assert math.isclose(quality.cnr(img, roi, bg), ref, rel_tol=1e-12)
    assert 8.0 < quality.cnr(img, roi, bg) < 12.0


def test_snr_closed_form():
    rng = np.random.default_rng(1)
    truth = rng.random((32, 32))
    err = 0.01 * rng.standard_normal((32, 32))
    f = truth + err
    ref = 10 * math.log10(np.sum((f - f.mean()) ** 2) / np.sum(err ** 2))
    assert math.isclose(quality.snr_db(f, truth), ref, rel_tol=1e-12)
    assert quality.snr_db(truth + 2 * err, truth) < quality.snr_db(f, truth)


def test_rois_lie_on_the_intended_structures():
    for name in ("tiny", "mid_a"):
        c = synth.case(name)
        g = c.geom
        for phase in (0, 5):
            ells = synth.phantom_ellipses(g.nx, g.pixel_mm, phase, g.n_phases, c.with_spine_diaphragm)
            truth = synth.rasterize(ells, g.nx, g.ny, g.pixel_mm)
            r = quality.rois(c, phase)
            roi, bg = r["roi1"]
            assert roi.sum() > 4 and bg.sum() > 10 and not (roi & bg).any()
            np.testing.assert_allclose(truth[roi], 0.021)
            np.testing.assert_allclose(truth[bg], 0.004)
            if c.with_spine_diaphragm:
                roi, bg = r["roi2"]
                assert roi.sum() > 4 and bg.sum() > 10 and not (roi & bg).any()
                np.testing.assert_allclose(truth[roi], 0.04)
                np.testing.assert_allclose(truth[bg], 0.019)


def test_less_noise_means_higher_cnr_and_snr():
    c = synth.case("tiny")
    truth = np.stack([synth.rasterize(synth.phantom_ellipses(64, 1.0, k, 10, False), 64, 64, 1.0)
                      for k in range(10)])
    rng = np.random.default_rng(2)
    noise = rng.standard_normal(truth.shape)
    lo = quality.evaluate(c, truth + 0.001 * noise, truth)
    hi = quality.evaluate(c, truth + 0.004 * noise, truth)
    assert lo["snr_db"] > hi["snr_db"] + 10
    assert lo["cnr_roi1"] > 3 * hi["cnr_roi1"]
