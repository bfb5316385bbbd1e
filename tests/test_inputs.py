"""The seeded input recipe (CPU): analytic line integrals and the noise model.

The synthetic workloads (paper_1009_1351_gb300/synth.py) stand in for the
paper's phantom studies: ellipse phantoms whose line integrals are computed
in closed form, then Poisson counts lambda = I0 exp(-p), y = log(I0 / n)
and the weights w = Sigma^{-1} = lambda (Eq. 1's statistical weighting).
Checked against things other than the formulas themselves:
  * the closed-form line integrals are the limit of the oracle's Siddon
    projections of ever finer rasterised copies of the same phantom (the
    gap is the raster's edge error and halves with each refinement);
  * for rays with many counts, (y - p) sqrt(w) has mean ~0 and mean square
    ~1 (the first-order variance of log n for Poisson n is 1 / lambda).
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth


def raster_projection_error(oracle_mod, c, factor):
    """Relative L2 gap between synth's line integrals and the oracle's
    projection of the phantom rasterised 'factor' times finer."""
    g = c.geom
    ells = [synth.phantom_ellipses(g.nx, g.pixel_mm, k, g.n_phases, c.with_spine_diaphragm)
            for k in range(g.n_phases)]
    p = synth.line_integrals(ells, g)
    fine = synth.Geometry(nx=g.nx * factor, ny=g.ny * factor, pixel_mm=g.pixel_mm / factor,
                          n_phases=g.n_phases, n_views=g.n_views, n_bins=g.n_bins, bin_mm=g.bin_mm,
                          sid_mm=g.sid_mm, sdd_mm=g.sdd_mm)
    img = np.stack([synth.rasterize(e, fine.nx, fine.ny, fine.pixel_mm) for e in ells])
    q = oracle_mod.project(oracle_mod.Geom(fine), img)
    return float(np.linalg.norm(q - p) / np.linalg.norm(p))


def test_closed_form_line_integrals_match_the_projected_phantom(oracle_mod):
    """The gap is the raster's edge error: first order in the raster pixel
    (halves with each refinement: 1.9 %, 0.93 %, 0.46 % on the 64^2
    workload), so the closed form is the limit the projections converge to;
    a wrong chord factor or centre would leave a gap that does not shrink."""
    c = synth.case("tiny")
    e1, e2, e4 = (raster_projection_error(oracle_mod, c, f) for f in (1, 2, 4))
    assert e4 < 6e-3
    assert 1.8 < e1 / e2 < 2.3 and 1.8 < e2 / e4 < 2.3


def test_noise_is_poisson_in_the_counts():
    c = synth.case("mid_b")             # I0 = 1e6: every ray has many counts
    d = synth.make_inputs(c)
    lam = d["w"]
    z = (d["y"] - d["pbar"]) * np.sqrt(lam)
    sel = lam > 1e3
    assert sel.mean() > 0.9
    assert abs(z[sel].mean()) < 0.01
    assert np.mean(z[sel] ** 2) == pytest.approx(1.0, abs=0.01)
    # the weights are the expected counts of the same rays
    assert np.allclose(lam, c.i0 * np.exp(-d["pbar"]), rtol=1e-12)
