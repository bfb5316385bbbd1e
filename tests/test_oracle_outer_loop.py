"""The step order of the oracle's TNLM algorithm box (Sec. 2.2), pinned by
composing its separately pinned parts (CPU).

The box, per outer iteration k:
  step 2  g^(k) = CGLS from f^(k-1)                 (orc_cgls: Krylov/lstsq pins)
  step 3  weights of Eq. 8 from g^(k), not f^(k-1)  (orc_weights: box-sum pins)
  step 4  M2 Gauss-Jacobi sweeps from u^(0) = g^(k) (orc_gj: dense-solve pins)
  step 5  f^(k) = max(u^(M2), 0), after Gauss-Jacobi only

orc_reconstruct must equal that composition to rounding (its loop shares
no arithmetic with the test beyond the pinned parts it calls).  The inputs
are chosen so that each plausible misreading changes the result by far more
than the tolerance: the weights taken from f^(k-1) instead of g^(k), the
clamp applied to g before the sweeps, the sweeps started from f^(k-1), or
the clamp skipped.  The checks that the misreadings differ guard the test
itself: a composition test that cannot tell them apart pins nothing.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

GEOM = synth.Geometry(nx=20, ny=16, pixel_mm=1.0, n_phases=3, n_views=9, n_bins=40,
                      bin_mm=1.2, sid_mm=200.0, sdd_mm=320.0)
P = synth.Params(mu_hat=0.8, h=0.01, patch=3, window=5, m1=2, m2=3, k_outer=1, clamp=1)


@pytest.fixture(scope="module")
def problem(oracle_mod):
    G = oracle_mod.Geom(GEOM)
    rng = np.random.default_rng(77)
    truth = np.stack([np.roll(0.02 * (rng.random((GEOM.ny, GEOM.nx)) > 0.5), k, axis=1)
                      for k in range(GEOM.n_phases)])
    y = oracle_mod.project(G, truth) + 0.05 * rng.standard_normal(G.sino_shape)
    w = rng.uniform(0.5, 2.0, G.sino_shape)
    # a start image far from the data, so g^(1) and f^(0) differ strongly
    f0 = 0.02 * rng.random(G.img_shape)[:, ::-1, :].copy()
    return G, y, w, f0


def compose(oracle_mod, G, y, w, f, p, weights_from="g", clamp_g=False, gj_start="g",
            clamp=True):
    g, res = oracle_mod.cgls(G, y, w, f, p.m1)
    src = g if weights_from == "g" else f
    wn, wp = oracle_mod.weights(src, p.patch, p.window, p.h)
    gg = np.maximum(g, 0.0) if clamp_g else g
    u = oracle_mod.gj(gg if gj_start == "g" else f, wn, wp, p.window, p.mu_hat, p.m2)
    return (np.maximum(u, 0.0) if clamp else u), float(res.sum())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_one_outer_iteration_is_the_composition_of_the_box_steps(oracle_mod, problem):
    G, y, w, f0 = problem
    f1, rel_hist, res_hist = oracle_mod.reconstruct(G, y, w, f0, P)
    want, res0 = compose(oracle_mod, G, y, w, f0, P)
    np.testing.assert_allclose(f1, want, rtol=1e-12, atol=1e-15)
    # the data residual monitor is that of f^(k-1), the CGLS start
    assert res_hist[0] == pytest.approx(res0, rel=1e-12)
    assert rel_hist[0] == pytest.approx(np.linalg.norm(f1 - f0) / np.linalg.norm(f1), rel=1e-12)


def test_two_outer_iterations_chain_the_composition(oracle_mod, problem):
    G, y, w, f0 = problem
    p2 = synth.Params(**{**P.__dict__, "k_outer": 2})
    f2, _, _ = oracle_mod.reconstruct(G, y, w, f0, p2)
    f1, _ = compose(oracle_mod, G, y, w, f0, P)
    want, _ = compose(oracle_mod, G, y, w, f1, P)
    np.testing.assert_allclose(f2, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("misreading", [dict(weights_from="f"), dict(clamp_g=True),
                                        dict(gj_start="f"), dict(clamp=False)],
                         ids=["weights_from_f", "clamp_before_gj", "gj_from_f", "no_clamp"])
def test_each_misreading_changes_the_result(oracle_mod, problem, misreading):
    G, y, w, f0 = problem
    f1, _, _ = oracle_mod.reconstruct(G, y, w, f0, P)
    wrong, _ = compose(oracle_mod, G, y, w, f0, P, **misreading)
    assert rel(wrong, f1) > 1e-3


def test_inputs_exercise_the_clamp(oracle_mod, problem):
    """g^(1) has negative pixels (so clamping g or skipping the clamp matter)."""
    G, y, w, f0 = problem
    g, _ = oracle_mod.cgls(G, y, w, f0, P.m1)
    assert (g < 0).mean() > 0.05
