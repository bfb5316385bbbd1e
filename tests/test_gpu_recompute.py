"""The Gauss-Jacobi sweeps with the patch distances recomputed in every
sweep (params.recompute = 1) instead of streamed from the stored array.

Same arithmetic as the stored form (Eq. 8 with the row minima, the sweep of
Eq. 7); only the FP32 association of the backward distances can differ in
the last bit.  Checked against the FP64 oracle at the bar of every fixed-K
reconstruction (relative L2 <= 1e-4), next to the stored form (1e-5), on
every patch / window the mode supports and at 512^2 with d = 7, W = 15."""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import paper_1009_1351_gb300 as tn
    from paper_1009_1351_gb300 import build
    build.build()
    tn.load_library()
    return tn


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(tn, g, p, y, w, f0):
    geo = tn.tnlm_create_geometry(g)
    f = dev(f0)
    rep = tn.tnlm_reconstruct(geo, p, dev(y), dev(w), f)
    torch.cuda.synchronize()
    return f.double().cpu().numpy(), rep


@pytest.mark.parametrize("W,d", [(3, 1), (5, 3), (9, 3), (11, 5), (15, 7), (13, 7)])
def test_recompute_sweep_matches_oracle_on_ragged_images(tn, oracle_mod, W, d):
    g = synth.Geometry(nx=83, ny=45, pixel_mm=1.0, n_phases=3, n_views=6, n_bins=64,
                       bin_mm=1.2, sid_mm=500.0, sdd_mm=800.0)
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(W + 10 * d)
    base = 0.02 * rng.random((g.ny, g.nx))
    f0 = np.stack([np.roll(base, k, axis=0) + 0.001 * rng.random((g.ny, g.nx)) for k in range(3)])
    y = np.zeros(G.sino_shape)
    w = np.ones(G.sino_shape)
    p = synth.Params(mu_hat=0.7, h=0.002 * d, patch=d, window=W, m1=0, m2=3, k_outer=1, clamp=0)
    stored, _ = run(tn, g, p, y, w, f0)
    pr = synth.Params(**{**p.__dict__, "recompute": 1})
    got, _ = run(tn, g, pr, y, w, f0)
    ref, _, _ = oracle_mod.reconstruct(G, y.astype(np.float32), w.astype(np.float32), f0.astype(np.float32), p)
    assert rel(got, ref) <= 1e-5
    assert rel(got, stored) <= 1e-5


@pytest.mark.parametrize("name,k", [("tiny", 20), ("large_b", 3)])
def test_recompute_reconstruction_matches_oracle(tn, oracle_mod, name, k):
    c = synth.case(name)
    d = synth.make_inputs(c)
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01, np.float32)
    p = synth.Params(**{**c.params.__dict__, "k_outer": k})
    stored, rep_s = run(tn, c.geom, p, y32, w32, f0)
    got, rep = run(tn, c.geom, synth.Params(**{**p.__dict__, "recompute": 1}), y32, w32, f0)
    ref, rel_h, _ = oracle_mod.reconstruct(oracle_mod.Geom(c.geom), y32, w32, f0, p)
    assert rep["iterations"] == k
    assert rel(got, ref) <= 1e-4
    assert rel(got, stored) <= 1e-5
    assert rep["clamped"] == rep_s["clamped"] or abs(rep["clamped"] - rep_s["clamped"]) <= 3


def test_recompute_rejects_mixed_precision(tn):
    c = synth.case("tiny")
    geo = tn.tnlm_create_geometry(c.geom)
    p = synth.Params(**{**c.params.__dict__, "recompute": 1, "precision": tn.PREC_MIXED})
    t = torch.zeros((10, 60, 128), device="cuda")
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, p, t, t, torch.zeros((10, 64, 64), device="cuda"))
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG
