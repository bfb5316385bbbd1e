"""The FP64 monitors of the TNLM algorithm box on the GPU (Sec. 2.1-2.2).

With params.monitor = 1 every outer iteration reduces the TNLM term of Eq. 1
(J of Eq. 2 toward both neighbours, with that iteration's weights, at the
iteration's result) and the call ends with the data term of the final
image; the positivity step counts the pixels it clamps.  Checked against
the oracle:

  * one iteration with M1 = 0 (so the weights come from the start image,
    which the test knows exactly): the GPU's weights are exported by
    tnlm_weights from the same image, and the oracle evaluates Eq. 2 and
    the data term on the GPU's result with them.  What remains is the
    monitor's own arithmetic: FP32 terms (each weight from ex2.approx,
    relative error ~2^-22, of an argument rounded to FP32: about 1e-6 of
    the argument for the weights that matter) summed in FP64, so relative
    2e-6 for the TNLM term; the data term carries the FP32 projector's
    ~1e-6 relative error per ray, 1e-5 allowed;
  * three iterations of the default step (CGLS, M2 = 5) against the oracle's
    own composition of the box steps: relative 1e-4, the bar of the whole
    FP32 iteration;
  * the clamp count equals the number of negative pixels of the same
    iteration run without the clamp (bitwise the same iterate), and the
    oracle's count within a few pixels whose sign FP32 rounding can flip;
  * the monitor does not change the iterate.
"""
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


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    rng = np.random.default_rng(21)
    f0 = (d["truth"] + 0.003 * rng.standard_normal(d["truth"].shape)).astype(np.float32)
    return c, d["y"].astype(np.float32), d["w"].astype(np.float32), f0


def gpu_row_weights(D, norm, W, h):
    """omega_{i,i+1}(x, x+s) and omega_{i,i-1}(x, x+s) in FP64 from the stored form."""
    N, W2, ny, nx = D.shape
    rho = (W - 1) // 2
    Dn = np.moveaxis(D, 1, -1)
    wn = np.where(np.isinf(Dn), 0.0, np.exp(-(Dn - norm[0][..., None]) / h ** 2)) / norm[1][..., None]
    wp = np.zeros_like(wn)
    for i in range(N):
        Dm = Dn[(i - 1) % N]
        for sy in range(-rho, rho + 1):
            for sx in range(-rho, rho + 1):
                k = (sy + rho) * W + sx + rho
                kn = (-sy + rho) * W + (-sx + rho)
                for y in range(ny):
                    y1 = y + sy
                    if not (0 <= y1 < ny):
                        continue
                    x0, x1 = max(0, -sx), min(nx, nx - sx)
                    dv = Dm[y1, x0 + sx:x1 + sx, kn]
                    wp[i, y, x0:x1, k] = np.exp(-(dv - norm[2][i, y, x0:x1]) / h ** 2) / norm[3][i, y, x0:x1]
    return wn, wp


def test_monitor_terms_match_the_oracle_with_the_gpu_weights(tn, oracle_mod, tiny):
    c, y, w, f0 = tiny
    p = synth.Params(mu_hat=0.6, h=0.006, beta=2.0, patch=3, window=5, m1=0, m2=3, k_outer=1,
                     clamp=1, monitor=1)
    geo = tn.tnlm_create_geometry(c.geom)
    f = dev(f0)
    rep = tn.tnlm_reconstruct(geo, p, dev(y), dev(w), f)
    f1 = host(f)
    nd, nn = tn.tnlm_weights_size(geo, p)
    N, ny, nx = f0.shape
    dist = torch.zeros((N, p.window ** 2, ny, nx), device="cuda")
    norm = torch.zeros((4, N, ny, nx), device="cuda")
    tn.tnlm_weights(geo, p, dev(f0), dist, norm)
    wn, wp = gpu_row_weights(host(dist), host(norm), p.window, p.h)
    G = oracle_mod.Geom(c.geom)
    t_ref = oracle_mod.tnlm_term(f1, wn, wp, p.window)
    d_ref = oracle_mod.data_term(G, y, w, f1)
    assert t_ref > 0
    assert rep["tnlm_term"] == pytest.approx(t_ref, rel=2e-6)
    assert rep["tnlm_hist"] == [rep["tnlm_term"]]
    assert rep["data_hist"][0] == pytest.approx(d_ref, rel=1e-5)
    mu = p.mu_hat * p.beta
    assert rep["objective"] == pytest.approx(d_ref + 0.5 * mu * t_ref, rel=1e-5)
    assert rep["objective_hist"] == [rep["objective"]]


def test_monitor_history_matches_the_oracle_box(tn, oracle_mod, tiny):
    c, y, w, _ = tiny
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3, "beta": 1.5, "monitor": 1})
    f0 = np.full((10, 64, 64), 0.01, np.float32)
    geo = tn.tnlm_create_geometry(c.geom)
    rep = tn.tnlm_reconstruct(geo, p, dev(y), dev(w), dev(f0))
    G = oracle_mod.Geom(c.geom)
    f = f0.astype(np.float64)
    for k in range(3):
        g, _ = oracle_mod.cgls(G, y, w, f, p.m1)
        wn, wp = oracle_mod.weights(g, p.patch, p.window, p.h)
        u = oracle_mod.gj(g, wn, wp, p.window, p.mu_hat, p.m2)
        ncl = int((u < 0).sum())
        f = np.maximum(u, 0.0)
        t_ref = oracle_mod.tnlm_term(f, wn, wp, p.window)
        d_ref = oracle_mod.data_term(G, y, w, f)
        assert rep["tnlm_hist"][k] == pytest.approx(t_ref, rel=1e-4)
        assert rep["data_hist"][k] == pytest.approx(d_ref, rel=1e-4)
        assert rep["objective_hist"][k] == pytest.approx(d_ref + 0.5 * p.mu_hat * p.beta * t_ref, rel=1e-4)
        assert abs(rep["clamped_hist"][k] - ncl) <= max(3, 0.005 * ncl)
    # the data term after iteration k is the residual iteration k + 1 starts from
    assert rep["data_hist"][:2] == rep["residual_hist"][1:]


def test_clamp_count_is_the_negative_pixels_of_the_unclamped_iterate(tn, tiny):
    c, y, w, _ = tiny
    f0 = np.full((10, 64, 64), 0.01, np.float32)
    geo = tn.tnlm_create_geometry(c.geom)
    base = {**c.params.__dict__, "k_outer": 1}
    a, b = dev(f0), dev(f0)
    rep_c = tn.tnlm_reconstruct(geo, synth.Params(**{**base, "clamp": 1}), dev(y), dev(w), a)
    rep_n = tn.tnlm_reconstruct(geo, synth.Params(**{**base, "clamp": 0}), dev(y), dev(w), b)
    neg = int((b < 0).sum())
    assert neg > 0
    assert rep_c["clamped"] == neg == rep_c["clamped_hist"][0]
    assert rep_n["clamped"] == 0
    assert torch.equal(a, torch.clamp(b, min=0.0))


def test_monitor_leaves_the_iterate_unchanged(tn, tiny):
    c, y, w, _ = tiny
    f0 = np.full((10, 64, 64), 0.01, np.float32)
    geo = tn.tnlm_create_geometry(c.geom)
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3})
    a, b = dev(f0), dev(f0)
    tn.tnlm_reconstruct(geo, p, dev(y), dev(w), a)
    tn.tnlm_reconstruct(geo, synth.Params(**{**p.__dict__, "monitor": 1}), dev(y), dev(w), b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
