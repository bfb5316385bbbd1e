"""GPU (FP32, CUDA kernels via the C ABI) vs the FP64 oracle, element by element.

Tolerances: single operators (P, P^T, patch distances) are FP32 sums of a few
hundred terms, relative L2 <= 1e-5.  The full TNLM iteration after a fixed
K must agree with the oracle to relative L2 <= 1e-4.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
REC_TOL = 1e-4
# Largest single-entry error of an operator, relative to the largest entry.
# The kernels derive each ray's position from FP32 geometry (error ~3e-5
# pixel); for a ray within ~1e-3 rad of an image axis the point where it
# crosses from one pixel row to the next moves by that error divided by the
# slope, so a few near-axis rays differ from the FP64 oracle by up to ~1e-3
# relative while the relative L2 error stays below 1e-5.
OP_MAX_TOL = 5e-3


@pytest.fixture(scope="module")
def tn():
    import paper_1009_1351_gb300 as tn
    from paper_1009_1351_gb300 import build
    build.build()
    tn.load_library()
    assert torch.cuda.is_available()
    return tn


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


RAGGED = synth.Geometry(nx=37, ny=29, pixel_mm=1.1, n_phases=3, n_views=7, n_bins=45,
                        bin_mm=1.3, sid_mm=500.0, sdd_mm=800.0)
# a 110-degree fan: some views' rays change marching class twice
WIDEFAN = synth.Geometry(nx=18, ny=14, pixel_mm=2.0, n_phases=3, n_views=8, n_bins=96,
                         bin_mm=2.0, sid_mm=60.0, sdd_mm=100.0)
GEOMS = {
    "tiny": synth.case("tiny").geom,
    "ragged": RAGGED,
    "widefan": WIDEFAN,
    "small": synth.small_geometry(),
    "mid_a": synth.case("mid_a").geom,
    "large_b": synth.case("large_b").geom,
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_project_matches_oracle(tn, oracle_mod, name):
    g = GEOMS[name]
    G = oracle_mod.Geom(g)
    f = synth.random_images(G.img_shape, 1)
    ref = oracle_mod.project(G, f)
    geo = tn.tnlm_create_geometry(g)
    out = torch.zeros(G.sino_shape, device="cuda")
    tn.tnlm_project(geo, dev(f), out)
    got = host(out)
    assert rel_l2(got, ref) <= OP_TOL
    assert np.abs(got - ref).max() <= OP_MAX_TOL * np.abs(ref).max()


@pytest.mark.parametrize("name", list(GEOMS))
def test_backproject_matches_oracle(tn, oracle_mod, name):
    g = GEOMS[name]
    G = oracle_mod.Geom(g)
    q = synth.random_images(G.sino_shape, 2, scale=1.0)
    ref = oracle_mod.backproject(G, q)
    geo = tn.tnlm_create_geometry(g)
    out = torch.zeros(G.img_shape, device="cuda")
    tn.tnlm_backproject(geo, dev(q), out)
    got = host(out)
    assert rel_l2(got, ref) <= OP_TOL
    assert np.abs(got - ref).max() <= OP_MAX_TOL * np.abs(ref).max()


def test_all_ones_image_projects_to_chords(tn):
    from test_oracle_projector import slab_chord
    g = GEOMS["tiny"]
    geo = tn.tnlm_create_geometry(g)
    out = torch.zeros((g.n_phases, g.n_views, g.n_bins), device="cuda")
    tn.tnlm_project(geo, torch.ones((g.n_phases, g.ny, g.nx), device="cuda"), out)
    src, d = synth.ray_endpoints(g)
    hx = g.nx * g.pixel_mm / 2
    ref = slab_chord(src[..., 0], src[..., 1], d[..., 0], d[..., 1], g.sdd_mm, -hx, hx, -hx, hx)
    np.testing.assert_allclose(host(out), ref, rtol=1e-5, atol=OP_MAX_TOL * ref.max())


@pytest.mark.parametrize("name", ["tiny", "ragged", "widefan", "mid_a"])
def test_adjointness_on_gpu(tn, name):
    g = GEOMS[name]
    geo = tn.tnlm_create_geometry(g)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((g.n_phases, g.ny, g.nx))
    q = rng.standard_normal((g.n_phases, g.n_views, g.n_bins))
    Pf = torch.zeros(q.shape, device="cuda")
    Ptq = torch.zeros(f.shape, device="cuda")
    tn.tnlm_project(geo, dev(f), Pf)
    tn.tnlm_backproject(geo, dev(q), Ptq)
    lhs = float(np.vdot(host(Pf), q))
    rhs = float(np.vdot(f, host(Ptq)))
    scale = float(np.abs(host(Pf)).sum() * np.abs(q).max())
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_projector_is_deterministic(tn):
    g = GEOMS["tiny"]
    geo = tn.tnlm_create_geometry(g)
    q = dev(synth.random_images((g.n_phases, g.n_views, g.n_bins), 5))
    a = torch.zeros((g.n_phases, g.ny, g.nx), device="cuda")
    b = torch.zeros_like(a)
    tn.tnlm_backproject(geo, q, a)
    tn.tnlm_backproject(geo, q, b)
    assert torch.equal(a, b)


# ---------------------------------------------------------------- weights
def gpu_weights(tn, geo, g, d, W, h):
    p = synth.Params(patch=d, window=W, h=h)
    nd, nn = tn.tnlm_weights_size(geo, p)
    N, ny, nx = g.shape
    dist = torch.zeros((N, W * W, ny, nx), device="cuda")
    norm = torch.zeros((4, N, ny, nx), device="cuda")
    assert dist.numel() * 4 == nd and norm.numel() * 4 == nn
    tn.tnlm_weights(geo, p, dev(g), dist, norm)
    return host(dist), host(norm)


def normalised_from_gpu(D, norm, W, h):
    """Rebuild omega_{i,i+1}(x, x+s) and omega_{i,i-1}(x, x+s) from the stored form."""
    N, W2, ny, nx = D.shape
    rho = (W - 1) // 2
    Dn = np.moveaxis(D, 1, -1)                       # [N, ny, nx, W2]
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


@pytest.mark.parametrize("shape,d,W", [((4, 21, 35), 3, 5), ((3, 40, 70), 5, 11),
                                       ((3, 37, 45), 7, 15), ((5, 17, 33), 1, 3),
                                       ((3, 512, 512), 5, 11), ((3, 30, 41), 9, 5),
                                       ((3, 29, 50), 3, 17)])
def test_weights_match_oracle(tn, oracle_mod, shape, d, W):
    """Ragged shapes (partial tiles, backward minima combined across tiles by
    the integer atomic min) and 512 x 512 x 3; patch <= 7 with window <= 15
    takes the sliding-window horizontal pass, the last two cases (patch 9,
    window 17) the reloading one."""
    N, ny, nx = shape
    geom = synth.Geometry(nx=nx, ny=ny, pixel_mm=min(1.0, 128.0 / max(nx, ny)), n_phases=N, n_views=4,
                          n_bins=16, bin_mm=1.0, sid_mm=500.0, sdd_mm=800.0)
    geo = tn.tnlm_create_geometry(geom)
    rng = np.random.default_rng(10 + d)
    base = 0.02 * rng.random((ny, nx))
    g = np.stack([np.roll(base, k, axis=1) + 0.002 * rng.random((ny, nx)) for k in range(N)])
    g = g.astype(np.float32).astype(np.float64)     # both sides see the same FP32 values
    h = 0.002 * d
    D, norm = gpu_weights(tn, geo, g, d, W, h)
    wn_ref, wp_ref, dn_ref = oracle_mod.weights(g, d, W, h, with_dist=True)
    Dref = np.moveaxis(dn_ref, -1, 1)
    assert np.array_equal(np.isinf(D), np.isinf(Dref))
    fin = np.isfinite(Dref)
    np.testing.assert_allclose(D[fin], Dref[fin], rtol=2e-5, atol=1e-9)
    wn, wp = normalised_from_gpu(D, norm, W, h)
    np.testing.assert_allclose(wn, wn_ref, atol=2e-5)
    np.testing.assert_allclose(wp, wp_ref, atol=2e-5)
    assert (norm[1] >= 1 - 1e-6).all() and (norm[3] >= 1 - 1e-6).all()


# ---------------------------------------------------------------- iteration
def run_both(tn, oracle_mod, g, inputs, p, f0):
    G = oracle_mod.Geom(g)
    geo = tn.tnlm_create_geometry(g)
    y, w = inputs["y"], inputs["w"]
    f = dev(f0)
    rep = tn.tnlm_reconstruct(geo, p, dev(y), dev(w), f)
    ref, rel, res = oracle_mod.reconstruct(G, y.astype(np.float32), w.astype(np.float32),
                                           np.asarray(f0, np.float32), p)
    return host(f), ref, rep, rel, res


@pytest.fixture(scope="module")
def tiny_case():
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    f0 = np.full((10, 64, 64), 0.01)
    return c, d, f0


def test_cgls_step_matches_oracle(tn, oracle_mod, tiny_case):
    """mu_hat = 0 makes the Gauss-Jacobi sweep return g: f = CGLS output."""
    c, d, f0 = tiny_case
    p = synth.Params(mu_hat=0.0, h=0.006, patch=3, window=5, m1=3, m2=1, k_outer=1, clamp=0)
    got, ref, rep, rel, res = run_both(tn, oracle_mod, c.geom, d, p, f0)
    assert rel_l2(got, ref) <= OP_TOL * 3
    assert abs(rep["residual_hist"][0] - res[0]) <= 1e-5 * res[0]


def test_gauss_jacobi_step_matches_oracle(tn, oracle_mod, tiny_case):
    """m1 = 0 makes g = f^(0): f = weights + 3 Gauss-Jacobi sweeps of the start image."""
    c, d, _ = tiny_case
    f0 = (d["truth"] + 0.002 * np.random.default_rng(4).standard_normal(d["truth"].shape))
    p = synth.Params(mu_hat=0.8, h=0.006, patch=3, window=5, m1=0, m2=3, k_outer=1, clamp=0)
    got, ref, rep, rel, res = run_both(tn, oracle_mod, c.geom, d, p, f0)
    assert rel_l2(got, ref) <= OP_TOL


def test_tiny_reconstruction_matches_oracle(tn, oracle_mod, tiny_case):
    c, d, f0 = tiny_case
    got, ref, rep, rel, res = run_both(tn, oracle_mod, c.geom, d, c.params, f0)
    assert rep["iterations"] == c.params.k_outer
    assert rel_l2(got, ref) <= REC_TOL
    np.testing.assert_allclose(rep["rel_change_hist"], rel, rtol=2e-3, atol=1e-6)
    np.testing.assert_allclose(rep["residual_hist"], res, rtol=1e-4)
    assert (got >= 0).all()


def lambda_max(oracle_mod, G, w, iters=30):
    """Largest eigenvalue of P^T w P by power iteration on the oracle."""
    v = np.ones(G.img_shape)
    lam = 0.0
    for _ in range(iters):
        u = oracle_mod.backproject(G, w * oracle_mod.project(G, v))
        lam = float(np.linalg.norm(u) / np.linalg.norm(v))
        v = u / np.linalg.norm(u)
    return lam


@pytest.mark.parametrize("variant", ["grad", "noclamp", "m2zero", "m1one"])
def test_variants_match_oracle(tn, oracle_mod, tiny_case, variant):
    c, d, f0 = tiny_case
    base = dict(mu_hat=0.5, h=0.006, patch=3, window=5, m1=3, m2=5, k_outer=4, clamp=1)
    if variant == "grad":
        beta = 1.1 * lambda_max(oracle_mod, oracle_mod.Geom(c.geom), d["w"])
        base.update(data_step=1, beta=beta)
    elif variant == "noclamp":
        base.update(clamp=0)
    elif variant == "m2zero":
        base.update(m2=0)
    else:
        base.update(m1=1)
    p = synth.Params(**base)
    got, ref, rep, rel, res = run_both(tn, oracle_mod, c.geom, d, p, f0)
    assert rel_l2(got, ref) <= REC_TOL


def test_ragged_reconstruction_matches_oracle(tn, oracle_mod):
    g = RAGGED
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(9)
    truth = 0.02 * rng.random(G.img_shape)
    y = oracle_mod.project(G, truth) + 0.01 * rng.standard_normal(G.sino_shape)
    w = rng.uniform(50, 200, G.sino_shape)
    p = synth.Params(mu_hat=0.6, h=0.01, patch=3, window=7, m1=2, m2=3, k_outer=5)
    got, ref, rep, rel, res = run_both(tn, oracle_mod, g, {"y": y, "w": w}, p,
                                       np.full(G.img_shape, 0.005))
    assert rel_l2(got, ref) <= REC_TOL


def test_reconstruction_is_deterministic_and_resumable(tn, tiny_case):
    c, d, f0 = tiny_case
    geo = tn.tnlm_create_geometry(c.geom)
    y, w = dev(d["y"]), dev(d["w"])
    p4 = synth.Params(**{**c.params.__dict__, "k_outer": 4})
    p2 = synth.Params(**{**c.params.__dict__, "k_outer": 2})
    a = dev(f0)
    b = dev(f0)
    r = dev(f0)
    tn.tnlm_reconstruct(geo, p4, y, w, a)
    tn.tnlm_reconstruct(geo, p4, y, w, b)
    tn.tnlm_reconstruct(geo, p2, y, w, r)
    tn.tnlm_reconstruct(geo, p2, y, w, r)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a, r)


def test_mid_size_reconstruction_matches_oracle(tn, oracle_mod):
    """256^2, 60 views (the undersampled dose scenario), d = 5, W = 11, K = 3."""
    c = synth.case("mid_c")
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3})
    got, ref, rep, rel, res = run_both(tn, oracle_mod, c.geom, d, p, np.full((10, 256, 256), 0.01))
    assert rel_l2(got, ref) <= REC_TOL


def test_bench_workload_slice_matches_oracle(tn, oracle_mod):
    """The benchmark's 360-view slice (256^2, 10 phases, d = 5, W = 11) run
    the way bench.py runs it -- the FBP of all views as the start image,
    then the outer iterations through the captured graph -- for K = 5,
    against the oracle run from its own FBP: the start images agree to
    2e-5 and the reconstructions to relative L2 1e-4."""
    c = synth.case("mid_a")
    d = synth.make_inputs(c)
    G = oracle_mod.Geom(c.geom)
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    geo = tn.tnlm_create_geometry(c.geom)
    f = torch.zeros(G.img_shape, device="cuda")
    tn.tnlm_fbp(geo, dev(y32), f)
    f0_ref = oracle_mod.fbp(G, y32.astype(np.float64))
    assert rel_l2(host(f), f0_ref) <= 2e-5
    p = synth.Params(**{**c.params.__dict__, "k_outer": 5})
    rep = tn.tnlm_reconstruct(geo, p, dev(y32), dev(w32), f)
    ref, rel, res = oracle_mod.reconstruct(G, y32, w32, f0_ref.astype(np.float32), p)
    assert rep["iterations"] == 5
    assert rel_l2(host(f), ref) <= REC_TOL
    np.testing.assert_allclose(rep["rel_change_hist"], rel, rtol=1e-3)


def test_graph_replay_matches_eager_launches(tn, tiny_case):
    """With kernel timing on, iterations are launched one kernel at a time;
    otherwise a captured CUDA graph of one iteration is replayed.  Both must
    give bitwise the same result, and the launch counters must agree."""
    c, d, f0 = tiny_case
    geo = tn.tnlm_create_geometry(c.geom)
    y, w = dev(d["y"]), dev(d["w"])
    a, b = dev(f0), dev(f0)
    tn.tnlm_reconstruct(geo, c.params, y, w, dev(f0))      # workspace set-up, graph capture
    tn.tnlm_profile_read(geo)
    tn.tnlm_reconstruct(geo, c.params, y, w, a)            # graph replay
    n_graph = tn.tnlm_profile_read(geo)
    tn.tnlm_profile_enable(geo, ("gj",))
    tn.tnlm_reconstruct(geo, c.params, y, w, b)            # eager
    n_eager = tn.tnlm_profile_read(geo)
    tn.tnlm_profile_enable(geo, ())
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert {k: v["launches"] for k, v in n_graph.items()} == {k: v["launches"] for k, v in n_eager.items()}
    assert n_eager["gj"]["ms"] > 0


@pytest.mark.parametrize("W,d", [(3, 1), (9, 3), (13, 5), (15, 7), (17, 3)])
def test_gauss_jacobi_window_sizes_match_oracle(tn, oracle_mod, W, d):
    """Weights + 2 sweeps (m1 = 0) on a ragged 3-phase image for every
    compiled window size (and one above them, which takes the generic sweep)."""
    g = synth.Geometry(nx=83, ny=45, pixel_mm=1.0, n_phases=3, n_views=6, n_bins=64,
                       bin_mm=1.2, sid_mm=500.0, sdd_mm=800.0)
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(W)
    base = 0.02 * rng.random((g.ny, g.nx))
    f0 = np.stack([np.roll(base, k, axis=0) + 0.001 * rng.random((g.ny, g.nx)) for k in range(3)])
    y = np.zeros(G.sino_shape)
    w = np.ones(G.sino_shape)
    p = synth.Params(mu_hat=0.7, h=0.002 * d, patch=d, window=W, m1=0, m2=2, k_outer=1, clamp=0)
    got, ref, rep, rel, res = run_both(tn, oracle_mod, g, {"y": y, "w": w}, p, f0)
    assert rel_l2(got, ref) <= OP_TOL


@pytest.mark.parametrize("name", ["tiny", "ragged", "mid_c"])
def test_fbp_initial_image_matches_oracle(tn, oracle_mod, name):
    """Step 1 of the TNLM algorithm box: FBP of all phases' projections."""
    g = GEOMS[name] if name in GEOMS else synth.case(name).geom
    G = oracle_mod.Geom(g)
    if name == "ragged":
        y = oracle_mod.project(G, 0.02 * np.random.default_rng(2).random(G.img_shape))
    else:
        y = synth.make_inputs(synth.case(name))["y"]
    y = y.astype(np.float32).astype(np.float64)
    ref = oracle_mod.fbp(G, y)
    geo = tn.tnlm_create_geometry(g)
    out = torch.zeros(G.img_shape, device="cuda")
    tn.tnlm_fbp(geo, dev(y), out)
    got = host(out)
    assert rel_l2(got, ref) <= 2e-5
    assert all(np.array_equal(got[0], got[i]) for i in range(1, g.n_phases))


def test_tiny_reconstruction_matches_the_stored_oracle_values(tn):
    """The CUDA path against the stored FP64-oracle values of
    tests/golden/tiny_k3.txt (no oracle run needed): sampled pixels within
    relative L2 1e-4, the per-iteration monitors within 1e-4 relative."""
    from tests.golden import make_golden
    iters, pix = make_golden.read_tiny_k3()
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": make_golden.K})
    geo = tn.tnlm_create_geometry(c.geom)
    f = dev(np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01))
    rep = tn.tnlm_reconstruct(geo, p, dev(d["y"]), dev(d["w"]), f)
    got_f = host(f)
    got = np.array([got_f[i, y, x] for i, y, x, _ in pix])
    want = np.array([v for _, _, _, v in pix])
    assert rel_l2(got, want) <= REC_TOL
    np.testing.assert_allclose(rep["rel_change_hist"], [r for _, r, _ in iters], rtol=1e-4)
    np.testing.assert_allclose(rep["residual_hist"], [r for _, _, r in iters], rtol=1e-4)
