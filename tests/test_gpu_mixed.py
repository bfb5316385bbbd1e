"""Mixed precision: patch-distance cross terms on the tensor cores.

The distances come from |P_i(x)|^2 + |P_j(y)|^2 - 2 <P_i(x), P_j(y)> with the
cross term as split-FP16 tcgen05 products (FP32 accumulation) and the
self-norms in FP32.  Against the FP64 oracle the distances must agree to an
absolute 1e-7 (the patch energies are ~1e-2, h^2 ~ 1e-4), the normalised
weights to 1e-4, and a full reconstruction to the mixed-precision bound of
relative L2 <= 1e-3 (it lands far inside it), also on the 512 x 512 slice
with 7 x 7 patches and a 15 x 15 window, whose 660 candidates per tile take
two passes through the tensor-memory accumulator.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-3


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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_weights(tn, geo, g, d, W, h, precision):
    p = synth.Params(patch=d, window=W, h=h, precision=precision)
    N, ny, nx = g.shape
    dist = torch.zeros((N, W * W, ny, nx), device="cuda")
    norm = torch.zeros((4, N, ny, nx), device="cuda")
    tn.tnlm_weights(geo, p, dev(g), dist, norm)
    return host(dist), host(norm)


@pytest.mark.parametrize("shape,d,W", [((3, 21, 35), 3, 5), ((3, 40, 70), 5, 11),
                                       ((4, 17, 33), 1, 3), ((3, 29, 50), 5, 7),
                                       ((3, 37, 45), 7, 15), ((3, 40, 52), 7, 11),
                                       ((3, 33, 40), 5, 15), ((3, 30, 41), 7, 5)])
def test_mixed_distances_match_oracle(tn, oracle_mod, shape, d, W):
    N, ny, nx = shape
    geom = synth.Geometry(nx=nx, ny=ny, pixel_mm=1.0, n_phases=N, n_views=4, n_bins=16,
                          bin_mm=1.0, sid_mm=500.0, sdd_mm=800.0)
    geo = tn.tnlm_create_geometry(geom)
    rng = np.random.default_rng(30 + d)
    base = 0.02 * rng.random((ny, nx))
    g = np.stack([np.roll(base, k, axis=1) + 0.002 * rng.random((ny, nx)) for k in range(N)])
    g = g.astype(np.float32).astype(np.float64)
    h = 0.002 * d
    D, norm = gpu_weights(tn, geo, g, d, W, h, tn.PREC_MIXED)
    _, _, dn_ref = oracle_mod.weights(g, d, W, h, with_dist=True)
    Dref = np.moveaxis(dn_ref, -1, 1)
    assert np.array_equal(np.isinf(D), np.isinf(Dref))
    fin = np.isfinite(Dref)
    err = np.abs(D[fin] - Dref[fin]).max()
    assert err <= 1e-7, err
    # minima and normalisers agree with the FP32 kernel's
    D32, norm32 = gpu_weights(tn, geo, g, d, W, h, tn.PREC_FP32)
    np.testing.assert_allclose(norm[0], norm32[0], atol=1e-7)
    np.testing.assert_allclose(norm[2], norm32[2], atol=1e-7)
    np.testing.assert_allclose(norm[1], norm32[1], rtol=1e-3)
    np.testing.assert_allclose(norm[3], norm32[3], rtol=1e-3)


@pytest.mark.parametrize("name,k", [("tiny", 20), ("mid_c", 3), ("mid_c", 50), ("large_b", 3)])
def test_mixed_reconstruction_matches_oracle(tn, oracle_mod, name, k):
    c = synth.case(name)
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": k, "precision": tn.PREC_MIXED})
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01)
    geo = tn.tnlm_create_geometry(c.geom)
    f = dev(f0)
    tn.tnlm_reconstruct(geo, p, dev(d["y"]), dev(d["w"]), f)
    got = host(f)
    p64 = synth.Params(**{**c.params.__dict__, "k_outer": k})
    ref, _, _ = oracle_mod.reconstruct(oracle_mod.Geom(c.geom), d["y"].astype(np.float32),
                                       d["w"].astype(np.float32), f0.astype(np.float32), p64)
    err = rel_l2(got, ref)
    assert err <= MIXED_TOL, err
    # and next to the FP32 path
    f32 = dev(f0)
    tn.tnlm_reconstruct(geo, p64, dev(d["y"]), dev(d["w"]), f32)
    assert rel_l2(got, host(f32)) <= 1e-4


def test_mixed_rejects_unsupported_shapes(tn):
    c = synth.case("tiny")
    geo = tn.tnlm_create_geometry(c.geom)
    p = synth.Params(patch=9, window=5, h=0.01, precision=tn.PREC_MIXED)
    g = torch.zeros((10, 64, 64), device="cuda")
    dist = torch.zeros((10, 25, 64, 64), device="cuda")
    norm = torch.zeros((4, 10, 64, 64), device="cuda")
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_weights(geo, p, g, dist, norm)
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG
