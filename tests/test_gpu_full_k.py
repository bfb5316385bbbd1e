"""Full-length reconstructions on the GPU against the FP64 oracle.

The workloads are run the way bench.py runs them: the FBP of all views as
the start image (box step 1, computed by each side on its own: the start
images agree to 2e-5), then the outer iterations (the first one launched
kernel by kernel, the rest as replays of the captured one-iteration graph
when the report is requested).  Tolerance: relative L2 <= 1e-4 over the
whole [N][ny][nx] result, the bar every fixed-K reconstruction is held to.

  * the three 256 x 256 dose scenarios at their own K = 50;
  * the 512 x 512 workload (d = 7, W = 15) at 360 and at 90 views per
    phase, K = 3, with the oracle run here;
  * the 512 x 512 workload at its full K = 100 against the stored oracle
    values of tests/golden/large_<s>_k100.txt (written by
    tests/golden/make_golden.py from the oracle alone): 8192 seeded pixels
    and the relative-change history.

The oracle runs on the host cores (OpenMP); the 256^2 cases take about a
minute each, the 512^2 ones about 20 s per outer iteration.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REC_TOL = 1e-4


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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_from_fbp(tn, c, y32, w32, k):
    geo = tn.tnlm_create_geometry(c.geom)
    f = torch.zeros((c.geom.n_phases, c.geom.ny, c.geom.nx), device="cuda")
    y, w = dev(y32), dev(w32)
    tn.tnlm_fbp(geo, y, f)
    p = synth.Params(**{**c.params.__dict__, "k_outer": k})
    rep = tn.tnlm_reconstruct(geo, p, y, w, f)
    torch.cuda.synchronize()
    return f.double().cpu().numpy(), rep


def both_from_fbp(tn, oracle_mod, name, k):
    c = synth.case(name)
    d = synth.make_inputs(c)
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    got, rep = gpu_from_fbp(tn, c, y32, w32, k)
    G = oracle_mod.Geom(c.geom)
    f0 = oracle_mod.fbp(G, y32)
    p = synth.Params(**{**c.params.__dict__, "k_outer": k})
    ref, rel, res = oracle_mod.reconstruct(G, y32, w32, f0, p)
    return got, rep, ref, rel, res


@pytest.mark.parametrize("name", ["mid_a", "mid_b", "mid_c"])
def test_256_scenarios_at_their_full_k_match_oracle(tn, oracle_mod, name):
    """256 x 256, d = 5, W = 11: (a) 360 views, (b, c) 60 views, K = 50."""
    k = synth.case(name).params.k_outer
    assert k == 50
    got, rep, ref, rel, res = both_from_fbp(tn, oracle_mod, name, k)
    assert rep["iterations"] == k
    assert rel_l2(got, ref) <= REC_TOL
    np.testing.assert_allclose(rep["residual_hist"], res, rtol=1e-3)
    assert (got >= 0).all()


@pytest.mark.parametrize("name", ["large_a", "large_b"])
def test_512_workload_matches_oracle(tn, oracle_mod, name):
    """512 x 512, d = 7, W = 15: 360 views (large_a) and 90 views (large_b), K = 3."""
    got, rep, ref, rel, res = both_from_fbp(tn, oracle_mod, name, 3)
    assert rep["iterations"] == 3
    assert rel_l2(got, ref) <= REC_TOL
    np.testing.assert_allclose(rep["rel_change_hist"], rel, rtol=1e-3)
    np.testing.assert_allclose(rep["residual_hist"], res, rtol=1e-4)


@pytest.mark.parametrize("name", ["large_a", "large_b"])
def test_512_workload_at_k100_matches_the_stored_oracle_values(tn, name):
    from tests.golden import make_golden
    gold = make_golden.read_large(name)
    if gold is None:
        pytest.skip(f"tests/golden/{name}_k100.txt not written")
    iters, pix = gold
    c = synth.case(name)
    d = synth.make_inputs(c)
    got_f, rep = gpu_from_fbp(tn, c, d["y"].astype(np.float32), d["w"].astype(np.float32),
                              make_golden.LARGE_K)
    assert rep["iterations"] == make_golden.LARGE_K == len(iters)
    got = np.array([got_f[i, y, x] for i, y, x, _ in pix])
    want = np.array([v for _, _, _, v in pix])
    assert rel_l2(got, want) <= REC_TOL
    np.testing.assert_allclose(rep["residual_hist"], [r for _, _, r in iters], rtol=1e-3)
