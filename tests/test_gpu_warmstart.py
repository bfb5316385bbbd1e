"""What the learned warm start gains, on the GPU, checked against the oracle.

A small U-Net (16 base channels, 3 levels) is trained by the library's own
kernels on pairs the plain method makes (per-phase FBP -> TNLM run to the
stopping tolerance) for the 256 x 256, 10-phase slices of the two 60-view
dose scenarios (I0 = 1e6 and 1e4; d = 5, W = 11).  On held-out seeds
the plain TNLM iteration then runs to the same stopping tolerance from the
usual start (the FBP of all views, box step 1: cold) and from the network's
output (warm).  The network is only a start image: both final images are
the TNLM iteration's own, and each is compared element by element with the
FP64 oracle run from the same start image for the same number of outer
iterations (relative L2 <= 1e-4, the bar of every fixed-K reconstruction).
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 4e-3          # stopping rule: ||f^k - f^(k-1)|| / ||f^k|| < TOL (the relative
                    # change of this iteration levels off at 1-3e-3 on these slices)
KMAX = 100
SCEN = ("mid_b", "mid_c")


@pytest.fixture(scope="module")
def trained(oracle_mod):
    import paper_1009_1351_gb300 as tn
    from paper_1009_1351_gb300 import build, warmstart as ws
    build.build()
    tn.load_library()
    maker = ws.PairMaker(torch, tn, slots=16, k_outer=KMAX, tol=TOL, scenarios=SCEN)
    train = maker.make(list(range(500, 500 + 192)), keep_all=False)
    test = maker.make(list(range(900, 904)))
    X = torch.stack(train["inp"]) * ws.SCALE
    Y = torch.stack(train["target"]) * ws.SCALE
    net = tn.UNet(10, 10, 16, 3)
    net.set_params(ws.init_params(10, 10, 16, 3, 1))
    rng = np.random.default_rng(1)
    epochs, steps = 16, len(X) // 8
    for ep in range(epochs):
        order = rng.permutation(len(X))
        for s in range(steps):
            idx = torch.as_tensor(order[8 * s:8 * s + 8], device=X.device)
            net.grads(X[idx].contiguous(), Y[idx].contiguous())
            net.adam_step(2e-3 * 0.5 * (1 + np.cos(np.pi * (ep * steps + s) / (epochs * steps))))
    rows = ws.evaluate(torch, tn, net, maker, test, TOL, KMAX)
    return tn, maker, test, rows


def test_trained_network_cuts_iterations_to_the_tolerance(trained):
    tn, maker, test, rows = trained
    cold = np.mean([r["iters_cold"] for r in rows])
    warm = np.mean([r["iters_warm"] for r in rows])
    print(f"iterations to tol {TOL}: cold {cold:.1f}, warm {warm:.1f} "
          f"(device ms {np.mean([r['ms_cold'] for r in rows]):.1f} -> {np.mean([r['ms_warm'] for r in rows]):.1f})")
    assert all(r["iters_cold"] < KMAX and r["iters_warm"] < KMAX for r in rows)
    assert warm <= 0.7 * cold


def test_warm_and_cold_results_match_the_oracle_from_their_starts(trained, oracle_mod):
    tn, maker, test, rows = trained
    for i in (0, 1):
        c = maker.cases[test["scenario"][i]]
        G = oracle_mod.Geom(c.geom)
        y = test["y"][i].double().cpu().numpy().astype(np.float32)
        w = test["lam"][i].double().cpu().numpy().astype(np.float32)
        for mode in ("cold", "warm"):
            f0 = test["start"][i][mode].cpu().numpy()
            got, k = test["result"][i][mode]
            p = synth.Params(**{**c.params.__dict__, "k_outer": k})
            ref, _, _ = oracle_mod.reconstruct(G, y, w, f0, p)
            err = float(np.linalg.norm(got.double().cpu().numpy() - ref) / np.linalg.norm(ref))
            print(f"slice {i} {mode}: {k} iterations, rel. L2 vs FP64 oracle {err:.2e}")
            assert err <= 1e-4
