"""Batched reconstruction and the launch autotuner (GPU, through the C ABI).

A batch must give every slice bitwise the result of its own
tnlm_reconstruct call, including where it stops under its own tolerance.  The autotuner's sweep tiling leaves results bitwise
unchanged; its choice of backprojection view groups reorders FP32 sums, so
results after it agree with the default to rounding (rel. L2 <= 1e-6).  One
slice of the batch is also checked against the FP64 oracle.
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


def small_slices():
    """Uneven slices: sizes, view counts, windows and iteration counts differ."""
    out = []
    specs = [(64, 48, 40, 96, 3, 5, 3), (48, 48, 24, 80, 3, 7, 4), (70, 52, 30, 110, 5, 5, 2),
             (32, 40, 16, 64, 1, 3, 3)]
    for k, (nx, ny, V, B, d, W, K) in enumerate(specs):
        g = synth.Geometry(nx=nx, ny=ny, pixel_mm=64.0 / max(nx, ny), n_phases=4 + k % 2, n_views=V,
                           n_bins=B, bin_mm=1.2, sid_mm=500.0, sdd_mm=800.0)
        c = synth.Case(f"s{k}", g, synth.Params(patch=d, window=W, k_outer=K, m2=3, h=0.002 * d),
                       1e4 * (k + 1), 1100 + k, k % 2 == 1)
        out.append(c)
    return out


def inputs(c):
    d = synth.make_inputs(c)
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01)
    return d, f0


def test_batch_replays_match_single_calls_bitwise(tn, monkeypatch):
    """The replay path (one graph of one outer iteration of the live slices,
    launched once per iteration) gives every slice its single-call result."""
    monkeypatch.setenv("TNLM_BATCH_REPLAY", "1")
    cases = small_slices()
    geoms, ys, ws, fs, ref = [], [], [], [], []
    for c in cases:
        d, f0 = inputs(c)
        g = tn.tnlm_create_geometry(c.geom)
        f = dev(f0)
        rep = tn.tnlm_reconstruct(g, c.params, dev(d["y"]), dev(d["w"]), f)
        ref.append((f.clone(), rep))
        geoms.append(tn.tnlm_create_geometry(c.geom))
        ys.append(dev(d["y"]))
        ws.append(dev(d["w"]))
        fs.append(dev(f0))
    reps = tn.tnlm_reconstruct_batch(geoms, [c.params for c in cases], ys, ws, fs, autotune=False)
    torch.cuda.synchronize()
    assert not tn.tnlm_batch_last_was_loop()
    for c, f, (fr, rr), r in zip(cases, fs, ref, reps):
        assert torch.equal(f, fr), c.name
        assert r["iterations"] == c.params.k_outer
        assert r["rel_change_hist"] == rr["rel_change_hist"]
        assert r["residual_hist"] == rr["residual_hist"]
    # a second call replays the cached graph and continues from the results
    fs2 = [f.clone() for f in fs]
    tn.tnlm_reconstruct_batch(geoms, [c.params for c in cases], ys, ws, fs2, autotune=False)
    for c, g, y, w, f, f2 in zip(cases, geoms, ys, ws, fs, fs2):
        f1 = f.clone()
        tn.tnlm_reconstruct(g, c.params, y, w, f1)
        assert torch.equal(f1, f2), c.name


def run_pair(tn, cases, plist):
    """Single tnlm_reconstruct calls and one batched call on the same inputs."""
    geoms, ys, ws, fs, ref, ref_it = [], [], [], [], [], []
    for c, p in zip(cases, plist):
        d, f0 = inputs(c)
        g = tn.tnlm_create_geometry(c.geom)
        f = dev(f0)
        rep = tn.tnlm_reconstruct(g, p, dev(d["y"]), dev(d["w"]), f)
        ref.append(f)
        ref_it.append(rep["iterations"])
        geoms.append(tn.tnlm_create_geometry(c.geom))
        ys.append(dev(d["y"])); ws.append(dev(d["w"])); fs.append(dev(f0))
    return geoms, ys, ws, fs, ref, ref_it


def test_batch_runs_as_one_loop_graph_and_matches_single_calls(tn):
    """Uneven iteration counts: the whole run is one graph launch (a
    device-side WHILE loop whose gate runs each slice's iteration while it
    has one left); the results are bitwise those of separate calls, also
    when the cached loop graph is launched again."""
    cases = small_slices()
    plist = [c.params for c in cases]
    assert len({p.k_outer for p in plist}) > 1
    geoms, ys, ws, fs, ref, ref_it = run_pair(tn, cases, plist)
    for rep in range(2):
        fr = [f.clone() for f in fs]
        reps = tn.tnlm_reconstruct_batch(geoms, plist, ys, ws, fr, autotune=False)
        torch.cuda.synchronize()
        assert tn.tnlm_batch_last_was_loop()
        for c, f, r, rp in zip(cases, fr, ref, reps):
            assert torch.equal(f, r), (rep, c.name)
            assert rp["iterations"] == c.params.k_outer


def tol_params(cases, rules):
    import types
    return [types.SimpleNamespace(**{**c.params.__dict__, "k_outer": k, "tol": tol, "tol_check_every": ev})
            for c, (k, tol, ev) in zip(cases, rules)]


@pytest.mark.parametrize("replay", [False, True])
def test_batch_stops_each_slice_at_its_tolerance(tn, monkeypatch, replay):
    """Every slice its own stopping rule (tolerance, check interval, cap):
    the batched launch (gate on the device; or, replaying, checks on the
    host) stops each slice at the iteration where its own tnlm_reconstruct
    call stops, with bitwise the same image.  A second call with other
    tolerances reuses the cached loop graph (the rules live in device
    memory, not in the graph)."""
    if replay:
        monkeypatch.setenv("TNLM_BATCH_REPLAY", "1")
    cases = small_slices()
    for rules in ([(12, 0.03, 1), (12, 0.01, 2), (7, 0.0, 1), (12, 0.05, 3)],
                  [(12, 0.015, 1), (12, 0.02, 2), (9, 0.0, 1), (12, 0.03, 2)]):
        plist = tol_params(cases, rules)
        geoms, ys, ws, fs, ref, ref_it = run_pair(tn, cases, plist)
        assert any(it < p.k_outer for it, p in zip(ref_it, plist))   # some tolerance fired
        assert len(set(ref_it)) > 1
        reps = tn.tnlm_reconstruct_batch(geoms, plist, ys, ws, fs, autotune=False)
        torch.cuda.synchronize()
        assert tn.tnlm_batch_last_was_loop() != replay
        for c, f, r, it, rp in zip(cases, fs, ref, ref_it, reps):
            assert rp["iterations"] == it, (c.name, rp["iterations"], it)
            assert torch.equal(f, r), c.name


def test_batch_slice_matches_oracle(tn, oracle_mod):
    c = small_slices()[1]
    d, f0 = inputs(c)
    others = small_slices()[2:]
    geoms = [tn.tnlm_create_geometry(c.geom)] + [tn.tnlm_create_geometry(o.geom) for o in others]
    ins = [(d, f0)] + [inputs(o) for o in others]
    fs = [dev(x[1]) for x in ins]
    tn.tnlm_reconstruct_batch(geoms, [c.params] + [o.params for o in others],
                              [dev(x[0]["y"]) for x in ins], [dev(x[0]["w"]) for x in ins], fs)
    torch.cuda.synchronize()
    fo, _, _ = oracle_mod.reconstruct(oracle_mod.Geom(c.geom), d["y"], d["w"], f0, c.params)
    got = fs[0].double().cpu().numpy()
    err = np.linalg.norm(got - fo) / np.linalg.norm(fo)
    assert err <= REC_TOL, err


def test_autotune_choices_leave_results_unchanged(tn):
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3})
    y, w = dev(d["y"]), dev(d["w"])
    f0 = dev(np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01))
    g = tn.tnlm_create_geometry(c.geom)
    f_default = f0.clone()
    tn.tnlm_reconstruct(g, p, y, w, f_default)
    keep = f0.clone()
    choice = tn.tnlm_autotune(g, p, y, w, f0)
    assert torch.equal(f0, keep)                       # the start image is untouched
    assert 1 <= choice["bp_groups"] <= 4 and 1 <= choice["gj_tiles"] <= 3 and choice["gj_split"] in (1, 2)
    f_tuned = f0.clone()
    tn.tnlm_reconstruct(g, p, y, w, f_tuned)
    a, b = f_tuned.double(), f_default.double()
    assert float((a - b).norm() / b.norm()) <= 1e-6
    f_again = f0.clone()
    tn.tnlm_reconstruct(g, p, y, w, f_again)
    assert torch.equal(f_again, f_tuned)               # deterministic under the choice
    # a second handle of the same shape takes the cached choice
    g2 = tn.tnlm_create_geometry(c.geom)
    assert tn.tnlm_autotune(g2, p, y, w, f0) == choice


def test_batch_rejects_repeated_handles(tn):
    c = small_slices()[0]
    d, f0 = inputs(c)
    g = tn.tnlm_create_geometry(c.geom)
    y, w, f = dev(d["y"]), dev(d["w"]), dev(f0)
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct_batch([g, g], [c.params, c.params], [y, y], [w, w], [f, f.clone()])
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG
    assert "repeats" in str(e.value)
    assert torch.equal(f, dev(f0))                     # nothing ran


def test_batch_workload_sampled_slices_match_oracle(tn, oracle_mod):
    """Four slices sampled from the 64-slice batched workload (one per side
    length and a 60-view one), mixed-precision patch distances, batched and
    autotuned, after K = 2 outer iterations: relative L2 <= 1e-3 against the
    FP64 oracle (the workload's accuracy bound)."""
    from tests.golden import make_golden
    items = synth.batch_cases(64)
    pick = make_golden.batch_pick(items)
    geoms, ps, ys, ws, fs, ins = [], [], [], [], [], []
    for i in pick:
        c, off = items[i]
        d = synth.make_inputs(c, off)
        p = synth.Params(**{**c.params.__dict__, "k_outer": 2})
        f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01)
        geoms.append(tn.tnlm_create_geometry(c.geom))
        ps.append(p)
        ys.append(dev(d["y"]))
        ws.append(dev(d["w"]))
        fs.append(dev(f0))
        ins.append((c, d, f0, p))
    tn.tnlm_reconstruct_batch(geoms, ps, ys, ws, fs, autotune=True)
    torch.cuda.synchronize()
    for (c, d, f0, p), f in zip(ins, fs):
        ref, _, _ = oracle_mod.reconstruct(oracle_mod.Geom(c.geom), d["y"].astype(np.float32),
                                           d["w"].astype(np.float32), f0.astype(np.float32), p)
        got = f.double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (c.name, err)


def test_batch_workload_sampled_slices_at_full_k_match_the_stored_oracle(tn):
    """The same four sampled slices at the workload's own K = 50, run the way
    the batched workload runs (mixed-precision patch distances, autotuned,
    one batched launch), against the FP64 oracle's values stored in
    tests/golden/batch<i>_k50.txt (written by tests/golden/make_golden.py
    from the oracle alone): 4096 seeded pixels per slice within relative L2
    1e-3, the workload's accuracy bound."""
    from tests.golden import make_golden
    items = synth.batch_cases(64)
    pick = make_golden.batch_pick(items)
    golds = [make_golden.read_batch(i) for i in pick]
    if any(gd is None for gd in golds):
        pytest.skip("tests/golden/batch*_k50.txt not written")
    geoms, ps, ys, ws, fs = [], [], [], [], []
    for i in pick:
        c, off = items[i]
        assert c.params.k_outer == make_golden.BATCH_K and c.params.precision == tn.PREC_MIXED
        d = synth.make_inputs(c, off)
        geoms.append(tn.tnlm_create_geometry(c.geom))
        ps.append(c.params)
        ys.append(dev(d["y"]))
        ws.append(dev(d["w"]))
        fs.append(dev(np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01)))
    reps = tn.tnlm_reconstruct_batch(geoms, ps, ys, ws, fs, autotune=True)
    torch.cuda.synchronize()
    for i, f, gd, r in zip(pick, fs, golds, reps):
        assert r["iterations"] == make_golden.BATCH_K
        pix = gd[1]
        got_f = f.double().cpu().numpy()
        got = np.array([got_f[a, y, x] for a, y, x, _ in pix])
        want = np.array([v for _, _, _, v in pix])
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        assert err <= 1e-3, (i, err)


def test_batch_edge_rules_zero_iterations_and_first_check(tn):
    """Degenerate stopping rules in one batched launch: a slice with K = 0
    is left untouched, a slice whose tolerance holds at its first check stops
    after one iteration, the others run their K; each matches its single
    call bitwise."""
    cases = small_slices()
    rules = [(0, 0.0, 1), (6, 1.0, 1), (4, 0.0, 1), (5, 0.0, 1)]
    plist = tol_params(cases, rules)
    geoms, ys, ws, fs, ref, ref_it = run_pair(tn, cases, plist)
    assert ref_it == [0, 1, 4, 5]
    f_before = [f.clone() for f in fs]
    reps = tn.tnlm_reconstruct_batch(geoms, plist, ys, ws, fs, autotune=False)
    torch.cuda.synchronize()
    assert tn.tnlm_batch_last_was_loop()
    assert [r["iterations"] for r in reps] == ref_it
    assert torch.equal(fs[0], f_before[0])
    for c, f, r in zip(cases, fs, ref):
        assert torch.equal(f, r), c.name
