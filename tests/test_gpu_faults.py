"""Failure handling of the C ABI on a GPU, all provoked from the host:
bad arguments, an injected allocation failure, non-finite inputs, and a
pipeline wait of the TMA sweep that runs out (its poll limit lowered to
zero, so no wait blocks at all).  No test here makes a kernel fault, trap
or hang."""
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


@pytest.fixture(scope="module")
def case():
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    dv = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    return c, dv(d["y"]), dv(d["w"]), dv(np.full((10, 64, 64), 0.01))


@pytest.mark.parametrize("bad", [dict(patch=4), dict(patch=17), dict(window=33), dict(window=0),
                                 dict(h=0.0), dict(h=float("nan")), dict(mu_hat=-1.0),
                                 dict(data_step=2), dict(data_step=1, beta=0.0), dict(m1=-1),
                                 dict(clamp=2)])
def test_invalid_params_are_rejected(tn, case, bad):
    c, y, w, f0 = case
    geo = tn.tnlm_create_geometry(c.geom)
    p = synth.Params(**{**c.params.__dict__, **bad})
    f = f0.clone()
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, p, y, w, f)
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG
    assert torch.equal(f, f0)


def test_misaligned_pointer_is_rejected(tn, case):
    c, y, w, f0 = case
    geo = tn.tnlm_create_geometry(c.geom)
    big = torch.zeros(f0.numel() + 4, device="cuda")
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, c.params, y, w, big.data_ptr() + 4)
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG


def test_injected_allocation_failure_reports_oom_and_recovers(tn, case):
    c, y, w, f0 = case
    p = synth.Params(**{**c.params.__dict__, "k_outer": 2})
    # one full create / reconstruct / destroy cycle first: the driver keeps
    # some memory after the first CUDA-graph instantiation, which is not a leak
    warm = tn.tnlm_create_geometry(c.geom)
    tn.tnlm_reconstruct(warm, p, y, w, f0.clone())
    warm.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    tn.tnlm_debug_fail_alloc_after(1)          # the geometry's first table
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_create_geometry(c.geom)
    assert e.value.status == tn.TNLM_ERR_OOM
    geo = tn.tnlm_create_geometry(c.geom)
    tn.tnlm_debug_fail_alloc_after(1)          # the workspace
    f = f0.clone()
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, p, y, w, f)
    assert e.value.status == tn.TNLM_ERR_OOM
    assert torch.equal(f, f0)
    tn.tnlm_reconstruct(geo, p, y, w, f)       # works afterwards
    geo2 = tn.tnlm_create_geometry(c.geom)
    f2 = f0.clone()
    tn.tnlm_reconstruct(geo2, p, y, w, f2)
    assert torch.equal(f, f2)
    geo.close()
    geo2.close()
    torch.cuda.synchronize()
    # nothing leaked (free memory may also grow when the driver trims its caches)
    assert free0 - torch.cuda.mem_get_info()[0] < (4 << 20)


def test_nonfinite_input_raises_numeric(tn, case):
    c, y, w, f0 = case
    geo = tn.tnlm_create_geometry(c.geom)
    p = synth.Params(**{**c.params.__dict__, "k_outer": 1})
    ybad = y.clone()
    ybad[3, 10, 20] = float("nan")
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, p, ybad, w, f0.clone())
    assert e.value.status == tn.TNLM_ERR_NUMERIC
    wbad = w.clone()
    wbad[0, 0, 0] = -1.0
    with pytest.raises(tn.TnlmError) as e:
        tn.tnlm_reconstruct(geo, p, y, wbad, f0.clone())
    assert e.value.status == tn.TNLM_ERR_NUMERIC
    # the flag is cleared once reported
    tn.tnlm_reconstruct(geo, p, y, w, f0.clone())


def test_sweep_wait_timeout_is_reported_and_the_handle_recovers(tn, case):
    """With the sweep's pipeline waits limited to zero polls every wait gives
    up at once: the sweep blocks stop issuing copies, drain the ones in
    flight (with the normal limit) and flag a timeout, which the
    synchronising call reports as TNLM_ERR_TIMEOUT.  With the limit restored
    the same handle reconstructs exactly as a fresh one."""
    c, y, w, f0 = case
    p = synth.Params(**{**c.params.__dict__, "k_outer": 1})   # eager launches, no captured graph
    geo = tn.tnlm_create_geometry(c.geom)
    f = f0.clone()
    tn.tnlm_debug_wait_limit(0)
    try:
        with pytest.raises(tn.TnlmError) as e:
            tn.tnlm_reconstruct(geo, p, y, w, f)
    finally:
        tn.tnlm_debug_wait_limit(-1)
    assert e.value.status == tn.TNLM_ERR_TIMEOUT
    assert "timed out" in str(e.value)
    torch.cuda.synchronize()
    a = f0.clone()
    rep = tn.tnlm_reconstruct(geo, p, y, w, a)
    fresh = tn.tnlm_create_geometry(c.geom)
    b = f0.clone()
    tn.tnlm_reconstruct(fresh, p, y, w, b)
    torch.cuda.synchronize()
    assert rep["iterations"] == 1
    assert torch.equal(a, b)


def test_wait_limit_applies_to_cached_graphs(tn, case):
    """A reconstruction with K > 1 replays a captured graph of one outer
    iteration; the sweep's wait limit is a kernel argument, so lowering it
    must re-capture (every replay then times out) and restoring it must
    re-capture again (the handle then matches a fresh one bitwise)."""
    c, y, w, f0 = case
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3})
    geo = tn.tnlm_create_geometry(c.geom)
    tn.tnlm_reconstruct(geo, p, y, w, f0.clone())          # graph captured with the normal limit
    tn.tnlm_debug_wait_limit(0)
    try:
        with pytest.raises(tn.TnlmError) as e:
            tn.tnlm_reconstruct(geo, p, y, w, f0.clone())
    finally:
        tn.tnlm_debug_wait_limit(-1)
    assert e.value.status == tn.TNLM_ERR_TIMEOUT
    a = f0.clone()
    tn.tnlm_reconstruct(geo, p, y, w, a)
    b = f0.clone()
    tn.tnlm_reconstruct(tn.tnlm_create_geometry(c.geom), p, y, w, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_cached_graph_follows_workspace_reallocation(tn, case):
    """The weights call with a wider window grows (re-allocates) the
    handle's workspace, whose buffer offsets depend on the window; a later
    reconstruction with the first parameters must not replay the graph
    captured on the old layout, even if the new allocation reuses its
    address."""
    c, y, w, f0 = case
    p = synth.Params(**{**c.params.__dict__, "k_outer": 3})
    geo = tn.tnlm_create_geometry(c.geom)
    tn.tnlm_reconstruct(geo, p, y, w, f0.clone())
    N, ny, nx = f0.shape
    for W in (9, 11):
        q = synth.Params(**{**c.params.__dict__, "window": W})
        nd, nn = tn.tnlm_weights_size(geo, q)
        dist = torch.empty(nd // 4, device="cuda")
        norm = torch.empty(nn // 4, device="cuda")
        tn.tnlm_weights(geo, q, f0, dist, norm)
        del dist, norm
    a = f0.clone()
    tn.tnlm_reconstruct(geo, p, y, w, a)
    b = f0.clone()
    tn.tnlm_reconstruct(tn.tnlm_create_geometry(c.geom), p, y, w, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
