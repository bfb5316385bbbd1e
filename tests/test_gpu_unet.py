"""Learned warm start on the GPU: per-phase FBP and the U-Net kernels
against the FP64 oracles.

The network oracle emulates the GPU's BF16 storage points, so the two
differ by FP32 accumulation order only, plus the activations whose BF16
rounding flips with it.  Each flip is one BF16 unit, so the difference is
bounded by the size of the BF16 storage effect itself (oracle with vs
without BF16 rounding), which grows with depth.  Forward outputs must agree
to relative L2 <= max(2e-3, that effect), parameter gradients per layer to
<= max(1e-2, twice the effect on that layer's gradient).
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
    assert torch.cuda.is_available()
    return tn


@pytest.fixture(scope="module")
def un():
    from oracle import unet_oracle
    return unet_oracle


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def unflat(v, params):
    out, o = [], 0
    for w, b in params:
        out.append((v[o:o + w.size].reshape(w.shape).astype(np.float64),
                    v[o + w.size:o + w.size + b.size].astype(np.float64)))
        o += w.size + b.size
    return out


def random_net(un, cin, cout, base, L, seed):
    rng = np.random.default_rng(seed)
    p = un.init_params(cin, cout, base, L, seed)
    p = [(w + 0.05 * rng.standard_normal(w.shape), b + 0.05 * rng.standard_normal(b.shape)) for w, b in p]
    return [(w.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for w, b in p]


def test_fbp_phases_matches_oracle(tn, oracle_mod):
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    g = c.geom
    geo = tn.tnlm_create_geometry(g)
    out = torch.zeros((g.n_phases, g.ny, g.nx), device="cuda")
    tn.tnlm_fbp_phases(geo, dev(d["y"]), out)
    got = out.double().cpu().numpy()
    ang = g.view_angles().reshape(g.n_phases, g.n_views)
    for i in (0, 3, 9):
        yi = np.tile(d["y"][i].astype(np.float32), (g.n_phases, 1, 1))
        ref = oracle_mod.fbp(oracle_mod.Geom(g, angles=np.tile(ang[i], g.n_phases)), yi)[0]
        assert rel(got[i], ref) <= 1e-5


@pytest.mark.parametrize("cin,base,L,H,W,B", [(3, 4, 2, 16, 24, 2), (10, 8, 3, 32, 32, 2), (10, 32, 4, 64, 64, 1)])
def test_unet_forward_and_gradients_match_oracle(tn, un, cin, base, L, H, W, B):
    params = random_net(un, cin, cin, base, L, seed=100 + L)
    rng = np.random.default_rng(7)
    x = rng.random((B, cin, H, W)).astype(np.float32).astype(np.float64)
    t = (x + 0.1 * rng.standard_normal(x.shape)).astype(np.float32).astype(np.float64)
    net = tn.UNet(cin, cin, base, L)
    assert net.param_count == flat(params).size
    net.set_params(flat(params))
    out = torch.zeros((B, cin, H, W), device="cuda")
    net.forward(dev(x), out)
    ref_out, _ = un.forward(params, x, L, bf16_storage=True)
    fp_out, _ = un.forward(params, x, L, bf16_storage=False)
    eff = rel(ref_out, fp_out)
    assert rel(out.double().cpu().numpy(), ref_out) <= max(2e-3, eff)
    loss = net.grads(dev(x), dev(t))
    ref_loss, ref_grads, _ = un.loss_and_grads(params, x, t, L, bf16_storage=True)
    _, fp_grads, _ = un.loss_and_grads(params, x, t, L, bf16_storage=False)
    assert abs(loss - ref_loss) <= max(1e-3, eff) * ref_loss
    _, g = net.get_params(grads=True)
    got = unflat(g, params)
    for k, ((gw, gb), (rw, rb), (fw, fb)) in enumerate(zip(got, ref_grads, fp_grads)):
        assert rel(gw, rw) <= max(1e-2, 2 * rel(rw, fw)), (k, rel(gw, rw), rel(rw, fw))
        assert rel(gb, rb) <= max(1e-2, 2 * rel(rb, fb)), (k, rel(gb, rb), rel(rb, fb))


def test_unet_training_lowers_the_loss_and_is_deterministic(tn, un):
    params = random_net(un, 4, 4, 8, 3, seed=3)
    rng = np.random.default_rng(11)
    x = rng.random((4, 4, 32, 32))
    t = 0.5 * x + 0.1
    losses = []
    finals = []
    for rep in range(2):
        net = tn.UNet(4, 4, 8, 3)
        net.set_params(flat(params))
        ls = []
        for _ in range(20):
            ls.append(net.grads(dev(x), dev(t)))
            net.adam_step(1e-3)
        losses.append(ls)
        finals.append(net.get_params())
    assert losses[0][-1] < 0.5 * losses[0][0]
    assert losses[0] == losses[1]
    assert np.array_equal(finals[0], finals[1])


def test_unet_rejects_bad_sizes(tn):
    net = tn.UNet(4, 4, 8, 3)
    x = torch.zeros((1, 4, 30, 32), device="cuda")
    with pytest.raises(tn.TnlmError) as e:
        net.forward(x, x.clone())
    assert e.value.status == tn.TNLM_ERR_INVALID_ARG
