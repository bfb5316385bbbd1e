"""Learned warm start on the GPU: per-phase FBP and the U-Net kernels
against the FP64 oracles.

The GPU stores the input, the weights and every post-ReLU activation in
BF16 and takes the gradient entering each 3x3 backward product as BF16
(the tensor cores multiply two operands of one 16-bit type), accumulating
in FP32.  The kernels are held to a fixed bound derived from BF16's unit
roundoff u = 2^-8 and the depth of the network, against the plain FP64
oracle (no rounding anywhere) and against the oracle that rounds at the
GPU's points.  To first order each rounding point perturbs what flows
through it by at most u relative (a ReLU mask that flips does so only for a
pre-activation within that perturbation of zero), and the perturbations add
along the paths.  With n3 the number of 3x3 layers:
  * the network's correction (output - input) passes 2 + 2 n3 rounding
    points (input, every layer's weights and output, the final weights):
    relative L2 <= u (2 + 2 n3);
  * every parameter gradient depends on the whole forward pass and on the
    gradients rounded at each 3x3 backward product: relative L2 <=
    u (1 + 3 n3);
  * the loss (a sum of squares of the residual): relative <= u (2 + 2 n3).
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


U_BF16 = 2.0 ** -8


@pytest.mark.parametrize("cin,base,L,H,W,B", [(3, 4, 2, 16, 24, 2), (10, 8, 3, 32, 32, 2), (10, 32, 4, 64, 64, 1)])
def test_unet_forward_and_gradients_match_oracle(tn, un, cin, base, L, H, W, B):
    params = random_net(un, cin, cin, base, L, seed=100 + L)
    rng = np.random.default_rng(7)
    x = rng.random((B, cin, H, W)).astype(np.float32).astype(np.float64)
    t = (x + 0.1 * rng.standard_normal(x.shape)).astype(np.float32).astype(np.float64)
    n3 = 2 * L + 2 * (L - 1)
    tol_fwd = U_BF16 * (2 + 2 * n3)
    tol_grad = U_BF16 * (1 + 3 * n3)
    net = tn.UNet(cin, cin, base, L)
    assert net.param_count == flat(params).size
    net.set_params(flat(params))
    out = torch.zeros((B, cin, H, W), device="cuda")
    net.forward(dev(x), out)
    got_out = out.double().cpu().numpy()
    xq = un.bf16(x)                      # the input as the network stores it
    loss = net.grads(dev(x), dev(t))
    _, g = net.get_params(grads=True)
    got = unflat(g, params)
    for emulate in (False, True):
        ref_out, _ = un.forward(params, x, L, bf16_storage=emulate)
        ref_loss, ref_grads, _ = un.loss_and_grads(params, x, t, L, bf16_storage=emulate)
        base_in = xq if emulate else x
        # the correction the network adds to its (BF16-stored) input
        assert rel(got_out - xq, ref_out - base_in) <= tol_fwd, (emulate, rel(got_out - xq, ref_out - base_in))
        assert rel(got_out, ref_out) <= tol_fwd
        assert abs(loss - ref_loss) <= tol_fwd * ref_loss
        for k, ((gw, gb), (rw, rb)) in enumerate(zip(got, ref_grads)):
            assert rel(gw, rw) <= tol_grad, (emulate, k, rel(gw, rw), tol_grad)
            assert rel(gb, rb) <= tol_grad, (emulate, k, rel(gb, rb), tol_grad)


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
