"""Pins of the warm-start network oracle (oracle/unet_oracle.py).

Gradients are checked against central finite differences (FP64, no BF16
rounding), the convolution against scipy's correlation, and the network's
structure by the identity it computes with a zero final layer.
"""
import numpy as np
import pytest

scipy_signal = pytest.importorskip("scipy.signal")


@pytest.fixture(scope="module")
def un():
    from oracle import unet_oracle
    return unet_oracle


def test_conv3_is_a_padded_correlation(un):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = un.conv3(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = sum(scipy_signal.correlate2d(x[bi, c], w[o, c], mode="same") for c in range(3)) + b[o]
            np.testing.assert_allclose(got[bi, o], ref, rtol=1e-12, atol=1e-12)


def test_zero_final_layer_gives_the_identity(un):
    rng = np.random.default_rng(2)
    params = un.init_params(3, 3, 2, 3, seed=5)
    x = rng.random((1, 3, 16, 16))
    out, _ = un.forward(params, x, 3, bf16_storage=False)
    np.testing.assert_array_equal(out, x)


def test_pool_and_upsample_adjoint_pairs(un):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 8, 6))
    g = rng.standard_normal((2, 3, 4, 3))
    # <up2(g), x> = <g, up2^T(x)>
    assert abs(np.sum(un.up2(g) * x) - np.sum(g * un.up2_backward(x))) < 1e-12
    # the pooling gradient routes each output gradient to one argmax
    gp = un.maxpool2_backward(x, g)
    assert np.count_nonzero(gp) == np.count_nonzero(g)
    assert abs(gp.sum() - g.sum()) < 1e-12


def test_gradients_match_finite_differences(un):
    rng = np.random.default_rng(4)
    L = 2
    params = un.init_params(3, 3, 2, L, seed=7)
    params = [(w + 0.1 * rng.standard_normal(w.shape), b + 0.1 * rng.standard_normal(b.shape))
              for w, b in params]
    x = rng.random((2, 3, 8, 8))
    t = rng.random((2, 3, 8, 8))
    loss, grads, _ = un.loss_and_grads(params, x, t, L, bf16_storage=False)
    eps = 1e-6
    for li in range(len(params)):
        w, b = params[li]
        for which, arr in ((0, w), (1, b)):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = un.loss_and_grads(params, x, t, L, bf16_storage=False)[0]
                flat[idx] = old - eps
                lm = un.loss_and_grads(params, x, t, L, bf16_storage=False)[0]
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                an = grads[li][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (li, which, idx, fd, an)


def test_bf16_rounding_is_nearest_even(un):
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8, -3.140625, 1e-3], dtype=np.float32)
    r = un.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # halfway, ties to even
    assert r[2] == 1.0 + 2 ** -6           # halfway, ties to even (odd lsb rounds up)
    assert r[3] == -3.140625
    assert abs(r[4] - 1e-3) <= 2 ** -9 * 1e-3


@pytest.mark.parametrize("cin,base,L,H,W,B", [(3, 4, 2, 16, 24, 2), (10, 8, 3, 32, 32, 2)])
def test_bf16_storage_stays_within_the_roundoff_bound(cin, base, L, H, W, B):
    """The oracle rounding at the GPU's points differs from the plain FP64
    network by less than the first-order bound the GPU tests use: u = 2^-8
    per rounding point, 2 + 2 n3 points on the correction, 1 + 3 n3 on every
    parameter gradient (n3 = number of 3x3 layers)."""
    from oracle import unet_oracle as un
    rng = np.random.default_rng(100 + L)
    p = un.init_params(cin, cin, base, L, 100 + L)
    p = [((w + 0.05 * rng.standard_normal(w.shape)).astype(np.float32).astype(np.float64),
          (b + 0.05 * rng.standard_normal(b.shape)).astype(np.float32).astype(np.float64)) for w, b in p]
    x = np.random.default_rng(7).random((B, cin, H, W)).astype(np.float32).astype(np.float64)
    t = x + 0.1 * np.random.default_rng(8).standard_normal(x.shape)
    n3 = 2 * L + 2 * (L - 1)
    u = 2.0 ** -8
    o1, _ = un.forward(p, x, L, bf16_storage=True)
    o0, _ = un.forward(p, x, L, bf16_storage=False)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(o1 - un.bf16(x), o0 - x) <= u * (2 + 2 * n3)
    _, g1, _ = un.loss_and_grads(p, x, t, L, bf16_storage=True)
    _, g0, _ = un.loss_and_grads(p, x, t, L, bf16_storage=False)
    for (w1, b1), (w0, b0) in zip(g1, g0):
        assert rel(w1, w0) <= u * (1 + 3 * n3)
        assert rel(b1, b0) <= u * (1 + 3 * n3)
