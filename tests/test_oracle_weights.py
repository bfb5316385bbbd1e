"""Pins of the oracle's TNLM weights (Eq. 8, Eq. 3 normalisation, Sec. 2.3).

Pinned against: an independent numpy box-sum evaluation of the patch
distances, the row normalisation sum_y omega = 1, the symmetric reuse of
the unnormalised weight between the two directions of a pair (Sec. 2.3),
and the uniform / concentrated limits of the Gaussian kernel.
"""
import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view


def numpy_distances(g, d, W):
    """D[i, y, x, s] = sum over the d x d patch of (g_i(x+p) - g_{i+1}(x+s+p))^2,
    zero outside the image, +inf where x+s is outside.  Box sums by windows."""
    N, ny, nx = g.shape
    r, rho = (d - 1) // 2, (W - 1) // 2
    pad = r + rho
    gp = np.pad(g, ((0, 0), (pad, pad), (pad, pad)))
    out = np.full((N, ny, nx, W * W), np.inf)
    yy, xx = np.mgrid[0:ny, 0:nx]
    for i in range(N):
        a = gp[i]
        b = gp[(i + 1) % N]
        for sy in range(-rho, rho + 1):
            for sx in range(-rho, rho + 1):
                bs = np.roll(b, (-sy, -sx), axis=(0, 1))
                e2 = (a - bs) ** 2
                box = sliding_window_view(e2, (d, d)).sum(axis=(2, 3))
                Dm = box[rho:rho + ny, rho:rho + nx]
                valid = (xx + sx >= 0) & (xx + sx < nx) & (yy + sy >= 0) & (yy + sy < ny)
                out[i, :, :, (sy + rho) * W + sx + rho] = np.where(valid, Dm, np.inf)
    return out


def stable_rows(D, h):
    m = D.min(axis=-1, keepdims=True)
    e = np.where(np.isinf(D), 0.0, np.exp(-(D - m) / h ** 2))
    return e / e.sum(axis=-1, keepdims=True)


@pytest.fixture(scope="module")
def imgs():
    rng = np.random.default_rng(11)
    return 0.02 * rng.random((4, 9, 11))


@pytest.mark.parametrize("d,W", [(3, 5), (5, 3), (1, 3), (3, 7)])
def test_patch_distances_match_independent_box_sums(oracle_mod, imgs, d, W):
    wn, wp, dn = oracle_mod.weights(imgs, d, W, 0.01, with_dist=True)
    ref = numpy_distances(imgs, d, W)
    assert np.array_equal(np.isinf(dn), np.isinf(ref))
    fin = np.isfinite(ref)
    np.testing.assert_allclose(dn[fin], ref[fin], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(wn, stable_rows(ref, 0.01), rtol=1e-10, atol=1e-14)


def test_rows_sum_to_one_and_are_nonnegative(oracle_mod, imgs):
    wn, wp = oracle_mod.weights(imgs, 3, 5, 0.005)
    for w in (wn, wp):
        assert (w >= 0).all()
        np.testing.assert_allclose(w.sum(-1), 1.0, rtol=0, atol=1e-12)


def test_symmetric_reuse_between_directions(oracle_mod, imgs):
    """omega_{i+1,i}(y, y+s') is the row-normalised exp(-D_{i,i+1}(y+s', -s')/h^2):
    the unnormalised weight of a pair is shared by both directions."""
    d, W, h = 3, 5, 0.008
    wn, wp, dn = oracle_mod.weights(imgs, d, W, h, with_dist=True)
    N, ny, nx, _ = dn.shape
    rho = (W - 1) // 2
    for i in range(N):
        j = (i + 1) % N
        Drev = np.full((ny, nx, W * W), np.inf)
        for sy in range(-rho, rho + 1):
            for sx in range(-rho, rho + 1):
                k = (sy + rho) * W + sx + rho
                kneg = (-sy + rho) * W + (-sx + rho)
                for y in range(ny):
                    for x in range(nx):
                        x1, y1 = x + sx, y + sy
                        if 0 <= x1 < nx and 0 <= y1 < ny:
                            Drev[y, x, k] = dn[i, y1, x1, kneg]
        np.testing.assert_allclose(wp[j], stable_rows(Drev, h), rtol=1e-10, atol=1e-14)


def _valid_counts(ny, nx, W):
    rho = (W - 1) // 2
    yy, xx = np.mgrid[0:ny, 0:nx]
    cx = np.minimum(xx + rho, nx - 1) - np.maximum(xx - rho, 0) + 1
    cy = np.minimum(yy + rho, ny - 1) - np.maximum(yy - rho, 0) + 1
    return cx * cy


def test_constant_images_give_uniform_weights(oracle_mod):
    """Constant, equal images: every candidate in the image is equally similar
    in the interior; rows are uniform over the valid candidates there."""
    g = np.full((3, 10, 12), 0.015)
    wn, wp = oracle_mod.weights(g, 1, 5, 0.001)
    cnt = _valid_counts(10, 12, 5)
    for w in (wn, wp):
        nz = w > 0
        np.testing.assert_array_equal(nz.sum(-1), np.broadcast_to(cnt, nz.sum(-1).shape))
        np.testing.assert_allclose(w.max(-1), np.broadcast_to(1.0 / cnt, w.shape[:-1]), rtol=1e-12)


def test_large_h_gives_uniform_weights(oracle_mod, imgs):
    wn, wp = oracle_mod.weights(imgs, 3, 5, 1e6)
    cnt = _valid_counts(imgs.shape[1], imgs.shape[2], 5)
    for w in (wn, wp):
        ref = np.broadcast_to(1.0 / cnt, w.shape[:-1])
        np.testing.assert_allclose(w.max(-1), ref, rtol=1e-9)
        np.testing.assert_allclose(np.where(w > 0, w, np.inf).min(-1), ref, rtol=1e-9)


def test_shifted_phase_concentrates_weight_at_the_shift(oracle_mod):
    """g_{i+1}(x) = g_i(x - s0): as h -> 0 the weight of an interior pixel
    concentrates on the candidate x + s0."""
    rng = np.random.default_rng(5)
    base = 0.02 * rng.random((24, 24))
    s0 = (1, -2)  # (sy, sx)
    g = np.stack([base, np.roll(base, s0, axis=(0, 1)), base])
    W, d = 7, 3
    wn, _ = oracle_mod.weights(g, d, W, 1e-4)
    rho = (W - 1) // 2
    k0 = (s0[0] + rho) * W + (s0[1] + rho)
    inner = wn[0, 6:18, 6:18]
    assert (inner[..., k0] > 0.999).all()
