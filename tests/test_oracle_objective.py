"""Pins of the oracle's two terms of Eq. 1 (CPU).

T(f) = sum_i [J(f_i, f_{i-1}) + J(f_i, f_{i+1})], J as Eq. 2 defines it, is
checked against
  * the same quantity written with dense weight matrices: for W_ij with
    entries omega_{i,j}(x, y), J(f_i, f_j) = f_i^T diag(W_ij 1) f_i
    - 2 f_i^T W_ij f_j + f_j^T diag(W_ij^T 1) f_j (expanding the square);
  * constant images (rows of Eq. 3 sum to one, every difference is zero): 0;
  * all weight on the zero shift: J(f_i, f_j) = ||f_i - f_j||^2;
and the data term against the dense system matrix of the oracle's projector:
sum_i ||Sigma^{-1/2} (A_i f_i - y_i)||^2.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth


def dense_weights(w, W, ny, nx):
    """[npx, npx] matrix of one phase's row weights w[ny, nx, W*W]."""
    rho = (W - 1) // 2
    M = np.zeros((ny * nx, ny * nx))
    for y in range(ny):
        for x in range(nx):
            for sy in range(-rho, rho + 1):
                for sx in range(-rho, rho + 1):
                    y1, x1 = y + sy, x + sx
                    if 0 <= y1 < ny and 0 <= x1 < nx:
                        M[y * nx + x, y1 * nx + x1] = w[y, x, (sy + rho) * W + sx + rho]
    return M


@pytest.mark.parametrize("shape,d,W", [((3, 7, 9), 3, 5), ((4, 6, 5), 1, 3), ((3, 8, 8), 5, 7)])
def test_tnlm_term_equals_the_dense_matrix_form(oracle_mod, shape, d, W):
    N, ny, nx = shape
    rng = np.random.default_rng(sum(shape) + W)
    g = 0.02 * rng.random(shape)
    f = 0.02 * rng.random(shape)
    wn, wp = oracle_mod.weights(g, d, W, 0.01)
    want = 0.0
    for i in range(N):
        fi = f[i].ravel()
        for j, w in (((i + 1) % N, wn[i]), ((i - 1) % N, wp[i])):
            M = dense_weights(w, W, ny, nx)
            fj = f[j].ravel()
            want += fi @ (M.sum(1) * fi) - 2 * fi @ (M @ fj) + fj @ (M.sum(0) * fj)
    assert oracle_mod.tnlm_term(f, wn, wp, W) == pytest.approx(want, rel=1e-12)


def test_tnlm_term_vanishes_on_constant_images(oracle_mod):
    rng = np.random.default_rng(5)
    wn, wp = oracle_mod.weights(0.02 * rng.random((3, 10, 12)), 3, 5, 0.01)
    f = np.full((3, 10, 12), 0.017)
    assert abs(oracle_mod.tnlm_term(f, wn, wp, 5)) <= 1e-20


def test_tnlm_term_with_all_weight_on_the_zero_shift(oracle_mod):
    N, ny, nx, W = 4, 6, 7, 3
    rng = np.random.default_rng(6)
    f = rng.random((N, ny, nx))
    w = np.zeros((N, ny, nx, W * W))
    w[..., (W * W) // 2] = 1.0
    want = sum(np.sum((f[i] - f[(i + 1) % N]) ** 2) + np.sum((f[i] - f[(i - 1) % N]) ** 2)
               for i in range(N))
    assert oracle_mod.tnlm_term(f, w, w, W) == pytest.approx(want, rel=1e-13)


def test_data_term_equals_the_dense_matrix_form(oracle_mod):
    g = synth.small_geometry(nx=7, ny=5, N=3, V=5, B=11)
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(8)
    f = rng.random(G.img_shape)
    y = rng.random(G.sino_shape)
    w = rng.uniform(0.5, 2.0, G.sino_shape)
    want = 0.0
    for i in range(g.n_phases):
        A = oracle_mod.system_matrix(G, i)
        r = A @ f[i].ravel() - y[i].ravel()
        want += np.sum(w[i].ravel() * r * r)
    assert oracle_mod.data_term(G, y, w, f) == pytest.approx(want, rel=1e-12)
    wn = np.zeros(G.img_shape + (9,))
    assert oracle_mod.objective(G, y, w, f, wn, wn, 3, 0.0) == pytest.approx(want, rel=1e-12)
