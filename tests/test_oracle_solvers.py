"""Pins of the oracle's data step, Gauss-Jacobi and outer iteration (Sec. 2.2).

Pinned against dense FP64 linear algebra on small problems:
  * CGLS (the CGLS box): u^(m) minimises ||P_n u - y_n|| over the Krylov
    space u^(0) + K_m(P_n^T P_n, s^(0));
  * Eq. 4 against the dense formula;
  * Gauss-Jacobi (its box, Eq. 7): the fixed point solves
    (mu+1) u - (mu/2) W_cyc u = g, sweeps contract by mu/(mu+1) in the max
    norm, mu = 0 returns g;
  * the outer iteration with frozen weights and the Eq. 4 step: its fixed
    point solves [mu (I - W_cyc/2) + P^T w P] f = P^T w y with mu = mu_hat*beta;
  * with W = I and beta >= lambda_max(P^T w P) the energy whose exact prox
    step is Eq. 7 decreases monotonically.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth


@pytest.fixture(scope="module")
def small(oracle_mod):
    g = synth.small_geometry()
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(21)
    f_true = 0.02 * rng.random(G.img_shape)
    A = [oracle_mod.system_matrix(G, i) for i in range(g.n_phases)]
    y = np.stack([(A[i] @ f_true[i].reshape(-1)).reshape(g.n_views, g.n_bins) for i in range(g.n_phases)])
    y = y + 0.01 * rng.standard_normal(y.shape)
    w = rng.uniform(0.5, 2.0, size=y.shape)
    return G, A, y, w, rng


def test_cgls_iterates_minimise_over_the_krylov_space(oracle_mod, small):
    G, A, y, w, rng = small
    f0 = 0.01 * rng.random(G.img_shape)
    for m in (1, 2, 3):
        g, res0 = oracle_mod.cgls(G, y, w, f0, m)
        for i in range(G.g.n_phases):
            sw = np.sqrt(w[i].reshape(-1))
            Pn = sw[:, None] * A[i]
            yn = sw * y[i].reshape(-1)
            u0 = f0[i].reshape(-1)
            r0 = yn - Pn @ u0
            assert np.isclose(res0[i], r0 @ r0, rtol=1e-12)
            M = Pn.T @ Pn
            K = [Pn.T @ r0]
            for _ in range(m - 1):
                K.append(M @ K[-1])
            Q, _ = np.linalg.qr(np.stack(K, 1))
            c, *_ = np.linalg.lstsq(Pn @ Q, r0, rcond=None)
            ref = u0 + Q @ c
            np.testing.assert_allclose(g[i].reshape(-1), ref, rtol=1e-8, atol=1e-10)


def test_cgls_with_zero_steps_returns_the_start(oracle_mod, small):
    G, A, y, w, rng = small
    f0 = rng.random(G.img_shape)
    g, _ = oracle_mod.cgls(G, y, w, f0, 0)
    np.testing.assert_array_equal(g, f0)


def test_cgls_zero_residual_phase_stops(oracle_mod, small):
    """y = P f0 exactly for one phase: its residual and gradient vanish and
    CGLS leaves it at f0 (zero denominator reading)."""
    G, A, y, w, rng = small
    f0 = 0.01 * rng.random(G.img_shape)
    y2 = y.copy()
    y2[1] = (A[1] @ f0[1].reshape(-1)).reshape(y2[1].shape)
    g, res0 = oracle_mod.cgls(G, y2, w, f0, 3)
    assert res0[1] < 1e-24
    np.testing.assert_allclose(g[1], f0[1], atol=1e-14)
    assert np.abs(g[0] - f0[0]).max() > 1e-6


def test_gradient_step_matches_dense_formula(oracle_mod, small):
    G, A, y, w, rng = small
    f = 0.01 * rng.random(G.img_shape)
    beta = 37.0
    g = oracle_mod.grad_step(G, y, w, f, beta)
    for i in range(G.g.n_phases):
        fi = f[i].reshape(-1)
        ref = fi - (A[i].T @ (w[i].reshape(-1) * (A[i] @ fi - y[i].reshape(-1)))) / beta
        np.testing.assert_allclose(g[i].reshape(-1), ref, rtol=1e-12, atol=1e-14)


def dense_wcyc(wnext, wprev, W):
    N, ny, nx, _ = wnext.shape
    rho = (W - 1) // 2
    n = ny * nx
    M = np.zeros((N * n, N * n))
    for i in range(N):
        for y in range(ny):
            for x in range(nx):
                row = i * n + y * nx + x
                for sy in range(-rho, rho + 1):
                    for sx in range(-rho, rho + 1):
                        x1, y1 = x + sx, y + sy
                        if not (0 <= x1 < nx and 0 <= y1 < ny):
                            continue
                        k = (sy + rho) * W + sx + rho
                        M[row, ((i + 1) % N) * n + y1 * nx + x1] += wnext[i, y, x, k]
                        M[row, ((i - 1) % N) * n + y1 * nx + x1] += wprev[i, y, x, k]
    return M


@pytest.fixture(scope="module")
def gj_case(oracle_mod):
    rng = np.random.default_rng(8)
    g = 0.02 * rng.random((4, 6, 7))
    W = 3
    wn, wp = oracle_mod.weights(g, 3, W, 0.01)
    return g, wn, wp, W


def test_gauss_jacobi_fixed_point_is_the_dense_solution(oracle_mod, gj_case):
    g, wn, wp, W = gj_case
    mu = 0.7
    M = (mu + 1.0) * np.eye(g.size) - 0.5 * mu * dense_wcyc(wn, wp, W)
    ustar = np.linalg.solve(M, g.reshape(-1))
    u = oracle_mod.gj(g, wn, wp, W, mu, 120)
    np.testing.assert_allclose(u.reshape(-1), ustar, rtol=1e-12, atol=1e-14)


def test_gauss_jacobi_contracts_in_max_norm(oracle_mod, gj_case):
    g, wn, wp, W = gj_case
    mu = 2.0
    M = (mu + 1.0) * np.eye(g.size) - 0.5 * mu * dense_wcyc(wn, wp, W)
    ustar = np.linalg.solve(M, g.reshape(-1))
    prev = np.abs(g.reshape(-1) - ustar).max()
    for m in range(1, 8):
        e = np.abs(oracle_mod.gj(g, wn, wp, W, mu, m).reshape(-1) - ustar).max()
        assert e <= mu / (mu + 1.0) * prev * (1 + 1e-12) + 1e-16
        prev = e


def test_gauss_jacobi_one_sweep_matches_eq7(oracle_mod, gj_case):
    g, wn, wp, W = gj_case
    mu = 0.5
    Wc = dense_wcyc(wn, wp, W)
    ref = g.reshape(-1) / (mu + 1) + mu / (2 * mu + 2) * (Wc @ g.reshape(-1))
    np.testing.assert_allclose(oracle_mod.gj(g, wn, wp, W, mu, 1).reshape(-1), ref, rtol=1e-13)


def test_gauss_jacobi_mu_zero_returns_g(oracle_mod, gj_case):
    g, wn, wp, W = gj_case
    np.testing.assert_array_equal(oracle_mod.gj(g, wn, wp, W, 0.0, 4), g)


def _identity_weights(N, ny, nx, W):
    w = np.zeros((N, ny, nx, W * W))
    w[..., (W * W) // 2] = 1.0
    return w


def _dense_normal(A, w):
    n = A[0].shape[1]
    N = len(A)
    H = np.zeros((N * n, N * n))
    b_of = []
    for i in range(N):
        wi = w[i].reshape(-1)
        H[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i].T @ (wi[:, None] * A[i])
    return H


def test_outer_iteration_fixed_point_with_frozen_weights(oracle_mod, small):
    """Eq. 4 step + exact Gauss-Jacobi (M2 large), frozen weights, no clamp:
    the fixed point solves [mu (I - W_cyc/2) + P^T w P] f = P^T w y."""
    G, A, y, w, rng = small
    N, ny, nx = G.img_shape
    W = 3
    gimg = 0.02 * rng.random(G.img_shape)
    wn, wp = oracle_mod.weights(gimg, 3, W, 0.01)
    H = _dense_normal(A, w)
    lam = np.linalg.eigvalsh(H).max()
    beta, mu_hat = 1.2 * lam, 0.8
    mu = mu_hat * beta
    Wc = dense_wcyc(wn, wp, W)
    rhs = np.concatenate([A[i].T @ (w[i].reshape(-1) * y[i].reshape(-1)) for i in range(N)])
    fstar = np.linalg.solve(mu * (np.eye(H.shape[0]) - 0.5 * Wc) + H, rhs).reshape(G.img_shape)
    p = synth.Params(mu_hat=mu_hat, beta=beta, patch=3, window=W, m1=0, m2=200, k_outer=1,
                     data_step=1, clamp=0)
    f1, _, _ = oracle_mod.reconstruct(G, y, w, fstar, p, frozen=(wn, wp))
    np.testing.assert_allclose(f1, fstar, rtol=1e-9, atol=1e-12)
    # and from elsewhere the iteration moves toward it
    p2 = synth.Params(mu_hat=mu_hat, beta=beta, patch=3, window=W, m1=0, m2=200, k_outer=30,
                      data_step=1, clamp=0)
    f0 = np.zeros(G.img_shape)
    fk, _, _ = oracle_mod.reconstruct(G, y, w, f0, p2, frozen=(wn, wp))
    assert np.linalg.norm(fk - fstar) < 0.5 * np.linalg.norm(f0 - fstar)


def test_energy_decreases_monotonically_for_the_convex_case(oracle_mod, small):
    """W = I (symmetric, doubly stochastic), beta >= lambda_max(P^T w P), exact
    prox (M2 large), no clamp: forward-backward splitting is monotone in
    E(f) = sum_i ||P_i f_i - y_i||_w^2 + mu sum_i [||f_i||^2 - <f_i, f_{i+1}>]."""
    G, A, y, w, rng = small
    N, ny, nx = G.img_shape
    W = 3
    I_w = _identity_weights(N, ny, nx, W)
    lam = np.linalg.eigvalsh(_dense_normal(A, w)).max()
    beta, mu_hat = 1.05 * lam, 0.5
    f = np.zeros(G.img_shape)
    e_prev = oracle_mod.objective_op(G, y, w, f, I_w, W, mu_hat * beta)
    p = synth.Params(mu_hat=mu_hat, beta=beta, patch=3, window=W, m1=0, m2=80, k_outer=1,
                     data_step=1, clamp=0)
    drops = 0
    for _ in range(25):
        f, _, _ = oracle_mod.reconstruct(G, y, w, f, p, frozen=(I_w, I_w))
        e = oracle_mod.objective_op(G, y, w, f, I_w, W, mu_hat * beta)
        assert e <= e_prev * (1 + 1e-12)
        drops += e < e_prev
        e_prev = e
    assert drops >= 20


def test_clamp_makes_images_nonnegative(oracle_mod):
    c = synth.case("tiny")
    G = oracle_mod.Geom(c.geom)
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": 2})
    f, rel, res = oracle_mod.reconstruct(G, d["y"], d["w"], np.zeros(G.img_shape), p)
    assert (f >= 0).all() and f.max() > 0.01
    assert res[1] < res[0]
