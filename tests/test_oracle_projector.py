"""Pins of the oracle's projector P_i and its transpose (Eq. 1, Sec. 3).

The oracle traces rays with Siddon's plane-crossing method.  These tests pin
it to results fixed by geometry alone: the closed-form chord of a line
through an axis-aligned square (slab clipping), the analytic line integral
of a uniform disc, and the transpose identity.
"""
import numpy as np
import pytest

from paper_1009_1351_gb300 import synth


def slab_chord(sx, sy, ux, uy, tmax, x0, x1, y0, y1):
    """Length of the segment S + t u, t in [0, tmax], inside [x0,x1]x[y0,y1]."""
    lo = np.zeros_like(sx)
    hi = np.full_like(sx, tmax)
    for s, u, a, b in ((sx, ux, x0, x1), (sy, uy, y0, y1)):
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (a - s) / u
            t1 = (b - s) / u
        par = u == 0
        inside = (s >= a) & (s < b)
        tl = np.where(par, np.where(inside, -np.inf, np.inf), np.minimum(t0, t1))
        th = np.where(par, np.where(inside, np.inf, -np.inf), np.maximum(t0, t1))
        lo = np.maximum(lo, tl)
        hi = np.minimum(hi, th)
    return np.maximum(hi - lo, 0.0)


def _rays(g):
    src, d = synth.ray_endpoints(g)
    return src[..., 0], src[..., 1], d[..., 0], d[..., 1]


@pytest.mark.parametrize("cfg", ["small", "tiny"])
def test_all_ones_image_gives_chord_through_image_square(oracle_mod, cfg):
    g = synth.small_geometry() if cfg == "small" else synth.case("tiny").geom
    G = oracle_mod.Geom(g)
    q = oracle_mod.project(G, np.ones(G.img_shape))
    sx, sy, ux, uy = _rays(g)
    hx, hy = g.nx * g.pixel_mm / 2, g.ny * g.pixel_mm / 2
    ref = slab_chord(sx, sy, ux, uy, g.sdd_mm, -hx, hx, -hy, hy)
    assert ref.max() > 0
    np.testing.assert_allclose(q, ref, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("ix,iy", [(5, 2), (0, 7), (3, 3)])
def test_single_pixel_image_gives_chord_through_that_pixel(oracle_mod, ix, iy):
    g = synth.small_geometry()
    G = oracle_mod.Geom(g)
    f = np.zeros(G.img_shape)
    f[:, iy, ix] = 1.0
    q = oracle_mod.project(G, f)
    sx, sy, ux, uy = _rays(g)
    d = g.pixel_mm
    x0 = (ix - g.nx / 2) * d
    y0 = (iy - g.ny / 2) * d
    ref = slab_chord(sx, sy, ux, uy, g.sdd_mm, x0, x0 + d, y0, y0 + d)
    assert (ref > 0).sum() > 10
    np.testing.assert_allclose(q, ref, rtol=1e-12, atol=1e-12)


def test_every_matrix_entry_is_the_pixel_chord(oracle_mod):
    """Each system-matrix entry equals the closed-form chord of that ray through
    that pixel square (catches swapped axes, off-by-one pixel indices, wrong
    sign of the fan angle)."""
    g = synth.small_geometry(nx=7, ny=5, N=2, V=5, B=11)
    G = oracle_mod.Geom(g)
    sx, sy, ux, uy = (a.reshape(-1) for a in _rays(g))
    d = g.pixel_mm
    for phase in range(g.n_phases):
        A = oracle_mod.system_matrix(G, phase)
        sl = slice(phase * g.n_views * g.n_bins, (phase + 1) * g.n_views * g.n_bins)
        for iy in range(g.ny):
            for ix in range(g.nx):
                x0 = (ix - g.nx / 2) * d
                y0 = (iy - g.ny / 2) * d
                ref = slab_chord(sx[sl], sy[sl], ux[sl], uy[sl], g.sdd_mm, x0, x0 + d, y0, y0 + d)
                np.testing.assert_allclose(A[:, iy * g.nx + ix], ref, atol=1e-12)


@pytest.mark.parametrize("cfg", ["small", "tiny"])
def test_adjointness(oracle_mod, cfg):
    g = synth.small_geometry() if cfg == "small" else synth.case("tiny").geom
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(G.img_shape)
    q = rng.standard_normal(G.sino_shape)
    lhs = np.vdot(oracle_mod.project(G, f), q)
    rhs = np.vdot(f, oracle_mod.backproject(G, q))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_backprojection_is_the_dense_transpose(oracle_mod):
    g = synth.small_geometry()
    G = oracle_mod.Geom(g)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(G.sino_shape)
    bp = oracle_mod.backproject(G, q)
    for i in range(g.n_phases):
        A = oracle_mod.system_matrix(G, i)
        np.testing.assert_allclose(bp[i].reshape(-1), A.T @ q[i].reshape(-1), rtol=1e-12, atol=1e-12)


def _disc_error(oracle_mod, L, fov_mm=64.0):
    pix = fov_mm / L
    g = synth.Geometry(nx=L, ny=L, pixel_mm=pix, n_phases=1, n_views=8, n_bins=96,
                       bin_mm=1.0, sid_mm=1000.0, sdd_mm=1500.0)
    G = oracle_mod.Geom(g)
    cx, cy, R, mu = 3.3, -2.1, 20.0, 0.02
    img = synth.rasterize([(cx, cy, R, R, mu, 0.0)], L, L, pix, ss=8)[None]
    q = oracle_mod.project(G, img)
    sx, sy, ux, uy = _rays(g)
    p = np.abs((sx - cx) * uy - (sy - cy) * ux)       # distance of the line to the disc centre
    ref = 2.0 * mu * np.sqrt(np.maximum(R * R - p * p, 0.0))
    return np.abs(q - ref).mean(), ref.max()


def test_uniform_disc_line_integrals_converge_first_order(oracle_mod):
    """Line integrals of a rasterised uniform disc approach 2 mu sqrt(R^2 - p^2);
    the error comes from the pixelised boundary and is O(pixel)."""
    errs = []
    for L in (32, 64, 128):
        e, peak = _disc_error(oracle_mod, L)
        errs.append(e)
        assert e < 0.02 * peak * (64.0 / L)
    assert errs[1] < 0.75 * errs[0]
    assert errs[2] < 0.75 * errs[1]
