"""Seeded synthetic 4DCT inputs: geometry, phantom, noisy sinogram, weights.

This module only *makes inputs*; it holds none of the reconstruction
method's arithmetic (no projector, no CGLS, no patch weights, no
Gauss-Jacobi).  Both the CUDA path and the FP64 oracle consume what it
returns, so a parity test feeds both sides identical arrays.

Stand-ins for the paper's experiment (Sec. 3):
  * The paper uses the digital NCAT thorax phantom, which is not available
    here.  A family of ellipses (body, two lungs, tumour disc; spine disc and
    a moving diaphragm edge at the larger sizes) plays its role.
  * The paper simulates projections with Siddon ray tracing of a voxel
    phantom; here the noise-free sinogram is the exact line integral through
    the analytic ellipses (no inverse crime with the pixel-based projector).
  * Noise: the paper draws Gaussian noise with the variance of Eq. 9; here
    photon counts are Poisson with mean I0*exp(-p) and the sinogram is the
    log of I0 / counts (a zero count is clamped to one).  The data-term
    weight is the inverse variance of Eq. 9 evaluated on the noise-free
    line integral, w = I0 * exp(-p).

Geometry reading (the paper only names an arc detector, Sec. 3):
  * pixel (ix, iy) has centre ((ix - (nx-1)/2) * pixel, (iy - (ny-1)/2) * pixel),
    images are stored row-major f[phase][iy][ix];
  * view v of phase i has source angle theta = 2*pi*v/V + 2*pi*i/(N*V): the N
    phases interleave evenly over 360 degrees;
  * the source sits at sid*(cos theta, sin theta); the equiangular arc
    detector is centred on the source; bin b has fan angle
    gamma_b = (b - (B-1)/2) * bin_mm / sdd measured counter-clockwise from the
    central ray, which points from the source through the isocentre.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Geometry:
    nx: int
    ny: int
    pixel_mm: float
    n_phases: int
    n_views: int
    n_bins: int
    bin_mm: float
    sid_mm: float
    sdd_mm: float

    def view_angles(self) -> np.ndarray:
        """Source angles [N*V] (radians), phase-major."""
        N, V = self.n_phases, self.n_views
        i = np.arange(N)[:, None]
        v = np.arange(V)[None, :]
        return (2.0 * np.pi * v / V + 2.0 * np.pi * i / (N * V)).reshape(-1).astype(np.float64)

    def fan_angles(self) -> np.ndarray:
        b = np.arange(self.n_bins, dtype=np.float64)
        return (b - (self.n_bins - 1) / 2.0) * (self.bin_mm / self.sdd_mm)


@dataclasses.dataclass(frozen=True)
class Params:
    """TNLM iteration parameters (see Sec. 2.2 and the algorithm boxes)."""
    mu_hat: float = 0.5
    h: float = 0.006          # weight bandwidth of Eq. 8, in units of the image values
    beta: float = 0.0         # only for the gradient data step of Eq. 4
    patch: int = 3            # d
    window: int = 5           # W
    m1: int = 3               # CGLS steps per outer iteration
    m2: int = 5               # Gauss-Jacobi sweeps per outer iteration
    k_outer: int = 20         # outer iterations
    data_step: int = 0        # 0 = CGLS, 1 = gradient step (Eq. 4)
    clamp: int = 1            # positivity truncation after each outer iteration
    precision: int = 0        # 0: FP32; 1: split-FP16 tensor-core patch cross terms
    monitor: int = 0          # 1: FP64 TNLM term / objective of Eq. 1 every iteration
    recompute: int = 0        # 1: sweeps recompute the patch distances (no stored array)


@dataclasses.dataclass(frozen=True)
class Case:
    name: str
    geom: Geometry
    params: Params
    i0: float
    seed: int
    with_spine_diaphragm: bool


# ----------------------------------------------------------------------------
# The workload family: a tiny case, a 256^2 case in three dose scenarios and a
# 512^2 case in four.  Sizes, geometry, doses, patch/window and iteration
# counts are those of the stated workloads; h = 0.002 * d.
# ----------------------------------------------------------------------------

def _geom(L, pix, V, B, binmm):
    return Geometry(nx=L, ny=L, pixel_mm=pix, n_phases=10, n_views=V, n_bins=B,
                    bin_mm=binmm, sid_mm=1000.0, sdd_mm=1500.0)


def case(name: str) -> Case:
    """Named workloads.

    tiny   : 64^2 @1 mm, 60 views, 128 bins @1.2 mm, I0=1e4, d=3, W=5, K=20, M2=5
    mid_a  : 256^2 @1.5 mm, 360 views, 512 bins @1 mm, I0=1e4, d=5, W=11, K=50
    mid_b  : as mid_a with 60 views, I0=1e6
    mid_c  : as mid_a with 60 views, I0=1e4
    large_a: 512^2 @0.8 mm, 360 views, 888 bins @1 mm, I0=5e3, d=7, W=15, K=100
    large_b: as large_a with 90 views, I0=1e5
    large_c: 360 views, I0=1e5;  large_d: 90 views, I0=5e3
    """
    if name == "tiny":
        return Case(name, _geom(64, 1.0, 60, 128, 1.2),
                    Params(patch=3, window=5, k_outer=20, m2=5, h=0.002 * 3),
                    1e4, 1010, False)
    if name.startswith("mid_"):
        sc = name[-1]
        V, i0 = {"a": (360, 1e4), "b": (60, 1e6), "c": (60, 1e4)}[sc]
        return Case(name, _geom(256, 1.5, V, 512, 1.0),
                    Params(patch=5, window=11, k_outer=50, m2=5, h=0.002 * 5),
                    i0, 1020 + "abc".index(sc), True)
    if name.startswith("large_"):
        sc = name[-1]
        V, i0 = {"a": (360, 5e3), "b": (90, 1e5), "c": (360, 1e5), "d": (90, 5e3)}[sc]
        return Case(name, _geom(512, 0.8, V, 888, 1.0),
                    Params(patch=7, window=15, k_outer=100, m2=5, h=0.002 * 7),
                    i0, 1030 + "abcd".index(sc), True)
    raise KeyError(name)


BATCH_SIDES = (256, 384, 512)
BATCH_VIEWS = (60, 90, 180, 360)
BATCH_BINS = {256: 512, 384: 700, 512: 888}


def batch_cases(n: int = 64, seed: int = 1040, k_outer: int = 50, precision: int = 1
                ) -> List[Tuple[Case, Tuple[float, float]]]:
    """The batched workload: n independent 10-phase slices.

    Side L drawn uniformly from {256, 384, 512} (pixel 384 mm / L, so every
    slice covers the same 384 mm field), views per phase from {60, 90, 180,
    360}, I0 log-uniform in [5e3, 1e6], the anatomy shifted by up to 5 % of L
    along each axis; 1 mm bins (512 / 700 / 888 of them); d = 5, W = 11 (the
    256^2 workload's patch and window) and, by default, the mixed-precision
    patch distances (precision = 1).  Returns (case, anatomy offset in
    pixels) per slice.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(rng.choice(BATCH_SIDES))
        V = int(rng.choice(BATCH_VIEWS))
        i0 = float(math.exp(rng.uniform(math.log(5e3), math.log(1e6))))
        off = (float(rng.uniform(-0.05, 0.05) * L), float(rng.uniform(-0.05, 0.05) * L))
        d, W = 5, 11
        c = Case(f"batch{i:02d}", _geom(L, 384.0 / L, V, BATCH_BINS[L], 1.0),
                 Params(patch=d, window=W, k_outer=k_outer, m2=5, h=0.002 * d, precision=precision),
                 i0, seed + 1 + i, True)
        out.append((c, off))
    return out


# ----------------------------------------------------------------------------
# Phantom: ellipses painted in order (later ones replace earlier values).
# Sizes are fractions of the image side L (in pixels); centre = isocentre.
# ----------------------------------------------------------------------------

def phantom_ellipses(L: int, pixel_mm: float, phase: int, n_phases: int,
                     spine_diaphragm: bool, offset_px: Tuple[float, float] = (0.0, 0.0)
                     ) -> List[Tuple[float, float, float, float, float, float]]:
    """Painted ellipses (cx_mm, cy_mm, ax_mm, ay_mm, mu, mu_under) of one phase.

    Each ellipse replaces the value mu_under of the region it is painted on
    (it lies wholly inside that region), so its additive density is
    mu - mu_under.  Body mu=0.019/mm (semi-axes 28/64 L x 20/64 L); lungs
    mu=0.004/mm centred at (+-0.22 L, 0), semi-axes 0.12 L x 0.2 L; tumour
    disc mu=0.021/mm of radius 4/64 L in the right lung, displaced along +y by
    3/64 L * cos^4(pi k / N).  With spine_diaphragm: spine disc mu=0.04/mm at
    (0, -0.25 L), radius 0.05 L, and the lower (-y) edge of both lungs moved
    down by 10 mm * cos^4(pi k / N) (10 mm peak to peak) with the upper edge
    fixed.  offset_px shifts the whole anatomy (per-slice variation).
    """
    s = pixel_mm
    ox, oy = offset_px[0] * s, offset_px[1] * s
    c4 = math.cos(math.pi * phase / n_phases) ** 4
    body = 0.019
    out = [(ox, oy, 28.0 / 64 * L * s, 20.0 / 64 * L * s, body, 0.0)]
    lung_ax, lung_ay = 0.12 * L * s, 0.2 * L * s
    dia = 10.0 * c4 if spine_diaphragm else 0.0
    for sgn in (-1.0, 1.0):
        out.append((ox + sgn * 0.22 * L * s, oy - dia / 2.0, lung_ax, lung_ay + dia / 2.0, 0.004, body))
    if spine_diaphragm:
        out.append((ox, oy - 0.25 * L * s, 0.05 * L * s, 0.05 * L * s, 0.04, body))
    r_t = 4.0 / 64 * L * s
    out.append((ox + 0.22 * L * s, oy + 3.0 / 64 * L * s * c4, r_t, r_t, 0.021, 0.004))
    return out


def rasterize(ells, nx: int, ny: int, pixel_mm: float, ss: int = 4) -> np.ndarray:
    """Painted phantom on the pixel grid, each pixel averaged over ss x ss points."""
    off = (np.arange(ss) + 0.5) / ss - 0.5
    ix = np.arange(nx)[None, :, None] + off[None, None, :]
    iy = np.arange(ny)[:, None, None] + off[None, None, :]
    x = (ix - (nx - 1) / 2.0) * pixel_mm  # [1, nx, ss]
    y = (iy - (ny - 1) / 2.0) * pixel_mm  # [ny, 1, ss]
    X = x[:, :, None, :]                 # [1, nx, 1, ssx]
    Y = y[:, :, :, None]                 # [ny, 1, ssy, 1]
    img = np.zeros((ny, nx, ss, ss))
    for cx, cy, ax, ay, mu, _ in ells:
        inside = ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 <= 1.0
        img = np.where(inside, mu, img)
    return img.mean(axis=(2, 3))


def ray_endpoints(geom: Geometry) -> Tuple[np.ndarray, np.ndarray]:
    """Source points and unit directions of every ray, shape [N, V, B, 2]."""
    th = geom.view_angles().reshape(geom.n_phases, geom.n_views)
    ga = geom.fan_angles()
    src = geom.sid_mm * np.stack([np.cos(th), np.sin(th)], -1)[:, :, None, :]
    ang = th[:, :, None] + np.pi + ga[None, None, :]
    d = np.stack([np.cos(ang), np.sin(ang)], -1)
    src = np.broadcast_to(src, d.shape)
    return src, d


def line_integrals(ells_per_phase, geom: Geometry) -> np.ndarray:
    """Exact line integrals through the (additive) ellipses: p[N][V][B]."""
    src, d = ray_endpoints(geom)
    p = np.zeros(src.shape[:3])
    for i in range(geom.n_phases):
        for cx, cy, ax, ay, mu, under in ells_per_phase[i]:
            px = (src[i, ..., 0] - cx) / ax
            py = (src[i, ..., 1] - cy) / ay
            dx = d[i, ..., 0] / ax
            dy = d[i, ..., 1] / ay
            a = dx * dx + dy * dy
            b = px * dx + py * dy
            c = px * px + py * py - 1.0
            disc = b * b - a * c
            chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / a, 0.0)
            p[i] += (mu - under) * chord
    return p


def make_inputs(c: Case, offset_px=(0.0, 0.0)) -> Dict[str, np.ndarray]:
    """Everything one reconstruction needs, FP64 host arrays.

    Returns dict with truth [N][ny][nx], pbar/y/w [N][V][B], angles [N*V].
    """
    g = c.geom
    rng = np.random.default_rng(c.seed)
    ells = [phantom_ellipses(g.nx, g.pixel_mm, k, g.n_phases, c.with_spine_diaphragm, offset_px)
            for k in range(g.n_phases)]
    truth = np.stack([rasterize(e, g.nx, g.ny, g.pixel_mm) for e in ells])
    pbar = line_integrals(ells, g)
    lam = c.i0 * np.exp(-pbar)
    counts = rng.poisson(lam)
    y = np.log(c.i0 / np.maximum(counts, 1))
    w = lam.copy()
    return {"truth": truth, "pbar": pbar, "y": y, "w": w, "angles": g.view_angles()}


def random_images(shape, seed: int, scale: float = 0.02) -> np.ndarray:
    """Smooth-ish non-negative random images for operator tests."""
    rng = np.random.default_rng(seed)
    return scale * rng.random(shape)


def small_geometry(nx=8, ny=8, N=3, V=6, B=12, pixel=1.0, bin_mm=1.5) -> Geometry:
    """A tiny geometry for dense-matrix checks (FOV covers the image)."""
    return Geometry(nx=nx, ny=ny, pixel_mm=pixel, n_phases=N, n_views=V, n_bins=B,
                    bin_mm=bin_mm, sid_mm=100.0, sdd_mm=150.0)
