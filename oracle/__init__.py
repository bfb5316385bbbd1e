"""FP64 CPU oracle of the TNLM 4DCT reconstruction path (arXiv:1009.1351).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(the CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``tnlm_oracle.c`` (plain C, FP64, OpenMP only over
independent rays / phases / pixels).  This module compiles it with gcc and
wraps each entry point for numpy arrays.  Every function states the paper
passage it follows; see the C file's header for the readings taken where
the paper is silent.

Parity status: every function here is pinned by a CPU test against a
closed form, a dense linear-algebra solve or an invariant (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnlm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
# A test that plants a mistake compiles a changed copy of tnlm_oracle.c and
# points this variable at it (tests/test_oracle_mutations.py); the pins then
# run against that copy.
_LIB_OVERRIDE = os.environ.get("TNLM_ORACLE_LIB")
_lib = None

# the compiler flags of the oracle (FP64, no fast-math, no FMA contraction)
CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11"]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into a shared library at 'out'."""
    subprocess.run(["gcc"] + CFLAGS + [src, "-o", out + ".tmp", "-lm"], check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no fast-math, no FMA contraction)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_ray_entries.restype = ctypes.c_int
        lib.orc_objective_op.restype = ctypes.c_double
        lib.orc_tnlm_term.restype = ctypes.c_double
        lib.orc_data_term.restype = ctypes.c_double
        _lib = lib
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count."""
    return _load().orc_threads(int(n))


class Geom:
    """Geometry arrays in the oracle's own form (built from a synth.Geometry)."""

    def __init__(self, g, angles: Optional[np.ndarray] = None):
        self.g = g
        self.gi = np.array([g.nx, g.ny, g.n_phases, g.n_views, g.n_bins], dtype=np.int32)
        self.gd = np.array([g.pixel_mm, g.bin_mm, g.sid_mm, g.sdd_mm], dtype=np.float64)
        self.ang = _f64(g.view_angles() if angles is None else angles)
        self.img_shape = (g.n_phases, g.ny, g.nx)
        self.sino_shape = (g.n_phases, g.n_views, g.n_bins)

    def args(self):
        return (self.gi.ctypes.data_as(_ip), _d(self.gd), _d(self.ang))


def project(G: Geom, f) -> np.ndarray:
    """P_i f_i for every phase (Eq. 1; Siddon ray tracing as in Sec. 3)."""
    f = _f64(f).reshape(G.img_shape)
    q = np.zeros(G.sino_shape)
    _load().orc_project(*G.args(), _d(f), _d(q))
    return q


def backproject(G: Geom, q) -> np.ndarray:
    """P_i^T q_i for every phase (the exact transpose of ``project``)."""
    q = _f64(q).reshape(G.sino_shape)
    f = np.zeros(G.img_shape)
    _load().orc_backproject(*G.args(), _d(q), _d(f))
    return f


def ray_entries(G: Geom, ray: int) -> Tuple[np.ndarray, np.ndarray]:
    """Non-zero entries (pixel index, length) of one row of the system matrix."""
    cap = G.g.nx + G.g.ny + 4
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap)
    n = _load().orc_ray_entries(*G.args(), ctypes.c_long(ray), idx.ctypes.data_as(_lp), _d(ln))
    return idx[:n].copy(), ln[:n].copy()


def system_matrix(G: Geom, phase: int = 0) -> np.ndarray:
    """Dense A_i (rays of one phase x pixels); small geometries only."""
    V, B = G.g.n_views, G.g.n_bins
    A = np.zeros((V * B, G.g.nx * G.g.ny))
    for rr in range(V * B):
        idx, ln = ray_entries(G, phase * V * B + rr)
        np.add.at(A[rr], idx, ln)
    return A


def cgls(G: Geom, y, w, f0, m1: int) -> Tuple[np.ndarray, np.ndarray]:
    """CGLS box of Sec. 2.2 per phase; returns (g = u^(M1), ||r^(0)||^2 per phase)."""
    u = _f64(f0).reshape(G.img_shape).copy()
    res = np.zeros(G.g.n_phases)
    _load().orc_cgls(*G.args(), _d(_f64(y)), _d(_f64(w)), _d(u), ctypes.c_int(m1), _d(res))
    return u, res


def grad_step(G: Geom, y, w, f, beta: float) -> np.ndarray:
    """Eq. 4: g = f - (1/beta) P^T Sigma^{-1} (P f - y)."""
    f = _f64(f).reshape(G.img_shape)
    g = np.zeros(G.img_shape)
    res = np.zeros(G.g.n_phases)
    _load().orc_grad_step(*G.args(), _d(_f64(y)), _d(_f64(w)), _d(f), ctypes.c_double(beta),
                          _d(g), _d(res))
    return g


def weights(g, d: int, W: int, h: float, with_dist: bool = False):
    """Eq. 8 weights for both neighbours of every phase.

    Returns (wnext, wprev[, dnext]) with shape [N, ny, nx, W*W]:
      wnext[i, y, x, s] = omega_{i,i+1}(x, x+s), wprev[i, y, x, s] = omega_{i,i-1}(x, x+s),
      dnext[i, y, x, s] = ||R_{g_i}(x) - R_{g_{i+1}}(x+s)||^2 (+inf outside the image),
    s = (sy + rho) * W + (sx + rho).
    """
    g = _f64(g)
    N, ny, nx = g.shape
    wn = np.zeros((N, ny, nx, W * W))
    wp = np.zeros_like(wn)
    dn = np.zeros_like(wn) if with_dist else None
    _load().orc_weights(ctypes.c_int(N), ctypes.c_int(nx), ctypes.c_int(ny), _d(g), ctypes.c_int(d),
                        ctypes.c_int(W), ctypes.c_double(h), _d(wn), _d(wp),
                        _d(dn) if with_dist else None)
    return (wn, wp, dn) if with_dist else (wn, wp)


def gj(g, wnext, wprev, W: int, mu_hat: float, m2: int) -> np.ndarray:
    """Gauss-Jacobi box of Sec. 2.2 (M2 sweeps from u^(0) = g)."""
    g = _f64(g)
    N, ny, nx = g.shape
    u = np.zeros_like(g)
    _load().orc_gj(ctypes.c_int(N), ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(W), _d(g),
                   _d(_f64(wnext)), _d(_f64(wprev)), ctypes.c_double(mu_hat), ctypes.c_int(m2), _d(u))
    return u


def reconstruct(G: Geom, y, w, f0, p, frozen=None):
    """TNLM algorithm box of Sec. 2.2.

    p: synth.Params.  frozen: optional (wnext, wprev) used instead of Eq. 8.
    Returns (f^(K), rel_change[K], data_residual[K]).
    """
    f = _f64(f0).reshape(G.img_shape).copy()
    ip = np.array([p.patch, p.window, p.m1, p.m2, p.k_outer, p.data_step, p.clamp], dtype=np.int32)
    dp = np.array([p.mu_hat, p.h, p.beta], dtype=np.float64)
    rel = np.zeros(p.k_outer)
    res = np.zeros(p.k_outer)
    fw = (None, None) if frozen is None else (_f64(frozen[0]), _f64(frozen[1]))
    _load().orc_reconstruct(*G.args(), _d(_f64(y)), _d(_f64(w)), _d(f), ip.ctypes.data_as(_ip),
                            _d(dp), _d(fw[0]) if fw[0] is not None else None,
                            _d(fw[1]) if fw[1] is not None else None, _d(rel), _d(res))
    return f, rel, res


def objective_op(G: Geom, y, w, f, wnext, W: int, mu: float) -> float:
    """Data term of Eq. 1 plus mu * sum_i [||f_i||^2 - <f_i, W_{i,i+1} f_{i+1}>]."""
    return float(_load().orc_objective_op(*G.args(), _d(_f64(y)), _d(_f64(w)), _d(_f64(f)),
                                          _d(_f64(wnext)), ctypes.c_int(W), ctypes.c_double(mu)))


def tnlm_term(f, wnext, wprev, W: int) -> float:
    """The bracket of Eq. 1 summed over phases: sum_i [J(f_i, f_{i-1}) + J(f_i, f_{i+1})]
    with J of Eq. 2 and the weights laid out as ``weights`` returns them."""
    f = _f64(f)
    N, ny, nx = f.shape
    return float(_load().orc_tnlm_term(ctypes.c_int(N), ctypes.c_int(nx), ctypes.c_int(ny),
                                       ctypes.c_int(W), _d(f), _d(_f64(wnext)), _d(_f64(wprev))))


def data_term(G: Geom, y, w, f) -> float:
    """Data term of Eq. 1: sum_i (P_i f_i - y_i)^T Sigma^{-1} (P_i f_i - y_i)."""
    return float(_load().orc_data_term(*G.args(), _d(_f64(y)), _d(_f64(w)), _d(_f64(f))))


def objective(G: Geom, y, w, f, wnext, wprev, W: int, mu: float) -> float:
    """Eq. 1: data term + (mu / 2) * sum_i [J(f_i, f_{i-1}) + J(f_i, f_{i+1})]."""
    return data_term(G, y, w, f) + 0.5 * mu * tnlm_term(f, wnext, wprev, W)


def fbp(G: Geom, y) -> np.ndarray:
    """Initial image of the TNLM algorithm box (step 1): fan-beam FBP of all
    phases' projections together (equiangular form, discrete ramp kernel);
    every phase receives the same image."""
    f = np.zeros(G.img_shape)
    _load().orc_fbp(*G.args(), _d(_f64(y).reshape(G.sino_shape)), _d(f))
    return f
