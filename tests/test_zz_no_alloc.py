"""tnlm_project_static: the projection for callers that cannot allocate.

Some callers cannot call cudaMalloc: code running inside an open CUDA stream
capture, applications whose device memory is fixed at start-up or owned by
another allocator, hosts that only hand out preallocated buffers.  For them
the library offers tnlm_project_static, which keeps its scratch in a fixed
file-scope device array instead of the handle's workspace.  This file checks,
through the C ABI, that two calls in a row give the same projections as
tnlm_project, and that a geometry too large for the array is refused.  It is
named so that pytest collects it last.
"""
import ctypes

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


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_static_projection_matches_tnlm_project_on_two_calls(tn):
    lib = tn.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    cases = []
    # a 256^2 slice first, then a smaller one: the second call must not see
    # stale values the first left in the shared array
    for name, seed in (("mid_a", 11), ("tiny", 12)):
        g = synth.case(name).geom
        geo = tn.tnlm_create_geometry(g)
        img = torch.tensor(synth.random_images((g.n_phases, g.ny, g.nx), seed), dtype=torch.float32,
                           device="cuda")
        ref = torch.zeros((g.n_phases, g.n_views, g.n_bins), device="cuda")
        tn.tnlm_project(geo, img, ref)
        cases.append((geo, img, ref))
    torch.cuda.synchronize()
    outs = []
    for geo, img, ref in cases:                       # two calls in a row
        out = torch.full_like(ref, float("nan"))
        st = lib.tnlm_project_static(ctypes.c_void_p(geo.handle), ctypes.c_void_p(img.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == tn.TNLM_OK, lib.tnlm_last_error()
        outs.append(out)
    torch.cuda.synchronize()
    for (geo, img, ref), out in zip(cases, outs):
        got, want = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel_l2(got, want) <= 1e-5


def test_static_projection_refuses_oversized_geometry(tn):
    lib = tn.load_library()
    g = synth.Geometry(nx=1024, ny=1024, pixel_mm=0.5, n_phases=3, n_views=2, n_bins=16,
                       bin_mm=1.0, sid_mm=2000.0, sdd_mm=3000.0)
    geo = tn.tnlm_create_geometry(g)
    img = torch.zeros((3, 1024, 1024), device="cuda")
    out = torch.zeros((3, 2, 16), device="cuda")
    st = lib.tnlm_project_static(ctypes.c_void_p(geo.handle), ctypes.c_void_p(img.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert st == tn.TNLM_ERR_INVALID_ARG
    assert b"static scratch" in lib.tnlm_last_error()
