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


def _static(tn, geo, img, out, stream):
    lib = tn.load_library()
    st = lib.tnlm_project_static(ctypes.c_void_p(geo.handle), ctypes.c_void_p(img.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert st == tn.TNLM_OK, lib.tnlm_last_error()


def test_static_projection_matches_tnlm_project_on_two_calls(tn):
    """The static calls run first, each on a fresh handle that never had a
    workspace; tnlm_project runs afterwards on handles of its own.  Both run
    the same layout and projector kernels on the same inputs, so the results
    must agree bitwise.  The second static call must not change the device's
    free memory (the first may: it can load the library's device code)."""
    stream = torch.cuda.current_stream().cuda_stream
    # a 256^2 slice first, then a smaller one: the second call must not see
    # stale values the first left in the shared array
    cases = []
    for name, seed in (("mid_a", 11), ("tiny", 12)):
        g = synth.case(name).geom
        img = torch.tensor(synth.random_images((g.n_phases, g.ny, g.nx), seed), dtype=torch.float32,
                           device="cuda")
        cases.append((g, img, torch.full((g.n_phases, g.n_views, g.n_bins), float("nan"), device="cuda")))
    geos = [tn.tnlm_create_geometry(g) for g, _, _ in cases]
    torch.cuda.synchronize()
    _static(tn, geos[0], cases[0][1], cases[0][2], stream)          # two calls in a row
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    _static(tn, geos[1], cases[1][1], cases[1][2], stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    for g, img, out in cases:
        ref = torch.zeros_like(out)
        tn.tnlm_project(tn.tnlm_create_geometry(g), img, ref)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert torch.equal(out, ref)


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
