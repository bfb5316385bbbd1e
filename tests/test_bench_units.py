"""The algorithmic amounts behind bench.py's roofline figures (CPU).

The projector pair's roofline counts lane operations per non-zero of the
system matrix, with the non-zeros counted from the ray geometry alone
(bench.system_nnz: a segment inside the image square crosses one pixel plus
one per grid line it passes).  Here that count is checked against the
oracle's explicit matrix, entry by entry, on several geometries (odd sizes,
a wide fan, the workload's own geometry scaled down), so the reported
fraction does not rest on the counting formula alone.
"""
import numpy as np
import pytest

import bench
from paper_1009_1351_gb300 import synth

GEOMS = [
    synth.small_geometry(nx=7, ny=5, N=2, V=5, B=11),
    synth.small_geometry(),
    synth.Geometry(nx=32, ny=32, pixel_mm=1.5, n_phases=3, n_views=12, n_bins=64, bin_mm=1.0,
                   sid_mm=1000.0, sdd_mm=1500.0),
    synth.Geometry(nx=37, ny=29, pixel_mm=1.1, n_phases=3, n_views=7, n_bins=45, bin_mm=1.3,
                   sid_mm=500.0, sdd_mm=800.0),
    synth.Geometry(nx=18, ny=14, pixel_mm=2.0, n_phases=3, n_views=8, n_bins=96, bin_mm=2.0,
                   sid_mm=60.0, sdd_mm=100.0),
]


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: f"{g.nx}x{g.ny}_{g.n_views}v_{g.n_bins}b")
def test_nnz_count_equals_the_oracle_matrix(oracle_mod, g):
    G = oracle_mod.Geom(g)
    nnz = sum(int((oracle_mod.system_matrix(G, p) > 0).sum()) for p in range(g.n_phases))
    assert bench.system_nnz(g) == nnz


def test_projector_roofline_amount_is_seven_operations_per_nonzero():
    c = synth.case("tiny")
    amount, unit, bound = bench.roofline_units(c, "project")
    assert (unit, bound) == ("Tops/s", "alu")
    assert amount == 7.0 * bench.system_nnz(c.geom)


def test_sweep_and_weights_bytes_follow_the_distance_array():
    """4 bytes per stored distance (N pairs x W^2 shifts x pixels) plus the
    per-pixel images each kernel reads or writes."""
    c = synth.case("mid_a")
    g, p = c.geom, c.params
    n_dist = g.n_phases * g.nx * g.ny * p.window ** 2
    gj, _, bound_gj = bench.roofline_units(c, "gj")
    w, _, bound_w = bench.roofline_units(c, "weights")
    assert (bound_gj, bound_w) == ("hbm", "hbm")
    assert gj == 4 * n_dist + 24 * g.n_phases * g.nx * g.ny
    assert w == 4 * n_dist + 20 * g.n_phases * g.nx * g.ny
    assert np.isclose(n_dist, 79.3e6, rtol=1e-3)


def test_traffic_rows_are_used_only_while_their_sources_hash_to_them(tmp_path, monkeypatch):
    """profiles/traffic.txt rows carry the hash of the files their counters
    depend on ('+'-joined); a changed file voids the row, and the mixed
    precision weights class looks up rows of its own."""
    import hashlib
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_text("kernel a\n")
    (tmp_path / "b.cu").write_text("layout b\n")
    h = hashlib.sha1(b"kernel a\nlayout b\n").hexdigest()[:12]
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# header\n"
        f"weights  c1  100  20  a.cu+b.cu  {h}\n"
        f"weights  c2  300  40  a.cu+b.cu  {h}\n"
        f"gj       c1  7    1   a.cu  {hashlib.sha1(b'kernel a').hexdigest()[:12]}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("weights", ["c1", "c2"]) == pytest.approx(230.0)
    assert bench.measured_traffic("weights", ["c1", "c3"]) is None      # a case without a row
    assert bench.measured_traffic("gj", ["c1"]) is None                 # hash of another content
    assert bench.measured_traffic(bench.traffic_class("weights", True), ["c1"]) is None
    assert bench.traffic_class("weights", False) == "weights"
    (tmp_path / "b.cu").write_text("layout b, changed\n")
    assert bench.measured_traffic("weights", ["c1"]) is None
